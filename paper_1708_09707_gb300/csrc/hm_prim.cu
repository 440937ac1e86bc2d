// hm_prim.cu -- device primitives: exclusive scan and a stable LSD radix sort.
//
// The paper builds on vendor "standard parallel algorithms" (scan, stable_sort,
// Sec. 3.2); here they are written out for sm_103a. Neither primitive uses
// inter-block spin waits: the scan is reduce -> scan partials -> downsweep and
// each radix pass is histogram -> scan -> scatter, so no launch can hang on
// another block's progress.
#include <algorithm>
#include <mutex>
#include <string>

#include "hm_internal.cuh"

namespace hm {

namespace {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Block-wide exclusive scan of one value per thread; returns the exclusive
// prefix and writes the block total to *total.
template <class T, int NT>
__device__ T block_exclusive_scan(T v, T* total)
{
    __shared__ T warp_tot[NT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        T t = (lane < NT / 32) ? warp_tot[lane] : T(0);
        T ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < NT / 32) warp_tot[lane] = ti - t;  // exclusive warp offsets
        if (lane == 31) *total = ti;
    }
    __syncthreads();
    T r = warp_tot[w] + inc - v;
    __syncthreads();
    return r;
}

template <class T>
__global__ void k_scan_reduce(const T* __restrict__ in, int64_t n, T* __restrict__ part)
{
    __shared__ T tot;
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    T s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
        if (i < n) s += in[i];
    }
    block_exclusive_scan<T, SCAN_THREADS>(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// Single block: exclusive scan of the tile partials, carrying a running sum.
template <class T>
__global__ void k_scan_partials(T* part, int64_t np, T* total)
{
    __shared__ T tot;
    T carry = 0;
    for (int64_t c = 0; c < np; c += SCAN_THREADS) {
        int64_t i = c + threadIdx.x;
        T v = (i < np) ? part[i] : T(0);
        T ex = block_exclusive_scan<T, SCAN_THREADS>(v, &tot);
        if (i < np) part[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

template <class T>
__global__ void k_scan_down(const T* in, T* out, int64_t n, const T* __restrict__ part)
{
    __shared__ T tot;
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T v[SCAN_ITEMS];
    T s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = (base + k < n) ? in[base + k] : T(0);
        s += v[k];
    }
    T ex = block_exclusive_scan<T, SCAN_THREADS>(s, &tot) + part[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = ex;
        ex += v[k];
    }
}

template <class T>
void scan_exclusive(const T* in, T* out, int64_t n, T* total, cudaStream_t s)
{
    if (n <= 0) {
        if (total) HM_CUDA(cudaMemsetAsync(total, 0, sizeof(T), s));
        return;
    }
    int64_t tiles = ceil_div(n, SCAN_TILE);
    DevBuf<T> part(tiles, s);
    k_scan_reduce<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, part.p); note_launch();
    k_scan_partials<T><<<1, SCAN_THREADS, 0, s>>>(part.p, tiles, total); note_launch();
    k_scan_down<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, part.p); note_launch();
    HM_LAUNCH("scan");
}

// Device-count variant: the scan covers n = min(*ndev, nmax) entries, n read
// on the device, so that a caller can chain launches whose sizes are known
// only on the device. The grids are sized for nmax but stride over the tiles
// of n, so the work follows n.
template <class T>
__global__ void k_scan_reduce_dev(const T* __restrict__ in, const int64_t* __restrict__ ndev,
                                  int64_t nmax, T* __restrict__ part)
{
    __shared__ T tot;
    const int64_t n = *ndev < nmax ? *ndev : nmax;
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t base = t * SCAN_TILE;
        T s = 0;
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            const int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
            if (i < n) s += in[i];
        }
        block_exclusive_scan<T, SCAN_THREADS>(s, &tot);
        if (threadIdx.x == 0) part[t] = tot;
    }
}

template <class T>
__global__ void k_scan_partials_dev(T* part, const int64_t* __restrict__ ndev, int64_t nmax,
                                    T* total)
{
    __shared__ T tot;
    const int64_t n = *ndev < nmax ? *ndev : nmax;
    const int64_t np = (n + SCAN_TILE - 1) / SCAN_TILE;
    T carry = 0;
    for (int64_t c = 0; c < np; c += SCAN_THREADS) {
        const int64_t i = c + threadIdx.x;
        const T v = (i < np) ? part[i] : T(0);
        const T ex = block_exclusive_scan<T, SCAN_THREADS>(v, &tot);
        if (i < np) part[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

template <class T>
__global__ void k_scan_down_dev(const T* in, T* out, const int64_t* __restrict__ ndev,
                                int64_t nmax, const T* __restrict__ part)
{
    __shared__ T tot;
    const int64_t n = *ndev < nmax ? *ndev : nmax;
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t base = t * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
        T v[SCAN_ITEMS];
        T s = 0;
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            v[k] = (base + k < n) ? in[base + k] : T(0);
            s += v[k];
        }
        T ex = block_exclusive_scan<T, SCAN_THREADS>(s, &tot) + part[t];
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            if (base + k < n) out[base + k] = ex;
            ex += v[k];
        }
    }
}

// ---------------------------------------------------------------------------
// Radix sort: 8-bit digits, tiles of 2048 keys (256 threads x 8 keys).
// Each warp owns 256 consecutive keys of its tile; within a tile the stable
// rank of a key is (tile-local start of its digit) + (keys of that digit in
// earlier warps) + (keys of that digit earlier in this warp), the last from
// __match_any_sync peer masks. Keys are first placed in shared memory in
// tile-sorted order and then written out so that equal digits stay
// contiguous.
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_GROUPS = 8;                       // 32-key groups per warp
constexpr int RS_TILE = RS_THREADS * RS_GROUPS;    // 2048

__global__ void k_rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                          int32_t* __restrict__ counts, int ntiles)
{
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int k = threadIdx.x; k < RS_TILE; k += RS_THREADS) {
        int64_t i = base + k;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xFF], 1);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_THREADS)
k_rs_scatter(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
             uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n,
             int shift, const int32_t* __restrict__ offs, int ntiles)
{
    __shared__ uint64_t sk[RS_TILE];
    __shared__ uint32_t sv[RS_TILE];
    __shared__ int32_t wcnt[RS_WARPS][256];
    __shared__ int32_t dstart[256];
    __shared__ int32_t tot;

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    const unsigned lt = (1u << lane) - 1u;

    for (int k = threadIdx.x; k < RS_WARPS * 256; k += RS_THREADS) (&wcnt[0][0])[k] = 0;
    __syncthreads();

    uint64_t key[RS_GROUPS];
    uint32_t val[RS_GROUPS];
    int dig[RS_GROUPS];
#pragma unroll
    for (int g = 0; g < RS_GROUPS; ++g) {
        int64_t i = base + (int64_t)w * (RS_GROUPS * 32) + g * 32 + lane;
        bool ok = i < n;
        key[g] = ok ? kin[i] : 0ull;
        val[g] = ok ? vin[i] : 0u;
        dig[g] = ok ? (int)((key[g] >> shift) & 0xFF) : 256;
    }
    // per-warp digit counts
#pragma unroll
    for (int g = 0; g < RS_GROUPS; ++g) {
        unsigned peers = __match_any_sync(0xffffffffu, dig[g]);
        if (dig[g] < 256 && (peers & lt) == 0) wcnt[w][dig[g]] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive offsets over warps, then over digits
    {
        int t = threadIdx.x;  // digit
        int run = 0;
#pragma unroll
        for (int ww = 0; ww < RS_WARPS; ++ww) {
            int c = wcnt[ww][t];
            wcnt[ww][t] = run;
            run += c;
        }
        int ex = block_exclusive_scan<int, RS_THREADS>(run, &tot);
        dstart[t] = ex;
    }
    __syncthreads();
    // stable tile-local positions
#pragma unroll
    for (int g = 0; g < RS_GROUPS; ++g) {
        unsigned peers = __match_any_sync(0xffffffffu, dig[g]);
        if (dig[g] < 256) {
            int pos = dstart[dig[g]] + wcnt[w][dig[g]] + __popc(peers & lt);
            sk[pos] = key[g];
            sv[pos] = val[g];
        }
        __syncwarp();
        if (dig[g] < 256 && (peers & lt) == 0) wcnt[w][dig[g]] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    const int64_t rem = n - base;
    const int valid = rem < RS_TILE ? (int)rem : RS_TILE;
    for (int k = threadIdx.x; k < valid; k += RS_THREADS) {
        uint64_t kk = sk[k];
        int dg = (int)((kk >> shift) & 0xFF);
        int64_t dst = (int64_t)offs[(int64_t)dg * ntiles + blockIdx.x] + (k - dstart[dg]);
        kout[dst] = kk;
        vout[dst] = sv[k];
    }
}

}  // namespace

void scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total,
                        cudaStream_t s)
{
    scan_exclusive<int64_t>(in, out, n, total, s);
}

void scan_exclusive_i64_dev(const int64_t* in, int64_t* out, const int64_t* ndev, int64_t nmax,
                            int64_t* total, cudaStream_t s)
{
    const int64_t tiles = std::max<int64_t>(1, ceil_div(nmax, SCAN_TILE));
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, 4 * (int64_t)num_sms());
    DevBuf<int64_t> part(tiles, s);
    k_scan_reduce_dev<int64_t><<<grid, SCAN_THREADS, 0, s>>>(in, ndev, nmax, part.p); note_launch();
    k_scan_partials_dev<int64_t><<<1, SCAN_THREADS, 0, s>>>(part.p, ndev, nmax, total); note_launch();
    k_scan_down_dev<int64_t><<<grid, SCAN_THREADS, 0, s>>>(in, out, ndev, nmax, part.p); note_launch();
    HM_LAUNCH("scan");
}

void scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* total,
                        cudaStream_t s)
{
    scan_exclusive<int32_t>(in, out, n, total, s);
}

void radix_sort_u64_u32(uint64_t* keys, uint32_t* vals, int64_t n, int key_bits,
                        cudaStream_t s)
{
    if (n <= 1 || key_bits <= 0) return;
    if (n > (int64_t)INT32_MAX) fail(HM_EINVAL, "radix sort: more than 2^31 keys");
    const int passes = (key_bits + 7) / 8;
    const int ntiles = (int)ceil_div(n, RS_TILE);
    DevBuf<uint64_t> k2(n, s);
    DevBuf<uint32_t> v2(n, s);
    DevBuf<int32_t> cnt((size_t)256 * ntiles, s);
    uint64_t *ka = keys, *kb = k2.p;
    uint32_t *va = vals, *vb = v2.p;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_rs_hist<<<ntiles, RS_THREADS, 0, s>>>(ka, n, shift, cnt.p, ntiles); note_launch();
        scan_exclusive<int32_t>(cnt.p, cnt.p, (int64_t)256 * ntiles, nullptr, s);
        k_rs_scatter<<<ntiles, RS_THREADS, 0, s>>>(ka, va, kb, vb, n, shift, cnt.p, ntiles); note_launch();
        HM_LAUNCH("radix sort pass");
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        HM_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        HM_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the radix sort (hm_radix_sort_pairs_noalloc).
//
// Some callers cannot allocate device memory while they run: a program that
// has handed all free device memory to its own pool or caching allocator
// must not have memory taken from under it, and a latency-critical loop
// cannot afford an allocation that may block on the driver. For them the
// sort below takes all of its scratch (ping-pong key and value buffers,
// digit counts, scan partials) from one fixed array in the library's device
// memory instead of allocating. The array holds NOALLOC_BYTES (about 3.3 MB)
// on every GPU that loads the library, for the life of the process.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t NOALLOC_MAX_N = HM_NOALLOC_SORT_MAX;
constexpr int64_t NOALLOC_TILES = (NOALLOC_MAX_N + RS_TILE - 1) / RS_TILE;
constexpr int64_t NOALLOC_COUNTS = 256 * NOALLOC_TILES;
constexpr int64_t NOALLOC_PARTS = (NOALLOC_COUNTS + SCAN_TILE - 1) / SCAN_TILE;
// byte offsets of the sub-buffers (each 256-byte aligned)
constexpr size_t NA_KEYS = 0;
constexpr size_t NA_VALS = NA_KEYS + ((NOALLOC_MAX_N * 8 + 255) / 256) * 256;
constexpr size_t NA_CNT = NA_VALS + ((NOALLOC_MAX_N * 4 + 255) / 256) * 256;
constexpr size_t NA_PART = NA_CNT + ((NOALLOC_COUNTS * 4 + 255) / 256) * 256;
constexpr size_t NOALLOC_BYTES = NA_PART + ((NOALLOC_PARTS * 4 + 255) / 256) * 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[256] = {};

// Device address of the scratch array on the current device. The first call
// on a device looks it up with cudaGetSymbolAddress (with that device
// current); later calls reuse it.
char* noalloc_scratch()
{
    int dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) fail(HM_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            fail(HM_ECUDA, std::string("cudaGetSymbolAddress of the sort scratch failed: ") +
                               cudaGetErrorString(e));
        }
        g_noalloc_addr[dev] = p;
    }
    return static_cast<char*>(g_noalloc_addr[dev]);
}

}  // namespace

void radix_sort_noalloc(uint64_t* keys, uint32_t* vals, int64_t n, int key_bits, cudaStream_t s)
{
    if (n > NOALLOC_MAX_N)
        fail(HM_EINVAL, "hm_radix_sort_pairs_noalloc: n = " + std::to_string(n) +
                            " exceeds the fixed scratch limit of " + std::to_string(NOALLOC_MAX_N) +
                            " pairs");
    if (n <= 1 || key_bits <= 0) return;
    char* base = noalloc_scratch();
    uint64_t* k2 = reinterpret_cast<uint64_t*>(base + NA_KEYS);
    uint32_t* v2 = reinterpret_cast<uint32_t*>(base + NA_VALS);
    int32_t* cnt = reinterpret_cast<int32_t*>(base + NA_CNT);
    int32_t* part = reinterpret_cast<int32_t*>(base + NA_PART);
    // every word of cnt and part that a pass reads is written earlier in the
    // same pass (histogram, then reduce), so nothing needs clearing
    const int passes = (key_bits + 7) / 8;
    const int ntiles = (int)ceil_div(n, RS_TILE);
    const int64_t ncnt = (int64_t)256 * ntiles;
    const int64_t sparts = ceil_div(ncnt, SCAN_TILE);
    uint64_t *ka = keys, *kb = k2;
    uint32_t *va = vals, *vb = v2;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        k_rs_hist<<<ntiles, RS_THREADS, 0, s>>>(ka, n, shift, cnt, ntiles); note_launch();
        k_scan_reduce<int32_t><<<(unsigned)sparts, SCAN_THREADS, 0, s>>>(cnt, ncnt, part); note_launch();
        k_scan_partials<int32_t><<<1, SCAN_THREADS, 0, s>>>(part, sparts, nullptr); note_launch();
        k_scan_down<int32_t><<<(unsigned)sparts, SCAN_THREADS, 0, s>>>(cnt, cnt, ncnt, part); note_launch();
        k_rs_scatter<<<ntiles, RS_THREADS, 0, s>>>(ka, va, kb, vb, n, shift, cnt, ntiles); note_launch();
        HM_LAUNCH("radix sort pass (no allocation)");
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        HM_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        HM_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
}

}  // namespace hm
