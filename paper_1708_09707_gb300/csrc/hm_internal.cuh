// hm_internal.cuh -- shared declarations of the CUDA H-matrix library.
//
// Layout conventions (all device memory, owned by a handle):
//  * Points are kept in Morton order as three structure-of-arrays coordinate
//    vectors X[0..2][row] (double, and float for mixed precision). Sets with
//    d < 3 are padded with zero coordinates: the padded terms add exact zeros
//    to every squared distance, so results are the same as with d terms.
//  * Several independent point sets are concatenated; a block descriptor
//    holds absolute Morton rows (row0, m) and columns (col0, n).
//  * Cluster-tree nodes use heap numbering per set (root 0, children 2v+1,
//    2v+2), offset by the set's node base in the concatenated node arrays.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/hm.h"

namespace hm {

// ---------------------------------------------------------------------------
// Errors: internal host code throws hm::Error; every C-ABI entry point catches
// it and converts it into an HM_* status plus the thread's last-error text.
// ---------------------------------------------------------------------------
struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string& msg) : std::runtime_error(msg), code(c) {}
};

void check_cuda(cudaError_t e, const char* what, const char* file, int line);
#define HM_CUDA(call) ::hm::check_cuda((call), #call, __FILE__, __LINE__)
#define HM_LAUNCH(what) ::hm::check_cuda(cudaGetLastError(), what, __FILE__, __LINE__)

[[noreturn]] void fail(int code, const std::string& msg);

// Stream-ordered device allocations (cudaMallocAsync on the handle's stream).
void* dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

template <class T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaStream_t s = 0;
    DevBuf() = default;
    DevBuf(size_t count, cudaStream_t st) { alloc(count, st); }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept { *this = std::move(o); }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) {
            release();
            p = o.p; n = o.n; s = o.s;
            o.p = nullptr; o.n = 0;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t count, cudaStream_t st) {
        release();
        s = st;
        n = count;
        p = count ? static_cast<T*>(dev_alloc(count * sizeof(T), st)) : nullptr;
    }
    void release() {
        if (p) dev_free(p, s);
        p = nullptr;
        n = 0;
    }
    size_t bytes() const { return n * sizeof(T); }
};

// Copy helpers that accept host or device pointers on either side.
bool is_device_ptr(const void* p);
void copy_in(void* dst_dev, const void* src, size_t bytes, cudaStream_t s);
void copy_out(void* dst, const void* src_dev, size_t bytes, cudaStream_t s);

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
int num_sms();
double alu_peak(int precision);   // FLOP/s of FMA chains on the current device

// Count of kernels this library has launched in the process (hm_kernel_launches).
void note_launch();

// ---------------------------------------------------------------------------
// Device primitives (hm_prim.cu)
// ---------------------------------------------------------------------------
// Exclusive scan of n int64 values (in may alias out); total (device, may be
// null) receives the sum.
void scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t n,
                        int64_t* total, cudaStream_t s);
void scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t n,
                        int32_t* total, cudaStream_t s);
// The same over n = min(*ndev, nmax) entries, n read on the device (ndev a
// device pointer); no host synchronisation.
void scan_exclusive_i64_dev(const int64_t* in, int64_t* out, const int64_t* ndev, int64_t nmax,
                            int64_t* total, cudaStream_t s);
// Stable LSD radix sort of (key, value) on the low key_bits bits.
void radix_sort_u64_u32(uint64_t* keys, uint32_t* vals, int64_t n, int key_bits,
                        cudaStream_t s);
// The same sort with all scratch in a fixed device array (no allocation).
void radix_sort_noalloc(uint64_t* keys, uint32_t* vals, int64_t n, int key_bits,
                        cudaStream_t s);

// ---------------------------------------------------------------------------
// Kernel function parameters
// ---------------------------------------------------------------------------
struct KernelParams {
    int kernel;    // HM_GAUSSIAN | HM_MATERN32 | HM_MATERN_K1
    double c64;    // 1/l^2 (Gaussian), sqrt(3)/l (Matern-3/2) or 1/(4 l^2) (Matern K_1)
    float c32;
    int dmax = 3;  // largest dimension of the handle's point sets (the planes
                   // above it hold zeros, so kernels may skip them)
};

KernelParams make_kernel_params(int kernel, double ell);

// Block descriptor in absolute Morton rows / columns.
struct Blk {
    int64_t row0, col0;
    int32_t m, n;
};

// ---------------------------------------------------------------------------
// Structure of one point set (built by build_structure in hm_build.cu).
// ---------------------------------------------------------------------------
struct SetStructure {
    int64_t N = 0;
    int d = 0, C = 0, depth = 0;
    int64_t n_nodes = 0;
    int64_t row0 = 0;      // first Morton row of this set in the concatenation
    int64_t node0 = 0;     // first node of this set in the node arrays
    int64_t n_adm = 0, n_dense = 0;
    int traversal_reruns = 0;  // traversals run again with larger level bounds
};

}  // namespace hm
