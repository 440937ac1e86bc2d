"""ctypes binding of libhm.so (include/hm.h): argument marshalling only.

Every step of the build and the product runs in the CUDA library; this module
converts numpy arrays / torch tensors into pointers, fills the option struct
and turns negative status codes into exceptions. There is no CPU fallback:
if the library is missing, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

GAUSSIAN, MATERN32, MATERN_K1 = 0, 1, 2
PREC_FP64, PREC_MIXED = 0, 1
NEAR_AUTO, NEAR_FP64, NEAR_FP32, NEAR_BF16X2, NEAR_BF16 = range(5)
MLP_NPARAM = 4801
OK, EINVAL, ENOMEM, EOVERFLOW, ECUDA, ETIMEOUT, ENOTSUP = 0, -1, -2, -3, -4, -5, -6

_STATUS = {0: "HM_OK", -1: "HM_EINVAL", -2: "HM_ENOMEM", -3: "HM_EOVERFLOW",
           -4: "HM_ECUDA", -5: "HM_ETIMEOUT", -6: "HM_ENOTSUP"}


class HMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (_STATUS.get(code, code), msg))
        self.code = code


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("near_format", C.c_int),
                ("adm_max", C.c_int), ("k_cap", C.c_int),
                ("aca_eta", C.c_double), ("eps0", C.c_double),
                ("accumulate", C.c_int), ("rank_model", C.c_int),
                ("rank_model_theta", C.c_void_p), ("scratch_gb", C.c_double),
                ("stream", C.c_void_p), ("profile", C.c_int),
                ("structure_only", C.c_int), ("symmetric", C.c_int),
                ("on_the_fly", C.c_int), ("row_lo", C.c_int64), ("row_hi", C.c_int64)]


class Stats(C.Structure):
    _fields_ = [("n_points", C.c_int64), ("n_nodes", C.c_int64),
                ("n_adm", C.c_int64), ("n_dense", C.c_int64),
                ("n_tiles", C.c_int64), ("depth", C.c_int), ("d", C.c_int),
                ("sum_rank", C.c_int64), ("max_rank", C.c_int),
                ("rank_cap_hits", C.c_int64), ("n_rejected", C.c_int64),
                ("n_mispredicted", C.c_int64), ("factor_entries", C.c_int64),
                ("near_entries", C.c_int64), ("factor_bytes", C.c_int64),
                ("near_bytes", C.c_int64), ("mvp_bytes", C.c_int64),
                ("reserved_factor_entries", C.c_int64),
                ("t_structure_ms", C.c_double), ("t_aca_ms", C.c_double),
                ("t_dense_ms", C.c_double), ("t_total_ms", C.c_double),
                ("aca_passes", C.c_int), ("precision", C.c_int),
                ("near_format", C.c_int), ("aca_evals", C.c_int64),
                ("aca_flops", C.c_double), ("mvp_count", C.c_int64),
                ("t_mvp_ms", C.c_double), ("t_mvp_gather_ms", C.c_double),
                ("t_mvp_vtx_ms", C.c_double), ("t_mvp_tile_ms", C.c_double),
                ("mvp_vtx_bytes", C.c_int64), ("mvp_tile_bytes", C.c_int64),
                ("t_aca_class_ms", C.c_double * 12),
                ("t_np_aca_ms", C.c_double), ("t_np_lowrank_ms", C.c_double),
                ("t_np_near_ms", C.c_double), ("traversal_reruns", C.c_int),
                ("t_mvp_tail_ms", C.c_double), ("mvp_tail_bytes", C.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["t_aca_class_ms"] = list(self.t_aca_class_ms)
        return d


_lib = None
_vp = C.c_void_p


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libhm.so (built by __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError("libhm.so not built: run python -m paper_1708_09707_gb300.build")
        L = C.CDLL(path)
        _declare(L)
        _lib = L
    return _lib


def _declare(L):
    i64, pi = C.c_int64, C.POINTER(C.c_int)
    L.hm_options_default.argtypes = [C.POINTER(Options)]
    L.hm_last_error.restype = C.c_char_p
    L.hm_kernel_launches.restype = C.c_uint64
    L.hm_set_gather_shape.argtypes = [C.c_int]
    L.hm_set_aca_shape.argtypes = [C.c_int, C.c_int]
    L.hm_set_test_hook.argtypes = [C.c_int, C.c_int64]
    L.hm_set_batch_limits.argtypes = [C.c_int64, C.c_int64]
    L.hm_tune_aca_shapes.argtypes = [_vp, i64, C.c_int, C.c_int, _vp, C.c_int, C.c_double,
                                     C.c_double, C.POINTER(Options), C.c_int, _vp]
    L.hm_check_status.argtypes = [_vp]
    L.hm_device_bytes.restype = C.c_uint64
    L.hm_device_bytes.argtypes = []
    L.hm_alu_peak.argtypes = [C.c_int, C.POINTER(C.c_double)]
    L.hm_build_ex.restype = _vp
    L.hm_build_ex.argtypes = [_vp, i64, C.c_int, C.c_int, _vp, C.c_int, C.c_double,
                              C.c_double, C.POINTER(Options), pi]
    L.hm_build_rect.restype = _vp
    L.hm_build_rect.argtypes = [_vp, i64, _vp, i64, C.c_int, C.c_int, _vp, C.c_int, C.c_double,
                                C.c_double, C.POINTER(Options), pi]
    L.hm_build.restype = _vp
    L.hm_build.argtypes = [_vp, i64, C.c_int, C.c_int, _vp, C.c_int, C.c_double, C.c_double]
    L.hm_matvec.argtypes = [_vp, _vp, _vp]
    L.hm_matvec_ex.argtypes = [_vp, _vp, _vp, C.c_int, _vp]
    L.hm_free.argtypes = [_vp]
    L.hm_get_stats.argtypes = [_vp, C.POINTER(Stats)]
    L.hm_export_structure.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
    L.hm_export_tree.argtypes = [_vp, _vp, _vp, _vp, _vp]
    L.hm_export_factors.argtypes = [_vp, i64, _vp, _vp, pi]
    L.hm_cg.argtypes = [_vp, _vp, _vp, C.c_double, C.c_int, pi, C.POINTER(C.c_double)]
    L.hm_build_batch.restype = _vp
    L.hm_build_batch.argtypes = [C.c_int, _vp, _vp, _vp, C.c_int, _vp, C.c_int, C.c_double,
                                 C.c_double, C.POINTER(Options), pi]
    L.hm_matvec_batch.argtypes = [_vp, _vp, _vp]
    L.hm_batch_stats.argtypes = [_vp, C.POINTER(Stats)]
    L.hm_free_batch.argtypes = [_vp]
    L.hm_block_features.argtypes = [_vp, _vp, _vp]
    L.hm_mlp_forward.argtypes = [_vp, _vp, i64, _vp, _vp]
    L.hm_mlp_loss_grad.argtypes = [_vp, _vp, _vp, i64, _vp, _vp, _vp]
    L.hm_mlp_adam.argtypes = [_vp, _vp, _vp, _vp, i64, C.c_float, C.c_float, C.c_float,
                              C.c_float, _vp]
    L.hm_morton_codes.argtypes = [_vp, i64, C.c_int, _vp, _vp]
    L.hm_radix_sort_pairs.argtypes = [_vp, _vp, i64, C.c_int, _vp]
    L.hm_radix_sort_pairs_noalloc.argtypes = [_vp, _vp, i64, C.c_int, _vp]


def _check(code: int):
    if code != 0:
        raise HMError(code, lib().hm_last_error().decode())


def _ptr(a):
    """Address of a numpy array or torch tensor (must be contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return a.data_ptr()


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _stream_ptr(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


def options(precision=PREC_FP64, near_format=NEAR_AUTO, adm_max=False, k_cap=64,
            aca_eta=0.0, eps0=0.0, accumulate=False, rank_model_theta=None,
            scratch_gb=0.0, stream=None, profile=False, symmetric=False,
            structure_only=False, on_the_fly=False, row_range=None) -> Options:
    o = Options()
    lib().hm_options_default(C.byref(o))
    o.precision = precision
    o.near_format = near_format
    o.adm_max = int(adm_max)
    o.k_cap = k_cap
    o.aca_eta = aca_eta
    o.eps0 = eps0
    o.accumulate = int(accumulate)
    o.rank_model = int(rank_model_theta is not None)
    o.rank_model_theta = _ptr(rank_model_theta)
    o.scratch_gb = scratch_gb
    o.stream = _stream_ptr(stream)
    o.profile = int(profile)
    o.symmetric = int(symmetric)
    o.structure_only = int(structure_only)
    o.on_the_fly = int(on_the_fly)
    if row_range is not None:
        o.row_lo, o.row_hi = int(row_range[0]), int(row_range[1])
    return o


class HMatrix:
    """H-matrix of A_{phi, Y x Y} (+ sigma^2 I) built on the GPU (hm_build_ex),
    or of A_{phi, Y1 x Y2} with cols = Y2 (hm_build_rect; points = Y1).

    points: (N, d) float64 numpy array (host) or torch tensor (host or cuda).
    """

    def __init__(self, points, kernel: int, ell: float, leaf: int, eta: float,
                 aca_eps: float, sigma2: float = 0.0, cols=None, **opts):
        L = lib()
        if isinstance(points, np.ndarray):
            points = np.ascontiguousarray(points, dtype=np.float64)
        if isinstance(cols, np.ndarray):
            cols = np.ascontiguousarray(cols, dtype=np.float64)
        self.n, self.d = int(points.shape[0]), int(points.shape[1])
        self.rect = cols is not None
        self.n_cols = int(cols.shape[0]) if self.rect else self.n
        self._theta = opts.get("rank_model_theta")
        self.opt = options(**opts)
        prm = np.array([ell, sigma2], dtype=np.float64)
        st = C.c_int(0)
        if self.rect:
            if int(cols.shape[1]) != self.d:
                raise HMError(-1, "both point sets need the same dimension")
            self._h = L.hm_build_rect(_ptr(points), self.n, _ptr(cols), self.n_cols, self.d,
                                      kernel, prm.ctypes.data, leaf, eta, aca_eps,
                                      C.byref(self.opt), C.byref(st))
        else:
            self._h = L.hm_build_ex(_ptr(points), self.n, self.d, kernel, prm.ctypes.data, leaf,
                                    eta, aca_eps, C.byref(self.opt), C.byref(st))
        if not self._h:
            raise HMError(st.value, L.hm_last_error().decode())
        self.kernel, self.ell, self.leaf, self.eta = kernel, ell, leaf, eta
        self.aca_eps, self.sigma2 = aca_eps, sigma2

    def free(self):
        if getattr(self, "_h", None):
            lib().hm_free(self._h)
            self._h = None

    __del__ = free

    def matvec(self, x, y=None, stream=None):
        """y = H x + sigma^2 x; numpy in -> numpy out, torch in -> torch out.
        For two point sets x has n_cols entries per vector and y n."""
        if _is_torch(x):
            import torch
            nrhs = 1 if x.dim() == 1 else x.shape[0]
            if y is None:
                shape = (self.n,) if x.dim() == 1 else (nrhs, self.n)
                y = torch.empty(shape, dtype=x.dtype, device=x.device)
        else:
            x = np.ascontiguousarray(x, dtype=np.float64)
            nrhs = 1 if x.ndim == 1 else x.shape[0]
            if y is None:
                y = np.empty((self.n,) if x.ndim == 1 else (nrhs, self.n))
        _check(lib().hm_matvec_ex(self._h, _ptr(x), _ptr(y), nrhs, _stream_ptr(stream)))
        return y

    def check_status(self) -> None:
        """hm_check_status: raise HMError(HM_ETIMEOUT) if a bounded device
        loop or wait of an earlier call gave up."""
        _check(lib().hm_check_status(self._h))

    def stats(self) -> dict:
        s = Stats()
        _check(lib().hm_get_stats(self._h, C.byref(s)))
        return s.as_dict()

    def structure(self):
        st = self.stats()
        ntot = self.n + self.n_cols if self.rect else self.n
        codes = np.zeros(ntot, np.uint64)
        perm = np.zeros(ntot, np.int64)
        adm = np.zeros((max(st["n_adm"], 1), 2), np.int64)
        dense = np.zeros((max(st["n_dense"], 1), 2), np.int64)
        ranks = np.zeros(max(st["n_adm"], 1), np.int32)
        _check(lib().hm_export_structure(self._h, _ptr(codes), _ptr(perm), _ptr(adm),
                                         _ptr(dense), _ptr(ranks)))
        return dict(codes=codes, perm=perm, adm=adm[: st["n_adm"]],
                    dense=dense[: st["n_dense"]], ranks=ranks[: st["n_adm"]])

    def tree(self):
        nn = self.stats()["n_nodes"]
        lo = np.zeros(nn, np.int64)
        hi = np.zeros(nn, np.int64)
        bmin = np.zeros((nn, self.d))
        bmax = np.zeros((nn, self.d))
        _check(lib().hm_export_tree(self._h, _ptr(lo), _ptr(hi), _ptr(bmin), _ptr(bmax)))
        return lo, hi, bmin, bmax

    def factors(self, b: int, m: int, n: int):
        k = self.opt.k_cap
        U = np.zeros((k, m))
        V = np.zeros((k, n))
        r = C.c_int(0)
        _check(lib().hm_export_factors(self._h, b, _ptr(U), _ptr(V), C.byref(r)))
        r = r.value
        return (U.reshape(-1)[: r * m].reshape(r, m).T.copy(),
                V.reshape(-1)[: r * n].reshape(r, n).T.copy())

    def cg(self, b, rtol=1e-6, maxit=1000, x0=None):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.n) if x0 is None else np.array(x0, dtype=np.float64)
        it = C.c_int(0)
        rr = C.c_double(0)
        _check(lib().hm_cg(self._h, _ptr(b), _ptr(x), rtol, maxit, C.byref(it), C.byref(rr)))
        return x, it.value, rr.value

    def features(self):
        na = self.stats()["n_adm"]
        F = np.zeros((max(na, 1), 8), np.float32)
        T = np.zeros(max(na, 1), np.float32)
        _check(lib().hm_block_features(self._h, _ptr(F), _ptr(T)))
        return F[:na], T[:na]


class HBatch:
    """Many independent point sets built and multiplied together."""

    def __init__(self, point_sets, kernel: int, ell: float, leaf: int, eta: float,
                 aca_eps: float, sigma2: float = 0.0, flat=None, sizes=None, dims=None,
                 **opts):
        """point_sets: list of (N_s, d_s) arrays; or None with flat (the sets
        one after another, row-major; numpy or a host / cuda torch tensor),
        sizes and dims."""
        L = lib()
        if point_sets is not None:
            self.sizes = np.array([p.shape[0] for p in point_sets], np.int64)
            self.dims = np.array([p.shape[1] for p in point_sets], np.int32)
            allp = np.ascontiguousarray(np.concatenate([np.asarray(p, np.float64).ravel()
                                                        for p in point_sets]))
        else:
            self.sizes = np.asarray(sizes, np.int64)
            self.dims = np.asarray(dims, np.int32)
            allp = flat if _is_torch(flat) else np.ascontiguousarray(flat, dtype=np.float64)
            npt = int((self.sizes * self.dims).sum())
            assert allp.numel() == npt if _is_torch(allp) else allp.size == npt
        self.opt = options(**opts)
        prm = np.array([ell, sigma2], dtype=np.float64)
        st = C.c_int(0)
        self._b = L.hm_build_batch(len(self.sizes), _ptr(allp), _ptr(self.sizes),
                                   _ptr(self.dims), kernel, prm.ctypes.data, leaf, eta,
                                   aca_eps, C.byref(self.opt), C.byref(st))
        if not self._b:
            raise HMError(st.value, L.hm_last_error().decode())
        self.n = int(self.sizes.sum())

    def free(self):
        if getattr(self, "_b", None):
            lib().hm_free_batch(self._b)
            self._b = None

    __del__ = free

    def matvec(self, x, y=None):
        if _is_torch(x):
            import torch
            y = torch.empty_like(x) if y is None else y
        else:
            x = np.ascontiguousarray(x, dtype=np.float64)
            y = np.empty_like(x) if y is None else y
        _check(lib().hm_matvec_batch(self._b, _ptr(x), _ptr(y)))
        return y

    def stats(self) -> dict:
        s = Stats()
        _check(lib().hm_batch_stats(self._b, C.byref(s)))
        return s.as_dict()


# ------------------------------------------------------------- step helpers
def morton_codes(points_dev, codes_dev, stream=None):
    n, d = points_dev.shape
    _check(lib().hm_morton_codes(_ptr(points_dev), n, d, _ptr(codes_dev), _stream_ptr(stream)))


def radix_sort_pairs(keys_dev, vals_dev, key_bits: int, stream=None):
    _check(lib().hm_radix_sort_pairs(_ptr(keys_dev), _ptr(vals_dev), keys_dev.numel(),
                                     key_bits, _stream_ptr(stream)))


def radix_sort_pairs_noalloc(keys_dev, vals_dev, key_bits: int, stream=None):
    """hm_radix_sort_pairs_noalloc: the sort without any device allocation."""
    _check(lib().hm_radix_sort_pairs_noalloc(_ptr(keys_dev), _ptr(vals_dev), keys_dev.numel(),
                                             key_bits, _stream_ptr(stream)))


def mlp_forward(theta, F, out, stream=None):
    _check(lib().hm_mlp_forward(_ptr(theta), _ptr(F), F.shape[0], _ptr(out),
                                _stream_ptr(stream)))


def mlp_loss_grad(theta, F, target, grad, loss=None, stream=None):
    _check(lib().hm_mlp_loss_grad(_ptr(theta), _ptr(F), _ptr(target), F.shape[0], _ptr(grad),
                                  _ptr(loss), _stream_ptr(stream)))


def mlp_adam(theta, grad, m, v, t: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    _check(lib().hm_mlp_adam(_ptr(theta), _ptr(grad), _ptr(m), _ptr(v), t, lr, b1, b2, eps,
                             _stream_ptr(stream)))


def set_gather_shape(shape: int) -> None:
    """Force the product gather's launch shape (0..4), or -1 to tune."""
    _check(lib().hm_set_gather_shape(int(shape)))


def set_aca_shape(cls: int, shape: int) -> None:
    """hm_set_aca_shape: launch shape of the batched ACA of one size class
    (-1 every class); shape -1 default, 0 the cluster kernels, 1 the default team
    shape, 2 another team shape."""
    _check(lib().hm_set_aca_shape(int(cls), int(shape)))


def tune_aca_shapes(points, kernel: int, ell: float, leaf: int, eta: float, aca_eps: float,
                    sigma2: float = 0.0, reps: int = 2, **opts) -> list:
    """hm_tune_aca_shapes: time the ACA shapes 0, 1, 2 per size class on this
    problem (stored build, classes serial) and keep the fastest for later
    builds; returns the 12 chosen shapes (-1: empty class)."""
    import numpy as _np
    o = options(**opts)
    n, d = int(points.shape[0]), int(points.shape[1])
    if isinstance(points, _np.ndarray):
        points = _np.ascontiguousarray(points, dtype=_np.float64)
    prm = _np.array([ell, sigma2], _np.float64)
    out = (C.c_int * 12)()
    _check(lib().hm_tune_aca_shapes(_ptr(points), n, d, int(kernel), _ptr(prm), int(leaf),
                                    float(eta), float(aca_eps), C.byref(o), int(reps), out))
    return list(out)


def set_batch_limits(aca_entries: int = 0, gather_items: int = 0) -> None:
    """hm_set_batch_limits: reserved factor entries per ACA launch and work
    items per gather launch (0: one launch per size class / one gather
    launch); a control for the batching study, not part of the method."""
    _check(lib().hm_set_batch_limits(int(aca_entries), int(gather_items)))


HOOK_ACA_STEP_LIMIT, HOOK_WAIT_LIMIT_NS, HOOK_GATHER_WITHHOLD, HOOK_FAIL_ALLOC = 0, 1, 2, 3
HOOK_TRAVERSAL_KAPPA, HOOK_TRAVERSAL_TRIES = 4, 5


def set_test_hook(hook: int, value: int) -> None:
    """hm_set_test_hook: a test hook of the failure paths (0 restores the default)."""
    _check(lib().hm_set_test_hook(int(hook), int(value)))


def device_bytes() -> int:
    """hm_device_bytes: device bytes the library holds right now."""
    return int(lib().hm_device_bytes())


def kernel_launches() -> int:
    """Kernels the library has launched in this process."""
    return int(lib().hm_kernel_launches())


def alu_peak(precision: int = PREC_MIXED) -> float:
    """Measured FMA throughput (FLOP/s) of the current device (hm_alu_peak)."""
    v = C.c_double(0.0)
    _check(lib().hm_alu_peak(precision, C.byref(v)))
    return v.value
