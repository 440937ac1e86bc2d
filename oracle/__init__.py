"""CPU oracle of the H-matrix build and H-MVP (test infrastructure only).

Thin numpy/ctypes wrapper around ``hm_oracle.c``: plain single-threaded C in
double precision, compiled with ``-ffp-contract=off``. Only the test suite, the
package smoke check and the benchmark's CPU-baseline leg use it; the CUDA
library never imports, links or calls anything here.

Parity unpinned: the paper prints no numeric worked example, so no value here
is checked against a number the paper prints; every function is pinned instead
by closed forms, invariants, library routines and brute force (tests/
test_oracle_*.py and the fixtures in tests/golden/).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libhm_oracle.so")
_SRC = os.path.join(_HERE, "hm_oracle.c")

NPARAM = 4801


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (force or not os.path.exists(_SO)
            or os.path.getmtime(_SO) < max(os.path.getmtime(_SRC),
                                           os.path.getmtime(_SRC[:-1] + "h"))):
        tmp = _SO + ".%d.tmp" % os.getpid()
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                "-shared", _SRC, "-o", tmp, "-lm"]
        # OpenMP only spreads the block loops over threads when asked
        # (set_threads); without it the same code runs on one thread
        if subprocess.run(base + ["-fopenmp"], capture_output=True).returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


_d = C.POINTER(C.c_double)
_i64 = C.POINTER(C.c_int64)
_u64 = C.POINTER(C.c_uint64)
_i32 = C.POINTER(C.c_int32)


def _declare(L):
    L.or_kernel_eval.restype = C.c_double
    L.or_kernel_eval.argtypes = [C.c_int, C.c_double, _d, _d, C.c_int]
    L.or_morton.restype = C.c_int
    L.or_morton.argtypes = [_d, C.c_int64, C.c_int, _u64, _d, _d, _d]
    L.or_sort.argtypes = [_u64, C.c_int64, _i64]
    L.or_tree_depth.restype = C.c_int
    L.or_tree_depth.argtypes = [C.c_int64, C.c_int]
    L.or_tree_nodes.restype = C.c_int64
    L.or_tree_nodes.argtypes = [C.c_int64, C.c_int]
    L.or_tree_ranges.argtypes = [C.c_int64, C.c_int, _i64, _i64]
    L.or_bbox.argtypes = [_d, C.c_int64, C.c_int, C.c_int, _i64, _i64, _d, _d]
    L.or_admissible.restype = C.c_int
    L.or_admissible.argtypes = [_d, _d, _d, _d, C.c_int, C.c_double, C.c_int]
    L.or_aca_dense.restype = C.c_int
    L.or_aca_dense.argtypes = [_d, C.c_int64, C.c_int64, C.c_double, C.c_int,
                               C.c_double, C.c_double, _d, _d, _i64, _i64, _i64]
    L.or_build.restype = C.c_void_p
    L.or_build.argtypes = [_d, C.c_int64, C.c_int, C.c_int, _d, C.c_int,
                           C.c_double, C.c_int, C.c_double, C.c_int,
                           C.c_double, C.c_double]
    L.or_build_rect.restype = C.c_void_p
    L.or_build_rect.argtypes = [_d, C.c_int64, _d, C.c_int64, C.c_int, C.c_int, _d, C.c_int,
                                C.c_double, C.c_int, C.c_double, C.c_int,
                                C.c_double, C.c_double]
    L.or_build_structure_rect.restype = C.c_void_p
    L.or_build_structure_rect.argtypes = [_d, C.c_int64, _d, C.c_int64, C.c_int, C.c_int, _d,
                                          C.c_int, C.c_double, C.c_int]
    for f in ("or_n_cols", "or_n_nodes_cols"):
        getattr(L, f).restype = C.c_int64
        getattr(L, f).argtypes = [C.c_void_p]
    L.or_get_col_perm.argtypes = [C.c_void_p, _i64]
    L.or_get_col_tree.argtypes = [C.c_void_p, _i64, _i64, _d, _d]
    L.or_dense_matvec_rect.argtypes = [_d, C.c_int64, _d, C.c_int64, C.c_int, C.c_int, _d,
                                       _d, _d]
    L.or_build_structure.restype = C.c_void_p
    L.or_build_structure.argtypes = [_d, C.c_int64, C.c_int, C.c_int, _d,
                                     C.c_int, C.c_double, C.c_int]
    L.or_compress_range.argtypes = [C.c_void_p, C.c_int64, C.c_int64,
                                    C.c_double, C.c_int, C.c_double, C.c_double]
    L.or_compress_ids.argtypes = [C.c_void_p, _i64, C.c_int64,
                                  C.c_double, C.c_int, C.c_double, C.c_double]
    L.or_set_threads.argtypes = [C.c_int]
    L.or_free.argtypes = [C.c_void_p]
    L.or_mirror_transposed.argtypes = [C.c_void_p]
    for f in ("or_n_adm", "or_n_dense", "or_n_nodes"):
        getattr(L, f).restype = C.c_int64
        getattr(L, f).argtypes = [C.c_void_p]
    L.or_get_codes.argtypes = [C.c_void_p, _u64]
    L.or_get_perm.argtypes = [C.c_void_p, _i64]
    L.or_get_coords.argtypes = [C.c_void_p, _d]
    L.or_get_tree.argtypes = [C.c_void_p, _i64, _i64, _d, _d]
    L.or_get_adm.argtypes = [C.c_void_p, _i64]
    L.or_get_dense.argtypes = [C.c_void_p, _i64]
    L.or_get_ranks.argtypes = [C.c_void_p, _i32, _i64]
    L.or_get_factors.argtypes = [C.c_void_p, C.c_int64, _d, _d]
    L.or_get_pivots.argtypes = [C.c_void_p, C.c_int64, _i64, _i64]
    L.or_matvec.argtypes = [C.c_void_p, _d, _d]
    L.or_matvec_rows.argtypes = [C.c_void_p, _d, C.c_int64, C.c_int64, _d]
    L.or_dense_matvec.argtypes = [_d, C.c_int64, C.c_int, C.c_int, _d, _d, _d]
    L.or_dense_rows.argtypes = [_d, C.c_int64, C.c_int, C.c_int, _d, _i64,
                                C.c_int64, _d, _d]
    L.or_cg.restype = C.c_int
    L.or_cg.argtypes = [C.c_void_p, _d, _d, C.c_double, C.c_int, _d]
    L.or_block_features.argtypes = [C.c_void_p, C.c_double, _d]
    L.or_mlp_forward.argtypes = [_d, _d, C.c_int64, _d]
    L.or_mlp_loss_grad.restype = C.c_double
    L.or_mlp_loss_grad.argtypes = [_d, _d, _d, C.c_int64, _d]
    L.or_adam_step.argtypes = [_d, _d, _d, _d, C.c_int64, C.c_int64,
                               C.c_double, C.c_double, C.c_double, C.c_double]


def _p(a, t=_d):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# Step-level functions
# ---------------------------------------------------------------------------

def kernel_eval(kernel: int, ell: float, a, b) -> float:
    a = _f64(a)
    b = _f64(b)
    return lib().or_kernel_eval(kernel, ell, _p(a), _p(b), a.size)


def morton(pts):
    pts = _f64(pts)
    n, d = pts.shape
    codes = np.zeros(n, np.uint64)
    lo, hi, sc = np.zeros(d), np.zeros(d), np.zeros(d)
    bits = lib().or_morton(_p(pts), n, d, _p(codes, _u64), _p(lo), _p(hi), _p(sc))
    return codes, bits, lo, hi, sc


def sort(codes):
    codes = np.ascontiguousarray(codes, dtype=np.uint64)
    perm = np.zeros(codes.size, np.int64)
    lib().or_sort(_p(codes, _u64), codes.size, _p(perm, _i64))
    return perm


def tree_depth(n: int, leaf: int) -> int:
    return lib().or_tree_depth(n, leaf)


def tree_ranges(n: int, leaf: int):
    nn = lib().or_tree_nodes(n, leaf)
    lo = np.zeros(nn, np.int64)
    hi = np.zeros(nn, np.int64)
    lib().or_tree_ranges(n, leaf, _p(lo, _i64), _p(hi, _i64))
    return lo, hi


def bbox(coords_m, leaf: int):
    coords_m = _f64(coords_m)
    n, d = coords_m.shape
    lo, hi = tree_ranges(n, leaf)
    bmin = np.zeros((lo.size, d))
    bmax = np.zeros((lo.size, d))
    lib().or_bbox(_p(coords_m), n, d, leaf, _p(lo, _i64), _p(hi, _i64),
                  _p(bmin), _p(bmax))
    return lo, hi, bmin, bmax


def admissible(amin, amax, bmin, bmax, eta: float, use_max: bool = False) -> bool:
    amin, amax, bmin, bmax = map(_f64, (amin, amax, bmin, bmax))
    return bool(lib().or_admissible(_p(amin), _p(amax), _p(bmin), _p(bmax),
                                    amin.size, eta * eta, int(use_max)))


def aca_dense(A, eps: float, k_cap: int = 64, aca_eta: float = 0.0,
              eps0: float = 0.0):
    """ACA (Alg. 2) of an explicit (m, n) matrix. Returns U, V, pivots, n_rej."""
    A = np.asfortranarray(A, dtype=np.float64)
    m, n = A.shape
    U = np.zeros((k_cap, m))
    V = np.zeros((k_cap, n))
    pi = np.zeros(k_cap, np.int64)
    pj = np.zeros(k_cap, np.int64)
    rej = np.zeros(1, np.int64)
    r = lib().or_aca_dense(A.ctypes.data_as(_d), m, n, eps, k_cap, aca_eta,
                           eps0, _p(U), _p(V), _p(pi, _i64), _p(pj, _i64),
                           _p(rej, _i64))
    return U[:r].T.copy(), V[:r].T.copy(), pi[:r], pj[:r], int(rej[0])


def dense_matvec(pts, kernel: int, ell: float, sigma2: float, x):
    pts = _f64(pts)
    x = _f64(x)
    n, d = pts.shape
    y = np.zeros(n)
    prm = np.array([ell, sigma2])
    lib().or_dense_matvec(_p(pts), n, d, kernel, _p(prm), _p(x), _p(y))
    return y


def dense_matvec_rect(rows, cols, kernel: int, ell: float, x):
    """Brute force y = A_{phi, Y1 x Y2} x, rows = Y1 (N1, d), cols = Y2 (N2, d)."""
    rows = _f64(rows)
    cols = _f64(cols)
    x = _f64(x)
    y = np.zeros(rows.shape[0])
    prm = np.array([ell, 0.0])
    lib().or_dense_matvec_rect(_p(rows), rows.shape[0], _p(cols), cols.shape[0], rows.shape[1],
                               kernel, _p(prm), _p(x), _p(y))
    return y


def dense_rows(pts, kernel: int, ell: float, sigma2: float, rows, x):
    pts = _f64(pts)
    x = _f64(x)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    n, d = pts.shape
    y = np.zeros(rows.size)
    prm = np.array([ell, sigma2])
    lib().or_dense_rows(_p(pts), n, d, kernel, _p(prm), _p(rows, _i64),
                        rows.size, _p(x), _p(y))
    return y


# ---------------------------------------------------------------------------
# Whole H-matrix
# ---------------------------------------------------------------------------

class HMatrix:
    """Oracle H-matrix: Morton/sort/tree/Alg. 1 structure plus Alg. 2 factors."""

    def __init__(self, pts, kernel: int, ell: float, leaf: int, eta: float,
                 aca_eps: float, sigma2: float = 0.0, adm_max: bool = False,
                 k_cap: int = 64, aca_eta: float = 0.0, eps0: float = 0.0,
                 compress: bool = True, symmetric: bool = False, cols=None):
        """cols: a second point set Y2 for A_{phi, Y1 x Y2} (pts = Y1); the
        product then maps x of length len(cols) to y of length len(pts)."""
        self.pts = _f64(pts)
        self.n, self.d = self.pts.shape
        self.cols = None if cols is None else _f64(cols)
        self.kernel, self.ell, self.leaf, self.eta = kernel, ell, leaf, eta
        self.aca_eps, self.sigma2, self.k_cap = aca_eps, sigma2, k_cap
        prm = np.array([ell, sigma2])
        L = lib()
        if self.cols is not None:
            n2 = self.cols.shape[0]
            if compress:
                self._h = L.or_build_rect(_p(self.pts), self.n, _p(self.cols), n2, self.d,
                                          kernel, _p(prm), leaf, eta, int(adm_max), aca_eps,
                                          k_cap, aca_eta, eps0)
            else:
                self._h = L.or_build_structure_rect(_p(self.pts), self.n, _p(self.cols), n2,
                                                    self.d, kernel, _p(prm), leaf, eta,
                                                    int(adm_max))
        elif compress:
            self._h = L.or_build(_p(self.pts), self.n, self.d, kernel, _p(prm),
                                 leaf, eta, int(adm_max), aca_eps, k_cap,
                                 aca_eta, eps0)
            if symmetric:
                L.or_mirror_transposed(self._h)
        else:
            self._h = L.or_build_structure(_p(self.pts), self.n, self.d, kernel,
                                           _p(prm), leaf, eta, int(adm_max))
        self.n_adm = L.or_n_adm(self._h)
        self.n_dense = L.or_n_dense(self._h)
        self.n_nodes = L.or_n_nodes(self._h)
        self.n_cols = L.or_n_cols(self._h)
        self.n_nodes_cols = L.or_n_nodes_cols(self._h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_free(h)
            self._h = None

    def compress_range(self, b0: int, b1: int, aca_eps=None, k_cap=None,
                       aca_eta: float = 0.0, eps0: float = 0.0):
        lib().or_compress_range(self._h, b0, b1,
                                self.aca_eps if aca_eps is None else aca_eps,
                                self.k_cap if k_cap is None else k_cap,
                                aca_eta, eps0)

    def compress_ids(self, ids, aca_eps=None, k_cap=None, aca_eta: float = 0.0,
                     eps0: float = 0.0):
        """ACA of the listed admissible leaves (the factors of earlier calls
        are dropped), on the threads set by set_threads."""
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        lib().or_compress_ids(self._h, _p(ids, _i64), ids.size,
                              self.aca_eps if aca_eps is None else aca_eps,
                              self.k_cap if k_cap is None else k_cap, aca_eta, eps0)

    def codes(self):
        c = np.zeros(self.n, np.uint64)
        lib().or_get_codes(self._h, _p(c, _u64))
        return c

    def perm(self):
        p = np.zeros(self.n, np.int64)
        lib().or_get_perm(self._h, _p(p, _i64))
        return p

    def coords(self):
        c = np.zeros((self.n, self.d))
        lib().or_get_coords(self._h, _p(c))
        return c

    def col_perm(self):
        p = np.zeros(self.n_cols, np.int64)
        lib().or_get_col_perm(self._h, _p(p, _i64))
        return p

    def col_tree(self):
        k = self.n_nodes_cols
        lo = np.zeros(k, np.int64)
        hi = np.zeros(k, np.int64)
        bmin = np.zeros((k, self.d))
        bmax = np.zeros((k, self.d))
        lib().or_get_col_tree(self._h, _p(lo, _i64), _p(hi, _i64), _p(bmin), _p(bmax))
        return lo, hi, bmin, bmax

    def tree(self):
        lo = np.zeros(self.n_nodes, np.int64)
        hi = np.zeros(self.n_nodes, np.int64)
        bmin = np.zeros((self.n_nodes, self.d))
        bmax = np.zeros((self.n_nodes, self.d))
        lib().or_get_tree(self._h, _p(lo, _i64), _p(hi, _i64), _p(bmin), _p(bmax))
        return lo, hi, bmin, bmax

    def adm_leaves(self):
        a = np.zeros((max(self.n_adm, 1), 2), np.int64)
        lib().or_get_adm(self._h, _p(a, _i64))
        return a[: self.n_adm]

    def dense_leaves(self):
        a = np.zeros((max(self.n_dense, 1), 2), np.int64)
        lib().or_get_dense(self._h, _p(a, _i64))
        return a[: self.n_dense]

    def ranks(self):
        r = np.zeros(max(self.n_adm, 1), np.int32)
        rej = np.zeros(max(self.n_adm, 1), np.int64)
        lib().or_get_ranks(self._h, _p(r, _i32), _p(rej, _i64))
        return r[: self.n_adm], rej[: self.n_adm]

    def factors(self, b: int):
        lo, hi, _, _ = self.tree()
        lo2, hi2, _, _ = self.col_tree()
        t, s = self.adm_leaves()[b]
        m, n = hi[t] - lo[t], hi2[s] - lo2[s]
        r = int(self.ranks()[0][b])
        U = np.zeros((r, m))
        V = np.zeros((r, n))
        lib().or_get_factors(self._h, b, _p(U), _p(V))
        return U.T.copy(), V.T.copy()

    def pivots(self, b: int):
        r = int(self.ranks()[0][b])
        pi = np.zeros(max(r, 1), np.int64)
        pj = np.zeros(max(r, 1), np.int64)
        lib().or_get_pivots(self._h, b, _p(pi, _i64), _p(pj, _i64))
        return pi[:r], pj[:r]

    def matvec(self, x):
        x = _f64(x)
        y = np.zeros(self.n)
        lib().or_matvec(self._h, _p(x), _p(y))
        return y

    def matvec_rows(self, xm, r0: int, r1: int):
        """Rows [r0, r1) of the Morton-ordered product from the Morton-ordered
        x_m, from the leaves that touch them (a block-row share)."""
        xm = _f64(xm)
        y = np.zeros(max(r1 - r0, 0))
        lib().or_matvec_rows(self._h, _p(xm), r0, r1, _p(y))
        return y

    def cg(self, b, rtol: float = 1e-6, maxit: int = 1000, x0=None):
        b = _f64(b)
        x = np.zeros(self.n) if x0 is None else _f64(x0).copy()
        rr = np.zeros(1)
        it = lib().or_cg(self._h, _p(b), _p(x), rtol, maxit, _p(rr))
        return x, it, float(rr[0])

    def features(self):
        f = np.zeros((max(self.n_adm, 1), 8))
        lib().or_block_features(self._h, self.aca_eps, _p(f))
        return f[: self.n_adm]


# ---------------------------------------------------------------------------
# Rank-model MLP
# ---------------------------------------------------------------------------

def set_threads(n: int) -> None:
    """Threads of the oracle's block loops (ACA and the product); 1 = the
    plain loops. Used to time the oracle on all host cores."""
    lib().or_set_threads(int(n))


def mlp_forward(theta, F):
    theta = _f64(theta)
    F = _f64(F)
    out = np.zeros(F.shape[0])
    lib().or_mlp_forward(_p(theta), _p(F), F.shape[0], _p(out))
    return out


def mlp_loss_grad(theta, F, target):
    theta, F, target = _f64(theta), _f64(F), _f64(target)
    g = np.zeros(NPARAM)
    loss = lib().or_mlp_loss_grad(_p(theta), _p(F), _p(target), F.shape[0], _p(g))
    return loss, g


def adam_step(theta, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam step on float64 arrays theta, m, v."""
    grad = _f64(grad)
    lib().or_adam_step(_p(theta), _p(grad), _p(m), _p(v), theta.size, t, lr,
                       b1, b2, eps)
