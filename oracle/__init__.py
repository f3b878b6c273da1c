"""Python access to the LAMG+ CPU oracle (``lamg_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it. The CUDA library never imports, links or calls anything here.

The oracle is plain serial FP64 C compiled with ``gcc -O2 -ffp-contract=off`` (no fused
multiply-add contraction, no fast-math), loaded through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lamg_oracle.c")
_SO = os.path.join(_HERE, "liblamg_oracle.so")
_lock = threading.Lock()
_lib = None

DEFAULTS = dict(K=4, nu_tv=3, dmax=4, nu_pre=1, nu_post=2, coarsest_max=0, max_levels=100,
                veto=1, caliber2=1, tv_lex=0, symmetric=0, seed=3, dense_rows=4096,
                cheb_colours=32, cheb_degree=1,
                Q=2.5, tau_soc=0.05, elim_min_frac=0.01, snap=1e-3, guard_eps=1e-10,
                gamma_fixed=0.0)
_IKEYS = ["K", "nu_tv", "dmax", "nu_pre", "nu_post", "coarsest_max", "max_levels", "veto",
          "caliber2", "tv_lex", "symmetric", "seed", "dense_rows", "cheb_colours", "cheb_degree"]
_DKEYS = ["Q", "tau_soc", "elim_min_frac", "snap", "guard_eps", "gamma_fixed"]

KIND = {0: "elim", 1: "agg", 2: "coarsest"}


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            tmp = _SO + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        P = C.c_void_p
        L.oracle_setup.restype = C.c_int
        L.oracle_setup.argtypes = [C.c_int64, P, P, P, P, P, C.POINTER(C.c_void_p)]
        L.oracle_free.argtypes = [P]
        L.oracle_nlevels.restype = C.c_int
        L.oracle_nlevels.argtypes = [P]
        L.oracle_level_meta.argtypes = [P, C.c_int, P, P]
        L.oracle_level_array.restype = C.c_int64
        L.oracle_level_array.argtypes = [P, C.c_int, C.c_char_p, P]
        L.oracle_cycle.argtypes = [P, P, P]
        L.oracle_fcg.restype = C.c_int64
        L.oracle_fcg.argtypes = [P, P, P, C.c_double, C.c_int64, P, P]
        L.oracle_stationary.restype = C.c_int64
        L.oracle_stationary.argtypes = [P, P, P, C.c_double, C.c_int64, C.c_int, P, P]
        L.oracle_visit_counts.argtypes = [P, P]
        L.oracle_set_gamma.argtypes = [P, C.c_int, C.c_double]
        L.oracle_testvectors.argtypes = [C.c_int64, P, P, P, P, C.c_int, C.c_uint64, C.c_int, C.c_int, P]
        L.oracle_aggregate.restype = C.c_int64
        L.oracle_aggregate.argtypes = [C.c_int64, P, P, P, P, P, C.c_int, P, P, C.c_double, C.c_double, P]
        L.oracle_splitmix64.restype = C.c_uint64
        L.oracle_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
        L.oracle_random_start.restype = C.c_double
        L.oracle_random_start.argtypes = [C.c_uint64, C.c_int, C.c_int64, C.c_int]
        L.oracle_guard_q.restype = C.c_double
        L.oracle_guard_q.argtypes = [P, P, P, P, C.c_int, C.c_double]
        L.oracle_laplacian.restype = C.c_int
        L.oracle_laplacian.argtypes = [C.c_int64, P, P, P, P, P]
        L.oracle_colour.restype = C.c_int
        L.oracle_colour.argtypes = [C.c_int64, P, P, P]
        L.oracle_gs.argtypes = [C.c_int64, P, P, P, P, P, P, C.c_int, C.c_int]
        L.oracle_residual.argtypes = [C.c_int64, P, P, P, P, P, P, P]
        L.oracle_affinity.restype = C.c_double
        L.oracle_affinity.argtypes = [P, P, C.c_int]
        L.oracle_eliminate.restype = C.c_int64
        L.oracle_eliminate.argtypes = [C.c_int64, P, P, P, P, C.c_int, P, C.POINTER(C.c_void_p)]
        L.oracle_galerkin.restype = C.c_void_p
        L.oracle_galerkin.argtypes = [C.c_int64, P, P, P, P, C.c_int64, P, P, P]
        L.oracle_pinv.restype = C.c_int
        L.oracle_pinv.argtypes = [C.c_int64, P, P, P, P, P]
        L.oracle_cheb_apply.argtypes = [C.c_int64, P, P, P, P, C.c_int, P, P, P]
        L.oracle_mat_meta.argtypes = [P, P]
        L.oracle_mat_get.argtypes = [P, P, P, P, P]
        L.oracle_mat_free.argtypes = [P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class Matrix:
    """A level operator: off-diagonal CSR (rp, ci, val) plus the diagonal."""

    def __init__(self, rp, ci, val, diag):
        self.rp = _c(rp, np.int64); self.ci = _c(ci, np.int32)
        self.val = _c(val, np.float64); self.diag = _c(diag, np.float64)
        self.n = len(self.diag)

    def dense(self) -> np.ndarray:
        M = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rp))
        M[rows, self.ci] = self.val
        M[np.arange(self.n), np.arange(self.n)] += self.diag
        return M

    def args(self):
        return (self.n, _p(self.rp), _p(self.ci), _p(self.val), _p(self.diag))


def _take_mat(ptr) -> Matrix:
    L = lib()
    meta = np.zeros(2, np.int64)
    L.oracle_mat_meta(ptr, _p(meta))
    n, nnz = int(meta[0]), int(meta[1])
    rp = np.zeros(n + 1, np.int64); ci = np.zeros(nnz, np.int32)
    val = np.zeros(nnz); diag = np.zeros(n)
    L.oracle_mat_get(ptr, _p(rp), _p(ci), _p(val), _p(diag))
    L.oracle_mat_free(ptr)
    return Matrix(rp, ci, val, diag)


def laplacian(g) -> Matrix:
    """L = D - W of a graph from ``graphgen`` (Eq. 1)."""
    val = np.zeros(g.nnz_off); diag = np.zeros(g.n)
    rp, ci, w = _c(g.rp, np.int64), _c(g.ci, np.int32), _c(g.w, np.float64)
    rc = lib().oracle_laplacian(g.n, _p(rp), _p(ci), _p(w), _p(val), _p(diag))
    if rc:
        raise ValueError(f"invalid graph (code {rc})")
    return Matrix(rp, ci, val, diag)


def colour(A: Matrix):
    col = np.zeros(A.n, np.int32)
    nc = lib().oracle_colour(A.n, _p(A.rp), _p(A.ci), _p(col))
    return col, nc


def gs(A: Matrix, x, b=None, order: str = "forward", sweeps: int = 1) -> np.ndarray:
    x = _c(x, np.float64).copy()
    bb = None if b is None else _c(b, np.float64)
    o = {"forward": 0, "reverse": 1, "lex": 2}[order]
    lib().oracle_gs(*A.args(), _p(x), _p(bb), o, sweeps)
    return x


def residual(A: Matrix, x, b) -> np.ndarray:
    x = _c(x, np.float64); b = _c(b, np.float64)
    r = np.zeros(A.n)
    lib().oracle_residual(*A.args(), _p(x), _p(b), _p(r))
    return r


def affinity(xu, xv) -> float:
    xu = _c(xu, np.float64); xv = _c(xv, np.float64)
    return lib().oracle_affinity(_p(xu), _p(xv), len(xu))


def guard_q(s0: float, s1, s2, xs, guard_eps: float = 1e-10) -> float:
    s0a = np.array([s0], np.float64)
    s1 = _c(s1, np.float64); s2 = _c(s2, np.float64); xs = _c(xs, np.float64)
    return lib().oracle_guard_q(_p(s0a), _p(s1), _p(s2), _p(xs), len(s1), guard_eps)


def splitmix64(seed: int, i: int) -> int:
    return int(lib().oracle_splitmix64(seed & (2**64 - 1), i & (2**64 - 1)))


def random_start(seed: int, level: int, u: int, k: int) -> float:
    return lib().oracle_random_start(seed, level, u, k)


def eliminate(A: Matrix, dmax: int = 4):
    inF = np.zeros(A.n, np.uint8)
    ptr = C.c_void_p()
    nf = lib().oracle_eliminate(*A.args(), dmax, _p(inF), C.byref(ptr))
    return inF.astype(bool), int(nf), _take_mat(ptr)


def galerkin(A: Matrix, nc: int, agg, agg2=None, wt=None) -> Matrix:
    agg = _c(agg, np.int32)
    agg2 = _c(np.full(A.n, -1) if agg2 is None else agg2, np.int32)
    wt = _c(np.ones(A.n) if wt is None else wt, np.float64)
    ptr = lib().oracle_galerkin(*A.args(), nc, _p(agg), _p(agg2), _p(wt))
    return _take_mat(ptr)


def pinv(A: Matrix) -> np.ndarray:
    out = np.zeros((A.n, A.n))
    rc = lib().oracle_pinv(*A.args(), _p(out))
    if rc:
        raise ValueError("operator is not connected")
    return out


def testvectors(A: Matrix, level: int, seed: int = 3, K: int = 4, nu: int = 3) -> np.ndarray:
    """K test vectors of a level operator (greedy colour order, Section 2): n x K."""
    X = np.zeros((A.n, K))
    lib().oracle_testvectors(*A.args(), level, seed, K, nu, _p(X))
    return X


def aggregate(A: Matrix, X, aff, strong, Q: float = 2.5, guard_eps: float = 1e-10):
    """Caliber-1 aggregation on given test vectors, affinities and strong flags; returns
    (seed_of, number of aggregates)."""
    X = _c(X, np.float64); aff = _c(aff, np.float64); strong = _c(strong, np.uint8)
    seed_of = np.zeros(A.n, np.int32)
    nc = lib().oracle_aggregate(*A.args(), _p(X), X.shape[1], _p(aff), _p(strong), Q, guard_eps, _p(seed_of))
    return seed_of, int(nc)


def cheb_apply(A: Matrix, x, b, m: int = 2):
    """One Chebyshev smoothing polynomial of degree m on A x = b; returns (x, lambda)."""
    x = _c(x, np.float64).copy()
    b = _c(b, np.float64)
    coef = np.zeros(17)
    lib().oracle_cheb_apply(*A.args(), m, _p(x), _p(b), _p(coef))
    return x, float(coef[0])


class Hierarchy:
    """An oracle hierarchy built from a graph (Section 2 setup)."""

    def __init__(self, g, **opts):
        o = dict(DEFAULTS); o.update(opts)
        self.opts = o
        iopt = np.array([o[k] for k in _IKEYS], np.int64)
        dopt = np.array([o[k] for k in _DKEYS], np.float64)
        self._rp, self._ci, self._w = _c(g.rp, np.int64), _c(g.ci, np.int32), _c(g.w, np.float64)
        ptr = C.c_void_p()
        rc = lib().oracle_setup(g.n, _p(self._rp), _p(self._ci), _p(self._w), _p(iopt), _p(dopt),
                                C.byref(ptr))
        if rc:
            raise ValueError(f"oracle setup failed (code {rc})")
        self._h = ptr
        self.n = g.n
        self._levels = None

    def __del__(self):
        if getattr(self, "_h", None):
            lib().oracle_free(self._h)
            self._h = None

    @property
    def nlevels(self) -> int:
        return lib().oracle_nlevels(self._h)

    def level(self, l: int) -> dict:
        L = lib()
        meta = np.zeros(7, np.int64); dmeta = np.zeros(18)
        L.oracle_level_meta(self._h, l, _p(meta), _p(dmeta))
        d = dict(kind=KIND[int(meta[0])], n=int(meta[1]), nnz=int(meta[2]), ncol=int(meta[3]),
                 nc=int(meta[4]), n_caliber2=int(meta[5]), gamma=float(dmeta[0]),
                 cheb=bool(meta[6]), cheb_lambda=float(dmeta[1]), cheb_c1=dmeta[2:10].copy(),
                 cheb_c2=dmeta[10:18].copy())
        dtypes = dict(rp=np.int64, ci=np.int32, val=np.float64, diag=np.float64, colour=np.int32,
                      cidx=np.int32, agg=np.int32, agg2=np.int32, wt=np.float64, seed_of=np.int32,
                      X=np.float64, aff=np.float64, strong=np.uint8, pinv=np.float64)
        for name, dt in dtypes.items():
            cnt = L.oracle_level_array(self._h, l, name.encode(), None)
            if cnt:
                a = np.zeros(cnt, dt)
                L.oracle_level_array(self._h, l, name.encode(), _p(a))
                d[name] = a
            elif name in ("ci", "val"):
                d[name] = np.zeros(0, dt)
        if "X" in d:
            d["X"] = d["X"].reshape(d["n"], -1)
        if "pinv" in d:
            d["pinv"] = d["pinv"].reshape(d["n"], d["n"])
        d["A"] = Matrix(d["rp"], d["ci"], d["val"], d["diag"])
        return d

    @property
    def levels(self) -> list:
        if self._levels is None:
            self._levels = [self.level(l) for l in range(self.nlevels)]
        return self._levels

    def cycle(self, r) -> np.ndarray:
        r = _c(r, np.float64)
        z = np.zeros(self.n)
        lib().oracle_cycle(self._h, _p(r), _p(z))
        return z

    def fcg(self, b, tol: float = 1e-8, maxit: int = 100, record: bool = False):
        b = _c(b, np.float64)
        x = np.zeros(self.n)
        hist = np.zeros(maxit + 1)
        xs = np.zeros((maxit, self.n)) if record else None
        it = lib().oracle_fcg(self._h, _p(b), _p(x), tol, maxit, _p(hist), _p(xs))
        out = dict(x=x, iters=int(it), hist=hist[: it + 1])
        if record:
            out["iterates"] = xs[:it]
        return out

    def stationary(self, b, tol: float = 1e-8, maxit: int = 100, kappa: int = 0, record: bool = False):
        """Stationary cycles with recombination of the last kappa iterates; with record, also
        the iterate after each cycle's correction ("pre") and the recombined iterate that was
        saved, before the projection ("saved")."""
        b = _c(b, np.float64)
        x = np.zeros(self.n)
        hist = np.zeros(maxit + 1)
        xs = np.zeros((2 * maxit, self.n)) if record else None
        it = lib().oracle_stationary(self._h, _p(b), _p(x), tol, maxit, kappa, _p(hist), _p(xs))
        out = dict(x=x, iters=int(it), hist=hist[: it + 1])
        if record:
            out["pre"] = xs[0:2 * it:2]
            out["saved"] = xs[1:2 * it:2]
        return out

    def set_gamma(self, level: int, gamma: float):
        """Override the cycle index of one aggregation level."""
        lib().oracle_set_gamma(self._h, level, gamma)
        self._levels = None

    def visit_counts(self) -> list:
        """Visits of each level during the most recent cycle."""
        out = np.zeros(self.nlevels, np.int64)
        lib().oracle_visit_counts(self._h, _p(out))
        return out.tolist()

    def summary(self) -> list:
        return [(l["kind"], l["n"], l["nnz"] // 2, l["ncol"], l["n_caliber2"], l["gamma"])
                for l in self.levels]


def acf(hist) -> float:
    """Asymptotic convergence factor: geometric mean of the last five per-cycle residual
    reductions (Section 4.1)."""
    h = np.asarray(hist, dtype=np.float64)
    h = h[h > 0]
    k = min(5, len(h) - 1)
    if k < 1:
        return 0.0
    return float((h[-1] / h[-1 - k]) ** (1.0 / k))
