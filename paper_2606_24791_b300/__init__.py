"""Python binding of the B300 LAMG+ solve-phase library (``include/lamg.h``).

Argument marshalling only: every step of setup kernels, cycle and CG runs inside
``_lib/liblamg_b300.so``. There is no CPU fallback: if the shared library cannot be loaded,
every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None

LAMG_OK = 0
ERRORS = {1: "INVALID", 2: "DISCONNECTED", 3: "SETUP", 4: "OOM", 5: "NOT_CONVERGED", 6: "CUDA",
          7: "TIMEOUT", 8: "ADMISSION", 9: "NO_DEVICE"}
DEVICE_PTRS = 1
PERSISTENT = 2
FP64, FP32 = 0, 1
KINDS = {"elim": 0, "agg": 1, "coarsest": 2}
KIND_NAMES = {v: k for k, v in KINDS.items()}


class LamgError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({_strerror(code)})")


class Options(C.Structure):
    _fields_ = [("K", C.c_int32), ("nu_tv", C.c_int32), ("dmax", C.c_int32), ("nu_pre", C.c_int32),
                ("nu_post", C.c_int32), ("coarsest_max", C.c_int32), ("max_levels", C.c_int32),
                ("veto", C.c_int32), ("caliber2", C.c_int32), ("precision", C.c_int32),
                ("seed", C.c_uint64), ("Q", C.c_double), ("tau_soc", C.c_double),
                ("elim_min_frac", C.c_double), ("snap", C.c_double), ("guard_eps", C.c_double),
                ("gamma_fixed", C.c_double), ("device", C.c_int32), ("tail_rows", C.c_int32),
                ("cluster_rows", C.c_int32), ("row_tpr", C.c_int32), ("sell", C.c_int32), ("autotune", C.c_int32), ("dense_rows", C.c_int32), ("cheb_colours", C.c_int32), ("cheb_degree", C.c_int32),
                ("tv_order", C.c_int32), ("agg_gpu_rows", C.c_int32), ("reserved", C.c_int32 * 1)]


class Graph(C.Structure):
    _fields_ = [("n", C.c_int64), ("rp", C.c_void_p), ("ci", C.c_void_p), ("w", C.c_void_p)]


class LevelDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32), ("n", C.c_int64), ("rp", C.c_void_p),
                ("ci", C.c_void_p), ("val", C.c_void_p), ("diag", C.c_void_p),
                ("colour", C.c_void_p), ("nc", C.c_int64), ("cidx", C.c_void_p),
                ("agg", C.c_void_p), ("agg2", C.c_void_p), ("wt", C.c_void_p),
                ("gamma", C.c_double)]


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int32), ("flags", C.c_uint32),
                ("stream", C.c_void_p), ("wait_us", C.c_int32), ("pad", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("nlevels", C.c_int32), ("relres", C.c_double),
                ("relres_true", C.c_double), ("b_mean", C.c_double), ("solve_ms", C.c_double),
                ("hist", C.c_void_p), ("kernel_ms", C.c_double), ("alg_bytes", C.c_double),
                ("launches", C.c_int64)]


class ServerOpts(C.Structure):
    _fields_ = [("budget_bytes", C.c_double), ("max_inflight", C.c_int32), ("setup_threads", C.c_int32),
                ("tol", C.c_double), ("maxit", C.c_int32), ("device", C.c_int32)]


class TicketInfo(C.Structure):
    _fields_ = [("done", C.c_int32), ("status", C.c_int32), ("iters", C.c_int32), ("pad", C.c_int32),
                ("relres", C.c_double), ("relres_true", C.c_double), ("t_submit_ms", C.c_double),
                ("t_admit_ms", C.c_double), ("t_ready_ms", C.c_double), ("t_done_ms", C.c_double)]


def lib_path() -> str:
    return _build.SO


def lib():
    """Load the shared library (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        L.lamg_options_default.argtypes = [C.POINTER(Options)]
        L.lamg_strerror.restype = C.c_char_p
        L.lamg_strerror.argtypes = [C.c_int]
        L.lamg_setup.argtypes = [C.POINTER(Graph), C.POINTER(Options), C.POINTER(P)]
        L.lamg_import.argtypes = [C.POINTER(LevelDesc), C.c_int32, C.POINTER(Options), C.POINTER(P)]
        L.lamg_solve.argtypes = [P, P, P, C.POINTER(SolveOpts), C.POINTER(Stats)]
        L.lamg_solve_batch.argtypes = [P, C.c_int32, P, P, C.POINTER(SolveOpts), P]
        L.lamg_cycle.argtypes = [P, P, P, C.c_uint32]
        L.lamg_hier_info.argtypes = [P, C.POINTER(C.c_int64), P, P]
        L.lamg_level_get.argtypes = [P, C.c_int32, C.c_char_p, P, C.POINTER(C.c_int64)]
        L.lamg_destroy.argtypes = [P]
        L.lamg_destroy.restype = None
        L.lamg_testvectors.argtypes = [C.c_int64, P, P, P, P, P, C.c_int32, C.c_uint64, C.c_int32,
                                       C.c_int32, P, C.c_int32]
        L.lamg_affinity.argtypes = [C.c_int64, P, P, P, P, C.c_int32, C.c_double, P, P]
        L.lamg_time_kernel.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, P]
        L.lamg_time_kernel_batch.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P]
        L.lamg_profile_cycle.argtypes = [P, P, C.c_int64, C.POINTER(C.c_int64)]
        L.lamg_testvectors_noalloc.argtypes = [C.c_int64, P, P, P, P, P, C.c_int32, C.c_int32, C.c_uint64,
                                               C.c_int32, C.c_int32, P, P, C.c_int32]
        L.lamg_server_create.argtypes = [C.POINTER(ServerOpts), C.POINTER(Options), C.POINTER(P)]
        L.lamg_serve.argtypes = [P, C.POINTER(Graph), P, C.POINTER(C.c_int64)]
        L.lamg_serve_poll.argtypes = [P, C.c_int64, C.POINTER(TicketInfo), P]
        L.lamg_server_drain.argtypes = [P, C.c_double]
        L.lamg_server_stats.argtypes = [P, P]
        L.lamg_server_destroy.argtypes = [P]
        L.lamg_server_destroy.restype = None
        L.lamg_op_list.argtypes = [P, P, C.c_int64, C.POINTER(C.c_int64)]
        L.lamg_schedule_info.argtypes = [P, P, C.c_int64, C.POINTER(C.c_int64)]
        L.lamg_solve_many.argtypes = [C.c_int32, P, P, P, C.POINTER(SolveOpts), P]
        L.lamg_setup_times.argtypes = [P, P, C.c_int32]
        L.lamg_solve_stationary.argtypes = [P, P, P, C.c_int32, C.POINTER(SolveOpts), P]
        L.lamg_profile_schedule.argtypes = [P, C.c_int32, P, C.c_int64, C.POINTER(C.c_int64)]
        _lib = L
    return _lib


def _strerror(code: int) -> str:
    try:
        return lib().lamg_strerror(code).decode()
    except Exception:  # noqa: BLE001 - only used inside error formatting
        return "?"


def _check(rc: int, where: str, allow=(LAMG_OK,)):
    if rc not in allow:
        raise LamgError(rc, where)
    return rc


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def options(**kw) -> Options:
    o = Options()
    lib().lamg_options_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Hierarchy:
    """A device-resident LAMG+ hierarchy (from ``setup`` or ``import_levels``)."""

    def __init__(self, handle, keep=None):
        self._h = handle
        self._keep = keep
        n = C.c_int64()
        _check(lib().lamg_hier_info(self._h, C.byref(n), None, None), "lamg_hier_info")
        self.nlevels = int(n.value)
        meta = np.zeros(7 * self.nlevels, np.int64)
        gam = np.zeros(self.nlevels)
        lib().lamg_hier_info(self._h, C.byref(n), _p(meta), _p(gam))
        meta = meta.reshape(-1, 7)
        self.info = [dict(kind=KIND_NAMES[int(m[0])], n=int(m[1]), nnz=int(m[2]), ncol=int(m[3]),
                          nc=int(m[4]), n_caliber2=int(m[5]), gamma=float(g))
                     for m, g in zip(meta, gam)]
        self.n = self.info[0]["n"]

    def close(self):
        if self._h:
            lib().lamg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def array(self, level: int, name: str):
        cnt = C.c_int64()
        _check(lib().lamg_level_get(self._h, level, name.encode(), None, C.byref(cnt)), "lamg_level_get")
        dt = {"rp": np.int64, "ci": np.int32, "val": np.float64, "diag": np.float64,
              "colour": np.int32, "cidx": np.int32, "agg": np.int32, "agg2": np.int32,
              "wt": np.float64, "X": np.float64, "aff": np.float64, "strong": np.uint8,
              "pinv": np.float64}[name]
        out = np.zeros(cnt.value, dt)
        if cnt.value:
            lib().lamg_level_get(self._h, level, name.encode(), _p(out), C.byref(cnt))
        return out

    def solve(self, b, tol: float = 1e-8, maxit: int = 100, allow_unconverged: bool = False,
              persistent: bool = False, wait_us: int = 0):
        """Host-pointer solve; returns (phi, stats dict with the residual history). wait_us: limit
        of each device-side wait (0: the library's 2 s; < 0: every wait gives up at once)."""
        b = _c(b, np.float64)
        if b.shape != (self.n,):
            raise ValueError("b has the wrong shape")
        phi = np.zeros(self.n)
        hist = np.zeros(maxit + 1)
        so = SolveOpts(tol, maxit, PERSISTENT if persistent else 0, None, wait_us)
        st = Stats()
        st.hist = hist.ctypes.data
        rc = lib().lamg_solve(self._h, _p(b), _p(phi), C.byref(so), C.byref(st))
        _check(rc, "lamg_solve", (LAMG_OK, 5) if allow_unconverged else (LAMG_OK,))
        return phi, _stats(st, hist)

    def stationary(self, b, tol: float = 1e-8, maxit: int = 100, kappa: int = 4,
                   allow_unconverged: bool = False):
        """lamg_solve_stationary: cycles with min-residual recombination of the last kappa
        iterates (the paper's solver loop); returns (phi, stats with the residual history)."""
        b = _c(b, np.float64)
        x = np.zeros(self.n)
        so = SolveOpts(tol, maxit, 0, None)
        st = Stats()
        h = np.zeros(maxit + 1)
        st.hist = h.ctypes.data
        rc = lib().lamg_solve_stationary(self._h, _p(b), _p(x), kappa, C.byref(so), C.byref(st))
        _check(rc, "lamg_solve_stationary", (LAMG_OK, 5) if allow_unconverged else (LAMG_OK,))
        return x, _stats(st, h)

    def solve_ptr(self, b_ptr: int, phi_ptr: int, tol: float = 1e-8, maxit: int = 100,
                  stream: int = 0, device: bool = True, hist: bool = False, persistent: bool = False):
        """Solve with raw pointers (device pointers when ``device``), e.g. torch ``data_ptr()``."""
        flags = (DEVICE_PTRS if device else 0) | (PERSISTENT if persistent else 0)
        so = SolveOpts(tol, maxit, flags, C.c_void_p(stream) if stream else None)
        st = Stats()
        h = np.zeros(maxit + 1) if hist else None
        if h is not None:
            st.hist = h.ctypes.data
        rc = lib().lamg_solve(self._h, C.c_void_p(b_ptr), C.c_void_p(phi_ptr), C.byref(so), C.byref(st))
        _check(rc, "lamg_solve", (LAMG_OK, 5))
        return _stats(st, h)

    def solve_batch(self, B, tol: float = 1e-8, maxit: int = 100, allow_unconverged: bool = False, out=None):
        """k right-hand sides (B: n x k) in one SpMM-form solve; returns (PHI, [stats per column]).
        out: an optional C-contiguous float64 n x k array that receives PHI (reused between calls,
        it saves the first-touch cost of a fresh output array)."""
        B = _c(B, np.float64)
        if B.ndim != 2 or B.shape[0] != self.n:
            raise ValueError("B must be n x k")
        k = B.shape[1]
        if out is not None:
            if out.shape != B.shape or out.dtype != np.float64 or not out.flags["C_CONTIGUOUS"]:
                raise ValueError("out must be a C-contiguous float64 array shaped like B")
            PHI = out
        else:
            PHI = np.zeros_like(B)
        hists = [np.zeros(maxit + 1) for _ in range(k)]
        st = (Stats * k)()
        for j in range(k):
            st[j].hist = hists[j].ctypes.data
        so = SolveOpts(tol, maxit, 0, None)
        rc = lib().lamg_solve_batch(self._h, k, _p(B), _p(PHI), C.byref(so), st)
        _check(rc, "lamg_solve_batch", (LAMG_OK, 5) if allow_unconverged else (LAMG_OK,))
        return PHI, [_stats(st[j], hists[j]) for j in range(k)]

    def solve_batch_ptr(self, k: int, B_ptr: int, PHI_ptr: int, tol: float = 1e-8, maxit: int = 100,
                        stream: int = 0, device: bool = True):
        """Batched solve on raw (device) pointers to n x k row-major blocks."""
        so = SolveOpts(tol, maxit, DEVICE_PTRS if device else 0, C.c_void_p(stream) if stream else None)
        st = (Stats * k)()
        rc = lib().lamg_solve_batch(self._h, k, C.c_void_p(B_ptr), C.c_void_p(PHI_ptr), C.byref(so), st)
        _check(rc, "lamg_solve_batch", (LAMG_OK, 5))
        return [_stats(st[j], None) for j in range(k)]

    KERNELS = {"resid": 0, "gs_sweep": 1, "spmv_dot": 2, "restrict": 3, "prolong": 4}

    def time_kernel(self, which: str, level: int, reps: int = 20) -> dict:
        """Cold-L2 device time of one kernel (``KERNELS``) and its algorithmic bytes."""
        out = np.zeros(3)
        _check(lib().lamg_time_kernel(self._h, self.KERNELS[which], level, reps, _p(out)),
               "lamg_time_kernel")
        return dict(ms=float(out[0]), bytes=float(out[1]), launches=int(out[2]),
                    gbs=float(out[1]) / (float(out[0]) * 1e-3) / 1e9)

    BATCH_KERNELS = {"resid": 0, "sweep": 1, "spmv_dot": 2, "cheb_step": 3}

    def time_kernel_batch(self, which: str, level: int, k: int, reps: int = 5) -> dict:
        """Cold-L2 device time of one k-column kernel sequence (``BATCH_KERNELS``), its
        algorithmic bytes and flops."""
        out = np.zeros(4)
        _check(lib().lamg_time_kernel_batch(self._h, self.BATCH_KERNELS[which], level, k, reps, _p(out)),
               "lamg_time_kernel_batch")
        ms = float(out[0])
        return dict(ms=ms, bytes=float(out[1]), launches=int(out[2]), flops=float(out[3]),
                    gbs=float(out[1]) / (ms * 1e-3) / 1e9, tflops=float(out[3]) / (ms * 1e-3) / 1e12)

    OP_KINDS = ["gs_first", "gs", "zero", "resid", "restrict", "prolong", "elim_restrict",
                "elim_interp", "coarse", "cheb", "cheb_copy", "cheb_first"]

    def op_list(self) -> list:
        cnt = C.c_int64()
        _check(lib().lamg_op_list(self._h, None, 0, C.byref(cnt)), "lamg_op_list")
        out = np.zeros(3 * cnt.value, np.int32)
        lib().lamg_op_list(self._h, _p(out), cnt.value, C.byref(cnt))
        return [(self.OP_KINDS[k], int(l), int(c)) for k, l, c in out.reshape(-1, 3)]

    SETUP_PHASES = ("input", "elimination", "colouring", "testvectors_affinity", "aggregation",
                    "galerkin", "dense_coarsest", "device_layout", "schedule")

    def setup_times(self) -> dict:
        """Wall milliseconds of each setup phase (lamg_setup hierarchies)."""
        out = np.zeros(len(self.SETUP_PHASES) + 1)
        _check(lib().lamg_setup_times(self._h, _p(out), out.size), "lamg_setup_times")
        d = {k: round(float(v), 3) for k, v in zip(self.SETUP_PHASES, out)}
        d["gpu_aggregation_rounds"] = int(out[-1])
        return d

    def schedule(self) -> dict:
        """Launch schedule of the graph path: first level of the cluster sub-cycle (-1: none),
        CTAs per cluster, kernels and steps per cycle, and the cycle times of the schedules
        the automatic choice compared."""
        out = np.zeros(5 + 2 * 128 + 2 * 16, np.int64)
        cnt = C.c_int64()
        _check(lib().lamg_schedule_info(self._h, _p(out), out.size, C.byref(cnt)), "lamg_schedule_info")
        nl = int(out[4])
        forms = [(int(out[5 + 2 * l]), int(out[6 + 2 * l])) for l in range(nl)]
        k0 = 5 + 2 * nl
        tuned = [(int(out[k]), out[k + 1] / 1e6) for k in range(k0, cnt.value, 2)]
        return {"cluster_from": int(out[0]), "cluster_ctas": int(out[1]), "launches_per_cycle": int(out[2]),
                "steps_per_cycle": int(out[3]), "forms": forms, "tuned_ms": tuned}

    def profile_schedule(self, from_level: int) -> list:
        """[(step, in_cluster, ns)] for one cycle with the steps on levels >= from_level run
        as cluster launches (from_level < 0: one kernel per step)."""
        cnt = C.c_int64()
        nops = len(self.op_list())
        out = np.zeros(3 * nops, np.int64)
        _check(lib().lamg_profile_schedule(self._h, from_level, _p(out), out.size, C.byref(cnt)),
               "lamg_profile_schedule")
        return [(int(a), bool(b), int(c)) for a, b, c in out.reshape(-1, 3)]

    def profile_cycle(self) -> list:
        """[(first step index after the barrier, ns)] for one cycle of the persistent kernel."""
        cap = len(self.op_list()) + 4
        out = np.zeros(2 * cap, np.int64)
        cnt = C.c_int64()
        _check(lib().lamg_profile_cycle(self._h, _p(out), cap, C.byref(cnt)), "lamg_profile_cycle")
        return [(int(a), int(b)) for a, b in out[: 2 * cnt.value].reshape(-1, 2)]

    def cycle(self, r, persistent: bool = False):
        r = _c(r, np.float64)
        z = np.zeros(self.n)
        _check(lib().lamg_cycle(self._h, _p(r), _p(z), PERSISTENT if persistent else 0), "lamg_cycle")
        return z


def _stats(st: Stats, hist) -> dict:
    d = dict(iters=st.iters, nlevels=st.nlevels, relres=st.relres, relres_true=st.relres_true,
             b_mean=st.b_mean, solve_ms=st.solve_ms, kernel_ms=st.kernel_ms,
             alg_bytes=st.alg_bytes, launches=st.launches)
    if hist is not None:
        d["hist"] = hist[: st.iters + 1].copy()
    return d


def solve_many(hs: list, bs: list, tol: float = 1e-8, maxit: int = 100, hist: bool = False,
               allow_unconverged: bool = False):
    """lamg_solve_many: G independent systems, one hierarchy each, in one kernel launch (one
    thread-block cluster per system). Returns ([phi_g], [stats_g])."""
    G = len(hs)
    if G != len(bs) or G == 0:
        raise ValueError("one right-hand side per hierarchy")
    barr = [_c(b, np.float64) for b in bs]
    for h, b in zip(hs, barr):
        if b.shape != (h.n,):
            raise ValueError("right-hand side size")
    xs = [np.zeros(h.n) for h in hs]
    hp = (C.c_void_p * G)(*[h._h for h in hs])
    bp = (C.c_void_p * G)(*[b.ctypes.data for b in barr])
    xp = (C.c_void_p * G)(*[x.ctypes.data for x in xs])
    so = SolveOpts(tol, maxit, 0, None)
    st = (Stats * G)()
    hbuf = [np.zeros(maxit + 1) for _ in range(G)] if hist else [None] * G
    for j in range(G):
        if hbuf[j] is not None:
            st[j].hist = hbuf[j].ctypes.data
    rc = lib().lamg_solve_many(G, hp, bp, xp, C.byref(so), st)
    _check(rc, "lamg_solve_many", (LAMG_OK, 5) if allow_unconverged else (LAMG_OK,))
    return xs, [_stats(st[j], hbuf[j]) for j in range(G)]


class Server:
    """Continuous-batching solve server (lamg_server_*): submit (graph, b) requests, poll tickets."""

    def __init__(self, budget_bytes: float, max_inflight: int = 64, setup_threads: int = 4,
                 tol: float = 1e-8, maxit: int = 200, device: int = 0, **opts):
        so = ServerOpts(float(budget_bytes), max_inflight, setup_threads, tol, maxit, device)
        o = options(**opts)
        h = C.c_void_p()
        _check(lib().lamg_server_create(C.byref(so), C.byref(o), C.byref(h)), "lamg_server_create")
        self._s = h

    def submit(self, g, b) -> int:
        rp, ci, w = _c(g.rp, np.int64), _c(g.ci, np.int32), _c(g.w, np.float64)
        b = _c(b, np.float64)
        G = Graph(g.n, rp.ctypes.data, ci.ctypes.data, w.ctypes.data)
        t = C.c_int64()
        _check(lib().lamg_serve(self._s, C.byref(G), _p(b), C.byref(t)), "lamg_serve")
        return int(t.value)

    def poll(self, ticket: int, n: int = 0) -> dict:
        info = TicketInfo()
        phi = np.zeros(n) if n else None
        _check(lib().lamg_serve_poll(self._s, ticket, C.byref(info), _p(phi)), "lamg_serve_poll")
        d = {f: getattr(info, f) for f, _ in TicketInfo._fields_ if f != "pad"}
        if phi is not None and info.done:
            d["phi"] = phi
        return d

    def drain(self, timeout_s: float = 600.0):
        _check(lib().lamg_server_drain(self._s, timeout_s), "lamg_server_drain")

    def stats(self) -> dict:
        out = np.zeros(8, np.int64)
        lib().lamg_server_stats(self._s, _p(out))
        return dict(bytes_in_flight=int(out[0]), inflight=int(out[1]), waiting=int(out[2]),
                    unfinished=int(out[3]), grouped_launches=int(out[4]), grouped_requests=int(out[5]),
                    largest_group=int(out[6]), overlapped_starts=int(out[7]))

    def close(self):
        if getattr(self, "_s", None):
            lib().lamg_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def setup(g, **opts) -> Hierarchy:
    """lamg_setup on a ``graphgen.Graph``-like object (n, rp, ci, w)."""
    rp, ci, w = _c(g.rp, np.int64), _c(g.ci, np.int32), _c(g.w, np.float64)
    G = Graph(g.n, rp.ctypes.data, ci.ctypes.data, w.ctypes.data)
    o = options(**opts)
    h = C.c_void_p()
    _check(lib().lamg_setup(C.byref(G), C.byref(o), C.byref(h)), "lamg_setup")
    return Hierarchy(h)


def import_levels(levels: list, **opts) -> Hierarchy:
    """lamg_import from level dicts with keys kind ('elim'|'agg'|'coarsest'), n, rp, ci, val,
    diag and, per kind, colour/nc/agg/agg2/wt/gamma or nc/cidx (natural numbering)."""
    keep = []
    descs = (LevelDesc * len(levels))()
    for d, L in zip(descs, levels):
        def arr(name, dt):
            if name not in L or L[name] is None:
                return None
            a = _c(L[name], dt)
            keep.append(a)
            return a.ctypes.data
        d.kind = KINDS[L["kind"]]
        d.n = int(L["n"])
        d.rp = arr("rp", np.int64); d.ci = arr("ci", np.int32)
        d.val = arr("val", np.float64); d.diag = arr("diag", np.float64)
        d.colour = arr("colour", np.int32)
        d.nc = int(L.get("nc", 0) or 0)
        d.cidx = arr("cidx", np.int32)
        d.agg = arr("agg", np.int32); d.agg2 = arr("agg2", np.int32); d.wt = arr("wt", np.float64)
        d.gamma = float(L.get("gamma", 0.0) or 0.0)
    o = options(**opts)
    h = C.c_void_p()
    _check(lib().lamg_import(descs, len(levels), C.byref(o), C.byref(h)), "lamg_import")
    return Hierarchy(h, keep)


TV_STRIDED, TV_STORED = 0, 1


def testvectors(rp, ci, val, diag, colour, level: int, seed: int, K: int = 4, nu: int = 3,
                order: int = TV_STRIDED):
    rp, ci = _c(rp, np.int64), _c(ci, np.int32)
    val, diag, colour = _c(val, np.float64), _c(diag, np.float64), _c(colour, np.int32)
    n = len(diag)
    X = np.zeros((n, K))
    _check(lib().lamg_testvectors(n, _p(rp), _p(ci), _p(val), _p(diag), _p(colour), level, seed, K,
                                  nu, _p(X), order), "lamg_testvectors")
    return X


def testvectors_noalloc(n: int, rp_ptr: int, ci_ptr: int, val_ptr: int, diag_ptr: int, colour_ptr: int,
                        ncol: int, level: int, seed: int, K: int, nu: int, X_ptr: int, stream: int = 0,
                        order: int = TV_STRIDED):
    """lamg_testvectors_noalloc on caller-owned device memory (raw device pointers); queued on
    `stream`, returns without waiting. For callers that cannot allocate device memory."""
    _check(lib().lamg_testvectors_noalloc(n, C.c_void_p(rp_ptr), C.c_void_p(ci_ptr), C.c_void_p(val_ptr),
                                          C.c_void_p(diag_ptr), C.c_void_p(colour_ptr), ncol, level, seed,
                                          K, nu, C.c_void_p(X_ptr), C.c_void_p(stream) if stream else None,
                                          order),
           "lamg_testvectors_noalloc")


def affinity(rp, ci, val, X, tau: float = 0.05):
    rp, ci, val = _c(rp, np.int64), _c(ci, np.int32), _c(val, np.float64)
    X = _c(X, np.float64)
    n, K = X.shape
    aff = np.zeros(len(ci)); strong = np.zeros(len(ci), np.uint8)
    _check(lib().lamg_affinity(n, _p(rp), _p(ci), _p(val), _p(X), K, tau, _p(aff), _p(strong)),
           "lamg_affinity")
    return aff, strong


EXPORTS = ["lamg_time_kernel_batch", "lamg_options_default", "lamg_setup", "lamg_import", "lamg_solve", "lamg_solve_batch",
           "lamg_cycle", "lamg_hier_info", "lamg_level_get", "lamg_destroy", "lamg_testvectors",
           "lamg_affinity", "lamg_strerror", "lamg_server_create", "lamg_serve", "lamg_serve_poll",
           "lamg_server_drain", "lamg_server_destroy", "lamg_time_kernel"]
