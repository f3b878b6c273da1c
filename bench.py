"""Benchmark of the LAMG+ solve phase on B300 (one JSON line on stdout).

Workload (N=1 line): the Chung-Lu power-law graph of 4,000,000 nodes (expected degrees from a
Pareto density with exponent 2.1, mean degree 16, capped at sqrt(sum); largest connected
component: 3,902,576 nodes, nnz(L) = n + 2m = 67,055,822), weights U(0.5, 1.5], 32 mean-zero
Gaussian right-hand sides b = L x (seeds: graph 1, RHS 2, test vectors 3), solved together in
SpMM form: FP64 cycle inside FP64 flexible CG, every column to ||b - L phi|| / ||b|| <= 1e-8.

A step is one complete 32-column solve (projection of b, CG with one cycle per iteration, final
true residuals) with B and PHI resident in device memory; the hierarchy is set up once before the
timed region. The metric is ns per nonzero of L per digit of residual reduction per right-hand
side, t_solve / sum_j (nnz(L) * log10(||b_j|| / ||b_j - L phi_j||)); lower is better.

--impl reference times the CPU oracle (serial FP64 C) on a bounded sample of the same family
(a 250,000-node Chung-Lu graph of the same generator, one right-hand side per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "ns/nnz/digit to 1e-8 residual"
UNIT = "ns/nnz/digit"
K_RHS = 32
WORKLOAD = ("chunglu4m x 32 RHS: Chung-Lu power-law graph n=4,000,000 (Pareto exponent 2.1, mean "
            "degree 16, largest connected component), weights U(0.5,1.5], 32 mean-zero N(0,1) RHS "
            "b = L x solved together (SpMM-form cycles), FP64 cycle in FP64 flexible CG, tol 1e-8 per "
            "column; metric per right-hand side")
ANISO = ("aniso1024: 2D 5-point grid 1024x1024, x-weight 1, y-weight 1e-3, one mean-zero N(0,1) RHS "
         "b = L x, FP64 cycle in FP64 flexible CG, tol 1e-8")
SAMPLE_N = 250_000
TOL = 1e-8
FP64_PEAK_TFLOPS = 1.25   # nominal B300 FP64 rate: 148 SMs x 2.032 GHz x ~4.16 flop/clock/SM


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="the main line only (no other forms)")
    ap.add_argument("--tail-rows", type=int, default=8192,
                    help="levels with at most this many rows run inside one CTA (persistent path)")
    ap.add_argument("--serve", action="store_true", help="run the serving workload instead")
    ap.add_argument("--profile-cycle", action="store_true",
                    help="per-step timing of one persistent-kernel cycle of the aniso1024 workload")
    ap.add_argument("--solve-once", default=None,
                    choices=["main", "main-fp32", "aniso1024", "aniso1024-fp32", "grid192", "grid192-fp32"],
                    help="set up the named workload and run one solve, nothing else (for a launch-list capture)")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-max-n", type=int, default=200000)
    ap.add_argument("--serve-threads", type=int, default=8)
    ap.add_argument("--profile-sweep", type=int, default=-1, metavar="LEVEL",
                    help="set up aniso1024, run one cold-L2 Gauss-Seidel sweep at LEVEL, exit (a target for ncu)")
    ap.add_argument("--profile-kernels", default=None,
                    choices=["single", "single32", "single_powerlaw", "batch", "batch16", "setup"],
                    help="run each kernel of one family a few times after an L2 flush, nothing else (a target "
                         "for one-kernel ncu captures): single = the one-RHS cycle and CG kernels on aniso1024, "
                         "single32 = two FP32-cycle iterations on aniso1024, single_powerlaw = two one-RHS "
                         "iterations on a 500k-node Chung-Lu graph (Chebyshev levels), batch = the 32-column kernels on a 500k-node Chung-Lu graph, batch16 = the 16-column "
                         "Gauss-Seidel kernels on a 512^2 anisotropic grid, setup = the setup kernels on a "
                         "200k-node Barabasi-Albert graph")
    ap.add_argument("--profile-batch", default=None, metavar="N:LEVEL:WHICH",
                    help="set up a Chung-Lu graph of N nodes, run one cold-L2 32-column kernel sequence "
                         "(WHICH: sweep, resid, spmv_dot) at LEVEL, exit (a target for ncu)")
    return ap.parse_args()


def serve_bench(args):
    """Serving workload: Poisson arrivals of single-RHS requests whose graphs are drawn uniformly
    from three families (2D grids with sides log-uniform in [32, 512], random geometric graphs
    and Barabasi-Albert graphs with n log-uniform up to args.serve_max_n), weights U(0.5, 1.5],
    one mean-zero Gaussian RHS each, tol 1e-8, device memory budget 120 GB. The graphs come from
    a pre-generated pool of 24 family members (input generation is outside the timed region);
    every request is set up and solved independently. The arrival rate is 0.8 x the server's
    measured closed-loop throughput on the same pool."""
    import graphgen as gg
    import paper_2606_24791_b300 as lamg
    rng = np.random.default_rng(1)
    pool = []
    top = math.log10(args.serve_max_n)
    for i in range(24):
        fam = i % 3
        if fam == 0:
            side = int(round(10 ** rng.uniform(math.log10(32), math.log10(min(512, math.sqrt(args.serve_max_n))))))
            g = gg.grid2d_random(side, side, seed=100 + i)
        elif fam == 1:
            g = gg.rgg(int(10 ** rng.uniform(4, max(4.0, top))), 10, seed=100 + i)
        else:
            g = gg.barabasi_albert(int(10 ** rng.uniform(3, top)), 4, seed=100 + i)
        pool.append((g, gg.rhs(g, seed=200 + i)))
    S = lamg.Server(budget_bytes=120e9, max_inflight=64, setup_threads=args.serve_threads, tol=TOL, maxit=200)
    # closed-loop capacity on the pool
    t0 = time.perf_counter()
    tk = [S.submit(g, b) for g, b in pool]
    S.drain(3600)
    cap = len(pool) / (time.perf_counter() - t0)
    # open loop: Poisson arrivals at 0.8 x capacity
    lam = 0.8 * cap
    nreq = args.serve_requests
    picks = rng.integers(0, len(pool), nreq)
    gaps = rng.exponential(1.0 / lam, nreq)
    tickets = []
    t_start = time.perf_counter()
    t_next = t_start
    for i in range(nreq):
        t_next += gaps[i]
        dt = t_next - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        g, b = pool[picks[i]]
        tickets.append(S.submit(g, b))
    S.drain(3600)
    infos = [S.poll(t) for t in tickets]
    S.close()
    lat = np.array([i["t_done_ms"] - i["t_submit_ms"] for i in infos])
    setup = np.array([i["t_ready_ms"] - i["t_admit_ms"] for i in infos])
    wait = np.array([i["t_admit_ms"] - i["t_submit_ms"] for i in infos])
    solve = np.array([i["t_done_ms"] - i["t_ready_ms"] for i in infos])
    span = (max(i["t_done_ms"] for i in infos) - min(i["t_submit_ms"] for i in infos)) / 1e3
    ok = sum(1 for i in infos if i["status"] == 0 and i["relres_true"] <= 2e-8)
    sizes = [pool[p][0].n for p in picks]
    print(json.dumps({
        "metric": "served solves/s + p50/p99", "value": round(nreq / span, 3), "unit": "solves/s",
        "p50_ms": round(float(np.percentile(lat, 50)), 2), "p99_ms": round(float(np.percentile(lat, 99)), 2),
        "requests": nreq, "converged_1e-8": ok, "arrival_rate_per_s": round(lam, 3),
        "closed_loop_capacity_per_s": round(cap, 3),
        "latency_parts_p50_ms": {"admission_wait": round(float(np.median(wait)), 2),
                                 "setup": round(float(np.median(setup)), 2),
                                 "device_solve": round(float(np.median(solve)), 2)},
        "n_range": [int(min(sizes)), int(max(sizes))], "setup_threads": args.serve_threads,
        "config": {"workload": "serving: Poisson arrivals, grids/RGG/BA pool (24 graphs), "
                               f"n <= {args.serve_max_n}, weights U(0.5,1.5], tol 1e-8, budget 120 GB"},
    }), flush=True)


def profile_cycle():
    """Per-step device time of one cycle of the persistent kernel (%globaltimer at every grid
    barrier), grouped by (step kind, level), for the aniso1024 hierarchy."""
    import collections
    import paper_2606_24791_b300 as lamg
    g, b = aniso_workload()
    P = lamg.setup(g)
    ops = P.op_list()
    for _ in range(3):
        P.profile_cycle()
    prof = P.profile_cycle()
    groups = collections.defaultdict(lambda: [0, 0])
    prev = 0
    for nxt, ns in prof:
        kinds = sorted(set((ops[i][0], ops[i][1]) for i in range(prev, nxt) if ops[i][0] != "resid"))
        key = "single-CTA segment" if len(kinds) > 1 else (f"{kinds[0][0]}@L{kinds[0][1]}" if kinds else "?")
        groups[key][0] += 1
        groups[key][1] += ns
        prev = nxt
    x, st = P.solve(b, TOL, 200)
    x2, st2 = P.solve(b, TOL, 200, persistent=True)
    print(json.dumps({
        "levels": [(i["kind"], i["n"], i["ncol"]) for i in P.info],
        "cycle_us": sum(t for _, t in prof) / 1e3, "barrier_steps": len(prof),
        "steps": {k: {"count": c, "total_us": round(t / 1e3, 1), "avg_us": round(t / c / 1e3, 2)}
                  for k, (c, t) in sorted(groups.items(), key=lambda kv: -kv[1][1])},
        "graph_path_solve_ms": st["solve_ms"], "persistent_solve_ms": st2["solve_ms"],
        "iterations": st["iters"]}))


def solve_once(which: str):
    """Setup and exactly one solve of the named workload (device buffers): the launch list of a
    profiler run over this process is the setup kernels followed by one solve."""
    import torch
    import paper_2606_24791_b300 as lamg
    if which in ("aniso1024", "aniso1024-fp32"):
        g, b = aniso_workload()
        P = lamg.setup(g, precision=lamg.FP32 if which == "aniso1024-fp32" else lamg.FP64)
        bt = torch.from_numpy(b).cuda()
        xt = torch.zeros_like(bt)
        sts = [P.solve_ptr(bt.data_ptr(), xt.data_ptr(), TOL, 200)]
    elif which in ("grid192", "grid192-fp32"):
        # the 192^3 heterogeneous 3D grid with 16 right-hand sides
        import graphgen as gg
        g = gg.config_graph("grid3d192_hetero")
        B = gg.rhs(g, seed=2, k=16)
        P = lamg.setup(g, precision=lamg.FP32 if which == "grid192-fp32" else lamg.FP64)
        bt = torch.from_numpy(B).cuda()
        xt = torch.zeros_like(bt)
        sts = P.solve_batch_ptr(16, bt.data_ptr(), xt.data_ptr(), TOL, 200)
    else:
        g, B = workload()
        P = lamg.setup(g, precision=lamg.FP32 if which == "main-fp32" else lamg.FP64)
        bt = torch.from_numpy(B).cuda()
        xt = torch.zeros_like(bt)
        sts = P.solve_batch_ptr(K_RHS, bt.data_ptr(), xt.data_ptr(), TOL, 200)
    torch.cuda.synchronize()
    print(json.dumps({"iterations": max(s["iters"] for s in sts), "relres_true": max(s["relres_true"] for s in sts),
                      "launches": sts[0]["launches"]}))


def profile_sweep(level: int):
    import paper_2606_24791_b300 as lamg
    g, b = aniso_workload()
    P = lamg.setup(g)
    # fill the level vectors with a real cycle iterate through the persistent kernel, so that
    # the only k_gs launches of this process are the profiled sweep
    P.cycle(b - b.mean(), persistent=True)
    r = P.time_kernel("gs_sweep", level, reps=1)
    print(json.dumps({"level": level, "info": P.info[level], "sweep": r}))


def profile_batch(spec: str):
    """One cold-L2 32-column kernel sequence on a Chung-Lu graph of N nodes from the workload's
    generator: a small N for multi-pass captures (a few GB on the device), N = 4,000,000 (the
    workload itself) for one-pass counters."""
    import graphgen as gg
    import paper_2606_24791_b300 as lamg
    n, level, which = spec.split(":")
    g = gg.chung_lu(int(n), 2.1, 16.0, seed=1)
    P = lamg.setup(g)
    # the kernel sequence runs once, on the batch context's vectors as allocated (values do not
    # change the work or the traffic), so it is the only launch of its kind in the process
    r = P.time_kernel_batch(which, int(level), K_RHS, reps=1)
    print(json.dumps({"n": g.n, "nnz_L": g.nnz_L, "level": int(level), "info": P.info[int(level)], "which": which,
                      "kernel": r}))


def profile_kernels(family: str):
    """Each kernel of a family run a few times from a cold L2 (lamg_time_kernel*), plus one cycle or
    one iteration for the transfer kernels; prints what ran."""
    import torch
    import graphgen as gg
    import paper_2606_24791_b300 as lamg
    out = {"family": family}
    if family == "single":
        g, b = aniso_workload()
        P = lamg.setup(g)
        P.cycle(b - b.mean())
        for which, lvl in (("resid", 1), ("resid", 2), ("gs_sweep", 1), ("gs_sweep", 2), ("spmv_dot", 0),
                           ("restrict", 1), ("prolong", 1)):
            if which != "spmv_dot" and P.info[lvl]["kind"] != "agg":
                continue
            out[f"{which}@L{lvl}"] = P.time_kernel(which, lvl, reps=2)
        P.solve(b, TOL, 2, allow_unconverged=True)
        out["levels"] = [(i["kind"], i["n"], i["nnz"]) for i in P.info]
        out["forms"] = P.schedule()["forms"]
    elif family == "single32":
        # the FP32 cycle with one right-hand side (the multi-column kernels at one column) and
        # its FP64 outer CG: two iterations
        g, b = aniso_workload()
        P = lamg.setup(g, precision=lamg.FP32)
        P.solve(b, TOL, 2, allow_unconverged=True)
        out["levels"] = [(i["kind"], i["n"], i["nnz"]) for i in P.info]
    elif family == "single_powerlaw":
        g = gg.chung_lu(500_000, 2.1, 16.0, seed=1)
        b = gg.rhs(g, seed=2)
        P = lamg.setup(g)
        P.solve(b, TOL, 2, allow_unconverged=True)
        out["levels"] = [(i["kind"], i["n"], i["nnz"], i["ncol"]) for i in P.info]
    elif family in ("batch", "batch16"):
        if family == "batch":
            g = gg.chung_lu(500_000, 2.1, 16.0, seed=1)
            k = K_RHS
        else:
            g = gg.grid2d(512, 512, 1.0, 1e-3)
            k = 16
        B = gg.rhs(g, seed=2, k=k)
        P = lamg.setup(g)
        bt = torch.from_numpy(B).cuda()
        xt = torch.zeros_like(bt)
        P.solve_batch_ptr(k, bt.data_ptr(), xt.data_ptr(), TOL, 2)
        torch.cuda.synchronize()
        for l, L in enumerate(P.info):
            if L["kind"] == "agg" and L["n"] >= 50_000:
                out[f"sweep@L{l}"] = P.time_kernel_batch("sweep", l, k, reps=2)
                out[f"resid@L{l}"] = P.time_kernel_batch("resid", l, k, reps=2)
        out["spmv_dot@L0"] = P.time_kernel_batch("spmv_dot", 0, k, reps=2)
        out["levels"] = [(i["kind"], i["n"], i["nnz"], i["ncol"]) for i in P.info]
    else:
        g = gg.barabasi_albert(200_000, 4, seed=1)
        P = lamg.setup(g)
        out["levels"] = [(i["kind"], i["n"], i["nnz"], i["ncol"]) for i in P.info]
        out["setup_ms"] = P.setup_times()
    torch.cuda.synchronize()
    print(json.dumps(out, default=str))


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def workload():
    """The N=1 workload: the 4M-node Chung-Lu graph and its 32 right-hand sides (n x 32)."""
    import graphgen as gg
    g = gg.config_graph("chunglu4m")
    return g, gg.rhs(g, seed=2, k=K_RHS)


def aniso_workload():
    import graphgen as gg
    g = gg.config_graph("aniso1024")
    return g, gg.rhs(g, 2)


def digits(relres: float) -> float:
    return -math.log10(max(relres, 1e-300))


def oracle_sample(reps: int, warmup: int = 0) -> dict:
    """The oracle as it stands (serial FP64 C, one thread) on a bounded sample of the workload's
    family: a Chung-Lu graph of SAMPLE_N nodes from the same generator, one right-hand side,
    `reps` timed FCG solves to 1e-8 after an untimed setup (and `warmup` untimed solves)."""
    import graphgen as gg
    import oracle
    g = gg.chung_lu(SAMPLE_N, 2.1, 16.0, seed=1)
    b = gg.rhs(g, 2)
    t0 = time.perf_counter()
    H = oracle.Hierarchy(g)
    setup_s = time.perf_counter() - t0
    for _ in range(warmup):
        H.fcg(b, TOL, 200)
    times, units = 0.0, 0.0
    for _ in range(reps):
        t0 = time.perf_counter()
        out = H.fcg(b, TOL, 200)
        times += time.perf_counter() - t0
        r = gg.laplacian_apply(g, out["x"]) - (b - b.mean())
        units += g.nnz_L * digits(np.linalg.norm(r) / np.linalg.norm(b - b.mean()))
    return {"value": times * 1e9 / units, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"Chung-Lu n={SAMPLE_N} from the workload's generator (largest component {g.n} "
                      f"nodes, nnz(L) = {g.nnz_L}), one RHS, {reps} FCG solves to 1e-8 after a "
                      f"{setup_s:.1f} s untimed oracle setup; ns/nnz/digit is per nonzero and digit, so "
                      f"it compares with the 4M workload's per-RHS figure; single-threaded C, gcc -O2",
            "setup_s": round(setup_s, 2), "ms_per_solve": round(times * 1e3 / max(reps, 1), 2),
            "n": g.n, "nnz_L": g.nnz_L}


# the source a kernel's counters depend on: its file, its own definition and the device helpers
# it calls
KERNEL_SOURCES = {
    "k_gs": ("cycle_kernels.cu", ["struct RowPre {", "RowPre row_pre(", "double row_finish(", "double block_row(",
                                  "void __launch_bounds__(BS) k_gs("]),
    "bk_cheb": ("batch.cu", ["void add_entries(", "T rowsum_k(", "T block_row_k(",
                             "__global__ void __launch_bounds__(BBS) bk_cheb("]),
}


def _definition(src: str, signature: str) -> str:
    """Text of the definition that starts at `signature`, up to its matching closing brace."""
    i = src.index(signature)
    j = src.index("{", i)
    depth = 0
    for k in range(j, len(src)):
        if src[k] == "{":
            depth += 1
        elif src[k] == "}":
            depth -= 1
            if depth == 0:
                return src[i:k + 1]
    raise ValueError(signature)


def kernel_source_sha(kernel: str) -> str:
    fname, sigs = KERNEL_SOURCES[kernel]
    src = open(os.path.join(ROOT, "paper_2606_24791_b300", "csrc", fname)).read()
    text = "\n".join(_definition(src, sig) for sig in sigs)
    return hashlib.sha256(text.encode()).hexdigest()


def traffic_for(kernel: str, units: float = 1.0):
    """ncu DRAM bytes per roofline unit recorded for `kernel` (scaled by `units` when the record
    is per unit of a smaller capture), if the kernel's source is unchanged."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path) or kernel not in KERNEL_SOURCES:
        return None
    rec = json.load(open(path))
    k = rec.get("kernels", {}).get(kernel)
    if not k or k.get("source_sha256") != kernel_source_sha(kernel):
        return None
    if "dram_bytes_per_unit" in k:
        return k["dram_bytes_per_unit"] * units
    return k.get("dram_bytes")


def schedule_counts(P, iters: int) -> dict:
    """Per-solve launch counts of the cycle kernels (the cycle's static schedule)."""
    import math as m
    counts = {}
    lv = P.info
    visits = [0] * len(lv)

    def visit(l):
        visits[l] += 1
        L = lv[l]
        if L["kind"] == "coarsest":
            return
        if L["kind"] == "elim":
            visit(l + 1)
            return
        j = counts.setdefault(("j", l), 0)
        counts[("j", l)] = j + 1
        nv = m.floor((j + 1) * L["gamma"]) - m.floor(j * L["gamma"])
        for _ in range(nv):
            visit(l + 1)
    visit(0)
    return visits


def combine_ranks(total_ms: float, units: float, device="cpu"):
    """Whole-job figures of independent replicas: the slowest rank's time and the units of all
    ranks (timing metadata only; the solves exchange no data)."""
    import torch
    import torch.distributed as td
    tmax = torch.tensor([total_ms], dtype=torch.float64, device=device)
    tsum = torch.tensor([units], dtype=torch.float64, device=device)
    td.all_reduce(tmax, op=td.ReduceOp.MAX)
    td.all_reduce(tsum, op=td.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[0])


def timed_batch(P, Bt, Xt, k, stream, flush, reps, warm=1):
    """Device-timed k-column solves (cold L2): per-solve ms, stats of the last solve, and the sum of
    digits over the timed solves' columns."""
    import torch
    ms, units, sts = [], 0.0, None
    for rep in range(warm + reps):
        flush.fill_(rep & 0xff)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if k == 1:
            sts = [P.solve_ptr(Bt.data_ptr(), Xt.data_ptr(), TOL, 200, stream=stream.cuda_stream)]
        else:
            sts = P.solve_batch_ptr(k, Bt.data_ptr(), Xt.data_ptr(), TOL, 200, stream=stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if rep >= warm:
            ms.append(e0.elapsed_time(e1))
            units += sum(digits(s_["relres_true"]) for s_ in sts)
    return ms, sts, units


def run_ours(args, ws, rank, local):
    import torch
    import graphgen as gg
    import paper_2606_24791_b300 as lamg
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    g, B = workload()
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    P = lamg.setup(g, device=local, tail_rows=args.tail_rows)
    setup_s = time.perf_counter() - t0
    # one explicit stream for the L2 flush, the events and the solves, so that every timed
    # interval covers exactly the work between its two events
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    Bt = torch.from_numpy(B).to(dev)
    Xt = torch.zeros_like(Bt)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def solve():
        return P.solve_batch_ptr(K_RHS, Bt.data_ptr(), Xt.data_ptr(), TOL, 200, stream=stream.cuda_stream)

    for _ in range(max(args.warmup, 0)):
        flush.fill_(1)
        st = solve()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i & 0xff)                 # evict the 126 MB L2 between steps
        ev[i][0].record(stream)
        stats.append(solve())
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if ws > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(bb) for a, bb in ev]
    total_ms = float(sum(step_ms))
    units = float(sum(g.nnz_L * digits(c["relres_true"]) for sts in stats for c in sts))
    iters = [max(c["iters"] for c in sts) for sts in stats]
    worst = max(c["relres_true"] for sts in stats for c in sts)
    launches = int(sum(sts[0]["launches"] for sts in stats))
    kern_ms = [sts[0]["kernel_ms"] for sts in stats]
    alg_bytes = [sum(c["alg_bytes"] for c in sts) for sts in stats]
    X64 = Xt.cpu().numpy()

    # e2e: the same solves through the C ABI with host buffers (H2D of B, D2H of PHI inside the
    # timed interval), right after the device-timed steps, one untimed call first, the L2 flushed
    # before each call (outside the interval) as for the device steps
    Xout = np.empty_like(B)
    P.solve_batch(B, TOL, 200, out=Xout)        # untimed; also touches the caller's output array
    e2e_t, e2e_units = 0.0, 0.0
    for i in range(max(2, min(args.steps, 3))):
        flush.fill_(i & 0xff)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Xh, sth = P.solve_batch(B, TOL, 200, out=Xout)
        e2e_t += time.perf_counter() - t0
        e2e_units += sum(g.nnz_L * digits(c["relres_true"]) for c in sth)

    # one right-hand side of the same workload (the graph path, FP64): column 0, device buffers
    b0 = Bt[:, 0].contiguous()
    x0 = torch.zeros_like(b0)
    one = []
    for i in range(4):
        flush.fill_(i & 0xff)
        st1 = P.solve_ptr(b0.data_ptr(), x0.data_ptr(), TOL, 200, stream=stream.cuda_stream)
        one.append(st1)
    torch.cuda.synchronize()
    ms1 = float(np.median([c["solve_ms"] for c in one[1:]]))
    single_rhs = {"value": round(ms1 * 1e6 / (g.nnz_L * digits(one[-1]["relres_true"])), 5), "unit": UNIT,
                  "rhs": 1, "ms_per_solve": round(ms1, 3), "iterations": one[-1]["iters"],
                  "relres_true": one[-1]["relres_true"]}
    del b0, x0

    # roofline of the dominant kernel: cold-L2 time of each candidate sequence alone, weighted by
    # how often a solve runs it (the cycle's static step list times the iterations); per level
    # the same figures (the levels table)
    visits = schedule_counts(P, iters[0])
    o = lamg.options()
    nsweeps = o.nu_pre + o.nu_post
    cand, levels = [], []
    per_cycle = {}
    for kind, lv, _ in P.op_list():
        per_cycle[(kind, lv)] = per_cycle.get((kind, lv), 0) + 1
    cheb_levels = {lv for kind, lv in per_cycle if kind == "cheb"}
    for l, L in enumerate(P.info):
        if L["kind"] != "agg":
            continue
        sw = P.time_kernel_batch("sweep", l, K_RHS, reps=3)
        rs = P.time_kernel_batch("resid", l, K_RHS, reps=3)
        smoother = "chebyshev" if l in cheb_levels else "gauss-seidel"
        if l in cheb_levels:
            # one Chebyshev step (bk_cheb alone) as the unit: a cycle runs per_cycle of them here
            cs = P.time_kernel_batch("cheb_step", l, K_RHS, reps=3)
            cand.append((cs["ms"] * per_cycle[("cheb", l)] * iters[0], f"cheb_step@L{l}", cs, smoother))
        else:
            cand.append((sw["ms"] * nsweeps * visits[l] * iters[0], f"sweep@L{l}", sw, smoother))
        op_bytes = 12 * L["nnz"] + 20 * L["n"]
        vec_bytes = 3 * 8 * K_RHS * L["n"]
        levels.append({"level": l, "n": L["n"], "nnz": L["nnz"], "colours": L["ncol"], "smoother": smoother,
                       "visits_per_cycle": visits[l],
                       "sweep_ms": round(sw["ms"], 4), "sweep_tflops": round(sw["tflops"], 3),
                       "sweep_gbs": round(sw["gbs"], 1), "resid_ms": round(rs["ms"], 4),
                       "resid_tflops": round(rs["tflops"], 3), "resid_gbs": round(rs["gbs"], 1),
                       "l2_resident": op_bytes + vec_bytes <= 126e6})
        if l in cheb_levels:
            levels[-1].update({"cheb_steps_per_cycle": per_cycle[("cheb", l)],
                               "first_steps_per_cycle": per_cycle.get(("cheb_first", l), 0),
                               "copies_per_cycle": per_cycle.get(("cheb_copy", l), 0),
                               "cheb_step_ms": round(cs["ms"], 4), "cheb_step_tflops": round(cs["tflops"], 3),
                               "cheb_step_gbs": round(cs["gbs"], 1)})
        cand.append((rs["ms"] * visits[l] * iters[0], f"resid@L{l}", rs, "residual"))
    sp = P.time_kernel_batch("spmv_dot", 0, K_RHS, reps=3)
    cand.append((sp["ms"] * iters[0], "spmv_dot@L0", sp, "outer CG product"))
    cand.sort(key=lambda t: -t[0])
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    share_ms, dom_name, dom, dom_kind = cand[0]
    kname = {"chebyshev": "bk_cheb", "gauss-seidel": "bk_gs", "residual": "bk_resid",
             "outer CG product": "bk_spmv_dot"}[dom_kind]
    roofline = {"bound": "alu", "kernel": f"{kname}<double,32,1> ({dom_name}: {dom['launches']} launches, "
                f"32 columns, {dom_kind})", "achieved": round(dom["tflops"], 4), "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": round(dom["tflops"] / FP64_PEAK_TFLOPS, 4),
                "traffic": traffic_for(kname) if dom_name == "cheb_step@L2" else None,
                "algorithmic_flops": dom["flops"], "algorithmic_bytes": dom["bytes"],
                "launch_ms": round(dom["ms"], 5), "launches_per_unit": dom["launches"],
                "estimated_share_of_solve": round(share_ms / float(np.mean(step_ms)), 3),
                "peak_source": "nominal B300 FP64 rate (148 SMs x 2.032 GHz x ~4.16 flop/clock/SM); FP64 "
                               "multiply-adds bound the 32-column kernels",
                "hbm_view": {"achieved_gbs": round(dom["gbs"], 1), "peak_gbs": hbm_peak,
                             "frac": round(dom["gbs"] / hbm_peak, 4),
                             "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy), of measured"}}
    ach = float(np.mean([bb / (ms * 1e-3) / 1e9 for bb, ms in zip(alg_bytes, kern_ms)]))
    solve_roofline = {"achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s", "frac": round(ach / hbm_peak, 4),
                      "algorithmic_bytes": float(np.mean(alg_bytes)), "ms": float(np.mean(kern_ms))}
    kernels = {name: {"ms": round(rr["ms"], 4), "tflops": round(rr["tflops"], 3), "gbs": round(rr["gbs"], 1),
                      "est_ms_per_solve": round(sh, 2)} for sh, name, rr, _ in cand}
    kernels["launches_per_solve"] = launches // max(args.steps, 1)
    P.close()
    del Bt, Xt

    variants = {"chunglu4m_1rhs_fp64": single_rhs}
    if not args.no_variants:
        variants.update(run_variants(g, B, X64, dev, stream, flush, local))

    if ws > 1:
        total_ms, units_all = combine_ranks(total_ms, units, dev)
    else:
        units_all = units
    value = total_ms * 1e6 / units_all
    out = {
        "metric": METRIC, "value": round(value, 5), "unit": UNIT + " (per right-hand side)", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": g.n, "nnz_L": g.nnz_L, "rhs": K_RHS, "levels": len(P.info),
                   "iterations": iters[0], "relres_true_max": worst,
                   "digits_min": round(digits(worst), 3), "setup_s": round(setup_s, 2),
                   "generation_s": round(gen_s, 1), "parallelism": f"replicas{ws}",
                   "l2": "flushed between steps (256 MB write); the 32-column vectors alone exceed L2",
                   "seeds": {"graph": 1, "rhs": 2, "test_vectors": 3},
                   "hierarchy": [(i["kind"], i["n"], i["nnz"], i["ncol"]) for i in P.info]},
        "e2e": {"value": round(e2e_t * 1e9 / e2e_units, 5), "unit": UNIT + " (per right-hand side)",
                "h2d_bytes_per_step": 8 * g.n * K_RHS, "d2h_bytes_per_step": 8 * g.n * K_RHS + 128 * K_RHS},
        "gpu_launches": launches,
        "roofline": roofline,
        "levels": levels,
        "solve_roofline": solve_roofline,
        "variants": variants,
        "kernels": kernels,
        "clocks": clocks,
        "wall_s_timed": round(wall, 3),
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_sample(reps=3)
    return out


def run_variants(g, B, X64, dev, stream, flush, local) -> dict:
    """Other forms of the solve, same metric (per right-hand side): the workload with the FP32
    cycle inside FP64 CG (the precision the Chung-Lu configuration names), and the 1024^2
    anisotropic grid (single RHS FP64 and FP32 cycle, 16 RHS), many small systems in one launch,
    and the paper's own stationary loop."""
    import torch
    import graphgen as gg
    import paper_2606_24791_b300 as lamg
    variants = {}
    t0 = time.perf_counter()
    P32 = lamg.setup(g, device=local, precision=lamg.FP32)
    s32 = time.perf_counter() - t0
    Bt = torch.from_numpy(B).to(dev)
    Xt = torch.zeros_like(Bt)
    ms, sts, dsum = timed_batch(P32, Bt, Xt, K_RHS, stream, flush, reps=3)
    X32 = Xt.cpu().numpy()
    err = float(max(np.linalg.norm(X32[:, j] - X64[:, j]) / np.linalg.norm(X64[:, j]) for j in range(K_RHS)))
    units = g.nnz_L * dsum
    variants["chunglu4m_fp32_cycle"] = {
        "value": round(float(np.sum(ms)) * 1e6 / units, 5), "unit": UNIT + " (per right-hand side)",
        "rhs": K_RHS, "ms_per_solve": round(float(np.mean(ms)), 3), "iterations": max(c["iters"] for c in sts),
        "relres_true_max": max(c["relres_true"] for c in sts), "setup_s": round(s32, 2),
        "max_col_rel_err_vs_fp64_solution": err}
    k32 = P32.time_kernel_batch("sweep", 2, K_RHS, reps=3) if P32.info[2]["kind"] == "agg" else None
    if k32:
        variants["chunglu4m_fp32_cycle"]["sweep_L2"] = {"ms": round(k32["ms"], 4), "gbs": round(k32["gbs"], 1),
                                                       "tflops": round(k32["tflops"], 3)}
    P32.close()
    del Bt, Xt

    ga, ba = aniso_workload()
    Pa = lamg.setup(ga, device=local)
    Pa32 = lamg.setup(ga, device=local, precision=lamg.FP32)
    xa64 = None
    for name, PP, k in (("aniso1024_fp64", Pa, 1), ("aniso1024_fp32_cycle", Pa32, 1),
                        ("aniso1024_batch16_fp64", Pa, 16), ("aniso1024_batch16_fp32_cycle", Pa32, 16)):
        Bk = torch.from_numpy(gg.rhs(ga, seed=2, k=k) if k > 1 else ba).to(dev)
        Xk = torch.zeros_like(Bk)
        ms, sts, dsum = timed_batch(PP, Bk, Xk, k, stream, flush, reps=3, warm=2)
        units = ga.nnz_L * dsum
        v = {"value": round(float(np.sum(ms)) * 1e6 / units, 5), "unit": UNIT + " (per right-hand side)",
             "rhs": k, "ms_per_solve": round(float(np.mean(ms)), 3), "iterations": max(c["iters"] for c in sts),
             "relres_true_max": max(c["relres_true"] for c in sts)}
        if k == 1 and PP is Pa:
            xa64 = Xk.cpu().numpy()
            v["launches_per_solve"] = sts[0]["launches"]
            # the one-column path's dominant kernel on this workload: one level-2 colour-ordered sweep
            r = Pa.time_kernel("gs_sweep", 2, reps=10)
            v["k_gs_sweep_L2"] = {"ms": round(r["ms"], 5), "gbs": round(r["gbs"], 1), "bytes": r["bytes"],
                                  "traffic": traffic_for("k_gs")}
            # per-level table of the one-column cycle passes (cold L2, of the measured copy peak)
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
                os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
            hbm = peaks.get("hbm_gbs", 6400.0)
            sp = Pa.time_kernel("spmv_dot", 0, reps=5)
            rows = [{"level": 0, "kind": Pa.info[0]["kind"], "n": Pa.info[0]["n"], "nnz": Pa.info[0]["nnz"],
                     "spmv_dot_ms": round(sp["ms"], 5), "spmv_dot_gbs": round(sp["gbs"], 1),
                     "spmv_dot_frac": round(sp["gbs"] / hbm, 3)}]
            for l, L in enumerate(Pa.info):
                if L["kind"] != "agg":
                    continue
                sw = Pa.time_kernel("gs_sweep", l, reps=5)
                rs = Pa.time_kernel("resid", l, reps=5)
                rows.append({"level": l, "kind": "agg", "n": L["n"], "nnz": L["nnz"], "colours": L["ncol"],
                             "sweep_ms": round(sw["ms"], 5), "sweep_gbs": round(sw["gbs"], 1),
                             "sweep_frac": round(sw["gbs"] / hbm, 3), "sweep_launches": sw["launches"],
                             "resid_ms": round(rs["ms"], 5), "resid_gbs": round(rs["gbs"], 1),
                             "resid_frac": round(rs["gbs"] / hbm, 3),
                             "l2_resident": 12 * L["nnz"] + 48 * L["n"] <= 126e6})
            v["levels"] = rows
        if k == 1 and PP is Pa32 and xa64 is not None:
            v["rel_err_vs_fp64_solution"] = float(np.linalg.norm(Xk.cpu().numpy() - xa64) / np.linalg.norm(xa64))
        variants[name] = v
    for _ in range(2):
        xs_st, st_st = Pa.stationary(ba, TOL, 200, kappa=4, allow_unconverged=True)
    h = np.asarray(st_st["hist"])
    kk = min(5, len(h) - 1)
    variants["aniso1024_stationary_recombination_kappa4"] = {
        "value": round(st_st["solve_ms"] * 1e6 / (ga.nnz_L * digits(st_st["relres_true"])), 5),
        "unit": UNIT + " (host buffers, copies included)", "cycles": st_st["iters"],
        "ms_per_solve": round(st_st["solve_ms"], 3), "relres_true": st_st["relres_true"],
        "acf_last5": round(float((h[-1] / h[-1 - kk]) ** (1.0 / kk)), 4) if kk > 0 else None}
    Pa.close()
    Pa32.close()

    # many small systems in one launch (one thread-block cluster per system): 64 systems shaped
    # like the 64x64 unit grid (seeded weights U(0.5,1.5], so each system has its own
    # hierarchy), against the same systems solved one after another
    smalls = [gg.grid2d_random(64, 64, seed=100 + i) for i in range(64)]
    hs = [lamg.setup(gsm, device=local) for gsm in smalls]
    bsm = [gg.rhs(gsm, seed=2) for gsm in smalls]
    for _ in range(2):
        lamg.solve_many(hs, bsm, TOL, 200)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    xs_m, st_m = lamg.solve_many(hs, bsm, TOL, 200)
    wall_many = time.perf_counter() - t0
    t0 = time.perf_counter()
    st_1 = [hh.solve(bb, TOL, 200)[1] for hh, bb in zip(hs, bsm)]
    wall_one = time.perf_counter() - t0
    units_m = sum(gsm.nnz_L * digits(st_["relres_true"]) for gsm, st_ in zip(smalls, st_m))
    variants["many64_grid64"] = {
        "value": round(st_m[0]["kernel_ms"] * 1e6 / units_m, 5), "unit": UNIT + " (per system)",
        "systems": len(smalls), "launches": 1, "kernel_ms": round(st_m[0]["kernel_ms"], 3),
        "solves_per_s_device": round(len(smalls) / (st_m[0]["kernel_ms"] * 1e-3), 1),
        "wall_ms_one_launch": round(wall_many * 1e3, 3),
        "wall_ms_one_by_one": round(wall_one * 1e3, 3),
        "device_ms_one_by_one": round(float(sum(x["solve_ms"] for x in st_1)), 3),
        "iterations_max": max(x["iters"] for x in st_m),
        "relres_true_max": max(x["relres_true"] for x in st_m)}
    for hh in hs:
        hh.close()
    return variants


def run_reference(args, ws, rank):
    """The oracle on the host cores (rank 0 only): one solve of the bounded sample per step."""
    if rank != 0:
        return None
    t0w = time.perf_counter()
    cb = oracle_sample(reps=args.steps, warmup=max(args.warmup, 0))
    value = cb["value"]
    cb["value"] = round(value, 4)
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT + " (per right-hand side)",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": cb["ms_per_solve"], "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": cb["sample"]},
        "cpu_baseline": cb,
        "e2e": {"value": round(value, 4), "unit": UNIT + " (per right-hand side)", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "wall_s_timed": round(time.perf_counter() - t0w, 2),
    }


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.profile_sweep >= 0:
        profile_sweep(args.profile_sweep)
        return
    if args.profile_cycle:
        profile_cycle()
        return
    if args.solve_once:
        solve_once(args.solve_once)
        return
    if args.profile_batch:
        profile_batch(args.profile_batch)
        return
    if args.profile_kernels:
        profile_kernels(args.profile_kernels)
        return
    if args.serve:
        if rank == 0:
            serve_bench(args)
        return
    if args.impl == "reference":
        out = run_reference(args, ws, rank)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if ws > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(local)
        td.init_process_group("nccl")
    out = run_ours(args, ws, rank, local)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as td
        td.destroy_process_group()


if __name__ == "__main__":
    main()
