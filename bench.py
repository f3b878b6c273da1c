"""Benchmark of the LAMG+ solve phase on B300 (one JSON line on stdout).

Workload (N=1 line): the 1024 x 1024 grid-aligned anisotropic 5-point Laplacian (x-edges 1,
y-edges 1e-3; n = 1,048,576, nnz(L) = n + 2m = 5,238,784), one mean-zero Gaussian right-hand
side b = L x (seeds: graph 1, RHS 2, test vectors 3), FP64 cycle inside FP64 flexible CG, run to
||b - L phi|| / ||b|| <= 1e-8.

A step is one complete solve (projection of b, CG with one cycle per iteration, final true
residual) with b and phi resident in device memory; the hierarchy is set up once before the
timed region. The metric is ns per nonzero of L per digit of residual reduction,
t_solve / (nnz(L) * log10(||b|| / ||b - L phi||)); lower is better.

--impl reference times the CPU oracle (serial FP64 C) on the same workload and metric.
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
WORKLOAD = ("aniso1024: 2D 5-point grid 1024x1024, x-weight 1, y-weight 1e-3, one mean-zero "
            "N(0,1) RHS b = L x, FP64 cycle in FP64 flexible CG, tol 1e-8")
TOL = 1e-8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tail-rows", type=int, default=8192,
                    help="levels with at most this many rows run inside one CTA (persistent path)")
    ap.add_argument("--serve", action="store_true", help="run the serving workload instead")
    ap.add_argument("--profile-cycle", action="store_true",
                    help="per-step timing of one persistent-kernel cycle of the workload")
    ap.add_argument("--solve-once", action="store_true",
                    help="set up the workload and run one solve, nothing else (for a launch-list capture)")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-max-n", type=int, default=200000)
    ap.add_argument("--serve-threads", type=int, default=8)
    ap.add_argument("--profile-sweep", type=int, default=-1, metavar="LEVEL",
                    help="set up the workload, run one cold-L2 Gauss-Seidel sweep at LEVEL, exit "
                         "(a target for ncu)")
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
    barrier), grouped by (step kind, level), for the workload's hierarchy."""
    import collections
    import paper_2606_24791_b300 as lamg
    g, b = workload()
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


def solve_once():
    """Setup and exactly one solve of the workload (device buffers): the launch list of a
    profiler run over this process is the setup kernels followed by one solve."""
    import torch
    import paper_2606_24791_b300 as lamg
    g, b = workload()
    P = lamg.setup(g)
    bt = torch.from_numpy(b).cuda()
    xt = torch.zeros_like(bt)
    st = P.solve_ptr(bt.data_ptr(), xt.data_ptr(), TOL, 200)
    torch.cuda.synchronize()
    print(json.dumps({"iterations": st["iters"], "relres_true": st["relres_true"], "launches": st["launches"]}))


def profile_sweep(level: int):
    import paper_2606_24791_b300 as lamg
    g, b = workload()
    P = lamg.setup(g)
    # fill the level vectors with a real cycle iterate through the persistent kernel, so that
    # the only k_gs launches of this process are the profiled sweep
    P.cycle(b - b.mean(), persistent=True)
    r = P.time_kernel("gs_sweep", level, reps=1)
    print(json.dumps({"level": level, "info": P.info[level], "sweep": r}))


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
    import graphgen as gg
    g = gg.config_graph("aniso1024")
    b = gg.rhs(g, 2)
    return g, b


def digits(relres: float) -> float:
    return -math.log10(max(relres, 1e-300))


def cpu_baseline(g, b, reps: int = 3) -> dict:
    """The oracle as it stands (serial FP64 C, one thread) on the same workload."""
    import oracle
    t0 = time.perf_counter()
    H = oracle.Hierarchy(g)
    setup_s = time.perf_counter() - t0
    times, units = 0.0, 0.0
    for _ in range(reps):
        t0 = time.perf_counter()
        out = H.fcg(b, TOL, 200)
        dt = time.perf_counter() - t0
        x = out["x"]
        import graphgen as gg
        r = gg.laplacian_apply(g, x) - (b - b.mean())
        rel = np.linalg.norm(r) / np.linalg.norm(b - b.mean())
        times += dt
        units += g.nnz_L * digits(rel)
    return {"value": times * 1e9 / units, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{reps} full solves of the aniso1024 workload (FCG to 1e-8) after a "
                      f"{setup_s:.1f} s untimed oracle setup; single-threaded C, gcc -O2",
            "setup_s": setup_s}


# the source a kernel's counters depend on: its own definition and the device helpers it calls
KERNEL_SOURCES = {"k_gs": ["struct RowPre {", "RowPre row_pre(", "double row_finish(", "double block_row(",
                           "void __launch_bounds__(BS) k_gs("]}


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
    src = open(os.path.join(ROOT, "paper_2606_24791_b300", "csrc", "cycle_kernels.cu")).read()
    text = "\n".join(_definition(src, sig) for sig in KERNEL_SOURCES[kernel])
    return hashlib.sha256(text.encode()).hexdigest()


def traffic_for(kernel: str):
    """ncu DRAM bytes per launch recorded for `kernel`, if the kernel's source is unchanged."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path) or kernel not in KERNEL_SOURCES:
        return None
    rec = json.load(open(path))
    k = rec.get("kernels", {}).get(kernel)
    if not k or k.get("source_sha256") != kernel_source_sha(kernel):
        return None
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


def run_ours(args, ws, rank, local):
    import torch
    import paper_2606_24791_b300 as lamg
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    g, b = workload()
    t0 = time.perf_counter()
    P = lamg.setup(g, device=local, tail_rows=args.tail_rows)
    setup_s = time.perf_counter() - t0
    # one explicit stream for the L2 flush, the events and the solves, so that every timed
    # interval covers exactly the work between its two events
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    bt = torch.from_numpy(b).to(dev)
    xt = torch.zeros_like(bt)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def solve():
        return P.solve_ptr(bt.data_ptr(), xt.data_ptr(), TOL, 200, stream=stream.cuda_stream)

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
    units = float(sum(g.nnz_L * digits(s["relres_true"]) for s in stats))
    iters = [s["iters"] for s in stats]

    # kernels launched in the timed region (the persistent solve kernel: one per solve)
    launches = int(sum(s["launches"] for s in stats))
    kern_ms = [s["kernel_ms"] for s in stats]
    alg_bytes = [s["alg_bytes"] for s in stats]

    # e2e: the same solve through the C ABI with host buffers (H2D of b, D2H of phi inside the
    # timed interval), right after the device-timed steps, one untimed call first, the L2
    # flushed before each call (outside the interval) as for the device steps
    P.solve(b, TOL, 200)
    e2e_t, e2e_units = 0.0, 0.0
    for i in range(max(3, args.steps)):
        flush.fill_(i & 0xff)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, st = P.solve(b, TOL, 200)
        e2e_t += time.perf_counter() - t0
        e2e_units += g.nnz_L * digits(st["relres_true"])

    # the same solves as one persistent cooperative kernel, for comparison
    graph_ms = []
    for _ in range(3):
        flush.fill_(7)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        P.solve_ptr(bt.data_ptr(), xt.data_ptr(), TOL, 200, stream=stream.cuda_stream, persistent=True)
        e1.record(stream)
        torch.cuda.synchronize()
        graph_ms.append(e0.elapsed_time(e1))


    # roofline of the dominant kernel: cold-L2 timing of each candidate, weighted by how often
    # a solve runs it
    visits = schedule_counts(P, iters[0])
    cand = []
    it0 = iters[0]
    for l, L in enumerate(P.info):
        if L["kind"] != "agg" or L["n"] < 100_000:
            continue
        for k, per_cycle in (("gs_sweep", 3 * visits[l]), ("resid", visits[l])):
            r = P.time_kernel(k, l, reps=10)
            cand.append((r["ms"] * per_cycle * it0, f"{k}@L{l}", r))
    r = P.time_kernel("spmv_dot", 0, reps=10)
    cand.append((r["ms"] * it0, "spmv_dot@L0", r))
    cand.sort(key=lambda t: -t[0])
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("hbm_gbs", 6400.0)
    # dominant kernel: the candidate with the largest estimated share of a solve (cold-L2 time
    # alone x launches per solve); timed alone, so compared with the burst copy peak
    _, dom_name, dom = cand[0]
    kname = {"gs_sweep": "k_gs", "resid": "k_resid", "spmv_dot": "k_spmv_dot"}[dom_name.split("@")[0]]
    roofline = {"bound": "hbm", "kernel": f"{kname} ({dom_name}: " +
                ("one full colour-ordered sweep, all colour classes)" if kname == "k_gs" else "one launch)"),
                "achieved": round(dom["gbs"], 1), "peak": peak, "unit": "GB/s",
                "frac": round(dom["gbs"] / peak, 4), "traffic": traffic_for(kname),
                "algorithmic_bytes": dom["bytes"], "launch_ms": round(dom["ms"], 5),
                "launches_per_unit": dom["launches"],
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy), of measured" if peaks
                else "fallback 6400 GB/s"}
    # the whole solve: algorithmic bytes of every step / device time of the solve
    ach = float(np.mean([bb / (ms * 1e-3) / 1e9 for bb, ms in zip(alg_bytes, kern_ms)]))
    solve_roofline = {"achieved": round(ach, 1), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
                      "algorithmic_bytes": float(np.mean(alg_bytes)), "ms": float(np.mean(kern_ms))}
    kernels = {name + " (per-step kernel, cold L2, alone)": {"gbs": round(rr["gbs"], 1), "ms": round(rr["ms"], 4)}
               for _, name, rr in cand}
    kernels["persistent_path_ms_per_solve"] = round(float(np.median(graph_ms)), 3)
    kernels["graph_path_launches_per_solve"] = launches // max(args.steps, 1)
    kernels["schedule"] = P.schedule()
    # the same solve with every cycle step its own kernel (no cluster sub-cycle)
    Pq = lamg.setup(g, device=local, cluster_rows=-1)
    qms = []
    for _ in range(3):
        flush.fill_(9)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Pq.solve_ptr(bt.data_ptr(), xt.data_ptr(), TOL, 200, stream=stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        qms.append(e0.elapsed_time(e1))
    kernels["per_step_schedule_ms_per_solve"] = round(float(np.median(qms)), 3)
    Pq.close()

    # other forms of the same solve on the same workload (same metric, per right-hand side):
    # FP32 cycle inside FP64 CG, and 16 right-hand sides per SpMM-form solve (FP64 / FP32 cycle)
    variants = {}
    x64 = xt.cpu().numpy()
    P32 = lamg.setup(g, device=local, precision=lamg.FP32)
    for name, PP, k in (("fp32_cycle", P32, 1), ("batch16_fp64", P, 16), ("batch16_fp32_cycle", P32, 16)):
        import graphgen as gg
        # k independent mean-zero Gaussian right-hand sides b = L x (seed 2); k = 1 is the main b
        Bk = torch.from_numpy(gg.rhs(g, seed=2, k=k) if k > 1 else b).to(dev)
        Xk = torch.zeros_like(Bk)
        ms, unit_sum, its, rts = [], 0.0, [], []
        for rep in range(2 + 3):
            flush.fill_(rep & 0xff)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if k == 1:
                sts = [PP.solve_ptr(Bk.data_ptr(), Xk.data_ptr(), TOL, 200, stream=stream.cuda_stream)]
            else:
                sts = PP.solve_batch_ptr(k, Bk.data_ptr(), Xk.data_ptr(), TOL, 200, stream=stream.cuda_stream)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep >= 2:
                ms.append(e0.elapsed_time(e1))
                unit_sum += sum(g.nnz_L * digits(s["relres_true"]) for s in sts)
                its.append(max(s["iters"] for s in sts))
                rts.append(max(s["relres_true"] for s in sts))
        v = {"value": round(float(np.sum(ms)) * 1e6 / unit_sum, 5), "unit": UNIT + " (per right-hand side)",
             "rhs": k, "ms_per_solve": round(float(np.mean(ms)), 3), "iterations": its[-1],
             "relres_true_max": max(rts),
             "achieved_gbs": round(float(np.mean([s["alg_bytes"] for s in sts])) * k / (np.mean(ms) * 1e-3) / 1e9, 1)}
        if k == 1:
            v["rel_err_vs_fp64_solution"] = float(np.linalg.norm(Xk.cpu().numpy() - x64) / np.linalg.norm(x64))
        variants[name] = v
    P32.close()

    # the paper's own outer loop: stationary cycles with recombination of the last 4 iterates
    # (host buffers; its convergence factor beside FCG's iteration count)
    for _ in range(2):
        xs_st, st_st = P.stationary(b, TOL, 200, kappa=4, allow_unconverged=True)
    h = np.asarray(st_st["hist"])
    kk = min(5, len(h) - 1)
    variants["stationary_recombination_kappa4"] = {
        "value": round(st_st["solve_ms"] * 1e6 / (g.nnz_L * digits(st_st["relres_true"])), 5),
        "unit": UNIT + " (host buffers, copies included)", "cycles": st_st["iters"],
        "ms_per_solve": round(st_st["solve_ms"], 3), "relres_true": st_st["relres_true"],
        "acf_last5": round(float((h[-1] / h[-1 - kk]) ** (1.0 / kk)), 4) if kk > 0 else None}

    # many small systems in one launch (one thread-block cluster per system): 64 systems shaped
    # like the 64x64 unit grid (seeded weights U(0.5,1.5], so each system has its own
    # hierarchy), against the same systems solved one after another
    import graphgen as gg
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

    # whole-job value across ranks: max time over ranks / sum of units
    if ws > 1:
        total_ms, units_all = combine_ranks(total_ms, units, dev)
    else:
        units_all = units
    value = total_ms * 1e6 / units_all
    out = {
        "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": g.n, "nnz_L": g.nnz_L, "levels": P.nlevels,
                   "iterations": iters[0], "relres_true": stats[-1]["relres_true"],
                   "digits": round(digits(stats[-1]["relres_true"]), 3), "setup_s": round(setup_s, 2),
                   "parallelism": f"replicas{ws}", "l2": "flushed between steps (256 MB write)",
                   "seeds": {"graph": 1, "rhs": 2, "test_vectors": 3}},
        "e2e": {"value": round(e2e_t * 1e9 / e2e_units, 5), "unit": UNIT,
                "h2d_bytes_per_step": 8 * g.n, "d2h_bytes_per_step": 8 * g.n + 128},
        "gpu_launches": launches,
        "roofline": roofline,
        "solve_roofline": solve_roofline,
        "variants": variants,
        "kernels": kernels,
        "clocks": clocks,
        "wall_s_timed": round(wall, 3),
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(g, b)
    P.close()
    return out


def run_reference(args, ws, rank):
    """The oracle on the host cores, same workload and metric (rank 0 only)."""
    if rank != 0:
        return None
    import oracle
    import graphgen as gg
    g, b = workload()
    H = oracle.Hierarchy(g)
    for _ in range(max(args.warmup, 0)):
        H.fcg(b, TOL, 200)
    t_total, units = 0.0, 0.0
    t0w = time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        out = H.fcg(b, TOL, 200)
        t_total += time.perf_counter() - t0
        r = gg.laplacian_apply(g, out["x"]) - (b - b.mean())
        units += g.nnz_L * digits(np.linalg.norm(r) / np.linalg.norm(b - b.mean()))
    value = t_total * 1e9 / units
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t_total * 1e3 / args.steps, 2), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": g.n, "nnz_L": g.nnz_L},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "kind": "oracle", "cores": 1,
                         "sample": f"{args.steps} full oracle solves of the workload after an untimed setup"},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
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
        solve_once()
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
