"""Benchmark: restarted-PDHG iterations per second on the GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload large|qp|tiny|batch|warmstart|sweep|mlp] [--no-ttt] [--lp-scale S]

Workload (default): the planted-optimum LP with m = 1e6 rows (4e5
equalities), n = 2e6 variables, nnz = 2e7 with Zipf(1.5) row lengths and
lognormal(0, 2) values, FP64 (seeded synthetic data; the paper's MIPLIB /
Mittelmann instances are not available).  One benchmark step is one check
period of the solver: P = 64 accepted PDHG iterations (Algorithm 2 trials
including any rejected ones) followed by the restart / termination check of
Sec. 3.4 / Sec. 4.1 -- every kernel of the hot path.  The matrix (K + K' =
480 MB) is far larger than the 129 MB L2, so every step streams it from HBM.

value  = accepted PDHG iterations per second, inputs resident in HBM;
e2e    = the same metric through the C ABI with (page-locked) host buffers:
         pdlp_create (host -> device copy, transpose, scaling) + pdlp_solve for the same
         number of iterations + device -> host copy of (x, y);
roofline = the dominant kernel's algorithmic HBM bytes per launch over its
         CUDA-event-timed average duration, against the measured copy
         bandwidth in MEASURED_PEAKS.json; `roofs` adds, per step kernel, the
         random-gather ceiling (one gather per nonzero), the same with the
         SpMV's index and value stream beside the gathers, and the FP64-pipe
         ceiling (FP64 instructions counted from the source), all measured
         on the GPU by pdlp_probe_rates / pdlp_probe_stream_gathers, and
         names the binding one;
time_to_tol = after the timed region, a solve from zero to each --ttt-tols
         tolerance (default 1e-4): seconds, iterations, objective error
         against the planted optimum (--trace-out FILE writes each of these
         solves' per-check records as JSON lines);
cpu_baseline = the FP64 CPU oracle (single thread) on a bounded sample of
         the same LP.

--workload qp runs the same measurement on a QP: the default LP with a
diagonal quadratic objective x'Qx/2 + c'x whose planted pair stays optimal;
--workload mlp times training steps of the warm-start network.

Multi-GPU: the plain path has an exchange per half-step (Kx', K'y'), so this
benchmark runs independent replicas, one per rank, and reports the sum.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PDHG iters/s"
UNIT = "iters/s"

# Per-launch DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum, bytes,
# mean of two launches) of the step kernels from one ncu capture of the
# 1e6 x 2e6 LP (FP64 values), keyed by (kernel, sha256 prefix of the kernel
# source it was taken on, value bits); reported as null once the source has
# changed.
NCU_TRAFFIC = {
    ("k_primal", "a9f0cfd18556e7b5", 64): 348776064.0,
    ("k_dual", "a9f0cfd18556e7b5", 64): 301759147.0,
}


def pinned_lp(lp):
    """A view of `lp` whose arrays live in page-locked host memory (returns the
    view and the torch tensors that own the memory)."""
    import types

    import numpy as np
    import torch

    owners, fields = [], {"m": lp.m, "n": lp.n, "n_eq": lp.n_eq}
    names = ["c", "row_ptr", "col_idx", "val", "q", "l", "u"]
    if getattr(lp, "qdiag", None) is not None:
        names.append("qdiag")
    for f in names:
        t = torch.from_numpy(np.ascontiguousarray(getattr(lp, f))).pin_memory()
        owners.append(t)
        fields[f] = t.numpy()
    return types.SimpleNamespace(**fields), owners


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    for f in ("pdlp_kernels.cu", "pdlp_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2311_12180_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """Samples nvidia-smi clocks / throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        import tempfile

        # the raw samples; BENCH_CLOCKS_CSV keeps them at a chosen path
        self.path = os.environ.get("BENCH_CLOCKS_CSV") or os.path.join(tempfile.gettempdir(),
                                                                         "pdlp_bench_clocks_%d.csv" % os.getpid())

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx = float(f[2])
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        except Exception:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate_replicas(ms: float, iters: float, pg=None, device: str = "cpu"):
    """Whole-job numbers of independent replicas: the slowest rank's time
    (max) and the iterations of all ranks (sum); pg is torch.distributed or
    None for one process."""
    import torch

    ms_t = torch.tensor([ms], dtype=torch.float64, device=device)
    it_t = torch.tensor([float(iters)], dtype=torch.float64, device=device)
    if pg is not None:
        pg.all_reduce(ms_t, op=pg.ReduceOp.MAX)
        pg.all_reduce(it_t, op=pg.ReduceOp.SUM)
    return float(ms_t.item()), float(it_t.item())


def batch_shard(work, rank: int, world: int):
    """This rank's members of a batch sharded over `world` ranks: members in
    decreasing expected work dealt out in a snake order (ranks 0 .. world - 1,
    then world - 1 .. 0, ...), so every rank gets a near-equal share;
    disjoint, covering, deterministic."""
    import numpy as np

    order = np.argsort(-np.asarray(work, dtype=np.float64), kind="stable")
    mine = []
    for k, i in enumerate(order):
        rnd, pos = divmod(k, world)
        if (pos if rnd % 2 == 0 else world - 1 - pos) == rank:
            mine.append(int(i))
    return sorted(mine)


def aggregate_batch(seconds: float, optimal: int, iters: int, count: int, pg=None, device: str = "cpu"):
    """Whole-job numbers of a sharded batch: the slowest rank's solve time
    and the summed optimal count, iterations and LP count."""
    import torch

    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    c = torch.tensor([float(optimal), float(iters), float(count)], dtype=torch.float64, device=device)
    if pg is not None:
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        pg.all_reduce(c, op=pg.ReduceOp.SUM)
    return float(t.item()), int(c[0].item()), int(c[1].item()), int(c[2].item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_workload(name: str, seed: int = 0, scale: float = 1.0, permute: int = -1):
    import lpgen

    if name == "large":
        m, n, nnz = int(round(1e6 * scale)), int(round(2e6 * scale)), int(round(2e7 * scale))
        lp = lpgen.large_lp(seed, m=m, n=n, nnz=nnz)
        desc = ("planted LP m=%d (40%% eq) n=%d nnz=%d, Zipf(1.5) row lengths (max %d), lognormal(0,2) values, "
                "bounds 50%% [0,inf) 30%% [l,u] 20%% free" % (m, n, lp.nnz, lp.meta["max_row"]))
        if permute >= 0:
            lp = lpgen.permuted(lp, permute)
            desc += ", rows and columns permuted (seed %d)" % permute
    elif name == "qp":
        # the same LP with a diagonal quadratic objective x'Qx/2 + c'x
        # (Q_jj ~ U(0, 2) on 60 % of the columns, c shifted so that the
        # planted pair stays optimal)
        m, n, nnz = int(round(1e6 * scale)), int(round(2e6 * scale)), int(round(2e7 * scale))
        lp = lpgen.planted_qp(lpgen.large_lp(seed, m=m, n=n, nnz=nnz), seed)
        desc = ("planted QP min x'Qx/2 + c'x, Q diagonal (60%% of Q_jj ~ U(0,2), the rest 0), over the planted LP "
                "m=%d (40%% eq) n=%d nnz=%d, Zipf(1.5) row lengths (max %d), lognormal(0,2) values"
                % (m, n, lp.nnz, lp.meta["max_row"]))
    elif name == "tiny":
        lp = lpgen.tiny_lp(seed)
        desc = "planted LP m=200 (100 eq) n=500 nnz=%d, 2%% density, N(0,1), 0<=x<=10" % lp.nnz
    else:
        raise SystemExit("unknown workload " + name)
    return lp, desc


def algorithmic_bytes(lp, kernel: str, value_bytes: int = 8) -> float:
    """HBM bytes one launch must move at minimum (int32 indices, FP64 values):
    k_primal: K' (row_ptr, col_idx, val) + gather of y (m) + read x, c, l, u,
              sx + write g, x', sx' (8 n-vectors);
    k_dual:   K + gather of x' (n) + read y, q, Kx, sy + write y', Kx', sy'
              (7 m-vectors).
    A QP's primal step also reads the diagonal of Q (one more n-vector)."""
    m, n, nnz = lp.m, lp.n, lp.nnz
    per_nz = 4.0 + value_bytes
    qp = 8.0 * n if getattr(lp, "qdiag", None) is not None else 0.0
    if kernel == "k_primal":
        return 4.0 * (n + 1) + per_nz * nnz + 8.0 * m + 8 * 8.0 * n + qp
    if kernel == "k_dual":
        return 4.0 * (m + 1) + per_nz * nnz + 8.0 * n + 7 * 8.0 * m
    if kernel == "k_primal_reuse_g":
        return 9 * 8.0 * n + qp
    raise KeyError(kernel)


def objective(lp, x) -> float:
    """c'x, plus x'Qx/2 for a QP (Q = diag(qdiag))."""
    import numpy as np

    qd = getattr(lp, "qdiag", None)
    obj = float(np.dot(lp.c, x))
    return obj + 0.5 * float(np.dot(qd * x, x)) if qd is not None else obj


def fp64_warp_instructions(layout: dict, kernel: str, qp: bool = False) -> float:
    """FP64 warp instructions one launch issues, counted from the kernels'
    source: one FMA per stored entry (a warp instruction covers 32 stored
    entries), one epilogue per slice (k_dual 8 FP64 operations per row:
    2 FMA + 1 subtraction for the extrapolated dual step, 1 FMA for the
    running sum, 1 subtraction + 2 FMA + 1 subtraction for the two partial
    sums; k_primal 5: 1 subtraction + 1 FMA for the step, 1 FMA for the
    running sum, 1 subtraction + 1 FMA for ||x' - x||^2), and per 32 long
    rows a 31-addition butterfly plus one epilogue.  A QP's primal step adds
    an FMA and a division per row, each counted as one instruction (so the
    count is a lower bound there)."""
    if kernel == "k_dual":
        stored, slices, longs, epi = layout["K_stored"], layout["K_slices"], layout["K_long_rows"], 8
    elif kernel == "k_primal":
        stored, slices, longs, epi = layout["KT_stored"], layout["KT_slices"], layout["KT_long_rows"], 7 if qp else 5
    else:
        raise KeyError(kernel)
    return stored / 32.0 + epi * slices + (31 + epi) * ((longs + 31) // 32)


def write_trace(path: str, trace, tol: float, recorded: int) -> None:
    """Appends the check records of one solve (the device ring's, copied
    once after the solve) to `path` as JSON lines."""
    import numpy as np

    with open(path, "a") as f:
        for r in trace:
            rec = {"tol": tol, "checks_recorded": recorded}
            for name in trace.dtype.names:
                v = r[name]
                rec[name] = int(v) if np.issubdtype(trace.dtype[name], np.integer) else float(v)
            f.write(json.dumps(rec) + "\n")


def cpu_baseline(lp, budget_s: float = 20.0):
    """The FP64 oracle as it stands (single thread), timed on a bounded sample:
    solves with max_iter = a and b; the difference isolates the iteration rate
    from the (shared) scaling set-up."""
    import oracle

    oracle.build()
    t = time.perf_counter()
    oracle.solve(lp, tol=1e-14, max_iter=2, trace_cap=1)
    t_small = time.perf_counter() - t
    # estimate per-iteration cost from a short run, then size the sample
    t = time.perf_counter()
    oracle.solve(lp, tol=1e-14, max_iter=6, trace_cap=1)
    t6 = time.perf_counter() - t
    per_it = max((t6 - t_small) / 4.0, 1e-6)
    b = int(max(6, min(2000, budget_s / per_it)))
    t = time.perf_counter()
    oracle.solve(lp, tol=1e-14, max_iter=b, trace_cap=1)
    tb = time.perf_counter() - t
    rate = (b - 2) / max(tb - t_small, 1e-9)
    return {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d accepted PDHG iterations of the same LP (rate from a %d-iteration minus a 2-iteration "
                      "solve, so the shared Sec. 2.2 scaling set-up cancels)" % (b - 2, b)}


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle on the host cores, same metric.
    Each step is one oracle solve of 1 + I iterations; the set-up of a solve
    (Sec. 2.2 scaling, the median of three 1-iteration solves) is subtracted,
    and I is sized so that the iterations take about 1.5 s per step."""
    if rank != 0:
        return
    import oracle

    oracle.build()
    lp, desc = make_workload(args.workload, seed=args.seed, scale=args.lp_scale, permute=args.permute_seed)

    def timed(k):
        t = time.perf_counter()
        r = oracle.solve(lp, tol=0.0, max_iter=k, trace_cap=1)
        return time.perf_counter() - t, r.iters

    t_setup = statistics.median(timed(1)[0] for _ in range(3))
    c = 2
    while True:  # calibrate the per-iteration cost on a sample well above the timer noise
        dt, k = timed(1 + c)
        per_it = (dt - t_setup) / max(k - 1, 1)
        if per_it * c > 0.05 or c >= 1 << 20:
            break
        c *= 8
    per_it = max(per_it, 1e-9)
    iters_per_step = int(max(2, min(1 << 22, 1.5 / per_it)))
    for _ in range(min(args.warmup, 1)):
        timed(1 + iters_per_step)
    el, total_iters = 0.0, 0
    for _ in range(args.steps):
        dt, k = timed(1 + iters_per_step)
        el += dt - t_setup
        total_iters += k - 1
    if el <= 0:
        el = per_it * total_iters
    val = total_iters / el
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * el / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d oracle iterations per step, one thread (the %.2f s set-up of a solve "
                                       "subtracted per step)" % (iters_per_step, t_setup)},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def mlp_step_flops(din: int, hidden: int, dout: int, batch: int) -> float:
    """FLOPs of one training step of the din-hidden-hidden-dout MLP: per
    weight, 2 (forward) + 4 (the two backward products) per batch row."""
    return 6.0 * batch * (din * hidden + hidden * hidden + hidden * dout)


def run_mlp(args, rank, world):
    """Training-step rate of the warm-start MLP (the tensor-core GEMMs, the
    fused loss, Adam): the 16-256-256-60500 network of the transportation
    workload at batch 256, He-uniform weights, 2048 random (theta, target)
    rows; 5 untimed Adam steps, then --mlp-steps timed ones (wall clock
    around the call, which waits for its per-step losses).  Rank 0 only."""
    if rank != 0:
        return
    import numpy as np

    from paper_2311_12180_gb300 import _build
    from paper_2311_12180_gb300 import pdlp as P
    from paper_2311_12180_gb300.warmstart import init_params

    _build.build()
    din, hid, dout, B = 16, 256, 60500, 256
    rng = np.random.default_rng(0)
    X = rng.standard_normal((2048, din)).astype(np.float32)
    T = rng.standard_normal((2048, dout)).astype(np.float32)
    steps = int(args.mlp_steps)
    with P.Mlp(din, hid, dout, max_batch=B) as net:
        net.set_params(init_params(din, hid, dout, 0))
        net.set_data(X, T)
        idx = rng.integers(0, 2048, (steps, B)).astype(np.int32)
        net.train(idx[:5])
        t = time.perf_counter()
        losses = net.train(idx)
        dt = time.perf_counter() - t
    flops = mlp_step_flops(din, hid, dout, B)
    line = {"metric": "MLP training steps/s", "value": steps / dt, "unit": "steps/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "bf16 (FP32 accumulate, FP32 masters)", "data": "synthetic",
            "config": {"workload": "MLP %d-%d-%d-%d, batch %d, 2048 random (theta, target) rows, Adam" %
                       (din, hid, hid, dout, B)},
            "ms_per_step": 1000.0 * dt / steps, "tflops": flops * steps / dt / 1e12,
            "flops_per_step": flops, "steps": steps, "loss_first_last": [float(losses[0]), float(losses[-1])]}
    print(json.dumps(line), flush=True)


def run_batch(args, rank, world):
    """Batched mode: many uneven planted LPs (m ~ logU[50,4000], n ~ logU[2m/3,
    2.5m], density ~ U[0.5%,5%], N(0,1) values, half equality rows, 0<=x<=10)
    solved to tol in one persistent launch; compared with the single-instance
    GPU solver run one LP after another on a sample of the same LPs.  With N
    ranks the LPs are sharded by expected work (batch_shard), each rank solves
    its share in its own launch with no collective on the data path, and the
    job's time is the slowest rank's (aggregate_batch)."""
    import numpy as np
    import torch

    import lpgen
    from paper_2311_12180_gb300 import _build
    from paper_2311_12180_gb300 import pdlp as P
    from paper_2311_12180_gb300.metrics import shifted_geometric_mean

    _build.build()
    pg = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(dist_env()[2])
        dist.init_process_group("nccl", device_id=torch.device("cuda", dist_env()[2]))
        pg = dist
    tol = args.batch_tol
    t = time.perf_counter()
    if world > 1:
        mine = batch_shard(lpgen.batch_work(args.batch_count, seed=0), rank, world)
        lps = lpgen.batch_subset(mine, args.batch_count, seed=0)
    else:
        lps = lpgen.batch_lps(args.batch_count, seed=0)
    gen_s = time.perf_counter() - t
    t = time.perf_counter()
    b = P.BatchSolver(lps)
    create_s = time.perf_counter() - t
    b.solve(tol=tol, max_iter=2)  # graph capture outside the timed solve
    if pg is not None:
        torch.cuda.synchronize()
        pg.barrier()
    t = time.perf_counter()
    xs, ys, st, it = b.solve(tol=tol, max_iter=args.batch_max_iter)
    solve_s = time.perf_counter() - t
    if pg is not None:
        job_s, job_opt, job_iters, job_count = aggregate_batch(solve_s, int(np.sum(st == P.OPTIMAL)), int(np.sum(it)),
                                                               len(lps), pg, device="cuda")
        if rank != 0:
            b.close()
            pg.destroy_process_group()
            return
        line = {"metric": "batch time-to-%g KKT (s)" % tol, "value": job_s, "unit": "s", "n_gpus": world,
                "higher_is_better": False, "scaling": "strong", "dtype": "f64", "data": "synthetic",
                "config": {"workload": "%d planted LPs sharded over %d ranks by expected work" % (job_count, world)},
                "optimal": job_opt, "count": job_count, "iters_total": job_iters,
                "agg_iters_per_s": job_iters / job_s, "rank0": {"lps": len(lps), "seconds": solve_s}}
        b.close()
        print(json.dumps(line), flush=True)
        pg.destroy_process_group()
        return
    stats = b.stats()
    t0s, t1s = b.times()
    b.close()
    nnzs = np.array([lp.nnz for lp in lps])
    team = nnzs >= stats["team_min_nnz"] if stats["team_lps"] else np.zeros(len(lps), bool)
    dur = t1s - t0s
    schedule = {
        "kernel_span_s": float(t1s.max()),
        "team_lps": int(team.sum()), "team_size": stats["team_size"],
        "team_phase_end_s": float(t1s[team].max()) if team.any() else None,
        "team_seconds": float(dur[team].sum()),
        "single_cta_seconds": float(dur[~team].sum()),
        "resident_lps": stats["resident"],
        "longest": [{"index": int(i), "m": lps[i].m, "n": lps[i].n, "nnz": lps[i].nnz, "iters": int(it[i]),
                     "team": bool(team[i]), "start_s": float(t0s[i]), "seconds": float(dur[i])}
                    for i in np.argsort(-dur)[:3]],
        "last_to_finish": [{"index": int(i), "nnz": lps[i].nnz, "iters": int(it[i]), "team": bool(team[i]),
                            "start_s": float(t0s[i]), "end_s": float(t1s[i])} for i in np.argsort(-t1s)[:3]],
    }
    ok = int(np.sum(st == P.OPTIMAL))
    rng = np.random.default_rng(1)
    sample = sorted(rng.choice(len(lps), size=min(args.batch_sample, len(lps)), replace=False).tolist())
    seq_s, seq_it, seq_times = 0.0, 0, []
    for i in sample:
        with P.Solver(lps[i]) as s1:
            t = time.perf_counter()
            _, _, s1st, s1it = s1.solve(tol=tol, max_iter=args.batch_max_iter)
            seq_times.append(time.perf_counter() - t)
            seq_s += seq_times[-1]
            seq_it += s1it
    seq_est = seq_s * len(lps) / len(sample)
    line = {"metric": "batch time-to-%g KKT (s)" % tol, "value": solve_s, "unit": "s", "n_gpus": 1,
            "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "%d planted LPs, m~logU[50,4000], n~logU[2m/3,2.5m], density~U[0.5%%,5%%], "
                                   "N(0,1), half equality rows, 0<=x<=10; sum nnz %d" % (len(lps), stats["sum_nnz"])},
            "optimal": ok, "count": len(lps), "iters_total": int(np.sum(it)), "iters_max": int(np.max(it)),
            "agg_iters_per_s": float(np.sum(it)) / solve_s, "create_s": create_s, "generate_s": gen_s,
            "autotune_entries_per_lane": stats["entries_per_lane"], "grid": stats["grid"],
            "slowest": [{"index": int(i), "m": lps[i].m, "n": lps[i].n, "nnz": lps[i].nnz, "iters": int(it[i]),
                         "status": int(st[i])} for i in np.argsort(-it)[:3]],
            "sequential_single_instance": {"sample": len(sample), "seconds_sample": seq_s,
                                           "estimated_seconds_all": seq_est, "iters_sample": seq_it,
                                           "sgm10_seconds": shifted_geometric_mean(seq_times)},
            "sgm10_seconds_per_lp_in_batch": shifted_geometric_mean(dur),
            "speedup_vs_sequential": seq_est / solve_s, "schedule": schedule}
    print(json.dumps(line), flush=True)


def run_sweep(args, rank, world):
    """Size sweep: planted LPs of the large recipe (Zipf(1.5) row lengths,
    lognormal(0,2) values, m = nnz/20, n = nnz/10) from 1e5 to 1e8 nonzeros;
    per size the device-timed PDHG iteration rate (as the large workload:
    warm-up periods, then timed check periods) and the FP64 oracle's rate on
    a bounded sample, and their ratio (the paper reports the GPU's advantage
    growing with the LP's size), with the step kernels' event-timed durations
    and their HBM roofline fraction per size."""
    if rank != 0:
        return
    import numpy as np
    import torch

    import lpgen
    from paper_2311_12180_gb300 import _build
    from paper_2311_12180_gb300 import pdlp as P

    _build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    rows = []
    for nnz in [int(float(v)) for v in args.sweep_nnz.split(",")]:
        lp = lpgen.large_lp(0, m=max(nnz // 20, 10), n=max(nnz // 10, 20), nnz=nnz)
        with P.Solver(lp, stream=stream.cuda_stream) as s:
            s.begin(tol=0.0, max_iter=10**12)
            s.run_periods(args.warmup)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            periods, ms = args.steps, 0.0
            while True:  # at least 0.2 s of timed work
                torch.cuda.synchronize()
                _, k0 = s.poll()
                ev0.record(stream)
                s.run_periods(periods)
                ev1.record(stream)
                ev1.synchronize()
                st1, k1 = s.poll()
                ms = ev0.elapsed_time(ev1)
                if st1 != -1:
                    raise SystemExit("sweep solve ended inside the timed region (status %d)" % st1)
                if ms >= 200.0 or periods >= 100000:
                    break
                periods = int(periods * max(2.0, 250.0 / max(ms, 1e-3)))
            gpu = (k1 - k0) / (ms / 1000.0)
            kt = s.time_kernels(2)
        peak, _ = measured_peaks()
        t_p = kt["k_primal"][0] / max(kt["k_primal"][1], 1) / 1000.0
        t_d = kt["k_dual"][0] / max(kt["k_dual"][1], 1) / 1000.0
        pair_bytes = algorithmic_bytes(lp, "k_primal") + algorithmic_bytes(lp, "k_dual")
        cpu = None if args.no_cpu else cpu_baseline(lp, budget_s=args.sweep_cpu_s)
        rows.append({"nnz": lp.nnz, "m": lp.m, "n": lp.n, "gpu_iters_per_s": gpu, "periods_timed": periods,
                     "k_primal_us": 1e6 * t_p, "k_dual_us": 1e6 * t_d,
                     "hbm_frac_step_kernels": pair_bytes / (t_p + t_d) / (peak * 1e9),
                     "cpu_iters_per_s": cpu["value"] if cpu else None,
                     "gpu_over_cpu": gpu / cpu["value"] if cpu else None,
                     "cpu_sample": cpu["sample"] if cpu else None})
        del lp
    line = {"metric": "PDHG iters/s by LP size", "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "planted LPs, Zipf(1.5) row lengths, lognormal(0,2) values, m = nnz/20, "
                                   "n = nnz/10, bounds 50% [0,inf) 30% [l,u] 20% free"},
            "cpu": "FP64 oracle, one host core, bounded sample per size", "sizes": rows}
    print(json.dumps(line), flush=True)


def run_warmstart(args, rank, world):
    """Learned warm start on the parametric transportation family: sources x
    sinks flows, costs / supplies / demands affine in a 16-dim latent theta
    plus N(0, noise) noise.  Training targets are the batched solver's own
    solutions; the BF16 MLP theta -> (x, y) is trained by the library's
    kernels; the held-out thetas are then solved to tol from the cold start,
    from the MLP's prediction (with cold fallback), and from two naive starts
    (mean training solution; solution of the nearest training theta) and two
    hybrids: a second MLP (theta, theta_nn - theta) -> T - T_nn that corrects
    the nearest training solution, and the neighbour's x with the MLP's y."""
    if rank != 0:
        return
    import numpy as np

    import lpgen
    from paper_2311_12180_gb300 import _build
    from paper_2311_12180_gb300 import warmstart as W

    _build.build()
    tol = args.ws_tol
    fam = lpgen.transport_family(0, sources=args.ws_sources, sinks=args.ws_sinks, dim=16, noise=args.ws_noise,
                                 cost_scale=args.ws_cost_scale)
    n, m = fam.n, fam.m
    th_tr = lpgen.transport_thetas(args.ws_train, 1)
    th_te = lpgen.transport_thetas(args.ws_test, 2)

    def mk_tr(i):
        return lpgen.transport_lp(fam, th_tr[i], i)

    def mk_te(i):
        return lpgen.transport_lp(fam, th_te[i], 10_000_000 + i)

    T = np.empty((args.ws_train, n + m), np.float32)

    def keep(i, x, y):
        T[i, :n] = x
        T[i, n:] = y

    t = time.perf_counter()
    st, it, data_solve_s, _ = W.solve_many(mk_tr, args.ws_train, args.ws_data_tol, on_solution=keep)
    data_s = time.perf_counter() - t
    steps = args.ws_steps
    sched = ((int(steps * 0.6), 1e-3), (int(steps * 0.3), 3e-4), (steps - int(steps * 0.6) - int(steps * 0.3), 1e-4))
    t = time.perf_counter()
    net, losses = W.train(th_tr, T, hidden=256, schedule=sched, batch=256, seed=0)
    train_s = time.perf_counter() - t
    # neighbour-residual model: (theta, theta_nn - theta) -> T - T_nn with the
    # leave-one-out neighbour inside the training set
    nn_tr = W.nearest_index(th_tr, th_tr, exclude_self=True)
    t = time.perf_counter()
    net_r, losses_r = W.train(W.residual_inputs(th_tr, th_tr[nn_tr]), T - T[nn_tr], hidden=256, schedule=sched,
                              batch=256, seed=1)
    train_r_s = time.perf_counter() - t
    flops_step = 6.0 * 256 * (16 * 256 + 256 * 256 + 256 * (n + m))
    near = W.nearest_index(th_tr, th_te)
    t = time.perf_counter()
    Yp = net.predict(th_te).astype(np.float64)
    predict_s = time.perf_counter() - t
    net.close()
    Yr = T[near].astype(np.float64) + net_r.predict(W.residual_inputs(th_te, th_tr[near])).astype(np.float64)
    net_r.close()

    Tc = np.empty((args.ws_test, n + m))

    def keep_c(i, x, y):
        Tc[i, :n] = x
        Tc[i, n:] = y

    arms = {}
    st_c, it_c, cold_s, _ = W.solve_many(mk_te, args.ws_test, tol, on_solution=keep_c)
    arms["cold"] = {"solve_s": cold_s, "optimal": int(np.sum(st_c == 0)), "iters_median": float(np.median(it_c)),
                    "iters_p90": float(np.percentile(it_c, 90)), "iters_mean": float(np.mean(it_c))}
    mx, my = W.mean_start(T, n)
    Ymix = np.concatenate([T[near][:, :n].astype(np.float64), Yp[:, n:]], axis=1)
    starts = {"mlp": lambda i: (Yp[i, :n], Yp[i, n:]), "mean": lambda i: (mx, my),
              "nearest": lambda i: (T[near[i], :n], T[near[i], n:]),
              "mlp_nn_residual": lambda i: (Yr[i, :n], Yr[i, n:]),
              "nearest_x_mlp_y": lambda i: (Ymix[i, :n], Ymix[i, n:])}
    preds = {"mlp": Yp, "mean": np.tile(np.concatenate([mx, my]), (args.ws_test, 1)), "nearest": T[near],
             "mlp_nn_residual": Yr, "nearest_x_mlp_y": Ymix}
    for name, fn in starts.items():
        r = W.solve_with_fallback(mk_te, args.ws_test, tol, fn)
        P_ = preds[name]
        ex = np.linalg.norm(P_[:, :n] - Tc[:, :n], axis=1) / np.maximum(np.linalg.norm(Tc[:, :n], axis=1), 1e-30)
        ey = np.linalg.norm(P_[:, n:] - Tc[:, n:], axis=1) / np.maximum(np.linalg.norm(Tc[:, n:], axis=1), 1e-30)
        arms[name] = {"solve_s": r["solve_s"], "optimal": int(np.sum(r["status"] == 0)), "fallbacks": r["fallbacks"],
                      "iters_median": float(np.median(r["iters"])), "iters_p90": float(np.percentile(r["iters"], 90)),
                      "iters_mean": float(np.mean(r["iters"])),
                      "iters_ratio_vs_cold_median": float(np.median(r["iters"] / np.maximum(it_c, 1))),
                      "rel_err_x_median": float(np.median(ex)), "rel_err_y_median": float(np.median(ey))}
    warm_total = arms["mlp"]["solve_s"] + predict_s
    line = {"metric": "warm-start time-to-%g KKT (s)" % tol, "value": warm_total, "unit": "s", "n_gpus": 1,
            "higher_is_better": False, "dtype": "f64 solve, bf16 MLP (f32 accumulate)", "data": "synthetic",
            "config": {"workload": "transportation family %dx%d (n=%d, m=%d), theta~N(0,I16), noise %g, cost directions "
                                   "x%g; %d training solutions (tol %g), %d held-out"
                                   % (fam.sources, fam.sinks, n, m, args.ws_noise, args.ws_cost_scale, args.ws_train,
                                      args.ws_data_tol, args.ws_test),
                       "mlp": "16-256-256-%d, batch 256, Adam %d steps (lr 1e-3 / 3e-4 / 1e-4)" % (n + m, steps)},
            "cold_s": cold_s, "speedup_vs_cold": cold_s / warm_total, "predict_s": predict_s,
            "data_generation_s": data_s, "data_solve_s": data_solve_s, "data_optimal": int(np.sum(st == 0)),
            "data_iters_median": float(np.median(it)), "train_s": train_s,
            "train_tflops": flops_step * steps / train_s / 1e12,
            "loss_first": float(losses[:10].mean()), "loss_last": float(losses[-50:].mean()),
            "residual_model": {"train_s": train_r_s, "loss_first": float(losses_r[:10].mean()),
                               "loss_last": float(losses_r[-50:].mean())},
            "arms": arms}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=["large", "qp", "tiny", "batch", "warmstart", "sweep", "mlp"])
    ap.add_argument("--mlp-steps", type=int, default=200, help="mlp workload: timed training steps")
    ap.add_argument("--sweep-nnz", default="1e5,1e6,1e7,5e7,1e8", help="comma-separated nonzero counts (sweep)")
    ap.add_argument("--sweep-cpu-s", type=float, default=5.0, help="oracle sample budget per size (sweep)")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--batch-tol", type=float, default=1e-6)
    ap.add_argument("--batch-max-iter", type=int, default=1_000_000)
    ap.add_argument("--batch-sample", type=int, default=32)
    ap.add_argument("--ws-sources", type=int, default=200)
    ap.add_argument("--ws-sinks", type=int, default=300)
    ap.add_argument("--ws-noise", type=float, default=0.1)
    ap.add_argument("--ws-cost-scale", type=float, default=1.0, help="0: costs fixed, only supplies/demands move")
    ap.add_argument("--ws-train", type=int, default=20000)
    ap.add_argument("--ws-test", type=int, default=1000)
    ap.add_argument("--ws-steps", type=int, default=4000)
    ap.add_argument("--ws-tol", type=float, default=1e-6)
    ap.add_argument("--ws-data-tol", type=float, default=1e-6)
    ap.add_argument("--no-ttt", action="store_true", help="skip the time-to-tolerance solves after the timed region")
    ap.add_argument("--ttt-limit", type=float, default=600.0, help="time limit per time-to-tolerance solve (s)")
    ap.add_argument("--ttt-tols", default="1e-4", help="comma-separated tolerances of the time-to-tolerance solves")
    ap.add_argument("--trace-out", default="", help="append each time-to-tolerance solve's per-check records "
                                                    "(k, trials, restarts, KKT, omega, step, Sec. 4.1 measures) "
                                                    "to this file as JSON lines")
    ap.add_argument("--seed", type=int, default=0, help="generator seed of the large / qp / tiny workload")
    ap.add_argument("--permute-seed", type=int, default=-1,
                    help="large workload: the same LP with rows (within their group) and columns permuted")
    ap.add_argument("--lp-scale", type=float, default=1.0,
                    help="large / qp workload: m, n and nnz scaled by this factor (1 = the 1e6 x 2e6 LP)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--value-bits", type=int, default=64, choices=[64, 32],
                    help="32: step kernels read an FP32 copy of K (FP64 gathers, accumulation, iterates)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local = dist_env()

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batch":
        run_batch(args, rank, world)
        return
    if args.workload == "warmstart":
        run_warmstart(args, rank, world)
        return
    if args.workload == "sweep":
        run_sweep(args, rank, world)
        return
    if args.workload == "mlp":
        run_mlp(args, rank, world)
        return

    import numpy as np
    import torch

    from paper_2311_12180_gb300 import _build
    from paper_2311_12180_gb300 import pdlp as P

    if not torch.cuda.is_available():
        raise SystemExit("bench needs a CUDA GPU")
    torch.cuda.set_device(local)
    _build.build()
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist

    lp, desc = make_workload(args.workload, seed=args.seed, scale=args.lp_scale, permute=args.permute_seed)
    stream = torch.cuda.Stream()
    solver = P.Solver(lp, stream=stream.cuda_stream, value_bits=args.value_bits)
    period = P.pdlp_default_params().check_period

    # ---- warm-up (cold start, then W periods) ----
    solver.begin(tol=1e-14, max_iter=10**12)
    solver.run_periods(args.warmup)
    st0, k0 = solver.poll()

    # ---- timed region ----
    def barrier():
        torch.cuda.synchronize()
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        solver.run_periods(args.steps)
        ev1.record(stream)
        ev1.synchronize()
    barrier()
    st1, k1 = solver.poll()
    ms = ev0.elapsed_time(ev1)
    iters = k1 - k0
    if st1 != -1:
        raise SystemExit("solve ended inside the timed region (status %d): timing invalid" % st1)
    ms_max, total_iters = aggregate_replicas(ms, iters, pg, "cuda")
    value = total_iters / (ms_max / 1000.0)

    # ---- per-kernel event timing (same workload, direct launches) ----
    times = solver.time_kernels(max(2, min(args.steps, 8)))
    peak, peak_kind = measured_peaks()
    cands = {k: v for k, v in times.items() if k in ("k_primal", "k_dual") and v[1] > 0}
    dom = max(cands, key=lambda k: cands[k][0])
    dom_ms = cands[dom][0] / cands[dom][1]
    vb = 8 if args.value_bits == 64 else 4
    dom_bytes = algorithmic_bytes(lp, dom, vb)
    achieved = dom_bytes / (dom_ms / 1000.0) / 1e9
    sha = kernel_source_sha()
    tr = NCU_TRAFFIC.get((dom, sha, args.value_bits)) if args.workload == "large" and args.lp_scale == 1.0 else None
    # the on-chip ceilings next to HBM: random gathers (one per nonzero) and
    # the FP64 pipe (FP64 instructions counted from the kernels' source)
    g_rate, f_rate = P.probe_rates()
    gs_rate = P.probe_stream_gathers()
    lay = solver.layout()
    roofs = {}
    for k in ("k_primal", "k_dual"):
        if k not in cands:
            continue
        t_k = cands[k][0] / cands[k][1] / 1000.0
        wi = fp64_warp_instructions(lay, k, qp=getattr(lp, "qdiag", None) is not None)
        roofs[k] = {
            "seconds": t_k,
            "hbm": {"floor_s": algorithmic_bytes(lp, k, vb) / (peak * 1e9),
                    "frac": algorithmic_bytes(lp, k, vb) / t_k / (peak * 1e9)},
            "gather": {"per_launch": lp.nnz, "peak_per_s": g_rate, "floor_s": lp.nnz / g_rate,
                       "frac": lp.nnz / t_k / g_rate},
            "gather_stream": {"per_launch": lp.nnz, "peak_per_s": gs_rate, "floor_s": lp.nnz / gs_rate,
                              "frac": lp.nnz / t_k / gs_rate},
            "fp64": {"warp_instructions": wi, "lane_ops": 32 * wi, "peak_lane_ops_per_s": f_rate,
                     "floor_s": 32 * wi / f_rate, "frac": 32 * wi / t_k / f_rate},
        }
        roofs[k]["binding"] = max(("hbm", "gather", "gather_stream", "fp64"), key=lambda r: roofs[k][r]["frac"])
    solver.finish()
    info = solver.info()

    # ---- end to end through the C ABI with host buffers (page-locked, as a
    # serving process keeps its request buffers) ----
    e2e_iters = int(max(1, round(iters / max(world, 1))))
    lp_host, _pinned = pinned_lp(lp)
    torch.cuda.synchronize()
    t = time.perf_counter()
    s2 = P.Solver(lp_host, value_bits=args.value_bits)
    x, y, st, it2 = s2.solve(tol=1e-14, max_iter=e2e_iters)
    e2e_s = time.perf_counter() - t
    e2e_setup_ms = s2.info()["setup_ms"]
    s2.close()
    # in: K (row starts, columns, values), c, l, u, q (K' is built on the device);
    # out: K''s row starts (read back at create for its sliced-ELL layout), x, y
    h2d = (4 * (lp.m + 1) + 12 * lp.nnz + 8 * 3 * lp.n + 8 * lp.m)
    d2h = 4 * (lp.n + 1) + 4 + 8 * (lp.n + lp.m)
    if getattr(lp, "qdiag", None) is not None:
        h2d += 8 * lp.n
    e2e_val = it2 / e2e_s * world

    ttt = None
    if not args.no_ttt:
        ttt = {}
        with P.Solver(lp, time_limit_s=args.ttt_limit, value_bits=args.value_bits) as s3:
            for tol in [float(v) for v in args.ttt_tols.split(",")]:
                t = time.perf_counter()
                _ = s3.solve(tol=tol, max_iter=10**9)
                stt, itt = _[2], _[3]
                x_t, y_t = _[0], _[1]
                obj = objective(lp, x_t)
                ttt["%g" % tol] = {"seconds": time.perf_counter() - t, "status": P.STATUS_NAMES.get(stt, stt),
                                   "iters": itt, "setup_excluded": True, "objective": obj,
                                   "obj_rel_err_vs_planted": abs(obj - lp.obj_star) / abs(lp.obj_star)}
                inf = s3.info()
                ttt["%g" % tol]["seconds_with_setup"] = ttt["%g" % tol]["seconds"] + inf["setup_ms"] / 1000.0
                ttt["%g" % tol].update({
                    "restarts": inf["restarts"], "f64_switch_iter": inf["f64_switch_iter"],
                    "rel_gap": abs(inf["pobj"] - inf["dobj"]) / (1 + abs(inf["pobj"]) + abs(inf["dobj"])),
                    "rel_primal_res": inf["rp_norm"] / (1 + inf["q_norm"]),
                    "rel_dual_res": inf["rd_norm"] / (1 + inf["c_norm"])})
                if args.trace_out and rank == 0:
                    write_trace(args.trace_out, s3.trace(), tol, s3.checks_recorded())

    if rank != 0:
        if pg is not None:
            pg.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu and world == 1:
        cpu = cpu_baseline(lp)

    kernels_per_period = 2 * (period + max(4, period // 8)) + 4  # + check_primal, infeas, check_dual, restart
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if args.value_bits == 64 else "f64 (K values stored f32)",
        "data": "synthetic",
        "config": {"workload": desc, "value_bits": args.value_bits, "step": "one check period: %d accepted PDHG iterations + restart/termination "
                   "check" % period, "l2": "inputs larger than L2 (K + K' = %.0f MB)" % (24 * lp.nnz / 1e6),
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "iters_timed": int(total_iters),
        "attempts_per_iter": info["attempts"] / max(info["iters"], 1),
        "effective_hbm_gbs": (algorithmic_bytes(lp, "k_primal", vb) + algorithmic_bytes(lp, "k_dual", vb)) * value / 1e9,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind, "traffic": tr, "traffic_unit": "bytes per launch (ncu)",
                     "algorithmic_bytes_per_launch": dom_bytes, "avg_launch_ms": dom_ms,
                     "kernel_ms": {k: (v[0] / v[1] if v[1] else None) for k, v in times.items()},
                     "roofs": roofs, "binding": roofs[dom]["binding"],
                     "binding_frac": roofs[dom][roofs[dom]["binding"]]["frac"],
                     "roofs_note": "gather and FP64 peaks measured on this GPU by pdlp_probe_rates (random "
                                   "8-byte gathers of a 16 MB vector; FP64 FMA lane operations); gather_stream "
                                   "by pdlp_probe_stream_gathers (the same gathers with a 4-byte index and an "
                                   "8-byte value streamed per entry, one FMA each: an SpMV's bytes per nonzero)"},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "iters": it2, "seconds": e2e_s, "create_ms": e2e_setup_ms, "note": "one step = create + solve(%d iterations) + outputs" % it2},
        "gpu_launches": kernels_per_period * args.steps,
        "clocks": clk.summary(),
    }
    if ttt is not None:
        line["time_to_tol"] = ttt
    print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
