#!/usr/bin/env python3
"""Benchmark of the Barnes-Hut dipole-sum hot path: one step = build the octree
and node geometry, refit the node moments, forward (primal) queries and the
two-stage adjoint over one batch of ray-sample queries.

Workload (default): 1,000,000 points on a noisy torus + two spheres with 2%
outliers, 4 float32 attribute channels, 524,288 queries = 4,096 camera rays x
128 stratified samples, beta = 2, leaf size 8.  Synthetic, seeded.

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank runs its own query batch on its own GPU against the
same point cloud (weak scaling, no collective on the data path).
Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2405_16788_gb300 import synthetic as syn  # noqa: E402

METRIC = "dipole-sum queries/sec (fwd+adjoint) at N=1M pts; % of L2/HBM roofline; BF16 vs FP32"
UNIT = "queries/s"
BETA = 2.0
LEAF = 8


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="scene-1m")
    p.add_argument("--cpu-seconds", type=float, default=15.0,
                   help="budget of the oracle's CPU-baseline sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-bf16", action="store_true")
    p.add_argument("--no-next", action="store_true",
                   help="skip the timings of the gradient, grid and training-loop rows")
    p.add_argument("--loop-steps", type=int, default=10)
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_workload(name: str, rank: int):
    w = syn.workload(name)
    if rank > 0:  # weak scaling: every rank gets its own batch of rays
        o, d, tn, tf = syn.camera_rays(len(w.queries) // 128, seed=3003 + 101 * rank)
        w.queries, _ = syn.stratified_samples(o, d, tn, tf, 128, seed=4003 + 101 * rank)
    return w


def max_over_ranks(value: float, td=None, device=None) -> float:
    """The largest value over all ranks (the job is as slow as its slowest rank)."""
    if td is None or not td.is_available() or not td.is_initialized() or td.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_rank: int, steps: int, max_ms: float) -> float:
    """Units processed by all ranks divided by the slowest rank's timed span."""
    return world * units_per_rank * steps / (max_ms * 1e-3)


def config_of(w, flush: str):
    return {"workload": w.name, "points": w.cloud.n, "queries": int(len(w.queries)),
            "channels": int(w.mu.shape[1]), "attr_dtype": "f32", "beta": BETA,
            "leaf_size": LEAF, "tree": "built every step",
            "api": "dipole_build_tree, dipole_refit, dipole_forward_planned, dipole_adjoint_planned",
            "l2": flush, "step": "build + refit + forward + adjoint (stage 1 + 2)"}


# ------------------------------------------------------------------ oracle

def oracle_sample(w, seconds: float, keep: bool = False):
    """Time the oracle (as it stands) on a bounded sample of the workload and
    scale to one full step: tree build and update once, forward and adjoint
    per query, adjoint's per-call fixed cost (stage 2) measured separately."""
    import oracle
    c = w.cloud
    Q = len(w.queries)
    t0 = time.perf_counter()
    T = oracle.Tree(c.points, c.normals, c.areas, c.eps, leaf_size=LEAF)
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    T.update(w.mu)
    t_update = time.perf_counter() - t0
    rng = np.random.default_rng(12345)
    probe = w.queries[rng.choice(Q, 512, replace=False)]
    t0 = time.perf_counter()
    T.forward(probe, BETA)
    per_q_probe = (time.perf_counter() - t0) / len(probe)
    # size the sample to the budget (forward + adjoint ~ 5x forward)
    n_s = int(min(Q, max(1024, seconds / max(per_q_probe * 6.0, 1e-9))))
    idx = rng.choice(Q, n_s, replace=False)
    q = w.queries[idx]
    g = syn.upstream_grad(n_s, w.mu.shape[1], seed=77).astype(np.float64)
    t0 = time.perf_counter()
    fwd_ref = T.forward(q, BETA)
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    T.adjoint(q[:1], BETA, g[:1])
    t_adj_fixed = time.perf_counter() - t0
    t0 = time.perf_counter()
    adj_ref = T.adjoint(q, BETA, g)
    t_adj = time.perf_counter() - t0
    # the plain O(NQ) sum on a few queries, as interactions per second
    nb = 128
    t0 = time.perf_counter()
    oracle.brute_forward(c.points, c.normals, c.areas, c.eps, w.mu, q[:nb])
    brute_ips = nb * c.n / (time.perf_counter() - t0)
    per_q = t_fwd / n_s + max(t_adj - t_adj_fixed, 0.0) / n_s
    est = t_build + t_update + t_adj_fixed + Q * per_q
    return dict(value=Q / est, unit=UNIT, cores=oracle.num_threads(), kind="oracle",
                sample=(f"double-precision CPU Barnes-Hut (same tree rules, beta={BETA}): tree "
                        f"build + update over all {c.n} points, forward and two-stage adjoint "
                        f"over {n_s} of the {Q} queries, scaled to the full step"),
                seconds_per_step_est=est, build_s=t_build, update_s=t_update,
                fwd_us_per_query=1e6 * t_fwd / n_s,
                adj_us_per_query=1e6 * max(t_adj - t_adj_fixed, 0.0) / n_s,
                adj_fixed_s=t_adj_fixed, brute_force_interactions_per_s=brute_ips,
                brute_force_sample=f"{nb} queries x {c.n} points"), \
        (dict(idx=idx, g=g, fwd=fwd_ref, adj=adj_ref) if keep else None)


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = rank_workload(args.workload, 0)
    per = max(2.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(w, per)
    vals = [oracle_sample(w, per)[0] for _ in range(args.steps)]
    secs = [v["seconds_per_step_est"] for v in vals]
    value = len(w.queries) / statistics.mean(secs)
    cb = dict(vals[-1])
    cb["value"] = value
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(w, "n/a (CPU)"), "impl": "reference", "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.lines = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", gpu_id], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        return self.summarize(self.lines)

    @staticmethod
    def summarize(lines):
        """Median SM clock, maximum clock and the throttle reasons seen active,
        from `--format=csv,noheader,nounits` lines of FIELDS; None without a sample."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------ ours

def kernel_source_sha() -> str:
    h = hashlib.sha256()
    for f in ["traverse.cu", "query.cuh", "kernels.cuh", "common.cuh"]:
        with open(os.path.join(ROOT, "paper_2405_16788_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu capture, if it was taken on
    the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        e = d.get(kernel)
        if e and e.get("source_sha") == kernel_source_sha():
            return e
    except Exception:
        pass
    return None


def l2_probe(torch, dev, dp):
    """Best-of-10 L2 read bandwidth: one kernel reads a 48 MB buffer (inside the
    L2) 20 times with L2-only loads (dipole_probe_l2), timed with CUDA events."""
    buf = torch.empty(12 * 1024 * 1024, dtype=torch.float32, device=dev).uniform_()
    sink = torch.empty(1024 * torch.cuda.get_device_properties(dev).multi_processor_count,
                       dtype=torch.float32, device=dev)
    passes = 20
    for _ in range(3):
        dp.dipole_probe_l2(buf, passes, sink)
    best = 0.0
    for _ in range(10):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dp.dipole_probe_l2(buf, passes, sink)
        e1.record()
        e1.synchronize()
        best = max(best, passes * buf.numel() * 4 / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    return best


def run_ours(args):
    import torch
    import torch.distributed as td
    from paper_2405_16788_gb300 import dipole as dp

    world, rank, local = dist_env()
    if world > 1:
        td.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            td.barrier()

    w = rank_workload(args.workload, rank)
    c = w.cloud
    Q, C, N = len(w.queries), w.mu.shape[1], c.n
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    P, Nr, A, E = T(c.points), T(c.normals), T(c.areas), T(c.eps)
    MU, X = T(w.mu), T(w.queries)
    G = T(syn.upstream_grad(Q, C, seed=555 + rank))
    OUT = torch.empty((Q, C), device=dev)
    GRAD = torch.empty((N, C), device=dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)  # 512 MB > L2

    PLAN = dp.QueryPlan(Q, dev)

    def step(mu=MU):
        h = dp.dipole_build_tree(P, Nr, A, E, LEAF, 10)
        dp.dipole_refit(h, mu)
        dp.dipole_forward_planned(h, X, BETA, OUT, PLAN)
        dp.dipole_adjoint_planned(h, X, BETA, G, GRAD, PLAN, False)
        return h

    for _ in range(args.warmup):
        h = step()
        torch.cuda.synchronize()
        dp.dipole_tree_destroy(h)
    h = step()
    dp.dipole_sync_status(h)
    dp.dipole_tree_destroy(h)

    gpu_uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_uuid) if rank == 0 else None
    launches0 = dp.dipole_kernel_launches()
    total_ms = 0.0
    for _ in range(args.steps):
        flush.fill_(1)  # evict L2 between timed steps (not timed)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h = step()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        dp.dipole_tree_destroy(h)
    launches = (dp.dipole_kernel_launches() - launches0) // args.steps
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop() if sampler else None
    max_ms = max_over_ranks(total_ms, td, dev)
    value = job_throughput(world, Q, args.steps, max_ms)
    ms_per_step = max_ms / args.steps

    # ---- phase breakdown and roofline (untimed for `value`) ----
    def phase_times(reps=3, mu=MU):
        acc = np.zeros(4)
        for _ in range(reps):
            flush.fill_(1)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            ev[0].record(stream)
            hh = dp.dipole_build_tree(P, Nr, A, E, LEAF, 10)
            ev[1].record(stream)
            dp.dipole_refit(hh, mu)
            ev[2].record(stream)
            dp.dipole_forward_planned(hh, X, BETA, OUT, PLAN)
            ev[3].record(stream)
            dp.dipole_adjoint_planned(hh, X, BETA, G, GRAD, PLAN, False)
            ev[4].record(stream)
            ev[4].synchronize()
            acc += [ev[i].elapsed_time(ev[i + 1]) for i in range(4)]
            dp.dipole_tree_destroy(hh)
        return acc / reps

    ph = phase_times()
    h = step()
    cnt = torch.empty((Q, 3), dtype=torch.int32, device=dev)
    dp.dipole_query_counts(h, X, BETA, cnt)
    sums = cnt.to(torch.int64).sum(0).tolist()
    info = dp.dipole_tree_info_get(h)
    dp.dipole_tree_destroy(h)
    Tn, An, Ln = sums
    alg_bytes = 16 * Tn + (4 + 12 * C) * An + (16 + 12 + 4 * C) * Ln + (12 + 4 * C) * Q
    dom = "adjoint" if ph[3] >= ph[2] else "forward"
    t_dom = ph[3] if dom == "adjoint" else ph[2]
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm_peak else "fallback"
    hbm_peak = hbm_peak or 6800.0
    achieved = alg_bytes / (t_dom * 1e-3) / 1e9
    kern = f"k_query<{dp_cp(C)},float,{dom}>"
    tr = measured_traffic(kern)
    l2 = l2_probe(torch, dev, dp) if rank == 0 else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                "traffic": tr["dram_bytes_per_launch"] if tr else None,
                "kernel": kern + f" (the dipole_{dom} call, incl. its query sort)",
                "algorithmic_bytes_per_launch": alg_bytes,
                "bytes_formula": "16*tested + (4+12C)*far + (28+4C)*leaf_points + (12+4C)*queries",
                "per_query": {"tested": Tn / Q, "far": An / Q, "leaf_points": Ln / Q},
                "launch_ms": t_dom,
                "l2_probe_gbs": l2, "frac_of_l2_probe": (achieved / l2) if l2 else None,
                "working_set_mb": (N * (32 + 4 * C) + info["n_nodes"] * (32 + 4 * srow(C))) / 2 ** 20}
    breakdown = {"build_ms": ph[0], "refit_ms": ph[1], "forward_ms": ph[2], "adjoint_ms": ph[3],
                 "forward_queries_per_s": Q / (ph[2] * 1e-3),
                 "adjoint_queries_per_s": Q / (ph[3] * 1e-3),
                 "refit_forward_adjoint_queries_per_s": Q / ((ph[1] + ph[2] + ph[3]) * 1e-3),
                 "interactions_per_s": world * (An + Ln) * 2 / (ms_per_step * 1e-3),
                 "nodes": info["n_nodes"]}

    # ---- bf16 attribute storage, same workload ----
    bf16 = None
    if not args.no_bf16:
        MUb = MU.to(torch.bfloat16)
        for _ in range(2):
            hb = step(MUb)
            torch.cuda.synchronize()
            dp.dipole_tree_destroy(hb)
        phb = phase_times(mu=MUb)
        bf16 = {"forward_ms": phb[2], "adjoint_ms": phb[3], "refit_ms": phb[1],
                "step_ms": float(phb.sum()),
                "speedup_vs_f32_step": float(ph.sum() / phb.sum())}

    # ---- rows beyond the hot path: spatial gradient, normal/radius adjoint,
    # dense grid, training loop (timed with CUDA events, untimed for `value`) ----
    nxt = None
    if rank == 0 and not args.no_next:
        nxt = next_rows(torch, dp, dev, stream, flush, P, Nr, A, E, MU, X, G, Q, C, N, args,
                        (Tn, An, Ln), hbm_peak)

    # ---- end to end through the public API with host buffers ----
    e2e = None
    if not args.no_e2e:
        host = [a.cpu().pin_memory() for a in (P, Nr, A, E, MU, X, G)]
        dbuf = [torch.empty_like(a) for a in (P, Nr, A, E, MU, X, G)]
        out_h = torch.empty((Q, C)).pin_memory()
        grad_h = torch.empty((N, C)).pin_memory()
        h2d = sum(a.numel() * a.element_size() for a in host)
        d2h = out_h.numel() * 4 + grad_h.numel() * 4
        k_e2e = max(1, min(args.steps, 5))

        side = torch.cuda.Stream(device=dev)

        def e2e_step():
            # the cloud on the compute stream (the build needs it first); the
            # attributes, queries and upstream gradient on a side stream, under
            # the build; the forward's output read back under the adjoint
            for d_, h_ in zip(dbuf[:4], host[:4]):
                d_.copy_(h_, non_blocking=True)
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                for d_, h_ in zip(dbuf[4:], host[4:]):
                    d_.copy_(h_, non_blocking=True)
            hh = dp.dipole_build_tree(dbuf[0], dbuf[1], dbuf[2], dbuf[3], LEAF, 10)
            torch.cuda.current_stream().wait_stream(side)
            dp.dipole_refit(hh, dbuf[4])
            dp.dipole_forward_planned(hh, dbuf[5], BETA, OUT, PLAN)
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                out_h.copy_(OUT, non_blocking=True)
            dp.dipole_adjoint_planned(hh, dbuf[5], BETA, dbuf[6], GRAD, PLAN, False)
            grad_h.copy_(GRAD, non_blocking=True)
            torch.cuda.synchronize()
            return hh

        dp.dipole_tree_destroy(e2e_step())
        barrier()
        el = 0.0
        for _ in range(k_e2e):
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hh = e2e_step()
            el += time.perf_counter() - t0
            dp.dipole_tree_destroy(hh)
        el_max = max_over_ranks(el, td, dev)
        e2e = {"value": job_throughput(world, Q, k_e2e, el_max * 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "steps": k_e2e, "timing": "host wall clock, pinned host buffers, sync per step; "
                                          "attribute/query/gradient uploads overlap the build, "
                                          "the output read-back overlaps the adjoint"}

    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, ref = oracle_sample(w, args.cpu_seconds, keep=True)
        accuracy = sample_errors(torch, dp, dev, P, Nr, A, E, MU, X, Q, C, N, ref)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": config_of(w, "flushed between timed steps (512 MB write)"),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clocks, "breakdown": breakdown,
                "bf16_attrs": bf16, "next_rows": nxt, "accuracy": accuracy, "impl": "ours"}
        print(json.dumps(line), flush=True)
    if world > 1:
        td.destroy_process_group()
    return 0


def sample_errors(torch, dp, dev, P, Nr, A, E, MU, X, Q, C, N, ref):
    """Errors of the GPU path against the oracle's FP64 Barnes-Hut on the CPU
    baseline's query sample: forward on those queries, adjoint with the
    upstream gradient nonzero on them only (so the oracle's adjoint over the
    sample is the whole answer).  Per channel max|y - r| / max|r|."""
    def normwise(y, r):
        y, r = np.asarray(y, np.float64), np.asarray(r, np.float64)
        den = np.max(np.abs(r), axis=0)
        return (np.max(np.abs(y - r), axis=0) / np.where(den > 0, den, 1.0)).tolist()
    h = dp.dipole_build_tree(P, Nr, A, E, LEAF, 10)
    dp.dipole_refit(h, MU)
    out = torch.empty((Q, C), device=dev)
    dp.dipole_forward(h, X, BETA, out)
    gfull = torch.zeros((Q, C), device=dev)
    idx = torch.from_numpy(ref["idx"]).to(dev)
    gfull[idx] = torch.from_numpy(ref["g"].astype(np.float32)).to(dev)
    grad = torch.empty((N, C), device=dev)
    dp.dipole_adjoint(h, X, BETA, gfull, grad, False)
    dp.dipole_sync_status(h)
    fwd = out[idx].cpu().numpy()
    adj = grad.cpu().numpy()
    dp.dipole_tree_destroy(h)
    return {"forward_normwise": normwise(fwd, ref["fwd"]), "adjoint_normwise": normwise(adj, ref["adj"]),
            "queries": int(len(ref["idx"])),
            "against": "oracle FP64 Barnes-Hut, same tree rules; gates 1e-4 forward, 1e-3 adjoint"}


def next_rows(torch, dp, dev, stream, flush, P, Nr, A, E, MU, X, G, Q, C, N, args, counts,
              hbm_peak):
    """Timings of the rows built beyond the forward/adjoint step, each the
    median of 5 launches after one warm-up, L2 flushed before each."""
    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    h = dp.dipole_build_tree(P, Nr, A, E, LEAF, 10)
    dp.dipole_refit(h, MU)
    plan = dp.QueryPlan(Q, dev)
    OUT = torch.empty((Q, C), device=dev)
    GX = torch.empty((Q, C, 3), device=dev)
    GG = torch.from_numpy(np.random.default_rng(1).normal(size=(Q, C, 3)).astype(np.float32)).to(dev)
    GM = torch.empty((N, C), device=dev)
    GN = torch.empty((N, 3), device=dev)
    GE = torch.empty((N,), device=dev)
    f_ms = timed(lambda: dp.dipole_forward_grad(h, X, BETA, OUT, GX, plan))
    a_ms = timed(lambda: dp.dipole_adjoint_grad(h, X, BETA, G, GG, GM, False, plan))
    geo_ms = timed(lambda: dp.dipole_adjoint_geom(h, X, BETA, G, GG, GM, GN, GE, False, plan))
    # algorithmic bytes per launch, same walk as the forward (per-query counts):
    # forward_grad writes D and grad D (16C B per query); the normal/radius
    # adjoint reads g and G (16C), the moments of every far node (12C + 4) and
    # the attributes of every leaf point (4C) besides the point records (32)
    Tn, An, Ln = counts
    b_fg = 16 * Tn + (4 + 12 * C) * An + (28 + 4 * C) * Ln + (12 + 16 * C) * Q
    b_geo = 16 * Tn + (4 + 12 * C) * An + (32 + 4 * C) * Ln + (12 + 16 * C) * Q
    res = {"spatial_gradient": {
        "forward_grad_ms": f_ms, "adjoint_grad_ms": a_ms,
        "queries_per_s_fwd_adj": Q / ((f_ms + a_ms) * 1e-3),
        "adjoint_geom_ms": geo_ms,
        "forward_grad_logical_gbs": b_fg / (f_ms * 1e-3) / 1e9,
        "forward_grad_frac_of_hbm": b_fg / (f_ms * 1e-3) / 1e9 / hbm_peak,
        "adjoint_geom_logical_gbs": b_geo / (geo_ms * 1e-3) / 1e9,
        "adjoint_geom_frac_of_hbm": b_geo / (geo_ms * 1e-3) / 1e9 / hbm_peak,
        "bytes_formulas": {"forward_grad": "16*tested + (4+12C)*far + (28+4C)*leaf + (12+16C)*queries",
                           "adjoint_geom": "16*tested + (4+12C)*far + (32+4C)*leaf + (12+16C)*queries"},
        "workload": "the bench workload's tree and queries, C=4, plan from forward_grad"}}
    dims = (512, 512, 512)
    grid_out = torch.empty((dims[2], dims[1], dims[0], C), device=dev)
    g_ms = timed(lambda: dp.dipole_forward_grid(h, (-1.5, -1.5, -1.5), 3.0 / 511, dims, BETA,
                                                grid_out), reps=3)
    res["dense_grid"] = {"dims": list(dims), "forward_ms": g_ms,
                         "queries_per_s": dims[0] * dims[1] * dims[2] / (g_ms * 1e-3)}
    dp.dipole_sync_status(h)
    dp.dipole_tree_destroy(h)
    del grid_out
    if args.loop_steps > 0:
        res["training_loop"] = loop_row(torch, dev, args.loop_steps)
    return res


def loop_row(torch, dev, steps):
    """Adam on the attributes of the 5M-point loop scene through the renderer
    (camera + shadow rays, tree built once and refit per step)."""
    from paper_2405_16788_gb300 import render
    w = syn.workload("scene-5m-loop")
    o, d, t = w.meta["rays"]
    c = w.cloud
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev)
    rd = render.Renderer(T(c.points), T(c.normals), T(c.areas), T(c.eps), T(o), T(d), T(t),
                         T(w.meta["t_near"]), T(w.meta["light"]), n_shadow=64,
                         shadow_jitter=T(w.meta["shadow_jitter"]), queries=T(w.queries))
    with torch.no_grad():
        target, _, _ = rd.render(T(w.mu))
    mu0 = w.mu.copy()
    mu0[:, 0] = 1.0
    master = T(mu0).requires_grad_(True)
    opt = torch.optim.Adam([master], lr=1e-2)

    def one():
        opt.zero_grad(set_to_none=True)
        L, _ = rd.loss(master, target)
        L.backward()
        opt.step()
        return L

    for _ in range(3):
        one()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        L = one()
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    nq = rd.R * rd.S + rd.R * rd.K
    rd.tree.sync_status()
    return {"workload": "scene-5m-loop", "points": c.n, "queries_per_step": nq,
            "step_ms": ms, "queries_per_s": nq / (ms * 1e-3), "steps": steps,
            "loss_last": float(L.detach()),
            "step": "refit + forward/gradient on camera and shadow rays + their adjoints + "
                    "PyTorch rendering and Adam"}


def dp_cp(C: int) -> int:
    for k in (1, 2, 4, 8, 16, 32, 64):
        if C <= k:
            return k
    return 64


def srow(C: int) -> int:
    return (3 * dp_cp(C) + 3) & ~3


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
