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
    p.add_argument("--loop-steps", type=int, default=200,
                   help="Adam steps of the 5M-point training-loop row")
    p.add_argument("--no-configs", action="store_true",
                   help="skip the rows of the other workloads (sphere-2k, scene-200k, scene-3m-bf16)")
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
            "l2": flush, "step": "build + refit + forward + adjoint (stage 1 + 2)",
            "cpu_baseline": "the oracle (FP64 CPU Barnes-Hut) timed on a sample of the queries "
                            "and extrapolated to the full step (sampled and extrapolated)"}


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
    for f in ["traverse.cu", "traverse_grad.cu", "query.cuh", "kernels.cuh", "common.cuh", "tree.cuh"]:
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


def l2_size_bytes(torch, dev) -> int:
    """The GPU's L2 size (cudaDevAttrL2CacheSize, as torch reports it)."""
    return int(getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 0) or 0)


def roofline_block(torch, dev, dp, C, Q, N, NN, sums, usums, kernel_ms, clocks, rank):
    """The roofline of the dominant traversal kernel (the slower of the
    forward and the adjoint stage 1, each timed by CUDA events around its
    launches in the timed region).

    The bound follows the workload: L2 when the working set (node records and
    moments, point records and attributes) fits in the L2, else HBM; the
    L2 peak is measured here (dipole_probe_l2, best of 10), the HBM peak is
    MEASURED_PEAKS.json's copy bandwidth.  Three figures side by side:
      per_lane  the algorithmic bytes of every query's own walk (tested node
                16 B, far node 4 + 12C B, leaf point 28 + 4C B, query 12 + 4C B),
                what a query must touch; the lanes of a warp share most of it
                as broadcasts, so this can exceed the memory peaks;
      per_warp  what the warps must fetch: a 32-byte node record per warp
                step, a 12C-byte moment row when some lane takes the node as
                far, 32 + 4C bytes per point of a leaf some lane opens, and the
                queries' own 12 + 4C bytes (dipole_query_packet_counts);
      issue     warp instructions per launch (ncu smsp__inst_executed.sum
                from profiles/traffic.json, taken on the current kernel
                source) over (SMs x 4 schedulers x SM clock x kernel time),
                the SM clock being the median sampled in the timed region.
    `frac` is the per-lane figure against the bound's peak; `binding` names
    the largest of the per-warp and issue fractions."""
    Tn, An, Ln = sums
    Us, Uf, Up, _ = usums
    per_lane = 16 * Tn + (4 + 12 * C) * An + (28 + 4 * C) * Ln + (12 + 4 * C) * Q
    per_warp = 32 * Us + 12 * C * Uf + (32 + 4 * C) * Up + (12 + 4 * C) * Q
    dom = "adjoint" if kernel_ms["adjoint"] >= kernel_ms["forward"] else "forward"
    t_k = kernel_ms[dom]
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs")
    hbm_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if hbm else "fallback (profiling recipe, 6.8 TB/s)"
    hbm = hbm or 6800.0
    l2_bytes = l2_size_bytes(torch, dev)
    ws = N * (32 + 4 * C) + NN * (32 + 4 * srow(C))
    l2_probe_gbs = l2_probe(torch, dev, dp) if rank == 0 else None
    if l2_bytes and ws <= l2_bytes and l2_probe_gbs:
        bound, peak, peak_src = "l2", l2_probe_gbs, "measured in this run (dipole_probe_l2, 48 MB x 20, best of 10)"
    else:
        bound, peak, peak_src = "hbm", hbm, hbm_src
    kern = f"k_query<{dp_cp(C)},float,{dom}>"
    tr = measured_traffic(kern)
    gbs = lambda b: b / (t_k * 1e-3) / 1e9
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    issue = None
    if tr and tr.get("inst_executed") and clocks and clocks.get("sm_mhz"):
        cap = sms * 4 * clocks["sm_mhz"] * 1e6 * t_k * 1e-3
        issue = {"warp_inst_per_launch": tr["inst_executed"], "sm_mhz": clocks["sm_mhz"],
                 "schedulers": sms * 4, "frac": tr["inst_executed"] / cap,
                 "inst_per_warp_step": tr["inst_executed"] / max(Us, 1),
                 "source": "profiles/traffic.json (ncu, same kernel source)"}
    figures = {
        "per_lane": {"bytes": per_lane, "achieved_gbs": gbs(per_lane), "frac": gbs(per_lane) / peak,
                     "formula": "16*tested + (4+12C)*far + (28+4C)*leaf_points + (12+4C)*queries"},
        "per_warp": {"bytes": per_warp, "achieved_gbs": gbs(per_warp), "frac": gbs(per_warp) / peak,
                     "formula": "32*warp_steps + 12C*far_steps + (32+4C)*opened_leaf_points + (12+4C)*queries"},
        "issue": issue,
    }
    cands = [("per_warp", figures["per_warp"]["frac"])] + ([("issue", issue["frac"])] if issue else [])
    binding = max(cands, key=lambda kv: kv[1])[0]
    return {"bound": bound, "achieved": gbs(per_lane), "peak": peak, "unit": "GB/s",
            "frac": gbs(per_lane) / peak, "peak_source": peak_src,
            "traffic": tr["dram_bytes_per_launch"] if tr else None,
            "kernel": kern + " (its traversal launches only: CUDA events in the timed region)",
            "launch_ms": t_k, "figures": figures, "binding": binding,
            "algorithmic_bytes_per_launch": per_lane,
            "per_query": {"tested": Tn / Q, "far": An / Q, "leaf_points": Ln / Q},
            "per_packet": {"warp_steps": Us / ((Q + 31) // 32), "far_steps": Uf / ((Q + 31) // 32),
                           "opened_leaf_points": Up / ((Q + 31) // 32)},
            "working_set_mb": ws / 2 ** 20, "l2_mb": l2_bytes / 2 ** 20, "hbm_peak_gbs": hbm,
            "l2_probe_gbs": l2_probe_gbs,
            "ncu": ({k: tr.get(k) for k in ("lts_pct", "dram_pct", "issue_active_pct",
                                               "warps_active_pct", "long_scoreboard_per_issue")}
                    if tr else None)}


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
    dp.dipole_traversal_elapsed("forward")  # drop anything recorded before
    dp.dipole_traversal_elapsed("adjoint")
    dp.dipole_traversal_timer(True)  # CUDA events around each traversal kernel
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
    dp.dipole_traversal_timer(False)
    torch.cuda.synchronize()
    kf_ms, kf_n = dp.dipole_traversal_elapsed("forward")
    ka_ms, ka_n = dp.dipole_traversal_elapsed("adjoint")
    kernel_ms = {"forward": kf_ms / max(kf_n, 1), "adjoint": ka_ms / max(ka_n, 1)}
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
    npk = (Q + 31) // 32
    cnt = torch.empty((Q, 3), dtype=torch.int32, device=dev)
    pcnt = torch.empty((npk, 4), dtype=torch.int32, device=dev)
    dp.dipole_query_packet_counts(h, X, BETA, pcnt, counts=cnt)
    sums = cnt.to(torch.int64).sum(0).tolist()
    usums = pcnt.to(torch.int64).sum(0).tolist()
    info = dp.dipole_tree_info_get(h)
    dp.dipole_tree_destroy(h)
    roofline = roofline_block(torch, dev, dp, C, Q, N, info["n_nodes"], sums, usums, kernel_ms,
                              clocks, rank)
    breakdown = {"build_ms": ph[0], "refit_ms": ph[1], "forward_ms": ph[2], "adjoint_ms": ph[3],
                 "forward_queries_per_s": Q / (ph[2] * 1e-3),
                 "adjoint_queries_per_s": Q / (ph[3] * 1e-3),
                 "refit_forward_adjoint_queries_per_s": Q / ((ph[1] + ph[2] + ph[3]) * 1e-3),
                 "interactions_per_s": world * (sums[1] + sums[2]) * 2 / (ms_per_step * 1e-3),
                 "forward_kernel_ms": kernel_ms["forward"], "adjoint_kernel_ms": kernel_ms["adjoint"],
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
                        sums, roofline["peak"])

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

    # ---- the other workloads, each with its error against the oracle ----
    configs = None
    if rank == 0 and world == 1 and not args.no_configs:
        del flush
        torch.cuda.empty_cache()
        configs = config_rows(torch, dp, dev, stream, clocks)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": config_of(w, "flushed between timed steps (512 MB write)"),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clocks, "breakdown": breakdown,
                "bf16_attrs": bf16, "next_rows": nxt, "accuracy": accuracy,
                "configs": configs, "impl": "ours"}
        print(json.dumps(line), flush=True)
    if world > 1:
        td.destroy_process_group()
    return 0


def _normwise(y, r):
    y, r = np.asarray(y, np.float64), np.asarray(r, np.float64)
    den = np.max(np.abs(r), axis=0)
    return np.max(np.abs(y - r), axis=0) / np.where(den > 0, den, 1.0)


def _rel2(y, r):
    y, r = np.asarray(y, np.float64), np.asarray(r, np.float64)
    return np.linalg.norm(y - r, axis=0) / np.maximum(np.linalg.norm(r, axis=0), 1e-300)


def _bf16_round(a):
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    return (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16).astype(np.uint32).view(np.float32).reshape(a.shape)


def config_rows(torch, dp, dev, stream, clocks=None):
    """The workloads besides the headline one (sphere-2k and scene-200k
    forward only, scene-3m-bf16 forward + adjoint in bf16 and in float32),
    each timed with CUDA events (median of 5, a 512 MB L2 flush before each)
    and checked against the oracle's FP64 Barnes-Hut on a query sample (all
    queries for sphere-2k, where the plain O(NQ) sum is also given).  The
    scene-3m-bf16 row carries the roofline block of its float32 traversals
    (working set beyond the L2: the HBM bound)."""
    import oracle
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)

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

    def kernel_ms(mode):
        ms, n = dp.dipole_traversal_elapsed(mode)
        return ms / max(n, 1)

    rows = {}
    for name, n_err in (("sphere-2k", None), ("scene-200k", 4096)):
        w = syn.workload(name)
        c = w.cloud
        Q, C = len(w.queries), w.mu.shape[1]
        P_, N_, A_, E_ = T(c.points), T(c.normals), T(c.areas), T(c.eps)
        X_, MU_ = T(w.queries), T(w.mu)
        out = torch.empty((Q, C), device=dev)
        b_ms = timed(lambda: dp.dipole_tree_destroy(dp.dipole_build_tree(P_, N_, A_, E_, LEAF, 10)))
        h = dp.dipole_build_tree(P_, N_, A_, E_, LEAF, 10)
        dp.dipole_refit(h, MU_)
        dp.dipole_traversal_elapsed("forward")
        dp.dipole_traversal_timer(True)
        f_ms = timed(lambda: dp.dipole_forward(h, X_, BETA, out))
        dp.dipole_traversal_timer(False)
        fk_ms = kernel_ms("forward")
        y = out.cpu().numpy()
        dp.dipole_sync_status(h)
        dp.dipole_tree_destroy(h)
        ot = oracle.Tree(c.points, c.normals, c.areas, c.eps, leaf_size=LEAF)
        ot.update(w.mu)
        idx = np.arange(Q) if n_err is None else np.random.default_rng(7).choice(Q, n_err, replace=False)
        t0 = time.perf_counter()
        ref = ot.forward(w.queries[idx], BETA)
        cpu_qps = len(idx) / (time.perf_counter() - t0)
        row = {"points": c.n, "queries": Q, "channels": C, "build_ms": b_ms, "forward_ms": f_ms,
               "forward_kernel_ms": fk_ms, "forward_queries_per_s": Q / (f_ms * 1e-3),
               "error_vs_oracle_bh_normwise": _normwise(y[idx], ref).tolist(),
               "error_queries": int(len(idx)),
               "cpu_oracle_forward_queries_per_s": cpu_qps, "cpu_cores": oracle.num_threads(),
               "cpu_sample": f"oracle FP64 Barnes-Hut forward on {len(idx)} queries (wall clock)"}
        if n_err is None:
            bf = oracle.brute_forward(c.points, c.normals, c.areas, c.eps, w.mu, w.queries)
            row["bh_vs_brute_force_normwise"] = _normwise(ref, bf).tolist()
            row["gpu_vs_brute_force_normwise"] = _normwise(y, bf).tolist()
        rows[name] = row
        del P_, N_, A_, E_, X_, MU_, out

    # scene-3m-bf16: float32 and bf16 attribute storage on the same GPU, and bf16
    # attributes with bf16 node moments (DIPOLE_BF16_MOMENTS)
    w = syn.workload("scene-3m-bf16")
    c = w.cloud
    Q, C = len(w.queries), w.mu.shape[1]
    P_, N_, A_, E_ = T(c.points), T(c.normals), T(c.areas), T(c.eps)
    X_ = T(w.queries)
    G_ = T(syn.upstream_grad(Q, C, seed=404))
    out = torch.empty((Q, C), device=dev)
    grad = torch.empty((c.n, C), device=dev)
    plan = dp.QueryPlan(Q, dev)
    b_ms = timed(lambda: dp.dipole_tree_destroy(dp.dipole_build_tree(P_, N_, A_, E_, LEAF, 10)), reps=3)
    h = dp.dipole_build_tree(P_, N_, A_, E_, LEAF, 10)
    res = {"points": c.n, "queries": Q, "channels": C, "build_ms": b_ms}
    idx = np.random.default_rng(4).choice(Q, 10000, replace=False)
    outs = {}
    for dt, mu, m16 in (("f32", T(w.mu), False), ("bf16", T(w.mu).to(torch.bfloat16), False),
                        ("bf16_moments", T(w.mu).to(torch.bfloat16), True)):
        r_ms = timed(lambda: dp.dipole_refit(h, mu, bf16_moments=m16), reps=3)
        dp.dipole_traversal_elapsed("forward")
        dp.dipole_traversal_elapsed("adjoint")
        dp.dipole_traversal_timer(True)
        f_ms = timed(lambda: dp.dipole_forward_planned(h, X_, BETA, out, plan), reps=3)
        a_ms = timed(lambda: dp.dipole_adjoint_planned(h, X_, BETA, G_, grad, plan, False), reps=3)
        dp.dipole_traversal_timer(False)
        res[dt] = {"refit_ms": r_ms, "forward_ms": f_ms, "adjoint_ms": a_ms,
                   "forward_kernel_ms": kernel_ms("forward"), "adjoint_kernel_ms": kernel_ms("adjoint"),
                   "refit_forward_adjoint_ms": r_ms + f_ms + a_ms,
                   "queries_per_s": Q / ((r_ms + f_ms + a_ms) * 1e-3)}
        dp.dipole_refit(h, mu, bf16_moments=m16)
        dp.dipole_forward(h, X_, BETA, out)
        outs[dt] = out[torch.from_numpy(idx).to(dev)].cpu().numpy()
        # the adjoint with the upstream gradient on the sample only
        gs = torch.zeros((Q, C), device=dev)
        gs[torch.from_numpy(idx).to(dev)] = G_[torch.from_numpy(idx).to(dev)]
        dp.dipole_adjoint(h, X_, BETA, gs, grad, False)
        outs[dt + "_adj"] = grad.cpu().numpy()
        del mu
    # roofline of the float32 traversals: per-query and per-packet counts of this tree
    dp.dipole_refit(h, T(w.mu))
    npk = (Q + 31) // 32
    cnt = torch.empty((Q, 3), dtype=torch.int32, device=dev)
    pcnt = torch.empty((npk, 4), dtype=torch.int32, device=dev)
    dp.dipole_query_packet_counts(h, X_, BETA, pcnt, counts=cnt)
    sums = cnt.to(torch.int64).sum(0).tolist()
    usums = pcnt.to(torch.int64).sum(0).tolist()
    nodes = dp.dipole_tree_info_get(h)["n_nodes"]
    del cnt, pcnt
    res["roofline"] = roofline_block(
        torch, dev, dp, C, Q, c.n, nodes, sums, usums,
        {"forward": res["f32"]["forward_kernel_ms"], "adjoint": res["f32"]["adjoint_kernel_ms"]},
        clocks, 0)
    dp.dipole_sync_status(h)
    dp.dipole_tree_destroy(h)
    res["speedup_bf16_vs_f32"] = {
        "refit_forward_adjoint": res["f32"]["refit_forward_adjoint_ms"] / res["bf16"]["refit_forward_adjoint_ms"],
        "step_with_build": (b_ms + res["f32"]["refit_forward_adjoint_ms"]) /
                           (b_ms + res["bf16"]["refit_forward_adjoint_ms"]),
        "forward_kernel": res["f32"]["forward_kernel_ms"] / res["bf16"]["forward_kernel_ms"],
        "adjoint_kernel": res["f32"]["adjoint_kernel_ms"] / res["bf16"]["adjoint_kernel_ms"]}
    res["speedup_bf16_moments_vs_f32"] = {
        "refit_forward_adjoint": res["f32"]["refit_forward_adjoint_ms"] /
                                 res["bf16_moments"]["refit_forward_adjoint_ms"],
        "forward_kernel": res["f32"]["forward_kernel_ms"] / res["bf16_moments"]["forward_kernel_ms"]}
    ot = oracle.Tree(c.points, c.normals, c.areas, c.eps, leaf_size=LEAF)
    g_s = syn.upstream_grad(Q, C, seed=404)[idx].astype(np.float64)
    ot.update(w.mu)
    ref_f = ot.forward(w.queries[idx], BETA)
    aref_f = ot.adjoint(w.queries[idx], BETA, g_s)
    ot.update(_bf16_round(w.mu))
    ref_b = ot.forward(w.queries[idx], BETA)
    aref_b = ot.adjoint(w.queries[idx], BETA, g_s)
    ot.update(_bf16_round(w.mu), bf16_moments=True)
    ref_m, allow_m = ot.forward_bf16_allowance(w.queries[idx], BETA)
    den_m = np.max(np.abs(ref_m), axis=0)
    beyond_m = np.max(np.abs(outs["bf16_moments"] - ref_m) - allow_m, axis=0) / np.where(den_m > 0, den_m, 1.0)
    res["accuracy"] = {
        "queries": 10000,
        "f32_forward_normwise": _normwise(outs["f32"], ref_f).tolist(),
        "f32_adjoint_normwise": _normwise(outs["f32_adj"], aref_f).tolist(),
        "bf16_forward_normwise_vs_f32_attrs": _normwise(outs["bf16"], ref_f).tolist(),
        "bf16_forward_rel_l2_vs_f32_attrs": _rel2(outs["bf16"], ref_f).tolist(),
        "bf16_forward_normwise_vs_bf16_attrs": _normwise(outs["bf16"], ref_b).tolist(),
        "bf16_adjoint_normwise_vs_bf16_attrs": _normwise(outs["bf16_adj"], aref_b).tolist(),
        "input_rounding_alone_normwise": _normwise(ref_b, ref_f).tolist(),
        "input_rounding_alone_rel_l2": _rel2(ref_b, ref_f).tolist(),
        "bf16_moments_forward_normwise_vs_f32_attrs": _normwise(outs["bf16_moments"], ref_f).tolist(),
        "bf16_moments_forward_rel_l2_vs_f32_attrs": _rel2(outs["bf16_moments"], ref_f).tolist(),
        "bf16_moments_forward_normwise_vs_oracle_bf16_moments":
            _normwise(outs["bf16_moments"], ref_m).tolist(),
        "bf16_moments_forward_beyond_rounding_allowance": beyond_m.tolist(),
        "bf16_moments_queries_with_allowance": float(np.mean(np.any(allow_m > 0, axis=1))),
        "input_and_moment_rounding_alone_normwise": _normwise(ref_m, ref_f).tolist(),
        "gate": "3e-3 max-norm per channel vs the float32 attributes (met where the input "
                "rounding alone is below it); 1e-4 vs the oracle on the bf16-rounded inputs"}
    rows["scene-3m-bf16"] = res
    return rows


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
              peak):
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
        "forward_grad_frac_of_peak": b_fg / (f_ms * 1e-3) / 1e9 / peak,
        "adjoint_geom_logical_gbs": b_geo / (geo_ms * 1e-3) / 1e9,
        "adjoint_geom_frac_of_peak": b_geo / (geo_ms * 1e-3) / 1e9 / peak,
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
    for k in (1, 2, 4, 8, 16, 32, 36, 64):
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
