#!/usr/bin/env python
"""Benchmark: PartialACO iterations on the 200,000-city clustered workload on GB300s.

One step = one ACO iteration of the whole colony (1024 ants): tour construction (PartialACO
rebuild of at most 1% of every ant's l_best by Eq. 1 over 16-nearest candidate lists) and the
pheromone update (l_best commit, C_gbest, candidate-edge pheromone rebuild).  Setup (candidate
lists, initial tours) is untimed.  Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun the ranks run one colony split by ants (every rank the whole colony state, its
share of the ants built, one all-gather of the improved ants' commits per iteration): the same
work as on one GPU, so the N-GPU figure is strong-scaled.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import aco_synth  # noqa: E402

METRIC = "city decisions/s and ACO iterations/s at n=200K on 1 GB300; % of mem roofline"
# DRAM bytes (read + write) per decision of construct_lbest_kernel from one ncu capture of the
# 200,000-city workload at m = 256 (62.83 MB for 266,770 decisions), valid for the code it was
# taken on: code_sha1 hashes the kernel's sources (the construction's device code and its
# single-colony launch) without their comments and blank lines, and the bench reports null
# traffic once the code changes.
CONSTRUCT_SOURCES = ("construct_dev.cuh", "construct.cu")
CONSTRUCT_TRAFFIC = {"code_sha1_12": "c8c114747692", "bytes_per_decision": 62828032.0 / 266769.67}
L2_FLUSH_BYTES = 512 << 20  # > 126 MB L2


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="lbest200k",
                    choices=sorted(aco_synth.WORKLOADS) + ["batch512", "learned20k", "schedule20k", "ls200k",
                                                           "async200k", "ir200k"])
    ap.add_argument("--ants", type=int, default=0, help="override m (profiling of smaller cases)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the short runs of the other forms")
    ap.add_argument("--cpu-sample", type=int, default=32, help="ants in the oracle's timed sample")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def aggregate_over_ranks(t_step: float, units: float, world: int, device="cpu"):
    """Whole-job figures: the slowest rank's timed seconds and the units all ranks processed."""
    if world == 1:
        return float(t_step), float(units)
    import torch
    import torch.distributed as dist

    tt = torch.tensor([float(t_step)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    uu = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(uu, op=dist.ReduceOp.SUM)
    return float(tt.item()), float(uu.item())


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.15)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for ln in f:
                parts = [x.strip() for x in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ algorithmic bytes
def code_sha1(*names: str) -> str:
    """SHA-1 (12 hex digits) of kernel sources, in order, with their // comments, trailing blanks
    and blank lines removed: comment edits keep an ncu capture of the code valid, code edits do
    not."""
    import hashlib
    import re

    lines = []
    for name in names:
        with open(os.path.join(ROOT, "paper_1709_03187_gb300", "csrc", name), encoding="utf-8") as f:
            for line in f:
                line = re.sub(r"//.*$", "", line).rstrip()
                if line:
                    lines.append(line)
    return hashlib.sha1("\n".join(lines).encode()).hexdigest()[:12]


def construct_bytes_model(decisions: int, fallbacks: int, fallback_rebuilt: int, k: int, m: int) -> int:
    """Algorithmic bytes of one construction launch by the method's byte model.

    Per decision: the current city's candidate row, its pheromone and its heuristic entries, one
    FP32 word each per candidate (3 x 4k B), and the 4 B segment write.  Per exhausted-list step:
    the current city's neighbour row over all ants (8 m B) and the ant's list of discarded cities
    (4 M B, M = the ant's rebuilt count, summed over the steps by a device counter).  Per ant: the
    segment read and written (8 M B) and the incremental length over 2 M coordinate gathers
    (16 B each); summed over the ants, M is the number of decisions."""
    return decisions * (12 * k + 4) + fallbacks * 8 * m + 4 * fallback_rebuilt + decisions * (8 + 32)


def construct_bytes_layout(decisions: int, k: int, m: int) -> int:
    """The bytes this kernel's own layout needs, narrower than the model: per decision one
    candidate row of (4 B city + 4 B FP32 weight) x k and the 4 B segment write; per rebuilt city
    its old l_best entry (4 B), the segment read back (4 B) and one coordinate pair for each of
    the old and the new path (2 x 16 B); per ant the two closing coordinate pairs of each path."""
    return decisions * (8 * k + 4) + decisions * (4 + 4 + 32) + 64 * m


def rebuild_bytes(n: int, m: int, k: int) -> int:
    """Algorithmic bytes of one pheromone rebuild: the n x m table of neighbour ranks (2 B per
    city and ant), eta^beta in (8 B), FP64 weight out (8 B) and FP32 weight out (4 B) per
    candidate edge, and the m per-ant weights (8 B)."""
    return 2 * n * m + n * k * (8 + 8 + 4) + 8 * m


def measure_l2_peak(stream, nbytes: int = 32 << 20, passes: int = 64):
    """L2 bandwidth from the library's STREAM-style probe on a buffer well inside L2 (32 MB of the
    126 MB): read GB/s (16-byte loads cached in L2 only) and copy GB/s (bytes read + written)."""
    import torch

    from paper_1709_03187_gb300 import aco_probe_bandwidth

    buf = torch.ones(nbytes // 4, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    best_r = best_c = 0.0
    for _ in range(3):
        ms = aco_probe_bandwidth(buf, nbytes, 0, passes, stream)
        best_r = max(best_r, (nbytes - 16) * passes / (ms / 1e3) / 1e9)
        ms = aco_probe_bandwidth(buf, nbytes, 1, passes, stream)
        best_c = max(best_c, nbytes * passes / (ms / 1e3) / 1e9)
    del buf
    return {"read_gbs": best_r, "copy_gbs": best_c, "buffer_mb": nbytes >> 20, "passes": passes,
            "how": "aco_probe_bandwidth, best of 3 launches of 64 passes, CUDA events"}


def instance_desc(wl) -> str:
    """The coordinates of a workload, as its generator draws them."""
    kind, g = wl["gen"]
    if kind == "clustered":
        return f"clustered ({g['n_clusters']} Gaussian clusters, sigma={g['sigma']})"
    if kind == "mixed":
        return f"half uniform in [0,1)^2, half in {g['n_clusters']} Gaussian clusters (sigma={g['sigma']})"
    return "uniform in [0,1)^2"


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1709_03187_gb300 import Colony, ShardedColony

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wl = aco_synth.WORKLOADS[args.workload]
    params = dict(wl["params"])
    if args.ants:
        params["m"] = args.ants
    n, m, k = params["n"], params["m"], params["k"]

    def make_colony(coords):
        # N ranks: one colony split by ants (every rank the same instance and seed)
        if world > 1:
            return ShardedColony(coords, rank=rank, world=world, stream=stream, **params)
        return Colony(coords, stream=stream, **params)
    xy = aco_synth.make(args.workload)
    stream = torch.cuda.Stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    t0 = time.perf_counter()
    col = make_colony(xy)
    col.build_candidates()
    col.iterate(0)  # Algorithm 1: initial tours
    s0 = col.stats()
    setup_s = time.perf_counter() - t0
    it = 1
    for _ in range(args.warmup):
        col.iterate(it)
        it += 1
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    evs = [(E(), E(), E()) for _ in range(args.steps)]
    barrier()
    st_before = col.stats()
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    with torch.cuda.stream(stream):
        for (e0, e1, e2) in evs:
            flush.zero_()  # L2 flush between timed steps (outside the events)
            e0.record(stream)
            col.construct(it)
            e1.record(stream)
            if world > 1:
                col.exchange()  # every rank's commits (export, all-gather, import)
            col.update()
            e2.record(stream)
            it += 1
    barrier()
    clocks = sampler.stop()
    st_after = col.stats()
    t_con = sum(a.elapsed_time(b) for a, b, _ in evs) / 1e3
    t_upd = sum(b.elapsed_time(c) for _, b, c in evs) / 1e3
    t_step = t_con + t_upd
    decisions = st_after["decisions"] - st_before["decisions"]
    t_max, dec_all = aggregate_over_ranks(t_step, decisions, world, "cuda")
    value = dec_all / t_max
    its = args.steps / t_max  # one colony (split over the ranks when N > 1)

    hbm_peak, peak_kind = read_peaks()
    launches = args.steps
    fb = st_after["fallbacks"] - st_before["fallbacks"]
    fb_m = st_after["fallback_rebuilt"] - st_before["fallback_rebuilt"]
    fb_scan = st_after["fallback_scanned"] - st_before["fallback_scanned"]
    c_bytes = construct_bytes_model(decisions, fb, fb_m, k, m) / launches
    c_layout = construct_bytes_layout(decisions, k, m) / launches
    r_bytes = rebuild_bytes(n, m, k)
    c_avg = t_con / launches
    u_avg = t_upd / launches
    l2 = measure_l2_peak(stream)
    kernels = {
        "construct_lbest_kernel": {"avg_ms": c_avg * 1e3, "alg_bytes": c_bytes, "achieved_gbs": c_bytes / c_avg / 1e9,
                                   "layout_bytes": c_layout, "layout_gbs": c_layout / c_avg / 1e9},
        "update (commit + gbest_q + rebuild)": {"avg_ms": u_avg * 1e3, "alg_bytes": r_bytes,
                                                "achieved_gbs": r_bytes / u_avg / 1e9},
    }
    dom = "construct_lbest_kernel" if c_avg >= u_avg else "update (commit + gbest_q + rebuild)"
    ach = kernels[dom]["achieved_gbs"]
    traffic = None
    # the stored figure is per decision of the 200,000-city workload (k = 16) at this code
    if (dom == "construct_lbest_kernel" and args.workload == "lbest200k"
            and code_sha1(*CONSTRUCT_SOURCES) == CONSTRUCT_TRAFFIC["code_sha1_12"]):
        traffic = round(CONSTRUCT_TRAFFIC["bytes_per_decision"] * decisions / launches)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(ach, 2), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(ach / hbm_peak, 5), "peak_source": f"{peak_kind} hbm_gbs", "traffic": traffic,
                "bytes_model": "per decision 12k + 4 B (candidate, pheromone, heuristic rows in FP32; segment "
                               "write); per exhausted step 8m B (neighbour row) + 4M B (discarded list, M from "
                               "a device counter); per rebuilt city 8 + 32 B (segment, coordinate gathers)",
                "exhausted_steps_per_launch": fb / launches, "mean_M_at_exhausted_step": fb_m / max(1, fb),
                "mean_list_scanned_at_exhausted_step": fb_scan / max(1, fb),
                "l2_peak_gbs": round(l2["read_gbs"], 1), "frac_l2": round(ach / l2["read_gbs"], 5),
                "l2_probe": l2,
                "layout_frac_l2": round(kernels["construct_lbest_kernel"]["layout_gbs"] / l2["read_gbs"], 5),
                "note": "each ant is a dependent chain of Eq. 1 decisions; a launch lasts as long as the "
                        "longest chain, so the kernel is latency-bound; its working set sits in L2",
                "kernels": {kn: {kk: round(v, 4) for kk, v in kv.items()} for kn, kv in kernels.items()}}

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, xy, params, stream, make_colony, world)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload.startswith("lbest"):
        cpu = cpu_baseline_oracle(xy, params, it, args.cpu_sample)
    col.close()
    secondary = None
    if rank == 0 and world == 1 and not args.no_secondary and args.workload == "lbest200k" and not args.ants:
        secondary = secondary_results()
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "decisions/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_max / args.steps * 1e3, 4), "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "iterations_per_s": round(its, 2),
        "config": {"workload": f"{args.workload}: n={n} {instance_desc(wl)}, k={k}, m={m}, "
                               f"f={params['max_mod_frac']}, alpha={params['alpha']}, beta={params['beta']}, "
                               f"tau0={params['tau0']}, p_partial={params['p_partial']}",
                   "n": n, "m": m, "k": k, "parallelism": f"one colony split by ants over {world} GPUs" if world > 1 else "single colony",
                   "l2": "flushed (512 MB write) before every timed step, outside the events",
                   "decisions_per_step": decisions / args.steps,
                   # every ant's new tour has n positions; those not decided this step stay in
                   # place in l_best (the preserved part, never copied) or are a drawn start city
                   "positions_per_step": float(m * n),
                   "kept_positions_per_step": m * n - decisions / args.steps,
                   "fallbacks_per_step": (st_after["fallbacks"] - st_before["fallbacks"]) / args.steps,
                   "exact_resolves_per_step": (st_after["exact_resolves"] - st_before["exact_resolves"]) / args.steps,
                   "improved_per_step": (st_after["improved"] - st_before["improved"]) / args.steps,
                   "setup_s": round(setup_s, 3), "setup_decisions": s0["decisions"],
                   "gbest_after": st_after["gbest"]},
        "roofline": roofline,
        "clocks": clocks,
        "gpu_launches": 4 * args.steps,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "secondary": secondary,
    }
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def secondary_results():
    """Short runs of the other forms of the hot path, reported beside the headline (after its timed
    region): the dense Section 2 form (dense100, 50 timed iterations), the batched form against
    per-instance launches on the first 64 of batch512's instances (16 of them timed one by one),
    and the learned proposal's time to the plain form's quality at n = 20,000 on one seed, with
    its training time beside it (the training runs once and serves every later instance)."""
    import types

    a = types.SimpleNamespace(steps=50, warmup=5, cpu_sample=16)
    out = {}
    d = run_dense(a, emit=False)
    out["dense100"] = {kk: d[kk] for kk in ("value", "unit", "iterations_per_s", "ms_construct", "ms_update")}
    out["dense100"]["cpu_oracle_decisions_per_s"] = d["cpu_baseline"]["value"]
    b = run_batch(a, count=64, per_instance_sample=16, emit=False)
    out["batch64"] = {kk: b[kk] for kk in ("workload", "batched_instances_per_s", "per_instance_instances_per_s",
                                           "speedup", "schedule", "schedule_kind", "per_instance_sample")}
    lr = run_learned(a, seeds=(1,), emit=False)
    tr = lr["training"]
    out["learned20k"] = {"ratio_learned_over_plain": lr["value"], "seed": lr["per_seed"],
                         "training_gpu_ms": round(tr["plain_ms"] + tr["train_ms"], 1), "training": tr,
                         "note": "ratio of GPU wall-clock to the plain form's final C_gbest; the training (plain "
                                 "runs for labels, then Adam) is reported beside it, not inside it"}
    return out


def run_e2e(args, xy, params, stream, make_colony, world=1):
    """The same metric through the public API from host buffers: pinned coordinates copied in,
    candidate lists, initial tours and `steps` iterations, C_gbest read back every step and the
    best tour read back at the end.  Decisions of the `steps` iterations / wall time of the whole
    solve (set-up time counted, set-up decisions not); with N ranks, the decisions of every rank
    over the slowest rank's wall time."""
    import torch

    host = torch.from_numpy(xy).pin_memory()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        dev = host.to("cuda", non_blocking=True)
    stream.synchronize()
    col = make_colony(dev)
    col.build_candidates()
    gb = []
    dec0 = 0
    for it in range(args.steps + 1):
        col.iterate(it)
        s_it = col.stats()  # device -> host read of the step's result (C_gbest, 8 B)
        gb.append(s_it["gbest"])
        if it == 0:
            dec0 = s_it["decisions"]  # the initial tours are set-up, not steps of the metric
            t_setup = time.perf_counter() - t0  # the read above waited for the first update
    st = col.stats()
    lb, cl, _ = col.state()
    best = lb[st["gbest_ant"]].cpu()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    col.close()
    del best
    wall, dec = aggregate_over_ranks(wall, st["decisions"] - dec0, world, "cuda")
    t_setup, _ = aggregate_over_ranks(t_setup, 0, world, "cuda")
    t_setup_note = ("wall time includes instance creation, candidate lists and the initial tours; decisions "
                    "are those of the timed iterations only; setup_s is the wall time up to the first "
                    "update's result, after_setup the same rate over the rest of the wall time")
    return {"value": round(dec / wall, 1), "unit": "decisions/s",
            "h2d_bytes_per_step": round(host.numel() * 8 / (args.steps + 1), 1),
            "d2h_bytes_per_step": round(8 + 4 * params["n"] / (args.steps + 1), 1),
            "wall_s": round(wall, 3), "iterations": args.steps + 1, "setup_s": round(t_setup, 3),
            "after_setup": round(dec / max(wall - t_setup, 1e-9), 1), "note": t_setup_note}


def oracle_start(xy, params, seeds=2):
    """The oracle's own starting colony, built with no input from the device: candidate lists by
    the exact x-sweep, initial tours of `seeds` ants (one host thread each), repeated over the m
    ants as their l_best, and the pheromone rebuild (timed, one core).  Returns (oracle, rebuild
    seconds)."""
    import oracle

    m, k = params["m"], params["k"]
    cand = oracle.knn_sweep(xy, k)
    ref = oracle.Oracle(xy, cand=cand, **params)
    ref.construct(0, ants=np.arange(seeds, dtype=np.int32), threads=seeds)  # oracle-built initial tours
    T = ref.newtours[:seeds]
    L = oracle.tour_lengths(xy, T)
    ref.set_lbest(np.ascontiguousarray(T[np.arange(m) % seeds]), L[np.arange(m) % seeds])
    t0 = time.perf_counter()
    ref.construct(1, ants=[])
    return ref, time.perf_counter() - t0


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def time_oracle_sample(ref, iteration, ants, threads):
    """Seconds and decisions of one PartialACO iteration of the listed ants (pheromone kept)."""
    ref.reset_counters()
    t0 = time.perf_counter()
    ref.construct(iteration, ants=ants, rebuild=False, threads=threads)
    return max(time.perf_counter() - t0, 1e-9), ref.counters()["decisions"]


def cpu_baseline_oracle(xy, params, iteration, sample):
    """The oracle timed on this host on its own colony (oracle_start): one PartialACO iteration of
    a sample of ants on one core, and of a larger sample spread over every core; each projected to
    the full colony as t_rebuild + (m / sample) * t_construct (the rebuild runs on one core)."""
    ref, t_rb = oracle_start(xy, params)
    m = params["m"]
    rng = np.random.default_rng(0)
    cores = host_cores()
    out = {}
    for label, threads, size in (("one_core", 1, min(sample, m)), ("all_cores", cores, min(m, 8 * cores))):
        ants = rng.choice(m, size=size, replace=False).astype(np.int32)
        t_cs, dec = time_oracle_sample(ref, iteration, ants, threads)
        full_dec = dec * m / ants.size
        full_t = t_rb + t_cs * m / ants.size
        out[label] = {"value": round(full_dec / full_t, 1), "cores": threads, "sample_ants": int(ants.size),
                      "construct_s": round(t_cs, 3), "projected_iteration_s": round(full_t, 3)}
    best = out["all_cores"]
    return {"value": best["value"], "unit": "decisions/s", "cores": best["cores"], "kind": "oracle",
            "sample": f"one iteration of sampled ants of the {m}-ant colony of the oracle's own start (its initial "
                      f"tours of 2 ants repeated as l_best): {out['all_cores']['sample_ants']} ants over "
                      f"{cores} threads, and {out['one_core']['sample_ants']} on one core; plus the full "
                      f"pheromone rebuild on one core ({t_rb:.2f} s); projected t_rebuild + (m/sample) t_construct",
            "one_core": out["one_core"], "all_cores": out["all_cores"], "host_cores": cores}


# ------------------------------------------------------------------ reference arm (the oracle)
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle

    t_run = time.perf_counter()
    wl = aco_synth.WORKLOADS[args.workload]
    params = dict(wl["params"])
    n, m, k = params["n"], params["m"], params["k"]
    xy = aco_synth.make(args.workload)
    t0 = time.perf_counter()
    if params["mode"] == 1:
        ref, t_rb = oracle_start(xy, params)
    else:
        ref = oracle.Oracle(xy, **params)
        t_rb = 0.0
    setup = time.perf_counter() - t0
    cores = host_cores()
    sample = max(1, min(m, cores))  # one sampled ant per host thread and step
    rng = np.random.default_rng(1)
    per = []
    sampled = []  # measured seconds of each step's sampled ants
    for step in range(args.warmup + args.steps):
        if params["mode"] == 1:
            ants = rng.choice(m, size=sample, replace=False).astype(np.int32)
            t_cs, dec = time_oracle_sample(ref, step + 2, ants, cores)
            sampled.append(t_cs)
            # the rebuild (measured once in set-up) plus the sampled ants projected to the colony
            t_full = t_rb + t_cs * m / sample
            per.append((dec * m / sample, t_full))
        else:
            ref.reset_counters()
            t1 = time.perf_counter()
            ref.iterate(step)
            per.append((ref.counters()["decisions"], time.perf_counter() - t1))
    timed = per[args.warmup:]
    dec = sum(d for d, _ in timed)
    tt = sum(t for _, t in timed)
    value = dec / tt
    if params["mode"] == 1:
        how = (f"each step: {sample} random ants of the {m}-ant colony over {cores} host threads (the oracle's own "
               f"start: initial tours of 2 ants, repeated as l_best), plus the pheromone rebuild over all ants on one "
               f"core ({t_rb:.2f} s, measured once); the step time is projected as t_rebuild + (m/sample) "
               f"t_construct; set-up {setup:.1f} s")
    else:
        how = f"every step is a whole iteration of the colony, one core; set-up {setup:.1f} s"
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "decisions/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tt / max(1, len(timed)) * 1e3, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "projected": params["mode"] == 1,
           # what ran: the whole run's wall time, and per timed step the sampled ants' seconds
           "wall_s": round(time.perf_counter() - t_run, 3),
           "sampled_ms_per_step": round(sum(sampled[args.warmup:]) / max(1, len(timed)) * 1e3, 3) if sampled else None,
           "config": {"workload": args.workload, "n": n, "m": m, "k": k},
           "cpu_baseline": {"value": round(value, 1), "unit": "decisions/s",
                            "cores": cores if params["mode"] == 1 else 1, "kind": "oracle", "sample": how},
           "e2e": {"value": round(value, 1), "unit": "decisions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ------------------------------------------------------------------ batched form
def run_batch(args, count=512, per_instance_sample=None, emit=True):
    """512 instances, n log-uniform in [50, 5000] (uniform cities), k = 20, m = min(n, 256),
    f = 1, 100 iterations each.  Batched: one launch per step over all colonies, CUDA-graph
    replay, autotuned schedule.  Per-instance: the same calls instance by instance; a stratified
    sample of instances is timed and scaled to all 512.  Instances/s of the whole job (candidate
    lists + initial tours + iterations; allocation excluded in both arms)."""
    import torch

    from paper_1709_03187_gb300 import Batch, Colony

    torch.cuda.set_device(0)
    iters = 100
    ns = aco_synth.batch_sizes(512, 50, 5000, 4)[:count]
    xys = [aco_synth.uniform(int(n), 4000 + i) for i, n in enumerate(ns)]
    kw = dict(k=20, alpha=1.0, beta=2.0, tau0=1.0, max_mod_frac=1.0, seed=4)
    stream = torch.cuda.Stream()
    b = Batch(xys, m=256, stream=stream, **kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.build_candidates()
    b.run(0, iters + 1, tune=True)
    stream.synchronize()
    t_batch = time.perf_counter() - t0
    (sched, warps, minb, pull), tune_ms = b.schedule()
    best = b.best()
    b.close()
    order = np.argsort(ns)
    ns_sample = per_instance_sample or (args.cpu_sample if args.cpu_sample <= 64 else 24)
    sample = order[np.linspace(0, count - 1, min(ns_sample, count)).astype(int)]
    t_inst = 0.0
    for i in sample:
        n = int(ns[i])
        col = Colony(xys[i], mode=1, n=n, m=min(n, 256), stream=stream, **dict(kw, seed=4 + int(i)))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        col.build_candidates()
        for it in range(iters + 1):
            col.iterate(it)
        stream.synchronize()
        t_inst += time.perf_counter() - t0
        col.close()
    t_inst_all = t_inst * count / len(sample)
    out = {"metric": "instances/s (batched form vs per-instance launches)", "workload": "batch512: 512 instances, n "
           "log-uniform in [50, 5000], uniform cities, k=20, m=min(n,256), f=1, 101 iterations incl. initial tours",
           "batched_instances_per_s": round(count / t_batch, 2), "batched_s": round(t_batch, 3),
           "per_instance_instances_per_s": round(count / t_inst_all, 3),
           "per_instance_s_estimated": round(t_inst_all, 2), "per_instance_sample": int(len(sample)),
           "speedup": round(t_inst_all / t_batch, 1), "schedule": sched,
           "schedule_kind": "persistent launch" if sched >= 8 else "four launches per iteration, CUDA graph",
           "schedule_warps_per_block": warps, "schedule_min_blocks": minb, "schedule_ants_per_pull": pull,
           "tune_ms": [round(float(x), 3) for x in tune_ms], "mean_gbest": float(np.mean(best))}
    if count != 512:
        out["workload"] = out["workload"].replace("512 instances", f"the first {count} of its 512 instances")
    if emit:
        print(json.dumps(out))
    return out


# ------------------------------------------------------------------ learned proposal
def _colony_curve(xy, n, m, k, f, seed, iters, scorer=None, target=None):
    """One colony run: candidate lists, initial tours, (scores,) iterations; C_gbest read after
    every iteration.  Returns (elapsed ms at each iteration, C_gbest at each iteration, ms of
    the scoring step)."""
    import torch

    from paper_1709_03187_gb300 import Colony

    col = Colony(xy, mode=1, n=n, m=m, k=k, max_mod_frac=f, seed=seed)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(iters + 3)]
    torch.cuda.synchronize()
    ev[0].record()
    col.build_candidates()
    col.iterate(0)
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record()
    if scorer is not None:
        scorer.score(col.handle, n, k, 16, beta=2.0)
    s1.record()
    best = [col.stats()["gbest"]]
    ev[1].record()
    for it in range(1, iters):
        col.iterate(it)
        best.append(col.stats()["gbest"])
        ev[it + 1].record()
        if target is not None and best[-1] <= target:
            break
    torch.cuda.synchronize()
    ms = [ev[0].elapsed_time(ev[i + 1]) for i in range(len(best))]
    col.close()
    return ms, best, s0.elapsed_time(s1)


def run_learned(args, seeds=(1, 2, 3), emit=True):
    """Learned proposal against the plain heuristic at n = 20,000 (clustered, 100 clusters,
    sigma = 0.01, k = 20, m = 512, f = 0.1).  Training: plain runs on 2,000 clustered instances of
    n = 1,000 (5 clusters, sigma = 0.01: the evaluation's 200 cities per cluster), m = 32, k = 20,
    f = 1, 40 iterations; labels from each instance's best tour; Adam over minibatches of 2,048
    cities.  The plain arm runs 100 iterations; the learned arm runs until its C_gbest reaches the
    plain arm's final C_gbest (at most 300 iterations).  Both arms read C_gbest after every
    iteration and are timed with CUDA events from candidate lists to that iteration (each arm run
    twice; the faster timing counts).  The learned score is exp(z)^beta with the instance's beta = 2."""
    import torch

    from paper_1709_03187_gb300 import EdgeScorer
    from paper_1709_03187_gb300.learned import training_data

    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    xys = [aco_synth.clustered(1000, 5, 0.01, 10_000 + i) for i in range(2000)]
    t_gen = time.perf_counter() - t0
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record()
    X, T, train_best = training_data(xys, m=32, k=20, iterations=40, max_mod_frac=1.0, seed=11)
    e[1].record()
    sc = EdgeScorer(aco_synth.mlp_weights(1), max_rows=2048 * 20)
    loss = sc.train(X, T, 20, batch_cities=2048, steps=2000, lr=2e-3)
    e[2].record()
    torch.cuda.synchronize()
    loss = loss.cpu().numpy()
    n, m, k, f, iters = 20_000, 512, 20, 0.1, 100
    rows = []
    for s in seeds:
        xy = aco_synth.clustered(n, 100, 0.01, 20_000 + s)
        # each arm twice (the runs are deterministic): the faster timing of each
        runs_p = [_colony_curve(xy, n, m, k, f, s, iters) for _ in range(2)]
        ms_p, best_p, _ = min(runs_p, key=lambda r: r[0][-1])
        runs_l = [_colony_curve(xy, n, m, k, f, s, 3 * iters, scorer=sc, target=best_p[-1]) for _ in range(2)]
        ms_l, best_l, ms_score = min(runs_l, key=lambda r: r[0][-1])
        reached = best_l[-1] <= best_p[-1]
        rows.append(dict(seed=s, plain_len=best_p[-1], plain_ms=ms_p[-1], plain_iters=iters,
                         learned_iters=len(best_l) if reached else None, learned_ms=ms_l[-1] if reached else None,
                         ratio=(ms_l[-1] / ms_p[-1]) if reached else None,
                         score_ms=ms_score,
                         len_at_iter_25=(best_p[24], best_l[24] if len(best_l) > 24 else None)))
    ratios = [r["ratio"] for r in rows]
    out = {"metric": "GPU wall-clock to reach the plain heuristic's mean tour length, learned / plain",
           "value": round(float(np.mean(ratios)), 3) if all(r is not None for r in ratios) else None,
           "unit": "ratio", "higher_is_better": False,
           "workload": "learned20k: n=20,000 clustered (100 clusters, sigma=0.01), k=20, m=512, f=0.1, beta=2, plain "
                       "100 iterations vs learned (score exp(z)^beta) until it reaches the plain final C_gbest; "
                       f"seeds {list(seeds)}",
           "per_seed": rows,
           "training": {"instances": 2000, "n": 1000, "plain_iterations": 40, "m": 32,
                        "plain_ms": round(e[0].elapsed_time(e[1]), 1), "train_ms": round(e[1].elapsed_time(e[2]), 1),
                        "steps": 2000, "batch_cities": 2048, "rows": int(X.shape[0]),
                        "loss_first": float(loss[:20].mean()), "loss_last": float(loss[-20:].mean()),
                        "train_instances_mean_gbest": float(np.mean(train_best)), "generate_s": round(t_gen, 1)}}
    sc.close()
    if emit:
        print(json.dumps(out))
    return out


# ------------------------------------------------------------------ modification schedule
def run_schedule(args):
    """The paper's proposed growing modification limit (Section 7) against a fixed one at
    n = 20,000 (the learned20k instances), m = 512, k = 20: 100 iterations with f = 0.1 fixed,
    100 iterations with f growing linearly from 0.01 to 0.1 over the first 50, and 100 iterations
    at f = 0.1 where an ant rebuilds only part of its l_best with probability 0.95 and builds a
    full tour otherwise (Table 4's setting).  Per seed: the CUDA-event time of the iterations and
    the final C_gbest."""
    import torch

    from paper_1709_03187_gb300 import Colony, linear_f_schedule

    torch.cuda.set_device(0)
    n, m, k, iters = 20_000, 512, 20, 100
    seeds = (1, 2, 3)
    rows = []
    for s in seeds:
        xy = aco_synth.clustered(n, 100, 0.01, 20_000 + s)
        res = {}
        for name, sched, pp in (("fixed", lambda t: 0.1, 1.0), ("growing", linear_f_schedule(0.01, 0.1, 50), 1.0),
                                ("partial95", lambda t: 0.1, 0.95)):
            col = Colony(xy, mode=1, n=n, m=m, k=k, max_mod_frac=0.1, seed=s)
            col.build_candidates()
            col.iterate(0)
            col.set_p_partial(pp)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for it in range(1, iters):
                col.set_max_mod_frac(sched(it))
                col.iterate(it)
            e1.record()
            torch.cuda.synchronize()
            res[name] = (e0.elapsed_time(e1), col.stats()["gbest"])
            col.close()
        rows.append({"seed": s, "fixed_ms": round(res["fixed"][0], 1), "fixed_gbest": res["fixed"][1],
                     "growing_ms": round(res["growing"][0], 1), "growing_gbest": res["growing"][1],
                     "partial95_ms": round(res["partial95"][0], 1), "partial95_gbest": res["partial95"][1]})
    out = {"metric": "C_gbest after 100 iterations and GPU time: growing vs fixed modification limit, and "
                     "p_partial = 0.95 at the fixed limit",
           "workload": "schedule20k: n=20,000 clustered (100 clusters, sigma=0.01), k=20, m=512; f=0.1 fixed vs "
                       "f from 0.01 to 0.1 over 50 iterations vs f=0.1 with p_partial=0.95; 3 seeds",
           "per_seed": rows,
           "mean_fixed_gbest": float(np.mean([r["fixed_gbest"] for r in rows])),
           "mean_growing_gbest": float(np.mean([r["growing_gbest"] for r in rows])),
           "mean_fixed_ms": float(np.mean([r["fixed_ms"] for r in rows])),
           "mean_growing_ms": float(np.mean([r["growing_ms"] for r in rows])),
           "mean_partial95_gbest": float(np.mean([r["partial95_gbest"] for r in rows])),
           "mean_partial95_ms": float(np.mean([r["partial95_ms"] for r in rows]))}
    print(json.dumps(out))


# ------------------------------------------------------------------ local search
def run_ls(args):
    """Windowed 2-opt (Section 3.2, Section 5's setting: probability 0.001 per tour, window 500) on
    the 200,000-city workload (m = 1024, k = 16, f = 0.01), 50 iterations after the initial tours,
    with and without local search: CUDA-event time per iteration, 2-opt moves, final C_gbest."""
    import torch

    from paper_1709_03187_gb300 import Colony

    torch.cuda.set_device(0)
    wl = aco_synth.WORKLOADS["lbest200k"]
    params = dict(wl["params"])
    xy = aco_synth.make("lbest200k")
    res = {}
    for name, p_ls in (("plain", 0.0), ("local_search", 0.001)):
        col = Colony(xy, **params)
        col.build_candidates()
        col.iterate(0)
        col.set_local_search(p_ls, 500)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for it in range(1, 51):
            col.iterate(it)
        e1.record()
        torch.cuda.synchronize()
        st = col.stats()
        res[name] = {"ms_per_iteration": round(e0.elapsed_time(e1) / 50, 4), "gbest": st["gbest"],
                     "ls_moves": int(st["ls_moves"])}
        col.close()
    out = {"metric": "ms per iteration and C_gbest after 50 iterations, windowed 2-opt (p=0.001, W=500) vs none",
           "workload": "ls200k: n=200,000 clustered (200 clusters, sigma=0.005), k=16, m=1024, f=0.01",
           "plain": res["plain"], "local_search": res["local_search"],
           "time_ratio": round(res["local_search"]["ms_per_iteration"] / res["plain"]["ms_per_iteration"], 3)}
    print(json.dumps(out))


# ------------------------------------------------------------------ dense form (Section 2)
def run_dense(args, emit=True):
    """The Section 2 form on its workload (dense100: n = 100 uniform cities, m = 100 ants; Eq. 1
    over every unvisited city, then Eq. 2 and Eq. 3-5 on the n x n matrix): CUDA-event time of the
    construction and of the update per iteration, decisions and iterations per second, the
    construction's roofline (per decision the current city's FP32 weight row, 4 n bytes; per ant
    its tour, 4 n bytes) and the update's (tau read and written, eta^beta read, FP64 and FP32
    weights written: 36 n^2 bytes; tours, successors and predecessors: 12 m n bytes), and the
    oracle's iterations timed on one host core."""
    import torch

    import oracle
    from paper_1709_03187_gb300 import Colony

    torch.cuda.set_device(0)
    params = dict(aco_synth.WORKLOADS["dense100"]["params"])
    xy = aco_synth.make("dense100")
    n, m = params["n"], params["m"]
    col = Colony(xy, **params)
    col.build_candidates()
    for it in range(args.warmup):
        col.iterate(it)
    ev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(args.steps)]
    st0 = col.stats()
    torch.cuda.synchronize()
    for i, (e0, e1, e2) in enumerate(ev):
        e0.record()
        col.construct(args.warmup + i)
        e1.record()
        col.update()
        e2.record()
    torch.cuda.synchronize()
    st = col.stats()
    t_con = sum(a.elapsed_time(b) for a, b, _ in ev) / 1e3
    t_upd = sum(b.elapsed_time(c) for _, b, c in ev) / 1e3
    col.close()
    dec = st["decisions"] - st0["decisions"]
    hbm_peak, peak_kind = read_peaks()
    c_bytes = (dec * 4 * n + m * 4 * n) / args.steps
    u_bytes = 36 * n * n + 12 * m * n
    c_gbs = c_bytes / (t_con / args.steps) / 1e9
    u_gbs = u_bytes / (t_upd / args.steps) / 1e9
    ref = oracle.Oracle(xy, **params)
    ref.reset_counters()
    t0 = time.perf_counter()
    for it in range(3):
        ref.iterate(it)
    t_or = time.perf_counter() - t0
    dec_or = ref.counters()["decisions"]
    out = {"metric": "decisions/s and iterations/s, dense Section 2 form", "workload":
           "dense100: n=100 uniform, m=100, alpha=1, beta=2, rho=0.5, tau0=1 (Eq. 1 over all unvisited; Eq. 2, 3-5)",
           "value": round(dec / (t_con + t_upd), 1), "unit": "decisions/s",
           "iterations_per_s": round(args.steps / (t_con + t_upd), 1), "steps": args.steps, "warmup": args.warmup,
           "ms_construct": round(t_con / args.steps * 1e3, 4), "ms_update": round(t_upd / args.steps * 1e3, 4),
           "roofline": {"bound": "hbm", "peak": hbm_peak, "unit": "GB/s", "peak_source": f"{peak_kind} hbm_gbs",
                        "construct_dense_kernel": {"alg_bytes": c_bytes, "achieved": round(c_gbs, 2),
                                                   "frac": round(c_gbs / hbm_peak, 6)},
                        "update (dense_tau + dense_weights)": {"alg_bytes": u_bytes, "achieved": round(u_gbs, 2),
                                                               "frac": round(u_gbs / hbm_peak, 6)},
                        "note": "the whole state (80 KB tau) is L2-resident; one block per ant and a few "
                                "launches per iteration: launch- and latency-bound"},
           "cpu_baseline": {"value": round(dec_or / t_or, 1), "unit": "decisions/s", "cores": 1,
                            "kind": "oracle", "sample": "3 full iterations of the oracle's own dense colony"}}
    if emit:
        print(json.dumps(out))
    return out


# ------------------------------------------------------------------ Independent Roulette
def run_ir(args):
    """Independent Roulette (the paper's Section 3 selection rule, argmax of tau^alpha eta^beta
    times a uniform draw) against the Eq. 1 wheel on the 200,000-city workload (m = 1024, k = 16,
    f = 0.01): 100 iterations after each colony's initial tours, CUDA-event time per iteration,
    decisions per second and the final C_gbest."""
    import torch

    from paper_1709_03187_gb300 import Colony

    torch.cuda.set_device(0)
    params = dict(aco_synth.WORKLOADS["lbest200k"]["params"])
    xy = aco_synth.make("lbest200k")
    iters = 100
    res = {}
    for name, sel in (("eq1_wheel", 0), ("independent_roulette", 1)):
        col = Colony(xy, selection=sel, **params)
        col.build_candidates()
        col.iterate(0)
        st0 = col.stats()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for it in range(1, iters + 1):
            col.iterate(it)
        e1.record()
        torch.cuda.synchronize()
        st = col.stats()
        ms = e0.elapsed_time(e1)
        res[name] = {"ms_per_iteration": round(ms / iters, 4),
                     "decisions_per_s": round((st["decisions"] - st0["decisions"]) / (ms / 1e3), 1),
                     "initial_gbest": st0["gbest"], "gbest": st["gbest"]}
        col.close()
    out = {"metric": "ms per iteration, decisions/s and C_gbest after 100 iterations, Independent Roulette vs Eq. 1",
           "workload": "ir200k: n=200,000 clustered (200 clusters, sigma=0.005), k=16, m=1024, f=0.01", **res}
    print(json.dumps(out))


# ------------------------------------------------------------------ asynchronous sharing
def run_async(args):
    """Asynchronous l_best sharing (improved partial rebuilds commit inside the construction launch,
    as in the paper's asynchronous CPU colony) against the synchronous iteration on the 200,000-city
    workload (m = 1024, k = 16, f = 0.01): 100 iterations after the same initial tours, CUDA-event
    time per iteration, decisions per second and the final C_gbest.  The asynchronous runs are not
    reproducible, so three are taken."""
    import torch

    from paper_1709_03187_gb300 import Colony

    torch.cuda.set_device(0)
    params = dict(aco_synth.WORKLOADS["lbest200k"]["params"])
    xy = aco_synth.make("lbest200k")
    iters = 100
    res = {}
    for name, on, runs in (("synchronous", False, 1), ("asynchronous", True, 3)):
        out = []
        for _ in range(runs):
            col = Colony(xy, **params)
            col.build_candidates()
            col.iterate(0)
            col.set_async_share(on)
            st0 = col.stats()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for it in range(1, iters + 1):
                col.iterate(it)
            e1.record()
            torch.cuda.synchronize()
            st = col.stats()
            ms = e0.elapsed_time(e1)
            out.append({"ms_per_iteration": round(ms / iters, 4),
                        "decisions_per_s": round((st["decisions"] - st0["decisions"]) / (ms / 1e3), 1),
                        "improved_per_iteration": round((st["improved"] - st0["improved"]) / iters, 1),
                        "gbest": st["gbest"]})
            col.close()
        res[name] = out
    out = {"metric": "ms per iteration, decisions/s and C_gbest after 100 iterations, asynchronous vs synchronous l_best sharing",
           "workload": "async200k: n=200,000 clustered (200 clusters, sigma=0.005), k=16, m=1024, f=0.01",
           "synchronous": res["synchronous"][0], "asynchronous": res["asynchronous"]}
    print(json.dumps(out))


def main():
    args = parse_args()
    if args.workload == "async200k" and args.impl == "ours":
        run_async(args)
        return
    if args.workload == "dense100" and args.impl == "ours":
        run_dense(args)
        return
    if args.workload == "ir200k" and args.impl == "ours":
        run_ir(args)
        return
    if args.workload == "ls200k" and args.impl == "ours":
        run_ls(args)
        return
    if args.workload == "schedule20k" and args.impl == "ours":
        run_schedule(args)
        return
    if args.workload == "batch512" and args.impl == "ours":
        run_batch(args)
    elif args.workload == "learned20k" and args.impl == "ours":
        run_learned(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
