"""Benchmark: frames relocalised per second at 640x480 (paper-shaped query:
5 trees of depth 15, 1024 hypotheses, 500-pixel batches halving to one, LM,
depth-residual ranking of the last 16), with p50/p99 latency batched and
per-frame.

One JSON line on rank 0.  A step relocalises one batch of --batch frames
whose inputs are already resident in device memory; L2 is flushed before
every timed step (a 256 MB write) and each step is timed with CUDA events on
the stream the library launches on.  `e2e` times the same work through the
C ABI from pinned host buffers, host<->device copies included.  Multi-GPU
runs are independent replicas (queries shard with no exchange): every rank
relocalises its own batches and `value` counts all ranks' frames over the
slowest rank's time.

--impl reference times the CPU oracle on the host cores, one query per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import workloads  # noqa: E402

METRIC = "frames relocalised/s at 640x480"
UNIT = "frames/s"
FP32_LANES_PER_SM = 128
F_REF = 585.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--train-frames", type=int, default=None)
    ap.add_argument("--cpu-sample", type=int, default=4, help="oracle queries in the CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving", action="store_true",
                    help="serving workload (3 rooms, 8 streams, cascade): latency and saturation sweep")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="length of the 30 Hz serving run")
    ap.add_argument("--sweep-seconds", type=float, default=4.0, help="length of each saturation point")
    ap.add_argument("--no-serving-leg", action="store_true",
                    help="skip the short serving leg (batched vs per-frame) of the default line")
    ap.add_argument("--leg-seconds", type=float, default=2.0, help="length of each serving-leg point")
    ap.add_argument("--profile-only", action="store_true",
                    help="short run for an external profiler (no baselines)")
    ap.add_argument("--streams", type=int, default=0,
                    help="sub-batches of each call on concurrent streams (1, 2, 4 or 8; default: autotuned); "
                         "1 gives an external profiler the launch sequence of the per-kernel profiled pass")
    ap.add_argument("--arena-gb", type=float, default=24.0,
                    help="device memory handed to the library (smaller for profiler captures)")
    ap.add_argument("--robustness", action="store_true",
                    help="success vs missing depth and depth-dependent noise (training and queries corrupted), "
                         "without and with ICP")
    ap.add_argument("--robust-queries", type=int, default=64)
    ap.add_argument("--tracking-loss", action="store_true",
                    help="tracking-loss recovery along a fresh trajectory from empty leaves")
    ap.add_argument("--track-frames", type=int, default=120)
    ap.add_argument("--track-depth", type=int, default=15,
                    help="tree depth of the tracking-loss forest (13: 5 x 8192 = 40,960 leaves)")
    ap.add_argument("--track-leaves", default="256,8192,65536",
                    help="leaves re-clustered per frame, one arm each (comma separated)")
    ap.add_argument("--rqs-leaves", type=int, default=0,
                    help="time Really Quick Shift on this many leaves of the trained config-2 forest")
    ap.add_argument("--streaming", action="store_true",
                    help="relocalisation throughput with adaptation running on a second stream")
    ap.add_argument("--icp-poses", type=int, default=0,
                    help="standalone ICP: refine this many poses against one 640x480 frame "
                         "(1 GB of device memory; the small case for profiling the ICP kernel)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def replica_seeds(rank, step, batch):
    """Seeds of one step's queries on one replica: disjoint across ranks
    (high bits) and steps."""
    return [(rank << 40) + (step + 1) * batch + i for i in range(batch)]


def max_over_ranks(x, device):
    """Largest value over the ranks: the slowest replica sets the job's time."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(frames_per_rank, world, seconds):
    """Whole-job frames/s: every rank's frames over the slowest rank's time."""
    return frames_per_rank * world / seconds


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def training_set(w, n):
    frames = []
    for i, fr in enumerate(w.training_frames()):
        if i >= n:
            break
        frames.append(fr)
    return frames


# --------------------------------------------------------------------------- oracle
def oracle_model(w, frames):
    import oracle
    f = w.forest
    nodes = oracle.forest_random(f["n_trees"], f["depth"], f["p_depth"], (f["delta_lo"], f["delta_hi"]),
                                 (f["tau_depth_lo"], f["tau_depth_hi"]), (f["tau_rgb_lo"], f["tau_rgb_hi"]),
                                 bool(f["tau_zero"]), w.forest_seed)
    res = oracle.Reservoirs(nodes, f["kappa"], w.forest_seed)
    for d, c, T in frames:
        res.add_frame(d, c, w.K, T, f["grid_step"], f["grid_origin"])
    modes = oracle.Modes(res.n_leaves, f["m_max"])
    oracle.update_modes(res, modes, f["sigma"], f["tau_c"], f["min_cluster_size"],
                        cov_eps=f["cov_eps"], fp16_offsets=bool(f["mode_precision"]))
    return nodes, modes


def oracle_step(w, nodes, modes, q):
    import oracle
    d, c, T, seed = q
    lv = oracle.forest_leaves(nodes, d, c, w.K.fx, n_trees=w.ransac["n_trees_used"])
    return oracle.relocalise(w.ransac, d, c, w.K, lv, modes, w.room().lo, w.room().hi, seed,
                             1 << w.forest["depth"])



def cpu_model_name():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


# Oracle workers for the all-cores baseline: spawned processes (the parent
# already holds a CUDA context), each running the single-threaded oracle on
# whole queries.
_ORACLE_MODEL = None


def _oracle_worker_init(path):
    global _ORACLE_MODEL
    import pickle
    import oracle
    oracle.set_threads(1)
    with open(path, "rb") as f:
        _ORACLE_MODEL = pickle.load(f)


def _oracle_worker_idle(_):
    time.sleep(0.2)
    return os.getpid()


def _oracle_worker_run(q):
    w, nodes, modes = _ORACLE_MODEL
    oracle_step(w, nodes, modes, q)
    return 1


def oracle_all_cores(w, nodes, modes, queries):
    """Wall-clock frames/s of the oracle on every host core: one single-threaded
    oracle per core, queries spread over them."""
    import multiprocessing
    import pickle
    ncores = os.cpu_count() or 1
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "model.pkl")
        with open(path, "wb") as f:
            pickle.dump((w, nodes, modes), f, protocol=pickle.HIGHEST_PROTOCOL)
        ctx = multiprocessing.get_context("spawn")
        with ctx.Pool(ncores, initializer=_oracle_worker_init, initargs=(path,)) as pool:
            pool.map(_oracle_worker_idle, range(2 * ncores), chunksize=1)
            t0 = time.perf_counter()
            pool.map(_oracle_worker_run, queries, chunksize=1)
            dt = time.perf_counter() - t0
    return len(queries) / dt, ncores, dt


def pose_err(A, B):
    A = np.asarray(A, np.float64).reshape(4, 4)
    B = np.asarray(B, np.float64).reshape(4, 4)
    dt = float(np.linalg.norm(A[:3, 3] - B[:3, 3]))
    c = (np.trace(A[:3, :3].T @ B[:3, :3]) - 1.0) / 2.0
    return dt, float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))


def oracle_threads():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    w = workloads.CONFIG2
    frames = training_set(w, args.train_frames or w.n_train)
    nodes, modes = oracle_model(w, frames)
    oracle.set_threads(1)  # one core, as the line states
    qs = w.queries(max(1, min(8, args.steps + args.warmup)))
    for i in range(args.warmup):
        oracle_step(w, nodes, modes, qs[i % len(qs)])
    times = []
    for i in range(args.steps):
        t = time.perf_counter()
        oracle_step(w, nodes, modes, qs[(args.warmup + i) % len(qs)])
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = args.steps / total
    sample = f"{args.steps} config-2 queries (640x480, 5 trees d15, 1024 hypotheses), one per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w.name, "global_batch": 1, "seq_len": 640 * 480,
                                        "parallelism": "replicas"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "cpu": cpu_model_name()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- roofline
def algorithmic_flops(kernel, work, p):
    """Algorithmic FP32 work of one kernel, from its counted work units.
    Energy (Eq. 5): 20 flops per (H, pixel) (transform 18, sqrt + add 2) and
    per (H, pixel, mode) 18 with the Mahalanobis factor (3 sub, U v 9,
    squared norm 5, min 1) or 9 Euclidean.  LM: pass 1 as the energy per
    (H, pixel, mode) plus 18 per (H, pixel) transform and 190 per inlier
    (J rows 12, J^T J 126, J^T r 36, cost 6, residual 10); trial pass 34 per
    inlier.  Raycast: 45 per ray.  ICP: 50 per valid-pixel evaluation in the
    face-binned world-frame form (camera ray 4, rotation 12, exit face 6,
    gap and inlier test 9, rotated point and residual 4, nine normal-equation
    terms 15)."""
    per_mode = 18 if p["use_cov"] else 9
    if kernel == "energy":
        return 20 * work["energy_pairs"] + per_mode * work["energy_modes"]
    if kernel == "lm":
        return (18 * work["lm_pairs"] + per_mode * work["lm_modes"] + 190 * work["lm_inliers"]
                + 34 * work["lm_trial"])
    if kernel == "raycast_score":
        return 45 * work["rays"]
    if kernel == "icp":
        return 50 * work["icp_pixels"]
    return None


# Hypothesis generation is integer work: per stage-1 attempt two Philox4x32-10
# blocks (10 rounds of two 32x32->64 products = 4 ops, 4 xor, 2 key adds:
# 100 ops each) and 3 multiply-shift draws, 3 mask loads and a bit test
# (10 ops): 210; per stage-2 evaluation 150 (3 record decodes 30, 3 mode
# positions 12, spread 3 x 8, 3 back-projections 3 x 12, rigidity 3 x 16).
HYP_OPS_ATTEMPT, HYP_OPS_STAGE2 = 210, 150


def algorithmic_int_ops(kernel, work):
    if kernel == "hypgen":
        return HYP_OPS_ATTEMPT * work["hyp_attempts"] + HYP_OPS_STAGE2 * work["hyp_stage2"]
    return None


# DRAM traffic (read + write) of a kernel from one ncu capture, per frame
# and launch (profiles/launches_relocalise_config2_b64.md: mean over the six
# rounds of a 32-frame call), valid only for the source it was measured on:
# when the file's hash differs, traffic is reported as null.
PROFILED_TRAFFIC = {
    "lm": {"bytes_per_frame_launch": 5.26e6, "source": "paper_1810_12163_gb300/csrc/lm.cu",
           "sha256_16": "61b14d376512a1d7"},
}


def profiled_traffic(kernel, frames):
    e = PROFILED_TRAFFIC.get(kernel)
    if not e:
        return None
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), e["source"])
    with open(path, "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()[:16]
    return e["bytes_per_frame_launch"] * frames if h == e["sha256_16"] else None


def roofline(kernels, work, p, n_frames_profiled, w, sm_count, pk, batch=1):
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    kd = kernels[dom]
    fp32_peak = sm_count * FP32_LANES_PER_SM * 2 * (pk.get("sm_max_mhz", 2070.0) if pk else 2070.0) * 1e6 / 1e12
    flops = algorithmic_flops(dom, work, p)
    avg_s = kd["ms"] / 1e3 / max(1, kd["launches"])
    out = {"kernel": dom, "avg_launch_ms": kd["ms"] / max(1, kd["launches"]), "launches": kd["launches"]}
    if flops is not None:
        ach = flops / max(1, kd["launches"]) / avg_s / 1e12
        out.update({"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": ach / fp32_peak, "traffic": profiled_traffic(dom, batch),
                    "peak_source": f"derived: {sm_count} SMs x 128 FP32 lanes x 2 x max SM clock"})
    elif dom == "leaves":
        bpf = w.width * w.height * (4 + 3 + 2 * p["n_trees_used"])
        ach = bpf * n_frames_profiled / max(1, kd["launches"]) / avg_s / 1e9
        hp = pk["hbm_gbs"] if pk else 6800.0
        out.update({"bound": "hbm", "achieved": ach, "peak": hp, "unit": "GB/s", "frac": ach / hp,
                    "traffic": None, "peak_source": "MEASURED_PEAKS.json hbm_gbs" if pk else "fallback"})
    elif algorithmic_int_ops(dom, work) is not None:
        ops = algorithmic_int_ops(dom, work)
        int_peak = fp32_peak / 2  # one 32-bit integer op per lane per clock
        ach = ops / max(1, kd["launches"]) / avg_s / 1e12
        out.update({"bound": "alu", "achieved": ach, "peak": int_peak, "unit": "Tops/s",
                    "frac": ach / int_peak, "traffic": None,
                    "peak_source": f"derived: {sm_count} SMs x 128 INT32 lanes x max SM clock"})
    else:
        out.update({"bound": "alu", "achieved": None, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": None, "traffic": None})
    return out


# Forest walk (Eq. 1-3): per pixel with depth, 4 B of depth, 3 B of colour
# and 2 B of leaf index per tree are the algorithmic HBM bytes; each node test
# is about 8 FP32 operations (offset scale, probe rounding, feature, compare).
LEAF_OPS_PER_TEST = 8


def leaves_roofline(kernels, n_frames, w, pk, fp32_peak):
    kd = kernels.get("leaves")
    if not kd or kd["ms"] <= 0:
        return None
    s = kd["ms"] / 1e3
    px = n_frames * w.width * w.height
    T, depth = w.ransac["n_trees_used"], w.forest["depth"]
    hbm = (pk["hbm_gbs"] if pk else 6800.0)
    bytes_ = px * (4 + 3 + 2 * T)
    flops = px * T * depth * LEAF_OPS_PER_TEST
    return {"hbm": {"achieved": bytes_ / s / 1e9, "unit": "GB/s", "frac": bytes_ / s / 1e9 / hbm},
            "fp32": {"achieved": flops / s / 1e12, "unit": "TFLOP/s", "frac": flops / s / 1e12 / fp32_peak},
            "note": "a gather-latency kernel: neither fraction is its bound"}


def kernel_rooflines(kernels, work, p, sm_count, pk, n_frames=None, w=None, accepted=None):
    """Achieved fraction of each kernel with an algorithmic work model."""
    fp32_peak = sm_count * FP32_LANES_PER_SM * 2 * (pk.get("sm_max_mhz", 2070.0) if pk else 2070.0) * 1e6 / 1e12
    out = {}
    if n_frames and w is not None:
        lr = leaves_roofline(kernels, n_frames, w, pk, fp32_peak)
        if lr:
            out["leaves"] = lr
    for k, kd in kernels.items():
        if not kd["launches"] or kd["ms"] <= 0:
            continue
        s = kd["ms"] / 1e3
        f = algorithmic_flops(k, work, p)
        if f is not None:
            out[k] = {"achieved": f / s / 1e12, "unit": "TFLOP/s", "frac": f / s / 1e12 / fp32_peak}
            continue
        o = algorithmic_int_ops(k, work)
        if o is not None:
            out[k] = {"achieved": o / s / 1e12, "unit": "Tops/s", "frac": o / s / 1e12 / (fp32_peak / 2)}
            if k == "hypgen":
                out[k]["attempts_per_s"] = work["hyp_attempts"] / s
                if accepted is not None:
                    out[k]["accepted_per_s"] = accepted / s
    return out


def end_to_end_roofline(work, p, frames, seconds, sm_count, pk):
    """FP32 work of the scoring kernels per frame (energy, LM, raycast; the
    models of algorithmic_flops) against the FP32 peak: the frames/s the
    device would reach if those flops ran at peak, and the fraction of it
    achieved.  Generation is integer work and the forest walk a gather, both
    outside this figure."""
    fp32_peak = sm_count * FP32_LANES_PER_SM * 2 * (pk.get("sm_max_mhz", 2070.0) if pk else 2070.0) * 1e6
    flops = sum(algorithmic_flops(k, work, p) or 0.0 for k in ("energy", "lm", "raycast_score"))
    per_frame = flops / frames
    roof = fp32_peak / per_frame
    achieved = frames / seconds
    return {"flops_per_frame": per_frame, "roofline_frames_per_s": roof, "achieved_frames_per_s": achieved,
            "frac": achieved / roof}


def _success(P, T):
    P = np.asarray(P).reshape(4, 4)
    dt, dr = pose_err(P, T)
    return dt <= 0.05 and dr <= 5.0


def run_icp_variant(rg, forest, scene, w, D, C, B, qs, stream, seeds, args, sm_count, pk, tuning):
    """The same workload with ICP before ranking (Sec. 3.2.4): throughput,
    the ICP kernel's share and roofline, and the 5 cm / 5 deg success rate
    with and without ICP on the same distinct queries and seeds."""
    import torch
    p = dict(w.ransac, **workloads.ICP_ON)
    rel = rg.Relocaliser(forest, scene, p, w.width, w.height, B)
    rel.set_tuning(tuning)
    for k in range(2):
        rel.relocalise_batch(D, C, w.K, seeds(600_000 + k), stream=stream, raw=True)
    torch.cuda.synchronize()
    steps = max(3, args.steps // 2)
    rel.profile(True)
    ms = []
    for k in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rel.relocalise_batch(D, C, w.K, seeds(k), stream=stream, raw=True)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    kernels, work = rel.profile_read()
    rel.profile(False)
    # success with and without ICP over the distinct queries, same seeds
    n = len(qs)
    Dq = D[:n]
    Cq = C[:n]
    sd = [q[3] for q in qs]
    with_icp = rel.relocalise_batch(Dq, Cq, w.K, sd, stream=stream)
    rel0 = rg.Relocaliser(forest, scene, w.ransac, w.width, w.height, B)
    without = rel0.relocalise_batch(Dq, Cq, w.K, sd, stream=stream)
    rel0.close()
    rel.close()
    err = lambda rs: [pose_err(r["pose"], q[2]) for r, q in zip(rs, qs)]
    e1, e0 = np.array(err(with_icp)), np.array(err(without))
    kr = kernel_rooflines(kernels, work, p, sm_count, pk)
    return {
        "frames_per_s": B * steps / (sum(ms) / 1e3), "ms_per_step": float(np.mean(ms)),
        "icp_ms_per_step": kernels["icp"]["ms"] / steps, "icp_roofline": kr.get("icp"),
        "icp_pixel_evals_per_step": work["icp_pixels"] // steps,
        "queries": n,
        "success_5cm_5deg": {"icp": float(np.mean([_success(r["pose"], q[2]) for r, q in zip(with_icp, qs)])),
                             "no_icp": float(np.mean([_success(r["pose"], q[2]) for r, q in zip(without, qs)]))},
        "median_error": {"icp": [float(np.median(e1[:, 0])), float(np.median(e1[:, 1]))],
                         "no_icp": [float(np.median(e0[:, 0])), float(np.median(e0[:, 1]))],
                         "unit": ["m", "deg"]},
        "icp_success_fraction": float(np.mean([bin(r["icp_mask"]).count("1") / max(1, r["n_chosen"])
                                               for r in with_icp])),
        "params": {k: (list(v) if isinstance(v, tuple) else v) for k, v in workloads.ICP_ON.items()},
    }


# --------------------------------------------------------------------------- ours
def run_cascade_variant(rg, forest, scene, w, D, C, B, truth, stream, seeds, args, flush):
    """Config 3: the three-level cascade (160x120 / 64 hypotheses / 1 tree,
    320x240 / 256 / 5 trees, 640x480 / 1024 / 5 trees; thresholds drawn by
    seed 7) over the same forest and the same 64 device-resident frames,
    every level of every frame in one captured CUDA graph per batch size."""
    import torch
    levels = [rg.Relocaliser(forest, scene, p, w.width // s, w.height // s, B) for s, p in workloads.CASCADE_LEVELS]
    cas = rg.Cascade(levels, workloads.cascade_thresholds(), [s for s, _ in workloads.CASCADE_LEVELS])
    for k in range(args.warmup):
        cas.relocalise_batch(D, C, w.K, seeds(700_000 + k), stream=stream)
    torch.cuda.synchronize()
    ms, res = [], None
    for k in range(args.steps):
        flush.fill_(k & 255)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = cas.relocalise_batch(D, C, w.K, seeds(k), stream=stream)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    cas.close()
    for lv in levels:
        lv.close()
    lv_used = [int(r["level"]) for r in res]
    return {"frames_per_s": 1000.0 * B / float(np.mean(ms)), "ms_per_step": float(np.mean(ms)), "batch": B,
            "levels_used": {str(l): lv_used.count(l) for l in range(len(workloads.CASCADE_LEVELS))},
            "thresholds_m": workloads.cascade_thresholds(),
            "success_5cm_5deg": float(np.mean([_success(r["pose"], t) for r, t in zip(res, truth)])),
            "timed_path": "CUDA graph replay of all levels"}


def run_ours(args):
    import torch
    import paper_1810_12163_gb300 as rg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = workloads.CONFIG2
    B = args.batch
    pk = peaks()
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count

    n_train = args.train_frames or w.n_train
    frames = training_set(w, n_train)
    ctx = rg.Context(local, arena_bytes=int(args.arena_gb * (1 << 30)))
    forest = rg.Forest.random(ctx, w.forest, w.forest_seed)
    for d, c, T in frames:
        forest.adapt(d, c, w.K, T)
    forest.update_modes(-1)
    scene = rg.Scene(ctx, w.room().lo, w.room().hi)
    rel = rg.Relocaliser(forest, scene, w.ransac, w.width, w.height, B)

    # distinct query frames for this rank, resident in device memory
    n_distinct = B
    qs = [w.query(rank * 1000 + i) for i in range(n_distinct)]
    D = torch.from_numpy(np.stack([qs[i % n_distinct][0] for i in range(B)])).cuda()
    C = torch.from_numpy(np.stack([qs[i % n_distinct][1] for i in range(B)])).cuda()
    truth = [qs[i % n_distinct][2] for i in range(B)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def seeds(step):
        return replica_seeds(rank, step, B)

    # launch shapes picked by the autotuner on this workload (results do not depend on them)
    tuning = rel.autotune(D, C, w.K, seeds(900_000), stream=stream)
    if args.streams:
        rel.set_tuning(dict(streams=args.streams))
        tuning = rel.tuning
    for k in range(args.warmup):
        rel.relocalise_batch(D, C, w.K, seeds(500_000 + k), stream=stream, raw=True)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()

    # the timed region: the product path (each step replays the captured
    # CUDA graph of the 64-frame launch sequence)
    step_ms = []
    results = None
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(k & 255)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            torch.cuda.nvtx.range_push("timed_step")  # lets an external profiler select these launches
            results = rel.relocalise_batch(D, C, w.K, seeds(k), stream=stream, raw=True)
            torch.cuda.nvtx.range_pop()
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
    total_s = sum(step_ms) / 1e3
    graph_kernels = rel.graph_kernels(B)  # kernels each timed step replayed
    # a profiled pass of the same steps (same seeds, so the same work):
    # kernels launched one by one with CUDA events around each launch and
    # work counters on the device; the per-kernel rooflines come from it
    rel.profile(True)
    prof_ms = []
    for k in range(args.steps):
        flush.fill_(k & 255)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rel.relocalise_batch(D, C, w.K, seeds(k), stream=stream, raw=True)
        e1.record(stream)
        e1.synchronize()
        prof_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    kernels, work = rel.profile_read()
    rel.profile(False)
    if world > 1:
        torch.distributed.barrier()
    total_s = max_over_ranks(total_s, "cuda")
    value = job_throughput(B * args.steps, world, total_s)

    # accuracy of the last step's poses (5 cm / 5 deg)
    ok = 0
    for i in range(B):
        P = np.array(results[i].pose).reshape(4, 4)
        dt = np.linalg.norm(P[:3, 3] - truth[i][:3, 3])
        ang = math.degrees(math.acos(max(-1, min(1, (np.trace(P[:3, :3].T @ truth[i][:3, :3]) - 1) / 2))))
        ok += dt <= 0.05 and ang <= 5.0

    # end to end through the C ABI from pinned host memory
    Dh = torch.empty(D.shape, dtype=torch.float32, pin_memory=True)
    Ch = torch.empty(C.shape, dtype=torch.uint8, pin_memory=True)
    Dh.copy_(D)
    Ch.copy_(C)
    Dn, Cn = Dh.numpy(), Ch.numpy()
    e2e_steps = max(3, args.steps // 2)
    rel.relocalise_batch(Dn, Cn, w.K, seeds(10_000), stream=stream, raw=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        rel.relocalise_batch(Dn, Cn, w.K, seeds(20_000 + k), stream=stream, raw=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, "cuda")
    h2d = int(Dn.nbytes + Cn.nbytes)
    d2h = B * (128 + 16 * 12 * 8 + 3 * 16 * 4)

    # per-frame latency (batch of one) vs batched step latency
    rel1 = rg.Relocaliser(forest, scene, w.ransac, w.width, w.height, 1)
    lat1 = []
    for i in range(max(8, min(32, args.steps * 2))):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rel1.relocalise_batch(D[i % B: i % B + 1], C[i % B: i % B + 1], w.K, [77_000 + i], stream=stream, raw=True)
        e1.record(stream)
        e1.synchronize()
        lat1.append(e0.elapsed_time(e1))
    lat1 = lat1[2:]

    icp = None if args.profile_only else run_icp_variant(rg, forest, scene, w, D, C, B, qs, stream, seeds, args,
                                                          sm_count, pk, tuning)
    cascade = None if args.profile_only else run_cascade_variant(rg, forest, scene, w, D, C, B, truth, stream,
                                                                 seeds, args, flush)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "fp32",
        "data": "synthetic (seeded textured box room, 200 posed training frames)",
        "config": {"workload": w.name, "global_batch": B * world, "seq_len": w.width * w.height,
                   "parallelism": f"replicas x{world}", "n_hyp": w.ransac["n_hyp"],
                   "eta": w.ransac["eta"], "k_out": w.ransac["k_out"],
                   "l2": "flushed before every timed step (256 MB write)", "tuning": tuning},
        "latency_ms": {
            "batched": {"batch": B, "p50": float(np.percentile(step_ms, 50)),
                        "p99": float(np.percentile(step_ms, 99))},
            "per_frame": {"p50": float(np.percentile(lat1, 50)), "p99": float(np.percentile(lat1, 99)),
                          "frames_per_s": 1000.0 / float(np.mean(lat1))},
        },
        "success_5cm_5deg": ok / B,
        "e2e": {"value": job_throughput(B * e2e_steps, world, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(graph_kernels * args.steps) if graph_kernels > 0 else None,
        "gpu_launches_per_step": {"graph_kernel_nodes": graph_kernels,
                                  "profiled_pass": int(sum(k["launches"] for k in kernels.values())) // args.steps},
        "timed_path": "CUDA graph replay (one graph per batch size); per-kernel figures from a "
                      "profiled pass of the same steps launched kernel by kernel",
        "profiled_pass_ms_per_step": float(np.mean(prof_ms)),
        "kernels_ms": {k: round(v["ms"], 4) for k, v in kernels.items()},
        "roofline": roofline(kernels, work, w.ransac, B * args.steps, w, sm_count, pk, batch=B),
        "kernel_rooflines": kernel_rooflines(kernels, work, w.ransac, sm_count, pk, n_frames=B * args.steps, w=w,
                                             accepted=args.steps * sum(int(r.n_hypotheses) for r in results)),
        "roofline_end_to_end": end_to_end_roofline(work, w.ransac, B * args.steps, total_s, sm_count, pk),
        "work_per_step": {k: v // max(1, args.steps) for k, v in work.items()},
        "clocks": clk.summary(),
        "icp_variant": icp,
        "cascade_config3": cascade,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.profile_only:
        import oracle
        nodes, modes = oracle_model(w, frames)
        oq = [w.query(i) for i in range(args.cpu_sample)]
        oracle.set_threads(1)
        t0 = time.perf_counter()
        ores = [oracle_step(w, nodes, modes, q) for q in oq]
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": len(oq) / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{len(oq)} config-2 queries relocalised one at a time "
                                          f"(one thread, {dt:.1f} s)", "cpu": cpu_model_name()}
        # the oracle on every host core, one query per process at a time
        allq = [w.query(i) for i in range(2 * (os.cpu_count() or 1))]
        v, ncores, dta = oracle_all_cores(w, nodes, modes, allq)
        line["cpu_baseline_all_cores"] = {
            "value": v, "unit": UNIT, "cores": ncores, "kind": "oracle", "cpu": cpu_model_name(),
            "sample": f"{len(allq)} config-2 queries, {ncores} single-threaded oracle processes ({dta:.1f} s)"}
        # error of the GPU results against the FP64 oracle on the same queries and seeds
        Dq = torch.from_numpy(np.stack([q[0] for q in oq])).cuda()
        Cq = torch.from_numpy(np.stack([q[1] for q in oq])).cuda()
        gres = rel.relocalise_batch(Dq, Cq, w.K, [q[3] for q in oq], stream=stream)
        torch.cuda.synchronize()
        errs = []
        for g, o in zip(gres, ores):
            dtp, drp = pose_err(g["pose"], o["pose"])
            e_rel = abs(g["energy"] - o["energy"]) / max(abs(o["energy"]), 1e-30)
            s_rel = (abs(g["score"] - o["score"]) / max(abs(o["score"]), 1e-30)
                     if np.isfinite(o["score"]) and np.isfinite(g["score"]) else 0.0)
            errs.append((dtp, drp, e_rel, s_rel))
        e = np.array(errs)
        line["oracle_error"] = {
            "queries": len(errs), "max_pose_m": float(e[:, 0].max()), "max_pose_deg": float(e[:, 1].max()),
            "max_energy_rel": float(e[:, 2].max()), "max_score_rel": float(e[:, 3].max()),
            "within_1mm_0.05deg": int(((e[:, 0] <= 1e-3) & (e[:, 1] <= 0.05)).sum())}
    line["arena_peak_gb"] = ctx.usage()[1] / (1 << 30)
    if rank == 0 and world == 1 and not args.no_serving_leg and not args.profile_only:
        sctx = rg.Context(local, arena_bytes=32 << 30)
        line["serving"] = serving_leg(rg, sctx, args.leg_seconds)
        sctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    rel1.close()
    rel.close()
    if world > 1:
        torch.distributed.destroy_process_group()


# --------------------------------------------------------------------------- serving
def _render_training(args):
    w, i = args
    from synth.rooms import render, training_trajectory
    room = w.room()
    T = training_trajectory(room, w.n_train)[i]
    d, c = render(room, w.K, T, w.noise_sigma, noise_seed=100 + i)
    return d, c, T


def _serving_pools(per_stream=8):
    """Pre-rendered queries per stream: (depth, rgb, K, truth, seed)."""
    from synth import rooms
    pools = []
    for s in range(workloads.SERVING_STREAMS):
        w = workloads.SERVING_ROOMS[s % 3]
        pool = []
        for k in range(per_stream):
            d, c, T, seed = w.query(100 * s + k)
            if s % 2:
                d, c, K = rooms.subsample(d, c, w.K, 2)
            else:
                K = w.K
            pool.append((d, c, K, T, seed))
        pools.append(pool)
    return pools


def _serve(srv, models, pools, arrivals):
    """Replays the arrivals in real time (one submitting thread per stream),
    releases every ticket, and returns the server's statistics plus the
    success rate of the served poses."""
    import queue
    streams = workloads.SERVING_STREAMS
    per = [[t for t, s in arrivals if s == k] for k in range(streams)]
    done_q = queue.Queue()
    ok = [0]
    served = [0]

    def collector():
        while True:
            item = done_q.get()
            if item is None:
                return
            ticket, truth = item
            r = srv.wait(ticket, 600_000)
            served[0] += 1
            dt, dr = pose_err(r["pose"], truth)
            ok[0] += int(dt <= 0.05 and dr <= 5.0)

    col = threading.Thread(target=collector)
    col.start()
    t0 = time.perf_counter() + 0.05

    def submitter(k):
        pool = pools[k]
        for n, t in enumerate(per[k]):
            delay = t0 + t - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            d, c, K, T, seed = pool[n % len(pool)]
            done_q.put((srv.submit(models[k % 3], d, c, K, seed + 7919 * n), T))

    subs = [threading.Thread(target=submitter, args=(k,)) for k in range(streams)]
    for th in subs:
        th.start()
    for th in subs:
        th.join()
    submit_s = time.perf_counter() - t0
    done_q.put(None)
    col.join()
    st = srv.stats()
    st["success_5cm_5deg"] = ok[0] / max(1, served[0])
    st["offered_per_s"] = len(arrivals) / (arrivals[-1][0] if arrivals else 1.0)
    st["submitted_per_s"] = len(arrivals) / max(submit_s, 1e-9)
    return st


class ServingBench:
    """Config 4: three rooms, each with its own five-tree forest trained on
    its 200-frame trajectory, served through the library's serving loop
    with the config-3 cascade per room."""

    def __init__(self, rg, ctx):
        import multiprocessing
        self.rg, self.ctx = rg, ctx
        forests, scenes = [], []
        mp = multiprocessing.get_context("spawn")
        with mp.Pool(min(16, os.cpu_count() or 1)) as pool:
            for w in workloads.SERVING_ROOMS:
                f = rg.Forest.random(ctx, w.forest, w.forest_seed)
                for d, c, T in pool.map(_render_training, [(w, i) for i in range(w.n_train)], chunksize=4):
                    f.adapt(d, c, w.K, T)
                f.update_modes(-1)
                forests.append(f)
                scenes.append(rg.Scene(ctx, w.room().lo, w.room().hi))
        self.forests, self.scenes = forests, scenes
        self.pools = _serving_pools()

    def make_server(self, max_batch):
        srv = self.rg.Server(self.ctx, max_batch=max_batch, memory_budget=2 << 30)
        subsample = [s for s, _ in workloads.CASCADE_LEVELS]
        levels = [p for _, p in workloads.CASCADE_LEVELS]
        thresholds = workloads.cascade_thresholds()
        models = [srv.add_cascade_model(self.forests[r], self.scenes[r], levels, subsample, thresholds, 640, 480)
                  for r in range(3)]
        # warm the graphs of every batch size the run can form
        d, c, K, T, seed = self.pools[0][0]
        for n in range(1, max_batch + 1):
            ts = [srv.submit(models[0], d, c, K, seed + i) for i in range(n)]
            for t in ts:
                srv.wait(t, 600_000)
        return srv, models

    def point(self, max_batch, seconds, scale):
        srv, models = self.make_server(max_batch)
        srv.reset_stats()
        st = _serve(srv, models, self.pools, workloads.serving_arrivals(seconds, scale))
        srv.close()
        keys = ("p50_ms", "p99_ms", "mean_ms", "frames_per_s", "success_5cm_5deg", "offered_per_s",
                "submitted_per_s", "refused")
        out = {k: st[k] for k in keys}
        out["completed"] = st["completed"]
        out["rate_scale"] = scale
        return out

    def close(self):
        for s in self.scenes:
            s.close()
        for f in self.forests:
            f.close()


def serving_leg(rg, ctx, seconds):
    """Short serving run for the default line: the config-4 load at x8 and
    x32 the 30 Hz rate, continuous batching (<= 16 frames) vs per-frame."""
    sb = ServingBench(rg, ctx)
    out = {"workload": "3 rooms, 8 streams (even 640x480, odd 320x240), Poisson arrivals, 3-level cascade",
           "seconds_per_point": seconds}
    for scale in (8, 32):
        out[f"x{scale}"] = {"batched_max16": sb.point(16, seconds, scale), "per_frame": sb.point(1, seconds, scale)}
    sb.close()
    return out


def run_serving(args):
    import torch
    import paper_1810_12163_gb300 as rg
    torch.cuda.set_device(0)
    ctx = rg.Context(0, arena_bytes=32 << 30)
    sb = ServingBench(rg, ctx)
    run_point = sb.point
    # three rooms, each with its own forest trained on its 200-frame trajectory
    line = {"impl": "ours", "metric": "serving: frames relocalised/s with p50/p99 latency",
            "workload": "3 rooms (4x3x2.5, 6x5x3, 10x8x3 m), 5-tree d15 forest each, 8 streams "
                        "(even 640x480, odd 320x240), Poisson 30 Hz per stream, 3-level cascade",
            "data": "synthetic", "n_gpus": 1}
    line["x1"] = run_point(16, args.serve_seconds, 1.0)
    # per-frame serving saturates far earlier: beyond x32 its queue only grows
    sweep = {"batched_max16": [], "per_frame": []}
    for scale in (2, 4, 8, 16, 32, 64, 128):
        sweep["batched_max16"].append(run_point(16, args.sweep_seconds, scale))
        if scale <= 32:
            sweep["per_frame"].append(run_point(1, args.sweep_seconds, scale))
    line["sweep"] = sweep
    for k, pts in sweep.items():
        good = [p["frames_per_s"] for p in pts if p["p99_ms"] <= 100.0]
        line[f"max_frames_per_s_p99_le_100ms_{k}"] = max(good) if good else None
    print(json.dumps(line), flush=True)


def run_icp_poses(args):
    """ICP (Sec. 3.2.4) of N poses, 3 cm / 2 deg around the true pose of a
    640x480 query of the config-2 room, in one rl_icp_poses call per step."""
    import torch
    import paper_1810_12163_gb300 as rg
    w = workloads.CONFIG2
    room = w.room()
    ctx = rg.Context(0, arena_bytes=1 << 30)
    scene = rg.Scene(ctx, room.lo, room.hi)
    d, c, T, seed = w.query(0)
    rng = np.random.default_rng(0)
    poses = []
    for _ in range(args.icp_poses):
        P = T.copy()
        axis = rng.normal(size=3)
        P[:3, :3] = rodrigues(axis / np.linalg.norm(axis), math.radians(2.0)) @ T[:3, :3]
        v = rng.normal(size=3)
        P[:3, 3] += v / np.linalg.norm(v) * 0.03
        poses.append(P)
    poses = np.stack(poses)
    dd = torch.from_numpy(d).cuda()
    for _ in range(args.warmup):
        scene.icp_poses(dd, w.K, poses, **workloads.ICP_ON)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        out, ok, frac = scene.icp_poses(dd, w.K, poses, **workloads.ICP_ON)
    dt = time.perf_counter() - t0
    print(json.dumps({"metric": "ICP pose refinements/s (640x480, 3 levels)", "value": args.icp_poses * args.steps / dt,
                      "unit": "poses/s", "poses": args.icp_poses, "steps": args.steps, "ok": float(ok.mean()),
                      "note": "host-timed through rl_icp_poses, pose copies included"}), flush=True)
    scene.close()


def run_robustness(args):
    """Robustness sweeps (reading R22): per corruption level, a config-2
    forest adapted from the corrupted training frames, then the corrupted
    queries relocalised in one batch without and with ICP before ranking;
    5 cm / 5 deg success and median error against the true poses."""
    import torch
    import paper_1810_12163_gb300 as rg
    w = workloads.CONFIG2
    nq = args.robust_queries
    train = list(w.training_frames())
    queries = w.queries(nq)
    ctx = rg.Context(0, arena_bytes=24 << 30)
    room = w.room()
    scene = rg.Scene(ctx, room.lo, room.hi)
    t0 = time.perf_counter()
    out = {}
    arms = (("missing", "missing", workloads.MISSING_LEVELS, True),
            ("missing_queries_only", "missing", workloads.MISSING_LEVELS, False),
            ("noise", "noise", workloads.NOISE_LEVELS, True))
    clean = None
    for arm, kind, levels, train_corrupted in arms:
        rows = []
        for lvl in levels:
            if train_corrupted or clean is None:
                forest = rg.Forest.random(ctx, w.forest, w.forest_seed)
                for i, (d, c, T) in enumerate(train):
                    forest.adapt(workloads.corrupt(d, kind, lvl, i) if train_corrupted else d, c, w.K, T)
                forest.update_modes(-1)
                if not train_corrupted:
                    clean = forest
            else:
                forest = clean
            D = torch.from_numpy(np.stack([workloads.corrupt(q[0], kind, lvl, 10000 + i)
                                           for i, q in enumerate(queries)])).cuda()
            C = torch.from_numpy(np.stack([q[1] for q in queries])).cuda()
            row = {"level": lvl, "valid_depth": float((D > 0).float().mean())}
            # readings R8 (an unusable draw fails its iteration) and R8b
            # (redrawn within the iteration), each without and with ICP
            variants = (("no_icp", w.ransac), ("icp", dict(w.ransac, **workloads.ICP_ON)),
                        ("redraw_no_icp", dict(w.ransac, redraw=1)),
                        ("redraw_icp", dict(w.ransac, redraw=1, **workloads.ICP_ON)))
            for name, p in variants:
                rel = rg.Relocaliser(forest, scene, p, w.width, w.height, nq)
                rs = rel.relocalise_batch(D, C, w.K, [q[3] for q in queries])
                rel.close()
                e = np.array([pose_err(r["pose"], q[2]) for r, q in zip(rs, queries)])
                row[name] = {"success": float(np.mean((e[:, 0] <= 0.05) & (e[:, 1] <= 5.0))),
                             "median_m": float(np.median(e[:, 0])), "median_deg": float(np.median(e[:, 1])),
                             "mean_hypotheses": float(np.mean([r["n_hypotheses"] for r in rs]))}
            if forest is not clean:
                forest.close()
            rows.append(row)
        out[arm] = rows
    line = {"metric": "5 cm / 5 deg success vs depth corruption", "workload": w.name, "queries": nq,
            "arms": {"missing": "training frames and queries masked",
                     "missing_queries_only": "queries masked, forest adapted from clean frames",
                     "noise": "training frames and queries noisy",
                     "redraw_*": "reading R8b: generation redraws an unusable pixel within its iteration"}, **out,
            "icp": {k: (list(v) if isinstance(v, tuple) else v) for k, v in workloads.ICP_ON.items()},
            "seconds": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)
    scene.close()


def _device_frames(frames):
    import torch
    return [(torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda(), T) for d, c, T in frames]


def run_tracking_loss(args):
    """Tracking-loss recovery (Sec. 4): along a fresh 640x480 trajectory of
    the config-2 room, starting from a random forest with empty leaves,
    frame t is relocalised with the forest as it stands (stream R), then
    added with its true pose: reservoir adaptation and a round-robin
    re-clustering of k leaves (stream T, double-buffered modes).  Success
    per frame, first success, per-frame training time (CUDA events on T)
    and relocalisation latency (events on R), for k = 256 (the paper's
    budget) and larger GB300 budgets."""
    import torch
    import paper_1810_12163_gb300 as rg
    from synth import rooms
    w = workloads.CONFIG2
    fp = dict(w.forest, depth=args.track_depth)
    room = w.room()
    n = args.track_frames
    poses = rooms.training_trajectory(room, n, seed=21)
    frames = []
    for t, T in enumerate(poses):
        d, c = rooms.render(room, w.K, T, w.noise_sigma, noise_seed=60000 + t)
        frames.append((d, c, T))
    dev = _device_frames(frames)
    ctx = rg.Context(0, arena_bytes=24 << 30)
    scene = rg.Scene(ctx, room.lo, room.hi)
    out = []
    for k in [int(x) for x in args.track_leaves.split(",")]:
        forest = rg.Forest.random(ctx, fp, w.forest_seed)
        forest.set_streaming(True)
        rel = rg.Relocaliser(forest, scene, w.ransac, w.width, w.height, 1)
        sR, sT = torch.cuda.Stream(), torch.cuda.Stream()
        ok, train_ms, reloc_ms = [], [], []
        for t, (dd, cc, T) in enumerate(dev):
            eR = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            eT = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            if t >= 1:
                eR[0].record(sR)
                rel.relocalise_batch_async(dd[None], cc[None], w.K, [80000 + t], stream=sR)
                eR[1].record(sR)
            eT[0].record(sT)
            forest.adapt(dd, cc, w.K, T, stream=sT)
            forest.update_modes(k, stream=sT)
            eT[1].record(sT)
            if t >= 1:
                r = rel.fetch(stream=sR)[0]
                ok.append(bool(_success(r["pose"], T)))
                reloc_ms.append(eR[0].elapsed_time(eR[1]))
            eT[1].synchronize()
            train_ms.append(eT[0].elapsed_time(eT[1]))
        rel.close()
        forest.close()
        first = next((i + 1 for i, v in enumerate(ok) if v), None)
        out.append({"leaves_per_frame": k, "first_success_frame": first,
                    "success_frames_1_10": float(np.mean(ok[:10])),
                    "success_frames_11_end": float(np.mean(ok[10:])) if len(ok) > 10 else None,
                    "success_curve_by_10": [float(np.mean(ok[i:i + 10])) for i in range(0, len(ok), 10)],
                    "train_ms_per_frame": {"median": float(np.median(train_ms[1:])),
                                           "p99": float(np.percentile(train_ms[1:], 99))},
                    "reloc_ms": {"median": float(np.median(reloc_ms)), "p99": float(np.percentile(reloc_ms, 99))}})
    line = {"metric": "tracking-loss recovery: 5 cm / 5 deg success per frame", "workload": w.name,
            "frames": n, "tree_depth": args.track_depth, "forest_leaves": int(fp["n_trees"] << fp["depth"]),
            "sequence": "seeded trajectory (seed 21) of the config-2 room, 2 mm depth noise", "arms": out}
    print(json.dumps(line), flush=True)
    scene.close()


def run_streaming(args):
    """Adaptation concurrent with relocalisation (Sec. 3.2.2): the config-2
    batched relocalisation (64 frames per launch) runs back to back on one
    stream; a second stream adapts the forest from one posed frame and
    re-clusters 256 leaves (round robin) per relocalisation launch.
    Relocalisation frames/s without and with the training stream, training
    time per frame under load (CUDA events on the training stream)."""
    import torch
    import paper_1810_12163_gb300 as rg
    w = workloads.CONFIG2
    B = args.batch
    frames = training_set(w, w.n_train)
    ctx = rg.Context(0, arena_bytes=24 << 30)
    forest = rg.Forest.random(ctx, w.forest, w.forest_seed)
    for d, c, T in frames:
        forest.adapt(d, c, w.K, T)
    forest.update_modes(-1)
    forest.set_streaming(True)
    scene = rg.Scene(ctx, w.room().lo, w.room().hi)
    rel = rg.Relocaliser(forest, scene, w.ransac, w.width, w.height, B)
    qs = [w.query(i) for i in range(min(B, 32))]
    D = torch.from_numpy(np.stack([qs[i % len(qs)][0] for i in range(B)])).cuda()
    C = torch.from_numpy(np.stack([qs[i % len(qs)][1] for i in range(B)])).cuda()
    dev = _device_frames(frames)
    sR, sT = torch.cuda.Stream(), torch.cuda.Stream()
    steps = max(args.steps, 4)
    for k in range(args.warmup):
        rel.relocalise_batch_async(D, C, w.K, list(range(k * B, k * B + B)), stream=sR)
        rel.fetch(stream=sR, raw=True)
        forest.adapt(dev[k][0], dev[k][1], w.K, dev[k][2], stream=sT)
        forest.update_modes(256, stream=sT)
    torch.cuda.synchronize()

    def phase(train):
        t_ms = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(steps):
            rel.relocalise_batch_async(D, C, w.K, list(range(10_000 + k * B, 10_000 + k * B + B)), stream=sR)
            if train:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                dd, cc, T = dev[(args.warmup + k) % len(dev)]
                e0.record(sT)
                forest.adapt(dd, cc, w.K, T, stream=sT)
                forest.update_modes(256, stream=sT)
                e1.record(sT)
                t_ms.append((e0, e1))
            rel.fetch(stream=sR, raw=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        return B * steps / dt, [a.elapsed_time(b) for a, b in t_ms]

    alone, _ = phase(False)
    mixed, tms = phase(True)
    line = {"metric": "relocalisation frames/s with concurrent adaptation", "workload": w.name, "batch": B,
            "steps": steps, "frames_per_s_alone": alone, "frames_per_s_with_training": mixed,
            "training_ms_per_frame_under_load": {"median": float(np.median(tms)), "p99": float(np.percentile(tms, 99))},
            "leaves_per_frame": 256, "note": "host-timed, results fetched every launch"}
    print(json.dumps(line), flush=True)
    rel.close()
    scene.close()


def run_rqs(args):
    """Really Quick Shift (Sec. 3.2.2 step 3) on N consecutive leaves of the
    config-2 forest adapted from its 200 training frames: CUDA-event time per
    launch and per leaf, and the leaves' reservoir fill."""
    import torch
    import paper_1810_12163_gb300 as rg
    w = workloads.CONFIG2
    frames = training_set(w, args.train_frames or w.n_train)
    ctx = rg.Context(0, arena_bytes=16 << 30)
    forest = rg.Forest.random(ctx, w.forest, w.forest_seed)
    for d, c, T in frames:
        forest.adapt(d, c, w.K, T)
    s = torch.cuda.current_stream()
    ms = []
    for k in range(args.warmup + args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        forest.update_modes(args.rqs_leaves, stream=s)
        e1.record(s)
        e1.synchronize()
        if k >= args.warmup:
            ms.append(e0.elapsed_time(e1))
    count = forest.export(reservoirs=True)["res_count"]
    kappa = w.forest["kappa"]
    print(json.dumps({"metric": "Really Quick Shift time per leaf", "leaves_per_launch": args.rqs_leaves,
                      "ms_per_launch": float(np.median(ms)), "us_per_leaf": 1000 * float(np.median(ms)) / args.rqs_leaves,
                      "reservoir_fill": {"mean": float(np.minimum(count, kappa).mean()),
                                         "full_fraction": float((count >= kappa).mean()),
                                         "empty_fraction": float((count == 0).mean())}}), flush=True)
    forest.close()


def rodrigues(axis, angle):
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * (K @ K)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.icp_poses:
        run_icp_poses(args)
    elif args.robustness:
        run_robustness(args)
    elif args.tracking_loss:
        run_tracking_loss(args)
    elif args.streaming:
        run_streaming(args)
    elif args.rqs_leaves:
        run_rqs(args)
    elif args.serving:
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
