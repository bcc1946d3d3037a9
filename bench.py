#!/usr/bin/env python3
"""Throughput of the IMU-seeded ICP tracking path on GB300.

One step = the whole hot path over one batch of synthetic Kinect-sized frame
pairs already resident in HBM: bilateral filter, depth pyramid, vertex and
normal maps (kf_set_frame_batch), then the coarse-to-fine regularised ICP
with the distance histogram, median filter and convergence control
(kf_align_batch, one CUDA graph). The value is alignments per second over
all ranks; e2e repeats the measurement with the depth frames copied from
pinned host memory and the poses read back every step, pipelined as a
serving loop would run it (two tracker sets: the copy engine uploads the
next batch while the current one aligns), with the one-batch-at-a-time
figure beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the FP64 CPU oracle (the only reference this method
has: the paper ships no code) on the host cores, on the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ICP alignments/s at 640x480 3-level pyramid"
UNIT = "alignments/s"
W, H = 640, 480
CAPS = (10, 5, 4)
LAM = 1e3
# ncu DRAM bytes (read + write) of the dominant kernel per pixel-iteration,
# by (kernel, precision), from the captures summarised in profiles/ for the
# kernel as it stands: one launch over 64 pairs of 640x480 each (FP32:
# 3.477 + 0.189 GB over 82,310,400 pixel-iterations; FP16: 1.801 + 0.171 GB
# over 83,980,800). Larger batches are scaled by the pixel-iterations their
# launch processes (the traffic per pixel-iteration does not depend on how
# many independent pairs share the launch).
NCU_TRAFFIC_PER_PX_ITER = {("k_icp_sched", "fp32"): (3477426688 + 188985088) / 82310400,
                           ("k_icp_sched", "fp16"): (1800692224 + 170857472) / 83980800}


BATCH64_SIZES = [(320, 240), (640, 480), (960, 720), (1280, 960)]


def workload_name(pairs, precision, workload="kinect640"):
    if workload == "batch64":
        return (f"batch64 mixed-resolution {precision}: {pairs} independent frame-to-model pairs per step, "
                f"16 each at 320x240, 640x480, 960x720, 1280x960 (4 seeded random scenes, motion <=8 deg / "
                f"8 cm, outliers uniform in [0, 30%], per-pair IMU prior (0.5 deg noise) and lambda "
                f"log-uniform in [1, 1e3], caps 10/5/4 coarse-to-fine)")
    return (f"kinect-640x480-3level {precision}: {pairs} independent frame-to-model pairs per step "
            f"(synthetic room, 10% uniform-depth outliers, motion <=5 deg / 5 cm, IMU prior noise "
            f"0.3 deg, 5x5 bilateral, caps 10/5/4 coarse-to-fine, lambda 1e3)")


def case_pixels(workload, case):
    """Level-0 pixels of a case (the unit the shards balance)."""
    if workload == "batch64":
        w, h = BATCH64_SIZES[case // 16]
        return w * h
    return W * H


def shard_by_pixels(pixels, rank, world):
    """Cases of one rank: the cases sorted by pixel count (largest first, ties
    by index) dealt round-robin to the ranks, so that per-rank pixel loads
    differ by at most one case. Ranks align disjoint, independent pair sets:
    no collective on the data path."""
    assert 0 <= rank < world
    order = sorted(range(len(pixels)), key=lambda c: (-pixels[c], c))
    return sorted(order[rank::world])


def job_cases(workload, per_rank, world):
    """The job's cases: the default workload gives every rank per_rank pairs
    of its own (weak scaling); batch64 splits the one 64-pair batch (strong)."""
    if workload == "batch64":
        return list(range(64)), "strong"
    return list(range(per_rank * world)), "weak"


def shard(rank, world, per_rank, workload="kinect640"):
    cases, _ = job_cases(workload, per_rank, world)
    return shard_by_pixels([case_pixels(workload, c) for c in cases], rank, world)


def max_over_ranks(x, dist=None, device="cpu"):
    """Timing reduction: the slowest rank defines the job's time."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_case(workload, case):
    from synth import scenes as S
    return S.config4_batch(case) if workload == "batch64" else S.config2_kinect(case)


def _make_pair(wc):
    return wc[1], make_case(*wc)


def make_pairs(cases, workload="kinect640"):
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1),
                                mp_context=mp.get_context("spawn")) as ex:
        out = dict(ex.map(_make_pair, [(workload, c) for c in cases]))
    return [out[c] for c in cases]


# ---------------------------------------------------------------------------
# CPU oracle legs (the oracle is test infrastructure; only these legs run it)
# ---------------------------------------------------------------------------
def _oracle_align_case(case, workload="kinect640"):
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    from oracle import kf_oracle as O
    pr = make_case(workload, case)
    op = O.Params(levels=3, max_iters=CAPS)
    c = O.Cam(*pr.K.as_tuple())
    t0 = time.perf_counter()
    r = O.align_from_depth(pr.depth, c, pr.model_vertex, pr.model_normal, c, pr.model_pose,
                           pr.prior_R, pr.init_pose, pr.lam, op)
    return case, time.perf_counter() - t0, r.pose, r.status, list(r.iters)


def _oracle_worker(cases, budget_s, q, workload="kinect640"):
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    os.environ["OMP_NUM_THREADS"] = "1"
    out = []
    spent = 0.0
    for c in cases:
        case, dt, pose, st, iters = _oracle_align_case(c, workload)
        out.append((case, dt, pose.tolist(), st, iters))
        spent += dt
        if spent >= budget_s:
            break
    q.put(out)


def run_oracle(cases, budget_s, workload="kinect640"):
    """Time the oracle on up to len(cases) pairs, single-threaded, in a spawned
    process (so its BLAS runs with one thread). Returns [(case, s, pose, st, iters)]."""
    import multiprocessing as mp
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    os.environ["OMP_NUM_THREADS"] = "1"
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_oracle_worker, args=(cases, budget_s, q, workload))
    p.start()
    res = q.get()
    p.join()
    return res


def _oracle_share(args):
    cases, budget_s, workload = args
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    os.environ["OMP_NUM_THREADS"] = "1"
    n, spent = 0, 0.0
    for c in cases:
        spent += _oracle_align_case(c, workload)[1]
        n += 1
        if spent >= budget_s:
            break
    return n


def run_oracle_all_cores(cases, budget_s, workload="kinect640"):
    """The oracle on every host core: one spawned single-threaded process per
    core, each aligning its share of independent pairs until the budget is
    spent (the oracle itself unchanged). Returns (alignments, wall s, cores)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    os.environ["OMP_NUM_THREADS"] = "1"
    cores = max(1, os.cpu_count() or 1)
    shares = [([cases[i % len(cases)] for i in range(w, 4 * len(cases), cores)], budget_s, workload)
              for w in range(cores)]
    shares = [sh for sh in shares if sh[0]]
    t0 = time.perf_counter()
    with cf.ProcessPoolExecutor(max_workers=len(shares), mp_context=mp.get_context("spawn")) as ex:
        done = sum(ex.map(_oracle_share, shares))
    return done, time.perf_counter() - t0, len(shares)


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n = args.steps + args.warmup
    res = run_oracle(list(range(n)), budget_s=1e9)
    timed = [r[1] for r in res[args.warmup:]]
    total = sum(timed)
    value = len(timed) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * total / len(timed), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(1, "fp64 oracle"), "pairs_per_step": 1},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{len(timed)} alignments (pyramid + ICP), one per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        import tempfile
        try:
            fd, self.path = tempfile.mkstemp(prefix=f"clocks{self.dev}_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()
            with open(self.path) as f:
                self.lines = f.readlines()
            os.unlink(self.path)

    def summary(self):
        if self.proc is None:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
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
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


# ---------------------------------------------------------------------------
# the GB300 arm
# ---------------------------------------------------------------------------
def rot_angle(R):
    return float(np.arccos(np.clip((np.trace(R) - 1.0) / 2.0, -1.0, 1.0)))


def rot_between(Ra, Rb):
    """Angle of Ra Rb^T from the chord |Ra - Rb|_F = 2 sqrt(2) sin(angle / 2)
    (full precision for tiny angles, where arccos of the trace loses half the
    digits)."""
    f = float(np.linalg.norm(np.asarray(Ra, np.float64) - np.asarray(Rb, np.float64)))
    return 2.0 * math.asin(min(1.0, f / (2.0 * math.sqrt(2.0))))


def ablation(kf, pairs, K, stream, steps, precision):
    """The paper's timing comparison on the same pairs (synthetic analog of its
    KinectFusion-vs-IMU-seeded table): the paper's mode with caps 4/5/10 and
    2/2/3 coarse to fine, and the original KinectFusion loop (no IMU seed, no
    median filter, no convergence rule, lambda 0, fixed 4/5/10, normal-angle
    gate at 20 degrees). Per variant:
    alignments/s (device-timed front end + alignment per step), mean
    iterations, pose error against the ground truth (median), failures
    (rotation error > 5 deg or translation error > 10 cm)."""
    import torch
    n = len(pairs)
    dd = [torch.from_numpy(pr.depth).cuda() for pr in pairs]
    dptrs = [d.data_ptr() for d in dd]
    priors = np.stack([pr.prior_R for pr in pairs])
    inits = np.stack([pr.init_pose for pr in pairs])
    out = {}
    for name, caps, flags, lam, extra in [
            ("paper_4_5_10", (10, 5, 4), 7, LAM, {}),
            ("paper_2_2_3", (3, 2, 2), 7, LAM, {}),
            # KinectFusion's own loop: no seed, filter or convergence rule,
            # lambda 0, fixed 4/5/10, its normal-angle gate at 20 degrees
            ("original_kinectfusion_4_5_10", (10, 5, 4), 0, 0.0,
             {"cos_angle_min": math.cos(math.radians(20.0))}),
            # the paper's own normal and association choices (Sec. 3.3)
            ("paper_integral_normals", (10, 5, 4), 7, LAM, {"normal_mode": kf.KF_NORMALS_INTEGRAL}),
            ("paper_normal_shooting_w2", (10, 5, 4), 7, LAM, {"shoot_radius": 2}),
            ("paper_integral_normals_shooting_w2", (10, 5, 4), 7, LAM,
             {"normal_mode": kf.KF_NORMALS_INTEGRAL, "shoot_radius": 2})]:
        p = kf.kf_default_params()
        for i, c in enumerate(caps):
            p.max_iters[i] = c
        p.flags = flags
        for k_, v_ in extra.items():
            setattr(p, k_, v_)
        p.precision = kf.KF_FP16 if precision == "fp16" else kf.KF_FP32
        trk = [kf.kf_track_create(p, W, H, stream.cuda_stream) for _ in pairs]
        try:
            with torch.cuda.stream(stream):
                for t, pr in zip(trk, pairs):
                    mv = torch.from_numpy(np.ascontiguousarray(pr.model_vertex)).cuda()
                    mn = torch.from_numpy(np.ascontiguousarray(pr.model_normal)).cuda()
                    kf.kf_set_model(t, mv.data_ptr(), mn.data_ptr(), pr.model_pose, K, True)
                    stream.synchronize()
            lams = np.full(n, lam)
            pri = priors if flags & 1 else None

            def step():
                kf.kf_set_frame_batch(trk, dptrs, [K] * n, True)
                return kf.kf_align_batch(trk, pri, inits, lams)

            for _ in range(3):
                step()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                st, poses, res = step()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            # the front end alone (set-frame of the batch)
            e0.record(stream)
            for _ in range(steps):
                kf.kf_set_frame_batch(trk, dptrs, [K] * n, True)
            e1.record(stream)
            torch.cuda.synchronize()
            fe_ms = e0.elapsed_time(e1) / steps
            rot = [math.degrees(rot_angle(poses[i][:3, :3] @ pr.gt_pose[:3, :3].T)) for i, pr in enumerate(pairs)]
            tr = [1e3 * float(np.linalg.norm(poses[i][:3, 3] - pr.gt_pose[:3, 3])) for i, pr in enumerate(pairs)]
            out[name] = {"alignments_per_s": n / (ms / 1000.0), "ms_per_step": ms, "frontend_ms": fe_ms,
                         "mean_iters": sum(r.total_iters for r in res) / n,
                         "median_rot_err_deg": float(np.median(rot)), "median_trans_err_mm": float(np.median(tr)),
                         "failures": int(sum(a > 5.0 or b > 100.0 for a, b in zip(rot, tr)))}
        finally:
            for t in trk:
                kf.kf_track_destroy(t)
    return out


def _models_to_device(kf, torch, trk, pairs, stream):
    with torch.cuda.stream(stream):
        for t, pr in zip(trk, pairs):
            mv = torch.from_numpy(np.ascontiguousarray(pr.model_vertex)).cuda()
            mn = torch.from_numpy(np.ascontiguousarray(pr.model_normal)).cuda()
            kf.kf_set_model(t, mv.data_ptr(), mn.data_ptr(), pr.model_pose, pr.K.as_tuple(), True)
            stream.synchronize()


def pose_errors(poses, pairs, oracle=None):
    """Pose error summaries: against the ground truth (all pairs, deg / mm) and
    against the FP64 oracle's poses (the sampled pairs, rad / m)."""
    rot = [math.degrees(rot_angle(poses[i][:3, :3] @ pr.gt_pose[:3, :3].T)) for i, pr in enumerate(pairs)]
    tr = [1e3 * float(np.linalg.norm(poses[i][:3, 3] - pr.gt_pose[:3, 3])) for i, pr in enumerate(pairs)]
    out = {"vs_truth": {"median_rot_deg": float(np.median(rot)), "max_rot_deg": float(np.max(rot)),
                        "median_trans_mm": float(np.median(tr)), "max_trans_mm": float(np.max(tr))}}
    if oracle:
        ro = [rot_between(poses[i][:3, :3], np.asarray(ref)[:3, :3]) for i, ref in oracle.items()]
        to = [float(np.linalg.norm(poses[i][:3, 3] - np.asarray(ref)[:3, 3])) for i, ref in oracle.items()]
        out["vs_oracle"] = {"pairs": len(oracle), "median_rot_rad": float(np.median(ro)),
                            "max_rot_rad": float(np.max(ro)), "median_trans_m": float(np.median(to)),
                            "max_trans_m": float(np.max(to))}
    return out


def precision_form(kf, torch, pairs, stream, steps, oracle, main=None):
    """The comparison the batching and precision patterns are built for, on the
    same pairs: FP16-stored maps (FP32 arithmetic, FP64 solve) in the batched
    persistent launch against the plain FP32 single-frame form (one pair per
    call). Each with its alignments/s (device-timed front end + alignment; the
    batched form also end to end from page-locked host frames, one batch at a
    time) and its pose errors against the FP64 oracle and the ground truth.
    main: the FP16 batched figures when the main run already was FP16."""
    n = len(pairs)
    Ks = [pr.K.as_tuple() for pr in pairs]
    priors = np.stack([pr.prior_R for pr in pairs])
    inits = np.stack([pr.init_pose for pr in pairs])
    lams = np.array([pr.lam for pr in pairs])
    mw, mh = max(k[0] for k in Ks), max(k[1] for k in Ks)
    dd = [torch.from_numpy(pr.depth).cuda() for pr in pairs]
    dptrs = [d.data_ptr() for d in dd]
    out = {}
    if main is None:
        p = kf.kf_default_params()
        for i, c in enumerate(CAPS):
            p.max_iters[i] = c
        p.precision = kf.KF_FP16
        trk = [kf.kf_track_create(p, mw, mh, stream.cuda_stream) for _ in pairs]
        try:
            _models_to_device(kf, torch, trk, pairs, stream)

            def step():
                kf.kf_set_frame_batch(trk, dptrs, Ks, True)
                return kf.kf_align_batch(trk, priors, inits, lams)

            for _ in range(3):
                step()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                st, poses, res = step()
            e1.record(stream)
            torch.cuda.synchronize()
            value = n * steps / (e0.elapsed_time(e1) / 1000.0)
            pinned = [torch.from_numpy(pr.depth).pin_memory() for pr in pairs]
            hptrs = [x.data_ptr() for x in pinned]
            kf.kf_set_frame_batch(trk, hptrs, Ks, kf.KF_FRAME_HOST)
            kf.kf_align_batch(trk, priors, inits, lams)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(steps):
                kf.kf_set_frame_batch(trk, hptrs, Ks, kf.KF_FRAME_HOST)
                kf.kf_align_batch(trk, priors, inits, lams)
            torch.cuda.synchronize()
            e2e = n * steps / (time.perf_counter() - t0)
            main = {"alignments_per_s": value, "e2e_alignments_per_s": e2e, "poses": poses}
        finally:
            for t in trk:
                kf.kf_track_destroy(t)
    out["fp16_batched"] = {"alignments_per_s": main["alignments_per_s"],
                           "e2e_alignments_per_s": main["e2e_alignments_per_s"],
                           "pairs_per_call": n, **pose_errors(main["poses"], pairs, oracle)}
    # the plain FP32 single-frame form: one pair per call, device-resident depth
    p = kf.kf_default_params()
    for i, c in enumerate(CAPS):
        p.max_iters[i] = c
    ns = min(n, 64)
    trk = [kf.kf_track_create(p, mw, mh, stream.cuda_stream) for _ in range(ns)]
    try:
        _models_to_device(kf, torch, trk, pairs[:ns], stream)
        for i in range(ns):  # builds each tracker's single-pair graph
            kf.kf_set_frame(trk[i], dptrs[i], Ks[i], True)
            kf.kf_align(trk[i], priors[i], inits[i], lams[i])
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        poses1 = np.zeros((ns, 4, 4))
        s0.record(stream)
        for i in range(ns):
            kf.kf_set_frame(trk[i], dptrs[i], Ks[i], True)
            st, poses1[i], _ = kf.kf_align(trk[i], priors[i], inits[i], lams[i])
        s1.record(stream)
        torch.cuda.synchronize()
        orc = {i: v for i, v in (oracle or {}).items() if i < ns}
        out["fp32_single_frame"] = {"alignments_per_s": ns / (s0.elapsed_time(s1) / 1000.0),
                                    "pairs_per_call": 1, **pose_errors(poses1, pairs[:ns], orc)}
    finally:
        for t in trk:
            kf.kf_track_destroy(t)
    out["fp16_batched_over_fp32_single_frame"] = (out["fp16_batched"]["alignments_per_s"]
                                                  / out["fp32_single_frame"]["alignments_per_s"])
    return out


def gb300_arm(args):
    import numpy as np
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    wl = args.workload
    all_cases, scaling = job_cases(wl, args.pairs, world)
    cases = shard(rank, world, args.pairs, wl)
    npairs = len(cases)
    pairs = make_pairs(cases, wl)                   # spawn pool, before any CUDA call
    cpu_cases = cases[:min(args.cpu_pairs, npairs)]
    cpu = run_oracle(cpu_cases, args.cpu_budget, wl) if (rank == 0 and world == 1 and not args.no_cpu) else []
    cpu_all = (run_oracle_all_cores(cases, args.cpu_budget, wl)
               if (rank == 0 and world == 1 and not args.no_cpu) else None)

    import torch
    import paper_1802_03980_gb300 as kf
    from paper_1802_03980_gb300 import tune
    kf.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    p = kf.kf_default_params()
    for i, c in enumerate(CAPS):
        p.max_iters[i] = c
    p.precision = kf.KF_FP16 if args.precision == "fp16" else kf.KF_FP32
    Ks = [pr.K.as_tuple() for pr in pairs]
    mw, mh = max(k[0] for k in Ks), max(k[1] for k in Ks)
    trk = [kf.kf_track_create(p, mw, mh, sh) for _ in pairs]
    depth_dev = [torch.from_numpy(pr.depth).cuda() for pr in pairs]
    _models_to_device(kf, torch, trk, pairs, stream)
    priors = np.stack([pr.prior_R for pr in pairs])
    inits = np.stack([pr.init_pose for pr in pairs])
    lams = np.array([pr.lam for pr in pairs])
    dptrs = [d.data_ptr() for d in depth_dev]

    def step():
        kf.kf_set_frame_batch(trk, dptrs, Ks, True)
        return kf.kf_align_batch(trk, priors, inits, lams)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            st, poses, res = step()
        ev1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
    # stage times from a second, profiled run of the same steps (the plans
    # with event nodes are built in its warm-up; the timed run above has none)
    kf.kf_profile_enable(trk[0], True)
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    kf.kf_profile_enable(trk[0], True)  # resets the counters
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    prof = kf.kf_profile_read(trk[0])
    kf.kf_profile_enable(trk[0], False)
    total_align = len(all_cases) * args.steps
    value = total_align / (ms / 1000.0)

    # end to end through the public API: pinned host depth in, poses out.
    # (a) one batch at a time: set-frame pulls the page-locked frames with a
    # kernel, align returns the poses;
    # The batch's frames lie back to back in one page-locked buffer, as a
    # frame grabber's ring holds them: a copy-engine upload moves them as one
    # copy (each copy costs the host ~10 us to issue, whatever its size).
    sizes = [int(pr.depth.size) for pr in pairs]
    flat = torch.empty(sum(sizes), dtype=torch.float32).pin_memory()
    hptrs, off = [], 0
    for pr, sz in zip(pairs, sizes):
        flat[off:off + sz].copy_(torch.from_numpy(np.ascontiguousarray(pr.depth, np.float32)).reshape(-1))
        hptrs.append(flat.data_ptr() + 4 * off)
        off += sz

    def e2e_step():
        kf.kf_set_frame_batch(trk, hptrs, Ks, kf.KF_FRAME_HOST)
        return kf.kf_align_batch(trk, priors, inits, lams)

    for _ in range(2):
        e2e_step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_serial_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    # (b) pipelined, as a serving loop runs it: a second set of trackers on a
    # second stream; while one set aligns batch i, the copy engine uploads
    # batch i + 1 into the other (every batch's frames still cross the host
    # link inside the timed region, every batch's poses come back)
    stream2 = torch.cuda.Stream()
    trk2 = [kf.kf_track_create(p, mw, mh, stream2.cuda_stream) for _ in pairs]
    _models_to_device(kf, torch, trk2, pairs, stream2)
    sets = (trk, trk2)

    def e2e_pipelined(steps):
        kf.kf_set_frame_batch(sets[0], hptrs, Ks, kf.KF_FRAME_HOST_COPY_ENGINE)
        for i in range(steps):
            if i + 1 < steps:
                kf.kf_set_frame_batch(sets[(i + 1) % 2], hptrs, Ks, kf.KF_FRAME_HOST_COPY_ENGINE)
            out = kf.kf_align_batch(sets[i % 2], priors, inits, lams)
        return out

    e2e_pipelined(4)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st2, poses2, res2 = e2e_pipelined(args.steps)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e_value = total_align / e2e_s
    e2e_serial_value = total_align / e2e_serial_s
    assert np.array_equal(poses2, poses), "the pipelined loop must give the same poses"
    for t in trk2:
        kf.kf_track_destroy(t)
    h2d = sum(int(pr.depth.nbytes) for pr in pairs) + len(pairs) * (9 + 16 + 1) * 8
    d2h = len(pairs) * (16 * 8 + 56)
    # (c) a tracking loop also replaces the model every frame: the same loop one
    # batch at a time with every pair's model maps uploaded from page-locked
    # host memory too (kf_set_model, host pointers)
    mpin = [(torch.from_numpy(np.ascontiguousarray(pr.model_vertex)).pin_memory(),
             torch.from_numpy(np.ascontiguousarray(pr.model_normal)).pin_memory()) for pr in pairs]
    nm = min(args.steps, 10)

    def e2e_model_step():
        for t, pr, (v, n_) in zip(trk, pairs, mpin):
            kf.kf_set_model(t, v.data_ptr(), n_.data_ptr(), pr.model_pose, pr.K.as_tuple(), False)
        return e2e_step()

    e2e_model_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(nm):
        e2e_model_step()
    torch.cuda.synchronize()
    e2e_model_value = len(all_cases) * nm / max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    h2d_model = sum(int(v.numel() * 4 + n_.numel() * 4) for v, n_ in mpin)

    # parity of the timed run: statuses, and the oracle's poses for the CPU sample
    assert all(r.status >= 0 for r in res), [r.status for r in res]
    parity = None
    oracle_poses = {}
    if cpu:
        idx = {c: i for i, c in enumerate(cases)}
        oracle_poses = {idx[c]: np.array(pose) for c, _, pose, _, _ in cpu}
        errs = [rot_between(poses[idx[c]][:3, :3], np.array(pose)[:3, :3]) for c, _, pose, _, _ in cpu]
        terr = [float(np.linalg.norm(poses[idx[c]][:3, 3] - np.array(pose)[:3, 3])) for c, _, pose, _, _ in cpu]
        parity = {"pairs_checked": len(cpu), "max_rot_rad": max(errs), "max_trans_m": max(terr),
                  "iters_equal": all(list(res[idx[c]].iters)[:3] == it for c, _, _, _, it in cpu)}
        if args.precision == "fp32":
            assert max(errs) < 1e-5 and max(terr) < 1e-5, parity
        else:  # the oracle aligns the FP32 maps: the difference is the storage quantisation
            parity["note"] = ("FP16 maps against the oracle on FP32 maps (storage quantisation); "
                              "the parity bar applies to FP32 maps")

    # roofline of the dominant kernel (time share over the timed region).
    # Frame pixels each kernel processed per step, from the pairs' iteration
    # records (every step repeats the same iterations: same inputs).
    px_iters = px_rereads = 0
    n_hit = n_iters = 0
    solve_ns = []
    for t, k in zip(trk, Ks):
        lv_px = [(k[0] >> l) * (k[1] >> l) for l in range(3)]
        for r in kf.kf_debug_trace(t):
            n_iters += 1
            n_hit += r.passes == 1
            solve_ns.append(r.solve_ns)
            px_iters += lv_px[r.level]
            if r.passes == 2:
                px_rereads += lv_px[r.level]
    # algorithmic bytes per pixel-iteration (the fixed unit of the roofline):
    # one read of the frame vertex plus one gathered model vertex and normal,
    # 3 x 12 B in FP32 storage, 3 x 6 B in FP16. An iteration whose band edge
    # left the expected window reads its frame a second time (px_rereads):
    # the fraction below counts useful work only; the ncu traffic is what moved.
    unit_b = 18 if args.precision == "fp16" else 36
    kern = {"k_assoc_hist": (prof.assoc_ms, prof.assoc_launches, unit_b * px_iters),
            "k_reduce_solve": (prof.reduce_ms, prof.reduce_launches, 0),
            "k_icp_sched": (prof.sched_ms, prof.sched_launches, unit_b * px_iters)}
    dom = max(kern, key=lambda k: kern[k][0])
    kms, klaunch, kbytes_step = kern[dom]
    peak, peak_src = hbm_peak()
    bytes_per_launch = kbytes_step * args.steps / max(1, klaunch)
    achieved = bytes_per_launch / (kms / max(1, klaunch) / 1000.0) / 1e9 if kms > 0 else 0.0
    # DRAM bytes of one launch of this kernel on this workload, from ncu
    # (dram__bytes_read.sum + dram__bytes_write.sum); null when not captured
    per_px = NCU_TRAFFIC_PER_PX_ITER.get((dom, args.precision)) if wl == "kinect640" else None
    traffic = per_px * (px_iters * args.steps / max(1, klaunch)) if per_px else None
    corr = prof.pixel_iters / (prof.align_ms / 1000.0) / 1e6 if prof.align_ms > 0 else None
    # kernels of ours per step: the front end, then the scheduled launch, or
    # init + per-iteration launches + finish
    per_iter = prof.assoc_launches + prof.reduce_launches
    fe_per_call = -(-npairs // 64)  # the front end takes 64 frames per launch
    launches_per_step = (prof.frontend_calls * fe_per_call + prof.sched_launches + per_iter
                         + (2 * prof.graph_launches if per_iter else 0)) / max(1, args.steps)
    abl = None
    if world == 1 and not args.no_ablation and wl == "kinect640":
        abl = ablation(kf, pairs, Ks[0], stream, min(args.steps, 50), args.precision)
    pform = None
    if world == 1 and not args.no_precision_form:
        main = None
        if args.precision == "fp16":
            main = {"alignments_per_s": value, "e2e_alignments_per_s": e2e_serial_value, "poses": poses}
        pform = precision_form(kf, torch, pairs, stream, min(args.steps, 50), oracle_poses, main)
    metric = METRIC if wl == "kinect640" else "ICP alignments/s, 64-pair mixed-resolution batch (320x240 to 1280x960)"
    line = {
        "metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": scaling, "vs_baseline": None,
        "dtype": "f16" if args.precision == "fp16" else "f32", "data": "synthetic",
        "config": {"workload": workload_name(len(all_cases), args.precision, wl),
                   "pairs_per_step": len(all_cases), "pairs_per_rank": npairs,
                   "precision": args.precision, "arithmetic": "f32 (FP64 solve and pose)",
                   "parallelism": f"replicas x{world} (pairs sharded by pixel count, no collective)",
                   "l2": "inputs larger than L2 (>1 GB of frame and model maps per step)"},
        "tuned": {"defines": tune.tuned_defines() or "library defaults (no tuned.json)"},
        "correspondences_M_per_s": corr,
        "stage_ms_per_step": {"frontend": prof.frontend_ms / args.steps,
                              "icp_sched": prof.sched_ms / args.steps,
                              "assoc_hist": prof.assoc_ms / args.steps,
                              "reduce_solve": prof.reduce_ms / args.steps,
                              "align_graph": prof.align_ms / args.steps},
        "window_hits": f"{n_hit} of {n_iters} iterations (frame read once); "
                       f"{px_rereads / max(1, px_iters):.3f} of the pixel-iterations read twice",
        "solve_us_median": float(np.median(solve_ns)) / 1000.0 if solve_ns else None,
        "roofline": {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "traffic_source": ("ncu dram bytes per pixel-iteration of one 64-pair launch, "
                                        "scaled to this launch's pixel-iterations") if traffic else None,
                     "peak_source": peak_src, "bytes_per_launch": bytes_per_launch,
                     "bytes_per_px_iter": unit_b, "px_iters_per_launch": px_iters * args.steps / max(1, klaunch),
                     "launches": klaunch, "avg_launch_us": 1000.0 * kms / max(1, klaunch)},
        # two serving forms through the public API, both timed in this run
        # with the same bytes crossing the host link; the line reports the
        # faster one (which one wins has differed between runs)
        "e2e": {"value": max(e2e_value, e2e_serial_value), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "form": ("pipelined" if e2e_value >= e2e_serial_value else "one_batch_at_a_time"),
                "pipelined": e2e_value,
                "pipelined_form": "two tracker sets on two streams, the copy engine uploads batch i+1 "
                                  "while batch i aligns; the batch's frames lie back to back in one "
                                  "page-locked buffer (one copy per batch)",
                "one_batch_at_a_time": e2e_serial_value,
                "one_batch_at_a_time_form": "one tracker set; set-frame pulls the page-locked frames "
                                            "with one gather kernel, align returns the poses",
                "model_maps": "resident: set once before the timed region, not uploaded per step",
                "with_model_upload": {"value": e2e_model_value, "steps": nm,
                                      "h2d_bytes_per_step": h2d + h2d_model,
                                      "form": "one batch at a time; every pair's model vertex and normal "
                                              "maps also uploaded from page-locked host memory each step"}},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "clocks": clk.summary(),
        "parity_vs_oracle": parity,
        "mean_iters": sum(r.total_iters for r in res) / len(res),
        "pose_errors": pose_errors(poses, pairs, oracle_poses),
        "precision_form": pform,
        "ablation": abl,
    }
    if cpu:
        ctime = sum(r[1] for r in cpu)
        n_all, wall_all, cores_all = cpu_all
        line["cpu_baseline"] = {"value": n_all / wall_all, "unit": UNIT, "cores": cores_all, "kind": "oracle",
                                "sample": f"{n_all} alignments of the same pairs (pyramid + ICP each) on "
                                          f"{cores_all} single-threaded FP64 numpy processes, {wall_all:.1f} s "
                                          f"wall including start-up",
                                "single_thread": {"value": len(cpu) / ctime, "cores": 1,
                                                  "sample": f"{len(cpu)} of the {npairs} pairs, {ctime:.1f} s"}}
    if rank == 0:
        print(json.dumps(line))
    for t in trk:
        kf.kf_track_destroy(t)
    if dist:
        dist.destroy_process_group()
    return 0


def _make_angular(ij):
    from synth import scenes as S
    return ij, S.angular_case(ij[0], ij[1])


def frontend_experiment(args):
    """The front end alone (bilateral filter, pyramid, vertex and normal maps
    of every level) for a batch of --pairs 640x480 frames, with
    KinectFusion's cross-product normals or the integral-image normals of
    Sec. 3.3 (--normals). Device-timed set-frame of the whole batch, device
    frames. One JSON line."""
    import torch
    import paper_1802_03980_gb300 as kf
    kf.build()
    n = args.pairs
    pairs = make_pairs(list(range(n)))
    K = pairs[0].K.as_tuple()
    p = kf.kf_default_params()
    p.normal_mode = kf.KF_NORMALS_INTEGRAL if args.normals == "integral" else kf.KF_NORMALS_CROSS
    stream = torch.cuda.Stream()
    trk = [kf.kf_track_create(p, W, H, stream.cuda_stream) for _ in range(n)]
    try:
        dd = [torch.from_numpy(pr.depth).cuda() for pr in pairs]
        torch.cuda.synchronize()
        ptrs = [d.data_ptr() for d in dd]
        for _ in range(args.warmup):
            kf.kf_set_frame_batch(trk, ptrs, [K] * n, True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            kf.kf_set_frame_batch(trk, ptrs, [K] * n, True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        kept = []
        for l in range(3):
            _, V, _ = kf.kf_debug_frame_level(trk[0], l)
            kept.append(float(np.isfinite(V[..., 0]).mean()))
    finally:
        for t in trk:
            kf.kf_track_destroy(t)
    print(json.dumps({"experiment": "frontend", "normals": args.normals, "frames": n,
                      "size": [W, H], "levels": 3, "ms_per_batch": ms,
                      "ns_per_level0_pixel": 1e6 * ms / (n * W * H),
                      "pixels_with_normal_frame0": kept, "data": "synthetic (10 % outliers)"}))
    return 0


def angular_experiment(args):
    """Synthetic analog of the paper's large-rotation experiment (Sec. 4.2):
    16 pairs of 640x480 per rotation angle, aligned with the IMU seed (paper
    mode, lambda 1e3) and without it (previous pose, lambda 0, filter and
    convergence rule kept). Failure: rotation error > 5 deg or translation
    error > 10 cm against the ground truth. One JSON line."""
    import concurrent.futures as cf
    import multiprocessing as mp
    from synth import scenes as S
    keys = [(a, c) for a in range(len(S.ANGULAR_SWEEP_DEG)) for c in range(16)]
    with cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1),
                                mp_context=mp.get_context("spawn")) as ex:
        got = dict(ex.map(_make_angular, keys))
    import torch
    import paper_1802_03980_gb300 as kf
    kf.build()
    stream = torch.cuda.Stream()
    res = {"experiment": "angular_failure_sweep", "pairs_per_angle": 16,
           "angles_deg": list(S.ANGULAR_SWEEP_DEG),
           "failure": "rotation error > 5 deg or translation error > 10 cm",
           "data": "synthetic"}
    for label, flags, lam in [("seeded", 7, LAM), ("unseeded", 6, 0.0)]:
        p = kf.kf_default_params()
        for i, c in enumerate(CAPS):
            p.max_iters[i] = c
        p.flags = flags
        trk = [kf.kf_track_create(p, W, H, stream.cuda_stream) for _ in range(16)]
        fails, med = [], []
        try:
            for a in range(len(S.ANGULAR_SWEEP_DEG)):
                prs = [got[(a, c)] for c in range(16)]
                K = prs[0].K.as_tuple()
                with torch.cuda.stream(stream):
                    for t, pr in zip(trk, prs):
                        mv = torch.from_numpy(np.ascontiguousarray(pr.model_vertex)).cuda()
                        mn = torch.from_numpy(np.ascontiguousarray(pr.model_normal)).cuda()
                        dz = torch.from_numpy(pr.depth).cuda()
                        kf.kf_set_model(t, mv.data_ptr(), mn.data_ptr(), pr.model_pose, K, True)
                        kf.kf_set_frame(t, dz.data_ptr(), K, True)
                        stream.synchronize()
                st, poses, rr = kf.kf_align_batch(trk, np.stack([pr.prior_R for pr in prs]) if flags & 1 else None,
                                                  np.stack([pr.init_pose for pr in prs]), np.full(16, lam))
                rot = [math.degrees(rot_angle(poses[i][:3, :3] @ pr.gt_pose[:3, :3].T)) for i, pr in enumerate(prs)]
                tr = [float(np.linalg.norm(poses[i][:3, 3] - pr.gt_pose[:3, 3])) for i, pr in enumerate(prs)]
                fails.append(int(sum(x > 5.0 or y > 0.1 for x, y in zip(rot, tr))))
                med.append(float(np.median(rot)))
        finally:
            for t in trk:
                kf.kf_track_destroy(t)
        res[label + "_failures"] = fails
        res[label + "_median_rot_err_deg"] = med
    print(json.dumps(res))
    return 0


def _traj_depth(args):
    i, pose, seed, outliers, holes = args
    from synth import scenes as S
    rng = np.random.default_rng(seed)
    return i, S.render_depth(S.room_6x6x3(), pose, S.kinect_intrinsics(), rng, outliers=outliers, holes=holes)


def _kinectfusion_loop(args, kf, torch, p, gt, priors, depths, K):
    """The full loop on the GPU: each frame is tracked against the raycast of
    the map fused so far (512^3 cube of 6.6 m around the room, mu 5 cm), then
    integrated at its estimated pose, and the map is raycast at that pose for
    the next frame. Two trackers on two streams take the frames in turn:
    frame i + 1's upload (copy engine, page-locked frames) and front end are
    queued before frame i is aligned, so they overlap its alignment,
    integration and raycast; the volume has its own stream and the next
    tracker waits for the raycast by an event."""
    n = args.frames
    Kt = K.as_tuple()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    vstream = torch.cuda.Stream()
    trk = [kf.kf_track_create(p, W, H, st.cuda_stream) for st in streams]
    vp = kf.kf_volume_default_params()
    vp.res, vp.side, vp.mu = 512, 6.6, 0.05
    for a in range(3):
        vp.origin[a] = -3.3
    vol = kf.kf_volume_create(vp, vstream.cuda_stream)
    pinned = {i: torch.from_numpy(np.ascontiguousarray(depths[i], np.float32)).pin_memory() for i in depths}
    Vd = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
    Nd = torch.empty_like(Vd)
    torch.cuda.synchronize()
    ray = (0.3, 6.0, 0.02)
    est, lat, t_int, t_ray, iters, diag = [gt[0].copy()], [], [], [], [], []
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ready = torch.cuda.Event()
    try:
        kf.kf_volume_integrate(vol, pinned[0].data_ptr(), Kt, gt[0], False)
        kf.kf_volume_raycast(vol, Kt, gt[0], *ray, Vd.data_ptr(), Nd.data_ptr(), True)
        ready.record(vstream)
        kf.kf_set_frame(trk[1], pinned[1].data_ptr(), Kt, kf.KF_FRAME_HOST_COPY_ENGINE)
        t_start = time.perf_counter()
        for i in range(1, n):
            cur, nxt = trk[i % 2], trk[(i + 1) % 2]
            t0 = time.perf_counter()
            streams[i % 2].wait_event(ready)   # the raycast maps are written
            mp_ = gt[i - 1] if args.map_poses == "gt" else est[-1]
            kf.kf_set_model(cur, Vd.data_ptr(), Nd.data_ptr(), mp_, Kt, True)
            if i + 1 < n:
                kf.kf_set_frame(nxt, pinned[i + 1].data_ptr(), Kt, kf.KF_FRAME_HOST_COPY_ENGINE)
            st, pose, res = kf.kf_align(cur, priors[i], est[-1], args.lam)
            ev[0].record(vstream)
            mp_ = gt[i] if args.map_poses == "gt" else pose
            kf.kf_volume_integrate(vol, pinned[i].data_ptr(), Kt, mp_, False)
            ev[1].record(vstream)
            kf.kf_volume_raycast(vol, Kt, mp_, *ray, Vd.data_ptr(), Nd.data_ptr(), True)
            ev[2].record(vstream)
            ready.record(vstream)
            vstream.synchronize()
            lat.append(time.perf_counter() - t0)
            t_int.append(ev[0].elapsed_time(ev[1]))
            t_ray.append(ev[1].elapsed_time(ev[2]))
            iters.append(res.total_iters)
            est.append(pose)
            if args.dump:
                diag.append((st, res.inliers, torch.isfinite(Vd[..., 0]).float().mean().item()))
            if args.verbose and (i < 40 or i % 25 == 0):
                cov = torch.isfinite(Vd[..., 0]).float().mean().item()
                print(f"frame {i} status {st} iters {res.total_iters} inliers {res.inliers} "
                      f"err {1e3 * np.linalg.norm(pose[:3, 3] - gt[i][:3, 3]):.1f} mm "
                      f"rot {math.degrees(rot_angle(pose[:3, :3] @ gt[i][:3, :3].T)):.2f} deg "
                      f"step {1e3 * np.linalg.norm(gt[i][:3, 3] - gt[i - 1][:3, 3]):.1f} mm "
                      f"raycast coverage {cov:.2f}", file=sys.stderr)
        wall = time.perf_counter() - t_start
    finally:
        for t in trk:
            kf.kf_track_destroy(t)
        kf.kf_volume_destroy(vol)
    err = [float(np.linalg.norm(e[:3, 3] - g[:3, 3])) for e, g in zip(est, gt)]
    rot = [math.degrees(rot_angle(e[:3, :3] @ g[:3, :3].T)) for e, g in zip(est, gt)]
    if args.dump:
        np.savez(args.dump, est=np.array(est), gt=np.array(gt[:n]), priors=np.array(priors[:n]),
                 diag=np.array(diag, np.float64))
    lat_ms = 1e3 * np.array(lat[3:])
    print(json.dumps({"experiment": "kinectfusion_loop", "frames": n, "data": "synthetic",
                      "outliers": args.outliers, "holes": args.holes, "precision": args.precision,
                      "volume": {"res": 512, "side_m": 6.6, "mu_m": 0.05}, "lambda": args.lam,
                      "map_poses": args.map_poses,
                      "caps": list(CAPS),
                      "frame_latency_ms": {"p50": float(np.percentile(lat_ms, 50)),
                                           "p99": float(np.percentile(lat_ms, 99))},
                      "frames_per_s": (n - 1) / wall,
                      "latency_includes": "set-model (raycast maps) + queueing the next frame's upload and "
                                          "front end on the other tracker + align + integrate + raycast; "
                                          "this frame's front end ran during the previous frame",
                      "integrate_ms_median": float(np.median(t_int)),
                      "raycast_ms_median": float(np.median(t_ray)),
                      "mean_iters": float(np.mean(iters)), "ate_m": math.sqrt(float(np.mean(np.square(err)))),
                      "final_err_m": err[-1], "final_rot_err_deg": rot[-1]}))
    return 0


def trajectory_experiment(args):
    """Long-trajectory form (frame-to-model tracking, synthetic): a smooth
    640x480 path at 30 Hz in a 6 x 6 x 3 m room, IMU priors with white noise
    and bias drift, 15 % outliers and 5 % holes; each frame is aligned to the
    model rendered at the previous ESTIMATED pose (the stand-in for the
    raycast of the reconstruction), one frame per call as a live tracker
    would. Reports the per-frame latency of set-frame + set-model + align on
    the host clock (p50 / p99) and the ATE. One JSON line."""
    import concurrent.futures as cf
    import multiprocessing as mp
    from synth import scenes as S
    n = args.frames
    rng = S.rng_for(5, 1)
    gt = S.trajectory(n, rng)
    priors = S.imu_priors(gt, rng)
    jobs = [(i, gt[i], 180203980 + 500 + i, args.outliers, args.holes) for i in range(1, n)]
    with cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1),
                                mp_context=mp.get_context("spawn")) as ex:
        depths = dict(ex.map(_traj_depth, jobs))
    import torch
    import paper_1802_03980_gb300 as kf
    kf.build()
    torch.cuda.synchronize()
    scene, K = S.room_6x6x3(), S.kinect_intrinsics()
    Kt = K.as_tuple()
    p = kf.kf_default_params()
    for i, c in enumerate(CAPS):
        p.max_iters[i] = c
    p.precision = kf.KF_FP16 if args.precision == "fp16" else kf.KF_FP32
    if args.model == "tsdf":
        depths[0] = _traj_depth((0, gt[0], 180203980 + 500, args.outliers, args.holes))[1]
        return _kinectfusion_loop(args, kf, torch, p, gt, priors, depths, K)
    # two trackers on two streams, frames in page-locked memory: frame i + 1's
    # upload (copy engine) and front end are queued on the other tracker
    # before frame i is aligned, as a streaming tracker overlaps them
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    trk = [kf.kf_track_create(p, W, H, st.cuda_stream) for st in streams]
    pinned = {i: torch.from_numpy(np.ascontiguousarray(depths[i], np.float32)).pin_memory() for i in depths}
    est, lat, render_s, iters = [gt[0].copy()], [], 0.0, []
    try:
        kf.kf_set_frame(trk[1], pinned[1].data_ptr(), Kt, kf.KF_FRAME_HOST_COPY_ENGINE)
        for i in range(1, n):
            cur, nxt = trk[i % 2], trk[(i + 1) % 2]
            r0 = time.perf_counter()
            mv, mn = S.render_model(scene, est[-1], K)
            render_s += time.perf_counter() - r0
            # the model maps live on the device, as a raycast of the
            # reconstruction would leave them
            mvd = torch.from_numpy(np.ascontiguousarray(mv)).cuda()
            mnd = torch.from_numpy(np.ascontiguousarray(mn)).cuda()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            kf.kf_set_model(cur, mvd.data_ptr(), mnd.data_ptr(), est[-1], Kt, True)
            if i + 1 < n:
                kf.kf_set_frame(nxt, pinned[i + 1].data_ptr(), Kt, kf.KF_FRAME_HOST_COPY_ENGINE)
            st, pose, res = kf.kf_align(cur, priors[i], est[-1], args.lam)
            lat.append(time.perf_counter() - t0)
            iters.append(res.total_iters)
            est.append(pose)
    finally:
        for t in trk:
            kf.kf_track_destroy(t)
    err = [float(np.linalg.norm(e[:3, 3] - g[:3, 3])) for e, g in zip(est, gt)]
    if args.dump:
        np.savez(args.dump, est=np.array(est), gt=np.array(gt[:n]), priors=np.array(priors[:n]))
    ate = math.sqrt(float(np.mean(np.square(err))))
    lat_ms = 1e3 * np.array(lat[3:])  # the first calls build the tracker's plan
    print(json.dumps({"experiment": "long_trajectory", "frames": n, "data": "synthetic",
                      "outliers": args.outliers, "holes": args.holes,
                      "lambda": args.lam, "caps": list(CAPS),
                      "latency_ms": {"p50": float(np.percentile(lat_ms, 50)),
                                     "p99": float(np.percentile(lat_ms, 99)),
                                     "mean": float(lat_ms.mean())},
                      "frames_per_s": 1000.0 / float(lat_ms.mean()),
                      "precision": args.precision,
                      "latency_includes": "set-model (device maps) + queueing the next frame's upload and "
                                          "front end on the other tracker + align; this frame's front end "
                                          "ran while the previous frame aligned",
                      "mean_iters": float(np.mean(iters)), "ate_m": ate, "final_err_m": err[-1],
                      "cpu_model_render_s": render_s}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--pairs", type=int, default=256,
                    help="independent 640x480 frame pairs per step (per rank; kinect640 workload)")
    ap.add_argument("--workload", choices=["kinect640", "batch64"], default="kinect640",
                    help="kinect640: the metric's workload; batch64: 64 mixed-resolution pairs "
                         "(320x240 to 1280x960), split over the ranks")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16"])
    ap.add_argument("--cpu-pairs", type=int, default=20)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ablation", action="store_true")
    ap.add_argument("--no-precision-form", action="store_true")
    ap.add_argument("--experiment", choices=["angular", "trajectory", "frontend"], default=None,
                    help="run a method experiment instead of the benchmark (one JSON line)")
    ap.add_argument("--frames", type=int, default=300, help="trajectory experiment length")
    ap.add_argument("--verbose", action="store_true", help="experiments: per-frame diagnostics on stderr")
    ap.add_argument("--dump", default="", help="trajectory: save poses (and per-frame diagnostics) to this .npz")
    ap.add_argument("--lam", type=float, default=5.0, help="trajectory: orientation prior weight (0: no prior)")
    ap.add_argument("--map-poses", choices=["est", "gt"], default="est",
                    help="trajectory --model tsdf: fuse and raycast at the estimated (est) or true (gt) poses")
    ap.add_argument("--outliers", type=float, default=0.15, help="trajectory: uniform-depth outlier fraction")
    ap.add_argument("--holes", type=float, default=0.05, help="trajectory: missing-depth fraction")
    ap.add_argument("--model", choices=["render", "tsdf"], default="render",
                    help="trajectory experiment: model rendered at the estimate, or the fused TSDF map")
    ap.add_argument("--normals", choices=["cross", "integral"], default="cross",
                    help="frontend experiment: cross-product or integral-image normals")
    args = ap.parse_args()
    if args.experiment == "frontend":
        return frontend_experiment(args)
    if args.experiment == "angular":
        return angular_experiment(args)
    if args.experiment == "trajectory":
        return trajectory_experiment(args)
    if args.warmup < 3 and args.impl == "gb300":
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)
    return gb300_arm(args)


if __name__ == "__main__":
    sys.exit(main())
