#!/usr/bin/env python
"""Tracked + fused frames/s of the pose search and fusion hot path.

Workload: a 30 Hz synthetic trajectory of 640x480 depth frames (f = 525,
c = (319.5, 239.5), noise sigma = 0.0012 z^2) through an analytic two-room
scene held in a 512^3 TSDF at 1 cm (truncation 3 cm, f32 tsdf + f32 weight);
every frame runs the randomized pose search (3072 particles x 20 iterations
over all valid points, advantage-set update) from a ground-truth relative
pose perturbed by 3 deg / 3 cm, then fuses the frame.  One step = one frame.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

value      frames/s with every depth frame resident in HBM (CUDA events around
           K back-to-back device-resident frames; no host round trip).
e2e        the same frames through the host API (pinned depth H2D, pose and
           stats D2H per frame), wall clock.
roofline   of the dominant kernel (the fitness gather-reduce), from CUDA
           events around each of its launches during the timed region.
Multi-GPU: the path does not shard within a frame; N ranks run N independent
sequences (replicas) and value = all frames / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tracked+fused frames/s (640x480, 512^3 TSDF); point-particle samples/s vs plain FP32"
K_PARTICLES = 3072
N_ITERS = 20
# FP32 work of one sample (one point under one particle): transform 9 FMA,
# fractional cell coordinates 3 subtractions, 7 linear interpolations
# (1 subtraction + 1 FMA each), |.| accumulation 1 add; FMA counted as 2.
FLOP_PER_SAMPLE = 9 * 2 + 3 + 7 * 3 + 1
GATHER_BYTES_PER_SAMPLE = 8 * 4  # eight f32 nodes
# Bytes of the cell record one sample reads: the eight corners of its cell,
# as float (f32 storage) or as stored (the 16- and 8-bit records lanes on
# points read; with a full view lanes on particles read the 32-byte float
# record).
RECORD_BYTES = {"f32": 32, "f16": 16, "bf16": 16, "fp8": 8}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variant", type=int, default=0, help="fitness kernel: 0 encoded (default), 1 plain")
    ap.add_argument("--update-mode", type=int, default=0)
    ap.add_argument("--compose-mode", type=int, default=1)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--tsdf-dtype", default="f32", choices=["f32", "f16", "bf16", "fp8"],
                    help="storage type of the TSDF and its cell view (arithmetic stays f32); "
                         "fp8 = e4m3 holding 256 x the value")
    ap.add_argument("--weight-u8", action="store_true", help="store fusion weights as uint8")
    ap.add_argument("--search-dtype", default="same", choices=["same", "f16", "bf16", "fp8"],
                    help="storage of the cell view the search reads: the tsdf's (same), or a narrow search view "
                         "of the float master grid, rounded once per refresh (fusion stays float)")
    ap.add_argument("--cell-view", type=int, default=0, choices=[-1, 0, 1, 2],
                    help="cell view of the volumes: 0 automatic, 1 full, 2 narrow records only, -1 none")
    ap.add_argument("--schedule", default="fixed", choices=["fixed", "paper"],
                    help="fixed: 3072 particles x 20 iterations over all points (the benchmark configuration); "
                         "paper: particles alternating 1024/3072/10240 with points decimated 1/8, 1/16, 1/32")
    ap.add_argument("--frame-step", type=int, default=1,
                    help="process every n-th frame of the trajectory (frames in between dropped)")
    ap.add_argument("--polish", type=int, default=0,
                    help="Gauss-Newton polish steps (pf_polish) after each frame's search, before fusion")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-frames", type=int, default=2,
                    help="frames 1..n of the device pass re-run by the FP64 oracle (the same closed loop on the "
                         "host: its own fusion and poses); the bench line reports the position differences and "
                         "both trajectories' errors against ground truth (0: skip)")
    ap.add_argument("--ref-particles", type=int, default=192,
                    help="particles per reference-arm step (a bounded slice of one iteration)")
    ap.add_argument("--kernel", default=None,
                    choices=["fitness", "integrate", "align", "batch", "room64", "precision", "probe"],
                    help="time one kernel on the multiroom volume instead of the frame loop (profiling); "
                         "align: loss + pose and node gradients of 64 320x240 frames against a 256^3 volume, "
                         "and the 10-step polish; batch: 32 sequences of mixed camera and volume size stepped "
                         "together (pf_batch, CUDA graph) against the same sequences one after another; room64: "
                         "the single-frame room workload (160x120, 64^3 at 5 cm, 1024 particles x 10 iterations, "
                         "seeds 0-9) with each layout, and the oracle on the host; precision: 640x480 into 768^3 at "
                         "8 mm with f32 / f16 / bf16 tsdf and uint8 weights -- fusion at the true poses (TSDF "
                         "deviation from the f32 volume) and tracking (frames/s, ATE), over --steps frames")
    ap.add_argument("--frames", type=int, default=300,
                    help="--kernel precision: length of the multiroom trajectory (30 Hz); --steps + 1 frames of it "
                         "are used")
    ap.add_argument("--vs-oracle", type=int, default=0,
                    help="--kernel precision: compare with the FP64 oracle instead of the f32 volume -- fusion of "
                         "--steps + 1 frames at the true poses (TSDF RMS / max per storage type against the oracle's "
                         "FP64 grid), then this many frames tracked once each on every storage type and by the "
                         "oracle on its grid (per-frame pose difference)")
    ap.add_argument("--fusion-only", action="store_true",
                    help="--kernel precision: fuse every frame at its true pose and report the storage deviation "
                         "only (no tracking pass)")
    ap.add_argument("--spread", type=float, default=3.0,
                    help="--kernel fitness: poses perturbed up to this many degrees and centimetres")
    ap.add_argument("--reps", type=int, default=3, help="--kernel: timed launches after one warm-up launch")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------

def _render(args):
    import synth
    n_frames, seed, f, step = args
    seq = synth.multiroom_sequence(n_frames, seed)
    return seq.depth(f * step), seq.relative_init(f * step, step) if f > 0 else np.eye(4)


def render_frames(n_needed: int, seed: int, step: int = 1):
    """Depth frames 0, step, ..., (n_needed-1) step and the perturbed relative
    poses between consecutive ones, rendered in a spawn pool (started before
    any CUDA call)."""
    import multiprocessing as mp

    import synth
    seq = synth.multiroom_sequence(300, seed)
    jobs = [(300, seed, f, step) for f in range(n_needed)]
    workers = max(1, min(len(jobs), (os.cpu_count() or 2) - 1, 16))
    if workers > 1:
        with mp.get_context("spawn").Pool(workers) as pool:
            out = pool.map(_render, jobs)
    else:
        out = [_render(j) for j in jobs]
    depths = [o[0] for o in out]
    rels = [o[1] for o in out]
    return seq, depths, rels


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, val in zip(names, r[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max([num(r[3]) for r in rows if num(r[3]) is not None], default=None)}


# ---------------------------------------------------------------------------
# the oracle on the host cores
# ---------------------------------------------------------------------------

def oracle_sample(seq, depths, rels, compose_mode: int, n_particles: int, repeats: int = 1):
    """Oracle timing on a bounded sample of the workload: fuse frame 0 (not
    timed), then time `repeats` evaluations of `n_particles` particles of one
    search iteration of frame 1 over all its points, and the fusion of frame 1.
    Returns (frames/s extrapolated to 3072 particles x 20 iterations + fusion,
    description, cores, per-repeat timings)."""
    import oracle
    import synth
    oracle.build()
    grid, intr = seq.grid, seq.intr
    vol = oracle.Volume(grid)
    oracle.integrate(vol, depths[0], intr, seq.gt[0])
    P0 = seq.gt[0] @ rels[1]
    pts = oracle.backproject(depths[1], intr)
    templ = synth.templates(K_PARTICLES, 0)
    T = oracle.particles(templ, K_PARTICLES, P0, 10.0, 10.0, compose_mode)
    times = []
    for r in range(repeats):
        lo = (r * n_particles) % K_PARTICLES
        sel = T[lo:lo + n_particles]
        t0 = time.perf_counter()
        oracle.fitness(vol, pts, sel)
        times.append(time.perf_counter() - t0)
    vol2 = oracle.Volume(grid, vol.tsdf.copy(), vol.weight.copy())
    t0 = time.perf_counter()
    oracle.integrate(vol2, depths[1], intr, P0)
    t_int = time.perf_counter() - t0
    t_particle = float(np.median(times)) / n_particles
    t_frame = N_ITERS * (K_PARTICLES + 1) * t_particle + t_int
    desc = (f"oracle (C, FP64, OpenMP): fusion of frame 0 untimed; timed {repeats}x fitness of {n_particles} "
            f"particles over all {pts.shape[0]} points of frame 1 and one 512^3 fusion; per-frame time "
            f"extrapolated to {N_ITERS} x ({K_PARTICLES}+1) particle evaluations + 1 fusion")
    return 1.0 / t_frame, desc, oracle.num_threads(), times, t_int, pts.shape[0]


# ---------------------------------------------------------------------------
# ranks (replicas: one independent sequence per GPU, no data-path collective)
# ---------------------------------------------------------------------------

def world_info():
    """(world size, rank, local rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_seed(base_seed: int, rank: int) -> int:
    """Each rank tracks its own sequence (different noise and perturbations)."""
    return base_seed + rank


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The largest of the ranks' values (the job's time is the slowest rank's)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / (ms_max / 1e3)


def oracle_closed_loop(seq, depths, rels, gt, poses, args, n: int) -> dict:
    """The FP64 oracle re-runs frames 1..n of the device pass's loop on the
    host (fusion of frame 0 at its true pose, then per frame the search from
    P_(t-1) P_(t,t-1) and fusion at the pose found): the GPU's positions
    against the oracle's, and both trajectories' errors against ground
    truth over those frames."""
    import oracle
    import synth
    f32 = lambda v: float(np.float32(v))
    intr, grid = seq.intr, seq.grid
    ointr = synth.Intrinsics(intr.width, intr.height, f32(intr.fx), f32(intr.fy), f32(intr.cx), f32(intr.cy),
                             f32(intr.depth_min), f32(intr.depth_max))
    ogrid = synth.Grid(grid.nx, grid.ny, grid.nz, f32(grid.voxel_size), f32(grid.trunc),
                       tuple(f32(o) for o in grid.origin))
    prm = oracle.TrackParams(n_iters=N_ITERS, k_sched=(K_PARTICLES,) * 3, decim_sched=(1, 1, 1), s0_deg=10.0,
                             s0_cm=10.0, beta=0.1, update_mode=args.update_mode, compose_mode=args.compose_mode,
                             min_valid_frac=0.05)
    templ = synth.templates(K_PARTICLES, args.seed)
    t0 = time.perf_counter()
    vol = oracle.Volume(ogrid)
    oracle.integrate(vol, depths[0], ointr, gt[0])
    P = gt[0]
    diff, e_gpu, e_orc = [], [], []
    for f in range(1, n + 1):
        P = oracle.track(vol, depths[f], ointr, templ, P @ rels[f], prm).pose
        oracle.integrate(vol, depths[f], ointr, P)
        diff.append(float(np.linalg.norm(poses[f][:3, 3] - P[:3, 3])))
        e_gpu.append(float(np.linalg.norm(poses[f][:3, 3] - gt[f][:3, 3])))
        e_orc.append(float(np.linalg.norm(P[:3, 3] - gt[f][:3, 3])))
    rms = lambda e: 100 * float(np.sqrt(np.mean(np.square(e))))
    return {"frames": n, "position_diff_mm": [1e3 * d for d in diff], "ate_cm_gpu": rms(e_gpu),
            "ate_cm_oracle": rms(e_orc), "oracle_threads": oracle.num_threads(),
            "seconds": time.perf_counter() - t0}


def run_reference(args):
    """The oracle (plain C, FP64) as the reference arm.  One step is one timed
    slice of a frame's work: the fitness of --ref-particles particles over all
    points of frame 1.  A frame is 20 x 3073 particle evaluations plus one
    fusion, so a step covers a fraction phi of a frame (phi = the slice's time
    over the frame time that the slice and the timed fusion extrapolate to);
    value = phi / (seconds per step) frames/s and ms_per_step is the slice's
    measured time, so steps x ms_per_step is the time the arm really ran."""
    world, rank, _ = world_info()
    if rank != 0:
        return 0
    steps, warm = max(1, args.steps), max(0, args.warmup)
    seq, depths, rels = render_frames(2, args.seed)
    fps, desc, cores, times, t_int, npts = oracle_sample(seq, depths, rels, args.compose_mode, args.ref_particles,
                                                         repeats=steps + warm)
    times = times[warm:]
    t_step = float(np.mean(times))
    t_particle = t_step / args.ref_particles
    t_frame = N_ITERS * (K_PARTICLES + 1) * t_particle + t_int
    frames_per_step = t_step / t_frame
    value = frames_per_step / t_step
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": 1e3 * t_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args),
        "step": {"work": f"fitness of {args.ref_particles} particles (10 deg / 10 cm spread) over all {npts} "
                         f"points of frame 1", "frames_per_step": frames_per_step,
                 "frame_ms_extrapolated": 1e3 * t_frame, "fusion_ms": 1e3 * t_int,
                 "note": "value = frames_per_step / step time; a frame = 20 x 3073 particle evaluations + 1 "
                         "fusion (fusion timed once, outside the steps)"},
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": cores, "kind": "oracle",
                         "sample": desc.replace(f"timed {steps + warm}x", f"timed {steps}x (after {warm} warm-up)")},
        "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "samples_per_s": npts / t_particle,
    }
    print(json.dumps(line))
    return 0


def storage_desc(args) -> str:
    view = {0: "", 1: ", full cell view", 2: ", narrow cell view", -1: ", no cell view"}[int(getattr(args, "cell_view", 0))]
    sv = getattr(args, "search_dtype", "same")
    search = "" if sv == "same" else f", {sv} search view of the float grid"
    return (f"{getattr(args, 'tsdf_dtype', 'f32')} tsdf + {'u8' if getattr(args, 'weight_u8', False) else 'f32'} "
            f"weight{view}{search}")


def search_dtype(args) -> str:
    """Storage type of the records the search reads."""
    sv = getattr(args, "search_dtype", "same")
    return args.tsdf_dtype if sv == "same" else sv


def new_volume(pf, grid, args):
    codes = {"f32": pf.PF_F32, "f16": pf.PF_F16, "bf16": pf.PF_BF16, "fp8": pf.PF_FP8E4M3}
    sv = getattr(args, "search_dtype", "same")
    return pf.Volume.from_grid(grid, tsdf_dtype=codes[args.tsdf_dtype], weight_u8=int(args.weight_u8),
                               cell_view=int(getattr(args, "cell_view", 0)),
                               search_dtype=pf.PF_F32 if sv == "same" else codes[sv])


def schedule(args):
    """(k_sched, decim_sched, k_max) of the search."""
    if getattr(args, "schedule", "fixed") == "paper":
        return (1024, 3072, 10240), (8, 16, 32), 10240
    return (K_PARTICLES,) * 3, (1, 1, 1), K_PARTICLES


def workload_config(args) -> dict:
    paper = getattr(args, "schedule", "fixed") == "paper"
    step = getattr(args, "frame_step", 1)
    search = ("3072 particles x 20 iterations over all points" if not paper else
              "20 iterations, particles 1024/3072/10240 with points decimated 1/8, 1/16, 1/32 (paper schedule)")
    drop = "" if step == 1 else f", every {step}th frame (the others dropped)"
    polish = getattr(args, "polish", 0)
    if polish:
        drop += f", {polish}-step Gauss-Newton polish after each search"
    k_sched, d_sched, _ = schedule(args)
    return {
        "workload": f"multiroom: 640x480 depth, 512^3 TSDF @ 1 cm (tau 3 cm, {storage_desc(args)}), "
                    f"{search}, then fusion{drop}",
        "resolution": "640x480", "volume": "512^3", "voxel_m": 0.01, "trunc_m": 0.03,
        "particles": list(k_sched) if paper else K_PARTICLES, "iterations": N_ITERS,
        "decimation": list(d_sched) if paper else 1, "frame_step": step,
        "update": "advantage-set mean" if args.update_mode == 0 else "best particle",
        "compose": "about the world origin" if args.compose_mode == 0 else "about the camera centre",
        "init_perturbation": "3 deg / 3 cm", "seed": args.seed,
        "l2": "inputs larger than L2: fusion reads and writes the 1.07 GB volume frustum every step",
        "parallelism": f"replicas x{args.gpus}",
        "storage": storage_desc(args),
    }


# ---------------------------------------------------------------------------
# our path
# ---------------------------------------------------------------------------

def run_ours(args):
    world, rank, local = world_info()
    W, K = max(3, args.warmup), max(1, args.steps)
    n_frames = 1 + W + K
    step = max(1, args.frame_step)
    if (n_frames - 1) * step > 299:
        raise SystemExit("(--warmup + --steps) x --frame-step must be <= 299 (300-frame trajectory)")
    seq, depths, rels = render_frames(n_frames, replica_seed(args.seed, rank), step)
    gt = [seq.gt[f * step] for f in range(n_frames)]  # the processed frames

    import torch
    import paper_2509_24236_gb300 as pf
    from paper_2509_24236_gb300 import build as pfbuild
    pfbuild.build()
    pf.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    intr, grid = seq.intr, seq.grid
    stream = torch.cuda.current_stream()
    vol = new_volume(pf, grid, args)
    vol.set_fitness_variant(args.variant)
    k_sched, d_sched, k_max = schedule(args)
    vol.reserve(intr.width * intr.height, k_max)
    import synth
    templ = torch.from_numpy(synth.templates(k_max, args.seed)).to(dev)
    params = pf.track_params(templ, n_iters=N_ITERS, k_sched=k_sched, decim_sched=d_sched,
                             update_mode=args.update_mode, compose_mode=args.compose_mode, min_valid_frac=0.05)
    depth_dev = [torch.from_numpy(d).to(dev) for d in depths]
    rel_dev = torch.from_numpy(np.stack([r.reshape(16) for r in rels])).to(dev)
    init_dev = torch.zeros((n_frames, 16), dtype=torch.float64, device=dev)
    pose_dev = torch.zeros((n_frames, 16), dtype=torch.float64, device=dev)
    stats_sz = __import__("ctypes").sizeof(pf.pf_track_stats)
    stats_dev = torch.zeros((n_frames, stats_sz), dtype=torch.uint8, device=dev)
    pose_dev[0] = torch.from_numpy(gt[0].reshape(16)).to(dev)

    polish_pts = torch.empty((intr.width * intr.height, 4), dtype=torch.float32, device=dev)
    polish_n = torch.zeros(1, dtype=torch.int32, device=dev)

    def device_frame(f):
        pf.pf_pose_compose(pose_dev[f - 1], rel_dev[f], init_dev[f])
        vol.track_frame_async(depth_dev[f], intr, params, init_dev[f], pose_dev[f], stats_dev[f])
        if args.polish > 0:
            pf.pf_backproject(depth_dev[f], intr, polish_pts, polish_n)
            vol.polish(polish_pts, pose_dev[f], steps=args.polish, n_dev=polish_n)
        vol.integrate_async(depth_dev[f], intr, pose_dev[f])

    # ---- device-resident pass -------------------------------------------
    vol.integrate_async(depth_dev[0], intr, pose_dev[0])
    for f in range(1, W + 1):
        device_frame(f)
    torch.cuda.synchronize()
    barrier()
    pf.pf_set_kernel_timing(True)
    for cls in ("fitness", "fitness1", "integrate", "refresh", "backproject"):
        pf.pf_kernel_timing(cls)
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = pf.pf_launch_count()
    torch.cuda.synchronize()
    barrier()
    t_begin = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_begin.record(stream)
    for f in range(W + 1, W + K + 1):
        device_frame(f)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = pf.pf_launch_count() - launches0
    clock_info = clocks.stop()
    ms = t_begin.elapsed_time(t_end)
    kt = {cls: pf.pf_kernel_timing(cls) for cls in ("fitness", "fitness1", "integrate", "refresh", "backproject")}
    pf.pf_set_kernel_timing(False)
    ms_max = max_over_ranks(ms, dist, dev)

    # per-frame statistics of the timed frames
    stats_host = stats_dev.cpu().numpy()
    samples = 0
    n_lost = 0
    for f in range(W + 1, W + K + 1):
        st = pf.pf_track_stats.from_buffer_copy(stats_host[f].tobytes()).to_dict()
        samples += int(np.sum(st["k_used"].astype(np.int64) * st["n_eval"]))
        n_lost += int(st["status"] == pf.PF_ERR_TRACK_LOST)
    poses = pose_dev.cpu().numpy().reshape(-1, 4, 4)
    err = [np.linalg.norm(poses[f][:3, 3] - gt[f][:3, 3]) for f in range(1, W + K + 1)]
    ate_cm = 100.0 * float(np.sqrt(np.mean(np.square(err))))

    # ---- fitness kernel throughput, encoded vs plain layout --------------
    # (the plain layout exists for float storage only)
    vs_plain = fitness_vs_plain(pf, vol, depth_dev[W + 1], intr, poses[W], dev) if args.tsdf_dtype == "f32" \
        and not args.weight_u8 and getattr(args, "search_dtype", "same") == "same" else None

    # ---- end-to-end pass through the host API ----------------------------
    e2e = None
    if not args.no_e2e and not args.polish:  # (the host-API pass has no polish step)
        e2e = run_e2e(pf, vol, gt, depths, rels, intr, params, W, K, dev)

    value = job_rate(K, world, ms_max)
    fit_ms, fit_n = kt["fitness"]
    fit_avg_ms = fit_ms / max(1, fit_n)
    samples_per_launch = samples / max(1, fit_n)
    achieved_tflops = samples_per_launch * FLOP_PER_SAMPLE / (fit_avg_ms / 1e3) / 1e12
    peak_tflops = fp32_peak_tflops()
    ceilings = gather_ceilings(pf, dev)
    rec_bytes = RECORD_BYTES[search_dtype(args)]
    achieved_gbs = samples_per_launch * rec_bytes / (fit_avg_ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic", "config": workload_config(args),
        "samples_per_s": samples / (ms / 1e3),
        "fitness_samples_per_s": samples / (fit_ms / 1e3) if fit_ms > 0 else None,
        "fitness_vs_plain": vs_plain,
        "roofline": {"bound": "l2_gather", "kernel": "fitness_kernel<search>", "achieved": achieved_gbs,
                     "peak": ceilings["l2_gbs"], "unit": "GB/s", "frac": achieved_gbs / ceilings["l2_gbs"],
                     "traffic": committed_traffic(), "bytes_per_sample": rec_bytes,
                     "peak_source": "measured in this run: pf_gather_probe mode 0 (L2 -> SM, 1 KiB per warp-load "
                                    f"at random positions in a {ceilings['mib']} MiB L2-resident buffer, L1 "
                                    "bypassed), CUDA events",
                     "scattered_gather_gbs": ceilings["scattered_gbs"],
                     "frac_of_scattered_gather": achieved_gbs / ceilings["scattered_gbs"],
                     "hbm_gbs_measured": measured_peak("hbm_gbs"),
                     "avg_launch_ms": fit_avg_ms, "launches": fit_n, "samples_per_launch": samples_per_launch,
                     "alu": {"achieved": achieved_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                             "frac": achieved_tflops / peak_tflops, "flop_per_sample": FLOP_PER_SAMPLE,
                             "peak_source": "FP32 lanes x clock: 152 SMs x 128 x 2 flop x 2070 MHz (derived)"},
                     "binding_unit": committed_l1_pipe()},
        "kernel_ms": {cls: {"total_ms": v[0], "launches": v[1]} for cls, v in kt.items()},
        "gpu_launches": launches,
        "clocks": clock_info,
        "ate_cm": ate_cm, "frames_lost": n_lost,
        "e2e": e2e,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.schedule == "fixed":
        fps, desc, cores, times, t_int, npts = oracle_sample(seq, depths, rels, args.compose_mode, 1024, repeats=1)
        line["cpu_baseline"] = {"value": fps, "unit": "frames/s", "cores": cores, "kind": "oracle", "sample": desc}
    if rank == 0 and args.oracle_frames > 0 and args.schedule == "fixed" and step == 1 and not args.polish \
            and args.tsdf_dtype == "f32" and not args.weight_u8 and args.search_dtype == "same":
        line["oracle_closed_loop"] = oracle_closed_loop(seq, depths, rels, gt, poses, args,
                                                        min(args.oracle_frames, W + K))
    if rank == 0:
        print(json.dumps(line))
    vol.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def fitness_source_sha(sources=None) -> str:
    """sha256 prefix of the fitness kernel's device code, as recorded beside
    the committed ncu capture: csrc/track.cu from the fitness section
    (FIT_THREADS) to the end of fitness_kernel_batch, followed by the value
    encoding and storage conversions of csrc/pf_internal.cuh (up to its
    volume and workspace section).  Host-side edits elsewhere in those files
    leave it unchanged.  `sources` = (track.cu text, pf_internal.cuh text)."""
    import hashlib
    if sources is None:
        csrc = os.path.join(ROOT, "paper_2509_24236_gb300", "csrc")
        sources = tuple(open(os.path.join(csrc, n)).read() for n in ("track.cu", "pf_internal.cuh"))
    track, internal = sources
    a = track.index("constexpr int FIT_THREADS")
    b = track.index("__global__ void track_begin_kernel")
    c = internal.index("// Volume and workspace")
    h = hashlib.sha256()
    h.update(track[a:b].encode())
    h.update(internal[:c].encode())
    return h.hexdigest()[:16]


def committed_traffic():
    """DRAM bytes per launch of the fitness kernel from the committed ncu
    summary, or None when the kernel's sources (csrc/track.cu and
    csrc/pf_internal.cuh) have changed since that capture."""
    import re
    path = os.path.join(ROOT, "profiles", "fitness_kernel_multiroom.md")
    try:
        text = open(path).read()
        sha = fitness_source_sha()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*(\d+)", text)
    h = re.search(r"kernel_source_sha256_prefix:\s*([0-9a-f]+)", text)
    if not m or not h or h.group(1) != sha:
        return None
    return int(m.group(1))


def committed_l1_pipe():
    """The unit that bounds the fitness kernel, from the same committed ncu
    summary: L1 data-pipe wavefronts as a fraction of peak in each lane
    mapping (None when the kernel's sources have changed since)."""
    import re
    path = os.path.join(ROOT, "profiles", "fitness_kernel_multiroom.md")
    try:
        text = open(path).read()
        sha = fitness_source_sha()
    except OSError:
        return None
    h = re.search(r"kernel_source_sha256_prefix:\s*([0-9a-f]+)", text)
    a = re.search(r"l1_data_pipe_frac_points_on_lanes:\s*([0-9.]+)", text)
    b = re.search(r"l1_data_pipe_frac_particles_on_lanes:\s*([0-9.]+)", text)
    if not h or h.group(1) != sha or not a or not b:
        return None
    return {"unit": "L1 data-pipe wavefronts, fraction of peak (ncu)", "points_on_lanes": float(a.group(1)),
            "particles_on_lanes": float(b.group(1)), "source": "profiles/fitness_kernel_multiroom.md"}


def fp32_peak_tflops() -> float:
    return 152 * 128 * 2 * 2.070e9 / 1e12


def measured_peak(key: str):
    """A figure of the measured MEASURED_PEAKS.json, or None."""
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get(key)
    except (OSError, ValueError):
        return None


def gather_ceilings(pf, dev, mib: int = 48, loads: int = 2048, reps: int = 5) -> dict:
    """GB/s of the two memory ceilings of the fitness kernel, measured with
    pf_gather_probe over an L2-resident buffer of `mib` MiB: mode 0 (L2 -> SM,
    coalesced 1 KiB warp-loads, L1 bypassed) and mode 1 (one 32-byte record
    per lane at random positions).  CUDA events on the current stream, after
    one warm-up launch that also brings the buffer into L2."""
    import torch
    n_rec = mib * (1 << 20) // 32
    buf = torch.rand(n_rec * 8, device=dev)
    threads = pf.pf_gather_probe(buf, n_rec, 0, loads)
    out = torch.empty(threads, device=dev)
    res = {"mib": mib, "loads_per_thread": loads, "threads": threads}
    for mode, key in ((0, "l2_gbs"), (1, "scattered_gbs")):
        pf.pf_gather_probe(buf, n_rec, mode, loads, out)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            pf.pf_gather_probe(buf, n_rec, mode, loads, out)
        b.record()
        torch.cuda.synchronize()
        res[key] = reps * threads * loads * 32 / (a.elapsed_time(b) / 1e3) / 1e9
    return res


def fitness_vs_plain(pf, vol, depth, intr, pose, dev, reps=5):
    """Samples/s of pf_fitness with 3072 poses around `pose` over one frame's
    points: the encoded (default) kernel against the plain f32 one."""
    import torch

    import synth
    pts, n = pf.backproject(depth, intr)
    n = int(n.item())
    pts = pts[:n].contiguous()
    u = synth.uniform01(77, 2 * K_PARTICLES)
    P = np.stack([(pose @ synth.perturbation(78, k, 10.0 * u[2 * k], 10.0 * u[2 * k + 1]))[:3, :4].reshape(12)
                  for k in range(K_PARTICLES)]).astype(np.float32)
    poses = torch.from_numpy(P).to(dev)
    out = {}
    for variant, name in ((0, "encoded"), (1, "plain")):
        vol.set_fitness_variant(variant)
        vol.fitness(pts, poses)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            vol.fitness(pts, poses)
        b.record()
        torch.cuda.synchronize()
        out[name] = reps * n * K_PARTICLES / (a.elapsed_time(b) / 1e3)
    vol.set_fitness_variant(0)
    out["ratio"] = out["encoded"] / out["plain"]
    out["points"] = n
    return out


def run_e2e(pf, vol, gt, depths, rels, intr, params, W, K, dev):
    """The frames end to end through the C ABI from host memory: per frame
    the depth image and the relative pose go host -> device (pinned), the
    initial pose P_t^(0) = P_(t-1) P_(t,t-1) is formed by pf_pose_compose,
    pf_track_frame_async searches and pf_integrate_async fuses, and the pose
    and the search record come back device -> host before the next frame
    (wall clock)."""
    import ctypes

    import torch
    vol.reset()
    pinned = [torch.from_numpy(d).pin_memory() for d in depths]
    rel_host = [torch.from_numpy(np.ascontiguousarray(r.reshape(16))).pin_memory() for r in rels]
    stats_sz = ctypes.sizeof(pf.pf_track_stats)
    pose_host = torch.empty(16, dtype=torch.float64).pin_memory()
    stats_host = torch.empty(stats_sz, dtype=torch.uint8).pin_memory()
    buf = torch.empty_like(pinned[0], device=dev)
    rel_dev = torch.empty(16, dtype=torch.float64, device=dev)
    # the pose of frame f lives in pose_dev[f % 2] (the previous one in the other slot)
    pose_dev = torch.empty((2, 16), dtype=torch.float64, device=dev)
    pose_dev[0].copy_(torch.from_numpy(gt[0].reshape(16).copy()))
    init_dev = torch.empty(16, dtype=torch.float64, device=dev)
    stats_dev = torch.empty(stats_sz, dtype=torch.uint8, device=dev)
    buf.copy_(pinned[0], non_blocking=True)
    vol.integrate_async(buf, intr, pose_dev[0])

    def frame(f):
        prev_dev, out_dev = pose_dev[(f - 1) % 2], pose_dev[f % 2]
        buf.copy_(pinned[f], non_blocking=True)
        rel_dev.copy_(rel_host[f], non_blocking=True)
        pf.pf_pose_compose(prev_dev, rel_dev, init_dev)
        vol.track_frame_async(buf, intr, params, init_dev, out_dev, stats_dev)
        vol.integrate_async(buf, intr, out_dev)
        pose_host.copy_(out_dev, non_blocking=True)
        stats_host.copy_(stats_dev, non_blocking=True)
        torch.cuda.current_stream().synchronize()   # the host reads the frame's result

    for f in range(1, W + 1):
        frame(f)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for f in range(W + 1, W + K + 1):
        frame(f)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    h2d = depths[0].nbytes + 16 * 8
    d2h = 16 * 8 + stats_sz
    return {"value": K / dt, "unit": "frames/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "path": "pinned host depth + relative pose -> pf_pose_compose -> pf_track_frame_async -> "
                    "pf_integrate_async -> pose + search record to host, synchronised per frame"}


def run_kernel(args):
    """One kernel on the multiroom workload, for profiling: the volume fuses
    frames 0 and 2 at their true poses; `fitness` evaluates 3072 poses within
    --spread degrees / centimetres of frame 1's pose over all of frame 1's
    points (pf_fitness, --variant); `integrate` fuses frame 1 (pf_integrate).
    Prints one JSON line with the mean CUDA-event time per launch."""
    import torch

    import paper_2509_24236_gb300 as pf
    import synth
    from paper_2509_24236_gb300 import build as pfbuild
    seq, depths, rels = render_frames(3, args.seed)
    pfbuild.build()
    pf.load()
    dev = torch.device("cuda", 0)
    intr = seq.intr
    vol = new_volume(pf, seq.grid, args)
    for f in (0, 2):
        vol.integrate(torch.from_numpy(depths[f]).to(dev), intr, seq.gt[f])
    depth1 = torch.from_numpy(depths[1]).to(dev)
    if args.kernel == "fitness":
        pts, n = pf.backproject(depth1, intr)
        n = int(n.item())
        pts = pts[:n].contiguous()
        u = synth.uniform01(77, 2 * K_PARTICLES)
        P = seq.gt[1]
        poses = np.stack([P[:3, :4].reshape(12)] + [
            (P @ synth.perturbation(78, k, args.spread * u[2 * k], args.spread * u[2 * k + 1]))[:3, :4].reshape(12)
            for k in range(1, K_PARTICLES)]).astype(np.float32)
        poses = torch.from_numpy(poses).to(dev)
        vol.set_fitness_variant(args.variant)
        launch = lambda: vol.fitness(pts, poses)
        units, unit = n * K_PARTICLES, "samples"
    else:
        launch = lambda: vol.integrate(depth1, intr, seq.gt[1])
        units, unit = seq.grid.n_nodes, "nodes"
    launch()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.reps):
        launch()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.reps
    print(json.dumps({"kernel": args.kernel, "variant": args.variant, "spread": args.spread, "reps": args.reps,
                      "storage": storage_desc(args),
                      "ms_per_launch": ms, f"{unit}_per_s": units / (ms / 1e3)}))
    vol.close()
    return 0


ALIGN_FRAMES = 64


def align_sequence(seed: int):
    """64 frames of 320x240 against a 256^3 TSDF at 2 cm (tau 6 cm) of the
    multiroom scene, every 4th frame of its trajectory."""
    import synth
    intr = synth.Intrinsics(320, 240, 262.5, 262.5, 159.5, 119.5, 0.1, 8.0)
    grid = synth.Grid(256, 256, 256, 0.02, 0.06, (0.0, 0.0, 0.0))
    return synth.multiroom_sequence(300, seed, grid=grid, intr=intr)


def _render_align(args):
    seed, f = args
    return align_sequence(seed).depth(f)


def run_align(args):
    """Alignment loss with pose and node-value gradients (pf_align_loss) for
    64 frames at once, each at its true pose perturbed by 1 deg / 1 cm, and
    the 10-step Gauss-Newton polish (pf_polish) of one frame.  Prints one
    JSON line."""
    import multiprocessing as mp
    frames = [4 * i for i in range(ALIGN_FRAMES)]
    with mp.get_context("spawn").Pool(max(1, min(16, (os.cpu_count() or 2) - 1))) as pool:
        depths = pool.map(_render_align, [(args.seed, f) for f in frames])
    import torch

    import paper_2509_24236_gb300 as pf
    import synth
    from paper_2509_24236_gb300 import build as pfbuild
    pfbuild.build()
    pf.load()
    dev = torch.device("cuda", 0)
    seq = align_sequence(args.seed)
    intr = seq.intr
    vol = new_volume(pf, seq.grid, args)
    n_max = intr.width * intr.height
    pts = torch.empty((ALIGN_FRAMES, n_max, 4), dtype=torch.float32, device=dev)
    counts = torch.empty(ALIGN_FRAMES, dtype=torch.int32, device=dev)
    for i, f in enumerate(frames):
        d = torch.from_numpy(depths[i]).to(dev)
        vol.integrate(d, intr, seq.gt[f])
        p, n = pf.backproject(d, intr)
        pts[i].copy_(p)
        counts[i:i + 1].copy_(n)
    u = synth.uniform01(91, 2 * ALIGN_FRAMES)
    poses = torch.from_numpy(np.stack([seq.gt[f] @ synth.perturbation(92, i, 1.0 * u[2 * i], 1.0 * u[2 * i + 1])
                                       for i, f in enumerate(frames)])).to(dev)
    call = lambda: vol.align_loss(pts, poses, counts=counts, grad_xi=True, grad_tsdf=True)
    call()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.reps):
        loss, cnt, gx, gv = call()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.reps
    samples = int(counts.sum().item())
    # polish of frame 0 from its perturbed pose
    pose0 = poses[0].reshape(16).clone()
    vol.polish(pts[0], pose0, steps=10, n_dev=counts[0:1])
    torch.cuda.synchronize()
    a.record()
    for _ in range(args.reps):
        pose0.copy_(poses[0].reshape(16))
        trace, acc = vol.polish(pts[0], pose0, steps=10, n_dev=counts[0:1])
    b.record()
    torch.cuda.synchronize()
    ms_polish = a.elapsed_time(b) / args.reps
    P0 = pose0.cpu().numpy().reshape(4, 4)
    print(json.dumps({
        "kernel": "align", "storage": storage_desc(args), "frames": ALIGN_FRAMES, "resolution": "320x240",
        "volume": "256^3 @ 2 cm, tau 6 cm", "reps": args.reps, "points": samples,
        "ms_per_call": ms, "frames_per_s": ALIGN_FRAMES / (ms / 1e3), "samples_per_s": samples / (ms / 1e3),
        "valid_fraction": float(cnt.sum().item()) / max(1, samples),
        "polish": {"steps": 10, "ms": ms_polish, "accepted": int(acc.item()),
                   "objective_first_last": [float(trace[0]), float(trace[-1])],
                   "trans_err_cm_before_after": [100 * float(np.linalg.norm(poses[0].cpu().numpy()[:3, 3] -
                                                                           seq.gt[frames[0]][:3, 3])),
                                                 100 * float(np.linalg.norm(P0[:3, 3] - seq.gt[frames[0]][:3, 3]))]},
    }))
    vol.close()
    return 0


BATCH_SEQS = 32
BATCH_RES = [(160, 120), (320, 240), (640, 480)]
BATCH_GRIDS = [128, 256, 384]          # nodes per axis over the 5.12 m multiroom cube (4, 2, 1.33 cm)
BATCH_K = [1024, 2048, 3072, 4096]


def batch_sequence(res: int, grid: int, seed: int):
    import synth
    w, h = BATCH_RES[res]
    f = 525.0 * w / 640.0
    intr = synth.Intrinsics(w, h, f, f, (w - 1) / 2.0, (h - 1) / 2.0, 0.1, 8.0)
    vs = 5.12 / BATCH_GRIDS[grid]
    g = synth.Grid(BATCH_GRIDS[grid], BATCH_GRIDS[grid], BATCH_GRIDS[grid], vs, 3.0 * vs, (0.0, 0.0, 0.0))
    return synth.multiroom_sequence(300, seed, grid=g, intr=intr)


def _render_batch(args):
    res, f, seed = args
    return batch_sequence(res, 0, seed).depth(f)


def run_batch(args):
    """C4-style batch: 32 sequences, camera i % 3 of 160x120 / 320x240 /
    640x480, volume (i // 3) % 3 of 128^3 / 256^3 / 384^3 over the same
    5.12 m scene, K = 1024 / 2048 / 3072 / 4096 by i % 4, 20 iterations over
    all points.  Frames 1..W+S of the multiroom trajectory (one rendering per
    camera size, shared by the sequences of that size); frame 0 is fused at
    its true pose.  Times S steps of all sequences (0) one sequence after
    another with the plain float form (float volumes, fitness layout 1), (a)
    one after another with the chosen storage and the default kernel
    (pf_track_frame_async + pf_integrate_async), (b) as a batch with direct
    launches, (c) as a batch replaying a CUDA graph.  Inputs are
    resident on the device.  Prints one JSON line (aggregate frames/s)."""
    import multiprocessing as mp
    W, S = max(1, args.warmup), max(1, args.steps)
    n_frames = 1 + W + S
    jobs = [(r, f, args.seed) for r in range(len(BATCH_RES)) for f in range(n_frames)]
    with mp.get_context("spawn").Pool(max(1, min(16, (os.cpu_count() or 2) - 1))) as pool:
        rendered = pool.map(_render_batch, jobs)
    import torch

    import paper_2509_24236_gb300 as pf
    import synth
    from paper_2509_24236_gb300 import build as pfbuild
    pfbuild.build()
    pf.load()
    dev = torch.device("cuda", 0)
    depth = {}
    for (r, f, _), d in zip(jobs, rendered):
        depth[r, f] = torch.from_numpy(d).to(dev)
    seqs, vols, params = [], [], []
    templ = torch.from_numpy(synth.templates(max(BATCH_K), args.seed)).to(dev)
    for i in range(BATCH_SEQS):
        r, g, K = i % 3, (i // 3) % 3, BATCH_K[i % 4]
        seq = batch_sequence(r, g, args.seed + i)
        seqs.append((r, seq))
        vols.append(new_volume(pf, seq.grid, args))
        params.append(pf.track_params(templ, n_iters=N_ITERS, k_sched=(K, K, K), decim_sched=(1, 1, 1),
                                      update_mode=args.update_mode, compose_mode=args.compose_mode,
                                      min_valid_frac=0.05))
    rels = [torch.from_numpy(np.stack([seq.relative_init(f).reshape(16) if f else np.eye(4).reshape(16)
                                       for f in range(n_frames)])).to(dev) for _, seq in seqs]

    def timed(run_steps):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        run_steps()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    pose = torch.zeros((BATCH_SEQS, n_frames, 16), dtype=torch.float64, device=dev)
    init = torch.zeros_like(pose)

    def sequential(vs):
        """Frames 1..W warm-up, then S timed frames of every sequence, one
        sequence after another (pf_track_frame_async + pf_integrate_async)."""
        for v in vs:
            v.reserve(640 * 480, max(BATCH_K))
        for i, (r, seq) in enumerate(seqs):
            pose[i, 0] = torch.from_numpy(seq.gt[0].reshape(16)).to(dev)
            vs[i].integrate_async(depth[r, 0], seq.intr, pose[i, 0])

        def frames(f0, f1):
            for f in range(f0, f1):
                for i, (r, seq) in enumerate(seqs):
                    pf.pf_pose_compose(pose[i, f - 1], rels[i][f], init[i, f])
                    vs[i].track_frame_async(depth[r, f], seq.intr, params[i], init[i, f], pose[i, f])
                    vs[i].integrate_async(depth[r, f], seq.intr, pose[i, f])

        frames(1, W + 1)
        return timed(lambda: frames(W + 1, W + S + 1))

    # (0) the plain float form (float storage, fitness layout 1), one after another
    plain = []
    for _, seq in seqs:
        v = pf.Volume.from_grid(seq.grid)
        v.set_fitness_variant(1)
        plain.append(v)
    ms_plain = sequential(plain)
    for v in plain:
        v.close()
    del plain
    # (a) this storage and the default kernel, one after another
    ms_seq = sequential(vols)
    pose_seq = pose.cpu().numpy()

    # (b), (c) batches, from the same start
    out = {}
    for use_graph in (False, True):
        for v in vols:
            v.reset()
        batch = pf.Batch(vols, [seq.intr for _, seq in seqs], params, use_graph=use_graph)
        for i, (r, seq) in enumerate(seqs):
            batch.pose[i].copy_(torch.from_numpy(seq.gt[0]).to(dev))
            batch.depth[i].copy_(depth[r, 0])
        batch.fuse()

        def load(f):
            for i, (r, seq) in enumerate(seqs):
                batch.depth[i].copy_(depth[r, f])
                batch.rel[i].copy_(rels[i][f].reshape(4, 4))

        if use_graph:
            load(1)
            out["points_per_block"] = batch.autotune()
            out["mapping_threshold"] = batch.tuning()["mapping_threshold"]
        for f in range(1, W + 1):
            load(f)
            batch.step()
            if f == 1:
                p1 = np.stack([batch.pose[i].cpu().numpy().reshape(16) for i in range(BATCH_SEQS)])
                out["pose_diff_1_m"] = float(np.max(np.abs(p1[:, 3::4][:, :3] - pose_seq[:, 1, 3::4][:, :3])))
        times = []
        for f in range(W + 1, W + S + 1):
            load(f)  # input copies stay outside the timed region
            times.append(timed(batch.step))
        out["graph" if use_graph else "direct"] = sum(times)
        poses_b = np.stack([batch.pose[i].cpu().numpy().reshape(16) for i in range(BATCH_SEQS)])
        out["pose_diff_m"] = float(np.max(np.abs(poses_b[:, 3::4][:, :3] - pose_seq[:, W + S, 3::4][:, :3])))
        batch.close()
    frames = BATCH_SEQS * S
    print(json.dumps({
        "kernel": "batch", "sequences": BATCH_SEQS, "steps": S, "warmup": W, "storage": storage_desc(args),
        "mix": "cameras 160x120/320x240/640x480 by i%3, volumes 128^3/256^3/384^3 over 5.12 m by (i//3)%3, "
               "K 1024/2048/3072/4096 by i%4, 20 iterations, all points",
        "frames_per_s_plain_f32_sequential": frames / (ms_plain / 1e3),
        "frames_per_s_sequential": frames / (ms_seq / 1e3),
        "frames_per_s_batch_direct": frames / (out["direct"] / 1e3),
        "frames_per_s_batch_graph": frames / (out["graph"] / 1e3),
        "speedup_graph_vs_sequential": ms_seq / out["graph"],
        "speedup_graph_vs_plain_f32_sequential": ms_plain / out["graph"],
        "points_per_block": out.get("points_per_block"),
        "mapping_threshold_voxels": out.get("mapping_threshold"),
        "max_position_difference_batch_vs_sequential_after_first_step_m": out.get("pose_diff_1_m"),
        "max_final_position_difference_batch_vs_sequential_m": out["pose_diff_m"],
    }))
    for v in vols:
        v.close()
    return 0


def run_room64(args):
    """The single-frame room workload: 160x120 depth (1 mm noise) of the
    3.2 m room with three spheres, a 64^3 TSDF at 5 cm (tau 15 cm) of the
    analytic scene, initial pose 5 deg / 5 cm off, 1024 particles x 10
    iterations over all points, mean update; seeds 0-9.  Device ms per frame
    (pf_track_frame_async, CUDA events over --reps repeats) for the default
    kernel and the plain float layout, pose error, and the oracle's time for
    the same frames on the host cores."""
    import time

    import synth
    seeds = list(range(10))
    frames = [synth.room64_frame(sd) for sd in seeds]
    vols_np = [synth.analytic_tsdf(sc, synth.ROOM64_GRID, hole_bricks=0.0, seed=sd) for (sc, fr), sd in
               zip(frames, seeds)]
    K, I = 1024, 10
    templ_np = synth.templates(K, 0)
    # oracle on the host (before any CUDA call)
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    for (sc, fr), (t, w) in zip(frames, vols_np):
        ov = oracle.Volume(synth.ROOM64_GRID, t, w)
        oracle.track(ov, fr.depth, synth.ROOM64_INTR, templ_np, fr.init_pose,
                     oracle.TrackParams(n_iters=I, k_sched=(K, K, K), decim_sched=(1, 1, 1), update_mode=0,
                                        compose_mode=args.compose_mode))
    oracle_ms = (time.perf_counter() - t0) / len(seeds) * 1e3
    import torch

    import paper_2509_24236_gb300 as pf
    from paper_2509_24236_gb300 import build as pfbuild
    pfbuild.build()
    pf.load()
    dev = torch.device("cuda", 0)
    templ = torch.from_numpy(templ_np).to(dev)
    params = pf.track_params(templ, n_iters=I, k_sched=(K, K, K), decim_sched=(1, 1, 1), update_mode=0,
                             compose_mode=args.compose_mode)
    out = {}
    for name, variant in (("default", 0), ("plain_f32", 1)):
        ms, errs = [], []
        for (sc, fr), (t, w) in zip(frames, vols_np):
            vol = pf.Volume.from_grid(synth.ROOM64_GRID)
            vol.upload(t, w)
            vol.set_fitness_variant(variant)
            vol.reserve(synth.ROOM64_INTR.width * synth.ROOM64_INTR.height, K)
            d = torch.from_numpy(fr.depth).to(dev)
            init = torch.from_numpy(fr.init_pose.reshape(16)).to(dev)
            outp = torch.zeros(16, dtype=torch.float64, device=dev)
            vol.track_frame_async(d, synth.ROOM64_INTR, params, init, outp)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(args.reps):
                vol.track_frame_async(d, synth.ROOM64_INTR, params, init, outp)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b) / args.reps)
            P = outp.cpu().numpy().reshape(4, 4)
            errs.append(float(np.linalg.norm(P[:3, 3] - fr.gt_pose[:3, 3])))
            vol.close()
        out[name] = {"ms_per_frame": float(np.mean(ms)), "frames_per_s": 1e3 / float(np.mean(ms)),
                     "samples_per_s": K * I * 19200 / (float(np.mean(ms)) / 1e3),
                     "pose_error_cm_mean": 100 * float(np.mean(errs)), "pose_error_cm_max": 100 * float(np.max(errs))}
    print(json.dumps({
        "kernel": "room64", "workload": "160x120, 64^3 TSDF @ 5 cm (tau 15 cm), 1024 particles x 10 iterations, "
                                        "all points, mean update, init 5 deg / 5 cm, seeds 0-9",
        "reps": args.reps, "gpu": out,
        "cpu_baseline": {"ms_per_frame": oracle_ms, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": "the same 10 frames, full search"},
    }))
    return 0


def run_precision_oracle(args):
    """Reduced-precision storage at scale against the FP64 oracle (640x480
    into 768^3 at 8 mm, tau 2.4 cm, uint8 weights, automatic cell view).
    (a) Fusion of frames 0..--steps at their true poses by every storage type
    and by the oracle in FP64: RMS and max of the stored tsdf minus the
    oracle's over nodes observed by both, and whether the weights agree.
    (b) For frames 1..--vs-oracle: the search of frame f (3072 particles x 20
    iterations from P_(f-1) P_(f,f-1), perturbed) on each storage type's grid
    and on the oracle's, both fused at the true poses of frames 0..f-1, then
    frame f fused at its true pose: the per-frame difference of the found
    poses from the oracle's, and each one's error against ground truth."""
    import synth
    import oracle
    n = max(2, args.steps + 1)
    n_pose = max(0, min(args.vs_oracle, n - 1))
    n_traj = max(args.frames, n)
    grid = synth.Grid(768, 768, 768, 0.008, 0.024, (-0.5, -0.5, -0.5))
    seq = synth.multiroom_sequence(n_traj, args.seed, grid=grid)
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(max(1, min(16, (os.cpu_count() or 2) - 1))) as pool:
        out = pool.map(_render, [(n_traj, args.seed, f, 1) for f in range(n)])
    depths = [o[0] for o in out]
    rels = [o[1] for o in out]
    import torch

    import paper_2509_24236_gb300 as pf
    from paper_2509_24236_gb300 import build as pfbuild
    pfbuild.build()
    pf.load()
    dev = torch.device("cuda", 0)
    intr = seq.intr
    f32 = lambda v: float(np.float32(v))
    ointr = synth.Intrinsics(intr.width, intr.height, f32(intr.fx), f32(intr.fy), f32(intr.cx), f32(intr.cy),
                             f32(intr.depth_min), f32(intr.depth_max))
    ogrid = synth.Grid(grid.nx, grid.ny, grid.nz, f32(grid.voxel_size), f32(grid.trunc),
                       tuple(f32(o) for o in grid.origin))
    templ_np = synth.templates(K_PARTICLES, args.seed)
    templ = torch.from_numpy(templ_np).to(dev)
    params = pf.track_params(templ, n_iters=N_ITERS, k_sched=(K_PARTICLES,) * 3, decim_sched=(1, 1, 1),
                             update_mode=args.update_mode, compose_mode=args.compose_mode, min_valid_frac=0.05)
    oparams = oracle.TrackParams(n_iters=N_ITERS, k_sched=(K_PARTICLES,) * 3, decim_sched=(1, 1, 1), s0_deg=10.0,
                                 s0_cm=10.0, beta=0.1, update_mode=args.update_mode, compose_mode=args.compose_mode,
                                 min_valid_frac=0.05)
    dd = [torch.from_numpy(d).to(dev) for d in depths]
    codes = {"f32": pf.PF_F32, "f16": pf.PF_F16, "bf16": pf.PF_BF16, "fp8": pf.PF_FP8E4M3}
    # the oracle: per-frame searches on its grid fused at the true poses, then the remaining fusions
    ovol = oracle.Volume(ogrid)
    opose = {}
    # nodes whose update, in some frame, sits within 1e-3 px of a pixel-rounding
    # boundary or 1e-6 m of the -tau cut or the camera plane: FP32 and FP64 may
    # take either side there (another pixel's depth), so they are counted apart
    amb = np.zeros(grid.n_nodes, dtype=bool)
    t0 = time.perf_counter()
    for f in range(n):
        if 1 <= f <= n_pose:
            opose[f] = oracle.track(ovol, depths[f], ointr, templ_np, seq.gt[f - 1] @ rels[f], oparams).pose
        amb |= oracle.integrate(ovol, depths[f], ointr, seq.gt[f], ambiguity=True).astype(bool)
    t_oracle = time.perf_counter() - t0
    res = {}
    configs = (("f32", "f32"), ("f32", "f16"), ("f32", "bf16"), ("f16", "f16"), ("bf16", "bf16"), ("fp8", "fp8"))
    for name, search in configs:
        vol = pf.Volume.from_grid(grid, tsdf_dtype=codes[name], weight_u8=1,
                                  search_dtype=pf.PF_F32 if search == name else codes[search])
        vol.reserve(intr.width * intr.height, K_PARTICLES)
        r = {"frames": {}}
        for f in range(n):
            if 1 <= f <= n_pose:
                st, P, _ = vol.track_frame(dd[f], intr, params, seq.gt[f - 1] @ rels[f])
                r["frames"][f] = {
                    "diff_to_oracle_mm": 1e3 * float(np.linalg.norm(P[:3, 3] - opose[f][:3, 3])),
                    "diff_to_oracle_rad": float(np.arccos(np.clip((np.trace(P[:3, :3].T @ opose[f][:3, :3]) - 1) / 2,
                                                                  -1, 1))),
                    "err_to_truth_cm": 100 * float(np.linalg.norm(P[:3, 3] - seq.gt[f][:3, 3])),
                    "oracle_err_to_truth_cm": 100 * float(np.linalg.norm(opose[f][:3, 3] - seq.gt[f][:3, 3]))}
            vol.integrate(dd[f], intr, seq.gt[f])
        t, w = vol.download()
        both = (w > 0) & (ovol.weight > 0)
        clean = both & ~amb
        diff = np.abs(t[clean].astype(np.float64) - ovol.tsdf[clean])
        diff_all = np.abs(t[both].astype(np.float64) - ovol.tsdf[both])
        r["tsdf_vs_oracle"] = {"rms": float(np.sqrt(np.mean(diff ** 2))), "max": float(diff.max()),
                               "nodes": int(clean.sum()),
                               "weights_equal": bool(np.array_equal(w[~amb].astype(np.float64), ovol.weight[~amb])),
                               "ambiguous_nodes": int((both & amb).sum()),
                               "rms_all_nodes": float(np.sqrt(np.mean(diff_all ** 2)))}
        res[name + "+u8" + ("" if search == name else f" ({search} search view)")] = r
        del t, w, diff, diff_all, both, clean
        vol.close()
    print(json.dumps({"kernel": "precision", "against": "FP64 oracle",
                      "workload": f"multiroom 640x480 ({n_traj}-frame trajectory), {n} frames fused at their true "
                                  f"poses, frames 1-{n_pose} each searched once (3072 particles x 20 iterations) on "
                                  "grids fused at the true poses of the frames before; 768^3 TSDF @ 8 mm (tau 2.4 cm), "
                                  "uint8 weights", "oracle_seconds": t_oracle, "oracle_threads": oracle.num_threads(),
                      "results": res}))
    return 0


def run_precision(args):
    """Reduced-precision storage at scale: the multiroom trajectory (frames
    0..--steps) at 640x480 into a 768^3 TSDF at 8 mm (tau 2.4 cm), tsdf in
    f32 / f16 / bf16 / scaled e4m3 with uint8 weights; the narrow storages
    with the automatic (full) cell view and with the narrow one.  Per run:
    the view taken and the device bytes per node.  (a) Fusion of every frame
    at its true pose: RMS and max deviation of the narrow volumes from the
    f32 one over nodes observed in both (the f32 fusion matches the FP64
    oracle to 1e-5, see the parity tests).  (b) Tracking + fusion of the same
    frames: frames/s (CUDA events), ATE and the largest distance between each
    trajectory and the f32 one."""
    import synth
    n = max(2, args.steps + 1)
    n_traj = max(args.frames, n)
    grid = synth.Grid(768, 768, 768, 0.008, 0.024, (-0.5, -0.5, -0.5))
    seq = synth.multiroom_sequence(n_traj, args.seed, grid=grid)
    depths, rels = [], []
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(max(1, min(16, (os.cpu_count() or 2) - 1))) as pool:
        out = pool.map(_render, [(n_traj, args.seed, f, 1) for f in range(n)])
    depths = [o[0] for o in out]
    rels = [o[1] for o in out]
    import torch

    import paper_2509_24236_gb300 as pf
    from paper_2509_24236_gb300 import build as pfbuild
    pfbuild.build()
    pf.load()
    dev = torch.device("cuda", 0)
    intr = seq.intr
    dd = [torch.from_numpy(d).to(dev) for d in depths]
    codes = {"f32": pf.PF_F32, "f16": pf.PF_F16, "bf16": pf.PF_BF16, "fp8": pf.PF_FP8E4M3}
    templ = torch.from_numpy(synth.templates(K_PARTICLES, args.seed)).to(dev)
    params = pf.track_params(templ, n_iters=N_ITERS, k_sched=(K_PARTICLES,) * 3, decim_sched=(1, 1, 1),
                             update_mode=args.update_mode, compose_mode=args.compose_mode, min_valid_frac=0.05)
    rel_dev = torch.from_numpy(np.stack([r.reshape(16) for r in rels])).to(dev)
    res, ref_tsdf, ref_w, ref_traj = {}, None, None, None
    configs = (("f32", 0, None), ("f32", 0, "f16"), ("f32", 0, "bf16"), ("f16", 0, None), ("f16", 2, None),
               ("bf16", 0, None), ("bf16", 2, None), ("fp8", 0, None), ("fp8", 2, None))
    for name, view, search in configs:
        vol = pf.Volume.from_grid(grid, tsdf_dtype=codes[name], weight_u8=1, cell_view=view,
                                  search_dtype=codes[search] if search else pf.PF_F32)
        info = vol.info()
        for f in range(n):
            vol.integrate(dd[f], intr, seq.gt[f])
        t, w = vol.download()
        r = {"cell_view": {1: "full", 2: "narrow", -1: "none"}[info["cell_view"]],
             "storage_bytes_per_node": info["storage_bytes"] / grid.n_nodes}
        if ref_tsdf is None:
            ref_tsdf, ref_w = t, w
        else:
            both = (w > 0) & (ref_w > 0)
            diff = np.abs(t[both].astype(np.float64) - ref_tsdf[both])
            r["tsdf_vs_f32"] = {"rms": float(np.sqrt(np.mean(diff ** 2))), "max": float(diff.max()),
                                "nodes": int(both.sum()), "weights_equal": bool(np.array_equal(w, ref_w))}
        del t, w
        key = name + "+u8" + ("+narrow" if view == 2 else "") + (f" ({search} search view)" if search else "")
        if args.fusion_only:
            res[key] = r
            vol.close()
            continue
        vol.reset()
        pose = torch.zeros((n, 16), dtype=torch.float64, device=dev)
        init = torch.zeros_like(pose)
        pose[0] = torch.from_numpy(seq.gt[0].reshape(16)).to(dev)
        vol.reserve(intr.width * intr.height, K_PARTICLES)
        vol.integrate_async(dd[0], intr, pose[0])
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for f in range(1, n):
            pf.pf_pose_compose(pose[f - 1], rel_dev[f], init[f])
            vol.track_frame_async(dd[f], intr, params, init[f], pose[f])
            vol.integrate_async(dd[f], intr, pose[f])
        b.record()
        torch.cuda.synchronize()
        P = pose.cpu().numpy().reshape(-1, 4, 4)
        err = np.array([np.linalg.norm(P[f][:3, 3] - seq.gt[f][:3, 3]) for f in range(1, n)])
        r.update({"frames_per_s": (n - 1) / (a.elapsed_time(b) / 1e3), "ate_cm": 100 * float(np.sqrt(np.mean(err ** 2)))})
        if ref_traj is None:
            ref_traj = P
        else:
            r["max_position_difference_to_f32_cm"] = 100 * float(np.max(np.linalg.norm(P[1:, :3, 3] - ref_traj[1:, :3, 3],
                                                                                       axis=1)))
        res[key] = r
        vol.close()
    what = f"{n} frames fused at their true poses" if args.fusion_only else f"{n - 1} tracked frames"
    print(json.dumps({"kernel": "precision", "workload": f"multiroom 640x480 ({n_traj}-frame trajectory), {what}, "
                      "768^3 TSDF @ 8 mm (tau 2.4 cm), 3072 particles x 20 iterations, uint8 weights",
                      "results": res}))
    return 0


def run_probe(args):
    """The fitness kernel's memory ceilings (pf_gather_probe) over buffers of
    growing size: L2-resident ones give the L2 -> SM bandwidth (mode 0) and
    the scattered-record gather rate (mode 1); the largest spills to HBM."""
    import torch

    import paper_2509_24236_gb300 as pf
    from paper_2509_24236_gb300 import build as pfbuild
    pfbuild.build()
    pf.load()
    dev = torch.device("cuda", 0)
    rows = []
    for mib in (8, 16, 32, 48, 64, 96, 128, 1024):
        r = gather_ceilings(pf, dev, mib=mib, loads=2048, reps=max(1, args.reps))
        rows.append({"mib": mib, "l2_stream_gbs": r["l2_gbs"], "scattered_gbs": r["scattered_gbs"]})
    print(json.dumps({"kernel": "probe", "threads": r["threads"], "loads_per_thread": 2048, "bytes_per_load": 32,
                      "rows": rows, "hbm_gbs_measured": measured_peak("hbm_gbs")}))
    return 0


def main():
    args = parse()
    if args.kernel == "probe":
        return run_probe(args)
    if args.kernel == "precision":
        return run_precision_oracle(args) if args.vs_oracle > 0 else run_precision(args)
    if args.kernel == "room64":
        return run_room64(args)
    if args.kernel == "batch":
        return run_batch(args)
    if args.kernel == "align":
        return run_align(args)
    if args.kernel:
        return run_kernel(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
