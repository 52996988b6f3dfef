#!/usr/bin/env python
"""Throughput of one IB-LBM time step (arXiv 2206.01683, Sec. III-B) on B300.

Workload: the skinned swimmer in its moving frame -- a 256x128x128 D3Q27
channel (velocity inlet u = 0.02 at -x, outflow at +x, free-slip side walls),
tau = 0.52, a 6000-marker fish of body length 64 on a 5-segment spine driven
by a travelling joint wave, and a seeded frame trajectory (Eq. 3).  One step
= IB interpolation + direct forcing + spreading, fused stream/collide/
boundary, FP64 force/torque/mass reduction; the marker pose of each step is
an input (precomputed, resident in HBM for ``value``).

Prints one JSON line (rank 0).  ``value`` is MLUPS over all ranks with the
inputs resident in HBM; ``e2e`` is the same metric through the C ABI with
the step's marker data copied from pinned host memory and the body force
read back every step.  ``--impl reference`` times the FP64 CPU oracle instead
(the only reference there is; rank 0 only).
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

REPEATS = 5   # timed repetitions of K steps; the median is reported
E2E_WARM = 60  # untimed fg_step_io calls before the end-to-end repetitions
E2E_STEPS = 200  # fg_step_io calls per end-to-end repetition, at least

METRIC = "MLUPS and % HBM roofline per step (FP32 vs FP16-storage vs batched), 1×B300"
OPEN_X = (1, 2, 3, 3, 3, 3)   # inlet, outflow, free-slip walls

# DRAM traffic of the stream-collide kernel per cell update from an ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum divided by the cells of
# the launch; the mean of two launches, one of each sweep direction, or in
# place of an even and an odd step), keyed by the kernel source it was taken
# on, the variant in use, the storage and the population layout, and valid
# only for those.  Swimmer channel, 4,194,304 cells.
NCU_TRAFFIC = {
    # k_stream_collide<StoreF32, false, true>: 440.53 MB read + 401.60 MB written
    ("a8391d8732973f3c32b44a42a94abfa4b32accb5560a824b805624a767a6f2eb", "plain", "f32", "pull"): 200.78,
    # k_stream_collide_staged<StoreF16, 512, 3, false, true>: 220.59 MB read + 174.88 MB written
    ("a8391d8732973f3c32b44a42a94abfa4b32accb5560a824b805624a767a6f2eb", "staged512", "f16", "pull"): 94.29,
    # k_stream_collide_staged<StoreBF16, 512, 3, false, true>: 220.58 MB read + 175.03 MB written
    ("a8391d8732973f3c32b44a42a94abfa4b32accb5560a824b805624a767a6f2eb", "staged512", "bf16", "pull"): 94.32,
    # in place: k_aa_boundary + k_stream_collide_aa<StoreF32, false, true, K>, the mean of an
    # even and an odd step: (13.85 + 439.96 + 379.68 MB + 13.85 + 440.17 + 390.67 MB) / 2
    ("ac85ed78c44d57df172a48785d85a2c587c414341033a1f1697f90ded12e7d7b", "plain", "f32", "aa"): 200.06,
    # the same with StoreF16: (6.94 + 220.47 + 160.58 MB + 6.94 + 220.55 + 164.98 MB) / 2
    ("ac85ed78c44d57df172a48785d85a2c587c414341033a1f1697f90ded12e7d7b", "plain", "f16", "aa"): 93.04,
}


NOMINAL_HBM_GBS = 8000.0   # B300 HBM3e, nominal (context only; the fraction that counts is of measured)


def kernel_source_hash(layout="pull"):
    """sha256 over the sources the stream-collide kernels of a population
    layout are compiled from."""
    h = hashlib.sha256()
    names = ("step_kernels.cuh", "lattice.cuh", "async_copy.cuh") + (("aa_kernels.cuh",) if layout == "aa" else ())
    for name in names:
        h.update(open(os.path.join(ROOT, "paper_2206_01683_b300", "csrc", name), "rb").read())
    return h.hexdigest()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[4:]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for name, flag in zip(names, r[3][1:]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        sm = sorted(r[0] for r in rows)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows),
                "reasons": sorted(reasons)}


# --------------------------------------------------------------- workload

def fish_workload(total_steps, shape=(256, 128, 128), length=64.0, n_markers=6000):
    from paper_2206_01683_b300 import inputs
    fish = inputs.fish_for_grid(shape, length, n_markers)
    traj = inputs.FrameTrajectory(inputs.seed_for(2), inputs.domain_centre(shape))
    X = np.zeros((total_steps, n_markers, 3), np.float32)
    U = np.zeros((total_steps, n_markers, 3), np.float32)
    for n0 in range(0, total_steps, 256):
        ts = np.arange(n0, min(n0 + 256, total_steps))
        X[ts], U[ts] = fish.poses(ts)
    frames = [traj.at(n) for n in range(total_steps)]
    return fish, X, U, np.array(frames)


def _barrier(world):
    import torch
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
        torch.cuda.synchronize()


def _sleep_ahead(stream, ms):
    """A spin kernel on the stream ahead of the start event: the host enqueues
    the timed steps while it runs, so no host launch gap falls inside the
    timed region (the e2e metric keeps the host's time)."""
    import torch
    if ms > 0:
        with torch.cuda.stream(stream):
            torch.cuda._sleep(int(ms * 2.1e6))   # clock cycles, at up to 2.1 GHz


def _ahead_ms(host_ms_per_step, steps):
    """How long the GPU is kept busy before a timed region of `steps` steps:
    1.5 x the host's enqueue time for them (measured on the warm-up steps),
    at least 0.5 ms, at most 200 ms."""
    return min(200.0, max(0.5, 1.5 * host_ms_per_step * steps))


def _warm(fn, steps):
    """Run the warm-up steps; returns the host's enqueue time per step (ms)
    over the second half of them (the first step may run the autotuner)."""
    steps = list(steps)
    half = len(steps) // 2
    for n in steps[:half]:
        fn(n)
    t0 = time.perf_counter()
    for n in steps[half:]:
        fn(n)
    return (time.perf_counter() - t0) * 1e3 / max(len(steps) - half, 1)


def _timed(stream, world, fn, steps, ahead_ms=0.0):
    """Milliseconds for fn(n) over the given step indices, CUDA events on the
    library's stream, barrier + synchronize on both sides."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    _barrier(world)
    _sleep_ahead(stream, ahead_ms)
    e0.record(stream)
    for n in steps:
        fn(n)
    e1.record(stream)
    _barrier(world)
    return e0.elapsed_time(e1)


def job_mlups(world, cells, steps, ms):
    """Whole-job throughput of `world` replicas, each updating `cells` cells
    `steps` times, the job taking `ms` (the slowest rank's time)."""
    return world * cells * steps / (ms * 1e-3) / 1e6


def _max_over_ranks(x, world):
    """Max of x over ranks (the slowest rank sets the job's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def adjoint_form():
    """Cost of the thrust gradient (forward with checkpoints + recompute and
    adjoint backward) on the 128x64x64 channel, one fish of 1500 markers,
    200 steps, checkpoint every 20, as a multiple of the forward."""
    import torch
    from paper_2206_01683_b300 import adjoint, inputs
    cfg = inputs.ADJOINT_CHANNEL
    prob = adjoint.ThrustProblem(cfg["shape"], cfg["tau"], cfg["length"], cfg["n_markers"], cfg["steps"],
                                 checkpoint=cfg["checkpoint"])
    reps = []
    for r in range(5):   # the first repetition warms up
        th = adjoint.default_theta().requires_grad_(True)
        L = adjoint.SwimThrust.apply(th, prob)
        (g,) = torch.autograd.grad(L, th)
        if r > 0:
            reps.append((prob.backward_ms / prob.forward_ms, prob.forward_ms, prob.backward_ms, float(L.detach()),
                         g.detach().numpy().tolist()))
    # the repetition with the median cost multiple (a single one can meet a
    # disturbance on the host)
    _, fwd, bwd, L, g = sorted(reps, key=lambda t: t[0])[len(reps) // 2]
    return {"workload": "adjoint_channel_128x64x64_periodic", "steps": cfg["steps"],
            "checkpoint": cfg["checkpoint"], "markers": cfg["n_markers"],
            "forward_ms": round(fwd, 3), "backward_ms": round(bwd, 3),
            "cost_multiple": round(bwd / fwd, 3), "loss_thrust": L, "grad_norm": float(np.linalg.norm(g)),
            "repetitions": len(reps), "cost_multiple_each": [round(t[0], 3) for t in reps]}


def _kernel_ms(dom, fn, steps):
    """Mean event-timed duration (ms) of each kernel over the given steps."""
    from paper_2206_01683_b300 import fishlbm
    dom.profile(True)
    for n in steps:
        fn(n)
    kms, cnt = dom.profile_read()
    dom.profile(False)
    return [kms[k] / max(cnt[k], 1) for k in range(fishlbm.FG_K_COUNT)]


def _variant_kw(args):
    """Domain options for --variant: autotune (default) or a fixed kernel."""
    if args.variant == "autotune":
        return {"autotune": True}
    return {"variant": args.variant}


def storage_form(storage, shape, tau, u_in, fish, Xd, Ud, dVd, segd, ref, fr, W, K, world, peak, vkw,
                 ib_iters=1, deterministic=False, eq_order=2, layout="pull"):
    """The swimmer-channel step with populations stored as FP16 / BF16 (or
    FP32 with ib_iters direct-forcing passes), in either population layout
    (two buffers, or one updated in place)."""
    import torch
    from paper_2206_01683_b300 import fishlbm
    stream = torch.cuda.Stream()
    dom = fishlbm.Domain([fishlbm.env_desc(shape, tau, OPEN_X, (u_in, 0, 0), 1.0, (u_in, 0, 0))],
                         storage=storage, stream=stream.cuda_stream, ib_iters=ib_iters,
                         deterministic=deterministic, eq_order=eq_order, layout=layout, **vkw)
    dom.set_markers(Xd[0], Ud[0], dVd, segd, n_seg=5, ref=ref)

    def step(n):
        dom.step_markers(Xd[n], Ud[n], [fr[n]])

    hms = _warm(step, range(W))
    ms = _max_over_ranks(_timed(stream, world, step, range(W, W + K), _ahead_ms(hms, K)), world)
    dom.get_body_force_torque()
    k = _kernel_ms(dom, step, range(W + K, W + 2 * K))
    ncell = shape[0] * shape[1] * shape[2]
    gbs = dom.stream_collide_bytes() / (k[1] * 1e-3) / 1e9
    variant = dom.stream_collide_variant()
    # (the captured kernels: second-order equilibrium, this grid; the IB
    # options do not change the stream-collide kernel)
    bpc = (NCU_TRAFFIC.get((kernel_source_hash(layout), variant, storage, layout))
           if eq_order == 2 and tuple(shape) == (256, 128, 128) else None)
    dom.close()
    return {"value": round(world * ncell * K / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS",
            "ms_per_step": round(ms / K, 5), "storage": storage, "kernel_variant": variant,
            "ib_iters": ib_iters, "deterministic": bool(deterministic), "eq_order": eq_order,
            "layout": layout, "population_bytes": (1 if layout == "aa" else 2) * 27 * ncell * (4 if storage == "f32" else 2),
            "roofline": {"bound": "hbm", "kernel": "k_stream_collide_aa" if layout == "aa" else "k_stream_collide",
                         "achieved": round(gbs, 1),
                         "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4),
                         "algorithmic_bytes_per_cell": 216 if storage == "f32" else 108,
                         "traffic": round(bpc * ncell) if bpc else None,
                         "kernel_ms": round(k[1], 5), "ib_ms": round(k[0], 5)}}


def storage_accuracy(storage, shape, tau, u_in, fish, Xd, Ud, dVd, segd, ref, fr, steps, vkw):
    """Velocity rel-L2 of the step with populations stored as `storage`
    against the same steps in FP32 (same inputs, same initial state)."""
    import torch
    from paper_2206_01683_b300 import fishlbm
    us = []
    for st in ("f32", storage):
        dom = fishlbm.Domain([fishlbm.env_desc(shape, tau, OPEN_X, (u_in, 0, 0), 1.0, (u_in, 0, 0))],
                             storage=st, **vkw)
        dom.set_markers(Xd[0], Ud[0], dVd, segd, n_seg=5, ref=ref)
        for n in range(steps):
            dom.step_markers(Xd[n], Ud[n], [fr[n]])
        torch.cuda.synchronize()
        us.append(dom.fields()[1])
        dom.close()
    return float(np.linalg.norm(us[1] - us[0]) / np.linalg.norm(us[0]))


# rel-L2 bars of u and F against the FP64 oracle (frozen in the precision tests)
STORAGE_BAR = {"f16": 2e-3, "bf16": 5e-2}


def school_form(W, K, world, peak, vkw):
    """Two fish in tandem in one 150x50x100 open channel (the paper's
    two-fish schooling domain), one marker set of 2 x 2500 markers with ten
    segments, each fish's torque about its own first joint, in the leader's
    moving frame."""
    import torch
    from paper_2206_01683_b300 import fishlbm, inputs
    cfg = inputs.SCHOOL_CHANNEL
    shape, tau, u_in = cfg["shape"], cfg["tau"], cfg["u_in"]
    school = inputs.School(shape, cfg["length"], cfg["n_markers"], cfg["gap"], cfg["phase_lag"])
    traj = inputs.FrameTrajectory(inputs.seed_for(6), inputs.domain_centre(shape))
    T = W + 2 * K
    X = np.zeros((T, school.n, 3), np.float32)
    U = np.zeros((T, school.n, 3), np.float32)
    fr = []
    for n in range(T):
        X[n], U[n] = school.pose(n)
        fr.append(fishlbm.frame_from_array(traj.at(n)))
    Xd, Ud = torch.from_numpy(X).cuda(), torch.from_numpy(U).cuda()
    dVd = torch.from_numpy(school.dV.astype(np.float32)).cuda()
    segd = torch.from_numpy(school.seg).cuda()
    stream = torch.cuda.Stream()
    dom = fishlbm.Domain([fishlbm.env_desc(shape, tau, OPEN_X, (u_in, 0, 0), 1.0, (u_in, 0, 0))],
                         stream=stream.cuda_stream, **vkw)
    dom.set_markers(Xd[0], Ud[0], dVd, segd, n_seg=school.n_seg, ref=tuple(school.ref))
    dom.set_segment_refs(school.seg_refs)

    def step(n):
        dom.step_markers(Xd[n], Ud[n], [fr[n]])

    hms = _warm(step, range(W))
    ms = _max_over_ranks(_timed(stream, world, step, range(W, W + K), _ahead_ms(hms, K)), world)
    ft = dom.get_body_force_torque()
    k = _kernel_ms(dom, step, range(W + K, W + 2 * K))
    ncell = shape[0] * shape[1] * shape[2]
    gbs = dom.stream_collide_bytes() / (k[1] * 1e-3) / 1e9
    variant = dom.stream_collide_variant()
    dom.close()
    return {"value": round(world * ncell * K / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS",
            "ms_per_step": round(ms / K, 5), "workload": "two_fish_school_150x50x100",
            "markers": int(school.n), "segments": int(school.n_seg), "kernel_variant": variant,
            "leader_fx": round(float(ft[:5, 0].sum()), 8), "follower_fx": round(float(ft[5:10, 0].sum()), 8),
            "roofline": {"bound": "hbm", "kernel": "k_stream_collide", "achieved": round(gbs, 1),
                         "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4),
                         "kernel_ms": round(k[1], 5), "ib_ms": round(k[0], 5)}}


def free_sphere_form(W, K, world, vkw):
    """A free sphere (R = 8, density ratio 1.08, gravity 1e-4 along -z) in a
    128^3 periodic box, two-way coupled every step.  The body update runs on
    the device in the step's own launches (fg_attach_sphere: markers from
    the body state, inner-fluid sums, FP64 Newton-Euler step), so the timed
    steps need no synchronisation; ``host_coupled`` times the same sphere
    advanced on the host (rigid.FreeSphere: the force/torque and the
    inner-fluid momentum read back every step, two synchronisations)."""
    import torch
    from paper_2206_01683_b300 import fishlbm, rigid
    shape = (128, 128, 128)
    ncell = shape[0] * shape[1] * shape[2]
    out = {}
    for mode in ("device", "host"):
        stream = torch.cuda.Stream()
        dom = fishlbm.Domain([fishlbm.env_desc(shape, 0.6)], stream=stream.cuda_stream, **vkw)
        cls = rigid.DeviceFreeSphere if mode == "device" else rigid.FreeSphere
        body = cls(dom, 8.0, (63.5, 63.5, 80.0), 1.08, (0.0, 0.0, -1e-4))
        hms = _warm(lambda n: body.step(), range(W))
        ahead = _ahead_ms(hms, K) if mode == "device" else 0.0
        ms = _max_over_ranks(_timed(stream, world, lambda n: body.step(), range(K), ahead), world)
        r = {"value": round(world * ncell * K / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS",
             "ms_per_step": round(ms / K, 5), "velocity_z": round(float(body.vel[2]), 8),
             "host_syncs_per_step": 0 if mode == "device" else 2}
        if mode == "device":
            out.update(r)
            out.update({"workload": "free_sphere_128cube_R8_ratio1.08", "markers": int(len(body.dirs)),
                        "body_update": "device (fg_attach_sphere)"})
        else:
            out["host_coupled"] = r
        dom.close()
    return out


def large_sphere_form(W, K, world, peak, vkw):
    """The precision workload: a 13,500-marker sphere (R = 32.78, dV = 1)
    translating at 0.05 lu/step through a 384x192x192 periodic box at tau =
    0.56, with populations stored as FP32, FP16 and BF16 (f - w), FP32
    arithmetic; marker poses resident in HBM.  Each storage's MLUPS and
    stream-collide roofline, and its speed-up over the FP32 storage."""
    import torch
    from paper_2206_01683_b300 import fishlbm, inputs
    shape, tau, nm = (384, 192, 192), 0.56, 13500
    centre = (383 / 2 - 48.0, 95.5, 95.5)
    R = (nm / (4 * np.pi)) ** 0.5
    X0, dV = inputs.fibonacci_sphere(nm, R, centre)
    T = W + 2 * K
    U1 = np.array([0.05, 0.0, 0.0])
    X = np.stack([X0 + U1 * n for n in range(T)]).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    Ud = torch.from_numpy(np.tile(U1, (nm, 1)).astype(np.float32)).cuda()
    dVd = torch.from_numpy(dV.astype(np.float32)).cuda()
    ncell = shape[0] * shape[1] * shape[2]
    out = {"workload": "large_sphere_box_384x192x192", "markers": nm,
           "accuracy": "FP64-oracle parity per storage: tests/test_gpu_full_configs.py (bars f32 1e-5, f16 2e-3, "
                       "bf16 5e-2)"}
    for st in ("f32", "f16", "bf16"):
        stream = torch.cuda.Stream()
        dom = fishlbm.Domain([fishlbm.env_desc(shape, tau)], storage=st, stream=stream.cuda_stream, **vkw)
        dom.set_markers(Xd[0], Ud, dVd)

        def step(n):
            dom.step_markers(Xd[n], Ud)

        hms = _warm(step, range(W))
        ms = _max_over_ranks(_timed(stream, world, step, range(W, W + K), _ahead_ms(hms, K)), world)
        dom.get_body_force_torque()
        k = _kernel_ms(dom, step, range(W + K, W + 2 * K))
        gbs = dom.stream_collide_bytes() / (k[1] * 1e-3) / 1e9
        out[st] = {"value": round(world * ncell * K / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS",
                   "ms_per_step": round(ms / K, 5), "kernel_variant": dom.stream_collide_variant(),
                   "roofline": {"bound": "hbm", "kernel": "k_stream_collide", "achieved": round(gbs, 1),
                                "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4),
                                "algorithmic_bytes_per_cell": 216 if st == "f32" else 108,
                                "kernel_ms": round(k[1], 5), "ib_ms": round(k[0], 5)}}
        dom.close()
        del dom
    for st in ("f16", "bf16"):
        out[st]["speedup_vs_f32_storage"] = round(out[st]["value"] / out["f32"]["value"], 3)
    return out


def batched_form(W, K, world, peak, vkw, n_envs=64):
    """n_envs (64) independent single-fish environments, grid sizes drawn by seed from
    {96x64x64, 128x64x64, 160x80x80, 192x96x96}, fish of 0.4 x grid length
    with 1500-4000 markers and its own wave amplitude and frame trajectory,
    all advanced by the same launches: one marker update for all
    environments and one graph replay per step."""
    import torch
    from paper_2206_01683_b300 import fishlbm, inputs
    draws = inputs.batch_envs(n_envs, inputs.seed_for(4))
    descs, fishes, trajs = [], [], []
    for d in draws:
        shape = d["shape"]
        descs.append(fishlbm.env_desc(shape, 0.52, OPEN_X, (0.02, 0, 0), 1.0, (0.02, 0, 0)))
        j = np.arange(1, 5)
        fishes.append(inputs.fish_for_grid(shape, 0.4 * shape[0], d["n_markers"],
                                           amplitudes=d["amplitude"] * j / 4.0))
        trajs.append(inputs.FrameTrajectory(d["frame_seed"], inputs.domain_centre(shape)))
    T = W + 2 * K
    ts = np.arange(T)
    Xs, Us = [], []
    for f in fishes:
        X, U = f.poses(ts)
        Xs.append(X.astype(np.float32))
        Us.append(U.astype(np.float32))
    # every step's markers of all environments, resident in HBM in the compact order
    Xall = torch.from_numpy(np.concatenate(Xs, axis=1)).cuda()
    Uall = torch.from_numpy(np.concatenate(Us, axis=1)).cuda()
    frames = [[fishlbm.frame_from_array(t.at(n)) for t in trajs] for n in range(T)]
    cells = sum(d["shape"][0] * d["shape"][1] * d["shape"][2] for d in draws)

    def run(kw):
        stream = torch.cuda.Stream()
        dom = fishlbm.Domain(descs, stream=stream.cuda_stream, **kw)
        for e, f in enumerate(fishes):
            ref = tuple(float(v) for v in f.joints_rest[0])
            dom.set_markers(torch.from_numpy(Xs[e][0]).cuda(), torch.from_numpy(Us[e][0]).cuda(),
                            torch.from_numpy(f.dV.astype(np.float32)).cuda(), torch.from_numpy(f.seg).cuda(),
                            n_seg=5, ref=ref, env=e)

        def step(n):
            dom.step_markers(Xall[n], Uall[n], frames[n])

        hms = _warm(step, range(W))
        ms = _max_over_ranks(_timed(stream, world, step, range(W, W + K), _ahead_ms(hms, K)), world)
        for e in range(n_envs):
            dom.get_body_force_torque(env=e)
        k = _kernel_ms(dom, step, range(W + K, W + 2 * K))
        gbs = dom.stream_collide_bytes() / (k[1] * 1e-3) / 1e9
        variant = dom.stream_collide_variant()
        dom.close()
        return ms, k, gbs, variant, stream

    ms, k, gbs, variant, stream = run(vkw)
    # the same batch with the fused persistent kernel: one launch per step for
    # the IB phases and stream-collide blocks of all environments
    ms_f, k_f, gbs_f, _, _ = run({"variant": "fused"})

    # the same environments as as many plain FP32 single-environment domains,
    # stepped one after another on the same stream (no batching)
    doms = []
    for e, f in enumerate(fishes):
        de = fishlbm.Domain([descs[e]], stream=stream.cuda_stream, **vkw)
        ref = tuple(float(v) for v in f.joints_rest[0])
        de.set_markers(torch.from_numpy(Xs[e][0]).cuda(), torch.from_numpy(Us[e][0]).cuda(),
                       torch.from_numpy(f.dV.astype(np.float32)).cuda(), torch.from_numpy(f.seg).cuda(),
                       n_seg=5, ref=ref)
        doms.append((de, torch.from_numpy(Xs[e]).cuda(), torch.from_numpy(Us[e]).cuda(), ref))

    def step_each(n):
        for e, (de, Xe, Ue, ref) in enumerate(doms):
            de.step_markers(Xe[n], Ue[n], [frames[n][e]])

    hms = _warm(step_each, range(W))
    ms_seq = _max_over_ranks(_timed(stream, world, step_each, range(W, W + K), _ahead_ms(hms, K)), world)
    for de, _, _, _ in doms:
        de.get_body_force_torque()
        de.close()
    return {"value": round(world * cells * K / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS",
            "ms_per_step": round(ms / K, 5), "envs": n_envs, "cells": int(cells), "kernel_variant": variant,
            "markers": int(sum(d["n_markers"] for d in draws)),
            "one_domain_per_env": {"value": round(world * cells * K / (ms_seq * 1e-3) / 1e6, 1), "unit": "MLUPS",
                                   "ms_per_step": round(ms_seq / K, 5),
                                   "what": "the same envs as 64 FP32 single-env domains stepped in turn"},
            "speedup_vs_one_domain_per_env": round(ms_seq / ms, 3),
            "fused_persistent": {"value": round(world * cells * K / (ms_f * 1e-3) / 1e6, 1), "unit": "MLUPS",
                                 "ms_per_step": round(ms_f / K, 5), "kernel_ms": round(k_f[1], 5),
                                 "reduce_ms": round(k_f[2], 5),
                                 "what": "k_step_fused: IB phases and stream-collide blocks of all %d envs in "
                                         "one persistent launch per step (+ the reduction)" % n_envs},
            "roofline": {"bound": "hbm", "kernel": "k_stream_collide", "achieved": round(gbs, 1),
                         "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4),
                         "kernel_ms": round(k[1], 5), "ib_ms": round(k[0], 5), "reduce_ms": round(k[2], 5),
                         "what": "the stream-collide section of the step; with kernel_variant overlap it also "
                                 "holds the IB phases running beside the cell blocks"}}


def run_ours(args):
    import torch

    from paper_2206_01683_b300 import fishlbm

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    shape, tau, u_in = (256, 128, 128), 0.52, 0.02
    ncell = shape[0] * shape[1] * shape[2]
    W, K = args.warmup, args.steps
    T = 2 * W + 2 * REPEATS * K   # warm-up, timed repetitions, roofline pass and e2e (warm-up, repetitions)
    fish, X, U, frames = fish_workload(T, shape)
    fr = [fishlbm.frame_from_array(f) for f in frames]
    stream = torch.cuda.Stream()
    dom = fishlbm.Domain([fishlbm.env_desc(shape, tau, OPEN_X, (u_in, 0, 0), 1.0, (u_in, 0, 0))],
                         stream=stream.cuda_stream, storage=args.storage, layout=args.layout, **_variant_kw(args))
    Xd = torch.from_numpy(X).cuda()
    Ud = torch.from_numpy(U).cuda()
    dVd = torch.from_numpy(fish.dV.astype(np.float32)).cuda()
    segd = torch.from_numpy(fish.seg.astype(np.int32)).cuda()
    ref = tuple(float(v) for v in fish.joints_rest[0])
    torch.cuda.synchronize()
    dom.set_markers(Xd[0], Ud[0], dVd, segd, n_seg=5, ref=ref)

    def dev_step(n):
        dom.step_markers(Xd[n], Ud[n], [fr[n]])

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    for n in range(W):
        dev_step(n)
    barrier()
    dom.get_body_force_torque()

    # ---- timed region: inputs resident in HBM.  The clock sampler starts
    # first and the warm-up steps run after it, so the GPU does not sit idle
    # (and drop its clocks) between the warm-up and the timed steps; the K
    # steps are timed REPEATS times back to back and the median is reported.
    clocks = ClockSampler(local)
    clocks.start()
    hms = _warm(dev_step, range(W))
    reps, host_ms = [], []
    for r in range(REPEATS):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        _sleep_ahead(stream, _ahead_ms(hms, K))
        e0.record(stream)
        t0 = time.perf_counter()
        for n in range(W + r * K, W + (r + 1) * K):
            dev_step(n)
        t1 = time.perf_counter()
        e1.record(stream)
        barrier()
        reps.append(e0.elapsed_time(e1))
        host_ms.append((t1 - t0) * 1e3)
    clock_info = clocks.stop()
    ms = float(np.median(reps))
    dom.get_body_force_torque()   # raises on a numeric fault
    base = W + REPEATS * K

    # ---- per-kernel durations over a second timed region (events around each launch)
    dom.profile(True)
    for n in range(base, base + K):
        dev_step(n)
    kms, kcount = dom.profile_read()
    dom.profile(False)
    k1_ms = kms[fishlbm.FG_K_STREAM_COLLIDE] / max(kcount[fishlbm.FG_K_STREAM_COLLIDE], 1)
    ib_ms = kms[fishlbm.FG_K_IB] / max(kcount[fishlbm.FG_K_IB], 1)
    red_ms = kms[fishlbm.FG_K_REDUCE] / max(kcount[fishlbm.FG_K_REDUCE], 1)
    algo_bytes = dom.stream_collide_bytes()

    # ---- end to end: host (pinned) marker buffers in, body force out, every
    # step; W untimed calls first (the first calls load kernels lazily)
    Xh = torch.from_numpy(X).pin_memory()
    Uh = torch.from_numpy(U).pin_memory()
    # each step's marker buffers and frame as the caller holds them (the
    # slicing is the caller's, not part of the call)
    io_in = [(Xh[n], Uh[n], [fr[n]]) for n in range(T)]
    out = np.zeros((6, 6))
    # at least 60 untimed calls: after 10, the first of five 200-step
    # repetitions ran 27% slower than the last on one box
    for n in range(max(W, E2E_WARM)):
        out = dom.step_io(*io_in[(base + n) % T])
    # repetitions of at least E2E_STEPS calls: the calls are host-bound, and
    # short repetitions between synchronisations measured the host's clock
    # ramp (20-call repetitions ran 0.23 ms per call where 200-call ones ran
    # 0.213 on the same box)
    Ke = max(K, E2E_STEPS)
    e2e_reps = []
    for r in range(REPEATS):
        barrier()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        for n in range(base + r * Ke, base + (r + 1) * Ke):
            out = dom.step_io(*io_in[n % T])   # markers in, one step, force/torque out
        h1.record(stream)
        barrier()
        e2e_reps.append(h0.elapsed_time(h1) / Ke)   # ms per step
    e2e_ms = float(np.median(e2e_reps)) * K   # per K steps, as ms

    ms = _max_over_ranks(ms, world)
    e2e_ms = _max_over_ranks(e2e_ms, world)
    peak, peak_kind = measured_peaks()
    forms = None
    if not args.no_forms:
        # every rank runs every form (their barriers and reductions pair up)
        Kf = min(K, args.form_steps)
        # ordered so that the reduced-precision, large-sphere and batched forms
        # come last in the printed line
        forms = {
            "mdf3": storage_form("f32", shape, tau, u_in, fish, Xd, Ud, dVd, segd, ref, fr, W, Kf, world, peak,
                                 _variant_kw(args), ib_iters=3),
            "deterministic": storage_form("f32", shape, tau, u_in, fish, Xd, Ud, dVd, segd, ref, fr, W, Kf, world,
                                          peak, _variant_kw(args), deterministic=True),
            "eq3": storage_form("f32", shape, tau, u_in, fish, Xd, Ud, dVd, segd, ref, fr, W, Kf, world, peak,
                                _variant_kw(args), eq_order=3),
            "school": school_form(W, Kf, world, peak, _variant_kw(args)),
            "free_sphere": free_sphere_form(W, Kf, world, _variant_kw(args)),
            "adjoint": adjoint_form(),
            "f16": storage_form("f16", shape, tau, u_in, fish, Xd, Ud, dVd, segd, ref, fr, W, Kf, world, peak,
                                _variant_kw(args)),
            "bf16": storage_form("bf16", shape, tau, u_in, fish, Xd, Ud, dVd, segd, ref, fr, W, Kf, world, peak,
                                 _variant_kw(args)),
            # one population array updated in place (the plain kernel's own in-place form)
            "aa": storage_form("f32", shape, tau, u_in, fish, Xd, Ud, dVd, segd, ref, fr, W, Kf, world, peak, {},
                               layout="aa"),
            "aa_f16": storage_form("f16", shape, tau, u_in, fish, Xd, Ud, dVd, segd, ref, fr, W, Kf, world, peak,
                                   {}, layout="aa"),
            "large_sphere": large_sphere_form(W, Kf, world, peak, _variant_kw(args)),
            "batched": batched_form(W, Kf, world, peak, _variant_kw(args)),
        }
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return None
    achieved = algo_bytes / (k1_ms * 1e-3) / 1e9
    bpc = NCU_TRAFFIC.get((kernel_source_hash(args.layout), dom.stream_collide_variant(), args.storage, args.layout))
    mlups = job_mlups(world, ncell, K, ms)
    # X and U (read by the step's IB kernel from pinned memory), then one copy
    # of the frame (25 floats, padded to 112 bytes) and the 24-byte marker source
    h2d = 2 * X[0].nbytes + 112 + 24
    d2h = out.size * 8 + 4        # the force/torque rows as FP32 pairs, and the status word
    line = {
        "metric": METRIC,
        "value": round(mlups, 1),
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": round(ms / K, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "swimmer_channel_256x128x128", "grid": list(shape), "tau": tau,
                   "faces": "inlet -x (u=0.02), outflow +x, free-slip y/z",
                   "markers": int(X.shape[1]), "segments": 5, "storage": args.storage,
                   "frame": "seeded accelerating + rotating (Eq. 3)",
                   "l2": "inputs exceed L2 (populations 453 MB per buffer, %s)"
                         % ("1 buffer in place" if args.layout == "aa" else "2 buffers"),
                   "layout": args.layout,
                   "parallelism": "replicas" if world > 1 else "single",
                   "kernel_variant": dom.stream_collide_variant()},
        "roofline": {"bound": "hbm", "kernel": "k_stream_collide_aa" if args.layout == "aa" else "k_stream_collide",
                     "achieved": round(achieved, 1),
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": round(achieved / peak, 4),
                     "nominal_peak": NOMINAL_HBM_GBS, "frac_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                     "traffic": (round(bpc * ncell) if bpc else None),
                     "algorithmic_bytes": int(algo_bytes),
                     "kernel_ms": round(k1_ms, 5), "ib_ms": round(ib_ms, 5),
                     "reduce_ms": round(red_ms, 5)},
        "e2e": {"value": round(job_mlups(world, ncell, K, e2e_ms), 1), "unit": "MLUPS",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": 3 * K,   # per timed repetition: k_ib_step (which reads the step's markers), stream-collide, k_reduce
        "clocks": clock_info,
        "timing": {"repeats": REPEATS, "ms_per_step_each": [round(r / K, 5) for r in reps],
                   "e2e_ms_per_step_each": [round(r, 5) for r in e2e_reps],
                   "host_submit_ms_per_step": round(float(np.median(host_ms)) / K, 5),
                   "what": "median of the repetitions; host_submit = host time to enqueue a step (no "
                           "sync); a spin kernel ahead of each timed region lets the host enqueue the K steps "
                           "before the GPU reaches them (e2e keeps the host's time; its repetitions are "
                           "max(K, %d) calls)" % E2E_STEPS},
    }
    if forms is not None:
        line["forms"] = dict(
            f32={"value": line["value"], "unit": "MLUPS", "ms_per_step": line["ms_per_step"],
                 "roofline": {"achieved": line["roofline"]["achieved"], "frac": line["roofline"]["frac"],
                              "algorithmic_bytes_per_cell": 216}}, **forms)
    if forms is not None:
        for name, form in line["forms"].items():
            if name != "f32" and isinstance(form, dict) and form.get("unit") == "MLUPS" and form.get("value"):
                form["speedup_vs_f32"] = round(form["value"] / line["value"], 3)
        na = min(60, len(fr))
        for st in ("f16", "bf16"):
            line["forms"][st]["accuracy"] = {
                "u_rel_l2_vs_f32": round(storage_accuracy(st, shape, tau, u_in, fish, Xd, Ud, dVd, segd, ref, fr,
                                                          na, _variant_kw(args)), 8),
                "steps": na, "bar_vs_fp64_oracle": STORAGE_BAR[st]}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(fish, X, U, frames, shape, tau, u_in, steps=args.cpu_steps)
    if world > 1:
        torch.distributed.destroy_process_group()
    return line


# -------------------------------------------------------------- oracle

def oracle_steps(shape, tau, u_in, fish, X, U, frames, steps):
    import oracle
    o = oracle.Oracle(shape, tau, faces=OPEN_X, u_in=(u_in, 0, 0))
    o.init_fields(None, np.tile([u_in, 0.0, 0.0], (o.ncell, 1)))
    ref = fish.joints_rest[0]
    times = []
    for n in range(steps):
        o.set_markers(X[n].astype(np.float64), U[n].astype(np.float64), fish.dV, seg=fish.seg,
                      nseg=5, ref=ref)
        t = time.perf_counter()
        o.step(frames[n])
        times.append(time.perf_counter() - t)
    return times


def cpu_baseline(fish, X, U, frames, shape, tau, u_in, steps):
    import oracle
    ncell = shape[0] * shape[1] * shape[2]
    cores = oracle.set_threads(0)
    times = oracle_steps(shape, tau, u_in, fish, X, U, frames, steps)
    oracle.set_threads(1)
    t1 = oracle_steps(shape, tau, u_in, fish, X, U, frames, 1)
    oracle.set_threads(cores)
    return {"value": round(ncell * steps / sum(times) / 1e6, 3), "unit": "MLUPS", "cores": cores,
            "kind": "oracle",
            "sample": "%d steps of the full %dx%dx%d swimmer channel (FP64 C oracle, OpenMP)"
                      % (steps, *shape),
            "single_thread": {"value": round(ncell / t1[0] / 1e6, 3), "unit": "MLUPS", "cores": 1,
                              "sample": "1 step of the same channel"}}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return None
    # each step: one oracle step of the same physics on a 128x64x64 sample of
    # the channel (body length 32, 1500 markers), so that K steps fit in minutes
    shape, tau, u_in = (128, 64, 64), 0.52, 0.02
    W, K = args.warmup, args.steps
    fish, X, U, frames = fish_workload(W + K, shape, length=32.0, n_markers=1500)
    import oracle
    o = oracle.Oracle(shape, tau, faces=OPEN_X, u_in=(u_in, 0, 0))
    o.init_fields(None, np.tile([u_in, 0.0, 0.0], (o.ncell, 1)))
    ref = fish.joints_rest[0]
    for n in range(W):
        o.set_markers(X[n].astype(np.float64), U[n].astype(np.float64), fish.dV, seg=fish.seg, nseg=5, ref=ref)
        o.step(frames[n])
    t0 = time.perf_counter()
    for n in range(W, W + K):
        o.set_markers(X[n].astype(np.float64), U[n].astype(np.float64), fish.dV, seg=fish.seg, nseg=5, ref=ref)
        o.step(frames[n])
    dt = time.perf_counter() - t0
    ncell = shape[0] * shape[1] * shape[2]
    v = ncell * K / dt / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = "each step: one FP64 oracle step on a 128x64x64 sample of the swimmer channel (L=32, 1500 markers)"
    return {
        "impl": "reference",
        "metric": METRIC, "value": round(v, 3), "unit": "MLUPS", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": round(dt / K * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "swimmer_channel_256x128x128", "sample": sample},
        "cpu_baseline": {"value": round(v, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(v, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }


def run_form(args):
    """One form alone on one GPU (no headline step, no CPU baseline)."""
    import torch
    torch.cuda.set_device(0)
    W, K, vkw = args.warmup, args.steps, _variant_kw(args)
    peak = measured_peaks()[0]
    if args.form == "batched":
        return batched_form(W, K, 1, peak, vkw, n_envs=args.batch_envs)
    if args.form == "school":
        return school_form(W, K, 1, peak, vkw)
    if args.form == "large_sphere":
        return large_sphere_form(W, K, 1, peak, vkw)
    if args.form == "free_sphere":
        return free_sphere_form(W, K, 1, vkw)
    return adjoint_form()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-steps", type=int, default=6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the FP16/BF16/batched forms")
    ap.add_argument("--form-steps", type=int, default=50)
    ap.add_argument("--layout", default="pull", choices=["pull", "aa"],
                    help="population layout of the main line: two buffers (pull) or one in place (aa)")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"],
                    help="population storage of the main workload (f32 is the headline; the others for profiling)")
    ap.add_argument("--variant", default="autotune", choices=["autotune", "plain", "staged", "staged512"],
                    help="stream-collide kernel: autotuned at creation (default) or fixed")
    ap.add_argument("--form", choices=["batched", "school", "large_sphere", "free_sphere", "adjoint"],
                    help="run only this form (W warm-up and K timed steps) and print its result, for profiling")
    ap.add_argument("--batch-envs", type=int, default=64,
                    help="environments of the batched form (the first of the 64 seeded draws)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.form:
        print(json.dumps({"form": args.form, **run_form(args)}), flush=True)
        return
    line = run_reference(args) if args.impl == "reference" else run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
