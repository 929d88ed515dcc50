#!/usr/bin/env python3
"""Benchmark of the plain FP64 VL2 + PLM + HLLD + CT step on one GB300 per process.

Workload: 3D Orszag-Tang-style vortex (seeded phases, seed 2005) on a 256^3 periodic grid split into
512 MeshBlocks of 32^3 with 2 ghost layers; gamma = 5/3, CFL 0.3, VL2 (donor-cell predictor, PLM
corrector), HLLD fluxes, upwind CT.  One "step" = one VL2 cycle plus the CFL time step of the new
state (new_dt), all through the C ABI.

Printed JSON line (rank 0):
  value       zone-cycles/s of the whole job, timed with CUDA events on the mesh's stream over exactly
              --steps cycles (state already resident; the 1.07 GB state register exceeds the 129 MB
              L2, so no flush is needed)
  e2e         the same metric when every step also uploads its input state from pinned host memory
              (set_prims) and reads the new state back to pinned host memory (get_cons)
  roofline    the dominant kernel (largest device time in the timed region): achieved FP64 FLOP/s =
              algorithmic FP64 operations per face (counted with the oracle's operation-counting scalar:
              add/sub, mul, div, sqrt each one) x the method's faces per launch ((mb+1) mb^2 per MeshBlock)
              / event-timed launch duration, against the FP64 FMA throughput measured on the same GPU by
              vl2_debug_fp64_peak (the figure derived from 152 SMs x 2 FP64 FMA per clock x 2 FLOP x
              2.07 GHz is printed beside it)
  hbm         320 algorithmic bytes per zone-cycle (8 doubles read+written in the predictor, a stencil
              read, a base read and a write of 8 doubles in the corrector) x value / measured HBM copy
              bandwidth
  cpu_baseline the CPU oracle timed on this host's cores on a bounded sample (N = 1, rank 0)
  forms       the other forms and workloads, each with its own config: mixed precision (512^3 decaying
              turbulence), batched (1024 uneven boxes, 200 cycles in one graph launch), adjoint (checkpointed
              rollout), integrators (RK2, RK3, VL2 / RK3 with PPM, four passive scalars), blast (the paper's
              blast wave at 256^3), meshblocks (single 64^3 MeshBlock rates, MeshBlock-size sweep at 128^3)
              and linear_waves (the Alfven, slow and fast waves at 16^3, 32^3, 64^3: GPU and oracle L1 error)

--impl reference times the CPU oracle itself on the same workload (the full 256^3 vortex in 512 MeshBlocks
of 32^3): every step is one oracle VL2 cycle of the whole mesh on the host's cores.
Under torchrun every rank advances its own replica (the method is not sharded: replicas only).
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MHD zone-cycles/s at 256^3 (FP64 plain vs mixed/batched), % of HBM roofline"
UNIT = "zone-cycles/s"
HBM_BYTES_PER_ZONE_CYCLE = 320.0
# FP64 operations of one face flux (add/sub + mul + div + sqrt), counted by instantiating the oracle's
# pointwise reconstruction and Riemann functions with its operation-counting scalar and averaging over
# 3000 faces of the seed-2005 vortex (oracle/count_flops.py).
FLOPS_PER_FACE = {("plm", "hlld"): 484.9, ("dc", "hlld"): 394.1, ("plm", "hlle"): 299.8, ("dc", "hlle"): 209.0}
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM traffic of the dominant kernel from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum of
# the k_flux_plm x sweep on the 128^3 vortex, 2,162,688 faces), scaled to a launch by its faces; valid only
# for the kernel source it was taken on (hash of the flux and physics sources), else reported as null.
NCU_TRAFFIC = {"hash": "46271050d8027eb8", "bytes_per_face": 131.92}


def flux_source_hash():
    h = hashlib.sha256()
    for f in ("vl2_flux.cu", "vl2_physics.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2005_06651_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, n = [], None, set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            n += 1
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": n}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, pg, device):
    """The largest value of x over all ranks (the job's time is its slowest rank's); x itself when there is
    no process group."""
    if not pg:
        return x
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(cells_per_rank, steps, seconds, world):
    """Zone-cycles/s of the whole job: every rank advances its own replica of `cells_per_rank` cells for
    `steps` cycles, and the job takes `seconds` (the max over ranks)."""
    return world * cells_per_rank * steps / seconds


def oracle_rate(n, mb, steps, warmup, seed=2005, min_seconds=0.0, max_steps=None):
    """Time the CPU oracle on an n^3 sample of the vortex; returns (zone-cycles/s, steps, threads, s)."""
    from oracle import orc
    from paper_2005_06651_gb300 import inputs

    prob = inputs.orszag_tang(n=n, mb=mb, seed=seed)
    m = orc.Mesh.from_problem(prob)
    for _ in range(warmup):
        m.step(m.new_dt(0.3))
    t0 = time.perf_counter()
    done = 0
    while True:
        m.step(m.new_dt(0.3))
        done += 1
        el = time.perf_counter() - t0
        if done >= steps and el >= min_seconds:
            break
        if max_steps is not None and done >= max_steps:
            break
    el = time.perf_counter() - t0
    threads = orc_threads()
    return prob.ncells * done / el, done, threads, el


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the CPU baseline's record."""
    import subprocess

    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def set_orc_threads(n):
    """Thread count of the oracle's OpenMP loops (libgomp, loaded by the oracle library)."""
    import ctypes

    gomp = ctypes.CDLL("libgomp.so.1")
    gomp.omp_set_num_threads(int(n))


def orc_threads():
    try:
        import ctypes

        gomp = ctypes.CDLL("libgomp.so.1")
        gomp.omp_get_max_threads.restype = ctypes.c_int
        return int(gomp.omp_get_max_threads())
    except Exception:
        return os.cpu_count()


def run_reference(args, world, rank):
    """The oracle as it stands on the host's cores, on this arm's own workload (the full args.n^3 vortex in
    args.mb^3 MeshBlocks): W untimed cycles, then K timed ones (about 2.7 s per 256^3 cycle on 16 cores)."""
    if rank != 0:
        return
    n, mb = args.n, args.mb
    rate, done, threads, el = oracle_rate(n, mb, args.steps, args.warmup)
    sample = "%d VL2 cycles of the full %d^3 vortex (%d MeshBlocks of %d^3) after %d untimed ones, FP64 CPU " \
        "oracle" % (done, n, (n // mb) ** 3, mb, args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / done, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args),
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                             "cpu": cpu_model()},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(args):
    return {"workload": "orszag_tang_3d_%d^3_%dx%d^3_blocks_vl2_plm_hlld_ct_fp64" % (
        args.n, (args.n // args.mb) ** 3, args.mb), "grid": [args.n] * 3, "meshblock": [args.mb] * 3,
        "meshblocks": (args.n // args.mb) ** 3, "ghosts": 2, "gamma": 5.0 / 3.0, "cfl": 0.3,
        "integrator": "vl2", "reconstruction": "plm (donor cell predictor)", "riemann": "hlld", "seed": 2005,
        "l2": "state (1.07 GB per register at 256^3) exceeds the 129 MB L2; no flush", "parallelism": "replicas",
        **({"flux_shape": list(args.flux_shape)} if getattr(args, "flux_shape", None) else {})}


def timed_steps(mesh, steps, stream, dts=None):
    """Device time (ms) of `steps` cycles (new_dt + step, or the given dt sequence); returns (ms, dts)."""
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = []
    e0.record(stream)
    for s in range(steps):
        dt = mesh.new_dt() if dts is None else dts[s]
        mesh.step(dt)
        out.append(dt)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def mixed_form(args, dev, stream, vl2, inputs):
    """Mixed-precision form on decaying turbulence (Mach 2, beta 10) at forms_n^3 in 32^3 MeshBlocks, next
    to plain FP64 on the same state and the same dt sequence; plus the 64^3 linear-wave L1 error of both."""
    import torch

    n, mb, K = args.forms_n, args.mb, args.forms_steps
    prob = inputs.turbulence(n=n, mb=mb, seed=3003, mach=2.0, beta=10.0)
    res = {"config": {"workload": "decaying_turbulence_%d^3_%dx%d^3_blocks_mach2_beta10" % (n, (n // mb) ** 3, mb),
                      "seed": 3003, "steps": K, "dtype": "f32 reconstruction/fluxes/CT, f64 state/cons->prim/accumulation"}}
    states, times = {}, {}
    dts = None
    for name, prec in (("fp64", vl2.FP64), ("mixed", vl2.MIXED)):
        m = vl2.Mesh.from_problem(prob, device=dev, stream=stream, precision=prec)
        if args.flux_shape:
            m.set_flux_shape(*args.flux_shape)
        for _ in range(3):
            m.step(m.new_dt())
        m.set_prims(prob.w, prob.b1, prob.b2, prob.b3)
        torch.cuda.synchronize(dev)
        ms, used = timed_steps(m, K, stream, dts)
        if dts is None:
            dts = used
        times[name] = ms
        u = torch.empty((5,) + m.shape, dtype=torch.float64, device=dev)
        m.get_cons((u, None, None, None))
        c = n // 2
        sl = slice(c - 64, c + 64) if n >= 128 else slice(0, n)
        states[name] = (u[0, sl, sl, sl].clone(), u[4, sl, sl, sl].clone())
        del m, u
        torch.cuda.empty_cache()
    rho_err = float(((states["mixed"][0] - states["fp64"][0]).abs() / states["fp64"][0].abs()).max())
    e_err = float(((states["mixed"][1] - states["fp64"][1]).abs() / states["fp64"][1].abs()).max())
    ncell = prob.ncells
    res.update({"value": ncell * K / (times["mixed"] / 1e3), "unit": UNIT, "ms_per_step": times["mixed"] / K,
                "fp64_value": ncell * K / (times["fp64"] / 1e3), "fp64_ms_per_step": times["fp64"] / K,
                "speedup_vs_fp64": times["fp64"] / times["mixed"],
                "hbm_frac": HBM_BYTES_PER_ZONE_CYCLE * ncell * K / (times["mixed"] / 1e3) / 1e9 /
                float(measured_peaks().get("hbm_gbs", 6800.0)),
                "max_rel_err_vs_fp64_central_128": {"rho": rho_err, "E": e_err,
                                                    "after_steps": K, "same_dt_sequence": True}})
    # linear-wave L1 error (eq. RMS-error) at 64^3, one period, both precisions
    wave = inputs.linear_wave(64, mb=32, kind="alfven", amp=1e-6)
    l1 = {}
    for name, prec in (("fp64", vl2.FP64), ("mixed", vl2.MIXED)):
        m = vl2.Mesh.from_problem(wave, device=dev, stream=stream, precision=prec)
        ref = m.get_cons()
        m.run(wave.meta["period"])
        l1[name] = rms_l1(m.get_cons(), ref)
        del m
    res["linear_wave_l1_64"] = {"amplitude": 1e-6, "fp64": l1["fp64"], "mixed": l1["mixed"]}
    return res


def batched_form(args, dev, stream, vl2, inputs):
    """Batched form: boxes of sizes drawn from {16, 32, 48, 64}^3 (seed 3003), one MeshBlock each, periodic
    turbulence (Mach 1, beta 1), FP64.  The per-box launch path (new_dt + step per box) is timed over
    --per-box-steps cycles; the batch (autotuned flux shapes, per-box CFL steps on the device) then runs the
    same cycles as one CUDA-graph launch and must end bitwise equal to the per-box path on the checked boxes.
    Finally the batch runs --batch-steps cycles (200: the configuration's run) from the initial state as one
    graph launch, timed with events; the state after it is summarised per box."""
    import numpy as np
    import torch

    nbox, K, Kp = args.batch_boxes, args.batch_steps, min(args.per_box_steps, args.batch_steps)
    rng = np.random.Generator(np.random.PCG64(3003))
    sizes = rng.choice([16, 32, 48, 64], size=nbox)
    probs = [inputs.turbulence(n=int(n), mb=int(n), seed=3003 + q, mach=1.0, beta=1.0) for q, n in enumerate(sizes)]
    meshes = [vl2.Mesh(p.nx, p.mb, p.xmin, p.xmax, p.gamma, device=dev, stream=stream) for p in probs]
    ncell = sum(p.ncells for p in probs)

    def reset():
        for m, p in zip(meshes, probs):
            m.set_prims(p.w, p.b1, p.b2, p.b3)

    reset()
    tot0 = np.array([m.totals() for m in meshes])
    for m in meshes:  # warm-up
        m.step(m.new_dt(allow_nonphys=True))
    reset()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = sum(m.launch_count() for m in meshes)
    t0 = time.perf_counter()
    for _ in range(Kp):
        for m in meshes:
            m.step(m.new_dt(allow_nonphys=True))  # a floor is part of the method: counted, not fatal
    torch.cuda.synchronize(dev)
    per_box_s = time.perf_counter() - t0
    per_box_launches = sum(m.launch_count() for m in meshes) - launches0
    check = [q for q in range(0, nbox, max(1, nbox // 8))]
    ref = {q: meshes[q].get_cons() for q in check}
    reset()
    batch = vl2.Batch(meshes)
    dc, pl = batch.autotune()
    reset()
    batch.run(Kp, want_dt=False)
    same = all(all(np.array_equal(a, b) for a, b in zip(meshes[q].get_cons(), ref[q])) for q in check)
    reset()
    floors0 = [m.floor_count() for m in meshes]
    torch.cuda.synchronize(dev)
    l0 = batch.launch_count()
    t0 = time.perf_counter()
    e0.record(stream)
    batch.run(K, want_dt=False)  # captures the K-cycle graph, then launches it once
    e1.record(stream)
    torch.cuda.synchronize(dev)
    batched_s = time.perf_counter() - t0
    batched_ms = e0.elapsed_time(e1)
    batched_launches = batch.launch_count() - l0
    floor_events = [m.floor_count() - floors0[q] for q, m in enumerate(meshes)]
    floor_boxes = [q for q, f in enumerate(floor_events) if f > 0]
    tot = np.array([m.totals() for m in meshes])
    divb = max(m.divb_norm() for m in meshes)
    dt_next = np.array([m.new_dt(allow_nonphys=True) for m in meshes])
    mass_drift = float(np.max(np.abs(tot[:, 0] - tot0[:, 0]) / tot0[:, 0]))
    tuned = batch.flux_shape()

    # the persistent, TMA-staged PLM kernel (bounded mbarrier waits), forced, against the autotuned shapes over
    # the per-box cycles: the tallest tile that fits the largest box in shared memory
    def timed_cycles(shape):
        batch.set_flux_shape(*shape)
        reset()
        batch.run(Kp, want_dt=False)  # captures the graph of this shape
        reset()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        batch.run(Kp, want_dt=False)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / Kp

    persistent = None
    for lines in (16, 8, 4):
        try:
            pms = timed_cycles((tuned[0], lines, 1))
        except vl2.VL2Error:
            continue
        ams = timed_cycles(tuned)
        persistent = {"plm_lines": lines, "steps": Kp, "ms_per_step": pms, "value": ncell / (pms / 1e3),
                      "unit": UNIT, "autotuned_ms_per_step_same_cycles": ams, "autotuned_over_persistent": ams / pms}
        break
    del batch
    counts = {int(v): int((sizes == v).sum()) for v in (16, 32, 48, 64)}
    return {"config": {"workload": "%d_turbulence_boxes_sizes_16_32_48_64_cubed_one_block_each" % nbox,
                       "box_counts": counts, "cells": ncell, "steps": K, "seed": 3003, "mach": 1.0, "beta": 1.0,
                       "dtype": "f64"},
            "value": ncell * K / (batched_ms / 1e3), "unit": UNIT, "ms_per_step": batched_ms / K,
            "wall_ms_per_step": 1e3 * batched_s / K, "gpu_launches_per_step": batched_launches / K,
            "timing": "one graph launch of %d cycles, CUDA events on the mesh stream; the wall time also holds "
                      "the graph's capture and instantiation" % K,
            "per_box_value": ncell * Kp / per_box_s, "per_box_ms_per_step": 1e3 * per_box_s / Kp,
            "per_box_steps": Kp, "per_box_launches_per_step": per_box_launches / Kp,
            "speedup_vs_per_box": (1e3 * per_box_s / Kp) / (batched_ms / K),
            "autotuned": {"dc_threads": tuned[0], "plm_lines": tuned[1], "plm_kernel": "persistent TMA-staged tiles"
                          if tuned[2] else "line tiles"},
            "persistent_tma_plm": persistent,
            "bitwise_equal_to_per_box_path": bool(same), "checked_boxes": len(check), "checked_steps": Kp,
            "after_steps": {"steps": K, "boxes_with_floor_events": len(floor_boxes),
                            "floor_events": int(sum(floor_events)),
                            "most_floored_boxes": sorted(floor_boxes, key=lambda q: -floor_events[q])[:8],
                            "max_divb_norm": divb, "max_relative_mass_drift": mass_drift,
                            "next_dt_min": float(np.min(dt_next)), "next_dt_median": float(np.median(dt_next)),
                            "boxes_next_dt_below_1e-6": [int(q) for q in np.nonzero(dt_next < 1e-6)[0]][:16]}}


def adjoint_form(args, dev, stream, vl2, inputs):
    """Differentiation form, FP64, 64^3 periodic box in 8 MeshBlocks of 32^3, adj_steps VL2 cycles behind
    torch.autograd with a checkpoint every ~sqrt(N) cycles.  Loss = sum over cells of (rho_final - target)^2
    dV with target = 1 + 0.01 N(0,1) (seed 5005); gradient with respect to the initial velocity (3 x 64^3).
    Timing and peak memory: seeded decaying turbulence (Mach 1, beta 10, seed 3003), forward and backward
    device time and their ratio.  Gradient check: a fast magnetosonic wave (amplitude 1e-2) carried by a
    uniform flow, central finite differences along smooth directions with the same time steps."""
    import numpy as np
    import torch

    from paper_2005_06651_gb300 import adjoint

    n, K = args.adj_n, args.adj_steps
    mb = min(32, n)
    k = max(1, int(round(K ** 0.5)))
    target = torch.from_numpy(1.0 + 0.01 * np.random.Generator(np.random.PCG64(5005)).standard_normal((n, n, n)))
    target = target.to(dev)

    def setup(prob):
        runner = adjoint.Rollout(prob, nsteps=K, checkpoint_every=k, device=dev)
        dv = float(np.prod(prob.dx))
        v_init = torch.from_numpy(np.ascontiguousarray(prob.w[1:4])).to(dev)
        return runner, v_init, (lambda u: ((u[0] - target) ** 2).sum() * dv)

    # timing and memory on the turbulence state
    turb = inputs.turbulence(n=n, mb=mb, seed=3003, mach=1.0, beta=10.0)
    torch.cuda.synchronize(dev)
    torch.cuda.empty_cache()
    base_mem = torch.cuda.memory_allocated(dev)
    torch.cuda.reset_peak_memory_stats(dev)
    runner, v_init, loss_of = setup(turb)
    times = {"forward": [], "backward": []}
    for rep in range(3):  # the first repetition is the warm-up
        v = v_init.clone().requires_grad_(True)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        loss = loss_of(adjoint.rollout(v, runner))
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        loss.backward()
        torch.cuda.synchronize(dev)
        t2 = time.perf_counter()
        if rep:
            times["forward"].append(t1 - t0)
            times["backward"].append(t2 - t1)
    peak = torch.cuda.max_memory_allocated(dev) - base_mem
    floors = runner.mesh.floor_count()
    runner.mesh.close()
    state_bytes = 8 * (5 * turb.ncells + sum(int(np.prod(b.shape)) for b in (turb.b1, turb.b2, turb.b3)))

    # gradient check on the advected wave
    wave = inputs.linear_wave(n, mb=mb, kind="fast", amp=1e-2, v0=(0.7, 0.4, 0.2))
    runner, v_init, loss_of = setup(wave)
    v = v_init.clone().requires_grad_(True)
    loss_of(adjoint.rollout(v, runner)).backward()
    grad = v.grad.detach().clone()
    runner.fixed_dts = list(runner.dts)
    x, y, z = inputs._cell_coords(wave.nx, wave.xmin, wave.xmax)
    rng = np.random.Generator(np.random.PCG64(5006))
    fd_checks = []
    for trial in range(2):
        ph = rng.uniform(0, 2 * np.pi, size=(3, 3))
        d = np.stack([np.sin(2 * np.pi * x + ph[c, 0]) * np.cos(2 * np.pi * y + ph[c, 1]) *
                      np.sin(2 * np.pi * z + ph[c, 2]) for c in range(3)])
        d = torch.from_numpy(np.ascontiguousarray(d)).to(dev)
        h = 1e-8  # small enough that the step crosses almost no limiter switch at this size
        with torch.no_grad():
            lp = float(loss_of(runner.run_forward(v_init + h * d)))
            lm = float(loss_of(runner.run_forward(v_init - h * d)))
        fd = (lp - lm) / (2 * h)
        ad = float((grad * d).sum())
        fd_checks.append({"fd": fd, "adjoint": ad, "rel_err": abs(fd - ad) / abs(ad)})
    runner.mesh.close()
    fwd, bwd = float(np.median(times["forward"])), float(np.median(times["backward"]))
    return {"config": {"workload": "decaying_turbulence_%d^3_%dx%d^3_blocks_mach1_beta10" % (n, (n // mb) ** 3, mb),
                       "seed": 3003, "steps": K, "checkpoint_every": k, "checkpoints": (K + k - 1) // k,
                       "loss": "sum (rho_final - target)^2 dV, target = 1 + 0.01 N(0,1), seed 5005",
                       "wrt": "initial velocity (3 x %d^3)" % n, "dtype": "f64", "riemann": "hlld",
                       "reconstruction": "plm", "fd_check_workload": "fast_wave_%d^3_amp1e-2_flow_0.7_0.4_0.2" % n},
            "forward_s": fwd, "backward_s": bwd, "backward_over_forward": bwd / fwd,
            "forward_value": turb.ncells * K / fwd, "unit": UNIT, "floor_events": floors,
            "peak_mem_bytes": int(peak), "state_bytes": state_bytes,
            "peak_mem_over_state": peak / state_bytes,
            "fd_check": {"h": 1e-8, "directions": "smooth sin/cos products, random phases (seed 5006)",
                         "checks": fd_checks, "max_rel_err": max(c["rel_err"] for c in fd_checks)}}


def integrators_form(args, dev, stream, vl2, inputs):
    """The other 2S integrators of Sec. 3.2.3 and PPM (Sec. 3.2.1) on the plain workload (256^3 vortex, 512
    MeshBlocks of 32^3, FP64, HLLD): RK2 (SSPRK(2,2)) and RK3 (SSPRK(3,3)) with PLM in every stage, and VL2
    and RK3 with PPM (three ghost layers), VL2 and RK3 with PLM and PPM on characteristic variables, VL2 + PLM
    carrying four passive scalars (eq. passive_scalars), and
    VL2 + PLM with the smoothed CT upwind weight (delta 1e-4, where most faces saturate, and delta 1, where
    none does), and VL2 + PLM with HLLE (the states' own speeds, and Einfeldt's Roe-averaged ones),
    zone-cycles/s next to VL2 + PLM + HLLD (the bench line).  A cycle has 2 or 3 PLM / PPM stages against VL2's donor-cell + PLM / PPM."""
    import torch

    prob = inputs.orszag_tang(n=args.n, mb=args.mb, seed=2005)
    out = {"config": {"workload": "orszag_tang_3d_%d^3_%dx%d^3_blocks_plm_hlld_ct_fp64" % (
        args.n, (args.n // args.mb) ** 3, args.mb), "steps": args.rk_steps, "dtype": "f64"}}
    import numpy as np

    H = vl2.HLLD
    for name, integ, recon, nsc, delta, rs in (("rk2", vl2.RK2, vl2.PLM, 0, 0.0, H), ("rk3", vl2.RK3, vl2.PLM, 0, 0.0, H),
                                               ("vl2_ppm", vl2.VL2, vl2.PPM, 0, 0.0, H),
                                               ("rk3_ppm", vl2.RK3, vl2.PPM, 0, 0.0, H),
                                               ("vl2_4_scalars", vl2.VL2, vl2.PLM, 4, 0.0, H),
                                               ("vl2_plm_char", vl2.VL2, vl2.PLM_CHAR, 0, 0.0, H),
                                               ("rk3_plm_char", vl2.RK3, vl2.PLM_CHAR, 0, 0.0, H),
                                               ("vl2_ppm_char", vl2.VL2, vl2.PPM_CHAR, 0, 0.0, H),
                                               ("rk3_ppm_char", vl2.RK3, vl2.PPM_CHAR, 0, 0.0, H),
                                               ("vl2_ct_smooth", vl2.VL2, vl2.PLM, 0, 1e-4, H),
                                               ("vl2_ct_smooth_wide", vl2.VL2, vl2.PLM, 0, 1.0, H),
                                               ("vl2_hlle", vl2.VL2, vl2.PLM, 0, 0.0, vl2.HLLE),
                                               ("vl2_hlle_roe", vl2.VL2, vl2.PLM, 0, 0.0, vl2.HLLE_ROE)):
        m = vl2.Mesh.from_problem(prob, device=dev, stream=stream, integrator=integ, recon=recon, nscalars=nsc,
                                  ct_delta=delta, riemann=rs)
        if nsc:
            rng = np.random.default_rng(4004)
            m.set_scalars(rng.uniform(0.0, 1.0, size=(nsc,) + prob.w.shape[1:]))
        for _ in range(2):
            m.step(m.new_dt())
        torch.cuda.synchronize(dev)
        ms, _ = timed_steps(m, args.rk_steps, stream)
        m.profile(True)
        m.profile_read()
        m.step(m.new_dt())
        prof = {k: v[0] for k, v in m.profile_read().items() if v[1] > 0}
        m.profile(False)
        out[name] = {"value": prob.ncells * args.rk_steps / (ms / 1e3), "unit": UNIT,
                     "ms_per_step": ms / args.rk_steps, "floor_events": m.floor_count(),
                     "kernel_ms_one_cycle": prof}
        m.close()
        del m
        torch.cuda.empty_cache()
    return out


def blast_form(args, dev, stream, vl2, inputs):
    """The paper's performance problem: the 3D MHD blast wave (rho = 1, p = 1e-3, total internal energy 1
    within r = 0.01 of the centre, B = (sqrt 3, 1, 0)) on the 256^3 mesh of 512 MeshBlocks of 32^3, FP64
    VL2 + PLM + HLLD + CT.  Ambient beta is 5e-4: floors fire (and are counted) as the pressure is
    recovered from E - rho v^2/2 - B^2/2 around the blast."""
    import torch

    prob = inputs.blast(n=args.n, mb=args.mb, r0=0.01)
    m = vl2.Mesh.from_problem(prob, device=dev, stream=stream)
    for _ in range(2):
        m.step(m.new_dt(allow_nonphys=True))
    torch.cuda.synchronize(dev)
    K = args.blast_steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        m.step(m.new_dt(allow_nonphys=True))
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    out = {"config": {"workload": "mhd_blast_%d^3_%dx%d^3_blocks_r0.01_etot1_p1e-3_b_sqrt3_1_0" % (
               args.n, (args.n // args.mb) ** 3, args.mb), "steps": K, "dtype": "f64",
               "cells_inside": prob.meta["cells_inside"], "p_in": prob.meta["p_in"]},
           "value": prob.ncells * K / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / K,
           "floor_events": m.floor_count(), "divb_norm": m.divb_norm()}
    m.close()
    return out


def _graph_ms_per_cycle(vl2, prob, mb, riemann, K, dev, stream):
    """ms per VL2 cycle of prob on MeshBlocks of mb^3 cells: K cycles with device-side CFL steps as one
    CUDA-graph launch (vl2_batch_run on a batch of this one mesh), so that no host call sits between the
    cycles.  Returns (ms, floor events, div B norm)."""
    import torch

    m = vl2.Mesh.from_problem(prob, mb=(mb,) * 3, riemann=riemann, device=dev, stream=stream)
    batch = vl2.Batch([m])
    batch.run(K, want_dt=False)  # capture the K-cycle graph (untimed), then reset and time it
    m.set_prims(prob.w, prob.b1, prob.b2, prob.b3)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    batch.run(K, want_dt=False)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / K
    out = (ms, m.floor_count(), m.divb_norm())
    batch.close()
    m.close()
    return out


def meshblocks_form(args, dev, stream, vl2, inputs):
    """MeshBlock size and cost, on the paper's blast wave (its Secs. on single-core performance and on the
    size of MeshBlocks):
    - sweep: the 128^3 MHD blast (HLLD) on MeshBlocks of x^3 cells, x = 4 ... 128, each cost normalised to
      the single 128^3 MeshBlock and fitted by least squares to W(x) = A + b/x + c/x^3 (active-cell work,
      a surface term, a per-MeshBlock term); the same on the 128^3 vortex, whose faces all carry distinct
      states (most of the blast's faces are between equal states at rest, which the solvers short-cut);
    - single 64^3 MeshBlock: the rate of each solver, MHD and hydro (HLLD at B = 0 is HLLC).
    The energy goes to the cells whose centres lie within r0 = max(0.01, sqrt(3) dx / 2 (1 + 1e-6)) of the
    centre: at 128^3 and at 64^3 these are the 8 cells around it (at 64^3 no centre lies within 0.01)."""
    import numpy as np

    K = args.mb_sweep_steps

    def r0_of(n):
        return max(0.01, 0.5 * np.sqrt(3.0) / n * (1.0 + 1e-6))

    n = 128
    sizes = [4, 8, 16, 32, 64, 128]
    xs = np.array(sizes, dtype=float)
    sweep = {}
    blast128 = inputs.blast(n=n, mb=n, r0=r0_of(n))
    for name, prob in (("mhd_blast_128^3_hlld_%d_cells_inside" % blast128.meta["cells_inside"], blast128),
                       ("orszag_tang_128^3_hlld", inputs.orszag_tang(n=n, mb=n, seed=2005))):
        ms = {x: _graph_ms_per_cycle(vl2, prob, x, vl2.HLLD, K, dev, stream)[0] for x in sizes}
        w = np.array([ms[x] / ms[128] for x in sizes])
        A, b, c = np.linalg.lstsq(np.stack([np.ones_like(xs), 1.0 / xs, xs ** -3], axis=1), w, rcond=None)[0]
        sweep[name] = {"cycles": K, "ms_per_cycle": {str(x): ms[x] for x in sizes},
                       "normalised_cost": {str(x): float(v) for x, v in zip(sizes, w)},
                       "fit_W_A_b_c": [float(A), float(b), float(c)],
                       "fit_max_abs_residual": float(np.max(np.abs(A + b / xs + c / xs ** 3 - w))),
                       "surface_term_exceeds_A_below_x": float(b / A) if A > 0 else None}
    n = 64
    single = {}
    for mhd in (True, False):
        p64 = inputs.blast(n=n, mb=n, r0=r0_of(n), magnetized=mhd)
        for name, riemann in (("hlld", vl2.HLLD), ("hlle", vl2.HLLE)):
            t, floors, divb = _graph_ms_per_cycle(vl2, p64, n, riemann, K, dev, stream)
            single["%s_plm_%s" % ("mhd" if mhd else "hydro", name)] = {
                "value": p64.ncells / (t / 1e3), "unit": UNIT, "ms_per_cycle": t, "floor_events": floors}
    return {"sweep": sweep, "single_64cubed_block": single,
            "config": {"dtype": "f64", "integrator": "vl2", "recon": "plm",
                       "timing": "K cycles with device-side dt as one CUDA graph (vl2_batch_run)"}}


def linear_waves_form(args, dev, stream, vl2, inputs):
    """Config 1 (Sec. 3.3.1, eq. RMS-error): the Alfven, slow and fast waves of amplitude 1e-6 along the unit
    cube's diagonal (|B| = 1, CFL 0.3), one MeshBlock, VL2 + PLM + HLLD + CT, one wave period with the last
    step clipped, at N = 16, 32, 64 (32^3 is the configuration).  The GPU's L1 error next to the oracle's
    (16^3 MeshBlocks on the host's cores, its own CFL steps), and the GPU's slopes between the sizes."""
    import math

    out = {"config": {"workload": "linear_waves_unit_cube_diagonal_amp1e-6_one_block_cfl0.3_one_period",
                      "sizes": list(args.wave_sizes), "dtype": "f64"}}
    from oracle import orc

    for kind in ("alfven", "slow", "fast"):
        rec = {}
        for n in args.wave_sizes:
            prob = inputs.linear_wave(n, kind=kind, amp=1e-6)
            m = vl2.Mesh.from_problem(prob, device=dev, stream=stream)
            ref = m.get_cons()
            steps = m.run(prob.meta["period"])
            gl1 = rms_l1(m.get_cons(), ref)
            del m
            o = orc.Mesh.from_problem(prob, mb=(min(16, n),) * 3)
            oref = o.get_cons()
            o.run(prob.meta["period"], cfl=0.3)
            ol1 = rms_l1(o.get_cons(), oref)
            del o
            rec[str(n)] = {"gpu_l1": gl1, "oracle_l1": ol1, "steps": steps,
                           "relative_difference": abs(gl1 - ol1) / ol1}
        ns = [str(n) for n in args.wave_sizes]
        rec["gpu_slopes"] = {"%s->%s" % (a, b): math.log2(rec[a]["gpu_l1"] / rec[b]["gpu_l1"]) for a, b in zip(ns, ns[1:])}
        out[kind] = rec
    return out


def run_forms(args, dev, stream, vl2, inputs):
    import torch

    fns = {"mixed": mixed_form, "batched": batched_form, "adjoint": adjoint_form, "integrators": integrators_form,
           "blast": blast_form, "meshblocks": meshblocks_form, "linear_waves": linear_waves_form}
    forms = {}
    for name in [f for f in args.forms.split(",") if f]:
        if name not in fns:
            raise SystemExit("unknown form %r (choose from %s)" % (name, ", ".join(fns)))
        forms[name] = compact(fns[name](args, dev, stream, vl2, inputs))
        torch.cuda.empty_cache()
    return forms


def compact(x, digits=6):
    """Floats rounded to `digits` significant digits, recursively (keeps the one JSON line short)."""
    if isinstance(x, float):
        return float("%.*g" % (digits, x))
    if isinstance(x, dict):
        return {k: compact(v, digits) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [compact(v, digits) for v in x]
    return x


def rms_l1(state, ref):
    import numpy as np

    def cb(b1, b2, b3):
        return (0.5 * (b1[:, :, 1:] + b1[:, :, :-1]), 0.5 * (b2[:, 1:, :] + b2[:, :-1, :]), 0.5 * (b3[1:] + b3[:-1]))

    u, b = state[0], cb(*state[1:])
    u0, b0 = ref[0], cb(*ref[1:])
    e = [np.mean(np.abs(u[v] - u0[v])) for v in range(5)] + [np.mean(np.abs(b[d] - b0[d])) for d in range(3)]
    return float(np.sqrt(np.sum(np.square(e))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", "--grid", dest="n", type=int, default=256, help="cells per direction of the vortex")
    ap.add_argument("--mb", type=int, default=32)
    ap.add_argument("--flux-shape", type=lambda t: tuple(int(v) for v in t.split(",")), default=None,
                    help="DC_THREADS,PLM_LINES,TMA for the headline and mixed-form meshes (default: the library's)")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the mixed-precision, batched and differentiation forms")
    ap.add_argument("--forms-n", type=int, default=512, help="grid of the mixed-precision form")
    ap.add_argument("--forms-steps", type=int, default=50)
    ap.add_argument("--batch-boxes", type=int, default=1024)
    ap.add_argument("--batch-steps", type=int, default=200, help="cycles of the batched form's graph launch")
    ap.add_argument("--per-box-steps", type=int, default=20, help="cycles of the per-box path it is compared with")
    ap.add_argument("--adj-n", type=int, default=64, help="grid of the differentiation form")
    ap.add_argument("--adj-steps", type=int, default=100)
    ap.add_argument("--wave-sizes", type=lambda t: [int(v) for v in t.split(",")], default=[16, 32, 64],
                    help="grids of the linear-wave form")
    ap.add_argument("--forms", default="mixed,adjoint,integrators,blast,meshblocks,batched,linear_waves",
                    help="comma list of the forms to run")
    ap.add_argument("--mb-sweep-steps", type=int, default=20, help="timed cycles per MeshBlock size")
    ap.add_argument("--blast-steps", type=int, default=20, help="timed cycles of the blast-wave form")
    ap.add_argument("--rk-steps", type=int, default=10, help="timed cycles of each RK integrator")
    ap.add_argument("--forms-only", action="store_true",
                    help="run only the forms (a profiling aid: prints {'forms': ...}, not the bench line)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import numpy as np
    import torch

    from paper_2005_06651_gb300 import build, inputs, vl2

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    build.build()
    vl2.load()
    if args.forms_only:
        stream = torch.cuda.current_stream(dev)
        print(json.dumps({"forms": run_forms(args, dev, stream, vl2, inputs)}), flush=True)
        return
    prob = inputs.orszag_tang(n=args.n, mb=args.mb, seed=2005)
    stream = torch.cuda.current_stream(dev)
    mesh = vl2.Mesh.from_problem(prob, device=dev, stream=stream)
    if args.flux_shape:
        mesh.set_flux_shape(*args.flux_shape)
    for _ in range(args.warmup):
        mesh.step(mesh.new_dt())
    torch.cuda.synchronize(dev)

    props = torch.cuda.get_device_properties(dev)
    gpu_id = ("GPU-" + str(props.uuid)) if getattr(props, "uuid", None) else str(local)
    sampler = ClockSampler(gpu_id)
    mesh.profile(True)
    mesh.profile_read()
    launches0 = mesh.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    time.sleep(0.3)
    # events at the borders of five equal blocks of the timed steps, for the median of five runs
    nblk_runs = 5 if args.steps >= 5 else 1
    marks = {(r * args.steps) // nblk_runs: torch.cuda.Event(enable_timing=True) for r in range(1, nblk_runs)}
    e0.record(stream)
    for s_ in range(args.steps):
        if s_ in marks:
            marks[s_].record(stream)
        mesh.step(mesh.new_dt())
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    border = [(0, e0)] + sorted(marks.items()) + [(args.steps, e1)]
    run_ms = [border[r][1].elapsed_time(border[r + 1][1]) / (border[r + 1][0] - border[r][0])
              for r in range(len(border) - 1)]
    if pg:
        pg.barrier()
    ms_total = e0.elapsed_time(e1)
    launches = mesh.launch_count() - launches0
    prof = mesh.profile_read()
    mesh.profile(False)
    ms_total = max_over_ranks(ms_total, pg, dev)
    ms_step = ms_total / args.steps
    value = whole_job_rate(prob.ncells, args.steps, ms_total / 1e3, world)

    # roofline of the dominant kernel, against the FP64 peak measured on this GPU right after the timed region
    kinds = {k: v for k, v in prof.items() if v[1] > 0}
    tot = sum(v[0] for v in kinds.values())
    dom = max(kinds, key=lambda k: kinds[k][0])
    dms, dn, dunits = kinds[dom]
    rec = {"flux_plm": "plm", "flux_dc": "dc"}.get(dom)
    sampler2 = ClockSampler(gpu_id)
    sampler2.start()
    time.sleep(0.3)
    pk = vl2.fp64_peak(dev)
    pk_clocks = sampler2.stop()
    roofline = {"kernel": dom, "bound": "alu", "unit": "TFLOP/s", "peak": pk["tflops"],
                "peak_source": "measured: vl2_debug_fp64_peak, %d CTAs x %d threads x 16 independent FMA chains, "
                               "best of 5 event-timed launches of %.0f ms" % (pk["ctas"], pk["threads"], pk["ms"]),
                "peak_clocks": pk_clocks, "peak_derived": round(FP64_PEAK_TFLOPS, 4),
                "launches": dn, "ms_per_launch": dms / dn, "kernel_units_per_launch": dunits / dn}
    if rec:
        fpu = FLOPS_PER_FACE[(rec, "hlld")]
        # the method's faces: (mb + 1) mb^2 per MeshBlock and sweep direction (both block-surface faces counted)
        faces = (prob.ncells // args.mb ** 3) * (args.mb + 1) * args.mb ** 2
        achieved = fpu * faces / (dms / dn / 1e3) / 1e12
        roofline.update({"achieved": achieved, "frac": achieved / pk["tflops"], "flops_per_unit": fpu,
                         "unit_kind": "face", "units_per_launch": faces})
        if NCU_TRAFFIC["hash"] == flux_source_hash() and NCU_TRAFFIC["bytes_per_face"]:
            roofline["traffic"] = NCU_TRAFFIC["bytes_per_face"] * dunits / dn
        else:
            roofline["traffic"] = None
    else:
        roofline.update({"achieved": None, "frac": None, "traffic": None})
    kernel_share = {k: {"ms_per_step": v[0] / args.steps, "share": v[0] / tot, "launches_per_step": v[1] / args.steps}
                    for k, v in kinds.items()}
    peaks = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm = {"bytes_per_zone_cycle": HBM_BYTES_PER_ZONE_CYCLE,
           "achieved_GBps": HBM_BYTES_PER_ZONE_CYCLE * value / world / 1e9, "peak_GBps": hbm_peak,
           "frac": HBM_BYTES_PER_ZONE_CYCLE * value / world / 1e9 / hbm_peak,
           "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}

    # end to end through the C ABI with pinned host buffers
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hw, hb1, hb2, hb3 = (pin(a) for a in (prob.w, prob.b1, prob.b2, prob.b3))
    outs = (torch.empty((5,) + mesh.shape, dtype=torch.float64).pin_memory(),
            *[torch.empty(s, dtype=torch.float64).pin_memory() for s in mesh.face_shapes()])
    h2d = sum(t.numel() * 8 for t in (hw, hb1, hb2, hb3))
    d2h = sum(t.numel() * 8 for t in outs)
    ke = max(1, min(args.e2e_steps, args.steps))
    mesh.set_prims(hw, hb1, hb2, hb3)
    mesh.step(mesh.new_dt())
    mesh.get_cons(outs)
    mesh.streamed_steps((hw, hb1, hb2, hb3), outs, 2)
    torch.cuda.synchronize(dev)
    # synchronous: each call waits for the device
    if pg:
        pg.barrier()
    t0 = time.perf_counter()
    for _ in range(ke):
        mesh.set_prims(hw, hb1, hb2, hb3)
        mesh.step(mesh.new_dt())
        mesh.get_cons(outs)
    torch.cuda.synchronize(dev)
    serial_s = max_over_ranks(time.perf_counter() - t0, pg, dev)
    # streamed: the same per-step copies and cycles, stream-ordered, so that one step's copies overlap the
    # neighbouring steps' cycles
    if pg:
        pg.barrier()
    t0 = time.perf_counter()
    mesh.streamed_steps((hw, hb1, hb2, hb3), outs, ke)
    torch.cuda.synchronize(dev)
    e2e_s = max_over_ranks(time.perf_counter() - t0, pg, dev)
    e2e = {"value": whole_job_rate(prob.ncells, ke, e2e_s, world), "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "steps": ke,
           "path": "per step: page-locked inputs to the device on a copy stream, vl2_set_prims_async, vl2_step_cfl "
                   "(CFL dt formed on the device), vl2_get_cons to device buffers, result to page-locked host on a "
                   "second copy stream; double-buffered, event-ordered (Mesh.streamed_steps)",
           "synchronous": {"value": whole_job_rate(prob.ncells, ke, serial_s, world), "unit": UNIT,
                           "path": "vl2_set_prims (page-locked host) + vl2_new_dt + vl2_step + vl2_get_cons "
                                   "(page-locked host) per step, each waiting for the device"}}
    divb = mesh.divb_norm()
    floors = mesh.floor_count()
    mesh.close()
    mesh = None
    torch.cuda.empty_cache()
    forms = None
    if not args.no_forms:
        forms = run_forms(args, dev, stream, vl2, inputs)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, done, threads, el = oracle_rate(args.n, args.mb, 1, 0, min_seconds=10.0, max_steps=3)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu": cpu_model(),
               "sample": "%d VL2 cycle(s) of the full %d^3 workload (%d MeshBlocks), %.1f s" % (
                   done, args.n, (args.n // args.mb) ** 3, el)}
        # one thread, on a 64^3 sample of the same vortex (one cycle)
        set_orc_threads(1)
        r1, d1, _, e1 = oracle_rate(64, 32, 1, 0, max_steps=1)
        set_orc_threads(threads)
        cpu["single_thread"] = {"value": r1, "unit": UNIT, "cores": 1,
                                "sample": "%d VL2 cycle of a 64^3 sample of the vortex (8 MeshBlocks), %.1f s" % (d1, e1)}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(args),
                "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "hbm": hbm,
                "kernels": kernel_share, "cpu_baseline": cpu, "divb_norm": divb, "floor_events": floors,
                "runs": {"blocks": len(run_ms), "ms_per_step": [round(x, 4) for x in run_ms],
                         "median_ms_per_step": float(np.median(run_ms)),
                         "note": "the timed steps in equal consecutive blocks, event-timed; value uses all of them"},
                "forms": forms}
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
