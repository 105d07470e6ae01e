#!/usr/bin/env python
"""Benchmark: grid-point updates/s of the Lax-Wendroff Teukolsky step on GB300.

Workload: the paper-scale single mode (s=-2, m=2, a=0.9; N_r*=16384 over r* in
[-200, 800], N_theta=256; circular-orbit source at r0=8M; extraction at r*=700).
One bench step = --chunk-steps full time steps (predictor + corrector + source +
extraction) of that grid.  The headline value is the FP32-Kahan path; the FP64
path is timed beside it, and the oracle (single-threaded FP64 C) is timed on the
host cores on a bounded sample.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank advances its own replica of the grid (weak scaling);
times are the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "paper-scale single mode 16384x256 (s=-2, m=2, a=0.9, r*=[-200,800], r0=8M, r*_ext=700)"
KAHAN_BYTES_PER_UPDATE = 64   # read + write of (hi, c) for Phi and Pi, FP32
FP64_BYTES_PER_UPDATE = 64    # read + write of Phi and Pi, FP64 (and double-float)
FP32_BYTES_PER_UPDATE = 32    # read + write of Phi and Pi, plain FP32
FP64_FLOPS_PER_UPDATE = 156   # FP64 flops of one point update in the kernel's formulation (FMA = 2)
FP64_PEAK_TFLOPS = 1.25       # GB300 FP64 (non-tensor) nominal: 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_hash():
    """Hash of the step kernel's sources with comments and blank lines removed (what
    the compiler sees), so that a comment edit keeps the recorded counters valid."""
    h = hashlib.sha256()
    for f in ("teuk_step.cu", "teuk_step_common.cuh", "teuk_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1001_3631_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        src = "\n".join(line.rstrip() for line in src.splitlines() if line.strip())
        h.update(src.encode())
    return h.hexdigest()[:16]


def ncu_traffic(prec):
    """DRAM bytes per launch of the step kernel from the committed ncu summary, if the
    kernel source is unchanged since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        ent = d.get(prec)
        if ent and ent.get("kernel_hash") == kernel_hash():
            return float(ent["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(times_ms, units_per_rank):
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    t = max(times_ms)
    return sum(units_per_rank) / (t * 1e-3), t


def reduce_max(x, world):
    if world == 1:
        return [x]
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    out = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(out, t)
    return [float(o.item()) for o in out]


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def moving_path(dt, n_steps):
    """Samples of the bench's moving particle for n_steps time steps: a Keplerian path
    (p = 10, e = 0.4, inclination 0.3, from anomaly 1.0)."""
    from paper_1001_3631_gb300 import inputs
    return inputs.eccentric_trajectory(2 * n_steps + 2, dt, semi_latus=10.0, ecc=0.4, incl=0.3,
                                       chi0=1.0)


def time_path(prec, cfg, S, K, W, world, dev_index, moving=False):
    import torch

    from paper_1001_3631_gb300 import TeukSolver
    p = cfg["params"]
    s = TeukSolver(dict(p, prec=prec))
    if moving:
        s.set_trajectory(moving_path(s.geometry()["dt"], (W + K) * S))
    else:
        s.set_source(cfg["r0"])
    for _ in range(W):
        s.step(S)
    torch.cuda.synchronize()
    barrier(world)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = s.kernel_launches()
    clk = Clocks(dev_index)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(K):
        s.step(S)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    barrier(world)
    ms = e0.elapsed_time(e1)
    launches = s.kernel_launches() - l0
    npts = p["n_rstar"] * p["n_theta"]
    s.sync()
    return s, ms, launches, npts, clocks


def moving_leg(cfg, S, world, dev_index, K=4, W=3):
    """The paper-scale grid with the particle on a sampled eccentric, inclined path
    (FP32-Kahan): per-step Gaussian factor tables instead of a fixed profile."""
    s, ms, launches, npts, clocks = time_path("fp32_kahan", cfg, S, K, W, world, dev_index,
                                              moving=True)
    dt = s.geometry()["dt"]
    s.close()
    r = moving_path(dt, (W + K) * S)[:, 0]
    peak, kind = measured_peaks()
    ach = KAHAN_BYTES_PER_UPDATE * npts / (ms / (K * S) * 1e-3) / 1e9
    return {"value": K * S * npts / (ms * 1e-3), "unit": "updates/s", "ms_per_step": ms / K,
            "time_steps": K * S, "gpu_launches": int(launches),
            "path": "Keplerian p = 10, e = 0.4, inclination 0.3; r_p %.2f-%.2f over the run"
                    % (r.min(), r.max()),
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": ach / peak, "traffic": ncu_traffic("fp32_kahan_moving"),
                         "peak_source": kind, "bytes_per_update": KAHAN_BYTES_PER_UPDATE,
                         "kernel": "step_kernel_s<PK, true>"},
            "clocks": clocks}


def e2e_path(prec, cfg, S, K, W):
    """Same metric through the C ABI with host buffers: each step uploads the initial
    state from pinned host memory, advances S steps and reads the waveform back."""
    import numpy as np
    import torch

    from paper_1001_3631_gb300 import TeukSolver, inputs
    p = cfg["params"]
    s = TeukSolver(dict(p, prec=prec, wave_capacity=S + 1))
    s.set_source(cfg["r0"])
    host_u = torch.empty((4, p["n_theta"], p["n_rstar"]), dtype=torch.float64,
                         pin_memory=True).numpy()
    host_u[...] = inputs.smooth_state(p["n_theta"], p["n_rstar"], seed=5)
    host_w = torch.empty((S + 1, p["n_theta"], 2), dtype=torch.float64, pin_memory=True).numpy()
    import ctypes

    from paper_1001_3631_gb300 import _lib
    lib = _lib.load()
    nw, first = ctypes.c_int64(0), ctypes.c_int64(0)

    def one():
        _lib.check(lib.teuk_set_state(s.ctx, 0, _lib.ptr(host_u), 0), s.ctx)
        _lib.check(lib.teuk_step_n(s.ctx, S), s.ctx)
        _lib.check(lib.teuk_extract(s.ctx, 0, _lib.ptr(host_w), None, S + 1, ctypes.byref(nw),
                                    ctypes.byref(first)), s.ctx)

    for _ in range(W):
        one()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        one()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    npts = p["n_rstar"] * p["n_theta"]
    s.close()
    return {"value": K * S * npts / dt, "unit": "updates/s",
            "h2d_bytes_per_step": int(host_u.nbytes), "d2h_bytes_per_step": int(host_w.nbytes)}


GOLDEN_PAPER_SCALE = os.path.join(ROOT, "tests", "golden", "paper_scale_16384x256_probe.npz")


def accuracy(cfg, n_steps=4000, probe=12.0, every=100):
    """Every path on the paper-scale grid against the oracle: the oracle's waveform at a
    near-zone probe r* = 12 every 100 steps and its final state at every 512th r* column
    after 4000 steps (a stored file written by tests/golden/make_paper_scale_probe.py,
    which calls only the oracle); without the file, against the FP64 path.  The extraction
    radius of the workload (r* = 700) is not reached in a few thousand steps of
    dt ~ 1e-3, so the waveform is taken next to the particle (r*(r0) = 10.2).  Waveform
    error: largest |W - W_ref| / |W_ref| over the checkpoints (theta rows as the vector);
    state error: relative L2 over the stored columns."""
    import numpy as np

    from paper_1001_3631_gb300 import TeukSolver
    p = dict(cfg["params"], rstar_ext=probe)
    golden = None
    if os.path.exists(GOLDEN_PAPER_SCALE):
        g = np.load(GOLDEN_PAPER_SCALE)
        if int(g["steps"][-1]) == n_steps and int(g["steps"][1] - g["steps"][0]) == every:
            golden = g
    res = {"steps": n_steps, "probe_rstar": probe, "every": every,
           "reference": "oracle (stored records)" if golden is not None else "FP64 GPU path"}
    runs = {}
    for prec in ("fp64", "fp64_df", "fp32_kahan", "fp32"):
        with TeukSolver(dict(p, prec=prec, wave_capacity=n_steps + 1)) as s:
            s.set_source(cfg["r0"])
            s.step(n_steps)
            u = s.get_state()
            w, first = s.extract()
            s.sync()
        runs[prec] = (u, w[::every])
    if golden is not None:
        ref_w, cols = golden["probe12"], golden["final_cols"]
        ref_u = golden["final_state"]
    else:
        ref_w, cols = runs["fp64"][1], np.arange(0, p["n_rstar"], 512)
        ref_u = runs["fp64"][0][:, :, cols]
    norms = np.linalg.norm(ref_w.reshape(len(ref_w), -1), axis=1)
    # checkpoints at which the particle's field has reached the probe (above 1e-3 of its
    # largest value; the earlier records are a numerical precursor of ~1e-14)
    arrived = [k for k in range(1, len(ref_w)) if norms[k] >= 1e-3 * norms.max()]
    res["signal_from_step"] = int(arrived[0] * every)
    for prec, (u, w) in runs.items():
        if golden is None and prec == "fp64":
            continue
        errs = [float(np.linalg.norm(w[k] - ref_w[k]) / norms[k]) for k in arrived]
        res[prec] = {"waveform_rel_err_max": max(errs), "waveform_rel_err_final": errs[-1],
                     "state_rel_l2": float(np.linalg.norm(u[:, :, cols] - ref_u) / np.linalg.norm(ref_u))}
    return res


def batched_leg(n_calls=2, steps_per_call=100, warm_calls=1):
    """The 128-instance uneven workload (8 modes x 16 orbits) in FP32-Kahan: one
    persistent launch per block-size class and call (100 steps), replayed from a CUDA
    graph on a side stream, tiles from the autotuner's cached table."""
    import torch

    from paper_1001_3631_gb300 import TeukSolver, inputs
    insts = inputs.batched_uneven()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = TeukSolver([dict(i["params"], prec="fp32_kahan") for i in insts], stream=stream)
        for k, inst in enumerate(insts):
            s.set_source(inst["r0"], instance=k)
        chunks = s.autotune(trial_steps=5)   # strips timed on the whole batch
        for _ in range(warm_calls):
            s.step(steps_per_call)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        l0 = s.kernel_launches()
        e0.record(stream)
        for _ in range(n_calls):
            s.step(steps_per_call)
        e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1)
        launches = (s.kernel_launches() - l0) // n_calls
        s.sync()
        npts = sum(i["params"]["n_rstar"] * i["params"]["n_theta"] for i in insts)
        s.close()
    return {"workload": "128 instances: m=1..8 x 16 orbits, N_r* in {2048..16384}, "
                        "N_theta in {64,128,256} (seed 3003), FP32-Kahan",
            "value": npts * n_calls * steps_per_call / (ms * 1e-3), "unit": "updates/s",
            "points": npts, "steps_timed": n_calls * steps_per_call,
            "ms_per_call": ms / n_calls, "launches_per_call": int(launches),
            "distinct_strips": sorted(set(chunks))}


def single_mode_leg(steps=2000):
    """The 800 x 64 single mode (51,200 points, L2-resident): one kernel per step, the
    persistent batched kernel replayed from a CUDA graph (strip length from the
    autotuner), and resident launches (the grid in shared memory, one cooperative launch
    per call; halo 1 .. 4 and 1 .. 3 blocks per SM timed, the fastest reported), blocked
    launches (1 .. 4 steps a launch of the grid held in shared memory, no exchange; shapes
    timed the same way), for FP64,
    the FP64-equivalent
    double-float path, FP32-Kahan and FP32.  hbm_frac is the algorithmic bytes per update
    against the measured HBM copy bandwidth (the grid is L2-resident, so this is the
    fraction of the HBM roofline, not a DRAM measurement); native FP64 is also stated
    against its ALU ceiling (156 flops per update at the nominal FP64 rate)."""
    import torch

    from paper_1001_3631_gb300 import TeukSolver, inputs
    cfg = inputs.SINGLE_MODE_800x64
    out = {"workload": "single mode 800x64 (s=-2, m=2, a=0.9), %d steps" % steps}
    peak, _ = measured_peaks()
    frac = {}
    for prec in ("fp64", "fp64_df", "fp32_kahan", "fp32"):
        bpu = FP32_BYTES_PER_UPDATE if prec == "fp32" else 64
        for mode in ("per_step", "persistent", "resident", "blocked"):
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                s = TeukSolver(dict(cfg["params"], prec=prec), stream=stream)
                s.set_tiling(0, 0 if mode == "persistent" else 1)
                s.set_source(cfg["r0"])
                if mode == "persistent":
                    # strip length of the persistent kernel from the autotuner (timed on
                    # this context; a fresh table so that it always measures)
                    with tempfile.TemporaryDirectory() as td:
                        out["%s_persistent_strip" % prec] = int(
                            s.autotune(trial_steps=20, cache_path=os.path.join(td, "t.json"))[0])
                elif mode in ("resident", "blocked"):
                    best = None
                    for h, bps in [(h, b) for b in (1, 2, 3) for h in (1, 2, 3, 4)]:
                        try:
                            if mode == "resident":
                                s.set_resident(h, bps)
                            else:
                                s.set_blocked(h, bps)
                        except Exception:
                            continue
                        s.step(200)
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        stream.synchronize()
                        e0.record(stream)
                        s.step(400)
                        e1.record(stream)
                        stream.synchronize()
                        ms = e0.elapsed_time(e1)
                        if best is None or ms < best[0]:
                            best = (ms, h, bps)
                    if mode == "resident":
                        s.set_resident(best[1], best[2])
                    else:
                        s.set_blocked(best[1], best[2])
                    out["%s_%s_halo" % (prec, mode)] = best[1]
                    out["%s_%s_blocks_per_sm" % (prec, mode)] = best[2]
                s.step(steps)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                stream.synchronize()
                e0.record(stream)
                s.step(steps)
                e1.record(stream)
                stream.synchronize()
                ms = e0.elapsed_time(e1)
                s.sync()
                s.close()
            ups = 51200 * steps / (ms * 1e-3)
            out["%s_%s" % (prec, mode)] = ups
            frac["%s_%s" % (prec, mode)] = bpu * ups / 1e9 / peak
    out["unit"] = "updates/s"
    out["hbm_frac"] = frac
    alu_cap = FP64_PEAK_TFLOPS * 1e12 / FP64_FLOPS_PER_UPDATE
    out["fp64_alu_cap"] = alu_cap
    out["fp64_alu_frac"] = {m: out["fp64_" + m] / alu_cap for m in ("per_step", "persistent", "resident", "blocked")}
    out["best"] = {p: max(("per_step", "persistent", "resident", "blocked"), key=lambda m: out["%s_%s" % (p, m)])
                   for p in ("fp64", "fp64_df", "fp32_kahan", "fp32")}
    return out


def adjoint_leg(peaks=None):
    """The adjoint workload (4096 x 128, 10000 steps, A_n ~ N(1, 0.1) seed 5005, loss at a
    near-zone probe r* = 12.5): the forward run alone; the built-in-loss gradient call
    without checkpoints (forward sweep keeping every record's cotangent, then the reverse
    sweep) and with a checkpoint every 100 steps (each segment's records recomputed from
    its checkpoint in the reverse sweep), each timed on the host around a synchronising
    call; and the reverse sweep alone (cotangent mode) timed with CUDA events, with its
    bytes per update: the co-state read and written once a step (FP32 instances: value
    and compensation planes of lam_Phi and lam_Pi, 4 x 8 B each way; FP64: 2 x 16 B each
    way) = 64 B.  The 4096 x 128 co-state (2 x 16.8 MB) stays in L2, so the fraction of
    the measured HBM copy rate can exceed what DRAM alone would allow."""
    import numpy as np
    import torch

    from paper_1001_3631_gb300 import TeukSolver, inputs
    cfg = inputs.ADJOINT_4096x128
    p = dict(cfg["params"], rstar_ext=12.5)
    n, npts = cfg["steps"], cfg["params"]["n_rstar"] * cfg["params"]["n_theta"]
    nth = cfg["params"]["n_theta"]
    amps = inputs.amplitudes(n, seed=cfg["amp_seed"])
    out = {"workload": "adjoint 4096x128, %d steps; checkpointed mode: every %d steps" % (n, cfg["ckpt_every"])}
    gw = np.random.default_rng(cfg["amp_seed"]).standard_normal((n, nth, 2))
    hbm = (peaks or {}).get("hbm_gbs")
    for prec in ("fp64", "fp32_kahan"):
        with TeukSolver(dict(p, prec=prec)) as s:
            s.set_source(cfg["r0"], amps)
            s.adjoint(10, step0=0, grad_wave=gw[:10])   # warm-up (tables, buffers)
            s.set_state(np.zeros(s.shape()), 0)
            t0 = time.perf_counter()
            s.step(n)
            s.sync()
            tf = time.perf_counter() - t0
            res = {"forward_s": tf}
            for ck, key in ((0, "gradient"), (cfg["ckpt_every"], "gradient_ckpt")):
                s.set_state(np.zeros(s.shape()), 0)
                t0 = time.perf_counter()
                s.adjoint(n, step0=0, ckpt_every=ck)
                ta = time.perf_counter() - t0
                res[key + "_s"] = ta
                res[key + "_over_forward"] = ta / tf
            st = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            s.adjoint(n, step0=0, grad_wave=gw)
            e1.record(st)
            torch.cuda.synchronize()
            us = e0.elapsed_time(e1) * 1e3 / n
            gbs = 64.0 * npts / (us * 1e-6) / 1e9
            res.update({"reverse_us_per_step": us, "reverse_bytes_per_update": 64,
                        "reverse_gbs": gbs, "reverse_frac_of_measured_hbm": (gbs / hbm) if hbm else None,
                        "gradient_updates_per_s": npts * n / res["gradient_s"]})
        out[prec] = res
    out["unit_note"] = ("gradient_updates_per_s = forward point-updates covered per second of the "
                        "gradient call; reverse_us_per_step includes the cotangent upload (pageable host "
                        "memory) of the timed call")
    return out


# FP64 flops of the flux diagnostic per (mode, row, record): the two trapezoid updates
# (N, H: 12), |N|^2 and its E and Pz terms (7), Im(conj(N) H) and its Jz term (5),
# N conj(N') times the momentum weight and its two sums (14).
FLUX_FLOPS_PER_ENTRY = 38


def radiated_flux_leg(peaks=None, n_modes=8, n_steps=4000):
    """The recoil diagnostic (teuk_radiated_flux): the modes m = 1..8 of one particle on a
    circular orbit at r0 = 10 (2048 x 256 grid, a = 0.9, FP32-Kahan, the time step of
    the m = 8 mode's rule shared by all) stepped 4000 steps in one batched context, then
    the energy, momentum and Jz fluxes of all 4001 records at r* = 14, next to the
    particle (r* = 12.8).  Timed with CUDA events on the context's stream around the call (it
    allocates its scratch, runs the kernels, copies the [R][10] result back and
    synchronizes), and on the host.  Bytes: the records read once (16 B per mode, row
    and record) are the algorithmic minimum; the kernels read them twice (the chunk
    totals, then the sums).  The work is FP64 arithmetic (38 flops per mode, row and
    record), which bounds the call on GB300 before its bytes do: the roofline is the FP64
    rate."""
    import torch

    from paper_1001_3631_gb300 import TeukSolver
    ms = list(range(1, n_modes + 1))
    dt = 0.5 * (math.pi / 256) / (n_modes + 2 + 2)    # dt_rule 1 of the largest |m|
    p = dict(s=-2, a=0.9, rstar_min=-60.0, rstar_max=140.0, n_rstar=2048, n_theta=256,
             rstar_ext=14.0, dt=dt, prec="fp32_kahan")
    with TeukSolver([dict(p, m=m) for m in ms]) as s:
        for k in range(len(ms)):
            s.set_source(10.0, instance=k)
        s.step(n_steps)
        s.radiated_flux(0, 64)                     # warm-up (module load, allocator)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        R = n_steps + 1
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0.record(st)
        out = s.radiated_flux(0, R)
        e1.record(st)
        torch.cuda.synchronize()
        th = time.perf_counter() - t0
        ms_ev = e0.elapsed_time(e1)
        s.sync()
    ent = len(ms) * p["n_theta"] * R
    tflops = FLUX_FLOPS_PER_ENTRY * ent / (ms_ev * 1e-3) / 1e12
    gbs = 16.0 * ent / (ms_ev * 1e-3) / 1e9
    hbm = (peaks or {}).get("hbm_gbs")
    return {"workload": "%d modes x %d rows x %d records (2048x256 grid, FP32-Kahan records)"
                        % (len(ms), p["n_theta"], R),
            "ms": ms_ev, "host_ms": th * 1e3, "records_per_s": R / (ms_ev * 1e-3),
            "entry_records_per_s": ent / (ms_ev * 1e-3),
            "roofline": {"bound": "alu", "achieved": tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": tflops / FP64_PEAK_TFLOPS, "flops_per_entry_record": FLUX_FLOPS_PER_ENTRY,
                         "peak_note": "FP64 nominal (152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz)",
                         "pipe_note": "about 39 FP64 instructions per entry and record, mostly "
                                      "adds and multiplies; ncu: the sums kernel keeps the FP64 "
                                      "pipe 86 % busy",
                         "record_bytes_gbs": gbs, "hbm_frac": (gbs / hbm) if hbm else None,
                         "kernel": "the whole call (allocation, four kernels, copy back)"},
            "E_total": float(out[-1, 5]), "P_total": [float(x) for x in out[-1, 6:9]],
            "Jz_total": float(out[-1, 9])}


def cpu_baseline(cfg, budget_s=12.0):
    """The oracle (single-threaded FP64 C) on the same grid, per-step time from the
    difference of two run lengths (so its setup is excluded)."""
    from oracle import teuk_oracle as orc
    p = orc.params(**cfg["params"], r0=cfg["r0"])
    src = orc.orbit_source(p)
    t0 = time.perf_counter()
    orc.run(p, None, 1, src, wave=False)
    t1 = time.perf_counter()
    orc.run(p, None, 3, src, wave=False)
    t2 = time.perf_counter()
    per_step = max((t2 - t1) - (t1 - t0), 1e-9) / 2.0
    n = max(2, int(budget_s / per_step))
    t3 = time.perf_counter()
    orc.run(p, None, n + 1, src, wave=False)
    t4 = time.perf_counter()
    per_step = ((t4 - t3) - (t1 - t0)) / n
    npts = p.n_rstar * p.n_theta
    return {"value": npts / per_step, "unit": "updates/s", "cores": 1, "kind": "oracle",
            "sample": "%d full steps of the %dx%d grid (setup excluded by differencing)"
                      % (n, p.n_rstar, p.n_theta)}


def run_reference(args, world, rank):
    """The reference arm: the oracle (single-threaded FP64 C, the only reference this
    paper has) on the host cores, on the same 16384 x 256 workload.  One bench step is
    one full time step; the per-step time comes from two run lengths (warmup and
    warmup + steps) so the oracle's setup is excluded."""
    if rank != 0:
        return 0
    from oracle import teuk_oracle as orc
    from paper_1001_3631_gb300 import inputs
    cfg = inputs.PAPER_SCALE_16384x256
    p = orc.params(**cfg["params"], r0=cfg["r0"])
    src = orc.orbit_source(p)
    W, K = max(1, args.warmup), max(1, args.steps)
    t0 = time.perf_counter()
    orc.run(p, None, W, src, wave=False)
    t1 = time.perf_counter()
    orc.run(p, None, W + K, src, wave=False)
    t2 = time.perf_counter()
    per_step = max((t2 - t1) - (t1 - t0), 1e-9) / K
    npts = p.n_rstar * p.n_theta
    value = npts / per_step
    cb = {"value": value, "unit": "updates/s", "cores": 1, "kind": "oracle",
          "sample": "%d timed full steps of the %dx%d grid (setup excluded by differencing)"
                    % (K, p.n_rstar, p.n_theta)}
    line = {"impl": "reference", "metric": "grid-point updates/s", "value": value,
            "unit": "updates/s", "n_gpus": args.gpus, "steps": K, "warmup": W,
            "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "impl": "oracle on host cores",
                       "time_steps_per_bench_step": 1},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


GOLDEN_LONG_RUN = os.path.join(ROOT, "tests", "golden", "long_run_8192x128_probe.npz")


def precision_sweep(steps=100000, every=1000, probe=30.0):
    """Long run of the 8192 x 128 single mode at a = 0.99 (r* in [-200, 800], r0 = 8M,
    dt rule 1): the waveform record every `every` steps of FP64, the FP64-equivalent
    double-float path, FP32-Kahan and FP32, against the oracle's records (a stored file
    written by tests/golden/make_long_run_probe.py, which calls only the oracle) or, if it
    is absent, against the FP64 path.  The waveform is taken at the near-zone probe
    r* = 30: at the stated extraction radius r* = 400 it is identically zero over the run
    (the particle's signal needs about 390 M, the run spans 204 M).  Error of a record:
    |W - W_ref| / |W_ref| over the theta rows.  Also the growth of a perturbation: two
    double-float runs whose initial states differ by 1e-12 (max norm, grid-scale random),
    compared at the probe every 10000 steps -- a property of the discretized equation on
    this grid, the factor by which any rounding difference is amplified."""
    import numpy as np
    import torch

    from paper_1001_3631_gb300 import TeukSolver, inputs
    cfg = inputs.LONG_RUN_8192x128
    par = dict(cfg["params"], rstar_ext=probe, wave_capacity=2)
    golden = None
    if os.path.exists(GOLDEN_LONG_RUN):
        g = np.load(GOLDEN_LONG_RUN)
        if int(g["steps"][-1]) >= steps and int(g["steps"][1] - g["steps"][0]) == every:
            golden = g["probe30"]
    out = {"workload": "long run 8192x128 (s=-2, m=2, a=0.99, r*=[-200,800], r0=8M), %d steps" % steps,
           "every": every, "probe_rstar": probe,
           "reference": "oracle records (stored)" if golden is not None else "FP64 GPU path",
           "rstar_400": "waveform identically zero over the run (signal arrives after ~390 M)"}
    recs = {}
    for prec in ("fp64", "fp64_df", "fp32_kahan", "fp32"):
        s = TeukSolver(dict(par, prec=prec))
        s.set_source(cfg["r0"])
        r = np.zeros((steps // every + 1, par["n_theta"], 2))
        t0 = time.perf_counter()
        for k in range(1, steps // every + 1):
            s.step(every)
            r[k] = s.extract(cap=1)[0][0]
        s.sync()
        out["seconds_" + prec] = time.perf_counter() - t0
        s.close()
        recs[prec] = r
    ref = golden if golden is not None else recs["fp64"]
    ck = list(range(every, steps + 1, every))
    # checkpoints at which the particle's signal has reached the probe (|W| above 1e-3 of
    # its largest value over the run; before that the record is a numerical precursor
    # ~1e-30 .. 1e-120, which FP32 does not represent)
    norms = np.array([np.linalg.norm(ref[k]) for k in range(steps // every + 1)])
    arrived = norms >= 1e-3 * norms.max()
    out["signal_from_step"] = int(ck[int(np.argmax(arrived[1:]))])
    for prec in ("fp64", "fp64_df", "fp32_kahan", "fp32"):
        if golden is None and prec == "fp64":
            continue
        e = [float(np.linalg.norm(recs[prec][k] - ref[k]) / norms[k]) if arrived[k] else None
             for k in range(1, steps // every + 1)]
        valid = [(n, x) for n, x in zip(ck, e) if x is not None]
        first_above = next((n for n, x in valid if x > 1e-6), None)
        out[prec] = {"rel_err_every_5000": [x for n, x in zip(ck, e) if n % 5000 == 0],
                     "max_to_40000": max(x for n, x in valid if n <= 40000),
                     "final": valid[-1][1], "max": max(x for _, x in valid),
                     "first_step_above_1e-6": first_above}
    # amplification of a grid-scale perturbation, FP64-class arithmetic only
    eps = 1e-12
    du = np.random.default_rng(1).standard_normal((4, par["n_theta"], par["n_rstar"]))
    du[:, :, 0] = du[:, :, -1] = 0
    du *= eps / np.abs(du).max()
    a, b = TeukSolver(dict(par, prec="fp64_df")), TeukSolver(dict(par, prec="fp64_df"))
    for x in (a, b):
        x.set_source(cfg["r0"])
    b.set_state(du, 0)
    amp = []
    for k in range(1, steps // 10000 + 1):
        a.step(10000)
        b.step(10000)
        wa, wb = a.extract(cap=1)[0][0], b.extract(cap=1)[0][0]
        amp.append(float(np.linalg.norm(wb - wa) / np.linalg.norm(wa) / eps))
    a.close()
    b.close()
    out["perturbation_growth"] = {"eps_max_norm": eps, "every": 10000,
                                  "waveform_rel_change_over_eps": amp}
    return out


def batched_accuracy(steps=10000, n_pick=16):
    """FP32-Kahan against the FP64-equivalent double-float path (which equals the oracle
    to 1e-12 in the tests) on n_pick instances of the 128-instance workload, one per
    (N_theta, N_r*) class and both pole parities, each in one batched context, after the
    workload's 10000 steps: waveform at a near-zone probe r* = r*(r0) + 2 (the stated
    r* = 700 is not reached in 10000 steps of dt = 5e-4 .. 5e-3) and the final state."""
    import numpy as np

    from paper_1001_3631_gb300 import TeukSolver, inputs
    insts = inputs.batched_uneven()
    seen, picks = set(), []
    for k, i in enumerate(insts):
        key = (i["params"]["n_theta"], i["params"]["n_rstar"], i["params"]["m"] % 2)
        if key not in seen:
            seen.add(key)
            picks.append(k)
    picks = picks[:n_pick]
    res = {}
    for prec in ("fp64_df", "fp32_kahan"):
        ps = []
        for k in picks:
            p = dict(insts[k]["params"], prec=prec, wave_capacity=steps + 1)
            M, a, r0 = p["M"], p["a"], insts[k]["r0"]
            rp = M + (M * M - a * a) ** 0.5
            rm = M - (M * M - a * a) ** 0.5
            kk = 2.0 * M / (rp - rm)
            rs0 = r0 + kk * rp * np.log((r0 - rp) / (2 * M)) - kk * rm * np.log((r0 - rm) / (2 * M))
            p["rstar_ext"] = float(rs0 + 2.0)
            ps.append(p)
        with TeukSolver(ps) as s:
            for q, k in enumerate(picks):
                s.set_source(insts[k]["r0"], instance=q)
            s.step(steps)
            res[prec] = [(s.get_state(q), s.extract(instance=q)[0]) for q in range(len(picks))]
            s.sync()
    ew, es = [], []
    for q in range(len(picks)):
        (u0, w0), (u1, w1) = res["fp64_df"][q], res["fp32_kahan"][q]
        ew.append(float(np.linalg.norm(w1 - w0) / np.linalg.norm(w0)))
        es.append(float(np.linalg.norm(u1 - u0) / np.linalg.norm(u0)))
    return {"instances": picks, "steps": steps, "reference": "FP64-equivalent double-float path",
            "waveform_rel_err_max": max(ew), "waveform_rel_err_median": float(np.median(ew)),
            "state_rel_err_max": max(es)}


def summary(line):
    """The headline figures of every leg in a few keys (printed last in the JSON line)."""
    def g(*ks):
        d = line
        for k in ks:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return d
    sm = line.get("single_mode_800x64", {})
    best = sm.get("best", {})
    return {
        "16384x256_updates_per_s": {"fp32_kahan": line.get("value"), "fp64": g("fp64", "value"),
                                    "fp64_df": g("fp64_df", "value"), "fp32": g("fp32", "value")},
        "16384x256_hbm_frac": {"fp32_kahan": g("roofline", "frac"), "fp64_df": g("fp64_df", "roofline", "frac"),
                               "fp32": g("fp32", "roofline", "frac")},
        "fp64_alu_frac": g("fp64", "roofline", "frac"),
        "800x64_best_updates_per_s": {p: sm.get("%s_%s" % (p, m)) for p, m in best.items()},
        "800x64_best_mode": best,
        "batched_updates_per_s": g("batched", "value"),
        "batched_kahan_waveform_err_max": g("batched", "accuracy", "waveform_rel_err_max"),
        "16384x256_waveform_err_vs_oracle": {p: g("accuracy", p, "waveform_rel_err_max")
                                             for p in ("fp64", "fp64_df", "fp32_kahan", "fp32")},
        "moving_particle_hbm_frac": g("moving_particle", "roofline", "frac"),
        "long_run_first_step_above_1e-6": {p: g("precision_sweep", p, "first_step_above_1e-6")
                                           for p in ("fp32_kahan", "fp32", "fp64_df")},
        "long_run_final_err": {p: g("precision_sweep", p, "final") for p in ("fp32_kahan", "fp32", "fp64_df", "fp64")},
        "adjoint_gradient_over_forward": {p: g("adjoint", p, "gradient_over_forward") for p in ("fp64", "fp32_kahan")},
        "adjoint_ckpt_gradient_over_forward": {p: g("adjoint", p, "gradient_ckpt_over_forward")
                                               for p in ("fp64", "fp32_kahan")},
        "adjoint_reverse_us_per_step": {p: g("adjoint", p, "reverse_us_per_step") for p in ("fp64", "fp32_kahan")},
        "radiated_flux_ms": g("radiated_flux", "ms"),
        "cpu_baseline": g("cpu_baseline", "value"),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--chunk-steps", type=int, default=500)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the accuracy, end-to-end and CPU-baseline legs")
    ap.add_argument("--only", choices=["fp32_kahan", "fp64", "fp64_df", "fp32", "moving"], default=None,
                    help="time one path only (for profiler captures)")
    ap.add_argument("--accuracy-steps", type=int, default=4000)
    ap.add_argument("--precision-sweep", action="store_true",
                    help="run the 8192x128 long-run precision sweep alone and print its JSON")
    ap.add_argument("--no-sweep", action="store_true", help="skip the long-run precision sweep")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    args.warmup = max(args.warmup, 3)

    import torch
    torch.cuda.set_device(local)
    if args.precision_sweep:
        from paper_1001_3631_gb300 import build as b
        b.build()
        print(json.dumps(precision_sweep()))
        return 0
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1001_3631_gb300 import build as b
    from paper_1001_3631_gb300 import inputs
    b.build()
    cfg = inputs.PAPER_SCALE_16384x256
    S, K, W = args.chunk_steps, args.steps, args.warmup

    if args.only:
        if args.only == "moving":
            s_o, ms_o, _, _, _ = time_path("fp32_kahan", cfg, S, K, W, world, local, moving=True)
        else:
            s_o, ms_o, _, _, _ = time_path(args.only, cfg, S, K, W, world, local)
        s_o.close()
        if rank == 0:
            print(json.dumps({"only": args.only, "ms": ms_o, "time_steps": K * S}))
        return 0
    s_k, ms_k, launches_k, npts, clocks = time_path("fp32_kahan", cfg, S, K, W, world, local)
    s_k.close()
    s_d, ms_d, launches_d, _, clocks_d = time_path("fp64", cfg, S, K, W, world, local)
    s_d.close()
    s_f, ms_f, _, _, clocks_f = time_path("fp64_df", cfg, S, K, W, world, local)
    s_f.close()
    s_p, ms_p, _, _, _ = time_path("fp32", cfg, S, K, W, world, local)
    s_p.close()
    ms_p_all = reduce_max(ms_p, world)
    ms_k_all = reduce_max(ms_k, world)
    ms_d_all = reduce_max(ms_d, world)
    ms_f_all = reduce_max(ms_f, world)
    units = K * S * npts
    val_k, tk = aggregate(ms_k_all, [units] * world)
    val_d, td = aggregate(ms_d_all, [units] * world)
    val_f, tf = aggregate(ms_f_all, [units] * world)
    val_p, tp = aggregate(ms_p_all, [units] * world)

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0

    peak, peak_kind = measured_peaks()
    step_launches = K * S
    avg_k = tk / step_launches          # ms per step-kernel launch (extract kernel included)
    avg_d = td / step_launches
    ach_k = KAHAN_BYTES_PER_UPDATE * npts / (avg_k * 1e-3) / 1e9
    traffic = ncu_traffic("fp32_kahan")
    fp64_tflops = FP64_FLOPS_PER_UPDATE * npts / (avg_d * 1e-3) / 1e12
    line = {
        "metric": "grid-point updates/s", "value": val_k, "unit": "updates/s",
        "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": tk / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32-kahan", "data": "synthetic",
        "config": {"workload": WORKLOAD, "time_steps_per_bench_step": S,
                   "precision": "FP32 stencil, Kahan-compensated state; FP64 tables/source/extraction",
                   "l2": "inputs larger than L2 (ping-pong state 268 MB FP32-Kahan, 268 MB + 604 MB tables FP64)",
                   "parallelism": "replica per GPU" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": ach_k, "peak": peak, "unit": "GB/s",
                     "frac": ach_k / peak, "traffic": traffic,
                     "peak_source": peak_kind, "bytes_per_update": KAHAN_BYTES_PER_UPDATE,
                     "kernel": "step_kernel<PK>"},
        "fp64": {"value": val_d, "unit": "updates/s", "ms_per_step": td / K,
                 "roofline": {"bound": "alu", "achieved": fp64_tflops, "peak": FP64_PEAK_TFLOPS,
                              "unit": "TFLOP/s", "frac": fp64_tflops / FP64_PEAK_TFLOPS,
                              "flops_per_update": FP64_FLOPS_PER_UPDATE,
                              "hbm_frac": FP64_BYTES_PER_UPDATE * npts / (avg_d * 1e-3) / 1e9 / peak,
                              "kernel": "step_kernel<P64>"},
                 "clocks": clocks_d},
        "fp64_df": {"value": val_f, "unit": "updates/s", "ms_per_step": tf / K,
                    "note": "FP64-equivalent double-float path (hi + lo FP32 pairs) on the FP32 units",
                    "roofline": {"bound": "hbm", "achieved": FP64_BYTES_PER_UPDATE * npts / (tf / step_launches * 1e-3) / 1e9,
                                 "peak": peak, "unit": "GB/s",
                                 "frac": FP64_BYTES_PER_UPDATE * npts / (tf / step_launches * 1e-3) / 1e9 / peak,
                                 "traffic": ncu_traffic("fp64_df"),
                                 "bytes_per_update": FP64_BYTES_PER_UPDATE, "kernel": "step_kernel<PD>"},
                    "over_fp64": val_f / val_d, "clocks": clocks_f},
        "fp32": {"value": val_p, "unit": "updates/s", "ms_per_step": tp / K,
                 "note": "plain FP32 state and arithmetic",
                 "roofline": {"bound": "hbm", "achieved": FP32_BYTES_PER_UPDATE * npts / (tp / step_launches * 1e-3) / 1e9,
                              "peak": peak, "unit": "GB/s",
                              "frac": FP32_BYTES_PER_UPDATE * npts / (tp / step_launches * 1e-3) / 1e9 / peak,
                              "bytes_per_update": FP32_BYTES_PER_UPDATE, "kernel": "step_kernel<P32>"}},
        "fp32_kahan_over_fp64": val_k / val_d,
        "gpu_launches": int(launches_k),
        "clocks": clocks,
    }
    if not args.no_extras:
        line["batched"] = batched_leg()
        line["batched"]["accuracy"] = batched_accuracy()
        mv = moving_leg(cfg, S, world, local)
        mv["over_circular_orbit"] = mv["value"] / val_k
        line["moving_particle"] = mv
        line["single_mode_800x64"] = single_mode_leg()
        line["accuracy"] = accuracy(cfg, n_steps=args.accuracy_steps)
        line["e2e"] = e2e_path("fp32_kahan", cfg, S, max(2, K // 2), 1)
        line["adjoint"] = adjoint_leg({"hbm_gbs": measured_peaks()[0]})
        line["radiated_flux"] = radiated_flux_leg({"hbm_gbs": measured_peaks()[0]})
        if not args.no_sweep:
            line["precision_sweep"] = precision_sweep()
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(cfg)
    line["summary"] = summary(line)
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
