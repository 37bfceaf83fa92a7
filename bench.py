"""Benchmark: active-cell-steps/s of the real-time RK4 GPE step on the
anisotropic thin-shell workload (1024^3 box, ~2.9e7 active cells, g = 2000),
complex64 bulk with FP64 reductions, on one GB300; complex128 reported beside.

One bench step = STEPS_PER_BENCH (100) RK4 time steps over the whole active
set plus one FP64 observables reduction (norm, energy, mu).  Inputs (state,
potential, masks) are larger than L2 and already resident when timing starts.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica (the single-shell step
has no data-parallel exchange); value = cell-steps of all ranks / max time.
--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (a slab of the shell).
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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

STEPS_PER_BENCH = 100
BATCH_STATES = {"c64": (2, np.complex64, "complex64"), "r32": (4, np.float32, "real float")}  # gpe state type ids
FLOOR_CHECKS = 10                 # batch workload: checks that measure the complex64 |dmu| floor
B_ALG = {"c64": 20.0, "c128": 40.0}   # algorithmic bytes per active cell-step (read psi, V; write psi)
METRIC = "shell-grid GPE cell-steps/s: FP32 vs FP64 at stated error; % of HBM roofline"
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "rk4_shell1024_c64_traffic.json")


def kernel_source_hash():
    """Hash of the sources that define the timed RK4 stage kernels (their
    launch code, device code and shared internals)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2603_05447_gb300", "csrc")
    for f in ("gpe_internal.cuh", "stencil.cuh", "step.cu"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.out = index, None, ""

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self):
        rows = [r.split(", ") for r in self.out.strip().splitlines() if r.strip()]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip() == "Active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------- workload
WORKLOADS = {"shell1024": "SHELL_1024", "shell512": "SHELL_512"}
EXTRA = ("ramp2048", "adjoint512", "batch", "roi_sweep", "stages512", "ramp_traced")
_workload_name = "shell1024"


def shell_workload():
    from paper_2603_05447_gb300 import inputs
    return getattr(inputs, WORKLOADS[_workload_name])


def build_grid(gpe, wl, brick=(8, 8, 4), sched=0, chunk=0):
    b = wl.box
    gb = gpe.make_box(b.nx, b.ny, b.nz, b.hx)
    pot = gpe.make_potential(gpe.GPE_POT_ELLIPSOID_SHELL, wl.w, *wl.axes)
    return gpe.gpe_grid_create_analytic(gb, pot, wl.V_cut, gpe.make_opts(brick, sched=sched, chunk=chunk))


def initial_compact(gpe, inputs, wl, grid):
    """Shell profile with smooth seeded phase noise at every active cell, in
    the compact layout."""
    info = gpe.gpe_grid_get_info(grid)
    idx, i, j, k = gpe.packed_coords(grid)
    b = wl.box
    out = np.zeros(info.n_packed, np.complex128)
    step = 1 << 22
    for s in range(0, idx.size, step):
        sl = slice(s, s + step)
        out[idx[sl]] = inputs.shell_initial_psi(wl, b.x0 + i[sl] * b.hx, b.y0 + j[sl] * b.hy, b.z0 + k[sl] * b.hz)
    out *= math.sqrt(wl.N / (np.sum(np.abs(out) ** 2) * b.dV))
    return out


# ----------------------------------------------------------------- CPU oracle sample
def oracle_sample(wl, target_s=12.0, layers=48):
    """A slab of `layers` z-planes through the shell's equator: (grid, V, psi)."""
    import oracle
    from paper_2603_05447_gb300 import inputs
    b = wl.box
    x, y, z = b.axes()
    k0 = b.nz // 2 - layers // 2
    zs = z[k0:k0 + layers]
    Z, Y, X = np.meshgrid(zs, y, x, indexing="ij")
    V = wl.potential(X, Y, Z)
    mask = V < wl.V_cut
    g = oracle.Grid(mask, b.hx)
    xc, yc, zc = X[mask], Y[mask], Z[mask]
    psi = inputs.shell_initial_psi(wl, xc, yc, zc)
    psi *= math.sqrt(1.0 / (np.sum(np.abs(psi) ** 2) * b.dV))
    return g, g.compact(V), psi


def _oracle_rk4_rate(oracle, g, V, psi, gg, dt, steps):
    """Active-cell RK4 steps per second of the FP64 oracle over `steps` steps."""
    y = oracle.rk4_step(g, V, psi, gg, 0.0, dt)                  # first touch
    t0 = time.perf_counter()
    for q in range(steps):
        y = oracle.rk4_step(g, V, y, gg, (q + 1) * dt, dt)
    el = time.perf_counter() - t0
    return {"value": g.n * steps / el, "unit": "cell-steps/s", "steps": steps, "n_active": g.n,
            "seconds": round(el, 3)}


def cpu_baseline(wl):
    """The FP64 oracle on the host cores: the headline shell (a slab of it, 100
    RK4 steps), the all-active 64^3 harmonic trap (C1, 100 RK4 steps), and
    both on a single thread (the paper's CPU figures are single-threaded);
    cores = the CPUs this process may run on (its affinity mask)."""
    import oracle
    from paper_2603_05447_gb300 import inputs
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    used = oracle.set_threads(cores)
    g, V, psi = oracle_sample(wl)
    dt = wl.stable_dt()
    c2 = _oracle_rk4_rate(oracle, g, V, psi, wl.g, dt, 100)
    box = inputs.cubic_box(64, 0.25)
    Vd = inputs.dense_potential(box, inputs.Harmonic())
    g1 = oracle.Grid(np.ones(box.shape, bool), box.hx)
    psi1 = g1.compact(inputs.gaussian_with_noise(box, seed=1, noise=1e-3))
    V1 = g1.compact(Vd)
    c1 = _oracle_rk4_rate(oracle, g1, V1, psi1, 100.0, 1e-3, 100)
    oracle.set_threads(1)
    single = {"c1_64cubed": _oracle_rk4_rate(oracle, g1, V1, psi1, 100.0, 1e-3, 100),
              "c2_slab": _oracle_rk4_rate(oracle, g, V, psi, wl.g, dt, 10)}
    oracle.set_threads(used)
    return {"value": c2["value"], "unit": "cell-steps/s", "cores": used, "kind": "oracle",
            "sample": f"FP64 oracle RK4, 100 steps on a {g.n}-cell slab (48 z-planes through the equator) of "
                      f"the headline shell, {c2['seconds']} s on {used} threads",
            "c1_64cubed_all_active": c1, "single_thread": single}


# ----------------------------------------------------------------- ranks
def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(local)
    return world, rank, local


def barrier(world):
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()


def max_over_ranks(world, x):
    import torch
    if world == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------- our arm
def time_rk4(gpe, torch, st, params, steps, warmup, n_active, g):
    """Warm up, then time `steps` bench steps; returns (ms per bench step,
    ms per RK4 step of the stage kernels alone)."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        gpe.gpe_step_real(st, params, STEPS_PER_BENCH)
        gpe.gpe_observables(st, g)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for e0, e1, e2 in ev:
        e0.record(stream)
        gpe.gpe_step_real(st, params, STEPS_PER_BENCH)
        e1.record(stream)
        gpe.gpe_observables(st, g)
        e2.record(stream)
    torch.cuda.synchronize()
    total = sum(e0.elapsed_time(e2) for e0, _, e2 in ev)
    rk = sum(e0.elapsed_time(e1) for e0, e1, _ in ev)
    return total, rk / (steps * STEPS_PER_BENCH)


# FP64 operations per cell and RK4 step of the stage kernels (static V; an
# FMA counts 2): Laplacian 20 per stage; update 15, 21, 15, 19 for stages 0-3.
# Counted per ACTIVE cell: the inactive cells of stored segments are skipped
# by the update, and their Laplacian is padding work, not the method's.
FP64_FLOPS_PER_CELL_STEP = 4 * 20 + 15 + 21 + 15 + 19
FP32_VS_FP64_STEPS = 10000        # the FP32-vs-FP64 comparison window (RK4 steps)


def fp64_roofline(gpe, n_active, rk_ms):
    """The complex128 step is bound by the GPU's FP64 arithmetic: its roof is
    the FP64 FMA rate measured on this GPU (gpe_fma_peak, CUDA events)."""
    peak, sec = gpe.gpe_fma_peak(gpe.GPE_F64, 20000)
    achieved = FP64_FLOPS_PER_CELL_STEP * n_active / (rk_ms / 1e3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "flops_per_active_cell_step": FP64_FLOPS_PER_CELL_STEP,
            "peak_kind": "measured: FP64 FMA chains on every SM, %.2f s, CUDA events (gpe_fma_peak)" % sec}


def fp32_vs_fp64(gpe, torch, grid, psi64, params, g, n_stored, checkpoints=(100, 1000, FP32_VS_FP64_STEPS)):
    """complex64 and complex128 runs from the same (complex64-rounded) input,
    compared at each checkpoint: relative L2 error of the FP32 state against
    the FP64 one, and the norm drift |N32 - N64| / N64.  The complex128 run is
    timed (CUDA events, observables excluded)."""
    st64 = gpe.gpe_state_create(grid, gpe.GPE_C64)
    st128 = gpe.gpe_state_create(grid, gpe.GPE_C128)
    gpe.gpe_state_load(st64, psi64, gpe.GPE_LAYOUT_COMPACT)
    gpe.gpe_state_load(st128, np.ascontiguousarray(psi64.astype(np.complex128)), gpe.GPE_LAYOUT_COMPACT)
    stream = torch.cuda.current_stream()
    a = np.empty(n_stored, np.complex64)
    c = np.empty(n_stored, np.complex128)
    done, ms128, out = 0, 0.0, []
    for cp in checkpoints:
        n = cp - done
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        gpe.gpe_step_real(st128, params, n, done * params.dt)
        e1.record(stream)
        gpe.gpe_step_real(st64, params, n, done * params.dt)
        torch.cuda.synchronize()
        ms128 += e0.elapsed_time(e1)
        done = cp
        gpe.gpe_state_store(st64, a, gpe.GPE_LAYOUT_COMPACT)
        gpe.gpe_state_store(st128, c, gpe.GPE_LAYOUT_COMPACT)
        o64, o128 = gpe.gpe_observables(st64, g), gpe.gpe_observables(st128, g)
        out.append({"steps": cp,
                    "rel_l2": float(np.linalg.norm(a.astype(np.complex128) - c) / np.linalg.norm(c)),
                    "norm_drift": abs(o64["norm"] - o128["norm"]) / o128["norm"],
                    "norm_fp32": o64["norm"], "norm_fp64": o128["norm"]})
    gpe.gpe_state_destroy(st64)
    gpe.gpe_state_destroy(st128)
    return out, ms128 / done


def time_itp(gpe, torch, st, ip, steps, warmup):
    """Imaginary-time steps (two stencil passes and the norm each): ms per
    step, after warm-up, CUDA events on the launching stream."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        gpe.gpe_step_imag(st, ip, STEPS_PER_BENCH)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        gpe.gpe_step_imag(st, ip, STEPS_PER_BENCH)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / (steps * STEPS_PER_BENCH)


def run_ours(args):
    import torch
    world, rank, local = dist_setup()
    # a non-default stream: the library replays its step loops as CUDA graphs there
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        _run_ours(args, torch, world, rank, local)


def _run_ours(args, torch, world, rank, local):
    from paper_2603_05447_gb300 import _build, gpe, inputs
    if rank == 0 or world > 1:
        _build.build()
    barrier(world)
    gpe.load()
    wl = shell_workload()
    t_build = time.perf_counter()
    grid = build_grid(gpe, wl, tuple(args.brick), args.sched, args.chunk)
    info = gpe.gpe_grid_get_info(grid)
    t_build = time.perf_counter() - t_build  # the builder synchronises before returning
    n_active, n_stored = info.n_active, info.n_packed
    psi0 = initial_compact(gpe, inputs, wl, grid)
    dt = wl.stable_dt()
    params = gpe.real_params(wl.g, dt)

    quick128 = args.quick and args.dtype == "c128"
    st64 = gpe.gpe_state_create(grid, gpe.GPE_C128 if quick128 else gpe.GPE_C64)
    psi64 = np.ascontiguousarray(psi0 if quick128 else psi0.astype(np.complex64))
    gpe.gpe_state_load(st64, psi64, gpe.GPE_LAYOUT_COMPACT)

    # ---- device-resident timing (complex64, the headline)
    barrier(world)
    launches0 = gpe.gpe_launch_count()
    with ClockSampler(local) as clk:
        total_ms, rk_ms = time_rk4(gpe, torch, st64, params, args.steps, args.warmup, n_active, wl.g)
    launches = gpe.gpe_launch_count() - launches0
    per_warm = (launches // (args.steps + args.warmup))
    gpu_launches = per_warm * args.steps
    barrier(world)
    total_ms = max_over_ranks(world, total_ms)
    cell_steps = n_active * STEPS_PER_BENCH * args.steps * world
    value = cell_steps / (total_ms / 1e3)
    peak, peak_kind = measured_peaks()
    achieved = B_ALG["c64"] * n_active / (rk_ms / 1e3) / 1e9

    # DRAM bytes per RK4 step from the committed ncu capture: valid only for
    # the captured kernels (source hash), workload and launch shape
    traffic = None
    if (os.path.exists(TRAFFIC_FILE) and args.sched == 0 and tuple(args.brick) == (8, 8, 4)
            and args.workload == "shell1024"):
        t = json.load(open(TRAFFIC_FILE))
        if t.get("kernel_source_hash") == kernel_source_hash():
            traffic = t.get("bytes_per_step")

    # ---- the other memory-optimised integrators of App. A on the same grid
    integ = {}
    if not args.quick or args.integrators:
        for name, code, ylim in (("RKHE3", gpe.GPE_RKHE3, 3 ** 0.5), ("RKCK", gpe.GPE_RKCK, 0.43)):
            gpe.gpe_state_load(st64, psi64, gpe.GPE_LAYOUT_COMPACT)
            # the headline dt (dt lambda_max = 0.2) is inside both limits
            p_i = gpe.real_params(wl.g, dt, integrator=code)
            for _ in range(max(1, args.warmup)):
                gpe.gpe_step_real(st64, p_i, STEPS_PER_BENCH // 10)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(torch.cuda.current_stream())
            gpe.gpe_step_real(st64, p_i, STEPS_PER_BENCH)
            e1.record(torch.cuda.current_stream())
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / STEPS_PER_BENCH
            integ[name] = {"value": n_active / (ms / 1e3), "unit": "cell-steps/s", "ms_per_step": ms,
                           "stages": 3 if name == "RKHE3" else 6}

    # ---- the 19-point stencil of App. B on the same shell (its own grid)
    st19 = None
    if not args.quick or args.integrators:
        b_ = wl.box
        g19 = gpe.gpe_grid_create_analytic(gpe.make_box(b_.nx, b_.ny, b_.nz, b_.hx),
                                           gpe.make_potential(gpe.GPE_POT_ELLIPSOID_SHELL, wl.w, *wl.axes),
                                           wl.V_cut, gpe.make_opts(tuple(args.brick), stencil=19))
        s19 = gpe.gpe_state_create(g19, gpe.GPE_C64)
        gpe.gpe_state_load(s19, psi64, gpe.GPE_LAYOUT_COMPACT)
        for _ in range(max(1, args.warmup)):
            gpe.gpe_step_real(s19, params, STEPS_PER_BENCH // 10)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(torch.cuda.current_stream())
        gpe.gpe_step_real(s19, params, STEPS_PER_BENCH)
        e1.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        ms19 = e0.elapsed_time(e1) / STEPS_PER_BENCH
        gpe.gpe_state_load(s19, psi64, gpe.GPE_LAYOUT_COMPACT)
        itp19 = time_itp(gpe, torch, s19, gpe.gpe_imag_params(wl.g, dt, wl.N), 1, 1)
        st19 = {"value": n_active / (ms19 / 1e3), "unit": "cell-steps/s", "ms_per_rk4_step": ms19,
                "ms_per_itp_step": itp19}
        gpe.gpe_state_destroy(s19)
        gpe.gpe_grid_destroy(g19)

    # ---- imaginary-time steps on the same grid (complex64, FP64 norm)
    gpe.gpe_state_load(st64, psi64, gpe.GPE_LAYOUT_COMPACT)
    ip = gpe.gpe_imag_params(wl.g, dt, wl.N)
    itp_ms = time_itp(gpe, torch, st64, ip, args.steps, args.warmup)
    itp = {"value": n_active / (itp_ms / 1e3), "unit": "cell-steps/s", "ms_per_itp_step": itp_ms,
           "achieved_gbs": B_ALG["c64"] * n_active / (itp_ms / 1e3) / 1e9,
           "alg_bytes_per_cell_step": B_ALG["c64"], "launches_per_step": 1 if args.sched == 3 else 2}
    gpe.gpe_state_load(st64, psi64, gpe.GPE_LAYOUT_COMPACT)
    # the same imaginary-time steps on a real-valued float state (|psi|)
    str_ = gpe.gpe_state_create(grid, gpe.GPE_R32)
    gpe.gpe_state_load(str_, np.ascontiguousarray(np.abs(psi0).astype(np.float32)), gpe.GPE_LAYOUT_COMPACT)
    itpr_ms = time_itp(gpe, torch, str_, ip, args.steps, args.warmup)
    gpe.gpe_state_destroy(str_)
    itp["real_f32"] = {"value": n_active / (itpr_ms / 1e3), "unit": "cell-steps/s", "ms_per_itp_step": itpr_ms,
                       "achieved_gbs": 12.0 * n_active / (itpr_ms / 1e3) / 1e9, "alg_bytes_per_cell_step": 12.0}

    # ---- the fused-pair schedule on the same shell (its own grid): RK4 in
    # two launches per step, imaginary time in one
    pair = None
    if not args.quick and args.sched == 0:
        gp = build_grid(gpe, wl, tuple(args.brick), 3, 0)
        sp = gpe.gpe_state_create(gp, gpe.GPE_C64)
        gpe.gpe_state_load(sp, psi64, gpe.GPE_LAYOUT_COMPACT)
        _, rkp_ms = time_rk4(gpe, torch, sp, params, 2, 1, n_active, wl.g)
        gpe.gpe_state_load(sp, psi64, gpe.GPE_LAYOUT_COMPACT)
        itpp_ms = time_itp(gpe, torch, sp, ip, 2, 1)
        pair = {"ms_per_rk4_step": rkp_ms, "rk4_launches_per_step": 2,
                "rk4_achieved_gbs": B_ALG["c64"] * n_active / (rkp_ms / 1e3) / 1e9,
                "ms_per_itp_step": itpp_ms, "itp_launches_per_step": 1,
                "itp_achieved_gbs": B_ALG["c64"] * n_active / (itpp_ms / 1e3) / 1e9}
        gpe.gpe_state_destroy(sp)
        gpe.gpe_grid_destroy(gp)

    if args.quick:
        gpe.gpe_state_destroy(st64)
        gpe.gpe_grid_destroy(grid)
        if rank == 0:
            print(json.dumps({"quick": True, "workload": _workload_name, "dtype": args.dtype, "value": value,
                              "grid_build_s": round(t_build, 4),
                              "ms_per_rk4_step": rk_ms, "achieved_gbs": achieved, "n_active": n_active,
                              "ms_per_itp_step": itp_ms, "ms_per_itp_step_real": itpr_ms,
                              "integrators": integ or None, "stencil19": st19,
                              "gpu_launches": gpu_launches}), flush=True)
        return

    # ---- end to end: host buffers through the C ABI, copies inside the timed region
    pinned_in = torch.empty(n_stored, dtype=torch.complex64, pin_memory=True)
    pinned_out = torch.empty(n_stored, dtype=torch.complex64, pin_memory=True)
    pinned_in.numpy()[:] = psi64
    gpe.gpe_state_load(st64, pinned_in, gpe.GPE_LAYOUT_COMPACT)
    e2e_steps = max(2, min(args.steps, 3))
    barrier(world)
    # the page-locked host tensors are passed as they are (a numpy view made
    # inside the loop would add milliseconds of host time per call)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        gpe.gpe_state_load(st64, pinned_in, gpe.GPE_LAYOUT_COMPACT)
        gpe.gpe_step_real(st64, params, STEPS_PER_BENCH)
        gpe.gpe_state_store(st64, pinned_out, gpe.GPE_LAYOUT_COMPACT)
        gpe.gpe_observables(st64, wl.g)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(world, time.perf_counter() - t0)
    e2e_value = n_active * STEPS_PER_BENCH * e2e_steps * world / e2e_s

    # ---- complex128 path and the FP32-vs-FP64 error after 10^4 RK4 steps
    gpe.gpe_state_destroy(st64)
    cmp, rk128_ms = fp32_vs_fp64(gpe, torch, grid, psi64, params, wl.g, n_stored)
    fp64_value = n_active * world / (max_over_ranks(world, rk128_ms) / 1e3)
    last = cmp[-1]

    gpe.gpe_grid_destroy(grid)

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "cell-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "anisotropic thin ellipsoidal shell, 1024^3 box, semi-axes 490/441/392 cells, "
                               "g=2000, N=1, mask V<5mu0, RK4 real time, complex64 bulk + FP64 reductions",
                   "n_active": n_active, "n_packed": n_stored, "brick": f"{info.bx}x{info.by}x{info.bz}",
                   "grid_build_s": round(t_build, 4),
                   "schedule": {0: "staged", 1: "wavefront", 2: "wavefront (stage pairs)", 3: "fused stage pairs"}[args.sched],
                   "rk4_steps_per_bench_step": STEPS_PER_BENCH, "dt": dt,
                   "l2": "inputs larger than L2 (state %.0f MB + potential %.0f MB)" % (n_stored * 8 / 1e6, n_stored * 4 / 1e6),
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": {0: "RK4 step (k_rk4_staged, four launches per step)",
                                1: "RK4 step (k_rk4_wave, one launch per step)",
                                2: "RK4 step (k_rk4_wave, two launches of two stages per step)",
                                3: "RK4 step (k_rk4_fused, two launches of two fused stages per step)"}[args.sched],
                     "peak_kind": peak_kind,
                     "alg_bytes_per_cell_step": B_ALG["c64"], "ms_per_rk4_step": rk_ms,
                     "traffic_gbs": traffic / (rk_ms / 1e3) / 1e9 if traffic else None,
                     "traffic_frac": traffic / (rk_ms / 1e3) / 1e9 / peak if traffic else None},
        "fp64": {"value": fp64_value, "unit": "cell-steps/s", "ms_per_rk4_step": rk128_ms,
                 "roofline": fp64_roofline(gpe, n_active, rk128_ms),
                 "fp32_over_fp64": (n_active / (rk_ms / 1e3)) / fp64_value,
                 "rel_l2_fp32_vs_fp64": last["rel_l2"], "norm_drift_fp32_vs_fp64": last["norm_drift"],
                 "steps_compared": last["steps"], "checkpoints": cmp,
                 "targets": {"rel_l2": 1e-5, "norm_drift": 1e-6},
                 "same_input": "both runs start from the complex64-rounded initial state"},
        "e2e": {"value": e2e_value, "unit": "cell-steps/s", "h2d_bytes_per_step": n_stored * 8,
                "d2h_bytes_per_step": n_stored * 8 + 7 * 8},
        "itp": itp,
        "pair_schedule": pair,
        "integrators": integ,
        "stencil19": st19,
        "gpu_launches": gpu_launches,
        "clocks": clk.summary(),
    }
    if world == 1:
        line["cpu_baseline"] = cpu_baseline(wl)
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- reference arm
def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = oracle.set_threads(len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
                               else (os.cpu_count() or 1))
    wl = shell_workload()
    g, V, psi = oracle_sample(wl)
    dt = wl.stable_dt()
    y = psi
    for q in range(args.warmup):
        y = oracle.rk4_step(g, V, y, wl.g, q * dt, dt)
    times = []
    for q in range(args.steps):
        t0 = time.perf_counter()
        y = oracle.rk4_step(g, V, y, wl.g, q * dt, dt)
        times.append(time.perf_counter() - t0)
    el = sum(times)
    value = g.n * args.steps / el
    sample = (f"FP64 oracle RK4 on a {g.n}-cell slab (48 z-planes through the equator) of the "
              f"same shell, one RK4 step per bench step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cell-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "anisotropic thin ellipsoidal shell, 1024^3 box, semi-axes 490/441/392 "
                                   "cells, g=2000 (bounded CPU sample)", "n_active_sample": g.n},
            "cpu_baseline": {"value": value, "unit": "cell-steps/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "cell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- other workloads
def _ramp_grid(gpe, rw):
    b = rw.shell.box
    gb = gpe.make_box(b.nx, b.ny, b.nz, b.hx)
    p0 = gpe.make_potential(gpe.GPE_POT_HARMONIC, rw.W, rw.W, rw.W)
    p1 = gpe.make_potential(gpe.GPE_POT_ELLIPSOID_SHELL, rw.shell.w, *rw.shell.axes)
    return gpe.gpe_grid_create_blend(gb, p0, rw.cut0, p1, rw.cut1)


def _core_state(gpe, inputs, rw, grid, dtype):
    """Normalised parabolic core cloud sqrt(max(mu0 - V0, 0)) on the grid."""
    idx, i, j, k = gpe.packed_coords(grid)
    info = gpe.gpe_grid_get_info(grid)
    b = rw.shell.box
    out = np.zeros(info.n_packed, np.complex128)
    x, y, z = b.x0 + i * b.hx, b.y0 + j * b.hy, b.z0 + k * b.hz
    out[idx] = np.sqrt(np.maximum(rw.mu0_core - rw.v0(x, y, z), 0.0))
    out *= math.sqrt(1.0 / (np.sum(np.abs(out) ** 2) * b.dV))
    return np.ascontiguousarray(out.astype(np.complex64 if dtype == gpe.GPE_C64 else np.complex128))


def _final_shell_ground_state(gpe, rw, dst):
    """The imaginary-time ground state of the ramp's final potential (the
    shell alone): solved on its own grid (region V1 < 5 mu_TF, Thomas-Fermi
    start, complex64, |dmu| < 1e-7 mu), then remapped onto dst's grid (the
    ramp's union region).  Returns what the solve reported."""
    b = rw.shell.box
    gb = gpe.make_box(b.nx, b.ny, b.nz, b.hx)
    pot = gpe.make_potential(gpe.GPE_POT_ELLIPSOID_SHELL, rw.shell.w, *rw.shell.axes)
    mu = gpe.gpe_tf_mu_analytic(gb, pot, rw.shell.g, rw.shell.N)
    g1 = gpe.gpe_grid_create_analytic(gb, pot, 5.0 * mu, gpe.make_opts((8, 8, 4)))
    s1 = gpe.gpe_state_create(g1, gpe.GPE_C64)
    try:
        idx, i, j, k = gpe.packed_coords(g1)
        psi = np.zeros(gpe.gpe_grid_get_info(g1).n_packed, np.complex64)
        psi[idx] = np.sqrt(np.maximum(mu - rw.shell.potential(b.x0 + i * b.hx, b.y0 + j * b.hy, b.z0 + k * b.hz),
                                      0.0) / rw.shell.g)
        gpe.gpe_state_load(s1, psi, gpe.GPE_LAYOUT_COMPACT)
        dti = min(0.5 * rw.shell.h ** 2, 0.5 / mu)
        try:
            n, o = gpe.gpe_ground_state(s1, gpe.gpe_imag_params(rw.shell.g, dti, rw.shell.N), 1e-7 * mu, 100, 20000)
            conv = True
        except gpe.GpeError:
            n, o, conv = 20000, gpe.gpe_observables(s1, rw.shell.g), False
        gpe.gpe_state_remap(dst, s1)
        kept = gpe.gpe_observables(dst, rw.shell.g, 1.0)["norm"]
        return {"steps": n, "converged": conv, "mu": o["mu"], "n_active": gpe.gpe_grid_get_info(g1).n_active,
                "norm_on_ramp_grid": kept}
    finally:
        gpe.gpe_state_destroy(s1)
        gpe.gpe_grid_destroy(g1)


def stages_run(gpe, inputs, torch, n_stages=66, steps_per_stage=20):
    """Multi-stage ramp (Sec. V) on a 512^3 shell: 67 dense FP32 potentials
    on the device, evenly spaced blends of the shell and a softer, slightly
    rounder shell (inputs.stage_fractions); every stage selects its region
    again at 5 max(mu_i, mu_{i+1}) and remaps the state.  Timed twice: with
    `steps_per_stage` RK4 steps a stage, and with one, whose difference gives
    the step rate; the report gives each stage's regrid time."""
    wl = inputs.SHELL_512
    b = wl.box
    gb = gpe.make_box(b.nx, b.ny, b.nz, b.hx)
    a, bb, c = wl.axes
    end = inputs.EllipsoidShell(0.6 * wl.w, a, bb + 0.01, c + 0.02)
    dev = torch.device("cuda", torch.cuda.current_device())
    # endpoint potentials, evaluated on the host in z-slabs, FP64 on the device
    V0 = torch.empty((b.nz, b.ny, b.nx), dtype=torch.float64, device=dev)
    V1 = torch.empty_like(V0)
    x, y, z = b.axes()
    for k0 in range(0, b.nz, 32):
        Z, Y, X = np.meshgrid(z[k0:k0 + 32], y, x, indexing="ij")
        V0[k0:k0 + 32].copy_(torch.from_numpy(wl.potential(X, Y, Z)))
        V1[k0:k0 + 32].copy_(torch.from_numpy(end(X, Y, Z)))
    pots = [((1.0 - s) * V0 + s * V1).to(torch.float32) for s in inputs.stage_fractions(n_stages)]
    del V0, V1
    mu0 = gpe.gpe_tf_mu_dense(gb, pots[0], wl.g, wl.N)
    g0 = gpe.gpe_grid_create_dense(gb, pots[0], 5.0 * mu0, gpe.make_opts((8, 8, 4)))
    info0 = gpe.gpe_grid_get_info(g0)
    dt = 0.2 / (6.0 / wl.h ** 2 + 2.0 * info0.v_max)     # the softer shells only lower |V|
    s0 = gpe.gpe_state_create(g0, gpe.GPE_C64)
    idx, i, j, k = gpe.packed_coords(g0)
    psi = np.zeros(info0.n_packed, np.complex128)
    psi[idx] = np.sqrt(np.maximum(mu0 - wl.potential(b.x0 + i * b.hx, b.y0 + j * b.hy, b.z0 + k * b.hz), 0.0)
                       / wl.g)
    psi *= math.sqrt(wl.N / (np.sum(np.abs(psi) ** 2) * b.dV))
    gpe.gpe_state_load(s0, np.ascontiguousarray(psi.astype(np.complex64)), gpe.GPE_LAYOUT_COMPACT)
    params = gpe.stage_params(wl.g, wl.N, dt, 5.0)
    runs = {}
    for n in (1, steps_per_stage, steps_per_stage):      # the first run warms up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        grid, st, rep = gpe.gpe_ramp_stages(s0, pots, [n * dt] * n_stages, params)
        el = time.perf_counter() - t0
        gpe.gpe_state_destroy(st)
        gpe.gpe_grid_destroy(grid)
        runs[n] = (el, rep)
    gpe.gpe_state_destroy(s0)
    gpe.gpe_grid_destroy(g0)
    (t1, rep1), (tn, rep) = runs[1], runs[steps_per_stage]
    cell_steps = sum(r["n_active"] * r["steps"] for r in rep)
    step_s = (tn - t1) / (steps_per_stage - 1) / n_stages        # one step of an average stage
    regrid_s = sum(r["regrid_s"] for r in rep)
    return dict(metric="multi-stage ramp: active-cell RK4 steps/s including every regrid (complex64)",
                unit="cell-steps/s", value=cell_steps / tn, seconds=tn, stages=n_stages,
                steps_per_stage=steps_per_stage, dt=dt,
                step_cell_steps_per_s=sum(r["n_active"] for r in rep) / n_stages / step_s,
                regrid_ms_per_stage=regrid_s / n_stages * 1e3,
                other_ms_per_stage=(tn - regrid_s - n_stages * steps_per_stage * step_s) / n_stages * 1e3,
                n_active_first=rep[0]["n_active"], n_active_last=rep[-1]["n_active"],
                norm_kept_min=min(r["norm_kept"] for r in rep), norm_end=rep[-1]["norm_end"],
                config="512^3 box, shell semi-axes 240/216/192 cells, g=2000; 67 dense FP32 potentials blending "
                       "it into a shell of 0.6x the stiffness and semi-axes +0.01/+0.02; region "
                       "5 max(mu_i, mu_i+1) per stage")


def roi_sweep(gpe, inputs, torch):
    """Boundary error of the region of interest (the study of Sec. IV,
    Fig. 2c, on a synthetic shell): ground states on regions V < r mu_TF in
    cell and brick mode against the ground state on the full box, error
    (1/N) sum ||psi_0|^2 - |psi|^2| dV.  Same finite-difference operator and
    time step everywhere, so the difference is the boundary's alone."""
    wl = inputs.SHELL_64
    b = wl.box
    gb = gpe.make_box(b.nx, b.ny, b.nz, b.hx)
    V = inputs.dense_potential(b, wl.potential)
    mu_tf = gpe.gpe_tf_mu_dense(gb, V, wl.g, wl.N)
    dt = 2.0 / (3 * 2.0 / b.hx ** 2)          # half the Euler substep limit
    p = gpe.gpe_imag_params(wl.g, dt, wl.N)
    psi0 = np.sqrt(np.maximum(mu_tf - V, 0.0) / wl.g)

    def ground(V_cut, mode):
        grid = gpe.gpe_grid_create_dense(gb, V, V_cut, gpe.make_opts((8, 8, 8), mode))
        st = gpe.gpe_state_create(grid, gpe.GPE_R64)
        try:
            gpe.gpe_state_load(st, np.ascontiguousarray(psi0), gpe.GPE_LAYOUT_DENSE)
            # mu is stationary to second order: relax for a fixed imaginary time
            # (tau ~ 2) before the |dmu| test, so slow surface modes decay too
            gpe.gpe_step_imag(st, p, 4000)
            steps, o = gpe.gpe_ground_state(st, p, 1e-11, 100, 400000)
            steps += 4000
            out = np.zeros(b.shape)
            gpe.gpe_state_store(st, out, gpe.GPE_LAYOUT_DENSE)
            return out, gpe.gpe_grid_get_info(grid).n_active, steps, o["mu"]
        finally:
            gpe.gpe_state_destroy(st)
            gpe.gpe_grid_destroy(grid)

    t0 = time.perf_counter()
    ref, n_ref, steps_ref, mu_ref = ground(np.inf, gpe.GPE_MASK_CELL)
    ratios = [1.25, 1.5, 2.0, 3.0, 4.0, 5.0, 6.0]
    res = {"cell": [], "brick": []}
    for mode, key in ((gpe.GPE_MASK_CELL, "cell"), (gpe.GPE_MASK_BRICK, "brick")):
        for r in ratios:
            psi, n, steps, mu = ground(r * mu_tf, mode)
            err = float(np.sum(np.abs(ref ** 2 - psi ** 2)) * b.dV / wl.N)
            res[key].append({"ratio": r, "error": err, "n_active": int(n), "steps": int(steps),
                             "dmu": float(mu - mu_ref)})
    return {"metric": "ROI boundary error (1/N) sum ||psi_0|^2 - |psi|^2| dV vs cutoff ratio V_cut / mu_TF",
            "unit": "relative", "mu_tf": mu_tf, "mu_full_box": mu_ref, "n_full_box": int(n_ref),
            "steps_full_box": int(steps_ref), "results": res, "seconds": time.perf_counter() - t0,
            "config": "64^3 shell (semi-axis 26 cells, g=2000, N=1), real FP64 ground states, |dmu| < 1e-11, "
                      "8^3 bricks; brick mode keeps every cell of a brick holding a selected cell"}


def ramp_traced(gpe, inputs, torch, nsteps=5000, every=500, n_overlap=5, nsteps_overlap=4000):
    """The hollowing ramp of the 2048^3 box tracked over a run of `nsteps` RK4
    steps (the configuration names 5e4; 5000 by default): norm and energy
    every `every` steps through gpe_step_real_traced.  The overlap with the
    instantaneous ground state needs a ground-state solve of V(s(t)) per
    trace point, so it is tracked on the 512^3 version of the same ramp:
    at n_overlap points of an `nsteps_overlap`-step run, the ground state of
    (1 - s) V0 + s V1 (complex64, Thomas-Fermi start, region V < 5 mu_TF) is
    solved and |<psi_gs | psi(t)>|^2 taken after remapping psi(t) onto its
    grid (cells of psi(t) outside that region are dropped)."""
    out = {}
    knots = inputs.monotone_knots(16, seed=3)
    # 2048^3: traced norm and energy
    rw = inputs.RAMP_2048
    grid = _ramp_grid(gpe, rw)
    info = gpe.gpe_grid_get_info(grid)
    st = gpe.gpe_state_create(grid, gpe.GPE_C64)
    gpe.gpe_state_load(st, _core_state(gpe, inputs, rw, grid, gpe.GPE_C64), gpe.GPE_LAYOUT_COMPACT)
    dt = 0.2 / (6.0 / rw.shell.h ** 2 + info.v_max)
    p = gpe.real_params(rw.shell.g, dt, gpe.GPE_V_BLEND, knots, nsteps * dt)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    trace = gpe.gpe_step_real_traced(st, p, nsteps, every)
    el = time.perf_counter() - t0
    out["box2048"] = {"n_active": info.n_active, "steps": nsteps, "every": every, "dt": dt, "seconds": el,
                      "cell_steps_per_s": info.n_active * nsteps / el,
                      "trace": [{"step": (k + 1) * every, "norm": o["norm"], "energy": o["energy"], "mu": o["mu"]}
                                for k, o in enumerate(trace)]}
    gpe.gpe_state_destroy(st)
    gpe.gpe_grid_destroy(grid)
    # 512^3: overlap with the instantaneous ground state
    rw = inputs.RAMP_512
    b = rw.shell.box
    gb = gpe.make_box(b.nx, b.ny, b.nz, b.hx)
    grid = _ramp_grid(gpe, rw)
    info = gpe.gpe_grid_get_info(grid)
    st = gpe.gpe_state_create(grid, gpe.GPE_C64)
    gpe.gpe_state_load(st, _core_state(gpe, inputs, rw, grid, gpe.GPE_C64), gpe.GPE_LAYOUT_COMPACT)
    dt = 0.2 / (6.0 / rw.shell.h ** 2 + info.v_max)
    T = nsteps_overlap * dt
    p = gpe.real_params(rw.shell.g, dt, gpe.GPE_V_BLEND, knots, T)
    dev = torch.device("cuda", torch.cuda.current_device())
    V0 = torch.empty((b.nz, b.ny, b.nx), dtype=torch.float64, device=dev)
    V1 = torch.empty_like(V0)
    x, y, z = b.axes()
    for k0 in range(0, b.nz, 32):
        Z, Y, X = np.meshgrid(z[k0:k0 + 32], y, x, indexing="ij")
        V0[k0:k0 + 32].copy_(torch.from_numpy(rw.v0(X, Y, Z)))
        V1[k0:k0 + 32].copy_(torch.from_numpy(rw.shell.potential(X, Y, Z)))
    tknots = np.linspace(0.0, T, len(knots))
    points, done = [], 0
    marks = [int(round(q * nsteps_overlap / (n_overlap - 1))) for q in range(n_overlap)]
    for m in marks:
        if m > done:
            gpe.gpe_step_real(st, p, m - done, done * dt)
            done = m
        s_t = float(np.interp(done * dt, tknots, knots))
        Vs = ((1.0 - s_t) * V0 + s_t * V1).contiguous()
        mu = gpe.gpe_tf_mu_dense(gb, Vs, rw.shell.g, rw.shell.N)
        g2 = gpe.gpe_grid_create_dense(gb, Vs, 5.0 * mu, gpe.make_opts((8, 8, 4)))
        gs = gpe.gpe_state_create(g2, gpe.GPE_C64)
        gpe.gpe_state_load(gs, torch.sqrt(torch.clamp(mu - Vs, min=0.0) / rw.shell.g).to(torch.complex64).contiguous(),
                           gpe.GPE_LAYOUT_DENSE)
        dti = min(0.5 * rw.shell.h ** 2, 0.5 / mu)
        try:
            n_gs, ogs = gpe.gpe_ground_state(gs, gpe.gpe_imag_params(rw.shell.g, dti, rw.shell.N), 1e-7 * mu, 100,
                                             20000)
            conv = True
        except gpe.GpeError:
            n_gs, ogs, conv = 20000, gpe.gpe_observables(gs, rw.shell.g), False
        tmp = gpe.gpe_state_create(g2, gpe.GPE_C64)
        gpe.gpe_state_remap(tmp, st)
        c = gpe.gpe_overlap(gs, tmp)
        o_t = gpe.gpe_observables(st, rw.shell.g, s_t)
        points.append({"step": done, "s": s_t, "fidelity": abs(c) ** 2, "norm": o_t["norm"],
                       "energy": o_t["energy"], "mu_ground": ogs["mu"], "ground_steps": n_gs,
                       "ground_converged": conv, "n_active_ground": gpe.gpe_grid_get_info(g2).n_active})
        for h_ in (tmp, gs):
            gpe.gpe_state_destroy(h_)
        gpe.gpe_grid_destroy(g2)
        del Vs
    out["box512_overlap"] = {"n_active": info.n_active, "steps": nsteps_overlap, "dt": dt, "points": points}
    gpe.gpe_state_destroy(st)
    gpe.gpe_grid_destroy(grid)
    return {"metric": "hollowing ramp tracked: norm, energy (2048^3) and overlap with the instantaneous ground "
                      "state (512^3)", "unit": "various", **out,
            "config": "ramp workload (harmonic core -> thin shell, g=5000, 16 seeded monotone knots over the run), "
                      "complex64 RK4; the configuration's 5e4 steps cut to the step counts stated"}


def alg_roofline(cell_steps_per_s, alg_bytes, what):
    """Algorithmic bytes per active cell-step x rate, over the measured copy
    bandwidth (whole-run rate: includes launch gaps and reductions)."""
    peak, kind = measured_peaks()
    achieved = cell_steps_per_s * alg_bytes / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "alg_bytes_per_cell_step": alg_bytes, "alg_bytes": what, "peak_kind": kind}


def run_extra(args):
    """Ramp (2048^3, ~1e8 active), adjoint (512^3) and batch workloads: one
    JSON line each, beside the headline line of the default run."""
    import torch
    from paper_2603_05447_gb300 import _build, gpe, inputs
    from paper_2603_05447_gb300 import dist as gdist
    rank, world, local = gdist.env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    gpe.load()
    side = torch.cuda.Stream()
    line = {"workload": args.workload, "n_gpus": world, "data": "synthetic"}
    with torch.cuda.stream(side):
        if args.workload == "roi_sweep":
            line.update(roi_sweep(gpe, inputs, torch))
        elif args.workload == "stages512":
            line.update(stages_run(gpe, inputs, torch))
        elif args.workload == "ramp_traced":
            line.update(ramp_traced(gpe, inputs, torch, nsteps=args.ramp_steps, every=max(1, args.ramp_steps // 10)))
        elif args.workload in ("ramp2048", "adjoint512"):
            rw = inputs.RAMP_2048 if args.workload == "ramp2048" else inputs.RAMP_512
            grid = _ramp_grid(gpe, rw)
            info = gpe.gpe_grid_get_info(grid)
            st = gpe.gpe_state_create(grid, gpe.GPE_C64)
            gpe.gpe_state_load(st, _core_state(gpe, inputs, rw, grid, gpe.GPE_C64), gpe.GPE_LAYOUT_COMPACT)
            # the union region holds the shell potential at the trap centre and the trap
            # potential on the shell: the explicit step must resolve the largest |V|
            h = rw.shell.h
            dt = 0.2 / (6.0 / h ** 2 + info.v_max)
            nsteps = args.steps * STEPS_PER_BENCH
            knots = inputs.monotone_knots(16, seed=3)
            p = gpe.real_params(rw.shell.g, dt, gpe.GPE_V_BLEND, knots, nsteps * dt)
            if args.workload == "ramp2048":
                gpe.gpe_step_real(st, p, args.warmup * 10)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                gpe.gpe_step_real(st, p, nsteps)
                e1.record()
                torch.cuda.synchronize()
                ms = gdist.max_over_ranks(e0.elapsed_time(e1))
                o = gpe.gpe_observables(st, rw.shell.g, float(knots[-1]))
                # regrid as between ramp stages (Sec. V): a region selected with
                # 0.8x the cutoffs, the state remapped onto it
                b = rw.shell.box
                g2 = gpe.gpe_grid_create_blend(
                    gpe.make_box(b.nx, b.ny, b.nz, b.hx),
                    gpe.make_potential(gpe.GPE_POT_HARMONIC, rw.W, rw.W, rw.W), 0.8 * rw.cut0,
                    gpe.make_potential(gpe.GPE_POT_ELLIPSOID_SHELL, rw.shell.w, *rw.shell.axes), 0.8 * rw.cut1)
                st2 = gpe.gpe_state_create(g2, gpe.GPE_C64)
                gpe.gpe_state_remap(st2, st)
                torch.cuda.synchronize()
                r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                r0.record()
                gpe.gpe_state_remap(st2, st)
                r1.record()
                torch.cuda.synchronize()
                info2 = gpe.gpe_grid_get_info(g2)
                remap = {"ms": r0.elapsed_time(r1), "n_packed_dst": info2.n_packed,
                         "cells_per_s": info2.n_packed / (r0.elapsed_time(r1) / 1e3)}
                gpe.gpe_state_destroy(st2)
                gpe.gpe_grid_destroy(g2)
                line.update(metric="ramp cell-steps/s (RK4, complex64, V(t) blend)", unit="cell-steps/s", remap=remap,
                            value=info.n_active * nsteps * world / (ms / 1e3), n_active=info.n_active,
                            n_packed=info.n_packed, steps=nsteps, ms_per_step=ms / nsteps, norm_after=o["norm"],
                            dt=dt, v_max=info.v_max,
                            roofline=alg_roofline(info.n_active * nsteps / (ms / 1e3), 24.0,
                                                  "read psi, V0, V1; write psi"),
                            config="2048^3 box, shell semi-axis 800 cells + harmonic core radius 0.24, g=5000, "
                                   "16 seeded monotone knots over the run")
            else:
                # the target: the imaginary-time ground state of the final shell
                tg = gpe.gpe_state_create(grid, gpe.GPE_C64)
                target = _final_shell_ground_state(gpe, rw, tg)
                # a second target the run's state still overlaps: the initial
                # core (the shell's ground state vanishes where the core is)
                tg0 = gpe.gpe_state_create(grid, gpe.GPE_C64)
                gpe.gpe_state_copy(tg0, st)
                nsteps = 4000
                K = 64
                p = gpe.real_params(rw.shell.g, dt, gpe.GPE_V_BLEND, knots, nsteps * dt)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                tape = gpe.gpe_ramp_forward(st, p, nsteps, 0.0, K)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                loss, grad = gpe.gpe_ramp_backward(tape, tg, 16)
                t2 = time.perf_counter()
                loss0, grad0 = gpe.gpe_ramp_backward(tape, tg0, 16)  # the same tape, untimed
                gpe.gpe_tape_destroy(tape)
                gpe.gpe_state_destroy(tg)
                gpe.gpe_state_destroy(tg0)
                line.update(metric="adjoint ramp gradient (4000 RK4 steps, K=64, complex64 + FP64 gradient)",
                            unit="s", value=t2 - t0, forward_s=t1 - t0, backward_s=t2 - t1,
                            n_active=info.n_active, loss=loss, grad_norm=float(np.linalg.norm(grad)),
                            forward_cell_steps_per_s=info.n_active * nsteps / (t1 - t0), target=target,
                            initial_state_target={"loss": loss0, "grad_norm": float(np.linalg.norm(grad0)),
                                                  "grad": [float(x) for x in grad0]},
                            config="512^3 box, shell semi-axis 200 cells + harmonic core, ~5e6 active, target = "
                                   "imaginary-time ground state of the final shell")
            gpe.gpe_state_destroy(st)
            gpe.gpe_grid_destroy(grid)
        else:
            shells = inputs.batch_shells(args.shells)
            dtype_id = BATCH_STATES[args.batch_state][0]

            def shell_args(wl):
                b = wl.box
                return (gpe.make_box(b.nx, b.ny, b.nz, b.hx),
                        gpe.make_potential(gpe.GPE_POT_ELLIPSOID_SHELL, wl.w, *wl.axes), wl.V_cut)

            # brick shape from the batch autotuner (every shell, the batch
            # kernels, 20 imaginary-time steps per candidate)
            sa = [shell_args(wl) for wl in shells]
            best, tuned = gpe.gpe_batch_autotune([x[0] for x in sa], [x[1] for x in sa], [x[2] for x in sa],
                                                 dtype_id, 20)
            brick = (best["bx"], best["by"], best["bz"])
            grids, states, cells = [], [], []
            for wl in shells:
                g = gpe.gpe_grid_create_analytic(*shell_args(wl), gpe.make_opts(brick))
                grids.append(g)
                cells.append(gpe.gpe_grid_get_info(g).n_active)
            mine = gdist.shard(cells, world, rank)
            for i in mine:
                wl, g = shells[i], grids[i]
                idx, ii, jj, kk = gpe.packed_coords(g)
                b = wl.box
                x, y, z = b.x0 + ii * b.hx, b.y0 + jj * b.hy, b.z0 + kk * b.hz
                psi = np.zeros(gpe.gpe_grid_get_info(g).n_packed, BATCH_STATES[args.batch_state][1])
                psi[idx] = np.sqrt(np.maximum(wl.mu0 - wl.potential(x, y, z), 0.0) / wl.g)
                st = gpe.gpe_state_create(g, BATCH_STATES[args.batch_state][0])
                gpe.gpe_state_load(st, psi, gpe.GPE_LAYOUT_COMPACT)
                states.append(st)
            batch = gpe.gpe_batch_create(states)
            params = [gpe.gpe_imag_params(shells[i].g, shells[i].stable_dt() * 20, 1.0) for i in mine]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, conv, steps, obs = gpe.gpe_batch_ground_state(batch, params, args.tol, 100,
                                                              args.steps * STEPS_PER_BENCH, check=False)
            el = gdist.max_over_ranks(time.perf_counter() - t0)
            done = gdist.sum_over_ranks(sum(cells[i] * s for i, s in zip(mine, steps)))
            # the single-precision floor: per shell, |dmu| between FLOOR_CHECKS further
            # checks of 100 steps each (outside the timed region)
            floors = []
            for k, i in enumerate(mine):
                mus = []
                for _ in range(FLOOR_CHECKS + 1):
                    gpe.gpe_step_imag(states[k], params[k], 100)
                    mus.append(gpe.gpe_observables(states[k], shells[i].g)["mu"])
                d = np.abs(np.diff(mus))
                floors.append({"shell": i, "n_active": cells[i], "converged": bool(conv[k]), "steps": int(steps[k]),
                               "mu": mus[-1], "dmu_median": float(np.median(d)), "dmu_max": float(np.max(d)),
                               "dmu_median_rel": float(np.median(d) / abs(mus[-1]))})
            med = np.array([f["dmu_median"] for f in floors])
            line.update(metric=f"batched ground states: active-cell ITP steps/s ({BATCH_STATES[args.batch_state][2]}, "
                               "FP64 norms)", dtype=args.batch_state,
                        unit="cell-steps/s", value=done / el, shells=len(shells), n_active_total=int(sum(cells)),
                        roofline=alg_roofline(done / el, 20.0 if args.batch_state == "c64" else 12.0,
                                              "psi in and out, E in"),
                        converged=int(gdist.sum_over_ranks(sum(conv))), tol_dmu=args.tol,
                        floor={"checks": FLOOR_CHECKS, "every": 100,
                               "below_tol": int(np.sum(med < args.tol)),
                               "dmu_median_quantiles": [float(np.quantile(med, q)) for q in (0, 0.5, 0.9, 1)],
                               "per_shell": floors},
                        max_steps=args.steps * STEPS_PER_BENCH, seconds=el, scaling="strong",
                        brick=list(brick), autotune=[{"brick": [r["bx"], r["by"], r["bz"]],
                                                      "ms_per_step": r["ms_per_step"],
                                                      "cell_steps_per_s": r["cell_steps_per_s"]} for r in tuned],
                        config="seeded uneven ellipsoidal shells (radius U[0.5,1] x 360 cells, aspects U[0.7,1], "
                               "thickness U[4,10] cells, g U[100,3000]), one persistent launch, graph-replayed, "
                               "brick shape from the autotuner")
            gpe.gpe_batch_destroy(batch)
            for st in states:
                gpe.gpe_state_destroy(st)
            for g in grids:
                gpe.gpe_grid_destroy(g)
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + list(EXTRA), default="shell1024",
                    help="shell512 is the smaller case used for ncu captures; ramp2048, adjoint512 and batch "
                         "time the other workloads (one JSON line each)")
    ap.add_argument("--shells", type=int, default=64, help="batch workload: number of shells")
    ap.add_argument("--tol", type=float, default=1e-8, help="batch workload: |dmu| tolerance")
    ap.add_argument("--ramp-steps", type=int, default=5000,
                    help="ramp_traced workload: RK4 steps of the tracked 2048^3 ramp (the configuration names 5e4)")
    ap.add_argument("--batch-state", choices=sorted(BATCH_STATES), default="c64",
                    help="batch workload: state type (r32: real float, half the bytes of c64)")
    ap.add_argument("--integrators", action="store_true", help="a --quick run also times RKHE3 and RKCK")
    ap.add_argument("--quick", action="store_true",
                    help="device-resident complex64 timing only (for profiling runs)")
    ap.add_argument("--sched", type=int, default=0,
                    help="0 staged, 1 wavefront, 2 two-stage wavefront, 3 fused stage pairs")
    ap.add_argument("--chunk", type=int, default=0, help="bricks per wavefront task (0: default)")
    ap.add_argument("--brick", type=int, nargs=3, default=[8, 8, 4])
    ap.add_argument("--dtype", choices=["c64", "c128"], default="c64", help="state type of a --quick run")
    args = ap.parse_args()
    global _workload_name
    _workload_name = args.workload
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in EXTRA:
        run_extra(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
