"""Benchmark: Mcell-updates/s per IMEX step of the AP IMEX-RK D2V6 solver.

Workload (default): Taylor-Green vortex on a periodic 2048 x 2048 grid,
eps = 1e-4, Ma = 1e-3, tau = 0.05, CFL 0.5, second-order GSA IMEX tableau
(c = 2.25) with WENO5 + fourth-order central differences.  One "step" is one
full IMEX step (both stages: explicit operators, closed-form relaxation,
Helmholtz solve, u/q update) of the whole grid.  The FP64 form is the
headline value; the FP32 deviation form is reported beside it with its
velocity/pressure error against the FP64 result.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 is launched with torchrun: every rank runs an independent replica on
its own GPU (the solve does not shard; replicas only), the time is the max
over ranks and the value counts the cells of all ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mcell-updates/s per IMEX step (FP64 vs FP32-dev) at stated error; served p99"
UNIT = "Mcell-updates/s"


# ----------------------------------------------------------------- algorithmic counts
# Flops per cell of each kernel kind for one IMEX step of the second-order
# tableau (both stages), counting every +, -, *, / as one flop, derived from
# the formulas (halo recomputation and redundant loads are not counted).
def weno_flux_pair_flops(scheme: str) -> int:
    """Flops per cell for one flux/partner pair along one axis: two
    reconstructions per interface + split + sum, and the difference."""
    if scheme == "WENO5_C4":
        return 2 * 69 + 1 + 4 + 2
    if scheme == "WENO3_C4":
        return 2 * 20 + 1 + 4 + 2
    return 4 + 2


def step_flops_per_cell(scheme: str, n: int) -> dict:
    FP = weno_flux_pair_flops(scheme)
    c1 = 6 if scheme != "LF1_C2" else 2           # first central difference
    c2 = 8 if scheme != "LF1_C2" else 4           # second central difference
    lg = math.log2(n)
    # stage 1: E, D0.u^n and the closed-form v^(2); stage 2: all derived operators and v^(3)
    explicit = (2 * c1 + 1) * 2 + 2 * FP + 13 + (2 * c1 + 1) + 14
    explicit += (2 * c1 + 1) * 2 + 2 * FP + 13 + (2 * c1 + 1) + (2 * c2 + 1) + 2 * c1 + 4 * FP + 2 + 22
    dbf = 2 * c2 + 2 * c1 + 3
    rhs = (dbf + 5 + 1) + (dbf + 11)
    # radix-2 butterflies (10 flops) of the two real-row, column and inverse-row passes, two solves
    rows = 2 * (2.5 * lg + 2)
    cols = 2 * (5 * lg + 2.5)
    update = (6 + 4 * FP + 2 + 2 * c1 + (2 * c1 + 1) + 6 + 4 + 8) + (10 + 4 * FP + 2 + 2 * c1 + (2 * c1 + 1) + 12 + 4 + 13)
    return {"explicit": explicit, "rhs": rhs, "fft_rows_fwd": rows, "fft_cols": cols,
            "fft_rows_inv": rows, "update": update}


def step_bytes_per_cell(f32: bool) -> dict:
    """Algorithmic DRAM bytes per cell of each kernel kind for one step:
    every plane a kernel must read or write, once."""
    e = 4 if f32 else 8
    planes = {
        # stage 1: read u, v, q (5), write E, D0.u, v^(2) (5);
        # stage 2: read X^(2) (6), E^(1), v^n (4), write E, D0.u, D_Delta theta, D_LF.B(v) + D0 theta, v^(3) (8)
        "explicit": (5 + 5) + (10 + 8),
        # stage 2: read v^(2), theta^n, D0.u^n (4), write DB, R (2);
        # stage 3: read v^(3), theta^n, D0.u^n, D0.u^(2), DB^(2), D_Delta theta^(2) (7), write R
        # (the last stage's DB is read by no later stage)
        "rhs": (4 + 2) + (7 + 1),
        # each pass reads and writes one plane-equivalent (real plane or half spectrum), two solves
        "fft_rows_fwd": 4, "fft_cols": 4, "fft_rows_inv": 4,
        # stage 2: read theta, v, u^(1), u^n, q^n (8), write u, q, D0.v (4);
        # stage 3: read theta, v, u^(1), u^(2), u^n, q^n, D_LF.B(v)^(2) + D0 theta^(2), D0.v^(2), q^(2) (14),
        # and close the step: write X^{n+1} (6; FP32 forms: the populations and the next step's
        # FP64-summed moments, 12)
        "update": (8 + 4) + (14 + (12 if f32 else 6))}
    return {k: v * e for k, v in planes.items()}


# ----------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- workload
def workload(n: int, eps: float, mach: float, tau: float):
    from paper_2512_19847_gb300 import workloads as W
    u1, u2, p = W.taylor_green(n)
    dt = W.stable_dt(u1, u2, 2 * math.pi / n, tau)
    return (u1, u2, p), dt


def make_solver(n, eps, mach, tau, dt, f32: bool, scheme="WENO5_C4"):
    from paper_2512_19847_gb300 import api, tableaux
    p = api.default_params(n, n, eps=eps, dt=dt, tau=tau, mach=mach, space_scheme=scheme,
                           tableau=tableaux.gsa2(), precision=api.FP32_DEV if f32 else api.FP64)
    return api.Solver(p)


def time_form(torch, fields, n, eps, mach, tau, dt, f32, steps, warmup, barrier, graph_steps=1, tile=None):
    s = make_solver(n, eps, mach, tau, dt, f32)
    s.set_equilibrium(*[torch.from_numpy(a).cuda() for a in fields])
    if tile is not None:                                 # a fixed tile shape (profiling runs)
        s.set_tile(tile)
        s.tuned = {"tile": tile, "ms_per_step": {}, "cached": False, "fixed": True}
    else:                                                # the autotuner (state saved and restored bit for bit)
        from paper_2512_19847_gb300 import autotune
        s.tuned = autotune.tune(s, steps=2, path=None)
    s.set_graph_steps(graph_steps)
    s.step(warmup)
    s.sync_status()
    torch.cuda.synchronize()
    barrier()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    s.step(steps)
    e1.record(st)
    e1.synchronize()
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    s.sync_status()
    return s, ms


def profile_form(s, steps):
    s.profile(True)
    s.step(steps)
    prof = s.profile_read()
    s.profile(False)
    return prof


TRAFFIC_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", "dram_traffic_tg2048.json")


def csrc_digest() -> str:
    """SHA-256 over the CUDA sources (names and contents): DRAM counters taken
    with ncu are only reported while the kernels are unchanged."""
    import hashlib
    d = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2512_19847_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".h", ".inc")):
            h.update(name.encode())
            with open(os.path.join(d, name), "rb") as f:
                h.update(f.read())
    return h.hexdigest()


def measured_traffic(kind: str, f32: bool, n: int):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch of `kind` from the
    committed ncu capture, or None when it was taken on other kernels or sizes."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("n") != n or rec.get("csrc_sha256") != csrc_digest():
        return None
    v = rec.get("fp32" if f32 else "fp64", {}).get(kind)
    return None if v is None else float(v)


def roofline(prof: dict, steps: int, cells: int, f32: bool, scheme: str, n: int, peaks: dict, fp64_peak: dict | None = None):
    flops = step_flops_per_cell(scheme, n)
    byts = step_bytes_per_cell(f32)
    kind, (tot_ms, launches) = max(prof.items(), key=lambda kv: kv[1][0])
    per_launch_ms = tot_ms / launches
    launches_per_step = launches / steps
    if f32:
        alg = byts[kind] * cells / launches_per_step            # bytes per launch
        achieved = alg / (per_launch_ms * 1e-3) / 1e9
        peak = peaks.get("hbm_gbs") or 6800.0
        return kind, {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                      "frac": round(achieved / peak, 4), "traffic": measured_traffic(kind, True, n), "kernel": kind,
                      "algorithmic_bytes_per_launch": alg, "ms_per_launch": round(per_launch_ms, 4),
                      "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if "hbm_gbs" in peaks else "fallback"}
    alg = flops[kind] * cells / launches_per_step                # flops per launch
    achieved = alg / (per_launch_ms * 1e-3) / 1e12
    peak = fp64_peak["tflops_at_run_clock"]
    return kind, {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
                  "frac": round(achieved / peak, 4), "traffic": measured_traffic(kind, False, n), "kernel": kind,
                  "algorithmic_flops_per_launch": alg, "ms_per_launch": round(per_launch_ms, 4),
                  "peak_source": fp64_peak["source"]}


def fma_peak_leg(local: int, precision: int, iters: int, reps: int = 60) -> dict:
    """The measured FMA peak (ap_dvm_fma_peak: a kernel of independent FMA chains,
    CUDA events on the launching stream) with the SM clock sampled while it runs."""
    from paper_2512_19847_gb300 import api
    api.fma_peak(precision, iters, 2)                   # warm-up (module load, clocks up)
    with ClockSampler(local) as clk:
        tf, ms = api.fma_peak(precision, iters, reps)
    c = clk.summary()
    return {"tflops": round(tf, 4), "ms_per_launch": round(ms, 3), "launches": reps, "clocks": c,
            "dtype": "f64" if precision == api.FP64 else "f32"}


def scaled_peak(leg: dict, run_clocks: dict) -> dict:
    """The leg's peak scaled to the timed run's median SM clock (the FMA rate is
    proportional to the clock)."""
    f_leg, f_run = leg["clocks"].get("sm_mhz"), run_clocks.get("sm_mhz")
    scale = (f_run / f_leg) if (f_leg and f_run) else 1.0
    src = (f"bench.py FP64 FMA-chain leg (ap_dvm_fma_peak): {leg['tflops']} TFLOP/s at {f_leg} MHz median SM clock, "
           f"scaled to the timed run's {f_run} MHz")
    return {"tflops_at_run_clock": leg["tflops"] * scale, "source": src}


# ----------------------------------------------------------------- the oracle on the host cores
_ORACLE_STATE = {}


def _oracle_init(n, eps, tau, dt):
    """Worker set-up (spawned process): the workload's initial state and parameters."""
    from oracle import ap_dvm_oracle as O
    from paper_2512_19847_gb300 import workloads as W
    A_ex, _, A_im, _ = O.tableau_gsa2()
    _ORACLE_STATE["p"] = O.Params(n, n, eps, tau, dt, A_ex, A_im, scheme="WENO5_C4")
    _ORACLE_STATE["X"] = O.equilibrium_state(*W.taylor_green(n))


def _oracle_steps(nsteps):
    """Advance this worker's replica by nsteps oracle IMEX steps; returns the seconds taken."""
    from oracle import ap_dvm_oracle as O
    t0 = time.perf_counter()
    for _ in range(nsteps):
        _ORACLE_STATE["X"] = O.step(_ORACLE_STATE["X"], _ORACLE_STATE["p"])
    return time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_pool_size(n: int, want: int) -> int:
    """Workers for the all-core figure: every host core, capped so that the
    replicas (about 80 planes of n^2 float64 each, stage caches included) fit in
    half of the host memory."""
    try:
        mem = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    except (ValueError, OSError, AttributeError):
        mem = 64e9
    per = 80 * n * n * 8
    return max(1, min(want, int(0.5 * mem // per)))


class OraclePool:
    """P spawned processes, each holding its own replica of the workload: one
    'step' advances every replica by one oracle IMEX step (independent
    replicas on the host cores, the oracle's all-core throughput).  Started
    with 'spawn' so that no worker inherits a CUDA context."""

    def __init__(self, procs: int, n, eps, tau, dt):
        import multiprocessing as mp
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        self.procs = procs
        self.pool = mp.get_context("spawn").Pool(procs, initializer=_oracle_init, initargs=(n, eps, tau, dt))

    def step(self, nsteps: int = 1) -> float:
        t0 = time.perf_counter()
        self.pool.map(_oracle_steps, [nsteps] * self.procs, chunksize=1)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(n, eps, mach, tau, dt, fields, nsteps=1):
    """The oracle as it stands on the host: one IMEX step of the full-size
    workload on one core, and one step on each of P independent replicas in P
    processes (all host cores, memory permitting)."""
    from oracle import ap_dvm_oracle as O
    A_ex, _, A_im, _ = O.tableau_gsa2()
    X = O.equilibrium_state(*fields)
    p = O.Params(n, n, eps, tau, dt, A_ex, A_im, scheme="WENO5_C4")
    t0 = time.perf_counter()
    for _ in range(nsteps):
        X = O.step(X, p)
    el1 = time.perf_counter() - t0
    v1 = n * n * nsteps / el1 / 1e6
    ncores = host_cores()
    procs = oracle_pool_size(n, ncores)
    pool = OraclePool(procs, n, eps, tau, dt)
    try:
        pool.step(0)                     # workers up, state built
        elp = pool.step(nsteps)
    finally:
        pool.close()
    vp = procs * n * n * nsteps / elp / 1e6
    return {"value": round(vp, 4), "unit": UNIT, "cores": procs, "kind": "oracle", "nproc": ncores,
            "single_core_value": round(v1, 4),
            "sample": (f"{nsteps} IMEX step(s) of the {n}x{n} workload (numpy float64): on {procs} independent "
                       f"replicas in {procs} spawned processes, one thread each ({elp:.1f} s; value), and on one "
                       f"core ({el1:.1f} s; single_core_value); host nproc = {ncores}")}


def fp32_errors(X32: np.ndarray, X64: np.ndarray) -> tuple[float, float]:
    """Max relative velocity error and pressure error (p = theta - |u|^2/2, mean
    removed, relative to the FP64 pressure's range) of an FP32-form state
    against the FP64 form's state after the same steps."""
    umax = float(np.max(np.hypot(X64[0], X64[1])))
    vel = float(np.max(np.hypot(X32[0] - X64[0], X32[1] - X64[1])) / umax)
    p64 = X64[2] - 0.5 * (X64[0] ** 2 + X64[1] ** 2)
    p32 = X32[2] - 0.5 * (X32[0] ** 2 + X32[1] ** 2)
    p64, p32 = p64 - p64.mean(), p32 - p32.mean()
    return vel, float(np.max(np.abs(p32 - p64)) / max(float(np.max(np.abs(p64))), 1e-300))


def _finite_slots(b, slots) -> list:
    """Slots whose state is finite (the batch's non-finite flag is global)."""
    import torch
    return [k for k in slots if bool(torch.isfinite(b.get_state(k)).all())]


def _sync_allow_nonfinite(b) -> bool:
    """sync_status that reports a non-finite state instead of raising; other errors raise."""
    from paper_2512_19847_gb300 import api
    try:
        b.sync_status()
        return True
    except api.ApDvmError as e:
        if e.status != 5:
            raise
        return False


def run_batched(torch, count=256, steps=200, seed=2512, sample=16):
    """Batched form: `count` seeded uneven instances (side uniform in
    {64,128,256,512}, eps log-uniform [1e-6,1], Ma log-uniform [1e-3,1e-1],
    random divergence-free fields, tau = 0.05), FP32 deviation storage, tile
    chosen by the autotuner, all `steps` steps replayed as one CUDA graph.  At
    eps ~ 1 (far from the low-Mach regime) some random fields grow without bound
    under the time-step rule: the oracle does the same at the same step
    (tests/test_gpu_experiments.py), so they are counted, not removed.  The FP32
    form's velocity and pressure errors are stated against the FP64 form on a
    seeded sample of `sample` of the instances that stay finite."""
    from paper_2512_19847_gb300 import api, autotune, tableaux, workloads as W
    draws = W.batched_draws(count, seed=seed, steps=steps, eps_range=(1e-6, 1.0))
    tmpl = api.default_params(512, 512, eps=1e-2, dt=1e-3, tau=0.05, tableau=tableaux.gsa2(), precision=api.FP32_DEV)
    b = api.Batch(tmpl, capacity=count)
    cells = 0
    prms = []
    for k, d in enumerate(draws):
        u1, u2, p = W.random_divfree(d.n, d.seed)
        prm = tmpl.copy()
        prm.nx = prm.ny = d.n
        prm.eps, prm.mach = d.eps, d.mach
        prm.dt = W.stable_dt(u1, u2, 2 * math.pi / d.n, prm.tau)
        b.attach(k, prm)
        b.set_equilibrium(*[torch.from_numpy(a).cuda() for a in (u1, u2, p)], slot=k)
        prms.append(prm)
        cells += d.n * d.n
    tuned = autotune.tune(b, steps=2, path=None)
    b.set_graph_steps(steps)
    b.step(steps)                          # warm-up (also builds the graph)
    _sync_allow_nonfinite(b)
    torch.cuda.synchronize()
    for k, d in enumerate(draws):          # restart from the initial data
        u1, u2, p = W.random_divfree(d.n, d.seed)
        b.set_equilibrium(*[torch.from_numpy(a).cuda() for a in (u1, u2, p)], slot=k)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    b.step(steps)                          # one graph launch
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    _sync_allow_nonfinite(b)
    finite = _finite_slots(b, range(count))
    blown = [{"n": draws[k].n, "eps": round(draws[k].eps, 4)} for k in range(count) if k not in set(finite)]
    # FP32 error against the FP64 form on a seeded sample of the finite instances
    rng = np.random.default_rng(seed + 1)
    pick = sorted(rng.choice(finite, size=min(sample, len(finite)), replace=False).tolist())
    t64 = tmpl.copy()
    t64.precision = api.FP64
    b64 = api.Batch(t64, capacity=len(pick))
    for j, k in enumerate(pick):
        q = prms[k].copy()
        q.precision = api.FP64
        b64.attach(j, q)
        u1, u2, p = W.random_divfree(draws[k].n, draws[k].seed)
        b64.set_equilibrium(*[torch.from_numpy(a).cuda() for a in (u1, u2, p)], slot=j)
    b64.set_tile(3)
    b64.step(steps)
    b64.sync_status()
    errs = [fp32_errors(b.get_state(k).cpu().numpy(), b64.get_state(j).cpu().numpy()) for j, k in enumerate(pick)]
    return {"value": round(cells * steps / (ms * 1e-3) / 1e6, 2), "unit": UNIT, "instances": count,
            "cells": cells, "steps": steps, "ms": round(ms, 2), "graph_launches": 1,
            "kernel_launches": b.launches_per_step * steps, "tile": tuned["tile"],
            "tile_ms_per_step": tuned["ms_per_step"], "dtype": "f32 deviation storage",
            "eps_range": [1e-6, 1.0], "nonfinite_instances": blown,
            "velocity_rel_err_vs_fp64": max(e[0] for e in errs), "pressure_rel_err_vs_fp64": max(e[1] for e in errs),
            "error_sample": f"max over {len(pick)} seeded instances of the {len(finite)} finite ones (FP64 form, same draws)"}


def run_served(torch, n_requests=500, budget=120e9, load=0.8, v_ref=None, seed=7, sample=8, alone=True):
    """Served form: open-loop Poisson stream (side uniform {128,256,512,1024},
    eps log-uniform [1e-6,1e-1], 50-500 steps, tau = 0.05) at `load` times the
    stream rate the batched form sustains (v_ref Mcell-updates/s), admitted by an
    HBM budget into one continuous batch (FP32 deviation form), against the same
    stream served one solve at a time with the plain per-solve path.  The FP32
    form's errors are stated against the FP64 form, each of a seeded sample of
    `sample` requests re-run alone in FP64."""
    from paper_2512_19847_gb300 import api, serve, tableaux, workloads as W
    sides, steps_rng = (128, 256, 512, 1024), (50, 500)
    mean_work = np.mean([n * n for n in sides]) * np.mean(steps_rng)
    rate = load * (v_ref or 1000.0) * 1e6 / mean_work
    reqs = W.poisson_requests(n_requests, rate_hz=rate, seed=seed, sides=sides, steps_range=steps_rng)
    tmpl = api.default_params(1024, 1024, eps=1e-2, dt=1e-3, tau=0.05, mach=1e-2, tableau=tableaux.gsa2(),
                              precision=api.FP32_DEV)
    cache = {}

    def fields(n, s):
        if (n, s) not in cache:
            u1, u2, p = W.random_divfree(n, s)
            cache[(n, s)] = (u1, u2, p, W.stable_dt(u1, u2, 2 * math.pi / n, 0.05))
        return cache[(n, s)]
    jobs = serve.make_jobs(reqs, tmpl, fields)
    tile = 2                                             # 16x8: the autotuner's pick for the FP32 form at 2048^2 and for the batched mix
    srv = serve.Server(tmpl, capacity=n_requests, hbm_budget=budget, chunk=10, tile=tile)
    mixed = srv.run(jobs).summary()
    mixed.update({"load": load, "rate_hz": round(rate, 3), "hbm_budget_gb": budget / 1e9, "chunk_steps": 10, "tile": tile})
    # FP32 errors: a seeded sample of the served results against FP64 re-runs of the same requests
    rng = np.random.default_rng(seed + 1)
    errs = []
    for k in sorted(rng.choice(len(jobs), size=min(sample, len(jobs)), replace=False).tolist()):
        j = jobs[k]
        q = j.params.copy()
        q.precision = api.FP64
        s64 = api.Solver(q)
        s64.set_tile(3)
        s64.set_graph_steps(1)
        s64.set_equilibrium(*[t.to("cuda") for t in j.fields])
        s64.step(j.steps)
        s64.sync_status()
        errs.append(fp32_errors(j.result.numpy(), s64.get_state().cpu().numpy()))
    mixed.update({"velocity_rel_err_vs_fp64": max(e[0] for e in errs), "pressure_rel_err_vs_fp64": max(e[1] for e in errs),
                  "error_sample": f"max over {len(errs)} seeded requests, each re-run alone in FP64"})
    out = {"continuous_batching": mixed}
    if alone:
        alone_jobs = serve.make_jobs(reqs, tmpl, fields)
        out["alone_per_solve"] = serve.run_alone(alone_jobs, tile=tile).summary()
    return out


def run_size_sweep(torch, cells=2048 * 2048, steps=5, tile=2):
    """Per-cell step cost of the FP32 deviation form in batches of equal total cells and
    one grid size each (1 x 2048^2, 16 x 512^2, 64 x 256^2, 256 x 128^2, 1024 x 64^2;
    Taylor-Green-like random divergence-free field, eps = 1e-4, Ma = 1e-2, tile 16x8):
    per-kernel CUDA-event time per step divided by the cells, in ns."""
    from paper_2512_19847_gb300 import api, tableaux, workloads as W
    out = []
    for n in (2048, 512, 256, 128, 64):
        count = cells // (n * n)
        t = api.default_params(n, n, eps=1e-4, dt=1e-3, tau=0.05, mach=1e-2, tableau=tableaux.gsa2(),
                               precision=api.FP32_DEV)
        b = api.Batch(t, capacity=count)
        u1, u2, p = W.random_divfree(n, 7)
        dt = W.stable_dt(u1, u2, 2 * math.pi / n, 0.05)
        f = [torch.from_numpy(a).cuda() for a in (u1, u2, p)]
        for k in range(count):
            q = t.copy()
            q.dt = dt
            b.attach(k, q)
            b.set_equilibrium(*f, slot=k)
        b.set_tile(tile)
        b.step(3)
        torch.cuda.synchronize()
        b.profile(True)
        b.step(steps)
        prof = b.profile_read()
        b.profile(False)
        per = {k: round(v[0] / steps * 1e6 / (n * n * count), 4) for k, v in prof.items()}
        out.append({"n": n, "instances": count, "ns_per_cell": round(sum(per.values()), 4), "kernels_ns_per_cell": per})
        del b
        torch.cuda.empty_cache()
    return out


def run_served_sweep(torch, v_ref, loads=(0.5, 0.7, 0.9), n_requests=500):
    """p50/p99 and Mcell-updates/s of the served form and of the per-solve path at
    several arrival rates (fractions of the batched form's sustained rate)."""
    rows = []
    for ld in loads:
        r = run_served(torch, n_requests=n_requests, load=ld, v_ref=v_ref, sample=2)
        c, a = r["continuous_batching"], r["alone_per_solve"]
        rows.append({"load": ld, "rate_hz": c["rate_hz"], "batched_p50_ms": c["p50_ms"], "batched_p99_ms": c["p99_ms"],
                     "batched_mcells": c["value"], "alone_p50_ms": a["p50_ms"], "alone_p99_ms": a["p99_ms"],
                     "alone_mcells": a["value"], "max_resident": c["max_resident"]})
    return rows


def replica_rate(ms_local: float, cells: int, steps: int, dist=None, device: str = "cuda"):
    """Whole-job throughput of N independent replicas (the solve does not shard):
    the slowest rank's time (max over ranks) and the cells of all ranks.
    Returns (Mcell-updates/s, max ms)."""
    import torch
    world = 1
    ms = float(ms_local)
    if dist is not None:
        world = dist.get_world_size()
        t = torch.tensor([ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * cells * steps / (ms * 1e-3) / 1e6, ms


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ----------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The reference arm: the oracle (the only other implementation of the
    method) as it stands, on the host cores, on the same 2048^2 workload.  A
    step advances P independent replicas (P spawned processes, one per host
    core, memory permitting) by one oracle IMEX step each."""
    if rank != 0:
        return
    n = args.n
    _, dt = workload(n, args.eps, args.mach, args.tau)
    ncores = host_cores()
    procs = oracle_pool_size(n, ncores)
    pool = OraclePool(procs, n, args.eps, args.tau, dt)
    try:
        pool.step(0)
        for _ in range(args.warmup):
            pool.step(1)
        el = pool.step(args.steps)
    finally:
        pool.close()
    v = procs * n * n * args.steps / el / 1e6
    sample = (f"one IMEX step of the {n}x{n} workload on each of {procs} independent replicas per step "
              f"({procs} spawned processes, one numpy thread each; host nproc = {ncores})")
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(args),
            "cpu_baseline": {"value": round(v, 4), "unit": UNIT, "cores": procs, "nproc": ncores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(v, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(args):
    return {"workload": f"taylor_green_{args.n}x{args.n}_eps{args.eps:g}_Ma{args.mach:g}",
            "grid": [args.n, args.n], "eps": args.eps, "mach": args.mach, "tau": args.tau,
            "dt_rule": "min(0.4 dx/max|u|, 0.32 dx^2/(tau/4))",
            "tableau": "GSA2 c=2.25", "space": "WENO5+C4", "l2": l2_note(args.n)}


def l2_note(n: int) -> str:
    """The timing rule's L2 statement for an n x n workload (129 MB of L2; the step's
    working set scales with the cells, about 1.7 GB at 2048^2)."""
    state, work = 48 * n * n / 1e6, 1.7 * n * n / 2048 ** 2
    side = "larger" if state > 129 else "smaller"
    return f"inputs {side} than L2 (FP64 state {state:.0f} MB, step working set ~{work:.2g} GB)"


# ----------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--eps", type=float, default=1e-4)
    ap.add_argument("--mach", type=float, default=1e-3)
    ap.add_argument("--tau", type=float, default=0.05)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=3)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--fp64-peak", action="store_true", help="print only the FMA-peak legs (FP64 and FP32) and exit")
    ap.add_argument("--served-sweep", action="store_true", help="also sweep the served form's arrival rate")
    ap.add_argument("--size-sweep", action="store_true",
                    help="print only the per-cell step cost of equal-cell FP32 batches of one grid size each and exit")
    ap.add_argument("--tiles", default=None,
                    help="FP64,FP32 tile indices (autotune.TILES) instead of the autotuner, e.g. 5,2 for profiling "
                         "runs, whose perturbed timings would make the autotuner pick other shapes")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    n, cells = args.n, args.n * args.n
    from paper_2512_19847_gb300 import api
    if args.fp64_peak:
        legs = {"fp64": fma_peak_leg(local, api.FP64, 256), "fp32": fma_peak_leg(local, api.FP32_DEV, 16384)}
        if rank == 0:
            print(json.dumps({"fma_peak": legs}), flush=True)
        return
    if args.size_sweep:
        sweep = run_size_sweep(torch)
        if rank == 0:
            print(json.dumps({"size_sweep": sweep}), flush=True)
        return
    fields, dt = workload(n, args.eps, args.mach, args.tau)
    peaks = load_peaks()
    tile64, tile32 = (int(t) for t in args.tiles.split(",")) if args.tiles else (None, None)

    with ClockSampler(local) as clk:
        s64, ms64 = time_form(torch, fields, n, args.eps, args.mach, args.tau, dt, False, args.steps, args.warmup, barrier,
                              tile=tile64)
    clocks = clk.summary()
    fp64_leg = fma_peak_leg(local, api.FP64, 256)
    fp64_peak = scaled_peak(fp64_leg, clocks)
    s32, ms32 = time_form(torch, fields, n, args.eps, args.mach, args.tau, dt, True, args.steps, args.warmup, barrier,
                          tile=tile32)

    v64, ms64 = replica_rate(ms64, cells, args.steps, dist, "cuda")
    v32, ms32 = replica_rate(ms32, cells, args.steps, dist, "cuda")

    # accuracy of the FP32 deviation form against the FP64 result after the same steps
    X64 = s64.get_state().cpu().numpy()
    X32 = s32.get_state().cpu().numpy()
    vel_err, pr_err = fp32_errors(X32, X64)

    # per-kernel CUDA-event profile on the launching stream, dominant kernel roofline
    prof64 = profile_form(s64, args.profile_steps)
    prof32 = profile_form(s32, args.profile_steps)
    k64, roof64 = roofline(prof64, args.profile_steps, cells, False, "WENO5_C4", n, peaks, fp64_peak)
    k32, roof32 = roofline(prof32, args.profile_steps, cells, True, "WENO5_C4", n, peaks)
    launches64 = s64.launches_per_step * args.steps

    # end to end through the public API with host buffers: per step, H2D of the
    # state from pinned memory, the step, and D2H of the resulting state
    Xh = torch.from_numpy(X64).pin_memory()
    e2e_steps = max(2, min(args.steps, 5))
    s64.run_host(Xh, 1)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        Xh = s64.run_host(Xh, 1)
    e2e_rate, _ = replica_rate((time.perf_counter() - t0) * 1e3, cells, e2e_steps, dist, "cuda")
    e2e = {"value": round(e2e_rate, 3), "unit": UNIT,
           "h2d_bytes_per_step": 6 * cells * 8, "d2h_bytes_per_step": 6 * cells * 8}

    def leg(fn, *a, **kw):
        # a failing secondary leg is reported in the line instead of losing the line
        try:
            return fn(*a, **kw)
        except Exception as e:            # noqa: BLE001
            torch.cuda.synchronize()
            return {"error": f"{type(e).__name__}: {e}"[:300]}

    batched = None if args.no_batched else leg(run_batched, torch)
    v_ref = (batched or {}).get("value", v32) if isinstance(batched, dict) and "value" in (batched or {}) else v32
    served = None if args.no_served else leg(run_served, torch, v_ref=v_ref)
    sweep = leg(run_served_sweep, torch, v_ref) if args.served_sweep else None
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline(n, args.eps, args.mach, args.tau, dt, fields)
    from paper_2512_19847_gb300.autotune import TILES as autotune_tiles
    line = {
        "metric": METRIC, "value": round(v64, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms64 / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(config_dict(args), tile_fp64=list(autotune_tiles[s64.tile]), tile_fp32=list(autotune_tiles[s32.tile])),
        "roofline": roof64,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches64,
        "clocks": clocks,
        "fma_peak_fp64": fp64_leg,
        "fp32_dev": {"value": round(v32, 3), "unit": UNIT, "ms_per_step": round(ms32 / args.steps, 4),
                     "dtype": "f32 transport, f64 moment sums and relaxation (eps<=1e-4)",
                     "velocity_rel_err_vs_fp64": vel_err, "pressure_rel_err_vs_fp64": pr_err,
                     "roofline": roof32, "gpu_launches": s32.launches_per_step * args.steps},
        "batched": batched,
        "served": served,
        "served_sweep": sweep,
        "kernels_fp64_ms_per_step": {k: round(v[0] / args.profile_steps, 4) for k, v in prof64.items()},
        "kernels_fp32_ms_per_step": {k: round(v[0] / args.profile_steps, 4) for k, v in prof32.items()},
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
