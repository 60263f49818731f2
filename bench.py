"""Benchmark: DVM cell-velocity updates/s of the GSIS kinetic step on one GB300.

A step is one outer iteration through the library's C ABI (gsis_step_async): per-cell
reference-distribution coefficients, wall densities, the implicit second-order
finite-volume sweep of the four gas planes and of the photon intensities with block
Gauss-Seidel point relaxation, the velocity moments, the FP64 macroscopic fields and
the convergence measure.  Workload: 2-D heated lid-driven cavity, 20 000 seeded
triangles, 28 x 28 closed Newton-Cotes (trapezoid) velocity grid, 64 photon directions, FP32 f and I.

``value``  device-timed, distributions resident in HBM (both f buffers exceed L2).
``e2e``    same metric through the C ABI with host buffers: every step uploads f and I
           from pinned host memory, iterates, and reads the fields back.
``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same
workload (the only other place this script runs the oracle).

Further keys of the line (each leg can be skipped with its --no-* flag):
``time_to_steady``  wall time to eps < 1e-6 on the 32 x 32 cavity: plain FP64 GSIS
                    against the FP32 forms and the learned warm start;
``normal_shock``    CIS and GSIS iterations on the Mach-5 normal shock;
``cylinder``        CIS and GSIS iterations and seconds on the Mach-5 cylinder;
``cpu_baseline``    the oracle timed on a bounded sample, on the host cores.

With ``--gpus N`` (torchrun, one rank per GPU) the velocity and photon sets are cut into N
contiguous ranges, one per rank (paper_2601_03935_gb300.shard): every rank sweeps all
cells for its velocities, and one NCCL all-reduce per iteration sums the per-cell moment
sums and wall outflow.  The work of one step is fixed (strong scaling); the timing is
the maximum over ranks and value is the updates of the whole problem per second.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "DVM cell-velocity updates/s (% HBM roofline); time-to-steady vs plain FP64 GSIS"
# DRAM bytes (read + write) of one gas slope pass + sweep on the 20 000-cell cavity (FP32,
# order 2) come from the ncu capture summarised in this file.  It records them with the
# SHA-256 of the kernel sources the capture ran; the figure is reported only while those
# sources are unchanged, and as null once a kernel has changed since the counters were taken.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "sweep_gas_cavity20k_order2.md")
KERNEL_SOURCES = ("kernels.cu", "gsis_impl.cuh", "tc_moments.cuh")


def kernel_sources_sha256(csrc=None):
    import hashlib
    csrc = csrc or os.path.join(ROOT, "paper_2601_03935_gb300", "csrc")
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def sweep_traffic(precision, order, path=TRAFFIC_FILE, csrc=None):
    """(bytes per launch pair or None, note) from the recorded capture."""
    import re
    if (precision, order) != ("fp32", 2):
        return None, "no capture of this precision and order"
    try:
        text = open(path).read()
    except OSError:
        return None, "no capture recorded"
    t = re.search(r"^traffic_bytes_per_launch_pair: (\d+)\s*$", text, re.M)
    h = re.search(r"^kernel_sources_sha256: ([0-9a-f]{64})\s*$", text, re.M)
    if not t or not h:
        return None, "no capture recorded"
    if h.group(1) != kernel_sources_sha256(csrc):
        return None, "kernel sources changed since the capture"
    return float(t.group(1)), "ncu capture of these kernel sources"
UNIT = "updates/s"


def workload(args):
    import gsis_inputs as gi
    wl = gi.workloads.cavity(n_side=100, Kn=args.kn, Kn_p=args.kn_p)
    return gi.workloads.with_solver(wl, precision=args.precision, order=args.order, relax_block=args.block,
                                    tc_moments=args.tc_moments)


def config(args, wl):
    return {"workload": "cavity 2-D, %d triangles, 28x28 closed Newton-Cotes (trapezoid) velocities (%d), %d photon directions"
                        % (wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0]),
            "n_cells": wl.mesh.n_cells, "n_xi": int(wl.xi.shape[0]), "n_omega": int(wl.omega.shape[0]),
            "order": args.order, "relax_block": args.block, "tc_moments": args.tc_moments, "Kn": args.kn, "Kn_photon": args.kn_p,
            "step": ("one CIS outer iteration (kinetic sweep + moments + fields + epsilon)" if args.mode == "cis" else
                     "one GSIS outer iteration (kinetic sweep + moments + high-order terms + synthetic solve + "
                     "synchronisation + epsilon)"),
            "l2": "inputs larger than L2 (f: 2 x %.0f MB)" % (wl.mesh.n_cells * 896 * 16 / 1e6),
            "parallelism": "1 GPU"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if len(s) > 8 and s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if len(s) > 8 and s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples if len(s) > 8 for k in range(4)
                          if s[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def create_ctx(wl, stream):
    from paper_2601_03935_gb300 import gsis as G
    m = wl.mesh
    return G.gsis_create(m.dim, m.face_owner, m.face_nbr, m.face_normal, m.face_area, m.face_centroid,
                         m.cell_volume, m.cell_centroid, m.patches, wl.xi, wl.w, wl.omega, wl.wo, wl.model,
                         wl.solver, stream, period=getattr(m, "period", 0.0))


def initial_state(wl):
    """Uniform gas at rest, rho = T = 1 (the paper's cases start from a uniform state)."""
    import gsis_inputs as gi
    M = gi.fields.uniform_fields(wl.mesh.n_cells, rho=1.0, T=1.0)
    return gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 2, wl.model.d_r, wl.model.d_v, wl.model.sigma_R,
                                       seed=1, noise=0.0)


_ORACLE = {}


def _oracle_worker_init(kn, kn_p, precision, order, block, tc_moments):
    """Builds the workload, its initial state and the oracle's geometry once per worker."""
    import types
    from oracle import kinetic as K
    args = types.SimpleNamespace(kn=kn, kn_p=kn_p, precision=precision, order=order, block=block,
                                 tc_moments=tc_moments)
    wl = workload(args)
    f, I = initial_state(wl)
    _ORACLE.update(wl=wl, f=f, I=I, geo=K.Geometry(wl.mesh))


def _oracle_worker_run(seconds, seed):
    """FP64 oracle sweeps of whole random relaxation blocks for about `seconds`: the cells
    swept and the elapsed time.  Blocks are independent within one sweep (Jacobi between
    blocks), so workers on different blocks do the work one sweep does, in parallel."""
    from oracle import kinetic as K
    wl, f, I, geo = _ORACLE["wl"], _ORACLE["f"], _ORACLE["I"], _ORACLE["geo"]
    B = wl.solver.relax_block
    n_blocks = (wl.mesh.n_cells + B - 1) // B
    rng = np.random.default_rng(seed)
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        b = int(rng.integers(n_blocks))
        cells = np.arange(b * B, min(b * B + B, wl.mesh.n_cells))
        K.kinetic_sweep(f, I, wl, geo=geo, cells=cells, relax_block=B)
        done += len(cells)
    return done, time.perf_counter() - t0


def cpu_baseline(args, seconds=12.0, cores=None):
    """The FP64 oracle on the host cores: a spawn process pool (safe after CUDA use), one
    worker per core, each sweeping random whole relaxation blocks for ~`seconds`; also one
    worker alone for the single-thread rate."""
    import concurrent.futures as cf
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    init = (args.kn, args.kn_p, args.precision, args.order, args.block, args.tc_moments)
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=ctx, initializer=_oracle_worker_init,
                                initargs=init) as ex:
        list(ex.map(_oracle_worker_run, [0.01] * cores, range(cores)))          # every worker set up
        res = list(ex.map(_oracle_worker_run, [seconds] * cores, range(100, 100 + cores)))
        one = ex.submit(_oracle_worker_run, seconds / 2, 999).result()
    n_xi = _n_xi_of(args)
    cells = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return {"value": cells * n_xi / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_thread_value": one[0] * n_xi / one[1],
            "sample": "%d cells (random whole relaxation blocks of %d) x %d velocities, FP64 NumPy oracle, "
                      "%d spawn processes on %d host cores (one NumPy thread each), %.1f s" % (
                          cells, args.block, n_xi, cores, cores, wall)}


def _n_xi_of(args):
    import gsis_inputs as gi
    return gi.workloads.cavity(n_side=2).xi.shape[0]


def _oracle_worker_block(seed):
    """One random whole relaxation block swept by the FP64 oracle: the cells swept."""
    from oracle import kinetic as K
    wl, f, I, geo = _ORACLE["wl"], _ORACLE["f"], _ORACLE["I"], _ORACLE["geo"]
    B = wl.solver.relax_block
    b = int(np.random.default_rng(seed).integers((wl.mesh.n_cells + B - 1) // B))
    cells = np.arange(b * B, min(b * B + B, wl.mesh.n_cells))
    K.kinetic_sweep(f, I, wl, geo=geo, cells=cells, relax_block=B)
    return len(cells)


def run_reference(args):
    """The FP64 oracle as it stands on the host cores: a spawn process pool with one worker
    per core; a step sweeps one random whole relaxation block on every worker."""
    import concurrent.futures as cf
    import multiprocessing as mp
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = workload(args)
    cores = os.cpu_count() or 1
    init = (args.kn, args.kn_p, args.precision, args.order, args.block, args.tc_moments)
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn"),
                                initializer=_oracle_worker_init, initargs=init) as ex:
        seed = [0]

        def step():
            seeds = list(range(seed[0], seed[0] + cores))
            seed[0] += cores
            return sum(ex.map(_oracle_worker_block, seeds))

        for _ in range(args.warmup):
            step()
        t0 = time.perf_counter()
        cells = sum(step() for _ in range(args.steps))
        dt = time.perf_counter() - t0
    value = cells * wl.xi.shape[0] / dt
    sample = ("%d steps x %d random relaxation blocks of %d cells (one per worker) x %d velocities (FP64 NumPy oracle, "
              "%d spawn processes on %d host cores)" % (args.steps, cores, args.block, wl.xi.shape[0], cores, cores))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(args, wl),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def time_to_steady(stream, n_side=32, kn=0.01, kn_p=10.0, tol=1e-6, max_outer=150, inner=100,
                   train_kn=(0.02, 0.05)):
    """Wall time from a uniform rest state to eps < tol (Section 6 criterion) with GSIS and
    the paper's inner budget (100 synthetic iterations, tolerance 1e-7): plain FP64; FP32
    distributions with tensor-core moments; the same with the synthetic residual side and
    the relaxation's flux increments in FP32 for all but the last 16 inner iterations
    (macro_fp32 = 2); and that with the
    learned warm start.  The network is trained on the solver's own samples from runs at
    other Knudsen numbers; collection and training are timed separately from the solve."""
    import torch
    import gsis_inputs as gi
    from paper_2601_03935_gb300 import gsis as G

    def make(prec, k, mixed=False):
        wl = gi.workloads.cavity(n_side=n_side, Kn=k, Kn_p=kn_p)
        return gi.workloads.with_solver(wl, precision=prec, order=1, relax_block=16, max_inner=inner,
                                        n_cis_precond=10, macro_fp32=2 if mixed else 0)

    def fresh(wl):
        ctx = create_ctx(wl, stream.cuda_stream)
        f, I = initial_state(wl)
        G.gsis_set_distributions(ctx, f, I)
        torch.cuda.synchronize()
        return ctx

    def run(prec, params=None, mixed=False):
        wl = make(prec, kn, mixed)
        ctx = fresh(wl)
        try:
            t0 = time.perf_counter()
            tw = 0.0
            if params is not None:
                G.gsis_mlp_set_params(ctx, params)
                G.gsis_warm_start(ctx, 2, use_mlp=True)
                tw = time.perf_counter() - t0
            it, hist = G.gsis_solve(ctx, G.GSIS_MODE_GSIS, max_outer, tol)
            dt = time.perf_counter() - t0
        finally:
            G.gsis_destroy(ctx)
        return {"seconds": dt, "iterations": it, "final_eps": float(hist[-1]) if len(hist) else None,
                "converged": bool(len(hist) and hist[-1] < tol), "warm_start_seconds": tw}

    out = {"workload": "cavity 2-D, %d triangles (%dx%d), Kn=%g, Kn_p=%g, order 1, %d inner iterations"
                       % (2 * n_side * n_side, n_side, n_side, kn, kn_p, inner), "tol": tol}
    out["fp64_plain"] = run("fp64")
    out["fp32_plain"] = run("fp32")
    out["fp32_mixed"] = run("fp32", mixed=True)
    t0 = time.perf_counter()
    Xs, Ys = [], []
    for k in train_kn:
        wl = make("fp32", k)
        ctx = fresh(wl)
        try:
            for j in range(40):
                G.gsis_step(ctx, G.GSIS_MODE_GSIS if j >= 10 else G.GSIS_MODE_CIS)
                if j >= 10:
                    X, Y = G.gsis_mlp_samples(ctx, wl.mesh.n_cells)
                    Xs.append(X)
                    Ys.append(Y)
            if k == train_kn[-1]:
                collect = time.perf_counter() - t0
                G.gsis_mlp_init(ctx, 3)
                t1 = time.perf_counter()
                loss = G.gsis_mlp_train(ctx, np.concatenate(Xs), np.concatenate(Ys), epochs=40, batch=2048,
                                        lr=1e-3, seed=4)
                train = time.perf_counter() - t1
                params = G.gsis_mlp_get_params(ctx)
        finally:
            G.gsis_destroy(ctx)
    out["fp32_learned"] = run("fp32", params, mixed=True)
    out["fp32_learned"].update({"train_samples": int(sum(x.shape[0] for x in Xs)), "collect_seconds": collect,
                                "train_seconds": train, "train_loss": loss, "trained_on_Kn": list(train_kn)})
    out["speedup_fp32_mixed_vs_fp64_plain"] = out["fp64_plain"]["seconds"] / out["fp32_mixed"]["seconds"]
    out["speedup_fp32_learned_vs_fp64_plain"] = out["fp64_plain"]["seconds"] / out["fp32_learned"]["seconds"]
    return out


def time_to_steady_full(stream, kn=0.01, kn_p=10.0, tol=1e-6, max_gsis=900, max_cis=3000, inner=100):
    """Time to eps < tol on the full 20 000-cell cavity at Kn = 0.01 (order 1, blocks of 16,
    100 synthetic iterations of six relaxation sweeps per outer iteration, the paper's
    settings): GSIS in plain FP64 and in FP32 with the mixed synthetic schedule, and CIS in
    FP32 (stopped at max_cis) for context; then both GSIS forms with 200 inner iterations
    of two sweeps, the fastest setting of a scan.  From uniform rest; the timing excludes
    creation, as the paper's does."""
    import torch
    import gsis_inputs as gi
    from paper_2601_03935_gb300 import gsis as G

    def run(prec, mode, mixed, n, max_inner=inner, sweeps=6):
        wl = gi.workloads.with_solver(gi.workloads.cavity(n_side=100, Kn=kn, Kn_p=kn_p), precision=prec, order=1,
                                      relax_block=16, max_inner=max_inner, macro_sweeps=sweeps, n_cis_precond=10,
                                      macro_fp32=2 if mixed else 0)
        ctx = create_ctx(wl, stream.cuda_stream)
        try:
            G.gsis_init_fields(ctx, gi.fields.uniform_fields(wl.mesh.n_cells))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it, hist = G.gsis_solve(ctx, mode, n, tol)
            dt = time.perf_counter() - t0
        finally:
            G.gsis_destroy(ctx)
        return {"seconds": dt, "iterations": int(it), "final_eps": float(hist[-1]) if len(hist) else None,
                "converged": bool(len(hist) and hist[-1] < tol),
                "eps_every_100": [float(hist[k]) for k in range(99, len(hist), 100)]}

    out = {"workload": "cavity 2-D, 20000 triangles, 28x28 velocities, 64 directions, Kn=%g, Kn_p=%g, order 1, "
                       "%d synthetic iterations per GSIS iteration" % (kn, kn_p, inner), "tol": tol}
    out["gsis_fp64_plain"] = run("fp64", G.GSIS_MODE_GSIS, False, max_gsis)
    out["gsis_fp32_mixed"] = run("fp32", G.GSIS_MODE_GSIS, True, max_gsis)
    out["cis_fp32"] = run("fp32", G.GSIS_MODE_CIS, False, max_cis)
    if out["gsis_fp32_mixed"]["converged"] and out["gsis_fp64_plain"]["converged"]:
        out["speedup_fp32_mixed_vs_fp64_plain"] = out["gsis_fp64_plain"]["seconds"] / out["gsis_fp32_mixed"]["seconds"]
    out["gsis_fp64_plain_200x2"] = run("fp64", G.GSIS_MODE_GSIS, False, max_gsis, 200, 2)
    out["gsis_fp32_mixed_200x2"] = run("fp32", G.GSIS_MODE_GSIS, True, max_gsis, 200, 2)
    a, b = out["gsis_fp64_plain_200x2"], out["gsis_fp32_mixed_200x2"]
    if a["converged"] and b["converged"]:
        out["speedup_fp32_mixed_vs_fp64_plain_200x2"] = a["seconds"] / b["seconds"]
    if b["converged"] and out["gsis_fp64_plain"]["converged"]:
        out["speedup_fp32_mixed_200x2_vs_fp64_plain_paper_settings"] = out["gsis_fp64_plain"]["seconds"] / b["seconds"]
    return out


def time_to_steady_handover(args, kn=0.1, kn_p=10.0, w=0.7, tol=1e-6, switch=3e-6, nmax=3000):
    """Time to eps < tol on the 20 000-cell cavity at Kn = 0.1 (order 1, blocks of 16, the
    paper's inner settings, the synchronisation damped to w), where eps of FP32
    distributions stops near 1.5e-6: plain FP64 GSIS, against FP32 distributions with the
    mixed synthetic schedule until eps < switch, then the state handed to an FP64 context
    through the C ABI (gsis_get_distributions / gsis_set_distributions, doubles at the
    boundary) and FP64 GSIS to tol.  From uniform rest; the hand-over is timed."""
    import torch
    import gsis_inputs as gi
    from paper_2601_03935_gb300 import build
    from paper_2601_03935_gb300 import gsis as G
    build.build()
    G.load()
    stream = torch.cuda.Stream()
    base = gi.workloads.cavity(n_side=100, Kn=kn, Kn_p=kn_p)
    nc, V, NO = base.mesh.n_cells, base.xi.shape[0], base.omega.shape[0]

    def make(prec, mixed, cis_first):
        wl = gi.workloads.with_solver(base, precision=prec, order=1, relax_block=16, n_cis_precond=cis_first,
                                      macro_fp32=2 if mixed else 0, sync_relax=w)
        return create_ctx(wl, stream.cuda_stream)

    def solve(ctx, n, stop):
        it, hist = G.gsis_solve(ctx, G.GSIS_MODE_GSIS, n, stop)
        return int(it), (float(hist[-1]) if len(hist) else None)

    out = {"workload": "cavity 2-D, 20000 triangles, 28x28 velocities, 64 directions, Kn=%g, Kn_p=%g, order 1, "
                       "100 synthetic iterations of six sweeps, synchronisation weight %g" % (kn, kn_p, w),
           "tol": tol, "switch": switch}
    ctx = make("fp64", False, 10)
    try:
        G.gsis_init_fields(ctx, gi.fields.uniform_fields(nc))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it, eps = solve(ctx, nmax, tol)
        out["gsis_fp64_plain"] = {"iterations": it, "seconds": time.perf_counter() - t0, "final_eps": eps,
                                  "converged": bool(eps is not None and eps < tol)}
    finally:
        G.gsis_destroy(ctx)
    ctx = make("fp32", True, 10)
    try:
        G.gsis_init_fields(ctx, gi.fields.uniform_fields(nc))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it1, eps1 = solve(ctx, nmax, switch)
        t1 = time.perf_counter() - t0
        t0 = time.perf_counter()
        f, I = G.gsis_get_distributions(ctx, nc, V, NO)
    finally:
        G.gsis_destroy(ctx)
    ctx = make("fp64", False, 0)
    try:
        G.gsis_set_distributions(ctx, f, I)
        torch.cuda.synchronize()
        th = time.perf_counter() - t0
        t0 = time.perf_counter()
        it2, eps2 = solve(ctx, nmax, tol)
        t2 = time.perf_counter() - t0
    finally:
        G.gsis_destroy(ctx)
    out["gsis_fp32_mixed_then_fp64"] = {"fp32_iterations": it1, "fp32_seconds": t1, "fp32_final_eps": eps1,
                                        "handover_seconds": th, "fp64_iterations": it2, "fp64_seconds": t2,
                                        "final_eps": eps2, "seconds": t1 + th + t2,
                                        "converged": bool(eps2 is not None and eps2 < tol)}
    a, b = out["gsis_fp64_plain"], out["gsis_fp32_mixed_then_fp64"]
    if a["converged"] and b["converged"]:
        out["speedup"] = a["seconds"] / b["seconds"]
    print(json.dumps({"handover": out}))
    return 0


def time_to_steady_capsule(stream, n=12, n_v=16, Mach=3.0, tol=1e-6, max_gsis=300, max_cis=3000):
    """Time to eps < tol on a reduced 3-D capsule (the sphere-cone capsule geometry on 6 n^3 tetrahedra
    less the body, n_v^3 velocities, 8 x 16 directions, Kn = 0.01) at Mach 3, where 16^3
    velocities resolve the free stream, order 1, from the uniform free stream: GSIS in
    plain FP64 and with FP32 distributions and the mixed synthetic schedule, and CIS in FP32."""
    import torch
    import gsis_inputs as gi
    from paper_2601_03935_gb300 import gsis as G
    base = gi.workloads.capsule(n=n, n_v=n_v, Mach=Mach)
    far = base.mesh.patches[1]

    def run(prec, mode, mixed, nmax):
        wl = gi.workloads.with_solver(base, precision=prec, order=1, relax_block=16, max_inner=100, n_cis_precond=10,
                                      macro_fp32=2 if mixed else 0, venkat_K=0.01)
        ctx = create_ctx(wl, stream.cuda_stream)
        try:
            G.gsis_init_fields(ctx, gi.fields.uniform_fields(wl.mesh.n_cells, rho=far.rho, u=far.u, T=far.T_t))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it, hist = G.gsis_solve(ctx, mode, nmax, tol)
            dt = time.perf_counter() - t0
        finally:
            G.gsis_destroy(ctx)
        return {"seconds": dt, "iterations": int(it), "final_eps": float(hist[-1]) if len(hist) else None,
                "converged": bool(len(hist) and hist[-1] < tol)}

    out = {"workload": "capsule 3-D Mach %g, %d tetrahedra, %d^3 velocities, %d directions, Kn=0.01, order 1, "
                       "100 synthetic iterations per GSIS iteration" % (Mach, base.mesh.n_cells, n_v,
                                                                          base.omega.shape[0]), "tol": tol}
    out["gsis_fp64_plain"] = run("fp64", G.GSIS_MODE_GSIS, False, max_gsis)
    out["gsis_fp32_mixed"] = run("fp32", G.GSIS_MODE_GSIS, True, max_gsis)
    out["cis_fp32"] = run("fp32", G.GSIS_MODE_CIS, False, max_cis)
    if out["gsis_fp32_mixed"]["converged"] and out["gsis_fp64_plain"]["converged"]:
        out["speedup_fp32_mixed_vs_fp64_plain"] = out["gsis_fp64_plain"]["seconds"] / out["gsis_fp32_mixed"]["seconds"]
    return out


def normal_shock(max_gsis=300):
    """The paper's Mach-5 normal shock (FP64, order 2): CIS and GSIS outer iterations to
    eps < 2e-6 for (Z_r, Z_v) = (2.6, 26) on 200 L0 and (8, 100) on 350 L0, with the
    paper's iteration counts beside them; and GSIS with the defect-corrected synthetic
    equations and 400 inner iterations.  GSIS stops at max_gsis iterations."""
    import torch
    import gsis_inputs as gi
    from paper_2601_03935_gb300 import gsis as G
    paper = {26.0: {"cis": 991, "gsis": 68}, 100.0: {"cis": 2566, "gsis": 90}}
    out = {}
    for Zr, Zv, L in ((2.6, 26.0, 200.0), (8.0, 100.0, 350.0)):
        wl = gi.workloads.with_solver(gi.workloads.normal_shock(Z_r=Zr, Z_v=Zv, length=L), precision="fp64",
                                      order=2, relax_block=16, venkat_K=0.01, max_inner=100, tol_inner=1e-7)
        M = gi.fields.shock_fields(wl)
        f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 1, wl.model.d_r, wl.model.d_v, wl.model.sigma_R,
                                           0, noise=0.0)
        res = {"cells": wl.mesh.n_cells, "n_xi": wl.xi.shape[0], "n_omega": wl.omega.shape[0],
               "paper_iterations": paper[Zv]}
        wl_dc = gi.workloads.with_solver(wl, defect_correction=1, max_inner=400)
        for mode, name, mx, w_ in ((G.GSIS_MODE_CIS, "cis", 6000, wl), (G.GSIS_MODE_GSIS, "gsis", max_gsis, wl),
                                   (G.GSIS_MODE_GSIS, "gsis_defect_corrected_400_inner", max_gsis, wl_dc)):
            ctx = create_ctx(w_, 0)
            G.gsis_set_distributions(ctx, f, I)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it, hist = G.gsis_solve(ctx, mode, mx, 2e-6)
            torch.cuda.synchronize()
            res[name] = {"iterations": it, "seconds": time.perf_counter() - t0, "final_eps": float(hist[-1]),
                         "converged": bool(hist[-1] < 2e-6),
                         "eps_at": {str(k): float(hist[k]) for k in (9, 49, 99, 199) if k < len(hist)}}
            G.gsis_destroy(ctx)
        out["Zr%g_Zv%g_L%g" % (Zr, Zv, L)] = res
    return out


def slab_time_to_steady(oracle_seconds=40.0):
    """The 1-D planar slab (64 cells between walls at T = 1 and 1.5, optical
    thickness 1, 32 Gauss-Hermite velocities, 16 Gauss-Legendre directions, order 2, FP64)
    from the uniform rest state at T = 1.25: outer iterations and seconds to eps < 1e-8
    on the GPU for CIS and for GSIS (3 CIS iterations first), at the config's Kn = 0.1 and
    at Kn = 0.01, at Kn = 0.1 also GSIS with the defect correction and the synchronisation
    weight 0.8; and the FP64 oracle's time to the same tolerance on one host core (stopped
    after about `oracle_seconds`)."""
    import torch
    import gsis_inputs as gi
    from oracle import gsis as OG
    from oracle import kinetic as K
    from oracle import macro as MA
    from paper_2601_03935_gb300 import gsis as G
    out = {}
    for kn, inner, oracle_mode in ((0.1, 100, "cis"), (0.01, 200, "gsis")):
        wl = gi.workloads.with_solver(gi.workloads.slab(64, Kn=kn), precision="fp64", order=2, relax_block=16,
                                      max_inner=inner, tol_inner=1e-7, n_cis_precond=3)
        M = gi.fields.uniform_fields(64, T=1.25)
        f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 1, wl.model.d_r, wl.model.d_v, wl.model.sigma_R, 0,
                                           noise=0.0)
        res = {"workload": "slab 1-D, 64 cells, 32 velocities, 16 directions, Kn %g, Kn_p 1, FP64, order 2, "
                           "%d inner iterations, eps < 1e-8" % (kn, inner)}
        runs = [(G.GSIS_MODE_GSIS, "gsis", 200, wl), (G.GSIS_MODE_CIS, "cis", 20000, wl)]
        if kn == 0.1:
            runs.append((G.GSIS_MODE_GSIS, "gsis_defect_corrected_w0.8", 600,
                         gi.workloads.with_solver(wl, defect_correction=1, sync_relax=0.8)))
        for mode, name, mx, w_ in runs:
            ctx = create_ctx(w_, 0)
            G.gsis_set_distributions(ctx, f, I)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it, hist = G.gsis_solve(ctx, mode, mx, 1e-8)
            torch.cuda.synchronize()
            res[name] = {"iterations": it, "seconds": time.perf_counter() - t0, "final_eps": float(hist[-1]),
                         "converged": bool(hist[-1] < 1e-8)}
            G.gsis_destroy(ctx)
        geo = K.Geometry(wl.mesh)
        faces = MA.Faces(geo)
        fo, Io, F, h = f.copy(), I.copy(), None, []
        t0 = time.perf_counter()
        for k in range(20000):
            if oracle_mode == "cis" or k < wl.solver.n_cis_precond:
                fo, Io, e, F = OG.cis_step(fo, Io, wl, geo)
            else:
                fo, Io, e, F = OG.gsis_step(fo, Io, wl, geo, faces, F)
            h.append(e)
            if e < 1e-8 or time.perf_counter() - t0 > oracle_seconds:
                break
        res["oracle_" + oracle_mode] = {"iterations": len(h), "seconds": time.perf_counter() - t0,
                                        "final_eps": float(h[-1]), "converged": bool(h[-1] < 1e-8), "cores": 1}
        out["Kn%g" % kn] = res
    return out


def cylinder(precond=150, max_iter=12000):
    """Mach-5 flow past the cylinder (Kn_p = 1000, sigma_R = 0.1, the paper's first column
    of its cylinder table), 3 072 triangles, 48 x 48 velocities, order 1, FP32 with the
    mixed synthetic solve: outer iterations and seconds to eps < 1e-6 for CIS alone and
    for GSIS switched on after `precond` CIS iterations, from the uniform free stream.
    The paper starts from an Euler solution; from the impulsive start the wake first
    empties, so GSIS begins once CIS has filled it."""
    import torch
    import gsis_inputs as gi
    from paper_2601_03935_gb300 import gsis as G
    paper = {0.1: {"cis": 499, "gsis": 24}, 0.01: {"cis": 9582, "gsis": 25}}
    out = {}
    for kn in (0.1, 0.01):
        base = gi.workloads.cylinder(n_theta=64, n_radial=24, n_v=48, n_polar=4, n_azim=8, Mach=5.0, Kn=kn,
                                     Kn_p=1000.0, sigma_R=0.1)
        res = {"cells": base.mesh.n_cells, "n_xi": base.xi.shape[0], "paper_iterations": paper[kn]}
        for name, n0 in (("cis", max_iter), ("gsis", precond)):
            wl = gi.workloads.with_solver(base, precision="fp32", order=1, relax_block=16, max_inner=100,
                                          tol_inner=1e-7, n_cis_precond=n0, macro_fp32=2)
            M = gi.fields.uniform_fields(wl.mesh.n_cells)
            far = wl.mesh.patches[1]
            M[:, 0], M[:, 1], M[:, 4:8] = far.rho, far.u[0], far.T_t
            f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 2, wl.model.d_r, wl.model.d_v,
                                               wl.model.sigma_R, 0, noise=0.0)
            stream = torch.cuda.Stream()
            ctx = create_ctx(wl, stream.cuda_stream)
            G.gsis_set_distributions(ctx, f, I)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it, hist = G.gsis_solve(ctx, G.GSIS_MODE_GSIS, max_iter, 1e-6)
            torch.cuda.synchronize()
            res[name] = {"iterations": it, "seconds": time.perf_counter() - t0, "final_eps": float(hist[-1]),
                         "converged": bool(hist[-1] < 1e-6)}
            if name == "gsis":
                res[name]["cis_first"] = n0
            G.gsis_destroy(ctx)
        res["speedup_seconds"] = res["cis"]["seconds"] / res["gsis"]["seconds"]
        out["Kn%g" % kn] = res
    return out


def _smooth_state(wl, seed):
    """Smooth seeded fields (around the free stream where the workload has one) and their
    noisy multi-temperature equilibrium, FP32-rounded."""
    import gsis_inputs as gi
    far = [p for p in wl.mesh.patches if p.kind == 1]
    if far:
        M = gi.fields.smooth_random_fields(wl.mesh.cell_centroid / 8.0, seed, u_scale=0.5)
        M[:, 1] += far[0].u[0]
        M[:, 4:8] *= far[0].T_t
    else:
        M = gi.fields.smooth_random_fields(wl.mesh.cell_centroid, seed, u_scale=0.2)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, wl.dim, wl.model.d_r, wl.model.d_v, wl.model.sigma_R,
                                       seed + 1, noise=0.02)
    return f.astype(np.float32).astype(np.float64), I.astype(np.float32).astype(np.float64)


def field_errors(stream):
    """Per-field error of one FP32 CIS iteration (order 2, blocks of 16) against the FP64
    oracle from the same state, for the slab (all 64 cells), the 20 000-cell cavity and
    the 40 000-cell Mach-5 cylinder (whole relaxation blocks at the start, middle and end
    and next to the boundaries).  Densities and temperatures relative to their value,
    velocities to sqrt(T), heat fluxes to rho T^1.5, stresses to rho T."""
    import gsis_inputs as gi
    from oracle import kinetic as K
    from paper_2601_03935_gb300 import gsis as G
    cases = {"slab64": gi.workloads.slab(64), "cavity20000": gi.workloads.cavity(n_side=100),
             "cylinder40000": gi.workloads.cylinder()}
    out = {}
    for name, wl0 in cases.items():
        wl = gi.workloads.with_solver(wl0, precision="fp32", order=2, relax_block=16)
        f, I = _smooth_state(wl, 31)
        nc = wl.mesh.n_cells
        ctx = create_ctx(wl, stream.cuda_stream)
        try:
            G.gsis_set_distributions(ctx, f, I)
            G.gsis_step(ctx, G.GSIS_MODE_CIS)
            Fg = G.gsis_get_fields(ctx, nc)
        finally:
            G.gsis_destroy(ctx)
        if nc <= 64:
            cells = np.arange(nc)
        else:
            m = wl.mesh
            bnd = m.face_owner[m.face_nbr < 0]
            blocks = sorted({0, nc // 32, int(bnd[len(bnd) // 3]) // 16, int(bnd[-1]) // 16, (nc - 1) // 16})
            cells = np.concatenate([np.arange(b * 16, min(b * 16 + 16, nc)) for b in blocks])
        fo, Io = K.kinetic_sweep(f, I, wl, relax_block=16, cells=cells)
        Fo = K.fields_to_record(K.moments(fo, Io, wl.xi, wl.w, wl.omega, wl.wo, wl.dim, wl.model))
        g, r = Fg[cells], Fo
        rho, T = r[:, 0], r[:, 4]
        d = wl.dim
        err = {"rho": np.abs(g[:, 0] - rho).max() / np.abs(rho).max()}
        for k, c in (("T_t", 4), ("T_r", 5), ("T_v", 6), ("T_R", 7)):
            err[k] = float((np.abs(g[:, c] - r[:, c]) / np.abs(r[:, c])).max())
        err["u"] = float((np.abs(g[:, 1:1 + d] - r[:, 1:1 + d]) / np.sqrt(T)[:, None]).max())
        for k, c in (("q_t", 8), ("q_r", 11), ("q_v", 14), ("q_R", 17)):
            err[k] = float((np.abs(g[:, c:c + d] - r[:, c:c + d]) / (rho * T ** 1.5)[:, None]).max())
        err["sigma"] = float((np.abs(g[:, 20:24] - r[:, 20:24]) / (rho * T)[:, None]).max())
        out[name] = {"cells_compared": int(len(cells)), "n_cells": nc, "n_xi": int(wl.xi.shape[0]),
                     "max_error": {k: float(v) for k, v in err.items()}}
    return out


def _stagnation_state(base):
    """Uniform gas at rest at the free stream's density and stagnation temperature
    T_0 = T_inf + (gamma - 1) / (2 gamma) |u_inf|^2: a hot state that the velocity grid
    (sized by T_0) resolves, unlike the cold free stream."""
    import gsis_inputs as gi
    far = base.mesh.patches[1]
    m = base.model
    gamma = (5.0 + m.d_r + m.d_v) / (3.0 + m.d_r + m.d_v)
    T0 = far.T_t + (gamma - 1.0) / (2.0 * gamma) * float(np.dot(far.u, far.u))
    return gi.fields.uniform_fields(base.mesh.n_cells, rho=far.rho, T=T0)


def _full_size_leg(stream, base, bytes_per_update, plan):
    """Throughput of one full-size case, FP32, blocks of 16, for each (label, order,
    fields, warmup, steps, limiter constant K, mode, positivity bound theta) of ``plan``
    (mode "cis", or "gsis": GSIS iterations with the mixed synthetic schedule):
    the state is set on the device (gsis_init_fields), then warmup and timed iterations.
    Reports updates/s and the gas sweep's fraction of HBM bandwidth per entry.  One
    context is alive at a time."""
    import torch
    import gsis_inputs as gi
    from paper_2601_03935_gb300 import gsis as G
    nc, V = base.mesh.n_cells, base.xi.shape[0]
    peak, kind = measured_peaks()
    out = {}
    for label, order, M, warmup, steps, K, how, theta in plan:
        mode = G.GSIS_MODE_GSIS if how == "gsis" else G.GSIS_MODE_CIS
        wl = gi.workloads.with_solver(base, precision="fp32", order=order, relax_block=16, venkat_K=K,
                                      macro_fp32=2 if how == "gsis" else 0, positivity=theta)
        ctx = create_ctx(wl, stream.cuda_stream)
        entry = {"order": order, "positivity": theta}
        try:
            G.gsis_init_fields(ctx, M)
            for _ in range(warmup):
                G.gsis_step_async(ctx, mode)
            G.gsis_last_eps(ctx)
            if how != "gsis":           # (profiling brackets would split the synthetic solve's graphs)
                G.gsis_profile_enable(ctx, True)
                G.gsis_profile_reset(ctx)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                G.gsis_step_async(ctx, mode)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            prof = G.gsis_profile_read(ctx)
            entry["last_eps"] = G.gsis_last_eps(ctx)
        except G.GsisError as e:
            out[label] = {"order": order, "note": "not timed: %s" % e}
            continue
        finally:
            G.gsis_destroy(ctx)
        if how == "gsis":
            entry.update({"mode": "GSIS, FP32 distributions, mixed synthetic schedule, 100 inner iterations",
                          "warmup": warmup, "steps": steps, "ms_per_gsis_iteration": ms,
                          "value": nc * V / (ms * 1e-3), "unit": UNIT})
            out[label] = entry
            continue
        names = ("slopes_gas", "sweep_gas") if order == 2 else ("sweep_gas",)
        sweep = sum(prof[k][0] / max(prof[k][1], 1) for k in names)
        alg = nc * V * bytes_per_update
        entry.update({"warmup": warmup, "steps": steps, "value": nc * V / (ms * 1e-3), "unit": UNIT,
                      "ms_per_step": ms,
                      "kernels": {k: {"ms_per_launch": v[0] / v[1], "launches": v[1]} for k, v in prof.items() if v[1]},
                      "roofline": {"kernel": "+".join(names), "bound": "hbm", "achieved": alg / (sweep * 1e-3) / 1e9,
                                   "peak": peak, "unit": "GB/s", "frac": alg / (sweep * 1e-3) / 1e9 / peak,
                                   "peak_kind": kind, "algorithmic_bytes_per_launch": alg, "ms_per_launch": sweep}})
        out[label] = entry
    return out


ORDER2_NOTE = ("order 2 from the impulsive free-stream start runs with the positivity bound of the "
               "implicit update (theta = 0.1: every value of f and I at least 0.1 times its previous "
               "value; steady states unchanged); without it the order-2 defect correction drives f "
               "negative at the body within a few iterations (oracle and GPU alike)")


def full_cylinder_throughput(stream):
    """The full-size Mach-5 cylinder (40 000 triangles, 48 x 48 velocities, 96 directions):
    32 B per update (four planes read and written once)."""
    import gsis_inputs as gi
    base = gi.workloads.cylinder()
    far = base.mesh.patches[1]
    free = gi.fields.uniform_fields(base.mesh.n_cells, rho=far.rho, u=far.u, T=far.T_t)
    plan = [("order2_free_stream", 2, free, 3, 10, 0.01, "cis", 0.1),
            ("order1_free_stream", 1, free, 3, 10, 0.01, "cis", 0.0)]
    return {"workload": "cylinder 2-D Mach 5, %d triangles, 48x48 velocities (%d), %d photon directions, FP32"
                        % (base.mesh.n_cells, base.xi.shape[0], base.omega.shape[0]),
            "note": ORDER2_NOTE, **_full_size_leg(stream, base, 32, plan)}


def capsule_throughput(stream):
    """The full-size 3-D sphere-cone capsule (193 009 tetrahedra, 24^3 = 13 824 velocities, 128
    directions, CUDA-core moments): 24 B per update (f0, f1, f2 read and written once;
    the fourth plane of the layout is zero in 3-D and counts as waste, not work)."""
    import gsis_inputs as gi
    base = gi.workloads.capsule()
    far = base.mesh.patches[1]
    free = gi.fields.uniform_fields(base.mesh.n_cells, rho=far.rho, u=far.u, T=far.T_t)
    plan = [("order2_free_stream", 2, free, 3, 5, 0.01, "cis", 0.1),
            ("order1_free_stream", 1, free, 3, 5, 0.01, "cis", 0.0),
            ("gsis_order1_stagnation_start", 1, _stagnation_state(base), 1, 2, 0.01, "gsis", 0.0)]
    return {"workload": "capsule 3-D Mach 10, %d tetrahedra, 24^3 velocities (%d), %d photon directions, FP32"
                        % (base.mesh.n_cells, base.xi.shape[0], base.omega.shape[0]),
            "note": ORDER2_NOTE, **_full_size_leg(stream, base, 24, plan)}


def capsule_probe(args):
    """A small 3-D capsule run for profiling: box of n^3 hexahedra (6 n^3 tetrahedra less the
    body), nv^3 velocities, 8 x 16 directions, FP32, order 2, from the stagnation state;
    --steps CIS iterations, then the per-kernel times of the library's own events."""
    import gsis_inputs as gi
    n, nv = (int(x) for x in args.capsule_probe.split(","))
    wl = gi.workloads.with_solver(gi.workloads.capsule(n=n, n_v=nv), precision="fp32", order=2, relax_block=16)
    return _probe(args, "capsule", wl, _stagnation_state(wl))


def cylinder_probe(args):
    """A smaller Mach-5 cylinder for profiling: the full case's O-grid with n_theta x n_radial
    quadrilaterals split into triangles, its 48 x 48 velocities and 96 directions, FP32, order
    2 with the positivity bound (theta = 0.1, limiter constant 0.01) from the free stream, as
    the full-size leg runs it; --steps CIS iterations."""
    import gsis_inputs as gi
    nt, nr = (int(x) for x in args.cylinder_probe.split(","))
    base = gi.workloads.cylinder(n_theta=nt, n_radial=nr)
    far = base.mesh.patches[1]
    wl = gi.workloads.with_solver(base, precision="fp32", order=2, relax_block=16, venkat_K=0.01, positivity=0.1)
    return _probe(args, "cylinder", wl, gi.fields.uniform_fields(base.mesh.n_cells, rho=far.rho, u=far.u, T=far.T_t))


def _probe(args, name, wl, M):
    from paper_2601_03935_gb300 import build
    from paper_2601_03935_gb300 import gsis as G
    build.build()
    G.load()
    ctx = create_ctx(wl, 0)
    try:
        G.gsis_init_fields(ctx, M)
        G.gsis_profile_enable(ctx, True)
        for _ in range(args.steps):
            G.gsis_step_async(ctx, G.GSIS_MODE_CIS)
        eps = G.gsis_last_eps(ctx)
        prof = G.gsis_profile_read(ctx)
    finally:
        G.gsis_destroy(ctx)
    print(json.dumps({"probe": name, "n_cells": wl.mesh.n_cells, "n_xi": int(wl.xi.shape[0]), "last_eps": eps,
                      "ms_per_launch": {k: v[0] / v[1] for k, v in prof.items() if v[1]}}))
    return 0


def run_sharded(args, dist, rank, local, world):
    """One problem cut into velocity shards, one per rank; NCCL sums the exchange buffers."""
    import torch
    from paper_2601_03935_gb300 import gsis as G
    from paper_2601_03935_gb300 import shard as SH
    wl = workload(args)
    nc, V, NO = wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0]
    stream = torch.cuda.Stream()
    sh = SH.VelocityShard(wl.mesh, wl.xi, wl.w, wl.omega, wl.wo, wl.model, wl.solver, rank, world, stream.cuda_stream)
    shards = [sh]
    f, I = initial_state(wl)
    sh.set_distributions(f, I)
    SH.refresh(shards, stream=stream)
    mode = G.GSIS_MODE_CIS if args.mode == "cis" else G.GSIS_MODE_GSIS
    for _ in range(args.warmup):
        SH.step(shards, mode, stream=stream)
    G.gsis_profile_enable(sh.ctx, True)
    G.gsis_profile_reset(sh.ctx)
    launches0 = G.gsis_launch_count(sh.ctx)
    dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            eps = SH.step(shards, mode, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
    dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    launches = G.gsis_launch_count(sh.ctx) - launches0
    prof = G.gsis_profile_read(sh.ctx)
    G.gsis_profile_enable(sh.ctx, False)
    t = torch.tensor([ms], device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    # end to end: this rank's slice uploaded from pinned host memory, the refresh (two
    # exchanges), the iteration, the fields read back
    rs = 4 if args.precision == "fp32" else 8
    f32 = np.float32 if args.precision == "fp32" else np.float64
    hf = torch.from_numpy(np.ascontiguousarray(f[:, sh.lo:sh.hi]).astype(f32)).pin_memory()
    hI = torch.from_numpy(np.ascontiguousarray(I[:, sh.olo:sh.ohi]).astype(f32)).pin_memory()
    hout = torch.empty((nc, G.GSIS_NF), dtype=torch.float64).pin_memory()
    e2e_steps = max(3, args.steps // 4)

    def e2e_step():
        G.gsis_upload_distributions(sh.ctx, hf.data_ptr(), hI.data_ptr())
        SH.refresh(shards, stream=stream)
        SH.step(shards, mode, stream=stream)
        G.gsis_download_fields_async(sh.ctx, hout.data_ptr(), nc)
        stream.synchronize()

    e2e_step()
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    t = torch.tensor([e2e_s], device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e2e_s = float(t.item())
    sh.destroy()
    if rank != 0:
        return 0
    sweep_names = ["slopes_gas", "sweep_gas"] if args.order == 2 else ["sweep_gas"]
    avg_sweep = sum(prof[k][0] / max(prof[k][1], 1) for k in sweep_names)
    alg_bytes = nc * (sh.hi - sh.lo) * 4 * rs * 2
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (avg_sweep * 1e-3) / 1e9
    cfg = config(args, wl)
    cfg["parallelism"] = "velocity-sharded x%d (NCCL all-reduce of per-cell moment sums per iteration)" % world
    line = {
        "metric": METRIC, "value": nc * V / (ms * 1e-3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
        "data": "synthetic (seeded cavity mesh and near-equilibrium distributions)", "config": cfg,
        "roofline": {"kernel": "+".join(sweep_names) + " (rank 0's velocity shard)", "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "traffic": None, "algorithmic_bytes_per_launch": alg_bytes,
                     "ms_per_launch": avg_sweep},
        "e2e": {"value": nc * V / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": nc * ((sh.hi - sh.lo) * 4 + (sh.ohi - sh.olo)) * rs * world,
                "d2h_bytes_per_step": nc * G.GSIS_NF * 8 * world},
        "gpu_launches": launches, "clocks": clk.summary(), "last_eps": eps,
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch
    from paper_2601_03935_gb300 import build
    from paper_2601_03935_gb300 import gsis as G

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        build.build()
    if dist is not None:
        dist.barrier()
    G.load()
    if dist is not None:
        try:
            return run_sharded(args, dist, rank, local, world)
        finally:
            dist.destroy_process_group()
    wl = workload(args)
    nc, V, NO = wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0]
    stream = torch.cuda.Stream()
    ctx = create_ctx(wl, stream.cuda_stream)
    f, I = initial_state(wl)
    G.gsis_set_distributions(ctx, f, I)
    mode = G.GSIS_MODE_CIS if args.mode == "cis" else G.GSIS_MODE_GSIS

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---- device-resident throughput
    for _ in range(args.warmup):
        G.gsis_step_async(ctx, mode)
    G.gsis_last_eps(ctx)
    G.gsis_profile_enable(ctx, True)
    G.gsis_profile_reset(ctx)
    launches0 = G.gsis_launch_count(ctx)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            G.gsis_step_async(ctx, mode)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    launches = G.gsis_launch_count(ctx) - launches0
    prof = G.gsis_profile_read(ctx)
    G.gsis_profile_enable(ctx, False)
    eps = G.gsis_last_eps(ctx)
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    # ---- end to end through the C ABI with host buffers
    f32 = np.float32 if args.precision == "fp32" else np.float64
    hf = torch.from_numpy(f.astype(f32)).pin_memory()
    hI = torch.from_numpy(I.astype(f32)).pin_memory()
    hout = torch.empty((nc, G.GSIS_NF), dtype=torch.float64).pin_memory()
    e2e_steps = max(3, args.steps // 4)

    # Every step uploads a full state from pinned host memory and reads the step's fields
    # back.  The upload of step k + 1 is staged on the context's copy stream while step k
    # computes (gsis_stage_distributions / gsis_commit_staged), so copy and compute overlap.
    def e2e_step():
        G.gsis_commit_staged(ctx)
        G.gsis_stage_distributions(ctx, hf.data_ptr(), hI.data_ptr())
        G.gsis_step_async(ctx, mode)
        G.gsis_download_fields_async(ctx, hout.data_ptr(), nc)
        stream.synchronize()

    G.gsis_stage_distributions(ctx, hf.data_ptr(), hI.data_ptr())
    for _ in range(2):
        e2e_step()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()                  # the last staged copy is inside the timed region
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    G.gsis_commit_staged(ctx)
    if dist is not None:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())

    # ---- the standalone moment pass (Eq. getmoment): in FP32 with tc_moments >= 1 the gas
    # moments are one split-TF32 tcgen05 contraction per (16-cell tile, 64 velocities)
    G.gsis_profile_enable(ctx, True)
    G.gsis_profile_reset(ctx)
    for _ in range(5):
        G.gsis_refresh_fields(ctx)
    torch.cuda.synchronize()
    mprof = G.gsis_profile_read(ctx)
    G.gsis_profile_enable(ctx, False)
    G.gsis_destroy(ctx)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    # the gas sweep of one iteration is the slope pass (order 2) plus the sweep proper
    sweep_names = ["slopes_gas", "sweep_gas"] if args.order == 2 else ["sweep_gas"]
    avg_sweep = sum(prof[k][0] / max(prof[k][1], 1) for k in sweep_names)
    rs = 4 if args.precision == "fp32" else 8
    alg_bytes = nc * V * 4 * rs * 2                     # read and write the four planes once
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (avg_sweep * 1e-3) / 1e9
    # moment pass: read f and I once, write the per-(cell, chunk) partials
    Vp, Op = -(-V // 64) * 64, -(-NO // 64) * 64
    m_bytes = nc * V * 4 * rs + nc * NO * rs + nc * (Vp // 64) * 20 * rs + nc * (Op // 64) * 4 * rs
    m_ms = mprof["moments_only"][0] / max(mprof["moments_only"][1], 1)
    tc_on = args.precision == "fp32" and args.tc_moments >= 1
    value = world * nc * V / (ms * 1e-3)
    traffic, traffic_note = sweep_traffic(args.precision, args.order)
    kernels = {k: {"ms_per_launch": (v[0] / v[1]) if v[1] else None, "launches": v[1],
                   "share": v[0] / max(sum(x[0] for x in prof.values()), 1e-30)} for k, v in prof.items() if v[1]}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
        "data": "synthetic (seeded cavity mesh and near-equilibrium distributions)",
        "config": config(args, wl),
        "roofline": {"kernel": "+".join(sweep_names), "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                     "traffic": traffic, "traffic_note": traffic_note,
                     "algorithmic_bytes_per_launch": alg_bytes, "ms_per_launch": avg_sweep},
        "e2e": {"value": world * nc * V / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": nc * (V * 4 + NO) * rs, "d2h_bytes_per_step": nc * G.GSIS_NF * 8},
        "gpu_launches": launches, "clocks": clk.summary(), "kernels": kernels,
        "kernels_note": "CUDA-event time per launch on the stream the kernel runs on, over the timed region; "
                        "the photon slope pass and sweep run on a side stream concurrently with the gas kernels, "
                        "so their brackets include the wait for free SMs",
        "last_eps": eps,
        "moment_pass": {"kernel": ("k_moments_gas_tc (tcgen05, split TF32)" if tc_on else "k_moments_gas (CUDA cores)")
                        + " + k_moments_photon", "bound": "hbm", "ms_per_launch": m_ms,
                        "algorithmic_bytes_per_launch": m_bytes, "achieved": m_bytes / (m_ms * 1e-3) / 1e9,
                        "peak": peak, "unit": "GB/s", "frac": m_bytes / (m_ms * 1e-3) / 1e9 / peak},
    }
    if not args.no_tts:
        line["time_to_steady"] = time_to_steady(stream)
    if not args.no_tts:
        line["slab_time_to_steady"] = slab_time_to_steady()
    if not args.no_tts:
        line["time_to_steady_20k"] = time_to_steady_full(stream)
        line["time_to_steady_capsule"] = time_to_steady_capsule(stream)
    if not args.no_shock:
        line["normal_shock"] = normal_shock()
    if not args.no_cylinder:
        line["cylinder"] = cylinder()
    if not args.no_full_cylinder:
        line["cylinder_full"] = full_cylinder_throughput(stream)
    if not args.no_capsule:
        line["capsule_3d"] = capsule_throughput(stream)
    if not args.no_field_errors:
        line["field_errors"] = field_errors(stream)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, seconds=args.cpu_seconds)
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--order", type=int, default=2)
    ap.add_argument("--block", type=int, default=16)
    ap.add_argument("--mode", default="cis", choices=["cis", "gsis"],
                    help="outer iteration timed: cis (the kinetic sweep and moments) or gsis (adds the synthetic "
                         "solve and the synchronisation pass)")
    ap.add_argument("--tc-moments", type=int, default=1, choices=[0, 1, 2],
                    help="FP32 gas moments: 0 CUDA cores, 1 tensor cores in the standalone and sync passes, "
                         "2 also in the sweep epilogue")
    ap.add_argument("--kn", type=float, default=0.01)
    ap.add_argument("--kn-p", type=float, default=10.0)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tts", action="store_true", help="skip the time-to-steady measurement")
    ap.add_argument("--no-shock", action="store_true", help="skip the normal-shock convergence measurement")
    ap.add_argument("--no-cylinder", action="store_true", help="skip the Mach-5 cylinder CIS/GSIS measurement")
    ap.add_argument("--capsule-probe", default=None, metavar="N,NV",
                    help="only run a small 3-D capsule case (N^3 hexahedra, NV^3 velocities) for profiling")
    ap.add_argument("--cylinder-probe", default=None, metavar="NT,NR",
                    help="only run a smaller Mach-5 cylinder (NT x NR O-grid, 2 NT NR triangles) for profiling")
    ap.add_argument("--handover", action="store_true",
                    help="only run the Kn = 0.1 cavity time to steady with the FP32 -> FP64 hand-over")
    ap.add_argument("--no-capsule", action="store_true",
                    help="skip the full-size 3-D capsule (tetrahedra) throughput leg")
    ap.add_argument("--no-full-cylinder", action="store_true",
                    help="skip the throughput of the full-size (40 000-cell, 2304-velocity) cylinder")
    ap.add_argument("--no-field-errors", action="store_true",
                    help="skip the per-field error of one FP32 iteration against the FP64 oracle")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.capsule_probe:
        return capsule_probe(args)
    if args.cylinder_probe:
        return cylinder_probe(args)
    if args.handover:
        return time_to_steady_handover(args)
    return run_reference(args) if args.impl == "reference" else run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
