"""Benchmark of the coupled Yee / molecular-ensemble step on GB300.

Headline workload (one step = the whole hot path: molecule window gather + density-
matrix step + current scatter + fused H/E pass with CPML, material map and source +
DFT flux planes): the Bragg-resonator ensemble, 512 x 512 x 384 cells with 10-cell CPML
on every face, a 12-layer quarter-wave stack (eps 2.25 / 1, 4 / 6 cells) along x split
around a 32-cell central slab holding 100,000 multilevel Lindblad systems (2..8 levels,
RK4; Hermitian z-dipoles with N(0, 0.01) entries, ladders 0.2 +- 5 %, decay rates
log-uniform in [1e-6, 1e-4], sigma = 1.5 cells), a z-polarised Gaussian-pulse sheet and
two 8-frequency flux planes; 8000 steps.  FP32 fields and molecules, FP64 DFT and
energy accumulators.  Synthetic, seeded inputs standing in for the Bragg resonator of
Sec. IV.C.  The other workloads (the 256^3 superradiant slab, the adjoint, batches,
dispersive media, energy transfer, cavity, laser drive) are sections of the same line.

  python bench.py [--gpus N --steps K --warmup W]      our CUDA path (C ABI)
  python bench.py --impl reference ...                  the FP64 CPU oracle

Under torchrun each rank advances an independent replica (seed offset by rank);
there is no data-path collective.  Rank 0 prints one JSON line.
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

METRIC = "coupled Yee Gcell-updates/s"
UNIT = "Gcell-updates/s"


def headline_problem(args, rank: int = 0):
    from paper_2512_06173_gb300 import workloads
    nx, ny, nz = args.bragg_shape
    return workloads.bragg_ensemble(nx=nx, ny=ny, nz=nz, nmol=args.bragg_nmol, seed=3 + rank)


def workload_text(prob) -> str:
    return (f"Bragg-resonator ensemble: {prob.nx}x{prob.ny}x{prob.nz} cells, 10-cell CPML on all faces, "
            f"12 quarter-wave layers (eps 2.25 / 1, 4 / 6 cells) along x around a 32-cell central slab, "
            f"{prob.molecules.count} multilevel Lindblad systems (2-8 levels, RK4; z-dipoles N(0,0.01), "
            f"ladders 0.2+-5%, decay log-U[1e-6,1e-4], sigma 1.5) in the slab, z-polarised Gaussian-pulse "
            f"sheet, 2 flux planes x 8 frequencies")


def config_of(prob, world: int) -> dict:
    level_gb = 6 * prob.cells * 4 / 1e9
    return {"workload": workload_text(prob), "cells": prob.cells, "molecules": prob.molecules.count,
            "grid": [prob.nx, prob.ny, prob.nz],
            "l2": f"inputs larger than L2 (fields {level_gb:.2f} GB per time level)",
            "parallelism": "replicas" if world > 1 else "single"}


# DRAM bytes (read + write) per field-pass launch, from one ncu capture of
# `yee_kernel` (dram__bytes_read.sum + dram__bytes_write.sum, --clock-control none) on
# the named workload; valid only for the source it was measured on, identified by the
# sha256 prefix of yee.cu.
FIELD_PASS_TRAFFIC = {
    ("bragg-512x512x384-100000ml", "6053a25796039c2f"): 6.2251e9,
    ("superradiant-slab-256^3-10000tls", "6053a25796039c2f"): 1.0410e9,
}


def field_pass_traffic(prob):
    import hashlib
    src = os.path.join(ROOT, "paper_2512_06173_gb300", "csrc", "yee.cu")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return FIELD_PASS_TRAFFIC.get((prob.name, h))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def field_pass_bytes(prob, esz: int) -> float:
    """Algorithmic bytes of one launch of the fused field pass: E and H read and
    written once (12 esz per cell), four CPML memory variables read and written per
    cell and layer axis (8 esz), 1 B material index per cell if present, esz per
    design-box cell, 6 esz per pole of a cell (its current J read and written) and 6
    esz more per Lorentz pole (its polarisation P).  Halo re-reads are not credited."""
    import numpy as np
    N = prob.cells
    b = 12 * esz * N
    dims = (prob.nx, prob.ny, prob.nz)
    for a in range(3):
        th = prob.pml[2 * a] + prob.pml[2 * a + 1]
        b += 8 * esz * th * (N // dims[a])
    if prob.mat is not None:
        b += N
        per = np.array([6 * esz * sum(1 + (w0 > 0) for _, _, w0 in m.poles()) for m in prob.materials])
        if per.any():
            b += int(per[np.asarray(prob.mat)].sum())
    if prob.design_box is not None:
        x0, y0, z0, sx, sy, sz = prob.design_box
        b += esz * sx * sy * sz
    return float(b)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms in the background."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        loaded = [r for r in rows if r[9].isdigit() and int(r[9]) > 50] or rows
        sm = [float(r[1]) for r in loaded if r[1].replace(".", "").isdigit()]
        reasons = sorted({names[q] for r in loaded for q in range(4) if r[5 + q].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "reasons": reasons, "samples": len(rows), "samples_under_load": len(loaded),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(world, x: float) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(world, x: float) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def cpu_oracle_run(prob, budget_s: float, max_steps: int, warm: int = 1):
    """Time the FP64 oracle as it stands on this host's cores on the same workload:
    `warm` untimed steps, then as many full steps as fit in about `budget_s` seconds
    (at least 2, at most max_steps).  Building the oracle's arrays is not timed."""
    import oracle
    sim = oracle.OracleSim(prob)
    t0 = time.perf_counter()
    sim.step(max(warm, 1))
    t_one = (time.perf_counter() - t0) / max(warm, 1)
    n = max(2, min(max_steps, int(budget_s / max(t_one, 1e-6))))
    t0 = time.perf_counter()
    sim.step(n)
    dt = time.perf_counter() - t0
    del sim
    return n, dt, oracle.threads()


def run_reference(args, world, rank):
    """Reference arm: the FP64 CPU oracle, rank 0 only, on the headline workload: W
    warm-up steps, then a bounded sample of full steps (about args.ref_budget seconds)."""
    if rank != 0:
        return
    prob = headline_problem(args, 0)
    n, dt, cores = cpu_oracle_run(prob, budget_s=args.ref_budget, max_steps=args.steps, warm=args.warmup)
    value = prob.cells * n / dt / 1e9
    sample = (f"{n} full steps (after {args.warmup} warm-up steps) of the {prob.nx}x{prob.ny}x{prob.nz} "
              f"workload with all {prob.molecules.count} systems, FP64, oracle as it stands")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": n, "warmup": args.warmup, "ms_per_step": dt / n * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(prob, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def adjoint_case(prob, S, K, stream):
    """Forward and adjoint wall time of one inverse-design problem: `reverse_ms` is the
    adjoint call minus a plain forward run of the same S steps (the checkpointed
    recompute plus the reversed steps), checkpoints every K steps."""
    import torch
    from paper_2512_06173_gb300 import maxlink

    sh = stream.cuda_stream
    g = maxlink.Grid(prob, maxlink.ML_F32, stream=sh)
    try:
        state0 = g.checkpoint()
        sx, sy, sz = prob.design_box[3:]
        ge = torch.zeros(sx * sy * sz, dtype=torch.float64, device="cuda")
        gg = torch.zeros(prob.molecules.count, dtype=torch.float64, device="cuda")
        # warm-up of both paths (module load, first allocations)
        g.step(20)
        g.sync()
        g.restore(state0)
        maxlink.ml_adjoint_run(g.h, 40, 20, 0, 0, ge.data_ptr(), gg.data_ptr(), True, sh)
        g.restore(state0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.step(S)
        g.sync()
        fwd = time.perf_counter() - t0
        fwd_flux = float(g.flux(0)[0])
        g.restore(state0)
        torch.cuda.synchronize()
        l0 = maxlink.ml_launch_count(g.h)
        t0 = time.perf_counter()
        obj = maxlink.ml_adjoint_run(g.h, S, K, 0, 0, ge.data_ptr(), gg.data_ptr(), True, sh)
        adj = time.perf_counter() - t0
        launches = maxlink.ml_launch_count(g.h) - l0
        return {"workload": prob.name, "steps": S, "ckpt_every": K, "dtype": "f32 fields, f64 gradient sums",
                "forward_ms": fwd * 1e3, "adjoint_call_ms": adj * 1e3, "reverse_ms": (adj - fwd) * 1e3,
                "ratio_reverse_to_forward": (adj - fwd) / fwd, "gpu_launches": int(launches),
                "objective": obj, "forward_flux_check": fwd_flux,
                "grad_eps_l2": float(torch.linalg.norm(ge)), "grad_gamma_l2": float(torch.linalg.norm(gg))}
    finally:
        g.close()


def measure_adjoint(args, stream):
    """The inverse-design workload (192^3 vacuum with CPML, 96^3 design box, 2000
    two-level emitters, 3000 steps, checkpoints every 100 steps), and the same problem
    with every part of the step the adjoint takes: emitters replaced by RK4 GKSL systems
    of 2..8 levels, a Lorentz layer and a Drude + Lorentz film behind the design box."""
    from paper_2512_06173_gb300 import workloads

    out = adjoint_case(workloads.adjoint_design(), args.adj_steps, 100, stream)
    out["full_step"] = adjoint_case(workloads.adjoint_design(multilevel=True, media=True), args.adj_steps, 100,
                                    stream)
    return out


def measure_bragg(args, stream):
    """Bragg-resonator ensemble: 512x512x384 cells, 12-layer stack, 100,000 multilevel
    Lindblad systems (2-8 levels, RK4), z-polarised pulse, FP32 fields; device time of
    args.bragg_steps steps after a warm-up, per-kernel split from the tracing events."""
    import torch
    from paper_2512_06173_gb300 import maxlink, workloads

    nx, ny, nz = args.bragg_shape
    prob = workloads.bragg_ensemble(nx=nx, ny=ny, nz=nz, nmol=args.bragg_nmol)
    sh = stream.cuda_stream
    g = maxlink.Grid(prob, maxlink.ML_F32, stream=sh)
    K = args.bragg_steps
    try:
        g.step(5)
        g.sync()
        # untraced: the launch chain overlaps as it does for a user
        u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        u0.record(stream)
        g.step(K)
        u1.record(stream)
        stream.synchronize()
        g.sync()
        ms_untraced = u0.elapsed_time(u1)
        maxlink.ml_set_timing(g.h, True)
        maxlink.ml_timing(g.h)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.step(K)
        e1.record(stream)
        stream.synchronize()
        g.sync()
        ms = e0.elapsed_time(e1)
        kms, _ = maxlink.ml_timing(g.h)
        maxlink.ml_set_timing(g.h, False)
        hbm, peak_kind = peaks()
        fp = kms[1] / K
        alg = field_pass_bytes(prob, 4)
        return {"workload": prob.name, "cells": prob.cells, "molecules": prob.molecules.count, "steps": K,
                "dtype": "f32", "gcells_per_s": prob.cells * K / ms / 1e6,
                "molecule_steps_per_s": prob.molecules.count * K / ms * 1e3, "ms_per_step_traced": ms / K,
                "ms_per_step": ms_untraced / K, "gcells_per_s_untraced": prob.cells * K / ms_untraced / 1e6,
                "field_pass": {"ms_per_step": fp, "alg_bytes": alg, "achieved_gbs": alg / (fp / 1e3) / 1e9,
                               "frac": alg / (fp / 1e3) / 1e9 / hbm, "peak": hbm, "peak_kind": peak_kind},
                "kernel_ms_per_step": {"gather": kms[5] / K, "molecules": kms[0] / K, "current": kms[4] / K,
                                       "field_pass": fp, "plane_fold": kms[3] / K}}
    finally:
        g.close()


def measure_dispersive(args, stream):
    """Dispersive stack: 512x512x256 cells periodic in x and y, a 32-cell Lorentz layer
    on an 8-cell Drude film, 20,000 two-level emitters in the Lorentz layer, FP32;
    device time of args.dispersive_steps steps after a warm-up, per-kernel split from
    the tracing events; the field pass's algorithmic bytes include the pole current and
    polarisation of every pole cell."""
    import torch
    from paper_2512_06173_gb300 import maxlink, workloads

    prob = workloads.dispersive_stack()
    sh = stream.cuda_stream
    g = maxlink.Grid(prob, maxlink.ML_F32, stream=sh)
    K = args.dispersive_steps
    try:
        g.step(5)
        g.sync()
        maxlink.ml_set_timing(g.h, True)
        maxlink.ml_timing(g.h)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.step(K)
        e1.record(stream)
        stream.synchronize()
        g.sync()
        ms = e0.elapsed_time(e1)
        kms, _ = maxlink.ml_timing(g.h)
        maxlink.ml_set_timing(g.h, False)
        hbm, peak_kind = peaks()
        fp = kms[1] / K
        alg = field_pass_bytes(prob, 4)
        pe = g.molecules(maxlink.ML_MOL_POP)[:, 1]
        return {"workload": prob.name, "cells": prob.cells, "molecules": prob.molecules.count, "steps": K,
                "dtype": "f32", "gcells_per_s": prob.cells * K / ms / 1e6,
                "molecule_steps_per_s": prob.molecules.count * K / ms * 1e3, "ms_per_step": ms / K,
                "field_pass": {"ms_per_step": fp, "alg_bytes": alg, "achieved_gbs": alg / (fp / 1e3) / 1e9,
                               "frac": alg / (fp / 1e3) / 1e9 / hbm, "peak": hbm, "peak_kind": peak_kind},
                "kernel_ms_per_step": {"molecules": kms[0] / K, "current": kms[4] / K, "field_pass": fp,
                                       "plane_fold": kms[3] / K},
                "pe_max": float(pe.max()), "flux_far_f3": float(g.flux(1)[3])}
    finally:
        g.close()


def measure_cavity(args, stream):
    """Single-mode cavity (Sec. II normal-mode solver, single-mode limit): 1,000,000
    two-level emitters resonant with the mode, in-plane dipoles, collective splitting
    about 5% of the mode frequency; FP32 molecules, FP64 mode.  Device time of
    args.cavity_steps steps after 20 warm-up steps.  Roofline: the algorithmic bytes per
    molecule-step (rho read + written 64 B, H0 32 B, mu_x and mu_y 64 B, gamma 4 B, the
    energy sum read + written 16 B, the field and dipole rate written 24 B: 204 B) over
    the step time."""
    import numpy as np
    import torch
    from paper_2512_06173_gb300 import maxlink, workloads

    M = args.cavity_molecules
    mols = workloads.cavity_ensemble(M)
    eps = 0.05 * 0.25 ** 2 / np.sqrt(2 * 0.25 * M * 0.05 ** 2 / 2)
    sh = stream.cuda_stream
    c = maxlink.Cavity(mols, 0.25, eps, 0.5, precision=maxlink.ML_F32, stream=sh)
    K = args.cavity_steps
    try:
        c.step(20)
        c.mode()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.step(K)
        e1.record(stream)
        stream.synchronize()
        mode = c.mode()
        ms = e0.elapsed_time(e1)
        hbm, peak_kind = peaks()
        alg = 204.0 * M
        gbs = alg / (ms / K / 1e3) / 1e9
        return {"workload": f"single-mode cavity, {M} two-level emitters, eps={eps:.3g}", "molecules": M, "steps": K,
                "dtype": "f32 molecules, f64 mode", "ms_per_step": ms / K,
                "molecule_steps_per_s": M * K / ms * 1e3, "launches_per_step": 1,
                "roofline": {"bound": "hbm", "alg_bytes_per_step": alg, "achieved_gbs": gbs, "peak": hbm,
                             "peak_kind": peak_kind, "frac": gbs / hbm},
                "mode_after": [float(x) for x in mode]}
    finally:
        c.close()


def measure_laser(args, stream):
    """Laser-driven molecules (classical path, Eq. E_analytical): 4,000,000 two-level
    emitters (the single-mode cavity workload's emitters) spread over z in [0, 1000),
    a resonant pulse of half width 200 crossing them; FP32.  One launch per step.
    Roofline: algorithmic bytes per molecule-step (rho read + written 64 B, H0 32 B,
    mu_x and mu_y 64 B, gamma 4 B, z 8 B, the energy sum read + written 16 B, the field
    and dipole rate written 24 B: 212 B) over the step time."""
    import numpy as np
    import torch
    from paper_2512_06173_gb300 import maxlink, workloads

    M = args.laser_molecules
    mols = workloads.cavity_ensemble(M)
    mols.pos[:, 2] = np.random.default_rng(7).uniform(0.0, 1000.0, M)
    sh = stream.cuda_stream
    d = maxlink.Drive(mols, 1e-3, 0.25, 0.0, -200.0, 200.0, (1.0, 0.0, 0.0), 0.5, precision=maxlink.ML_F32, stream=sh)
    K = args.laser_steps
    try:
        d.step(64)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d.step(K)
        e1.record(stream)
        stream.synchronize()
        pe = d.molecules(maxlink.ML_MOL_POP)[:, 1]
        ms = e0.elapsed_time(e1)
        hbm, peak_kind = peaks()
        alg = 212.0 * M
        gbs = alg / (ms / K / 1e3) / 1e9
        return {"workload": f"laser-driven, {M} two-level emitters, z in [0, 1000), resonant cos^2 pulse",
                "molecules": M, "steps": K, "dtype": "f32", "ms_per_step": ms / K,
                "molecule_steps_per_s": M * K / ms * 1e3, "launches_per_step": 1,
                "roofline": {"bound": "hbm", "alg_bytes_per_step": alg, "achieved_gbs": gbs, "peak": hbm,
                             "peak_kind": peak_kind, "frac": gbs / hbm},
                "pe_max": float(pe.max()), "pe_mean": float(pe.mean())}
    finally:
        d.close()


def measure_features(args, stream):
    """Field-pass time per step on the 256^3 bench grid with features removed one at a
    time (tracing events, 200 steps after 20 warm-up steps): where the pass loses time."""
    from paper_2512_06173_gb300 import maxlink, workloads

    sh = stream.cuda_stream
    base = workloads.superradiant_slab()
    vac = workloads.Problem(256, 256, 256, 0.5)
    none = workloads.empty_molecules()
    cases = [("bench: CPML 10, current box, 2 planes", base),
             ("CPML only", base.replace(molecules=none, planes=[])),
             ("PEC walls only", base.replace(pml=(0,) * 6, molecules=none, planes=[])),
             ("CPML on x faces only", vac.replace(pml=(10, 10, 0, 0, 0, 0))),
             ("CPML on y faces only", vac.replace(pml=(0, 0, 10, 10, 0, 0))),
             ("CPML on z faces only", vac.replace(pml=(0, 0, 0, 0, 10, 10)))]
    out = []
    for label, prob in cases:
        g = maxlink.Grid(prob, maxlink.ML_F32, stream=sh)
        try:
            g.step(20)
            g.sync()
            maxlink.ml_set_timing(g.h, True)
            maxlink.ml_timing(g.h)
            g.step(200)
            g.sync()
            ms, _ = maxlink.ml_timing(g.h)
            maxlink.ml_set_timing(g.h, False)
            us = ms[1] / 200 * 1e3
            out.append({"case": label, "field_pass_us": us, "tbs_at_48B_per_cell": prob.cells * 48 / us / 1e6})
        finally:
            g.close()
    return {"cases": out}


def measure_batch(args, stream):
    """64 plasmonic realisations of uneven size (edges 64..160, 200-5000 emitters each):
    K steps as one batch (one launch per kernel class per step, graph-replayed, field-pass
    grid from the autotuner) against the same K steps with ml_step on each grid in turn
    (the plain one-instance-per-launch method).  Both start from the same state.  The
    plain grids use the automatic short z chunks, the batched ones 32-plane chunks: the
    fields do not depend on the chunking, the per-instance absorbed energies agree to
    rounding (the per-block partial sums are grouped differently)."""
    import numpy as np
    import torch
    from paper_2512_06173_gb300 import maxlink, workloads

    probs = workloads.plasmonic_batch(count=args.batch_count)
    sh = stream.cuda_stream
    K = args.batch_steps
    cells = sum(p.cells for p in probs)
    # each method in its own best decomposition: a grid stepped alone needs the short
    # automatic z chunks to fill the GPU, batched grids take the long ones
    plain = [maxlink.Grid(p.replace(zchunk=0), maxlink.ML_F32, stream=sh) for p in probs]
    grids = [maxlink.Grid(p, maxlink.ML_F32, stream=sh) for p in probs]
    b = maxlink.Batch(grids, stream=sh)
    try:
        for g in plain:
            g.step(32)
        b.step(32)
        choice, tune_ms = b.autotune(64)
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        for g in plain:
            g.step(K)
        e1.record(stream)
        l0 = b.launches
        b.step(K)
        e2.record(stream)
        stream.synchronize()
        plain_ms, batch_ms = e0.elapsed_time(e1), e1.elapsed_time(e2)
        launches = b.launches - l0
        # per-kernel split of the batched step (traced, without the graph): the time a step
        # spends outside kernels (launch gaps, kernel tails) is what one fused persistent
        # launch per step could at most take away
        KT = 128
        maxlink.ml_batch_set_timing(b.h, True)
        maxlink.ml_batch_timing(b.h)
        b.step(KT)
        kms, _ = maxlink.ml_batch_timing(b.h)
        maxlink.ml_batch_set_timing(b.h, False)
        ksum = float(kms[0] + kms[1] + kms[3] + kms[4]) / KT
        ab_p = np.array([g.absorbed() for g in plain])
        ab_b = np.array([g.absorbed() for g in grids])
        # the batch's field passes move at least the algorithmic bytes of every instance's
        # field pass each step: that over the batched step time (which also holds the
        # molecule, current and fold kernels) is a lower bound of the field passes' rate
        hbm, peak_kind = peaks()
        alg = sum(field_pass_bytes(p, 4) for p in probs)
        step_gbs = alg / (batch_ms / K / 1e3) / 1e9
        return {"workload": f"{len(probs)} plasmonic realisations, edges {{64,96,128,160}}, Drude sphere r=edge/6, "
                            f"200-5000 emitters in a shell, z-polarised pulse", "instances": len(probs),
                "cells": cells, "molecules": int(sum(p.molecules.count for p in probs)), "steps": K,
                "dtype": "f32", "plain_ms": plain_ms, "batched_ms": batch_ms,
                "plain_gcells": cells * K / plain_ms / 1e6, "batched_gcells": cells * K / batch_ms / 1e6,
                "speedup": plain_ms / batch_ms, "blocks_per_sm": choice, "autotune_trial_ms": tune_ms,
                "kernel_ms_per_step_traced": {"molecules": kms[0] / KT, "current": kms[4] / KT,
                                              "field_pass": kms[1] / KT, "plane_fold": kms[3] / KT},
                "step_minus_kernel_sum_ms": batch_ms / K - ksum,
                "roofline": {"bound": "hbm", "alg_bytes_per_step": alg, "achieved_gbs_whole_step": step_gbs,
                             "peak": hbm, "peak_kind": peak_kind, "frac": step_gbs / hbm,
                             "note": "field-pass algorithmic bytes of all instances over the whole batched step"},
                "batched_launches": int(launches),
                "absorbed_max_rel_diff": float(np.max(np.abs(ab_p - ab_b) / np.maximum(np.abs(ab_p), 1e-300))),
                "absorbed_sum": float(ab_b.sum())}
    finally:
        b.close()
        for g in plain + grids:
            g.close()


def measure_transfer(args, stream):
    """Resonance energy transfer (Sec. IV.B setup with model acceptors): 64 independent
    96^3 realisations, each a two-level donor (dipole 2, coherent state) and a
    ground-state 2-, 4- or 8-level model acceptor (strongest dipole 0.02) 8-24 cells
    apart in vacuum; args.transfer_steps steps as one batch (one launch per kernel class
    per step, graph-replayed, field-pass grid from the autotuner).  Reports the batch's
    cell and molecule throughput and, as a readout of the physics, the acceptors' mean
    energy gain by model and the donors' mean excited population."""
    import numpy as np
    import torch
    from paper_2512_06173_gb300 import maxlink, workloads

    probs = workloads.energy_transfer_batch(count=args.transfer_count)
    sh = stream.cuda_stream
    K = args.transfer_steps
    cells = sum(p.cells for p in probs)
    grids = [maxlink.Grid(p, maxlink.ML_F32, stream=sh) for p in probs]
    b = maxlink.Batch(grids, stream=sh)
    try:
        b.step(32)
        choice, tune_ms = b.autotune(64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = b.launches
        e0.record(stream)
        b.step(K)
        e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1)
        launches = b.launches - l0
        gain, pe_d = {}, []
        for g, p in zip(grids, probs):
            n = int(p.molecules.nlev[1])
            H = p.molecules.matrix(p.molecules.H0, 1)
            gain.setdefault(n, []).append(float(np.real(np.trace(g.rho(1) @ H))))
            pe_d.append(float(g.rho(0)[1, 1].real))
        mol_steps = sum(p.molecules.count for p in probs) * K
        return {"workload": f"{len(probs)} energy-transfer realisations, 96^3 vacuum, 10-cell CPML, two-level donor "
                            f"(mu 2, coherent) + 2/4/8-level model acceptor (mu 0.02) 8-24 cells apart",
                "instances": len(probs), "cells": cells, "molecules": int(sum(p.molecules.count for p in probs)),
                "steps": K, "dtype": "f32", "ms_per_step": ms / K, "gcells_per_s": cells * K / ms / 1e6,
                "molecule_steps_per_s": mol_steps / ms * 1e3, "blocks_per_sm": choice,
                "batched_launches": int(launches),
                "acceptor_gain_mean": {str(n): float(np.mean(v)) for n, v in sorted(gain.items())},
                "donor_pe_mean": float(np.mean(pe_d))}
    finally:
        b.close()
        for g in grids:
            g.close()


def gpu_index_of(local: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            return int(vis.split(",")[local])
        except ValueError:
            pass
    return local


def measure_coupled(prob, args, stream, world, rank, local, K, W, with_clocks=True, with_e2e=True):
    """Whole-hot-path throughput of one workload: W warm-up steps, then K steps timed with
    CUDA events on the launching stream between barriers (untraced, so the programmatic
    launch chain overlaps as it does for a user), then a traced pass (events around every
    launch) for the per-kernel split and the field pass's roofline, then the end-to-end leg
    through the C ABI with host buffers."""
    import numpy as np
    import torch
    from paper_2512_06173_gb300 import maxlink

    sh = stream.cuda_stream
    esz = 4
    g = maxlink.Grid(prob, maxlink.ML_F32, stream=sh)
    out = {}
    try:
        g.step(W)
        g.sync()
        sampler = ClockSampler(gpu_index_of(local)) if (rank == 0 and with_clocks) else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        launches0 = maxlink.ml_launch_count(g.h)
        barrier(world)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.step(K)
        e1.record(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        barrier(world)
        out["clocks"] = sampler.stop() if sampler else None
        out["launches"] = maxlink.ml_launch_count(g.h) - launches0
        ms = e0.elapsed_time(e1)
        g.sync()
        # traced pass right after the timed region: CUDA events around every launch on the
        # launching stream give each kernel's average duration (the events separate the
        # kernels, so they do not overlap here as they do in the timed region)
        KT = max(1, min(K, args.traced_steps))
        maxlink.ml_set_timing(g.h, True)
        maxlink.ml_timing(g.h)  # clear
        g.step(KT)
        g.sync()
        kms, kcnt = maxlink.ml_timing(g.h)
        maxlink.ml_set_timing(g.h, False)
        ms_max = allreduce_max(world, ms)
        cells_total = allreduce_sum(world, float(prob.cells) * K)
        out["ms_per_step"] = ms_max / K
        out["value"] = cells_total / (ms_max / 1e3) / 1e9
        out["molecule_steps_per_s"] = allreduce_sum(world, float(prob.molecules.count) * K) / (ms_max / 1e3)
        hbm, peak_kind = peaks()
        k1_ms = kms[1] / KT
        alg = field_pass_bytes(prob, esz)
        achieved = alg / (k1_ms / 1e3) / 1e9
        out["roofline"] = {"bound": "hbm", "kernel": "yee_kernel (fused H/E + CPML + material + source + current "
                                                      "read + plane sampling)",
                           "timing": f"CUDA events around each launch on the launching stream, traced pass of {KT} "
                                     f"steps after the timed region",
                           "achieved": achieved, "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s",
                           "frac": achieved / hbm, "traffic": field_pass_traffic(prob), "alg_bytes_per_step": alg,
                           "field_pass_ms_per_step": k1_ms, "launches_per_step": kcnt[1] / KT}
        out["kernel_ms_per_step"] = {"gather": kms[5] / KT, "molecules": kms[0] / KT, "current": kms[4] / KT,
                                     "field_pass": k1_ms, "plane_fold": kms[3] / KT}
        pops = g.molecules(maxlink.ML_MOL_POP)
        flux = [g.flux(p) for p in range(len(prob.planes))]
        out["check"] = {"pop_excited_mean": float(np.mean(1.0 - pops[:, 0])), "flux_plane0_f0": float(flux[0][0])}
    finally:
        g.close()
    if not with_e2e:
        return out
    # ---- end to end through the C ABI with host buffers: every step's inputs are the
    # previous step's state on the device; the initial fields come from pinned host memory
    # inside the timed region, each step's populations reach pinned host memory through the
    # population sink, and the spectra are read at the end
    N = prob.cells
    g2 = maxlink.Grid(prob, maxlink.ML_F32, stream=sh)
    try:
        host_fields = torch.zeros((6, N), dtype=torch.float32, pin_memory=True)
        ring = 2
        host_pop = torch.zeros((ring * prob.molecules.count * maxlink.ML_MAX_LEVELS,), dtype=torch.float64,
                               pin_memory=True)
        maxlink.ml_set_population_sink(g2.h, host_pop.data_ptr(), ring)
        g2.step(W)
        g2.sync()
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        maxlink.ml_set_fields(g2.h, maxlink.ML_ALL, host_fields.data_ptr(), False, sh)
        for _ in range(K):
            maxlink.ml_step(g2.h, 1, sh)
        fl = [g2.flux(p) for p in range(len(prob.planes))]
        stream.synchronize()
        e2e_s = allreduce_max(world, time.perf_counter() - t0)
        g2.sync()
        last = (maxlink.ml_step_count(g2.h) - 1) % ring
        pe_e2e = float(1.0 - host_pop.view(ring, prob.molecules.count, maxlink.ML_MAX_LEVELS)[last, :, 0].mean())
        maxlink.ml_set_population_sink(g2.h, 0, 1)
        h2d = 6 * N * esz / K
        # the populations written to the host each step (nlev doubles per molecule) and the
        # spectra read once at the end
        d2h = int(prob.molecules.nlev.sum()) * 8 + sum(8 * len(p.omegas) for p in prob.planes) / K
        out["e2e"] = {"value": allreduce_sum(world, float(N) * K) / e2e_s / 1e9, "unit": UNIT,
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
        out["check"]["e2e_flux_plane0_f0"] = float(fl[0][0])
        out["check"]["e2e_pop_excited_mean"] = pe_e2e
    finally:
        g2.close()
    return out


def measure_superradiant(args, stream):
    """Superradiant slab (256^3 vacuum, 10-cell CPML, 10,000 two-level emitters in a
    32-cell central slab, two flux planes): the coupled step and its field pass's roofline,
    args.sr_steps steps after 20 warm-up steps."""
    from paper_2512_06173_gb300 import workloads
    prob = workloads.superradiant_slab(n=args.edge, nmol=args.nmol, seed=2)
    r = measure_coupled(prob, args, stream, 1, 0, 0, args.sr_steps, 20, with_clocks=False, with_e2e=False)
    return {"workload": prob.name, "cells": prob.cells, "molecules": prob.molecules.count, "steps": args.sr_steps,
            "dtype": "f32", "gcells_per_s": r["value"], "ms_per_step": r["ms_per_step"],
            "molecule_steps_per_s": r["molecule_steps_per_s"], "roofline": r["roofline"],
            "kernel_ms_per_step": r["kernel_ms_per_step"], "gpu_launches": r["launches"]}


def measure_static_gather(args, stream):
    """ml_gather_static at its molecule limit: 16,384 molecules at seeded positions in a
    256^3 FP32 field (periodic on every axis), widths sigma = 1.5 and the widest accepted
    sigma = 7/3 (a 16-plane window); CUDA events around 50 calls after 5 warm-up calls."""
    import numpy as np
    import torch
    from paper_2512_06173_gb300 import maxlink

    n, M = 256, maxlink.ML_STATIC_GATHER_MAX_MOLECULES
    rng = np.random.default_rng(11)
    E = torch.randn(3 * n ** 3, dtype=torch.float32, device="cuda")
    pos = torch.tensor(rng.uniform(0.0, n, (M, 3)), dtype=torch.float64, device="cuda")
    gamma = torch.ones(M, dtype=torch.float64, device="cuda")
    out = torch.empty((M, 3), dtype=torch.float32, device="cuda")
    sh = stream.cuda_stream
    res = {"molecules": M, "grid": f"{n}^3"}
    for sg in (1.5, 7.0 / 3.0):
        sigma = torch.full((M,), sg, dtype=torch.float64, device="cuda")
        call = lambda: maxlink.ml_gather_static(E.data_ptr(), n, n, n, (1, 1, 1), M, pos.data_ptr(),
                                                sigma.data_ptr(), gamma.data_ptr(), out.data_ptr(), sh)
        with torch.cuda.stream(stream):
            for _ in range(5):
                call()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(50):
                call()
            e1.record(stream)
        e1.synchronize()
        us = e0.elapsed_time(e1) / 50 * 1e3
        R = int(np.ceil(3 * sg))
        res[f"sigma_{sg:.3f}"] = {"us_per_call": us, "molecules_per_s": M / us * 1e6, "window": 2 * R + 2}
    return res


def run_ours(args, world, rank, local):
    import torch

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU for the CUDA path")
    torch.cuda.set_device(local)
    sections = {"adjoint": measure_adjoint, "batch": measure_batch, "bragg": measure_bragg,
                "superradiant": measure_superradiant, "dispersive": measure_dispersive,
                "transfer": measure_transfer, "features": measure_features, "cavity": measure_cavity,
                "laser": measure_laser, "static_gather": measure_static_gather}
    if args.section != "main":
        # one secondary measurement alone (profiling runs): its JSON object, rank 0
        out = sections[args.section](args, torch.cuda.Stream())
        if rank == 0:
            print(json.dumps({"section": args.section, **out}), flush=True)
        return
    prob = headline_problem(args, rank)
    stream = torch.cuda.Stream()
    K, W = args.steps, args.warmup
    main = measure_coupled(prob, args, stream, world, rank, local, K, W, with_clocks=True,
                           with_e2e=not args.no_e2e)
    if args.no_e2e:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": main["value"], "unit": UNIT, "steps": K,
                              "profiling_run": True}), flush=True)
        return
    solo = world == 1
    sec = {}
    for name, skip in (("superradiant", args.no_superradiant), ("adjoint", args.no_adjoint),
                       ("batch", args.no_batch), ("dispersive", args.no_dispersive),
                       ("transfer", args.no_transfer), ("cavity", args.no_cavity), ("laser", args.no_laser),
                       ("static_gather", args.no_static_gather)):
        sec[name] = sections[name](args, stream) if (solo and not skip) else None
    # ---- CPU baseline: the oracle on this host, rank 0 at N=1 only
    cpu = None
    if rank == 0 and solo and not args.no_cpu_baseline:
        n, dt, cores = cpu_oracle_run(prob, budget_s=args.cpu_budget, max_steps=50)
        cpu = {"value": prob.cells * n / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n} full steps (after 1 warm-up step) of the same {prob.nx}x{prob.ny}x{prob.nz} "
                         f"workload with all {prob.molecules.count} systems, FP64"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic", "config": config_of(prob, world),
            "roofline": main["roofline"], "cpu_baseline": cpu, "e2e": main["e2e"],
            "gpu_launches": int(main["launches"]), "clocks": main["clocks"],
            "molecule_steps_per_s": main["molecule_steps_per_s"],
            "kernel_ms_per_step": main["kernel_ms_per_step"], "check": main["check"],
        }
        line.update(sec)
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--ref-budget", type=float, default=40.0,
                    help="seconds of timed oracle steps in the reference arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--edge", type=int, default=256, help="superradiant slab: grid edge")
    ap.add_argument("--nmol", type=int, default=10000, help="superradiant slab: emitters")
    ap.add_argument("--sr-steps", type=int, default=2000, help="superradiant slab: timed steps")
    ap.add_argument("--no-superradiant", action="store_true", help="skip the superradiant slab")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint/forward timing")
    ap.add_argument("--traced-steps", type=int, default=400,
                    help="steps of the traced pass that times each kernel (roofline)")
    ap.add_argument("--section", default="main", choices=["main", "adjoint", "batch", "bragg", "superradiant",
                                                        "dispersive", "transfer", "features", "cavity", "laser",
                                                        "static_gather"],
                    help="run only this measurement (the default runs the main line with every section)")
    ap.add_argument("--adj-steps", type=int, default=3000)
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-realisations comparison")
    ap.add_argument("--batch-steps", type=int, default=3000)
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--no-bragg", action="store_true", help="skip the Bragg-resonator ensemble")
    ap.add_argument("--no-cavity", action="store_true", help="skip the single-mode cavity")
    ap.add_argument("--cavity-steps", type=int, default=2000)
    ap.add_argument("--cavity-molecules", type=int, default=1000000)
    ap.add_argument("--no-laser", action="store_true", help="skip the laser-driven molecules")
    ap.add_argument("--no-static-gather", action="store_true", help="skip the allocation-free gather timing")
    ap.add_argument("--laser-steps", type=int, default=2000)
    ap.add_argument("--laser-molecules", type=int, default=4000000)
    ap.add_argument("--bragg-steps", type=int, default=400)
    ap.add_argument("--bragg-shape", type=int, nargs=3, default=(512, 512, 384),
                    help="grid of the Bragg ensemble, the headline workload (profiling runs use a smaller copy)")
    ap.add_argument("--bragg-nmol", type=int, default=100000)
    ap.add_argument("--no-dispersive", action="store_true", help="skip the dispersive stack")
    ap.add_argument("--dispersive-steps", type=int, default=400)
    ap.add_argument("--no-transfer", action="store_true", help="skip the energy-transfer realisations")
    ap.add_argument("--transfer-steps", type=int, default=2000)
    ap.add_argument("--transfer-count", type=int, default=64)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
