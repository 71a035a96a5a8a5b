"""Throughput benchmark of the block-update hot path on GB300.

Workload (one "step" = one full SSPRK3 step = 3 stage launches of the update kernel plus
the ghost/CFL/GLM work around them): 3-D ideal MHD with GLM divergence cleaning on a
periodic 256^3 grid of 4096 blocks of 16^3 cells, Orszag-Tang-like fields plus seeded 1%
velocity noise, HLL, PLM van Leer, SSPRK3, CFL 0.4, dt from the on-device CFL reduction.
The headline value is the FP32-stencil run (FP64 kept for the CFL reduction); the FP64
run is reported beside it. Metric: zone-updates/s (one interior cell advanced by one RK
stage). The state (604 MB FP32, 1.2 GB FP64 per buffer) exceeds the 129 MB L2, so no
flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs independent replicas (one per rank, weak scaling): the path has no exchange
across GPUs on one mesh. --impl reference times the FP64 CPU oracle on a bounded sample of
the same workload.
"""
from __future__ import annotations

import argparse
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

METRIC = "zone-updates/s per GB300 (FP32 batched vs FP64 plain) and % HBM roofline; p50/p99 solve latency"
UNIT = "zone-updates/s"
N_SIDE = 256
WORKLOAD = "mhd_glm_orszag_tang_256^3_4096x16^3_hll_vanleer_ssprk3"


def spec():
    return dict(physics="mhd", limiter="vanleer", flux="hll", rk=3, cfl=0.4,
                base_blocks=(N_SIDE // 16,) * 3)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region (SM clock, throttle reasons)."""

    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self, t0=None, t1=None):
        """Median SM clock and active throttle reasons of the samples taken between the
        host times t0 and t1 (the timed region); the nearest later sample if none fell in."""
        import datetime
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        samples = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                samples.append((ts, float(parts[1]), float(parts[2]), parts[4:8]))
            except ValueError:
                continue
        inside = [x for x in samples if t0 is None or (t0 <= x[0] <= t1)]
        if not inside and samples and t0 is not None:
            later = [x for x in samples if x[0] >= t0]
            inside = later[:1] if later else samples[-1:]
        sm = [x[1] for x in inside]
        smax = [x[2] for x in inside]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for x in inside:
            for n, v in zip(names, x[3]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def replica_throughput(zones_per_rank, stages, steps, local_ms, world):
    """Whole-job zone-updates/s of `world` independent replicas (weak scaling): every rank
    advanced zones_per_rank cells by stages * steps substeps; the job time is the slowest
    rank's (max over ranks through the default process group when world > 1). Returns
    (zone-updates/s, max time in ms)."""
    t_ms = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([t_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_ms = float(t.item())
    return zones_per_rank * stages * steps * world / (t_ms / 1e3), t_ms


# Analytic floating-point operation count of one zone-update of the implemented scheme
# (MHD + GLM, HLL, PLM van Leer, SSPRK3 combine; each face flux once, +,-,*,/,sqrt,min,max
# count 1, FMA counts 2). Per face: PLM 9 x 21 = 189, GLM pair 10, prim->cons 2 x 18,
# physical fluxes 2 x 37, fast speeds 2 x 24, HLL combine 70 -> 427; 3 x 17/16 faces per
# zone-update -> 1361; primitive recovery 1.75 x 19 -> 33; divergence + stage combine 108.
MHD_HLL_VL_FLOPS = 1502
SMS = 152
FP32_LANES = 128     # FP32 FMA lanes per SM
FP64_LANES = 2       # FP64 FMA lanes per SM on GB300 (1.25 TFLOP/s measured at 2.07 GHz)


# DRAM bytes (read + write) per stage launch of the FP32 MHD stage kernel on this workload,
# from one ncu capture of the three stage launches of one SSPRK3 step (1.201, 1.839 and
# 1.804 GB; blocks taken in z-slab order), averaged; valid only while the kernel sources
# hash to STAGE_SRC_DIGEST.
STAGE_TRAFFIC_BYTES = (1.2008e9 + 1.8389e9 + 1.8044e9) / 3
STAGE_SRC_DIGEST = "0d29d99aee7755b5"
STAGE_SRC = ("kernels.cuh", "pair.cuh", "physics.cuh", "stage_go.cuh", "stage_mhd.cu")


def stage_traffic():
    """Measured per-launch DRAM traffic, or None when the kernel changed since the capture."""
    import hashlib
    h = hashlib.sha256()
    try:
        for f in STAGE_SRC:
            with open(os.path.join(ROOT, "paper_2607_19277_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
    except OSError:
        return None
    return STAGE_TRAFFIC_BYTES if h.hexdigest()[:16] == STAGE_SRC_DIGEST else None


def alu_peak_tflops(lanes, mhz):
    """Peak flop rate from unit counts and the SM clock seen during the run."""
    return SMS * lanes * 2 * mhz * 1e6 / 1e12


def ghost_inflated_bytes_per_zone(nvar, w, rk):
    """Bytes per zone-update of a storage scheme with 20^3 ghost-cell block arrays (the paper's
    layout, Section 3.1): the algorithmic bytes plus, per stage, the halo part of the stage
    input read (8000 / 4096 - 1 of the interior), the ghost-cell writes of the fill (3904 /
    4096) and the reads that fill them (as many). This build reads same-level halos in place
    and writes no ghost cells on uniform grids; the figure says what a ghost-copy
    implementation must move for the same rate."""
    g = nvar * w * (8000.0 / 4096.0 - 1.0 + 2.0 * 3904.0 / 4096.0)
    return algorithmic_bytes_per_zone(nvar, w, rk) + g


def algorithmic_bytes_per_zone(nvar, w, rk):
    """Compulsory bytes per zone-update, averaged over the stages of one step: read U_s and
    write U_out every stage, read U^n in the stages that combine with it."""
    per = [nvar * w * (2 + (0 if s == 0 else 1)) for s in range(rk)]
    return sum(per) / rk


def run_gpu(real_bytes, steps, warmup, rank, world, dev):
    import numpy as np
    import torch

    from paper_2607_19277_gb300 import agile, workloads as W

    sp = spec()
    nblk = (N_SIDE // 16) ** 3
    zones = nblk * 4096
    stream = torch.cuda.current_stream()
    m = agile.Mesh(agile.make_config(real_bytes=real_bytes, **sp), stream=stream)
    m.set_state(W.orszag_tang_3d(N_SIDE))
    clocks = Clocks(dev)
    clocks.start()          # started early so that it samples throughout the timed region
    for _ in range(warmup):
        m.step(0.0)
    m.sync()
    time.sleep(0.3)
    # ---- device-timed region: inputs resident in HBM
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    m.set_kernel_timing(True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    t_start = time.time()
    ev[0].record(stream)
    for i in range(steps):
        m.step(0.0)
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    t_end = time.time()
    clk = clocks.stop(t_start, t_end)
    if world > 1:
        torch.distributed.barrier()
    per_step = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    total_ms = ev[0].elapsed_time(ev[steps])
    stage_ms, stage_launches, total_launches = m.kernel_timing()
    m.set_kernel_timing(False)
    m.sync()
    # ---- end-to-end through the C ABI with pinned host buffers: upload the state, run
    # the steps (CFL dt on the device, as agile_step(0) takes it) with the conserved-sum
    # diagnostics read back after every step (the paper's high-cadence log), download the
    # final state.
    lev, ijk, cons = m.get_state()
    pinned_in = torch.from_numpy(cons).pin_memory()
    pinned_out = torch.empty_like(pinned_in).pin_memory()
    state_bytes = cons.nbytes
    del cons
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m.set_state_blocks(pinned_in.numpy())
    for _ in range(steps):
        m.step(0.0)
        m.conserved_sums()
    lib = m.lib
    import ctypes as C
    st = lib.agile_get_state(m.ptr, None, None,
                             C.cast(pinned_out.data_ptr(), C.POINTER(C.c_double)))
    if st:
        raise RuntimeError("agile_get_state failed: %d" % st)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    m.close()
    return dict(zones=zones, total_ms=total_ms, per_step=per_step, stage_ms=stage_ms,
                stage_launches=stage_launches, total_launches=total_launches, clocks=clk,
                e2e_s=e2e_s, state_bytes=state_bytes, nvar=9)


def run_error_vs_fp64(nsteps):
    """Error of the FP32 stencil on the headline workload against the FP64 stencil (whose
    agreement with the FP64 oracle the parity tests establish): both meshes start from the
    same state and take the same nsteps steps with the FP64 mesh's CFL dt; then the relative
    L1 error per variable, sum |a - b| / sum |b| over all cells. psi starts at zero and holds
    only the discretisation error of div B, so its error is also given on the c_max sum |B|
    scale it is rounded on."""
    from paper_2607_19277_gb300 import agile, workloads as W
    ms = {rb: agile.Mesh(agile.make_config(real_bytes=rb, **spec())) for rb in (8, 4)}
    for m in ms.values():
        m.set_state(W.orszag_tang_3d(N_SIDE))
    for _ in range(nsteps):
        dt = ms[8].cfl_dt()
        ms[8].step(dt)
        ms[4].step(dt)
    _, cmax = ms[8].max_speeds()
    _, _, r = ms[8].get_state()
    ms[8].close()
    _, _, g = ms[4].get_state()
    ms[4].close()
    num = np.array([np.abs(g[:, v] - r[:, v]).sum() for v in range(9)])
    den = np.array([np.abs(r[:, v]).sum() for v in range(9)])
    del g, r
    rel = num / den
    names = ["rho", "m_x", "m_y", "m_z", "e", "B_x", "B_y", "B_z", "psi"]
    # m_z and B_z start at (near) zero and stay small, so their own norms are small too; the
    # error of each vector component on the scale of its whole vector is given beside it
    vec = {"m": (1, 4), "B": (5, 8)}
    on_vec = {}
    for nm, (a, b) in vec.items():
        for v in range(a, b):
            on_vec[names[v]] = float(num[v] / den[a:b].sum())
    return {"steps": nsteps, "reference": "FP64 stencil, same dt per step",
            "rel_l1": {n: float(x) for n, x in zip(names, rel)},
            "rel_l1_on_vector_scale": on_vec,
            "max_rel_l1_rho_m_e_B": float(rel[:8].max()),
            "psi_rel_l1_on_cmax_B_scale": float(num[8] / (cmax * den[5:8].sum())),
            "psi_norm_over_cmax_B": float(den[8] / (cmax * den[5:8].sum()))}


BATCH_SIDES = (32, 48, 64, 80, 96, 112, 128)


def batch_workload(nsolve=256, seed=20260004):
    """Seeded batch of SRHD solves: side from {32, ..., 128} per solve, one shell each with
    radial Lorentz factor U[1, 10] (the configured range), radius U[0.2, 0.35], a Gaussian
    profile two cells wide, periodic (minimum-image) distances, ambient rho = p = 1. Thinner
    or multiple colliding shells, or radii of three cells at 32^3, reach states without a
    primitive solution within ten steps at these Lorentz factors (in FP64 as well)."""
    from paper_2607_19277_gb300 import workloads as W
    u = W.uniform01(seed, np.arange(nsolve))
    sides = [BATCH_SIDES[min(len(BATCH_SIDES) - 1, int(x * len(BATCH_SIDES)))] for x in u]
    ics = [W.srhd_shells(seed + 1 + i, sides[i], n_shells=1, lorentz_max=10.0, p_amb=1.0, smooth=True,
                         width=2.0, wrap=True, radius=(0.2, 0.35))
           for i in range(nsolve)]
    return sides, ics


def run_batched(steps, warmup, nsolve=256, fp64_solves=8):
    """Batched FP32 SRHD solves (one launch per RK stage over all of them, CUDA-graph
    steps) against the plain FP64 per-solve path on the first fp64_solves solves."""
    import torch
    from paper_2607_19277_gb300 import agile
    sides, ics = batch_workload(nsolve)

    def cfg(side, rb):
        return agile.make_config(physics="srhd", limiter="minmod", flux="tvdlf", rk=2, gamma=4.0 / 3.0,
                                 cfl=0.4, real_bytes=rb, base_blocks=(side // 16,) * 3)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = agile.Batch([cfg(sd, 4) for sd in sides], stream=stream)
        for i in range(nsolve):
            b.set_state(i, ics[i])
        tuned = b.autotune(trials=2)     # before the warm-up steps, which capture the graph
        for _ in range(warmup):
            b.step()
        b.sync()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        l0 = b.launches()
        ev[0].record(stream)
        for i in range(steps):
            b.step()
            ev[i + 1].record(stream)
        stream.synchronize()
        per = sorted(ev[i].elapsed_time(ev[i + 1]) for i in range(steps))
        total = ev[0].elapsed_time(ev[steps])
        b.sync()
        launches = b.launches() - l0
        b.close()
    zones = sum(sd ** 3 for sd in sides)
    out = {"value": zones * 2 * steps / (total / 1e3), "unit": UNIT, "solves": nsolve,
           "lorentz_factor_max_initial": max(sh["lorentz"] for ic in ics for sh in ic.shells),
           "cells": zones, "ms_per_step": total / steps, "step_latency_ms": {
               "p50": per[len(per) // 2], "p99": per[min(len(per) - 1, int(math.ceil(0.99 * len(per))) - 1)]},
           "dtype": "f32 stencil, f64 con2prim", "graph_launches_per_step": "1 graph (set_dt + 2 stages)",
           "kernel_launches_in_timed_region": launches,
           "autotune": {"grid": tuned[0], "dynamic_blocks": tuned[1],
                        "staging_layout": {1: "4 raw slots, 1 flux buffer", 2: "5 raw slots, 2 flux buffers",
                                           3: "3 raw slots, 2 flux buffers, stage input from L2"}[tuned[3]],
                        "stage1_ms": {"%s,%d/SM,%s" % (lay, g, a): tuned[2][6 * li + 2 * (g - 1) + ai]
                                      for li, lay in enumerate(("ring4", "ring5db", "ring3db"))
                                      for g in (1, 2, 3) for ai, a in enumerate(("counter", "strided"))}}}
    # plain FP64 per-solve path: each solve its own mesh, solved one after the other
    z64 = 0
    t64 = 0.0
    st64 = max(2, steps // 4)
    for i in range(fp64_solves):
        m = agile.Mesh(cfg(sides[i], 8))
        m.set_state(ics[i])
        m.step(0.0)
        m.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(st64):
            m.step(0.0)
        e1.record()
        torch.cuda.synchronize()
        t64 += e0.elapsed_time(e1)
        z64 += sides[i] ** 3 * 2 * st64
        m.close()
    out["fp64_plain_per_solve"] = {"value": z64 / (t64 / 1e3), "unit": UNIT, "solves": fp64_solves,
                                   "steps": st64}
    return out


def run_paper_scheme(steps=10, warmup=3):
    """The paper's single-device benchmark scheme (Section 3.1): hydrodynamics, LF (TVDLF),
    PLM van Leer, SSPRK3, periodic, 256^3 in 4096 blocks of 16^3, double shear layer
    stand-in for its double Kelvin-Helmholtz setup, FP64 (the paper's precision) and FP32.
    Paper context (FP64, NVIDIA B200, same grid and block size): 1.552e9 CUPS (Table 4, Appendix B)."""
    import torch
    from paper_2607_19277_gb300 import agile, workloads as W
    out = {"workload": "hd tvdlf vanleer ssprk3 periodic 256^3 (4096 x 16^3), double shear layer",
           "paper_b200_fp64_cups": 1.552e9}
    for rb, name in ((8, "fp64"), (4, "fp32")):
        m = agile.Mesh(agile.make_config(physics="hd", limiter="vanleer", flux="tvdlf", rk=3,
                                         real_bytes=rb, base_blocks=(16, 16, 16)))
        m.set_state(W.double_kelvin_helmholtz())
        for _ in range(warmup):
            m.step(0.0)
        m.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            m.step(0.0)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        m.close()
        out[name] = {"value": 16.0 ** 3 * 4096 * 3 * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps}
    return out


def run_cooling(steps=20, warmup=3):
    """MHD+GLM 256^3 (the headline workload, FP32 stencil) with optically thin radiative
    losses (Section 2.3.1; log-skew-normal loss table peaked at the Orszag-Tang temperature
    p / rho = 0.25, cooling time ~0.1 code units), against the same run without losses: the
    throughput cost of the source term (the paper reports 10.2% for its FFHD case on an
    H100, Section 4.4)."""
    import torch
    from paper_2607_19277_gb300 import agile, workloads as W
    T, L = W.skew_normal_cooling(n=256, t_min=1e-2, t_max=1e2, t_peak=0.25, peak=1.0)
    res = {}
    for name, cool in (("plain", False), ("cooling", True)):
        m = agile.Mesh(agile.make_config(real_bytes=4, **spec()))
        if cool:
            m.set_cooling(T, L)
        m.set_state(W.orszag_tang_3d(N_SIDE))
        for _ in range(warmup):
            m.step(0.0)
        m.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            m.step(0.0)
        e1.record()
        torch.cuda.synchronize()
        res[name] = e0.elapsed_time(e1) / steps
        m.close()
    zones = float(N_SIDE ** 3) * 3
    return {"workload": "mhd_glm 256^3 hll vanleer ssprk3 fp32 + radiative losses (256-node table)",
            "value": zones / (res["cooling"] / 1e3), "unit": UNIT,
            "ms_per_step": res["cooling"], "ms_per_step_without": res["plain"],
            "throughput_reduction": 1.0 - res["plain"] / res["cooling"]}


def run_batched_amr(nsolve=16, steps=20, regrid_every=10):
    """Batched refined solves (§8(f) item 1 with all levels in one launch per stage): 16
    Sedov blasts (seeded centres) on base 64^3 grids of 16^3 blocks, max level 3, HLL minmod
    SSPRK2, FP32, regrid of every solve every `regrid_every` steps, against the same solves
    as separate meshes stepped one after the other. Zone-updates count every leaf cell and
    stage; the timed regions include the regrids."""
    import torch
    from paper_2607_19277_gb300 import agile, workloads as W
    u = W.uniform01(W.SEED_BASE + 31, np.arange(3 * nsolve)).reshape(nsolve, 3)
    ics = [W.sedov(r0=0.06, centre=tuple(0.3 * (2.0 * u[i] - 1.0))) for i in range(nsolve)]
    cfg = agile.make_config(physics="hd", limiter="minmod", flux="hll", rk=2, real_bytes=4, base_blocks=(4, 4, 4),
                            xmin=(-0.5,) * 3, xmax=(0.5,) * 3, bc=("outflow",) * 6, max_level=3,
                            refine_vars=(0, 4), refine_weights=(0.5, 0.5), refine_tol=0.2)
    out = {"workload": "%d hd sedov solves, base 64^3, max level 3, hll minmod ssprk2 fp32, regrid every %d steps"
                       % (nsolve, regrid_every)}

    def run(stepper, layouts):
        zones = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for n in range(steps):
            zones += 2 * 4096 * sum(layouts())
            stepper(n)
        torch.cuda.synchronize()
        return zones / (time.perf_counter() - t0)

    b = agile.Batch([cfg] * nsolve)
    for i in range(nsolve):
        b.set_state(i, ics[i])
    for _ in range(2):                     # initial refinement around the blasts
        b.regrid(-1, init=True)

    def bstep(n):
        b.step()
        if n % regrid_every == regrid_every - 1:
            b.regrid(-1)                   # every solve, one new layout
    b.step()
    out["batched"] = {"value": run(bstep, lambda: [b.layout(i)[0] for i in range(nsolve)]), "unit": UNIT}
    out["blocks"] = sum(b.layout(i)[0] for i in range(nsolve))
    b.close()
    ms = []
    for i in range(nsolve):
        m = agile.Mesh(cfg)
        m.set_state(ics[i])
        for _ in range(2):
            m.regrid(init=True)
        ms.append(m)

    def mstep(n):
        for m in ms:
            m.step(0.0)
        if n % regrid_every == regrid_every - 1:
            for m in ms:
                m.regrid()
    for m in ms:
        m.step(0.0)
    out["separate_meshes"] = {"value": run(mstep, lambda: [m.layout()[0] for m in ms]), "unit": UNIT}
    for m in ms:
        m.close()
    return out


def _average_to_base(lev, ijk, cons, nbase):
    """Volume average of every leaf onto the uniform base grid (nbase cells per dimension,
    16 per base block): a level-l block covers 16 / 2^(l-1) base cells per edge."""
    nv = cons.shape[1]
    out = np.zeros((nv, nbase, nbase, nbase))
    for i in range(len(lev)):
        f = 1 << (int(lev[i]) - 1)
        n = 16 // f
        red = cons[i].reshape(nv, n, f, n, f, n, f).mean(axis=(2, 4, 6))
        z0, y0, x0 = (int(ijk[i, 2]) * n, int(ijk[i, 1]) * n, int(ijk[i, 0]) * n)
        out[:, z0:z0 + n, y0:y0 + n, x0:x0 + n] += red
    return out


def run_sedov_5level(steps=200, regrid_every=10):
    """The refined Sedov blast at its stated size (Fig. 2 time loop with regrids): hydro,
    gamma 5/3, [-1/2, 1/2]^3 with outflow boundaries, base 64^3 (4x4x4 blocks of 16^3), five
    levels (effective 1024^3), Loehner estimator on rho and e (weights 1/2), initial
    refinement by four regrids that re-apply the initial condition, regrid every 10 steps,
    HLL, minmod, SSPRK2, CFL 0.4, dt from the device. FP32 bulk (FP64 dt, sums and
    estimator) against the FP64 stencil. Zone-updates count every leaf cell and stage; the
    timed region includes the regrids. Reports the device time of each phase (stage kernel,
    coarse-fine ghost fill, flux fix-up, estimator; CUDA events), the regrid's wall time, and
    the FP32 state's relative L1 error per variable against the FP64 state after both are
    averaged to the base level (the two runs may refine differently)."""
    import torch
    from paper_2607_19277_gb300 import agile, workloads as W
    spec = dict(physics="hd", limiter="minmod", flux="hll", rk=2, cfl=0.4, base_blocks=(4, 4, 4),
                xmin=(-0.5,) * 3, xmax=(0.5,) * 3, bc=("outflow",) * 6, max_level=5,
                refine_vars=(0, 4), refine_weights=(0.5, 0.5), refine_tol=0.2)
    out = {"workload": "hd sedov, base 64^3, 5 levels, loehner rho+e, regrid every %d steps, hll minmod "
                       "ssprk2, %d steps" % (regrid_every, steps)}
    states = {}
    for rb, name in ((4, "fp32"), (8, "fp64")):
        m = agile.Mesh(agile.make_config(real_bytes=rb, **spec))
        m.set_state(W.sedov(r0=0.03))
        for _ in range(4):
            m.regrid(init=True)
        s0 = m.conserved_sums()
        m.sync()
        m.set_kernel_timing(True)
        zones = 0
        regrid_s = 0.0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for n in range(steps):
            zones += m.layout()[0] * 4096 * 2
            m.step(0.0)
            if n % regrid_every == regrid_every - 1:
                m.sync()                       # the steps queued so far are not the regrid's
                r0 = time.perf_counter()
                m.regrid()
                regrid_s += time.perf_counter() - r0
        m.sync()
        wall = time.perf_counter() - t0
        ph = m.phase_timing()
        m.set_kernel_timing(False)
        s1 = m.conserved_sums()
        lev, ijk, cons = m.get_state()
        m.close()
        states[name] = (lev, ijk, cons)
        out[name] = {"value": zones / wall, "unit": UNIT, "seconds": wall, "leaves_end": int(len(lev)),
                     "levels_used": sorted(set(int(x) for x in lev)),
                     "share": {"stage_kernel": ph["stage"][0] / 1e3 / wall,
                               "ghost_fill": ph["ghost_fill"][0] / 1e3 / wall,
                               "flux_fixup": ph["fixup"][0] / 1e3 / wall,
                               "estimator": ph["estimate"][0] / 1e3 / wall,
                               "regrid_incl_estimator": regrid_s / wall,
                               "note": "device time per phase (CUDA events) and the regrid's wall time "
                                       "(estimator, host planning, new pools and tables), as shares of the "
                                       "timed wall time"},
                     "mass_energy_rel_change": [float(abs(s1[v] - s0[v]) / abs(s0[v])) for v in (0, 4)]}
        torch.cuda.empty_cache()
    a = _average_to_base(*states["fp64"], 64)
    b = _average_to_base(*states["fp32"], 64)
    err = np.abs(b - a).sum(axis=(1, 2, 3)) / np.abs(a).sum(axis=(1, 2, 3))
    out["fp32_rel_l1_vs_fp64_on_base_grid"] = {n: float(x) for n, x in zip(("rho", "m_x", "m_y", "m_z", "e"), err)}
    return out


def run_ffhd(steps=20, warmup=3, kappa0=1e-3):
    """Frozen-field hydrodynamics (Section 2.3.2) on a periodic 256^3 grid of 16^3 blocks
    in a sheared frozen field, TVDLF, van Leer, SSPRK3, FP32 stencil: without source terms,
    with radiative losses, with hyperbolic thermal conduction (kappa0 T^(5/2), tau = 4 dt) and
    with both (the paper compares these four configurations for its FFHD case on an H100 and
    reports 10.2%, 21.8% and 29.4% lower throughput for losses, conduction and both, Section
    4.4; it reports relative costs, not this grid)."""
    import torch
    from paper_2607_19277_gb300 import agile, workloads as W
    T, L = W.skew_normal_cooling(n=256, t_min=5e-2, t_max=1e2, t_peak=1.0, peak=0.5)

    def ic(nv):
        def f(x, y, z):
            th = 0.7 * np.sin(2 * math.pi * x) + 0.5 * np.cos(2 * math.pi * (y + z))
            p = np.zeros((nv,) + np.shape(x))
            p[0] = 1.0 + 0.3 * np.sin(2 * math.pi * (x + 2 * y)) * np.cos(2 * math.pi * z)
            p[1] = 0.4 * np.cos(2 * math.pi * (x - y))
            p[2] = 1.0 + 0.2 * np.sin(2 * math.pi * (y + z))
            o = nv - 3                      # the frozen field follows q_par when present
            p[o] = np.cos(th) * np.cos(0.3 * th)
            p[o + 1] = np.sin(th) * np.cos(0.3 * th)
            p[o + 2] = np.sin(0.3 * th)
            return p
        return f
    out = {"workload": "ffhd 256^3 (4096 x 16^3) sheared frozen field, tvdlf vanleer ssprk3, fp32; "
                       "conduction kappa0 = %g" % kappa0}
    for name, cool, htc in (("plain", False, False), ("losses", True, False), ("conduction", False, True),
                            ("both", True, True)):
        m = agile.Mesh(agile.make_config(physics="ffhd_htc" if htc else "ffhd", htc_kappa0=kappa0 if htc else 0.0,
                                         limiter="vanleer", flux="tvdlf", rk=3, real_bytes=4,
                                         base_blocks=(N_SIDE // 16,) * 3))
        if cool:
            m.set_cooling(T, L)
        m.set_state(ic(7 if htc else 6))
        for _ in range(warmup):
            m.step(0.0)
        m.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            m.step(0.0)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        m.close()
        out[name] = {"value": float(N_SIDE ** 3) * 3 / (ms / 1e3), "unit": UNIT, "ms_per_step": ms}
    for name in ("losses", "conduction", "both"):
        out["throughput_reduction_" + name] = 1.0 - out["plain"]["ms_per_step"] / out[name]["ms_per_step"]
    out["paper_h100_reduction"] = {"losses": 0.102, "conduction": 0.218, "both": 0.294}
    return out


def run_serving(nreq=64, rate=50.0, budget_gb=160.0, fp64_subset=8):
    """Serving stream with the configured ranges (Poisson arrivals at mean 50/s of HD / MHD /
    SRHD solves, sides 32-256, 50-500 steps, admitted against a 160 GB HBM budget), a bounded
    sample of `nreq` requests: the FP32 stencils served by per-request streams and by
    per-module batches (continuous batching: one launch per stage over every admitted solve
    of a module, CUDA-graph steps; solves attach and detach without moving the others, and
    the cost of those calls is reported), and, on a stated subset (the first `fp64_subset`
    requests of side <= 64 in arrival order), the plain FP64 per-solve path beside both FP32
    forms. Each form reports
    p50/p99 latency (completion - arrival), aggregate zone-updates/s and the largest number
    of co-resident solves."""
    from paper_2607_19277_gb300 import serving
    budget = int(budget_gb * 2 ** 30)

    def stream():
        return serving.request_stream(nreq, rate=rate, sides=(32, 64, 128, 256), steps=(50, 500))

    out = {"workload": "%d requests, Poisson mean %g/s, physics hd/mhd/srhd, sides 32-256, 50-500 steps, "
                       "budget %g GB" % (nreq, rate, budget_gb)}
    out["fp32"] = serving.Server(budget, real_bytes=4, steps_per_poll=4).run(stream()).summary()
    out["fp32_batched"] = serving.BatchedServer(budget, real_bytes=4).run(stream()).summary()
    ids = [r.rid for r in stream() if r.side <= 64][:fp64_subset]

    def subset():
        return [r for r in stream() if r.rid in ids]
    sub = {"requests": ids, "note": "the same requests (arrival times kept) on each path"}
    sub["fp64_plain"] = serving.Server(budget, real_bytes=8, steps_per_poll=4).run(subset()).summary()
    sub["fp32"] = serving.Server(budget, real_bytes=4, steps_per_poll=4).run(subset()).summary()
    sub["fp32_batched"] = serving.BatchedServer(budget, real_bytes=4).run(subset()).summary()
    out["subset"] = sub
    # a burst of small solves (sides 32-64, arrivals at a mean 2000/s so that the servers'
    # capacity and not the arrival process sets the time), where one launch per stage over
    # many solves matters most against a launch sequence per solve
    small = {"workload": "%d requests, Poisson mean 2000/s (a burst), sides 32-64, 50-500 steps" % nreq}

    def small_stream():
        return serving.request_stream(nreq, rate=2000.0, sides=(32, 48, 64), steps=(50, 500),
                                      seed=serving.W.SEED_BASE + 15)
    small["fp32"] = serving.Server(budget, real_bytes=4, steps_per_poll=4).run(small_stream()).summary()
    small["fp32_batched"] = serving.BatchedServer(budget, real_bytes=4).run(small_stream()).summary()
    out["small_solves"] = small
    return out


def _oracle_mhd(side):
    from oracle import Config, Solver
    from paper_2607_19277_gb300 import workloads as W
    sp = spec()
    sp["base_blocks"] = (side // 16,) * 3
    s = Solver(Config(**sp))
    s.set_state(W.orszag_tang_3d(side))
    return s


def _oracle_worker(side, steps, barrier, q):
    """One spawned process of the all-cores run: the oracle's MHD sample, timed from a start
    barrier shared by all processes (monotonic clock, common to the processes of a host)."""
    s = _oracle_mhd(side)
    barrier.wait(timeout=900)
    t0 = time.monotonic()
    for _ in range(steps):
        s.step()
    q.put((t0, time.monotonic()))


def cpu_baseline(seconds_budget=12.0):
    """The FP64 oracle as it stands, on the host cores:
    * value: the MHD scheme of the workload on a 64^3 periodic box (64 blocks) of the same
      initial-condition family, whole SSPRK3 steps for about `seconds_budget` s, 1 thread;
    * all_cores: the same scheme on 32^3 boxes, one independent box per process on every
      host core (up to 16), aggregate zone-updates/s over the common wall time;
    * config1_full: the 64^3 HD Sod problem (4x4x4 blocks, minmod, HLL, SSPRK2, CFL 0.4)
      for its full 20 steps, 1 thread;
    * config3_sample / config4_sample: two steps of a refined Sedov problem and of one SRHD
      solve of the batch's family, 1 thread."""
    import multiprocessing as mp
    from oracle import Config, Solver
    from paper_2607_19277_gb300 import workloads as W
    s = _oracle_mhd(64)
    t0 = time.perf_counter()
    n = 0
    while True:
        s.step()
        n += 1
        if (time.perf_counter() - t0 > seconds_budget and n >= 2) or n >= 30:
            break
    el = time.perf_counter() - t0
    out = {"value": 64 * 4096 * 3 * n / el, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "mhd_glm OT 64^3 periodic (64 blocks), %d SSPRK3 steps in %.1f s, numpy FP64 on 1 "
                     "host thread" % (n, el)}
    del s
    # config 1 in full
    c1 = Solver(Config(physics="hd", limiter="minmod", flux="hll", rk=2, cfl=0.4, base_blocks=(4, 4, 4),
                       bc=("outflow", "outflow", "periodic", "periodic", "periodic", "periodic")))
    c1.set_state(W.sod_x)
    t0 = time.perf_counter()
    for _ in range(20):
        c1.step(c1.cfl_dt())
    el1 = time.perf_counter() - t0
    out["config1_full"] = {"value": 64 ** 3 * 2 * 20 / el1, "unit": UNIT, "seconds": el1, "cores": 1,
                           "workload": "hd sod 64^3 (4x4x4 blocks), minmod, hll, ssprk2, cfl 0.4, 20 steps, fp64"}
    del c1
    # bounded samples of the refined Sedov problem (config 3's scheme, base 32^3, three
    # levels after the initial refinement) and of one SRHD solve of the batch (config 4's
    # scheme, 32^3), a few steps each
    c3 = Solver(Config(physics="hd", limiter="minmod", flux="hll", rk=2, cfl=0.4, base_blocks=(2, 2, 2),
                       xmin=(-0.5,) * 3, xmax=(0.5,) * 3, bc=("outflow",) * 6, max_level=3,
                       refine_vars=(0, 4), refine_weights=(0.5, 0.5), refine_tol=0.2))
    c3.set_state(W.sedov(r0=0.06))
    for _ in range(2):
        c3.regrid(init=True)
    nleaf = len(c3.leaves)
    t0 = time.perf_counter()
    for _ in range(2):
        c3.step()
    el3 = time.perf_counter() - t0
    out["config3_sample"] = {"value": nleaf * 4096 * 2 * 2 / el3, "unit": UNIT, "seconds": el3, "cores": 1,
                             "workload": "hd sedov, base 32^3, max level 3 (%d leaves), minmod, hll, ssprk2, "
                                         "2 steps, fp64" % nleaf}
    del c3
    c4 = Solver(Config(physics="srhd", limiter="minmod", flux="tvdlf", rk=2, gamma=4.0 / 3.0, cfl=0.4,
                       base_blocks=(2, 2, 2)))
    c4.set_state(W.srhd_shells(20260005, 32, lorentz_max=2.0, p_amb=0.1, smooth=True))
    t0 = time.perf_counter()
    for _ in range(2):
        c4.step()
    el4 = time.perf_counter() - t0
    out["config4_sample"] = {"value": 32 ** 3 * 2 * 2 / el4, "unit": UNIT, "seconds": el4, "cores": 1,
                             "workload": "one srhd solve 32^3 of the batch's family, tvdlf, minmod, ssprk2, "
                                         "2 steps, fp64 newton"}
    del c4
    # every host core, independent boxes (the oracle's work splits over blocks/solves)
    nproc = max(1, min(os.cpu_count() or 1, 16))
    steps = 6
    try:
        ctx = mp.get_context("spawn")
        bar = ctx.Barrier(nproc)
        q = ctx.Queue()
        ps = [ctx.Process(target=_oracle_worker, args=(32, steps, bar, q)) for _ in range(nproc)]
        for p in ps:
            p.start()
        spans = [q.get(timeout=900) for _ in ps]
        for p in ps:
            p.join(timeout=60)
        wall = max(e for _, e in spans) - min(b for b, _ in spans)
        out["all_cores"] = {"value": nproc * 8 * 4096 * 3 * steps / wall, "unit": UNIT, "cores": nproc,
                            "kind": "oracle",
                            "sample": "%d processes, each a mhd_glm OT 32^3 periodic box (8 blocks), %d SSPRK3 "
                                      "steps, numpy FP64" % (nproc, steps)}
    except Exception as e:   # the single-thread figure stands on its own
        out["all_cores"] = {"error": str(e)}
    return out


def reference_arm(args):
    """--impl reference: the oracle timed as the reference, same workload family/metric."""
    from oracle import Config, Solver
    from paper_2607_19277_gb300 import workloads as W
    sp = spec()
    sp["base_blocks"] = (2, 2, 2)
    s = Solver(Config(**sp))
    s.set_state(W.orszag_tang_3d(32))
    for _ in range(args.warmup):
        s.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step()
    el = time.perf_counter() - t0
    zones = 8 * 4096 * 3 * args.steps
    v = zones / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "32^3 periodic sub-box (8 blocks) per step",
                       "parallelism": "replicas"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "mhd_glm OT 32^3 periodic (8 blocks), one SSPRK3 step per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def summary_of(line):
    """The headline numbers of every leg in one short object, printed last in the line."""
    def get(d, *path):
        for p in path:
            if not isinstance(d, dict) or p not in d:
                return None
            d = d[p]
        return d
    out = {"fp32_value": line.get("value"), "fp32_hbm_frac": get(line, "roofline", "frac"),
           "fp32_alu_frac": get(line, "roofline", "alu", "frac"),
           "fp32_stage_launch_ms": get(line, "roofline", "launch_ms"),
           "fp64_value": get(line, "fp64", "value"), "fp64_alu_frac": get(line, "fp64", "roofline", "frac"),
           "e2e": get(line, "e2e", "value"),
           "fp32_max_rel_l1_vs_fp64": get(line, "error_vs_fp64", "max_rel_l1_rho_m_e_B"),
           "fp32_psi_rel_l1_vs_fp64": get(line, "error_vs_fp64", "rel_l1", "psi"),
           "paper_scheme_hd_fp32": get(line, "paper_scheme_hd", "fp32", "value"),
           "paper_scheme_hd_fp64": get(line, "paper_scheme_hd", "fp64", "value"),
           "batched_srhd_fp32": get(line, "batched", "value"),
           "batched_srhd_fp64_plain": get(line, "batched", "fp64_plain_per_solve", "value"),
           "sedov_5level_fp32": get(line, "sedov_5level", "fp32", "value"),
           "sedov_5level_fp64": get(line, "sedov_5level", "fp64", "value"),
           "serving_fp32_batched_p99_s": get(line, "serving", "fp32_batched", "latency_p99_s"),
           "serving_fp32_batched_value": get(line, "serving", "fp32_batched", "zone_updates_per_s"),
           "serving_fp32_streams_p99_s": get(line, "serving", "fp32", "latency_p99_s"),
           "serving_fp32_streams_value": get(line, "serving", "fp32", "zone_updates_per_s"),
           "serving_max_concurrent": get(line, "serving", "fp32_batched", "max_concurrent"),
           "serving_membership_share": get(line, "serving", "fp32_batched", "membership",
                                           "membership_share_of_wall"),
           "serving_small_fp32_streams_value": get(line, "serving", "small_solves", "fp32", "zone_updates_per_s"),
           "serving_small_fp32_batched_value": get(line, "serving", "small_solves", "fp32_batched",
                                                   "zone_updates_per_s"),
           "serving_small_fp32_batched_p99_s": get(line, "serving", "small_solves", "fp32_batched",
                                                   "latency_p99_s"),
           "serving_small_fp32_streams_p99_s": get(line, "serving", "small_solves", "fp32", "latency_p99_s"),
           "serving_subset_fp64_plain_p99_s": get(line, "serving", "subset", "fp64_plain", "latency_p99_s"),
           "serving_subset_fp64_plain_value": get(line, "serving", "subset", "fp64_plain", "zone_updates_per_s"),
           "serving_subset_fp32_batched_value": get(line, "serving", "subset", "fp32_batched",
                                                    "zone_updates_per_s"),
           "cpu_oracle_1core": get(line, "cpu_baseline", "value")}
    return {k: v for k, v in out.items() if v is not None}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-paper-scheme", action="store_true")
    ap.add_argument("--no-cooling", action="store_true")
    ap.add_argument("--no-ffhd", action="store_true")
    ap.add_argument("--no-sedov", action="store_true")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            reference_arm(args)
        return
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        from paper_2607_19277_gb300 import build
        build.build()
    if world > 1:
        torch.distributed.barrier()
    args.warmup = max(args.warmup, 3)
    r32 = run_gpu(4, args.steps, args.warmup, rank, world, local)
    steps64 = max(2, min(args.steps // 4, 20))
    r64 = None if args.no_fp64 else run_gpu(8, steps64, args.warmup, rank, world, local)

    hbm, peak_kind = peaks()

    def summarize(r, w, steps):
        zu, t_ms = replica_throughput(r["zones"], 3, steps, r["total_ms"], world)
        ms_step = t_ms / steps
        bpz = algorithmic_bytes_per_zone(r["nvar"], w, 3)
        launch_ms = r["stage_ms"] / max(1, r["stage_launches"])
        achieved = bpz * r["zones"] / (launch_ms / 1e3) / 1e9
        e2e, _ = replica_throughput(r["zones"], 3, steps, 1e3 * r["e2e_s"], world)
        ps = sorted(r["per_step"])
        flops = MHD_HLL_VL_FLOPS * r["zones"] / (launch_ms / 1e3) / 1e12
        mhz = (r["clocks"] or {}).get("sm_mhz") or 2070.0
        peak_alu = alu_peak_tflops(FP32_LANES if w == 4 else FP64_LANES, mhz)
        return dict(value=zu, ms_per_step=ms_step, bytes_per_zone=bpz, launch_ms=launch_ms,
                    zps=r["zones"] / (launch_ms / 1e3), achieved=achieved, tflops=flops, peak_alu=peak_alu, mhz=mhz,
                    e2e=e2e, p50=ps[len(ps) // 2],
                    p99=ps[min(len(ps) - 1, int(math.ceil(0.99 * len(ps))) - 1)],
                    stage_share=r["stage_ms"] / max(1e-9, r["total_ms"]),
                    launches=r["total_launches"], clocks=r["clocks"])

    s32 = summarize(r32, 4, args.steps)
    s64 = summarize(r64, 8, steps64) if r64 else None
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    steps = args.steps
    traffic = stage_traffic()
    line = {
        "metric": METRIC, "value": s32["value"], "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": s32["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": N_SIDE ** 3, "blocks": (N_SIDE // 16) ** 3,
                   "stages_per_step": 3, "dt": "on-device CFL reduction",
                   "l2": "state 604 MB (fp32) / 1.2 GB (fp64) per buffer > 129 MB L2, no flush",
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": {"bound": "hbm", "achieved": s32["achieved"], "peak": hbm, "unit": "GB/s",
                     "frac": s32["achieved"] / hbm, "traffic": traffic,
                     "traffic_unit": "bytes per launch (ncu dram__bytes_read+write, mean of the 3 stages)",
                     "algorithmic_bytes_per_launch": s32["bytes_per_zone"] * N_SIDE ** 3,
                     "bytes_per_zone_update": s32["bytes_per_zone"],
                     "peak_kind": peak_kind + " hbm_gbs (MEASURED_PEAKS.json)",
                     "kernel": "stage_kernel<MhdPhys,float,vanleer,hll>",
                     "launch_ms": s32["launch_ms"],
                     "stage_kernel_share_of_step": s32["stage_share"],
                     "alu": {"achieved": s32["tflops"], "peak": s32["peak_alu"], "unit": "TFLOP/s",
                             "frac": s32["tflops"] / s32["peak_alu"],
                             "flops_per_zone_update": MHD_HLL_VL_FLOPS,
                             "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x %.0f MHz" % s32["mhz"],
                             "note": "the kernel is bound by FP32 instruction issue, not by HBM"}},
        "hbm_roofline": {"bound": "hbm", "achieved": s32["achieved"], "peak": hbm, "unit": "GB/s",
                         "frac": s32["achieved"] / hbm, "traffic": traffic,
                         "bytes_per_zone_update": s32["bytes_per_zone"],
                         "peak_kind": peak_kind + " hbm_gbs",
                         "ghost_inflated": {
                             "bytes_per_zone_update": ghost_inflated_bytes_per_zone(9, 4, 3),
                             "achieved": ghost_inflated_bytes_per_zone(9, 4, 3) * s32["zps"] / 1e9,
                             "frac": ghost_inflated_bytes_per_zone(9, 4, 3) * s32["zps"] / 1e9 / hbm,
                             "note": "equivalent rate of a 20^3 ghost-cell storage scheme at this "
                                     "stage-launch zone-update rate; not this build's traffic"}},
        "e2e": {"value": s32["e2e"], "unit": UNIT,
                "h2d_bytes_per_step": r32["state_bytes"] / steps,
                "d2h_bytes_per_step": r32["state_bytes"] / steps + 8 * (1 + 9),
                "loop": "set_state_blocks(pinned) + per step (step with device dt, conserved_sums read back) + get_state(pinned)"},
        "gpu_launches": s32["launches"],
        "step_latency_ms": {"p50": s32["p50"], "p99": s32["p99"]},
        "clocks": s32["clocks"],
    }
    if s64:
        line["fp64"] = {"value": s64["value"], "ms_per_step": s64["ms_per_step"], "dtype": "f64",
                        "roofline": {"bound": "alu", "achieved": s64["tflops"], "peak": s64["peak_alu"],
                                     "unit": "TFLOP/s", "frac": s64["tflops"] / s64["peak_alu"],
                                     "flops_per_zone_update": MHD_HLL_VL_FLOPS,
                                     "peak_kind": "derived: 152 SMs x 2 FP64 lanes x 2 x %.0f MHz" % s64["mhz"],
                                     "launch_ms": s64["launch_ms"]},
                        "hbm_roofline": {"bound": "hbm", "achieved": s64["achieved"], "peak": hbm,
                                         "unit": "GB/s", "frac": s64["achieved"] / hbm,
                                         "bytes_per_zone_update": s64["bytes_per_zone"]},
                        "e2e": s64["e2e"], "step_latency_ms": {"p50": s64["p50"], "p99": s64["p99"]},
                        "gpu_launches": s64["launches"], "clocks": s64["clocks"]}
    if not args.no_batched:
        try:
            line["batched"] = run_batched(max(4, min(args.steps // 20, 10)), args.warmup)
            line["batched"]["workload"] = ("256 SRHD solves 32^3-128^3 (16^3 blocks), one seeded shell each "
                                           "(Gaussian profile, 2 cells wide) with Lorentz factor U[1, 10], TVDLF "
                                           "minmod SSPRK2")
        except Exception as e:   # report, do not lose the headline line
            line["batched"] = {"error": str(e)}
    if not args.no_batched:
        try:
            line["batched_amr"] = run_batched_amr()
        except Exception as e:
            line["batched_amr"] = {"error": str(e)}
    if not args.no_paper_scheme:
        try:
            line["paper_scheme_hd"] = run_paper_scheme()
        except Exception as e:
            line["paper_scheme_hd"] = {"error": str(e)}
    if not args.no_cooling:
        try:
            line["cooling_mhd"] = run_cooling()
        except Exception as e:
            line["cooling_mhd"] = {"error": str(e)}
    if not args.no_sedov:
        try:
            line["sedov_5level"] = run_sedov_5level()
        except Exception as e:
            line["sedov_5level"] = {"error": str(e)}
    if not args.no_ffhd:
        try:
            line["ffhd"] = run_ffhd()
        except Exception as e:
            line["ffhd"] = {"error": str(e)}
    if not args.no_serving:
        try:
            line["serving"] = run_serving()
        except Exception as e:
            line["serving"] = {"error": str(e)}
    if not args.no_fp64 and world == 1:
        try:
            line["error_vs_fp64"] = run_error_vs_fp64(min(args.warmup + steps, 50))
        except Exception as e:
            line["error_vs_fp64"] = {"error": str(e)}
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline()
    line["summary"] = summary_of(line)
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
