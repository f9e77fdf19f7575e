#!/usr/bin/env python3
"""Throughput of the AMR level advance on GB300: leaf cell-updates/s.

Workload: the Sedov blast on a static graded octree, levels 7-10 (128^3 base
cells, nested refined balls of radius 0.12 / 0.06 / 0.03 around the centre,
about 2.4 M leaf cells), gamma = 5/3, synthetic seeded input.  One step is
one coarse time step of the level-by-level W-cycle through the C ABI
(amr_advance): device CFL reduction, then every level step (ghosts,
primitives, predictor, HLLC fluxes, update, reflux, restriction) with
2^(l-7) substeps per level; the static mesh's hash table, neighbour array
and ghost cache are built once, at creation.
The unit of work is one leaf cell advanced by one level step.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "sedov_l7-10_static_nested_balls"
L2_FLUSH_BYTES = 256 << 20
WORD = {8: 8, 4: 4}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", type=int, default=8, choices=[4, 8],
                    help="state precision of the headline value (the other is reported beside it)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=6,
                    help="coarse steps of the oracle in the CPU baseline (about 2 s each on one core)")
    ap.add_argument("--cpu-all-core-steps", type=int, default=2,
                    help="coarse steps of each per-core oracle replica in the all-core CPU "
                         "baseline (0: skip it)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 512-mesh batched ensemble measurement")
    ap.add_argument("--batched-members", type=int, default=512)
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-loop sweep")
    ap.add_argument("--no-poisson", action="store_true",
                    help="skip the multigrid V-cycle measurement")
    ap.add_argument("--no-adaptive", action="store_true",
                    help="skip the adaptive run (regrid before every coarse step)")
    ap.add_argument("--no-unigrid", action="store_true",
                    help="skip the uniform 256^3 blast (Godunov level step and coarse step)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the per-cell vs fused (nsubgrid) level-step comparison")
    ap.add_argument("--no-cic", action="store_true",
                    help="skip the Cloud-in-Cell particle deposition measurement")
    ap.add_argument("--cic-grid", type=int, default=512,
                    help="grid cells per axis of the deposition measurement (N_part = N_grid)")
    ap.add_argument("--profile-cic", type=int, default=0,
                    help="profiling mode: one sort and one deposit of each algorithm of n^3 "
                         "cosmological particles on the n^3 grid (--precision), then exit")
    ap.add_argument("--serving-requests", type=int, default=48)
    ap.add_argument("--no-other-precision", action="store_true",
                    help="run only --precision (skip the other precision's pass)")
    ap.add_argument("--tile", type=int, default=0,
                    help="work-tile size of every handle (0: autotune at the first step)")
    ap.add_argument("--schedule", type=int, default=-1,
                    help="1 persistent grids, 0 one tile per block, -1 autotune")
    ap.add_argument("--nsubgrid", type=int, default=-1,
                    help="level-step kernel: 0 per-cell passes, 1/2/4 fused kernel, -1 autotune")
    ap.add_argument("--planar", type=int, default=-1,
                    help="fused kernel: 0 cube staging (rock), 1 planar sweep (paper kernel), -1 default")
    ap.add_argument("--profile-poisson", type=int, default=0,
                    help="profiling mode: one multigrid V-cycle on a periodic 2^L grid, then exit")
    ap.add_argument("--profile-unigrid", type=int, default=0,
                    help="profiling mode: the blast on a uniform 2^L grid, one eager level step "
                         "(one launch of each level-step kernel), then exit")
    ap.add_argument("--profile-level", type=int, default=0,
                    help="profiling mode: build the mesh and run one eager level step of this "
                         "level (one launch of each level-step kernel), then exit")
    return ap.parse_args()


def dist_env():
    from paper_2607_20704_gb300 import dist
    return dist.env()


def work_per_step(info, levelmin=None):
    """Leaf cell-updates of one coarse step (level l runs 2^(l-levelmin)
    times), counted by the library over every member of the handle."""
    return int(info["work_per_step"])


# -- clocks ----------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            out, _ = self.proc.communicate(timeout=10)
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons, pw = [], [], set(), []
        for line in getattr(self, "lines", []):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                  "sw_power_cap"), f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(pw) if pw else None}


# -- roofline bookkeeping -----------------------------------------------------------
def kernel_units(info_levels, levelmin):
    """Per kernel: units processed in one coarse step (each level l runs
    2^(l-levelmin) times): local cells (real + ghost), real cells, ghost
    octs, real octs above levelmin."""
    loc = real = ghost = fine = 0
    for l in range(levelmin, 16):
        n, nc = info_levels["level_octs"][l], info_levels["level_cache"][l]
        if not n:
            continue
        reps = 2 ** (l - levelmin)
        loc += reps * 8 * (n + nc)
        real += reps * 8 * n
        ghost += reps * nc
        if l > levelmin:
            fine += reps * n
    return loc, real, ghost, fine


def kernel_traffic(info, levelmin, w, fused):
    """Algorithmic bytes of one coarse step per kernel: its inputs read once
    and its outputs written once (w = bytes per word).
      FP64 kernels (one pass each):
      prim        U in, W out                       10 w per real+ghost cell
      predict     W in, (W*, dW) out                25 w per real+ghost cell
      flux        (W*, dW) in, three fluxes out     35 w per real+ghost cell
      update      fluxes in (15 w), U in/out        25 w + 4 B per real cell
      FP32 kernels (fused):
      predict     U in, (W*, dW) out                25 w per real+ghost cell
      flux        (W*, dW) in (20 w per real+ghost cell), U in/out + slot
                  index (10 w + 4 B per real cell)
      both:
      prolong     7 sources in, 8 ghosts out        75 w per ghost oct
      reflux_restrict  24 slots + R in/out per ghost oct (130 w), 8 children
                  in + father out per real oct above levelmin (45 w)
    """
    loc, real, ghost, fine = kernel_units(info, levelmin)
    out = {"prolong": ghost * 75 * w, "reflux_restrict": ghost * 130 * w + fine * 45 * w}
    if fused:
        out["predict"] = loc * 25 * w
        out["flux"] = loc * 20 * w + real * (10 * w + 4)
    else:
        out["prim"] = loc * 10 * w
        out["predict"] = loc * 25 * w
        out["flux"] = loc * 35 * w
        out["update"] = real * (25 * w + 4)
    return out


# FP64 flops (2 per FMA) per real cell of the FP64 flux kernel (three HLLC
# faces), and DRAM bytes per cell of the flux kernels, from one ncu capture
# of the level-7 launch of the benchmark mesh (ncu: FP64 instruction counts,
# dram__bytes_read.sum + dram__bytes_write.sum)
FLUX_FP64_FLOPS_PER_CELL = 289.8
FLUX_DRAM_BYTES_PER_CELL = {8: 272.7, 4: 125.8}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def flush_l2(buf):
    buf.zero_()


# -- our arm ----------------------------------------------------------------------
LAUNCH = {"tile": 0, "schedule": -1, "nsubgrid": -1, "planar": -1}  # from --tile / --schedule / --nsubgrid / --planar
_STREAM = []


def bench_stream():
    """One CUDA stream for every handle of the run: a handle created on a
    stream of its own after others have existed in the process was measured
    4-6 % slower (FP32), one reusing the stream (and its freed memory) not."""
    import torch
    if not _STREAM:
        _STREAM.append(torch.cuda.Stream())
    return _STREAM[0]

def run_precision(prob, precision, steps, warmup, torch, device, flush, kernels=True):
    from paper_2607_20704_gb300 import amr
    mesh = amr.Mesh(*prob.mesh_args(), **prob.params(), precision=precision, stream=bench_stream(),
                    **LAUNCH)
    info = mesh.info()
    upd = work_per_step(info, prob.levelmin)
    st = mesh.stream
    for _ in range(warmup):
        mesh.advance(1)
        with torch.cuda.stream(st):
            flush_l2(flush)
    torch.cuda.synchronize(device)
    info = mesh.info()  # after the autotuner has picked tile and schedule
    mesh_tile, mesh_sched = info["tile"], info["schedule"]
    launches0 = info["kernel_launches"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    from paper_2607_20704_gb300 import dist
    dist.barrier()
    torch.cuda.synchronize(device)
    wall0 = time.perf_counter()
    for e0, e1 in ev:
        e0.record(st)
        mesh.advance(1)
        e1.record(st)
        with torch.cuda.stream(st):
            flush_l2(flush)
    torch.cuda.synchronize(device)
    wall = time.perf_counter() - wall0
    dist.barrier()
    ms = sum(e0.elapsed_time(e1) for e0, e1 in ev)
    launches = mesh.info()["kernel_launches"] - launches0
    res = {"ms": ms, "wall_s": wall, "updates_per_step": upd, "launches": launches, "info": info}
    mesh.close()
    if kernels:
        # per-kernel device time: same K steps, each launch bracketed by CUDA
        # events on the library's stream (eager launches, no graph)
        m2 = amr.Mesh(*prob.mesh_args(), **prob.params(), precision=precision,
                      tile=mesh_tile, schedule=mesh_sched, nsubgrid=info["nsubgrid"],
                      planar=info["planar"], stream=bench_stream())
        for _ in range(warmup):
            m2.advance(1)
        m2.sync()
        m2.set_timing(True)
        for _ in range(steps):
            m2.advance(1)
            with torch.cuda.stream(m2.stream):
                flush_l2(flush)
        res["kernels"] = m2.read_timing()
        m2.close()
    return res


def run_variants(prob, steps, torch, device, flush):
    """The level-step kernels side by side on the workload: the per-cell
    passes (autotuned tile and schedule) and the fused shared-memory kernels,
    cube staging (rock; nsubgrid 1, 2, and 4 in FP32) and planar sweep (paper
    kernel; nsubgrid 1, 2, 4), each schedule; median coarse-step time of
    `steps` graph-replayed steps, L2 flushed between them."""
    from paper_2607_20704_gb300 import amr
    out = {}
    for prec in (8, 4):
        rows = []
        shapes = [dict(nsubgrid=0)]
        for planar in (0, 1):
            for ns in ((1, 2) if (prec == 8 and planar == 0) else (1, 2, 4)):
                shapes += [dict(nsubgrid=ns, planar=planar, tile=128, schedule=sc) for sc in (0, 1)]
        for shp in shapes:
            m = amr.Mesh(*prob.mesh_args(), **prob.params(), precision=prec, stream=bench_stream(), **shp)
            upd = work_per_step(m.info(), prob.levelmin)
            st = m.stream
            for _ in range(3):
                m.advance(1)
            ts = []
            for _ in range(steps):
                with torch.cuda.stream(st):
                    flush_l2(flush)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                m.advance(1)
                e1.record(st)
                torch.cuda.synchronize(device)
                ts.append(e0.elapsed_time(e1))
            inf = m.info()
            ms = float(np.median(ts))
            rows.append({"nsubgrid": inf["nsubgrid"], "planar": inf["planar"], "tile": inf["tile"],
                         "schedule": inf["schedule"],
                         "ms_per_step": round(ms, 4), "cell_updates_per_s": upd / (ms * 1e-3)})
            m.close()
        out["fp64" if prec == 8 else "fp32"] = rows
    return out


def unigrid_problem(level):
    """The blast on a uniform 2^level grid: unit density at rest, pressure
    1e-5 outside a ball of radius 2 cells that holds unit energy."""
    from paper_2607_20704_gb300 import inputs
    n = 1 << level
    r0 = 2.0 / n

    def fn(x, y, z):
        r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2
        p = np.where(r2 < r0 * r0, (5.0 / 3.0 - 1.0) / (4.0 / 3.0 * np.pi * r0 ** 3), 1e-5)
        zero = 0.0 * x
        return 1.0 + zero, zero, zero, zero, p
    return inputs.uniform_grid(level, fn, gamma=5.0 / 3.0)


def run_unigrid(level, steps, torch, device):
    """The blast on a uniform 2^level grid (one level, no refinement): the
    Godunov level step alone (amr_step_level: primitives, predictor, HLLC
    fluxes, update) and the whole coarse step (re-index, time step, level
    step), median over `steps`, each precision.  The paper quotes its
    unigrid Sedov rates this way (rock kernel, H200, FP32)."""
    from paper_2607_20704_gb300 import amr
    n = 1 << level
    prob = unigrid_problem(level)
    out = {"grid": f"{n}^3 cells, one level", "cells": n ** 3}
    for prec in (8, 4):
        m = amr.Mesh(*prob.mesh_args(), **prob.params(), precision=prec, stream=bench_stream())
        st = m.stream
        m.advance(3, sync=True)
        dt = m.cfl_dt() * 1e-3
        ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        lv, cs = [], []
        for _ in range(steps):
            e0, e1 = ev()
            e0.record(st)
            m.step_level(level, dt)
            e1.record(st)
            torch.cuda.synchronize(device)
            lv.append(e0.elapsed_time(e1))
            e0, e1 = ev()
            e0.record(st)
            m.advance(1)
            e1.record(st)
            torch.cuda.synchronize(device)
            cs.append(e0.elapsed_time(e1))
        inf = m.info()
        lms, cms = float(np.median(lv)), float(np.median(cs))
        out["fp64" if prec == 8 else "fp32"] = {
            "level_step_ms": round(lms, 4), "level_step_cell_updates_per_s": n ** 3 / (lms * 1e-3),
            "coarse_step_ms": round(cms, 4), "coarse_step_cell_updates_per_s": n ** 3 / (cms * 1e-3),
            "tile": inf["tile"], "schedule": inf["schedule"], "nsubgrid": inf["nsubgrid"]}
        m.close()
        # each level-step kernel on its own: the per-cell passes and the rock
        # kernel with nsubgrid 2 and 4 (fixed launch shapes, no autotuning)
        kern = []
        for ns, tile, sched in ((0, 256, 0), (2, 128, 0), (4, 128, 0)):
            m = amr.Mesh(*prob.mesh_args(), **prob.params(), precision=prec, stream=bench_stream(),
                         nsubgrid=ns, planar=0, tile=tile, schedule=sched)
            st = m.stream
            m.advance(1, sync=True)
            dt = m.cfl_dt() * 1e-3
            lv = []
            for _ in range(steps):
                e0, e1 = ev()
                e0.record(st)
                m.step_level(level, dt)
                e1.record(st)
                torch.cuda.synchronize(device)
                lv.append(e0.elapsed_time(e1))
            lms = float(np.median(lv))
            kern.append({"nsubgrid": ns, "planar": 0, "tile": tile, "schedule": sched,
                         "level_step_ms": round(lms, 4),
                         "level_step_cell_updates_per_s": n ** 3 / (lms * 1e-3)})
            m.close()
        out["fp64" if prec == 8 else "fp32"]["kernels"] = kern
    out["paper_context"] = ("H200, FP32 with fast math, unigrid Sedov, Godunov only: rock kernel "
                            "nsubgrid 4 0.09 ns per cell (11.1e9 /s), paper kernel 0.2 ns (5e9 /s)")
    return out


def run_e2e(prob, precision, steps, torch):
    """Same metric through the public API with host buffers.  Per step: the
    whole state (every level, mesh order) is uploaded from pinned host memory
    (amr_load_state_async), one coarse step runs (amr_advance), and the
    resulting state is read back into pinned host memory
    (amr_store_state_async); the copies of neighbouring steps overlap the
    compute on the handle's upload and download copy streams.  Two input and two output host
    buffers alternate.  Wall clock from the first upload to the last
    download's completion.  `serial` is the same loop with the synchronous
    per-level amr_write / amr_read calls (copies not overlapped)."""
    from paper_2607_20704_gb300 import amr
    mesh = amr.Mesh(*prob.mesh_args(), **prob.params(), precision=precision, stream=bench_stream(),
                    **LAUNCH)
    info = mesh.info()
    upd = work_per_step(info, prob.levelmin)
    levels = mesh.levels()
    n = mesh.state_octs()
    pin = lambda: torch.empty((5, 8 * n), dtype=torch.float64, pin_memory=True).numpy()
    ins, outs = [pin(), pin()], [pin(), pin()]
    for b in ins:
        b[:] = np.concatenate([mesh.read(l)[1] for l in levels], axis=1)
    nbytes = ins[0].nbytes

    def pipelined(k):
        mesh.load_state_async(ins[k % 2])
        mesh.advance(1)
        mesh.store_state_async(outs[k % 2])

    for k in range(2):
        pipelined(k)
    mesh.sync()
    t0 = time.perf_counter()
    for k in range(steps):
        pipelined(k)
    mesh.sync()
    dt = time.perf_counter() - t0
    # the synchronous path, level by level
    host = {}
    for l in levels:
        host[l] = torch.empty((5, 8 * mesh.num_octs(l)), dtype=torch.float64, pin_memory=True).numpy()
        mesh.read(l, out_U=host[l], keys=False)

    def serial():
        for l in levels:
            mesh.write(l, host[l])
        mesh.advance(1)
        for l in levels:
            mesh.read(l, out_U=host[l], keys=False)

    serial()
    t1 = time.perf_counter()
    for _ in range(steps):
        serial()
    ds = time.perf_counter() - t1
    mesh.close()
    return {"value": upd * steps / dt, "unit": "leaf cell-updates/s",
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "ms_per_step": 1e3 * dt / steps, "copies": "overlapped with the steps (upload and download copy streams)",
            "serial": {"value": upd * steps / ds, "ms_per_step": 1e3 * ds / steps,
                       "copies": "synchronous per-level amr_write / amr_read"}}


def run_batched(members, steps, warmup, torch, device, flush):
    """Leaf cell-updates/s of the seeded ensemble of independent Sod/Sedov
    meshes, all advanced by the same launches (one handle), FP64 and FP32."""
    from paper_2607_20704_gb300 import amr
    out = {"members": len(members), "octs": int(sum(p.n_oct for p in members)),
           "leaf_cells": int(sum(p.leaf_cells() for p in members))}
    for prec, name in ((8, "fp64"), (4, "fp32")):
        b = amr.Mesh.batch(members, precision=prec, stream=bench_stream())
        info = b.info()
        upd = int(info["work_per_step"])
        st = b.stream
        b.advance(warmup)
        torch.cuda.synchronize(device)
        info = b.info()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        l0 = info["kernel_launches"]
        for e0, e1 in ev:
            e0.record(st)
            b.advance(1)
            e1.record(st)
            with torch.cuda.stream(st):
                flush_l2(flush)
        torch.cuda.synchronize(device)
        ms = sum(e0.elapsed_time(e1) for e0, e1 in ev)
        info = b.info()
        out[name] = {"value": upd * steps / (ms * 1e-3), "ms_per_step": ms / steps,
                     "cell_updates_per_step": upd, "phases": info["phases"],
                     "tile": info["tile"], "schedule": "persistent" if info["schedule"] else "one tile per block",
                     "gpu_launches": info["kernel_launches"] - l0,
                     "device_gb": round(info["device_bytes"] / 1e9, 2)}
        b.close()
    return out


def run_adaptive(prob, precision, steps, torch, device):
    """The blast with its mesh following it: a regrid (relative jump of rho
    or p above 0.1, one-cell expansion) before every coarse step.  Regrids
    synchronise with the host, so both phases are timed on the wall clock
    around a device synchronisation."""
    from paper_2607_20704_gb300 import amr
    m = amr.Mesh(*prob.mesh_args(), **prob.params(), precision=precision, stream=bench_stream(),
                 refine_grad_rho=0.1, refine_grad_p=0.1, **LAUNCH)
    octs0 = m.info()["n_oct"]
    for _ in range(2):
        m.regrid()
        m.advance(1)
    torch.cuda.synchronize(device)
    t_regrid, t_step, upd, changes = [], [], 0, []
    for _ in range(steps):
        t0 = time.perf_counter()
        changes.append(m.regrid())
        torch.cuda.synchronize(device)
        t1 = time.perf_counter()
        upd += int(m.info()["work_per_step"])
        m.advance(1)
        torch.cuda.synchronize(device)
        t2 = time.perf_counter()
        t_regrid.append(1e3 * (t1 - t0))
        t_step.append(1e3 * (t2 - t1))
    # kernel time inside regrids that change the mesh (CUDA events around
    # every launch of the regrid, none in the steps between them)
    for _ in range(3):
        m.set_timing(True)
        m.regrid()
        m.sync()
        m.set_timing(False)
        m.advance(1)
    m.sync()
    kt = m.read_timing()
    ktot = sum(v[0] for v in kt.values()) or 1.0
    regrid_kernels = {k: {"ms_per_regrid": round(v[0] / 3, 4), "share": round(v[0] / ktot, 4)}
                      for k, v in sorted(kt.items(), key=lambda kv: -kv[1][0])[:8]}
    inf = m.info()
    m.close()
    total_s = 1e-3 * (sum(t_regrid) + sum(t_step))
    return {"steps": steps, "criterion": "relative jump of rho or p to a face neighbour > 0.1, "
            "expand 1, regrid before every coarse step",
            "cell_updates_per_s": upd / total_s,
            "regrid_ms_median": round(statistics.median(t_regrid), 3),
            "step_ms_median": round(statistics.median(t_step), 3),
            "regrid_share": round(sum(t_regrid) / (sum(t_regrid) + sum(t_step)), 4),
            "octs_start": int(octs0), "octs_end": int(inf["n_oct"]),
            "leaf_cells_end": int(inf["n_leaf_cells"]),
            "octs_created_per_regrid": round(float(np.mean([c[0] for c in changes])), 1),
            "octs_removed_per_regrid": round(float(np.mean([c[1] for c in changes])), 1),
            "regrid_kernel_ms": round(ktot / 3, 4), "regrid_kernels": regrid_kernels}


def run_poisson(level, cycles, torch, device):
    """Multigrid V-cycles on a periodic 2^level grid holding a lognormal
    density (the cosmology-shaped configuration's base level): cell-updates
    per V-cycle per second (cells of the grid per V-cycle over its time, the
    paper's unit for the solver; one call of `cycles` V-cycles including the
    density gather and the potential scatter, no residual norms), residual
    reduction per V-cycle (from a separate call), and the kernel breakdown."""
    from paper_2607_20704_gb300 import amr
    rng = np.random.default_rng(7)
    n = 1 << level
    g, _ = inputs_gaussian(n, rng)
    rho_b = np.exp(g - 0.5 * 1.5 ** 2)

    def fn(x, y, z):
        bx = np.minimum((x * n).astype(np.int64), n - 1)
        by = np.minimum((y * n).astype(np.int64), n - 1)
        bz = np.minimum((z * n).astype(np.int64), n - 1)
        zero = 0.0 * x
        return rho_b[bx, by, bz], zero, zero, zero, 1.0 + zero
    from paper_2607_20704_gb300 import inputs
    prob = inputs.uniform_grid(level, fn)
    m = amr.Mesh(*prob.mesh_args(), **prob.params(), stream=bench_stream())
    st = m.stream
    res = m.poisson(1.0, 6)  # warm-up (allocates the hierarchy); convergence
    torch.cuda.synchronize(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    m.poisson(1.0, cycles, residuals=False)
    e1.record(st)
    torch.cuda.synchronize(device)
    ms = e0.elapsed_time(e1)
    m.set_timing(True)
    m.poisson(1.0, 2, residuals=False)
    kt = m.read_timing()
    m.set_timing(False)
    m.close()
    cells = n ** 3
    rates = res[1:] / res[:-1]
    ktot = sum(v[0] for v in kt.values()) or 1.0
    return {"grid": f"{n}^3 periodic", "cells": cells, "vcycles": cycles,
            "ms_per_vcycle": round(ms / cycles, 4),
            "cell_updates_per_s": cells * cycles / (ms * 1e-3),
            "residual_reduction_per_vcycle": round(float(np.median(rates)), 4),
            "smoother": "red-black Gauss-Seidel, 2 + 2 sweeps; restriction 1/8; trilinear prolongation",
            "kernels": {k: round(v[0] / ktot, 4) for k, v in sorted(kt.items(), key=lambda kv: -kv[1][0])}}


def run_poisson_levels(cycles, torch, device):
    """The potential of every level of the cosmology-shaped mesh (levels 8-11,
    Sec. 5: the base level's periodic solve, then each refined level from its
    father cells' values with Dirichlet data from the level below):
    cell-updates per V-cycle per second over all levels' cells (one call of
    `cycles` V-cycles per level, no residual norms), the per-level cell counts
    and residual reductions, and the first call's wall time (it also builds
    the level hierarchies' tables on the device)."""
    import time
    from paper_2607_20704_gb300 import amr, inputs
    prob = inputs.lognormal()
    m = amr.Mesh(*prob.mesh_args(), **prob.params(), stream=bench_stream())
    st = m.stream
    t0 = time.perf_counter()
    res = m.poisson_levels(1.0, cycles)  # builds the tables; convergence
    torch.cuda.synchronize(device)
    build_s = time.perf_counter() - t0
    m.poisson_levels(1.0, cycles, residuals=False)
    torch.cuda.synchronize(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    m.poisson_levels(1.0, cycles, residuals=False)
    e1.record(st)
    torch.cuda.synchronize(device)
    ms = e0.elapsed_time(e1)
    cells = {l: 8 * m.num_octs(l) for l in res}
    total = sum(cells.values())
    m.close()
    return {"mesh": "lognormal levels 8-11", "vcycles_per_level": cycles, "cells": cells,
            "ms": round(ms, 4), "cell_updates_per_s": total * cycles / (ms * 1e-3),
            "residual_reduction_per_vcycle": {l: round(float(np.median(r[1:] / r[:-1])), 4) for l, r in res.items()},
            "first_call_s": round(build_s, 3)}


def run_cic(n, reps, warmup, torch, peak_gbs, peak_src):
    """Cloud-in-Cell mass deposition (Sec. 4) of a cosmological particle set
    with N_part = N_grid = n^3 on the periodic n^3 grid: particle
    depositions per second of the atomic (warp-combining) kernel and of the
    deterministic segment kernel, grid zeroing included; of the source-cell
    Hilbert sort; and of sort + atomic deposit.  FP64 and FP32.  Particle
    arrays and the grid exceed L2, so nothing is flushed between repeats.
    The deposit kernel's algorithmic bytes: the 4 particle arrays read once,
    the grid read and written once."""
    from paper_2607_20704_gb300 import amr, inputs
    t0 = time.perf_counter()
    ps = inputs.particles(n, "cosmo", seed=2607)
    gen_s = time.perf_counter() - t0
    st = bench_stream()
    out = {"grid": f"{n}^3 periodic", "particles": ps.np,
           "set": "lattice of n^3 particles, Zel'dovich-like displacements (rms 0.75 cell at 512^3), "
                  "25% of the particles in Gaussian halos of ~4096 (radii 0.3-3 cells)",
           "l2": "inputs and grid larger than L2; not flushed", "input_generation_s": round(gen_s, 1)}

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    for prec in (8, 4):
        p = amr.Particles(*ps.args(), precision=prec, stream=st)
        p.sort()
        res = {}
        for name, fn in (("sort", p.sort), ("deposit_atomic", lambda: p.deposit("atomic")),
                         ("deposit_segment", lambda: p.deposit("segment")),
                         ("sort_and_deposit_atomic", lambda: (p.sort(), p.deposit("atomic")))):
            ms = timed(fn)
            res[name] = {"ms": round(ms, 4), "particles_per_s": ps.np / (ms * 1e-3)}
        p.set_timing(True)
        p.sort()
        p.deposit("atomic")
        p.deposit("segment")
        kt = p.read_timing()
        p.set_timing(False)
        res["segments"] = p.info()["n_segments"]
        esz = WORD[prec]
        k_ms = kt["cic_atomic"][0] / kt["cic_atomic"][1]
        alg = ps.np * 4 * esz + 2 * n ** 3 * esz
        hbm = {"bound": "hbm", "unit": "GB/s", "achieved": round(alg / (k_ms * 1e-3) / 1e9, 1),
               "peak": peak_gbs, "peak_source": peak_src,
               "frac": round(alg / (k_ms * 1e-3) / 1e9 / peak_gbs, 4),
               "algorithmic_bytes": alg, "kernel_ms": round(k_ms, 4)}
        if prec == 8:
            # bound by the FP64 pipe: FP64 thread instructions per particle
            # counted by ncu (15 DMUL + 3 DFMA + 3.9 DADD on this set) against
            # the pipe's issue rate; the SM clock is filled in after the run
            res["cic_atomic_roofline"] = {"bound": "alu", "unit": "G FP64 inst/s",
                                          "fp64_inst_per_particle": CIC_FP64_INST_PER_PARTICLE,
                                          "achieved": round(ps.np * CIC_FP64_INST_PER_PARTICLE
                                                            / (k_ms * 1e-3) / 1e9, 1),
                                          "kernel_ms": round(k_ms, 4), "hbm_view": hbm}
        else:
            res["cic_atomic_roofline"] = hbm
        res["kernels_ms"] = {k: round(v[0], 4) for k, v in sorted(kt.items(), key=lambda kv: -kv[1][0])}
        out["fp64" if prec == 8 else "fp32"] = res
        p.close()
    out["levels"] = run_cic_levels(timed, torch, st)
    return out


def run_cic_levels(timed, torch, st):
    """Deposition onto the AMR levels (Sec. 4: each level's particle list,
    then the split by host cells refined): the cosmological particle set
    with 256^3 particles on the cosmology-shaped mesh (levels 8-11, 2.5 M
    octs), from device arrays, list sizes per level, deposits per second
    (every list entry deposits once at its level)."""
    from paper_2607_20704_gb300 import amr, inputs
    ps = inputs.particles(256, "cosmo", seed=2607)
    prob = inputs.lognormal()
    out = {"mesh": "lognormal levels 8-11", "octs": int(prob.n_oct), "particles": int(ps.np)}
    for prec in (8, 4):
        m = amr.Mesh(*prob.mesh_args(), **prob.params(), precision=prec, stream=st)
        dt = torch.float64 if prec == 8 else torch.float32
        arrs = [torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt) for a in ps.args()[1:]]
        cnt = m.cic_deposit_levels_device(*arrs)
        ms = timed(lambda: m.cic_deposit_levels_device(*arrs, counts=False))
        total = int(cnt.sum())
        out["fp64" if prec == 8 else "fp32"] = {
            "ms": round(ms, 4), "list_sizes": {int(l): int(c) for l, c in enumerate(cnt) if c},
            "deposits_per_s": total / (ms * 1e-3)}
        m.close()
    return out


CIC_FP64_INST_PER_PARTICLE = 21.9


def cic_alu_peak(cic, sm_mhz):
    """FP64 issue peak of the CIC roofline: 152 SMs x 2 FP64 thread
    instructions per clock at the median SM clock of the run."""
    if cic is None or "fp64" not in cic:
        return
    rl = cic["fp64"]["cic_atomic_roofline"]
    peak = N_SM * FP64_FMA_PER_SM_CLK * sm_mhz * 1e6 / 1e9
    rl["peak"] = round(peak, 1)
    rl["peak_source"] = (f"derived: {N_SM} SMs x {FP64_FMA_PER_SM_CLK} FP64 instructions/clk x "
                         f"{sm_mhz:.0f} MHz (median SM clock under load)")
    rl["frac"] = round(rl["achieved"] / peak, 4)


def inputs_gaussian(n, rng):
    from paper_2607_20704_gb300 import inputs
    return inputs.gaussian_field(n, -2.0, 1.5, rng)


def run_serving(n_requests, rates, torch):
    """Serving loop under Poisson arrivals at each rate of the sweep: p50/p99
    latency (submit -> result on the host) and sustained leaf cell-updates/s
    (completed work / first submission -> last completion).  The low rates
    load the GPU below its capacity, so their latency is the solve itself;
    the high ones saturate it and add queueing."""
    import random
    from paper_2607_20704_gb300 import amr, inputs
    probs, reqs = inputs.serving_requests(n_requests, seed=13)
    # warm-up: one small request of each precision
    srv = amr.Server()
    for prec in (4, 8):
        srv.submit(probs[min(range(len(probs)), key=lambda t: probs[t].n_oct)], 2, prec)
    srv.wait(-1, 600.0)
    srv.close()
    out = {"requests": n_requests, "pool_meshes": len(probs),
           "pool_octs": int(sum(p.n_oct for p in probs)), "budget_gb": 120, "points": []}
    for rate in rates:
        rng = random.Random(13)
        srv = amr.Server()
        t0 = time.perf_counter()
        next_t = 0.0
        for pi, steps, prec in reqs:
            next_t += rng.expovariate(rate)
            dt = t0 + next_t - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            srv.submit(probs[pi], steps, prec)
        srv.wait(-1, 1800.0)
        st = srv.stats()
        srv.close()
        out["points"].append({"arrival_rate_per_s": rate, "completed": st["completed"],
                              "failed": st["failed"], "p50_ms": round(st["latency_p50_ms"], 2),
                              "p99_ms": round(st["latency_p99_ms"], 2),
                              "queue_p50_ms": round(st["queue_p50_ms"], 2),
                              "cell_updates_per_s": st["cell_updates"] / max(st["span_s"], 1e-9),
                              "span_s": round(st["span_s"], 3)})
    return out


def cpu_baseline(prob, nsteps, all_cores=0):
    import oracle
    m = oracle.Mesh(*prob.mesh_args(), **prob.params())
    upd = 0
    for l in m.levels():
        leaf = int(np.count_nonzero(m.read_split(l) == 0))
        upd += leaf * 2 ** (l - prob.levelmin)
    t0 = time.perf_counter()
    m.advance(nsteps)
    dt = time.perf_counter() - t0
    out = {"value": upd * nsteps / dt, "unit": "leaf cell-updates/s", "cores": 1,
           "kind": "oracle",
           "sample": f"{nsteps} coarse W-cycle steps of the same Sedov mesh (levels 7-10, "
                     f"{upd} cell-updates per step), single-threaded FP64 oracle, {dt:.1f} s"}
    if all_cores:
        out["all_cores"] = cpu_baseline_all_cores(upd, all_cores)
    return out


def _oracle_replica(nsteps):
    """One process of the all-core baseline: build the workload, time nsteps
    oracle coarse steps (the oracle as it stands, single-threaded)."""
    import oracle
    from paper_2607_20704_gb300 import inputs
    prob = inputs.sedov()
    m = oracle.Mesh(*prob.mesh_args(), **prob.params())
    t0 = time.perf_counter()
    m.advance(nsteps)
    return time.perf_counter() - t0


def cpu_baseline_all_cores(upd_per_step, nsteps):
    """The oracle on every host core: one independent replica of the workload
    per core (processes started with spawn), all stepping at once; rate =
    all replicas' cell-updates / the slowest replica's time.  The oracle is
    not parallelised or tuned: this is the host's throughput for independent
    solves, the CPU counterpart of the batched GPU handle."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    n = os.cpu_count() or 1
    ex = None
    try:
        # an executor (not a Pool) fails with BrokenProcessPool if a worker
        # dies, and every result has a deadline, so the run cannot hang here
        ex = ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn"))
        futs = [ex.submit(_oracle_replica, nsteps) for _ in range(n)]
        times = [f.result(timeout=300) for f in futs]
    except Exception as e:  # the single-thread figure stands alone
        return {"unavailable": f"{type(e).__name__}: {e}"[:200]}
    finally:
        if ex is not None:
            ex.shutdown(wait=False, cancel_futures=True)
    slowest = max(times)
    return {"value": n * nsteps * upd_per_step / slowest, "unit": "leaf cell-updates/s", "cores": n,
            "kind": "oracle",
            "sample": f"{n} processes, each {nsteps} coarse W-cycle steps of its own copy of the "
                      f"Sedov mesh, single-threaded FP64 oracle; slowest {slowest:.1f} s"}


def fp64_peak(torch, device):
    """FP64 rate of cuBLAS DGEMM on this GPU (denominator of the ALU roofline)."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device=device)
    b = torch.randn(n, n, dtype=torch.float64, device=device)
    torch.matmul(a, b)
    torch.cuda.synchronize(device)
    best = 1e30
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2 * n ** 3 / (best * 1e-3) / 1e12


# FP64 pipe of the GB300: 152 SMs, 2 FP64 FMA lanes per SM per clock (the
# nominal 1.25 TFLOP/s at the 2070 MHz maximum SM clock: 152 x 2 x 2 x 2.07e9)
N_SM = 152
FP64_FMA_PER_SM_CLK = 2


def fp64_peak_derived(sm_mhz):
    """FP64 TFLOP/s (2 per FMA) at the given SM clock."""
    return N_SM * FP64_FMA_PER_SM_CLK * 2 * sm_mhz * 1e6 / 1e12


def roofline(res, prec, levelmin, peak_gbs, peak_src, fp64_tflops=None, dgemm=None,
             sm_mhz=None, fma64=None):
    """Roofline object of the dominant kernel: achieved = its algorithmic
    bytes (FP32) or FP64 flops (FP64: the flux kernel is bound by the FP64
    pipe) per launch / its average CUDA-event launch time."""
    w = WORD[prec]
    traffic = kernel_traffic(res["info"], levelmin, w, fused=(prec == 4))
    kt = res.get("kernels", {})
    if not kt:
        return None, None
    tot = sum(v[0] for v in kt.values())
    table = {k: {"ms": round(v[0], 4), "launches": v[1], "share": round(v[0] / tot, 4)}
             for k, v in sorted(kt.items(), key=lambda kv: -kv[1][0])}
    name, (ms_tot, n_launch) = max(kt.items(), key=lambda kv: kv[1][0])
    if name not in traffic:
        return None, table
    steps = res["steps"]
    avg_s = ms_tot / n_launch * 1e-3
    bytes_per_launch = traffic[name] * steps / n_launch
    loc, real, _, _ = kernel_units(res["info"], levelmin)
    cells_per_launch = (real if prec == 8 else loc) * steps / n_launch
    hbm = {"bound": "hbm", "achieved": round(bytes_per_launch / avg_s / 1e9, 1), "peak": peak_gbs,
           "unit": "GB/s", "frac": round(bytes_per_launch / avg_s / 1e9 / peak_gbs, 4),
           "algorithmic_bytes_per_launch": int(bytes_per_launch), "peak_source": peak_src}
    traffic_launch = None
    if name == "flux":
        real_per_launch = real * steps / n_launch
        traffic_launch = int(FLUX_DRAM_BYTES_PER_CELL[prec] * real_per_launch)
    hbm["traffic"] = traffic_launch
    if prec == 8 and name == "flux" and fp64_tflops:
        flops = FLUX_FP64_FLOPS_PER_CELL * cells_per_launch
        ach = flops / avg_s / 1e12
        rl = {"kernel": name, "bound": "alu", "achieved": round(ach, 4),
              "peak": round(fp64_tflops, 4), "unit": "TFLOP/s", "frac": round(ach / fp64_tflops, 4),
              "traffic": traffic_launch,
              "peak_source": f"derived: {N_SM} SMs x {FP64_FMA_PER_SM_CLK} FP64 FMA/clk x 2 flops "
                             f"x {sm_mhz:.0f} MHz (median SM clock under load)",
              "flops_per_launch": int(flops), "avg_launch_us": round(avg_s * 1e6, 3),
              "dgemm_tflops": dgemm, "frac_of_dgemm": round(ach / dgemm, 4) if dgemm else None,
              "fma_microbench_tflops": fma64,
              "frac_of_fma_microbench": round(ach / fma64, 4) if fma64 else None,
              "hbm_view": hbm}
    else:
        rl = dict(hbm)
        rl["kernel"] = name
        rl["avg_launch_us"] = round(avg_s * 1e6, 3)
    return rl, table


def workload_config(n_oct, n_ghost, leaf, upd, world):
    """The workload as both arms name it (the GPU arm and the CPU reference
    arm print the same dict for the same mesh)."""
    return {"workload": WORKLOAD, "levelmin": 7, "levelmax": 10, "gamma": 5.0 / 3.0,
            "n_oct": int(n_oct), "n_ghost_oct": int(n_ghost), "leaf_cells": int(leaf),
            "cell_updates_per_step": int(upd),
            "step": "one coarse W-cycle step (CFL + 15 level steps; the static mesh is indexed "
                    "once, at creation)",
            "l2": f"GPU arm: a {L2_FLUSH_BYTES >> 20} MiB write between timed steps; CPU "
                  "reference arm: no device",
            "parallelism": (f"{world} GPU processes, replicas; the CPU reference arm runs on rank 0"
                            if world > 1 else "single GPU; the CPU reference arm on the host")}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.warmup < 3:
        args.warmup = 3
    LAUNCH.update(tile=args.tile, schedule=args.schedule, nsubgrid=args.nsubgrid, planar=args.planar)
    if args.impl == "reference" and rank != 0:
        return 0  # the reference arm runs on rank 0 alone
    from paper_2607_20704_gb300 import inputs
    prob = inputs.sedov()

    if args.impl == "reference":
        import oracle
        m = oracle.Mesh(*prob.mesh_args(), **prob.params())
        upd = sum(int(np.count_nonzero(m.read_split(l) == 0)) * 2 ** (l - prob.levelmin)
                  for l in m.levels())
        leaf = sum(int(np.count_nonzero(m.read_split(l) == 0)) for l in m.levels())
        n_ghost = sum(m.num_cache(l) for l in m.levels())
        m.advance(args.warmup)
        t0 = time.perf_counter()
        m.advance(args.steps)
        dt = time.perf_counter() - t0
        v = upd * args.steps / dt
        line = {"impl": "reference", "metric": "leaf cell-updates/s", "value": v,
                "unit": "leaf cell-updates/s", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": workload_config(prob.n_oct, n_ghost, leaf, upd, world),
                "cpu_baseline": {"value": v, "unit": "leaf cell-updates/s", "cores": 1,
                                 "kind": "oracle",
                                 "sample": f"{args.steps} full coarse steps of the workload, "
                                           "single-threaded FP64 oracle on the host"},
                "e2e": {"value": v, "unit": "leaf cell-updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch
    if args.profile_poisson:
        from paper_2607_20704_gb300 import amr, build
        build.build()
        amr.load()
        L = args.profile_poisson
        n = 1 << L
        pr = inputs.uniform_grid(L, lambda x, y, z: (1.0 + 0.5 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y),
                                                     0 * x, 0 * x, 0 * x, 1.0 + 0 * x))
        m = amr.Mesh(*pr.mesh_args(), **pr.params())
        m.poisson(1.0, 1, residuals=False)
        m.sync()
        print(json.dumps({"profile_poisson": L, "cells": n ** 3}))
        m.close()
        return 0
    if args.profile_cic:
        from paper_2607_20704_gb300 import amr, build
        build.build()
        amr.load()
        ps = inputs.particles(args.profile_cic, "cosmo", seed=2607)
        p = amr.Particles(*ps.args(), precision=args.precision)
        p.sort()
        p.deposit("atomic")
        p.deposit("segment")
        p.rho()
        print(json.dumps({"profile_cic": args.profile_cic, "particles": ps.np,
                          "precision": args.precision}))
        p.close()
        return 0
    if args.profile_unigrid:
        from paper_2607_20704_gb300 import amr, build
        build.build()
        amr.load()
        L = args.profile_unigrid
        up = unigrid_problem(L)
        m = amr.Mesh(*up.mesh_args(), **up.params(), precision=args.precision, **LAUNCH)
        m.step_level(L, m.cfl_dt() * 1e-3)
        m.sync()
        print(json.dumps({"profile_unigrid": L, "precision": args.precision, "cells": 8 * m.num_octs(L)}))
        m.close()
        return 0
    if args.profile_level:
        from paper_2607_20704_gb300 import amr, build
        build.build()
        amr.load()
        m = amr.Mesh(*prob.mesh_args(), **prob.params(), precision=args.precision, **LAUNCH)
        dt = m.cfl_dt() * 0.5 ** (args.profile_level - prob.levelmin)
        m.step_level(args.profile_level, dt)
        m.sync()
        print(json.dumps({"profile_level": args.profile_level, "precision": args.precision,
                          "octs": m.num_octs(args.profile_level)}))
        m.close()
        return 0
    from paper_2607_20704_gb300 import dist
    if world > 1:
        dist.init("nccl", torch.device("cuda", local))
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    from paper_2607_20704_gb300 import amr, build
    build.build()
    amr.load()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    peak_gbs, peak_src = load_peaks()

    prec_main = args.precision
    prec_other = 4 if prec_main == 8 else 8
    with ClockSampler(local) as clk:
        main_res = run_precision(prob, prec_main, args.steps, args.warmup, torch, device, flush)
        main_res["steps"] = args.steps
        other = None
        if not args.no_other_precision:
            other = run_precision(prob, prec_other, args.steps, args.warmup, torch, device, flush)
            other["steps"] = args.steps
        e2e = None if args.no_e2e else run_e2e(prob, prec_main, max(3, args.steps // 2), torch)
        poisson = None if args.no_poisson else run_poisson(8, 10, torch, device)
        if poisson is not None:
            poisson["levels"] = run_poisson_levels(4, torch, device)
        cic = None if args.no_cic else run_cic(args.cic_grid, 5, 3, torch, peak_gbs, peak_src)
        variants = None if args.no_variants else run_variants(prob, 7, torch, device, flush)
        unigrid = None if args.no_unigrid else run_unigrid(8, 7, torch, device)
        adaptive = None
        if not args.no_adaptive:
            adaptive = {("fp64" if p == 8 else "fp32"): run_adaptive(prob, p, 10, torch, device)
                        for p in (8, 4)}
        serving = None
        if not args.no_serving:
            serving = run_serving(args.serving_requests, (2.0, 4.0, 10.0, 40.0), torch)
        batched = None
        if not args.no_batched:
            ens = inputs.batched(args.batched_members, seed=11)
            batched = run_batched(ens, min(args.steps, 5), 2, torch, device, flush)
            del ens
    clocks = clk.summary()

    upd = main_res["updates_per_step"]
    # whole job: every rank's cell-updates over the slowest rank's time
    value, slowest_s = dist.throughput(upd * args.steps, main_res["ms"] * 1e-3, device)
    ms = slowest_s * 1e3
    if other is not None:
        other_value, other_s = dist.throughput(upd * args.steps, other["ms"] * 1e-3, device)
    try:
        dgemm = round(fp64_peak(torch, device), 4)
    except Exception:
        dgemm = None
    try:  # the FMA rates of this GPU from the library's own microbenchmark
        fma = {"fp64_tflops": round(amr.fma_rate(local, 8) / 1e12, 4),
               "fp32_tflops": round(amr.fma_rate(local, 4) / 1e12, 3)}
    except Exception:
        fma = None
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    fp64_pk = fp64_peak_derived(sm_mhz)
    cic_alu_peak(cic, sm_mhz)
    fma64 = fma["fp64_tflops"] if fma else None
    rl, table = roofline(main_res, prec_main, prob.levelmin, peak_gbs, peak_src, fp64_pk, dgemm, sm_mhz,
                         fma64)
    if other is not None:
        rl_o, table_o = roofline(other, prec_other, prob.levelmin, peak_gbs, peak_src, fp64_pk,
                                 dgemm, sm_mhz, fma64)
    step_bytes = 2 * 5 * WORD[prec_main]
    line = {
        "metric": "leaf cell-updates/s",
        "value": value,
        "unit": "leaf cell-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if prec_main == 8 else "f32",
        "data": "synthetic",
        "config": workload_config(main_res["info"]["n_oct"], main_res["info"]["n_cache"],
                                  main_res["info"]["n_leaf_cells"], upd, world),
        "roofline": rl,
        "step_roofline": {"bound": "hbm", "unit": "GB/s", "peak": peak_gbs,
                          "achieved": round(value / world * step_bytes / 1e9, 1),
                          "frac": round(value / world * step_bytes / 1e9 / peak_gbs, 4),
                          "bytes_per_cell_update": step_bytes},
        "kernels": table,
        "gpu_launches": main_res["launches"],
        "autotuned": {"tile": main_res["info"].get("tile"), "schedule": main_res["info"].get("schedule"),
                      "nsubgrid": main_res["info"].get("nsubgrid"), "planar": main_res["info"].get("planar")},
        "clocks": clocks,
        "e2e": e2e,
    }
    if other is not None:
        line["fp32" if prec_other == 4 else "fp64"] = {
            "value": other_value,
            "ms_per_step": other_s * 1e3 / args.steps,
            "roofline": rl_o, "kernels": table_o, "gpu_launches": other["launches"],
            "autotuned": {"tile": other["info"].get("tile"), "schedule": other["info"].get("schedule"),
                          "nsubgrid": other["info"].get("nsubgrid"), "planar": other["info"].get("planar")},
            "step_roofline_frac": round(other_value / world
                                        * 2 * 5 * WORD[prec_other] / 1e9 / peak_gbs, 4)}
    if adaptive is not None:
        line["adaptive"] = adaptive
    if poisson is not None:
        line["poisson"] = poisson
    if cic is not None:
        line["cic"] = cic
    if variants is not None:
        line["level_step_kernels"] = variants
    if unigrid is not None:
        line["unigrid"] = unigrid
    if batched is not None:
        line["batched"] = batched
    if serving is not None:
        line["serving"] = serving
    line["fp64_dgemm_tflops"] = dgemm
    line["fma_microbench"] = fma
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(prob, args.cpu_steps, args.cpu_all_core_steps)
    if world > 1:
        dist.finalize()
    if rank == 0:
        print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
