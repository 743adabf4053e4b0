#!/usr/bin/env python
"""Throughput of the fused particle step (DEM contacts + drag + heat + USCM kinetics +
deposition + gas update) on GB300, in parcel-updates per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on rank 0. The default workload is the 2,000,000-parcel two-ore bed with the
conical bottom and perforated distributor plate (64x64x384 gas cells), in the precision form
with FP32 forces and kinetics and compensated FP32 pairs for positions, layer masses and cell
sums (the FP64-position form and the all-FP64 form are timed beside it), stepped by replaying
CUDA graphs of ten steps. Under torchrun every rank steps its own replica of the workload (the
path has no exchange between beds): weak scaling, max-over-ranks time.
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

METRIC = "parcel-updates/s per fused DEM+reaction step; % HBM roofline; adjoint/fwd cost"
UNIT = "parcel-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ibm_2m", choices=["ibm_2m", "split_200k", "plain_2k", "batched_32"])
    ap.add_argument("--precision", default="split_kahan", choices=["split", "fp64", "split_kahan"],
                    help="split_kahan (default): FP32 forces and kinetics, positions, layer masses and cell "
                    "sums as compensated FP32 pairs; split: the same with FP64 positions and masses")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-form", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=100_000, help="parcels in the oracle's sample")
    ap.add_argument("--parcels", type=int, default=0, help="override the workload's parcel count "
                    "(smaller cases for profiler captures; same geometry and packing)")
    ap.add_argument("--form-steps", type=int, default=0, help="steps of the three-form comparison "
                    "(0: the workload's own step count)")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--graph-steps", type=int, default=10, help="steps per captured CUDA graph in the timed "
                    "loop (the graph is replayed; every step is computed)")
    ap.add_argument("--settle", type=int, default=300, help="untimed steps before the autotuner and the warm-up, so that the timed steps see the fluidised bed (contacts, list builds) rather than the packing at rest")
    ap.add_argument("--autotune", type=int, default=30, help="steps per autotuner candidate before the "
                    "warm-up (0: keep the default launch configuration)")
    ap.add_argument("--no-radiation-leg", action="store_true", help="skip the extra measurement of the "
                    "step with radiation switched on")
    ap.add_argument("--radiation", action="store_true", help="switch on the particle radiation of "
                    "eqs (3-16), (3-17), (3-51) in every bed (a widening of the step; off by default)")
    ap.add_argument("--conduction", action="store_true", help="switch on the contact heat conduction of "
                    "eqs (3-14)..(3-15-2) in every bed (off by default)")
    ap.add_argument("--tuning", default="", help="fixed launch configuration instead of the autotuner, "
                    "e.g. neighbour_lists=1,bs_key=64,skin_permille=50 (profiler runs repeat a plain run's)")
    ap.add_argument("--no-dense-leg", action="store_true", help="skip the contact-dominated 2M bed")
    ap.add_argument("--no-batched-leg", action="store_true", help="skip the 32-bed batch")
    ap.add_argument("--no-gas-solver-leg", action="store_true", help="skip the 2M bed with the gas phase solved")
    ap.add_argument("--only-leg", default="", choices=["", "gas_solver", "dense", "dense_conduction"],
                    help="run only this leg and print its line (for profiling one regime on a small case): "
                    "gas_solver on --workload (ibm_2m or split_200k), the dense legs with --parcels")
    ap.add_argument("--coupling", default="10,1,20", help="coupling intervals n = dt_CFD/dt_DEM of the "
                    "end-to-end legs; the first one is the e2e headline (Table 3: n = 10 for Bed II)")
    return ap.parse_args()


def make_workload(name: str, rank: int = 0, parcels: int = 0, radiation: bool = False, conduction: bool = False):
    from paper_2311_03908_gb300 import synth
    seed_shift = 7919 * rank
    kw = {"n": parcels} if parcels else {}
    if name == "ibm_2m":
        bed = synth.config_ibm_2m(seed=2311039083 + seed_shift, **kw)
    elif name == "split_200k":
        bed = synth.config_split_200k(seed=2311039082 + seed_shift, **kw)
    elif name == "plain_2k":
        bed = synth.config_plain_2k(seed=2311039081 + seed_shift, **kw)
    elif name == "batched_32":
        bed = synth.config_batched_32(seed=2311039085 + seed_shift)
    else:
        raise ValueError(name)
    for cfg in bed.beds:
        cfg.flags |= (synth.RADIATION if radiation else 0) | (synth.CONDUCTION if conduction else 0)
    return bed


# ---------------------------------------------------------------------------------------
# Algorithmic bytes per launch of each kernel: the traffic the method cannot avoid in this
# layout -- every parcel's own record read and written once, every cell's state once, the
# live contact slots (z_bar per parcel) and neighbour-list entries (L per parcel) once -- not
# counting the re-reads of neighbours' records, which the caches serve.
# ---------------------------------------------------------------------------------------
def algorithmic_bytes(kernel: str, n: int, ncells: int, zbar: float, L: float, rsize: int, passes: int,
                      fbuild: float = 0.0, fc: float = 1.0, frestore: float = None) -> float:
    """Per launch; fbuild = fraction of steps that rebuild the lists, frestore = fraction that
    re-store the state in cell order (default: every build), fc = fraction of parcels in
    contact (only those have a contact force and torque to pass on)."""
    if frestore is None:
        frestore = fbuild
    R = rsize
    slot = 4 + 3 * R                                  # partner id + tangential displacement
    state = 24 + 12 * R + 2 * R + 32 + 8 + 12         # x; v,w,a,al; T,d; masses; meta,orig; dsp
    if kernel == "k_key":            # in place: drift with the half-step velocity, displacement, key,
        # local coordinates; the previous step's sorted keys (to empty its cell ranges)
        return n * ((4 + 24 + 3 * R + 12 + 16 + 4 + R + 4) + (24 + 12 + 4 + 16))
    if kernel == "radix_sort":
        return n * passes * (8 + 8)
    if kernel == "resort":           # new keys in sorted order, re-sort, permutation and cell ranges
        return n * (16 + 16 + 8)
    if kernel == "k_restore":        # re-store steps: state, local coordinates, history back from the copy
        return frestore * n * (2 * (state + 16 + 1 + zbar * slot) + 8)
    if kernel == "k_pair_search":    # list builds (the cell-list search) only
        return fbuild * n * ((4 + 16 + 4) + (4 * L + 1 + 1 + 12 + 5 * zbar))
    if kernel == "k_ranges":         # ranges, inverse permutation; on re-store steps the records out
        return n * (4 + 4 + 4) + frestore * n * (2 * (state + 16 + 1 + zbar * slot) + 4)
    if kernel == "k_contact_screen":  # list test (between builds), wall pre-screen; empty histories
        return n * ((4 + 16 + 4 + 1 + 4 * L * (1 - fbuild) + fbuild * 1) + 1)
    if kernel == "k_contact_forces":  # parcels in contact: own state, partners, history in and out, F, T
        return n * (fbuild * 5 * zbar + zbar * (2 * slot + 8 * R + 32) + fc * (8 + 6 * R + 32 + 6 * R))
    if kernel == "k_gas_particle":   # the accelerations and 7 of the 13 source rows are stored on a
        # stepping call's last step only
        return n * ((4 + 4 + R + 3 * R + R + 32 + 1 + fc * 6 * R + 3 * R) + (6 * R + R + 32 + 6 * R)) + ncells * 13 * R
    if kernel == "k_cells":          # bed, mark, range, state in (rho and c_p are recomputed in the
        # FP32 forms, read in the FP64 form); state and properties out; the parcels' 6 source rows
        return ncells * ((4 + 1 + 8 + 5 * 8 + (2 * R if R == 8 else 0)) + (5 * 8 + 14 * R)) + n * (6 * R + 4)
    if kernel == "k_radiation":      # own meta, local coordinates, key, d, T (+ FP64 position); the
        # cell's eps_g and T_g; Q_rad out (the neighbours' records are cache re-reads)
        return n * ((4 + 16 + 4 + 2 * R + (24 if R == 8 else 0)) + R) + ncells * 2 * R
    return 0.0


def survey_step_bytes(n: int, ncells: int, zbar: float, rsize: int, passes: int) -> float:
    """Minimum traffic of one step by the per-parcel and per-cell list of the method's scope
    table (parcel state gathered and written once, key and sort passes, live contact history,
    per-parcel source staging as this layout does it, and ~256 B per gas cell), recomputed
    from this layout's sizes: the method's floor, against which the builder's kernel-by-kernel
    algorithmic bytes (which include neighbour lists, the list screen and the cell-property
    records) are the larger figure."""
    if rsize == 4:
        read, write, slot = 24 + 12 + 12 + 4 + 32 + 12, 24 + 12 + 12 + 4 + 32, 4 + 12
    else:
        read, write, slot = 24 + 24 + 24 + 8 + 32 + 16, 24 + 24 + 24 + 8 + 32, 4 + 24
    staging = (6 + 6) * rsize               # per-parcel sources written, then read by the cell sums
    return n * (read + write + 4 + passes * 16 + zbar * slot * 2 + staging) + ncells * 256


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum, one full-size ncu
# capture of the 2M-parcel bed in the split-Kahan form between list builds, after the
# 300-step settle; per parcel), valid only for the CUDA sources it was taken on.
TRAFFIC_SOURCE_SHA256 = "66daeeb47eb051fdb6b1ffcd5811fd31a9fd60d4f0eb426a743c327e62aca2d8"
TRAFFIC_WORKLOAD = ("ibm_2m", "split_kahan", 2_000_000)
TRAFFIC_BYTES_PER_PARCEL = {"k_gas_particle": 169.2, "k_key": 117.1, "k_cells": 99.6, "k_contact_screen": 58.4,
                            "k_contact_forces": 17.7, "k_ranges": 8.1}


def source_sha256() -> str:
    """Hash of the CUDA sources and the C header with comments and blank lines left out: a
    change of code invalidates the measured traffic, a change of comments does not."""
    import glob
    import hashlib
    import re
    h = hashlib.sha256()
    files = sorted(glob.glob(os.path.join(ROOT, "paper_2311_03908_gb300", "csrc", "*.cu")) +
                   glob.glob(os.path.join(ROOT, "paper_2311_03908_gb300", "csrc", "*.cuh")) +
                   [os.path.join(ROOT, "include", "dem.h")])
    for f in files:
        with open(f, encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        code = "\n".join(line.rstrip() for line in text.splitlines() if line.strip())
        h.update(os.path.basename(f).encode() + b"\0" + code.encode())
    return h.hexdigest()


def measured_traffic(kernel: str, workload: str, precision: str, n: int):
    """Bytes per launch from the committed ncu capture, or None when it does not apply."""
    if (workload, precision, n) != TRAFFIC_WORKLOAD or kernel not in TRAFFIC_BYTES_PER_PARCEL:
        return None
    if source_sha256() != TRAFFIC_SOURCE_SHA256:
        return None   # the kernels changed since the counters were taken
    return TRAFFIC_BYTES_PER_PARCEL[kernel] * n


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def cpu_baseline(bed, steps: int, sample: int):
    """The oracle as it stands on this host's cores, on a bounded sample of the workload."""
    import oracle
    n = min(sample, bed.n)
    sub = bed.subset(np.arange(n)) if n < bed.n else bed   # parcel indices are shuffled
    o = oracle.Oracle(sub)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return {"value": n * steps / dt, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
            "sample": f"{n} of {bed.n} parcels of the same bed (random subset), {steps} step(s), FP64"}


def radiation_leg(binding, stream, bed, tuning, settle, steps, precision):
    """The step with the particle radiation of eqs (3-16), (3-17), (3-51) switched on in every
    bed (off in the headline step): a fresh context of the same workload, settled like the
    main one, 10-step graphs timed with CUDA events, and the radiation kernel's own time
    from an eager pass."""
    import dataclasses
    import torch
    from paper_2311_03908_gb300 import synth
    rb = dataclasses.replace(bed, beds=[dataclasses.replace(c, flags=c.flags | synth.RADIATION) for c in bed.beds])
    cx = binding.Context(rb, precision=precision, stream=stream.cuda_stream)
    if settle > 0:
        cx.dem_step(settle)
    cx.dem_set_tuning(**tuning)
    G = 10
    steps = max(G, steps // G * G)
    cx.dem_step_graph(G)
    cx.dem_step_graph(G)
    cx.dem_sync()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(steps // G):
        cx.dem_step_graph(G)
    a1.record(stream)
    torch.cuda.synchronize()
    ms = a0.elapsed_time(a1)
    cx.dem_profile(True)
    cx.dem_step(20)
    t = cx.dem_kernel_times()
    cx.dem_profile(False)
    cx.close()
    nl, tot = t.get("k_radiation", (1, 0.0))
    return {"ms_per_step": ms / steps, "value": bed.n * steps / (ms * 1e-3), "unit": UNIT, "steps": steps,
            "settle_steps": settle, "k_radiation_ms": tot / max(nl, 1),
            "what": "eqs (3-16), (3-17), (3-51) on, same workload, tuning and stepping"}


def e2e_coupling(binding, stream, bed, ncouple, tuning, settle, steps):
    """End to end through the C ABI, the paper's coupling round trip (Sec. 4, Fig. 5): every
    n = coupling_interval steps the gas field comes in from page-locked host memory
    (dem_set_gas: mass fractions and temperature of every cell), the n steps run as one
    replayed graph, and the cell sources of the coupling step go back to page-locked host
    memory (dem_get_sources_occupied: 14 doubles and the index of every cell that holds
    parcels, the others' sources being zero) with the bed reduction degrees."""
    import dataclasses
    import torch
    b2 = dataclasses.replace(bed, beds=[dataclasses.replace(c, coupling_interval=ncouple) for c in bed.beds])
    cx = binding.Context(b2, precision=tuning.pop("_precision"), stream=stream.cuda_stream)
    if settle > 0:
        cx.dem_step(settle)
    cx.dem_set_tuning(**tuning)
    gas = cx.dem_get_gas()
    Y = torch.from_numpy(np.ascontiguousarray(gas[:, 1:4])).pin_memory()
    T = torch.from_numpy(np.ascontiguousarray(gas[:, 4])).pin_memory()
    cap = min(cx.n, cx.ncells)
    out = torch.empty((cap, 14), dtype=torch.float64).pin_memory()
    cells = torch.empty(cap, dtype=torch.int64).pin_memory()
    ncpl = max(3, steps // ncouple)
    for _ in range(2):             # warm-up couplings (graphs captured)
        cx.dem_set_gas(Y, T)
        cx.dem_step_graph(ncouple)
        cx.dem_get_sources_occupied(cells, out)
        cx.dem_reduction_degree()
    torch.cuda.synchronize()
    nocc = 0
    t0 = time.perf_counter()
    for _ in range(ncpl):
        cx.dem_set_gas(Y, T)
        cx.dem_step_graph(ncouple)
        occ, _ = cx.dem_get_sources_occupied(cells, out)
        nocc += len(occ)
        cx.dem_reduction_degree()
    torch.cuda.synchronize()
    te = time.perf_counter() - t0
    nsteps = ncpl * ncouple
    # the same steps without the round trip (same context, graphs replayed back to back)
    t1 = time.perf_counter()
    for _ in range(ncpl):
        cx.dem_step_graph(ncouple)
    torch.cuda.synchronize()
    ts = time.perf_counter() - t1
    cx.close()
    return {"coupling_interval": ncouple, "steps": nsteps, "seconds": te, "ms_per_step": 1e3 * te / nsteps,
            "steps_only_ms_per_step": 1e3 * ts / nsteps,
            "occupied_cells": nocc / ncpl, "cells": int(Y.shape[0]),
            "h2d_bytes_per_step": int(Y.numel() * 8 + T.numel() * 8) / ncouple,
            "d2h_bytes_per_step": (nocc / ncpl * (14 * 8 + 8) + 4 + len(bed.beds) * 16) / ncouple}


def dense_leg(binding, stream, tuning, settle, steps, precision, parcels=0, conduction=False):
    """The 2M cone-and-plate bed as a packed bed without gas flow: one parcel size, every
    site of a square lattice filled with touching neighbours, compressed by its own weight
    over the untimed settle steps into the contact-dominated regime (about 2.7 contacts per
    parcel, 97 % of the parcels in contact after 100 steps). Over thousands of steps the
    packing drains through the plate's holes (wider than the parcels), so it is timed early,
    like the headline step, and the mean number of live contacts is read after the timed
    steps. conduction: the same with the contact heat conduction of eqs (3-14)..(3-15-2)."""
    import torch
    from paper_2311_03908_gb300 import synth
    kw = {"n": parcels} if parcels else {}
    bed = synth.config_ibm_2m_dense(**kw)
    if conduction:
        for c in bed.beds:
            c.flags |= synth.CONDUCTION
    cx = binding.Context(bed, precision=precision, stream=stream.cuda_stream)
    cx.dem_step(settle)
    cx.dem_set_tuning(**tuning)
    G = 10
    steps = max(G, steps // G * G)
    cx.dem_step_graph(G)
    cx.dem_step_graph(G)
    cx.dem_sync()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(steps // G):
        cx.dem_step_graph(G)
    a1.record(stream)
    torch.cuda.synchronize()
    ms = a0.elapsed_time(a1)
    cnt, _, _ = cx.dem_get_contacts()
    cx.dem_profile(True)
    cx.dem_step(20)
    t = cx.dem_kernel_times()
    cx.dem_profile(False)
    cx.close()
    return {"workload": f"ibm_2m_dense ({bed.n} parcels of one size, touching square lattice under gravity, no gas flow)"
                        + (", contact conduction on" if conduction else ""),
            "ms_per_step": ms / steps, "value": bed.n * steps / (ms * 1e-3), "unit": UNIT, "steps": steps,
            "settle_steps": settle, "zbar_contacts": float(cnt.mean()), "fraction_in_contact": float((cnt > 0).mean()),
            "contact_kernels_ms": {k: v[1] / max(v[0], 1) for k, v in t.items()
                                   if k in ("k_contact_screen", "k_contact_forces", "k_pair_search")}}


def batched_leg(binding, stream, settle, steps, precision):
    """The 32-bed sweep (uneven parcel counts, 773-1073 K, 0.2-0.5 m/s inlet): one context,
    one sort and one launch per kernel for all beds, the steps replayed as CUDA graphs."""
    import torch
    bed = make_workload("batched_32")
    cx = binding.Context(bed, precision=precision, stream=stream.cuda_stream)
    cx.dem_step(settle)
    tuning = cx.dem_autotune(20)
    G = 10
    steps = max(G, steps // G * G)
    cx.dem_step_graph(G)
    cx.dem_step_graph(G)
    cx.dem_sync()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(steps // G):
        cx.dem_step_graph(G)
    a1.record(stream)
    torch.cuda.synchronize()
    ms = a0.elapsed_time(a1)
    mean, _ = cx.dem_reduction_degree()
    # launch overhead: the same steps launched kernel by kernel (no graph), and the sum of
    # the kernels' own device times (each bracketed by events, so no overlap between them)
    a0.record(stream)
    cx.dem_step(steps)
    a1.record(stream)
    torch.cuda.synchronize()
    ms_eager = a0.elapsed_time(a1)
    cx.dem_profile(True)
    cx.dem_step(G)
    t = cx.dem_kernel_times()
    cx.dem_profile(False)
    ksum = sum(v[1] for v in t.values()) / G
    cx.close()
    return {"workload": f"batched_32 ({bed.n} parcels in {len(bed.beds)} beds of "
                        f"{min(bed.meta['counts'])}..{max(bed.meta['counts'])})",
            "ms_per_step": ms / steps, "value": bed.n * steps / (ms * 1e-3), "unit": UNIT, "steps": steps,
            "settle_steps": settle, "tuning": tuning, "stepping": "one context, graphs of 10 steps",
            "eager_ms_per_step": ms_eager / steps, "kernel_sum_ms_per_step": ksum,
            "graph_over_kernel_sum": (ms / steps) / ksum if ksum > 0 else None,
            "f_ov_mean_per_bed_range": [float(mean.min()), float(mean.max())]}


def gas_solver_leg(binding, stream, tuning, steps, precision, workload="ibm_2m"):
    """A bed (by default the 2M cone-and-plate bed) with the gas phase solved on the GPU
    (momentum, energy and species every 10 steps, the pressure by multigrid-preconditioned
    CG): the whole coupled step, timed like the headline one, and the solver's share."""
    import torch
    from paper_2311_03908_gb300 import synth
    bed = make_workload(workload)
    for c in bed.beds:
        c.flags |= synth.GAS_SOLVER
        c.coupling_interval = 10
    cx = binding.Context(bed, precision=precision, stream=stream.cuda_stream)
    cx.dem_set_tuning(**{k: v for k, v in tuning.items() if not k.startswith("gas_")})
    G = 10
    steps = max(G, steps // G * G)
    cx.dem_step_graph(G)
    cx.dem_step_graph(G)
    cx.dem_sync()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(steps // G):
        cx.dem_step_graph(G)
    a1.record(stream)
    torch.cuda.synchronize()
    ms = a0.elapsed_time(a1)
    fl, iters = cx.dem_get_flow()
    cx.dem_profile(True)
    cx.dem_step(2 * G)
    t = cx.dem_kernel_times()
    cx.dem_profile(False)
    cx.close()
    gas = {k: v[1] / 2 for k, v in t.items() if k.startswith("k_gs_")}
    total = sum(v[1] for v in t.values()) / 2
    return {"workload": f"{workload} ({bed.n} parcels, {bed.beds[0].nx}x{bed.beds[0].ny}x{bed.beds[0].nz} gas cells) "
                        "with the gas phase solved, coupling interval 10",
            "ms_per_step": ms / steps, "value": bed.n * steps / (ms * 1e-3), "unit": UNIT, "steps": steps,
            "cg_iterations_last_solve": iters, "preconditioner": "multigrid V(2,2), coarse weight 1.5",
            "ms_per_solve": {k: round(v, 4) for k, v in gas.items()},
            "solver_share_of_10_steps": sum(gas.values()) / total if total > 0 else None,
            "max_gas_speed_m_s": float(np.abs(fl[:, :3]).max())}


def adjoint_cost(binding, stream):
    """Wall time of dem_adjoint with the gradient against its forward sweep alone."""
    import torch
    from paper_2311_03908_gb300 import synth
    abed = synth.config_adjoint_64k()
    steps, ck = int(abed.meta["steps"]), int(abed.meta["ckpt"])
    cx = binding.Context(abed, precision="fp64", stream=stream.cuda_stream)
    cx.dem_adjoint(ck, ck, want_grad=True)           # warm-up (buffers, code paths)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J, _ = cx.dem_adjoint(steps, ck, want_grad=False)
    torch.cuda.synchronize()
    tf = time.perf_counter() - t0
    t0 = time.perf_counter()
    J2, g = cx.dem_adjoint(steps, ck, want_grad=True)
    torch.cuda.synchronize()
    ta = time.perf_counter() - t0
    cx.close()
    return {"parcels": abed.n, "steps": steps, "ckpt_every": ck, "forward_ms": tf * 1e3,
            "adjoint_ms": ta * 1e3, "adjoint_over_forward": ta / tf, "J": J, "J_adjoint_run": J2,
            "grad": [float(v) for v in g]}


def max_over_ranks(value: float, dist=None, device: str = "cpu") -> float:
    """The largest of the ranks' values: a job's time is that of its slowest rank."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(n_per_rank: int, world: int, steps: int, ms_max: float) -> float:
    """Parcel-updates/s of the whole job: every rank's parcels, over the slowest rank's time."""
    return n_per_rank * world * steps / (ms_max * 1e-3)


def reference_arm(args):
    """--impl reference: the oracle (FP64 CPU) on the host cores, same workload and metric."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    bed = make_workload(args.workload, 0, args.parcels, args.radiation, args.conduction)
    import oracle
    n = min(args.cpu_sample, bed.n)
    sub = bed.subset(np.arange(n)) if n < bed.n else bed   # parcel indices are shuffled
    o = oracle.Oracle(sub)
    ksteps = max(1, min(args.steps, 20))
    wsteps = max(0, min(args.warmup, 3))   # the timing rules' minimum, bounded: the oracle is slow
    o.step(wsteps)
    t0 = time.perf_counter()
    o.step(ksteps)
    dt = time.perf_counter() - t0
    value = n * ksteps / dt
    sample = f"{n} of {bed.n} parcels (random subset), {ksteps} timed steps after {wsteps} warm-up, FP64"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": ksteps, "warmup": wsteps, "ms_per_step": 1e3 * dt / ksteps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}", "parcels_sampled": n, "precision": "fp64 oracle",
                       "radiation": bool(args.radiation)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2311_03908_gb300 import binding
    stream = torch.cuda.current_stream()
    if args.only_leg:
        tun = {k: int(v) for k, v in (kv.split("=") for kv in args.tuning.split(","))} if args.tuning else {}
        if args.only_leg == "gas_solver":
            leg = gas_solver_leg(binding, stream, tun, args.steps, args.precision, args.workload)
        else:
            leg = dense_leg(binding, stream, tun, 100, args.steps, args.precision, args.parcels,
                            conduction=args.only_leg == "dense_conduction")
        if rank == 0:
            print(json.dumps({"impl": "ours", args.only_leg: leg}), flush=True)
        return
    bed = make_workload(args.workload, rank, args.parcels, args.radiation, args.conduction)
    ctx = binding.Context(bed, precision=args.precision, stream=stream.cuda_stream)
    n = bed.n
    if args.settle > 0:
        ctx.dem_step(args.settle)
        ctx.dem_sync()
    if args.tuning:
        ctx.dem_set_tuning(**{k: int(v) for k, v in (kv.split("=") for kv in args.tuning.split(","))})
        tuning = ctx.dem_get_tuning()
    else:
        tuning = ctx.dem_autotune(args.autotune) if args.autotune > 0 else ctx.dem_get_tuning()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up: W untimed steps (this also captures the two one-step graphs), then one untimed
    # replay of the G-step graph (captured here)
    G = max(1, args.graph_steps)
    for _ in range(args.warmup):
        ctx.dem_step_graph(1)
    warm = args.warmup
    if G > 1 and args.steps >= G:
        ctx.dem_step_graph(G)
        warm += G
    ctx.dem_sync()
    c_pre = ctx.dem_get_counters()
    launches_per_step = None
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    time.sleep(0.2)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    total_launches = 0
    for _ in range(args.steps // G):
        ctx.dem_step_graph(G)
        total_launches += ctx.dem_last_launch_count()
    for _ in range(args.steps % G):
        ctx.dem_step_graph(1)
        total_launches += ctx.dem_last_launch_count()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ck = clocks.stop()
    ctx.dem_sync()
    c_post = ctx.dem_get_counters()
    ms_max = max_over_ranks(ms, dist, "cuda")
    value = job_throughput(n, world, args.steps, ms_max)

    # per-kernel device times (CUDA events on the library's stream) over K plain steps
    ctx.dem_profile(True)
    ksteps = args.steps
    ctx.dem_step(ksteps)
    times = ctx.dem_kernel_times()
    ctx.dem_profile(False)
    cnt, _, _ = ctx.dem_get_contacts()
    zbar = float(cnt.mean())
    fc = float((cnt > 0).mean())
    ncells = ctx.ncells
    steps_done, builds, entries = ctx.dem_get_counters()
    L = entries / n
    fbuild = (c_post[1] - c_pre[1]) / max(1, args.steps)
    rsize = 8 if args.precision == "fp64" else 4
    key_bits = max(1, math.ceil(math.log2(max(2, sum(c.nx * c.ny * c.nz for c in bed.beds)))))
    passes = (key_bits + 7) // 8
    peak, peak_kind = measured_peaks()
    kernels = {}
    for name, (nl, tot) in times.items():
        avg = tot / max(nl, 1)
        b = algorithmic_bytes(name, n, ncells, zbar, L, rsize, passes, fbuild, fc,
                              fbuild / max(1, int(tuning.get("restore_every", 1))))
        kernels[name] = {"launches": nl, "avg_ms": avg, "alg_bytes": b,
                         "gbs": (b / (avg * 1e-3) / 1e9) if avg > 0 and b > 0 else None}
    dom = max(kernels, key=lambda k: kernels[k]["avg_ms"]) if kernels else None
    roof = None
    if dom:
        ach = kernels[dom]["gbs"] or 0.0
        roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "peak_kind": f"{peak_kind} HBM copy bandwidth",
                "traffic": measured_traffic(dom, args.workload, args.precision, n),
                "traffic_unit": "bytes per launch (ncu dram read + write)"}
    step_alg = sum(v["alg_bytes"] for v in kernels.values())
    step_ms = ms_max / args.steps

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": warm, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64", "split": "f32+f64", "split_kahan": "f32"}[args.precision],
            "data": "synthetic",
            "config": {"workload": f"{args.workload} ({bed.n} parcels, {ncells} gas cells, {len(bed.beds)} bed(s))",
                       "precision": args.precision, "radiation": bool(args.radiation),
                       "conduction": bool(args.conduction), "stepping": f"CUDA graph of {G} step(s), replayed", "settle_steps": args.settle,
                       "l2": "inputs larger than L2 (parcel state and history ~ 1 GB)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roof, "gpu_launches": total_launches, "clocks": ck,
            "kernels": kernels, "step_alg_bytes": step_alg,
            "step_alg_gbs": step_alg / (step_ms * 1e-3) / 1e9,
            "step_alg_frac": step_alg / (step_ms * 1e-3) / 1e9 / peak,
            "step_survey_bytes": survey_step_bytes(n, ncells, zbar, rsize, passes),
            "step_survey_frac": survey_step_bytes(n, ncells, zbar, rsize, passes) / (step_ms * 1e-3) / 1e9 / peak,
            "zbar_contacts": zbar, "fraction_in_contact": fc,
            "neighbour_lists": {"mean_length": L, "builds_in_timed_steps": c_post[1] - c_pre[1], "builds_total": builds,
                                "steps_total": steps_done},
            "tuning": tuning}

    # the three forms on fresh copies of the workload, each run for the workload's own step
    # count: device time per step and the bed-mean reduction degree against the FP64 form
    if not args.no_fp64_form:
        fsteps = args.form_steps or int(bed.meta.get("steps", 500))
        forms = {}
        for prec in ("fp64", "split", "split_kahan"):
            cx = binding.Context(bed, precision=prec, stream=stream.cuda_stream)
            if prec != "fp64":
                cx.dem_set_tuning(**tuning)
            cx.dem_step_graph(1)          # captures the graphs; untimed, but counted in fsteps
            cx.dem_step_graph(1)
            cx.dem_sync()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(fsteps - 2):
                cx.dem_step_graph(1)
            a1.record(stream)
            torch.cuda.synchronize()
            msf = a0.elapsed_time(a1) / max(1, fsteps - 2)
            fm, _ = cx.dem_reduction_degree()
            forms[prec] = {"ms_per_step": msf, "value": n / (msf * 1e-3), "f_ov_mean": float(fm.mean())}
            cx.close()
        for prec in forms:
            forms[prec]["f_ov_abs_diff_vs_fp64"] = abs(forms[prec]["f_ov_mean"] - forms["fp64"]["f_ov_mean"])
        line["forms"] = {"steps": fsteps, "unit": UNIT, **forms}

    # cost of the adjoint (drag-heat-reaction sub-step, checkpoints + recomputation + reverse
    # sweep) against its forward sweep, on the 64,000-parcel adjoint workload
    if not args.no_radiation_leg and not args.radiation:
        line["radiation"] = radiation_leg(binding, stream, bed, tuning, args.settle, min(args.steps, 200),
                                          args.precision)
    if rank == 0 and not args.no_adjoint:
        line["adjoint"] = adjoint_cost(binding, stream)

    # end to end through the C ABI with host buffers: the coupling round trip of Sec. 4 at
    # each coupling interval n (gas field in, n steps, cell sources and reduction degree out)
    if not args.no_e2e:
        legs = {}
        ke = max(60, min(args.steps, 200))
        for k, ncouple in enumerate(int(v) for v in args.coupling.split(",")):
            barrier()
            r = e2e_coupling(binding, stream, bed, ncouple, dict(tuning, _precision=args.precision),
                             args.settle, ke)
            te = max_over_ranks(r["seconds"], dist, "cuda")
            r["value"] = job_throughput(n, world, r["steps"], te * 1e3)
            legs[str(ncouple)] = r
            if k == 0:
                line["e2e"] = {"value": r["value"], "unit": UNIT, "steps": r["steps"],
                               "h2d_bytes_per_step": int(r["h2d_bytes_per_step"]),
                               "d2h_bytes_per_step": int(r["d2h_bytes_per_step"]),
                               "coupling_interval": ncouple,
                               "api": "every n steps: dem_set_gas (pinned host Y, T) + dem_step_graph(n) + "
                                      "dem_get_sources_occupied (pinned host, 14 doubles and an index per cell "
                                      "holding parcels) + dem_reduction_degree"}
        line["e2e_coupling"] = legs
    if not args.no_dense_leg:
        line["dense"] = dense_leg(binding, stream, tuning, 100, 100, args.precision, args.parcels)
        line["dense_conduction"] = dense_leg(binding, stream, tuning, 100, 100, args.precision, args.parcels,
                                             conduction=True)
    if rank == 0 and not args.no_batched_leg and not args.parcels:
        line["batched_32"] = batched_leg(binding, stream, args.settle, min(max(args.steps, 100), 200),
                                         args.precision)

    if rank == 0 and not args.no_gas_solver_leg and not args.parcels:
        line["gas_solver"] = gas_solver_leg(binding, stream, tuning, min(max(args.steps, 40), 100), args.precision)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(bed, 1, args.cpu_sample)
    mean, _ = ctx.dem_reduction_degree()
    line["f_ov_mean"] = float(mean.mean())
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
