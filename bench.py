"""Benchmark: collided particle-steps/s of the GB300 collisional-PIC step.

Workload: the large 2D slab of solid Al, 8192 x 1024 cells of 5 nm, 80
electrons + 20 Al3+ per cell (0.84e9 macroparticles at the start), 1.8
keV / 80 fs / 5e17 W/cm^2 pulse peaking at 40 fs, every process on, FP32
particle state with FP64-grade (double-float) cell sums: the largest
workload that fits one GPU.  A step is one pass of the whole hot path
(march, sort, collisions, atomic processes, push, deposit, fields) over
the slab.

The slab is first advanced --advance-fs (10 fs, 500 steps) outside the
clock, so that the timed steps run on a plasma that the beam electrons and
the pulse have already ionized (several charge states per cell, more
electrons than at the start), not on the cold Al3+ of step 0; the mean
rate over the advance is reported beside the timed value.

value: particle-steps/s with the state resident in HBM (device-timed with
CUDA events on the context stream, K steps between a synchronize on each
side).  e2e: the same metric through the public API with host buffers:
the H2D load of the initial state and a D2H diagnostics read every step
inside the timed region.  The state (27 GB at the start, ~32 GB at the
timed steps) is far larger than L2.

--impl reference: the FP64 oracle on the host cores, on a bounded sample
of the same workload (a 64 x 64-cell patch of the slab).
"""
import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import pic_inputs as P  # noqa: E402

METRIC = "collided particle-steps/s"
UNIT = "particle-steps/s"
# algorithmic bytes per particle of the per-cell kernel: the 32 B record
# read and written once (written back in the cell's canonical order)
CELL_BYTES_PER_PARTICLE = 64
# whole step: cell kernel 64 B + scatter (36 B read, 32 B written)
STEP_BYTES_PER_PARTICLE = 132
# DRAM bytes per particle of the cell kernel, from one ncu capture of a
# smaller slab of the same make-up (1024 x 256 cells, 28.0 M particles:
# 1782.5 MB on a plain step, 1829.6 MB on a radiation step, 64.0 B per
# particle over the five-step cycle), scaled to a launch by the particle
# count; None when no capture of the current kernel exists
CELL_TRAFFIC_BYTES_PER_PARTICLE = 64.0
# warp instructions per particle of the cell kernel, from the same capture
# (104 on a radiation step, 89 on the others: 92 over the five-step cycle);
# the kernel is bound by instruction issue, so the bench also sets its
# time against the SM issue rate
CELL_WARP_INSTR_PER_PARTICLE = 92.0


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            return float(d.get("hbm_gbs") or d.get("hbm_GBps") or 6800.0), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    def __init__(self):
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-i", "0", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons)}


def aggregate(ms, particle_steps, dist=None, device="cpu"):
    """Whole-job throughput over the ranks: the slowest rank's time and the
    particle-steps of all ranks (replicas: no data-path collective, only
    this reduction of two numbers)."""
    if dist is None:
        return ms, particle_steps / (ms * 1e-3)
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    n = torch.tensor([particle_steps], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item()) / (float(t.item()) * 1e-3)


def workload(cells=None, which="large"):
    """The timed workload: the large 2D slab (8192 x 1024 cells, 80 e + 20 i)
    or, with which="foil", the 2D foil (2048 x 256 cells, 64 e + 16 i);
    cells: a smaller slab of the same make-up (profiling)."""
    if which == "foil":
        cfg, pl = P.cfg_foil_2d(), P.pulse_foil_2d()
    else:
        cfg, pl = P.cfg_large_2d(), P.pulse_large_2d()
    if cells:
        cfg.nx, cfg.ny = cells
        cfg.name = f"al_2d_{cells[0]}x{cells[1]}x5nm_{cfg.ppc_e}e{cfg.ppc_i}i"
    return cfg, pl


def cpu_baseline(steps=32, patch=128, which="large"):
    """The oracle as it stands on a patch of the workload (default 128 x 128
    cells, 1.6 M particles, 32 steps: about 10 s on 16 host cores)."""
    import oracle
    cfg, pl = workload(which=which)
    sub = P.SlabConfig(**{**cfg.to_dict(), "nx": patch, "ny": patch})
    st = P.init_particles(sub)
    o = oracle.OracleSlab(sub, P.standin_tables(), pl)
    o.load(st)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    o.step(1, threads=cores)
    n = st.n_e + st.n_i
    t0 = time.perf_counter()
    o.step(steps, threads=cores)
    dt = time.perf_counter() - t0
    return {"value": n * steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{patch}x{patch}-cell patch of {cfg.name} ({n} particles), {steps} steps after "
                      f"1 warm-up, OpenMP over cells"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg, _ = workload(which=args.workload)
    vals = []
    for _ in range(max(1, args.warmup)):
        cpu_baseline(steps=1, patch=64, which=args.workload)
    cb = None
    for _ in range(args.steps):
        cb = cpu_baseline(steps=2, patch=64, which=args.workload)
        vals.append(cb["value"])
    v = statistics.median(vals)
    cb["value"] = v
    out = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "impl": "reference", "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": cfg.name, "sample": cb["sample"]},
           "cpu_baseline": cb,
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def issue_rate(cell_ms, n_particles, n_sm, sm_mhz):
    """The cell kernel against the SM issue rate: warp instructions per
    particle x particles over its time, against four schedulers per SM
    issuing one warp instruction a cycle at the SM clock sampled during the
    timed steps (the maximum clock when no sample exists)."""
    mhz = sm_mhz if sm_mhz else 2070.0
    peak = 4.0 * n_sm * mhz * 1e6
    achieved = CELL_WARP_INSTR_PER_PARTICLE * n_particles / (cell_ms * 1e-3)
    return {"achieved": achieved, "peak": peak, "unit": "warp instructions/s", "frac": achieved / peak,
            "warp_instructions_per_particle": CELL_WARP_INSTR_PER_PARTICLE, "sm": n_sm, "sm_mhz": mhz,
            "source": "instructions per particle from ncu (profiles/)"}


def capacity(cfg, n_e, n_i):
    """Particle capacity of the timed slab: electrons for a mean charge up to
    9.5 on the large slab (the precision study's figure), for full
    stripping otherwise, within what 32-bit particle indices hold
    (cap_e + 3 cap_i below 2^31)."""
    import paper_1704_01202_gb300 as pkg
    ce, ci = pkg.default_capacity(n_e, n_i, cfg.Z_init)
    return min(ce, int(9.5 * n_i) + 1024, (1 << 31) - 1 - 3 * ci), ci


ENERGY_KEYS = ("ke_e", "ke_i", "e_ion", "e_phot", "e_field", "e_esc", "e_trans", "e_ka_esc")


def energy_total(d):
    """Total energy of the diagnostics' bookkeeping (eV x weight): kinetic,
    ionization, photons in the slab, fields, escaped and transmitted, minus
    what the pulse brought in."""
    return sum(d[k] for k in ENERGY_KEYS) - d["e_inc"]


def energy_drift(d0, d1, d2, n01, n12):
    """Relative change of the total energy per 1000 steps, over the advance
    (d0 -> d1, n01 steps) and the timed steps (d1 -> d2), against the energy
    the slab holds (kinetic + ionization + photons + fields) at d1."""
    held = sum(d1[k] for k in ("ke_e", "ke_i", "e_ion", "e_phot", "e_field"))
    out = {"reference": "energy held at the start of the timed steps", "held": held}
    for name, a, b, n in (("advance", d0, d1, n01), ("timed", d1, d2, n12)):
        out[name] = {"steps": n, "rel_per_1000_steps": (energy_total(b) - energy_total(a)) / held * 1000.0 / max(n, 1)}
    return out


def charge_states(csd, share=0.01):
    """Charge states holding more than `share` of the ions."""
    return [z for z, f in enumerate(csd) if f > share]


def run_gpu(args):
    import torch
    import paper_1704_01202_gb300 as pkg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    pkg.build()
    cfg, pl = workload(args.cells, args.workload)
    # replicas: every rank runs its own slab with its own seed
    cfg.seed = cfg.seed + rank
    tab = P.standin_tables()
    # one GPU: the initial state built on the host and loaded (the e2e leg
    # needs the host copy); several: seeded on each device (pic_seed, the
    # same distributions), since N host copies of a 0.84e9-particle state
    # would take N x ~80 GB of host memory
    host_state = world == 1
    t_gen = time.perf_counter()
    st = P.init_particles(cfg) if host_state else None
    t_gen = time.perf_counter() - t_gen
    n_e0, n_i0 = (st.n_e, st.n_i) if host_state else (cfg.ncell * cfg.ppc_e, cfg.ncell * cfg.ppc_i)
    n0 = n_e0 + n_i0
    cap_e, cap_i = capacity(cfg, n_e0, n_i0)
    slab = pkg.Slab(cfg, tab, pl, cap_e=cap_e, cap_i=cap_i)
    if host_state:
        slab.load(st)
    else:
        slab.seed()
    stream = torch.cuda.current_stream()

    # advance outside the clock, timed as a whole for the mean; its last
    # steps autotune the cell kernel's launch shape for the state the timed
    # steps see (these are real steps of the run)
    n_adv = int(round(args.advance_fs / cfg.dt_fs))
    tune_steps = 0 if args.no_autotune else min(9, n_adv)
    adv = {"steps": n_adv, "fs": n_adv * cfg.dt_fs}
    ne_a, ni_a = slab.counts()
    d_start = slab.diagnostics()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a0.record(stream)
    if n_adv > tune_steps:
        slab.step(n_adv - tune_steps)
    if tune_steps:
        slab.autotune(True)
        slab.step(tune_steps)
        slab.autotune(False)
    a1.record(stream)
    torch.cuda.synchronize()
    ne_b, ni_b = slab.counts()
    if n_adv:
        adv_ms = a0.elapsed_time(a1)
        adv["value"] = 0.5 * (ne_a + ni_a + ne_b + ni_b) * n_adv / (adv_ms * 1e-3)
        adv["ms_per_step"] = adv_ms / n_adv
    for _ in range(args.warmup):
        slab.step(1)
    slab.sync()
    tuned = slab.autotune()
    dw = slab.diagnostics()
    window = {"t_fs": [dw["t_fs"], dw["t_fs"] + args.steps * cfg.dt_fs], "Zbar": dw["Zbar"],
              "charge_states_over_1pct": charge_states(dw["csd"]), "T_e_eV": dw["T_e_eV"],
              "electrons_per_ion": dw["n_e"] / max(dw["n_i"], 1)}
    ne0, ni0 = slab.counts()
    if dist:
        dist.barrier()
    clocks = ClockSampler()
    clocks.start()
    slab.timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    slab.step(args.steps)
    launches = slab.launches
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    tms, nrec = slab.timing(None)
    slab.timing(False)
    ne1, ni1 = slab.counts()
    d_end = slab.diagnostics()
    energy = energy_drift(d_start, dw, d_end, n_adv + args.warmup, args.steps)
    n_mean = 0.5 * (ne0 + ni0 + ne1 + ni1)
    ms, value = aggregate(ms, n_mean * args.steps, dist, "cuda")

    # dominant kernel roofline: the per-cell kernel
    peak, peak_kind = measured_peaks()
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    cell_ms = tms["cell"] / max(nrec, 1)
    achieved = CELL_BYTES_PER_PARTICLE * n_mean / (cell_ms * 1e-3) / 1e9
    traffic = CELL_TRAFFIC_BYTES_PER_PARTICLE * n_mean if CELL_TRAFFIC_BYTES_PER_PARTICLE else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_note": "ncu DRAM bytes of a smaller slab of the same make-up, "
                                                "scaled by particles (profiles/)",
            "kernel": "k_cell", "peak_source": peak_kind,
            "bytes_per_particle": CELL_BYTES_PER_PARTICLE, "kernel_ms_per_step": cell_ms,
            "share_of_step": tms["cell"] / max(tms["step"], 1e-9),
            "issue": issue_rate(cell_ms, n_mean, n_sm, clk.get("sm_mhz"))}
    step_gbs = STEP_BYTES_PER_PARTICLE * n_mean / (ms / args.steps * 1e-3) / 1e9

    # end to end through the public API with host buffers
    slab.close()
    del slab
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    e2e = None
    if not args.no_e2e and host_state:
        e2e = run_e2e(pkg, cfg, tab, pl, st, args, world, n0, (cap_e, cap_i))
    elif not args.no_e2e:
        e2e = {"value": None, "skipped": "N > 1: a host copy of the initial state per rank would need N x ~80 GB "
                                         "of host memory; the state was seeded on each device"}
    del st
    torch.cuda.empty_cache()
    foil = run_foil(pkg, tab, args) if args.foil_steps > 0 and args.workload != "foil" else None
    rt = run_rt(pkg, tab, args) if args.rt_steps > 0 else None
    mc_energy = run_mc_energy(pkg, tab, args) if args.mc_energy_steps > 0 else None
    ensemble = run_ensemble(pkg, tab, args, rank) if args.ensemble > 0 else None
    served = run_served(pkg, tab, args) if args.serve_n > 0 else None
    kedge_scan = run_kedge(pkg, tab, args) if args.kedge_points > 0 else None
    thermal = run_thermal(pkg, tab, args) if args.thermal_horizon_fs > 0 else None
    extreme = run_extreme(pkg, tab, args) if args.extreme_horizon_fs > 0 else None
    if dist:
        dist.barrier()
    if rank == 0:
        cb = cpu_baseline(which=args.workload) if world == 1 and not args.no_cpu else None
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": cfg.name, "cells": [cfg.nx, cfg.ny], "particles": int(n_mean),
                          "particles_start": int(n0), "ppc": [cfg.ppc_e, cfg.ppc_i], "pulse_keV": pl.hv_eV / 1e3,
                          "pulse_Wcm2": pl.I_peak_Wcm2, "pulse_peak_fs": pl.t_peak_fs,
                          "l2": f"state ({n_mean * 32 / 1e9:.0f} GB) larger than L2; no flush",
                          "parallelism": "replicas", "host_generation_s": round(t_gen, 1),
                          "initial_state": "host generator, loaded" if host_state else "seeded on the device"},
               "timed_window": window, "advance": adv, "energy_drift": energy,
               "energy_drift_collisions_and_atomic": mc_energy,
               "roofline": roof, "step_hbm_gbs": step_gbs, "cpu_baseline": cb, "e2e": e2e,
               "gpu_launches": int(launches), "clocks": clk, "kernel_ms": {k: v / max(nrec, 1) for k, v in tms.items()},
               "autotune": {"cell_warps_per_cta": tuned[0], "cell_ms_1_2_4_8": [float(x) for x in tuned[1]]},
               "foil_2048x256": foil, "radiation_transport": rt, "ensemble": ensemble, "served": served, "kedge_scan": kedge_scan,
               "thermalization": thermal, "extreme_10keV": extreme}
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def run_rt(pkg, tab, args):
    """The 2D foil with radiation transport instead of the ballistic march
    (rad cells of 8 x 8 PIC cells, the beam plus 4 polar x 2 azimuthal
    ordinates, CIP): the same timing as the foil leg, with the transport's
    share of the step (the "march" group of the timing)."""
    import torch
    cfg, pl = workload(None, "foil")
    st = P.init_particles(cfg)
    slab = pkg.Slab(cfg, tab, pl)
    slab.load(st)
    del st
    slab.set_rt(coarsen=8, n_polar=4, n_azimuth=2, scheme=0)
    stream = torch.cuda.current_stream()
    slab.autotune(True)
    slab.step(9)
    slab.autotune(False)
    slab.step(max(args.warmup, 3))
    slab.sync()
    ne0, ni0 = slab.counts()
    slab.timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    slab.step(args.rt_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    tms, nrec = slab.timing(None)
    ne1, ni1 = slab.counts()
    d = slab.diagnostics()
    slab.close()
    n_mean = 0.5 * (ne0 + ni0 + ne1 + ni1)
    return {"workload": cfg.name + ", radiation transport: rad cells 8 x 8, 1 + 4 x 2 ordinates, CIP",
            "particles": int(n_mean), "steps": args.rt_steps, "value": n_mean * args.rt_steps / (ms * 1e-3),
            "unit": UNIT, "ms_per_step": ms / args.rt_steps,
            "transport_ms_per_step": tms["march"] / max(nrec, 1),
            "kernel_ms": {k: v / max(nrec, 1) for k, v in tms.items()},
            "transport_energy_gain_over_incident": d["e_rt_num"] / d["e_inc"] if d["e_inc"] > 0 else None}


def run_foil(pkg, tab, args):
    """The 2D foil (2048 x 256 cells of 5 nm, 64 e + 16 i per cell, 1.6 keV /
    1e17 W/cm^2), timed the same way from its first steps (autotuning,
    warm-up, then --foil-steps steps)."""
    import torch
    cfg, pl = workload(None, "foil")
    st = P.init_particles(cfg)
    slab = pkg.Slab(cfg, tab, pl)
    slab.load(st)
    del st
    stream = torch.cuda.current_stream()
    slab.autotune(True)
    slab.step(9)
    slab.autotune(False)
    slab.step(max(args.warmup, 3))
    slab.sync()
    ne0, ni0 = slab.counts()
    slab.timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    slab.step(args.foil_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    tms, nrec = slab.timing(None)
    ne1, ni1 = slab.counts()
    slab.close()
    n_mean = 0.5 * (ne0 + ni0 + ne1 + ni1)
    return {"workload": cfg.name, "particles": int(n_mean), "steps": args.foil_steps,
            "value": n_mean * args.foil_steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / args.foil_steps,
            "kernel_ms": {k: v / max(nrec, 1) for k, v in tms.items()}}


def run_mc_energy(pkg, tab, args):
    """Energy bookkeeping of the collision and atomic operators alone at
    scale: a 1024 x 256-cell slab of the headline's make-up with push and
    fields off (every other process on, the pulse peak moved to 2 fs so that
    photoionization and K decay run), --mc-energy-steps steps seeded on the
    device: the total energy's relative change per 1000 steps."""
    cfg, pl = workload((1024, 256), "large")
    cfg.flags = cfg.flags & ~(P.F_PUSH | P.F_FIELD)
    pl.t_peak_fs = 2.0
    slab = pkg.Slab(cfg, tab, pl)
    slab.seed()
    d0 = slab.diagnostics()
    slab.step(args.mc_energy_steps)
    d1 = slab.diagnostics()
    slab.close()
    held = sum(d1[k] for k in ("ke_e", "ke_i", "e_ion", "e_phot"))
    return {"workload": cfg.name + ", push and fields off, pulse peak at 2 fs", "steps": args.mc_energy_steps,
            "rel_per_1000_steps": (energy_total(d1) - energy_total(d0)) / held * 1000.0 / args.mc_energy_steps,
            "events": {k: d1["counts"][k] for k in ("ION", "REC", "PH0", "AUG", "KA", "EE", "EI")}}


def run_ensemble(pkg, tab, args, rank):
    """The batched ensemble: 256 independent 1D slabs (cells log-uniform
    64-4096, 32-512 particles per cell) stepped together, one launch of each
    kernel per step for all of them."""
    import torch
    ens = P.batched_ensemble(n=args.ensemble, seed=7 + rank)
    states = [P.init_particles(c) for c, _ in ens]
    cap_e = cap_i = 0
    for (c, _), st in zip(ens, states):
        e, i = pkg.default_capacity(st.n_e, st.n_i, c.Z_init)
        cap_e, cap_i = cap_e + e, cap_i + i
    slot_cells = max(c.nx for c, _ in ens)
    bt = pkg.Batch(tab, len(ens), slot_cells, cap_e, cap_i)
    for (c, pl), st in zip(ens, states):
        bt.admit(c, st, pl)
    bt.autotune(True)
    bt.step(9 + args.warmup)
    bt.autotune(False)
    bt.sync()
    tuned = bt.autotune()
    n0 = sum(sum(bt.counts(k)) for k in range(len(ens)))
    stream = torch.cuda.current_stream()
    bt.timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    bt.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = bt.launches
    tms, nrec = bt.timing(None)
    n1 = sum(sum(bt.counts(k)) for k in range(len(ens)))
    bt.close()
    n_mean = 0.5 * (n0 + n1)
    return {"workload": f"{len(ens)} 1D Al slabs, cells log-uniform 64-4096 (2 nm), 32-512 particles per cell, "
                        "I log-uniform 1e15-1e18 W/cm^2, hv U(1.58, 1.90) keV",
            "slabs": len(ens), "slot_cells": slot_cells, "particles": int(n_mean), "steps": args.steps,
            "value": n_mean * args.steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / args.steps,
            "gpu_launches": int(launches), "kernel_ms": {k: v / max(nrec, 1) for k, v in tms.items()},
            "autotune": {"cell_warps_per_cta": tuned[0], "cell_ms_1_2_4_8": [float(x) for x in tuned[1]]}}


def run_served(pkg, tab, args):
    """Served loop: Poisson arrivals of slab requests, continuous batching
    with admission by reserved footprint; more requests than fit at once,
    so that arrivals queue.  The plain one-at-a-time form runs a fixed
    sample of the same requests back to back (its rate under a backlog is
    one request per service time, whatever the arrival times)."""
    from paper_1704_01202_gb300 import serve
    tr = P.request_trace(n=args.serve_n, rate_hz=200.0, seed=11, horizon_fs=args.serve_horizon_fs)
    # request payloads (initial particles) are built before the clock starts:
    # a client sends them with the request
    payload = {r.rid: P.init_particles(r.cfg) for r in tr}
    init = lambda r: payload[r.rid]  # noqa: E731
    fp = [serve.footprint(r.cfg, r.pulse) for r in tr]
    slot_cells = max(r.cfg.nx for r in tr)
    # resident capacity: the slots, and room for about serve_room average
    # reservations at once
    room = args.serve_room
    cap_e = max(max(f[0] for f in fp), int(room * sum(f[0] for f in fp) / len(fp)))
    cap_i = max(max(f[1] for f in fp), int(room * sum(f[1] for f in fp) / len(fp)))
    b = serve.serve_batched(tr, tab, init, max_slabs=args.serve_slots, slot_cells=slot_cells,
                            cap_e=cap_e, cap_i=cap_i, tick_steps=args.serve_tick)
    sample = [dataclasses.replace(r, t_arrive=0.0) for r in tr[::args.serve_every]]
    o = serve.serve_one_at_a_time(sample, tab, init)
    psteps = sum(r.nsteps * r.cfg.ncell * (r.cfg.ppc_e + r.cfg.ppc_i) for r in tr)
    keys = ("slabs_per_s", "ttr_p50_s", "ttr_p99_s", "ttr_mean_s", "wall_s", "wait_p50_s", "wait_p99_s",
            "max_queue", "preempted", "busy_s")
    return {"trace": f"{len(tr)} Poisson arrivals at 200/s, ensemble draws + thickness U(0.2, 2) um, "
                     f"each run {args.serve_horizon_fs:g} fs ({tr[0].nsteps} steps)",
            "batched": {k: b[k] for k in keys}, "failed": len(b["failed"]),
            "one_at_a_time": {"slabs_per_s": o["slabs_per_s"], "wall_s": o["wall_s"],
                              "service_p50_s": float(np.percentile(np.diff([0.0] + sorted(o["ttr"].values())), 50)),
                              "sample": f"every {args.serve_every}th request ({len(sample)}), run back to back"},
            "speedup_slabs_per_s": b["slabs_per_s"] / o["slabs_per_s"],
            "particle_steps": int(psteps), "particle_steps_per_s": psteps / b["wall_s"],
            "max_slabs": args.serve_slots, "room_avg_requests": room, "slot_cells": slot_cells}


def run_kedge(pkg, tab, args):
    """K-edge transmission sweep (photon energy x continuum-lowering model),
    every point a slab of one batch."""
    from paper_1704_01202_gb300 import kedge
    hv = np.linspace(1540.0, 1870.0, args.kedge_points)
    slabs = kedge.scan_slabs(P, hv)
    nsteps = int(round(args.kedge_horizon_fs / slabs[0][0].dt_fs))
    res = kedge.run_scan(tab, slabs, P.init_particles, nsteps)
    curve = {}
    for r in res["points"]:
        curve.setdefault({1: "EK", 2: "SP"}.get(r["ipd"], str(r["ipd"])), []).append(round(r["transmission"], 5))
    return {"workload": f"{len(slabs)} 1D foils of 250 x 2 nm, 64 e + 16 i per cell, 10 fs / 1e17 W/cm^2 pulse, "
                        f"{args.kedge_horizon_fs:g} fs", "hv_eV": [float(x) for x in hv], "transmission": curve,
            "steps": nsteps, "wall_s": res["wall_s"], "particle_steps_per_s": res["particle_steps_per_s"]}


def run_thermal(pkg, tab, args):
    """Non-thermal against force-thermalized electrons: the small 1D slab
    under a 1.7 keV, 80 fs, 1.36e17 W/cm^2 pulse, both variants in one batch."""
    from paper_1704_01202_gb300 import thermal
    cfg = P.cfg_small_1d(nx=128, flags=P.F_ALL)
    pulse = P.Pulse(I_peak_Wcm2=1.36e17, fwhm_fs=80.0, t_peak_fs=80.0, hv_eV=1700.0)
    r = thermal.compare(tab, cfg, pulse, P.init_particles, args.thermal_horizon_fs, 10.0, P.F_THERM)
    r["workload"] = (f"al_1d_128x2nm_256e64i, 1.7 keV / 80 fs / 1.36e17 W/cm^2, {args.thermal_horizon_fs:g} fs, "
                     "with and without forced thermalization")
    for k in ("Zbar", "Zbar_therm", "T_e_eV", "T_e_eV_therm"):
        r[k] = [round(x, 4) for x in r[k]]
    return r


def run_extreme(pkg, tab, args):
    """The 10 keV extreme case (Sec. VI C): 8 keV photoelectrons and
    1.4 keV Auger electrons in the small slab under a 10 keV, 20 fs,
    1e19 W/cm^2 pulse, with and without forced thermalization, and the share
    of the free-electron energy above 700 eV."""
    from paper_1704_01202_gb300 import thermal
    cfg = P.cfg_small_1d(nx=128, flags=P.F_ALL)
    pulse = P.Pulse(I_peak_Wcm2=1.0e19, fwhm_fs=20.0, t_peak_fs=30.0, hv_eV=10000.0)
    r = thermal.compare(tab, cfg, pulse, P.init_particles, args.extreme_horizon_fs, 10.0, P.F_THERM, tail_eV=700.0)
    r["workload"] = (f"al_1d_128x2nm_256e64i, 10 keV / 20 fs / 1e19 W/cm^2 peak at 30 fs, "
                     f"{args.extreme_horizon_fs:g} fs, with and without forced thermalization")
    for k in ("Zbar", "Zbar_therm", "T_e_eV", "T_e_eV_therm", "tail_number_share", "tail_energy_share"):
        r[k] = [round(x, 4) for x in r[k]]
    return r


def run_e2e(pkg, cfg, tab, pl, st, args, world, n0, caps):
    """Public API with host buffers: context, H2D load, steps with a D2H
    diagnostics read after each; 100 steps (2 fs), so that the one-time
    set-up weighs as it would in a run."""
    e2e_steps = 100
    t0 = time.perf_counter()
    s2 = pkg.Slab(cfg, tab, pl, cap_e=caps[0], cap_i=caps[1])
    s2.load(st)
    d2h = 0
    for _ in range(e2e_steps):
        s2.step(1)
        d = s2.diagnostics(n_E=64)
        d2h += (pkg.NZ + 64) * 8 + 16 * 8 + 20 * 8
    t_e2e = time.perf_counter() - t0
    h2d = st.n_e * (8 + 8 + 12 + 4 + 8) + st.n_i * (8 + 8 + 12 + 4 + 4 + 4 + 4)
    s2.close()
    return {"value": world * n0 * e2e_steps / t_e2e, "unit": UNIT,
            "h2d_bytes_per_step": int(h2d / e2e_steps), "d2h_bytes_per_step": int(d2h / e2e_steps),
            "steps": e2e_steps, "includes": "context creation, H2D load of the initial state, "
                                           "per-step diagnostics D2H"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="large", choices=["large", "foil"],
                    help="timed slab: the large 2D slab (8192 x 1024) or the 2D foil (2048 x 256)")
    ap.add_argument("--cells", type=int, nargs=2, default=None, help="smaller slab of the same make-up (profiling)")
    ap.add_argument("--advance-fs", type=float, default=10.0,
                    help="simulated time run before the timed steps, outside the clock")
    ap.add_argument("--foil-steps", type=int, default=20, help="timed steps of the 2D foil leg (0: skip)")
    ap.add_argument("--rt-steps", type=int, default=20,
                    help="timed steps of the 2D foil with radiation transport (0: skip)")
    ap.add_argument("--mc-energy-steps", type=int, default=500,
                    help="steps of the collision / atomic energy bookkeeping leg (0: skip)")
    ap.add_argument("--ensemble", type=int, default=256, help="slabs of the batched ensemble (0: skip)")
    ap.add_argument("--serve-n", type=int, default=240, help="requests of the served trace (0: skip)")
    ap.add_argument("--serve-slots", type=int, default=128, help="slots of the served batch")
    ap.add_argument("--serve-room", type=float, default=96.0,
                    help="electron and ion capacity of the served batch, in average request reservations")
    ap.add_argument("--serve-tick", type=int, default=25, help="steps between admissions / retirements")
    ap.add_argument("--serve-every", type=int, default=16,
                    help="the one-at-a-time form runs every n-th request of the trace")
    ap.add_argument("--serve-horizon-fs", type=float, default=150.0,
                    help="simulated time per served request (the workload's 150 fs)")
    ap.add_argument("--kedge-points", type=int, default=12, help="photon energies of the K-edge sweep (0: skip)")
    ap.add_argument("--kedge-horizon-fs", type=float, default=30.0)
    ap.add_argument("--thermal-horizon-fs", type=float, default=60.0, help="0: skip")
    ap.add_argument("--extreme-horizon-fs", type=float, default=60.0, help="10 keV case; 0: skip")
    ap.add_argument("--no-autotune", action="store_true",
                    help="default launch shapes (profiling: timings under a profiler mislead the tuner)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "gb300" else args.warmup
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
