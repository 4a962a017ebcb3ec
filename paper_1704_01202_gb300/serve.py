"""Serving of independent slab simulations on one GPU.

`serve_batched` is continuous batching over the batch context of the C ABI
(pic_batch_*): requests are admitted as they arrive whenever a slot is free
and their worst-case particle footprint fits the arena, every kernel of a
step runs once for all resident slabs, and a slab leaves (diagnostics read,
slot retired) as soon as it has run its steps.  `serve_one_at_a_time` is
the plain form: one single-slab context per request, in arrival order.

Both replay the same arrival trace in real time and return per-request
time-to-result (result ready minus arrival) and the drained slabs/s.  A
slab's result is the same alone and in the mix (its random streams are
keyed by its own seed, ids and step count).

    python -m paper_1704_01202_gb300.serve --requests 40 --horizon-fs 150
    python -m paper_1704_01202_gb300.serve --static 48 --steps 4
"""
from __future__ import annotations

import time

import numpy as np

from . import Batch, Slab, default_capacity


F_PHOTO = 16          # the photoionization flag of pic_species


def footprint(cfg, pulse=None, partial_per_cell: int = 1) -> tuple[int, int]:
    """Electron and ion slots reserved for a slab at admission.

    Electrons: the slab's own, one per charge its ions can still lose by
    whole events (every ion stripped), and partial_per_cell partial-event
    electrons per photon bin per cell: an absorption of fewer photons than
    one ion weight (Sec. III, Eq. 2) creates an electron macroparticle of
    fractional weight and advances the ion's charge by that fraction only,
    so these electrons are not bounded by the charge the ions can lose.
    Their worst case, one per bin per cell per rad step (partial_bound), is
    far above what a slab creates; a slab that outgrows its reservation is
    stopped by its budget and run again with a larger one."""
    n_e, n_i = cfg.ncell * cfg.ppc_e, cfg.ncell * cfg.ppc_i
    nb = pulse.n_bins if pulse is not None and (cfg.flags & F_PHOTO) else 0
    return n_e + n_i * (13 - cfg.Z_init) + cfg.ncell * nb * partial_per_cell, n_i


def partial_bound(cfg, pulse, nsteps: int) -> int:
    """Most partial-event electrons a slab can create in nsteps: one per
    photon bin per cell per rad step."""
    if pulse is None or not (cfg.flags & F_PHOTO) or cfg.rad_every <= 0:
        return 0
    return cfg.ncell * pulse.n_bins * (-(-nsteps // cfg.rad_every))


def _summary(ttr: dict, t0: float, t_end: float, n: int) -> dict:
    v = np.array([ttr[k] for k in sorted(ttr)]) if ttr else np.zeros(1)
    return {"slabs": n, "wall_s": t_end - t0, "slabs_per_s": n / (t_end - t0),
            "ttr_p50_s": float(np.percentile(v, 50)), "ttr_p99_s": float(np.percentile(v, 99)),
            "ttr_mean_s": float(v.mean())}


def serve_batched(trace, tables, init_state, max_slabs: int, slot_cells: int, cap_e: int, cap_i: int,
                  tick_steps: int = 25, keep=None, diag_bins: int = 64, autotune: bool = False,
                  grow: int = 4, batch=None) -> dict:
    """Continuous batching of `trace` (requests sorted by arrival).

    init_state(request) -> ParticleState gives a request's particles (the
    request payload, on the host).  keep(rid) -> bool selects requests whose
    final particles are returned (for tests).

    Admission: first come first served, while a slot is free and the
    request's reservation (footprint) fits beside the others' in cap_e /
    cap_i; later arrivals wait in the queue.  Each admitted slab gets its
    reservation as its electron budget on the device, so the reservations
    never overcommit the shared capacity and a slab that outgrows its own is
    stopped alone (pic_batch_set_budget) while the others run on.  Such a
    slab is preempted: its slot and reservation are freed and it is queued
    again, at the head, with grow times the partial-event allowance; its
    result does not depend on where or when it runs, so the re-run returns
    what an unconstrained run would.  The allowance grows up to the worst
    case or the most cap_e holds; a request that outgrows that fails alone
    (reported in `failed`; beyond the worst case only when its ions are
    stripped again after recombining).  A request wider than a slot, or
    whose first reservation is beyond the batch's capacity, is refused alone
    on arrival (also in `failed`).  autotune: let the launch-shape autotuner time the cell
    kernel's warps per CTA for each new staging size (results do not depend
    on it).  batch: an object with the Batch interface to drive instead of
    a new Batch (host-logic tests)."""
    bt = batch if batch is not None else Batch(tables, max_slabs, slot_cells, cap_e, cap_i)
    if autotune:
        bt.autotune(True)
    pending = list(trace)
    allowance = {}                   # rid -> partial-event electrons per bin per cell
    active = {}                      # slot -> [request, steps left, reservation]
    res_e = res_i = 0
    ttr, results, finals, failed = {}, {}, {}, {}
    admitted_at, preempted, max_queue = {}, 0, 0
    busy = {"step": 0.0, "admit": 0.0, "results": 0.0}   # host wall time by phase
    t0 = time.perf_counter()
    try:
        while pending or active:
            now = time.perf_counter() - t0
            # admit what has arrived, in order, while it fits
            while pending and pending[0].t_arrive <= now:
                r = pending[0]
                a = allowance.setdefault(r.rid, 1)
                fe, fi = footprint(r.cfg, r.pulse, a)
                if r.cfg.nx > slot_cells or fe > cap_e or fi > cap_i:
                    # refused alone; the rest of the trace is served
                    if r.cfg.nx > slot_cells:
                        failed[r.rid] = f"{r.cfg.nx} cells, more than a slot's {slot_cells}"
                    elif a == 1:
                        failed[r.rid] = f"its footprint ({fe} electron, {fi} ion slots) is beyond the batch's " \
                                        f"capacity ({cap_e}, {cap_i})"
                    else:
                        failed[r.rid] = f"needs more than {cap_e} electron slots"
                    ttr[r.rid] = time.perf_counter() - t0 - r.t_arrive
                    pending.pop(0)
                    continue
                if len(active) >= max_slabs or res_e + fe > cap_e or res_i + fi > cap_i:
                    break
                ta = time.perf_counter()
                slot = bt.admit(r.cfg, init_state(r), r.pulse)
                bt.set_budget(slot, fe)
                busy["admit"] += time.perf_counter() - ta
                active[slot] = [r, r.nsteps, (fe, fi)]
                admitted_at.setdefault(r.rid, now)
                res_e, res_i = res_e + fe, res_i + fi
                pending.pop(0)
            max_queue = max(max_queue, sum(1 for q in pending if q.t_arrive <= now))
            if not active:
                if pending:
                    time.sleep(max(0.0, pending[0].t_arrive - (time.perf_counter() - t0)))
                continue
            n = min(tick_steps, min(a[1] for a in active.values()))
            ts = time.perf_counter()
            bt.step(n)
            stopped = set(bt.failed())
            tr_ = time.perf_counter()
            busy["step"] += tr_ - ts
            back = []
            for slot in list(active):
                a = active[slot]
                r = a[0]
                if slot in stopped:
                    # preempted: free the slot and the reservation, queue again
                    # with a larger one (up to one partial-event electron per
                    # bin per cell per rad step of the horizon)
                    bt.retire(slot)
                    res_e, res_i = res_e - a[2][0], res_i - a[2][1]
                    del active[slot]
                    worst = -(-r.nsteps // max(1, r.cfg.rad_every))
                    per = max(1, r.cfg.ncell * (r.pulse.n_bins if r.pulse is not None else 1))
                    fits = (cap_e - footprint(r.cfg, r.pulse, 0)[0]) // per    # the most the capacity holds
                    if allowance[r.rid] >= min(worst, fits):
                        failed[r.rid] = f"went beyond the {a[2][0]} electron slots of its " + \
                                        ("worst case" if allowance[r.rid] >= worst else "largest reservation")
                        ttr[r.rid] = time.perf_counter() - t0 - r.t_arrive
                        continue
                    allowance[r.rid] = min(worst, fits, allowance[r.rid] * grow)
                    preempted += 1
                    back.append(r)
                    continue
                a[1] -= n
                if a[1] == 0:
                    results[r.rid] = bt.diagnostics(slot, n_E=diag_bins)
                    if keep is not None and keep(r.rid):
                        finals[r.rid] = (bt.electrons(slot), bt.ions(slot))
                    ttr[r.rid] = time.perf_counter() - t0 - r.t_arrive
                    bt.retire(slot)
                    res_e, res_i = res_e - a[2][0], res_i - a[2][1]
                    del active[slot]
            pending[:0] = sorted(back, key=lambda q: q.t_arrive)
            busy["results"] += time.perf_counter() - tr_
        bt.sync()
        t_end = time.perf_counter()
    finally:
        if batch is None:
            bt.close()
    out = _summary(ttr, t0, t_end, len(trace))
    wait = np.array([admitted_at[k] - q.t_arrive for q in trace for k in [q.rid] if k in admitted_at])
    out.update(results=results, finals=finals, ttr=ttr, failed=failed, preempted=preempted,
               max_queue=max_queue, busy_s=busy, wait_p50_s=float(np.percentile(wait, 50)) if len(wait) else 0.0,
               wait_p99_s=float(np.percentile(wait, 99)) if len(wait) else 0.0)
    return out


def serve_one_at_a_time(trace, tables, init_state, keep=None, diag_bins: int = 64) -> dict:
    """The plain form: each request in arrival order gets its own
    single-slab context, runs to its horizon, and is freed."""
    ttr, results, finals = {}, {}, {}
    t0 = time.perf_counter()
    for r in trace:
        wait = r.t_arrive - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        st = init_state(r)
        ce, ci = default_capacity(st.n_e, st.n_i, r.cfg.Z_init)
        s = Slab(r.cfg, tables, r.pulse, cap_e=ce, cap_i=ci)
        try:
            s.load(st)
            s.step(r.nsteps)
            results[r.rid] = s.diagnostics(n_E=diag_bins)
            if keep is not None and keep(r.rid):
                finals[r.rid] = (s.electrons(), s.ions())
        finally:
            s.close()
        ttr[r.rid] = time.perf_counter() - t0 - r.t_arrive
    out = _summary(ttr, t0, time.perf_counter(), len(trace))
    out.update(results=results, finals=finals, ttr=ttr)
    return out


def main():
    """Replay the seeded request trace (continuous batching against one at a
    time), or with --static N admit the first N requests at once and run K
    steps of the batch (a fixed batch for profiling the batched kernels)."""
    import argparse
    import json
    import pic_inputs as P
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=40)
    ap.add_argument("--horizon-fs", type=float, default=150.0)
    ap.add_argument("--static", type=int, default=0, help="admit this many requests at once and step")
    ap.add_argument("--steps", type=int, default=4)
    args = ap.parse_args()
    tab = P.standin_tables()
    if args.static:
        tr = P.request_trace(n=args.static, rate_hz=200.0, seed=11, horizon_fs=args.horizon_fs)
        fp = [footprint(r.cfg, r.pulse) for r in tr]
        bt = Batch(tab, len(tr), max(r.cfg.nx for r in tr), sum(f[0] for f in fp) + 1024, sum(f[1] for f in fp) + 1024)
        try:
            bt.use_graphs(False)
            for r in tr:
                bt.admit(r.cfg, P.init_particles(r.cfg), r.pulse)
            t0 = time.perf_counter()
            bt.step(args.steps)
            bt.sync()
            wall = time.perf_counter() - t0
        finally:
            bt.close()
        print(json.dumps({"requests": len(tr), "steps": args.steps, "wall_s": wall,
                          "particles": int(sum(r.cfg.ncell * (r.cfg.ppc_e + r.cfg.ppc_i) for r in tr))}))
        return
    tr = P.request_trace(n=args.requests, rate_hz=200.0, seed=11, horizon_fs=args.horizon_fs)
    payload = {r.rid: P.init_particles(r.cfg) for r in tr}
    fp = [footprint(r.cfg, r.pulse) for r in tr]
    cap_e = max(max(f[0] for f in fp), int(64 * sum(f[0] for f in fp) / len(fp)))
    cap_i = max(max(f[1] for f in fp), int(64 * sum(f[1] for f in fp) / len(fp)))
    b = serve_batched(tr, tab, lambda r: payload[r.rid], 128, max(r.cfg.nx for r in tr), cap_e, cap_i)
    o = serve_one_at_a_time(tr, tab, lambda r: payload[r.rid])
    keys = ("slabs_per_s", "ttr_p50_s", "ttr_p99_s", "wall_s")
    print(json.dumps({"batched": {k: b[k] for k in keys}, "one_at_a_time": {k: o[k] for k in keys},
                      "speedup": b["slabs_per_s"] / o["slabs_per_s"]}))


if __name__ == "__main__":
    main()
