"""Host logic of the served loop, without a GPU: admission by reservation,
queueing, electron budgets, preemption of a slab that outgrows its
reservation and its re-run with a larger one, the failure of a request
that can never fit and the refusal on arrival of one wider than a slot or
larger than the batch, each alone, against a stand-in for the batch
context that grows each slab's electrons at a scripted rate."""
from dataclasses import dataclass, field

import pic_inputs as P
from paper_1704_01202_gb300 import SLOT_ACTIVE, SLOT_FAILED, serve


@dataclass
class FakeBatch:
    """Stand-in for paper_1704_01202_gb300.Batch: slab k holds
    n_e + growth[seed] * steps electrons; a step that takes it beyond its
    budget fails it (state 3), as the device does."""
    cap_e: int
    cap_i: int
    max_slabs: int
    growth: dict
    state: dict = field(default_factory=dict)      # slot -> [cfg, electrons, budget, steps, state]
    log: list = field(default_factory=list)
    peak_reserved: int = 0

    def autotune(self, on):
        pass

    def admit(self, cfg, st, pulse=None):
        slot = next(k for k in range(self.max_slabs) if k not in self.state)
        self.state[slot] = [cfg, cfg.ncell * cfg.ppc_e, 0, 0, SLOT_ACTIVE]
        self.log.append(("admit", cfg.seed))
        return slot

    def set_budget(self, slot, max_e):
        assert 0 < max_e <= self.cap_e
        self.state[slot][2] = max_e
        # the scheduler never reserves more than the shared capacity
        total = sum(s[2] for s in self.state.values() if s[4] == SLOT_ACTIVE)
        assert total <= self.cap_e
        self.peak_reserved = max(self.peak_reserved, total)

    def step(self, n):
        for s in self.state.values():
            if s[4] != SLOT_ACTIVE:
                continue
            s[1] += self.growth.get(s[0].seed, 0) * n
            s[3] += n
            if s[1] > s[2]:
                s[4] = SLOT_FAILED

    def failed(self):
        return [k for k, s in self.state.items() if s[4] == SLOT_FAILED]

    def retire(self, slot):
        self.log.append(("retire", self.state[slot][0].seed, self.state[slot][4]))
        del self.state[slot]

    def diagnostics(self, slot, n_E=64):
        s = self.state[slot]
        return {"steps": s[3], "n_e": s[1]}

    def sync(self):
        pass


def _request(rid, nx, ppc_i, nsteps, t=0.0):
    cfg = P.cfg_small_1d(nx=nx, ppc_e=4 * ppc_i, ppc_i=ppc_i, rad_every=5, flags=P.F_ALL, seed=100 + rid)
    return P.Request(rid=rid, t_arrive=t, cfg=cfg, pulse=P.Pulse(n_bins=2), nsteps=nsteps)


def test_footprint_reserves_partial_event_electrons():
    r = _request(0, nx=10, ppc_i=3, nsteps=100)
    fe, fi = serve.footprint(r.cfg, r.pulse)
    # own electrons + one per charge the ions can lose + one per bin per cell
    assert (fe, fi) == (10 * 12 + 30 * 10 + 10 * 2, 30)
    assert serve.footprint(r.cfg, r.pulse, 5)[0] == fe + 10 * 2 * 4
    assert serve.footprint(r.cfg)[0] == fe - 20                 # no pulse: no photoionization
    assert serve.partial_bound(r.cfg, r.pulse, 100) == 10 * 2 * 20
    r.cfg.flags = P.F_ALL & ~P.F_PHOTO
    assert serve.partial_bound(r.cfg, r.pulse, 100) == 0


def test_requests_queue_until_room_frees():
    tr = [_request(k, nx=10, ppc_i=2, nsteps=40) for k in range(7)]
    fe = serve.footprint(tr[0].cfg, tr[0].pulse)[0]
    fb = FakeBatch(cap_e=3 * fe, cap_i=10**6, max_slabs=8, growth={})
    out = serve.serve_batched(tr, None, lambda r: None, max_slabs=8, slot_cells=16, cap_e=3 * fe,
                              cap_i=10**6, tick_steps=10, batch=fb)
    assert sorted(out["results"]) == list(range(7)) and not out["failed"]
    assert all(d["steps"] == 40 for d in out["results"].values())
    assert fb.peak_reserved == 3 * fe and out["max_queue"] == 4 and out["preempted"] == 0
    # first come first served: admissions follow arrival order
    assert [e[1] for e in fb.log if e[0] == "admit"] == [100 + k for k in range(7)]
    assert out["wait_p99_s"] >= out["wait_p50_s"] >= 0.0


def test_a_slab_beyond_its_reservation_is_preempted_alone_and_rerun():
    tr = [_request(k, nx=10, ppc_i=2, nsteps=60) for k in range(4)]
    fe = serve.footprint(tr[0].cfg, tr[0].pulse)[0]
    # request 2 creates 5 electrons a step: 380 after 60 steps, beyond its
    # first reservation (300) and the one with 4 partial-event electrons per
    # bin per cell (360), within the one with 16 (600)
    grow = 5
    n_end = tr[2].cfg.ncell * tr[2].cfg.ppc_e + grow * 60
    assert serve.footprint(tr[2].cfg, tr[2].pulse, 4)[0] < n_end <= serve.footprint(tr[2].cfg, tr[2].pulse, 16)[0]
    fb = FakeBatch(cap_e=10 * fe, cap_i=10**6, max_slabs=8, growth={102: grow})
    out = serve.serve_batched(tr, None, lambda r: None, max_slabs=8, slot_cells=16, cap_e=10 * fe,
                              cap_i=10**6, tick_steps=10, batch=fb)
    assert sorted(out["results"]) == [0, 1, 2, 3] and not out["failed"]
    assert out["preempted"] == 2
    # the preempted run was retired as failed, the others only once each, done
    retired = [e for e in fb.log if e[0] == "retire"]
    assert [e[1] for e in retired if e[2] == SLOT_FAILED] == [102] * out["preempted"]
    assert sorted(e[1] for e in retired if e[2] == SLOT_ACTIVE) == [100, 101, 102, 103]
    # the re-run started from step 0 and ran the whole horizon
    assert out["results"][2]["steps"] == 60
    assert sum(1 for e in fb.log if e == ("admit", 102)) == out["preempted"] + 1


def test_a_request_that_cannot_fit_fails_alone():
    tr = [_request(k, nx=10, ppc_i=2, nsteps=60) for k in range(3)]
    fe = serve.footprint(tr[0].cfg, tr[0].pulse)[0]
    # request 1 grows without bound: its reservation outgrows the capacity
    fb = FakeBatch(cap_e=2 * fe, cap_i=10**6, max_slabs=4, growth={101: 10**4})
    out = serve.serve_batched(tr, None, lambda r: None, max_slabs=4, slot_cells=16, cap_e=2 * fe,
                              cap_i=10**6, tick_steps=10, batch=fb)
    assert sorted(out["results"]) == [0, 2]
    assert list(out["failed"]) == [1] and "electron slots" in out["failed"][1]
    assert out["slabs"] == 3


def test_a_request_larger_than_the_batch_is_refused_alone():
    """A request whose footprint is beyond the capacity, or which is wider
    than a slot, is refused on arrival; the others are served."""
    small = [_request(k, nx=10, ppc_i=2, nsteps=10) for k in (0, 2)]
    fe = serve.footprint(small[0].cfg, small[0].pulse)[0]
    big = _request(1, nx=12, ppc_i=40, nsteps=10)
    wide = _request(3, nx=20, ppc_i=2, nsteps=10)
    assert serve.footprint(big.cfg, big.pulse)[0] > 2 * fe
    tr = [small[0], big, small[1], wide]
    fb = FakeBatch(cap_e=2 * fe, cap_i=10**6, max_slabs=2, growth={})
    out = serve.serve_batched(tr, None, lambda r: None, max_slabs=2, slot_cells=16, cap_e=2 * fe,
                              cap_i=10**6, tick_steps=5, batch=fb)
    assert sorted(out["results"]) == [0, 2]
    assert sorted(out["failed"]) == [1, 3]
    assert "capacity" in out["failed"][1] and "slot" in out["failed"][3]
    assert [e[1] for e in fb.log if e[0] == "admit"] == [100, 102]


def test_the_reservation_grows_up_to_what_the_capacity_holds():
    """The preempted request's allowance grows by 4 each time, but not past
    the most the capacity holds: with cap_e = 500 (own electrons and
    charge reserve 280, 20 slots per allowance step) it runs at allowance 11,
    where the unclamped 16 would not fit and the request would fail."""
    tr = [_request(k, nx=10, ppc_i=2, nsteps=60) for k in range(2)]
    n_end = 80 + 6 * 60                                    # 440 electrons at the end
    assert serve.footprint(tr[0].cfg, tr[0].pulse, 4)[0] < n_end <= serve.footprint(tr[0].cfg, tr[0].pulse, 11)[0]
    fb = FakeBatch(cap_e=500, cap_i=10**6, max_slabs=4, growth={100: 6})
    out = serve.serve_batched(tr, None, lambda r: None, max_slabs=4, slot_cells=16, cap_e=500,
                              cap_i=10**6, tick_steps=10, batch=fb)
    assert sorted(out["results"]) == [0, 1] and not out["failed"]
    assert out["preempted"] == 2 and out["results"][0]["steps"] == 60
