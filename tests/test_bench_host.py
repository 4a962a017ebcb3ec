"""Host arithmetic of bench.py's report, without a GPU: the energy
bookkeeping and its drift per 1000 steps, the clock-sample parsing
(median SM clock, throttle reasons), the charge states listed, and the
single-rank aggregation."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _diag(**kw):
    d = {k: 0.0 for k in ("ke_e", "ke_i", "e_ion", "e_phot", "e_field", "e_esc", "e_trans", "e_ka_esc", "e_inc")}
    d.update(kw)
    return d


def test_energy_total_counts_every_store_once(bench):
    d = _diag(ke_e=10.0, ke_i=1.0, e_ion=3.0, e_phot=4.0, e_field=0.5, e_esc=0.25, e_trans=2.0, e_ka_esc=0.125,
              e_inc=7.0)
    assert bench.energy_total(d) == pytest.approx(10 + 1 + 3 + 4 + 0.5 + 0.25 + 2 + 0.125 - 7)


def test_energy_drift_per_1000_steps(bench):
    d0 = _diag(ke_e=100.0)
    # 500 steps: 20 units came in as photons, 19.5 of them absorbed and
    # 0.5 still photons, plus 1 unit of heating -> +1 on a held 121
    d1 = _diag(ke_e=119.0, e_ion=1.5, e_phot=0.5, e_inc=20.0)
    # 10 timed steps: nothing changes
    d2 = dict(d1)
    out = bench.energy_drift(d0, d1, d2, 500, 10)
    held = 119.0 + 1.5 + 0.5
    assert out["held"] == pytest.approx(held)
    assert out["advance"]["rel_per_1000_steps"] == pytest.approx(1.0 / held * 2.0)
    assert out["timed"]["rel_per_1000_steps"] == 0.0
    assert out["advance"]["steps"] == 500 and out["timed"]["steps"] == 10


def test_charge_states_over_a_share(bench):
    assert bench.charge_states([0.0, 0.005, 0.2, 0.011, 0.784], 0.01) == [2, 3, 4]


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples(bench):
    c = bench.ClockSampler()
    c.proc = _FakeProc()
    c.lines = ["2070, 2070, 0x0, Not Active, Not Active, Not Active, Not Active",
               "2055, 2070, 0x4, Not Active, Not Active, Not Active, Active",
               "2070, 2070, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage",
               "1980, 2070, 0x8, Active, Not Active, Not Active, Not Active"]
    out = c.stop()
    assert out["sm_mhz"] == pytest.approx(2062.5) and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]
    none = bench.ClockSampler().stop()
    assert none["sm_mhz"] is None and none["reasons"] == ["nvidia-smi unavailable"]


def test_single_rank_aggregate(bench):
    ms, value = bench.aggregate(250.0, 1.0e9 * 20)
    assert ms == 250.0 and value == pytest.approx(1.0e9 * 20 / 0.25)


def test_issue_rate(bench):
    """The cell kernel against the SM issue rate: 92 warp instructions per
    particle; four schedulers per SM, one warp instruction a cycle."""
    r = bench.issue_rate(100.0, 1.0e9, 152, 2000.0)
    assert r["peak"] == pytest.approx(4 * 152 * 2.0e9)
    assert r["achieved"] == pytest.approx(92.0 * 1.0e9 / 0.1)
    assert r["frac"] == pytest.approx(92.0e10 / (4 * 152 * 2.0e9))
    assert bench.issue_rate(100.0, 1.0e9, 152, None)["sm_mhz"] == 2070.0


def test_profile_commands_use_existing_bench_options(bench):
    """Every command under profiles/ that runs bench.py passes only options
    the bench parses (the summaries give runnable commands)."""
    import glob
    import re
    known = set(re.findall(r'add_argument\("(--[\w-]+)"', open(os.path.join(ROOT, "bench.py")).read()))
    assert "--steps" in known and "--no-cpu" in known
    seen = 0
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        text = open(path).read().replace("\\\n", " ")
        for line in text.splitlines():
            if "python bench.py" not in line:
                continue
            seen += 1
            args = line.split("python bench.py", 1)[1].split()
            for a in args:
                if a.startswith("--"):
                    assert a in known, (os.path.basename(path), a)
    assert seen >= 4
