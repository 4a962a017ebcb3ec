"""Pins of the oracle's random streams and pairing (CPU only).

The generator is Philox4x32-10 (Salmon et al., SC'11); the paper only asks
for random numbers 0 < r < 1 (Sec. III).  Without the Random123 answer
files the oracle's copy is pinned by statistics here and against cuRAND's
Philox4_32_10 in the GPU suite.  Pairing (Sec. IV, Takizuka-Abe by
citation) is pinned by brute-force enumeration of orderings.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

import oracle


def _block(n, step=0, purpose=1, key=(7, 11)):
    out = np.zeros((n, 4), dtype=np.uint32)
    for i in range(n):
        out[i] = oracle.philox([i, 0, step, purpose], key)
    return out


def test_philox_uniformity_chi2():
    x = _block(20000).ravel()
    u = (x >> np.uint32(24)).astype(np.int64)          # top byte, 256 classes
    cnt = np.bincount(u, minlength=256)
    chi2, p = stats.chisquare(cnt)
    assert p > 1e-4


def test_philox_bit_balance_and_avalanche():
    x = _block(4000)
    bits = np.unpackbits(x.view(np.uint8)).reshape(-1)
    assert abs(bits.mean() - 0.5) < 0.005
    # flipping one counter bit flips about half of the 128 output bits
    flips = []
    for i in range(300):
        a = oracle.philox([i, 5, 9, 3], [1, 2])
        b = oracle.philox([i ^ 1, 5, 9, 3], [1, 2])
        flips.append(np.unpackbits((a ^ b).view(np.uint8)).sum())
    assert 60 < np.mean(flips) < 68


def test_philox_distinct_counters_distinct_outputs():
    x = _block(50000)
    rows = {tuple(r) for r in x}
    assert len(rows) == x.shape[0]


def test_uniform_open_interval():
    L = oracle.lib()
    assert 0.0 < L.orc_u01(0) < 1e-7
    assert 1.0 - 1e-7 < L.orc_u01(0xFFFFFFFF) < 1.0
    # every uniform is exactly a single-precision number (the FP32 device
    # path draws the same value), the largest one included
    rng = np.random.default_rng(4)
    xs = np.concatenate([rng.integers(0, 2**32, 20000, dtype=np.uint64), [0, 2**31, 2**32 - 1, 2**32 - 512]])
    for x in xs:
        u = L.orc_u01(int(x))
        assert float(np.float32(u)) == u, x
    assert float(np.float32(L.orc_u01(0xFFFFFFFF))) < 1.0


def test_pair_order_is_uniform_permutation():
    # every ordering of 4 ids equally likely over many steps
    ids = np.array([3, 17, 4 << 32, 9], dtype=np.uint64)
    counts = {}
    n = 12000
    for step in range(n):
        p = tuple(oracle.pair_order(ids, step, 1, 12345))
        counts[p] = counts.get(p, 0) + 1
    assert len(counts) == 24
    chi2, pv = stats.chisquare(list(counts.values()))
    assert pv > 1e-4


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_pairing_brute_force(n):
    """Expected collision share of every particle pair from all n! orderings
    of the pairing rule (odd n: first three in a half-step triangle) against
    the oracle's pair frequencies over many steps."""
    pa, pb, fr = oracle.ee_pairs(n)
    # the rule is a perfect matching (even) or triangle + matching (odd)
    used = np.zeros(n, dtype=int)
    for a, b, f in zip(pa, pb, fr):
        used[a] += 1
        used[b] += 1
    if n % 2 == 0:
        assert (used == 1).all() and np.allclose(fr, 1.0)
    else:
        assert (used[:3] == 2).all() and (used[3:] == 1).all()
    expect = np.zeros((n, n))
    for perm in itertools.permutations(range(n)):
        for a, b, f in zip(pa, pb, fr):
            i, j = sorted((perm[a], perm[b]))
            expect[i, j] += f
    expect /= math.factorial(n)
    ids = np.arange(n, dtype=np.uint64) * 1000 + 7
    nsteps = 6000
    got = np.zeros((n, n))
    for step in range(nsteps):
        perm = oracle.pair_order(ids, step, 1, 99)
        for a, b, f in zip(pa, pb, fr):
            i, j = sorted((perm[a], perm[b]))
            got[i, j] += f
    iu = np.triu_indices(n, 1)
    e = expect[iu] * nsteps
    g = got[iu]
    # all pairs equally likely by symmetry, and the brute force says so
    assert np.allclose(e, e[0])
    chi2 = ((g - e) ** 2 / e).sum()
    dof = len(e) - 1
    assert stats.chi2.sf(chi2, dof) > 1e-4 if dof > 0 else abs(g[0] - e[0]) < 1e-9


def _kat():
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.json")
    for v in json.load(open(path))["vectors"]:
        yield ([int(x, 16) for x in v["ctr"]], [int(x, 16) for x in v["key"]], [int(x, 16) for x in v["out"]])


def test_philox_published_known_answers():
    """The oracle's Philox4x32-10 against the generator's published
    known-answer vectors (tests/golden/philox4x32_10_kat.json)."""
    for ctr, key, out in _kat():
        got = oracle.philox(np.array([ctr], dtype=np.uint32), tuple(key)).ravel()
        assert [int(x) for x in got] == out
