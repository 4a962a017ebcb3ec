"""The allocation-free Philox check (pic_philox_check_static) against the
allocating one (pic_philox_check), through the C ABI, and on its own
against the oracle's Philox4x32-10 (itself checked against cuRAND's
generator).  Kept in a file that is collected last so it also runs after
every other GPU test."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_1704_01202_gb300 as pkg  # noqa: E402

MAX = 4096      # PIC_PHILOX_STATIC_MAX in include/pic.h


def _call(fn, ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros_like(c)
    P = C.POINTER(C.c_uint32)
    st = fn(c.ctypes.data_as(P), k.ctypes.data_as(P), o.ctypes.data_as(P), c.shape[0])
    return st, o


@pytest.mark.parametrize("n", [1, 1000, MAX])
def test_static_matches_allocating_twice(n):
    pkg.build()
    L = pkg.lib()
    rng = np.random.default_rng(n)
    for call in range(2):                   # two calls in a row, new inputs each time
        ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2**32, size=2, dtype=np.uint64).astype(np.uint32)
        st_a, ref = _call(L.pic_philox_check, ctr, key)
        st_b, got = _call(L.pic_philox_check_static, ctr, key)
        assert st_a == 0 and st_b == 0, (call, st_a, st_b)
        assert np.array_equal(got, ref), call


def test_static_matches_oracle_at_max():
    """One call at the largest size, compared row by row (a sample of rows
    and both ends) with the oracle's independent Philox4x32-10."""
    pkg.build()
    L = pkg.lib()
    rng = np.random.default_rng(77)
    ctr = rng.integers(0, 2**32, size=(MAX, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    key = np.array([0xDEADBEEF, 0x01234567], dtype=np.uint32)
    st, got = _call(L.pic_philox_check_static, ctr, key)
    assert st == 0
    rows = np.concatenate([[0, 1, MAX - 1], rng.choice(MAX, 61, replace=False)])
    for r in rows:
        assert np.array_equal(got[r], oracle.philox(ctr[r], key)), r


def test_static_rejects_oversize():
    pkg.build()
    L = pkg.lib()
    st, _ = _call(L.pic_philox_check_static, np.zeros((MAX + 1, 4), np.uint32), np.zeros(2, np.uint32))
    assert pkg.STATUS[st] == "PIC_ERR_ARG"


def test_static_known_answers():
    """On its own: the static entry point against Philox4x32-10's published
    known-answer vectors (tests/golden/philox4x32_10_kat.json)."""
    import json
    import os
    pkg.build()
    L = pkg.lib()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.json")
    for v in json.load(open(path))["vectors"]:
        ctr = np.array([[int(x, 16) for x in v["ctr"]]], dtype=np.uint32)
        key = np.array([int(x, 16) for x in v["key"]], dtype=np.uint32)
        st, out = _call(L.pic_philox_check_static, ctr, key)
        assert st == 0 and [int(x) for x in out.ravel()] == [int(x, 16) for x in v["out"]]
