"""The precision split: particle state and scattering are FP32, the per-cell
energy, weight and charge sums that the energy restore (Sec. IV) and the
cell moments (Sec. II) need are double-float pairs (a float hi + lo).  Here
that arithmetic, run by the device as the cell kernel runs it, is held to
exact sums of the same FP32 terms: within 2^-44 of the sum of the terms'
magnitudes, where a plain FP32 accumulation misses by orders of magnitude;
the FP64 build's pairs of doubles to the correctly rounded sum."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1704_01202_gb300 as pkg  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()


def _cases():
    rng = np.random.default_rng(3)
    n = 4096
    bulk = rng.exponential(30.0, n)
    tail = np.where(rng.uniform(size=n) < 0.05, rng.exponential(1500.0, n), bulk)
    return {
        "kinetic_energies": rng.uniform(0.5, 1.5, n) * bulk,           # w * E of a cell
        "bulk_and_beam": rng.uniform(0.5, 1.5, n) * tail,
        "one_cell_max": rng.exponential(1.0, 2048),
        "many_terms": rng.exponential(1.0, 1 << 20),
        "signed_momenta": rng.normal(0.0, 1.0, 100000),
        "wide_range": 10.0 ** rng.uniform(-8, 8, 50000),
    }


@pytest.mark.parametrize("name", list(_cases()))
def test_double_float_sums_against_exact(name):
    x = _cases()[name].astype(np.float32)
    x64 = x.astype(np.float64)
    exact = math.fsum(x64)
    mag = float(np.abs(x64).sum())
    got = pkg.dd_sum_check(x)
    assert abs(got - exact) <= 2.0**-44 * mag, (name, got - exact, mag)
    # the FP64 build: pairs of doubles, the FP32 terms exact in them
    got64 = pkg.dd_sum_check(x, fp64=True)
    assert abs(got64 - exact) <= 2.0**-52 * mag, (name, got64 - exact, mag)
    if x.size >= 4096 and np.all(x > 0):
        # sequential FP32 accumulation: what the pairs are there to avoid
        naive = float(np.cumsum(x, dtype=np.float32)[-1])
        assert abs(naive - exact) > 2.0**-44 * mag * 64, (name, naive - exact)
