"""The 16-bit storage formats through the C ABI.

* E3M12 (sign, 3 exponent bits with bias 5, 12 mantissa bits, subnormals):
  set_populations rounds the stored value x = (f_j - omega_j rho0) * s_j
  (s_j the power of two nearest 1/omega_j times the range factor
  2^floor(log2(8 / R))) to nearest-even on the format's value grid, written
  out here from the format's definition (the spacing is 2^(e - 12) in the
  binade [2^e, 2^(e+1)) for e >= -4, 2^-16 below 2^-4, and the largest
  value 8 - 2^-10 takes everything that rounds beyond it); get_populations
  returns exactly that grid value.
* Stochastic rounding of rmrtlb_step (FP16, BF16, E3M12): from a uniform
  state at rest every node rounds the same post-collision value; the mean
  over the nodes of the stored values equals the oracle's post-collision
  value within the sampling error of a Bernoulli rounding, and both
  neighbouring grid values occur (round-to-nearest would give one of them
  at every node).
* A population beyond the E3M12 range is reported by the check (flag 8).
"""
import numpy as np
import pytest

import oracle.rmrt as R
from cases import Case, gpu_solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "the -m gpu tests need a CUDA device"
    from paper_2206_00366_gb300 import build
    build.build()


def pow2_scale(w):
    """The storage factor s_j: the power of two nearest 1/omega_j."""
    return np.ldexp(1.0, np.rint(-np.log2(w)).astype(int))


def e3m12_spacing(x):
    """Spacing of the E3M12 grid around |x| (scaled units)."""
    a = np.abs(x)
    e = np.floor(np.log2(np.maximum(a, 2.0 ** -4)))
    return np.where(a < 2.0 ** -4, 2.0 ** -16, 2.0 ** (e - 12))


def e3m12_nearest(x):
    """Round-to-nearest-even onto the E3M12 grid, saturating at 8 - 2^-10."""
    h = e3m12_spacing(x)
    q = np.abs(x) / h
    r = np.floor(q)
    frac = q - r
    r = np.where((frac > 0.5) | ((frac == 0.5) & (np.fmod(r, 2) == 1)), r + 1, r)
    v = np.minimum(r * h, 8.0 - 2.0 ** -10)
    return np.sign(x) * v


@pytest.mark.parametrize("lattice,shape,storage_range", [("D2Q9", (36, 20, 1), 0.0), ("D3Q27", (12, 9, 5), 0.0),
                                                         ("D2Q9", (36, 20, 1), 3.0), ("D3Q19", (8, 6, 5), 0.3)])
def test_e3m12_round_trip_on_the_format_grid(lattice, shape, storage_range):
    """storage_range 0 selects the NSE default 2; a range R otherwise maps
    onto the format's [0, 8) by 2^floor(log2(8 / R)) (3 -> 4, 0.3 -> 0.5)."""
    case = Case(lattice, shape, (1.0, 0.7, 0.55), extra={"storage_range": storage_range})
    lat = case.lat()
    s = gpu_solver(case, "e3m12")
    w = np.asarray(s.constants()[4:4 + lat.q])        # the library's weights: its rest state is w_j rho0
    rng = np.random.default_rng(5)
    nz, ny, nx = case.field_shape
    # stored values spanning the subnormal range, every binade and the saturation point
    mag = np.exp(rng.uniform(np.log(2.0 ** -22), np.log(12.0), size=(lat.q, nz, ny, nx)))
    x = mag * rng.choice([-1.0, 1.0], size=mag.shape)
    shift = np.floor(np.log2(8.0 / (storage_range if storage_range > 0 else 2.0)))
    sc = (pow2_scale(w) * 2.0 ** shift).reshape(lat.q, 1, 1, 1)
    rest = (w * case.rho0).reshape(lat.q, 1, 1, 1)
    f = rest + x / sc
    s.set_populations(f)
    back = s.get_populations()
    # the library forms x in FP32 before rounding it to the format
    x32 = ((f - rest) * sc).astype(np.float32).astype(np.float64)
    want = rest + e3m12_nearest(x32) / sc
    np.testing.assert_array_equal(back, want)


@pytest.mark.parametrize("storage", ["f16", "bf16", "e3m12"])
def test_stochastic_rounding_is_unbiased(storage):
    case = Case("D2Q9", (128, 128, 1), (1.0, 0.6, 1.0), nu=0.02, nu_bulk=0.03, s_free=1.1)
    lat, m, S = case.oracle_setup()
    nz, ny, nx = case.field_shape
    eps = 0.0123456789
    s = gpu_solver(case, storage)
    s.init_equilibrium(np.full(case.field_shape, case.rho0 + eps), np.zeros((2,) + case.field_shape))
    f0 = s.get_populations()
    assert np.ptp(f0.reshape(lat.q, -1), axis=1).max() == 0          # a uniform state
    want = R.collide(lat, m, S, f0.reshape(lat.q, -1)[:, :1])[:, 0]    # uniform at rest: streaming moves nothing
    s.step(1)
    f1 = s.get_populations().reshape(lat.q, -1)
    n = f1.shape[1]
    both = 0
    for j in range(lat.q):
        vals = np.unique(f1[j])
        assert len(vals) <= 2, (j, vals)            # the two grid values around the exact one
        both += len(vals) == 2
        gap = vals[-1] - vals[0] if len(vals) == 2 else 0.0
        # Bernoulli rounding: the mean deviates from want by at most a few gap * 0.5 / sqrt(n)
        tol = 6.0 * 0.5 * gap / np.sqrt(n) + 1e-6 * abs(want[j] - lat.w[j] * case.rho0)
        assert abs(f1[j].mean() - want[j]) <= tol, (j, f1[j].mean(), want[j], tol)
    assert both >= lat.q - 2          # rounding down at some nodes and up at others


def test_e3m12_saturation_is_reported():
    from paper_2206_00366_gb300 import rmrtlb as B
    case = Case("D2Q9", (16, 8, 1), (1.0, 0.6, 1.0))
    lat = case.lat()
    f = np.tile((lat.w * case.rho0).reshape(lat.q, 1, 1, 1), (1, 1, 8, 16))
    f[3, 0, 2, 5] += 5.0 / pow2_scale(lat.w)[3]                       # scaled deviation 5 > range 2 (NSE)
    s = gpu_solver(case, "e3m12")
    s.set_populations(f)
    with pytest.raises(B.RmrtlbError) as ei:
        s.stats()
    assert ei.value.status == B.EUNSTABLE
    assert int(s.stats(allow_unstable=True)[7]) & 8
