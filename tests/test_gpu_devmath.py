"""Accuracy of the device arithmetic that replaces CUDA's functions in the
transport kernels, evaluated on the GPU through mc_selftest_math.

  * -ln z of an optical-depth draw z = u 2^-53, u in [1, 2^53] (Sect. 2.6),
    and the logarithm of the Planck sampler (Sect. 2.4): Tang's table-driven
    method.  Bound: within 1.5 ulp of the true value (a long-double reference
    on the host; the table method's degree-8 polynomial and the final sum of
    three terms, 1.35 ulp seen over 1e5 draws) and within 2 ulp of CUDA's log.
  * Reciprocals of Doppler factors D in [1 - x_out, 1 + x_out] and of
    frequencies (Sect. 2.5 frame transforms): within 1 ulp of IEEE division.
  * Square roots of the move and shell-exit geometry (Sect. 2.6): within
    1 ulp of IEEE sqrt; sqrt(0) = 0.
  * The hardware approximations the reciprocal and square root start from:
    over every high word of [1, 4) (both exponent parities, four low words
    each) the residual |1 - x y^2| of rsqrt.approx.f64 stays below 2^-18.5,
    so the square root's omitted 5e^3/16 term is below 2^-56 relative, and
    |1 - x r| of rcp.approx.f64 below 2^-19.5, so the reciprocal's omitted
    e^3 term is below 2^-58.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1401_5469_gb300 import mc as mcmod
    mcmod.load()
    return mcmod


def _ulps(a, ref):
    """|a - ref| in units of the binary64 spacing at ref (ref a float64 array)."""
    return np.abs(a - ref) / np.spacing(np.abs(ref))


def _ulps_exact(a, exact):
    """|a - exact| in ulps of binary64, exact given in long double."""
    e64 = exact.astype(np.float64)
    return (np.abs(a.astype(np.longdouble) - exact) / np.spacing(np.abs(e64)).astype(np.longdouble)).astype(np.float64)


def _long_double_is_wider():
    return np.finfo(np.longdouble).nmant > 52


def _log_uniform(rng, n, lo_exp, hi_exp):
    return np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(lo_exp, hi_exp, n))


def test_neg_log_u53(mc):
    rng = np.random.default_rng(53)
    edges = np.array([1, 2, 3, 4, 5, 2**26, 2**52 - 1, 2**52, 2**52 + 1, 2**53 - 2, 2**53 - 1, 2**53],
                     dtype=np.uint64)
    # uniform over the whole range, plus small u (large -ln z) log-uniformly
    uni = rng.integers(1, 2**53, 10_000_000, dtype=np.uint64, endpoint=True)
    small = np.maximum(1, np.exp(rng.uniform(0, np.log(2.0**53), 200_000))).astype(np.uint64)
    u = np.concatenate([edges, uni, small])
    ours, ref = mc.mc_selftest_math(mc.MC_MATH_NEG_LOG_U53, u)
    assert ours[edges.size - 1] == 0.0           # -ln(1) = 0 exactly
    assert np.all(ours[:edges.size - 1] > 0)
    d = _ulps(ours, np.where(ref == 0, np.finfo(float).tiny, ref))
    d[edges.size - 1] = 0.0
    assert d.max() <= 2.0, (d.max(), u[np.argmax(d)])
    if _long_double_is_wider():
        pick = np.concatenate([np.arange(edges.size - 1), rng.choice(u.size, 100_000, replace=False)])
        pick = pick[u[pick] != 2**53]
        z = u[pick].astype(np.longdouble) * np.longdouble(2.0) ** -53
        exact = -np.log(z)
        assert _ulps_exact(ours[pick], exact).max() <= 1.5


def test_log_pos(mc):
    rng = np.random.default_rng(54)
    x = np.concatenate([[1.0, 2.0, 0.5, np.nextafter(1.0, 2.0), np.nextafter(1.0, 0.0), 2.0**-1000, 2.0**1000],
                        _log_uniform(rng, 2_000_000, -1000, 1000),
                        rng.uniform(0.5, 2.0, 1_000_000)])
    ours, ref = mc.mc_selftest_math(mc.MC_MATH_LOG, x)
    assert ours[0] == 0.0
    nz = ref != 0
    assert _ulps(ours[nz], ref[nz]).max() <= 2.0
    if _long_double_is_wider():
        pick = np.concatenate([np.arange(1, 7), rng.choice(x.size, 100_000, replace=False)])
        exact = np.log(x[pick].astype(np.longdouble))
        assert _ulps_exact(ours[pick], exact).max() <= 1.5


def test_rcp64(mc):
    rng = np.random.default_rng(55)
    x_out = 25_000e5 / 2.99792458e10  # the largest outer velocity of the models, in units of c
    d = rng.uniform(1.0 - x_out, 1.0 + x_out, 2_000_000)
    x = np.concatenate([[1.0 - x_out, 1.0 + x_out, 1.0, np.nextafter(1.0, 0.0), 1e14, 3e15, 2.0**-1000, 2.0**1000],
                        d, _log_uniform(rng, 2_000_000, -1000, 1000), -d[:1000]])
    ours, ref = mc.mc_selftest_math(mc.MC_MATH_RCP, x)
    assert _ulps(ours, ref).max() <= 1.0


def test_sqrt64(mc):
    rng = np.random.default_rng(56)
    x_out2 = (25_000e5 / 2.99792458e10) ** 2
    geo = rng.uniform(0.0, x_out2, 2_000_000)          # squared radii and x_b^2 - q of the models
    tiny = x_out2 * np.ldexp(1.0, -rng.integers(20, 60, 200_000))  # near-tangent shell exits
    x = np.concatenate([[0.0, 1.0, 4.0, 2.0, 2.0**-1000, 2.0**1000, np.nextafter(1.0, 2.0)],
                        geo, tiny, _log_uniform(rng, 2_000_000, -1000, 1000)])
    ours, ref = mc.mc_selftest_math(mc.MC_MATH_SQRT, x)
    assert ours[0] == 0.0
    nz = ref != 0
    assert _ulps(ours[nz], ref[nz]).max() <= 1.0


def test_approximation_residuals(mc):
    hi = np.arange(1 << 21, dtype=np.uint64)
    expo = (1023 + (hi >> np.uint64(20))) << np.uint64(52)
    mant = (hi & np.uint64(0xFFFFF)) << np.uint64(32)
    lows = np.array([0, 0x80000000, 0xFFFFFFFF, 0x12345678], dtype=np.uint64)
    bits = (expo[:, None] | mant[:, None] | lows[None, :]).ravel()
    x = bits.view(np.float64)
    assert x.min() >= 1.0 and x.max() < 4.0
    res_rsqrt, res_rcp = mc.mc_selftest_math(mc.MC_MATH_APPROX, x)
    assert np.abs(res_rsqrt).max() <= 2.0 ** -18.5, np.log2(np.abs(res_rsqrt).max())
    assert np.abs(res_rcp).max() <= 2.0 ** -19.5, np.log2(np.abs(res_rcp).max())
