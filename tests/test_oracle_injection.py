"""Pins of packet injection (Sect. 2.4, Eqs. 9-10) and of free streaming.

* Planck sampling: the sampled xi = h nu / kT has the Planck mean
  360 zeta(5) / pi^4 and the Planck shape x^3 / (e^x - 1) (chi^2 against
  scipy quadrature of that shape).
* Directions mu = sqrt(z): P(mu < m) = m^2 (zero limb darkening).
* Packet energies: N E = 4 pi r_i^2 sigma T^4 dt exactly (to rounding).
* With tau_S = 0 and n_e = 0 every packet escapes with its injection lab
  frequency and energy bit for bit, and the escaped luminosity is
  L_i <1/(1 - mu x_i)> = L_i 2 (-1/x - ln(1-x)/x^2).
"""
import numpy as np
from scipy import integrate, special, stats

import oracle
from paper_1401_5469_gb300 import synth

SIGMA_SB = 5.670374419e-5


def test_planck_sampler_mean_and_shape():
    rng = np.random.default_rng(21)
    n = 400_000
    z = np.empty((n, 5))
    z[:, 0] = rng.integers(0, 2**53, n, dtype=np.uint64) * 2.0**-53
    z[:, 1:] = (rng.integers(0, 2**53, (n, 4), dtype=np.uint64) + 1.0) * 2.0**-53
    xi = oracle.planck_xi(z)
    mean_exact = 360 * special.zeta(5) / np.pi**4
    assert abs(mean_exact - 3.83223) < 1e-5
    assert abs(xi.mean() - mean_exact) < 4 * xi.std() / np.sqrt(n)
    edges = np.linspace(0, 20, 81)
    counts, _ = np.histogram(xi, bins=edges)
    norm = np.pi**4 / 15
    p = np.array([integrate.quad(lambda x: x**3 / np.expm1(x), a, b)[0] for a, b in zip(edges[:-1], edges[1:])]) / norm
    exp_counts = p * n
    keep = exp_counts > 20
    chi2 = ((counts[keep] - exp_counts[keep]) ** 2 / exp_counts[keep]).sum()
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-4, chi2


def test_injection_state():
    spec = synth.scatter_model(n_lines=2000)
    om = oracle.OracleModel(spec)
    N = 200_000
    inj = oracle.inject_packets(om, 5469, 0, N, 1.0e4)
    mu = inj["mu"]
    assert np.all(mu > 0) and np.all(mu <= 1)
    assert stats.kstest(mu**2, "uniform").pvalue > 1e-4
    x_i = spec.v_inner[0] / 2.99792458e10
    D = 1 - mu * x_i
    np.testing.assert_allclose(inj["nu_lab"] * D, inj["nu_cmf"], rtol=2e-16 * 4)
    r_i = spec.v_inner[0] * spec.t_exp
    L = 4 * np.pi * r_i**2 * SIGMA_SB * 1.0e4**4
    e_cmf = inj["e_lab"] * D
    assert abs(e_cmf.sum() / L - 1) < 1e-12
    # first redward line: nu[j] < nu_cmf <= nu[j-1]
    j = inj["next_line"]
    nu = spec.nu
    inside = (j > 0) & (j < nu.size)
    assert np.all(nu[j[inside]] < inj["nu_cmf"][inside])
    assert np.all(nu[j[inside] - 1] >= inj["nu_cmf"][inside])
    assert np.all(inj["nu_cmf"][j == nu.size] <= nu[-1])
    assert np.all(inj["nu_cmf"][j == 0] > nu[0])


def test_free_streaming_recovers_injection_exactly():
    spec = synth.free_streaming_model(n_packets=100_000)
    om = oracle.OracleModel(spec)
    N = spec.n_packets
    inj = oracle.inject_packets(om, 99, 0, N, 1.0e4)
    r = oracle.run_iteration(om, 99, 0, N, 1.0e4)
    assert np.all(r.status == oracle.ESCAPED)
    assert np.array_equal(r.nu, inj["nu_lab"])
    assert np.array_equal(r.energy, inj["e_lab"])
    # escaped luminosity: L_i <1/D>, <1/D> = 2 (-1/x - ln(1-x)/x^2)
    x = spec.v_inner[0] / 2.99792458e10
    mean_invD = 2 * (-1 / x - np.log1p(-x) / x**2)
    r_i = spec.v_inner[0] * spec.t_exp
    L = 4 * np.pi * r_i**2 * SIGMA_SB * 1.0e4**4
    e = r.energy
    sigma = e.std() * np.sqrt(N)
    assert abs(e.sum() - L * mean_invD) < 4 * sigma
    # direct-binning spectrum equals the histogram of the injected lab frequencies
    edges = np.linspace(spec.spec_nu_lo, spec.spec_nu_hi, spec.spec_bins + 1)
    idx = np.digitize(inj["nu_lab"], edges) - 1
    inside = (idx >= 0) & (idx < spec.spec_bins)
    h = np.bincount(idx[inside], weights=inj["e_lab"][inside], minlength=spec.spec_bins)
    np.testing.assert_allclose(r.spectrum[:-2], h, rtol=1e-12, atol=1e-300)
    assert abs(r.spectrum[-2] - inj["e_lab"][inj["nu_lab"] < spec.spec_nu_lo].sum()) <= 1e-12 * e.sum()
    assert abs(r.spectrum[-1] - inj["e_lab"][inj["nu_lab"] >= spec.spec_nu_hi].sum()) <= 1e-12 * e.sum()
