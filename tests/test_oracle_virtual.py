"""Pins of the oracle's virtual packets (Sect. 2.9, Eqs. 19-21).

* v-packets draw from their own Philox stream: the r-packets' estimators and
  spectrum are bit-identical with and without them;
* transparent ejecta: every v-packet escapes with weight 2 mu_v / N_v (Eq. 20)
  at lab energy E/D, so the v-spectrum total per packet estimates
  E int_0^1 2 mu / (1 - mu x_i) dmu = E (-2/x - 2 ln(1 - x)/x^2) (closed form);
* tau_v of a radial ray through electron-scattering shells is the sum of
  kappa_s (1 - x_s)(x_out,s - x_s) over the shells (segment-start Doppler
  factor at each shell's inner radius, as for r-packets);
* one line with depth tau0: tau_v = tau0 exactly when the ray's resonance
  point (x mu = 1 - nu_line / nu_lab) lies on the ray before the outer
  boundary, else 0; with the depth in one shell only, exactly when the
  resonance radius lies in that shell;
* directions: a ray with mu just above mu_min = -sqrt(1 - (x_in/x)^2) stays
  clear of the inner boundary, one just below meets it (inf);
* the tau_v_max cut drops exactly the v-packets above it;
* in a scattering model the v-spectrum and the direct r-packet spectrum
  estimate the same emergent spectrum (agree within the Monte Carlo noise,
  16 seeds), and with N_v = 3 the v-spectrum has the lower noise per bin.
"""
import numpy as np
import pytest

import oracle
from paper_1401_5469_gb300 import synth

C = 2.99792458e10
SIGMA_T = 6.6524587321e-25


def _x(spec):
    return spec.v_inner / C, spec.v_outer / C


def test_r_packets_unchanged_by_virtual_packets():
    spec = synth.scatter_model(n_packets=3000)
    om = oracle.OracleModel(spec, tau=spec.tau)
    a = oracle.run_iteration(om, 11, 0, 3000, spec.t_inner, threads=1, record=True)
    om.set_virtual(3)
    b = oracle.run_iteration(om, 11, 0, 3000, spec.t_inner, threads=1, record=True)
    for k in ("j_est", "nu_bar", "spectrum", "status", "nu", "energy", "counters"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k))
    assert b.spectrum_v.sum() > 0


def test_free_streaming_total_matches_closed_form():
    spec = synth.free_streaming_model(n_packets=20000)
    om = oracle.OracleModel(spec)
    nv = 4
    om.set_virtual(nv)
    r = oracle.run_iteration(om, 3, 0, spec.n_packets, spec.t_inner, threads=4, record=False)
    x = spec.v_inner[0] / C
    # packet comoving energy (Eqs. 9-10)
    r_i = spec.v_inner[0] * spec.t_exp
    e = 4 * np.pi * r_i ** 2 * 5.670374419e-5 * spec.t_inner ** 4 / spec.n_packets
    mean = -2.0 / x - 2.0 * np.log1p(-x) / x ** 2  # int_0^1 2 mu / (1 - mu x) dmu
    mu = (np.arange(200000) + 0.5) / 200000
    var = np.mean((2 * mu / (1 - mu * x)) ** 2) - mean ** 2  # one v-packet, mu ~ U(0,1)
    want = e * spec.n_packets * mean
    sigma = e * np.sqrt(spec.n_packets * var / nv)
    got = r.spectrum_v.sum()
    assert abs(got - want) < 5 * sigma, (got, want, sigma)
    # every v-packet escapes, so no energy is lost to the inner boundary
    assert r.stats["escaped"] == spec.n_packets


def test_radial_electron_optical_depth():
    spec = synth.scatter_model(n_lines=10, n_shells=6)
    spec.tau = np.zeros_like(spec.tau)
    om = oracle.OracleModel(spec)
    x_in, x_out = _x(spec)
    kappa = SIGMA_T * spec.n_e * C * spec.t_exp
    want = np.sum(kappa * (1.0 - x_in) * (x_out - x_in))
    got = oracle.virtual_tau(om, x_in[0], 1.0, 0, 1e15, spec.nu.size)  # no lines left
    assert got == pytest.approx(want, rel=1e-13)
    # starting mid-way through shell 2, radially
    x0 = 0.5 * (x_in[2] + x_out[2])
    want2 = kappa[2] * (1 - x0) * (x_out[2] - x0) + np.sum((kappa * (1 - x_in) * (x_out - x_in))[3:])
    assert oracle.virtual_tau(om, x0, 1.0, 2, 1e15, spec.nu.size) == pytest.approx(want2, rel=1e-13)


def _one_line_model(tau0, shell=None):
    spec = synth.free_streaming_model(n_shells=6, n_lines=1)
    spec.nu = np.array([1.0e15])
    t = np.zeros((6, 1))
    if shell is None:
        t[:, 0] = tau0
    else:
        t[shell, 0] = tau0
    spec.tau = t
    return spec, oracle.OracleModel(spec)


@pytest.mark.parametrize("mu", [1.0, 0.6, 0.1, -0.3])
def test_single_line_depth_on_and_off_the_ray(mu):
    spec, om = _one_line_model(2.5)
    x_in, x_out = _x(spec)
    x = x_in[0] * 1.2 if mu < 0 else x_in[0]
    s = int(np.searchsorted(x_out, x, side="right"))
    p0, q = x * mu, x * x * (1 - mu * mu)
    p_end = np.sqrt(x_out[-1] ** 2 - q)  # the ray leaves through the outer sphere
    for frac in (0.2, 0.5, 0.9, 1.2):
        # lab frequency that puts the resonance at x mu = p0 + frac (p_end - p0)
        p_res = p0 + frac * (p_end - p0)
        nu_lab = spec.nu[0] / (1.0 - p_res)
        got = oracle.virtual_tau(om, x, mu, s, nu_lab, 0)
        assert got == (2.5 if frac < 1.0 else 0.0), (frac, got)


def test_single_line_depth_counts_only_in_its_shell():
    x_in, x_out = _x(_one_line_model(1.0)[0])
    for shell in range(6):
        spec, om = _one_line_model(1.7, shell)
        x = x_in[0]
        for frac in (0.1, 0.3, 0.5, 0.7, 0.95):
            p_res = x + frac * (x_out[-1] - x)  # radial ray: resonance radius = p_res
            nu_lab = spec.nu[0] / (1.0 - p_res)
            want = 1.7 if x_in[shell] <= p_res < x_out[shell] else 0.0
            assert oracle.virtual_tau(om, x, 1.0, 0, nu_lab, 0) == want, (shell, frac)


def test_directions_clear_the_inner_boundary():
    spec = synth.free_streaming_model(n_shells=5)
    om = oracle.OracleModel(spec)
    x_in, x_out = _x(spec)
    x = 0.5 * (x_in[3] + x_out[3])
    mu_min = -np.sqrt(1 - (x_in[0] / x) ** 2)
    assert np.isfinite(oracle.virtual_tau(om, x, mu_min + 1e-9, 3, 1e15, 0))
    assert oracle.virtual_tau(om, x, mu_min - 1e-9, 3, 1e15, 0) == np.inf


def test_tau_cut():
    spec, om = _one_line_model(40.0)
    x_in, x_out = _x(spec)
    nu_lab = spec.nu[0] / (1.0 - 0.5 * (x_in[0] + x_out[-1]))
    assert oracle.virtual_tau(om, x_in[0], 1.0, 0, nu_lab, 0) == 40.0
    om.set_virtual(0, tau_v_max=30.0)
    assert oracle.virtual_tau(om, x_in[0], 1.0, 0, nu_lab, 0) == np.inf
    om.set_virtual(0, tau_v_max=50.0)
    assert oracle.virtual_tau(om, x_in[0], 1.0, 0, nu_lab, 0) == 40.0


def test_scattering_model_v_and_r_spectra_agree_and_v_is_less_noisy():
    # scatter mode, electron scattering tau ~ 3 and median line depth 1
    spec = synth.scatter_model(n_packets=4000, n_shells=10, n_lines=400, n_e_inner=1e10, tau_mu=0.0)
    om = oracle.OracleModel(spec, tau=spec.tau)
    om.set_virtual(3)
    B = spec.spec_bins
    fine_r, fine_v = [], []
    for seed in range(16):
        r = oracle.run_iteration(om, 100 + seed, 0, spec.n_packets, spec.t_inner, threads=4, record=False)
        fine_r.append(r.spectrum[:B])
        fine_v.append(r.spectrum_v[:B])
    fine_r, fine_v = np.array(fine_r), np.array(fine_v)
    # the same emergent spectrum: totals and 10 coarse bins agree within 5 sigma
    d = fine_v.sum(axis=1) - fine_r.sum(axis=1)
    assert abs(d.mean()) < 5 * d.std(ddof=1) / np.sqrt(d.size)
    coarse_r, coarse_v = fine_r.reshape(16, 10, -1).sum(axis=2), fine_v.reshape(16, 10, -1).sum(axis=2)
    big = coarse_r.mean(axis=0) > 0.02 * coarse_r.mean(axis=0).sum()
    dc = coarse_v[:, big] - coarse_r[:, big]
    z = dc.mean(axis=0) / (dc.std(axis=0, ddof=1) / np.sqrt(dc.shape[0]))
    assert np.all(np.abs(z) < 5), z
    # the point of the method: less Monte Carlo noise per spectral bin (each
    # event's v-packets spread over neighbouring bins by their Doppler shifts)
    m = fine_r.mean(axis=0)
    pop = m > 0.3 * m.max()
    noise_r = fine_r[:, pop].std(axis=0, ddof=1) / fine_r[:, pop].mean(axis=0)
    noise_v = fine_v[:, pop].std(axis=0, ddof=1) / fine_v[:, pop].mean(axis=0)
    assert np.median(noise_r / noise_v) > 1.5, np.median(noise_r / noise_v)
