"""Pins of the plasma-state functions (Sect. 2.3, Eqs. 4, 5, 12) and of the
radiation-field update (Sect. 2.7, Eqs. 15-16; Sect. 2.8 initial W).

* Populations of an ion sum to the ion density; with W = 1 (or lte mode)
  level ratios are the Boltzmann ratios (numpy exp); non-metastable levels
  carry exactly the extra factor W relative to lte.
* The Sobolev constant pi e^2 / (m_e c) = 0.02654 cm^2 s^-1 (textbook value);
  tau scales as f, 1/nu, t_exp and the ion density; with W = 1 the
  stimulated-emission factor is 1 - exp(-(eps_u - eps_l) / kT).
* Eq. 15 inverts the Planck mean frequency: for the nu_bar / J ratio of a
  blackbody (computed with scipy quadrature), T_R = T; Eq. 16 returns W for
  J = W sigma T^4 / pi.  An empty shell keeps its previous T_R and W.
* Geometric dilution equals the solid-angle fraction of the inner sphere,
  found here by integrating over directions.
"""
import numpy as np
from scipy import integrate

import oracle
from paper_1401_5469_gb300 import synth

K_B = 1.380649e-16
H = 6.62607015e-27
EV = 1.602176634e-12
SIGMA_SB = 5.670374419e-5


def _spec(n_lines=500):
    return synth.downbranch_model(n_lines=n_lines, n_ions=3, n_levels=8, n_shells=4, n_packets=10)


def test_populations_sum_and_boltzmann_ratios():
    spec = _spec()
    S, I, K = spec.n_shells, spec.n_ions, spec.n_levels
    T = np.array([6000.0, 8000.0, 10000.0, 14000.0])
    w = np.array([0.5, 0.3, 0.2, 0.1])
    n = oracle.level_populations(spec, T, w)
    np.testing.assert_allclose(n.sum(axis=2), spec.n_ion.reshape(S, I), rtol=1e-14)
    n_lte = oracle.level_populations(spec, T, w, lte_excitation=True)
    e = spec.energy_ev.reshape(I, K)
    g = spec.g.reshape(I, K)
    meta = spec.metastable.reshape(I, K).astype(bool)
    for s in range(S):
        boltz = g * np.exp(-(e * EV) / (K_B * T[s]))
        np.testing.assert_allclose(n_lte[s] / n_lte[s][:, :1], boltz / boltz[:, :1], rtol=1e-13)
        dil = n[s] / n[s][:, :1]
        expect = np.where(meta, 1.0, w[s]) * boltz / boltz[:, :1]
        np.testing.assert_allclose(dil, expect, rtol=1e-13)


def test_sobolev_constant_and_scalings():
    assert abs(oracle.sobolev_constant() / 0.026540 - 1) < 2e-4
    spec = _spec()
    T = np.full(spec.n_shells, 1.0e4)
    w = np.ones(spec.n_shells)
    n = oracle.level_populations(spec, T, w)
    tau = oracle.sobolev_tau(spec, n)
    assert np.all(tau >= 0)
    # tau / (f lambda t n_l) is the constant times the stimulated-emission factor
    K = spec.n_levels
    lev_l = spec.ion * K + spec.lower
    lev_u = spec.ion * K + spec.upper
    e = spec.energy_ev
    for s in range(spec.n_shells):
        nl = n[s].reshape(-1)[lev_l]
        lam = 2.99792458e10 / spec.nu
        stim = 1 - np.exp(-((e[lev_u] - e[lev_l]) * EV) / (K_B * T[s]))
        expect = 0.02654008854 * spec.f * lam * spec.t_exp * nl * stim
        np.testing.assert_allclose(tau[s], expect, rtol=2e-9, atol=1e-300)
    # linear in the ion density, in f and in t_exp
    spec2 = _spec()
    spec2.n_ion = spec.n_ion * 3.0
    spec2.f = spec.f * 2.0
    spec2.t_exp = spec.t_exp * 1.5
    tau2 = oracle.sobolev_tau(spec2, oracle.level_populations(spec2, T, w))
    np.testing.assert_allclose(tau2, tau * 9.0, rtol=1e-13)


def test_radiation_field_update_inverts_planck_mean():
    spec = _spec()
    S = spec.n_shells
    norm = oracle.estimator_norm(spec)
    T = np.array([7000.0, 9000.0, 11000.0, 13000.0])
    W = np.array([0.4, 0.25, 0.15, 0.08])
    # blackbody mean frequency from quadrature of x^3/(e^x - 1)
    m3 = integrate.quad(lambda x: x**3 / np.expm1(x), 0, 200)[0]
    m4 = integrate.quad(lambda x: x**4 / np.expm1(x), 0, 200)[0]
    nu_mean = (K_B * T / H) * (m4 / m3)
    J = W * SIGMA_SB * T**4 / np.pi
    j_raw = J / norm
    nb_raw = j_raw * nu_mean
    t_new, w_new = oracle.update_radiation_field(spec, j_raw, nb_raw, np.zeros(S), np.zeros(S))
    np.testing.assert_allclose(t_new, T, rtol=1e-9)
    np.testing.assert_allclose(w_new, W, rtol=1e-8)
    # an empty shell keeps its previous state
    j_raw[2] = 0.0
    nb_raw[2] = 0.0
    t2, w2 = oracle.update_radiation_field(spec, j_raw, nb_raw, np.full(S, 1.0), np.full(S, 2.0))
    assert t2[2] == 1.0 and w2[2] == 2.0


def test_geometric_dilution_is_solid_angle_fraction():
    spec = _spec()
    w = oracle.geometric_dilution(spec)
    r_i = spec.v_inner[0]
    for s in range(spec.n_shells):
        r = 0.5 * (spec.v_inner[s] + spec.v_outer[s])
        # fraction of directions mu in [-1, 1] whose ray meets the inner sphere
        hit = lambda mu: 1.0 if r * r * (1 - mu * mu) <= r_i * r_i and mu > 0 else 0.0
        frac = integrate.quad(hit, -1, 1, points=[np.sqrt(1 - (r_i / r) ** 2)], limit=200)[0] / 2
        assert abs(w[s] - frac) < 1e-9
