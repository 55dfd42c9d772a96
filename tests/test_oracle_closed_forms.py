"""Closed-form pins of the oracle at finite v/c (Doppler factors) and of the
J_blue estimator and the line-by-line optical-depth accounting.

* Thomson opacity kappa_e = sigma_T n_e D (Eq. 11) with D evaluated at the
  segment start: for a transparent-to-lines shell at v/c ~ 0.1 the fraction
  of packets that leave without scattering is E_mu[exp(-kappa' (1 - p0) d)],
  p0 = x0 mu, d the straight path to the outer boundary (quadrature over the
  injected mu ~ 2 mu).
* Free-streaming estimators (Eqs. 13-14) at v/c ~ 0.1: a packet injected with
  direction mu crosses shell s on a straight line entering at x mu =
  p_s = sqrt(x_s^2 - q) (q the squared impact parameter); its contribution is
  E_lab D_s^2 (p_{s+1} - p_s), E_lab = E / (1 - x0 mu).  Expectations by
  quadrature.
* J_blue (Eq. 17, resonance path c t_exp): in free streaming with v/c -> 0 the
  mean intensity at the blue wing of every line is W(r) B_nu(T_inner), so
  sum_j J_b[s][j] / sum_j W_s B_nu(nu_j) -> 1.
* Two lines in one segment: a packet that reaches the second line's Sobolev
  point after passing the first is absorbed there with probability
  1 - exp(-tau_2) (memoryless; tau is reduced by the first line's depth).
"""
import numpy as np
import pytest
from scipy import integrate, special, stats

import oracle
from paper_1401_5469_gb300 import synth

C_LIGHT = 2.99792458e10
SIGMA_T = 6.6524587321e-25
SIGMA_SB = 5.670374419e-5
H = 6.62607015e-27
K_B = 1.380649e-16


def _shells(x_edges, n_e, nu, tau, t_days=13.0):
    S = len(x_edges) - 1
    return synth.ModelSpec(name="cf", v_inner=np.asarray(x_edges[:-1]) * C_LIGHT,
                           v_outer=np.asarray(x_edges[1:]) * C_LIGHT, n_e=np.full(S, n_e),
                           t_exp=t_days * 86400.0, nu=np.asarray(nu, float),
                           tau=np.asarray(tau, float).reshape(S, -1), spec_bins=10)


def test_thomson_opacity_doppler_factor():
    x0, x1 = 0.05, 0.15
    t = 13.0 * 86400.0
    kappa_p = 0.5  # sigma_T n_e c t_exp per unit x
    n_e = kappa_p / (SIGMA_T * C_LIGHT * t)
    spec = _shells([x0, x1], n_e, [1.0e12], [[0.0]])
    N = 1_000_000
    r = oracle.run_iteration(oracle.OracleModel(spec), 314, 0, N, 1.0e4, threads=4)
    no_scatter = int((r.counters[:, 4] == 0).sum())

    def p_no(mu):
        p0 = x0 * mu
        q = x0 * x0 * (1 - mu * mu)
        d = np.sqrt(x1 * x1 - q) - p0
        return 2 * mu * np.exp(-kappa_p * (1 - p0) * d)

    expect = integrate.quad(p_no, 0, 1, epsabs=1e-13)[0]
    assert stats.binomtest(no_scatter, N, expect).pvalue > 1e-4, (no_scatter / N, expect)


def test_free_streaming_estimators_at_finite_velocity():
    edges = np.array([0.05, 0.075, 0.1, 0.125, 0.15])
    spec = _shells(edges, 0.0, [1.0e12], np.zeros((4, 1)))
    om = oracle.OracleModel(spec)
    T = 1.0e4
    N = 50_000
    runs = [oracle.run_iteration(om, 900 + b, 0, N, T, record=False) for b in range(8)]
    J = np.array([r.j_est for r in runs])
    NB = np.array([r.nu_bar for r in runs])
    x0 = edges[0]
    r_i = x0 * C_LIGHT * spec.t_exp
    E0 = 4 * np.pi * r_i**2 * SIGMA_SB * T**4 / N
    nu_mean = (K_B * T / H) * 360 * special.zeta(5) / np.pi**4

    def p_at(x, mu):
        q = x0 * x0 * (1 - mu * mu)
        return np.sqrt(np.maximum(x * x - q, 0.0))

    for s in range(4):
        def fj(mu, power_d, power_inj):
            ps = x0 * mu if s == 0 else p_at(edges[s], mu)
            pe = p_at(edges[s + 1], mu)
            return 2 * mu * (1 - ps) ** power_d * (pe - ps) / (1 - x0 * mu) ** power_inj
        ej = N * E0 * integrate.quad(fj, 0, 1, args=(2, 1), epsabs=1e-15, limit=200)[0]
        enb = N * E0 * nu_mean * integrate.quad(fj, 0, 1, args=(3, 2), epsabs=1e-15, limit=200)[0]
        sj = J[:, s].std(ddof=1) / np.sqrt(len(runs))
        snb = NB[:, s].std(ddof=1) / np.sqrt(len(runs))
        assert abs(J[:, s].mean() - ej) < 4 * sj, (s, J[:, s].mean() / ej)
        assert abs(NB[:, s].mean() - enb) < 4 * snb, (s, NB[:, s].mean() / enb)


def test_j_blue_is_dilute_blackbody_in_free_streaming():
    edges = np.array([1.0e-3, 1.2e-3, 1.4e-3, 1.6e-3])
    rng = np.random.default_rng(2)
    nu = np.sort(np.exp(rng.uniform(np.log(2e14), np.log(2e15), 3000)))[::-1].copy()
    spec = _shells(edges, 0.0, nu, np.zeros((3, nu.size)))
    spec.j_blue = True
    om = oracle.OracleModel(spec)
    T = 1.0e4
    N = 400_000
    r = oracle.run_iteration(om, 77, 0, N, T, threads=4, record=False)
    norm = oracle.estimator_norm(spec)
    B = 2 * H * nu**3 / C_LIGHT**2 / np.expm1(H * nu / (K_B * T))
    r_i = edges[0]
    wgeo = lambda x: 0.5 * (1 - np.sqrt(1 - (r_i / x) ** 2))
    for s in range(3):
        a, b = edges[s], edges[s + 1]
        wv = integrate.quad(lambda x: wgeo(x) * x * x, a, b)[0] / ((b**3 - a**3) / 3)
        got = (r.j_blue[s] * norm[s]).sum()
        want = wv * B.sum()
        n_res = np.count_nonzero(r.j_blue[s])
        assert n_res > 2000
        assert abs(got / want - 1) < 4 / np.sqrt(n_res) + 5e-3, (s, got / want)


@pytest.mark.parametrize("tau1,tau2", [(0.5, 0.2), (0.1, 1.5)])
def test_second_line_absorbs_with_its_own_depth(tau1, tau2):
    spec = _shells([0.05, 0.25], 0.0, [6.0e14, 5.9e14], [[tau1, tau2]])
    om = oracle.OracleModel(spec, max_segments=1)  # first flight segment only
    r = oracle.run_iteration(om, 21, 0, 1_000_000, 1.0e4, threads=4)
    c = r.counters
    both = c[:, 2] == 2
    k = int((c[both, 3] == 1).sum())
    n = int(both.sum())
    assert n > 5000
    assert stats.binomtest(k, n, 1 - np.exp(-tau2)).pvalue > 1e-4, (k / n, 1 - np.exp(-tau2))
