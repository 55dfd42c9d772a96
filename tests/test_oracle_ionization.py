"""Pins of the oracle's ionization balance (Sect. 2.3, Eqs. 2-3).

* every shell conserves each element (sum over stages = element density) and
  charge (n_e = sum of stage x density over all stages);
* a hydrogen-like element (neutral stage with a 2-fold ground level, bare
  ion with Z = 1, chi = 13.6057 eV): the ionized fraction x solves
  x^2 N / (1 - x) = Phi with the textbook Saha constant
  (2 pi m_e k T / h^2)^(3/2) = 2.4147e15 T^(3/2) cm^-3, i.e.
  x = (-Phi + sqrt(Phi^2 + 4 N Phi)) / (2 N) -- in lte mode (Eq. 2) and, with
  Phi scaled by W [delta zeta + W (1 - zeta)] (0.9)^(1/2), in nebular mode
  (Eq. 3);
* more ionized at higher T_R; less at lower W (nebular mode).
"""
import numpy as np
import pytest

import oracle
from paper_1401_5469_gb300 import synth

K_EV = 8.617333262e-5  # eV / K


def _hydrogen_like(mode, n_h=1.0e10):
    spec = synth.free_streaming_model(n_shells=3)
    spec.n_ions, spec.n_levels = 1, 2
    spec.energy_ev = np.array([0.0, 10.2])
    spec.g = np.array([2.0, 8.0])
    spec.metastable = np.array([1, 0], dtype=np.uint8)
    spec.ionization_mode = mode
    spec.n_elements, spec.n_stages = 1, 2
    spec.ion_element = np.array([0], np.int32)
    spec.ion_stage = np.array([0], np.int32)
    spec.chi_ev = np.array([[13.6057]])
    spec.zeta = np.array([[0.4]])
    spec.delta = 1.0
    spec.n_element = np.full((3, 1), n_h)
    return spec


@pytest.mark.parametrize("mode", [1, 2])
def test_hydrogen_like_element_matches_the_saha_quadratic(mode):
    spec = _hydrogen_like(mode)
    t = np.array([6000.0, 9000.0, 14000.0])
    w = np.array([1.0, 0.3, 0.05])
    n_ion, n_e = oracle.ionization_state(spec, t, w)
    for s in range(3):
        kT = K_EV * t[s]
        z0 = 2.0 + 8.0 * np.exp(-10.2 / kT)  # LTE partition function of the neutral stage
        phi = 2.0 * (1.0 / z0) * 2.4147e15 * t[s] ** 1.5 * np.exp(-13.6057 / kT)
        if mode == 2:
            phi *= w[s] * (1.0 * 0.4 + w[s] * (1 - 0.4)) * np.sqrt(0.9)
        N = spec.n_element[s, 0]
        x = (-phi + np.sqrt(phi * phi + 4 * N * phi)) / (2 * N)
        assert n_e[s] == pytest.approx(x * N, rel=2e-4)  # the textbook constant has 5 digits
        assert n_ion[s, 0] == pytest.approx((1 - x) * N, rel=2e-4 * max(1.0, x / (1 - x)))


@pytest.mark.parametrize("mode", [1, 2])
def test_element_and_charge_conservation(mode):
    spec = synth.nebular_model(mode=mode, n_lines=2000, n_shells=6, n_packets=10)
    S, E, J = spec.n_shells, spec.n_elements, spec.n_stages
    for t0 in (5000.0, 9000.0, 15000.0):
        t = np.full(S, t0)
        w = oracle.geometric_dilution(spec)
        n_ion, n_e = oracle.ionization_state(spec, t, w)
        # bare stage = element density minus the stages with levels
        stages = np.zeros((S, E, J))
        for a in range(spec.n_ions):
            stages[:, spec.ion_element[a], spec.ion_stage[a]] = n_ion[:, a]
        bare = spec.n_element - stages[:, :, :J - 1].sum(axis=2)
        assert np.all(bare >= -1e-12 * spec.n_element)
        stages[:, :, J - 1] = bare
        charge = (stages * np.arange(J)).sum(axis=(1, 2))
        np.testing.assert_allclose(n_e, charge, rtol=1e-12)
        assert np.all(n_e > 0)


def test_ionization_rises_with_temperature_and_falls_with_dilution():
    spec = synth.nebular_model(mode=2, n_lines=2000, n_shells=4, n_packets=10)
    w = oracle.geometric_dilution(spec)
    ne = [oracle.ionization_state(spec, np.full(4, t), w)[1] for t in (5000.0, 8000.0, 12000.0)]
    assert np.all(ne[0] < ne[1]) and np.all(ne[1] < ne[2])
    ne_low_w = oracle.ionization_state(spec, np.full(4, 8000.0), 0.5 * w)[1]
    assert np.all(ne_low_w < ne[1])
