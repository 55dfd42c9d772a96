"""Ionization balance (Sect. 2.3, Eqs. 2-3) on the GPU against the oracle.

* the electron and ion densities from the ionization kernels equal the
  oracle's to 1e-12 relative in Saha (Eq. 2) and nebular (Eq. 3) mode, at a
  different T_R and W in every shell, and the Sobolev depths built from them
  agree to 1e-13 of the stimulated-emission bracket's magnitude;
* three iterations of the cycle in nebular mode (ionization, depths,
  transport, T_R/W update): the Thomson opacity follows the solved n_e on
  both sides, and every packet's fate, frequency, energy and counters agree
  as in the fixed-ion loop test, with J, nu_bar within 1e-9;
* mixed precision runs the same plasma kernels: its n_e is bit-identical to
  the binary64 model's;
* given Sobolev depths leave n_e at the geometry's values.
"""
import numpy as np
import pytest

import oracle
from paper_1401_5469_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL = 1e-12
EST_RTOL = 1e-9
NU_E_RTOL = 1e-12


@pytest.fixture(scope="module")
def mc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1401_5469_gb300 import mc as mcmod
    mcmod.load()
    return mcmod


def _plasma(spec):
    S = spec.n_shells
    t = np.linspace(6000.0, 14000.0, S)
    w = oracle.geometric_dilution(spec) * np.linspace(1.0, 0.4, S)
    return t, w


def _tau_close(tau_g, tau_o, spec, t, w, n_ion, rtol=1e-13):
    """Eq. 12 cancels between its two terms for levels close in energy:
    compare to the magnitude of the terms (as the fixed-ion parity test)."""
    n = oracle.level_populations(spec, t, w, n_ion=n_ion)
    K = spec.n_levels
    ll = spec.ion.astype(np.int64) * K + spec.lower
    lu = spec.ion.astype(np.int64) * K + spec.upper
    flat = n.reshape(spec.n_shells, -1)
    n_l, n_u = flat[:, ll], flat[:, lu]
    ratio = (spec.g[ll] * n_u) / (spec.g[lu] * n_l)
    pref = 0.026540088 * spec.f * (2.99792458e10 / spec.nu) * spec.t_exp
    mag = pref * n_l * (1.0 + ratio)
    err = np.abs(tau_g - tau_o) / mag
    assert np.all(err <= rtol), float(err.max())


@pytest.mark.parametrize("mode", [1, 2])
def test_ionization_state_and_depths_match_the_oracle(mc, mode):
    spec = synth.nebular_model(mode=mode, n_lines=20000, n_shells=12, n_packets=100)
    t, w = _plasma(spec)
    m = mc.Model(spec)
    m.set_plasma(t_rad=t, w=w)
    n_e, n_ion = m.ionization()
    _, _, tau = m.plasma()
    m.close()
    o_ion, o_e = oracle.ionization_state(spec, t, w)
    np.testing.assert_allclose(n_e, o_e, rtol=RTOL)
    np.testing.assert_allclose(n_ion, o_ion, rtol=RTOL, atol=1e-300)
    # the solution is not the fixed-ion input
    assert np.max(np.abs(n_ion / spec.n_ion.reshape(n_ion.shape) - 1)) > 0.1
    _tau_close(tau, oracle.plasma_tau(spec, t, w), spec, t, w, o_ion)


def test_nebular_loop_parity(mc):
    spec = synth.nebular_model(mode=2, n_lines=20000, n_shells=12, n_packets=4000)
    n = spec.n_packets
    m = mc.Model(spec, record_packets=True, max_packets=n, j_blue=False)
    m.set_plasma()
    ref = oracle.run_loop(spec, 3, n, spec.seed, record=True)
    for it in range(3):
        m.run_iteration(spec.seed, it, n, spec.t_inner)
        n_e, _ = m.ionization()
        np.testing.assert_allclose(n_e, ref[it].n_e, rtol=RTOL if it == 0 else 1e-8)
        if it == 0:
            # the Thomson opacity is not the geometry's
            assert np.max(np.abs(n_e / spec.n_e - 1)) > 0.1
        st, nu, e, cnt = m.packets(0, n)
        agree = st == ref[it].status
        assert (~agree).sum() <= int(1e-5 * n), (~agree).sum()
        np.testing.assert_allclose(nu[agree], ref[it].nu[agree], rtol=NU_E_RTOL)
        np.testing.assert_allclose(e[agree], ref[it].energy[agree], rtol=NU_E_RTOL)
        assert np.array_equal(cnt[agree], ref[it].counters[agree])
        j, nb, _, _ = m.estimators()
        if agree.all():
            np.testing.assert_allclose(j, ref[it].j_est, rtol=EST_RTOL)
            np.testing.assert_allclose(nb, ref[it].nu_bar, rtol=EST_RTOL)
        t_out, w_out = m.update_radiation_field()
        np.testing.assert_allclose(t_out, ref[it].t_rad_out, rtol=EST_RTOL)
        np.testing.assert_allclose(w_out, ref[it].w_out, rtol=EST_RTOL)
    m.close()


def test_mixed_precision_uses_the_same_solution(mc):
    spec = synth.nebular_model(mode=2, n_lines=5000, n_shells=10, n_packets=2000)
    t, w = _plasma(spec)
    out = []
    for prec in (mc.MC_PRECISION_FP64, mc.MC_PRECISION_MIXED):
        m = mc.Model(spec, precision=prec)
        m.set_plasma(t_rad=t, w=w)
        m.run_iteration(3, 0, spec.n_packets, spec.t_inner)
        n_e, n_ion = m.ionization()
        _, stats, _ = m.spectrum()
        assert stats["packets"] == spec.n_packets
        out.append((n_e, n_ion))
        m.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])


def test_given_depths_keep_the_geometry_electron_density(mc):
    spec = synth.nebular_model(mode=1, n_lines=2000, n_shells=6, n_packets=100)
    m = mc.Model(spec)
    m.set_plasma(tau=np.zeros((spec.n_shells, spec.n_lines)))
    n_e, _ = m.ionization()
    np.testing.assert_array_equal(n_e, spec.n_e)
    m.close()
