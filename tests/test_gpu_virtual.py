"""Virtual packets (Sect. 2.9, Eqs. 19-21) on the GPU against the oracle.

* the v-spectrum of the 2000-line scatter model (1e4 packets, N_v = 3) and of
  a 20k-line downbranch model (4e3 packets, N_v = 3, tau_v cut 30) equals the
  oracle's bin by bin within 1e-9 relative (binary64 on both sides; only the
  summation order of the bins differs);
* with v-packets on, every r-packet's fate, frequency, energy and counters
  are the same bit for bit as with them off, and so are J, nu_bar (the
  v-packets have their own draw stream);
* mixed-precision models reject v-packets; reading the v-spectrum with
  v-packets off is refused.
"""
import numpy as np
import pytest

import oracle
from paper_1401_5469_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1401_5469_gb300 import mc as mcmod
    mcmod.load()
    return mcmod


def _bins_close(g, o, rtol=1e-9):
    tol = rtol * np.abs(o) + 1e-12 * np.abs(o).max()
    bad = np.abs(g - o) > tol
    assert not bad.any(), (np.flatnonzero(bad)[:5], g[bad][:5], o[bad][:5])


def test_scatter_model_virtual_spectrum(mc):
    spec = synth.scatter_model()
    m = mc.Model(spec)
    m.set_plasma(tau=spec.tau)
    m.set_virtual_packets(3)
    m.run_iteration(5469, 0, spec.n_packets, spec.t_inner)
    g = m.virtual_spectrum()
    m.close()
    om = oracle.OracleModel(spec, tau=spec.tau)
    om.set_virtual(3)
    r = oracle.run_iteration(om, 5469, 0, spec.n_packets, spec.t_inner, threads=8, record=False)
    assert r.spectrum_v.sum() > 0
    _bins_close(g, r.spectrum_v)


def test_downbranch_model_virtual_spectrum_with_cut(mc):
    spec = synth.downbranch_model(n_lines=20000, n_shells=12, n_packets=4000, seed=77, j_blue=False)
    t_rad = np.full(spec.n_shells, 1.0e4)
    tau = oracle.plasma_tau(spec, t_rad, oracle.geometric_dilution(spec))
    m = mc.Model(spec)
    m.set_plasma(tau=tau)
    m.set_virtual_packets(3, 30.0)
    m.run_iteration(5469, 2, spec.n_packets, spec.t_inner)
    g = m.virtual_spectrum()
    m.close()
    om = oracle.OracleModel(spec, tau=tau)
    om.set_virtual(3, 30.0)
    r = oracle.run_iteration(om, 5469, 2, spec.n_packets, spec.t_inner, threads=8, record=False,
                             j_blue=False)
    assert r.spectrum_v.sum() > 0
    _bins_close(g, r.spectrum_v)


def test_r_packets_unchanged_by_virtual_packets(mc):
    spec = synth.downbranch_model(n_lines=20000, n_shells=12, n_packets=3000, seed=78)
    out = []
    for nv in (0, 4):
        m = mc.Model(spec, record_packets=True)
        m.set_plasma()
        if nv:
            m.set_virtual_packets(nv)
        m.run_iteration(11, 0, spec.n_packets, spec.t_inner)
        st, nu, e, cnt = m.packets(0, spec.n_packets)
        j, nb, _, _ = m.estimators()
        out.append((st, nu, e, cnt, j, nb))
        m.close()
    for a, b in zip(out[0][:4], out[1][:4]):
        np.testing.assert_array_equal(a, b)
    # binary64 estimator sums: summation order only
    np.testing.assert_allclose(out[1][4], out[0][4], rtol=1e-12)
    np.testing.assert_allclose(out[1][5], out[0][5], rtol=1e-12)


def test_virtual_packets_need_binary64_and_a_run(mc):
    spec = synth.scatter_model(n_packets=100)
    m = mc.Model(spec, precision=mc.MC_PRECISION_MIXED)
    with pytest.raises(mc.MCError) as ei:
        m.set_virtual_packets(3)
    assert ei.value.code == mc.MC_ERR_UNSUPPORTED
    m.close()
    m = mc.Model(spec)
    m.set_plasma(tau=spec.tau)
    m.run_iteration(1, 0, 100, spec.t_inner)
    with pytest.raises(mc.MCError):
        m.virtual_spectrum()  # v-packets off
    with pytest.raises(mc.MCError):
        m.set_virtual_packets(3, -1.0)
    m.close()
