"""Macro-atom mode (Sect. 2.5) on the GPU against the oracle, per packet.

Binary64 transport of a 20k-line macro-atom model (synthetic internal jumps,
Sobolev depths from the plasma kernels' inputs): every packet's fate agrees,
final lab frequency and energy within 1e-12, counters equal; J, nu_bar and the
spectrum within 1e-9.  A second case raises every jump probability to 0.99
(~100 jumps per interaction, many draws per segment) on 31 packets, whose
warps read warp-computed draws from the first segment and run past the end of
that buffer: the same per-packet parity must hold.
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


def _run_both(mc, spec, n, seed=5469, it=0):
    tau = oracle.plasma_tau(spec, np.full(spec.n_shells, 1.0e4), oracle.geometric_dilution(spec))
    m = mc.Model(spec, record_packets=True, max_packets=n, j_blue=False)
    m.set_plasma(tau=tau)
    m.run_iteration(seed, it, n, spec.t_inner)
    st, nu, e, cnt = m.packets(0, n)
    j, nb, _, _ = m.estimators()
    sp, stats, _ = m.spectrum()
    m.close()
    om = oracle.OracleModel(spec, tau=tau)
    r = oracle.run_iteration(om, seed, it, n, spec.t_inner, threads=8, record=True, j_blue=False)
    return (st, nu, e, cnt, j, nb, sp, stats), r


def _check(g, r):
    st, nu, e, cnt, j, nb, sp, stats = g
    agree = st == r.status
    assert (~agree).sum() <= max(0, int(1e-5 * st.size)), (~agree).sum()
    np.testing.assert_allclose(nu[agree], r.nu[agree], rtol=1e-12)
    np.testing.assert_allclose(e[agree], r.energy[agree], rtol=1e-12)
    assert np.array_equal(cnt[agree], r.counters[agree])
    if agree.all():
        np.testing.assert_allclose(j, r.j_est, rtol=1e-9)
        np.testing.assert_allclose(nb, r.nu_bar, rtol=1e-9)
        np.testing.assert_allclose(sp, r.spectrum, rtol=1e-9, atol=1e-12 * np.abs(r.spectrum).max())
    assert stats["line_interactions"] == r.stats["line_interactions"]


def test_macroatom_model_per_packet_parity(mc):
    spec = synth.macroatom_model(n_lines=20000, n_shells=12, n_packets=5000, seed=21)
    g, r = _run_both(mc, spec, spec.n_packets)
    assert r.stats["line_interactions"] > 10 * spec.n_packets
    _check(g, r)


def test_macroatom_many_jumps_few_packets(mc):
    spec = synth.macroatom_model(n_lines=8000, n_shells=8, n_packets=31, seed=22)
    spec.ma_jump_p = np.where(spec.ma_jump_p > 0, 0.99, 0.0)
    g, r = _run_both(mc, spec, 31)
    assert r.stats["line_interactions"] > 31
    _check(g, r)


def test_macroatom_needs_binary64(mc):
    spec = synth.macroatom_model(n_lines=2000, n_shells=4, n_packets=10)
    with pytest.raises(mc.MCError) as ei:
        mc.Model(spec, precision=mc.MC_PRECISION_MIXED)
    assert ei.value.code == mc.MC_ERR_UNSUPPORTED
