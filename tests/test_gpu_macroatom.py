"""Macro-atom mode (Sect. 2.5) on the GPU against the oracle, per packet.

Binary64 transport of a 20k-line macro-atom model (synthetic internal jumps,
Sobolev depths from the plasma kernels' inputs): every packet's fate agrees,
final lab frequency and energy within 1e-12, counters equal; J, nu_bar and the
spectrum within 1e-9.  A second case raises every jump probability to 0.99
(~100 jumps per interaction, many draws per segment) on 31 packets, whose
warps read warp-computed draws from the first segment and run past the end of
that buffer: the same per-packet parity must hold.  The mixed kernel runs
the same walk: within the Monte Carlo noise of binary64, and batched models
bit-identical to the same models alone.
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


def _mixed_run(mc, spec, tau, precision, seed):
    m = mc.Model(spec, precision=precision)
    m.set_plasma(tau=tau)
    m.run_iteration(seed, 0, spec.n_packets, spec.t_inner)
    j, nb, _, norm = m.estimators()
    _, st, _ = m.spectrum()
    m.close()
    return j * norm, nb * norm, st


def test_macroatom_mixed_precision_within_monte_carlo_noise(mc):
    """The mixed kernel's macro-atom walk (same integer thresholds and draws):
    J and nu_bar within 5 sigma of the binary64 run with the same seed, sigma
    from 8 binary64 seeds; interaction counts likewise."""
    spec = synth.macroatom_model(n_lines=20000, n_shells=12, n_packets=20000, seed=23)
    tau = oracle.plasma_tau(spec, np.full(spec.n_shells, 1.0e4), oracle.geometric_dilution(spec))
    ref = [_mixed_run(mc, spec, tau, mc.MC_PRECISION_FP64, 700 + k) for k in range(8)]
    J = np.array([r[0] for r in ref])
    NB = np.array([r[1] for r in ref])
    sJ, sNB = J.std(0, ddof=1), NB.std(0, ddof=1)
    j32, nb32, st32 = _mixed_run(mc, spec, tau, mc.MC_PRECISION_MIXED, 700)
    keep = sJ > 0
    assert np.all(np.abs(j32 - ref[0][0])[keep] <= 5 * sJ[keep] + 1e-12 * np.abs(ref[0][0][keep]))
    assert np.all(np.abs(nb32 - ref[0][1])[keep] <= 5 * sNB[keep] + 1e-12 * np.abs(ref[0][1][keep]))
    li = np.array([r[2]["line_interactions"] for r in ref], dtype=float)
    assert abs(st32["line_interactions"] - li[0]) <= 5 * li.std(ddof=1) + 1
    assert st32["line_interactions"] > 10 * spec.n_packets


def test_macroatom_batch_equals_solo(mc):
    """Macro-atom models in a batch compute what they compute alone (mixed
    precision; packets, J and nu_bar bit for bit)."""
    specs = [synth.macroatom_model(n_lines=L, n_shells=S, n_packets=N, seed=30 + k)
             for k, (S, L, N) in enumerate([(8, 4000, 800), (12, 9000, 1500), (10, 6000, 500)])]
    solo = []
    for k, spec in enumerate(specs):
        m = mc.Model(spec, precision=mc.MC_PRECISION_MIXED, record_packets=True)
        m.set_plasma()
        m.run_iteration(40 + k, 0, spec.n_packets, spec.t_inner)
        pk = m.packets(0, spec.n_packets)
        j, nb, _, _ = m.estimators()
        solo.append((pk, j, nb))
        m.close()
    models = [mc.Model(s, precision=mc.MC_PRECISION_MIXED, record_packets=True) for s in specs]
    for m in models:
        m.set_plasma()
    b = mc.Batch(models)
    b.run_iteration([40 + k for k in range(3)], 0, [s.n_packets for s in specs],
                    [s.t_inner for s in specs], update=False)
    b.synchronize()
    for k, m in enumerate(models):
        pk = m.packets(0, specs[k].n_packets)
        j, nb, _, _ = m.estimators()
        for a, c in zip(pk, solo[k][0]):
            assert np.array_equal(a, c), k
        assert np.array_equal(j, solo[k][1]) and np.array_equal(nb, solo[k][2]), k
    b.close()
    for m in models:
        m.close()
