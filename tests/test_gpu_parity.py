"""GPU <-> oracle parity through the C ABI.

Tolerances (floating point decides fates, so they are checked first):
  * packet fates: at most 1e-5 of packets may differ (expected 0 at these sizes);
  * per-packet final lab frequency and energy where fates agree: 1e-12 relative;
  * per-packet counters (segments, line checks, resonances, interactions):
    exactly equal where fates agree;
  * shell estimators J, nu_bar, the spectrum and J_blue: 1e-9 relative;
  * Sobolev depths from the plasma kernels: 1e-13 relative;
  * T_R, W after the radiation-field update: 1e-9 relative.
The GPU evaluates the same formulas with FMA and reciprocals and integer
comparison keys, so agreement is to rounding, not bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_1401_5469_gb300 import synth

pytestmark = pytest.mark.gpu

FATE_TOL = 1e-5
NU_E_RTOL = 1e-12
EST_RTOL = 1e-9
TAU_RTOL = 1e-13


@pytest.fixture(scope="module")
def mc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1401_5469_gb300 import mc as mcmod
    mcmod.load()
    return mcmod


def _compare_packets(st_g, nu_g, e_g, cnt_g, r):
    n = st_g.size
    agree = st_g == r.status
    assert (n - agree.sum()) <= max(0, int(FATE_TOL * n)), f"{n - agree.sum()} fate mismatches of {n}"
    np.testing.assert_allclose(nu_g[agree], r.nu[agree], rtol=NU_E_RTOL)
    np.testing.assert_allclose(e_g[agree], r.energy[agree], rtol=NU_E_RTOL)
    assert np.array_equal(cnt_g[agree], r.counters[agree])
    return agree


def _close(a, b, rtol):
    a, b = np.asarray(a), np.asarray(b)
    scale = np.maximum(np.abs(b), 1e-300)
    assert np.all(np.abs(a - b) <= rtol * scale + 1e-300), np.max(np.abs(a - b) / scale)


def _tau_close(tau_g, spec, t_rad, w, tau_o, t_rad_g=None, w_g=None, where=""):
    """Sobolev depths agree to 1e-13 of the magnitude of the two terms of the
    stimulated-emission bracket (Eq. 12 cancels when the levels are close in
    energy; both sides lose the same digits there), widened by the difference
    of the two sides' own T_R and W (after an update they differ by the
    estimators' summation order): d ln n / d ln T = eps / kT <= 60 here."""
    rel_t = 0.0 if t_rad_g is None else float(np.max(np.abs(t_rad_g / t_rad - 1)))
    rel_w = 0.0 if w_g is None else float(np.max(np.abs(w_g / w - 1)))
    rtol = TAU_RTOL + 60.0 * rel_t + 2.0 * rel_w
    n = oracle.level_populations(spec, t_rad, w)
    K = spec.n_levels
    ll = spec.ion.astype(np.int64) * K + spec.lower
    lu = spec.ion.astype(np.int64) * K + spec.upper
    flat = n.reshape(spec.n_shells, -1)
    n_l, n_u = flat[:, ll], flat[:, lu]
    ratio = (spec.g[ll] * n_u) / (spec.g[lu] * n_l)
    pref = 0.026540088 * spec.f * (2.99792458e10 / spec.nu) * spec.t_exp
    mag = pref * n_l * (1.0 + ratio)
    err = np.abs(tau_g - tau_o) / mag
    assert np.all(err <= rtol), (where, float(err.max()), rtol)


def _run_gpu(mc, spec, tau, n, seed, it=0, **kw):
    m = mc.Model(spec, record_packets=True, max_packets=n, **kw)
    m.set_plasma(tau=tau)
    m.run_iteration(seed, it, n, spec.t_inner)
    return m


@pytest.mark.parametrize("n_packets", [1, 31, 10_000])
def test_scatter_model_parity(mc, n_packets):
    """Plain scatter mode, 20 shells, 2000 lines, lognormal tau (full size at 1e4)."""
    spec = synth.scatter_model(n_lines=2000, n_packets=n_packets)
    m = _run_gpu(mc, spec, spec.tau, n_packets, 5469)
    st, nu, e, cnt = m.packets(0, n_packets)
    j, nb, _, norm = m.estimators()
    sp, stats, _ = m.spectrum()
    om = oracle.OracleModel(spec)
    r = oracle.run_iteration(om, 5469, 0, n_packets, spec.t_inner)
    agree = _compare_packets(st, nu, e, cnt, r)
    assert agree.all()
    _close(j, r.j_est, EST_RTOL)
    _close(nb, r.nu_bar, EST_RTOL)
    _close(sp, r.spectrum, EST_RTOL)
    assert stats["escaped"] == r.stats["escaped"]
    assert stats["line_checks"] == r.stats["line_checks"]
    assert stats["segments"] == r.stats["segments"]
    np.testing.assert_allclose(norm, oracle.estimator_norm(spec), rtol=1e-14)
    m.close()


def test_downbranch_loop_parity(mc):
    """Downbranch + J_blue, tau from the plasma kernels, 3 iterations with the
    T_R/W update between them (oracle iterates independently)."""
    spec = synth.downbranch_model(n_lines=20_000, n_packets=4000, n_iterations=3)
    n = spec.n_packets
    m = mc.Model(spec, record_packets=True, max_packets=n)
    m.set_plasma()
    ref = oracle.run_loop(spec, 3, n, spec.seed, record=True)
    for it in range(3):
        m.run_iteration(spec.seed, it, n, spec.t_inner)
        t_in, w_in, tau = m.plasma()
        np.testing.assert_allclose(t_in, ref[it].t_rad_in, rtol=EST_RTOL)
        np.testing.assert_allclose(w_in, ref[it].w_in, rtol=EST_RTOL)
        _tau_close(tau, spec, ref[it].t_rad_in, ref[it].w_in, ref[it].tau, t_in, w_in, f"iteration {it}")
        st, nu, e, cnt = m.packets(0, n)
        agree = _compare_packets(st, nu, e, cnt, ref[it])
        assert agree.all()
        j, nb, jb, _ = m.estimators(j_blue=True)
        _close(j, ref[it].j_est, EST_RTOL)
        _close(nb, ref[it].nu_bar, EST_RTOL)
        _close(jb, ref[it].j_blue, EST_RTOL)
        sp, stats, _ = m.spectrum()
        _close(sp, ref[it].spectrum, EST_RTOL)
        t_out, w_out = m.update_radiation_field()
        np.testing.assert_allclose(t_out, ref[it].t_rad_out, rtol=EST_RTOL)
        np.testing.assert_allclose(w_out, ref[it].w_out, rtol=EST_RTOL)
    m.close()


def test_full_size_downbranch_sampled_packets(mc):
    """500,000 lines, 1e6 packets in the benchmark's launch configuration; the
    oracle recomputes a sample of packets one by one (Philox is keyed by packet
    id, so any packet is reproducible alone)."""
    spec = synth.downbranch_model()
    n = spec.n_packets
    t_rad = np.full(spec.n_shells, 1.0e4)
    w = oracle.geometric_dilution(spec)
    m = mc.Model(spec, record_packets=True, max_packets=n)
    m.set_plasma(t_rad, w)
    m.run_iteration(spec.seed, 0, n, spec.t_inner)
    _, _, tau = m.plasma()
    tau_ref = oracle.plasma_tau(spec, t_rad, w)
    _tau_close(tau, spec, t_rad, w, tau_ref)
    om = oracle.OracleModel(spec, tau=tau_ref)
    rng = np.random.default_rng(8)
    ids = np.concatenate([np.arange(64), rng.choice(n, size=1500, replace=False), [n - 1]])
    st, nu, e, cnt = m.packets(0, n)
    sp, stats, _ = m.spectrum()
    for pid in ids:
        r = oracle.run_iteration(om, spec.seed, 0, n, spec.t_inner, first=int(pid), count=1, j_blue=False)
        sl = slice(int(pid), int(pid) + 1)
        _compare_packets(st[sl], nu[sl], e[sl], cnt[sl], r)
    # totals are sums of the per-packet records
    assert stats["escaped"] == int((st == 1).sum())
    assert stats["reabsorbed"] == int((st == 2).sum())
    assert stats["segments"] == int(cnt[:, 0].sum())
    assert stats["line_checks"] == int(cnt[:, 1].sum())
    esc = st == 1
    _close(sp[:-2].sum() + sp[-2] + sp[-1], e[esc].sum(), 1e-9)
    m.close()


def test_edge_cases(mc):
    # one shell, one line, no electrons; ragged packet count
    spec = synth.ModelSpec(name="edge", v_inner=np.array([1.1e9]), v_outer=np.array([2.0e9]),
                           n_e=np.array([0.0]), t_exp=13 * 86400.0, nu=np.array([6.0e14]),
                           tau=np.array([[1.0]]), spec_bins=7)
    for n in (1, 2, 33, 257):
        m = _run_gpu(mc, spec, spec.tau, n, 11)
        st, nu, e, cnt = m.packets(0, n)
        r = oracle.run_iteration(oracle.OracleModel(spec), 11, 0, n, spec.t_inner)
        assert _compare_packets(st, nu, e, cnt, r).all()
        m.close()
    # transparent ejecta: every packet escapes with its injection values
    fs = synth.free_streaming_model(n_packets=5000)
    m = _run_gpu(mc, fs, fs.tau, 5000, 3)
    st, nu, e, cnt = m.packets(0, 5000)
    inj = oracle.inject_packets(oracle.OracleModel(fs), 3, 0, 5000, fs.t_inner)
    assert np.all(st == 1)
    np.testing.assert_allclose(nu, inj["nu_lab"], rtol=NU_E_RTOL)
    np.testing.assert_allclose(e, inj["e_lab"], rtol=NU_E_RTOL)
    m.close()
    # segment cap: capped fates and counters agree with the oracle
    spec = synth.scatter_model(n_lines=2000, n_packets=3000)
    m = _run_gpu(mc, spec, spec.tau, 3000, 5, max_segments=4)
    st, nu, e, cnt = m.packets(0, 3000)
    _, stats, rc = m.spectrum()
    r = oracle.run_iteration(oracle.OracleModel(spec, max_segments=4), 5, 0, 3000, spec.t_inner)
    assert _compare_packets(st, nu, e, cnt, r).all()
    assert stats["capped"] == r.stats["capped"] > 0
    assert rc == mc.MC_WARN_CAPPED
    m.close()


def test_deadline_returns_timeout_status(mc):
    spec = synth.downbranch_model(n_lines=50_000, n_packets=200_000)
    m = mc.Model(spec, timeout_ns=1000)  # 1 microsecond
    m.set_plasma()
    m.run_iteration(1, 0, spec.n_packets, spec.t_inner)
    with pytest.raises(mc.MCError) as ei:
        m.estimators()
    assert ei.value.code == mc.MC_ERR_TIMEOUT
    # the context stays usable: a run without deadline afterwards succeeds
    m.close()
    m2 = mc.Model(spec)
    m2.set_plasma()
    m2.run_iteration(1, 0, 1000, spec.t_inner)
    m2.estimators()
    m2.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_maximum_shell_count(mc, precision):
    """1024 shells, the most the shell tables in shared memory hold (the
    binary64 kernel then needs more than 48 KB of dynamic shared memory):
    per-packet parity in binary64; in mixed precision every packet finishes
    and the escaped fraction matches the oracle's within the noise."""
    spec = synth.scatter_model(n_lines=2000, n_shells=1024, n_packets=2000)
    n = spec.n_packets
    m = _run_gpu(mc, spec, spec.tau, n, 21, precision=precision)
    st, nu, e, cnt = m.packets(0, n)
    _, stats, _ = m.spectrum()
    m.close()
    r = oracle.run_iteration(oracle.OracleModel(spec, tau=spec.tau), 21, 0, n, spec.t_inner, threads=8)
    assert stats["packets"] == n and stats["shell_crossings"] > 100 * n
    if precision == 0:
        assert _compare_packets(st, nu, e, cnt, r).all()
    else:
        esc, esc_o = (st == 1).mean(), (r.status == 1).mean()
        assert abs(esc - esc_o) < 5 * np.sqrt(esc_o * (1 - esc_o) / n) + 1e-3
