"""Pins of the oracle's macro-atom mode (Sect. 2.5).

An activated macro atom is an absorbing Markov chain over the levels of its
ion: from level r it jumps to r' with probability Q[r, r'] = p_r w_{r->r'}
and deactivates through line l with probability R[r, l] = (1 - p_r) b_{r,l}
(b: the level's branching ratios).  The probability of finally emitting line l
after activation in level r0 is therefore [(I - Q)^-1 R][r0, l], and the mean
number of jumps [(I - Q)^-1 Q 1][r0] -- linear algebra independent of the
walk.  The oracle's walks must reproduce both (multinomial chi-square and a
5-sigma mean), also with all jump probabilities zero (then the emission is
the downbranch choice) and with jump probabilities near 1 (the walk still
ends).  In transport, each macro-atom interaction conserves the comoving
energy and the emitted packet leaves from the absorbing line's Sobolev point.
"""
import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1401_5469_gb300 import synth


def _model(p_jump_max=0.5, seed=11):
    return synth.macroatom_model(n_lines=3000, n_shells=6, n_ions=3, n_levels=12, n_packets=500,
                                 seed=seed, p_jump_max=p_jump_max)


def _chain(spec, ion):
    """Q (jumps among the ion's levels), R (emission of each line) and the
    row and line index maps, from the model's tables."""
    K = spec.n_levels
    rows = list(range(ion * K, (ion + 1) * K))
    ridx = {r: i for i, r in enumerate(rows)}
    off = spec.dbr_offset.astype(np.int64)
    lines = sorted({int(spec.dbr_line[k]) for r in rows for k in range(off[r], off[r + 1])})
    lidx = {l: i for i, l in enumerate(lines)}
    Q = np.zeros((K, K))
    R = np.zeros((K, len(lines)))
    joff = spec.ma_jump_offset.astype(np.int64)
    for r in rows:
        p = spec.ma_jump_p[r]
        prev = 0.0
        for k in range(joff[r], joff[r + 1]):
            Q[ridx[r], ridx[int(spec.ma_jump_target[k])]] += p * (spec.ma_jump_cdf[k] - prev)
            prev = spec.ma_jump_cdf[k]
        prev = 0.0
        for k in range(off[r], off[r + 1]):
            R[ridx[r], lidx[int(spec.dbr_line[k])]] += (1.0 - p) * (spec.dbr_cdf[k] - prev)
            prev = spec.dbr_cdf[k]
    return rows, ridx, lines, lidx, Q, R


def _check_walks(spec, om, n=200_000):
    checked = 0
    for ion in range(spec.n_ions):
        rows, ridx, lines, lidx, Q, R = _chain(spec, ion)
        N = np.linalg.inv(np.eye(len(rows)) - Q)
        B = N @ R                      # emission probabilities
        mean_jumps = N @ Q @ np.ones(len(rows))
        for r0 in rows:
            if spec.dbr_offset[r0 + 1] == spec.dbr_offset[r0]:
                continue  # a level without emission lines is never activated
            assert B[ridx[r0]].sum() == pytest.approx(1.0, abs=1e-12)
            line, jumps = oracle.macroatom_walks(om, r0, 1234 + r0, n)
            counts = np.bincount([lidx[int(l)] for l in line], minlength=len(lines))
            exp = B[ridx[r0]] * n
            big = exp >= 5
            # lines with tiny expectation pooled into one cell
            obs = np.append(counts[big], counts[~big].sum())
            ex = np.append(exp[big], exp[~big].sum())
            keep = ex > 0
            chi2 = np.sum((obs[keep] - ex[keep]) ** 2 / ex[keep])
            pval = stats.chi2.sf(chi2, keep.sum() - 1)
            assert pval > 1e-5, (ion, r0, chi2, keep.sum())
            m, sd = jumps.mean(), jumps.std(ddof=1)
            assert abs(m - mean_jumps[ridx[r0]]) < 5 * sd / np.sqrt(n) + 1e-12, (r0, m, mean_jumps[ridx[r0]])
            checked += 1
            if checked >= 12:
                return


def test_walks_match_the_absorbing_markov_chain():
    spec = _model()
    _check_walks(spec, oracle.OracleModel(spec, tau=np.zeros((spec.n_shells, spec.n_lines))))


def test_without_jumps_the_atom_deactivates_from_the_activated_level():
    spec = _model()
    spec.ma_jump_p = np.zeros_like(spec.ma_jump_p)
    om = oracle.OracleModel(spec, tau=np.zeros((spec.n_shells, spec.n_lines)))
    _check_walks(spec, om, n=100_000)
    line, jumps = oracle.macroatom_walks(om, int(om.line_row[0]), 9, 1000)
    assert jumps.max() == 0


def test_walks_end_with_jump_probabilities_near_one():
    # p = 0.99: ~100 jumps per walk; the 1024-jump cap binds with probability
    # 0.99^1024 = 3e-5, so the walks still follow the chain
    spec = _model()
    spec.ma_jump_p = np.where(spec.ma_jump_p > 0, 0.99, 0.0)
    om = oracle.OracleModel(spec, tau=np.zeros((spec.n_shells, spec.n_lines)))
    _check_walks(spec, om, n=50_000)
    line, jumps = oracle.macroatom_walks(om, int(om.line_row[0]), 9, 2000)
    assert jumps.max() <= 1024 and jumps.mean() > 50


def test_macroatom_events_conserve_comoving_energy_at_the_sobolev_point():
    spec = _model()
    tau = oracle.plasma_tau(spec, np.full(spec.n_shells, 1e4), oracle.geometric_dilution(spec))
    om = oracle.OracleModel(spec, tau=tau)
    r = oracle.run_traced(om, 5, 0, 200, spec.t_inner, 0, 200, capacity=200_000)
    ev = r.events
    assert r.n_events <= 200_000
    ln = ev["kind"] == 2
    assert ln.sum() > 100
    line = ev["line"][ln].astype(int)
    emit = ev["emit"][ln].astype(int)
    np.testing.assert_allclose(ev["e_cmf_after"][ln], ev["e_cmf_before"][ln], rtol=4e-16)
    # absorbed at the Sobolev point of the absorbing line, emitted at the emitting line
    np.testing.assert_allclose(ev["nu_cmf_before"][ln], spec.nu[line], rtol=1e-13)
    np.testing.assert_allclose(ev["nu_cmf_after"][ln], spec.nu[emit], rtol=4e-16)
    # some emissions come from another level of the ion than the activated one
    row = lambda l: spec.ion[l] * spec.n_levels + spec.upper[l]
    assert np.any(row(line) != row(emit))
