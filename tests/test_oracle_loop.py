"""Pins of the oracle's iteration cycle (Sect. 2.8).

The state carried from one iteration to the next is T_R and W per shell
(and T_inner, a host value): draws are keyed by (seed, iteration, packet),
depths and ionization are recomputed from T_R and W.  So a run stopped
after iteration k and resumed from its saved T_R, W at iteration k + 1
reproduces the uninterrupted run bit for bit -- a check that no other
state leaks between iterations (a draw counter not keyed by the iteration,
estimators not zeroed, depths or n_e kept from an earlier plasma state).
"""
import numpy as np
import pytest

import oracle
from paper_1401_5469_gb300 import synth

FIELDS = ("j_est", "nu_bar", "spectrum", "status", "nu", "energy", "counters", "t_rad_in", "w_in",
          "t_rad_out", "w_out")


@pytest.mark.parametrize("kind", ["downbranch", "nebular"])
def test_loop_resumes_bit_identically_from_saved_state(kind):
    if kind == "downbranch":
        spec = synth.downbranch_model(n_lines=3000, n_shells=6, n_packets=400, seed=5)
    else:
        spec = synth.nebular_model(mode=2, n_lines=3000, n_shells=6, n_packets=400, seed=6)
    n = spec.n_packets
    full = oracle.run_loop(spec, 4, n, 77, threads=2, record=True)
    head = oracle.run_loop(spec, 2, n, 77, threads=2, record=True)
    tail = oracle.run_loop(spec, 2, n, 77, threads=2, record=True, t_rad=head[-1].t_rad_out,
                           w=head[-1].w_out, first_iteration=2)
    for a, b in zip(full[:2], head):
        for k in FIELDS:
            np.testing.assert_array_equal(getattr(a, k), getattr(b, k), err_msg=k)
    for a, b in zip(full[2:], tail):
        for k in FIELDS:
            np.testing.assert_array_equal(getattr(a, k), getattr(b, k), err_msg=k)
    # the state does change between iterations (the check is not vacuous)
    assert np.any(full[2].t_rad_in != full[0].t_rad_in)
    assert not np.array_equal(full[2].status, full[3].status)
