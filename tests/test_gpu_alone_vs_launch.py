"""A packet's history does not depend on where in a launch it runs.

Draws are keyed by (seed, iteration, packet), and the binary64 kernel has two
ways to obtain them: the lane's own Philox stream, or -- once a warp is down
to its last live packet -- a buffer that the warp's idle lanes fill ahead.  A
packet run alone (mc_run_iteration_range with one packet: its warp is in that
state from its first segment) must therefore reproduce, bit for bit, the
status, final frequency, energy and counters it has in a full launch (where it
mostly shares its warp).  The twelve longest walks of a 2e4-packet downbranch
iteration are checked, in binary64 and in mixed precision, with downbranch
and with macro-atom line interactions.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("precision,line_mode", [(0, 1), (1, 1), (0, 2), (1, 2)])
def test_packets_alone_equal_their_full_launch_records(mc, precision, line_mode):
    make = synth.downbranch_model if line_mode == 1 else synth.macroatom_model
    spec = make(n_lines=40000, n_shells=16, n_packets=20000, seed=4242)
    N = spec.n_packets
    m = mc.Model(spec, precision=precision, record_packets=True)
    m.set_plasma()
    m.run_iteration(5469, 0, N, spec.t_inner)
    st, nu, e, cnt = m.packets(0, N)
    longest = np.argsort(cnt[:, 0])[-12:]
    assert cnt[longest, 0].min() > 50  # long enough to run many segments alone
    for k in longest:
        m.run_iteration_range(5469, 0, int(k), 1, N, spec.t_inner)
        s1, nu1, e1, c1 = m.packets(0, 1)
        assert s1[0] == st[k], k
        assert nu1[0] == nu[k] and e1[0] == e[k], k
        assert np.array_equal(c1[0], cnt[k]), k
    m.close()
