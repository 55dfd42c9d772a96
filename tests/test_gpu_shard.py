"""Device estimator views and packet-range sharding on one GPU.

* mc_device_estimators returns the buffers the update kernel reads: doubling
  J and nu_bar in place leaves T_R unchanged and doubles W (Eqs. 15-16).
* Two disjoint packet ranges of one iteration, run by two models (as two
  ranks would, one after the other), sum to the whole iteration run at once.
* run_sharded_iteration over a one-process NCCL group equals run_iteration.
"""
import os
import socket

import numpy as np
import pytest

from paper_1401_5469_gb300 import shard, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1401_5469_gb300 import mc as mcmod
    mcmod.load()
    return mcmod


def _spec():
    return synth.downbranch_model(n_lines=20000, n_shells=12, n_packets=20000, seed=31)


@pytest.mark.parametrize("precision", [0, 1])
def test_views_are_the_update_inputs(mc, precision):
    spec = _spec()
    m = mc.Model(spec, precision=precision)
    m.set_plasma()
    m.run_iteration(5469, 0, spec.n_packets, spec.t_inner)
    j, nb, _, _ = m.estimators()
    v = m.device_estimators()
    m.synchronize()
    np.testing.assert_array_equal(v["j_est"].cpu().numpy(), j)
    np.testing.assert_array_equal(v["nu_bar"].cpu().numpy(), nb)
    sp, _, _ = m.spectrum()
    np.testing.assert_array_equal(v["spectrum"].cpu().numpy(), sp)
    # reference update from the untouched sums, on a twin model
    m2 = mc.Model(spec, precision=precision)
    m2.set_plasma()
    m2.run_iteration(5469, 0, spec.n_packets, spec.t_inner)
    t_ref, w_ref = m2.update_radiation_field()
    import torch
    v["j_est"].mul_(2.0)
    v["nu_bar"].mul_(2.0)
    torch.cuda.synchronize()
    t, w = m.update_radiation_field()
    # (the twin's binary64 sums differ from these by atomic summation order)
    np.testing.assert_allclose(t, t_ref, rtol=1e-12)
    np.testing.assert_allclose(w, 2.0 * w_ref, rtol=1e-12)
    m.close()
    m2.close()


def test_two_ranges_sum_to_the_whole_iteration(mc):
    spec = _spec()
    N = spec.n_packets
    whole = mc.Model(spec)
    whole.set_plasma()
    whole.run_iteration(5469, 0, N, spec.t_inner)
    j, nb, _, _ = whole.estimators()
    sp, _, _ = whole.spectrum()
    parts = []
    for r in range(2):
        first, count = shard.packet_range(r, 2, N)
        m = mc.Model(spec)
        m.set_plasma()
        m.run_iteration_range(5469, 0, first, count, N, spec.t_inner)
        jr, nbr, _, _ = m.estimators()
        spr, _, _ = m.spectrum()
        parts.append((jr, nbr, spr))
        m.close()
    np.testing.assert_allclose(parts[0][0] + parts[1][0], j, rtol=1e-12)
    np.testing.assert_allclose(parts[0][1] + parts[1][1], nb, rtol=1e-12)
    np.testing.assert_allclose(parts[0][2] + parts[1][2], sp, rtol=1e-12, atol=0.0)
    whole.close()


def test_sharded_iteration_over_one_process_group(mc):
    """Mixed precision sums J, nu_bar in fixed point, so the sharded run equals
    the plain run bit for bit; binary64 atomics leave summation-order noise."""
    import torch
    import torch.distributed as dist
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        spec = _spec()
        for precision in (1, 0):
            a = mc.Model(spec, precision=precision)
            a.set_plasma()
            b = mc.Model(spec, precision=precision)
            b.set_plasma()
            for it in range(2):
                t_s, w_s = shard.run_sharded_iteration(a, 5469, it, spec.n_packets, spec.t_inner)
                b.run_iteration(5469, it, spec.n_packets, spec.t_inner)
                t_b, w_b = b.update_radiation_field()
                if precision == 1:
                    np.testing.assert_array_equal(t_s, t_b)
                    np.testing.assert_array_equal(w_s, w_b)
                else:
                    np.testing.assert_allclose(t_s, t_b, rtol=1e-12)
                    np.testing.assert_allclose(w_s, w_b, rtol=1e-12)
            a.close()
            b.close()
    finally:
        dist.destroy_process_group()


def test_two_packet_ranges_sum_to_the_oracle_iteration(mc):
    """The full-size downbranch iteration (500,000 lines, 1e6 packets, J_blue)
    split into two packet ranges as two ranks would run them (one after the
    other on this GPU): the summed J, nu_bar, spectrum and every J_blue cell
    equal the oracle's whole iteration within 1e-9 relative, and each range's
    run statistics add up to the oracle's."""
    import oracle
    spec = synth.downbranch_model()
    n, S, L = spec.n_packets, spec.n_shells, spec.n_lines
    t_rad = np.full(S, 1.0e4)
    tau = oracle.plasma_tau(spec, t_rad, oracle.geometric_dilution(spec))
    sums = {"j": 0.0, "nb": 0.0, "jb": 0.0, "sp": 0.0}
    stats = {}
    for rank in range(2):
        first, count = shard.packet_range(rank, 2, n)
        m = mc.Model(spec)
        m.set_plasma(tau=tau)
        m.run_iteration_range(spec.seed, 0, first, count, n, spec.t_inner)
        j, nb, jb, _ = m.estimators(j_blue=True)
        sp, st, _ = m.spectrum()
        m.close()
        sums["j"] = sums["j"] + j
        sums["nb"] = sums["nb"] + nb
        sums["jb"] = sums["jb"] + jb.reshape(S, L)
        sums["sp"] = sums["sp"] + sp
        for k, v in st.items():
            stats[k] = stats.get(k, 0) + v
    r = oracle.run_iteration(oracle.OracleModel(spec, tau=tau), spec.seed, 0, n, spec.t_inner,
                             threads=os.cpu_count() or 1, record=False)
    for k in oracle.STAT_NAMES:
        assert stats[k] == r.stats[k], k
    for name, a, b in (("J", sums["j"], r.j_est), ("nu_bar", sums["nb"], r.nu_bar),
                       ("spectrum", sums["sp"], r.spectrum), ("J_blue", sums["jb"], r.j_blue)):
        zero = b == 0
        assert np.all(a[zero] == 0), name
        rel = np.abs(a[~zero] - b[~zero]) / np.abs(b[~zero])
        assert rel.max() <= 1e-9, (name, float(rel.max()))
