"""Packet-range sharding of one iteration across processes (CPU, gloo).

Two ranks each transport their contiguous share of the packets and sum the
estimators with an all-reduce (paper_1401_5469_gb300.shard).  Because every
packet's draws are keyed by its index, the summed J_est, nu_bar and spectrum
must equal the single-process iteration up to summation order, and both ranks
must reach the same T_R, W.  On CPU ranks the oracle stands in for the GPU
model (a test double with the same methods as mc.Model).
"""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1401_5469_gb300 import shard, synth


def test_packet_ranges_tile_the_iteration():
    for world in (1, 2, 3, 7):
        for n in (7, 8, 100, 1001):
            spans = [shard.packet_range(r, world, n) for r in range(world)]
            assert spans[0][0] == 0
            for (f0, c0), (f1, _) in zip(spans, spans[1:]):
                assert f0 + c0 == f1
            assert sum(c for _, c in spans) == n
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1
    with pytest.raises(ValueError):
        shard.packet_range(2, 2, 10)


def _spec():
    return synth.downbranch_model(n_lines=3000, n_shells=8, n_packets=3000, seed=77)


class OracleShardModel:
    """Test double of mc.Model for CPU ranks: the oracle transports the range."""

    def __init__(self, spec):
        import torch
        self.torch = torch
        self.spec = spec
        self.t_rad = np.full(spec.n_shells, 1.0e4)
        self.w = oracle.geometric_dilution(spec)
        self.om = oracle.OracleModel(spec, tau=oracle.plasma_tau(spec, self.t_rad, self.w))
        self.est = None

    def run_iteration_range(self, seed, iteration, first, count, n_total, t_inner):
        r = oracle.run_iteration(self.om, seed, iteration, n_total, t_inner, first=first, count=count,
                                 threads=1, record=False, j_blue=False)
        t = self.torch.from_numpy
        self.est = {"j_est": t(r.j_est.copy()), "nu_bar": t(r.nu_bar.copy()),
                    "spectrum": t(r.spectrum.copy()), "j_blue": None, "stream": None}

    def synchronize(self):
        return 0

    def device_estimators(self):
        return self.est

    def update_radiation_field(self):
        j, nb = self.est["j_est"].numpy(), self.est["nu_bar"].numpy()
        self.t_rad, self.w = oracle.update_radiation_field(self.spec, j, nb, self.t_rad, self.w)
        self.om.set_tau(oracle.plasma_tau(self.spec, self.t_rad, self.w))
        return self.t_rad, self.w


def _worker(rank, world, port, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        spec = _spec()
        m = OracleShardModel(spec)
        out = []
        for it in range(2):
            t, w = shard.run_sharded_iteration(m, 5469, it, spec.n_packets, spec.t_inner)
            out.append({k: m.est[k].numpy().copy() for k in ("j_est", "nu_bar", "spectrum")} |
                       {"t_rad": t.copy(), "w": w.copy()})
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_ranks_reproduce_the_single_process_iterations():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = oracle.run_loop(_spec(), 2, _spec().n_packets, 5469, threads=1)
    for it in range(2):
        for k in ("j_est", "nu_bar", "spectrum"):
            want = getattr(ref[it], k)
            for r in (0, 1):
                a = got[r][it][k]
                assert np.allclose(a, want, rtol=1e-12, atol=0.0), (it, k, r)
        np.testing.assert_array_equal(got[0][it]["t_rad"], got[1][it]["t_rad"])
        np.testing.assert_array_equal(got[0][it]["w"], got[1][it]["w"])
        assert np.allclose(got[0][it]["t_rad"], ref[it].t_rad_out, rtol=1e-11)
