"""Continuous batching: each request's result is the same alone and in the mix.

Five requests with different models and iteration counts arrive over three
ticks; the HBM budget admits at most three models at a time, so later
requests wait and then join models already running (their iterations share
batched launches).  Every request's per-iteration J, nu_bar, T_R and W must
equal, bit for bit, the same model iterated alone with the same seed (J and
nu_bar are fixed-point sums, so the summation order does not show).
"""
import numpy as np
import pytest

from paper_1401_5469_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1401_5469_gb300 import mc, serve
    mc.load()
    return mc, serve


def test_requests_same_alone_and_in_the_mix(env):
    mc, serve = env
    sizes = [(14, 4000, 1500, 3), (20, 9000, 3000, 2), (10, 2500, 800, 4), (25, 6000, 2000, 2),
             (16, 3000, 1200, 3)]
    specs = [synth.downbranch_model(n_lines=L, n_shells=S, n_packets=N, seed=1500 + k,
                                    t_inner=9000.0 + 300 * k)
             for k, (S, L, N, _) in enumerate(sizes)]
    reqs = [serve.Request(rid=k, spec=specs[k], n_iterations=sizes[k][3], seed=77 + k, keep_history=True)
            for k in range(len(specs))]
    fp = [serve.model_footprint_bytes(s) for s in specs]
    budget = sum(sorted(fp)[-3:]) + 1  # at most three resident models
    server = serve.Server(hbm_budget_bytes=budget)
    arrivals = {0: [0, 1], 1: [2], 2: [3, 4]}
    tick = 0
    max_resident = 0
    while tick < 40 and len(server.done) < len(reqs):
        for k in arrivals.get(tick, []):
            server.submit(reqs[k])
        server.step(float(tick))
        max_resident = max(max_resident, len(server.active) + sum(1 for r in server.done if r.finished == tick))
        tick += 1
    server.close()
    assert len(server.done) == len(reqs)
    assert server.ticks >= max(r.n_iterations for r in reqs)
    for r in reqs:
        assert len(r.history) == r.n_iterations
        m = mc.Model(r.spec, precision=mc.MC_PRECISION_MIXED)
        m.set_plasma()
        for it in range(r.n_iterations):
            m.run_iteration(r.seed, it, r.spec.n_packets, r.spec.t_inner)
            j, nb, _, _ = m.estimators()
            t, w = m.update_radiation_field()
            j_s, nb_s, t_s, w_s = r.history[it]
            assert np.array_equal(j_s, j) and np.array_equal(nb_s, nb), (r.rid, it)
            assert np.array_equal(t_s, t) and np.array_equal(w_s, w), (r.rid, it)
        m.close()
    lat = serve.percentiles([r.latency for r in reqs])
    assert lat["p50"] is not None and lat["p99"] >= lat["p50"]


def test_grouped_service_same_alone_and_in_the_mix(env):
    """Without ticks: two groups of models on their own streams, each group's
    next iteration enqueued as soon as its last one ends; requests join a
    group when its iteration ends.  Every request's per-iteration J, nu_bar,
    T_R and W equal, bit for bit, the model iterated alone."""
    mc, serve = env
    sizes = [(14, 4000, 1500, 3), (20, 9000, 3000, 2), (10, 2500, 800, 4), (25, 6000, 2000, 2),
             (16, 3000, 1200, 3)]
    specs = [synth.downbranch_model(n_lines=L, n_shells=S, n_packets=N, seed=1600 + k,
                                    t_inner=9000.0 + 300 * k)
             for k, (S, L, N, _) in enumerate(sizes)]
    reqs = [serve.Request(rid=k, spec=specs[k], n_iterations=sizes[k][3], seed=91 + k, keep_history=True)
            for k in range(len(specs))]
    server = serve.Server(hbm_budget_bytes=1e12, n_groups=2, max_tick_packets=8000)
    import time
    polls, t_end = 0, time.perf_counter() + 120.0
    while time.perf_counter() < t_end and len(server.done) < len(reqs):
        if polls < len(reqs):
            server.submit(reqs[polls])
        if server.poll(float(polls)) == 0:
            time.sleep(0.001)
        polls += 1
    server.close()
    assert len(server.done) == len(reqs)
    for r in reqs:
        assert len(r.history) == r.n_iterations
        m = mc.Model(r.spec, precision=mc.MC_PRECISION_MIXED)
        m.set_plasma()
        for it in range(r.n_iterations):
            m.run_iteration(r.seed, it, r.spec.n_packets, r.spec.t_inner)
            j, nb, _, _ = m.estimators()
            t, w = m.update_radiation_field()
            j_s, nb_s, t_s, w_s = r.history[it]
            assert np.array_equal(j_s, j) and np.array_equal(nb_s, nb), (r.rid, it)
            assert np.array_equal(t_s, t) and np.array_equal(w_s, w), (r.rid, it)
        m.close()
