"""Batched launches: every model's iteration inside a batch equals the same
model's iteration run alone.

Four mixed-precision models of uneven shell, line and packet counts run 3
iterations (Sobolev depths, transport, T_R/W update) as one batch -- the
second and third iterations replay the captured CUDA graph -- and the same
models run alone.  Per packet the fate, final frequency and energy and the
counters must be identical (the batched kernel performs the same arithmetic on
the same draws).  J, nu_bar and J_blue are summed in fixed point, so they and
the updated T_R, W are identical too; the spectrum is a binary64 atomic sum
and agrees to 1e-9 (summation order).
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


def _specs():
    out = []
    for k, (S, L, N) in enumerate([(12, 3000, 1500), (20, 20000, 6000), (31, 8000, 300), (16, 12000, 4000)]):
        out.append(synth.downbranch_model(n_lines=L, n_shells=S, n_packets=N, seed=1401 + k,
                                          v_in_kms=9000.0 + 500 * k, v_out_kms=21000.0 - 700 * k,
                                          t_exp_days=10.0 + 2 * k, t_inner=9000.0 + 700 * k))
    return out


def _close(a, b, rtol):
    scale = np.maximum(np.abs(b), 1e-300)
    assert np.all(np.abs(a - b) <= rtol * scale + 1e-300), float(np.max(np.abs(a - b) / scale))


def test_batch_equals_solo(mc):
    specs = _specs()
    seeds = [100 + k for k in range(len(specs))]
    n = [s.n_packets for s in specs]
    t_in = [s.t_inner for s in specs]
    solo = []
    for spec, seed in zip(specs, seeds):
        m = mc.Model(spec, precision=mc.MC_PRECISION_MIXED, record_packets=True)
        m.set_plasma()
        per_it = []
        for it in range(3):
            m.run_iteration(seed, it, spec.n_packets, spec.t_inner)
            pk = m.packets(0, spec.n_packets)
            j, nb, jb, _ = m.estimators(j_blue=True)
            sp, st, _ = m.spectrum()
            t, w = m.update_radiation_field()
            per_it.append((pk, j, nb, jb, sp, st, t, w))
        solo.append(per_it)
        m.close()
    models = [mc.Model(spec, precision=mc.MC_PRECISION_MIXED, record_packets=True) for spec in specs]
    for m in models:
        m.set_plasma()
    b = mc.Batch(models)
    for it in range(3):
        b.run_iteration(seeds, it, n, t_in, update=True)  # iteration it for every model
        b.synchronize()
        for k, m in enumerate(models):
            pk_s, j_s, nb_s, jb_s, sp_s, st_s, t_s, w_s = solo[k][it]
            st_b, nu_b, e_b, cnt_b = m.packets(0, n[k])
            assert np.array_equal(st_b, pk_s[0]), (k, it)
            assert np.array_equal(nu_b, pk_s[1]) and np.array_equal(e_b, pk_s[2]), (k, it)
            assert np.array_equal(cnt_b, pk_s[3]), (k, it)
            j, nb, jb, _ = m.estimators(j_blue=True)
            assert np.array_equal(j, j_s) and np.array_equal(nb, nb_s), (k, it)
            assert np.array_equal(jb, jb_s), (k, it)
            sp, st, _ = m.spectrum()
            _close(sp, sp_s, 1e-9)
            assert st == st_s
            t, w, _ = m.plasma()
            assert np.array_equal(t, t_s) and np.array_equal(w, w_s), (k, it)
    assert b.transport_ms() > 0
    queue_ms, tail_ms = b.phases()  # global-timer phases of the same launch
    assert queue_ms > 0 and tail_ms >= 0
    assert queue_ms + tail_ms <= 1.05 * b.transport_ms() + 0.05
    b.close()
    for m in models:
        m.close()


def test_batch_rejects_fp64_models(mc):
    spec = synth.downbranch_model(n_lines=2000, n_packets=100)
    m = mc.Model(spec)
    with pytest.raises(mc.MCError) as ei:
        mc.Batch([m])
    assert ei.value.code == mc.MC_ERR_UNSUPPORTED
    m.close()


def test_launch_shape_and_autotune_leave_results_unchanged(mc):
    """Block size, resident blocks per SM and queue order change only which
    thread carries a packet and when; J, nu_bar, T_R, W stay bit-identical and
    the packets' fates and frequencies identical.  The autotuner's trials
    (transport only) leave the models' state as it was, and so does running
    the iteration as plain launches instead of a graph replay."""
    specs = _specs()
    seeds = [7 + k for k in range(len(specs))]
    n = [s.n_packets for s in specs]
    t_in = [s.t_inner for s in specs]
    shapes = [None, dict(block=64, blocks_per_sm=1, order=mc.MC_ORDER_GIVEN),
              dict(block=256, blocks_per_sm=0, order=mc.MC_ORDER_WORK), "autotune",
              "direct", "graph_then_direct"]
    results = []
    for shape in shapes:
        models = [mc.Model(s, precision=mc.MC_PRECISION_MIXED, record_packets=True) for s in specs]
        for m in models:
            m.set_plasma()
        b = mc.Batch(models)
        if shape == "autotune":
            best, ms, trials = b.autotune(seeds, 0, n, t_in)
            assert best["block"] in (64, 128, 256) and best["blocks_per_sm"] >= 1 and ms > 0 and trials >= 4
            assert b.launch() == best
        elif shape == "direct":
            b.capture_graph(False)  # plain launches every iteration
        elif shape is not None and shape != "graph_then_direct":
            b.set_launch(**shape)
            got = b.launch()
            assert got["block"] == shape["block"] and got["order"] == shape["order"]
        out = []
        for it in range(2):
            if shape == "graph_then_direct" and it == 1:
                b.capture_graph(False)
            b.run_iteration(seeds, it, n, t_in, update=True)
            b.synchronize()
            per = []
            for k, m in enumerate(models):
                j, nb, _, _ = m.estimators()
                t, w, _ = m.plasma()
                st, nu, e, _ = m.packets(0, n[k])
                per.append((j, nb, t, w, st, nu, e))
            out.append(per)
        b.close()
        for m in models:
            m.close()
        results.append(out)
    for r in results[1:]:
        for it in range(2):
            for k in range(len(specs)):
                for a, c in zip(r[it][k], results[0][it][k]):
                    assert np.array_equal(a, c), (it, k)


def test_set_launch_rejects_unknown_shapes(mc):
    spec = synth.downbranch_model(n_lines=2000, n_packets=100)
    m = mc.Model(spec, precision=mc.MC_PRECISION_MIXED)
    m.set_plasma()
    b = mc.Batch([m])
    with pytest.raises(mc.MCError):
        b.set_launch(block=96)
    with pytest.raises(mc.MCError):
        b.set_launch(order=9)
    b.set_launch(block=256, blocks_per_sm=1000)  # clamped to what fits
    assert 1 <= b.launch()["blocks_per_sm"] <= 8
    assert mc.load().mc_batch_capture_graph(b.h, 2) == mc.MC_ERR_INVALID_ARG
    b.close()
    m.close()
