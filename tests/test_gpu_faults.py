"""Host-side failure injection on a GPU machine (no device fault is provoked).

* a caller-supplied allocator that fails at the k-th request: model creation
  returns MC_ERR_OOM with a message, and every block it had obtained is
  handed back through the allocator's free;
* after a successful create, run and destroy, the allocator holds nothing;
* the serving loop's footprint estimate (its HBM admission budget) covers
  every byte a model obtains, and is not more than 25% above it;
* mc_cancel stops a running launch within milliseconds (its reads report
  MC_ERR_TIMEOUT naming the cancel), stops a launch started while the request
  stands, and once withdrawn the model runs normally again;
* the transport deadline: covered by tests/test_gpu_parity.py.
"""
import ctypes as C
import time

import numpy as np
import pytest

from paper_1401_5469_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1401_5469_gb300 import mc as mcmod
    mcmod.load()
    return torch, mcmod


def _descs(mc, spec, keep):
    f64 = lambda a: keep.append(np.ascontiguousarray(a, np.float64)) or keep[-1].ctypes.data
    i32 = lambda a: keep.append(np.ascontiguousarray(a, np.int32)) or keep[-1].ctypes.data
    g = mc.mc_geometry_desc(n_shells=spec.n_shells, v_inner=f64(spec.v_inner), v_outer=f64(spec.v_outer),
                            n_e=f64(spec.n_e), t_exp=spec.t_exp)
    l = mc.mc_line_desc(n_lines=spec.n_lines, nu=f64(spec.nu), f=f64(spec.f), ion=i32(spec.ion),
                        lower=i32(spec.lower), upper=i32(spec.upper))
    a = mc.atomic_desc(spec, keep)
    r = mc.mc_run_desc(line_mode=int(spec.line_mode), precision=0, j_blue=1, record_packets=1,
                       spec_bins=100, spec_nu_lo=1e14, spec_nu_hi=3e15, max_packets=spec.n_packets,
                       max_segments=0, delta_t=1.0)
    return g, l, a, r


class _Allocator:
    """Device blocks from torch; the k-th request fails."""

    def __init__(self, torch, mc, fail_at=None):
        self.live, self.calls, self.fail_at = {}, 0, fail_at

        def alloc(nbytes, ctx):
            self.calls += 1
            if self.calls == self.fail_at:
                return None
            t = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device="cuda")
            self.live[t.data_ptr()] = t
            return t.data_ptr()

        self.bytes = lambda: sum(t.numel() for t in self.live.values())

        def free(ptr, ctx):
            self.live.pop(ptr)

        self._a, self._f = mc.ALLOC_FN(alloc), mc.FREE_FN(free)
        self.c = mc.mc_allocator(alloc=self._a, free=self._f, ctx=None)


def test_allocation_failure_is_reported_and_released(env):
    torch, mc = env
    spec = synth.downbranch_model(n_lines=2000, n_shells=6, n_packets=200)
    keep = []
    g, l, a, r = _descs(mc, spec, keep)
    L = mc.load()
    total = _Allocator(torch, mc)
    h = C.c_void_p()
    assert L.mc_model_create(C.byref(g), C.byref(l), C.byref(a), C.byref(r), C.byref(total.c), None,
                             C.byref(h)) == 0
    L.mc_model_destroy(h)
    torch.cuda.synchronize()
    assert total.calls > 10 and not total.live
    for k in (1, 2, total.calls // 2, total.calls):
        al = _Allocator(torch, mc, fail_at=k)
        h = C.c_void_p()
        rc = L.mc_model_create(C.byref(g), C.byref(l), C.byref(a), C.byref(r), C.byref(al.c), None,
                               C.byref(h))
        torch.cuda.synchronize()
        assert rc == mc.MC_ERR_OOM, (k, rc)
        assert not h.value
        assert "allocation" in L.mc_last_error_message(None).decode()
        assert not al.live, (k, len(al.live))


def test_run_and_destroy_release_everything(env):
    torch, mc = env
    spec = synth.downbranch_model(n_lines=2000, n_shells=6, n_packets=200)
    keep = []
    g, l, a, r = _descs(mc, spec, keep)
    L = mc.load()
    al = _Allocator(torch, mc)
    h = C.c_void_p()
    assert L.mc_model_create(C.byref(g), C.byref(l), C.byref(a), C.byref(r), C.byref(al.c), None,
                             C.byref(h)) == 0
    assert L.mc_set_plasma(h, None, None, None) == 0
    assert L.mc_run_iteration(h, 5, 0, spec.n_packets, spec.t_inner) == 0
    assert L.mc_synchronize(h) == 0
    L.mc_model_destroy(h)
    torch.cuda.synchronize()
    assert al.calls > 10 and not al.live


def test_cancel_stops_running_and_later_launches(env):
    torch, mc = env
    spec = synth.downbranch_model(n_lines=100_000, n_packets=300_000)
    n = spec.n_packets
    m = mc.Model(spec)
    m.set_plasma()
    m.run_iteration(1, 0, n, spec.t_inner)
    m.synchronize()
    t0 = time.perf_counter()
    m.run_iteration(1, 1, n, spec.t_inner)
    m.synchronize()
    full = time.perf_counter() - t0
    m.run_iteration(1, 2, n, spec.t_inner)  # asynchronous
    time.sleep(0.2 * full)
    t0 = time.perf_counter()
    m.cancel()
    with pytest.raises(mc.MCError) as ei:
        m.estimators()
    stopped = time.perf_counter() - t0
    assert ei.value.code == mc.MC_ERR_TIMEOUT and "mc_cancel" in str(ei.value)
    assert stopped < 0.5 * full, (stopped, full)
    m.run_iteration(1, 3, n, spec.t_inner)  # starts while the request stands
    with pytest.raises(mc.MCError) as ei:
        m.spectrum()
    assert ei.value.code == mc.MC_ERR_TIMEOUT
    m.cancel(False)
    m.run_iteration(1, 4, 2000, spec.t_inner)
    m.estimators()
    _, stats, rc = m.spectrum()
    assert stats["escaped"] + stats["reabsorbed"] == 2000
    m.close()


@pytest.mark.parametrize("precision,j_blue,kind", [(1, True, "downbranch"), (1, False, "downbranch"),
                                                   (0, True, "downbranch"), (1, True, "macroatom")])
def test_footprint_estimate_covers_the_allocations(env, precision, j_blue, kind):
    torch, mc = env
    from paper_1401_5469_gb300 import serve
    make = synth.downbranch_model if kind == "downbranch" else synth.macroatom_model
    spec = make(n_lines=30000, n_shells=15, n_packets=5000, j_blue=j_blue)
    keep = []
    g, l, a, r = _descs(mc, spec, keep)
    r.precision, r.j_blue, r.record_packets = precision, int(j_blue), 0
    L = mc.load()
    al = _Allocator(torch, mc)
    h = C.c_void_p()
    assert L.mc_model_create(C.byref(g), C.byref(l), C.byref(a), C.byref(r), C.byref(al.c), None,
                             C.byref(h)) == 0
    assert L.mc_set_plasma(h, None, None, None) == 0
    assert L.mc_run_iteration(h, 5, 0, spec.n_packets, spec.t_inner) == 0
    assert L.mc_synchronize(h) == 0
    used = al.bytes()
    est = serve.model_footprint_bytes(spec, j_blue, precision)
    L.mc_model_destroy(h)
    torch.cuda.synchronize()
    assert used <= est <= 1.25 * used, (used, est)
