"""Host logic of the continuous-batching service, on the CPU.

The GPU models and batches are replaced by stand-ins that record what the
service asks of them, so admission and retirement can be checked without a
device: requests are admitted first come, first served while the HBM budget
and the per-tick packet budget allow (the head of the queue is never skipped
for a smaller request behind it); a request larger than the whole budget is
still admitted when nothing else is resident; each tick advances every
resident model by exactly one iteration, with its own seed and iteration
index; a model leaves after its last iteration, its footprint is released
and the batch is rebuilt for the models that remain.
"""
import numpy as np
import pytest

from paper_1401_5469_gb300 import serve, synth


class _FakeModel:
    live = 0

    def __init__(self, spec, precision=None, j_blue=None, stream=None):
        self.spec, self.S, self.closed = spec, spec.n_shells, False
        self.iterations = []
        _FakeModel.live += 1

    def set_plasma(self, *a, **k):
        pass

    def estimators(self, j_blue=False):
        return np.zeros(self.S), np.zeros(self.S), None, np.ones(self.S)

    def spectrum(self):
        return np.zeros(self.spec.spec_bins + 2), {}, 0

    def close(self):
        assert not self.closed
        self.closed = True
        _FakeModel.live -= 1


class _FakeBatch:
    created = []

    def __init__(self, models):
        self.models, self.closed = list(models), False
        _FakeBatch.created.append(self)

    def run_iteration(self, seeds, iterations, n_packets, t_inner, update=True):
        assert not self.closed and update
        for m, s, it, n in zip(self.models, seeds, iterations, n_packets):
            assert not m.closed and n == m.spec.n_packets
            m.iterations.append((s, it))

    def synchronize(self):
        pass

    def transport_ms(self):
        return 1.0

    def close(self):
        self.closed = True


@pytest.fixture
def fake(monkeypatch):
    _FakeModel.live = 0
    _FakeBatch.created = []
    monkeypatch.setattr(serve.mc, "Model", _FakeModel)
    monkeypatch.setattr(serve.mc, "Batch", _FakeBatch)
    monkeypatch.setattr(serve, "_radiation_field", lambda m: (np.zeros(m.S), np.zeros(m.S)))
    return serve


def _spec(n_lines, n_packets):
    return synth.scatter_model(n_lines=n_lines, n_shells=4, n_packets=n_packets)


def test_fifo_admission_under_the_hbm_budget(fake):
    small, big = _spec(200, 100), _spec(4000, 100)
    fs = serve.model_footprint_bytes(small, True)
    fb = serve.model_footprint_bytes(big, True)
    srv = serve.Server(hbm_budget_bytes=fb + fs, j_blue=True)
    reqs = [serve.Request(rid=0, spec=big, n_iterations=2, seed=1),
            serve.Request(rid=1, spec=big, n_iterations=1, seed=2),   # does not fit beside rid 0
            serve.Request(rid=2, spec=small, n_iterations=1, seed=3)]  # would fit, must wait its turn
    for r in reqs:
        srv.submit(r)
    assert srv.step(0.0) == 1 and list(srv.active) == [0]
    assert srv.used == fb and srv.used <= srv.budget
    assert srv.step(1.0) == 1            # rid 0 ends; rids 1, 2 still queued (FIFO head blocked)
    assert [r.rid for r in srv.done] == [0] and srv.used == 0
    assert srv.step(2.0) == 2            # both fit now: fb + fs <= budget
    assert sorted(r.rid for r in srv.done) == [0, 1, 2] and not srv.active and srv.used == 0
    assert _FakeModel.live == 0


def test_each_tick_advances_every_model_once_with_its_own_draws(fake):
    specs = [_spec(300, 50 + k) for k in range(3)]
    srv = serve.Server(hbm_budget_bytes=1e12)
    reqs = [serve.Request(rid=k, spec=s, n_iterations=k + 1, seed=100 + k) for k, s in enumerate(specs)]
    for r in reqs:
        srv.submit(r)
    models = {}
    while srv.queue or srv.active:
        srv.step(float(srv.ticks))
        for rid, (req, m, _) in srv.active.items():
            models[rid] = m
    # every model ran iterations 0 .. n-1 with its own seed, one per tick
    assert srv.ticks == 3
    for k, r in enumerate(reqs):
        assert r.done_iterations == r.n_iterations and r.finished is not None
    assert _FakeModel.live == 0
    # the batch was rebuilt whenever the resident set changed, and closed
    assert len(_FakeBatch.created) == 3 and all(b.closed for b in _FakeBatch.created)
    seen = {}
    for b in _FakeBatch.created:
        for m in b.models:
            seen.setdefault(id(m), m)
    runs = sorted((m.spec.n_packets, m.iterations) for m in seen.values())
    assert runs == [(50, [(100, 0)]), (51, [(101, 0), (101, 1)]), (52, [(102, 0), (102, 1), (102, 2)])]


def test_tick_packet_budget_and_oversized_request(fake):
    a, b = _spec(200, 600), _spec(200, 600)
    huge = _spec(8000, 10)
    srv = serve.Server(hbm_budget_bytes=serve.model_footprint_bytes(a, True) * 3, max_tick_packets=1000)
    for k, s in enumerate((a, b)):
        srv.submit(serve.Request(rid=k, spec=s, n_iterations=1, seed=k))
    srv.step(0.0)
    # the second request would push the tick past 1000 packets: it waits
    assert [r.rid for r in srv.done] == [0] and list(srv.queue)[0].rid == 1
    srv.step(1.0)
    assert [r.rid for r in srv.done] == [0, 1]
    # a request larger than the whole budget runs alone rather than never
    assert serve.model_footprint_bytes(huge, True) > srv.budget
    srv.submit(serve.Request(rid=9, spec=huge, n_iterations=1, seed=9))
    assert srv.step(2.0) == 1 and srv.done[-1].rid == 9
    srv.close()
    assert _FakeModel.live == 0


def test_percentiles():
    p = serve.percentiles([1.0, 2.0, 3.0, 4.0, None])
    assert p["p50"] == pytest.approx(2.5) and p["p99"] == pytest.approx(3.97)
    assert serve.percentiles([None])["p50"] is None


def test_iterate_applies_luminosity_matching_every_third_iteration(monkeypatch):
    """mc.Model.iterate's host logic with the device calls stubbed: T_inner
    changes only after iterations 3, 6, ... by (L_req / L_emitted)^(1/4)
    (mc_t_inner_update from the C library, no GPU needed), each iteration
    runs with the T_inner then current, and the radiation field is updated
    after every iteration."""
    import oracle
    from paper_1401_5469_gb300 import mc
    calls = []
    monkeypatch.setattr(mc, "mc_update_radiation_field", lambda h, t, w: calls.append("update"))

    class _M(mc.Model):
        def __init__(self):
            self.h = None
            self.lum = iter([2.0, 3.0, 5.0, 7.0, 11.0, 13.0, 17.0])

        def run_iteration(self, seed, iteration, n_packets, t_inner):
            calls.append(("run", iteration, t_inner))

        def emitted_luminosity(self):
            return next(self.lum)

    m = _M()
    used, t_next = m.iterate(7, 7, 100, 1.0e4, l_requested=4.0)
    t3 = oracle.t_inner_update(1.0e4, 4.0, 2.0)      # after iteration 2: L_emitted of that iteration
    t6 = oracle.t_inner_update(t3, 4.0, 3.0)         # after iteration 5
    assert used == [1.0e4] * 3 + [t3] * 3 + [t6]
    assert t_next == t6
    assert calls.count("update") == 7
    assert [c[1] for c in calls if c != "update"] == list(range(7))


def test_withdrawn_requests_release_their_resources(fake):
    specs = [_spec(300, 100 + k) for k in range(4)]
    srv = serve.Server(hbm_budget_bytes=2.5 * serve.model_footprint_bytes(specs[0], True))
    for k, s in enumerate(specs):
        srv.submit(serve.Request(rid=k, spec=s, n_iterations=3, seed=k))
    srv.step(0.0)
    assert sorted(srv.active) == [0, 1] and [r.rid for r in srv.queue] == [2, 3]
    used_before = srv.used
    assert srv.withdraw(1)                 # resident: model released, budget freed
    assert srv.withdraw(3)                 # queued: simply dropped
    assert not srv.withdraw(42)
    assert srv.used < used_before and 1 not in srv.active
    assert [r.rid for r in srv.aborted] == [1, 3] and all(r.aborted for r in srv.aborted)
    while srv.queue or srv.active:
        srv.step(float(srv.ticks))
    assert sorted(r.rid for r in srv.done) == [0, 2]
    assert all(r.done_iterations == 3 for r in srv.done)
    assert srv.used == 0 and srv.tick_packets == 0 and _FakeModel.live == 0


class _FakeEvent:
    """Completes after a set number of polls of its group (the device time)."""
    duration = {}

    def __init__(self):
        self.left = None

    def record(self, stream):
        self.stream = stream
        self.left = _FakeEvent.duration.get(stream.name, 1)

    def query(self):
        self.left -= 1
        return self.left <= 0

    def synchronize(self):
        self.left = 0


class _FakeStream:
    count = 0

    def __init__(self):
        self.name = _FakeStream.count
        _FakeStream.count += 1


@pytest.fixture
def grouped(fake, monkeypatch):
    _FakeStream.count = 0
    _FakeEvent.duration = {}
    monkeypatch.setattr(serve, "_new_stream", _FakeStream)
    monkeypatch.setattr(serve, "_new_event", _FakeEvent)
    return serve


def test_groups_advance_independently(grouped):
    """Without ticks: a group whose iterations take long (stream 0, 5 polls
    each) does not hold back the other group (stream 1, 1 poll each); every
    model still runs iterations 0 .. n-1 with its own seed, exactly once."""
    _FakeEvent.duration = {0: 5, 1: 1}
    specs = [_spec(300, 100 + k) for k in range(4)]
    srv = serve.Server(hbm_budget_bytes=1e12, n_groups=2, max_tick_packets=250)
    reqs = [serve.Request(rid=k, spec=s, n_iterations=3, seed=10 + k) for k, s in enumerate(specs)]
    for r in reqs:
        srv.submit(r)
    polls = 0
    finished_at = {}
    while (srv.queue or srv.active) and polls < 200:
        srv.poll(float(polls))
        for r in srv.done:
            finished_at.setdefault(r.rid, polls)
        polls += 1
    srv.close()
    assert sorted(r.rid for r in srv.done) == [0, 1, 2, 3]
    # the packet cap (125 per group) puts one model in each group at a time:
    # rids 0 and 1 start together; rid 1 (fast group) finishes and rids 2, 3
    # follow it in the fast group while rid 0 is still in the slow one
    assert finished_at[1] < finished_at[0] and finished_at[2] < finished_at[0]
    seen = {}
    for b in _FakeBatch.created:
        for m in b.models:
            seen.setdefault(id(m), m)
    runs = sorted((m.spec.n_packets, m.iterations) for m in seen.values())
    assert runs == [(100 + k, [(10 + k, 0), (10 + k, 1), (10 + k, 2)]) for k in range(4)]
    assert _FakeModel.live == 0 and srv.used == 0


def test_grouped_withdraw_waits_for_the_group(grouped):
    _FakeEvent.duration = {0: 3, 1: 3}
    specs = [_spec(300, 100 + k) for k in range(2)]
    srv = serve.Server(hbm_budget_bytes=1e12, n_groups=2, max_tick_packets=250)
    for k, s in enumerate(specs):
        srv.submit(serve.Request(rid=k, spec=s, n_iterations=5, seed=k))
    srv.poll(0.0)
    assert sorted(srv.active) == [0, 1]
    assert srv.withdraw(0)      # its group's iteration in flight: it ends first, then the model goes
    assert 0 not in srv.active and srv.aborted[-1].rid == 0
    while srv.active:
        srv.poll(1.0)
    assert [r.rid for r in srv.done] == [1] and _FakeModel.live == 0
