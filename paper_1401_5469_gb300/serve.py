"""Continuous-batching service for spectral-fit model evaluations.

Each request is one ejecta model to be iterated K times (Sect. 2.8: Sobolev
depths from T_R and W, Monte Carlo transport, T_R/W update).  The service
keeps every admitted model resident on the GPU (plasma state, line data and
estimators stay in device memory across its iterations) and advances all
resident models together, one iteration each per tick.  Requests that arrive
while others are on the GPU are admitted first come, first served at the next
tick while the HBM budget (and the optional per-tick packet budget) allows, so
their iterations overlap on the device with the models already running; a
model leaves as soon as its last iteration is done, or when its request is
withdrawn between ticks (its memory and packet budget are released).

In mixed precision a tick is one batched transport launch for all resident
models (a captured CUDA graph).  In binary64 a tick launches every resident
model's own iteration on the model's own stream, so that one model's long
last random walks overlap the other models' work.

Without ticks (``n_groups`` > 1, driven by ``poll``): the resident models are
dealt into groups, each with its own CUDA stream and (in mixed precision) its
own batched launch.  A group's next iteration is enqueued as soon as its
previous one has ended, whatever the other groups are doing, so a model waits
only for the slowest walk of its own group, and one group's bulk runs in
another's tail.  Requests are admitted into a group when its iteration ends
(or while it is empty), and only that group's batch is rebuilt.

A request's results depend only on its own model, seed and iteration count:
packet draws are keyed by (seed, iteration, packet), single and batched
launches run the same kernel arithmetic, and in mixed precision J, nu_bar and
J_blue are summed in fixed point, so the same request gives bit-identical J,
nu_bar, J_blue, T_R and W alone and in any mix (only the spectrum sums, and in
binary64 the estimator sums, depend on summation order).
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque
from typing import Deque, Dict, List, Optional

import numpy as np

from . import mc


def model_footprint_bytes(spec, j_blue: Optional[bool] = None,
                          precision: int = mc.MC_PRECISION_MIXED) -> int:
    """Device bytes a model holds (Sobolev depths, J_blue, line list,
    branching tables, level data, spectrum)."""
    S, L = spec.n_shells, spec.n_lines
    jb = spec.j_blue if j_blue is None else j_blue
    nnz = L if spec.dbr_line is None else int(spec.dbr_line.shape[0])
    b = (4 if precision == mc.MC_PRECISION_MIXED else 8) * S * L  # Sobolev depths
    b += 8 * S * L if jb else 0        # J_blue sums
    b += L * (8 + 8 + 4 * 3 + 8 + 8)   # nu, f, ion/lower/upper, per-line constants, row info
    b += L * (4 * 3 + 8)               # staged line arrays used at set-up
    b += nnz * (4 + 4 + 8 + 32 + 32)   # branching table + guide records
    if spec.n_ions:
        b += spec.n_ions * spec.n_levels * (8 + 8 + 1) + S * spec.n_ions * (8 + 8 * spec.n_levels)
    if getattr(spec, "ma_jump_p", None) is not None:  # macro-atom level and jump tables
        b += spec.n_ions * spec.n_levels * 24 + int(np.asarray(spec.ma_jump_target).size) * 16
    if getattr(spec, "ionization_mode", 0):  # ionization tables and scratch
        E, J = int(spec.n_elements), int(spec.n_stages)
        b += 4 * E * J + 16 * E * (J - 1) + 8 * S * E + 8 * S * E * (J - 1)
    b += 8 * (spec.spec_bins + 2) + 64 * S + 16 * 1024
    return int(b)


@dataclasses.dataclass
class Request:
    rid: int
    spec: object
    n_iterations: int
    seed: int
    arrival: float = 0.0            # seconds on the service clock
    admitted: Optional[float] = None
    finished: Optional[float] = None
    done_iterations: int = 0
    t_rad: Optional[np.ndarray] = None
    w: Optional[np.ndarray] = None
    j_est: Optional[np.ndarray] = None
    nu_bar: Optional[np.ndarray] = None
    spectrum: Optional[np.ndarray] = None
    keep_history: bool = False
    history: List = dataclasses.field(default_factory=list)
    aborted: bool = False

    @property
    def latency(self) -> Optional[float]:
        return None if self.finished is None else self.finished - self.arrival


class Server:
    """Admits requests under an HBM budget and advances all resident models
    by one iteration per tick.

    hbm_budget_bytes: device bytes the resident models may hold together.
    max_tick_packets: admit no further request while the resident models'
        packets per iteration exceed this (None: no limit); bounds the tick
        length, so that finished models leave and waiting ones enter often.
    precision: mc.MC_PRECISION_MIXED (batched launch) or MC_PRECISION_FP64.
    """

    def __init__(self, hbm_budget_bytes: float = 150e9, j_blue: bool = True, stream=None,
                 precision: int = mc.MC_PRECISION_MIXED, max_tick_packets: Optional[int] = None,
                 n_groups: int = 1):
        self.budget = float(hbm_budget_bytes)
        self.n_groups = int(n_groups)
        self.groups: List[_Group] = []
        self.j_blue = j_blue
        self.stream = stream
        self.precision = precision
        self.max_tick_packets = max_tick_packets
        self.tick_packets = 0
        self.queue: Deque[Request] = deque()
        self.active: Dict[int, tuple] = {}   # rid -> (request, model, bytes)
        self.used = 0
        self.batch: Optional[mc.Batch] = None
        self.batch_ids: List[int] = []
        self.done: List[Request] = []
        self.aborted: List[Request] = []
        self.ticks = 0
        self.tick_ms: List[float] = []
        self.transport_ms: List[float] = []
        # host seconds spent creating models, building batches and launching,
        # and reading back results (without ticks)
        self.host_s = {"admit": 0.0, "launch": 0.0, "complete": 0.0}

    # -- admission
    def submit(self, req: Request):
        self.queue.append(req)

    def _admit(self, now: float):
        while self.queue:
            req = self.queue[0]
            need = model_footprint_bytes(req.spec, self.j_blue, self.precision)
            if self.active and self.used + need > self.budget:
                break
            if (self.active and self.max_tick_packets is not None
                    and self.tick_packets + req.spec.n_packets > self.max_tick_packets):
                break
            self.queue.popleft()
            m = mc.Model(req.spec, precision=self.precision, j_blue=self.j_blue,
                         stream=self.stream)
            m.set_plasma()
            req.admitted = now
            self.active[req.rid] = (req, m, need)
            self.used += need
            self.tick_packets += req.spec.n_packets

    def withdraw(self, rid: int) -> bool:
        """Abort request rid between ticks: drop it from the queue, or release
        its resident model (footprint and packet budget freed; the batch is
        rebuilt at the next tick).  Returns whether the request was found."""
        for r in self.queue:
            if r.rid == rid:
                self.queue.remove(r)
                r.aborted = True
                self.aborted.append(r)
                return True
        if rid not in self.active:
            return False
        for g in self.groups:  # without ticks: wait for the request's group to end its iteration
            if rid in g.ids:
                if g.event is not None:
                    g.event.synchronize()
                    self._complete_group(g, time.perf_counter())
                    if rid not in self.active:  # it finished with that iteration
                        return True
                if g.batch is not None:
                    g.batch.close()
                    g.batch, g.batch_ids = None, []
                g.ids.remove(rid)
                g.packets -= self.active[rid][0].spec.n_packets
        if self.batch is not None:
            self.batch.close()  # the batch goes before its models
            self.batch = None
            self.batch_ids = []
        req, m, need = self.active.pop(rid)
        m.close()
        self.used -= need
        self.tick_packets -= req.spec.n_packets
        req.aborted = True
        self.aborted.append(req)
        return True

    def _retire(self, rid: int, now: float):
        req, m, need = self.active.pop(rid)
        req.finished = now
        m.close()
        self.used -= need
        self.tick_packets -= req.spec.n_packets
        self.done.append(req)

    # -- one tick: every resident model advances by one iteration
    def step(self, now: float) -> int:
        self._admit(now)
        if not self.active:
            return 0
        ids = sorted(self.active)
        reqs = [self.active[r][0] for r in ids]
        if self.precision == mc.MC_PRECISION_MIXED:
            if ids != self.batch_ids:
                if self.batch is not None:
                    self.batch.close()
                self.batch = mc.Batch([self.active[r][1] for r in ids])
                self.batch_ids = ids
            t0 = time.perf_counter()
            # each model runs its own next iteration (draws keyed by its seed and index)
            self.batch.run_iteration([r.seed for r in reqs], [r.done_iterations for r in reqs],
                                     [r.spec.n_packets for r in reqs], [r.spec.t_inner for r in reqs],
                                     update=True)
            self.batch.synchronize()
            self.tick_ms.append(1e3 * (time.perf_counter() - t0))
            self.transport_ms.append(self.batch.transport_ms())
        else:
            t0 = time.perf_counter()
            models = [self.active[r][1] for r in ids]
            for r, m in zip(reqs, models):  # asynchronous, one stream per model
                m.run_iteration(r.seed, r.done_iterations, r.spec.n_packets, r.spec.t_inner)
                mc.mc_update_radiation_field(m.h, None, None)
            for m in models:
                m.synchronize()
            self.tick_ms.append(1e3 * (time.perf_counter() - t0))
        self.ticks += 1
        finished = []
        for r in reqs:
            m = self.active[r.rid][1]
            r.done_iterations += 1
            if r.keep_history:
                j, nb, _, _ = m.estimators()
                r.history.append((j, nb) + _radiation_field(m))
            if r.done_iterations >= r.n_iterations:
                r.j_est, r.nu_bar, _, _ = m.estimators()
                r.spectrum = m.spectrum()[0]
                r.t_rad, r.w = _radiation_field(m)
                finished.append(r.rid)
        end = now + (time.perf_counter() - t0)
        if finished and self.batch is not None:
            self.batch.close()  # the batch goes before its models
            self.batch = None
            self.batch_ids = []
        for rid in finished:
            self._retire(rid, end)
        return len(reqs)

    # -- without ticks: groups of models advancing on their own streams
    def poll(self, now: float) -> int:
        """Advance every group whose last iteration has ended: count the
        iteration for its models, retire the finished ones, admit waiting
        requests into it and enqueue its next iteration.  Never waits for the
        device.  Returns the number of model iterations completed."""
        if not self.groups:
            self.groups = [_Group(_new_stream()) for _ in range(max(1, self.n_groups))]
        completed = 0
        for g in self.groups:
            if g.event is not None:
                if not g.event.query():
                    continue
                g.event = None
                t0 = time.perf_counter()
                completed += self._complete_group(g, now)
                self.host_s["complete"] += time.perf_counter() - t0
            t0 = time.perf_counter()
            self._admit_group(g, now)
            t1 = time.perf_counter()
            if g.ids:
                self._launch_group(g)
            self.host_s["admit"] += t1 - t0
            self.host_s["launch"] += time.perf_counter() - t1
        return completed

    def _complete_group(self, g, now: float) -> int:
        if g.batch is not None:
            g.transport_ms.append(g.batch.transport_ms())
        self.tick_ms.append(1e3 * (time.perf_counter() - g.t_launch))
        self.ticks += 1
        finished = []
        for rid in g.ids:
            r, m, _ = self.active[rid]
            r.done_iterations += 1
            if r.keep_history:
                j, nb, _, _ = m.estimators()
                r.history.append((j, nb) + _radiation_field(m))
            if r.done_iterations >= r.n_iterations:
                r.j_est, r.nu_bar, _, _ = m.estimators()
                r.spectrum = m.spectrum()[0]
                r.t_rad, r.w = _radiation_field(m)
                finished.append(rid)
        if finished and g.batch is not None:
            g.batch.close()  # the batch goes before its models
            g.batch, g.batch_ids = None, []
        for rid in finished:
            g.ids.remove(rid)
            g.packets -= self.active[rid][0].spec.n_packets
            self._retire(rid, now)
        return len(g.ids) + len(finished)

    def _admit_group(self, g, now: float):
        cap = None if self.max_tick_packets is None else self.max_tick_packets / len(self.groups)
        while self.queue:
            req = self.queue[0]
            need = model_footprint_bytes(req.spec, self.j_blue, self.precision)
            if self.active and self.used + need > self.budget:
                break
            if g.ids and cap is not None and g.packets + req.spec.n_packets > cap:
                break
            self.queue.popleft()
            m = mc.Model(req.spec, precision=self.precision, j_blue=self.j_blue,
                         stream=g.stream_handle())
            m.set_plasma()
            req.admitted = now
            self.active[req.rid] = (req, m, need)
            self.used += need
            self.tick_packets += req.spec.n_packets
            g.ids.append(req.rid)
            g.packets += req.spec.n_packets

    def _launch_group(self, g):
        reqs = [self.active[r][0] for r in g.ids]
        models = [self.active[r][1] for r in g.ids]
        g.t_launch = time.perf_counter()
        if self.precision == mc.MC_PRECISION_MIXED:
            if g.ids != g.batch_ids:
                if g.batch is not None:
                    g.batch.close()
                g.batch = mc.Batch(models)
                g.batch_ids = list(g.ids)
            g.batch.run_iteration([r.seed for r in reqs], [r.done_iterations for r in reqs],
                                  [r.spec.n_packets for r in reqs], [r.spec.t_inner for r in reqs],
                                  update=True)
        else:
            for r, m in zip(reqs, models):  # in order on the group's stream
                m.run_iteration(r.seed, r.done_iterations, r.spec.n_packets, r.spec.t_inner)
                mc.mc_update_radiation_field(m.h, None, None)
        g.event = _new_event()
        g.event.record(g.stream)

    def close(self):
        if self.batch is not None:
            self.batch.close()
            self.batch = None
        for g in self.groups:
            if g.event is not None:
                g.event.synchronize()
            if g.batch is not None:
                g.batch.close()
                g.batch = None
            g.ids = []
        for rid in list(self.active):
            self._retire(rid, time.perf_counter())


def _new_stream():
    import torch
    return torch.cuda.Stream()


def _new_event():
    import torch
    return torch.cuda.Event()


class _Group:
    """A group of resident models sharing one CUDA stream and one batch."""

    def __init__(self, stream):
        self.stream = stream
        self.ids: List[int] = []
        self.batch: Optional[mc.Batch] = None
        self.batch_ids: List[int] = []
        self.event = None
        self.t_launch = 0.0
        self.packets = 0
        self.transport_ms: List[float] = []

    def stream_handle(self):
        import ctypes
        return ctypes.c_void_p(getattr(self.stream, "cuda_stream", 0))


def _radiation_field(m):
    t, w = np.zeros(m.S), np.zeros(m.S)
    mc.mc_read_plasma(m.h, t, w, None)
    return t, w


def percentiles(values, qs=(50, 95, 99)):
    v = np.asarray([x for x in values if x is not None], dtype=float)
    if v.size == 0:
        return {f"p{q}": None for q in qs}
    return {f"p{q}": float(np.percentile(v, q)) for q in qs}
