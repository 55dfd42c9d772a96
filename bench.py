"""Benchmark of the GB300 Monte Carlo transport library.

Workload (default): the full-loop downbranch model -- 20 shells
(11000-20000 km/s, 13 d), 500,000 lines, 30 ions x 40 levels, J_blue
estimators, 1e6 packets per iteration, binary64.  One step is one Monte Carlo
iteration of Sect. 2.8: Sobolev depths recomputed from the current T_R, W
(plasma kernels), estimators zeroed, 1e6 packets transported, T_R and W
updated from the estimators.  The iteration index advances every step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --workload batched [--models M]

Prints one JSON line.  ``--impl reference`` times the CPU oracle (the plain
FP64 C implementation used by the tests) on all host cores, over the same
iteration loop (each step the whole 1e6-packet iteration, then the T_R/W
update; ``BENCH_REF_SAMPLE`` bounds the packets per step).  The default line also carries the mixed-precision loop, the
2000-line scatter model, and a ``batched`` object: the batched workload below
(256 models, two groups, mixed precision) with its own roofline, and the
per-model binary64 path on the first 8 of those models.

``--workload batched``: 256 ejecta models of uneven size (shells U{10..40},
lines U{5e4..5e5}, packets log-uniform in [1e4, 1e6], velocities, epoch and
T_inner drawn per model), 10 iterations each with the T_R/W update.  The
batched mixed-precision path (one persistent launch per iteration for all
models, a captured CUDA graph, autotuned launch shape) is timed against the
plain per-model binary64 path on the same models, seeds and packet counts;
the metric is models/s (models completed with all 10 iterations per second).

``--workload spectrum``: the spectrum iteration with virtual packets (N_v = 3)
on the same model -- transport time with and without them, and the noise per
spectral bin of both spectra over 8 seeds.

``--workload macroatom``: the same model with macro-atom line interactions
(synthetic internal jumps) against downbranch, per-iteration transport time.

``--workload serve [--precision mixed|fp64] [--rate R]``: continuous-batching
service.  Requests arrive as a Poisson process (R = 50 models/s by default)
for 70 s; each is one model of the batched workload's distribution with
U{5..20} iterations.  Resident models are admitted first come, first served
under a 150 GB HBM budget and a per-tick packet budget.  The first 10 s are
warm-up; models/s and the p50/p95/p99 latency (arrival to last iteration) are
taken over the requests that arrive in the remaining 60 s and finish by its
end, with the backlog left at the end reported beside them.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "packets/s"
UNIT = "packets/s"
WORKLOAD = "downbranch-20sh-500k-lines-1e6-packets"
L2_BYTES = 129 * 2**20

# DRAM traffic of one transport_fp64 launch of this workload (1e6 packets,
# iteration 0), from the one-pass ncu capture summarised in
# profiles/transport_fp64_downbranch_500k_traffic.md.  It stands for the
# kernel built from these sources only: with any other source hash the
# bench reports traffic as null.
TRAFFIC_CAPTURE = {
    "dram_bytes_per_launch": 926.16e6 + 159.46e6,
    "sources": ("paper_1401_5469_gb300/csrc/mc_transport.cu", "paper_1401_5469_gb300/csrc/mc_device.cuh",
                "paper_1401_5469_gb300/csrc/mc_internal.h"),
    "sha256": "309bc2792b36959d9057086d024a7347dd831c4869688afaae1a866dbc6c0124",
}


# Binary64 warp instructions (FP64-pipe issue slots) per flight segment of the
# same kernel, from ncu's sm__inst_executed_pipe_fp64 on one full-size launch
# of this workload (profiles/transport_fp64_downbranch_500k_fp64_ops.md); null
# for other sources.  (Lane operations would count the redundant lanes of the
# lone-walker mode, where the whole warp runs one walk.)
FP64_OPS_CAPTURE = {
    "warp_instructions_per_segment": 8.950,
    "sources": TRAFFIC_CAPTURE["sources"],
    "sha256": TRAFFIC_CAPTURE["sha256"],
}
# Binary64 pipe peak in issue slots: one binary64 warp instruction per ~64
# cycles per SM sub-partition (measured on this GPU with one-warp probes,
# dependent or not), 4 sub-partitions per SM, 152 SMs, 2070 MHz.
FP64_PEAK_SLOTS = 4 * 152 * 2.070e9 / 64


def _sources_match(capture):
    import hashlib
    h = hashlib.sha256()
    for rel in capture["sources"]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest() == capture["sha256"]


def _captured_traffic():
    return TRAFFIC_CAPTURE["dram_bytes_per_launch"] if _sources_match(TRAFFIC_CAPTURE) else None


def _fp64_roofline(segments, seconds):
    per = FP64_OPS_CAPTURE["warp_instructions_per_segment"]
    if per is None or not _sources_match(FP64_OPS_CAPTURE):
        return None
    achieved = per * segments / seconds
    return {"bound": "alu", "achieved": achieved / 1e9, "peak": FP64_PEAK_SLOTS / 1e9,
            "unit": "G binary64 warp instructions/s", "frac": achieved / FP64_PEAK_SLOTS,
            "warp_instructions_per_segment": per, "kernel": "transport_fp64",
            "peak_kind": "derived: 1 binary64 warp instruction per 64 cycles per sub-partition (measured), "
                         "4 per SM x 152 SMs x 2070 MHz"}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo")
        return dist, dist.get_rank(), ws
    return None, 0, 1


def run_reference(args):
    """CPU oracle on the host cores, a bounded sample per step."""
    import oracle
    from paper_1401_5469_gb300 import synth
    dist, rank, ws = _dist()
    if rank != 0:
        return 0
    spec = synth.downbranch_model()
    threads = os.cpu_count() or 1
    sample = int(os.environ.get("BENCH_REF_SAMPLE", str(spec.n_packets)))
    t_rad = np.full(spec.n_shells, 1.0e4)
    w = oracle.geometric_dilution(spec)
    om = None
    times = []
    total = 0
    for step in range(args.warmup + args.steps):
        tau = oracle.plasma_tau(spec, t_rad, w)
        if om is None:
            om = oracle.OracleModel(spec, tau=tau)
        else:
            om.set_tau(tau)
        t0 = time.perf_counter()
        r = oracle.run_iteration(om, spec.seed, step, spec.n_packets, spec.t_inner, first=0,
                                 count=sample, threads=threads, record=False)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            total += sample
        if sample >= spec.n_packets:  # the iteration cycle: T_R, W from this step's estimators
            t_rad, w = oracle.update_radiation_field(spec, r.j_est, r.nu_bar, t_rad, w)
    value = total / sum(times)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample_packets_per_step": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": (f"the whole 1e6-packet iteration k per step (longest walks included), "
                                        f"T_R and W updated after each step" if sample >= spec.n_packets else
                                        f"first {sample} of 1e6 packets of iteration k, T_R and W held"),
                             "note": "transport only; each step's Sobolev depths are computed outside the timing"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_sample(spec, seconds_hint=10.0):
    """Oracle throughput on a bounded sample of the workload (first iteration),
    on all host cores and on one, with the counted work of the sample."""
    import oracle
    threads = os.cpu_count() or 1
    t_rad = np.full(spec.n_shells, 1.0e4)
    w = oracle.geometric_dilution(spec)
    om = oracle.OracleModel(spec, tau=oracle.plasma_tau(spec, t_rad, w))
    n = int(os.environ.get("BENCH_CPU_SAMPLE", str(spec.n_packets)))
    t0 = time.perf_counter()
    r = oracle.run_iteration(om, spec.seed, 0, spec.n_packets, spec.t_inner, first=0, count=n,
                             threads=threads, record=False)
    dt = time.perf_counter() - t0
    n1 = max(1, min(n, 62_500))
    t0 = time.perf_counter()
    oracle.run_iteration(om, spec.seed, 0, spec.n_packets, spec.t_inner, first=0, count=n1,
                         threads=1, record=False)
    dt1 = time.perf_counter() - t0
    st = r.stats
    whole = n >= spec.n_packets
    return {"value": n / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": (f"the whole 1e6-packet iteration 0, longest walks included ({dt:.1f} s)" if whole else
                       f"first {n} of the 1e6 packets of iteration 0 ({dt:.1f} s)"),
            "note": ("the iteration's transport only (the Sobolev depths are computed beforehand, "
                     "outside the timing)" if whole else
                     "a packet sample: the iteration's longest random walks are not in it"),
            "interactions_per_s": (st["line_interactions"] + st["e_scatters"]) / dt,
            "line_checks_per_s": st["line_checks"] / dt,
            "single_thread": {"value": n1 / dt1, "unit": UNIT,
                              "sample": f"first {n1} packets of iteration 0 ({dt1:.1f} s)"}}


def scatter_config(mc, synth):
    """The 2000-line scatter model (20 shells, 1e4 packets, tau given), one
    iteration: GPU transport time (CUDA events) and the oracle on all host
    cores, both over the whole iteration."""
    spec = synth.scatter_model()
    m = mc.Model(spec)
    m.set_plasma(tau=spec.tau)
    for it in range(3):  # warm-up
        m.run_iteration(spec.seed, it, spec.n_packets, spec.t_inner)
    ms = []
    for it in range(3, 8):
        m.run_iteration(spec.seed, it, spec.n_packets, spec.t_inner)
        ms.append(float(m.timing()[1]))
    m.close()
    out = {"workload": "scatter-20sh-2000-lines-1e4-packets", "gpu_transport_ms": float(np.median(ms)),
           "gpu_packets_per_s": spec.n_packets / (1e-3 * float(np.median(ms)))}
    if os.environ.get("BENCH_SKIP_CPU") != "1":
        import oracle
        om = oracle.OracleModel(spec, tau=spec.tau)
        t0 = time.perf_counter()
        oracle.run_iteration(om, spec.seed, 0, spec.n_packets, spec.t_inner, threads=os.cpu_count() or 1,
                             record=False)
        dt = time.perf_counter() - t0
        out["cpu_oracle_packets_per_s"] = spec.n_packets / dt
        out["cpu_cores"] = os.cpu_count() or 1
    return out


def run_ours(args):
    import torch
    from paper_1401_5469_gb300 import mc, synth
    dist, rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    spec = synth.downbranch_model()
    N = spec.n_packets
    seed = spec.seed
    m = mc.Model(spec)
    S, L = spec.n_shells, spec.n_lines
    m.set_plasma()  # T_R = 1e4 K, geometric W (Sect. 2.8)
    stream = torch.cuda.current_stream()
    if ws > 1:
        # one model iterated with ws x 1e6 packets per iteration: rank r transports
        # the packet range shard.packet_range(r, ws, ws N), the ranks sum J, nu_bar,
        # the spectrum and J_blue with one all-reduce each, and every rank applies
        # the T_R/W update to the identical sums (Sect. 2.8)
        from paper_1401_5469_gb300 import shard

        def step(it):
            shard.run_sharded_iteration(m, seed, it, ws * N, spec.t_inner, j_blue=True, update=False)
            mc.mc_update_radiation_field(m.h, None, None)
    else:
        def step(it):
            m.run_iteration(seed, it, N, spec.t_inner)
            mc.mc_update_radiation_field(m.h, None, None)

    # warm-up (W >= 3 enforced by the caller's arguments)
    it = 0
    for _ in range(args.warmup):
        step(it)
        it += 1
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = m.launches()
    k_ms = np.zeros(3)
    stats_acc = {}
    phase_ms = np.zeros(2)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step(it)
        # per-kernel device times of this step (events on the model's stream)
        k_ms += m.timing()
        phase_ms += m.phases()
        _, st, _ = m.spectrum()
        for k, v in st.items():
            stats_acc[k] = stats_acc.get(k, 0) + v
        it += 1
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    clk = clocks.stop()
    launches = m.launches() - l0
    if dist:
        t = torch.tensor([elapsed], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())

    # ---- end-to-end through the C ABI with host buffers
    pin = lambda n: torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    t_h, w_h = pin(S), pin(S)
    j_h, nb_h, jb_h = pin(S), pin(S), pin(S * L)
    sp_h = pin(spec.spec_bins + 2)
    t_h[:], w_h[:] = m.update_radiation_field()
    e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e_steps):
        mc.mc_set_plasma(m.h, t_h, w_h, None)
        if ws > 1:
            shard.run_sharded_iteration(m, seed, it, ws * N, spec.t_inner, j_blue=True, update=False)
        else:
            mc.mc_run_iteration(m.h, seed, it, N, spec.t_inner)
        mc.mc_read_estimators(m.h, j_h, nb_h, jb_h, None)
        mc.mc_read_spectrum(m.h, sp_h, None)
        mc.mc_update_radiation_field(m.h, t_h, w_h)
        it += 1
    e2e_s = (time.perf_counter() - t0) / e_steps
    h2d = 2 * S * 8
    d2h = (2 * S + S * L + spec.spec_bins + 2 + 2 * S) * 8

    m.close()
    mixed = measure_mixed(spec, seed, args) if os.environ.get("BENCH_SKIP_MIXED") != "1" else None
    scatter = scatter_config(mc, synth) if rank == 0 else None
    batched = None
    if rank == 0 and ws == 1 and os.environ.get("BENCH_SKIP_BATCHED") != "1":
        # the batched workload (256 uneven models x 10 iterations, mixed precision,
        # one persistent launch per group iteration); per-model binary64 on the
        # first 8 models for the ratio
        r = measure_batched(256, 2, True, fp64_models=8, noise_models=0)
        batched = {"metric": "models/s", "value": r["value"], "unit": "models/s",
                   "wall_s": r["batched_s"], "config": r["config"], "packets_per_s": r["packets_per_s"],
                   "segments_per_s": r["segments_per_s"], "interactions_per_s": r["interactions_per_s"],
                   "groups": r["groups"], "launches": len(r["transport_ms_per_group_iteration"]),
                   "roofline": r["roofline"], "autotune": r["autotune"],
                   "fp64_per_model": r["fp64_per_model"],
                   "speedup_vs_fp64_per_model": r["speedup_vs_fp64_per_model"],
                   "clocks": r["clocks"]}
    if rank != 0:
        return 0
    ms_step = 1e3 * elapsed / args.steps
    value = ws * N * args.steps / elapsed
    per = {k: v / args.steps for k, v in stats_acc.items()}
    k1_ms = k_ms[1] / args.steps
    # algorithmic bytes of the transport kernel per launch (units from its counters)
    alg_bytes = (8 * per["line_checks"] + 8 * per["resonances"]       # nu_line per check, tau per Sobolev point
                 + 8 * per["resonances"]                               # J_blue update per Sobolev point
                 + 40 * per["segments"]                                # shell row + 2 estimator updates
                 + 8 * per["escaped"])                                 # spectrum bin
    peak, peak_kind = _peaks()
    achieved = alg_bytes / (k1_ms * 1e-3) / 1e9
    cpu = cpu_baseline_sample(spec) if os.environ.get("BENCH_SKIP_CPU") != "1" else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "shells": S, "lines": L, "packets_per_step": ws * N,
                   "line_mode": "downbranch", "j_blue": True, "precision": "fp64",
                   "parallelism": (f"packet ranges of one {ws}x1e6-packet iteration over {ws} GPUs, "
                                   "estimators summed by all-reduce" if ws > 1 else "one GPU"),
                   "l2": "inputs larger than L2 (tau 80 MB + J_blue 80 MB rewritten every step)"},
        "interactions_per_s": ws * (per["line_interactions"] + per["e_scatters"]) / (ms_step * 1e-3),
        "line_checks_per_s": ws * per["line_checks"] / (ms_step * 1e-3),
        "kernel_ms": {"plasma": k_ms[0] / args.steps, "transport": k1_ms, "update": k_ms[2] / args.steps},
        "transport_phases_ms": {"queue_drain": phase_ms[0] / args.steps, "tail": phase_ms[1] / args.steps},
        "per_step": per,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": _captured_traffic(), "kernel": "transport_fp64",
                     "peak_kind": peak_kind, "algorithmic_bytes_per_launch": alg_bytes},
        "roofline_fp64": _fp64_roofline(per["segments"], k1_ms * 1e-3),
        # the same kernel while its packet queue lasts: most of a launch's line
        # checks, Sobolev points and segments happen before the queue empties
        # (then at most one packet per resident lane is still in flight), so the
        # launch's algorithmic bytes over the time to the empty queue approximate
        # (from above) the kernel's rate while the GPU is full
        "roofline_queue_phase": {
            "bound": "hbm", "achieved": alg_bytes / (phase_ms[0] / args.steps * 1e-3) / 1e9, "peak": peak,
            "unit": "GB/s", "frac": alg_bytes / (phase_ms[0] / args.steps * 1e-3) / 1e9 / peak,
            "queue_ms": phase_ms[0] / args.steps, "kernel": "transport_fp64", "peak_kind": peak_kind,
            "note": "launch's algorithmic bytes / time until the packet queue is empty; packets still "
                    "in flight then (at most one per resident lane) finish after it"},
        "cpu_baseline": cpu,
        "e2e": {"value": ws * N / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "mixed_precision": mixed,
        "scatter_config": scatter,
        "batched": batched,
    }
    print(json.dumps(line), flush=True)
    return 0


def measure_mixed(spec, seed, args):
    """The same iteration loop in mixed precision (binary32 distances and
    optical depths; binary64 frequencies, resonance tests and estimators)."""
    import torch
    from paper_1401_5469_gb300 import mc
    N = spec.n_packets
    m = mc.Model(spec, precision=mc.MC_PRECISION_MIXED)
    m.set_plasma()
    stream = torch.cuda.current_stream()
    it = 0
    for _ in range(args.warmup):
        m.run_iteration(seed, it, N, spec.t_inner)
        mc.mc_update_radiation_field(m.h, None, None)
        it += 1
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k_ms = np.zeros(3)
    tail = 0.0
    ev0.record(stream)
    for _ in range(args.steps):
        m.run_iteration(seed, it, N, spec.t_inner)
        mc.mc_update_radiation_field(m.h, None, None)
        k_ms += m.timing()
        tail += float(m.phases()[1])
        it += 1
    ev1.record(stream)
    torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    m.close()
    return {"value": N * args.steps / elapsed, "unit": UNIT, "ms_per_step": 1e3 * elapsed / args.steps,
            "kernel_ms": {"plasma": k_ms[0] / args.steps, "transport": k_ms[1] / args.steps,
                          "update": k_ms[2] / args.steps},
            "transport_tail_ms": tail / args.steps, "dtype": "f32/f64"}


def _log(msg):
    print(f"[bench] {msg}", file=sys.stderr, flush=True)


def measure_batched(n_models=256, groups=2, j_blue=True, fp64_models=None, noise_models=16, n_it=10,
                    order=None):
    """256 uneven models x 10 iterations: batched mixed vs per-model binary64.

    The per-model binary64 side runs the first ``fp64_models`` models of the
    generated list (all of them by default) with the same seeds and packet
    counts; ``noise_models`` of those are run again with another seed for the
    Monte Carlo spread of T_R."""
    import torch
    from paper_1401_5469_gb300 import mc, synth
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    specs = synth.batched_models(n_models=n_models, seed=1401, iterations=n_it)
    gen_s = time.perf_counter() - t0
    _log(f"generated {n_models} models in {gen_s:.1f} s")
    seeds = [5469 + k for k in range(n_models)]
    n = [s.n_packets for s in specs]
    t_in = [s.t_inner for s in specs]
    total_packets = int(sum(n))

    # ---- batched, mixed precision: G groups of models, one batch (persistent
    # launch, own stream) each; a group's next iteration is enqueued as soon as
    # its last one ends, so one group's bulk fills the SMs another's tail of
    # long random walks leaves idle (a model's results do not depend on its group)
    jb = bool(j_blue)
    G = max(1, min(groups, n_models))
    t0 = time.perf_counter()
    # deal models by work (packets x lines) round-robin, so the groups balance;
    # a group's models share one stream (the batch orders itself after it)
    by_work = sorted(range(n_models), key=lambda k: -n[k] * specs[k].n_lines)
    grp_of = [by_work[g::G] for g in range(G)]
    g_streams = [torch.cuda.Stream() for _ in range(G)]
    group_of = {k: g for g, grp in enumerate(grp_of) for k in grp}
    models = [mc.Model(s, precision=mc.MC_PRECISION_MIXED, j_blue=jb,
                       stream=ctypes.c_void_p(g_streams[group_of[k]].cuda_stream))
              for k, s in enumerate(specs)]
    for m in models:
        m.set_plasma()
    batches = [mc.Batch([models[k] for k in grp]) for grp in grp_of]
    gargs = [([seeds[k] for k in grp], [n[k] for k in grp], [t_in[k] for k in grp]) for grp in grp_of]
    torch.cuda.synchronize()
    _log(f"created mixed models in {time.perf_counter() - t0:.1f} s ({G} groups)")
    t0 = time.perf_counter()
    tuned, tuned_ms, trials = [], [], 0
    for b, (sd, np_, ti) in zip(batches, gargs):
        l_, ms_, tr_ = b.autotune(sd, 0, np_, ti)
        tuned.append(l_)
        tuned_ms.append(ms_)
        trials += tr_
    tune_s = time.perf_counter() - t0
    _log(f"autotune {tuned} {tuned_ms} ms after {trials} trials ({tune_s:.1f} s)")
    if order is not None:  # a given queue order with the tuned block size and residency
        for b, l_ in zip(batches, tuned):
            b.set_launch(block=l_["block"], blocks_per_sm=l_["blocks_per_sm"], order=order)
        tuned = [b.launch() for b in batches]
    clocks = ClockSampler(0)
    clocks.start()
    torch.cuda.synchronize()
    transport_ms = []
    keys = ("segments", "line_checks", "resonances", "line_interactions", "e_scatters", "escaped")
    work = {k: 0 for k in keys}
    alg_bytes = 0.0
    w0 = time.perf_counter()
    for b, (sd, np_, ti) in zip(batches, gargs):
        b.run_iteration(sd, 0, np_, ti, update=True)
    for it in range(n_it):
        for g, (b, (sd, np_, ti)) in enumerate(zip(batches, gargs)):
            transport_ms.append(b.transport_ms())  # waits for this group's iteration
            gw = {k: 0 for k in keys}
            for k in grp_of[g]:  # per-model run statistics (read after the iteration)
                st = models[k].spectrum()[1]
                for key in keys:
                    gw[key] += st[key]
            for key in keys:
                work[key] += gw[key]
            # algorithmic bytes of this launch: nu per line check, binary32 tau and
            # the 8-byte J_blue sum per Sobolev point, shell row + two estimator
            # sums per segment, spectrum bin per escaping packet
            alg_bytes += (8 * gw["line_checks"] + (4 + (8 if jb else 0)) * gw["resonances"]
                          + 40 * gw["segments"] + 8 * gw["escaped"])
            if it + 1 < n_it:
                b.run_iteration(sd, it + 1, np_, ti, update=True)
    for b in batches:
        b.synchronize()
    torch.cuda.synchronize()
    batched_s = time.perf_counter() - w0
    clk = clocks.stop()
    t_mixed = []
    for m in models:
        t, w, _ = m.plasma()
        t_mixed.append(t)
    for b in batches:
        b.close()
    for m in models:
        m.close()
    _log(f"batched: {batched_s:.2f} s for {n_it} iterations")

    # ---- per-model binary64, the same models, seeds and packets
    limit = n_models if fp64_models is None else min(int(fp64_models), n_models)
    fp64_s = 0.0
    t_fp64 = []

    def fp64_loop(spec, seed):
        m = mc.Model(spec, j_blue=jb)
        m.set_plasma()
        for it in range(n_it):
            m.run_iteration(seed, it, spec.n_packets, spec.t_inner)
            mc.mc_update_radiation_field(m.h, None, None)
        m.synchronize()
        t, _, _ = m.plasma()
        m.close()
        return t

    for k, spec in enumerate(specs[:limit]):
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        t_fp64.append(fp64_loop(spec, seeds[k]))
        fp64_s += time.perf_counter() - w0
    fp64_models_s = limit / fp64_s if limit else None
    _log(f"per-model fp64: {fp64_s:.2f} s for {limit} models")
    # Monte Carlo noise of the same statistic: binary64 with another seed
    rms = lambda a, b_: float(np.sqrt(np.mean(((a - b_) / b_) ** 2)))
    n_noise = min(noise_models, limit)
    d_mix = [rms(t_mixed[k], t_fp64[k]) for k in range(limit)]
    d_seed = [rms(fp64_loop(specs[k], seeds[k] + 1_000_000), t_fp64[k]) for k in range(n_noise)]
    med = lambda v: float(np.median(v)) if v else None
    value = n_models / batched_s
    peak, peak_kind = _peaks()
    k_s = 1e-3 * sum(transport_ms)
    return {
        "value": value, "batched_s": batched_s,
        "config": {"workload": f"batched-{n_models}-uneven-models-10-iterations",
                   "models": n_models, "iterations": n_it, "packets_per_iteration": total_packets,
                   "shells": [min(s.n_shells for s in specs), max(s.n_shells for s in specs)],
                   "lines": [min(s.n_lines for s in specs), max(s.n_lines for s in specs)],
                   "j_blue": jb, "line_mode": "downbranch", "precision": "mixed",
                   "l2": "inputs larger than L2 (Sobolev depths and J_blue of all models)"},
        "packets_per_s": total_packets * n_it / batched_s,
        "segments_per_s": work["segments"] / batched_s,
        "line_checks_per_s": work["line_checks"] / batched_s,
        "interactions_per_s": (work["line_interactions"] + work["e_scatters"]) / batched_s,
        "segments_per_packet": work["segments"] / (total_packets * n_it),
        "groups": G,
        "transport_ms_per_group_iteration": transport_ms,
        "roofline": {"bound": "hbm", "kernel": "transport_mixed (batched)",
                     "achieved": alg_bytes / k_s / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": alg_bytes / k_s / 1e9 / peak, "peak_kind": peak_kind,
                     "algorithmic_bytes": alg_bytes, "kernel_s": k_s,
                     "aggregate_gbs_over_wall": alg_bytes / batched_s / 1e9,
                     "note": "kernel_s sums the launches' CUDA-event durations; the two groups' "
                             "launches overlap, so the aggregate over the wall clock is also given"},
        "autotune": {"launch": tuned, "transport_ms": tuned_ms, "trials": trials, "seconds": tune_s},
        "fp64_per_model": {"models_per_s": fp64_models_s, "seconds": fp64_s, "models_timed": limit,
                           "which": f"the first {limit} of the {n_models} generated models (generation seed 1401)",
                           "packets_per_s": sum(n[:limit]) * n_it / fp64_s if limit else None,
                           "timing": "host clock around each model's 10 iterations (synchronised)"},
        "speedup_vs_fp64_per_model": value / fp64_models_s if limit else None,
        "t_rad_after_10_iterations": {
            "rms_rel_diff_mixed_vs_fp64": {"median": med(d_mix), "models": limit},
            "rms_rel_diff_fp64_seed_vs_seed": {"median": med(d_seed), "models": n_noise},
            "note": "per model, RMS over shells of the relative T_R difference; mixed and binary64 "
                    "share the seeds, but their histories part after rounding differences, so the "
                    "comparison is with the seed-to-seed Monte Carlo spread"},
        "generation_s": gen_s,
        "clocks": clk,
    }


def run_batched(args):
    """256 uneven models x 10 iterations: batched mixed vs per-model binary64."""
    limit = int(os.environ.get("BENCH_FP64_MODELS", str(args.models)))
    orders = {"auto": None, "packets": 0, "work": 1, "given": 2}
    r = measure_batched(args.models, args.groups, bool(args.j_blue), fp64_models=limit,
                        order=orders[args.order])
    value, batched_s = r.pop("value"), r.pop("batched_s")
    line = {
        "metric": "models/s", "value": value, "unit": "models/s", "n_gpus": 1, "steps": 10,
        "warmup": r["autotune"]["trials"], "ms_per_step": 1e3 * batched_s / 10, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
        "wall_s": batched_s, **r,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Poisson arrivals of batched-workload models, continuous batching."""
    import torch
    from paper_1401_5469_gb300 import mc, serve, synth
    torch.cuda.set_device(0)
    mixed = args.precision == "mixed"
    prec = mc.MC_PRECISION_MIXED if mixed else mc.MC_PRECISION_FP64
    warm_s, window_s = 10.0, 60.0
    t0 = time.perf_counter()
    pool = synth.batched_models(n_models=256, seed=1401)
    _log(f"generated the model pool in {time.perf_counter() - t0:.1f} s")
    rng = np.random.default_rng(50)
    arrivals = []
    t = 0.0
    while True:
        t += float(rng.exponential(1.0 / args.rate))
        if t >= warm_s + window_s:
            break
        arrivals.append(t)
    reqs = [serve.Request(rid=k, spec=pool[int(rng.integers(len(pool)))],
                          n_iterations=int(rng.integers(5, 21)), seed=5469 + k, arrival=a)
            for k, a in enumerate(arrivals)]
    tick_packets = args.tick_packets or (25_000_000 if mixed else 5_000_000)
    # model groups advancing independently: 2 for batched mixed precision (a
    # group's batch keeps a large packet budget), 8 for binary64 (single-model
    # launches on 8 streams overlap one another's tails); measured best of 1-16
    n_groups = args.serve_groups if args.serve_groups > 0 else (2 if mixed else 8)
    server = serve.Server(hbm_budget_bytes=150e9, j_blue=False, precision=prec,
                          max_tick_packets=tick_packets, n_groups=n_groups)
    clocks = ClockSampler(0)
    clocks.start()
    start = time.perf_counter()
    nxt = 0
    peak_resident = 0
    while True:
        now = time.perf_counter() - start
        if now >= warm_s + window_s:
            break
        while nxt < len(reqs) and reqs[nxt].arrival <= now:
            server.submit(reqs[nxt])
            nxt += 1
        if not server.active and not server.queue:
            if nxt >= len(reqs):
                break
            time.sleep(max(0.0, min(reqs[nxt].arrival - now, 0.05)))
            continue
        if n_groups > 1:
            # groups advance on their own streams; poll without waiting for the device
            if server.poll(now) == 0:
                time.sleep(0.0005)
        else:
            server.step(now)
        peak_resident = max(peak_resident, len(server.active))
    end = time.perf_counter() - start
    clk = clocks.stop()
    backlog_queued, backlog_active = len(server.queue), len(server.active)
    server.close()
    done = [r for r in reqs if r.finished is not None and r.finished <= warm_s + window_s
            and r.arrival >= warm_s]
    # requests retired by close() at the end are not finished work
    done = [r for r in done if r.done_iterations >= r.n_iterations]
    lat = serve.percentiles([r.latency for r in done])
    in_window = [r for r in reqs if r.arrival >= warm_s]
    offered = sum(r.spec.n_packets * r.n_iterations for r in in_window) / window_s
    served = sum(r.spec.n_packets * r.n_iterations for r in done) / window_s
    value = len(done) / window_s
    line = {
        "metric": "models/s", "value": value, "unit": "models/s", "n_gpus": 1,
        "steps": server.ticks, "warmup": 0, "ms_per_step": float(np.mean(server.tick_ms)) if server.tick_ms else None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32/f64" if mixed else "f64", "data": "synthetic",
        "config": {"workload": f"serve-poisson-{args.rate:g}-per-s-{args.precision}",
                   "arrival_rate": args.rate, "window_s": window_s, "warmup_s": warm_s,
                   "iterations": [5, 20], "hbm_budget_bytes": 150e9, "max_tick_packets": tick_packets,
                   "model_pool": "256 batched-workload models (seed 1401), one drawn per request",
                   "j_blue": False, "groups": n_groups,
                   "mode": ("groups of models on their own streams, each group's next iteration "
                            "enqueued when its last ends" if n_groups > 1 else
                            "ticks: every resident model advances by one iteration per tick")},
        "latency_s": lat,
        "requests": {"arrived_in_window": len(in_window), "finished_in_window": len(done),
                     "backlog_at_end": {"queued": backlog_queued, "resident": backlog_active}},
        "packet_iterations_per_s": {"offered": offered, "served": served},
        "ticks": server.ticks, "peak_resident_models": peak_resident,
        "tick_ms": {"p50": float(np.percentile(server.tick_ms, 50)) if server.tick_ms else None,
                    "max": float(np.max(server.tick_ms)) if server.tick_ms else None},
        "elapsed_s": end, "clocks": clk,
        "host_s": server.host_s,
        "admitted": sum(1 for r in reqs if r.admitted is not None),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_spectrum(args):
    """The spectrum iteration with virtual packets (Sect. 2.9).  Cost: the
    500k-line downbranch model after 3 iterations of the loop, 1e6 packets,
    N_v = 3, tau_v cut 30, transport time with and without v-packets (that
    model escapes almost only below its line list, so its optical spectrum is
    empty).  Noise: the 2000-line scatter model, 1e5 packets, 8 seeds, the
    relative spread per spectral bin of the r-packet and v-packet spectra."""
    import torch
    from paper_1401_5469_gb300 import mc, synth
    torch.cuda.set_device(0)
    clocks = ClockSampler(0)
    clocks.start()
    spec = synth.downbranch_model(j_blue=False)
    N, nv, cut = spec.n_packets, 3, 30.0
    m = mc.Model(spec)
    m.set_plasma()
    for it in range(3):
        m.run_iteration(spec.seed, it, N, spec.t_inner)
        mc.mc_update_radiation_field(m.h, None, None)
    t_rad, w, _ = m.plasma()
    m.set_plasma(t_rad, w)  # the same plasma state for both spectrum iterations
    m.run_iteration(spec.seed, 3, N, spec.t_inner)
    plain_ms = float(m.timing()[1])
    m.set_virtual_packets(nv, cut)
    m.run_iteration(spec.seed, 3, N, spec.t_inner)
    virt_ms = float(m.timing()[1])
    st = m.spectrum()[1]
    n_v = nv * (N + st["line_interactions"] + st["e_scatters"])
    sp = m.spectrum()[0]
    below = float(sp[spec.spec_bins] / max(sp.sum(), 1e-300))
    m.close()

    sc = synth.scatter_model(n_packets=100_000)
    ms = mc.Model(sc)
    ms.set_plasma(tau=sc.tau)
    ms.set_virtual_packets(nv)
    r_sp, v_sp = [], []
    for k in range(8):
        ms.run_iteration(5469 + k, 0, sc.n_packets, sc.t_inner)
        r_sp.append(ms.spectrum()[0][:sc.spec_bins])
        v_sp.append(ms.virtual_spectrum()[:sc.spec_bins])
    sc_ms = float(ms.timing()[1])
    ms.close()
    clk = clocks.stop()
    r_sp, v_sp = np.array(r_sp), np.array(v_sp)
    out = {}
    for name, g in (("fine_1000_bins", 1), ("coarse_100_bins", 10)):
        rr = r_sp.reshape(8, -1, g).sum(axis=2)
        vv = v_sp.reshape(8, -1, g).sum(axis=2)
        mean_r = rr.mean(axis=0)
        pop = mean_r > 0.01 * mean_r.max()  # bins above 1% of the peak
        nr = rr[:, pop].std(axis=0, ddof=1) / rr[:, pop].mean(axis=0)
        nvv = vv[:, pop].std(axis=0, ddof=1) / vv[:, pop].mean(axis=0)
        wgt = mean_r[pop] / mean_r[pop].sum()
        out[name] = {"bins": int(pop.sum()), "r_noise_median": float(np.median(nr)),
                     "v_noise_median": float(np.median(nvv)),
                     "noise_ratio_median": float(np.median(nr / nvv)),
                     "noise_ratio_energy_weighted": float(np.sum(wgt * nr) / np.sum(wgt * nvv))}
    line = {"metric": "virtual packets/s", "value": n_v / (1e-3 * virt_ms), "unit": "v-packets/s",
            "n_gpus": 1, "steps": 1, "warmup": 3, "ms_per_step": virt_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "spectrum-iteration-downbranch-500k-lines-1e6-packets-Nv3",
                       "n_virtual": nv, "tau_v_max": cut, "packets": N},
            "transport_ms": {"without_virtual": plain_ms, "with_virtual": virt_ms},
            "virtual_packets": n_v, "escaped_energy_below_line_list": below,
            "spectrum_noise_scatter_model_1e5_packets_8_seeds": out,
            "scatter_model_spectrum_iteration_ms": sc_ms, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_macroatom(args):
    """Macro-atom vs downbranch line interactions (Sect. 2.5) on the 500k-line,
    1e6-packet model (the same lines and branching rows; macro-atom mode adds
    synthetic internal jumps), binary64, 1 warm-up and 3 timed iterations of
    the loop each."""
    import torch
    from paper_1401_5469_gb300 import mc, synth
    torch.cuda.set_device(0)
    clocks = ClockSampler(0)
    clocks.start()
    res = {}
    for name, spec in (("downbranch", synth.downbranch_model(j_blue=False)),
                       ("macroatom", synth.macroatom_model(j_blue=False))):
        N = spec.n_packets
        m = mc.Model(spec)
        m.set_plasma()
        ms, inter = [], []
        for it in range(4):
            m.run_iteration(spec.seed, it, N, spec.t_inner)
            mc.mc_update_radiation_field(m.h, None, None)
            if it:
                ms.append(float(m.timing()[1]))
                st = m.spectrum()[1]
                inter.append(st["line_interactions"] + st["e_scatters"])
        m.close()
        t = float(np.median(ms))
        res[name] = {"transport_ms_median": t, "packets_per_s": N / (1e-3 * t),
                     "interactions_per_iteration": float(np.mean(inter)),
                     "interactions_per_s": float(np.mean(inter)) / (1e-3 * t)}
    clk = clocks.stop()
    ratio = res["macroatom"]["transport_ms_median"] / res["downbranch"]["transport_ms_median"]
    line = {"metric": "packets/s", "value": res["macroatom"]["packets_per_s"], "unit": "packets/s",
            "n_gpus": 1, "steps": 3, "warmup": 1, "ms_per_step": res["macroatom"]["transport_ms_median"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "macroatom-vs-downbranch-500k-lines-1e6-packets", "j_blue": False},
            "modes": res, "macroatom_time_over_downbranch": ratio, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="downbranch", choices=["downbranch", "batched", "serve", "spectrum", "macroatom"])
    ap.add_argument("--models", type=int, default=256)
    ap.add_argument("--groups", type=int, default=2, help="batched workload: model groups on their own streams")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--tick-packets", type=int, default=0)
    ap.add_argument("--serve-groups", type=int, default=0,
                    help="serving: model groups advancing independently (1 = one tick for all; "
                         "0 = 2 in mixed precision, 8 in binary64)")
    ap.add_argument("--j-blue", type=int, default=1, choices=[0, 1], help="J_blue estimators (batched workload)")
    ap.add_argument("--order", default="auto", choices=["auto", "packets", "work", "given"],
                    help="batched workload: packet queue order (auto = the autotuner's)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "spectrum":
        return run_spectrum(args)
    if args.workload == "macroatom":
        return run_macroatom(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
