"""Benchmark of the GB300 Monte Carlo transport library.

Workload (default): the full-loop downbranch model -- 20 shells
(11000-20000 km/s, 13 d), 500,000 lines, 30 ions x 40 levels, J_blue
estimators, 1e6 packets per iteration, binary64.  One step is one Monte Carlo
iteration of Sect. 2.8: Sobolev depths recomputed from the current T_R, W
(plasma kernels), estimators zeroed, 1e6 packets transported, T_R and W
updated from the estimators.  The iteration index advances every step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  ``--impl reference`` times the CPU oracle (the plain
FP64 C implementation used by the tests) on a bounded packet sample of the
same workload.
"""
from __future__ import annotations

import argparse
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
    sample = int(os.environ.get("BENCH_REF_SAMPLE", "100000"))
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
    value = total / sum(times)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample_packets_per_step": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"first {sample} of 1e6 packets of iteration k, tau held from T_R=1e4 K"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_sample(spec, seconds_hint=10.0):
    """Oracle throughput on a bounded sample of the workload (first iteration)."""
    import oracle
    threads = os.cpu_count() or 1
    t_rad = np.full(spec.n_shells, 1.0e4)
    w = oracle.geometric_dilution(spec)
    om = oracle.OracleModel(spec, tau=oracle.plasma_tau(spec, t_rad, w))
    n = int(os.environ.get("BENCH_CPU_SAMPLE", "100000"))
    t0 = time.perf_counter()
    oracle.run_iteration(om, spec.seed, 0, spec.n_packets, spec.t_inner, first=0, count=n,
                         threads=threads, record=False)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {n} of the 1e6 packets of iteration 0 ({dt:.1f} s)"}


def run_ours(args):
    import torch
    from paper_1401_5469_gb300 import mc, synth
    dist, rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    spec = synth.downbranch_model()
    N = spec.n_packets
    seed = spec.seed + 1000 * rank
    m = mc.Model(spec)
    S, L = spec.n_shells, spec.n_lines
    m.set_plasma()  # T_R = 1e4 K, geometric W (Sect. 2.8)
    stream = torch.cuda.current_stream()

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
        m.run_iteration(seed, it, N, spec.t_inner)
        mc.mc_update_radiation_field(m.h, None, None)
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
        "config": {"workload": WORKLOAD, "shells": S, "lines": L, "packets_per_step": N,
                   "line_mode": "downbranch", "j_blue": True, "precision": "fp64",
                   "l2": "inputs larger than L2 (tau 80 MB + J_blue 80 MB rewritten every step)"},
        "interactions_per_s": ws * (per["line_interactions"] + per["e_scatters"]) / (ms_step * 1e-3),
        "line_checks_per_s": ws * per["line_checks"] / (ms_step * 1e-3),
        "kernel_ms": {"plasma": k_ms[0] / args.steps, "transport": k1_ms, "update": k_ms[2] / args.steps},
        "transport_phases_ms": {"queue_drain": phase_ms[0] / args.steps, "tail": phase_ms[1] / args.steps},
        "per_step": per,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "transport_fp64",
                     "peak_kind": peak_kind},
        "cpu_baseline": cpu,
        "e2e": {"value": ws * N / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "mixed_precision": mixed,
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
