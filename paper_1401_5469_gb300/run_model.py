"""Run a synthetic ejecta model for a few Monte Carlo iterations on the GPU.

    python -m paper_1401_5469_gb300.run_model [--model downbranch|scatter]
        [--lines L] [--packets N] [--iterations K] [--precision fp64|mixed]
        [--first F --count C]
    python -m paper_1401_5469_gb300.run_model --batched M [--iterations K]

Each iteration recomputes the Sobolev depths from T_R and W (downbranch
model), transports the packets and updates T_R and W (Sect. 2.8).  With
--first/--count only packets [F, F+C) of the N-packet iteration are
transported (the draws of a packet depend only on its id), e.g. a single long
random walk.  With --batched M: the first M models of the batched workload
(generation seed 1401), mixed precision, one batched launch per iteration
with a fixed shape (128 threads per block, 4 resident blocks per SM, largest
models first).  Prints one JSON line of totals and kernel times per
iteration.  Used for profiling captures.
"""
from __future__ import annotations

import argparse
import json

from . import mc, synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--model", default="downbranch", choices=["downbranch", "scatter"])
    ap.add_argument("--lines", type=int, default=None)
    ap.add_argument("--packets", type=int, default=None)
    ap.add_argument("--iterations", type=int, default=2)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--seed", type=int, default=5469)
    ap.add_argument("--first", type=int, default=0)
    ap.add_argument("--count", type=int, default=None)
    ap.add_argument("--update", type=int, default=1, help="update T_R, W between iterations")
    ap.add_argument("--batched", type=int, default=0, help="run the first M batched-workload models")
    a = ap.parse_args()
    if a.batched:
        return run_batched(a)
    if a.model == "downbranch":
        kw = {}
        if a.lines:
            kw["n_lines"] = a.lines
        if a.packets:
            kw["n_packets"] = a.packets
        spec = synth.downbranch_model(**kw)
    else:
        spec = synth.scatter_model(n_lines=a.lines or 2000, n_packets=a.packets or 10_000)
    prec = mc.MC_PRECISION_FP64 if a.precision == "fp64" else mc.MC_PRECISION_MIXED
    m = mc.Model(spec, precision=prec)
    if spec.tau is not None:
        m.set_plasma(tau=spec.tau)
    else:
        m.set_plasma()
    n = spec.n_packets
    count = a.count if a.count is not None else n - a.first
    for it in range(a.iterations):
        m.run_iteration_range(a.seed, it, a.first, count, n, spec.t_inner)
        if spec.tau is None and a.update:
            m.update_radiation_field()
        _, st, _ = m.spectrum()
        ms = m.timing()
        ph = m.phases()
        us = float(ms[1]) * 1e3 / max(st["segments"], 1)
        print(json.dumps({"iteration": it, "ms": [float(x) for x in ms],
                          "bulk_ms": float(ph[0]), "tail_ms": float(ph[1]),
                          "us_per_segment": us, **st}), flush=True)
    m.close()


def run_batched(a):
    specs = synth.batched_models(n_models=a.batched, seed=1401, iterations=max(a.iterations, 1))
    models = [mc.Model(s, precision=mc.MC_PRECISION_MIXED) for s in specs]
    for m in models:
        m.set_plasma()
    b = mc.Batch(models)
    b.set_launch(block=128, blocks_per_sm=4, order=mc.MC_ORDER_PACKETS)
    seeds = [a.seed + k for k in range(len(specs))]
    n = [s.n_packets for s in specs]
    t = [s.t_inner for s in specs]
    for it in range(a.iterations):
        b.run_iteration(seeds, it, n, t, update=bool(a.update))
        ms = b.transport_ms()
        phases = b.phases()
        tot = {}
        for m in models:
            for k, v in m.spectrum()[1].items():
                tot[k] = tot.get(k, 0) + v
        print(json.dumps({"iteration": it, "models": len(specs), "transport_ms": ms, "queue_ms": phases[0],
                          "tail_ms": phases[1], **tot}), flush=True)
    b.close()
    for m in models:
        m.close()


if __name__ == "__main__":
    main()
