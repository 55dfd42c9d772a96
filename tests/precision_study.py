"""Mixed-precision error against the binary64 oracle, next to the Monte Carlo
noise (the 500,000-line downbranch model, Sect. 2.8 iteration cycle).

Three kinds of run of the same model, all starting from T_R = 1e4 K and the
geometric dilution factor:

* the CPU oracle (binary64, seed 5469),
* the GPU mixed-precision path (seed 5469),
* the GPU binary64 path with seeds 5469 + k, k = 0..n_seeds-1, whose spread
  is the Monte Carlo noise sigma per shell and per spectral bin.

Two stages are compared:

* ``iteration0``: the first iteration (identical Sobolev depths on every
  side, 1e6 packets).  Mixed and oracle share the draws, so their difference
  is the rounding of the binary32 geometry plus the packets whose histories
  that rounding sends elsewhere.
* ``final``: after n_loop iterations with the T_R/W update, one more
  iteration with n_final packets (4e6), no update.  The loop amplifies any
  difference into independent Monte Carlo histories, so here every run --
  the binary64 GPU run with the oracle's own seed included -- differs from the
  oracle by about the noise.

For J_est, nu_bar (per shell) and the escaping-packet spectrum (per bin) the
study reports z = (run - oracle) / sigma: its RMS and maximum, for the mixed
run and, as the control, the binary64 GPU run with the oracle's seed.  J_blue
is off on every side (it changes no packet history).

    python tests/precision_study.py [--loop 10] [--final 4000000] [--seeds 16]

prints one JSON object.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _gpu_run(mc, spec, precision, seed, n_loop, n_final):
    m = mc.Model(spec, precision=precision, j_blue=False)
    m.set_plasma()
    N = spec.n_packets
    out = {}
    for it in range(n_loop):
        m.run_iteration(seed, it, N, spec.t_inner)
        if it == 0:
            j, nb, _, _ = m.estimators()
            out["iteration0"] = (j, nb, m.spectrum()[0])
        m.update_radiation_field()
    if n_final:
        m.run_iteration(seed, n_loop, n_final, spec.t_inner)
        j, nb, _, _ = m.estimators()
        out["final"] = (j, nb, m.spectrum()[0])
    m.close()
    return out


def _oracle_run(oracle, spec, seed, n_loop, n_final, threads):
    N = spec.n_packets
    t_rad = np.full(spec.n_shells, 1.0e4)
    w = oracle.geometric_dilution(spec)
    om = None
    out = {}
    for it in range(n_loop + (1 if n_final else 0)):
        tau = oracle.plasma_tau(spec, t_rad, w)
        if om is None:
            om = oracle.OracleModel(spec, tau=tau)
        else:
            om.set_tau(tau)
        n = N if it < n_loop else n_final
        r = oracle.run_iteration(om, seed, it, n, spec.t_inner, threads=threads, record=False,
                                 j_blue=False)
        if it == 0:
            out["iteration0"] = (r.j_est, r.nu_bar, r.spectrum)
        if it < n_loop:
            t_rad, w = oracle.update_radiation_field(spec, r.j_est, r.nu_bar, t_rad, w)
        else:
            out["final"] = (r.j_est, r.nu_bar, r.spectrum)
    return out


def _z(run, ref, sigma):
    ok = sigma > 0
    z = (run[ok] - ref[ok]) / sigma[ok]
    return {"rms": float(np.sqrt(np.mean(z * z))), "max_abs": float(np.max(np.abs(z))),
            "n": int(ok.sum()),
            "rel_l2": float(np.linalg.norm(run - ref) / max(np.linalg.norm(ref), 1e-300))}


def study(n_loop=10, n_final=4_000_000, n_seeds=16, seed=5469, threads=None, spec=None):
    import oracle
    from paper_1401_5469_gb300 import mc, synth
    mc.load()
    spec = spec if spec is not None else synth.downbranch_model()
    threads = threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    fp64 = [_gpu_run(mc, spec, mc.MC_PRECISION_FP64, seed + k, n_loop, n_final) for k in range(n_seeds)]
    mixed = _gpu_run(mc, spec, mc.MC_PRECISION_MIXED, seed, n_loop, n_final)
    t_gpu = time.perf_counter() - t0
    t0 = time.perf_counter()
    orc = _oracle_run(oracle, spec, seed, n_loop, n_final, threads)
    t_cpu = time.perf_counter() - t0
    report = {"model": f"downbranch {spec.n_shells} shells, {spec.n_lines} lines, "
                       f"{spec.n_packets} packets per iteration",
              "n_loop": n_loop, "n_final": n_final, "n_seeds": n_seeds, "seed": seed,
              "gpu_seconds": t_gpu, "oracle_seconds": t_cpu, "oracle_threads": threads}
    for stage in ("iteration0", "final"):
        if stage not in orc:
            continue
        rows = {}
        for q, name in enumerate(("j_est", "nu_bar", "spectrum")):
            runs = np.array([f[stage][q] for f in fp64])
            sigma = runs.std(axis=0, ddof=1)
            ref = orc[stage][q]
            if name == "spectrum":  # the in-range bins only
                runs, sigma, ref = runs[:, :-2], sigma[:-2], ref[:-2]
                mix, f0 = mixed[stage][q][:-2], fp64[0][stage][q][:-2]
            else:
                mix, f0 = mixed[stage][q], fp64[0][stage][q]
            rows[name] = {"mixed_vs_oracle": _z(mix, ref, sigma),
                          "fp64_gpu_vs_oracle": _z(f0, ref, sigma),
                          "sigma_rel_median": float(np.median(sigma[sigma > 0] / np.abs(runs.mean(axis=0))[sigma > 0]))}
        report[stage] = rows
    return report


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--loop", type=int, default=10)
    ap.add_argument("--final", type=int, default=4_000_000)
    ap.add_argument("--seeds", type=int, default=16)
    a = ap.parse_args()
    print(json.dumps(study(a.loop, a.final, a.seeds)), flush=True)


if __name__ == "__main__":
    main()
