"""The allocation-free transport entry point (mc_transport_noalloc).

It exists for callers that cannot allocate device memory where they run the
transport (a framework's fixed memory pool, a plug-in handed raw buffers, a
loop that must not allocate).  They pass every buffer; the kernel's working
memory is a static device array inside the library.  Here the caller's
buffers come from torch, and two calls in a row (iterations 0 and 1) are
checked against the model-based entry point (mc_run_iteration) and against
the oracle, with the tolerances of the parity tests: estimators and spectrum
to 1e-9 relative, run statistics exactly.  The second call also shows that
the shared scratch is cleared between calls, and that a call allocates
nothing: torch's caching allocator, the device's default memory pool (its
high-water mark reset before the call) and the device's free memory are the
same after the call as before it.

This file is named so that pytest collects it last.
"""
import ctypes
import os

import numpy as np
import pytest

import oracle
from paper_1401_5469_gb300 import synth

pytestmark = pytest.mark.gpu

EST_RTOL = 1e-9


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1401_5469_gb300 import mc
    mc.load()
    return torch, mc


def _close(a, b, rtol):
    scale = np.maximum(np.abs(b), 1e-300)
    assert np.all(np.abs(a - b) <= rtol * scale + 1e-300), float(np.max(np.abs(a - b) / scale))


def _device(torch, a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=dtype), device="cuda")


class _DefaultPool:
    """Usage counters of the current device's default memory pool (the pool
    cudaMallocAsync draws from), read through the driver API."""

    USED_CURRENT, USED_HIGH = 7, 8  # CU_MEMPOOL_ATTR_USED_MEM_CURRENT / _HIGH

    def __init__(self, torch):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int(0)
        assert self.cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_HIGH, ctypes.byref(zero)) == 0


def _memory_state(torch):
    torch.cuda.synchronize()
    return {"reserved": torch.cuda.memory_reserved(), "allocated": torch.cuda.memory_allocated(),
            "free": torch.cuda.mem_get_info()[0]}


def _model_reference(mc, spec, tau, seed, iteration, n):
    m = mc.Model(spec)
    m.set_plasma(tau=tau)
    m.run_iteration(seed, iteration, n, spec.t_inner)
    j, nb, jb, _ = m.estimators(j_blue=bool(spec.j_blue))
    sp, st, _ = m.spectrum()
    m.close()
    return j, nb, jb, sp, st


@pytest.mark.parametrize("kind", ["scatter", "downbranch"])
def test_noalloc_matches_model_entry_point_twice(env, kind):
    torch, mc = env
    if kind == "scatter":
        spec = synth.scatter_model(n_lines=2000, n_packets=10_000)
        tau = spec.tau
    else:
        spec = synth.downbranch_model(n_lines=20_000, n_packets=4000)
        rng = np.random.default_rng(4)
        tau = np.exp(-2 + 2 * rng.standard_normal((spec.n_shells, spec.n_lines)))
    S, L, B, n = spec.n_shells, spec.n_lines, spec.spec_bins, spec.n_packets
    keep = {
        "v_inner": _device(torch, spec.v_inner, np.float64),
        "v_outer": _device(torch, spec.v_outer, np.float64),
        "n_e": _device(torch, spec.n_e, np.float64),
        "nu": _device(torch, spec.nu, np.float64),
        "tau": _device(torch, tau, np.float64),
        "j_est": torch.empty(S, dtype=torch.float64, device="cuda"),
        "nu_bar": torch.empty(S, dtype=torch.float64, device="cuda"),
        "spectrum": torch.empty(B + 2, dtype=torch.float64, device="cuda"),
        "stats": torch.empty(9, dtype=torch.int64, device="cuda"),
    }
    args = mc.mc_noalloc_args(
        n_shells=S, v_inner=keep["v_inner"].data_ptr(), v_outer=keep["v_outer"].data_ptr(),
        n_e=keep["n_e"].data_ptr(), v_inner_0=float(spec.v_inner[0]), t_exp=float(spec.t_exp),
        n_lines=L, nu=keep["nu"].data_ptr(), tau=keep["tau"].data_ptr(), line_mode=int(spec.line_mode),
        seed=spec.seed, n_packets=n, t_inner=float(spec.t_inner), max_segments=0, delta_t=1.0,
        j_est=keep["j_est"].data_ptr(), nu_bar=keep["nu_bar"].data_ptr(),
        spectrum=keep["spectrum"].data_ptr(), spec_bins=B, spec_nu_lo=float(spec.spec_nu_lo),
        spec_nu_hi=float(spec.spec_nu_hi), stats=keep["stats"].data_ptr())
    if spec.line_mode == 1:
        row = spec.ion.astype(np.int64) * spec.n_levels + spec.upper
        keep["line_row"] = _device(torch, row, np.int32)
        keep["dbr_offset"] = _device(torch, spec.dbr_offset.astype(np.int64), np.int64).to(torch.int32)
        keep["dbr_line"] = _device(torch, spec.dbr_line.astype(np.int64), np.int64).to(torch.int32)
        keep["dbr_cdf"] = _device(torch, spec.dbr_cdf, np.float64)
        args.line_row = keep["line_row"].data_ptr()
        args.dbr_offset = keep["dbr_offset"].data_ptr()
        args.dbr_line = keep["dbr_line"].data_ptr()
        args.dbr_cdf = keep["dbr_cdf"].data_ptr()
    if spec.j_blue:
        keep["j_blue"] = torch.empty(S * L, dtype=torch.float64, device="cuda")
        args.j_blue = keep["j_blue"].data_ptr()
    stream = torch.cuda.current_stream().cuda_stream
    om = oracle.OracleModel(spec, tau=tau)
    pool = _DefaultPool(torch)
    for iteration in (0, 1):
        args.iteration = iteration
        if iteration == 1:  # the set-up happened in the first call: this one allocates nothing
            before = _memory_state(torch)
            used_before = pool.get(pool.USED_CURRENT)
            pool.reset_high()
        mc.mc_transport_noalloc(args, stream)
        torch.cuda.synchronize()
        if iteration == 1:
            assert _memory_state(torch) == before
            assert pool.get(pool.USED_CURRENT) == used_before
            assert pool.get(pool.USED_HIGH) <= used_before
        got = {k: keep[k].cpu().numpy() for k in ("j_est", "nu_bar", "spectrum", "stats")}
        j, nb, jb, sp, st = _model_reference(mc, spec, tau, spec.seed, iteration, n)
        _close(got["j_est"], j, EST_RTOL)
        _close(got["nu_bar"], nb, EST_RTOL)
        _close(got["spectrum"], sp, EST_RTOL)
        if spec.j_blue:
            _close(keep["j_blue"].cpu().numpy().reshape(S, L), jb, EST_RTOL)
        want = [st[k] for k in ("escaped", "reabsorbed", "capped", "segments", "line_checks",
                                "resonances", "line_interactions", "e_scatters", "shell_crossings")]
        assert list(map(int, got["stats"])) == want
        # and the oracle, on the same inputs and draws
        r = oracle.run_iteration(om, spec.seed, iteration, n, spec.t_inner, threads=os.cpu_count() or 1,
                                 record=False)
        _close(got["j_est"], r.j_est, EST_RTOL)
        _close(got["nu_bar"], r.nu_bar, EST_RTOL)
        _close(got["spectrum"], r.spectrum, EST_RTOL)
        if spec.j_blue:
            _close(keep["j_blue"].cpu().numpy().reshape(S, L), r.j_blue, EST_RTOL)
        assert list(map(int, got["stats"])) == [r.stats[k] for k in oracle.STAT_NAMES]


def test_noalloc_rejects_too_many_shells(env):
    torch, mc = env
    args = mc.mc_noalloc_args(n_shells=mc.MC_NOALLOC_MAX_SHELLS + 1, n_lines=1)
    with pytest.raises(mc.MCError) as ei:
        mc.mc_transport_noalloc(args, None)
    assert ei.value.code == mc.MC_ERR_INVALID_ARG
    assert "MC_NOALLOC_MAX_SHELLS" in str(ei.value)


_FIRST_CALL_UNDER_CAPTURE = r"""
import sys
import torch
from paper_1401_5469_gb300 import mc
mc.load()
args = mc.mc_noalloc_args(n_shells=1, n_lines=1, spec_bins=10)
dummy = torch.zeros(64, dtype=torch.float64, device="cuda")
for name in ("v_inner", "v_outer", "n_e", "nu", "tau", "j_est", "nu_bar", "spectrum"):
    setattr(args, name, dummy.data_ptr())
args.v_inner_0, args.t_exp, args.t_inner, args.n_packets = 1e9, 1e6, 1e4, 10
args.spec_nu_lo, args.spec_nu_hi = 1e14, 3e15
torch.cuda.synchronize()
g = torch.cuda.CUDAGraph()
code = None
try:
    with torch.cuda.graph(g):
        try:
            mc.mc_transport_noalloc(args, torch.cuda.current_stream().cuda_stream)
        except mc.MCError as e:
            code = e.code
            print("refused:", e)
except Exception as e:  # an empty capture may be reported on exit
    print("capture end:", type(e).__name__)
sys.exit(0 if code == mc.MC_ERR_INVALID_ARG else 1)
"""


def test_noalloc_first_call_refused_while_capturing(env):
    """The first call on a device runs a set-up kernel; made on a capturing
    stream it would land in a graph that may never run, so it is refused
    (checked in a fresh process, where the call is the first on the device)."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FIRST_CALL_UNDER_CAPTURE], cwd=root, capture_output=True,
                       text=True, timeout=300, env={**os.environ, "PYTHONPATH": root})
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-2000:])
    assert "capturing" in r.stdout
