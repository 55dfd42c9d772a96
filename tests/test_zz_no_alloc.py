"""The allocation-free transport entry point (mc_transport_noalloc).

It exists for callers that cannot allocate device memory where they run the
transport (a framework's fixed memory pool, a plug-in handed raw buffers, a
loop that must not allocate).  They pass every buffer; the kernel's working
memory is a static device array inside the library.  Here the caller's
buffers come from torch, and two calls in a row (iterations 0 and 1) are
checked against the model-based entry point (mc_run_iteration) with the
tolerances of the parity tests: estimators and spectrum to 1e-9 relative,
run statistics exactly.  The second call also shows that the shared scratch
is cleared between calls.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

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
    for iteration in (0, 1):
        args.iteration = iteration
        mc.mc_transport_noalloc(args, stream)
        torch.cuda.synchronize()
        j, nb, jb, sp, st = _model_reference(mc, spec, tau, spec.seed, iteration, n)
        _close(keep["j_est"].cpu().numpy(), j, EST_RTOL)
        _close(keep["nu_bar"].cpu().numpy(), nb, EST_RTOL)
        _close(keep["spectrum"].cpu().numpy(), sp, EST_RTOL)
        if spec.j_blue:
            _close(keep["j_blue"].cpu().numpy().reshape(S, L), jb, EST_RTOL)
        got = keep["stats"].cpu().numpy()
        want = [st[k] for k in ("escaped", "reabsorbed", "capped", "segments", "line_checks",
                                "resonances", "line_interactions", "e_scatters", "shell_crossings")]
        assert list(map(int, got)) == want


def test_noalloc_rejects_too_many_shells(env):
    torch, mc = env
    args = mc.mc_noalloc_args(n_shells=mc.MC_NOALLOC_MAX_SHELLS + 1, n_lines=1)
    with pytest.raises(mc.MCError) as ei:
        mc.mc_transport_noalloc(args, None)
    assert ei.value.code == mc.MC_ERR_INVALID_ARG
    assert "MC_NOALLOC_MAX_SHELLS" in str(ei.value)
