"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point declared in include/mc_transport.h, and rejects invalid
models before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1401_5469_gb300 import mc, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "mc_transport.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mc_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = mc.load()
    names = _declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(L, n), n
    assert set(mc.EXPORTED) <= set(names)


def test_status_strings():
    L = mc.load()
    for code in (0, -1, -2, -3, -4, -5, -6, 1):
        assert L.mc_status_string(code).decode()


def _descs(spec, **run_kw):
    keep = []
    f64 = lambda a: keep.append(np.ascontiguousarray(a, np.float64)) or keep[-1].ctypes.data
    g = mc.mc_geometry_desc(n_shells=spec.n_shells, v_inner=f64(spec.v_inner), v_outer=f64(spec.v_outer),
                            n_e=f64(spec.n_e), t_exp=spec.t_exp)
    l = mc.mc_line_desc(n_lines=spec.n_lines, nu=f64(spec.nu))
    r = mc.mc_run_desc(line_mode=0, precision=0, j_blue=0, record_packets=0, spec_bins=10,
                       spec_nu_lo=1e14, spec_nu_hi=3e15, max_packets=100, max_segments=0, delta_t=1.0)
    for k, v in run_kw.items():
        setattr(r, k, v)
    return g, l, r, keep


@pytest.mark.parametrize("mutate,expect", [
    ("nu_ascending", mc.MC_ERR_INVALID_ARG),
    ("negative_ne", mc.MC_ERR_INVALID_ARG),
    ("gap", mc.MC_ERR_INVALID_ARG),
    ("bad_mode", mc.MC_ERR_INVALID_ARG),
    ("no_bins", mc.MC_ERR_INVALID_ARG),
    ("downbranch_without_table", mc.MC_ERR_INVALID_ARG),
    ("too_many_shells", mc.MC_ERR_INVALID_ARG),
])
def test_create_rejects_invalid_models(mutate, expect):
    spec = synth.scatter_model(n_lines=50, n_shells=4)
    if mutate == "nu_ascending":
        spec.nu = spec.nu[::-1].copy()
    elif mutate == "negative_ne":
        spec.n_e = spec.n_e.copy()
        spec.n_e[1] = -1.0
    elif mutate == "gap":
        spec.v_inner = spec.v_inner.copy()
        spec.v_inner[2] *= 1.01
    elif mutate == "too_many_shells":
        spec = synth.scatter_model(n_lines=50, n_shells=1025)
    g, l, r, keep = _descs(spec)
    if mutate == "bad_mode":
        r.line_mode = 7
    elif mutate == "no_bins":
        r.spec_bins = 0
    elif mutate == "downbranch_without_table":
        r.line_mode = 1
    L = mc.load()
    h = C.c_void_p()
    rc = L.mc_model_create(C.byref(g), C.byref(l), None, C.byref(r), None, None, C.byref(h))
    assert rc == expect
    assert not h.value
    assert L.mc_last_error_message(None).decode()


def test_batch_calls_reject_null_arguments():
    L = mc.load()
    c = mc.mc_batch_launch(128, 0, 0)
    assert L.mc_batch_set_launch(None, C.byref(c)) == mc.MC_ERR_INVALID_ARG
    assert L.mc_batch_get_launch(None, C.byref(c)) == mc.MC_ERR_INVALID_ARG
    assert L.mc_batch_autotune(None, None, None, None, None, None, None, None) == mc.MC_ERR_INVALID_ARG
    assert L.mc_batch_run_iteration(None, None, None, None, None, 1) == mc.MC_ERR_INVALID_ARG
    assert L.mc_batch_capture_graph(None, 1) == mc.MC_ERR_INVALID_ARG
    assert L.mc_cancel(None, 1) == mc.MC_ERR_INVALID_ARG
    h = C.c_void_p()
    assert L.mc_batch_create(None, 0, C.byref(h)) == mc.MC_ERR_INVALID_ARG
    assert not h.value


def test_t_inner_update_matches_the_oracle():
    import oracle
    for t, lr, le in ((9000.0, 4e42, 3.1e42), (12000.0, 1e41, 2e41), (8000.0, 1e42, 0.0)):
        assert mc.t_inner_update(t, lr, le) == oracle.t_inner_update(t, lr, le)


def _full_descs(spec):
    g, l, r, keep = _descs(spec, line_mode=int(spec.line_mode))
    for name in ("f", "ion", "lower", "upper"):
        a = getattr(spec, name)
        arr = np.ascontiguousarray(a, np.float64 if name == "f" else np.int32)
        keep.append(arr)
        setattr(l, name, arr.ctypes.data)
    a = mc.atomic_desc(spec, keep)
    return g, l, a, r, keep


@pytest.mark.parametrize("mutate,message", [
    ("mode", "ionization_mode"),
    ("one_stage", "ionization needs"),
    ("too_many_stages", "ionization needs"),
    ("bare_stage_ion", "out of range"),
    ("duplicate", "same (element, stage)"),
    ("chi", "ionization potentials"),
    ("zeta", "zeta"),
    ("no_zeta", "ionization needs"),
    ("delta", "delta"),
    ("n_element", "element densities"),
    ("fixed_without_n_ion", "atomic data needs"),
])
def test_create_rejects_invalid_ionization_data(mutate, message):
    spec = synth.nebular_model(mode=2, n_lines=300, n_shells=4, n_packets=10)
    if mutate == "one_stage":
        spec.n_stages = 1
    elif mutate == "too_many_stages":
        spec.n_stages = 17
    elif mutate == "bare_stage_ion":
        spec.ion_stage = spec.ion_stage.copy()
        spec.ion_stage[0] = spec.n_stages - 1
    elif mutate == "duplicate":
        spec.ion_stage = spec.ion_stage.copy()
        spec.ion_stage[1] = spec.ion_stage[0]
    elif mutate == "chi":
        spec.chi_ev = spec.chi_ev.copy()
        spec.chi_ev[0, 1] = 0.0
    elif mutate == "zeta":
        spec.zeta = spec.zeta.copy()
        spec.zeta[1, 0] = 1.5
    elif mutate == "no_zeta":
        spec.zeta = None
    elif mutate == "delta":
        spec.delta = 0.0
    elif mutate == "n_element":
        spec.n_element = spec.n_element.copy()
        spec.n_element[2, 0] = -1.0
    elif mutate == "fixed_without_n_ion":
        spec.ionization_mode = 0
        spec.n_ion = None
    g, l, a, r, keep = _full_descs(spec)
    if mutate == "mode":
        a.ionization_mode = 3
    L = mc.load()
    h = C.c_void_p()
    rc = L.mc_model_create(C.byref(g), C.byref(l), C.byref(a), C.byref(r), None, None, C.byref(h))
    assert rc == mc.MC_ERR_INVALID_ARG
    assert not h.value
    assert message in L.mc_last_error_message(None).decode()


def test_ionization_descriptor_matches_the_model():
    spec = synth.nebular_model(mode=1, n_lines=300, n_shells=4, n_packets=10)
    keep = []
    a = mc.atomic_desc(spec, keep)
    assert (a.ionization_mode, a.n_elements, a.n_stages) == (mc.MC_ION_SAHA, spec.n_elements, spec.n_stages)
    assert a.n_element == keep[-1].ctypes.data and keep[-1].shape == (4, spec.n_elements)
    assert a.delta == 1.0


def test_model_calls_reject_a_null_model():
    """Every per-model entry point answers a NULL handle with
    MC_ERR_INVALID_ARG before touching the device (destroy is a no-op)."""
    L = mc.load()
    inv = mc.MC_ERR_INVALID_ARG
    assert L.mc_set_plasma(None, None, None, None) == inv
    assert L.mc_run_iteration(None, 1, 0, 10, 1e4) == inv
    assert L.mc_run_iteration_range(None, 1, 0, 0, 10, 10, 1e4) == inv
    assert L.mc_update_radiation_field(None, None, None) == inv
    assert L.mc_read_estimators(None, None, None, None, None) == inv
    assert L.mc_read_spectrum(None, None, None) == inv
    assert L.mc_read_packets(None, 0, 1, None, None, None, None) == inv
    assert L.mc_read_plasma(None, None, None, None) == inv
    assert L.mc_read_ionization(None, None, None) == inv
    assert L.mc_synchronize(None) == inv
    L.mc_model_destroy(None)


@pytest.mark.parametrize("field,value", [("n_lines", 2**31), ("spec_bins", 2**31 - 2), ("n_shells", 0)])
def test_noalloc_rejects_out_of_range_sizes_before_device_work(field, value):
    """mc_transport_noalloc checks its sizes on the host before any CUDA call
    (counts that would not fit the kernels' signed 32-bit sizes included)."""
    args = mc.mc_noalloc_args(n_shells=1, n_lines=1, spec_bins=10)
    setattr(args, field, value)
    with pytest.raises(mc.MCError) as ei:
        mc.mc_transport_noalloc(args, None)
    assert ei.value.code == mc.MC_ERR_INVALID_ARG
