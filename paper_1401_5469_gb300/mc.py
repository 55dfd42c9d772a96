"""Python binding of the C ABI in ``include/mc_transport.h`` (ctypes).

Argument marshalling only: every computation runs in the CUDA library
``_lib/libmc_gb300.so``.  The functions keep the C names (``mc_model_create``,
``mc_set_plasma``, ``mc_run_iteration``, ...); ``Model`` wraps them for a
``synth.ModelSpec``.  PyTorch is used only for the CUDA stream (the model's
work is enqueued on torch's current stream) and, optionally, for device memory
through torch's caching allocator.  Importing this module without the built
library raises ``ImportError``: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import build as _build

MC_OK = 0
MC_ERR_INVALID_ARG = -1
MC_ERR_OOM = -2
MC_ERR_CUDA = -3
MC_ERR_NOT_READY = -4
MC_ERR_TIMEOUT = -5
MC_ERR_UNSUPPORTED = -6
MC_WARN_CAPPED = 1
MC_LINE_SCATTER, MC_LINE_DOWNBRANCH = 0, 1
MC_PRECISION_FP64, MC_PRECISION_MIXED = 0, 1
MC_LINE_SCATTER, MC_LINE_DOWNBRANCH, MC_LINE_MACROATOM = 0, 1, 2
MC_ION_FIXED, MC_ION_SAHA, MC_ION_NEBULAR = 0, 1, 2
MC_PACKET_ESCAPED, MC_PACKET_REABSORBED, MC_PACKET_CAPPED = 1, 2, 3
MC_N_COUNTERS = 6
COUNTER_NAMES = ("segments", "line_checks", "resonances", "line_interactions", "e_scatters",
                 "shell_crossings")

# Every entry point declared in include/mc_transport.h.
EXPORTED = ("mc_model_create", "mc_set_plasma", "mc_run_iteration", "mc_run_iteration_range",
            "mc_update_radiation_field",
            "mc_read_estimators", "mc_read_spectrum", "mc_read_packets", "mc_read_plasma",
            "mc_read_ionization", "mc_cancel",
            "mc_read_timing", "mc_read_transport_phases", "mc_launch_count", "mc_synchronize", "mc_model_destroy",
            "mc_status_string", "mc_last_error_message", "mc_transport_noalloc",
            "mc_batch_create", "mc_batch_run_iteration", "mc_batch_synchronize",
            "mc_batch_read_timing", "mc_batch_read_phases", "mc_batch_last_error_message", "mc_batch_destroy",
            "mc_batch_set_launch", "mc_batch_get_launch", "mc_batch_autotune", "mc_batch_capture_graph",
            "mc_device_estimators", "mc_set_virtual_packets", "mc_read_virtual_spectrum",
            "mc_t_inner_from_luminosity", "mc_emitted_luminosity", "mc_t_inner_update",
            "mc_selftest_math")

MC_ORDER_PACKETS, MC_ORDER_WORK, MC_ORDER_GIVEN = 0, 1, 2
MC_MATH_NEG_LOG_U53, MC_MATH_LOG, MC_MATH_RCP, MC_MATH_SQRT, MC_MATH_APPROX = 0, 1, 2, 3, 4


class mc_geometry_desc(C.Structure):
    _fields_ = [("n_shells", C.c_uint32), ("v_inner", C.c_void_p), ("v_outer", C.c_void_p),
                ("n_e", C.c_void_p), ("t_exp", C.c_double)]


class mc_line_desc(C.Structure):
    _fields_ = [("n_lines", C.c_uint32), ("nu", C.c_void_p), ("f", C.c_void_p),
                ("ion", C.c_void_p), ("lower", C.c_void_p), ("upper", C.c_void_p)]


class mc_atomic_desc(C.Structure):
    _fields_ = [("n_ions", C.c_uint32), ("n_levels", C.c_uint32), ("energy_ev", C.c_void_p),
                ("g", C.c_void_p), ("metastable", C.c_void_p), ("n_ion", C.c_void_p),
                ("dbr_offset", C.c_void_p), ("dbr_line", C.c_void_p), ("dbr_cdf", C.c_void_p),
                ("lte_excitation", C.c_int32),
                ("ma_jump_p", C.c_void_p), ("ma_jump_offset", C.c_void_p), ("ma_jump_target", C.c_void_p),
                ("ma_jump_cdf", C.c_void_p),
                ("ionization_mode", C.c_int32), ("n_elements", C.c_uint32), ("n_stages", C.c_uint32),
                ("ion_element", C.c_void_p), ("ion_stage", C.c_void_p), ("chi_ev", C.c_void_p),
                ("zeta", C.c_void_p), ("delta", C.c_double), ("n_element", C.c_void_p)]


class mc_run_desc(C.Structure):
    _fields_ = [("line_mode", C.c_int32), ("precision", C.c_int32), ("j_blue", C.c_int32),
                ("record_packets", C.c_int32), ("spec_bins", C.c_uint32),
                ("spec_nu_lo", C.c_double), ("spec_nu_hi", C.c_double),
                ("max_packets", C.c_uint64), ("max_segments", C.c_uint64),
                ("delta_t", C.c_double), ("timeout_ns", C.c_uint64)]


class mc_noalloc_args(C.Structure):
    """Arguments of mc_transport_noalloc: every pointer is a device pointer."""
    _fields_ = [("n_shells", C.c_uint32), ("v_inner", C.c_void_p), ("v_outer", C.c_void_p),
                ("n_e", C.c_void_p), ("v_inner_0", C.c_double), ("t_exp", C.c_double),
                ("n_lines", C.c_uint32), ("nu", C.c_void_p), ("tau", C.c_void_p),
                ("line_mode", C.c_int32), ("line_row", C.c_void_p), ("dbr_offset", C.c_void_p),
                ("dbr_line", C.c_void_p), ("dbr_cdf", C.c_void_p), ("seed", C.c_uint64),
                ("iteration", C.c_uint32), ("n_packets", C.c_uint64), ("t_inner", C.c_double),
                ("max_segments", C.c_uint64), ("delta_t", C.c_double), ("j_est", C.c_void_p),
                ("nu_bar", C.c_void_p), ("j_blue", C.c_void_p), ("spectrum", C.c_void_p),
                ("spec_bins", C.c_uint32), ("spec_nu_lo", C.c_double), ("spec_nu_hi", C.c_double),
                ("stats", C.c_void_p)]


MC_NOALLOC_MAX_SHELLS = 1024


class mc_estimator_views(C.Structure):
    _fields_ = [("j_est", C.c_void_p), ("nu_bar", C.c_void_p), ("j_blue", C.c_void_p),
                ("spectrum", C.c_void_p), ("n_shells", C.c_uint32), ("n_lines", C.c_uint32),
                ("spec_bins", C.c_uint32), ("stream", C.c_void_p)]


class _DeviceArray:
    """A non-owning device buffer exposed through __cuda_array_interface__."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f8",
                                         "data": (int(ptr), False), "version": 3, "strides": None}


class mc_batch_launch(C.Structure):
    _fields_ = [("block", C.c_uint32), ("blocks_per_sm", C.c_uint32), ("order", C.c_uint32)]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class mc_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class mc_packet_stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("packets", "escaped", "reabsorbed", "capped", "segments",
                                          "line_checks", "resonances", "line_interactions",
                                          "e_scatters", "shell_crossings")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"CUDA library not built: {_build.LIB}")
    L = C.CDLL(_build.LIB)
    vp, i32, u32, u64, d = C.c_void_p, C.c_int32, C.c_uint32, C.c_uint64, C.c_double
    P = C.POINTER
    L.mc_model_create.restype = i32
    L.mc_model_create.argtypes = [P(mc_geometry_desc), P(mc_line_desc), P(mc_atomic_desc),
                                  P(mc_run_desc), P(mc_allocator), vp, P(vp)]
    L.mc_set_plasma.restype = i32
    L.mc_set_plasma.argtypes = [vp, vp, vp, vp]
    L.mc_run_iteration.restype = i32
    L.mc_run_iteration.argtypes = [vp, u64, u32, u64, d]
    L.mc_run_iteration_range.restype = i32
    L.mc_run_iteration_range.argtypes = [vp, u64, u32, u64, u64, u64, d]
    L.mc_update_radiation_field.restype = i32
    L.mc_update_radiation_field.argtypes = [vp, vp, vp]
    L.mc_read_estimators.restype = i32
    L.mc_read_estimators.argtypes = [vp, vp, vp, vp, vp]
    L.mc_read_spectrum.restype = i32
    L.mc_read_spectrum.argtypes = [vp, vp, P(mc_packet_stats)]
    L.mc_read_packets.restype = i32
    L.mc_read_packets.argtypes = [vp, u64, u64, vp, vp, vp, vp]
    L.mc_read_plasma.restype = i32
    L.mc_read_plasma.argtypes = [vp, vp, vp, vp]
    L.mc_read_ionization.restype = i32
    L.mc_read_ionization.argtypes = [vp, vp, vp]
    L.mc_cancel.restype = i32
    L.mc_cancel.argtypes = [vp, i32]
    L.mc_read_timing.restype = i32
    L.mc_read_timing.argtypes = [vp, vp]
    L.mc_read_transport_phases.restype = i32
    L.mc_read_transport_phases.argtypes = [vp, vp]
    L.mc_launch_count.restype = i32
    L.mc_launch_count.argtypes = [vp, P(u64)]
    L.mc_synchronize.restype = i32
    L.mc_synchronize.argtypes = [vp]
    L.mc_model_destroy.restype = None
    L.mc_model_destroy.argtypes = [vp]
    L.mc_status_string.restype = C.c_char_p
    L.mc_status_string.argtypes = [i32]
    L.mc_last_error_message.restype = C.c_char_p
    L.mc_last_error_message.argtypes = [vp]
    L.mc_transport_noalloc.restype = i32
    L.mc_transport_noalloc.argtypes = [P(mc_noalloc_args), vp]
    L.mc_batch_create.restype = i32
    L.mc_batch_create.argtypes = [vp, u32, P(vp)]
    L.mc_batch_run_iteration.restype = i32
    L.mc_batch_run_iteration.argtypes = [vp, vp, vp, vp, vp, i32]
    L.mc_batch_synchronize.restype = i32
    L.mc_batch_synchronize.argtypes = [vp]
    L.mc_batch_read_timing.restype = i32
    L.mc_batch_read_timing.argtypes = [vp, vp]
    L.mc_batch_read_phases.restype = i32
    L.mc_batch_read_phases.argtypes = [vp, vp]
    L.mc_batch_last_error_message.restype = C.c_char_p
    L.mc_batch_last_error_message.argtypes = [vp]
    L.mc_batch_destroy.restype = None
    L.mc_batch_destroy.argtypes = [vp]
    L.mc_t_inner_from_luminosity.restype = i32
    L.mc_t_inner_from_luminosity.argtypes = [vp, d, P(d)]
    L.mc_emitted_luminosity.restype = i32
    L.mc_emitted_luminosity.argtypes = [vp, P(d)]
    L.mc_t_inner_update.restype = d
    L.mc_t_inner_update.argtypes = [d, d, d]
    L.mc_set_virtual_packets.restype = i32
    L.mc_set_virtual_packets.argtypes = [vp, u32, d]
    L.mc_read_virtual_spectrum.restype = i32
    L.mc_read_virtual_spectrum.argtypes = [vp, vp]
    L.mc_device_estimators.restype = i32
    L.mc_device_estimators.argtypes = [vp, P(mc_estimator_views)]
    L.mc_batch_set_launch.restype = i32
    L.mc_batch_set_launch.argtypes = [vp, P(mc_batch_launch)]
    L.mc_batch_get_launch.restype = i32
    L.mc_batch_get_launch.argtypes = [vp, P(mc_batch_launch)]
    L.mc_batch_capture_graph.restype = i32
    L.mc_batch_capture_graph.argtypes = [vp, i32]
    L.mc_batch_autotune.restype = i32
    L.mc_batch_autotune.argtypes = [vp, vp, vp, vp, vp, P(mc_batch_launch), vp, vp]
    L.mc_selftest_math.restype = i32
    L.mc_selftest_math.argtypes = [i32, vp, u64, vp, vp]
    _lib = L
    return L


class MCError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


def _p(a):
    return None if a is None else a.ctypes.data


def _check(code, handle=None, allow_warn=True):
    if code == MC_OK or (allow_warn and code > 0):
        return code
    L = load()
    msg = L.mc_last_error_message(handle).decode() or L.mc_status_string(code).decode()
    raise MCError(code, msg)


# ----------------------------------------------------------------- raw C names

def mc_model_create(geom, lines, atomic, run, alloc=None, stream=None):
    L = load()
    h = C.c_void_p()
    rc = L.mc_model_create(C.byref(geom), C.byref(lines), C.byref(atomic) if atomic else None,
                           C.byref(run), C.byref(alloc) if alloc else None, stream, C.byref(h))
    _check(rc, None)
    return h


def mc_set_plasma(h, t_rad=None, w=None, tau=None):
    return _check(load().mc_set_plasma(h, _p(t_rad), _p(w), _p(tau)), h)


def mc_run_iteration(h, seed, iteration, n_packets, t_inner):
    return _check(load().mc_run_iteration(h, seed, iteration, n_packets, float(t_inner)), h)


def mc_run_iteration_range(h, seed, iteration, first_packet, n_packets, n_total, t_inner):
    return _check(load().mc_run_iteration_range(h, seed, iteration, first_packet, n_packets, n_total,
                                                float(t_inner)), h)


def mc_update_radiation_field(h, t_rad_out=None, w_out=None):
    return _check(load().mc_update_radiation_field(h, _p(t_rad_out), _p(w_out)), h)


def mc_read_estimators(h, j_est=None, nu_bar=None, j_blue=None, norm=None):
    return _check(load().mc_read_estimators(h, _p(j_est), _p(nu_bar), _p(j_blue), _p(norm)), h)


def mc_read_spectrum(h, spectrum=None, stats=None):
    return _check(load().mc_read_spectrum(h, _p(spectrum), C.byref(stats) if stats is not None else None), h)


def mc_read_packets(h, first, count, status=None, nu=None, energy=None, counters=None):
    return _check(load().mc_read_packets(h, first, count, _p(status), _p(nu), _p(energy), _p(counters)), h)


def mc_read_plasma(h, t_rad=None, w=None, tau=None):
    return _check(load().mc_read_plasma(h, _p(t_rad), _p(w), _p(tau)), h)


def mc_read_ionization(h, n_e=None, n_ion=None):
    return _check(load().mc_read_ionization(h, _p(n_e), _p(n_ion)), h)


def mc_read_timing(h):
    ms = np.zeros(3, dtype=np.float32)
    _check(load().mc_read_timing(h, _p(ms)), h)
    return ms


def mc_read_transport_phases(h):
    ms = np.zeros(2, dtype=np.float32)
    _check(load().mc_read_transport_phases(h, _p(ms)), h)
    return ms


def mc_launch_count(h):
    c = C.c_uint64(0)
    _check(load().mc_launch_count(h, C.byref(c)), h)
    return int(c.value)


def mc_synchronize(h):
    return _check(load().mc_synchronize(h), h)


def mc_model_destroy(h):
    load().mc_model_destroy(h)


def mc_transport_noalloc(args, stream=None):
    """One transport launch on caller-owned device buffers; allocates nothing."""
    return _check(load().mc_transport_noalloc(C.byref(args), stream), None)


def mc_selftest_math(fn, values):
    """The kernels' own device arithmetic next to CUDA's (accuracy diagnostic):
    returns (ours, ref) for the host input array ``values`` (uint64 draws for
    MC_MATH_NEG_LOG_U53, binary64 otherwise)."""
    dt = np.uint64 if fn == MC_MATH_NEG_LOG_U53 else np.float64
    x = np.ascontiguousarray(values, dtype=dt)
    ours, ref = np.empty(x.size), np.empty(x.size)
    _check(load().mc_selftest_math(int(fn), _p(x), x.size, _p(ours), _p(ref)), None)
    return ours, ref


# ----------------------------------------------------------------- torch plumbing

def _torch_stream_handle():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class _TorchAllocator:
    """mc_allocator backed by torch's CUDA caching allocator."""

    def __init__(self, stream_handle):
        import torch
        self._torch = torch
        self._dev = torch.cuda.current_device()
        self._stream = stream_handle.value

        def _alloc(nbytes, ctx):
            try:
                return int(self._torch.cuda.caching_allocator_alloc(nbytes, self._dev, self._stream))
            except Exception:  # noqa: BLE001 -- report OOM through the C status
                return None

        def _free(ptr, ctx):
            self._torch.cuda.caching_allocator_delete(ptr)

        self._a = ALLOC_FN(_alloc)
        self._f = FREE_FN(_free)
        self.c = mc_allocator(alloc=self._a, free=self._f, ctx=None)


# ----------------------------------------------------------------- Model wrapper

def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


def _u32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.uint32)


def atomic_desc(spec, keep):
    """The mc_atomic_desc of a ``synth.ModelSpec`` (None without atomic data);
    the arrays it points to are appended to ``keep``."""
    if spec.energy_ev is None:
        return None
    e, g = _f64(spec.energy_ev), _f64(spec.g)
    meta = np.ascontiguousarray(spec.metastable, dtype=np.uint8)
    nion = _f64(spec.n_ion) if spec.n_ion is not None else None
    off, dl, cdf = _u32(spec.dbr_offset), _u32(spec.dbr_line), _f64(spec.dbr_cdf)
    keep += [e, g, meta, nion, off, dl, cdf]
    jp = jo = jt = jc = None
    if getattr(spec, "ma_jump_p", None) is not None:
        jp, jo = _f64(spec.ma_jump_p), _u32(spec.ma_jump_offset)
        jt, jc = _i32(spec.ma_jump_target), _f64(spec.ma_jump_cdf)
        keep += [jp, jo, jt, jc]
    a = mc_atomic_desc(n_ions=int(spec.n_ions), n_levels=int(spec.n_levels),
                       energy_ev=_p(e), g=_p(g), metastable=_p(meta),
                       n_ion=_p(nion), dbr_offset=_p(off), dbr_line=_p(dl),
                       dbr_cdf=_p(cdf), lte_excitation=0,
                       ma_jump_p=_p(jp), ma_jump_offset=_p(jo),
                       ma_jump_target=_p(jt), ma_jump_cdf=_p(jc))
    mode = int(getattr(spec, "ionization_mode", 0) or 0)
    if mode:
        ie, ist = _i32(spec.ion_element), _i32(spec.ion_stage)
        chi, nel = _f64(spec.chi_ev), _f64(spec.n_element)
        zeta = _f64(spec.zeta) if spec.zeta is not None else None
        keep += [ie, ist, chi, zeta, nel]
        a.ionization_mode, a.n_elements, a.n_stages = mode, int(spec.n_elements), int(spec.n_stages)
        a.ion_element, a.ion_stage = _p(ie), _p(ist)
        a.chi_ev, a.zeta, a.n_element = _p(chi), _p(zeta), _p(nel)
        a.delta = float(spec.delta)
    return a


class Model:
    """One ejecta model resident on the GPU (wraps a ``synth.ModelSpec``)."""

    def __init__(self, spec, precision: int = MC_PRECISION_FP64, record_packets: bool = False,
                 max_packets: Optional[int] = None, max_segments: int = 1_000_000,
                 j_blue: Optional[bool] = None, use_torch_allocator: bool = True,
                 timeout_ns: int = 0, stream=None):
        self.spec = spec
        self._keep = []
        k = self._keep
        vi, vo, ne = _f64(spec.v_inner), _f64(spec.v_outer), _f64(spec.n_e)
        nu = _f64(spec.nu)
        k += [vi, vo, ne, nu]
        self.geom = mc_geometry_desc(n_shells=vi.size, v_inner=_p(vi), v_outer=_p(vo), n_e=_p(ne),
                                     t_exp=float(spec.t_exp))
        f, ion, lo, up = _f64(spec.f), _i32(spec.ion), _i32(spec.lower), _i32(spec.upper)
        k += [f, ion, lo, up]
        self.lines = mc_line_desc(n_lines=nu.size, nu=_p(nu), f=_p(f), ion=_p(ion), lower=_p(lo),
                                  upper=_p(up))
        self.atomic = atomic_desc(spec, k)
        jb = spec.j_blue if j_blue is None else j_blue
        mp = int(max_packets if max_packets is not None else spec.n_packets)
        self.run = mc_run_desc(line_mode=int(spec.line_mode), precision=int(precision),
                               j_blue=int(bool(jb)), record_packets=int(bool(record_packets)),
                               spec_bins=int(spec.spec_bins), spec_nu_lo=float(spec.spec_nu_lo),
                               spec_nu_hi=float(spec.spec_nu_hi), max_packets=mp,
                               max_segments=int(max_segments), delta_t=1.0,
                               timeout_ns=int(timeout_ns))
        self.S, self.L = vi.size, nu.size
        self.I = int(spec.n_ions) if self.atomic is not None else 0
        self.bins = int(spec.spec_bins)
        self.stream = stream if stream is not None else _torch_stream_handle()
        self._alloc = _TorchAllocator(self.stream) if use_torch_allocator else None
        self.h = mc_model_create(self.geom, self.lines, self.atomic, self.run,
                                 self._alloc.c if self._alloc else None, self.stream)

    def close(self):
        if getattr(self, "h", None):
            mc_model_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    # -- plasma and runs
    def set_plasma(self, t_rad=None, w=None, tau=None):
        t_rad, w = _f64(t_rad), _f64(w)
        tau = None if tau is None else _f64(tau).reshape(-1)
        return mc_set_plasma(self.h, t_rad, w, tau)

    def run_iteration(self, seed, iteration, n_packets, t_inner):
        return mc_run_iteration(self.h, int(seed), int(iteration), int(n_packets), float(t_inner))

    def run_iteration_range(self, seed, iteration, first, n_packets, n_total, t_inner):
        return mc_run_iteration_range(self.h, int(seed), int(iteration), int(first), int(n_packets),
                                      int(n_total), float(t_inner))

    def update_radiation_field(self):
        t, w = np.zeros(self.S), np.zeros(self.S)
        mc_update_radiation_field(self.h, t, w)
        return t, w

    def estimators(self, j_blue=False):
        j, nb, norm = np.zeros(self.S), np.zeros(self.S), np.zeros(self.S)
        jb = np.zeros((self.S, self.L)) if j_blue else None
        mc_read_estimators(self.h, j, nb, jb, norm)
        return j, nb, jb, norm

    def t_inner_from_luminosity(self, l_outer: float) -> float:
        """Eq. 18: T_inner whose inner-boundary luminosity is l_outer."""
        t = C.c_double()
        _check(load().mc_t_inner_from_luminosity(self.h, float(l_outer), C.byref(t)), self.h)
        return t.value

    def emitted_luminosity(self) -> float:
        """Lab-frame energy of the last iteration's escaping packets per unit time."""
        v = C.c_double()
        _check(load().mc_emitted_luminosity(self.h, C.byref(v)), self.h)
        return v.value

    def iterate(self, seed, n_iterations, n_packets, t_inner, first_iteration=0, l_requested=None,
                t_inner_every=3, on_iteration=None):
        """The iteration cycle of Sect. 2.8 through the C ABI: run, update T_R
        and W (Eqs. 15-16), and with l_requested, after every
        t_inner_every-th iteration, mc_t_inner_update with this iteration's
        emitted luminosity.  on_iteration(it, t_inner) is called after each
        run, before the update.  Returns the T_inner each iteration ran with
        and the one the next iteration would use."""
        used = []
        for it in range(first_iteration, first_iteration + n_iterations):
            self.run_iteration(seed, it, n_packets, t_inner)
            used.append(t_inner)
            if on_iteration is not None:
                on_iteration(it, t_inner)
            mc_update_radiation_field(self.h, None, None)
            if l_requested is not None and (it - first_iteration + 1) % t_inner_every == 0:
                t_inner = t_inner_update(t_inner, l_requested, self.emitted_luminosity())
        return used, t_inner

    def set_virtual_packets(self, n_virtual: int, tau_v_max: float = 0.0):
        """Virtual packets (Sect. 2.9) in the following iterations (0: off)."""
        return _check(load().mc_set_virtual_packets(self.h, int(n_virtual), float(tau_v_max)), self.h)

    def virtual_spectrum(self):
        """Raw v-spectrum sums of the last iteration ([bins + 2])."""
        sp = np.zeros(self.bins + 2)
        _check(load().mc_read_virtual_spectrum(self.h, _p(sp)), self.h)
        return sp

    def device_estimators(self):
        """Torch views (no copy) of the model's device estimator buffers:
        {"j_est", "nu_bar", "spectrum", "j_blue" (None when off), "stream"}."""
        import torch
        v = mc_estimator_views()
        _check(load().mc_device_estimators(self.h, C.byref(v)), self.h)
        dev = torch.device("cuda", torch.cuda.current_device())
        view = lambda ptr, n: torch.as_tensor(_DeviceArray(ptr, n), device=dev)
        return {"j_est": view(v.j_est, v.n_shells), "nu_bar": view(v.nu_bar, v.n_shells),
                "spectrum": view(v.spectrum, v.spec_bins + 2),
                "j_blue": view(v.j_blue, v.n_shells * v.n_lines) if v.j_blue else None,
                "stream": v.stream}

    def spectrum(self):
        sp = np.zeros(self.bins + 2)
        st = mc_packet_stats()
        rc = mc_read_spectrum(self.h, sp, st)
        return sp, st.as_dict(), rc

    def packets(self, first=0, count=None):
        if count is None:
            count = int(self.spectrum()[1]["packets"]) - first
        status = np.zeros(count, dtype=np.int32)
        nu, e = np.zeros(count), np.zeros(count)
        cnt = np.zeros((count, MC_N_COUNTERS), dtype=np.uint64)
        mc_read_packets(self.h, first, count, status, nu, e, cnt)
        return status, nu, e, cnt

    def plasma(self):
        t, w = np.zeros(self.S), np.zeros(self.S)
        tau = np.zeros((self.S, self.L))
        mc_read_plasma(self.h, t, w, tau)
        return t, w, tau

    def cancel(self, stop: bool = True):
        """mc_cancel: ask running and later launches to stop (or withdraw)."""
        return _check(load().mc_cancel(self.h, int(bool(stop))), self.h)

    def ionization(self):
        """mc_read_ionization: electron densities [S] and ion densities [S, I]
        the transport uses (the ionization balance in an ionization mode)."""
        n_e = np.zeros(self.S)
        n_ion = np.zeros((self.S, self.I)) if self.I else None
        mc_read_ionization(self.h, n_e, n_ion)
        return n_e, n_ion

    def timing(self):
        return mc_read_timing(self.h)

    def phases(self):
        return mc_read_transport_phases(self.h)

    def launches(self):
        return mc_launch_count(self.h)

    def synchronize(self):
        return mc_synchronize(self.h)


def t_inner_update(t_inner: float, l_requested: float, l_emitted: float) -> float:
    """mc_t_inner_update: T_inner (l_requested / l_emitted)^(1/4)."""
    return float(load().mc_t_inner_update(float(t_inner), float(l_requested), float(l_emitted)))


# ----------------------------------------------------------------- batches

class Batch:
    """Several mixed-precision Models advanced together (mc_batch_*)."""

    def __init__(self, models):
        self.models = list(models)
        L = load()
        arr = (C.c_void_p * len(self.models))(*[m.h.value for m in self.models])
        self._arr = arr
        h = C.c_void_p()
        rc = L.mc_batch_create(C.cast(arr, C.c_void_p), len(self.models), C.byref(h))
        _check(rc, None)
        self.h = h

    def _bcheck(self, rc):
        if rc == MC_OK or rc > 0:
            return rc
        msg = load().mc_batch_last_error_message(self.h).decode() or load().mc_status_string(rc).decode()
        raise MCError(rc, msg)

    def _args(self, seeds, iterations, n_packets, t_inner):
        n = len(self.models)
        s = np.ascontiguousarray(np.broadcast_to(np.asarray(seeds, dtype=np.uint64), (n,)))
        its = np.ascontiguousarray(np.broadcast_to(np.asarray(iterations, dtype=np.uint32), (n,)))
        npk = np.ascontiguousarray(np.broadcast_to(np.asarray(n_packets, dtype=np.uint64), (n,)))
        t = np.ascontiguousarray(np.broadcast_to(np.asarray(t_inner, dtype=np.float64), (n,)))
        return s, its, npk, t

    def run_iteration(self, seeds, iterations, n_packets, t_inner, update=True):
        """Model i runs its iteration iterations[i] with seeds[i] (scalars broadcast)."""
        s, its, npk, t = self._args(seeds, iterations, n_packets, t_inner)
        return self._bcheck(load().mc_batch_run_iteration(self.h, _p(s), _p(its), _p(npk), _p(t),
                                                          int(bool(update))))

    def set_launch(self, block=0, blocks_per_sm=0, order=MC_ORDER_PACKETS):
        c = mc_batch_launch(block, blocks_per_sm, order)
        return self._bcheck(load().mc_batch_set_launch(self.h, C.byref(c)))

    def capture_graph(self, enable=True):
        """mc_batch_capture_graph: replay a captured CUDA graph (default) or
        enqueue the kernels directly every iteration."""
        return self._bcheck(load().mc_batch_capture_graph(self.h, int(bool(enable))))

    def launch(self):
        c = mc_batch_launch()
        self._bcheck(load().mc_batch_get_launch(self.h, C.byref(c)))
        return c.as_dict()

    def autotune(self, seeds, iterations, n_packets, t_inner):
        """mc_batch_autotune: returns (launch shape, its transport ms, trials)."""
        s, its, npk, t = self._args(seeds, iterations, n_packets, t_inner)
        best = mc_batch_launch()
        ms = np.zeros(1, dtype=np.float32)
        nt = np.zeros(1, dtype=np.uint32)
        self._bcheck(load().mc_batch_autotune(self.h, _p(s), _p(its), _p(npk), _p(t), C.byref(best),
                                              _p(ms), _p(nt)))
        return best.as_dict(), float(ms[0]), int(nt[0])

    def synchronize(self):
        return self._bcheck(load().mc_batch_synchronize(self.h))

    def transport_ms(self):
        ms = np.zeros(1, dtype=np.float32)
        self._bcheck(load().mc_batch_read_timing(self.h, _p(ms)))
        return float(ms[0])

    def phases(self):
        """mc_batch_read_phases: (ms until the packet queue ran empty, ms of the tail)."""
        ms = np.zeros(2, dtype=np.float32)
        self._bcheck(load().mc_batch_read_phases(self.h, _p(ms)))
        return float(ms[0]), float(ms[1])

    def close(self):
        if getattr(self, "h", None):
            load().mc_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass
