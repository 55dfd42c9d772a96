"""CPU oracle of the Monte Carlo packet transport (Kerzendorf & Sim 2014, Sects. 2.3-2.8).

TEST INFRASTRUCTURE ONLY.  This package is imported by the test suite, by the
smoke check and by the CPU-baseline leg of the benchmark, and by nothing in
the product path.  It wraps ``mc_oracle.c`` -- a plain FP64 C program written
step by step from the paper -- through ctypes, and shares no code with the
CUDA library.

Functions and the passage each follows:

* ``run_iteration``       -- packet injection (Sect. 2.4, Eqs. 9-10), propagation
                             (Sect. 2.6, Eq. 11), line interactions (Sect. 2.5,
                             scatter / downbranch), estimators (Sect. 2.7,
                             Eqs. 13, 14, 17) and direct-binning spectrum (Sect. 2.9)
* ``level_populations``   -- Eqs. 4-5 (lte / dilute-lte excitation)
* ``sobolev_tau``         -- Eq. 12
* ``geometric_dilution``  -- Sect. 2.8 initial W
* ``update_radiation_field`` -- Eqs. 15-16
* ``log`` / ``exp``       -- own series (A&S 4.1.27; Cody & Waite 1980)
* ``philox`` / ``uniforms`` -- Philox4x32-10 (Salmon et al. 2011) draw stream
* ``distance_shell``      -- shell-crossing distance of Sect. 2.6
* ``ionization_state``    -- ionization balance, Eqs. 2-3 (lte / nebular modes)
* ``plasma_tau``          -- Eqs. 2-5 and 12 together (the plasma-state step)
* ``virtual_tau``         -- optical depth of a virtual packet's ray (Sect. 2.9, Eq. 21)
* ``macroatom_walks``     -- macro-atom internal jumps and deactivation (Sect. 2.5)
* ``t_inner_from_luminosity`` / ``emitted_luminosity`` / ``t_inner_update``
                          -- inner-boundary temperature (Sect. 2.8, Eq. 18)
* ``run_loop``            -- the iteration cycle of Sect. 2.8 (resumable from T_R, W)

Every function has pins in ``tests/test_oracle_*.py`` (Philox4x32-10 against
its published known-answer values, ``tests/golden/philox4x32_10_kat.txt``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mc_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

NCOUNT = 6
NSTATS = 9
COUNTER_NAMES = ("segments", "line_checks", "resonances", "line_interactions", "e_scatters",
                 "shell_crossings")
STAT_NAMES = ("escaped", "reabsorbed", "capped", "segments", "line_checks", "resonances",
              "line_interactions", "e_scatters", "shell_crossings")
IN_FLIGHT, ESCAPED, REABSORBED, CAPPED = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc: IEEE binary64, no FMA contraction."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Model(C.Structure):
    _fields_ = [
        ("n_shells", C.c_int32),
        ("v_inner", C.c_void_p), ("v_outer", C.c_void_p), ("n_e", C.c_void_p),
        ("t_exp", C.c_double),
        ("n_lines", C.c_int32),
        ("nu", C.c_void_p), ("tau", C.c_void_p),
        ("line_mode", C.c_int32),
        ("line_row", C.c_void_p), ("dbr_offset", C.c_void_p), ("dbr_line", C.c_void_p),
        ("dbr_cdf", C.c_void_p),
        ("j_blue", C.c_int32),
        ("spec_bins", C.c_int32),
        ("spec_nu_lo", C.c_double), ("spec_nu_hi", C.c_double),
        ("max_segments", C.c_uint64),
        ("delta_t", C.c_double),
        ("n_virtual", C.c_int32),
        ("tau_v_max", C.c_double),
        ("ma_jump_p", C.c_void_p), ("ma_jump_offset", C.c_void_p), ("ma_jump_target", C.c_void_p),
        ("ma_jump_cdf", C.c_void_p),
    ]


class _Result(C.Structure):
    _fields_ = [
        ("j_est", C.c_void_p), ("nu_bar", C.c_void_p), ("j_blue", C.c_void_p),
        ("spectrum", C.c_void_p),
        ("stats", C.c_uint64 * NSTATS),
        ("status", C.c_void_p), ("nu_out", C.c_void_p), ("e_out", C.c_void_p),
        ("counters", C.c_void_p),
        ("spectrum_v", C.c_void_p),
    ]


class _Event(C.Structure):
    _fields_ = [("kind", C.c_int32), ("line", C.c_int32), ("emit", C.c_int32), ("shell", C.c_int32)] + [
        (n, C.c_double) for n in ("x", "mu_before", "mu_after", "nu_lab_before", "nu_lab_after",
                                  "e_lab_before", "e_lab_after", "e_cmf_before", "e_cmf_after",
                                  "nu_cmf_before", "nu_cmf_after")]


class _Trace(C.Structure):
    _fields_ = [("events", C.c_void_p), ("capacity", C.c_int64), ("count", C.c_int64)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_LIB: a separately built copy (used by the mutation tests)
            override = os.environ.get("ORACLE_LIB")
            if override:
                path = override
            else:
                build()
                path = _LIB
            L = C.CDLL(path)
            vp, i32, i64, u32, u64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double
            L.orc_log.restype = d; L.orc_log.argtypes = [d]
            L.orc_exp.restype = d; L.orc_exp.argtypes = [d]
            L.orc_log_array.argtypes = [i64, vp, vp]
            L.orc_exp_array.argtypes = [i64, vp, vp]
            L.orc_distance_shell.restype = d
            L.orc_distance_shell.argtypes = [d, d, d, d, C.POINTER(i32)]
            L.orc_run.restype = i32
            L.orc_run.argtypes = [C.POINTER(_Model), u64, u32, u64, d, u64, u64, i32, C.POINTER(_Result)]
            L.orc_run_traced.restype = i32
            L.orc_run_traced.argtypes = [C.POINTER(_Model), u64, u32, u64, d, u64, u64,
                                         C.POINTER(_Result), C.POINTER(_Trace)]
            L.orc_ionization.restype = i32
            L.orc_ionization.argtypes = [i32, i32, i32, i32, i32, vp, vp, vp, vp, vp, d, vp, vp, vp, i32, vp, vp]
            L.orc_t_inner_from_luminosity.restype = d
            L.orc_t_inner_from_luminosity.argtypes = [d, d]
            L.orc_emitted_luminosity.restype = d
            L.orc_emitted_luminosity.argtypes = [vp, i32, d]
            L.orc_t_inner_update.restype = d
            L.orc_t_inner_update.argtypes = [d, d, d]
            L.orc_macroatom_walks.argtypes = [C.POINTER(_Model), i32, u64, i64, vp, vp]
            L.orc_virtual_tau.restype = d
            L.orc_virtual_tau.argtypes = [C.POINTER(_Model), d, d, i32, d, i32]
            L.orc_inject_packets.restype = i32
            L.orc_inject_packets.argtypes = [C.POINTER(_Model), u64, u32, u64, d, u64, u64, vp, vp, vp, vp, vp]
            L.orc_uniforms.argtypes = [u64, u32, u32, u32, i64, vp]
            L.orc_philox.argtypes = [vp, vp, vp]
            L.orc_planck_xi.argtypes = [i64, vp, vp]
            L.orc_level_populations.argtypes = [i32, i32, i32, vp, vp, vp, vp, vp, vp, i32, vp]
            L.orc_sobolev_tau.argtypes = [i32, i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, d, vp]
            L.orc_sobolev_constant.restype = d
            L.orc_geometric_dilution.argtypes = [i32, vp, vp, vp]
            L.orc_estimator_norm.argtypes = [i32, vp, vp, d, d, vp]
            L.orc_update_radiation_field.argtypes = [i32, vp, vp, vp, vp, vp]
            L.orc_downbranch_pick.restype = i32
            L.orc_downbranch_pick.argtypes = [C.POINTER(_Model), i32, d]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------------ elementary functions

def log(x):
    x = _f64(x)
    out = np.empty_like(x)
    lib().orc_log_array(x.size, _p(x), _p(out))
    return out


def exp(x):
    x = _f64(x)
    out = np.empty_like(x)
    lib().orc_exp_array(x.size, _p(x), _p(out))
    return out


def distance_shell(x, mu, x_in, x_out):
    w = C.c_int32(0)
    d = lib().orc_distance_shell(float(x), float(mu), float(x_in), float(x_out), C.byref(w))
    return d, int(w.value)


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_p(c), _p(k), _p(out))
    return out


def uniforms(seed, iteration, packet, n, stream=0):
    out = np.empty(n, dtype=np.float64)
    lib().orc_uniforms(seed, iteration, packet, stream, n, _p(out))
    return out


def planck_xi(z):
    z = _f64(z).reshape(-1, 5)
    out = np.empty(z.shape[0])
    lib().orc_planck_xi(z.shape[0], _p(z), _p(out))
    return out


# ------------------------------------------------------------------ model marshalling

class OracleModel:
    """Holds the arrays of a model (a ``synth.ModelSpec``-like object) in the
    layout the C oracle reads, plus the Sobolev depths it transports through."""

    def __init__(self, spec, tau=None, max_segments=1_000_000, delta_t=1.0):
        self.spec = spec
        self.v_inner = _f64(spec.v_inner)
        self.v_outer = _f64(spec.v_outer)
        self.n_e = _f64(spec.n_e)
        self.nu = _f64(spec.nu)
        S, L = self.v_inner.size, self.nu.size
        t = spec.tau if tau is None else tau
        if t is None:
            t = np.zeros((S, L))
        self.tau = _f64(t).reshape(S, L)
        self.line_mode = int(spec.line_mode)
        self.j_blue = int(bool(spec.j_blue))
        self.line_row = None
        self.ma_jump_p = self.ma_jump_offset = self.ma_jump_target = self.ma_jump_cdf = None
        if self.line_mode >= 1:
            self.line_row = (np.asarray(spec.ion, np.int64) * int(spec.n_levels)
                             + np.asarray(spec.upper, np.int64)).astype(np.int32)
            self.dbr_offset = np.ascontiguousarray(spec.dbr_offset, dtype=np.uint32)
            self.dbr_line = np.ascontiguousarray(spec.dbr_line, dtype=np.uint32)
            self.dbr_cdf = _f64(spec.dbr_cdf)
            if self.line_mode == 2:
                self.ma_jump_p = _f64(spec.ma_jump_p)
                self.ma_jump_offset = np.ascontiguousarray(spec.ma_jump_offset, dtype=np.uint32)
                self.ma_jump_target = np.ascontiguousarray(spec.ma_jump_target, dtype=np.int32)
                self.ma_jump_cdf = _f64(spec.ma_jump_cdf)
        else:
            self.dbr_offset = self.dbr_line = self.dbr_cdf = None
        self.max_segments = int(max_segments)
        self.delta_t = float(delta_t)
        self.n_virtual = 0
        self.tau_v_max = 0.0
        self._refresh()

    def set_virtual(self, n_virtual: int, tau_v_max: float = 0.0):
        """Virtual packets (Sect. 2.9) in subsequent runs: N_v per launch;
        a v-packet whose optical depth exceeds tau_v_max (> 0) is dropped."""
        self.n_virtual = int(n_virtual)
        self.tau_v_max = float(tau_v_max)
        self._refresh()

    def set_electron_density(self, n_e):
        """Electron density per shell for the Thomson opacity (ionization modes)."""
        self.n_e = _f64(n_e).copy()
        self._refresh()

    def set_tau(self, tau):
        self.tau = _f64(tau).reshape(self.v_inner.size, self.nu.size)
        self._refresh()

    def _refresh(self):
        s = self.spec
        self.c = _Model(
            n_shells=self.v_inner.size, v_inner=_p(self.v_inner), v_outer=_p(self.v_outer),
            n_e=_p(self.n_e), t_exp=float(s.t_exp), n_lines=self.nu.size, nu=_p(self.nu),
            tau=_p(self.tau), line_mode=self.line_mode, line_row=_p(self.line_row),
            dbr_offset=_p(self.dbr_offset), dbr_line=_p(self.dbr_line), dbr_cdf=_p(self.dbr_cdf),
            j_blue=self.j_blue, spec_bins=int(s.spec_bins), spec_nu_lo=float(s.spec_nu_lo),
            spec_nu_hi=float(s.spec_nu_hi), max_segments=self.max_segments, delta_t=self.delta_t,
            n_virtual=self.n_virtual, tau_v_max=self.tau_v_max,
            ma_jump_p=_p(self.ma_jump_p), ma_jump_offset=_p(self.ma_jump_offset),
            ma_jump_target=_p(self.ma_jump_target), ma_jump_cdf=_p(self.ma_jump_cdf))


class OracleResult:
    pass


def run_iteration(om: OracleModel, seed: int, iteration: int, n_packets: int, t_inner: float,
                  first: int = 0, count: int = None, threads: int = 1, record: bool = True,
                  j_blue: bool = None):
    """Transport packets [first, first+count) of an n_packets iteration."""
    if count is None:
        count = n_packets - first
    S, L, B = om.v_inner.size, om.nu.size, int(om.spec.spec_bins)
    r = OracleResult()
    r.j_est = np.zeros(S)
    r.nu_bar = np.zeros(S)
    want_jb = om.j_blue if j_blue is None else j_blue
    r.j_blue = np.zeros((S, L)) if want_jb else None
    r.spectrum = np.zeros(B + 2)
    r.spectrum_v = np.zeros(B + 2) if om.n_virtual > 0 else None
    if record:
        r.status = np.zeros(count, dtype=np.int32)
        r.nu = np.zeros(count)
        r.energy = np.zeros(count)
        r.counters = np.zeros((count, NCOUNT), dtype=np.uint64)
    else:
        r.status = r.nu = r.energy = r.counters = None
    res = _Result(j_est=_p(r.j_est), nu_bar=_p(r.nu_bar), j_blue=_p(r.j_blue),
                  spectrum=_p(r.spectrum), status=_p(r.status), nu_out=_p(r.nu),
                  e_out=_p(r.energy), counters=_p(r.counters), spectrum_v=_p(r.spectrum_v))
    # the model's flag switches the accumulation on; j_blue= overrides it for this call
    saved = om.c.j_blue
    om.c.j_blue = int(bool(want_jb))
    try:
        rc = lib().orc_run(C.byref(om.c), seed, iteration, n_packets, float(t_inner), first, count,
                           threads, C.byref(res))
    finally:
        om.c.j_blue = saved
    if rc != 0:
        raise ValueError(f"oracle rejected the model (rc={rc})")
    r.stats = dict(zip(STAT_NAMES, [int(v) for v in res.stats]))
    return r


def run_traced(om: OracleModel, seed, iteration, n_packets, t_inner, first, count, capacity=100_000):
    S, L, B = om.v_inner.size, om.nu.size, int(om.spec.spec_bins)
    r = OracleResult()
    r.j_est, r.nu_bar, r.spectrum = np.zeros(S), np.zeros(S), np.zeros(B + 2)
    r.j_blue = np.zeros((S, L)) if om.j_blue else None
    r.spectrum_v = np.zeros(B + 2) if om.n_virtual > 0 else None
    r.status = np.zeros(count, dtype=np.int32)
    r.nu, r.energy = np.zeros(count), np.zeros(count)
    r.counters = np.zeros((count, NCOUNT), dtype=np.uint64)
    res = _Result(j_est=_p(r.j_est), nu_bar=_p(r.nu_bar), j_blue=_p(r.j_blue),
                  spectrum=_p(r.spectrum), status=_p(r.status), nu_out=_p(r.nu),
                  e_out=_p(r.energy), counters=_p(r.counters), spectrum_v=_p(r.spectrum_v))
    ev = (_Event * capacity)()
    tr = _Trace(events=C.cast(ev, C.c_void_p), capacity=capacity, count=0)
    rc = lib().orc_run_traced(C.byref(om.c), seed, iteration, n_packets, float(t_inner), first,
                              count, C.byref(res), C.byref(tr))
    if rc != 0:
        raise ValueError("oracle rejected the model")
    n = min(tr.count, capacity)
    names = [f[0] for f in _Event._fields_]
    r.events = {k: np.array([getattr(ev[i], k) for i in range(n)]) for k in names}
    r.n_events = int(tr.count)
    r.stats = dict(zip(STAT_NAMES, [int(v) for v in res.stats]))
    return r


def inject_packets(om: OracleModel, seed, iteration, n_packets, t_inner, first=0, count=None):
    if count is None:
        count = n_packets - first
    out = {k: np.zeros(count) for k in ("nu_cmf", "mu", "nu_lab", "e_lab")}
    nl = np.zeros(count, dtype=np.int32)
    rc = lib().orc_inject_packets(C.byref(om.c), seed, iteration, n_packets, float(t_inner), first,
                                  count, _p(out["nu_cmf"]), _p(out["mu"]), _p(out["nu_lab"]),
                                  _p(out["e_lab"]), _p(nl))
    if rc != 0:
        raise ValueError("oracle rejected the model")
    out["next_line"] = nl
    return out


def virtual_tau(om: OracleModel, x: float, mu: float, shell: int, nu_lab: float, next_line: int) -> float:
    """Optical depth tau_v of a virtual packet from radius x (units of c t_exp)
    in direction mu, shell `shell`, lab frequency nu_lab, lines from next_line
    on, to the outer boundary (Sect. 2.9); inf if it meets the inner boundary
    or exceeds the model's tau_v_max."""
    return float(lib().orc_virtual_tau(C.byref(om.c), float(x), float(mu), int(shell), float(nu_lab),
                                       int(next_line)))


def macroatom_walks(om: OracleModel, row: int, seed: int, n: int):
    """n macro-atom walks activated in level `row` (Sect. 2.5), walk i drawing
    from packet i's stream: (emitting line, number of internal jumps)."""
    line = np.zeros(n, dtype=np.int32)
    jumps = np.zeros(n, dtype=np.uint32)
    lib().orc_macroatom_walks(C.byref(om.c), int(row), int(seed), int(n), _p(line), _p(jumps))
    return line, jumps


def downbranch_pick(om: OracleModel, row: int, z: float) -> int:
    return int(lib().orc_downbranch_pick(C.byref(om.c), int(row), float(z)))


# ------------------------------------------------------------------ plasma / radiation field

def ion_of(spec):
    """[E * J] ion index of each (element, stage), -1 for stages without levels."""
    E, J = int(spec.n_elements), int(spec.n_stages)
    out = np.full(E * J, -1, dtype=np.int32)
    for a, (e, j) in enumerate(zip(spec.ion_element, spec.ion_stage)):
        out[int(e) * J + int(j)] = a
    return out


def ionization_state(spec, t_rad, w):
    """Ion densities [S, I] and electron density [S] from the ionization
    balance of Sect. 2.3 (Eq. 2 or 3, charge conservation)."""
    S, I, K = spec.n_shells, int(spec.n_ions), int(spec.n_levels)
    E, J = int(spec.n_elements), int(spec.n_stages)
    n_ion, n_e = np.zeros(S * I), np.zeros(S)
    rc = lib().orc_ionization(S, I, K, E, J, _p(ion_of(spec)), _p(_f64(spec.energy_ev)), _p(_f64(spec.g)),
                              _p(_f64(spec.chi_ev)), _p(_f64(spec.zeta)), float(spec.delta),
                              _p(_f64(spec.n_element)), _p(_f64(t_rad)), _p(_f64(w)),
                              int(spec.ionization_mode), _p(n_ion), _p(n_e))
    if rc != 0:
        raise ValueError("oracle rejected the ionization data")
    return n_ion.reshape(S, I), n_e


def level_populations(spec, t_rad, w, lte_excitation=False, n_ion=None):
    S, I, K = spec.n_shells, int(spec.n_ions), int(spec.n_levels)
    t_rad, w = _f64(t_rad), _f64(w)
    e, g = _f64(spec.energy_ev), _f64(spec.g)
    meta = np.ascontiguousarray(spec.metastable, dtype=np.uint8)
    n_ion = _f64(spec.n_ion if n_ion is None else n_ion)
    n = np.zeros(S * I * K)
    lib().orc_level_populations(S, I, K, _p(t_rad), _p(w), _p(e), _p(g), _p(meta), _p(n_ion),
                                int(bool(lte_excitation)), _p(n))
    return n.reshape(S, I, K)


def sobolev_tau(spec, n):
    S, L, I, K = spec.n_shells, spec.n_lines, int(spec.n_ions), int(spec.n_levels)
    nu, f, g = _f64(spec.nu), _f64(spec.f), _f64(spec.g)
    ion = np.ascontiguousarray(spec.ion, dtype=np.int32)
    lo = np.ascontiguousarray(spec.lower, dtype=np.int32)
    up = np.ascontiguousarray(spec.upper, dtype=np.int32)
    n = _f64(n)
    tau = np.zeros(S * L)
    lib().orc_sobolev_tau(S, L, I, K, _p(nu), _p(f), _p(ion), _p(lo), _p(up), _p(g), _p(n),
                          float(spec.t_exp), _p(tau))
    return tau.reshape(S, L)


def sobolev_constant() -> float:
    return float(lib().orc_sobolev_constant())


def geometric_dilution(spec):
    S = spec.n_shells
    w = np.zeros(S)
    lib().orc_geometric_dilution(S, _p(_f64(spec.v_inner)), _p(_f64(spec.v_outer)), _p(w))
    return w


def estimator_norm(spec, delta_t=1.0):
    S = spec.n_shells
    out = np.zeros(S)
    lib().orc_estimator_norm(S, _p(_f64(spec.v_inner)), _p(_f64(spec.v_outer)), float(spec.t_exp),
                             float(delta_t), _p(out))
    return out


def update_radiation_field(spec, j_raw, nu_bar_raw, t_rad, w, delta_t=1.0):
    """Returns new (t_rad, w); inputs are not modified."""
    S = spec.n_shells
    norm = estimator_norm(spec, delta_t)
    t, ww = _f64(t_rad).copy(), _f64(w).copy()
    lib().orc_update_radiation_field(S, _p(_f64(j_raw)), _p(_f64(nu_bar_raw)), _p(norm), _p(t), _p(ww))
    return t, ww


def t_inner_from_luminosity(spec, l_outer):
    """Eq. 18: T_inner with 4 pi r_i^2 sigma T_inner^4 = L_outer."""
    return float(lib().orc_t_inner_from_luminosity(float(spec.v_inner[0] * spec.t_exp), float(l_outer)))


def emitted_luminosity(spectrum, delta_t=1.0):
    """Lab-frame energy of the escaping packets per unit time (all bins)."""
    sp = _f64(spectrum)
    return float(lib().orc_emitted_luminosity(_p(sp), sp.size, float(delta_t)))


def t_inner_update(t_inner, l_requested, l_emitted):
    """T_inner (L_requested / L_emitted)^(1/4); unchanged if nothing escaped."""
    return float(lib().orc_t_inner_update(float(t_inner), float(l_requested), float(l_emitted)))


def plasma_tau(spec, t_rad, w):
    """Sobolev depths from dilute-lte populations (Eqs. 5 and 12); with an
    ionization mode the ion densities come from the ionization balance."""
    n_ion = ionization_state(spec, t_rad, w)[0] if getattr(spec, "ionization_mode", 0) else None
    return sobolev_tau(spec, level_populations(spec, t_rad, w, n_ion=n_ion))


def run_loop(spec, n_iterations, n_packets, seed, threads=1, t_inner=None, record=False,
             max_segments=1_000_000, t_rad=None, w=None, first_iteration=0, l_requested=None,
             t_inner_every=3):
    """The iteration cycle of Sect. 2.8 with T_R = 1e4 K and geometric W to
    start (or the given T_R, W: a run resumed from a saved state), tau
    recomputed from the plasma each iteration and T_R, W updated from the
    estimators after each; iterations are numbered from first_iteration.
    With l_requested, after every t_inner_every-th iteration T_inner is scaled
    by (l_requested / L_emitted)^(1/4) (L_emitted from that iteration's
    escaping packets).  Returns the per-iteration results (r.t_inner: the
    inner-boundary temperature the iteration ran with)."""
    S = spec.n_shells
    t_in = spec.t_inner if t_inner is None else t_inner
    t_rad = np.full(S, 1.0e4) if t_rad is None else _f64(t_rad).copy()
    w = geometric_dilution(spec) if w is None else _f64(w).copy()
    om = None
    out = []
    ionized = getattr(spec, "ionization_mode", 0) and spec.tau is None
    for it in range(first_iteration, first_iteration + n_iterations):
        tau = plasma_tau(spec, t_rad, w) if spec.tau is None else spec.tau
        if om is None:
            om = OracleModel(spec, tau=tau, max_segments=max_segments)
        else:
            om.set_tau(tau)
        n_e = None
        if ionized:  # the Thomson opacity follows the electron density
            n_e = ionization_state(spec, t_rad, w)[1]
            om.set_electron_density(n_e)
        r = run_iteration(om, seed, it, n_packets, t_in, threads=threads, record=record)
        r.t_rad_in, r.w_in, r.tau, r.n_e = t_rad.copy(), w.copy(), tau, n_e
        r.t_inner = t_in
        t_rad, w = update_radiation_field(spec, r.j_est, r.nu_bar, t_rad, w)
        r.t_rad_out, r.w_out = t_rad.copy(), w.copy()
        r.l_emitted = emitted_luminosity(r.spectrum, om.delta_t)
        if l_requested is not None and (it - first_iteration + 1) % t_inner_every == 0:
            t_in = t_inner_update(t_in, l_requested, r.l_emitted)
        out.append(r)
    return out
