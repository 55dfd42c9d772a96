"""Seeded synthetic supernova-ejecta models (input data only).

This module draws the *inputs* of the Monte Carlo transport: shell grids,
electron densities, frequency-sorted line lists, given Sobolev depths,
synthetic atomic data and downbranch branching tables.  It holds none of the
method's arithmetic (no transport, no Sobolev formula, no estimator): every
array it returns is fed unchanged both to the CUDA library and to the CPU
oracle used by the tests.

Workload shapes follow the paper's SN Ia setting: 20 equal-velocity shells
between 11000 and 20000 km/s at 13 days (the geometry of the code comparison
of Sect. 5.3 and the example of Appendix A), a density falling as v^-7
(Sect. 5.3), line frequencies spanning 1e14-3e15 Hz, and the dilute-lte
excitation inputs of Sect. 2.3 (Eq. 5: level energies, statistical weights,
metastable flags, ion densities).  Because the paper's atomic database is not
available, every atomic quantity is drawn from documented distributions.

Random numbers come from numpy's PCG64 generator seeded explicitly, never from
the transport's own counter-based stream.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

KM_S = 1.0e5          # cm/s per km/s
DAY_S = 86400.0       # s per day
SPEC_NU_LO = 1.0e14   # Hz, lower edge of the line range and of the spectrum
SPEC_NU_HI = 3.0e15   # Hz

# Scale A of the synthetic ion densities, N_ion[s] = A (v_mid/v_in)^-7 / n_ions.
# Chosen so that the median Sobolev depth of shell 0 in the first iteration
# (T_R = 1e4 K, geometric dilution factor) is e^-2, the median of the
# lognormal depths of the 2000-line scatter model.  The value is the one
# printed by oracle/calibrate_ion_density.py for the 500,000-line model.
ION_DENSITY_SCALE = 3809298.098545858


@dataclasses.dataclass
class ModelSpec:
    """All inputs of one ejecta model, in CGS units.

    Shells are contiguous and ordered by increasing velocity.  ``nu`` is
    strictly descending.  Either ``tau`` (given Sobolev depths, shell-major
    ``[S, L]``) or the atomic block (``f``, ``ion``, ``lower``, ``upper``,
    ``energy_ev``, ``g``, ``metastable``, ``n_ion``) is present.
    """

    name: str
    v_inner: np.ndarray
    v_outer: np.ndarray
    n_e: np.ndarray
    t_exp: float
    nu: np.ndarray
    tau: Optional[np.ndarray] = None
    f: Optional[np.ndarray] = None
    ion: Optional[np.ndarray] = None
    lower: Optional[np.ndarray] = None
    upper: Optional[np.ndarray] = None
    n_ions: int = 0
    n_levels: int = 0
    energy_ev: Optional[np.ndarray] = None
    g: Optional[np.ndarray] = None
    metastable: Optional[np.ndarray] = None
    n_ion: Optional[np.ndarray] = None
    dbr_offset: Optional[np.ndarray] = None
    dbr_line: Optional[np.ndarray] = None
    dbr_cdf: Optional[np.ndarray] = None
    # macro-atom internal jumps (line_mode 2), rows as the branching table
    ma_jump_p: Optional[np.ndarray] = None       # [rows] probability of a jump from the level
    ma_jump_offset: Optional[np.ndarray] = None  # [rows + 1] CSR over the rows
    ma_jump_target: Optional[np.ndarray] = None  # [n] row jumped to
    ma_jump_cdf: Optional[np.ndarray] = None     # [n] cumulative target probability (row ends at 1)
    # ionization balance (Sect. 2.3): 0 fixed ion densities (n_ion), 1 lte (Eq. 2),
    # 2 nebular (Eq. 3); ions with levels belong to (element, stage)
    ionization_mode: int = 0
    n_elements: int = 0
    n_stages: int = 0                       # stages per element, the last one bare
    ion_element: Optional[np.ndarray] = None  # [I]
    ion_stage: Optional[np.ndarray] = None    # [I]
    chi_ev: Optional[np.ndarray] = None       # [E, n_stages - 1] ionization potentials, eV
    zeta: Optional[np.ndarray] = None         # [E, n_stages - 1] fraction of recombinations to ground
    delta: float = 1.0
    n_element: Optional[np.ndarray] = None    # [S, E] element number densities, cm^-3
    line_mode: int = 0          # 0 scatter, 1 downbranch, 2 macro-atom
    j_blue: bool = False
    spec_bins: int = 1000
    spec_nu_lo: float = SPEC_NU_LO
    spec_nu_hi: float = SPEC_NU_HI
    t_inner: float = 1.0e4
    n_packets: int = 10_000
    n_iterations: int = 1
    seed: int = 5469

    @property
    def n_shells(self) -> int:
        return int(self.v_inner.shape[0])

    @property
    def n_lines(self) -> int:
        return int(self.nu.shape[0])

    def nbytes(self) -> int:
        tot = 0
        for fld in dataclasses.fields(self):
            v = getattr(self, fld.name)
            if isinstance(v, np.ndarray):
                tot += v.nbytes
        return tot


# ---------------------------------------------------------------- pieces

def shell_grid(n_shells: int, v_in_kms: float, v_out_kms: float):
    """Equal-velocity-width shells [v_inner, v_outer) in cm/s."""
    edges = np.linspace(v_in_kms, v_out_kms, n_shells + 1) * KM_S
    return edges[:-1].copy(), edges[1:].copy()


def power_law_profile(v_inner, v_outer, value_at_inner: float, index: float = -7.0):
    """value * (v_mid / v_inner[0])^index per shell, v_mid the shell mid-velocity."""
    v_mid = 0.5 * (v_inner + v_outer)
    return value_at_inner * (v_mid / v_inner[0]) ** index


def line_frequencies(rng, n_lines: int, lo: float = SPEC_NU_LO, hi: float = SPEC_NU_HI):
    """Log-uniform frequencies in [lo, hi], strictly descending."""
    while True:
        nu = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_lines))
        nu = np.sort(nu)[::-1].copy()
        if n_lines < 2 or np.all(np.diff(nu) < 0):
            return nu


def lognormal_tau(rng, n_shells, n_lines, shell_factor, mu=-2.0, sigma=2.0):
    """tau[s, j] = exp(mu + sigma g) * shell_factor[s], g ~ N(0, 1)."""
    g = rng.standard_normal(size=(n_shells, n_lines))
    return np.exp(mu + sigma * g) * shell_factor[:, None]


def atomic_levels(rng, n_ions: int, n_levels: int, e_max_ev: float = 15.0,
                  n_metastable: int = 5):
    """Level energies (level 0 at 0 eV, the rest sorted uniform draws in
    [0, e_max]), integer statistical weights in 1..9 and metastable flags
    (ground + the next ``n_metastable-1`` levels)."""
    energy = np.zeros((n_ions, n_levels))
    energy[:, 1:] = np.sort(rng.uniform(0.0, e_max_ev, size=(n_ions, n_levels - 1)), axis=1)
    g = rng.integers(1, 10, size=(n_ions, n_levels)).astype(np.float64)
    meta = np.zeros((n_ions, n_levels), dtype=np.uint8)
    meta[:, :n_metastable] = 1
    return energy.reshape(-1), g.reshape(-1), meta.reshape(-1)


def line_transitions(rng, n_lines: int, n_ions: int, n_levels: int):
    """Each line draws an ion and a level pair l < u uniformly."""
    ion = rng.integers(0, n_ions, size=n_lines).astype(np.int32)
    lo_idx, up_idx = np.triu_indices(n_levels, k=1)
    pair = rng.integers(0, lo_idx.shape[0], size=n_lines)
    return ion, lo_idx[pair].astype(np.int32), up_idx[pair].astype(np.int32)


def oscillator_strengths(rng, n_lines: int, lo: float = 1e-6, hi: float = 1.0):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_lines))


def downbranch_table(rng, ion, upper, n_ions: int, n_levels: int):
    """Branching table for downbranch emission, CSR over upper levels.

    Row r = ion * n_levels + upper holds, in line-index order, every line
    whose upper level is r.  Its weights are one Dirichlet(1,...,1) draw
    (normalised -ln z); ``cdf`` is the running sum divided by the total,
    with the row's last entry set to exactly 1.
    """
    n_rows = n_ions * n_levels
    row = ion.astype(np.int64) * n_levels + upper.astype(np.int64)
    order = np.argsort(row, kind="stable")
    counts = np.bincount(row, minlength=n_rows)
    offset = np.zeros(n_rows + 1, dtype=np.uint32)
    offset[1:] = np.cumsum(counts)
    w = -np.log(1.0 - rng.random(size=row.shape[0]))  # z in (0, 1]
    ws = w[order]
    csum = np.cumsum(ws)
    row_sorted = row[order]
    start = offset[:-1].astype(np.int64)[row_sorted]
    before = np.where(start > 0, csum[np.maximum(start - 1, 0)], 0.0)
    part = csum - before
    end = offset[1:].astype(np.int64)[row_sorted]
    total = csum[end - 1] - before
    cdf = part / total
    is_last = np.arange(row.shape[0]) == (end - 1)
    cdf[is_last] = 1.0
    return offset, order.astype(np.uint32), cdf


def macroatom_table(rng, dbr_offset, n_ions: int, n_levels: int, p_jump_max: float = 0.5,
                    n_targets: int = 8):
    """Synthetic macro-atom internal transitions (the paper uses radiative
    rates it does not list).  Every level that can deactivate (its branching
    row is not empty) jumps with probability p ~ U(0, p_jump_max) to one of up
    to n_targets other such levels of the same ion, with Dirichlet(1,...,1)
    target weights; otherwise it deactivates through its branching row.  Only
    levels that can deactivate are jump targets, so every walk ends.
    """
    n_rows = n_ions * n_levels
    counts = np.diff(np.asarray(dbr_offset, dtype=np.int64))
    p = np.zeros(n_rows)
    offset = np.zeros(n_rows + 1, dtype=np.uint32)
    targets, cdfs = [], []
    for ion in range(n_ions):
        rows = np.arange(ion * n_levels, (ion + 1) * n_levels)
        live = rows[counts[rows] > 0]
        for r in rows:
            if counts[r] > 0 and live.size > 1:
                others = live[live != r]
                k = min(n_targets, others.size)
                t = np.sort(rng.choice(others, size=k, replace=False))
                w = -np.log(1.0 - rng.random(size=k))
                c = np.cumsum(w) / w.sum()
                c[-1] = 1.0
                targets.append(t)
                cdfs.append(c)
                p[r] = rng.uniform(0.0, p_jump_max)
                offset[r + 1] = offset[r] + k
            else:
                offset[r + 1] = offset[r]
    target = np.concatenate(targets).astype(np.int32) if targets else np.zeros(0, np.int32)
    cdf = np.concatenate(cdfs) if cdfs else np.zeros(0)
    return p, offset, target, cdf


def ionization_data(rng, n_elements: int, n_levels_stages: int):
    """Synthetic ionization data (the paper's come from NIST and its atomic
    database): each element has n_levels_stages stages with levels plus a
    bare top stage; ionization potentials rise with the stage (U(6, 12),
    U(15, 25), U(30, 45), then +15 eV per stage), zeta ~ U(0.1, 0.9)."""
    J1 = n_levels_stages
    chi = np.zeros((n_elements, J1))
    lo, hi = [6.0, 15.0, 30.0], [12.0, 25.0, 45.0]
    for j in range(J1):
        a = lo[j] if j < 3 else 30.0 + 15.0 * (j - 2)
        b = hi[j] if j < 3 else 45.0 + 15.0 * (j - 2)
        chi[:, j] = rng.uniform(a, b, size=n_elements)
    zeta = rng.uniform(0.1, 0.9, size=(n_elements, J1))
    return chi, zeta


def nebular_model(mode: int = 2, stages: int = 3, **kw) -> ModelSpec:
    """The downbranch model with its ions grouped into elements (ion a is stage
    a % stages of element a // stages) and the ion densities from the
    ionization balance (mode 1 lte, Eq. 2; 2 nebular, Eq. 3) instead of fixed
    values; the electron density follows from charge conservation.  Element
    totals keep the fixed-ion model's total heavy-element density."""
    spec = downbranch_model(**kw)
    I, S = int(spec.n_ions), spec.n_shells
    if I % stages:
        raise ValueError("n_ions must be a multiple of stages")
    E = I // stages
    rng = np.random.default_rng(int(kw.get("seed", 1401)) + 11)
    spec.chi_ev, spec.zeta = ionization_data(rng, E, stages)
    spec.ionization_mode = int(mode)
    spec.n_elements, spec.n_stages = E, stages + 1
    spec.ion_element = (np.arange(I) // stages).astype(np.int32)
    spec.ion_stage = (np.arange(I) % stages).astype(np.int32)
    per_ion = spec.n_ion.reshape(S, I)
    spec.n_element = np.ascontiguousarray(per_ion.reshape(S, E, stages).sum(axis=2))
    spec.name = "nebular" if mode == 2 else "lte-ionization"
    return spec


def macroatom_model(p_jump_max: float = 0.5, **kw) -> ModelSpec:
    """The downbranch model in macro-atom mode (line_mode 2): the same atomic
    data and branching rows plus synthetic internal jumps."""
    spec = downbranch_model(line_mode=2, **kw)
    rng = np.random.default_rng(int(kw.get("seed", 1401)) + 7)
    (spec.ma_jump_p, spec.ma_jump_offset, spec.ma_jump_target,
     spec.ma_jump_cdf) = macroatom_table(rng, spec.dbr_offset, spec.n_ions, spec.n_levels, p_jump_max)
    spec.name = "macroatom"
    return spec


# ---------------------------------------------------------------- presets

def scatter_model(n_lines: int = 2000, n_shells: int = 20, n_packets: int = 10_000,
                  seed: int = 1401, v_in_kms: float = 11000.0, v_out_kms: float = 20000.0,
                  t_exp_days: float = 13.0, n_e_inner: float = 1.0e9,
                  tau_mu: float = -2.0, tau_sigma: float = 2.0,
                  spec_bins: int = 1000, name: str = "scatter") -> ModelSpec:
    """The plain scatter-mode model with given lognormal Sobolev depths.

    Default sizes are the 20-shell, 2000-line, 1e4-packet single-iteration
    workload: n_e = 1e9 (v_mid/v_in)^-7 cm^-3, tau lognormal(mu=-2, sigma=2)
    times (v_mid/v_in)^-7.
    """
    rng = np.random.default_rng(seed)
    v_in, v_out = shell_grid(n_shells, v_in_kms, v_out_kms)
    n_e = power_law_profile(v_in, v_out, n_e_inner)
    nu = line_frequencies(rng, n_lines)
    shell_factor = power_law_profile(v_in, v_out, 1.0)
    tau = lognormal_tau(rng, n_shells, n_lines, shell_factor, tau_mu, tau_sigma)
    return ModelSpec(name=name, v_inner=v_in, v_outer=v_out, n_e=n_e,
                     t_exp=t_exp_days * DAY_S, nu=nu, tau=np.ascontiguousarray(tau),
                     line_mode=0, j_blue=False, spec_bins=spec_bins,
                     n_packets=n_packets, n_iterations=1)


def downbranch_model(n_lines: int = 500_000, n_shells: int = 20, n_ions: int = 30,
                     n_levels: int = 40, n_packets: int = 1_000_000, n_iterations: int = 10,
                     seed: int = 1401, v_in_kms: float = 11000.0, v_out_kms: float = 20000.0,
                     t_exp_days: float = 13.0, n_e_inner: float = 1.0e9,
                     ion_density_scale: float = None, j_blue: bool = True,
                     line_mode: int = 1, t_inner: float = 1.0e4,
                     spec_bins: int = 1000, name: str = "downbranch") -> ModelSpec:
    """The full-loop downbranch model with synthetic atomic data.

    Defaults are the 500,000-line, 30-ion x 40-level, 1e6-packet, 10-iteration
    workload.  Lines draw (ion, l < u) uniformly; frequencies are log-uniform
    over 1e14-3e15 Hz (independent of the level energies, so that they stay
    distinct); oscillator strengths are log-uniform over 1e-6..1; branching
    rows are Dirichlet draws per upper level.  Ion densities are
    A (v_mid/v_in)^-7 split equally over the ions.
    """
    rng = np.random.default_rng(seed)
    v_in, v_out = shell_grid(n_shells, v_in_kms, v_out_kms)
    n_e = power_law_profile(v_in, v_out, n_e_inner)
    energy, g, meta = atomic_levels(rng, n_ions, n_levels)
    ion, lower, upper = line_transitions(rng, n_lines, n_ions, n_levels)
    f = oscillator_strengths(rng, n_lines)
    nu = line_frequencies(rng, n_lines)
    off, dline, cdf = downbranch_table(rng, ion, upper, n_ions, n_levels)
    A = ION_DENSITY_SCALE if ion_density_scale is None else ion_density_scale
    shell_factor = power_law_profile(v_in, v_out, A / n_ions)
    n_ion = np.repeat(shell_factor[:, None], n_ions, axis=1).reshape(-1).copy()
    return ModelSpec(name=name, v_inner=v_in, v_outer=v_out, n_e=n_e,
                     t_exp=t_exp_days * DAY_S, nu=nu, f=f, ion=ion, lower=lower,
                     upper=upper, n_ions=n_ions, n_levels=n_levels, energy_ev=energy,
                     g=g, metastable=meta, n_ion=n_ion, dbr_offset=off, dbr_line=dline,
                     dbr_cdf=cdf, line_mode=line_mode, j_blue=j_blue, spec_bins=spec_bins,
                     t_inner=t_inner, n_packets=n_packets, n_iterations=n_iterations)


def free_streaming_model(n_shells: int = 5, v_in_kms: float = 11000.0,
                         v_out_kms: float = 20000.0, t_exp_days: float = 13.0,
                         n_lines: int = 4, seed: int = 7, n_packets: int = 10_000) -> ModelSpec:
    """Transparent ejecta: zero electron density and zero Sobolev depths."""
    rng = np.random.default_rng(seed)
    v_in, v_out = shell_grid(n_shells, v_in_kms, v_out_kms)
    nu = line_frequencies(rng, n_lines)
    return ModelSpec(name="free", v_inner=v_in, v_outer=v_out, n_e=np.zeros(n_shells),
                     t_exp=t_exp_days * DAY_S, nu=nu, tau=np.zeros((n_shells, n_lines)),
                     n_packets=n_packets)


def batched_models(n_models: int = 256, seed: int = 1401, packets_lo: float = 1e4,
                   packets_hi: float = 1e6, lines_lo: int = 50_000, lines_hi: int = 500_000,
                   iterations: int = 10):
    """Uneven ejecta models for the batched launch, one seed per model.

    Per model: shells U{10..40}, v_in U(8000, 14000) km/s, v_out
    U(18000, 25000) km/s, t_exp U(8, 25) d, T_inner U(8000, 13000) K, line
    count U{lines_lo..lines_hi} with the downbranch-model distributions, and
    packets log-uniform in [packets_lo, packets_hi].
    """
    out = []
    for m in range(n_models):
        r = np.random.default_rng(seed + m)
        n_sh = int(r.integers(10, 41))
        v_i = float(r.uniform(8000.0, 14000.0))
        v_o = float(r.uniform(18000.0, 25000.0))
        t_d = float(r.uniform(8.0, 25.0))
        t_in = float(r.uniform(8000.0, 13000.0))
        n_l = int(r.integers(lines_lo, lines_hi + 1))
        n_p = int(round(float(np.exp(r.uniform(np.log(packets_lo), np.log(packets_hi))))))
        spec = downbranch_model(n_lines=n_l, n_shells=n_sh, n_packets=n_p,
                                n_iterations=iterations, seed=seed + 100_000 + m,
                                v_in_kms=v_i, v_out_kms=v_o, t_exp_days=t_d,
                                t_inner=t_in, name=f"batch{m}")
        out.append(spec)
    return out
