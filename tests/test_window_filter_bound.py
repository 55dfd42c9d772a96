"""The error bound of the lone walker's one-step window scan (Sect. 2.6 line
loop), checked on the CPU.

In lone-walker mode the transport kernels decide the first event among 32
consecutive lines at once, in binary32, and accept the decision only when
every sign involved lies outside an error bound M; otherwise they run the
exact scan.  The exact scan's threshold after line k is the chain of binary64
FMAs T_k = fma(tau_k, c_e, T_{k-1}) from T_{idx-1} = thr_e (binary64 kernel),
or T_k = T_{k-1} + double(float(tau_k * c_e)) (mixed kernel); line k lies
beyond d_e when nu_k <= T_{k-1} and absorbs when T_k > nu_k.  This file
restates the kernels' binary32 side (truncated conversions, a five-level
prefix sum of 32 lanes, the bound M) in numpy and asserts, on random windows
with near-ties planted at the deciding line, that every decision the filter
calls certain is the exact scan's.
"""
import ctypes
import ctypes.util

import numpy as np
import pytest

_libm = ctypes.CDLL(ctypes.util.find_library("m") or "libm.so.6")
_libm.fma.restype = ctypes.c_double
_libm.fma.argtypes = [ctypes.c_double] * 3
F32 = np.float32


def _rz32(x):
    """binary64 -> binary32 toward zero on the bit pattern, any sign; below the
    normal range -> signed 0, above it -> +-inf (the kernels' f32_rz_any)."""
    b = np.atleast_1d(np.asarray(x, dtype=np.float64)).view(np.uint64)
    e = ((b >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64) - 1023 + 127
    mant = ((b >> np.uint64(29)) & np.uint64(0x7FFFFF)).astype(np.uint32)
    mag = np.where(e <= 0, 0, np.where(e >= 255, 0x7F800000,
                                       (np.clip(e, 0, 255).astype(np.uint32) << np.uint32(23)) | mant))
    sign = (b >> np.uint64(63)).astype(np.uint32) << np.uint32(31)
    return (mag.astype(np.uint32) | sign).view(np.float32)


def _prefix32(v):
    """Inclusive Kogge-Stone prefix over 32 lanes in binary32 (offsets 1..16)."""
    p = v.astype(np.float32).copy()
    lane = np.arange(32)
    for o in (1, 2, 4, 8, 16):
        y = np.concatenate([np.zeros(o, np.float32), p[:-o]])
        p = np.where(lane >= o, (p + y).astype(np.float32), p)
    return p


def _first_stop(cand, e_no, a_yes, a_no):
    """(index of the first line that stops the scan, whether it is a certain absorption)."""
    passed = cand & e_no & a_no
    stop = cand & ~passed
    take = cand & e_no & a_yes
    if not stop.any():
        return None, False
    k = int(np.argmax(stop))
    return k, bool(take[k])


def _exact_fp64(nus, taus, ce, thr, idx):
    t = thr
    for k in range(idx, 32):
        if nus[k] <= t:
            return ("E", k)
        tn = _libm.fma(float(taus[k]), float(ce), float(t))
        if tn > nus[k]:
            return ("A", k)
        t = tn
    return (None, None)


def _filter_fp64(nus, taus, ce, thr, idx):
    cand = np.arange(32) >= idx
    dk = _rz32(nus - thr)
    p = _prefix32(np.where(cand, _rz32(taus), F32(0)))
    px = np.concatenate([np.zeros(1, np.float32), p[:-1]])
    cef = _rz32(ce)[0]
    c = (cef * p).astype(np.float32)
    a = (dk - (cef * px).astype(np.float32)).astype(np.float32)
    b = (dk - c).astype(np.float32)
    m = (F32(2.0**-20) * (np.abs(dk) + c) +
         (F32(2.0**-44) * np.abs(_rz32(thr)[0]) + (cef * F32(2.0**-119) + F32(2.0**-124)))).astype(np.float32)
    with np.errstate(invalid="ignore", over="ignore"):
        return _first_stop(cand, a > m, b < -m, b > m)


def _exact_mixed(nus, taus32, ce32, thr, idx):
    t = thr
    for k in range(idx, 32):
        if nus[k] <= t:
            return ("E", k)
        tn = t + float(np.float32(taus32[k] * ce32))
        if tn > nus[k]:
            return ("A", k)
        t = tn
    return (None, None)


def _filter_mixed(nus, taus32, ce32, thr, idx):
    cand = np.arange(32) >= idx
    dk = _rz32(nus - thr)
    p = _prefix32(np.where(cand, (taus32 * ce32).astype(np.float32), F32(0)))
    px = np.concatenate([np.zeros(1, np.float32), p[:-1]])
    a = (dk - px).astype(np.float32)
    b = (dk - p).astype(np.float32)
    m = (F32(2.0**-20) * (np.abs(dk) + p) + (F32(2.0**-44) * np.abs(_rz32(thr)[0]) + F32(2.0**-120))).astype(np.float32)
    with np.errstate(invalid="ignore", over="ignore"):
        return _first_stop(cand, a > m, b < -m, b > m)


def _window(rng, mixed):
    nu0 = 10 ** rng.uniform(14, 16)
    gap = nu0 * 10 ** rng.uniform(-8, -3)
    nus = nu0 - np.cumsum(rng.exponential(gap, 32))
    taus = 10 ** rng.normal(-2, 2, 32) * (rng.random(32) < 0.98)
    if rng.random() < 0.1:
        taus[rng.integers(32)] = 10 ** rng.uniform(-40, -30)
    if mixed:
        taus = taus.astype(np.float32)
    ce = nu0 * 10 ** rng.uniform(-6, 4)
    if mixed:
        ce = np.float32(ce)
    idx = int(rng.integers(0, 4)) if rng.random() < 0.5 else 0
    if rng.random() < 0.6:  # plant a near-tie at line k0: T_{k0} or T_{k0-1} within a few units of nu_k0
        k0 = int(rng.integers(idx, 32))
        prods = (taus * ce).astype(np.float32) if mixed else taus * ce
        s = float(np.sum(prods[idx:k0 + 1])) if rng.random() < 0.5 else float(np.sum(prods[idx:k0]))
        thr = nus[k0] - s + rng.normal(0, 1) * 10 ** rng.uniform(-3, 9)
    else:
        thr = nu0 + rng.normal(0, 3) * gap - rng.exponential(1.0) * ce * rng.choice([0.0, 1e-6, 1e-3, 1.0])
    return nus, taus, ce, float(thr), idx


@pytest.mark.parametrize("mixed", [False, True])
def test_certain_decisions_are_the_exact_scans(mixed):
    rng = np.random.default_rng(20140521 + int(mixed))
    n_fast = 0
    for _ in range(6000):
        nus, taus, ce, thr, idx = _window(rng, mixed)
        if mixed:
            k, take = _filter_mixed(nus, taus, ce, thr, idx)
            exact = _exact_mixed(nus, taus, ce, thr, idx)
        else:
            k, take = _filter_fp64(nus, taus, ce, thr, idx)
            exact = _exact_fp64(nus, taus, ce, thr, idx)
        if take:
            n_fast += 1
            assert exact == ("A", k), (exact, k, thr, ce)
    # the filter decides a good share of these adversarial windows by itself
    assert n_fast > 1000


def test_bound_is_needed():
    """A bound 2^8 times smaller lets the planted near-ties through: M is not
    so wide that the test above could not fail."""
    rng = np.random.default_rng(7)
    wrong = 0
    for _ in range(6000):
        nus, taus, ce, thr, idx = _window(rng, False)
        cand = np.arange(32) >= idx
        dk = _rz32(nus - thr)
        p = _prefix32(np.where(cand, _rz32(taus), F32(0)))
        px = np.concatenate([np.zeros(1, np.float32), p[:-1]])
        cef = _rz32(ce)[0]
        c = (cef * p).astype(np.float32)
        a = (dk - (cef * px).astype(np.float32)).astype(np.float32)
        b = (dk - c).astype(np.float32)
        m = (F32(2.0**-28) * (np.abs(dk) + c)).astype(np.float32)
        with np.errstate(invalid="ignore", over="ignore"):
            k, take = _first_stop(cand, a > m, b < -m, b > m)
        if take and _exact_fp64(nus, taus, ce, thr, idx) != ("A", k):
            wrong += 1
    assert wrong > 0
