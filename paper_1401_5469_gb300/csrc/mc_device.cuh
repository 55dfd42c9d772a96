// Device helpers of the transport kernels: the Philox4x32-10 draw stream,
// integer comparison keys of binary64 values, and the binary64
// logarithm and reciprocal used on the hot path.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mcgpu {

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32->64-bit products mixed with the other counter words and the key,
// the key advancing by the two Weyl increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Per-packet uniform stream.  Draw d uses Philox block d/2 with counter
// (d/2, packet, iteration, 0); words (x,y) for even d, (z,w) for odd d;
// u53 = (wa >> 5) 2^26 + (wb >> 6).
struct DrawStream {
  uint32_t k0, k1, packet, iteration;
  uint32_t d, spare_a, spare_b;

  __device__ __forceinline__ void init(uint32_t key0, uint32_t key1, uint32_t pid, uint32_t it) {
    k0 = key0; k1 = key1; packet = pid; iteration = it; d = 0; spare_a = 0; spare_b = 0;
  }
  __device__ __forceinline__ uint64_t next_u53() {
    uint32_t wa, wb;
    if ((d & 1u) == 0u) {
      const uint4 o = philox4x32_10(make_uint4(d >> 1, packet, iteration, 0u), k0, k1);
      wa = o.x; wb = o.y; spare_a = o.z; spare_b = o.w;
    } else {
      wa = spare_a; wb = spare_b;
    }
    ++d;
    return u53_of(wa, wb);
  }
  static __device__ __forceinline__ uint64_t u53_of(uint32_t wa, uint32_t wb) {
    return (static_cast<uint64_t>(wa >> 5) << 26) | static_cast<uint64_t>(wb >> 6);
  }
  // z in (0, 1]
  __device__ __forceinline__ double open0() { return __ull2double_rn(next_u53() + 1ull) * 0x1.0p-53; }
  // z in [0, 1)
  __device__ __forceinline__ double closed0() { return __ull2double_rn(next_u53()) * 0x1.0p-53; }
  // mu = 2 z - 1 for z = u53 2^-53 in [0, 1): (u53 - 2^52) 2^-52, exact.
  // Assembled from the integer's bits (no conversion instruction).
  __device__ __forceinline__ double mu_isotropic() { return mu_from_u53(next_u53()); }
  static __device__ __forceinline__ double mu_from_u53(unsigned long long u) {
    const long long v = static_cast<long long>(u) - (1ll << 52);
    const unsigned long long a = static_cast<unsigned long long>(v < 0 ? -v : v);  // <= 2^52
    if (a == 0ull) return 0.0;
    const int lz = __clzll(static_cast<long long>(a));
    const unsigned long long mant = ((a << lz) << 1) >> 12;
    const unsigned long long bits = (static_cast<unsigned long long>(63 - lz - 52 + 1023) << 52) |
                                    mant | (v < 0 ? (1ull << 63) : 0ull);
    return __longlong_as_double(static_cast<long long>(bits));
  }
};

// The bit pattern of a binary64 value read as a signed integer.  Compared
// with the pattern of a positive value (or +0) it orders exactly like the
// values do, negative values included (their patterns are negative
// integers), so every comparison in the transport kernels -- each has one
// operand known to be positive -- runs on the integer pipe.
__device__ __forceinline__ long long rawkey(double v) { return __double_as_longlong(v); }

// Pattern of -inf: below every non-negative value's pattern.
constexpr long long kKeyNegInf = (long long)0xfff0000000000000ll;

// A pattern below that of every non-negative value.
constexpr long long kRawBelowZero = (long long)0x8000000000000000ll;

// binary64 -> binary32 toward zero on the bit pattern, any sign: |result| <=
// |d| with a relative error below 2^-23, values below the binary32 normal
// range give (signed) 0, values above its range (and NaN) +-infinity.
__device__ __forceinline__ float f32_rz_any(double d) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(d));
  const int e = static_cast<int>((b >> 52) & 0x7ffull) - 1023 + 127;
  const unsigned int mag = e <= 0 ? 0u
                           : e >= 255 ? 0x7f800000u
                                      : (static_cast<unsigned int>(e) << 23) |
                                            static_cast<unsigned int>((b >> 29) & 0x7fffffull);
  return __int_as_float(static_cast<int>(mag | (static_cast<unsigned int>(b >> 63) << 31)));
}

// v < 0, excluding -0 (its pattern is the most negative integer).
__device__ __forceinline__ bool strictly_negative(double v) {
  const long long b = __double_as_longlong(v);
  return b < 0 && b != kRawBelowZero;
}

// A 32-bit word the host may write while the kernel runs (pinned, mapped
// host memory): system-scope load, so the host's store becomes visible.
__device__ __forceinline__ uint32_t load_sys_u32(const uint32_t *a) {
  uint32_t v;
  asm volatile("ld.relaxed.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}

// L2 eviction priority for the J_blue sums: a J_blue array is as large as the
// Sobolev depths (S x L cells) and is only written, by atomics, during a
// transport launch; marking those atomics evict-first keeps the line list,
// the depths and the branching records -- what the random walks read on
// their dependency chains -- resident in L2 instead.
__device__ __forceinline__ unsigned long long l2_evict_first_policy() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void red_add_evict_first(double *a, double v, unsigned long long pol) {
  asm volatile("red.global.add.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(a), "d"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void red_add_evict_first(unsigned long long *a, unsigned long long v,
                                                    unsigned long long pol) {
  asm volatile("red.global.add.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(a), "l"(v), "l"(pol) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Reciprocal from the hardware approximation r = rcp.approx.ftz.f64(x) by
// one second-order correction: with e = 1 - x r (exact up to one rounding),
// 1/x = r / (1 - e) = r (1 + e + e^2 + ...), so r + r (e + e^2) leaves a
// relative error of order e^3 -- the cubically convergent form of Newton's
// reciprocal iteration (Markstein 1990; J.-M. Muller, Elementary Functions,
// ch. 2).  Three binary64 operations instead of the four of two Newton steps.
// Within 1 ulp of 1/x for normal |x| in [2^-1000, 2^1000] (tested against
// IEEE division through mc_selftest_math).
__device__ __forceinline__ double rcp64(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

// Square root of x >= 0 (0 or a normal number) to within 1 ulp, in five
// binary64 operations: y = rsqrt.approx.ftz.f64(x), t = x y, e = 1 - t y, and
// sqrt(x) = sqrt(t / y) (1 + O(2^-53)) = t (1 - e)^(-1/2), taken from the
// Taylor series t (1 + e/2 + 3e^2/8) (the second-order Householder step for
// 1/sqrt; J.-M. Muller, Elementary Functions, ch. 2).  On GB300 |e| <= 2^-19.0
// over every high word of [1, 4) (measured), so the first omitted term,
// 5e^3/16, is below 2^-58 relative.  (CUDA's sqrt rounds correctly but takes
// about ten binary64 instructions; on GB300 each costs its sub-partition's
// FP64 pipe ~64 cycles.)
__device__ __forceinline__ double sqrt64(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double t = x * y;
  const double e = fma(-t, y, 1.0);
  const double p = fma(0.375, e, 0.5);
  const double r = fma(t * e, p, t);
  return __double_as_longlong(x) == 0ll ? 0.0 : r;
}

// ln(2) split so that k * kLn2Head is exact for |k| < 2^20.
constexpr double kLn2Head = 0x1.62e42fee00000p-1;
constexpr double kLn2Tail = 0x1.a39ef35793c76p-33;

// {c = 1/F, -ln(c)} per breakpoint F; see gen_log_table.py.
static __constant__ double2 c_log_tab[128] = {
#include "mc_log_table.inc"
};

// ln(m 2^k) for m in [1, 2) given by its 52 fraction bits, by Tang's
// table-driven method (ACM TOMS 16, 1990): m is moved to [0.75, 1.5) (k
// adjusted), r = m c - 1 with the nearest breakpoint's c = 1/F, and
// ln(1 + r) from its Taylor series to degree 8 (|r| < 2^-7).
__device__ __forceinline__ double log_core(int k, unsigned long long frac) {
  const int i = static_cast<int>(frac >> 45);
  long long mb = static_cast<long long>(0x3ff0000000000000ull | frac);
  if (i >= 64) { mb -= (1ll << 52); ++k; }  // m / 2, exponent field only
  const double m = __longlong_as_double(mb);
  const double2 ct = c_log_tab[i];
  const double r = fma(m, ct.x, -1.0);
  double p = -0.125;
  p = fma(p, r, 1.0 / 7.0);
  p = fma(p, r, -1.0 / 6.0);
  p = fma(p, r, 0.2);
  p = fma(p, r, -0.25);
  p = fma(p, r, 1.0 / 3.0);
  p = fma(p, r, -0.5);
  p = fma(p, r, 1.0);
  const double dk = static_cast<double>(k);
  return fma(dk, kLn2Head, ct.y) + fma(p, r, dk * kLn2Tail);
}

#define MC_KLN2(k) {(k) * kLn2Head, (k) * kLn2Tail}
#define MC_KLN2_8(b) MC_KLN2(b), MC_KLN2(b - 1), MC_KLN2(b - 2), MC_KLN2(b - 3), \
                     MC_KLN2(b - 4), MC_KLN2(b - 5), MC_KLN2(b - 6), MC_KLN2(b - 7)
// {k ln2 head, k ln2 tail} for k = 0, -1, ..., -55 (both products exact / correctly rounded).
static __constant__ double2 c_kln2[56] = {MC_KLN2_8(0), MC_KLN2_8(-8), MC_KLN2_8(-16), MC_KLN2_8(-24),
                                          MC_KLN2_8(-32), MC_KLN2_8(-40), MC_KLN2_8(-48)};
#undef MC_KLN2_8
#undef MC_KLN2

// -ln(z) for z = u 2^-53, 1 <= u <= 2^53 (the (0,1] draw): integer-only
// reduction, k ln2 from a table (no conversion instruction), then Tang's
// method as in log_core.
__device__ __forceinline__ double neg_log_u53(unsigned long long u) {
  const int lz = __clzll(static_cast<long long>(u));
  const unsigned long long frac = ((u << lz) << 1) >> 12;
  int k = 63 - lz - 53;  // in [-53, 0]
  const int i = static_cast<int>(frac >> 45);
  long long mb = static_cast<long long>(0x3ff0000000000000ull | frac);
  if (i >= 64) { mb -= (1ll << 52); ++k; }
  const double m = __longlong_as_double(mb);
  const double2 ct = c_log_tab[i];
  const double2 kl = c_kln2[-k];
  const double r = fma(m, ct.x, -1.0);
  double p = -0.125;
  p = fma(p, r, 1.0 / 7.0);
  p = fma(p, r, -1.0 / 6.0);
  p = fma(p, r, 0.2);
  p = fma(p, r, -0.25);
  p = fma(p, r, 1.0 / 3.0);
  p = fma(p, r, -0.5);
  p = fma(p, r, 1.0);
  return -((kl.x + ct.y) + fma(p, r, kl.y));
}

// Draws of a warp's last live packet, computed ahead by the whole warp.
// Once the packet queue is empty and one lane of a warp is left, the other
// 31 lanes have nothing to do; a draw's value depends only on (key, packet,
// iteration, draw index), so lane i computes Philox block base/2 + i and the
// -ln z of both its draws, and the live lane reads its next 64 draws from
// shared memory instead of running Philox and the log on its own dependency
// chain.  Values are identical to DrawStream's.  All state is warp-uniform.
// (Serving up to four live lanes, with per-lane slots, measured slower: the
// per-segment bookkeeping then costs more than the draws it saves.)
constexpr uint32_t kWarpDraws = 64;
constexpr uint32_t kNoPacket = 0xffffffffu;

// Draw i of a packet's stream computed on its own, for draws past the end of
// the warp buffer (only a macro atom's long walks get there).  Out of line
// and by value, so that the common path does not evaluate it.
static __device__ __noinline__ unsigned long long u53_past_buffer(uint32_t k0, uint32_t k1, uint32_t packet,
                                                           uint32_t iteration, uint32_t i) {
  const uint4 o = philox4x32_10(make_uint4(i >> 1, packet, iteration, 0u), k0, k1);
  return (i & 1u) ? DrawStream::u53_of(o.z, o.w) : DrawStream::u53_of(o.x, o.y);
}
static __device__ __noinline__ double tau_past_buffer(uint32_t k0, uint32_t k1, uint32_t packet, uint32_t iteration,
                                               uint32_t i) {
  return neg_log_u53(u53_past_buffer(k0, k1, packet, iteration, i) + 1ull);
}

struct WarpDraws {
  unsigned long long *u;  // [64] u53 of draws base .. base + 63 (shared memory, per warp)
  double *t;              // [64] -ln((u53 + 1) 2^-53) of the same draws
  uint32_t base, pid;     // first draw index held, packet (kNoPacket: none)
  bool on;                // the warp is down to one live lane, which reads the buffer

  __device__ __forceinline__ void init(unsigned long long *warp_buf) {
    u = warp_buf;
    t = reinterpret_cast<double *>(warp_buf + kWarpDraws);
    base = 0u;
    pid = kNoPacket;
    on = false;
  }

  // All 32 lanes, converged, after the claim step.  alive: this lane has a
  // packet; drained: the packet queue is empty.  With one live lane left,
  // refill the buffer when it holds fewer than the three draws a segment may
  // take (or belongs to another packet).
  __device__ __forceinline__ void prepare(bool alive, bool drained, const DrawStream &ds,
                                          uint32_t packet, uint32_t k0, uint32_t k1,
                                          uint32_t iteration, unsigned lane) {
    const unsigned live = __ballot_sync(0xffffffffu, alive);
    on = drained && __popc(live) == 1;
    if (!on) return;
    const int owner = __ffs(live) - 1;
    const uint32_t d = __shfl_sync(0xffffffffu, ds.d, owner);
    const uint32_t pk = __shfl_sync(0xffffffffu, packet, owner);
    if (pk == pid && d + 3u <= base + kWarpDraws) return;
    const uint32_t b = d & ~1u;
    const uint4 o = philox4x32_10(make_uint4((b >> 1) + lane, pk, iteration, 0u), k0, k1);
    const unsigned long long u0 = DrawStream::u53_of(o.x, o.y), u1 = DrawStream::u53_of(o.z, o.w);
    u[2 * lane] = u0;
    u[2 * lane + 1] = u1;
    t[2 * lane] = neg_log_u53(u0 + 1ull);
    t[2 * lane + 1] = neg_log_u53(u1 + 1ull);
    __syncwarp();
    base = b;
    pid = pk;
  }
  // Lone-walker mode (every lane of the warp holds the walker's draw stream):
  // refill when fewer than the three draws a segment may take are left.
  __device__ __forceinline__ void keep(const DrawStream &ds, uint32_t k0, uint32_t k1, uint32_t iteration,
                                       unsigned lane) {
    if (ds.packet == pid && ds.d + 3u <= base + kWarpDraws) return;
    const uint32_t b = ds.d & ~1u;
    const uint4 o = philox4x32_10(make_uint4((b >> 1) + lane, ds.packet, iteration, 0u), k0, k1);
    const unsigned long long u0 = DrawStream::u53_of(o.x, o.y), u1 = DrawStream::u53_of(o.z, o.w);
    __syncwarp();  // every lane has read the old contents
    u[2 * lane] = u0;
    u[2 * lane + 1] = u1;
    t[2 * lane] = neg_log_u53(u0 + 1ull);
    t[2 * lane + 1] = neg_log_u53(u1 + 1ull);
    __syncwarp();
    base = b;
    pid = ds.packet;
  }
  // As keep(), for a kernel that takes only the u53 values from the buffer
  // (the mixed-precision kernel's log is binary32): the -ln z half stays unset.
  __device__ __forceinline__ void keep_u(const DrawStream &ds, uint32_t k0, uint32_t k1, uint32_t iteration,
                                         unsigned lane) {
    if (ds.packet == pid && ds.d + 3u <= base + kWarpDraws) return;
    const uint32_t b = ds.d & ~1u;
    const uint4 o = philox4x32_10(make_uint4((b >> 1) + lane, ds.packet, iteration, 0u), k0, k1);
    __syncwarp();  // every lane has read the old contents
    u[2 * lane] = DrawStream::u53_of(o.x, o.y);
    u[2 * lane + 1] = DrawStream::u53_of(o.z, o.w);
    __syncwarp();
    base = b;
    pid = ds.packet;
  }
  // The lone walker's next draw, from the buffer that keep() or keep_u()
  // holds filled for the segment.
  __device__ __forceinline__ unsigned long long take_u53(DrawStream &ds) const { return u[ds.d++ - base]; }
  // The live lane's next draw (u53, or the -ln z of an open-interval draw).
  // UNBOUNDED: a segment may take more draws than the buffer holds (a macro
  // atom's internal jumps), and past its end a draw is computed on its own;
  // otherwise a segment takes at most three draws and prepare() keeps three
  // in the buffer.
  template <bool UNBOUNDED>
  __device__ __forceinline__ unsigned long long next_u53(DrawStream &ds) const {
    if (!on) return ds.next_u53();
    const uint32_t i = ds.d++ - base;
    if (!UNBOUNDED || i < kWarpDraws) return u[i];
    return u53_past_buffer(ds.k0, ds.k1, ds.packet, ds.iteration, ds.d - 1u);
  }
  // The draw next_u53 returns next, without taking it; only while the buffer
  // holds it (lone-walker mode, within a segment's three draws).
  __device__ __forceinline__ unsigned long long peek_u53(const DrawStream &ds) const { return u[ds.d - base]; }
  template <bool UNBOUNDED>
  __device__ __forceinline__ double next_tau(DrawStream &ds) const {
    if (!on) return neg_log_u53(ds.next_u53() + 1ull);
    const uint32_t i = ds.d++ - base;
    if (!UNBOUNDED || i < kWarpDraws) return t[i];
    return tau_past_buffer(ds.k0, ds.k1, ds.packet, ds.iteration, ds.d - 1u);
  }
};

// ln(x) for a positive normal binary64 x.
__device__ __forceinline__ double log_pos(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  return log_core(static_cast<int>((b >> 52) & 0x7ffull) - 1023, b & 0x000fffffffffffffull);
}

}  // namespace mcgpu
