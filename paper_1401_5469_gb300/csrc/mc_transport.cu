// Monte Carlo packet transport through homologously expanding shells
// (Kerzendorf & Sim 2014, Sects. 2.4-2.7 and 2.9), one packet per thread in a
// persistent grid.
//
// GB300 notes.  Binary64 add/mul/fma/compare issue at 1/64 of the binary32
// rate and every binary64 warp instruction holds its warp for ~64 cycles,
// whatever the number of active lanes.  A line-thick model is latency-bound by
// its longest random walks (the packet queue empties within a few percent of
// the kernel time), so the kernel minimises binary64 instructions per flight
// segment:
//  * the packet carries p = x mu and q = x^2 - p^2 (conserved in free flight;
//    radii in units of c t_exp): D = 1 - p, x^2 = q + p^2, the shell exit is
//    at p = +-sqrt(x_b^2 - q) -- a root taken only when a line is passed or
//    the shell event wins -- and a flight of length l is p += l;
//  * the line scan runs in the frequency domain: a Sobolev point is the
//    closest event while nu_line > max(nu_shell, nu_e), where nu_shell and
//    nu_e are the comoving frequencies reached at d_shell and d_e; passing a
//    line of depth tau moves nu_e up by tau nu_lab / k (one FMA), and the line
//    absorbs the packet exactly when that new nu_e exceeds nu_line (Sect. 2.6's
//    test tau_S + kappa d_line > tau with kappa d = (nu_cmf - nu) / (nu_lab/k));
//    every comparison is an integer compare of the values' bit patterns
//    (one operand is always positive, so the patterns order like the values);
//  * 1/D and 1/nu_lab are carried and refreshed with Newton reciprocals,
//    E/nu_lab is carried instead of E_lab (the same in both frames), and
//    -ln z comes from a table-driven logarithm;
//  * downbranch emission is an integer guide-table search, and the next
//    line's nu/tau loads are issued before the current line is resolved;
//  * lanes stay converged: a lane that finishes claims the next packet at the
//    loop head (warp-aggregated atomic); shell estimators accumulate in
//    registers and are flushed once per shell change;
//  * a warp down to its last live walk runs it with all 32 lanes (lone-walker
//    mode): the line list 32 lines at a time, the scan of such a window in
//    one step through a binary32 filter with an error bound (the scalar scan
//    wherever a sign is within the bound), the absorbing line's emission
//    record loaded as soon as the scan names it, and the walk's draws
//    computed ahead by the whole warp.
#include <cstdint>

#include "mc_device.cuh"
#include "mc_internal.h"

namespace mcgpu {

namespace {

constexpr int kBlock = 128;
constexpr int kShellArrays = 6;  // x_in^2, x_out^2, x_in, x_out, kappa, 1/kappa
constexpr int kLineEvent = 1, kElectronEvent = 2, kShellEvent = 3;

struct Packet {
  double p, q;               // x mu, x^2 - p^2
  // nu_lab, 1/nu_lab and E_lab / nu_lab = E_cmf / nu_cmf: the first-order
  // Doppler factor scales energy and frequency alike, so the ratio is the
  // same in both frames; it changes only when a line re-emits at another
  // frequency (Thomson and resonant scatterings keep both comoving values).
  double nu_lab, e_per_nu, inv_nu;
  // Frame quantities at the start of the next flight segment, carried from
  // the event that began it (valid while have_cmf): D = 1 - p, 1/D, the
  // comoving frequency nu_lab D and E_cmf D = E_lab D^2 (the estimators'
  // weight per unit length).  After an interaction they are known without
  // new products (nu_cmf is the emitted comoving frequency, E_cmf D = E_cmf' D
  // with the new direction's D); after a shell crossing they are recomputed.
  double D, inv_D, nu_cmf, eD2;
  int32_t shell, next_line;
  uint32_t pid;
  bool have_cmf;
  uint32_t cnt[kNCounters];
};

// First index j with nu[j] < v (nu strictly descending, positive): lower
// bound on the int64 images of the frequencies.
__device__ __forceinline__ int32_t first_redward(const double *nu, int32_t L, double v) {
  const long long kv = __double_as_longlong(v);
  const long long *nb = reinterpret_cast<const long long *>(nu);
  int32_t lo = 0, hi = L;
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (__ldg(nb + mid) < kv) hi = mid; else lo = mid + 1;
  }
  return lo;
}

struct Emission {
  double nu, inv_nu;
  int32_t line;
};

// Downbranch re-emission (Sect. 2.5): the first entry k of the activated
// upper level's branching row with z < cdf[k], z = u 2^-53.  With the guide
// table: z < cdf[k] <=> u < ceil(cdf[k] 2^53) = thr[k] exactly; the search
// starts at the guide entry of bucket floor(z n) and walks forward.
// The bucket slot of draw u in the branching row of rinfo (begin | length << 32).
__device__ __forceinline__ const DbrRec *bucket_slot(const TransportParams &p, unsigned long long rinfo,
                                                     unsigned long long u) {
  const uint32_t b = static_cast<uint32_t>(rinfo), len = static_cast<uint32_t>(rinfo >> 32);
  const uint32_t bucket = static_cast<uint32_t>(__umul64hi(u << 11, static_cast<unsigned long long>(len)));
  return p.dbr_bucket + b + bucket;
}

// A slot record as two 16-byte halves: {thr, nu} and {inv_nu, emit | guide << 32}.
__device__ __forceinline__ void load_slot(const DbrRec *slot, ulonglong2 &a, ulonglong2 &c) {
  a = __ldg(reinterpret_cast<const ulonglong2 *>(slot));
  c = __ldg(reinterpret_cast<const ulonglong2 *>(slot) + 1);
}

// The emission from a loaded slot record: the slot itself when u is below its
// threshold, else the walk forward from its guide entry.
__device__ __forceinline__ Emission pick_from_slot(const TransportParams &p, unsigned long long rinfo,
                                                   unsigned long long u, ulonglong2 a, ulonglong2 c) {
  Emission em;
  if (u < a.x) {
    em.nu = __longlong_as_double(static_cast<long long>(a.y));
    em.inv_nu = __longlong_as_double(static_cast<long long>(c.x));
    em.line = static_cast<int32_t>(static_cast<uint32_t>(c.y));
    return em;
  }
  const DbrRec *rec = p.dbr_rec;
  uint32_t i = static_cast<uint32_t>(rinfo) + static_cast<uint32_t>(c.y >> 32) + 1u;
  unsigned long long thr = __ldg(&rec[i].thr);
  while (u >= thr) { ++i; thr = __ldg(&rec[i].thr); }
  em.nu = __ldg(&rec[i].nu);
  em.inv_nu = __ldg(&rec[i].inv_nu);
  em.line = static_cast<int32_t>(__ldg(&rec[i].emit));
  return em;
}

// Lone-walker mode (all 32 lanes converged on one walk): the pick from the
// bucket slot's record, and past it the next 32 records of the row in one
// coalesced load per round (lane i takes entry i), the first with u below
// its threshold found by a vote.  The row's last threshold is 2^53 > u, so
// the search ends inside the row.
__device__ __forceinline__ Emission pick_from_slot_lone(const TransportParams &p, unsigned long long rinfo,
                                                        unsigned long long u, ulonglong2 a, ulonglong2 c,
                                                        unsigned lane) {
  Emission em;
  if (u < a.x) {
    em.nu = __longlong_as_double(static_cast<long long>(a.y));
    em.inv_nu = __longlong_as_double(static_cast<long long>(c.x));
    em.line = static_cast<int32_t>(static_cast<uint32_t>(c.y));
    return em;
  }
  const uint32_t end = static_cast<uint32_t>(rinfo) + static_cast<uint32_t>(rinfo >> 32);
  uint32_t i0 = static_cast<uint32_t>(rinfo) + static_cast<uint32_t>(c.y >> 32) + 1u;
  for (;;) {
    const uint32_t i = i0 + lane;
    ulonglong2 ra = make_ulonglong2(~0ull, 0ull), rc = make_ulonglong2(0ull, 0ull);
    if (i < end) load_slot(p.dbr_rec + i, ra, rc);
    const unsigned m = __ballot_sync(0xffffffffu, u < ra.x);  // lanes past the row's end vote yes
    if (m != 0u) {
      const int k = __ffs(m) - 1;
      em.nu = __longlong_as_double(__shfl_sync(0xffffffffu, static_cast<long long>(ra.y), k));
      em.inv_nu = __longlong_as_double(__shfl_sync(0xffffffffu, static_cast<long long>(rc.x), k));
      em.line = __shfl_sync(0xffffffffu, static_cast<int32_t>(static_cast<uint32_t>(rc.y)), k);
      return em;
    }
    i0 += 32u;
  }
}

__device__ __forceinline__ Emission downbranch_pick(const TransportParams &p, int32_t j,
                                                    unsigned long long rinfo, unsigned long long u) {
  Emission em;
  if (p.dbr_rec) {
    // bucket slot: a copy of the guide entry's record, so that the common case
    // (the guide entry is the answer) is one 32-byte record load
    ulonglong2 a, c;
    load_slot(bucket_slot(p, rinfo, u), a, c);
    return pick_from_slot(p, rinfo, u, a, c);
  }
  const int32_t row = __ldg(p.line_row + j);
  uint32_t lo = __ldg(p.dbr_offset + row), hi = __ldg(p.dbr_offset + row + 1) - 1u;
  const long long kz = __double_as_longlong(static_cast<double>(u) * 0x1.0p-53);
  const long long *cb = reinterpret_cast<const long long *>(p.dbr_cdf);
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (kz < __ldg(cb + mid)) hi = mid; else lo = mid + 1u;
  }
  em.line = static_cast<int32_t>(__ldg(p.dbr_line + lo));
  em.nu = __ldg(p.nu + em.line);
  em.inv_nu = rcp64(em.nu);
  return em;
}

// Macro atom (Sect. 2.5, mode macroatom): activated in level `row` (the
// absorbing line's upper level), the atom jumps -- decision draw u53 below
// the level's threshold, then a draw for the target -- until it deactivates;
// returns the branching-row info (begin | length << 32) of the level it
// deactivates from, for the emission pick.  After kMaMaxJumps jumps it
// deactivates without the decision draw.
__device__ __forceinline__ unsigned long long macroatom_walk(const TransportParams &p, int32_t row,
                                                             const WarpDraws &wd, DrawStream &ds) {
  for (uint32_t n = 0; n < kMaMaxJumps; ++n) {
    const MaRow *mr = p.ma_row + row;
    const unsigned long long thr = __ldg(&mr->jump_thr);
    const uint2 jb = __ldg(reinterpret_cast<const uint2 *>(&mr->jump_begin));  // begin, length
    const unsigned long long za = wd.template next_u53<true>(ds);
    if (!(za < thr)) {
      const uint2 db = __ldg(reinterpret_cast<const uint2 *>(&mr->dbr_begin));
      return static_cast<unsigned long long>(db.x) | (static_cast<unsigned long long>(db.y) << 32);
    }
    const unsigned long long zb = wd.template next_u53<true>(ds);
    const MaJump *jp = p.ma_jump + jb.x;
    int32_t next = __ldg(&jp[jb.y - 1].target);
    for (uint32_t k = 0; k < jb.y; ++k) {
      if (zb < __ldg(&jp[k].thr)) { next = __ldg(&jp[k].target); break; }
    }
    row = next;
  }
  const uint2 db = __ldg(reinterpret_cast<const uint2 *>(&p.ma_row[row].dbr_begin));
  return static_cast<unsigned long long>(db.x) | (static_cast<unsigned long long>(db.y) << 32);
}

// max(v, 0) through the integer keys (no binary64 instruction).
__device__ __forceinline__ double max0(double v) { return rawkey(v) > 0 ? v : 0.0; }

// x mu at the shell exit: +sqrt(x_out^2 - q), or -sqrt(x_in^2 - q) when the
// ray meets the inner sphere.
__device__ __forceinline__ double shell_exit(double q, bool inner, double xi2, double xo2) {
  const double root = sqrt64((inner ? xi2 : xo2) - q);
  return inner ? -root : root;
}

// Does an event at path length l (units of c t_exp) come before the shell
// exit?  Along the ray x mu grows by l and x^2 = q + (x mu)^2; pl = x mu and
// r2 = x^2 at the event point.  Outward exit: before it exactly when x^2 <
// x_out^2 there (a point with x mu < 0 has x^2 <= the current x^2).  Inner
// exit at x mu = -sqrt(x_in^2 - q): before it exactly when x mu < 0 and
// x^2 > x_in^2 there.
__device__ __forceinline__ bool inside_shell(double pl, double r2, bool inner, double xi2, double xo2) {
  const long long k2 = rawkey(r2);  // all three squares are >= 0
  return inner ? (strictly_negative(pl) && k2 > rawkey(xi2)) : k2 < rawkey(xo2);
}

// binary64 -> binary32 toward zero on the bit pattern (no conversion
// instruction: on GB300 those issue on the binary64 pipe), for d >= 0 below
// the binary32 overflow threshold; values below the binary32 normal range
// give 0 (an absolute error under 2^-126).
__device__ __forceinline__ float f32_rz(double d) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(d));
  const int e = static_cast<int>(b >> 52) - 1023 + 127;
  return e <= 0 ? 0.0f : __int_as_float((e << 23) | static_cast<int>((b >> 29) & 0x7fffffull));
}

// Bit pattern of the binary64 value of a positive normal binary32 (exact).
__device__ __forceinline__ long long f64_bits(float f) {
  const unsigned int b = static_cast<unsigned int>(__float_as_int(f));
  return static_cast<long long>(((static_cast<unsigned long long>(b >> 23) + (1023 - 127)) << 52) |
                                (static_cast<unsigned long long>(b & 0x7fffffu) << 29));
}

// The comoving frequency at the shell exit, K = nu_lab (1 - p_exit) with
// p_exit = +-sqrt64(x_b^2 - q) as shell_exit and the key below compute it
// in binary64, bracketed from binary32 arithmetic: on success K lies in
// [lo, hi] (binary64 bit patterns), so that a line frequency or threshold
// outside the bracket is ordered against K without the binary64 root; a
// value inside it needs the exact K.  Error budget (u = 2^-24): the
// operands truncated to binary32 (2u each), the difference (u), the
// approximate reciprocal square root (taken as 2^-20 relative), the
// products and sums (u each), and the binary64 path's own rounding (1 ulp
// root, 3 roundings); the bracket is widened by 2^-19 K beyond the sum so
// that rounding its ends keeps K inside.  Near-tangent exits (x_b^2 - q
// within 4x its own error) and roots of 0.5 or more are not bracketed.
struct ShellBracket {
  long long lo, hi;
  bool ok;
};
__device__ __forceinline__ ShellBracket shell_bracket(double q, double xb2, bool inner, double nu_lab) {
  ShellBracket b;
  const float a = f32_rz(xb2), c = f32_rz(q), nu = f32_rz(nu_lab);
  const float dq = a - c;
  const float e1 = 0x1.0p-22f * (a + dq);  // >= |dq - (x_b^2 - q)| + the binary64 difference's rounding
  b.ok = dq >= 4.0f * e1;
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(dq));
  const float P = dq * r;                                  // ~ sqrt(x_b^2 - q)
  const float ep = fmaf(0x1.0p-18f, P, 1.01f * (e1 * r));  // >= |p_exit| - P
  b.ok = b.ok && P < 0.5f;
  const float g = inner ? 1.0f + P : 1.0f - P;
  const float k = nu * g;
  const float ek = k * fmaf(2.5f, ep, 0x1.0p-19f);
  b.lo = f64_bits(k - ek);
  b.hi = f64_bits(k + ek);
  return b;
}

// Injection at the inner boundary, Sect. 2.4: Planck-sampled comoving
// frequency (Carter & Cashwell series method), mu = sqrt(z), equal comoving
// energy (Eq. 10), lab-frame values by the first-order Doppler factor.
__device__ __forceinline__ double inject(const TransportParams &p, const double *planck, double x0,
                                         double x0sq, Packet &pk, DrawStream &ds) {
  const double z0 = ds.closed0();
  const double z1 = ds.open0(), z2 = ds.open0(), z3 = ds.open0(), z4 = ds.open0();
  int l = 1;
  while (l < kPlanckLmax && planck[l] < z0) ++l;
  double xi = -log_pos(((z1 * z2) * z3) * z4);
  if (l > 1) xi = xi / static_cast<double>(l);
  const double nu_cmf = p.nu_scale * xi;
  const double mu = sqrt(ds.open0());
  const double pp = x0 * mu;
  const double D = 1.0 - pp;
  const double iD = rcp64(D);
  pk.p = pp;
  pk.q = max0(fma(-pp, pp, x0sq));
  const double inv_nu_cmf = rcp64(nu_cmf);
  pk.nu_lab = nu_cmf * iD;
  pk.e_per_nu = p.e_cmf * inv_nu_cmf;
  pk.inv_nu = inv_nu_cmf * D;
  pk.D = D;
  pk.inv_D = iD;
  pk.nu_cmf = nu_cmf;
  pk.eD2 = p.e_cmf * D;
  pk.have_cmf = true;
  pk.shell = 0;
  pk.next_line = first_redward(p.nu, p.L, nu_cmf);
#pragma unroll
  for (int c = 0; c < kNCounters; ++c) pk.cnt[c] = 0u;
  return nu_cmf;
}

// Spectrum bin of a lab frequency; below the range -> bins, above (or NaN)
// -> bins + 1 (Sect. 2.9 direct binning).
__device__ __forceinline__ int spectrum_bin(const TransportParams &p, double nu_lab) {
  if (nu_lab < p.spec_lo) return p.spec_bins;
  const double t = (nu_lab - p.spec_lo) / p.spec_dnu;
  return (t >= 0.0 && t < static_cast<double>(p.spec_bins)) ? static_cast<int>(floor(t)) : p.spec_bins + 1;
}

// ---- virtual packets (Sect. 2.9, Eqs. 19-21)
// Whenever an r-packet is about to start a trajectory (injection, or after an
// interaction), N_v v-packets leave its position with its comoving frequency
// and energy, in directions mu_v = mu_min + (1 - mu_min) z, z in (0, 1], with
// mu_min = -sqrt(1 - (x_in / x)^2) so that none meets the inner boundary.  A
// v-packet never interacts: it collects the Sobolev depths of the lines it
// passes and the electron-scattering depth kappa' D l of each segment (D at
// the segment start) on its way out, and adds exp(-tau_v) times its lab
// energy to the bin of its lab frequency.  Comoving energies: E (1 - mu_min)
// / (2 N_v) after an interaction (Eq. 19), E 2 mu_v / N_v at injection
// (Eq. 20).  Draws come from Philox stream 1 (counter word 3 = 1), the v-draw
// index counting on across the packet's launches, so the r-packet's own
// draws are untouched.

struct VirtualLaunch {
  double x, r2, nu_cmf, e_cmf;  // radius (units of c t_exp), its square, comoving nu and E
  int32_t shell, next_line;
  uint32_t pid, first_draw;
  bool injection;
};

__device__ __forceinline__ double vdraw_open0(const TransportParams &p, uint32_t pid, uint32_t d) {
  const uint4 o = philox4x32_10(make_uint4(d >> 1, pid, p.iteration, 1u), p.key0, p.key1);
  const unsigned long long u = (d & 1u) ? DrawStream::u53_of(o.z, o.w) : DrawStream::u53_of(o.x, o.y);
  return __ull2double_rn(u + 1ull) * 0x1.0p-53;
}

// Kept out of line: it runs only in the spectrum iteration and must not add
// registers to the transport loop.
__device__ __noinline__ void spawn_virtual(const TransportParams &p, const double *sh, VirtualLaunch v) {
  const int32_t S = p.S, L = p.L, nv = p.n_virtual;
  const double *s_xi2 = sh, *s_xo2 = sh + S, *s_kap = sh + 4 * S;
  const double ri = sh[2 * S] / v.x;  // x_in[0] / x
  const double arg = 1.0 - ri * ri;
  const double mu_min = -sqrt(rawkey(arg) > 0 ? arg : 0.0);
  const long long *nub = reinterpret_cast<const long long *>(p.nu);
  const bool cut = rawkey(p.tau_v_max) > 0;
  for (int32_t i = 0; i < nv; ++i) {
    const double mu_v = mu_min + (1.0 - mu_min) * vdraw_open0(p, v.pid, v.first_draw + i);
    double pc = v.x * mu_v;
    const double D = 1.0 - pc;
    const double q = max0(fma(-pc, pc, v.r2));
    const double e_v = v.injection ? (v.e_cmf * (2.0 * mu_v)) / nv : (v.e_cmf * (1.0 - mu_min)) / (2.0 * nv);
    const double nu_lab = v.nu_cmf / D;
    double tau = 0.0;
    int32_t s = v.shell, j = v.next_line;
    bool out = false;
    for (;;) {
      const double xi2 = s_xi2[s], xo2 = s_xo2[s];
      const bool inner = strictly_negative(pc) && rawkey(q) <= rawkey(xi2);
      const double p_exit = shell_exit(q, inner, xi2, xo2);
      // Sobolev points before the exit: nu_j > nu_lab (1 - p_exit)
      const long long key_exit = rawkey(nu_lab * (1.0 - p_exit));
      const double *tau_s = p.tau + static_cast<size_t>(s) * static_cast<size_t>(L);
      bool over = false;
      while (j < L && __ldg(nub + j) > key_exit) {
        tau += __ldg(tau_s + j);
        ++j;
        if (cut && rawkey(tau) > rawkey(p.tau_v_max)) { over = true; break; }
      }
      if (over) break;
      tau += (s_kap[s] * (1.0 - pc)) * max0(p_exit - pc);
      if (cut && rawkey(tau) > rawkey(p.tau_v_max)) break;
      pc = p_exit;
      s += inner ? -1 : 1;
      if (s >= S) { out = true; break; }
      if (s < 0) break;  // met the inner boundary (only by rounding)
    }
    if (out) atomicAdd(p.spectrum_v + spectrum_bin(p, nu_lab), (e_v / D) * exp(-tau));
  }
}

template <int MODE, bool JB, bool REC>
__global__ void __launch_bounds__(kBlock) transport_fp64(const TransportParams p) {
  extern __shared__ double sh[];
  const int32_t S = p.S, L = p.L;
  for (int i = threadIdx.x; i < S; i += blockDim.x) {
    const double xi = p.x_in[i], xo = p.x_out[i], kap = p.kappa[i];
    sh[i] = xi * xi;
    sh[S + i] = xo * xo;
    sh[2 * S + i] = xi;
    sh[3 * S + i] = xo;
    sh[4 * S + i] = kap;
    sh[5 * S + i] = p.inv_kappa ? p.inv_kappa[i] : (kap > 0.0 ? 1.0 / kap : 0.0);
  }
  __syncthreads();
  const double *s_xi2 = sh, *s_xo2 = sh + S, *s_ikap = sh + 5 * S;
  const double *s_kap = sh + 4 * S;
  const double x0 = sh[2 * S], x0sq = sh[0];

  const unsigned lane = threadIdx.x & 31u;
  const unsigned lanemask_lt = (1u << lane) - 1u;
  const unsigned long long jb_pol = l2_evict_first_policy();
  const unsigned long long t_start = global_ns();
  uint32_t polls = 0u;  // loop iterations between looks at the host's stop request
  if (lane == 0u) atomicCAS(p.flags + 3, 0ull, t_start);

  Packet pk;
  DrawStream ds;
  WarpDraws wd;
  wd.init(reinterpret_cast<unsigned long long *>(sh + kShellArrays * S) +
          2 * kWarpDraws * (threadIdx.x >> 5));
  bool alive = false, finished = false;
  // Lone-walker mode: once the packet queue is empty and a warp is down to
  // one live walk, every lane of the warp takes that walk's state and runs
  // its segments together with the owner lane (the same instructions on the
  // same values, so the walk's results are those of the owner alone).  The
  // lanes then load the line list 32 lines at a time in one coalesced load
  // (line lwin_j0 + lane in each lane) and pass line data by shuffles;
  // only the owner lane makes the walk's side effects (estimator and J_blue
  // atomics, spectrum, records, statistics).
  bool lone = false;
  int owner = 0;
  int32_t lwin_j0 = 0, lwin_s = -1;
  long long lwin_b = 0;
  double lwin_t = 0.0;
  unsigned long long lwin_r = 0ull;
  uint32_t vdraws = 0u;  // v-packet draws used by this lane's packet
  unsigned long long n_esc = 0, n_reab = 0, n_cap = 0, n_seg = 0, n_chk = 0, n_res = 0, n_lint = 0,
                     n_esca = 0, n_shell = 0;
  int32_t acc_s = -1;
  double acc_j = 0.0, acc_nb = 0.0;
  const long long *nub = reinterpret_cast<const long long *>(p.nu);
  // the lane's current shell and its constants (reloaded on a shell change)
  int32_t cs = -1;
  double c_kap = 0.0, c_ikap = 0.0, c_xi2 = 0.0, c_xo2 = 0.0;
  // Lines next_line and next_line + 1 of the next segment (frequency bits,
  // Sobolev depth in the segment's shell, branching-row info), loaded by the
  // event that began it as soon as next_line is known, so that their latency
  // overlaps the event's arithmetic instead of opening the next scan.
  bool lw_ok = false;
  long long lw_b0 = 0, lw_b1 = 0;
  double lw_t0 = 0.0, lw_t1 = 0.0;
  unsigned long long lw_r0 = 0ull, lw_r1 = 0ull;
  auto load_window = [&](int32_t s_, int32_t j_) {
    const double *ts = p.tau + static_cast<size_t>(s_) * static_cast<size_t>(L);
    lw_b0 = 0; lw_t0 = 0.0; lw_r0 = 0ull; lw_b1 = 0; lw_t1 = 0.0; lw_r1 = 0ull;
    if (j_ < L) {
      lw_b0 = __ldg(nub + j_);
      lw_t0 = __ldg(ts + j_);
      if (MODE >= 1 && p.row_info) lw_r0 = __ldg(p.row_info + j_);
    }
    if (j_ + 1 < L) {
      lw_b1 = __ldg(nub + j_ + 1);
      lw_t1 = __ldg(ts + j_ + 1);
      if (MODE >= 1 && p.row_info) lw_r1 = __ldg(p.row_info + j_ + 1);
    }
    lw_ok = true;
  };
  auto lone_reload = [&](int32_t s_, int32_t j0) {
    lwin_j0 = j0;
    lwin_s = s_;
    const int32_t jj = j0 + static_cast<int32_t>(lane);
    lwin_b = 0;
    lwin_t = 0.0;
    lwin_r = 0ull;
    if (jj < L) {
      lwin_b = __ldg(nub + jj);
      lwin_t = __ldg(p.tau + static_cast<size_t>(s_) * static_cast<size_t>(L) + jj);
      if (MODE >= 1 && p.row_info) lwin_r = __ldg(p.row_info + jj);
    }
  };
  auto lone_fetch = [&](int32_t s_, int32_t jj, long long &b, double &t, unsigned long long &r) {
    int idx = jj - lwin_j0;
    if (lwin_s != s_ || idx < 0 || idx >= 32) {
      lone_reload(s_, jj);
      idx = 0;
    }
    b = __shfl_sync(0xffffffffu, lwin_b, idx);
    t = __shfl_sync(0xffffffffu, lwin_t, idx);
    r = __shfl_sync(0xffffffffu, lwin_r, idx);
  };

  for (;;) {
    // ---- claim packets for idle lanes (one atomic per warp; none in lone mode,
    // where every lane carries the walk until it ends)
    const bool need = !lone && !alive && !finished;
    const unsigned needmask = lone ? 0u : __ballot_sync(0xffffffffu, need);
    if (needmask) {
      const int leader = __ffs(needmask) - 1;
      unsigned long long base = 0ull;
      if (static_cast<int>(lane) == leader)
        base = atomicAdd(p.work_counter, static_cast<unsigned long long>(__popc(needmask)));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        const unsigned long long id = base + __popc(needmask & lanemask_lt);
        if (id < p.n_packets) {
          pk.pid = static_cast<uint32_t>(p.first_packet + id);
          ds.init(p.key0, p.key1, pk.pid, p.iteration);
          const double nu_cmf0 = inject(p, p.planck_cdf, x0, x0sq, pk, ds);
          alive = true;
          lw_ok = false;
          vdraws = 0u;
          if (p.n_virtual) {
            spawn_virtual(p, sh, VirtualLaunch{x0, x0sq, nu_cmf0, p.e_cmf, 0, pk.next_line, pk.pid, 0u, true});
            vdraws = static_cast<uint32_t>(p.n_virtual);
          }
        } else {
          finished = true;
          atomicCAS(p.flags + 1, 0ull, global_ns());
        }
      }
    }
    if (!lone && __all_sync(0xffffffffu, finished)) break;
    if (p.timeout_ns) {
      bool late = false;
      if (lane == 0u) late = (global_ns() - t_start) > p.timeout_ns;
      late = __shfl_sync(0xffffffffu, late, 0);
      if (late) {
        if (lane == 0u) atomicExch(p.flags, 1ull);
        break;
      }
    }
    if (p.cancel && (++polls & 255u) == 0u) {  // the host's stop request (mc_cancel)
      uint32_t stop = 0u;
      if (lane == 0u) stop = load_sys_u32(p.cancel);
      stop = __shfl_sync(0xffffffffu, stop, 0);
      if (stop) {
        if (lane == 0u) atomicExch(p.flags, 2ull);
        break;
      }
    }
    // ---- a warp's last live walk: the idle lanes compute its draws ahead
    if (lone) {
      wd.keep(ds, p.key0, p.key1, p.iteration, lane);
    } else {
      wd.prepare(alive, __any_sync(0xffffffffu, finished), ds, pk.pid, p.key0, p.key1, p.iteration, lane);
      if (wd.on && !p.n_virtual) {
        // enter lone-walker mode: the other lanes' packets are done; they hand
        // their estimator sums over and take the walk's state
        owner = __ffs(__ballot_sync(0xffffffffu, alive)) - 1;
        if (!alive && acc_s >= 0) {
          atomicAdd(p.j_est + acc_s, acc_j);
          atomicAdd(p.nu_bar + acc_s, acc_nb);
        }
        const unsigned F = 0xffffffffu;
        pk.p = __shfl_sync(F, pk.p, owner);
        pk.q = __shfl_sync(F, pk.q, owner);
        pk.nu_lab = __shfl_sync(F, pk.nu_lab, owner);
        pk.e_per_nu = __shfl_sync(F, pk.e_per_nu, owner);
        pk.inv_nu = __shfl_sync(F, pk.inv_nu, owner);
        pk.D = __shfl_sync(F, pk.D, owner);
        pk.inv_D = __shfl_sync(F, pk.inv_D, owner);
        pk.nu_cmf = __shfl_sync(F, pk.nu_cmf, owner);
        pk.eD2 = __shfl_sync(F, pk.eD2, owner);
        pk.shell = __shfl_sync(F, pk.shell, owner);
        pk.next_line = __shfl_sync(F, pk.next_line, owner);
        pk.pid = __shfl_sync(F, pk.pid, owner);
        pk.have_cmf = __shfl_sync(F, static_cast<int>(pk.have_cmf), owner) != 0;
#pragma unroll
        for (int c = 0; c < kNCounters; ++c) pk.cnt[c] = __shfl_sync(F, pk.cnt[c], owner);
        ds.k0 = __shfl_sync(F, ds.k0, owner);
        ds.k1 = __shfl_sync(F, ds.k1, owner);
        ds.packet = __shfl_sync(F, ds.packet, owner);
        ds.iteration = __shfl_sync(F, ds.iteration, owner);
        ds.d = __shfl_sync(F, ds.d, owner);
        ds.spare_a = __shfl_sync(F, ds.spare_a, owner);
        ds.spare_b = __shfl_sync(F, ds.spare_b, owner);
        cs = __shfl_sync(F, cs, owner);
        c_kap = __shfl_sync(F, c_kap, owner);
        c_ikap = __shfl_sync(F, c_ikap, owner);
        c_xi2 = __shfl_sync(F, c_xi2, owner);
        c_xo2 = __shfl_sync(F, c_xo2, owner);
        acc_s = __shfl_sync(F, acc_s, owner);
        acc_j = __shfl_sync(F, acc_j, owner);
        acc_nb = __shfl_sync(F, acc_nb, owner);
        vdraws = __shfl_sync(F, vdraws, owner);
        lwin_s = -1;
        alive = true;
        lone = true;
      }
    }
    if (!alive) continue;
    const bool act = !lone || static_cast<int>(lane) == owner;  // makes the walk's side effects

    // ---- one flight segment (Sect. 2.6)
    int status = 0;
    if (pk.cnt[0] >= p.max_segments) {
      status = 3;  // capped
    } else {
      pk.cnt[0] += 1u;
      const int32_t s = pk.shell;
      const double pp = pk.p, q = pk.q, nu_lab = pk.nu_lab, inv_nu = pk.inv_nu;
      if (!pk.have_cmf) {
        // after a shell crossing: Doppler factor D = 1 - mu v/c at the boundary
        // point, comoving frequency and E_cmf D (Sect. 2.5)
        const double D0 = 1.0 - pp;
        pk.D = D0;
        pk.inv_D = rcp64(D0);
        pk.nu_cmf = nu_lab * D0;
        pk.eD2 = (pk.e_per_nu * pk.nu_cmf) * D0;  // E_cmf D
        pk.have_cmf = true;
      }
      const double D = pk.D, inv_D = pk.inv_D, nu_cmf = pk.nu_cmf, eD2 = pk.eD2;
      if (s != cs) {
        cs = s;
        c_kap = s_kap[s];
        c_ikap = s_ikap[s];
        c_xi2 = s_xi2[s];
        c_xo2 = s_xo2[s];
      }
      const bool thomson = rawkey(c_kap) > 0;
      // optical depth to the next event, tau = -ln z
      double tau_rem = wd.template next_tau<MODE == 2>(ds);
      // Shell boundary: at the exit point x mu = p_exit = +-sqrt(x_b^2 - q) (the
      // inner sphere is hit when moving inward with q <= x_in^2), so the path
      // length is p_exit - p and the comoving frequency there nu_lab (1 - p_exit).
      // That frequency orders the lines passed against the exit; it is first
      // bracketed in binary32 (shell_bracket) and taken exactly (binary64
      // root) only for a value inside the bracket or when the shell event
      // wins.  An event at path length l with no line passed before it is
      // placed against the exit through x^2 = q + (p+l)^2 at the event point,
      // the same p + l and x^2 the move to the event computes.
      const double xi2 = c_xi2, xo2 = c_xo2;
      const bool inner = strictly_negative(pp) && rawkey(q) <= rawkey(xi2);  // q, x_in^2 >= 0
      int shell_state = 0;  // 0 nothing known, 1 bracket [klo, khi], 2 exact (klo = khi = key)
      long long klo = 0, khi = 0;
      double p_exit = 0.0;
      auto exact_exit = [&]() {
        p_exit = shell_exit(q, inner, xi2, xo2);
        klo = khi = rawkey(nu_lab * (1.0 - p_exit));  // > 0
        shell_state = 2;
      };
      // is a Sobolev point or threshold at comoving frequency key beyond the exit?
      auto beyond_exit = [&](long long key) -> bool {
        if (key > khi) return false;
        if (key > klo) exact_exit();
        return key <= klo;
      };
      double c_e = 0.0, thr_e = 0.0;
      long long key_e = kKeyNegInf;
      if (thomson) {
        c_e = (nu_lab * c_ikap) * inv_D;  // nu_lab / k, k = kappa' D
        thr_e = fma(-tau_rem, c_e, nu_cmf);
        key_e = rawkey(thr_e);
      }
      // J_blue weight of this segment, E_lab / nu_lab^2 (Eq. 17 without its
      // line factor nu_j, applied per cell after the launch)
      const double e_inv2 = JB ? pk.e_per_nu * inv_nu : 0.0;
      const size_t row = static_cast<size_t>(s) * static_cast<size_t>(L);
      const double *tau_s = p.tau + row;
      int32_t j = pk.next_line;
      int kind = 0;
      double l = 0.0, nu_hit = 0.0;
      double pl_ev = 0.0, r2_ev = 0.0;  // x mu and x^2 at the event, when the exit test made them
      bool have_ev = false;
      double D1_ev = 0.0;  // Doppler factor at an electron-scattering point
      unsigned long long rinfo_hit = 0ull;
      // two lines ahead are always in flight while line j is resolved
      long long bj = 0, bj_n = 0;
      double taul = 0.0, tau_n = 0.0;
      unsigned long long rinfo = 0ull, rinfo_n = 0ull;
      // An absorbing line (Sect. 2.6): the Sobolev point nu_lab (1 - x mu) =
      // nu_j, so x mu = 1 - nu_j / nu_lab and D = nu_j / nu_lab there (a
      // resonance that rounding puts behind the packet is taken where the
      // packet is).  With no line passed yet the event point is also placed
      // against the shell exit; if the exit comes first the scan ends with no
      // event (kind stays 0).
      auto absorb = [&](long long b_, unsigned long long r_) {
        const double nuj = __longlong_as_double(b_);
        const double lj = max0(fma(-nuj, inv_nu, D));
        const bool ahead = rawkey(lj) > 0;
        pl_ev = ahead ? fma(-nuj, inv_nu, 1.0) : pp;
        r2_ev = fma(pl_ev, pl_ev, q);
        have_ev = true;
        if (shell_state == 0 && !inside_shell(pl_ev, r2_ev, inner, xi2, xo2)) return;  // exit comes first
        pk.cnt[2] += 1u;
        if (JB && act) red_add_evict_first(p.j_blue + row + j, e_inv2, jb_pol);
        kind = kLineEvent;
        l = lj;
        nu_hit = nuj;
        rinfo_hit = r_;
      };
      bool fast = false;  // the lone scan below settled the segment's line event
      // downbranch: the absorbing line's emission record, loaded as soon as the
      // lone scan names the line (the emission draw is the next in the buffer)
      bool have_slot = false;
      ulonglong2 slot_a = make_ulonglong2(0ull, 0ull), slot_c = make_ulonglong2(0ull, 0ull);
      if (lone) {
        int idx = j - lwin_j0;
        if (lwin_s != s || idx < 0 || idx >= 32) {
          lone_reload(s, j);
          idx = 0;
        }
        if (thomson) {
          // The scan of lines j0 + idx .. j0 + 31 of the window in one step, lane
          // k taking line j0 + k.  In exact arithmetic the scan below stops at
          // line k when nu_k <= T_{k-1} (beyond d_e), when nu_k lies beyond the
          // shell exit, or when T_k > nu_k (absorbed), with T_k = thr_e + c_e
          // (tau_idx + ... + tau_k).  Each lane forms A = nu_k - T_{k-1} and B =
          // nu_k - T_k in binary32 from the exact binary64 difference nu_k - thr_e
          // (one binary64 instruction for the whole window) and a prefix sum of
          // the depths, with a bound M on |error| that also covers the rounding
          // of the scan's own chain of fmas (at most 32 of them).  Where every
          // sign up to the first line that stops the scan is certain and that
          // line absorbs, the result is the scan's; otherwise (a sign within
          // the bound, the exit, d_e or the end of the window reached) the scan
          // below runs as usual.  Error budget (u = 2^-24): the difference
          // truncated to binary32 (2u), the depths truncated (2u) and summed in
          // five levels (5u), c_e truncated (2u), the product and the final
          // difference (u each), so |A|, |B| error <= 3u |d| + 11u C; the fma
          // chain adds at most 2^-48 (|thr_e| + C); depths below the binary32
          // normal range add at most 32 c_e 2^-126.  M = 2^-20 (|d| + C) +
          // 2^-44 |thr_e| + c_e 2^-119 + 2^-124 bounds all of it.
          const ShellBracket sb = shell_bracket(q, inner ? xi2 : xo2, inner, nu_lab);
          const int32_t jl = lwin_j0 + static_cast<int32_t>(lane);
          const bool cand = static_cast<int>(lane) >= idx;
          const bool valid = cand && jl < L;
          const float dk = f32_rz_any(__longlong_as_double(lwin_b) - thr_e);
          float P = valid ? f32_rz_any(lwin_t) : 0.0f;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const float y = __shfl_up_sync(0xffffffffu, P, o);
            if (static_cast<int>(lane) >= o) P = __fadd_rn(P, y);
          }
          float Px = __shfl_up_sync(0xffffffffu, P, 1);
          if (lane == 0u) Px = 0.0f;
          const float ce = f32_rz_any(c_e);
          const float C = __fmul_rn(ce, P);
          const float A = __fsub_rn(dk, __fmul_rn(ce, Px)), B = __fsub_rn(dk, C);
          const float M = __fadd_rn(__fmul_rn(0x1.0p-20f, __fadd_rn(fabsf(dk), C)),
                                    __fadd_rn(__fmul_rn(0x1.0p-44f, fabsf(f32_rz_any(thr_e))),
                                              __fmaf_rn(ce, 0x1.0p-119f, 0x1.0p-124f)));
          const bool e_no = A > M;                               // certainly before d_e
          const bool a_yes = B < -M, a_no = B > M;               // certainly absorbed / passed
          const bool x_no = sb.ok && lwin_b > sb.hi;             // certainly before the exit
          const bool pass = valid && e_no && a_no && x_no;
          const bool take = valid && e_no && a_yes && (static_cast<int>(lane) == idx || x_no);
          const unsigned stop = __ballot_sync(0xffffffffu, cand && !pass);
          const unsigned took = __ballot_sync(0xffffffffu, take);
          const int kstar = __ffs(stop) - 1;
          if (kstar >= 0 && ((took >> kstar) & 1u)) {
            fast = true;
            const int npass = kstar - idx;
            pk.cnt[1] += static_cast<uint32_t>(npass + 1);
            pk.cnt[2] += static_cast<uint32_t>(npass);
            if (JB && cand && static_cast<int>(lane) < kstar)  // the lines passed, one lane each
              red_add_evict_first(p.j_blue + row + jl, e_inv2, jb_pol);
            if (npass > 0) {  // as the scan leaves it after its first pass
              klo = sb.lo;
              khi = sb.hi;
              shell_state = 1;
            }
            j = lwin_j0 + kstar;
            bj = __shfl_sync(0xffffffffu, lwin_b, kstar);
            rinfo = __shfl_sync(0xffffffffu, lwin_r, kstar);
            if (MODE == 1 && p.dbr_rec) {
              load_slot(bucket_slot(p, rinfo, wd.peek_u53(ds)), slot_a, slot_c);
              have_slot = true;
            }
          }
        }
        if (!fast) {
          lone_fetch(s, j, bj, taul, rinfo);
          lone_fetch(s, j + 1, bj_n, tau_n, rinfo_n);
        }
      } else {
        if (!lw_ok) load_window(s, j);
        bj = lw_b0; taul = lw_t0; rinfo = lw_r0;
        bj_n = lw_b1; tau_n = lw_t1; rinfo_n = lw_r1;
      }
      lw_ok = false;
      long long bj_nn = 0;
      double tau_nn = 0.0;
      unsigned long long rinfo_nn = 0ull;
      if (fast) absorb(bj, rinfo);
      else while (j < L) {
        pk.cnt[1] += 1u;
        bj_nn = 0;
        tau_nn = 0.0;
        rinfo_nn = 0ull;
        if (lone) {
          lone_fetch(s, j + 2, bj_nn, tau_nn, rinfo_nn);
        } else if (j + 2 < L) {
          bj_nn = __ldg(nub + j + 2);
          tau_nn = __ldg(tau_s + j + 2);
          if (MODE >= 1 && p.row_info) rinfo_nn = __ldg(p.row_info + j + 2);
        }
        if (bj <= key_e) break;                             // the Sobolev point lies beyond d_e
        if (shell_state != 0 && beyond_exit(bj)) break;     // ... or beyond the shell exit
        bool absorbed;
        double t = 0.0;
        if (thomson) {
          t = fma(taul, c_e, thr_e);
          absorbed = rawkey(t) > bj;  // nu_j > 0
        } else {
          absorbed = rawkey(taul) > rawkey(tau_rem);  // both >= 0
        }
        if (absorbed) {
          absorb(bj, rinfo);
          break;
        }
        if (shell_state == 0) {  // a line is passed: the scan needs the exit frequency
          const ShellBracket sb = shell_bracket(q, inner ? xi2 : xo2, inner, nu_lab);
          if (sb.ok) {
            klo = sb.lo;
            khi = sb.hi;
            shell_state = 1;
          } else {
            exact_exit();
          }
          if (beyond_exit(bj)) break;  // this line lies beyond the exit
        }
        pk.cnt[2] += 1u;
        if (JB && act) red_add_evict_first(p.j_blue + row + j, e_inv2, jb_pol);
        if (thomson) {
          thr_e = t;
          key_e = rawkey(t);
        } else {
          tau_rem -= taul;
        }
        ++j;
        bj = bj_n; taul = tau_n; rinfo = rinfo_n;
        bj_n = bj_nn; tau_n = tau_nn; rinfo_n = rinfo_nn;
      }
      if (kind == 0) {
        bool electron;
        double le = 0.0;
        have_ev = false;  // an absorbed line that lay beyond the exit left its point here
        if (shell_state != 0) {
          electron = thomson && !beyond_exit(key_e);
          if (electron) le = max0(fma(-thr_e, inv_nu, D));
        } else {
          le = thomson ? max0(fma(-thr_e, inv_nu, D)) : 0.0;
          if (thomson) {
            pl_ev = pp + le;
            r2_ev = fma(pl_ev, pl_ev, q);
            have_ev = true;
          }
          electron = thomson && inside_shell(pl_ev, r2_ev, inner, xi2, xo2);
        }
        if (electron) {
          kind = kElectronEvent;
          l = le;
          if (!have_ev) {
            pl_ev = pp + le;
            r2_ev = fma(pl_ev, pl_ev, q);
            have_ev = true;
          }
          D1_ev = 1.0 - pl_ev;
        } else {
          if (shell_state != 2) exact_exit();
          kind = kShellEvent;
          l = max0(p_exit - pp);
          have_ev = false;
        }
      }
      // estimators, Eqs. 13-14 (segment-start comoving values)
      const double wgt = eD2 * l;
      if (s != acc_s) {
        if (acc_s >= 0 && act) {
          atomicAdd(p.j_est + acc_s, acc_j);
          atomicAdd(p.nu_bar + acc_s, acc_nb);
        }
        acc_s = s; acc_j = 0.0; acc_nb = 0.0;
      }
      acc_j += wgt;
      acc_nb = fma(wgt, nu_cmf, acc_nb);
      pk.next_line = j;
      if (kind == kShellEvent) {
        // move to the boundary; free flight keeps q, nu_lab and E_lab
        pk.cnt[5] += 1u;
        const int32_t ns = inner ? s - 1 : s + 1;
        pk.p = p_exit;
        pk.shell = ns;
        pk.have_cmf = false;
        lw_ok = false;
        if (ns >= S) status = 1;
        else if (ns < 0) status = 2;
      } else {
        // move to the event point (x mu, x^2 and D there from the scan)
        const double r2n = r2_ev;
        const double xn = sqrt64(r2n);
        // comoving energy at the event: E / nu times the comoving frequency
        // there (the line's own frequency at a Sobolev point)
        double nu_c, inv_nu_c, e_c;
        if (kind == kLineEvent) {
          pk.cnt[3] += 1u;
          e_c = pk.e_per_nu * nu_hit;
          if (MODE >= 1) {
            // MODE 2: macro atom, internal jumps before the emission pick
            const unsigned long long rinfo_em =
                MODE == 2 ? macroatom_walk(p, __ldg(p.line_row + j), wd, ds) : rinfo_hit;
            const unsigned long long u_em = wd.template next_u53<MODE == 2>(ds);
            const Emission em = have_slot ? pick_from_slot_lone(p, rinfo_em, u_em, slot_a, slot_c, lane)
                                          : downbranch_pick(p, j, rinfo_em, u_em);
            nu_c = em.nu;
            inv_nu_c = em.inv_nu;
            pk.e_per_nu = e_c * inv_nu_c;  // re-emitted at another frequency
            pk.next_line = em.line + 1;
            if (lone) lone_reload(s, pk.next_line);
            else load_window(s, pk.next_line);
          } else {
            nu_c = nu_hit;
            inv_nu_c = rcp64(nu_hit);
            pk.next_line = j + 1;
            lw_ok = true;  // lines j + 1, j + 2 are in the scan's registers
            lw_b0 = bj_n; lw_t0 = tau_n; lw_r0 = rinfo_n;
            lw_b1 = bj_nn; lw_t1 = tau_nn; lw_r1 = rinfo_nn;
          }
        } else {
          pk.cnt[4] += 1u;
          nu_c = nu_lab * D1_ev;
          inv_nu_c = inv_nu * rcp64(D1_ev);
          e_c = pk.e_per_nu * nu_c;
          lw_ok = true;  // the next segment starts at line j again
          lw_b0 = bj; lw_t0 = taul; lw_r0 = rinfo;
          lw_b1 = bj_n; lw_t1 = tau_n; lw_r1 = rinfo_n;
        }
        // isotropic re-emission: new direction, lab values from the comoving ones
        const double mu2 = DrawStream::mu_from_u53(wd.template next_u53<MODE == 2>(ds));
        const double pn = xn * mu2;
        const double D2 = 1.0 - pn;
        const double iD2 = rcp64(D2);
        pk.p = pn;
        pk.q = max0(fma(-pn, pn, r2n));
        pk.nu_lab = nu_c * iD2;
        pk.inv_nu = inv_nu_c * D2;
        pk.D = D2;
        pk.inv_D = iD2;
        pk.nu_cmf = nu_c;       // = nu_lab D2
        pk.eD2 = e_c * D2;      // = E_lab D2^2
        pk.have_cmf = true;
        if (p.n_virtual && act) {
          spawn_virtual(p, sh, VirtualLaunch{xn, r2n, nu_c, e_c, s, pk.next_line, pk.pid, vdraws, false});
          vdraws += static_cast<uint32_t>(p.n_virtual);
        }
      }
    }
    if (status != 0 && !act) {  // lone mode, not the owner lane: drop the adopted walk
      alive = false;
      lone = false;
      acc_s = -1;
      acc_j = 0.0;
      acc_nb = 0.0;
    } else if (status != 0) {
      lone = false;
      if (status == 1) ++n_esc;
      else if (status == 2) ++n_reab;
      else ++n_cap;
      n_seg += pk.cnt[0];
      n_chk += pk.cnt[1];
      n_res += pk.cnt[2];
      n_lint += pk.cnt[3];
      n_esca += pk.cnt[4];
      n_shell += pk.cnt[5];
      const double e_lab = pk.e_per_nu * pk.nu_lab;
      if (status == 1) atomicAdd(p.spectrum + spectrum_bin(p, pk.nu_lab), e_lab);
      if (REC) {
        p.rec_status[pk.pid - p.first_packet] = status;
        p.rec_nu[pk.pid - p.first_packet] = pk.nu_lab;
        p.rec_e[pk.pid - p.first_packet] = e_lab;
#pragma unroll
        for (int c = 0; c < kNCounters; ++c)
          p.rec_cnt[static_cast<size_t>(pk.pid - p.first_packet) * kNCounters + c] = pk.cnt[c];
      }
      alive = false;
    }
  }
  if (acc_s >= 0 && (!lone || static_cast<int>(lane) == owner)) {  // (a launch stopped in lone mode)
    atomicAdd(p.j_est + acc_s, acc_j);
    atomicAdd(p.nu_bar + acc_s, acc_nb);
  }
  unsigned long long st[kNStats] = {n_esc, n_reab, n_cap, n_seg, n_chk, n_res, n_lint, n_esca, n_shell};
#pragma unroll
  for (int i = 0; i < kNStats; ++i) {
    unsigned long long v = st[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0u && v) atomicAdd(p.stats + i, v);
  }
  if (lane == 0u) atomicMax(p.flags + 2, global_ns());
}

template <int MODE, bool JB, bool REC>
const void *kernel_ptr() {
  return reinterpret_cast<const void *>(&transport_fp64<MODE, JB, REC>);
}

const void *select_kernel(int line_mode, int precision, bool jb, bool rec) {
  if (precision == 1) return select_mixed_kernel(line_mode, jb, rec);
  if (line_mode == 0) {
    if (jb) return rec ? kernel_ptr<0, true, true>() : kernel_ptr<0, true, false>();
    return rec ? kernel_ptr<0, false, true>() : kernel_ptr<0, false, false>();
  }
  if (line_mode == 2) {
    if (jb) return rec ? kernel_ptr<2, true, true>() : kernel_ptr<2, true, false>();
    return rec ? kernel_ptr<2, false, true>() : kernel_ptr<2, false, false>();
  }
  if (jb) return rec ? kernel_ptr<1, true, true>() : kernel_ptr<1, true, false>();
  return rec ? kernel_ptr<1, false, true>() : kernel_ptr<1, false, false>();
}

size_t smem_bytes(int S, int precision) {
  // binary64: shell tables, then one WarpDraws buffer (u53 + -ln z) per warp
  return precision == 1 ? mixed_smem_bytes(S)
                        : static_cast<size_t>(kShellArrays) * S * sizeof(double) +
                              (kBlock / 32) * 2 * kWarpDraws * sizeof(double);
}

}  // namespace

int transport_block_size() { return kBlock; }

cudaError_t transport_occupancy(int line_mode, int precision, bool j_blue, bool record, int S,
                                int *blocks_per_sm) {
  const void *k = select_kernel(line_mode, precision, j_blue, record);
  const size_t smem = smem_bytes(S, precision);
  if (smem > 48 * 1024) {  // the query, like the launch, needs the opt-in above 48 KB
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(smem));
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, kBlock, smem);
}

cudaError_t launch_transport(const TransportParams &p, int line_mode, int precision, bool j_blue,
                             bool record, int grid, int block, cudaStream_t st) {
  // the shared-memory layout (one draw buffer per warp) is sized for kBlock
  if (block != kBlock) return cudaErrorInvalidValue;
  const void *k = select_kernel(line_mode, precision, j_blue, record);
  const size_t smem = smem_bytes(p.S, precision);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
  }
  void *args[] = {const_cast<TransportParams *>(&p)};
  return cudaLaunchKernel(k, dim3(grid), dim3(block), args, smem, st);
}

}  // namespace mcgpu
