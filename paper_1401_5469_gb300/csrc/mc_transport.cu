// Monte Carlo packet transport through homologously expanding shells
// (Kerzendorf & Sim 2014, Sects. 2.4-2.7 and 2.9), one packet per thread in a
// persistent grid.
//
// GB300 notes.  Binary64 add/mul/fma/compare issue at 1/64 of the binary32
// rate and every binary64 warp instruction holds its warp for ~64 cycles,
// whatever the number of active lanes.  The kernel therefore
//  * keeps lanes converged: a lane that finishes its packet claims the next
//    one at the loop head (warp-aggregated atomic), and the three event kinds
//    share one code path;
//  * runs every comparison of the line scan on the integer pipe, comparing
//    order-preserving int64 keys of binary64 values: the resonance test
//    "d_line < min(d_e, d_shell)" becomes "nu_line > nu_threshold" with
//    nu_threshold = nu_cmf - d_min nu_lab (d_line is linear in nu_line);
//  * accumulates the shell estimators in registers while a packet stays in
//    one shell and flushes them with one atomic per shell change.
#include <cstdint>

#include "mc_device.cuh"
#include "mc_internal.h"

namespace mcgpu {

namespace {

constexpr int kBlock = 128;
constexpr int kLineEvent = 1, kElectronEvent = 2, kShellEvent = 3;

struct Packet {
  double x, mu, nu_lab, e_lab;
  int32_t shell, next_line;
  uint32_t pid;
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

// First entry k of a branching row with z < cdf[k] (cdf non-decreasing, last
// entry 1 > z): binary search on int64 images (all values non-negative).
__device__ __forceinline__ int32_t downbranch_pick(const TransportParams &p, int32_t row, double z) {
  uint32_t lo = __ldg(p.dbr_offset + row), hi = __ldg(p.dbr_offset + row + 1) - 1u;
  const long long kz = __double_as_longlong(z);
  const long long *cb = reinterpret_cast<const long long *>(p.dbr_cdf);
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (kz < __ldg(cb + mid)) hi = mid; else lo = mid + 1u;
  }
  return static_cast<int32_t>(__ldg(p.dbr_line + lo));
}

// Injection at the inner boundary, Sect. 2.4: Planck-sampled comoving
// frequency (Carter & Cashwell series method), mu = sqrt(z), equal comoving
// energy (Eq. 10), lab-frame values by the first-order Doppler factor.
__device__ __forceinline__ void inject(const TransportParams &p, Packet &pk, DrawStream &ds) {
  const double z0 = ds.closed0();
  const double z1 = ds.open0(), z2 = ds.open0(), z3 = ds.open0(), z4 = ds.open0();
  int l = 1;
  while (l < kPlanckLmax && __ldg(p.planck_cdf + l) < z0) ++l;
  const double xi = -log(((z1 * z2) * z3) * z4) / static_cast<double>(l);
  const double nu_cmf = p.nu_scale * xi;
  const double mu = sqrt(ds.open0());
  const double x = __ldg(p.x_in);
  const double D = fma(-mu, x, 1.0);
  const double iD = 1.0 / D;
  pk.x = x;
  pk.mu = mu;
  pk.nu_lab = nu_cmf * iD;
  pk.e_lab = p.e_cmf * iD;
  pk.shell = 0;
  pk.next_line = first_redward(p.nu, p.L, nu_cmf);
#pragma unroll
  for (int c = 0; c < kNCounters; ++c) pk.cnt[c] = 0u;
}

template <int MODE, bool JB, bool REC>
__global__ void __launch_bounds__(kBlock) transport_fp64(const TransportParams p) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lanemask_lt = (1u << lane) - 1u;
  const int32_t S = p.S, L = p.L;
  const unsigned long long t_start = p.timeout_ns ? global_ns() : 0ull;

  Packet pk;
  DrawStream ds;
  bool alive = false, finished = false;
  unsigned long long st[kNStats];
#pragma unroll
  for (int i = 0; i < kNStats; ++i) st[i] = 0ull;
  int32_t acc_s = -1;
  double acc_j = 0.0, acc_nb = 0.0;

  for (;;) {
    // ---- claim packets for idle lanes (one atomic per warp)
    const bool need = !alive && !finished;
    const unsigned needmask = __ballot_sync(0xffffffffu, need);
    if (needmask) {
      const int leader = __ffs(needmask) - 1;
      unsigned long long base = 0ull;
      if (static_cast<int>(lane) == leader)
        base = atomicAdd(p.work_counter, static_cast<unsigned long long>(__popc(needmask)));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        const unsigned long long id = base + __popc(needmask & lanemask_lt);
        if (id < p.n_packets) {
          pk.pid = static_cast<uint32_t>(id);
          ds.init(p.key0, p.key1, pk.pid, p.iteration);
          inject(p, pk, ds);
          alive = true;
        } else {
          finished = true;
        }
      }
    }
    if (__all_sync(0xffffffffu, finished)) break;
    if (p.timeout_ns) {
      bool late = false;
      if (lane == 0u) late = (global_ns() - t_start) > p.timeout_ns;
      late = __shfl_sync(0xffffffffu, late, 0);
      if (late) {
        if (lane == 0u) atomicExch(p.flags, 1ull);
        break;
      }
    }
    if (!alive) continue;

    // ---- one flight segment (Sect. 2.6)
    int status = 0;
    if (pk.cnt[0] >= p.max_segments) {
      status = 3;  // capped
    } else {
      pk.cnt[0] += 1u;
      const int32_t s = pk.shell;
      const double x = pk.x, mu = pk.mu, nu_lab = pk.nu_lab;
      // Doppler factor, comoving frequency/energy, Thomson opacity (Eq. 11)
      const double D = fma(-mu, x, 1.0);
      const double nu_cmf = nu_lab * D;
      const double e_cmf = pk.e_lab * D;
      const double k = __ldg(p.kappa + s) * D;
      double tau_rem = -log(ds.open0());
      // distance to the shell boundary
      const double pm = x * mu;
      const double xo = __ldg(p.x_out + s), xi = __ldg(p.x_in + s);
      const double ao = (xo - x) * (xo + x);
      const double ai = (xi - x) * (xi + x);
      const bool inner = (mu < 0.0) && (fma(pm, pm, ai) >= 0.0);
      const double root = sqrt(fma(pm, pm, inner ? ai : ao));
      double num, den;
      if (inner) { num = -ai; den = root - pm; }
      else if (mu >= 0.0) { num = ao; den = root + pm; }
      else { num = root - pm; den = 1.0; }
      const double d_shell = fmax(num / den, 0.0);
      // resonance thresholds on the line frequency
      const double inv_nu = 1.0 / nu_lab;
      const long long key_shell = okey(fma(-d_shell, nu_lab, nu_cmf));
      double inv_k = 0.0, c_e = 0.0;
      long long key_e = kKeyNegInf;
      if (k > 0.0) {
        inv_k = 1.0 / k;
        c_e = nu_lab * inv_k;
        key_e = okey(fma(-tau_rem, c_e, nu_cmf));
      }
      long long key_thr = key_shell > key_e ? key_shell : key_e;
      const double e_inv2 = JB ? (pk.e_lab * inv_nu) * inv_nu : 0.0;
      const size_t row = static_cast<size_t>(s) * static_cast<size_t>(L);
      const long long *nub = reinterpret_cast<const long long *>(p.nu);
      int32_t j = pk.next_line;
      int kind = 0;
      double l = 0.0;
      // walk the redward lines while a Sobolev point is the closest event
      while (j < L) {
        pk.cnt[1] += 1u;
        const long long bj = __ldg(nub + j);
        if (bj <= key_thr) break;
        pk.cnt[2] += 1u;
        const double nuj = __longlong_as_double(bj);
        const double d_line = fmax(fma(-nuj, inv_nu, D), 0.0);
        if (JB) atomicAdd(p.j_blue + row + j, nuj * e_inv2);
        const double taul = __ldg(p.tau + row + j);
        if (okey(taul) > okey(fma(-k, d_line, tau_rem))) { kind = kLineEvent; l = d_line; break; }
        tau_rem -= taul;
        if (k > 0.0) {
          key_e = okey(fma(-tau_rem, c_e, nu_cmf));
          key_thr = key_shell > key_e ? key_shell : key_e;
        }
        ++j;
      }
      if (kind == 0) {
        if (key_e > key_shell) { kind = kElectronEvent; l = tau_rem * inv_k; }
        else { kind = kShellEvent; l = d_shell; }
      }
      // estimators, Eqs. 13-14 (segment-start comoving values)
      const double wgt = (e_cmf * l) * D;
      if (s != acc_s) {
        if (acc_s >= 0) {
          atomicAdd(p.j_est + acc_s, acc_j);
          atomicAdd(p.nu_bar + acc_s, acc_nb);
        }
        acc_s = s; acc_j = 0.0; acc_nb = 0.0;
      }
      acc_j += wgt;
      acc_nb = fma(wgt, nu_cmf, acc_nb);
      pk.next_line = j;
      if (kind == kShellEvent) {
        pk.cnt[5] += 1u;
        const int32_t ns = inner ? s - 1 : s + 1;
        const double xb = inner ? xi : xo;
        const double inv_xb = __ldg((inner ? p.inv_x_in : p.inv_x_out) + s);
        pk.mu = fmin(fmax((pm + l) * inv_xb, -1.0), 1.0);
        pk.x = xb;
        pk.shell = ns;
        if (ns >= S) status = 1;
        else if (ns < 0) status = 2;
      } else {
        // move to the event point (impact parameter conserved)
        const double q = fmax(fma(x, x, -pm * pm), 0.0);
        const double pl = pm + l;
        const double xn = sqrt(fma(pl, pl, q));
        const double mun = fmin(fmax(pl / xn, -1.0), 1.0);
        const double D1 = fma(-mun, xn, 1.0);
        const double e_c = pk.e_lab * D1;
        double nu_c;
        if (kind == kLineEvent) {
          pk.cnt[3] += 1u;
          int32_t emit = j;
          if (MODE == 1) emit = downbranch_pick(p, __ldg(p.line_row + j), ds.closed0());
          nu_c = __ldg(p.nu + emit);
          pk.next_line = emit + 1;
        } else {
          pk.cnt[4] += 1u;
          nu_c = nu_lab * D1;
        }
        const double mu2 = fma(2.0, ds.closed0(), -1.0);
        const double iD2 = 1.0 / fma(-mu2, xn, 1.0);
        pk.x = xn;
        pk.mu = mu2;
        pk.nu_lab = nu_c * iD2;
        pk.e_lab = e_c * iD2;
      }
    }
    if (status != 0) {
      st[status - 1] += 1ull;
      st[kStSegments] += pk.cnt[0];
      st[kStLineChecks] += pk.cnt[1];
      st[kStResonances] += pk.cnt[2];
      st[kStLineInteractions] += pk.cnt[3];
      st[kStEScatters] += pk.cnt[4];
      st[kStShellCrossings] += pk.cnt[5];
      if (status == 1) {
        // bin index; underflow -> bins, overflow (or NaN) -> bins + 1
        int b;
        if (pk.nu_lab < p.spec_lo) b = p.spec_bins;
        else {
          const double t = (pk.nu_lab - p.spec_lo) / p.spec_dnu;
          b = (t >= 0.0 && t < static_cast<double>(p.spec_bins)) ? static_cast<int>(floor(t))
                                                                   : p.spec_bins + 1;
        }
        atomicAdd(p.spectrum + b, pk.e_lab);
      }
      if (REC) {
        p.rec_status[pk.pid] = status;
        p.rec_nu[pk.pid] = pk.nu_lab;
        p.rec_e[pk.pid] = pk.e_lab;
#pragma unroll
        for (int c = 0; c < kNCounters; ++c)
          p.rec_cnt[static_cast<size_t>(pk.pid) * kNCounters + c] = pk.cnt[c];
      }
      alive = false;
    }
  }
  if (acc_s >= 0) {
    atomicAdd(p.j_est + acc_s, acc_j);
    atomicAdd(p.nu_bar + acc_s, acc_nb);
  }
#pragma unroll
  for (int i = 0; i < kNStats; ++i) {
    unsigned long long v = st[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0u && v) atomicAdd(p.stats + i, v);
  }
}

template <int MODE, bool JB, bool REC>
const void *kernel_ptr(int precision) {
  (void)precision;
  return reinterpret_cast<const void *>(&transport_fp64<MODE, JB, REC>);
}

const void *select_kernel(int line_mode, int precision, bool jb, bool rec) {
  if (line_mode == 0) {
    if (jb) return rec ? kernel_ptr<0, true, true>(precision) : kernel_ptr<0, true, false>(precision);
    return rec ? kernel_ptr<0, false, true>(precision) : kernel_ptr<0, false, false>(precision);
  }
  if (jb) return rec ? kernel_ptr<1, true, true>(precision) : kernel_ptr<1, true, false>(precision);
  return rec ? kernel_ptr<1, false, true>(precision) : kernel_ptr<1, false, false>(precision);
}

}  // namespace

int transport_block_size() { return kBlock; }

cudaError_t transport_occupancy(int line_mode, int precision, bool j_blue, bool record,
                                int *blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      blocks_per_sm, select_kernel(line_mode, precision, j_blue, record), kBlock, 0);
}

cudaError_t launch_transport(const TransportParams &p, int line_mode, int precision, bool j_blue,
                             bool record, int grid, int block, cudaStream_t st) {
  void *args[] = {const_cast<TransportParams *>(&p)};
  return cudaLaunchKernel(select_kernel(line_mode, precision, j_blue, record), dim3(grid),
                          dim3(block), args, 0, st);
}

}  // namespace mcgpu
