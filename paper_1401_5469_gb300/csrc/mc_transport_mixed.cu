// Mixed-precision Monte Carlo packet transport (same method as
// mc_transport.cu, Kerzendorf & Sim 2014 Sects. 2.4-2.7, 2.9).
//
// Precision split.  Geometry (x mu, impact parameter, radius), path lengths,
// optical depths, the logarithm of the event draw, packet energy and the
// frame factors are binary32.  Binary64 is kept where the method needs it:
// the lab and comoving frequencies, the Sobolev-resonance comparison against
// the frequency-sorted line list (integer keys of binary64 values), the
// frequency thresholds that the optical depth is accumulated into, and the
// estimator sums.  The lab frequency after a re-emission is nu_c / D to
// binary64 accuracy (Newton step on the binary32 reciprocal), so the comoving
// frequency at the emission point is the emitting line's frequency.
#include <cstdint>

#include "mc_device.cuh"
#include "mc_internal.h"

namespace mcgpu {

namespace {

constexpr int kBlock = 128;
constexpr int kShellArrays = 4;  // x_in^2, x_out^2, kappa, 1/kappa (binary32)
constexpr int kLineEvent = 1, kElectronEvent = 2, kShellEvent = 3;

struct PacketM {
  double nu_lab;             // binary64
  float p, q, r2;            // x mu, x^2 - p^2, x^2
  float e_lab, inv_nu, inv_D;
  int32_t shell, next_line;
  uint32_t pid;
  bool have_inv_D;
  uint32_t cnt[kNCounters];
};

__device__ __forceinline__ int32_t first_redward_m(const double *nu, int32_t L, double v) {
  const long long kv = __double_as_longlong(v);
  const long long *nb = reinterpret_cast<const long long *>(nu);
  int32_t lo = 0, hi = L;
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (__ldg(nb + mid) < kv) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// Same exact integer search as the binary64 kernel (downbranch emission).
__device__ __forceinline__ void pick_m(const TransportParams &p, unsigned long long rinfo,
                                       unsigned long long u, double &nu, float &inv_nu, int32_t &line) {
  const uint32_t b = static_cast<uint32_t>(rinfo), len = static_cast<uint32_t>(rinfo >> 32);
  const uint32_t bucket = static_cast<uint32_t>(__umul64hi(u << 11, static_cast<unsigned long long>(len)));
  const DbrRec *slot = p.dbr_bucket + b + bucket;
  unsigned long long thr = __ldg(&slot->thr);
  if (u < thr) {
    nu = __ldg(&slot->nu);
    inv_nu = static_cast<float>(__ldg(&slot->inv_nu));
    line = static_cast<int32_t>(__ldg(&slot->emit));
    return;
  }
  const DbrRec *rec = p.dbr_rec;
  uint32_t i = b + __ldg(&slot->guide) + 1u;
  thr = __ldg(&rec[i].thr);
  while (u >= thr) { ++i; thr = __ldg(&rec[i].thr); }
  nu = __ldg(&rec[i].nu);
  inv_nu = static_cast<float>(__ldg(&rec[i].inv_nu));
  line = static_cast<int32_t>(__ldg(&rec[i].emit));
}

__device__ __forceinline__ float max0f(float v) { return v > 0.0f ? v : 0.0f; }

// uniform in (0, 1] / [0, 1) with 24 random bits
__device__ __forceinline__ float open0f(unsigned long long u53) {
  return static_cast<float>((u53 >> 29) + 1ull) * 0x1.0p-24f;
}

template <int MODE, bool JB, bool REC>
__global__ void __launch_bounds__(kBlock) transport_mixed(const TransportParams p) {
  extern __shared__ float shf[];
  const int32_t S = p.S, L = p.L;
  for (int i = threadIdx.x; i < S; i += blockDim.x) {
    const float xi = static_cast<float>(p.x_in[i]), xo = static_cast<float>(p.x_out[i]);
    const double kap = p.kappa[i];
    shf[i] = xi * xi;
    shf[S + i] = xo * xo;
    shf[2 * S + i] = static_cast<float>(kap);
    shf[3 * S + i] = kap > 0.0 ? static_cast<float>(1.0 / kap) : 0.0f;
  }
  __syncthreads();
  const float *s_xi2 = shf, *s_xo2 = shf + S, *s_kap = shf + 2 * S, *s_ikap = shf + 3 * S;
  const double x0d = p.x_in[0];
  const float x0 = static_cast<float>(x0d), x0sq = s_xi2[0];

  const unsigned lane = threadIdx.x & 31u;
  const unsigned lanemask_lt = (1u << lane) - 1u;
  const unsigned long long t_start = global_ns();
  if (lane == 0u) atomicCAS(p.flags + 3, 0ull, t_start);

  PacketM pk;
  DrawStream ds;
  bool alive = false, finished = false;
  unsigned long long n_esc = 0, n_reab = 0, n_cap = 0, n_seg = 0, n_chk = 0, n_res = 0, n_lint = 0,
                     n_esca = 0, n_shell = 0;
  int32_t acc_s = -1;
  double acc_j = 0.0, acc_nb = 0.0;
  const long long *nub = reinterpret_cast<const long long *>(p.nu);
  const double e_cmf0 = p.e_cmf;  // binary32 energies are carried relative to this

  for (;;) {
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
          // injection (Sect. 2.4), same draws as the binary64 kernel
          pk.pid = static_cast<uint32_t>(p.first_packet + id);
          ds.init(p.key0, p.key1, pk.pid, p.iteration);
          const double z0 = ds.closed0();
          const double z1 = ds.open0(), z2 = ds.open0(), z3 = ds.open0(), z4 = ds.open0();
          int l = 1;
          while (l < kPlanckLmax && p.planck_cdf[l] < z0) ++l;
          double xi = -log_pos(((z1 * z2) * z3) * z4);
          if (l > 1) xi = xi / static_cast<double>(l);
          const double nu_cmf = p.nu_scale * xi;
          const float mu = sqrtf(open0f(ds.next_u53()));
          const float pp = x0 * mu;
          const float D = 1.0f - pp;
          const float iD = 1.0f / D;
          pk.p = pp;
          pk.r2 = x0sq;
          pk.q = max0f(fmaf(-pp, pp, x0sq));
          pk.nu_lab = nu_cmf * static_cast<double>(iD);
          pk.e_lab = iD;  // E_lab / E_cmf(injection)
          pk.inv_nu = static_cast<float>(1.0 / nu_cmf) * D;
          pk.inv_D = iD;
          pk.have_inv_D = true;
          pk.shell = 0;
          pk.next_line = first_redward_m(p.nu, L, nu_cmf);
#pragma unroll
          for (int c = 0; c < kNCounters; ++c) pk.cnt[c] = 0u;
          alive = true;
        } else {
          finished = true;
          atomicCAS(p.flags + 1, 0ull, global_ns());
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

    int status = 0;
    if (pk.cnt[0] >= p.max_segments) {
      status = 3;
    } else {
      pk.cnt[0] += 1u;
      const int32_t s = pk.shell;
      const float pp = pk.p, q = pk.q, r2 = pk.r2, inv_nu = pk.inv_nu;
      const double nu_lab = pk.nu_lab;
      const float Df = 1.0f - pp;
      const float inv_D = pk.have_inv_D ? pk.inv_D : 1.0f / Df;
      const double nu_cmf = nu_lab * static_cast<double>(Df);
      const float eD2 = (pk.e_lab * Df) * Df;
      const float kap = s_kap[s];
      const bool thomson = kap > 0.0f;
      const float tau0 = -__logf(open0f(ds.next_u53()));
      const float xi2 = s_xi2[s], xo2 = s_xo2[s];
      const bool inner = pp < 0.0f && q <= xi2;
      const float root = sqrtf(max0f((inner ? xi2 : xo2) - q));
      const float p_exit = inner ? -root : root;
      const long long key_shell = okey(nu_lab * static_cast<double>(1.0f - p_exit));
      float c_e = 0.0f, tau_rem = tau0;
      double thr_e = 0.0;
      long long key_e = kKeyNegInf;
      if (thomson) {
        c_e = (static_cast<float>(nu_lab) * s_ikap[s]) * inv_D;  // nu_lab / k
        thr_e = nu_cmf - static_cast<double>(tau0 * c_e);
        key_e = okey(thr_e);
      }
      long long key_thr = key_shell > key_e ? key_shell : key_e;
      const float e_inv2 = JB ? (pk.e_lab * inv_nu) * inv_nu : 0.0f;
      const size_t row = static_cast<size_t>(s) * static_cast<size_t>(L);
      const float *tau_s = p.tau32 + row;
      int32_t j = pk.next_line;
      int kind = 0;
      float l = 0.0f;
      double nu_hit = 0.0;
      unsigned long long rinfo_hit = 0ull;
      long long bj = 0, bj_n = 0;
      float taul = 0.0f, tau_n = 0.0f;
      unsigned long long rinfo = 0ull, rinfo_n = 0ull;
      if (j < L) {
        bj = __ldg(nub + j);
        taul = __ldg(tau_s + j);
        if (MODE == 1) rinfo = __ldg(p.row_info + j);
      }
      if (j + 1 < L) {
        bj_n = __ldg(nub + j + 1);
        tau_n = __ldg(tau_s + j + 1);
        if (MODE == 1) rinfo_n = __ldg(p.row_info + j + 1);
      }
      while (j < L) {
        pk.cnt[1] += 1u;
        long long bj_nn = 0;
        float tau_nn = 0.0f;
        unsigned long long rinfo_nn = 0ull;
        if (j + 2 < L) {
          bj_nn = __ldg(nub + j + 2);
          tau_nn = __ldg(tau_s + j + 2);
          if (MODE == 1) rinfo_nn = __ldg(p.row_info + j + 2);
        }
        if (bj <= key_thr) break;
        pk.cnt[2] += 1u;
        const double nuj = __longlong_as_double(bj);
        if (JB) atomicAdd(p.j_blue + row + j, static_cast<double>(static_cast<float>(nuj) * e_inv2) * e_cmf0);
        bool absorbed;
        if (thomson) {
          const double t = thr_e + static_cast<double>(taul * c_e);
          absorbed = okey(t) > bj;
          if (!absorbed) {
            thr_e = t;
            key_e = okey(t);
            key_thr = key_shell > key_e ? key_shell : key_e;
          }
        } else {
          absorbed = taul > tau_rem;
          if (!absorbed) tau_rem -= taul;
        }
        if (absorbed) {
          kind = kLineEvent;
          l = max0f(static_cast<float>(nu_cmf - nuj) * inv_nu);
          nu_hit = nuj;
          rinfo_hit = rinfo;
          break;
        }
        ++j;
        bj = bj_n; taul = tau_n; rinfo = rinfo_n;
        bj_n = bj_nn; tau_n = tau_nn; rinfo_n = rinfo_nn;
      }
      if (kind == 0) {
        if (key_e > key_shell) { kind = kElectronEvent; l = max0f(static_cast<float>(nu_cmf - thr_e) * inv_nu); }
        else { kind = kShellEvent; l = max0f(p_exit - pp); }
      }
      // estimators (binary32 contribution, binary64 sums)
      const double wgt = static_cast<double>(eD2 * l);
      if (s != acc_s) {
        if (acc_s >= 0) {
          atomicAdd(p.j_est + acc_s, acc_j * e_cmf0);
          atomicAdd(p.nu_bar + acc_s, acc_nb * e_cmf0);
        }
        acc_s = s; acc_j = 0.0; acc_nb = 0.0;
      }
      acc_j += wgt;
      acc_nb = fma(wgt, nu_cmf, acc_nb);
      pk.next_line = j;
      if (kind == kShellEvent) {
        pk.cnt[5] += 1u;
        const int32_t ns = inner ? s - 1 : s + 1;
        pk.p = p_exit;
        pk.r2 = inner ? xi2 : xo2;
        pk.shell = ns;
        pk.have_inv_D = false;
        if (ns >= S) status = 1;
        else if (ns < 0) status = 2;
      } else {
        const float pl = pp + l;
        const float r2n = fmaf(pl, pl, q);
        const float xn = sqrtf(r2n);
        const float D1 = 1.0f - pl;
        const float e_c = pk.e_lab * D1;
        double nu_c;
        float inv_nu_c;
        if (kind == kLineEvent) {
          pk.cnt[3] += 1u;
          if (MODE == 1) {
            int32_t emit;
            pick_m(p, rinfo_hit, ds.next_u53(), nu_c, inv_nu_c, emit);
            pk.next_line = emit + 1;
          } else {
            nu_c = nu_hit;
            inv_nu_c = static_cast<float>(1.0 / nu_hit);
            pk.next_line = j + 1;
          }
        } else {
          pk.cnt[4] += 1u;
          nu_c = nu_lab * static_cast<double>(D1);
          inv_nu_c = inv_nu / D1;
        }
        const unsigned long long um = ds.next_u53();
        const float mu2 = static_cast<float>(static_cast<long long>(um >> 29) - (1ll << 23)) * 0x1.0p-23f;
        const float pn = xn * mu2;
        const float D2 = 1.0f - pn;
        const float iD2 = 1.0f / D2;
        // nu_lab = nu_c / D2 to binary64 accuracy: one Newton step on 1/D2
        const double D2d = static_cast<double>(D2), r0 = static_cast<double>(iD2);
        const double r1 = fma(r0, fma(-D2d, r0, 1.0), r0);
        pk.p = pn;
        pk.q = max0f(fmaf(-pn, pn, r2n));
        pk.r2 = r2n;
        pk.nu_lab = nu_c * r1;
        pk.e_lab = e_c * iD2;
        pk.inv_nu = inv_nu_c * D2;
        pk.inv_D = iD2;
        pk.have_inv_D = true;
      }
    }
    if (status != 0) {
      if (status == 1) ++n_esc;
      else if (status == 2) ++n_reab;
      else ++n_cap;
      n_seg += pk.cnt[0];
      n_chk += pk.cnt[1];
      n_res += pk.cnt[2];
      n_lint += pk.cnt[3];
      n_esca += pk.cnt[4];
      n_shell += pk.cnt[5];
      const double e_lab = static_cast<double>(pk.e_lab) * e_cmf0;
      if (status == 1) {
        int b;
        if (pk.nu_lab < p.spec_lo) b = p.spec_bins;
        else {
          const double t = (pk.nu_lab - p.spec_lo) / p.spec_dnu;
          b = (t >= 0.0 && t < static_cast<double>(p.spec_bins)) ? static_cast<int>(floor(t))
                                                                   : p.spec_bins + 1;
        }
        atomicAdd(p.spectrum + b, e_lab);
      }
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
  if (acc_s >= 0) {
    atomicAdd(p.j_est + acc_s, acc_j * e_cmf0);
    atomicAdd(p.nu_bar + acc_s, acc_nb * e_cmf0);
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
const void *kptr() {
  return reinterpret_cast<const void *>(&transport_mixed<MODE, JB, REC>);
}

}  // namespace

const void *select_mixed_kernel(int line_mode, bool jb, bool rec) {
  if (line_mode == 0) {
    if (jb) return rec ? kptr<0, true, true>() : kptr<0, true, false>();
    return rec ? kptr<0, false, true>() : kptr<0, false, false>();
  }
  if (jb) return rec ? kptr<1, true, true>() : kptr<1, true, false>();
  return rec ? kptr<1, false, true>() : kptr<1, false, false>();
}

size_t mixed_smem_bytes(int S) { return static_cast<size_t>(kShellArrays) * S * sizeof(float); }

}  // namespace mcgpu
