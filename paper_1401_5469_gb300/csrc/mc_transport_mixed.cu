// Mixed-precision Monte Carlo packet transport (same method as
// mc_transport.cu, Kerzendorf & Sim 2014 Sects. 2.4-2.7, 2.9), for one model
// or for a batch of models in one persistent launch.
//
// Precision split.  Geometry (x mu, impact parameter, radius), path lengths,
// optical depths, the logarithm of the event draw, packet energies (relative
// to the injection energy) and the frame factors are binary32.  Binary64 is
// kept where the method needs it: the lab and comoving frequencies, the
// Sobolev-resonance comparison against the frequency-sorted line list
// (integer keys of binary64 values) and the frequency thresholds that the
// optical depth is accumulated into.  J, nu_bar and J_blue are summed exactly
// as 64-bit fixed point from binary32 contributions (order-independent).  The
// lab frequency after a re-emission is nu_c / D to binary64 accuracy (Newton
// step on the binary32 reciprocal), so the comoving frequency at the emission
// point is the emitting line's frequency.  Conversions between the two
// formats are done on the bit patterns with integer operations (on this GPU a
// conversion instruction takes the binary64 pipe).
//
// Batched launch.  Packets of all models are claimed from one queue (models
// laid out by a prefix sum of their packet counts, largest first so that the
// longest random walks start first); a lane that claims a packet of another
// model loads that model's context and first flushes its register
// accumulators to the previous model.
//
// Single-model launches also have the binary64 kernel's lone-walker mode: a
// warp down to its last live walk runs it with all 32 lanes (32-line windows
// scanned in one step through a binary32 filter against this kernel's own
// threshold chain, the emission record loaded as soon as the scan names the
// line, the walk's draws computed ahead by the warp).
#include <cstdint>

#include "mc_device.cuh"
#include "mc_internal.h"

namespace mcgpu {

namespace {

// single-model launches take 128 threads per block, batched ones 64, 128 or 256
constexpr int kMaxBlock = 256;
constexpr int kLineEvent = 1, kElectronEvent = 2, kShellEvent = 3;

struct PacketM {
  double nu_lab;               // binary64
  float p, q;                  // x mu, x^2 - p^2
  float e_lab, inv_nu, inv_D;  // e_lab relative to the injection energy
  int32_t shell, next_line;
  uint32_t pid;
  bool have_inv_D;
  uint32_t cnt[kNCounters];
};

// What a lane needs of its packet's model.
struct MCtx {
  const float *xi2, *xo2, *kap, *ikap;
  const double *nu;
  const float *tau32;
  const unsigned long long *row_info;
  const int32_t *line_row;           // macro atom: upper level of each line
  const MaRow *ma_row;               // macro atom: level table
  const MaJump *ma_jump;             // macro atom: jump entries
  const DbrRec *bucket, *rec;
  double *j_blue, *j_est, *nu_bar, *spectrum;
  unsigned long long *stats;
  unsigned long long *est_fix;  // [2 S] J, nu_bar in fixed point
  unsigned long long *jb_fix;   // [S L] J_blue in fixed point (the j_blue buffer, converted after the launch)
  float inv_nu_ref, nu_ref;
  const double *planck;
  int32_t S, L, spec_bins;
  uint32_t key0, key1, iteration;
  double spec_lo, spec_dnu, e_cmf, nu_scale;
  uint64_t max_segments, first_packet;
  float x0, x0sq;
  int32_t *rec_status;
  double *rec_nu, *rec_e;
  unsigned long long *rec_cnt;
};

__device__ __forceinline__ void load_ctx(MCtx &c, const TransportParams &q, const float *shell) {
  c.S = q.S;
  c.L = q.L;
  c.xi2 = shell;
  c.xo2 = shell + q.S;
  c.kap = shell + 2 * q.S;
  c.ikap = shell + 3 * q.S;
  c.nu = q.nu;
  c.tau32 = q.tau32;
  c.row_info = q.row_info;
  c.line_row = q.line_row;
  c.ma_row = q.ma_row;
  c.ma_jump = q.ma_jump;
  c.bucket = q.dbr_bucket;
  c.rec = q.dbr_rec;
  c.j_blue = q.j_blue;
  c.j_est = q.j_est;
  c.nu_bar = q.nu_bar;
  c.spectrum = q.spectrum;
  c.stats = q.stats;
  c.est_fix = q.est_fix;
  c.jb_fix = reinterpret_cast<unsigned long long *>(q.j_blue);
  c.inv_nu_ref = static_cast<float>(q.inv_nu_ref);
  c.nu_ref = static_cast<float>(q.nu_scale);
  c.planck = q.planck_cdf;
  c.spec_bins = q.spec_bins;
  c.key0 = q.key0;
  c.key1 = q.key1;
  c.iteration = q.iteration;
  c.spec_lo = q.spec_lo;
  c.spec_dnu = q.spec_dnu;
  c.e_cmf = q.e_cmf;
  c.nu_scale = q.nu_scale;
  c.max_segments = q.max_segments;
  c.first_packet = q.first_packet;
  c.x0 = static_cast<float>(q.x_in[0]);
  c.x0sq = shell[0];
  c.rec_status = q.rec_status;
  c.rec_nu = q.rec_nu;
  c.rec_e = q.rec_e;
  c.rec_cnt = q.rec_cnt;
}

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

// binary32 value of a positive binary64 (given as its bit pattern) inside
// binary32's normal range, rounded toward zero, with integer operations only
// (the line frequencies are validated to lie in that range).
__device__ __forceinline__ float f32_of_positive_f64(long long bits) {
  const unsigned long long b = static_cast<unsigned long long>(bits);
  const uint32_t e = static_cast<uint32_t>(b >> 52) - 1023u + 127u;
  const uint32_t m = static_cast<uint32_t>(b >> 29) & 0x7fffffu;
  return __uint_as_float((e << 23) | m);
}

// Conversions between binary32 and binary64 with integer operations only
// (on this GPU a conversion through the binary64 pipe costs as much as a
// binary64 multiply).  Exact binary64 value of a finite binary32 (binary32
// subnormals, below 1.2e-38, are taken as zero):
__device__ __forceinline__ double f64_of_f32(float x) {
  const uint32_t b = __float_as_uint(x);
  const uint32_t e = (b >> 23) & 0xffu;
  const unsigned long long bits = (static_cast<unsigned long long>(b >> 31) << 63) |
                                  (static_cast<unsigned long long>(e + (1023u - 127u)) << 52) |
                                  (static_cast<unsigned long long>(b & 0x7fffffu) << 29);
  return e ? __longlong_as_double(static_cast<long long>(bits)) : 0.0;
}
// binary32 of max(d, 0) for a binary64 d below binary32's overflow, rounded
// toward zero; values below binary32's normal range give zero.
__device__ __forceinline__ float f32_of_f64_max0(double d) {
  const long long bits = __double_as_longlong(d);
  const int e = static_cast<int>((static_cast<unsigned long long>(bits) >> 52) & 0x7ffu) - (1023 - 127);
  const uint32_t m = static_cast<uint32_t>(static_cast<unsigned long long>(bits) >> 29) & 0x7fffffu;
  return (bits > 0 && e > 0) ? __uint_as_float((static_cast<uint32_t>(e) << 23) | m) : 0.0f;
}

// Same exact integer search as the binary64 kernel (downbranch emission).
__device__ __forceinline__ void pick_m(const MCtx &c, unsigned long long rinfo, unsigned long long u,
                                       double &nu, float &inv_nu, int32_t &line) {
  const uint32_t b = static_cast<uint32_t>(rinfo), len = static_cast<uint32_t>(rinfo >> 32);
  const uint32_t bucket = static_cast<uint32_t>(__umul64hi(u << 11, static_cast<unsigned long long>(len)));
  const DbrRec *slot = c.bucket + b + bucket;
  unsigned long long thr = __ldg(&slot->thr);
  if (u < thr) {
    nu = __ldg(&slot->nu);
    inv_nu = f32_of_positive_f64(__ldg(reinterpret_cast<const long long *>(&slot->inv_nu)));
    line = static_cast<int32_t>(__ldg(&slot->emit));
    return;
  }
  const DbrRec *rec = c.rec;
  uint32_t i = b + __ldg(&slot->guide) + 1u;
  thr = __ldg(&rec[i].thr);
  while (u >= thr) { ++i; thr = __ldg(&rec[i].thr); }
  nu = __ldg(&rec[i].nu);
  inv_nu = f32_of_positive_f64(__ldg(reinterpret_cast<const long long *>(&rec[i].inv_nu)));
  line = static_cast<int32_t>(__ldg(&rec[i].emit));
}

__device__ __forceinline__ float max0f(float v) { return v > 0.0f ? v : 0.0f; }

// Lone-walker mode (all 32 lanes of the warp converged on one walk): the
// emission from a bucket slot loaded ahead as two 16-byte halves {thr, nu},
// {inv_nu, emit | guide << 32}; past the slot the next 32 records of the row
// in one coalesced load per round (lane i takes entry i), the first with u
// below its threshold found by a vote (the row's last threshold is 2^53 > u).
__device__ __forceinline__ void pick_lone_m(const MCtx &c, unsigned long long rinfo, unsigned long long u,
                                            ulonglong2 a, ulonglong2 h, unsigned lane, double &nu,
                                            float &inv_nu, int32_t &line) {
  if (u < a.x) {
    nu = __longlong_as_double(static_cast<long long>(a.y));
    inv_nu = f32_of_positive_f64(static_cast<long long>(h.x));
    line = static_cast<int32_t>(static_cast<uint32_t>(h.y));
    return;
  }
  const uint32_t end = static_cast<uint32_t>(rinfo) + static_cast<uint32_t>(rinfo >> 32);
  uint32_t i0 = static_cast<uint32_t>(rinfo) + static_cast<uint32_t>(h.y >> 32) + 1u;
  for (;;) {
    const uint32_t i = i0 + lane;
    ulonglong2 ra = make_ulonglong2(~0ull, 0ull), rh = make_ulonglong2(0ull, 0ull);
    if (i < end) {
      ra = __ldg(reinterpret_cast<const ulonglong2 *>(c.rec + i));
      rh = __ldg(reinterpret_cast<const ulonglong2 *>(c.rec + i) + 1);
    }
    const unsigned m = __ballot_sync(0xffffffffu, u < ra.x);  // lanes past the row's end vote yes
    if (m != 0u) {
      const int k = __ffs(m) - 1;
      nu = __longlong_as_double(__shfl_sync(0xffffffffu, static_cast<long long>(ra.y), k));
      inv_nu = f32_of_positive_f64(__shfl_sync(0xffffffffu, static_cast<long long>(rh.x), k));
      line = __shfl_sync(0xffffffffu, static_cast<int32_t>(static_cast<uint32_t>(rh.y)), k);
      return;
    }
    i0 += 32u;
  }
}

// Macro atom (Sect. 2.5): the binary64 kernel's walk (integer thresholds, the
// same draws in the same order) on a lane's model context; returns the
// branching-row info of the level the atom deactivates from.
// In lone-walker mode (wd non-null) the draws come from the warp's buffer,
// and past its end each is computed on its own: the same values either way.
__device__ __forceinline__ unsigned long long ma_draw(DrawStream &ds, const WarpDraws *wd) {
  if (!wd) return ds.next_u53();
  if (ds.d - wd->base < kWarpDraws) return wd->take_u53(ds);
  ++ds.d;
  return u53_past_buffer(ds.k0, ds.k1, ds.packet, ds.iteration, ds.d - 1u);
}

__device__ __forceinline__ unsigned long long macroatom_walk_m(const MCtx &c, int32_t row, DrawStream &ds,
                                                               const WarpDraws *wd) {
  for (uint32_t n = 0; n < kMaMaxJumps; ++n) {
    const MaRow *mr = c.ma_row + row;
    const unsigned long long thr = __ldg(&mr->jump_thr);
    const uint2 jb = __ldg(reinterpret_cast<const uint2 *>(&mr->jump_begin));  // begin, length
    const unsigned long long za = ma_draw(ds, wd);
    if (!(za < thr)) {
      const uint2 db = __ldg(reinterpret_cast<const uint2 *>(&mr->dbr_begin));
      return static_cast<unsigned long long>(db.x) | (static_cast<unsigned long long>(db.y) << 32);
    }
    const unsigned long long zb = ma_draw(ds, wd);
    const MaJump *jp = c.ma_jump + jb.x;
    int32_t next = __ldg(&jp[jb.y - 1].target);
    for (uint32_t k = 0; k < jb.y; ++k) {
      if (zb < __ldg(&jp[k].thr)) { next = __ldg(&jp[k].target); break; }
    }
    row = next;
  }
  const uint2 db = __ldg(reinterpret_cast<const uint2 *>(&c.ma_row[row].dbr_begin));
  return static_cast<unsigned long long>(db.x) | (static_cast<unsigned long long>(db.y) << 32);
}

// x mu at the shell exit, +sqrt(x_out^2 - q) or -sqrt(x_in^2 - q).
__device__ __forceinline__ float shell_exit_f(float q, bool inner, float xi2, float xo2) {
  const float root = sqrtf(max0f((inner ? xi2 : xo2) - q));
  return inner ? -root : root;
}

// Does an event at path length l come before the shell exit?  x mu grows by
// l along the ray and x^2 = q + (x mu)^2: before an outward exit exactly when
// x^2 < x_out^2 there; before an inner exit exactly when x mu < 0 and
// x^2 > x_in^2 there.
__device__ __forceinline__ bool inside_shell_f(float pp, float q, float l, bool inner, float xi2,
                                               float xo2) {
  const float pl = pp + l;
  const float r2 = fmaf(pl, pl, q);
  return inner ? (pl < 0.0f && r2 > xi2) : r2 < xo2;
}

// uniform in (0, 1] with 24 random bits (a 32-bit conversion)
__device__ __forceinline__ float open0f(unsigned long long u53) {
  return static_cast<float>(static_cast<uint32_t>(u53 >> 29) + 1u) * 0x1.0p-24f;
}

struct Stats {
  unsigned long long v[kNStats];
};

__device__ __forceinline__ void flush_stats(Stats &st, unsigned long long *dst) {
#pragma unroll
  for (int i = 0; i < kNStats; ++i) {
    if (st.v[i]) atomicAdd(dst + i, st.v[i]);
    st.v[i] = 0ull;
  }
}

// One kernel source serves a single model (p.n_models == 0) and a batch, so a
// model's results do not depend on the company it is launched in.  It is
// compiled twice: MINB = 1 for single models (blocks of 128 threads, three
// per SM at up to 168 registers, and the lone-walker mode for the last random
// walks) and MINB = 2 for batches (128 registers: 16 resident warps per SM,
// for the throughput phase that dominates a batch).  The arithmetic is the
// same instruction for instruction, lone-walker mode included; the batch
// tests check the bits.
template <int MODE, bool JB, bool REC, int MINB>
__global__ void __launch_bounds__(MINB == 1 ? 128 : kMaxBlock, MINB == 1 ? 3 : MINB)
    transport_mixed(const TransportParams p) {
  extern __shared__ unsigned long long smem_u64[];
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lanemask_lt = (1u << lane) - 1u;
  const unsigned long long jb_pol = l2_evict_first_policy();
  MCtx c;
  int32_t cur_model = -1;
  unsigned long long *prefix = smem_u64;
  const bool batch = p.n_models > 0;
  if (batch) {
    for (int i = threadIdx.x; i <= p.n_models; i += blockDim.x) prefix[i] = p.batch_prefix[i];
    __syncthreads();
  } else {
    float *shf = reinterpret_cast<float *>(smem_u64);
    for (int i = threadIdx.x; i < 4 * p.S; i += blockDim.x) shf[i] = p.shell32[i];
    __syncthreads();
    load_ctx(c, p, shf);
    cur_model = 0;
  }
  const unsigned long long t_start = global_ns();
  uint32_t polls = 0u;  // loop iterations between looks at the host's stop request
  if (lane == 0u) atomicCAS(p.flags + 3, 0ull, t_start);

  PacketM pk;
  DrawStream ds;
  bool alive = false, finished = false;
  // Lone-walker mode (single-model build): once the packet queue is empty and
  // a warp is down to one live walk, every lane takes that walk's state and
  // runs its segments with the owner lane, as in the binary64 kernel: the
  // lanes load the line list 32 lines at a time in one coalesced load (line
  // lwin_j0 + lane in each lane), scan the window in one step, compute the
  // walk's draws 64 at a time into a per-warp shared buffer, and only the
  // owner lane makes the walk's side effects.
  constexpr bool kLoneBuild = MINB == 1;
  WarpDraws wd;
  wd.init(batch ? nullptr : smem_u64 + 2 * static_cast<size_t>(p.S) + 2 * kWarpDraws * (threadIdx.x >> 5));
  bool drained = false;  // warp-uniform: the packet queue is empty
  bool lone = false;
  int owner = 0;
  int32_t lwin_j0 = 0, lwin_s = -1;
  long long lwin_b = 0;
  float lwin_t = 0.0f;
  unsigned long long lwin_r = 0ull;
  Stats st;
#pragma unroll
  for (int i = 0; i < kNStats; ++i) st.v[i] = 0ull;
  int32_t acc_s = -1;
  unsigned long long acc_j = 0ull, acc_nb = 0ull;  // fixed point, see kEstFixScale
  // the lane's current shell and its constants (reloaded on a shell or model change)
  int32_t cs = -1;
  float c_kap = 0.0f, c_ikap = 0.0f, c_xi2 = 0.0f, c_xo2 = 0.0f;
  // single-model build: lines next_line, next_line + 1 of the next segment,
  // loaded by the event that began it (see the binary64 kernel)
  bool lw_ok = false;
  long long lw_b0 = 0, lw_b1 = 0;
  float lw_t0 = 0.0f, lw_t1 = 0.0f;
  unsigned long long lw_r0 = 0ull, lw_r1 = 0ull;

  for (;;) {
    const bool need = !lone && !alive && !finished;
    const unsigned needmask = lone ? 0u : __ballot_sync(0xffffffffu, need);
    if (needmask) {
      const int leader = __ffs(needmask) - 1;
      unsigned long long base = 0ull;
      if (static_cast<int>(lane) == leader)
        base = atomicAdd(p.work_counter, static_cast<unsigned long long>(__popc(needmask)));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (base + __popc(needmask) > p.n_packets) drained = true;
      if (need) {
        unsigned long long id = base + __popc(needmask & lanemask_lt);
        if (id < p.n_packets) {
          if (batch) {
            int lo = 0, hi = p.n_models;  // model m with prefix[m] <= id < prefix[m+1]
            while (hi - lo > 1) {
              const int mid = (lo + hi) >> 1;
              if (prefix[mid] <= id) lo = mid; else hi = mid;
            }
            if (lo != cur_model) {
              if (cur_model >= 0) {
                if (acc_s >= 0) {
                  atomicAdd(c.est_fix + acc_s, acc_j);
                  atomicAdd(c.est_fix + c.S + acc_s, acc_nb);
                }
                flush_stats(st, c.stats);
              }
              acc_s = -1; acc_j = 0ull; acc_nb = 0ull;
              load_ctx(c, p.batch[lo], p.batch[lo].shell32);
              cur_model = lo;
              cs = -1;
            }
            id -= prefix[lo];
          }
          // injection (Sect. 2.4), same draws as the binary64 kernel
          pk.pid = static_cast<uint32_t>(c.first_packet + id);
          ds.init(c.key0, c.key1, pk.pid, c.iteration);
          const double z0 = ds.closed0();
          const double z1 = ds.open0(), z2 = ds.open0(), z3 = ds.open0(), z4 = ds.open0();
          int l = 1;
          while (l < kPlanckLmax && c.planck[l] < z0) ++l;
          double xi = -log_pos(((z1 * z2) * z3) * z4);
          if (l > 1) xi = xi / static_cast<double>(l);
          const double nu_cmf = c.nu_scale * xi;
          const float mu = sqrtf(open0f(ds.next_u53()));
          const float pp = c.x0 * mu;
          const float D = 1.0f - pp;
          const float iD = 1.0f / D;
          pk.p = pp;
          pk.q = max0f(fmaf(-pp, pp, c.x0sq));
          pk.nu_lab = nu_cmf * static_cast<double>(iD);
          pk.e_lab = iD;  // E_lab / E_cmf(injection)
          pk.inv_nu = static_cast<float>(1.0 / nu_cmf) * D;
          pk.inv_D = iD;
          pk.have_inv_D = true;
          pk.shell = 0;
          pk.next_line = first_redward_m(c.nu, c.L, nu_cmf);
#pragma unroll
          for (int k = 0; k < kNCounters; ++k) pk.cnt[k] = 0u;
          alive = true;
          lw_ok = false;
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
    if (kLoneBuild && !batch) {
      if (lone) {
        wd.keep_u(ds, c.key0, c.key1, c.iteration, lane);
      } else if (drained) {
        const unsigned live = __ballot_sync(0xffffffffu, alive);
        if (__popc(live) == 1) {
          // the other lanes' packets are done: they hand their estimator sums
          // over and take the walk's state
          owner = __ffs(live) - 1;
          if (!alive && acc_s >= 0) {
            atomicAdd(c.est_fix + acc_s, acc_j);
            atomicAdd(c.est_fix + c.S + acc_s, acc_nb);
          }
          const unsigned F = 0xffffffffu;
          pk.nu_lab = __shfl_sync(F, pk.nu_lab, owner);
          pk.p = __shfl_sync(F, pk.p, owner);
          pk.q = __shfl_sync(F, pk.q, owner);
          pk.e_lab = __shfl_sync(F, pk.e_lab, owner);
          pk.inv_nu = __shfl_sync(F, pk.inv_nu, owner);
          pk.inv_D = __shfl_sync(F, pk.inv_D, owner);
          pk.shell = __shfl_sync(F, pk.shell, owner);
          pk.next_line = __shfl_sync(F, pk.next_line, owner);
          pk.pid = __shfl_sync(F, pk.pid, owner);
          pk.have_inv_D = __shfl_sync(F, static_cast<int>(pk.have_inv_D), owner) != 0;
#pragma unroll
          for (int k = 0; k < kNCounters; ++k) pk.cnt[k] = __shfl_sync(F, pk.cnt[k], owner);
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
          lwin_s = -1;
          alive = true;
          lone = true;
          wd.keep_u(ds, c.key0, c.key1, c.iteration, lane);
        }
      }
    }
    if (!alive) continue;
    const bool act = !lone || static_cast<int>(lane) == owner;  // makes the walk's side effects
    // the walk's next draw: from the warp's buffer in lone mode
    // (a macro atom's internal jumps can take more draws than the buffer holds)
    auto next_u = [&]() -> unsigned long long {
      if (!lone) return ds.next_u53();
      return MODE == 2 ? ma_draw(ds, &wd) : wd.take_u53(ds);
    };
    auto lone_reload = [&](int32_t s_, int32_t j0) {
      lwin_j0 = j0;
      lwin_s = s_;
      const int32_t jj = j0 + static_cast<int32_t>(lane);
      lwin_b = 0;
      lwin_t = 0.0f;
      lwin_r = 0ull;
      if (jj < c.L) {
        lwin_b = __ldg(reinterpret_cast<const long long *>(c.nu) + jj);
        lwin_t = __ldg(c.tau32 + static_cast<size_t>(s_) * static_cast<size_t>(c.L) + jj);
        if (MODE == 1) lwin_r = __ldg(c.row_info + jj);
      }
    };
    auto lone_fetch = [&](int32_t s_, int32_t jj, long long &b, float &t, unsigned long long &r) {
      int idx = jj - lwin_j0;
      if (lwin_s != s_ || idx < 0 || idx >= 32) {
        lone_reload(s_, jj);
        idx = 0;
      }
      b = __shfl_sync(0xffffffffu, lwin_b, idx);
      t = __shfl_sync(0xffffffffu, lwin_t, idx);
      r = __shfl_sync(0xffffffffu, lwin_r, idx);
    };

    int status = 0;
    if (pk.cnt[0] >= c.max_segments) {
      status = 3;
    } else {
      pk.cnt[0] += 1u;
      const int32_t s = pk.shell;
      const int32_t L = c.L;
      const float pp = pk.p, q = pk.q, inv_nu = pk.inv_nu;
      const double nu_lab = pk.nu_lab;
      const float Df = 1.0f - pp;
      const float inv_D = pk.have_inv_D ? pk.inv_D : 1.0f / Df;
      const double nu_cmf = nu_lab * f64_of_f32(Df);
      const float eD2 = (pk.e_lab * Df) * Df;
      if (s != cs) {
        cs = s;
        c_kap = c.kap[s];
        c_ikap = c.ikap[s];
        c_xi2 = c.xi2[s];
        c_xo2 = c.xo2[s];
      }
      const float kap = c_kap;
      const bool thomson = kap > 0.0f;
      const float tau0 = -__logf(open0f(next_u()));
      const float xi2 = c_xi2, xo2 = c_xo2;
      const bool inner = pp < 0.0f && q <= xi2;
      // shell exit threshold only once a line is passed or the exit wins
      // (see inside_shell_f)
      float p_exit = 0.0f;
      long long key_shell = kKeyNegInf;
      bool have_shell = false;
      float c_e = 0.0f, tau_rem = tau0;
      double thr_e = 0.0;
      long long key_e = kKeyNegInf;
      if (thomson) {
        c_e = (f32_of_positive_f64(__double_as_longlong(nu_lab)) * c_ikap) * inv_D;  // nu_lab / k
        thr_e = nu_cmf - f64_of_f32(tau0 * c_e);
        key_e = rawkey(thr_e);  // compared only with positive keys
      }
      long long key_thr = key_e;
      // J_blue contribution E_lab (nu_j / nu_lab)^2 / nu_j = (nu_j / nu_lab) E_lab / nu_lab,
      // in units of E / nu_ref and 2^-32 (fixed point, like J and nu_bar)
      const float e_jb = JB ? ((pk.e_lab * inv_nu) * c.nu_ref) * kEstFixScaleF : 0.0f;
      const size_t row = static_cast<size_t>(s) * static_cast<size_t>(L);
      const float *tau_s = c.tau32 + row;
      const long long *nub = reinterpret_cast<const long long *>(c.nu);
      int32_t j = pk.next_line;
      int kind = 0;
      float l = 0.0f;
      double nu_hit = 0.0;
      unsigned long long rinfo_hit = 0ull;
      long long bj = 0, bj_n = 0;
      float taul = 0.0f, tau_n = 0.0f;
      unsigned long long rinfo = 0ull, rinfo_n = 0ull;
      // An absorbing line (Sect. 2.6): with no line passed yet its Sobolev
      // point is also placed against the shell exit; if the exit comes first
      // the scan ends with no event (kind stays 0).
      auto absorb = [&](long long b_, unsigned long long r_) {
        const double nuj = __longlong_as_double(b_);
        const float lj = f32_of_f64_max0(nu_cmf - nuj) * inv_nu;
        if (!have_shell && !inside_shell_f(pp, q, lj, inner, xi2, xo2)) return;  // exit comes first
        pk.cnt[2] += 1u;
        if (JB && act)
          red_add_evict_first(c.jb_fix + row + j, __float2ull_rn((f32_of_positive_f64(b_) * inv_nu) * e_jb), jb_pol);
        kind = kLineEvent;
        l = lj;
        nu_hit = nuj;
        rinfo_hit = r_;
      };
      bool fast = false;  // the lone scan settled the segment's line event
      // downbranch: the absorbing line's emission record, loaded as soon as the
      // lone scan names the line (the emission draw is the next in the buffer)
      bool have_slot = false;
      ulonglong2 slot_a = make_ulonglong2(0ull, 0ull), slot_h = make_ulonglong2(0ull, 0ull);
      if (lone) {
        int idx = j - lwin_j0;
        if (lwin_s != s || idx < 0 || idx >= 32) {
          lone_reload(s, j);
          idx = 0;
        }
        if (thomson) {
          // The scan of lines j0 + idx .. j0 + 31 of the window in one step (the
          // binary64 kernel's window scan in this kernel's arithmetic): in the
          // scan below the threshold after line k is T_k = thr_e + sum of the
          // binary32 products tau_i c_e (binary64 sums); it stops at line k when
          // nu_k <= T_{k-1} (beyond d_e), when nu_k lies beyond the shell exit
          // (exact key comparison), or when T_k > nu_k (absorbed).  Each lane
          // forms A = nu_k - T_{k-1} and B = nu_k - T_k in binary32 from the
          // binary64 difference nu_k - thr_e (truncated) and a prefix sum of the
          // same products, with a bound M on |error|: the truncation (2u) and
          // the five summation levels (5u), the final difference (u), the scan's
          // binary64 sums (at most 2^-48 (|thr_e| + C)) and products below the
          // binary32 normal range that the scan drops (32 2^-126):  M = 2^-20
          // (|d| + C) + 2^-44 |thr_e| + 2^-120.  Where every sign up to the first
          // line that stops the scan is certain and that line absorbs, the
          // result is the scan's; otherwise the scan below runs as usual.
          const float pe = shell_exit_f(q, inner, xi2, xo2);
          const long long ksh = rawkey(nu_lab * f64_of_f32(1.0f - pe));
          const int32_t jl = lwin_j0 + static_cast<int32_t>(lane);
          const bool cand = static_cast<int>(lane) >= idx;
          const bool valid = cand && jl < L;
          const float dk = f32_rz_any(__longlong_as_double(lwin_b) - thr_e);
          float P = valid ? lwin_t * c_e : 0.0f;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const float y = __shfl_up_sync(0xffffffffu, P, o);
            if (static_cast<int>(lane) >= o) P = __fadd_rn(P, y);
          }
          float Px = __shfl_up_sync(0xffffffffu, P, 1);
          if (lane == 0u) Px = 0.0f;
          const float A = __fsub_rn(dk, Px), B = __fsub_rn(dk, P);
          const float M = __fadd_rn(__fmul_rn(0x1.0p-20f, __fadd_rn(fabsf(dk), P)),
                                    __fadd_rn(__fmul_rn(0x1.0p-44f, fabsf(f32_rz_any(thr_e))), 0x1.0p-120f));
          const bool e_no = A > M;                      // certainly before d_e
          const bool a_yes = B < -M, a_no = B > M;      // certainly absorbed / passed
          const bool x_no = lwin_b > ksh;               // before the exit
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
              red_add_evict_first(c.jb_fix + row + jl,
                                  __float2ull_rn((f32_of_positive_f64(lwin_b) * inv_nu) * e_jb), jb_pol);
            if (npass > 0) {  // as the scan leaves it after its first pass
              p_exit = pe;
              key_shell = ksh;
              have_shell = true;
            }
            j = lwin_j0 + kstar;
            bj = __shfl_sync(0xffffffffu, lwin_b, kstar);
            rinfo = __shfl_sync(0xffffffffu, lwin_r, kstar);
            if (MODE == 1) {
              const uint32_t rb = static_cast<uint32_t>(rinfo), rlen = static_cast<uint32_t>(rinfo >> 32);
              const uint32_t bucket = static_cast<uint32_t>(
                  __umul64hi(wd.peek_u53(ds) << 11, static_cast<unsigned long long>(rlen)));
              const DbrRec *slot = c.bucket + rb + bucket;
              slot_a = __ldg(reinterpret_cast<const ulonglong2 *>(slot));
              slot_h = __ldg(reinterpret_cast<const ulonglong2 *>(slot) + 1);
              have_slot = true;
            }
          }
        }
        if (!fast) {
          lone_fetch(s, j, bj, taul, rinfo);
          lone_fetch(s, j + 1, bj_n, tau_n, rinfo_n);
        }
      } else if (MINB == 1 && lw_ok) {
        bj = lw_b0; taul = lw_t0; rinfo = lw_r0;
        bj_n = lw_b1; tau_n = lw_t1; rinfo_n = lw_r1;
      } else {
        if (j < L) {
          bj = __ldg(nub + j);
          taul = __ldg(tau_s + j);
          if (MODE == 1) rinfo = __ldg(c.row_info + j);
        }
        if (j + 1 < L) {
          bj_n = __ldg(nub + j + 1);
          tau_n = __ldg(tau_s + j + 1);
          if (MODE == 1) rinfo_n = __ldg(c.row_info + j + 1);
        }
      }
      lw_ok = false;
      long long bj_nn = 0;
      float tau_nn = 0.0f;
      unsigned long long rinfo_nn = 0ull;
      if (fast) absorb(bj, rinfo);
      else while (j < L) {
        pk.cnt[1] += 1u;
        bj_nn = 0;
        tau_nn = 0.0f;
        rinfo_nn = 0ull;
        if (lone) {
          lone_fetch(s, j + 2, bj_nn, tau_nn, rinfo_nn);
        } else if (j + 2 < L) {
          bj_nn = __ldg(nub + j + 2);
          tau_nn = __ldg(tau_s + j + 2);
          if (MODE == 1) rinfo_nn = __ldg(c.row_info + j + 2);
        }
        if (bj <= key_thr) break;
        const double nuj = __longlong_as_double(bj);
        bool absorbed;
        double t = 0.0;
        if (thomson) {
          t = thr_e + f64_of_f32(taul * c_e);
          absorbed = rawkey(t) > bj;  // nu_j > 0
        } else {
          absorbed = taul > tau_rem;
        }
        if (!absorbed) {
          if (!have_shell) {  // a line is passed: the scan needs the exit threshold
            p_exit = shell_exit_f(q, inner, xi2, xo2);
            key_shell = rawkey(nu_lab * f64_of_f32(1.0f - p_exit));  // > 0
            have_shell = true;
            key_thr = key_shell > key_e ? key_shell : key_e;
            if (bj <= key_shell) break;  // this line lies beyond the exit
          }
          pk.cnt[2] += 1u;
          if (JB && act) red_add_evict_first(c.jb_fix + row + j, __float2ull_rn((f32_of_positive_f64(bj) * inv_nu) * e_jb), jb_pol);
          if (thomson) {
            thr_e = t;
            key_e = rawkey(t);
            key_thr = key_shell > key_e ? key_shell : key_e;
          } else {
            tau_rem -= taul;
          }
        } else {
          absorb(bj, rinfo);
          break;
        }
        ++j;
        bj = bj_n; taul = tau_n; rinfo = rinfo_n;
        bj_n = bj_nn; tau_n = tau_nn; rinfo_n = rinfo_nn;
      }
      if (kind == 0) {
        const float le = thomson ? f32_of_f64_max0(nu_cmf - thr_e) * inv_nu : 0.0f;
        const bool electron = have_shell ? key_e > key_shell
                                         : thomson && inside_shell_f(pp, q, le, inner, xi2, xo2);
        if (electron) {
          kind = kElectronEvent;
          l = le;
        } else {
          if (!have_shell) p_exit = shell_exit_f(q, inner, xi2, xo2);
          kind = kShellEvent;
          l = max0f(p_exit - pp);
        }
      }
      // estimators: binary32 contribution (units of E), summed in fixed point
      const float wgt = eD2 * l;
      if (s != acc_s) {
        if (acc_s >= 0 && act) {
          atomicAdd(c.est_fix + acc_s, acc_j);
          atomicAdd(c.est_fix + c.S + acc_s, acc_nb);
        }
        acc_s = s; acc_j = 0ull; acc_nb = 0ull;
      }
      // (x 2^32 is exact; the binary32 to integer conversions do not touch
      // the binary64 pipe)
      acc_j += __float2ull_rn(wgt * kEstFixScaleF);
      acc_nb += __float2ull_rn((wgt * (f32_of_positive_f64(__double_as_longlong(nu_cmf)) * c.inv_nu_ref)) *
                               kEstFixScaleF);
      pk.next_line = j;
      if (kind == kShellEvent) {
        pk.cnt[5] += 1u;
        const int32_t ns = inner ? s - 1 : s + 1;
        pk.p = p_exit;
        pk.shell = ns;
        pk.have_inv_D = false;
        if (ns >= c.S) status = 1;
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
          if (MODE >= 1) {
            // MODE 2: macro atom, internal jumps before the emission pick
            const unsigned long long rinfo_em =
                MODE == 2 ? macroatom_walk_m(c, __ldg(c.line_row + j), ds, lone ? &wd : nullptr) : rinfo_hit;
            int32_t emit;
            const unsigned long long u_em = next_u();
            if (have_slot) pick_lone_m(c, rinfo_em, u_em, slot_a, slot_h, lane, nu_c, inv_nu_c, emit);
            else pick_m(c, rinfo_em, u_em, nu_c, inv_nu_c, emit);
            pk.next_line = emit + 1;
            if (lone) {
              lone_reload(s, pk.next_line);
            } else if (MINB == 1) {  // the next segment's first lines, loaded now
              const int32_t nl = pk.next_line;
              lw_b0 = 0; lw_t0 = 0.0f; lw_r0 = 0ull; lw_b1 = 0; lw_t1 = 0.0f; lw_r1 = 0ull;
              if (nl < L) {
                lw_b0 = __ldg(nub + nl);
                lw_t0 = __ldg(tau_s + nl);
                if (MODE == 1) lw_r0 = __ldg(c.row_info + nl);
              }
              if (nl + 1 < L) {
                lw_b1 = __ldg(nub + nl + 1);
                lw_t1 = __ldg(tau_s + nl + 1);
                if (MODE == 1) lw_r1 = __ldg(c.row_info + nl + 1);
              }
              lw_ok = true;
            }
          } else {
            nu_c = nu_hit;
            inv_nu_c = 1.0f / f32_of_positive_f64(__double_as_longlong(nu_hit));
            pk.next_line = j + 1;
            if (MINB == 1) {  // lines j + 1, j + 2 are in the scan's registers
              lw_b0 = bj_n; lw_t0 = tau_n; lw_r0 = rinfo_n;
              lw_b1 = bj_nn; lw_t1 = tau_nn; lw_r1 = rinfo_nn;
              lw_ok = true;
            }
          }
        } else {
          pk.cnt[4] += 1u;
          nu_c = nu_lab * f64_of_f32(D1);
          inv_nu_c = inv_nu / D1;
          if (MINB == 1) {  // the next segment starts at line j again
            lw_b0 = bj; lw_t0 = taul; lw_r0 = rinfo;
            lw_b1 = bj_n; lw_t1 = tau_n; lw_r1 = rinfo_n;
            lw_ok = true;
          }
        }
        const unsigned long long um = next_u();
        const float mu2 = static_cast<float>(static_cast<int32_t>(um >> 29) - (1 << 23)) * 0x1.0p-23f;
        const float pn = xn * mu2;
        const float D2 = 1.0f - pn;
        const float iD2 = 1.0f / D2;
        // nu_lab = nu_c / D2 to binary64 accuracy: one Newton step on 1/D2
        const double D2d = f64_of_f32(D2), r0 = f64_of_f32(iD2);
        const double r1 = fma(r0, fma(-D2d, r0, 1.0), r0);
        pk.p = pn;
        pk.q = max0f(fmaf(-pn, pn, r2n));
        pk.nu_lab = nu_c * r1;
        pk.e_lab = e_c * iD2;
        pk.inv_nu = inv_nu_c * D2;
        pk.inv_D = iD2;
        pk.have_inv_D = true;
      }
    }
    if (status != 0 && !act) {  // lone mode, not the owner lane: drop the adopted walk
      alive = false;
      lone = false;
      acc_s = -1;
      acc_j = 0ull;
      acc_nb = 0ull;
    } else if (status != 0) {
      lone = false;
      if (status == 1) st.v[kStEscaped] += 1ull;
      else if (status == 2) st.v[kStReabsorbed] += 1ull;
      else st.v[kStCapped] += 1ull;
      st.v[kStSegments] += pk.cnt[0];
      st.v[kStLineChecks] += pk.cnt[1];
      st.v[kStResonances] += pk.cnt[2];
      st.v[kStLineInteractions] += pk.cnt[3];
      st.v[kStEScatters] += pk.cnt[4];
      st.v[kStShellCrossings] += pk.cnt[5];
      const double e_lab = static_cast<double>(pk.e_lab) * c.e_cmf;
      if (status == 1) {
        int b;
        if (pk.nu_lab < c.spec_lo) b = c.spec_bins;
        else {
          const double t = (pk.nu_lab - c.spec_lo) / c.spec_dnu;
          b = (t >= 0.0 && t < static_cast<double>(c.spec_bins)) ? static_cast<int>(floor(t))
                                                                   : c.spec_bins + 1;
        }
        atomicAdd(c.spectrum + b, e_lab);
      }
      if (REC) {
        const uint64_t r = pk.pid - c.first_packet;
        c.rec_status[r] = status;
        c.rec_nu[r] = pk.nu_lab;
        c.rec_e[r] = e_lab;
#pragma unroll
        for (int k = 0; k < kNCounters; ++k) c.rec_cnt[r * kNCounters + k] = pk.cnt[k];
      }
      alive = false;
    }
  }
  if (cur_model >= 0) {
    if (acc_s >= 0 && (!lone || static_cast<int>(lane) == owner)) {  // (a launch stopped in lone mode)
      atomicAdd(c.est_fix + acc_s, acc_j);
      atomicAdd(c.est_fix + c.S + acc_s, acc_nb);
    }
    flush_stats(st, c.stats);
  }
  if (lane == 0u) atomicMax(p.flags + 2, global_ns());
}

template <int MODE, bool JB, bool REC, int MINB>
const void *kptr() {
  return reinterpret_cast<const void *>(&transport_mixed<MODE, JB, REC, MINB>);
}

template <int MINB>
const void *select_m(int line_mode, bool jb, bool rec) {
  if (line_mode == 0) {
    if (jb) return rec ? kptr<0, true, true, MINB>() : kptr<0, true, false, MINB>();
    return rec ? kptr<0, false, true, MINB>() : kptr<0, false, false, MINB>();
  }
  if (line_mode == 2) {
    if (jb) return rec ? kptr<2, true, true, MINB>() : kptr<2, true, false, MINB>();
    return rec ? kptr<2, false, true, MINB>() : kptr<2, false, false, MINB>();
  }
  if (jb) return rec ? kptr<1, true, true, MINB>() : kptr<1, true, false, MINB>();
  return rec ? kptr<1, false, true, MINB>() : kptr<1, false, false, MINB>();
}

const void *select_b(int line_mode, bool jb, bool rec) { return select_m<2>(line_mode, jb, rec); }

}  // namespace

const void *select_mixed_kernel(int line_mode, bool jb, bool rec) { return select_m<1>(line_mode, jb, rec); }

// single-model launches (128 threads): shell tables, then a lone walker's
// draw buffer per warp
size_t mixed_smem_bytes(int S) {
  return 4 * static_cast<size_t>(S) * sizeof(float) + (128 / 32) * 2 * kWarpDraws * sizeof(unsigned long long);
}

cudaError_t batch_occupancy(int line_mode, bool j_blue, bool record, int n_models, int block,
                            int *blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      blocks_per_sm, select_b(line_mode, j_blue, record), block,
      static_cast<size_t>(n_models + 1) * sizeof(unsigned long long));
}

cudaError_t launch_transport_batch(const TransportParams &p, int line_mode, bool j_blue, bool record,
                                   int grid, int block, cudaStream_t st) {
  void *args[] = {const_cast<TransportParams *>(&p)};
  return cudaLaunchKernel(select_b(line_mode, j_blue, record), dim3(grid), dim3(block), args,
                          static_cast<size_t>(p.n_models + 1) * sizeof(unsigned long long), st);
}

}  // namespace mcgpu
