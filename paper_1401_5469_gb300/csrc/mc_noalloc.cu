// mc_transport_noalloc: one Monte Carlo transport launch that allocates no
// memory at all.
//
// Some callers cannot allocate device memory on the path where they need the
// transport: code running inside another framework's memory pool or under a
// fixed memory budget, callers that hold no allocator of their own (for
// example a plug-in handed raw device buffers by its host application), and
// callers that must not trigger the implicit synchronisation or the failure
// modes of an allocation in the middle of a time-critical loop.  They pass
// every input and output buffer themselves; the little working memory the
// kernel still needs -- the packet work counter, the run statistics, the
// deadline flag, the per-shell geometry in units of c t_exp and the Planck
// sampling table -- lives in a fixed, file-scope device array that the
// library owns for the lifetime of the process.
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/mc_transport.h"
#include "mc_internal.h"

namespace mcgpu {
void set_create_error(const std::string &msg);
}

using namespace mcgpu;

namespace {

// Scratch layout (bytes).  Counters first, then the Planck table, then five
// per-shell arrays of MC_NOALLOC_MAX_SHELLS doubles each.
constexpr size_t kCountersOff = 0;                                  // stats, work counter, flag
constexpr size_t kPlanckOff = 256;
constexpr size_t kShellOff = kPlanckOff + ((kPlanckLmax + 1) * sizeof(double) + 255) / 256 * 256;
constexpr size_t kShellArrayBytes = MC_NOALLOC_MAX_SHELLS * sizeof(double);
constexpr size_t kScratchBytes = kShellOff + 5 * kShellArrayBytes;
static_assert(kScratchBytes <= 64 * 1024, "no-allocation scratch must stay at most 64 KiB");
static_assert(kNCounterSlots * sizeof(unsigned long long) <= kPlanckOff, "counter slots overlap the Planck table");

// The scratch itself: every GPU that loads the library holds these bytes
// until the process exits.  Calls share it (see the header).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_lock;
unsigned char *g_scratch_ptr[kMaxDevices] = {};

// Planck series partial sums (90/pi^4) sum_{j<=l} j^-4, written once per device.
__global__ void noalloc_planck_kernel() {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double *cdf = reinterpret_cast<double *>(g_scratch + kPlanckOff);
  const double c = 90.0 / (kPi * kPi * kPi * kPi);
  double acc = 0.0;
  cdf[0] = 0.0;
  for (int l = 1; l <= kPlanckLmax; ++l) {
    const double dl = static_cast<double>(l);
    acc = __dadd_rn(acc, 1.0 / __dmul_rn(__dmul_rn(__dmul_rn(dl, dl), dl), dl));
    cdf[l] = __dmul_rn(c, acc);
  }
}

// Per call: zero every counter slot (run statistics, work counter and the
// four flag words: deadline, queue-empty, last-warp and first-warp
// timestamps, which this entry point does not read but clears all the same,
// so that nothing of an earlier call survives in them) and derive the shell arrays from the caller's
// velocities and electron densities (radii in units of c t_exp, their
// inverses, and kappa' = sigma_T n_e c t_exp).
__global__ void noalloc_prepare_kernel(int S, const double *v_inner, const double *v_outer,
                                       const double *n_e, double t_exp) {
  unsigned long long *cnt = reinterpret_cast<unsigned long long *>(g_scratch + kCountersOff);
  double *xi = reinterpret_cast<double *>(g_scratch + kShellOff);
  double *xo = xi + MC_NOALLOC_MAX_SHELLS;
  double *ixi = xo + MC_NOALLOC_MAX_SHELLS;
  double *ixo = ixi + MC_NOALLOC_MAX_SHELLS;
  double *kap = ixo + MC_NOALLOC_MAX_SHELLS;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < kNCounterSlots) cnt[t] = 0ull;
  if (t < S) {
    xi[t] = v_inner[t] / kC;
    xo[t] = v_outer[t] / kC;
    ixi[t] = 1.0 / xi[t];
    ixo[t] = 1.0 / xo[t];
    kap[t] = __dmul_rn(__dmul_rn(__dmul_rn(kSigmaT, n_e[t]), kC), t_exp);
  }
}

mc_status reject(const std::string &msg) {
  set_create_error(std::string("mc_transport_noalloc: ") + msg);
  return MC_ERR_INVALID_ARG;
}

// Once per device, with that device current: find the device address of the
// scratch array and fill the Planck table.
mc_status scratch_for_current_device(cudaStream_t st, unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_create_error(std::string("mc_transport_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    return MC_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return reject("device index out of range");
  std::lock_guard<std::mutex> lk(g_setup_lock);
  if (!g_scratch_ptr[dev]) {
    // The set-up kernel must run, not land in a graph that may never be
    // launched: refuse a first call made while the stream is capturing.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) {
      set_create_error(std::string("mc_transport_noalloc: cudaStreamIsCapturing: ") + cudaGetErrorString(e));
      return MC_ERR_CUDA;
    }
    if (cap != cudaStreamCaptureStatusNone)
      return reject("the first call on a device does its set-up and must not be made while the stream is capturing");
    // Looking the array up loads this file's device code onto the device
    // (modules load lazily), which is when the array's memory is committed.
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_scratch);
    if (e != cudaSuccess || !ptr) {
      set_create_error(std::string("mc_transport_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return MC_ERR_CUDA;
    }
    noalloc_planck_kernel<<<1, 1, 0, st>>>();
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_create_error(std::string("mc_transport_noalloc: set-up kernel: ") + cudaGetErrorString(e));
      return MC_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<unsigned char *>(ptr);
  }
  *out = g_scratch_ptr[dev];
  return MC_OK;
}

}  // namespace

extern "C" mc_status mc_transport_noalloc(const mc_noalloc_args *a, void *stream) {
  if (!a) return reject("args is NULL");
  const uint32_t S = a->n_shells, L = a->n_lines;
  if (S == 0) return reject("n_shells must be >= 1");
  if (S > MC_NOALLOC_MAX_SHELLS)
    return reject("n_shells exceeds MC_NOALLOC_MAX_SHELLS (" + std::to_string(MC_NOALLOC_MAX_SHELLS) + ")");
  if (L == 0) return reject("n_lines must be >= 1");
  if (L > static_cast<uint32_t>(INT32_MAX)) return reject("n_lines must be below 2^31");
  if (a->spec_bins > static_cast<uint32_t>(INT32_MAX) - 2u) return reject("spec_bins must be below 2^31 - 2");
  if (!a->v_inner || !a->v_outer || !a->n_e || !a->nu || !a->tau)
    return reject("geometry, line and tau buffers are required");
  if (!a->j_est || !a->nu_bar || !a->spectrum) return reject("j_est, nu_bar and spectrum outputs are required");
  if (!(a->t_exp > 0.0) || !std::isfinite(a->t_exp)) return reject("t_exp must be positive");
  if (!(a->v_inner_0 > 0.0) || !std::isfinite(a->v_inner_0)) return reject("v_inner_0 must be positive");
  if (a->line_mode != MC_LINE_SCATTER && a->line_mode != MC_LINE_DOWNBRANCH) return reject("unknown line_mode");
  if (a->line_mode == MC_LINE_DOWNBRANCH && (!a->line_row || !a->dbr_offset || !a->dbr_line || !a->dbr_cdf))
    return reject("downbranch mode needs line_row and the branching table");
  if (a->n_packets == 0 || a->n_packets >= (1ull << 32)) return reject("need 0 < n_packets < 2^32");
  if (!(a->t_inner > 0.0) || !std::isfinite(a->t_inner)) return reject("t_inner must be positive");
  if (a->spec_bins == 0 || !(a->spec_nu_hi > a->spec_nu_lo)) return reject("spectrum needs bins > 0 and nu_lo < nu_hi");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);

  unsigned char *scratch = nullptr;
  mc_status rc = scratch_for_current_device(st, &scratch);
  if (rc != MC_OK) return rc;

  noalloc_prepare_kernel<<<(MC_NOALLOC_MAX_SHELLS + 127) / 128, 128, 0, st>>>(
      static_cast<int>(S), a->v_inner, a->v_outer, a->n_e, a->t_exp);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = launch_zero(a->j_est, S, a->nu_bar, S, a->spectrum, static_cast<size_t>(a->spec_bins) + 2, nullptr, 0, st);
  if (e == cudaSuccess && a->j_blue) e = launch_zero_large(a->j_blue, static_cast<size_t>(S) * L, st);
  if (e != cudaSuccess) {
    set_create_error(std::string("mc_transport_noalloc: ") + cudaGetErrorString(e));
    return MC_ERR_CUDA;
  }

  unsigned long long *cnt = reinterpret_cast<unsigned long long *>(scratch + kCountersOff);
  double *xi = reinterpret_cast<double *>(scratch + kShellOff);
  TransportParams p{};
  p.S = static_cast<int32_t>(S);
  p.L = static_cast<int32_t>(L);
  p.x_in = xi;
  p.x_out = xi + MC_NOALLOC_MAX_SHELLS;
  p.inv_x_in = xi + 2 * MC_NOALLOC_MAX_SHELLS;
  p.inv_x_out = xi + 3 * MC_NOALLOC_MAX_SHELLS;
  p.kappa = xi + 4 * MC_NOALLOC_MAX_SHELLS;
  p.nu = a->nu;
  p.tau = a->tau;
  p.line_row = a->line_row;
  p.dbr_offset = a->dbr_offset;
  p.dbr_line = a->dbr_line;
  p.dbr_cdf = a->dbr_cdf;
  p.j_est = a->j_est;
  p.nu_bar = a->nu_bar;
  p.j_blue = a->j_blue;
  p.spectrum = a->spectrum;
  p.stats = cnt;
  p.work_counter = cnt + kNStats;
  p.flags = cnt + kNStats + 1;
  p.spec_bins = static_cast<int32_t>(a->spec_bins);
  p.spec_lo = a->spec_nu_lo;
  p.spec_hi = a->spec_nu_hi;
  p.spec_dnu = (a->spec_nu_hi - a->spec_nu_lo) / static_cast<double>(a->spec_bins);
  p.n_packets = a->n_packets;
  p.iteration = a->iteration;
  p.key0 = static_cast<uint32_t>(a->seed);
  p.key1 = static_cast<uint32_t>(a->seed >> 32);
  const double dt = a->delta_t > 0.0 ? a->delta_t : 1.0;
  const double r_i = a->v_inner_0 * a->t_exp;
  const double lum = (((4.0 * kPi) * r_i) * r_i) * kSigmaSB * a->t_inner * a->t_inner * a->t_inner * a->t_inner;
  p.e_cmf = (lum * dt) / static_cast<double>(a->n_packets);
  p.nu_scale = (kKB * a->t_inner) / kH;
  p.planck_cdf = reinterpret_cast<const double *>(scratch + kPlanckOff);
  p.max_segments = a->max_segments ? a->max_segments : 1000000ull;
  p.timeout_ns = 0;

  int dev = 0, nsm = 1, bps = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  e = transport_occupancy(a->line_mode, MC_PRECISION_FP64, a->j_blue != nullptr, false,
                          static_cast<int>(S), &bps);
  if (e != cudaSuccess || bps <= 0) {
    set_create_error("mc_transport_noalloc: occupancy query failed");
    return MC_ERR_CUDA;
  }
  e = launch_transport(p, a->line_mode, MC_PRECISION_FP64, a->j_blue != nullptr, false, nsm * bps,
                       transport_block_size(), st);
  if (e == cudaSuccess && a->j_blue)  // cells hold sums of E_lab / nu_lab^2: times nu_j (Eq. 17)
    e = launch_jblue_times_nu(a->j_blue, a->nu, static_cast<int>(S), static_cast<int>(L), st);
  if (e == cudaSuccess && a->stats)
    e = cudaMemcpyAsync(a->stats, cnt, kNStats * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) {
    set_create_error(std::string("mc_transport_noalloc: ") + cudaGetErrorString(e));
    return MC_ERR_CUDA;
  }
  return MC_OK;
}
