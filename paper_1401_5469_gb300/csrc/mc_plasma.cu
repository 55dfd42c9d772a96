// Plasma-state kernels: ionization balance and level populations (Kerzendorf
// & Sim 2014, Sect. 2.3, Eqs. 2-5), Sobolev optical depths (Eq. 12), the
// radiation-field update from the Monte Carlo estimators (Eqs. 15-16) and
// estimator zeroing.
#include <cstdint>

#include "mc_internal.h"

namespace mcgpu {

namespace {

// One thread per (shell, ion): partition function over the ion's levels
// Z = sum_k w_k g_k exp(-eps_k / k T_R) with w_k = 1 for ground/metastable
// levels (Eq. 4) and w_k = W otherwise (Eq. 5); n_k = w_k g_k N exp(..) / Z.
__global__ void populations_kernel(const PlasmaParams p) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= p.S * p.I) return;
  const int s = idx / p.I, i = idx - s * p.I;
  const double inv_kT = 1.0 / (kKB * p.t_rad[s]);
  const double w = p.w[s];
  const size_t a0 = static_cast<size_t>(i) * p.K;
  double Z = 0.0;
  for (int k = 0; k < p.K; ++k) {
    const double wk = (p.lte_excitation || p.metastable[a0 + k]) ? 1.0 : w;
    Z += (wk * p.g[a0 + k]) * exp(-(p.eps_erg[a0 + k] * inv_kT));
  }
  const double scale = p.n_ion[static_cast<size_t>(s) * p.I + i] / Z;
  double *out = p.pop + (static_cast<size_t>(s) * p.I + i) * p.K;
  for (int k = 0; k < p.K; ++k) {
    const double wk = (p.lte_excitation || p.metastable[a0 + k]) ? 1.0 : w;
    out[k] = ((wk * p.g[a0 + k]) * exp(-(p.eps_erg[a0 + k] * inv_kT))) * scale;
  }
}

// Partition function of ion `a` from its levels, sum_k g_k exp(-eps_k / k T_R)
// (the populations of Eq. 4 summed); a stage without levels (a < 0) has 1.
__device__ double ion_partition(const IonParams &p, int a, double inv_kT) {
  if (a < 0) return 1.0;
  const size_t a0 = static_cast<size_t>(a) * p.K;
  double z = 0.0;
  for (int k = 0; k < p.K; ++k) z += p.g[a0 + k] * exp(-(p.eps_erg[a0 + k] * inv_kT));
  return z;
}

// One thread per (shell, element, stage j < J-1): Phi_j = n_{j+1} n_e / n_j
// from the Saha equation (Eq. 2), 2 (Z_{j+1}/Z_j) (2 pi m_e k T / h^2)^(3/2)
// exp(-chi_j / k T); in nebular mode (Eq. 3) times
// W [delta zeta + W (1 - zeta)] (T_e / T_R)^(1/2) with T_e = 0.9 T_R.
__global__ void ion_phi_kernel(const IonParams p) {
  const int J1 = p.J - 1;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= p.S * p.E * J1) return;
  const int s = idx / (p.E * J1);
  const int t = idx - s * (p.E * J1);
  const int e = t / J1, j = t - e * J1;
  const double kT = kKB * p.t_rad[s];
  const double inv_kT = 1.0 / kT;
  const double x = ((2.0 * kPi) * kMe * kT) / (kH * kH);
  const double saha = x * sqrt(x);
  const double z_lo = ion_partition(p, p.ion_of[e * p.J + j], inv_kT);
  const double z_hi = ion_partition(p, p.ion_of[e * p.J + j + 1], inv_kT);
  double phi = ((2.0 * z_hi) / z_lo) * saha * exp(-(p.chi_erg[t] * inv_kT));
  if (p.mode == 2) {
    const double W = p.w[s], z = p.zeta[t];
    phi = ((W * (p.delta * z + W * (1.0 - z))) * sqrt(0.9)) * phi;
  }
  p.phi[idx] = phi;
}

// Stage fractions of one element at electron density n_e: n_j / N from the
// ratios Phi_j / n_e (each stage relative to the one below).
__device__ void stage_fractions(int J, const double *phi, double n_e, double *f) {
  double r = 1.0, sum = 1.0;
  f[0] = 1.0;
  for (int j = 1; j < J; ++j) {
    r = r * (phi[j - 1] / n_e);
    f[j] = r;
    sum += r;
  }
  for (int j = 0; j < J; ++j) f[j] = f[j] / sum;
}

// Sum over the warp, the same value in every lane (lane 0's, broadcast).
__device__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}

// One warp per shell, lanes over elements: charge conservation,
// n_e = sum_e N_e sum_j j f_j(n_e), solved by bisection on ln n_e between
// 1e-40 and 1 times the charge of full ionization (charge(n_e) - n_e falls
// monotonically); then the ion densities N_e f_j, n_e and the Thomson opacity.
__global__ void ion_balance_kernel(const IonParams p) {
  const int s = static_cast<int>((blockIdx.x * static_cast<unsigned>(blockDim.x) + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= p.S) return;  // whole warps: blockDim is a multiple of 32
  const int E = p.E, J = p.J, J1 = J - 1;
  const double *phi = p.phi + static_cast<size_t>(s) * E * J1;
  const double *n_el = p.n_element + static_cast<size_t>(s) * E;
  double part = 0.0;
  for (int e = lane; e < E; e += 32) part += n_el[e] * static_cast<double>(J1);
  const double max_charge = warp_sum(part);
  double f[kIonMaxStages];
  double lo = max_charge * 1e-40, hi = max_charge;
  for (int it = 0; it < 200 && max_charge > 0.0; ++it) {
    const double mid = sqrt(lo * hi);
    if (!(mid > lo && mid < hi)) break;
    double c = 0.0;
    for (int e = lane; e < E; e += 32) {
      stage_fractions(J, phi + e * J1, mid, f);
      double ce = 0.0;
      for (int j = 1; j < J; ++j) ce += static_cast<double>(j) * f[j];
      c += n_el[e] * ce;
    }
    if (warp_sum(c) > mid) lo = mid; else hi = mid;
  }
  const double ne = (max_charge > 0.0) ? sqrt(lo * hi) : 0.0;
  for (int e = lane; e < E; e += 32) {
    if (ne > 0.0) {
      stage_fractions(J, phi + e * J1, ne, f);
    } else {
      f[0] = 1.0;
      for (int j = 1; j < J; ++j) f[j] = 0.0;
    }
    for (int j = 0; j < J; ++j) {
      const int a = p.ion_of[e * J + j];
      if (a >= 0) p.n_ion[static_cast<size_t>(s) * p.I + a] = n_el[e] * f[j];
    }
  }
  if (lane == 0) {
    const double kap = ((kSigmaT * ne) * kC) * p.t_exp;
    const double ikap = kap > 0.0 ? 1.0 / kap : 0.0;
    p.n_e[s] = ne;
    p.kappa[s] = kap;
    p.inv_kappa[s] = ikap;
    if (p.shell32) {
      p.shell32[2 * p.S + s] = static_cast<float>(kap);
      p.shell32[3 * p.S + s] = kap > 0.0 ? static_cast<float>(1.0 / kap) : 0.0f;
    }
  }
}

// One thread per line, looping over shells so that each shell row is written
// with coalesced stores.  Eq. 12 with the stimulated-emission bracket
// multiplied out: tau = pref (n_l - (g_l/g_u) n_u), pref = (pi e^2/m_e c) f
// lambda t_exp.  A line whose lower level is empty gets tau = 0.
__global__ void sobolev_tau_kernel(const PlasmaParams p) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p.L) return;
  const int ll = __ldg(p.lev_l + j), lu = __ldg(p.lev_u + j);
  const double pref = __ldg(p.line_pref + j), gr = __ldg(p.line_gratio + j);
  const size_t IK = static_cast<size_t>(p.I) * p.K;
  for (int s = 0; s < p.S; ++s) {
    const double n_l = __ldg(p.pop + s * IK + ll);
    const double n_u = __ldg(p.pop + s * IK + lu);
    const double t = (n_l > 0.0) ? pref * fma(-gr, n_u, n_l) : 0.0;
    const size_t o = static_cast<size_t>(s) * p.L + j;
    if (p.tau) p.tau[o] = t;
    if (p.tau32) p.tau32[o] = static_cast<float>(t);
  }
}

// Eqs. 15-16; shells without path length keep T_R and W.
__global__ void update_kernel(const UpdateParams p) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.S) return;
  const double j = p.j_est[s];
  if (!(j > 0.0)) return;
  const double T = p.c_tr * (p.nu_bar[s] / j);
  const double J = j * p.norm[s];
  const double T2 = T * T;
  p.t_rad[s] = T;
  p.w[s] = (kPi * J) / (kSigmaSB * (T2 * T2));
}

__global__ void zero_kernel(double *a, size_t n_a, double *b, size_t n_b, double *c, size_t n_c,
                            unsigned long long *u, size_t n_u) {
  const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;; i += stride) {
    bool any = false;
    if (i < n_a) { a[i] = 0.0; any = true; }
    if (i < n_b) { b[i] = 0.0; any = true; }
    if (i < n_c) { c[i] = 0.0; any = true; }
    if (i < n_u) { u[i] = 0ull; any = true; }
    if (!any) break;
  }
}

// Wide zeroing with 16-byte stores (n doubles, base 16-byte aligned).
__global__ void zero_large_kernel(double *a, size_t n) {
  const size_t n2 = n / 2;
  double2 *a2 = reinterpret_cast<double2 *>(a);
  const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  // streaming stores (evict-first): zeroing the J_blue sums must not push the
  // line data out of L2
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n2; i += stride)
    __stcs(a2 + i, make_double2(0.0, 0.0));
  if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) __stcs(a + n - 1, 0.0);
}

// Per-line constants of Eq. 12 and the level/branching-row indices.
__global__ void line_setup_kernel(int L, int K, const double *nu, const double *f,
                                  const int32_t *ion, const int32_t *lower, const int32_t *upper,
                                  const double *g, double t_exp, double sob, int32_t *lev_l,
                                  int32_t *lev_u, double *pref, double *gratio, int32_t *row) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= L) return;
  const int ll = ion[j] * K + lower[j], lu = ion[j] * K + upper[j];
  lev_l[j] = ll;
  lev_u[j] = lu;
  row[j] = lu;
  if (f) {
    pref[j] = ((sob * f[j]) * (kC / nu[j])) * t_exp;
    gratio[j] = g[ll] / g[lu];
  }
}

// Downbranch guide-table rows.  One thread per branching entry: its row is
// found by bisection of the row offsets; thr = ceil(cdf 2^53) is exact (a
// power-of-two scaling of a binary64 value); the guide entry of bucket k of a
// row of length n is the first position whose thr exceeds the smallest u53 of
// the bucket, ceil(k 2^53 / n).
__global__ void dbr_rec_kernel(uint32_t nnz, uint32_t n_rows, const uint32_t *off,
                               const uint32_t *line, const double *cdf, const double *nu,
                               DbrRec *rec) {
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  uint32_t lo = 0, hi = n_rows;  // row r with off[r] <= e < off[r+1]
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (off[mid] <= e) lo = mid; else hi = mid;
  }
  const uint32_t b = off[lo], n = off[lo + 1] - b, k = e - b;
  const double scaled = cdf[e] * 0x1.0p53;
  rec[e].thr = static_cast<unsigned long long>(ceil(scaled));
  rec[e].emit = line[e];
  rec[e].nu = nu[line[e]];
  rec[e].inv_nu = 1.0 / nu[line[e]];
  const unsigned __int128 num = (static_cast<unsigned __int128>(k) << 53) + (n - 1);
  const unsigned long long u_min = static_cast<unsigned long long>(num / n);
  uint32_t a = 0, z = n - 1;  // first position with thr > u_min (the last has thr = 2^53)
  while (a < z) {
    const uint32_t mid = (a + z) >> 1;
    const unsigned long long t = static_cast<unsigned long long>(ceil(cdf[b + mid] * 0x1.0p53));
    if (u_min < t) z = mid; else a = mid + 1;
  }
  rec[e].guide = a;
}

// Bucket slots: slot b + k holds the record of the row's guide entry G[k],
// with its guide field set to G[k].
__global__ void dbr_bucket_kernel(uint32_t nnz, uint32_t n_rows, const uint32_t *off,
                                  const DbrRec *rec, DbrRec *bucket) {
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  uint32_t lo = 0, hi = n_rows;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (off[mid] <= e) lo = mid; else hi = mid;
  }
  const uint32_t b = off[lo];
  const uint32_t g = rec[e].guide;
  DbrRec r = rec[b + g];
  r.guide = g;
  bucket[e] = r;
}

__global__ void row_info_kernel(uint32_t L, const int32_t *line_row, const uint32_t *off,
                                unsigned long long *row_info) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= L) return;
  const int32_t r = line_row[j];
  const unsigned long long b = off[r], n = off[r + 1] - off[r];
  row_info[j] = b | (n << 32);
}

// J_blue of a mixed-precision launch, in place: the buffer holds 64-bit
// fixed-point sums in units of 2^-32 E / nu_ref; overwrite each with
// sum 2^-32 E / nu_ref (E the packet energy).
__global__ void jblue_from_fix_kernel(double *jb, size_t n, double e_cmf, double inv_nu_ref) {
  unsigned long long *fix = reinterpret_cast<unsigned long long *>(jb);
  const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n; i += stride)
    __stcs(jb + i, ((static_cast<double>(__ldcs(fix + i)) * (1.0 / kEstFixScale)) * e_cmf) * inv_nu_ref);
}

// Binary64 J_blue: the transport adds E_lab / nu_lab^2 at each Sobolev point
// (the packet's weight, the same for every line of a flight segment); the
// line's own factor nu_j of Eq. 17's E_lab nu_j / nu_lab^2 is applied here,
// once per cell.  One thread per line, every shell: coalesced over lines.
__global__ void jblue_times_nu_kernel(double *jb, const double *nu, int S, int L) {
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < L; j += stride) {
    const double v = nu[j];
    for (int s = 0; s < S; ++s) {  // streaming loads and stores, as in the zeroing
      double *c = jb + static_cast<size_t>(s) * static_cast<size_t>(L) + j;
      __stcs(c, __ldcs(c) * v);
    }
  }
}

__global__ void est_from_fix_kernel(const unsigned long long *fix, int S, double e_cmf, double nu_ref,
                                    double *j_est, double *nu_bar) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  j_est[s] = (static_cast<double>(fix[s]) * (1.0 / kEstFixScale)) * e_cmf;
  nu_bar[s] = ((static_cast<double>(fix[S + s]) * (1.0 / kEstFixScale)) * e_cmf) * nu_ref;
}

__global__ void to_f32_kernel(const double *in, float *out, size_t n) {
  const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n; i += stride)
    out[i] = static_cast<float>(in[i]);
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

}  // namespace

cudaError_t launch_ionization(const IonParams &p, cudaStream_t st) {
  if (p.J < 2 || p.J > kIonMaxStages) return cudaErrorInvalidValue;
  const int n = p.S * p.E * (p.J - 1);
  ion_phi_kernel<<<(n + 127) / 128, 128, 0, st>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ion_balance_kernel<<<(p.S + 3) / 4, 128, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_populations(const PlasmaParams &p, cudaStream_t st) {
  const int n = p.S * p.I;
  populations_kernel<<<(n + 127) / 128, 128, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_sobolev_tau(const PlasmaParams &p, cudaStream_t st) {
  sobolev_tau_kernel<<<(p.L + 255) / 256, 256, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_update(const UpdateParams &p, cudaStream_t st) {
  update_kernel<<<(p.S + 63) / 64, 64, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_zero(double *a, size_t n_a, double *b, size_t n_b, double *c, size_t n_c,
                        unsigned long long *u, size_t n_u, cudaStream_t st) {
  size_t n = n_a;
  if (n_b > n) n = n_b;
  if (n_c > n) n = n_c;
  if (n_u > n) n = n_u;
  const int grid = static_cast<int>((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
  zero_kernel<<<grid > 0 ? grid : 1, 256, 0, st>>>(a, n_a, b, n_b, c, n_c, u, n_u);
  return cudaGetLastError();
}

cudaError_t launch_line_setup(int L, int K, const double *nu, const double *f, const int32_t *ion,
                              const int32_t *lower, const int32_t *upper, const double *g,
                              double t_exp, int32_t *lev_l, int32_t *lev_u, double *pref,
                              double *gratio, int32_t *row, cudaStream_t st) {
  const double sob = ((kPi * kEcharge) * kEcharge) / (kMe * kC);
  line_setup_kernel<<<(L + 255) / 256, 256, 0, st>>>(L, K, nu, f, ion, lower, upper, g, t_exp, sob,
                                                     lev_l, lev_u, pref, gratio, row);
  return cudaGetLastError();
}

cudaError_t launch_dbr_setup(uint32_t nnz, uint32_t n_rows, uint32_t L, int K,
                             const uint32_t *dbr_offset, const uint32_t *dbr_line,
                             const double *dbr_cdf, const double *nu, const int32_t *line_row,
                             DbrRec *rec, DbrRec *bucket, unsigned long long *row_info,
                             cudaStream_t st) {
  (void)K;
  if (nnz > 0) {
    dbr_rec_kernel<<<(nnz + 255) / 256, 256, 0, st>>>(nnz, n_rows, dbr_offset, dbr_line, dbr_cdf, nu, rec);
    dbr_bucket_kernel<<<(nnz + 255) / 256, 256, 0, st>>>(nnz, n_rows, dbr_offset, rec, bucket);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  row_info_kernel<<<(L + 255) / 256, 256, 0, st>>>(L, line_row, dbr_offset, row_info);
  return cudaGetLastError();
}

cudaError_t launch_jblue_from_fix(double *j_blue, size_t n, double e_cmf, double inv_nu_ref, cudaStream_t st) {
  jblue_from_fix_kernel<<<4 * 152, 256, 0, st>>>(j_blue, n, e_cmf, inv_nu_ref);
  return cudaGetLastError();
}

cudaError_t launch_jblue_times_nu(double *j_blue, const double *nu, int S, int L, cudaStream_t st) {
  const int blocks = (L + 255) / 256 < sm_count() * 8 ? (L + 255) / 256 : sm_count() * 8;
  jblue_times_nu_kernel<<<blocks, 256, 0, st>>>(j_blue, nu, S, L);
  return cudaGetLastError();
}

cudaError_t launch_est_from_fix(const unsigned long long *fix, int S, double e_cmf, double nu_ref,
                                double *j_est, double *nu_bar, cudaStream_t st) {
  est_from_fix_kernel<<<(S + 63) / 64, 64, 0, st>>>(fix, S, e_cmf, nu_ref, j_est, nu_bar);
  return cudaGetLastError();
}

cudaError_t launch_to_f32(const double *in, float *out, size_t n, cudaStream_t st) {
  to_f32_kernel<<<sm_count() * 8, 256, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_zero_large(double *a, size_t n, cudaStream_t st) {
  zero_large_kernel<<<sm_count() * 8, 256, 0, st>>>(a, n);
  return cudaGetLastError();
}

}  // namespace mcgpu
