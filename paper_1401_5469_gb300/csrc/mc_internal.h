// Internal declarations of the CUDA library (kernel parameter blocks and
// launchers).  Not part of the public ABI; see include/mc_transport.h.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mcgpu {

// Physical constants, CGS (CODATA 2018).
constexpr double kC = 2.99792458e10;
constexpr double kH = 6.62607015e-27;
constexpr double kKB = 1.380649e-16;
constexpr double kSigmaSB = 5.670374419e-5;
constexpr double kSigmaT = 6.6524587321e-25;
constexpr double kMe = 9.1093837015e-28;
constexpr double kEcharge = 4.803204712570263e-10;
constexpr double kEv = 1.602176634e-12;
constexpr double kPi = 3.14159265358979323846;
constexpr double kZeta5 = 1.0369277551433699263;

constexpr int kPlanckLmax = 1024;

// Run-statistics slots (device array of unsigned long long).
enum Stat : int {
  kStEscaped = 0, kStReabsorbed, kStCapped, kStSegments, kStLineChecks, kStResonances,
  kStLineInteractions, kStEScatters, kStShellCrossings, kNStats
};
constexpr int kNCounters = 6;

// One entry of a downbranch branching row, in the order of the row:
// thr = ceil(cdf * 2^53) (so that z < cdf <=> u53 < thr for z = u53 2^-53),
// the emitted line with its frequency and reciprocal, and the guide entry
// of bucket (this entry's position in the row): the first position whose
// thr exceeds the smallest u53 of that bucket.
struct DbrRec {
  unsigned long long thr;
  double nu;
  double inv_nu;
  uint32_t emit;
  uint32_t guide;
};

// Macro-atom level (mode MC_LINE_MACROATOM), one per downbranch row: jump
// when the decision draw u53 < jump_thr (= ceil(p 2^53), so exactly z < p),
// target from the row's jump entries (first with u53 < thr), deactivation
// through the downbranch row (begin, length).
struct MaRow {
  unsigned long long jump_thr;
  uint32_t jump_begin, jump_len;
  uint32_t dbr_begin, dbr_len;
};
struct MaJump {
  unsigned long long thr;  // ceil(cdf 2^53)
  int32_t target;          // row jumped to
  uint32_t pad;
};
constexpr uint32_t kMaMaxJumps = 1024;

// Everything the transport kernel reads or writes.
struct TransportParams {
  int32_t S, L;
  const double *x_in, *x_out;        // [S] radii in units of c t_exp
  const double *inv_x_in, *inv_x_out;// [S]
  const double *kappa;               // [S] sigma_T n_e c t_exp (per unit x)
  const double *nu;                  // [L] line frequencies, descending
  const double *tau;                 // [S*L] Sobolev depths (fp64 mode)
  const float *tau32;                // [S*L] Sobolev depths (mixed mode)
  const int32_t *line_row;           // [L] downbranch row of each line
  const uint32_t *dbr_offset, *dbr_line;
  const double *dbr_cdf;
  const double *inv_kappa;           // [S] 1/kappa (0 where kappa = 0), or nullptr
  const unsigned long long *row_info;// [L] row begin | row length << 32, or nullptr
  const DbrRec *dbr_rec;             // [nnz] guide-table rows, or nullptr
  const MaRow *ma_row;               // [rows] macro-atom levels, or nullptr (no internal jumps)
  const MaJump *ma_jump;             // [n] macro-atom jump entries
  const DbrRec *dbr_bucket;          // [nnz] bucket k of a row: copy of its guide entry's
                                     // record, guide field = that entry's position
  double *j_est, *nu_bar;            // [S] raw sums
  double *j_blue;                    // [S*L] raw sums or nullptr
  double *spectrum;                  // [bins + 2]
  unsigned long long *stats;         // [kNStats]
  int32_t spec_bins;
  double spec_lo, spec_hi, spec_dnu;
  uint64_t n_packets;                // packets of this launch
  uint64_t first_packet;             // global id of the first (records are relative)
  uint32_t iteration, key0, key1;
  double e_cmf;                      // comoving packet energy, Eq. 10
  double nu_scale;                   // k T_inner / h
  const double *planck_cdf;          // [kPlanckLmax + 1]
  uint64_t max_segments;
  unsigned long long *work_counter;  // next unclaimed packet id
  int32_t *rec_status;               // per-packet records or nullptrs
  double *rec_nu, *rec_e;
  unsigned long long *rec_cnt;       // [n * kNCounters]
  const float *shell32;              // [4 S] binary32 shell table (mixed; batched launch)
  unsigned long long *est_fix;       // [2 S] mixed: J, nu_bar sums in fixed point (see below)
  double inv_nu_ref;                 // mixed: 1 / (k T_inner / h), scale of nu in nu_bar
  const TransportParams *batch;      // batched launch: per-model parameters, or nullptr
  const unsigned long long *batch_prefix;  // [n_models + 1] packet offsets of the models
  int32_t n_models;
  unsigned long long timeout_ns;     // 0 = none
  const uint32_t *cancel;            // mapped host word: nonzero stops the launch (or nullptr)
  unsigned long long *flags;         // [0] deadline hit, [1] work queue empty (ns),
                                     // [2] last warp done (ns), [3] first warp start (ns)
  // virtual packets (Sect. 2.9; binary64 kernel)
  int32_t n_virtual;                 // N_v per launch of an r-packet trajectory, 0 = off
  double tau_v_max;                  // > 0: a v-packet is dropped once tau_v exceeds it
  double *spectrum_v;                // [bins + 2] sums of E_lab exp(-tau_v) (Eq. 21)
};

constexpr int kNCounterSlots = kNStats + 5;  // stats, work counter, flags[4]

// Mixed precision accumulates the J and nu_bar estimators as unsigned 64-bit
// fixed point: each segment's contribution (in units of the packet energy E,
// and nu_cmf in units of k T_inner / h) is rounded to a multiple of 2^-32 and
// added with integer atomics, so the sums do not depend on the order in which
// packets finish (the radiation-field update, and every later iteration, are
// then the same whatever the launch mixes).  Headroom: 2^64 / 2^32 = 4.3e9
// units per shell.
constexpr double kEstFixScale = 0x1.0p32;
constexpr float kEstFixScaleF = 0x1.0p32f;

struct PlasmaParams {
  int32_t S, I, K, L;
  const double *t_rad, *w;           // [S]
  const double *eps_erg, *g;         // [I*K]
  const uint8_t *metastable;         // [I*K]
  const double *n_ion;               // [S*I]
  int32_t lte_excitation;
  double *pop;                       // [S*I*K]
  const int32_t *lev_l, *lev_u;      // [L] level index ion*K + level
  const double *line_pref;           // [L] (pi e^2 / m_e c) f lambda t_exp
  const double *line_gratio;         // [L] g_l / g_u
  double *tau;                       // [S*L] or nullptr
  float *tau32;                      // [S*L] or nullptr
};

// Ionization balance (Sect. 2.3, Eqs. 2-3) of S shells, E elements of J
// stages each; ion_of[e*J + j] is the ion holding stage j of element e, or -1
// (partition function 1).  Writes n_ion, n_e and the Thomson opacity arrays.
struct IonParams {
  int32_t S, I, K, E, J;
  int32_t mode;                      // 1 Saha (Eq. 2), 2 modified nebular (Eq. 3)
  const double *t_rad, *w;           // [S]
  const double *eps_erg, *g;         // [I*K]
  const int32_t *ion_of;             // [E*J]
  const double *chi_erg, *zeta;      // [E*(J-1)]
  double delta;
  const double *n_element;           // [S*E]
  double *phi;                       // [S*E*(J-1)] scratch: n_{j+1} n_e / n_j
  double *n_ion;                     // [S*I]
  double *n_e;                       // [S]
  double *kappa, *inv_kappa;         // [S] sigma_T n_e c t_exp and its inverse (0 if kappa = 0)
  float *shell32;                    // [4S] or nullptr: binary32 copies at 2S (kappa), 3S (inverse)
  double t_exp;                      // s (kappa = ((sigma_T n_e) c) t_exp)
};
constexpr int kIonMaxStages = 16;

struct UpdateParams {
  int32_t S;
  const double *j_est, *nu_bar, *norm;
  double *t_rad, *w;
  double c_tr;                       // (h/k) pi^4 / (360 zeta(5))
};

// Launchers (return the launch error).  `line_mode` 0 scatter / 1 downbranch,
// `precision` 0 fp64 / 1 mixed.
cudaError_t launch_transport(const TransportParams &p, int line_mode, int precision, bool j_blue,
                             bool record, int grid, int block, cudaStream_t st);
int transport_block_size();
cudaError_t transport_occupancy(int line_mode, int precision, bool j_blue, bool record, int S,
                                int *blocks_per_sm);
const void *select_mixed_kernel(int line_mode, bool j_blue, bool record);
// Batched launches: `block` threads per block (64, 128 or 256).
cudaError_t batch_occupancy(int line_mode, bool j_blue, bool record, int n_models, int block,
                            int *blocks_per_sm);
cudaError_t launch_transport_batch(const TransportParams &p, int line_mode, bool j_blue, bool record,
                                   int grid, int block, cudaStream_t st);
size_t mixed_smem_bytes(int S);
cudaError_t launch_to_f32(const double *in, float *out, size_t n, cudaStream_t st);
// j_est = fix[s] 2^-32 E, nu_bar = fix[S + s] 2^-32 E nu_ref (mixed precision).
// J_blue of a mixed launch is summed in the j_blue buffer as 64-bit fixed
// point (units of 2^-32 E / nu_ref) and converted in place after the launch.
cudaError_t launch_jblue_from_fix(double *j_blue, size_t n, double e_cmf, double inv_nu_ref, cudaStream_t st);
// Binary64 J_blue: the transport sums E_lab / nu_lab^2 per (shell, line);
// this multiplies every cell by its line frequency nu_j (Eq. 17).
cudaError_t launch_jblue_times_nu(double *j_blue, const double *nu, int S, int L, cudaStream_t st);
cudaError_t launch_est_from_fix(const unsigned long long *fix, int S, double e_cmf, double nu_ref,
                                double *j_est, double *nu_bar, cudaStream_t st);
cudaError_t launch_ionization(const IonParams &p, cudaStream_t st);  // two kernels
cudaError_t launch_populations(const PlasmaParams &p, cudaStream_t st);
cudaError_t launch_sobolev_tau(const PlasmaParams &p, cudaStream_t st);
cudaError_t launch_update(const UpdateParams &p, cudaStream_t st);
cudaError_t launch_zero(double *a, size_t n_a, double *b, size_t n_b, double *c, size_t n_c,
                        unsigned long long *u, size_t n_u, cudaStream_t st);
cudaError_t launch_zero_large(double *a, size_t n, cudaStream_t st);
cudaError_t launch_dbr_setup(uint32_t nnz, uint32_t n_rows, uint32_t L, int K,
                             const uint32_t *dbr_offset, const uint32_t *dbr_line,
                             const double *dbr_cdf, const double *nu, const int32_t *line_row,
                             DbrRec *rec, DbrRec *bucket, unsigned long long *row_info,
                             cudaStream_t st);
cudaError_t launch_line_setup(int L, int K, const double *nu, const double *f, const int32_t *ion,
                              const int32_t *lower, const int32_t *upper, const double *g,
                              double t_exp, int32_t *lev_l, int32_t *lev_u, double *pref,
                              double *gratio, int32_t *row, cudaStream_t st);

}  // namespace mcgpu
