/*
 * mc_transport.h -- C ABI of the GB300 Monte Carlo packet-transport library.
 *
 * The library implements the per-iteration Monte Carlo radiative transfer of
 * Kerzendorf & Sim (2014, "A spectral synthesis code for rapid modelling of
 * supernovae"), Sect. 2: indivisible energy packets injected at the inner
 * boundary of homologously expanding spherical shells (Sect. 2.4, Eqs. 9-10),
 * propagated through Thomson and Sobolev line opacity (Sects. 2.5-2.6,
 * Eqs. 11-12), with scatter or downbranch line interactions (Sect. 2.5), the
 * J, nu_bar and J_blue estimators (Sect. 2.7, Eqs. 13, 14, 17), the
 * radiation-field update (Eqs. 15-16) and the direct-binning spectrum
 * (Sect. 2.9).  All compute runs in CUDA kernels for sm_103a.
 *
 * Conventions common to every entry point:
 *  - Units are CGS: velocities cm/s, densities cm^-3, times s, frequencies Hz,
 *    energies erg (level energies in eV where stated).
 *  - Pointers in descriptors and outputs are HOST pointers unless stated.
 *    Input arrays are copied to the device during the call; the caller keeps
 *    ownership.  Output arrays are caller-allocated host buffers.
 *  - Every function returns mc_status: 0 on success, negative on error
 *    (MC_ERR_*), positive for warnings (MC_WARN_*).  After an error,
 *    mc_last_error_message() explains it.  No C++ exception crosses the ABI.
 *  - A model is used by one host thread at a time; distinct models are
 *    independent.  Device work is enqueued on the model's CUDA stream.
 *  - Shell s covers [v_inner[s], v_outer[s]); shells are contiguous and
 *    ordered outward.  Lines are ordered by strictly DESCENDING frequency, so
 *    "the next redward line" of Sect. 2.6 is the next index.
 */
#ifndef MC_TRANSPORT_H
#define MC_TRANSPORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mc_status;

#define MC_OK 0
#define MC_ERR_INVALID_ARG (-1) /* NULL, empty, non-monotone, NaN or negative input */
#define MC_ERR_OOM (-2)         /* device allocation failed */
#define MC_ERR_CUDA (-3)        /* a CUDA runtime call failed */
#define MC_ERR_NOT_READY (-4)   /* run before mc_set_plasma, or read before a run */
#define MC_ERR_TIMEOUT (-5)     /* the transport kernel hit its deadline */
#define MC_ERR_UNSUPPORTED (-6) /* option not available for this model */
#define MC_WARN_CAPPED 1        /* some packets hit max_segments (counted in stats) */

/* Line-interaction modes (Table 1 of the paper). */
#define MC_LINE_SCATTER 0    /* resonance scattering: re-emit in the absorbing line */
#define MC_LINE_DOWNBRANCH 1 /* macro atom without internal jumps: re-emit via the
                                branching table of the activated upper level */
#define MC_LINE_MACROATOM 2  /* macro atom: internal jumps between the ion's levels
                                (ma_jump_* tables), then re-emission via the branching
                                table of the level it deactivates from */

/* Ionization balance (Sect. 2.3), mc_atomic_desc.ionization_mode. */
#define MC_ION_FIXED 0   /* ion densities and n_e as given */
#define MC_ION_SAHA 1    /* Saha equation at T_R (Eq. 2) */
#define MC_ION_NEBULAR 2 /* modified nebular approximation (Eq. 3), T_e = 0.9 T_R */
#define MC_ION_MAX_STAGES 16

/* Precision modes. */
#define MC_PRECISION_FP64 0  /* all transport arithmetic in binary64 */
#define MC_PRECISION_MIXED 1 /* distances and optical depths in binary32; comoving
                                frequency and line-resonance test in binary64; J, nu_bar
                                and J_blue summed exactly in 64-bit fixed point from
                                binary32 contributions (line frequencies must lie in
                                (1e-30, 1e30) Hz) */

/* Packet fates reported by mc_read_packets. */
#define MC_PACKET_ESCAPED 1
#define MC_PACKET_REABSORBED 2
#define MC_PACKET_CAPPED 3

/* Per-packet counters reported by mc_read_packets, in this order. */
#define MC_COUNTER_SEGMENTS 0         /* flight segments (one per event) */
#define MC_COUNTER_LINE_CHECKS 1      /* line-list entries examined */
#define MC_COUNTER_RESONANCES 2       /* Sobolev points reached within a segment */
#define MC_COUNTER_LINE_INTERACTIONS 3
#define MC_COUNTER_E_SCATTERS 4
#define MC_COUNTER_SHELL_CROSSINGS 5
#define MC_N_COUNTERS 6

typedef struct mc_model mc_model; /* opaque; owns all device memory of one model */

/* Model geometry, Sect. 2.1: homologous expansion, r = v t_exp. */
typedef struct {
    uint32_t n_shells;      /* S >= 1 */
    const double *v_inner;  /* [S] cm/s, v_inner[s+1] == v_outer[s] */
    const double *v_outer;  /* [S] cm/s, > v_inner, < c */
    const double *n_e;      /* [S] free-electron density, cm^-3, >= 0 */
    double t_exp;           /* time since explosion, s, > 0 */
} mc_geometry_desc;

/* Line list, Sects. 2.5-2.6.  f/ion/lower/upper are needed only when the
 * Sobolev depths are computed by the library (Eq. 12) or in downbranch mode. */
typedef struct {
    uint32_t n_lines;       /* L >= 1 */
    const double *nu;       /* [L] Hz, strictly descending, > 0 */
    const double *f;        /* [L] absorption oscillator strengths, or NULL */
    const int32_t *ion;     /* [L] ion index in [0, n_ions), or NULL */
    const int32_t *lower;   /* [L] lower level in [0, n_levels), or NULL */
    const int32_t *upper;   /* [L] upper level, > lower, or NULL */
} mc_line_desc;

/* Atomic data and ion densities for the level populations of Sect. 2.3
 * (Eqs. 4-5) and the downbranch table.  Level (i, k) is entry i*n_levels + k.
 * The downbranch table is CSR over upper levels: row r = ion*n_levels + upper
 * lists, in any fixed order, the lines whose upper level is r (dbr_line) and
 * the running branching probability (dbr_cdf, non-decreasing, last == 1). */
typedef struct {
    uint32_t n_ions, n_levels;
    const double *energy_ev;   /* [I*K] excitation energy above the ion ground state, eV */
    const double *g;           /* [I*K] statistical weights, > 0 */
    const uint8_t *metastable; /* [I*K] 1 = ground/metastable (Eq. 4), 0 = diluted (Eq. 5) */
    const double *n_ion;       /* [S*I] ion number densities, cm^-3 (may be NULL in an ionization mode) */
    const uint32_t *dbr_offset;/* [I*K + 1] or NULL (scatter mode) */
    const uint32_t *dbr_line;  /* [nnz] line index of each branch */
    const double *dbr_cdf;     /* [nnz] cumulative branching ratio within the row */
    int32_t lte_excitation;    /* 1: Eq. 4 for every level; 0: dilute-lte (Eq. 5) */
    /* Macro-atom internal jumps (MC_LINE_MACROATOM, else NULL), rows as the
     * downbranch table: from level r the atom jumps with probability
     * ma_jump_p[r] in [0, 1) to a level picked by the CSR row r of
     * (ma_jump_target, ma_jump_cdf) -- targets are rows with a non-empty
     * downbranch row, cdf non-decreasing with last == 1, and the row is not
     * empty when ma_jump_p[r] > 0 -- or deactivates through its downbranch
     * row.  Draws per step: the jump decision, then the target if it jumps;
     * then the emitting line.  After 1024 jumps the atom deactivates. */
    const double *ma_jump_p;          /* [I*K] */
    const uint32_t *ma_jump_offset;   /* [I*K + 1] */
    const int32_t *ma_jump_target;    /* [n] */
    const double *ma_jump_cdf;        /* [n] */
    /* Ionization balance (Sect. 2.3, Eqs. 2-3).  With MC_ION_SAHA or
     * MC_ION_NEBULAR every recomputation of the Sobolev depths first solves,
     * per shell at its T_R and W, for the stage fractions of each element and
     * the electron density that conserve charge (n_e = sum over elements and
     * stages of stage number x stage density), and replaces n_ion (which may
     * then be NULL) and the geometry's n_e -- hence the Thomson opacity -- by
     * the solution.  Partition functions: sum over the ion's levels of
     * g exp(-E/kT_R); a stage without an ion (in particular the bare top stage
     * J-1) has Z = 1.  Nebular mode scales Saha's Phi by
     * W [delta zeta + W (1 - zeta)] (T_e/T_R)^(1/2) with T_e = 0.9 T_R.
     * Given Sobolev depths (mc_set_plasma with tau) leave n_e and n_ion as
     * they are. */
    int32_t ionization_mode;          /* MC_ION_* */
    uint32_t n_elements, n_stages;    /* E >= 1; 2 <= J <= MC_ION_MAX_STAGES */
    const int32_t *ion_element;       /* [I] element of each ion, in [0, E) */
    const int32_t *ion_stage;         /* [I] its stage in [0, J-1); (element, stage) pairs distinct */
    const double *chi_ev;             /* [E*(J-1)] ionization potential of stage j, eV, > 0 */
    const double *zeta;               /* [E*(J-1)] recombination fraction to the ground state,
                                         in [0, 1] (nebular mode; else may be NULL) */
    double delta;                     /* Eq. 3 delta, > 0 (nebular mode) */
    const double *n_element;          /* [S*E] element number densities, cm^-3, >= 0 */
} mc_atomic_desc;

/* Run options. */
typedef struct {
    int32_t line_mode;          /* MC_LINE_* */
    int32_t precision;          /* MC_PRECISION_* */
    int32_t j_blue;             /* 1: accumulate J_blue estimators (Eq. 17) */
    int32_t record_packets;     /* 1: keep per-packet fates for mc_read_packets */
    uint32_t spec_bins;         /* spectrum bins, uniform in frequency */
    double spec_nu_lo, spec_nu_hi; /* spectrum range, Hz */
    uint64_t max_packets;       /* largest n_packets of any run (sizes packet records) */
    uint64_t max_segments;      /* per-packet segment cap; 0 = 1e6 */
    double delta_t;             /* simulated time interval of Eq. 10, s; 0 = 1 s */
    uint64_t timeout_ns;        /* transport-kernel deadline; 0 = none */
} mc_run_desc;

/* Optional device allocator (e.g. a framework's caching allocator).  alloc
 * returns device memory usable on the model's stream, or NULL on failure. */
typedef struct {
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, void *ctx);
    void *ctx;
} mc_allocator;

/* Totals of the last run. */
typedef struct {
    uint64_t packets, escaped, reabsorbed, capped;
    uint64_t segments, line_checks, resonances, line_interactions, e_scatters, shell_crossings;
} mc_packet_stats;

/* Create a model on the current CUDA device.
 *  geom, lines, run: required.  atomic: required when the library computes the
 *  Sobolev depths (mc_set_plasma with tau == NULL) or in downbranch mode.
 *  alloc: NULL = stream-ordered cudaMallocAsync.  stream: a cudaStream_t, or
 *  NULL for a stream owned by the model.
 *  Errors: MC_ERR_INVALID_ARG (shape/value checks listed above), MC_ERR_OOM,
 *  MC_ERR_CUDA.  On error *out is NULL. */
mc_status mc_model_create(const mc_geometry_desc *geom, const mc_line_desc *lines,
                          const mc_atomic_desc *atomic, const mc_run_desc *run,
                          const mc_allocator *alloc, void *stream, mc_model **out);

/* Set the plasma state: radiation temperature T_R and dilution factor W of
 * Eq. 1 per shell, and optionally the Sobolev depths.
 *  t_rad [S] K or NULL (= 1e4 K, Sect. 2.8); w [S] or NULL (= geometric
 *  dilution at the shell centre, Sect. 2.8).  tau [S*L] shell-major given
 *  Sobolev depths, or NULL to recompute them on the device from the
 *  populations of Eqs. 4-5 and Eq. 12 before the next run (needs atomic data).
 *  Errors: MC_ERR_INVALID_ARG (NaN/negative values, tau == NULL without
 *  atomic data). */
mc_status mc_set_plasma(mc_model *m, const double *t_rad, const double *w, const double *tau);

/* Enqueue one Monte Carlo iteration (Sects. 2.4-2.7, 2.9): recompute the
 * Sobolev depths if the plasma changed, zero the estimators, inject and
 * transport n_packets packets from a blackbody of temperature t_inner (K).
 * Random numbers: Philox4x32-10 (Salmon et al. 2011) with key = seed and
 * counter (draw block, packet id, iteration, 0), so results depend only on
 * (seed, iteration, packet id).  Asynchronous on the model's stream.
 *  Errors: MC_ERR_NOT_READY (no plasma set), MC_ERR_INVALID_ARG
 *  (n_packets == 0 or > max_packets when records are kept, n_packets >= 2^32,
 *  t_inner <= 0). */
mc_status mc_run_iteration(mc_model *m, uint64_t seed, uint32_t iteration, uint64_t n_packets,
                           double t_inner);

/* Packets [first_packet, first_packet + n_packets) of an iteration of n_total
 * packets (packet energy E = L_i dt / n_total, Eq. 10); the random draws of a
 * packet depend only on (seed, iteration, packet id), so disjoint ranges run
 * on different devices or at different times reproduce the whole iteration.
 * Estimators and spectrum hold the sums over this range; packet records are
 * indexed from first_packet.  mc_run_iteration(m, s, it, n, T) is
 * mc_run_iteration_range(m, s, it, 0, n, n, T).
 *  Errors: MC_ERR_INVALID_ARG (empty range, first + n_packets > n_total,
 *  n_total >= 2^32, records too small), MC_ERR_NOT_READY. */
mc_status mc_run_iteration_range(mc_model *m, uint64_t seed, uint32_t iteration, uint64_t first_packet,
                                 uint64_t n_packets, uint64_t n_total, double t_inner);

/* Ask this model's transport launches to stop (stop = 1) or withdraw the
 * request (stop = 0).  A single-model launch that is running, or starts,
 * while the request stands stops at its next look at it (each warp looks
 * every 256 loop iterations: microseconds to a millisecond), leaving
 * unfinished packets, and the run's reads return MC_ERR_TIMEOUT with a
 * message naming the cancel.  The request stands until withdrawn.  The call
 * writes one word of pinned host memory and may come from any host thread
 * while the launch runs.  Batched launches do not look at it.
 *  Errors: MC_ERR_INVALID_ARG (m NULL, stop not 0 or 1). */
mc_status mc_cancel(mc_model *m, int32_t stop);

/* Update T_R and W from the last run's estimators (Eqs. 15-16) on the device;
 * shells with no path length keep their values.  The next run recomputes the
 * Sobolev depths when they are not given.  Copies the new values to t_rad_out
 * and w_out ([S], either may be NULL); synchronises the stream when either is
 * given, and is asynchronous on the model's stream when both are NULL.
 *  Errors: MC_ERR_NOT_READY (no run yet), MC_ERR_CUDA. */
mc_status mc_update_radiation_field(mc_model *m, double *t_rad_out, double *w_out);

/* Read the last run's estimators (synchronises).  Raw sums, any may be NULL:
 *  j_est[S]   = sum E_cmf l D over segments in the shell, l in units of c t_exp
 *  nu_bar[S]  = sum E_cmf nu_cmf l D
 *  j_blue[S*L]= sum E_lab (nu_line/nu_lab)^2 / nu_line over Sobolev points passed
 *               (shell-major; requires run->j_blue)
 *  norm[S]    = c t_exp / (4 pi delta_t V): multiplying j_est, nu_bar or j_blue
 *               by it gives Eqs. 13, 14 and 17 (with the resonance path c t_exp).
 *  Errors: MC_ERR_NOT_READY, MC_ERR_UNSUPPORTED (j_blue requested but off). */
mc_status mc_read_estimators(mc_model *m, double *j_est, double *nu_bar, double *j_blue,
                             double *norm);

/* Read the last run's direct-binning spectrum and totals (synchronises).
 *  spectrum[spec_bins + 2]: sum of escaping lab energies per bin, then the
 *  underflow and overflow sums; divide by (delta_t * bin width) for L_nu.
 *  stats may be NULL.  Returns MC_WARN_CAPPED if any packet was capped. */
mc_status mc_read_spectrum(mc_model *m, double *spectrum, mc_packet_stats *stats);

/* Read per-packet results [first, first+count) of the last run (requires
 * record_packets).  Any output may be NULL.  status: MC_PACKET_*; nu, energy:
 * final lab frequency and energy; counters: [count * MC_N_COUNTERS].
 *  Errors: MC_ERR_UNSUPPORTED (records off), MC_ERR_INVALID_ARG (range). */
mc_status mc_read_packets(mc_model *m, uint64_t first, uint64_t count, int32_t *status,
                          double *nu, double *energy, uint64_t *counters);

/* Read the device-side plasma state: t_rad[S], w[S], tau[S*L] (shell-major,
 * binary64 even in mixed mode).  Recomputes tau first if it is stale. */
mc_status mc_read_plasma(mc_model *m, double *t_rad, double *w, double *tau);

/* Read the electron densities n_e[S] (cm^-3) and ion densities n_ion[S*I]
 * the transport uses: the solution of the ionization balance at the current
 * T_R and W (recomputed first if stale) in an ionization mode, else the
 * given values.  Either output may be NULL.  Synchronises.
 *  Errors: MC_ERR_NOT_READY (no plasma set), MC_ERR_INVALID_ARG (n_ion
 *  without atomic data). */
mc_status mc_read_ionization(mc_model *m, double *n_e, double *n_ion);

/* Device times of the last run, from CUDA events on the model's stream:
 * ms[0] Sobolev-depth recomputation (0 if none), ms[1] transport,
 * ms[2] radiation-field update (0 if not run).  Synchronises. */
mc_status mc_read_timing(mc_model *m, float *ms);

/* Phases of the last transport launch, from the GPU's global timer:
 * ms[0] from the first warp's start until the packet queue ran empty (every
 * packet claimed), ms[1] from then until the last warp finished (the tail of
 * long random walks).  Synchronises. */
mc_status mc_read_transport_phases(mc_model *m, float *ms);

/* Number of kernels this model has launched since creation. */
mc_status mc_launch_count(const mc_model *m, uint64_t *count);

/* Inner-boundary temperature (Sect. 2.8).  Eq. 18: *t_inner such that
 * 4 pi r_inner^2 sigma_SB t_inner^4 = l_outer (erg/s), r_inner = v_inner[0]
 * t_exp of the model.  Errors: MC_ERR_INVALID_ARG (NULL, l_outer <= 0). */
mc_status mc_t_inner_from_luminosity(const mc_model *m, double l_outer, double *t_inner);

/* Luminosity emitted in the last iteration: the lab-frame energy of the
 * escaping packets (every spectrum bin, including the two outside the
 * range, summed in bin order) divided by delta_t, in erg/s.  Synchronises
 * the model's stream.  Errors: MC_ERR_INVALID_ARG, MC_ERR_NOT_READY. */
mc_status mc_emitted_luminosity(mc_model *m, double *l_emitted);

/* T_inner for the next iteration so that the emitted luminosity would match
 * the requested one if it scaled like T_inner^4 (the paper raises T_inner
 * when too little escapes and lowers it otherwise):
 * t_inner (l_requested / l_emitted)^(1/4); t_inner when l_emitted <= 0. */
double mc_t_inner_update(double t_inner, double l_requested, double l_emitted);

/* Virtual packets (Sect. 2.9, Eqs. 19-21) in the following iterations: at
 * injection and after every interaction each packet spawns n_virtual
 * v-packets with directions uniform in (mu_min, 1], mu_min = -sqrt(1 -
 * (r_inner/r)^2), comoving energy E (1 - mu_min) / (2 n_virtual) (after an
 * interaction) or E 2 mu_v / n_virtual (at injection); each flies to the
 * outer boundary without interacting and adds exp(-tau_v) times its lab-frame
 * energy to the bin of its lab frequency in the v-spectrum.  tau_v_max > 0
 * drops a v-packet once tau_v exceeds it (changing the spectrum by less than
 * exp(-tau_v_max) of that packet); 0 keeps every v-packet.  The v-packets
 * draw from their own Philox stream, so the r-packets' histories, estimators
 * and spectrum are unchanged.  n_virtual = 0 turns them off.  Binary64
 * models only (MC_ERR_UNSUPPORTED otherwise); n_virtual <= 1024.
 * Errors: MC_ERR_INVALID_ARG, MC_ERR_UNSUPPORTED, MC_ERR_OOM. */
mc_status mc_set_virtual_packets(mc_model *m, uint32_t n_virtual, double tau_v_max);

/* v-spectrum of the last iteration: spectrum_v[spec_bins + 2] receives the
 * raw sums of E_lab exp(-tau_v) (erg) per bin, then the below-range and
 * above-range sums (the layout of mc_read_spectrum).  Synchronises the
 * model's stream.  Errors: MC_ERR_INVALID_ARG, MC_ERR_NOT_READY (no run, or
 * virtual packets off). */
mc_status mc_read_virtual_spectrum(mc_model *m, double *spectrum_v);

/* Device views of the model's estimator buffers, for callers that combine
 * the partial sums of several packet ranges in place (a sum all-reduce across
 * processes, one GPU each, each having run mc_run_iteration_range on its own
 * disjoint range of the same iteration) before mc_update_radiation_field,
 * which reads j_est and nu_bar from these same buffers (Eqs. 15-16).  Packet
 * draws are keyed by packet index, so the combined sums are those of the
 * whole iteration run on one GPU, up to summation order.
 *  out->j_est, nu_bar: [n_shells] binary64 raw sums (Eqs. 13-14);
 *  out->j_blue: [n_shells * n_lines] or NULL when J_blue is off;
 *  out->spectrum: [spec_bins + 2] (last two: below / above the range);
 *  out->stream: the model's stream (cudaStream_t); the buffers hold the last
 *  iteration's sums once the work queued there has completed.
 * The pointers are owned by the model and valid until mc_model_destroy; they
 * are device memory on the model's device.  Errors: MC_ERR_INVALID_ARG. */
typedef struct {
  double *j_est, *nu_bar, *j_blue, *spectrum;
  uint32_t n_shells, n_lines, spec_bins;
  void *stream;
} mc_estimator_views;
mc_status mc_device_estimators(mc_model *m, mc_estimator_views *out);

/* Wait for the model's stream. */
mc_status mc_synchronize(mc_model *m);

/* Free all device memory of the model (NULL is ignored). */
void mc_model_destroy(mc_model *m);

/* ---------------------------------------------------------------------------
 * Batched iterations of many models.
 *
 * A batch advances several mixed-precision models (MC_PRECISION_MIXED, one
 * device, the same line mode, J_blue and record settings) by one
 * Monte Carlo iteration each with a single persistent transport launch: the
 * packets of all models are drawn from one queue (largest model first by
 * default).  Each model's iteration is exactly its single-model iteration:
 * the same draws, the same compiled kernel, and J, nu_bar and J_blue summed
 * in fixed point, so they and the updated T_R, W are bit-identical to the
 * model run alone; only the binary64 spectrum sums depend on summation order.
 * The whole iteration -- Sobolev depths where stale, estimator zeroing, transport and,
 * when `update` is set, Eqs. 15-16 for every model -- is captured as one CUDA
 * graph on the first call and replayed while the batch's shape (models with
 * stale depths, update flag, total packets) is unchanged.  Results are read
 * per model with mc_read_estimators / mc_read_spectrum / mc_read_plasma /
 * mc_read_packets (ordered after the batch on the models' stream).  A model in
 * a batch cannot be run alone until the batch is destroyed.
 *  seeds, iterations, n_packets, t_inner: [n_models] in the order passed to
 *  mc_batch_create; model i runs its iteration iterations[i] with seeds[i]
 *  (the same draws as mc_run_iteration(m, seeds[i], iterations[i], ...)).  Errors: MC_ERR_INVALID_ARG, MC_ERR_UNSUPPORTED (a model
 *  not in mixed precision), MC_ERR_NOT_READY (no plasma state), MC_ERR_CUDA;
 *  messages via mc_batch_last_error_message. */
typedef struct mc_batch mc_batch;

mc_status mc_batch_create(mc_model *const *models, uint32_t n_models, mc_batch **out);
mc_status mc_batch_run_iteration(mc_batch *b, const uint64_t *seeds, const uint32_t *iterations,
                                 const uint64_t *n_packets, const double *t_inner, int32_t update);
mc_status mc_batch_synchronize(mc_batch *b);
/* Device time of the last batched transport launch, ms[0] (synchronises). */
mc_status mc_batch_read_timing(mc_batch *b, float *ms);
/* Phases of the last batched transport launch, as mc_read_transport_phases:
 * ms[0] until the packet queue of all models ran empty, ms[1] from then until
 * the last warp finished (synchronises). */
mc_status mc_batch_read_phases(mc_batch *b, float *ms);
const char *mc_batch_last_error_message(const mc_batch *b);
void mc_batch_destroy(mc_batch *b);

/* Launch shape of a batch.  None of these changes any model's results (the
 * packet histories and fixed-point J, nu_bar sums do not depend on which
 * thread transports a packet or when).
 *  block:         threads per block, 64, 128 or 256 (0: 128).
 *  blocks_per_sm: resident blocks per SM of the persistent grid (0: as many
 *                 as fit; larger values are clamped to what fits).
 *  order:         MC_ORDER_PACKETS -- models with more packets are queued
 *                 first; MC_ORDER_WORK -- by packets x lines; MC_ORDER_GIVEN --
 *                 the order passed to mc_batch_create. */
enum { MC_ORDER_PACKETS = 0, MC_ORDER_WORK = 1, MC_ORDER_GIVEN = 2 };
typedef struct {
  uint32_t block;
  uint32_t blocks_per_sm;
  uint32_t order;
} mc_batch_launch;

/* Set the launch shape (MC_ERR_INVALID_ARG for an unknown block size or
 * order); the next iteration recaptures the graph. */
mc_status mc_batch_set_launch(mc_batch *b, const mc_batch_launch *launch);
/* The launch shape in use, with blocks_per_sm resolved to the value used. */
mc_status mc_batch_get_launch(const mc_batch *b, mc_batch_launch *launch);

/* CUDA-graph capture of the batched iteration.  enable = 1 (the default):
 * capture on the first call and replay while the shape is unchanged, as
 * described at mc_batch_run_iteration; enable = 0: enqueue the kernels on the
 * batch's stream directly every iteration (for tools that step through
 * individual launches, or shapes that change every iteration).  No result
 * depends on it.  Waits for the iteration in flight.
 *  Errors: MC_ERR_INVALID_ARG (b NULL, enable not 0 or 1), MC_ERR_CUDA. */
mc_status mc_batch_capture_graph(mc_batch *b, int32_t enable);

/* Autotuner: pick the fastest launch shape for these iterations by timing
 * transport-only trial iterations (update = 0, the same arguments as
 * mc_batch_run_iteration).  Coordinate search: queue order, then block size,
 * then resident blocks per SM, each trial one full batched transport launch
 * timed with events on the batch stream.  Trials leave every model's T_R, W
 * and Sobolev depths as they were (the estimators and spectrum hold the last
 * trial's sums until the next iteration overwrites them).  On return the best
 * shape is set; `best` and `best_ms` (either may be NULL) receive it and its
 * transport time; `n_trials` (may be NULL) the number of trials run. */
mc_status mc_batch_autotune(mc_batch *b, const uint64_t *seeds, const uint32_t *iterations,
                            const uint64_t *n_packets, const double *t_inner,
                            mc_batch_launch *best, float *best_ms, uint32_t *n_trials);

/* ---------------------------------------------------------------------------
 * Transport without any allocation.
 *
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory where they run the transport: code living
 * inside another framework's memory pool or under a fixed memory budget,
 * plug-ins that are handed raw device buffers and hold no allocator of their
 * own, and loops that must not pay for (or risk failing on) an allocation in
 * the middle of a time-critical sequence.
 *
 * It runs one Monte Carlo iteration exactly like mc_run_iteration on a model
 * with given Sobolev depths, binary64, no packet records, but every buffer is
 * the caller's: all pointers in mc_noalloc_args are DEVICE pointers on the
 * current device, with the layouts and value constraints of mc_model_create
 * and mc_set_plasma (they are not re-validated, only checked for NULL).  The
 * kernel's own working memory -- work counter, run statistics, the per-shell
 * radii and Thomson opacities, the Planck sampling table -- lives in a static
 * 64 KiB device array that every GPU loading the library holds until the
 * process exits; hence n_shells <= MC_NOALLOC_MAX_SHELLS, and larger models
 * are rejected with MC_ERR_INVALID_ARG.  The call performs no cudaMalloc, no
 * cudaFree and no allocating library call.
 *
 *  - The first call on a device does a one-time set-up on that device (it
 *    looks up the device address of the static array and fills the Planck
 *    table), so make that first call before any stream capture: a first call
 *    on a capturing stream is refused with MC_ERR_INVALID_ARG.  Device code
 *    loads lazily, so that first call is also when the array and the
 *    kernels' code are committed on the device; under a full memory budget it
 *    can fail with MC_ERR_CUDA (later calls then retry the set-up).
 *  - n_lines must be below 2^31 and spec_bins below 2^31 - 2.
 *  - Every call on a device shares the same static array, and the array keeps
 *    the last call's contents; the call clears what must start at zero
 *    (counters, and the j_est, nu_bar, j_blue and spectrum outputs).  Calls
 *    whose work overlaps on the GPU (on different streams, or from different
 *    host threads) race on that array: serialise them.
 *  - Asynchronous on `stream` (a cudaStream_t, NULL = legacy default stream);
 *    outputs are ready when the stream is.  Errors are reported through the
 *    return code and mc_last_error_message(NULL). */
#define MC_NOALLOC_MAX_SHELLS 1024

typedef struct {
    uint32_t n_shells;
    const double *v_inner, *v_outer, *n_e; /* [S] device: cm/s, cm/s, cm^-3 */
    double v_inner_0;                     /* host copy of v_inner[0], cm/s */
    double t_exp;                         /* s */
    uint32_t n_lines;
    const double *nu;                     /* [L] device, strictly descending */
    const double *tau;                    /* [S*L] device, shell-major Sobolev depths */
    int32_t line_mode;                    /* MC_LINE_SCATTER or MC_LINE_DOWNBRANCH */
    const int32_t *line_row;              /* [L] device: ion*n_levels + upper (downbranch) */
    const uint32_t *dbr_offset, *dbr_line;/* device branching table (downbranch) */
    const double *dbr_cdf;
    uint64_t seed;
    uint32_t iteration;
    uint64_t n_packets;                   /* 0 < n_packets < 2^32 */
    double t_inner;                       /* K */
    uint64_t max_segments;                /* 0 = 1e6 */
    double delta_t;                       /* s, 0 = 1 s */
    double *j_est, *nu_bar;               /* [S] device outputs, raw sums as mc_read_estimators */
    double *j_blue;                       /* [S*L] device output or NULL (no J_blue) */
    double *spectrum;                     /* [spec_bins + 2] device output */
    uint32_t spec_bins;
    double spec_nu_lo, spec_nu_hi;
    uint64_t *stats;                      /* device output [9] or NULL: escaped, reabsorbed,
                                             capped, segments, line_checks, resonances,
                                             line_interactions, e_scatters, shell_crossings */
} mc_noalloc_args;

mc_status mc_transport_noalloc(const mc_noalloc_args *args, void *stream);

/* ---------------------------------------------------------------------------
 * Accuracy diagnostic of the device arithmetic.
 *
 * The transport kernels evaluate -ln z of a Sect. 2.6 optical-depth draw, the
 * logarithm of the Sect. 2.4 Planck sampler, reciprocals of Doppler factors
 * and frequencies (Sect. 2.5 frame transforms) and square roots of the
 * shell-crossing and move geometry (Sect. 2.6) with their own device code,
 * not with CUDA's functions.  mc_selftest_math evaluates one of them on the
 * current device for n inputs, next to CUDA's counterpart:
 *
 *   fn = MC_MATH_NEG_LOG_U53: in = uint64_t u[n], 1 <= u <= 2^53;
 *        ours = the kernels' -ln(u 2^-53), ref = -log(u 2^-53)
 *   fn = MC_MATH_LOG:  in = double x[n] > 0 (normal); ours = log, ref = log(x)
 *   fn = MC_MATH_RCP:  in = double x[n] (normal); ours = reciprocal, ref = 1.0 / x
 *   fn = MC_MATH_SQRT: in = double x[n] >= 0 (0 or normal); ours = square root,
 *        ref = sqrt(x) (IEEE, correctly rounded)
 *   fn = MC_MATH_APPROX: in = double x[n] > 0 (normal); ours = 1 - x y^2 with
 *        y = rsqrt.approx.ftz.f64(x), ref = 1 - x r with r = rcp.approx.ftz.f64(x)
 *        (each by one fma after the product x y): the residuals that the
 *        square root's and the reciprocal's corrections assume small
 *
 * `in`, `ours` and `ref` are HOST arrays of n elements (0 < n <= 2^28); the
 * call allocates device memory, runs synchronously and frees it (a test
 * utility, not for the transport path).  Returns MC_ERR_INVALID_ARG for an
 * unknown fn, NULL buffers or a bad n, MC_ERR_CUDA (message in
 * mc_last_error_message(NULL)) if a CUDA call fails. */
#define MC_MATH_NEG_LOG_U53 0
#define MC_MATH_LOG 1
#define MC_MATH_RCP 2
#define MC_MATH_SQRT 3
#define MC_MATH_APPROX 4
mc_status mc_selftest_math(int32_t fn, const void *in, uint64_t n, double *ours, double *ref);

/* Static description of a status code. */
const char *mc_status_string(mc_status s);

/* Message of the model's last error ("" if none); m may be NULL for errors
 * of mc_model_create. */
const char *mc_last_error_message(const mc_model *m);

#ifdef __cplusplus
}
#endif

#endif /* MC_TRANSPORT_H */
