// Internal definition of mc_model and the per-model steps of an iteration,
// shared by the single-model C ABI (mc_capi.cu) and the batched launch
// (mc_batch.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mc_transport.h"
#include "mc_internal.h"

namespace mcgpu {
enum Ev { kEvPlasma0 = 0, kEvPlasma1, kEvTransport0, kEvTransport1, kEvUpdate0, kEvUpdate1, kNEv };
}

struct mc_model {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  mc_allocator alloc{};
  bool has_alloc = false;
  std::vector<void *> allocations;
  std::string err;

  uint32_t S = 0, L = 0, I = 0, K = 0;
  uint64_t nnz = 0;
  mc_run_desc run{};
  double t_exp = 0.0;
  bool has_atomic = false, has_line_meta = false;

  double *x_in = nullptr, *x_out = nullptr, *inv_x_in = nullptr, *inv_x_out = nullptr;
  double *kappa = nullptr, *inv_kappa = nullptr;
  float *shell32 = nullptr;  // [4 S] binary32 x_in^2, x_out^2, kappa', 1/kappa' (mixed precision)
  unsigned long long *est_fix = nullptr;  // [2 S] fixed-point J, nu_bar sums (mixed precision)
  mcgpu::DbrRec *dbr_rec = nullptr, *dbr_bucket = nullptr;
  mcgpu::MaRow *ma_row = nullptr;    // macro-atom levels (MC_LINE_MACROATOM)
  mcgpu::MaJump *ma_jump = nullptr;
  unsigned long long *row_info = nullptr;
  double *nu = nullptr, *tau = nullptr;
  float *tau32 = nullptr;
  int32_t *line_row = nullptr, *lev_l = nullptr, *lev_u = nullptr;
  double *line_pref = nullptr, *line_gratio = nullptr;
  uint32_t *dbr_offset = nullptr, *dbr_line = nullptr;
  double *dbr_cdf = nullptr;
  double *t_rad = nullptr, *w = nullptr, *eps_erg = nullptr, *g = nullptr, *n_ion = nullptr,
         *pop = nullptr;
  uint8_t *meta = nullptr;
  // Ionization balance (atomic ionization_mode != 0): inputs, scratch and n_e.
  int32_t ion_mode = 0, ion_E = 0, ion_J = 0;
  double ion_delta = 0.0;
  int32_t *ion_of = nullptr;
  double *chi_erg = nullptr, *zeta = nullptr, *n_element = nullptr, *ion_phi = nullptr;
  double *n_e = nullptr;  // [S] electron densities the Thomson opacity is built from
  uint32_t *cancel_host = nullptr;  // pinned, mapped: the stop request (mc_cancel)
  const uint32_t *cancel_dev = nullptr;
  double *norm = nullptr;
  double *j_est = nullptr, *nu_bar = nullptr, *j_blue = nullptr, *spectrum = nullptr;
  double *spectrum_v = nullptr;  // [bins + 2] virtual-packet spectrum (allocated on first use)
  uint32_t n_virtual = 0;
  double tau_v_max = 0.0;
  unsigned long long *counters = nullptr;  // stats [kNStats], work counter, flags
  double *planck_cdf = nullptr;
  int32_t *rec_status = nullptr;
  double *rec_nu = nullptr, *rec_e = nullptr;
  unsigned long long *rec_cnt = nullptr;

  std::vector<double> host_norm, host_x_in, host_x_out;
  double r_inner = 0.0;
  bool plasma_set = false, tau_given = false, tau_dirty = true, have_run = false;
  bool ran_plasma = false, ran_update = false;
  uint64_t last_n = 0;
  cudaEvent_t ev[mcgpu::kNEv] = {};
  uint64_t launches = 0;
  int grid = 0;
  bool in_batch = false;
};

namespace mcgpu {

// Error helpers: set the model's message and return the code.
mc_status model_fail(mc_model *m, mc_status code, const std::string &msg);

// Enqueue the plasma kernels if the Sobolev depths are stale (recording the
// plasma events when `events`), then zero the estimators and counters.
mc_status model_prepare(mc_model *m, cudaStream_t st, bool events);

// Transport parameters of packets [first, first+n) of an n_total iteration.
void model_fill_transport(const mc_model *m, TransportParams &p, uint64_t seed, uint32_t iteration,
                          uint64_t first, uint64_t n, uint64_t n_total, double t_inner);

// After the transport launch: turn the fixed-point J, nu_bar sums of a
// mixed-precision model into the binary64 estimators (no-op otherwise).
mc_status model_finish_transport(mc_model *m, const TransportParams &p, cudaStream_t st);

// Eqs. 15-16 for this model on `st`; marks the Sobolev depths stale.
mc_status model_update(mc_model *m, cudaStream_t st, bool events);

// Pinned host blocks (mapped into the device's address space if `mapped`)
// from a process-wide cache: no device-wide synchronisation once a block of
// that size class has been allocated before.  nullptr if allocation fails.
void *pinned_get(size_t bytes, bool mapped);
void pinned_put(void *p);

}  // namespace mcgpu
