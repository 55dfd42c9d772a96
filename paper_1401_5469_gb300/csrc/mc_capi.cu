// C ABI of the Monte Carlo transport library (include/mc_transport.h):
// model creation and validation, device memory, the iteration sequence of
// Kerzendorf & Sim (2014) Sect. 2.8 (plasma -> Monte Carlo -> estimators ->
// radiation field) and result readout.  Host code only marshals, validates
// and launches; every step of the transport runs in the kernels of
// mc_transport.cu and mc_plasma.cu.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mc_transport.h"
#include "mc_internal.h"
#include "mc_model_internal.h"

using namespace mcgpu;

namespace {

thread_local std::string g_create_error;


}  // namespace


namespace {

mc_status fail(mc_model *m, mc_status code, const std::string &msg) {
  if (m) m->err = msg;
  else g_create_error = msg;
  return code;
}

mc_status cuda_fail(mc_model *m, cudaError_t e, const char *what) {
  return fail(m, MC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void *dev_alloc(mc_model *m, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~static_cast<size_t>(255);
  void *p = nullptr;
  if (m->has_alloc) {
    p = m->alloc.alloc(bytes, m->alloc.ctx);
  } else if (cudaMallocAsync(&p, bytes, m->stream) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) m->allocations.push_back(p);
  return p;
}

template <typename T>
bool alloc_n(mc_model *m, T **out, size_t n) {
  *out = static_cast<T *>(dev_alloc(m, n * sizeof(T)));
  return *out != nullptr;
}

template <typename T>
cudaError_t upload(mc_model *m, T *dst, const T *src, size_t n) {
  return cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyHostToDevice, m->stream);
}

bool finite_nonneg(const double *a, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!(a[i] >= 0.0) || !std::isfinite(a[i])) return false;
  return true;
}

void free_all(mc_model *m) {
  for (void *p : m->allocations) {
    if (m->has_alloc) m->alloc.free(p, m->alloc.ctx);
    else cudaFreeAsync(p, m->stream);
  }
  m->allocations.clear();
}

// Why a transport launch stopped early (the kernel's flag word).
const char *stop_message(unsigned long long flag) {
  return flag == 2ull ? "transport launch stopped by mc_cancel" : "transport kernel stopped at its deadline";
}

mc_status recompute_tau(mc_model *m) {
  PlasmaParams pp{};
  pp.S = static_cast<int32_t>(m->S);
  pp.I = static_cast<int32_t>(m->I);
  pp.K = static_cast<int32_t>(m->K);
  pp.L = static_cast<int32_t>(m->L);
  pp.t_rad = m->t_rad;
  pp.w = m->w;
  pp.eps_erg = m->eps_erg;
  pp.g = m->g;
  pp.metastable = m->meta;
  pp.n_ion = m->n_ion;
  pp.lte_excitation = 0;
  pp.pop = m->pop;
  pp.lev_l = m->lev_l;
  pp.lev_u = m->lev_u;
  pp.line_pref = m->line_pref;
  pp.line_gratio = m->line_gratio;
  pp.tau = m->tau;
  pp.tau32 = m->tau32;
  cudaError_t e = cudaSuccess;
  if (m->ion_mode) {
    IonParams ip{};
    ip.S = pp.S; ip.I = pp.I; ip.K = pp.K;
    ip.E = m->ion_E; ip.J = m->ion_J;
    ip.mode = m->ion_mode;
    ip.t_rad = m->t_rad; ip.w = m->w;
    ip.eps_erg = m->eps_erg; ip.g = m->g;
    ip.ion_of = m->ion_of;
    ip.chi_erg = m->chi_erg; ip.zeta = m->zeta;
    ip.delta = m->ion_delta;
    ip.n_element = m->n_element;
    ip.phi = m->ion_phi;
    ip.n_ion = m->n_ion; ip.n_e = m->n_e;
    ip.kappa = m->kappa; ip.inv_kappa = m->inv_kappa; ip.shell32 = m->shell32;
    ip.t_exp = m->t_exp;
    e = launch_ionization(ip, m->stream);
    if (e != cudaSuccess) return cuda_fail(m, e, "ionization kernels");
    m->launches += 2;
  }
  e = launch_populations(pp, m->stream);
  if (e == cudaSuccess) e = launch_sobolev_tau(pp, m->stream);
  if (e != cudaSuccess) return cuda_fail(m, e, "Sobolev-depth kernels");
  m->launches += 2;
  m->tau_dirty = false;
  return MC_OK;
}

}  // namespace

namespace mcgpu {
// Message returned by mc_last_error_message(NULL) (used by entry points that
// have no model handle).
void set_create_error(const std::string &msg) { g_create_error = msg; }
}  // namespace mcgpu

extern "C" {

const char *mc_status_string(mc_status s) {
  switch (s) {
    case MC_OK: return "ok";
    case MC_ERR_INVALID_ARG: return "invalid argument";
    case MC_ERR_OOM: return "device out of memory";
    case MC_ERR_CUDA: return "CUDA error";
    case MC_ERR_NOT_READY: return "not ready";
    case MC_ERR_TIMEOUT: return "transport deadline exceeded";
    case MC_ERR_UNSUPPORTED: return "unsupported option";
    case MC_WARN_CAPPED: return "some packets hit the segment cap";
    default: return "unknown status";
  }
}

const char *mc_last_error_message(const mc_model *m) {
  return m ? m->err.c_str() : g_create_error.c_str();
}

mc_status mc_model_create(const mc_geometry_desc *geom, const mc_line_desc *lines,
                          const mc_atomic_desc *atomic, const mc_run_desc *run,
                          const mc_allocator *alloc, void *stream, mc_model **out) {
  if (!out) return fail(nullptr, MC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!geom || !lines || !run) return fail(nullptr, MC_ERR_INVALID_ARG, "geometry, lines and run are required");
  const uint32_t S = geom->n_shells, L = lines->n_lines;
  if (S == 0 || L == 0) return fail(nullptr, MC_ERR_INVALID_ARG, "need at least one shell and one line");
  if (S > 1024) return fail(nullptr, MC_ERR_INVALID_ARG, "at most 1024 shells (the shell table lives in shared memory)");
  if (!geom->v_inner || !geom->v_outer || !geom->n_e || !lines->nu)
    return fail(nullptr, MC_ERR_INVALID_ARG, "NULL geometry or line array");
  if (!(geom->t_exp > 0.0) || !std::isfinite(geom->t_exp))
    return fail(nullptr, MC_ERR_INVALID_ARG, "t_exp must be positive");
  for (uint32_t s = 0; s < S; ++s) {
    const double a = geom->v_inner[s], b = geom->v_outer[s];
    if (!(a > 0.0) || !(b > a) || !(b < kC) || !std::isfinite(b))
      return fail(nullptr, MC_ERR_INVALID_ARG, "shell velocities must satisfy 0 < v_inner < v_outer < c");
    if (s > 0 && geom->v_inner[s] != geom->v_outer[s - 1])
      return fail(nullptr, MC_ERR_INVALID_ARG, "shells must be contiguous (v_inner[s] == v_outer[s-1])");
  }
  if (!finite_nonneg(geom->n_e, S)) return fail(nullptr, MC_ERR_INVALID_ARG, "n_e must be finite and >= 0");
  for (uint32_t j = 0; j < L; ++j) {
    if (!(lines->nu[j] > 0.0) || !std::isfinite(lines->nu[j]))
      return fail(nullptr, MC_ERR_INVALID_ARG, "line frequencies must be positive and finite");
    if (j > 0 && !(lines->nu[j] < lines->nu[j - 1]))
      return fail(nullptr, MC_ERR_INVALID_ARG, "line frequencies must be strictly descending");
  }
  if (run->precision == MC_PRECISION_MIXED && !(lines->nu[0] < 1e30 && lines->nu[L - 1] > 1e-30))
    return fail(nullptr, MC_ERR_INVALID_ARG, "mixed precision needs line frequencies in (1e-30, 1e30) Hz");
  if (run->line_mode != MC_LINE_SCATTER && run->line_mode != MC_LINE_DOWNBRANCH &&
      run->line_mode != MC_LINE_MACROATOM)
    return fail(nullptr, MC_ERR_INVALID_ARG, "unknown line_mode");
  if (run->precision != MC_PRECISION_FP64 && run->precision != MC_PRECISION_MIXED)
    return fail(nullptr, MC_ERR_INVALID_ARG, "unknown precision");
  if (run->precision == MC_PRECISION_MIXED && run->line_mode != MC_LINE_SCATTER &&
      !(atomic && atomic->dbr_offset))
    return fail(nullptr, MC_ERR_INVALID_ARG, "mixed-precision downbranch needs the branching table");
  if (run->spec_bins == 0 || !(run->spec_nu_hi > run->spec_nu_lo) || !(run->spec_nu_lo >= 0.0))
    return fail(nullptr, MC_ERR_INVALID_ARG, "spectrum needs bins > 0 and 0 <= nu_lo < nu_hi");
  if (run->record_packets && (run->max_packets == 0 || run->max_packets >= (1ull << 32)))
    return fail(nullptr, MC_ERR_INVALID_ARG, "record_packets needs 0 < max_packets < 2^32");
  const bool meta = lines->ion && lines->lower && lines->upper;
  if (run->line_mode != MC_LINE_SCATTER) {
    if (!atomic || !meta || !atomic->dbr_offset || !atomic->dbr_line || !atomic->dbr_cdf)
      return fail(nullptr, MC_ERR_INVALID_ARG, "downbranch mode needs ion/upper per line and the branching table");
  }
  if (run->line_mode == MC_LINE_MACROATOM &&
      (!atomic->ma_jump_p || !atomic->ma_jump_offset || !atomic->ma_jump_target || !atomic->ma_jump_cdf))
    return fail(nullptr, MC_ERR_INVALID_ARG, "macro-atom mode needs the ma_jump_* tables");
  uint32_t I = 0, K = 0;
  uint64_t nnz = 0;
  const int32_t ion_mode = atomic ? atomic->ionization_mode : MC_ION_FIXED;
  std::vector<int32_t> ion_of;  // [E*J] ion of each (element, stage), -1 none
  if (atomic) {
    I = atomic->n_ions;
    K = atomic->n_levels;
    if (ion_mode != MC_ION_FIXED && ion_mode != MC_ION_SAHA && ion_mode != MC_ION_NEBULAR)
      return fail(nullptr, MC_ERR_INVALID_ARG, "ionization_mode must be MC_ION_FIXED, MC_ION_SAHA or MC_ION_NEBULAR");
    if (I == 0 || K == 0 || !atomic->energy_ev || !atomic->g || !atomic->metastable ||
        (!atomic->n_ion && ion_mode == MC_ION_FIXED))
      return fail(nullptr, MC_ERR_INVALID_ARG, "atomic data needs n_ions, n_levels, energies, g, metastable, n_ion");
    if (!finite_nonneg(atomic->energy_ev, static_cast<size_t>(I) * K) ||
        (atomic->n_ion && !finite_nonneg(atomic->n_ion, static_cast<size_t>(S) * I)))
      return fail(nullptr, MC_ERR_INVALID_ARG, "level energies and ion densities must be finite and >= 0");
    if (ion_mode != MC_ION_FIXED) {
      const uint32_t E = atomic->n_elements, J = atomic->n_stages;
      if (E == 0 || J < 2 || J > MC_ION_MAX_STAGES || !atomic->ion_element || !atomic->ion_stage ||
          !atomic->chi_ev || !atomic->n_element || (ion_mode == MC_ION_NEBULAR && !atomic->zeta))
        return fail(nullptr, MC_ERR_INVALID_ARG,
                    "ionization needs n_elements >= 1, 2 <= n_stages <= 16, ion_element, ion_stage, chi_ev, "
                    "n_element (and zeta in nebular mode)");
      if (static_cast<uint64_t>(S) * E * J >= (1ull << 31))
        return fail(nullptr, MC_ERR_INVALID_ARG, "too many shells x elements x stages");
      ion_of.assign(static_cast<size_t>(E) * J, -1);
      for (uint32_t a = 0; a < I; ++a) {
        const int32_t e = atomic->ion_element[a], j = atomic->ion_stage[a];
        if (e < 0 || static_cast<uint32_t>(e) >= E || j < 0 || static_cast<uint32_t>(j) + 1 >= J)
          return fail(nullptr, MC_ERR_INVALID_ARG, "ion_element/ion_stage out of range (the top stage is bare)");
        int32_t &slot = ion_of[static_cast<size_t>(e) * J + j];
        if (slot >= 0) return fail(nullptr, MC_ERR_INVALID_ARG, "two ions hold the same (element, stage)");
        slot = static_cast<int32_t>(a);
      }
      const size_t EJ1 = static_cast<size_t>(E) * (J - 1);
      for (size_t t = 0; t < EJ1; ++t)
        if (!(atomic->chi_ev[t] > 0.0) || !std::isfinite(atomic->chi_ev[t]))
          return fail(nullptr, MC_ERR_INVALID_ARG, "ionization potentials must be positive and finite");
      if (ion_mode == MC_ION_NEBULAR) {
        for (size_t t = 0; t < EJ1; ++t)
          if (!(atomic->zeta[t] >= 0.0 && atomic->zeta[t] <= 1.0))
            return fail(nullptr, MC_ERR_INVALID_ARG, "zeta must be in [0, 1]");
        if (!(atomic->delta > 0.0) || !std::isfinite(atomic->delta))
          return fail(nullptr, MC_ERR_INVALID_ARG, "delta must be positive and finite");
      }
      if (!finite_nonneg(atomic->n_element, static_cast<size_t>(S) * E))
        return fail(nullptr, MC_ERR_INVALID_ARG, "element densities must be finite and >= 0");
    }
    for (size_t a = 0; a < static_cast<size_t>(I) * K; ++a)
      if (!(atomic->g[a] > 0.0)) return fail(nullptr, MC_ERR_INVALID_ARG, "statistical weights must be > 0");
    if (meta) {
      for (uint32_t j = 0; j < L; ++j) {
        if (lines->ion[j] < 0 || static_cast<uint32_t>(lines->ion[j]) >= I || lines->lower[j] < 0 ||
            lines->upper[j] <= lines->lower[j] || static_cast<uint32_t>(lines->upper[j]) >= K)
          return fail(nullptr, MC_ERR_INVALID_ARG, "line ion/lower/upper out of range");
      }
    }
    if (lines->f && !finite_nonneg(lines->f, L))
      return fail(nullptr, MC_ERR_INVALID_ARG, "oscillator strengths must be finite and >= 0");
    if (atomic->dbr_offset) {
      const uint64_t rows = static_cast<uint64_t>(I) * K;
      if (atomic->dbr_offset[0] != 0) return fail(nullptr, MC_ERR_INVALID_ARG, "dbr_offset[0] must be 0");
      for (uint64_t r = 0; r < rows; ++r)
        if (atomic->dbr_offset[r + 1] < atomic->dbr_offset[r])
          return fail(nullptr, MC_ERR_INVALID_ARG, "dbr_offset must be non-decreasing");
      nnz = atomic->dbr_offset[rows];
      for (uint64_t r = 0; r < rows; ++r) {
        const uint32_t b = atomic->dbr_offset[r], e = atomic->dbr_offset[r + 1];
        for (uint32_t k = b; k < e; ++k) {
          if (atomic->dbr_line[k] >= L) return fail(nullptr, MC_ERR_INVALID_ARG, "dbr_line out of range");
          if (!(atomic->dbr_cdf[k] >= 0.0) || (k > b && atomic->dbr_cdf[k] < atomic->dbr_cdf[k - 1]))
            return fail(nullptr, MC_ERR_INVALID_ARG, "dbr_cdf must be non-decreasing within a row");
        }
        if (e > b && atomic->dbr_cdf[e - 1] != 1.0)
          return fail(nullptr, MC_ERR_INVALID_ARG, "each branching row must end at cdf == 1");
      }
      if (run->line_mode != MC_LINE_SCATTER) {
        for (uint32_t j = 0; j < L; ++j) {
          const uint64_t r = static_cast<uint64_t>(lines->ion[j]) * K + lines->upper[j];
          if (atomic->dbr_offset[r + 1] == atomic->dbr_offset[r])
            return fail(nullptr, MC_ERR_INVALID_ARG, "a line's upper level has an empty branching row");
        }
      }
      if (run->line_mode == MC_LINE_MACROATOM) {
        const uint32_t *jo = atomic->ma_jump_offset;
        if (jo[0] != 0) return fail(nullptr, MC_ERR_INVALID_ARG, "ma_jump_offset[0] must be 0");
        for (uint64_t r = 0; r < rows; ++r) {
          const double pj = atomic->ma_jump_p[r];
          if (!(pj >= 0.0 && pj < 1.0)) return fail(nullptr, MC_ERR_INVALID_ARG, "ma_jump_p must be in [0, 1)");
          if (jo[r + 1] < jo[r]) return fail(nullptr, MC_ERR_INVALID_ARG, "ma_jump_offset must be non-decreasing");
          if (pj > 0.0 && jo[r + 1] == jo[r])
            return fail(nullptr, MC_ERR_INVALID_ARG, "a level that jumps needs jump targets");
          for (uint32_t k = jo[r]; k < jo[r + 1]; ++k) {
            const int32_t t = atomic->ma_jump_target[k];
            if (t < 0 || static_cast<uint64_t>(t) >= rows ||
                atomic->dbr_offset[t + 1] == atomic->dbr_offset[t])
              return fail(nullptr, MC_ERR_INVALID_ARG, "a jump target must be a level with a branching row");
            if (!(atomic->ma_jump_cdf[k] >= 0.0) || (k > jo[r] && atomic->ma_jump_cdf[k] < atomic->ma_jump_cdf[k - 1]))
              return fail(nullptr, MC_ERR_INVALID_ARG, "ma_jump_cdf must be non-decreasing within a row");
          }
          if (jo[r + 1] > jo[r] && atomic->ma_jump_cdf[jo[r + 1] - 1] != 1.0)
            return fail(nullptr, MC_ERR_INVALID_ARG, "each jump row must end at cdf == 1");
        }
      }
    }
  }

  mc_model *m = new (std::nothrow) mc_model();
  if (!m) return fail(nullptr, MC_ERR_OOM, "host allocation failed");
  cudaGetDevice(&m->device);
  if (stream) {
    m->stream = static_cast<cudaStream_t>(stream);
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete m;
      return fail(nullptr, MC_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
    }
    m->own_stream = true;
  }
  if (alloc && alloc->alloc && alloc->free) {
    m->alloc = *alloc;
    m->has_alloc = true;
  }
  m->S = S; m->L = L; m->I = I; m->K = K; m->nnz = nnz;
  m->run = *run;
  if (m->run.max_segments == 0) m->run.max_segments = 1000000ull;
  if (!(m->run.delta_t > 0.0)) m->run.delta_t = 1.0;
  m->t_exp = geom->t_exp;
  m->has_atomic = atomic != nullptr;
  m->has_line_meta = meta;
  for (int i = 0; i < kNEv; ++i) cudaEventCreate(&m->ev[i]);

  auto bail = [&](mc_status code, const std::string &msg) {
    g_create_error = msg;
    // copies already enqueued must finish before a caller's allocator gets
    // its blocks back (the default stream-ordered free needs no wait)
    cudaStreamSynchronize(m->stream);
    free_all(m);
    cudaStreamSynchronize(m->stream);
    pinned_put(m->cancel_host);
    for (int i = 0; i < kNEv; ++i) cudaEventDestroy(m->ev[i]);
    if (m->own_stream) cudaStreamDestroy(m->stream);
    delete m;
    return code;
  };

  const size_t SL = static_cast<size_t>(S) * L;
  bool ok = alloc_n(m, &m->x_in, S) && alloc_n(m, &m->x_out, S) && alloc_n(m, &m->inv_x_in, S) &&
            alloc_n(m, &m->inv_x_out, S) && alloc_n(m, &m->kappa, S) && alloc_n(m, &m->inv_kappa, S) && alloc_n(m, &m->nu, L) &&
            (run->precision == MC_PRECISION_MIXED ? alloc_n(m, &m->tau32, SL) : alloc_n(m, &m->tau, SL)) &&
            alloc_n(m, &m->t_rad, S) && alloc_n(m, &m->w, S) &&
            alloc_n(m, &m->norm, S) && alloc_n(m, &m->j_est, S) && alloc_n(m, &m->nu_bar, S) &&
            alloc_n(m, &m->spectrum, static_cast<size_t>(run->spec_bins) + 2) &&
            alloc_n(m, &m->counters, static_cast<size_t>(kNCounterSlots)) &&
            alloc_n(m, &m->planck_cdf, static_cast<size_t>(kPlanckLmax) + 1);
  if (ok && run->j_blue) ok = alloc_n(m, &m->j_blue, SL);
  if (ok && run->precision == MC_PRECISION_MIXED)
    ok = alloc_n(m, &m->shell32, 4 * static_cast<size_t>(S)) && alloc_n(m, &m->est_fix, 2 * static_cast<size_t>(S));
  if (ok && meta) ok = alloc_n(m, &m->line_row, L) && alloc_n(m, &m->lev_l, L) && alloc_n(m, &m->lev_u, L);
  if (ok && atomic) {
    const size_t IK = static_cast<size_t>(I) * K;
    ok = alloc_n(m, &m->eps_erg, IK) && alloc_n(m, &m->g, IK) && alloc_n(m, &m->meta, IK) &&
         alloc_n(m, &m->n_ion, static_cast<size_t>(S) * I) && alloc_n(m, &m->pop, S * IK);
    if (ok && meta && lines->f) ok = alloc_n(m, &m->line_pref, L) && alloc_n(m, &m->line_gratio, L);
    if (ok && atomic->dbr_offset)
      ok = alloc_n(m, &m->dbr_offset, IK + 1) && alloc_n(m, &m->dbr_line, nnz) &&
           alloc_n(m, &m->dbr_cdf, nnz);
    if (ok && atomic->dbr_offset && meta && run->line_mode != MC_LINE_SCATTER)
      ok = alloc_n(m, &m->dbr_rec, nnz) && alloc_n(m, &m->dbr_bucket, nnz) &&
           alloc_n(m, &m->row_info, L);
  }
  if (ok) ok = alloc_n(m, &m->n_e, S);
  if (ok) {  // the stop request: one pinned host word the kernels can read
    void *d = nullptr;
    void *h = pinned_get(sizeof(uint32_t), true);
    ok = h != nullptr;
    if (ok) {
      m->cancel_host = static_cast<uint32_t *>(h);
      *static_cast<volatile uint32_t *>(m->cancel_host) = 0u;
      ok = cudaHostGetDevicePointer(&d, h, 0) == cudaSuccess;
      m->cancel_dev = static_cast<const uint32_t *>(d);
    }
  }
  if (ok && ion_mode != MC_ION_FIXED) {
    const size_t E = atomic->n_elements, J = atomic->n_stages;
    m->ion_mode = ion_mode;
    m->ion_E = static_cast<int32_t>(E);
    m->ion_J = static_cast<int32_t>(J);
    m->ion_delta = ion_mode == MC_ION_NEBULAR ? atomic->delta : 0.0;
    ok = alloc_n(m, &m->ion_of, E * J) && alloc_n(m, &m->chi_erg, E * (J - 1)) &&
         alloc_n(m, &m->zeta, E * (J - 1)) && alloc_n(m, &m->n_element, S * E) &&
         alloc_n(m, &m->ion_phi, S * E * (J - 1));
  }
  if (ok && run->record_packets) {
    const size_t n = run->max_packets;
    ok = alloc_n(m, &m->rec_status, n) && alloc_n(m, &m->rec_nu, n) && alloc_n(m, &m->rec_e, n) &&
         alloc_n(m, &m->rec_cnt, n * kNCounters);
  }
  if (!ok) return bail(MC_ERR_OOM, "device allocation failed");

  // Geometry in units of c t_exp (v/c = r/(c t_exp)); kappa' = sigma_T n_e c t_exp.
  std::vector<double> xi(S), xo(S), ixi(S), ixo(S), kap(S), ikap(S), norm(S);
  for (uint32_t s = 0; s < S; ++s) {
    xi[s] = geom->v_inner[s] / kC;
    xo[s] = geom->v_outer[s] / kC;
    ixi[s] = 1.0 / xi[s];
    ixo[s] = 1.0 / xo[s];
    kap[s] = ((kSigmaT * geom->n_e[s]) * kC) * geom->t_exp;
    ikap[s] = kap[s] > 0.0 ? 1.0 / kap[s] : 0.0;
    const double ri = geom->v_inner[s] * geom->t_exp, ro = geom->v_outer[s] * geom->t_exp;
    const double V = ((4.0 / 3.0) * kPi) * (ro * ro * ro - ri * ri * ri);
    norm[s] = (kC * geom->t_exp) / (((4.0 * kPi) * m->run.delta_t) * V);
  }
  m->host_norm = norm;
  m->host_x_in = xi;
  m->host_x_out = xo;
  m->r_inner = geom->v_inner[0] * geom->t_exp;
  // Planck series partial sums (90/pi^4) sum_{j<=l} j^-4 for the frequency sampler.
  std::vector<double> cdf(kPlanckLmax + 1, 0.0);
  {
    const double c = 90.0 / (kPi * kPi * kPi * kPi);
    double acc = 0.0;
    for (int l = 1; l <= kPlanckLmax; ++l) {
      const double dl = static_cast<double>(l);
      acc += 1.0 / (dl * dl * dl * dl);
      cdf[l] = c * acc;
    }
  }
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  chk(upload(m, m->x_in, xi.data(), S));
  chk(upload(m, m->x_out, xo.data(), S));
  chk(upload(m, m->inv_x_in, ixi.data(), S));
  chk(upload(m, m->inv_x_out, ixo.data(), S));
  chk(upload(m, m->kappa, kap.data(), S));
  chk(upload(m, m->inv_kappa, ikap.data(), S));
  chk(upload(m, m->n_e, geom->n_e, S));
  std::vector<float> sh32;
  if (m->shell32) {
    sh32.resize(4 * static_cast<size_t>(S));
    for (uint32_t s = 0; s < S; ++s) {
      const float fi = static_cast<float>(xi[s]), fo = static_cast<float>(xo[s]);
      sh32[s] = fi * fi;
      sh32[S + s] = fo * fo;
      sh32[2 * S + s] = static_cast<float>(kap[s]);
      sh32[3 * S + s] = kap[s] > 0.0 ? static_cast<float>(1.0 / kap[s]) : 0.0f;
    }
    chk(upload(m, m->shell32, sh32.data(), sh32.size()));
  }
  chk(upload(m, m->norm, norm.data(), S));
  chk(upload(m, m->nu, lines->nu, L));
  chk(upload(m, m->planck_cdf, cdf.data(), cdf.size()));
  if (atomic) {
    const size_t IK = static_cast<size_t>(I) * K;
    std::vector<double> eps(IK);
    for (size_t a = 0; a < IK; ++a) eps[a] = atomic->energy_ev[a] * kEv;
    chk(upload(m, m->eps_erg, eps.data(), IK));
    chk(upload(m, m->g, atomic->g, IK));
    chk(upload(m, m->meta, atomic->metastable, IK));
    if (atomic->n_ion) chk(upload(m, m->n_ion, atomic->n_ion, static_cast<size_t>(S) * I));
    else chk(cudaMemsetAsync(m->n_ion, 0, static_cast<size_t>(S) * I * sizeof(double), m->stream));
    if (m->ion_mode) {
      const size_t E = atomic->n_elements, EJ1 = E * (atomic->n_stages - 1);
      std::vector<double> chi(EJ1), zeta(EJ1, 0.0);
      for (size_t t = 0; t < EJ1; ++t) chi[t] = atomic->chi_ev[t] * kEv;
      if (atomic->zeta) zeta.assign(atomic->zeta, atomic->zeta + EJ1);
      chk(upload(m, m->ion_of, ion_of.data(), ion_of.size()));
      chk(upload(m, m->chi_erg, chi.data(), EJ1));
      chk(upload(m, m->zeta, zeta.data(), EJ1));
      chk(upload(m, m->n_element, atomic->n_element, static_cast<size_t>(S) * E));
    }
    if (atomic->dbr_offset) {
      chk(upload(m, m->dbr_offset, atomic->dbr_offset, IK + 1));
      chk(upload(m, m->dbr_line, atomic->dbr_line, nnz));
      chk(upload(m, m->dbr_cdf, atomic->dbr_cdf, nnz));
    }
  }
  if (e != cudaSuccess) return bail(MC_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
  if (meta) {
    // Line indices (and Eq. 12 per-line constants when f is given) are built
    // on the device from staged copies of the host arrays.
    int32_t *ion_d = nullptr, *lo_d = nullptr, *up_d = nullptr;
    double *f_d = nullptr;
    ok = alloc_n(m, &ion_d, L) && alloc_n(m, &lo_d, L) && alloc_n(m, &up_d, L);
    if (ok && lines->f && atomic) ok = alloc_n(m, &f_d, L);
    if (!ok) return bail(MC_ERR_OOM, "device allocation failed");
    chk(upload(m, ion_d, lines->ion, L));
    chk(upload(m, lo_d, lines->lower, L));
    chk(upload(m, up_d, lines->upper, L));
    if (f_d) chk(upload(m, f_d, lines->f, L));
    const int Kc = static_cast<int>(K > 0 ? K : 1);
    chk(launch_line_setup(static_cast<int>(L), Kc, m->nu, f_d, ion_d, lo_d, up_d, m->g, m->t_exp,
                          m->lev_l, m->lev_u, m->line_pref, m->line_gratio, m->line_row, m->stream));
    m->launches += 1;
    if (m->dbr_rec) {
      chk(launch_dbr_setup(static_cast<uint32_t>(nnz), I * K, L, Kc, m->dbr_offset, m->dbr_line,
                           m->dbr_cdf, m->nu, m->line_row, m->dbr_rec, m->dbr_bucket,
                           m->row_info, m->stream));
      m->launches += 2;
    }
    std::vector<MaRow> ma_rows;
    std::vector<MaJump> ma_jumps;
    if (run->line_mode == MC_LINE_MACROATOM) {
      // decision thresholds ceil(p 2^53): z = u 2^-53 < p exactly when u < thr
      const auto thr53 = [](double v) {
        return static_cast<unsigned long long>(std::ceil(v * 9007199254740992.0));
      };
      const uint64_t rows = static_cast<uint64_t>(I) * K;
      const uint32_t nj = atomic->ma_jump_offset[rows];
      ma_rows.resize(rows);
      ma_jumps.resize(nj > 0 ? nj : 1);
      for (uint64_t r = 0; r < rows; ++r) {
        MaRow &mr = ma_rows[r];
        mr.jump_thr = thr53(atomic->ma_jump_p[r]);
        mr.jump_begin = atomic->ma_jump_offset[r];
        mr.jump_len = atomic->ma_jump_offset[r + 1] - atomic->ma_jump_offset[r];
        mr.dbr_begin = atomic->dbr_offset[r];
        mr.dbr_len = atomic->dbr_offset[r + 1] - atomic->dbr_offset[r];
      }
      for (uint32_t k = 0; k < nj; ++k) {
        ma_jumps[k].thr = thr53(atomic->ma_jump_cdf[k]);
        ma_jumps[k].target = atomic->ma_jump_target[k];
        ma_jumps[k].pad = 0u;
      }
      if (!alloc_n(m, &m->ma_row, ma_rows.size()) || !alloc_n(m, &m->ma_jump, ma_jumps.size()))
        return bail(MC_ERR_OOM, "device allocation failed");
      chk(upload(m, m->ma_row, ma_rows.data(), ma_rows.size()));
      chk(upload(m, m->ma_jump, ma_jumps.data(), ma_jumps.size()));
    }
    // Host buffers of the staged copies must outlive the async copies.
    chk(cudaStreamSynchronize(m->stream));
    if (e != cudaSuccess) return bail(MC_ERR_CUDA, std::string("line setup: ") + cudaGetErrorString(e));
  }
  int bps = 0;
  e = transport_occupancy(run->line_mode, run->precision, run->j_blue != 0, run->record_packets != 0,
                          static_cast<int>(S), &bps);
  if (e != cudaSuccess || bps <= 0) return bail(MC_ERR_CUDA, "transport occupancy query failed");
  int nsm = 1;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device);
  m->grid = nsm * bps;
  e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return bail(MC_ERR_CUDA, std::string("create: ") + cudaGetErrorString(e));
  *out = m;
  return MC_OK;
}

mc_status mc_set_plasma(mc_model *m, const double *t_rad, const double *w, const double *tau) {
  if (!m) return MC_ERR_INVALID_ARG;
  const uint32_t S = m->S;
  std::vector<double> t(S, 1.0e4), ww(S);
  if (t_rad) {
    for (uint32_t s = 0; s < S; ++s) {
      if (!(t_rad[s] > 0.0) || !std::isfinite(t_rad[s])) return fail(m, MC_ERR_INVALID_ARG, "t_rad must be positive");
      t[s] = t_rad[s];
    }
  }
  if (w) {
    for (uint32_t s = 0; s < S; ++s) {
      if (!(w[s] >= 0.0) || !std::isfinite(w[s])) return fail(m, MC_ERR_INVALID_ARG, "w must be finite and >= 0");
      ww[s] = w[s];
    }
  } else {
    // Geometric dilution at the shell centre, Sect. 2.8.
    const std::vector<double> &vi = m->host_x_in, &vo = m->host_x_out;
    for (uint32_t s = 0; s < S; ++s) {
      const double rr = vi[0] / ((vi[s] + vo[s]) * 0.5);
      ww[s] = 0.5 * (1.0 - std::sqrt(1.0 - rr * rr));
    }
  }
  if (!tau && !(m->has_atomic && m->line_pref))
    return fail(m, MC_ERR_INVALID_ARG, "tau == NULL needs atomic data and oscillator strengths");
  cudaError_t e = upload(m, m->t_rad, t.data(), S);
  if (e == cudaSuccess) e = upload(m, m->w, ww.data(), S);
  if (tau) {
    const size_t SL = static_cast<size_t>(S) * m->L;
    for (size_t i = 0; i < SL; ++i)
      if (!std::isfinite(tau[i])) return fail(m, MC_ERR_INVALID_ARG, "tau must be finite");
    if (m->tau32) {
      // mixed precision keeps binary32 depths only
      std::vector<float> t32(SL);
      for (size_t i = 0; i < SL; ++i) t32[i] = static_cast<float>(tau[i]);
      if (e == cudaSuccess) e = upload(m, m->tau32, t32.data(), SL);
      if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    } else if (e == cudaSuccess) {
      e = upload(m, m->tau, tau, SL);
    }
    m->tau_given = true;
    m->tau_dirty = false;
  } else {
    m->tau_given = false;
    m->tau_dirty = true;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_fail(m, e, "set_plasma");
  m->plasma_set = true;
  return MC_OK;
}

mc_status mc_run_iteration(mc_model *m, uint64_t seed, uint32_t iteration, uint64_t n_packets,
                           double t_inner) {
  return mc_run_iteration_range(m, seed, iteration, 0, n_packets, n_packets, t_inner);
}

mc_status mc_run_iteration_range(mc_model *m, uint64_t seed, uint32_t iteration, uint64_t first_packet,
                                 uint64_t n_packets, uint64_t n_total, double t_inner) {
  if (!m) return MC_ERR_INVALID_ARG;
  if (!m->plasma_set) return fail(m, MC_ERR_NOT_READY, "mc_set_plasma has not been called");
  if (n_packets == 0 || n_total >= (1ull << 32) || first_packet + n_packets > n_total ||
      first_packet + n_packets < first_packet)
    return fail(m, MC_ERR_INVALID_ARG, "need 0 < n_packets, first + n_packets <= n_total < 2^32");
  if (m->run.record_packets && n_packets > m->run.max_packets)
    return fail(m, MC_ERR_INVALID_ARG, "n_packets exceeds max_packets of the packet records");
  if (!(t_inner > 0.0) || !std::isfinite(t_inner)) return fail(m, MC_ERR_INVALID_ARG, "t_inner must be positive");
  if (m->in_batch) return fail(m, MC_ERR_INVALID_ARG, "the model belongs to a batch; run it through the batch");
  mc_status st = model_prepare(m, m->stream, true);
  if (st != MC_OK) return st;
  TransportParams p{};
  model_fill_transport(m, p, seed, iteration, first_packet, n_packets, n_total, t_inner);
  cudaEventRecord(m->ev[kEvTransport0], m->stream);
  cudaError_t e = launch_transport(p, m->run.line_mode, m->run.precision, m->j_blue != nullptr,
                                   m->run.record_packets != 0, m->grid, transport_block_size(), m->stream);
  if (e != cudaSuccess) return cuda_fail(m, e, "transport kernel");
  cudaEventRecord(m->ev[kEvTransport1], m->stream);
  m->launches += 1;
  st = model_finish_transport(m, p, m->stream);
  if (st != MC_OK) return st;
  m->have_run = true;
  m->ran_update = false;
  m->last_n = n_packets;
  return MC_OK;
}

}  // extern "C"

namespace mcgpu {

mc_status model_fail(mc_model *m, mc_status code, const std::string &msg) { return fail(m, code, msg); }

mc_status model_prepare(mc_model *m, cudaStream_t st, bool events) {
  m->ran_plasma = false;
  if (!m->tau_given && m->tau_dirty) {
    if (events) cudaEventRecord(m->ev[kEvPlasma0], st);
    cudaStream_t own = m->stream;
    m->stream = st;
    const mc_status rc = recompute_tau(m);
    m->stream = own;
    if (rc != MC_OK) return rc;
    if (events) cudaEventRecord(m->ev[kEvPlasma1], st);
    m->ran_plasma = events;
  }
  cudaError_t e = launch_zero(m->j_est, m->S, m->nu_bar, m->S, m->spectrum, m->run.spec_bins + 2,
                              m->counters, kNCounterSlots, st);
  if (e != cudaSuccess) return cuda_fail(m, e, "zero");
  m->launches += 1;
  if (m->j_blue) {
    e = launch_zero_large(m->j_blue, static_cast<size_t>(m->S) * m->L, st);
    if (e != cudaSuccess) return cuda_fail(m, e, "zero j_blue");
    m->launches += 1;
  }
  if (m->est_fix) {
    e = cudaMemsetAsync(m->est_fix, 0, 2 * static_cast<size_t>(m->S) * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_fail(m, e, "zero fixed-point estimators");
  }
  if (m->spectrum_v && m->n_virtual) {
    e = cudaMemsetAsync(m->spectrum_v, 0, (static_cast<size_t>(m->run.spec_bins) + 2) * sizeof(double), st);
    if (e != cudaSuccess) return cuda_fail(m, e, "zero virtual-packet spectrum");
  }
  return MC_OK;
}

mc_status model_finish_transport(mc_model *m, const TransportParams &p, cudaStream_t st) {
  if (!m->est_fix) {
    if (!m->j_blue) return MC_OK;
    // binary64: J_blue cells hold sums of E_lab / nu_lab^2; times nu_j
    const cudaError_t e = launch_jblue_times_nu(m->j_blue, m->nu, static_cast<int>(m->S),
                                                static_cast<int>(m->L), st);
    if (e != cudaSuccess) return cuda_fail(m, e, "J_blue line factor");
    m->launches += 1;
    return MC_OK;
  }
  cudaError_t e = launch_est_from_fix(m->est_fix, static_cast<int>(m->S), p.e_cmf, p.nu_scale,
                                      m->j_est, m->nu_bar, st);
  if (e != cudaSuccess) return cuda_fail(m, e, "estimator conversion");
  m->launches += 1;
  if (m->j_blue) {
    e = launch_jblue_from_fix(m->j_blue, static_cast<size_t>(m->S) * m->L, p.e_cmf, p.inv_nu_ref, st);
    if (e != cudaSuccess) return cuda_fail(m, e, "J_blue conversion");
    m->launches += 1;
  }
  return MC_OK;
}

void model_fill_transport(const mc_model *m, TransportParams &p, uint64_t seed, uint32_t iteration,
                          uint64_t first_packet, uint64_t n_packets, uint64_t n_total, double t_inner) {
  p = TransportParams{};
  p.S = static_cast<int32_t>(m->S);
  p.L = static_cast<int32_t>(m->L);
  p.x_in = m->x_in; p.x_out = m->x_out; p.inv_x_in = m->inv_x_in; p.inv_x_out = m->inv_x_out;
  p.inv_kappa = m->inv_kappa; p.row_info = m->row_info; p.dbr_rec = m->dbr_rec;
  p.dbr_bucket = m->dbr_bucket;
  p.kappa = m->kappa;
  p.nu = m->nu; p.tau = m->tau; p.tau32 = m->tau32;
  p.line_row = m->line_row; p.dbr_offset = m->dbr_offset; p.dbr_line = m->dbr_line; p.dbr_cdf = m->dbr_cdf;
  p.j_est = m->j_est; p.nu_bar = m->nu_bar; p.j_blue = m->j_blue; p.spectrum = m->spectrum;
  p.ma_row = m->ma_row;
  p.ma_jump = m->ma_jump;
  p.n_virtual = static_cast<int32_t>(m->n_virtual);
  p.tau_v_max = m->tau_v_max;
  p.spectrum_v = m->n_virtual ? m->spectrum_v : nullptr;
  p.stats = m->counters;
  p.work_counter = m->counters + kNStats;
  p.flags = m->counters + kNStats + 1;
  p.spec_bins = static_cast<int32_t>(m->run.spec_bins);
  p.spec_lo = m->run.spec_nu_lo;
  p.spec_hi = m->run.spec_nu_hi;
  p.spec_dnu = (m->run.spec_nu_hi - m->run.spec_nu_lo) / static_cast<double>(m->run.spec_bins);
  p.n_packets = n_packets;
  p.first_packet = first_packet;
  p.iteration = iteration;
  p.key0 = static_cast<uint32_t>(seed);
  p.key1 = static_cast<uint32_t>(seed >> 32);
  // Eqs. 9-10: E = 4 pi r_i^2 sigma T^4 dt / N (comoving, equal for all packets).
  const double r_i = m->r_inner;
  const double lum = (((4.0 * kPi) * r_i) * r_i) * kSigmaSB * t_inner * t_inner * t_inner * t_inner;
  p.e_cmf = (lum * m->run.delta_t) / static_cast<double>(n_total);
  p.nu_scale = (kKB * t_inner) / kH;
  p.planck_cdf = m->planck_cdf;
  p.max_segments = m->run.max_segments;
  p.rec_status = m->rec_status; p.rec_nu = m->rec_nu; p.rec_e = m->rec_e; p.rec_cnt = m->rec_cnt;
  p.timeout_ns = m->run.timeout_ns;
  p.cancel = m->cancel_dev;
  p.shell32 = m->shell32;
  p.est_fix = m->est_fix;
  p.inv_nu_ref = 1.0 / p.nu_scale;
}

mc_status model_update(mc_model *m, cudaStream_t st, bool events) {
  UpdateParams u{};
  u.S = static_cast<int32_t>(m->S);
  u.j_est = m->j_est; u.nu_bar = m->nu_bar; u.norm = m->norm;
  u.t_rad = m->t_rad; u.w = m->w;
  u.c_tr = (kH / kKB) * ((kPi * kPi * kPi * kPi) / (360.0 * kZeta5));
  if (events) cudaEventRecord(m->ev[kEvUpdate0], st);
  cudaError_t e = launch_update(u, st);
  if (e != cudaSuccess) return cuda_fail(m, e, "update kernel");
  if (events) cudaEventRecord(m->ev[kEvUpdate1], st);
  m->launches += 1;
  m->ran_update = events;
  if (!m->tau_given) m->tau_dirty = true;
  return MC_OK;
}

}  // namespace mcgpu

extern "C" {

mc_status mc_update_radiation_field(mc_model *m, double *t_rad_out, double *w_out) {
  if (!m) return MC_ERR_INVALID_ARG;
  if (!m->have_run) return fail(m, MC_ERR_NOT_READY, "no Monte Carlo run to update from");
  mc_status st = model_update(m, m->stream, true);
  if (st != MC_OK) return st;
  if (!t_rad_out && !w_out) return MC_OK;  // stays asynchronous on the model's stream
  cudaError_t e = cudaSuccess;
  if (t_rad_out) e = cudaMemcpyAsync(t_rad_out, m->t_rad, m->S * sizeof(double), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess && w_out) e = cudaMemcpyAsync(w_out, m->w, m->S * sizeof(double), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_fail(m, e, "update readout");
  return MC_OK;
}

mc_status mc_device_estimators(mc_model *m, mc_estimator_views *out) {
  if (!m || !out) return MC_ERR_INVALID_ARG;
  out->j_est = m->j_est;
  out->nu_bar = m->nu_bar;
  out->j_blue = m->j_blue;
  out->spectrum = m->spectrum;
  out->n_shells = m->S;
  out->n_lines = m->L;
  out->spec_bins = m->run.spec_bins;
  out->stream = m->stream;
  return MC_OK;
}

mc_status mc_read_estimators(mc_model *m, double *j_est, double *nu_bar, double *j_blue, double *norm) {
  if (!m) return MC_ERR_INVALID_ARG;
  if (!m->have_run) return fail(m, MC_ERR_NOT_READY, "no run yet");
  if (j_blue && !m->j_blue) return fail(m, MC_ERR_UNSUPPORTED, "J_blue estimators are off for this model");
  cudaError_t e = cudaSuccess;
  if (j_est) e = cudaMemcpyAsync(j_est, m->j_est, m->S * sizeof(double), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess && nu_bar)
    e = cudaMemcpyAsync(nu_bar, m->nu_bar, m->S * sizeof(double), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess && j_blue)
    e = cudaMemcpyAsync(j_blue, m->j_blue, static_cast<size_t>(m->S) * m->L * sizeof(double),
                        cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_fail(m, e, "read estimators");
  if (norm) std::memcpy(norm, m->host_norm.data(), m->S * sizeof(double));
  unsigned long long flag = 0;
  cudaMemcpy(&flag, m->counters + kNStats + 1, sizeof(flag), cudaMemcpyDeviceToHost);
  if (flag) return fail(m, MC_ERR_TIMEOUT, stop_message(flag));
  return MC_OK;
}

mc_status mc_read_spectrum(mc_model *m, double *spectrum, mc_packet_stats *stats) {
  if (!m) return MC_ERR_INVALID_ARG;
  if (!m->have_run) return fail(m, MC_ERR_NOT_READY, "no run yet");
  unsigned long long c[kNCounterSlots];
  cudaError_t e = cudaSuccess;
  if (spectrum)
    e = cudaMemcpyAsync(spectrum, m->spectrum, (m->run.spec_bins + 2) * sizeof(double),
                        cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c, m->counters, sizeof(c), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_fail(m, e, "read spectrum");
  if (stats) {
    stats->packets = m->last_n;
    stats->escaped = c[kStEscaped];
    stats->reabsorbed = c[kStReabsorbed];
    stats->capped = c[kStCapped];
    stats->segments = c[kStSegments];
    stats->line_checks = c[kStLineChecks];
    stats->resonances = c[kStResonances];
    stats->line_interactions = c[kStLineInteractions];
    stats->e_scatters = c[kStEScatters];
    stats->shell_crossings = c[kStShellCrossings];
  }
  if (c[kNStats + 1]) return fail(m, MC_ERR_TIMEOUT, stop_message(c[kNStats + 1]));
  return c[kStCapped] ? MC_WARN_CAPPED : MC_OK;
}

mc_status mc_t_inner_from_luminosity(const mc_model *m, double l_outer, double *t_inner) {
  if (!m || !t_inner || !(l_outer > 0.0) || !std::isfinite(l_outer)) return MC_ERR_INVALID_ARG;
  const double r_i = m->r_inner;
  *t_inner = std::sqrt(std::sqrt(l_outer / ((((4.0 * kPi) * r_i) * r_i) * kSigmaSB)));
  return MC_OK;
}

mc_status mc_emitted_luminosity(mc_model *m, double *l_emitted) {
  if (!m || !l_emitted) return MC_ERR_INVALID_ARG;
  if (!m->have_run) return fail(m, MC_ERR_NOT_READY, "no run yet");
  std::vector<double> sp(static_cast<size_t>(m->run.spec_bins) + 2);
  cudaError_t e = cudaMemcpyAsync(sp.data(), m->spectrum, sp.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                  m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_fail(m, e, "read spectrum");
  double s = 0.0;
  for (double v : sp) s += v;
  *l_emitted = s / m->run.delta_t;
  return MC_OK;
}

double mc_t_inner_update(double t_inner, double l_requested, double l_emitted) {
  if (!(l_emitted > 0.0)) return t_inner;
  return t_inner * std::sqrt(std::sqrt(l_requested / l_emitted));
}

mc_status mc_set_virtual_packets(mc_model *m, uint32_t n_virtual, double tau_v_max) {
  if (!m) return MC_ERR_INVALID_ARG;
  if (m->run.precision != MC_PRECISION_FP64)
    return fail(m, MC_ERR_UNSUPPORTED, "virtual packets run in the binary64 kernel");
  if (n_virtual > 1024) return fail(m, MC_ERR_INVALID_ARG, "at most 1024 virtual packets per launch");
  if (!(tau_v_max >= 0.0) || !std::isfinite(tau_v_max))
    return fail(m, MC_ERR_INVALID_ARG, "tau_v_max must be finite and >= 0");
  if (n_virtual && !m->spectrum_v) {
    if (!alloc_n(m, &m->spectrum_v, static_cast<size_t>(m->run.spec_bins) + 2))
      return fail(m, MC_ERR_OOM, "device allocation failed");
  }
  m->n_virtual = n_virtual;
  m->tau_v_max = tau_v_max;
  return MC_OK;
}

mc_status mc_read_virtual_spectrum(mc_model *m, double *spectrum_v) {
  if (!m || !spectrum_v) return MC_ERR_INVALID_ARG;
  if (!m->have_run) return fail(m, MC_ERR_NOT_READY, "no run yet");
  if (!m->spectrum_v || !m->n_virtual) return fail(m, MC_ERR_NOT_READY, "virtual packets are off");
  cudaError_t e = cudaMemcpyAsync(spectrum_v, m->spectrum_v, (m->run.spec_bins + 2) * sizeof(double),
                                  cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_fail(m, e, "read virtual spectrum");
  return MC_OK;
}

mc_status mc_read_packets(mc_model *m, uint64_t first, uint64_t count, int32_t *status, double *nu,
                          double *energy, uint64_t *counters) {
  if (!m) return MC_ERR_INVALID_ARG;
  if (!m->rec_status) return fail(m, MC_ERR_UNSUPPORTED, "packet records are off for this model");
  if (!m->have_run) return fail(m, MC_ERR_NOT_READY, "no run yet");
  if (first + count > m->last_n || first + count < first) return fail(m, MC_ERR_INVALID_ARG, "packet range out of bounds");
  cudaError_t e = cudaSuccess;
  if (status) e = cudaMemcpyAsync(status, m->rec_status + first, count * sizeof(int32_t), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess && nu) e = cudaMemcpyAsync(nu, m->rec_nu + first, count * sizeof(double), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess && energy)
    e = cudaMemcpyAsync(energy, m->rec_e + first, count * sizeof(double), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess && counters)
    e = cudaMemcpyAsync(counters, m->rec_cnt + first * kNCounters, count * kNCounters * sizeof(uint64_t),
                        cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_fail(m, e, "read packets");
  return MC_OK;
}

mc_status mc_read_plasma(mc_model *m, double *t_rad, double *w, double *tau) {
  if (!m) return MC_ERR_INVALID_ARG;
  if (!m->plasma_set) return fail(m, MC_ERR_NOT_READY, "mc_set_plasma has not been called");
  if (tau && !m->tau_given && m->tau_dirty) {
    mc_status st = recompute_tau(m);
    if (st != MC_OK) return st;
  }
  cudaError_t e = cudaSuccess;
  if (t_rad) e = cudaMemcpyAsync(t_rad, m->t_rad, m->S * sizeof(double), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess && w) e = cudaMemcpyAsync(w, m->w, m->S * sizeof(double), cudaMemcpyDeviceToHost, m->stream);
  const size_t SL = static_cast<size_t>(m->S) * m->L;
  std::vector<float> t32;
  if (e == cudaSuccess && tau) {
    if (m->tau32) {
      t32.resize(SL);
      e = cudaMemcpyAsync(t32.data(), m->tau32, SL * sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    } else {
      e = cudaMemcpyAsync(tau, m->tau, SL * sizeof(double), cudaMemcpyDeviceToHost, m->stream);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_fail(m, e, "read plasma");
  if (tau && m->tau32)
    for (size_t i = 0; i < SL; ++i) tau[i] = static_cast<double>(t32[i]);
  return MC_OK;
}

mc_status mc_read_ionization(mc_model *m, double *n_e, double *n_ion) {
  if (!m) return MC_ERR_INVALID_ARG;
  if (!m->plasma_set) return fail(m, MC_ERR_NOT_READY, "mc_set_plasma has not been called");
  if (n_ion && !m->n_ion) return fail(m, MC_ERR_INVALID_ARG, "no atomic data: no ion densities");
  if (m->ion_mode && !m->tau_given && m->tau_dirty) {
    mc_status st = recompute_tau(m);
    if (st != MC_OK) return st;
  }
  cudaError_t e = cudaSuccess;
  if (n_e) e = cudaMemcpyAsync(n_e, m->n_e, m->S * sizeof(double), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess && n_ion)
    e = cudaMemcpyAsync(n_ion, m->n_ion, static_cast<size_t>(m->S) * m->I * sizeof(double),
                        cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_fail(m, e, "read ionization");
  return MC_OK;
}

mc_status mc_read_timing(mc_model *m, float *ms) {
  if (!m || !ms) return MC_ERR_INVALID_ARG;
  if (!m->have_run) return fail(m, MC_ERR_NOT_READY, "no run yet");
  cudaError_t e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_fail(m, e, "timing");
  ms[0] = ms[1] = ms[2] = 0.0f;
  if (m->ran_plasma) cudaEventElapsedTime(&ms[0], m->ev[kEvPlasma0], m->ev[kEvPlasma1]);
  cudaEventElapsedTime(&ms[1], m->ev[kEvTransport0], m->ev[kEvTransport1]);
  if (m->ran_update) cudaEventElapsedTime(&ms[2], m->ev[kEvUpdate0], m->ev[kEvUpdate1]);
  return MC_OK;
}

mc_status mc_read_transport_phases(mc_model *m, float *ms) {
  if (!m || !ms) return MC_ERR_INVALID_ARG;
  if (!m->have_run) return fail(m, MC_ERR_NOT_READY, "no run yet");
  unsigned long long f[3];
  cudaError_t e = cudaMemcpyAsync(f, m->counters + kNStats + 2, sizeof(f), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_fail(m, e, "phases");
  const unsigned long long empty = f[0], done = f[1], start = f[2];
  ms[0] = (empty > start) ? static_cast<float>((empty - start) * 1e-6) : 0.0f;
  ms[1] = (done > empty && empty) ? static_cast<float>((done - empty) * 1e-6) : 0.0f;
  return MC_OK;
}

mc_status mc_launch_count(const mc_model *m, uint64_t *count) {
  if (!m || !count) return MC_ERR_INVALID_ARG;
  *count = m->launches;
  return MC_OK;
}

mc_status mc_synchronize(mc_model *m) {
  if (!m) return MC_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_fail(m, e, "synchronize");
  return MC_OK;
}

void mc_model_destroy(mc_model *m) {
  if (!m) return;
  cudaStreamSynchronize(m->stream);
  free_all(m);
  cudaStreamSynchronize(m->stream);
  pinned_put(m->cancel_host);
  for (int i = 0; i < kNEv; ++i) cudaEventDestroy(m->ev[i]);
  if (m->own_stream) cudaStreamDestroy(m->stream);
  delete m;
}

mc_status mc_cancel(mc_model *m, int32_t stop) {
  if (!m || (stop != 0 && stop != 1)) return MC_ERR_INVALID_ARG;
  *static_cast<volatile uint32_t *>(m->cancel_host) = static_cast<uint32_t>(stop);
  return MC_OK;
}

}  // extern "C"
