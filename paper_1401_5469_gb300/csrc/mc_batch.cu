// Batched Monte Carlo iterations: many ejecta models of uneven size advanced
// by one persistent transport launch per iteration, the whole iteration
// (Sobolev depths, estimator zeroing, transport, radiation-field update of
// every model) replayed as one captured CUDA graph.
//
// Each model keeps its own device arrays; the batch owns only the per-model
// transport parameter table, the packet prefix sums and a work counter.  The
// models' results are read with the single-model mc_read_* calls.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/mc_transport.h"
#include "mc_internal.h"
#include "mc_model_internal.h"

using namespace mcgpu;

namespace mcgpu {
void set_create_error(const std::string &msg);
}

struct mc_batch {
  std::vector<mc_model *> models;  // in launch order (largest packet count first)
  std::vector<uint32_t> order;     // launch position -> caller's index
  cudaStream_t stream = nullptr;   // the batch's own stream (graph capture)
  std::vector<cudaStream_t> user;  // the models' distinct streams
  int line_mode = 0;
  bool j_blue = false, record = false;
  int nsm = 1;
  int max_bps[3] = {0, 0, 0};      // resident blocks per SM at 64, 128, 256 threads
  uint32_t block = 128, bps_req = 0, order_policy = MC_ORDER_PACKETS;
  int grid = 0;
  TransportParams *d_params = nullptr, *h_params = nullptr;  // device table, pinned host staging
  unsigned long long *d_prefix = nullptr, *h_prefix = nullptr;
  unsigned long long *d_counters = nullptr;  // work counter, flags (kNCounterSlots)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<int> graph_shape;    // per model: 1 if its Sobolev depths were recomputed
  std::vector<uint32_t> graph_order;  // launch order captured in the graph
  std::vector<uint64_t> graph_np;     // per-model packets (packet energy is baked into the graph)
  std::vector<double> graph_tin;      // per-model T_inner
  bool graph_update = false;
  uint64_t graph_total = 0;
  bool use_graph = true;           // mc_batch_capture_graph
  uint64_t iterations = 0;         // batched iterations enqueued (graph or direct)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, t0 = nullptr, t1 = nullptr;
  uint64_t launches = 0, graph_launches = 0;
  std::string err;
};

namespace {

mc_status bfail(mc_batch *b, mc_status code, const std::string &msg) {
  if (b) b->err = msg;
  else set_create_error(msg);
  return code;
}

mc_status bcuda(mc_batch *b, cudaError_t e, const char *what) {
  return bfail(b, MC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int block_slot(uint32_t block) { return block == 64 ? 0 : block == 128 ? 1 : block == 256 ? 2 : -1; }

// Resident blocks per SM used for the current block size.
int resolved_bps(const mc_batch *b) {
  const int most = b->max_bps[block_slot(b->block)];
  return b->bps_req == 0 ? most : std::min<int>(most, static_cast<int>(b->bps_req));
}

void drop_graph(mc_batch *b) {
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
}

// Enqueue one iteration of every model on the batch stream (`capturing`:
// inside a stream capture, so the timing events become external event nodes).
mc_status enqueue_iteration(mc_batch *b, int update, bool capturing) {
  const unsigned ev_flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  for (mc_model *m : b->models) {
    const mc_status rc = model_prepare(m, b->stream, false);
    if (rc != MC_OK) return bfail(b, rc, m->err);
  }
  cudaError_t e = cudaMemsetAsync(b->d_counters, 0, kNCounterSlots * sizeof(unsigned long long), b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_params, b->h_params, b->models.size() * sizeof(TransportParams),
                        cudaMemcpyHostToDevice, b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "batch staging");
  TransportParams p{};
  p.batch = b->d_params;
  p.batch_prefix = b->d_prefix;
  p.n_models = static_cast<int32_t>(b->models.size());
  p.n_packets = b->h_prefix[b->models.size()];
  p.work_counter = b->d_counters;
  p.flags = b->d_counters + 1;
  e = cudaEventRecordWithFlags(b->t0, b->stream, ev_flags);
  if (e == cudaSuccess) e = launch_transport_batch(p, b->line_mode, b->j_blue, b->record, b->grid,
                                                    static_cast<int>(b->block), b->stream);
  if (e == cudaSuccess) e = cudaEventRecordWithFlags(b->t1, b->stream, ev_flags);
  if (e != cudaSuccess) return bcuda(b, e, "batched transport");
  b->launches += 1;
  for (size_t k = 0; k < b->models.size(); ++k) {
    const mc_status rc = model_finish_transport(b->models[k], b->h_params[k], b->stream);
    if (rc != MC_OK) return bfail(b, rc, b->models[k]->err);
  }
  if (update) {
    for (mc_model *m : b->models) {
      const mc_status rc = model_update(m, b->stream, false);
      if (rc != MC_OK) return bfail(b, rc, m->err);
    }
  }
  return MC_OK;
}

}  // namespace

extern "C" {

mc_status mc_batch_create(mc_model *const *models, uint32_t n_models, mc_batch **out) {
  if (!out) return bfail(nullptr, MC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!models || n_models == 0) return bfail(nullptr, MC_ERR_INVALID_ARG, "need at least one model");
  if (n_models > 4096) return bfail(nullptr, MC_ERR_INVALID_ARG, "at most 4096 models per batch");
  const mc_model *m0 = models[0];
  for (uint32_t i = 0; i < n_models; ++i) {
    const mc_model *m = models[i];
    if (!m) return bfail(nullptr, MC_ERR_INVALID_ARG, "NULL model");
    if (m->in_batch) return bfail(nullptr, MC_ERR_INVALID_ARG, "a model already belongs to a batch");
    if (m->run.precision != MC_PRECISION_MIXED)
      return bfail(nullptr, MC_ERR_UNSUPPORTED, "batched launches use mixed-precision models");
    if (m->device != m0->device || m->run.line_mode != m0->run.line_mode ||
        (m->j_blue != nullptr) != (m0->j_blue != nullptr) || m->run.record_packets != m0->run.record_packets)
      return bfail(nullptr, MC_ERR_INVALID_ARG, "batched models need one device, line mode, J_blue and record setting");
    for (uint32_t k = 0; k < i; ++k)
      if (models[k] == m) return bfail(nullptr, MC_ERR_INVALID_ARG, "a model appears twice");
  }
  mc_batch *b = new (std::nothrow) mc_batch();
  if (!b) return bfail(nullptr, MC_ERR_OOM, "host allocation failed");
  for (uint32_t i = 0; i < n_models; ++i)
    if (std::find(b->user.begin(), b->user.end(), models[i]->stream) == b->user.end())
      b->user.push_back(models[i]->stream);
  b->line_mode = m0->run.line_mode;
  b->j_blue = m0->j_blue != nullptr;
  b->record = m0->run.record_packets != 0;
  b->order.resize(n_models);
  std::iota(b->order.begin(), b->order.end(), 0u);
  for (uint32_t i = 0; i < n_models; ++i) b->models.push_back(models[i]);
  // Stream-ordered device buffers and cached pinned host buffers: creating or
  // destroying a batch does not synchronise the device, so batches of other
  // models keep running on their own streams meanwhile.
  cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMallocAsync(&b->d_params, n_models * sizeof(TransportParams), b->stream);
  if (e == cudaSuccess) e = cudaMallocAsync(&b->d_prefix, (n_models + 1) * sizeof(unsigned long long), b->stream);
  if (e == cudaSuccess) e = cudaMallocAsync(&b->d_counters, kNCounterSlots * sizeof(unsigned long long), b->stream);
  if (e == cudaSuccess) {
    b->h_params = static_cast<TransportParams *>(pinned_get(n_models * sizeof(TransportParams), false));
    b->h_prefix = static_cast<unsigned long long *>(pinned_get((n_models + 1) * sizeof(unsigned long long), false));
    if (!b->h_params || !b->h_prefix) e = cudaErrorMemoryAllocation;
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreate(&b->t0);
  if (e == cudaSuccess) e = cudaEventCreate(&b->t1);
  const int blocks[3] = {64, 128, 256};
  for (int k = 0; k < 3 && e == cudaSuccess; ++k)
    e = batch_occupancy(b->line_mode, b->j_blue, b->record, static_cast<int>(n_models), blocks[k],
                        &b->max_bps[k]);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, m0->device);
  if (e != cudaSuccess || b->max_bps[0] <= 0 || b->max_bps[1] <= 0 || b->max_bps[2] <= 0) {
    mc_batch_destroy(b);
    return bfail(nullptr, MC_ERR_CUDA, std::string("batch create: ") + cudaGetErrorString(e));
  }
  b->grid = b->nsm * resolved_bps(b);
  for (mc_model *m : b->models) m->in_batch = true;
  *out = b;
  return MC_OK;
}

mc_status mc_batch_run_iteration(mc_batch *b, const uint64_t *seeds, const uint32_t *iterations,
                                 const uint64_t *n_packets, const double *t_inner, int32_t update) {
  if (!b || !seeds || !iterations || !n_packets || !t_inner) return MC_ERR_INVALID_ARG;
  const size_t n = b->models.size();
  // the previous iteration reads the pinned parameter table when it starts;
  // wait until it has been copied before overwriting it
  if (b->iterations) {
    const cudaError_t ew = cudaEventSynchronize(b->t0);
    if (ew != cudaSuccess) return bcuda(b, ew, "previous iteration");
  }
  // queue order (MC_ORDER_PACKETS by default: largest packet count first, so
  // the longest walks start first)
  std::vector<uint32_t> order(n);
  std::iota(order.begin(), order.end(), 0u);
  std::vector<mc_model *> by_caller(n);
  for (size_t k = 0; k < n; ++k)
    by_caller[b->order[k]] = b->models[k];
  if (b->order_policy == MC_ORDER_PACKETS) {
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t a, uint32_t c) { return n_packets[a] > n_packets[c]; });
  } else if (b->order_policy == MC_ORDER_WORK) {
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t c) {
      return static_cast<double>(n_packets[a]) * by_caller[a]->L >
             static_cast<double>(n_packets[c]) * by_caller[c]->L;
    });
  }
  std::vector<mc_model *> launch_models(n);
  for (size_t k = 0; k < n; ++k) {
    const uint32_t i = order[k];
    mc_model *m = by_caller[i];
    launch_models[k] = m;
    if (!m->plasma_set) return bfail(b, MC_ERR_NOT_READY, "a model has no plasma state");
    if (n_packets[i] == 0 || n_packets[i] >= (1ull << 32))
      return bfail(b, MC_ERR_INVALID_ARG, "need 0 < n_packets < 2^32 for every model");
    if (m->run.record_packets && n_packets[i] > m->run.max_packets)
      return bfail(b, MC_ERR_INVALID_ARG, "n_packets exceeds a model's packet records");
    if (!(t_inner[i] > 0.0) || !std::isfinite(t_inner[i])) return bfail(b, MC_ERR_INVALID_ARG, "t_inner must be positive");
  }
  b->models = launch_models;
  b->order = order;
  b->h_prefix[0] = 0;
  std::vector<int> shape(n);
  for (size_t k = 0; k < n; ++k) {
    const uint32_t i = order[k];
    mc_model *m = b->models[k];
    model_fill_transport(m, b->h_params[k], seeds[i], iterations[i], 0, n_packets[i], n_packets[i], t_inner[i]);
    b->h_prefix[k + 1] = b->h_prefix[k] + n_packets[i];
    shape[k] = (!m->tau_given && m->tau_dirty) ? 1 : 0;
  }
  // the prefix table is constant across graph replays of the same shape
  cudaError_t e = cudaMemcpyAsync(b->d_prefix, b->h_prefix, (n + 1) * sizeof(unsigned long long),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "prefix upload");
  // order the batch after the models' own stream
  for (cudaStream_t us : b->user) {
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_in, us);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_in, 0);
  }
  if (e != cudaSuccess) return bcuda(b, e, "stream order");

  const std::vector<uint64_t> np(n_packets, n_packets + n);
  const std::vector<double> tin(t_inner, t_inner + n);
  if (!b->use_graph) {
    const mc_status rc = enqueue_iteration(b, update, false);
    if (rc != MC_OK) return rc;
  } else {
    const bool reuse = b->exec && b->graph_shape == shape && b->graph_order == order &&
                       b->graph_np == np && b->graph_tin == tin &&
                       b->graph_update == (update != 0) &&
                       b->graph_total == b->h_prefix[n];
    if (!reuse) {
      drop_graph(b);
      e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return bcuda(b, e, "begin capture");
      const mc_status rc = enqueue_iteration(b, update, true);
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(b->stream, &g);
      if (rc != MC_OK) { if (g) cudaGraphDestroy(g); return rc; }
      if (e != cudaSuccess) return bcuda(b, e, "end capture");
      b->graph = g;
      e = cudaGraphInstantiate(&b->exec, g, 0);
      if (e != cudaSuccess) return bcuda(b, e, "graph instantiate");
      b->graph_shape = shape;
      b->graph_order = order;
      b->graph_np = np;
      b->graph_tin = tin;
      b->graph_update = update != 0;
      b->graph_total = b->h_prefix[n];
    } else {
      // the captured steps mark the same state; keep the host-side flags in step
      for (mc_model *m : b->models) {
        m->ran_plasma = false;
        if (!m->tau_given && m->tau_dirty) m->tau_dirty = false;
      }
    }
    e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "graph launch");
    b->graph_launches += 1;
  }
  b->iterations += 1;
  for (size_t k = 0; k < n; ++k) {
    mc_model *m = b->models[k];
    m->have_run = true;
    m->last_n = n_packets[order[k]];
    if (update && !m->tau_given) m->tau_dirty = true;
  }
  e = cudaEventRecord(b->ev_out, b->stream);
  for (cudaStream_t us : b->user)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(us, b->ev_out, 0);
  if (e != cudaSuccess) return bcuda(b, e, "stream order");
  return MC_OK;
}

mc_status mc_batch_synchronize(mc_batch *b) {
  if (!b) return MC_ERR_INVALID_ARG;
  const cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "batch synchronize");
  return MC_OK;
}

mc_status mc_batch_read_timing(mc_batch *b, float *ms) {
  if (!b || !ms) return MC_ERR_INVALID_ARG;
  if (!b->iterations) return bfail(b, MC_ERR_NOT_READY, "no batched iteration yet");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, b->t0, b->t1);
  if (e != cudaSuccess) return bcuda(b, e, "batch timing");
  return MC_OK;
}

mc_status mc_batch_read_phases(mc_batch *b, float *ms) {
  if (!b || !ms) return MC_ERR_INVALID_ARG;
  if (!b->iterations) return bfail(b, MC_ERR_NOT_READY, "no batched iteration yet");
  unsigned long long f[3];  // flags [1] queue empty, [2] last warp done, [3] first warp start (ns)
  cudaError_t e = cudaMemcpyAsync(f, b->d_counters + 2, sizeof(f), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "batch phases");
  const unsigned long long empty = f[0], done = f[1], start = f[2];
  ms[0] = (empty > start) ? static_cast<float>((empty - start) * 1e-6) : 0.0f;
  ms[1] = (done > empty && empty) ? static_cast<float>((done - empty) * 1e-6) : 0.0f;
  return MC_OK;
}

const char *mc_batch_last_error_message(const mc_batch *b) { return b ? b->err.c_str() : ""; }

mc_status mc_batch_set_launch(mc_batch *b, const mc_batch_launch *launch) {
  if (!b || !launch) return MC_ERR_INVALID_ARG;
  const uint32_t block = launch->block == 0 ? 128u : launch->block;
  if (block_slot(block) < 0) return bfail(b, MC_ERR_INVALID_ARG, "block must be 64, 128 or 256");
  if (launch->order > MC_ORDER_GIVEN) return bfail(b, MC_ERR_INVALID_ARG, "unknown queue order");
  if (b->iterations) {  // the iteration in flight reads the parameter table
    const cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "set launch");
  }
  b->block = block;
  b->bps_req = launch->blocks_per_sm;
  b->order_policy = launch->order;
  b->grid = b->nsm * resolved_bps(b);
  drop_graph(b);
  return MC_OK;
}

mc_status mc_batch_capture_graph(mc_batch *b, int32_t enable) {
  if (!b || (enable != 0 && enable != 1)) return MC_ERR_INVALID_ARG;
  if (b->iterations) {  // the iteration in flight may still be the graph
    const cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "capture graph");
  }
  b->use_graph = enable == 1;
  drop_graph(b);
  return MC_OK;
}

mc_status mc_batch_get_launch(const mc_batch *b, mc_batch_launch *launch) {
  if (!b || !launch) return MC_ERR_INVALID_ARG;
  launch->block = b->block;
  launch->blocks_per_sm = static_cast<uint32_t>(resolved_bps(b));
  launch->order = b->order_policy;
  return MC_OK;
}

mc_status mc_batch_autotune(mc_batch *b, const uint64_t *seeds, const uint32_t *iterations,
                            const uint64_t *n_packets, const double *t_inner,
                            mc_batch_launch *best, float *best_ms, uint32_t *n_trials) {
  if (!b) return MC_ERR_INVALID_ARG;
  uint32_t trials = 0;
  // one transport-only iteration with shape c; its device time in *ms
  auto trial = [&](const mc_batch_launch &c, float *ms) -> mc_status {
    mc_status rc = mc_batch_set_launch(b, &c);
    if (rc == MC_OK) rc = mc_batch_run_iteration(b, seeds, iterations, n_packets, t_inner, 0);
    if (rc == MC_OK) rc = mc_batch_read_timing(b, ms);
    ++trials;
    return rc;
  };
  mc_batch_launch cur{b->block, 0u, b->order_policy};
  float cur_ms = 0.0f;
  // the first trial also absorbs one-time costs (stale Sobolev depths, first
  // capture); time the starting shape again so that it competes fairly
  mc_status rc = trial(cur, &cur_ms);
  if (rc == MC_OK) rc = trial(cur, &cur_ms);
  auto consider = [&](const mc_batch_launch &c) -> mc_status {
    float ms = 0.0f;
    const mc_status r = trial(c, &ms);
    if (r == MC_OK && ms < cur_ms) { cur = c; cur_ms = ms; }
    return r;
  };
  for (uint32_t o = MC_ORDER_PACKETS; o <= MC_ORDER_WORK && rc == MC_OK; ++o)
    if (o != cur.order) rc = consider(mc_batch_launch{cur.block, cur.blocks_per_sm, o});
  const uint32_t blocks[3] = {64u, 128u, 256u};
  const uint32_t start_block = cur.block;
  for (uint32_t bl : blocks)
    if (rc == MC_OK && bl != start_block) rc = consider(mc_batch_launch{bl, 0u, cur.order});
  const int most = b->max_bps[block_slot(cur.block)];
  const uint32_t start_bps = cur.blocks_per_sm;
  for (int k = 1; k < most && rc == MC_OK; ++k)  // 0 (= most) was timed above
    if (static_cast<uint32_t>(k) != start_bps) rc = consider(mc_batch_launch{cur.block, static_cast<uint32_t>(k), cur.order});
  if (rc == MC_OK) rc = mc_batch_set_launch(b, &cur);
  if (rc != MC_OK) return rc;
  if (best) mc_batch_get_launch(b, best);
  if (best_ms) *best_ms = cur_ms;
  if (n_trials) *n_trials = trials;
  return MC_OK;
}

void mc_batch_destroy(mc_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (mc_model *m : b->models) m->in_batch = false;
  drop_graph(b);
  if (b->d_params) cudaFreeAsync(b->d_params, b->stream);
  if (b->d_prefix) cudaFreeAsync(b->d_prefix, b->stream);
  if (b->d_counters) cudaFreeAsync(b->d_counters, b->stream);
  pinned_put(b->h_params);
  pinned_put(b->h_prefix);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->t0) cudaEventDestroy(b->t0);
  if (b->t1) cudaEventDestroy(b->t1);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // extern "C"
