// snn_serve.cu -- continuous batching of independent simulation requests
// (the serving entry points of include/snn.h).
//
// Requests queue in arrival order.  A builder thread admits the head request
// when its estimated device footprint fits the budget and builds its net
// (store construction on the net's own stream) while the admitted nets keep
// running on the server's stream.  A step advances every running net by its
// next interval with one batched update launch and one batched tiled-delivery
// launch for all nets (k_update_batch / k_deliver_tiled_batch): a device table
// holds each net's view, update constants and step count, and a block map
// sends every CTA to its (net, block) or (net, tile).  While the batch is
// unchanged a step may run several intervals, captured as one CUDA graph; a
// small autotuner picks that number from measured GPU time per interval.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "snn_net.cuh"

namespace {

int sfail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int sfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return code;
}

#define SCK(call)                                                           \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess)                                                  \
      return sfail(e_ == cudaErrorMemoryAllocation ? SNN_E_OOM : SNN_E_CUDA, \
                   "%s failed: %s", #call, cudaGetErrorString(e_));         \
  } while (0)

#define SREQ(cond, code, ...)                     \
  do {                                            \
    if (!(cond)) return sfail(code, __VA_ARGS__); \
  } while (0)

constexpr int kTuneCandidates[] = {1, 2, 4, 8};
constexpr int kTuneStepsPerCandidate = 4;
constexpr uint64_t kLogCapMax = 1ull << 22;  // recorded spikes per request
// Served nets share each delivery launch, so a net gets tiles in proportion
// to its synapses (one per kSynPerTile, at most one per SM) rather than one
// per SM: small nets then add few CTAs of fixed per-CTA cost to the batch.
constexpr uint64_t kSynPerTile = 1ull << 22;

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
  uint64_t id = 0;
  snn_request r{};
  snn_result res{};
  snn_net* net = nullptr;
  int64_t steps_left = 0;
  uint64_t est = 0;
  std::vector<uint32_t> sp_src;
  std::vector<int32_t> sp_t;
};

}  // namespace

struct snn_server {
  uint64_t budget = 0, used = 0;
  int fmt = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  double t0 = 0;

  std::mutex mu;                       // guards everything below it
  std::condition_variable cv;          // builder wake-ups
  std::deque<uint64_t> queue;          // ids waiting for admission
  std::map<uint64_t, Req> reqs;
  std::vector<Req*> ready;             // built, not yet in the batch
  uint64_t next_id = 1;
  bool stop = false;
  uint64_t submitted = 0, done = 0, failed = 0, events = 0, spikes = 0;

  // used by the stepping thread only (map nodes are stable: a request is
  // erased only after it finished)
  std::vector<Req*> active;
  std::vector<int> active_steps;       // n_steps per net in the tables
  BatchNet* d_nets = nullptr;
  uint2* d_umap = nullptr;
  uint2* d_dmap = nullptr;
  size_t cap_nets = 0, cap_umap = 0, cap_dmap = 0;
  uint32_t n_ublocks = 0, n_dctas = 0;
  size_t dsmem = 0;
  bool dirty = true;
  cudaGraphExec_t graph = nullptr;
  int graph_m = 0;
  // GPU time per step: two event pairs used in turn, so that the host
  // prepares step k+1 while step k runs and reads step k's time afterwards
  cudaEvent_t ev[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  bool ev_pending[2] = {false, false};
  int ev_m[2] = {0, 0};
  int ev_cur = 0;
  uint64_t steps = 0, intervals = 0, launches = 0;
  double gpu_ms = 0;
  // autotuner
  int ips = 1;            // intervals per step
  int tuned = 0;
  int tune_idx = 0, tune_count = 0;
  double tune_ms = 0;
  double tune_best = 1e300;
  int tune_best_m = 1;

  std::thread builder;
};

namespace {

// Device bytes a request will hold (the store with its build keys, tile
// index, ring buffer, state, interval list, spike log), plus slack for the
// allocator's granularity.
int32_t serve_tile_width(const snn_request& r) {
  const uint64_t n = (uint64_t)r.params.n_exc + r.params.n_inh;
  const uint64_t n_syn = n * ((uint64_t)r.conn.k_exc + r.conn.k_inh);
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t tiles = (n_syn + kSynPerTile - 1) / kSynPerTile;
  tiles = std::min<uint64_t>(std::max<uint64_t>(tiles, 1), (uint64_t)std::max(sms, 1));
  return (int32_t)std::min<uint64_t>((n + tiles - 1) / tiles, 1u << 30);
}

uint64_t estimate_bytes(const snn_request& r, int fmt) {
  const uint64_t n = (uint64_t)r.params.n_exc + r.params.n_inh;
  const uint64_t k = (uint64_t)r.conn.k_exc + r.conn.k_inh;
  const uint64_t n_syn = n * k;
  const uint64_t ch = (uint64_t)chunk_records(fmt);
  const uint64_t padded = (n_syn + ch - 1) / ch * ch + ch;
  const uint64_t rec = fmt == SNN_W_FP32_12B ? 12 : 8;
  uint64_t store = padded * rec + (fmt == SNN_W_FP32_12B ? padded * 8 : 0);
  const int iv = r.params.interval ? r.params.interval : r.conn.d_lo;
  uint32_t tw = 0, nt = 0;
  int lb = 0;
  tile_geometry((uint32_t)n, iv + (r.conn.d_hi - r.conn.d_lo),
                r.params.tile_width, &tw, &lb, &nt);
  const uint64_t index = n * (nt + 1ull) * 4;
  const uint64_t pitch = (n + 31) / 32 * 32;
  const uint64_t rb = (uint64_t)r.params.n_slots * pitch * 4;
  const uint64_t state = 16 * n + rb + n * (uint64_t)iv * 16 + (n + 1) * 8 +
                         n * 4 + r.params.spike_log_capacity * 8;
  return store + index + state + (8ull << 20);
}

void builder_main(snn_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    sv->cv.wait(lk, [&] {
      if (sv->stop) return true;
      if (sv->queue.empty()) return false;
      const Req& h = sv->reqs[sv->queue.front()];
      return sv->used + h.est <= sv->budget;
    });
    if (sv->stop) return;
    const uint64_t id = sv->queue.front();
    sv->queue.pop_front();
    Req& q = sv->reqs[id];
    q.res.state = SNN_REQ_BUILDING;
    q.res.t_admit = now_s() - sv->t0;
    sv->used += q.est;
    const snn_request r = q.r;
    lk.unlock();
    // build outside the lock, on the net's own stream
    snn_net* net = nullptr;
    int rc = snn_create(&r.params, nullptr, &net);
    if (rc == SNN_OK) rc = snn_connect_fixed_indegree(net, &r.conn);
    if (rc == SNN_OK) rc = snn_finalize(net);
    if (rc == SNN_OK && !(net->tile_off && net->n_syn > 0 &&
                          net->p.deliver_mode == SNN_DELIVER_TILED))
      rc = SNN_E_ARG;
    if (rc == SNN_OK) rc = snn_sync(net);
    lk.lock();
    Req& q2 = sv->reqs[id];
    if (rc == SNN_OK) {
      q2.net = net;
      q2.steps_left = r.n_steps;
      q2.res.n_synapses = net->n_syn;
      sv->ready.push_back(&q2);
    } else {
      if (net) snn_destroy(net);
      sv->used -= q2.est;
      q2.res.state = SNN_REQ_FAILED;
      q2.res.error = rc;
      q2.res.t_done = now_s() - sv->t0;
      sv->failed += 1;
    }
  }
}

template <class T>
int ensure_dev(T** p, size_t* cap, size_t n, cudaStream_t s) {
  if (n <= *cap) return SNN_OK;
  const size_t c = std::max<size_t>(n, 2 * *cap);
  pool_free(*p, s);
  *p = nullptr;
  *cap = 0;
  SCK(pool_alloc(reinterpret_cast<void**>(p), c * sizeof(T), s));
  *cap = c;
  return SNN_OK;
}

// Rebuild the batch table and block maps for the active nets.
int rebuild_tables(snn_server* sv) {
  // earlier steps may still read the tables: finish them first
  SCK(cudaStreamSynchronize(sv->stream));
  std::vector<BatchNet> nets(sv->active.size());
  std::vector<uint2> umap, dmap;
  size_t smem = 0;
  const uint32_t ut = update_threads();
  for (size_t k = 0; k < sv->active.size(); ++k) {
    snn_net* net = sv->active[k]->net;
    nets[k].v = net->view();
    nets[k].c = net->uc;
    nets[k].n_steps = sv->active_steps[k];
    nets[k].pad_ = 0;
    const uint32_t nb = (net->n + ut - 1) / ut;
    for (uint32_t b = 0; b < nb; ++b) umap.push_back(make_uint2((uint32_t)k, b));
    for (uint32_t t = 0; t < net->n_tiles; ++t)
      dmap.push_back(make_uint2((uint32_t)k, t));
    smem = std::max(smem, tiled_smem_bytes(nets[k].v));
  }
  int rc;
  if ((rc = ensure_dev(&sv->d_nets, &sv->cap_nets, nets.size(), sv->stream)) != SNN_OK) return rc;
  if ((rc = ensure_dev(&sv->d_umap, &sv->cap_umap, umap.size(), sv->stream)) != SNN_OK) return rc;
  if ((rc = ensure_dev(&sv->d_dmap, &sv->cap_dmap, dmap.size(), sv->stream)) != SNN_OK) return rc;
  SCK(cudaMemcpyAsync(sv->d_nets, nets.data(), nets.size() * sizeof(BatchNet),
                      cudaMemcpyHostToDevice, sv->stream));
  SCK(cudaMemcpyAsync(sv->d_umap, umap.data(), umap.size() * sizeof(uint2),
                      cudaMemcpyHostToDevice, sv->stream));
  SCK(cudaMemcpyAsync(sv->d_dmap, dmap.data(), dmap.size() * sizeof(uint2),
                      cudaMemcpyHostToDevice, sv->stream));
  SCK(cudaStreamSynchronize(sv->stream));  // host vectors go out of scope
  sv->n_ublocks = (uint32_t)umap.size();
  sv->n_dctas = (uint32_t)dmap.size();
  sv->dsmem = smem;
  if (sv->graph) {
    cudaGraphExecDestroy(sv->graph);
    sv->graph = nullptr;
  }
  sv->dirty = false;
  return SNN_OK;
}

int launch_intervals(snn_server* sv, int m) {
  for (int i = 0; i < m; ++i) {
    SCK(launch_update_batch(sv->d_nets, sv->d_umap, sv->n_ublocks, sv->stream));
    SCK(launch_deliver_tiled_batch(sv->fmt, sv->d_nets, sv->d_dmap, sv->n_dctas,
                                   sv->dsmem, sv->stream));
  }
  return SNN_OK;
}

int capture(snn_server* sv, int m) {
  if (sv->graph) {
    cudaGraphExecDestroy(sv->graph);
    sv->graph = nullptr;
  }
  cudaGraph_t g;
  SCK(cudaStreamBeginCapture(sv->stream, cudaStreamCaptureModeThreadLocal));
  int rc = launch_intervals(sv, m);
  cudaError_t e = cudaStreamEndCapture(sv->stream, &g);
  if (rc != SNN_OK) return rc;
  SCK(e);
  e = cudaGraphInstantiate(&sv->graph, g, 0);
  cudaGraphDestroy(g);
  SCK(e);
  sv->graph_m = m;
  return SNN_OK;
}

// Feed the autotuner with the GPU time of the last step (per interval).
void tune_observe(snn_server* sv, double ms, int m) {
  if (sv->tuned || m != kTuneCandidates[sv->tune_idx]) return;
  sv->tune_ms += ms / m;
  if (++sv->tune_count < kTuneStepsPerCandidate) return;
  const double avg = sv->tune_ms / sv->tune_count;
  if (avg < sv->tune_best) {
    sv->tune_best = avg;
    sv->tune_best_m = m;
  }
  sv->tune_ms = 0;
  sv->tune_count = 0;
  if (++sv->tune_idx == (int)(sizeof(kTuneCandidates) / sizeof(int))) {
    sv->tuned = 1;
    sv->ips = sv->tune_best_m;
  } else {
    sv->ips = kTuneCandidates[sv->tune_idx];
  }
}

// Add the GPU time of the step recorded in event pair `slot` if it has
// finished (or wait for it when `wait`).
int fold_step_time(snn_server* sv, int slot, bool wait) {
  if (!sv->ev_pending[slot]) return SNN_OK;
  if (wait) {
    SCK(cudaEventSynchronize(sv->ev[slot][1]));
  } else {
    const cudaError_t q = cudaEventQuery(sv->ev[slot][1]);
    if (q == cudaErrorNotReady) return SNN_OK;
    SCK(q);
  }
  float ms = 0;
  SCK(cudaEventElapsedTime(&ms, sv->ev[slot][0], sv->ev[slot][1]));
  sv->gpu_ms += ms;
  tune_observe(sv, ms, sv->ev_m[slot]);
  sv->ev_pending[slot] = false;
  return SNN_OK;
}

int retire(snn_server* sv, std::vector<Req*>& finished) {
  if (finished.empty()) return SNN_OK;
  SCK(cudaStreamSynchronize(sv->stream));
  for (Req* q : finished) {
    snn_net* net = q->net;
    const bool rec = q->r.record_spikes != 0;
    snn_stats st;
    int rc = snn_get_stats(net, &st);
    std::vector<uint32_t> src;
    std::vector<int32_t> t;
    if (rc == SNN_OK && rec && net->log_cap) {
      src.resize(net->log_cap);
      t.resize(net->log_cap);
      uint64_t n = 0;
      int r2 = snn_read_spikes(net, src.data(), t.data(), src.size(), &n,
                               SNN_MEM_HOST);
      if (r2 != SNN_OK && r2 != SNN_E_OVERFLOW) rc = r2;
      src.resize(std::min<uint64_t>(n, src.size()));
      t.resize(src.size());
    }
    snn_destroy(net);
    std::lock_guard<std::mutex> lk(sv->mu);
    q->net = nullptr;
    sv->used -= q->est;
    q->res.t_done = now_s() - sv->t0;
    if (rc == SNN_OK) {
      q->res.state = SNN_REQ_DONE;
      q->res.spikes = st.spikes;
      q->res.events = st.events_delivered;
      q->sp_src.swap(src);
      q->sp_t.swap(t);
      sv->done += 1;
      sv->events += st.events_delivered;
      sv->spikes += st.spikes;
    } else {
      q->res.state = SNN_REQ_FAILED;
      q->res.error = rc;
      sv->failed += 1;
    }
  }
  sv->cv.notify_all();
  return SNN_OK;
}

}  // namespace

extern "C" {

int snn_server_create(uint64_t mem_budget, int32_t weight_format, void* stream,
                      snn_server** out) {
  SREQ(out, SNN_E_ARG, "null argument");
  *out = nullptr;
  SREQ(weight_format == SNN_W_FP32_12B || weight_format == SNN_W_BF16_8B,
       SNN_E_ARG, "bad weight format");
  SREQ(mem_budget > 0, SNN_E_ARG, "zero memory budget");
  snn_server* sv = new snn_server();
  sv->budget = mem_budget;
  sv->fmt = weight_format;
  sv->t0 = now_s();
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    delete sv;
    return sfail(SNN_E_CUDA, "no CUDA device");
  }
  if (stream) {
    sv->stream = static_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreate(&sv->stream) != cudaSuccess) {
      delete sv;
      return sfail(SNN_E_CUDA, "stream creation failed");
    }
    sv->own_stream = true;
  }
  if (cudaEventCreate(&sv->ev[0][0]) != cudaSuccess ||
      cudaEventCreate(&sv->ev[0][1]) != cudaSuccess ||
      cudaEventCreate(&sv->ev[1][0]) != cudaSuccess ||
      cudaEventCreate(&sv->ev[1][1]) != cudaSuccess) {
    snn_server_destroy(sv);
    return sfail(SNN_E_CUDA, "event creation failed");
  }
  sv->ips = kTuneCandidates[0];
  sv->builder = std::thread(builder_main, sv);
  *out = sv;
  return SNN_OK;
}

int snn_server_submit(snn_server* sv, const snn_request* req, uint64_t* id) {
  SREQ(sv && req && id, SNN_E_ARG, "null argument");
  SREQ(req->params.weight_format == sv->fmt, SNN_E_ARG,
       "request weight format differs from the server's");
  SREQ(req->n_steps >= 1 && req->n_steps < (1ll << 31), SNN_E_ARG,
       "bad n_steps");
  SREQ(req->conn.k_exc + req->conn.k_inh >= 1, SNN_E_ARG,
       "a served net needs synapses");
  SREQ(req->params.deliver_mode == SNN_DELIVER_TILED, SNN_E_ARG,
       "served nets use the tiled delivery");
  Req q;
  q.r = *req;
  if (req->record_spikes) {
    // every neuron at most once per refractory period plus one step
    const double refr = floor(req->params.t_ref / req->params.h + 0.5);
    const uint64_t n = (uint64_t)req->params.n_exc + req->params.n_inh;
    const uint64_t bound =
        n * (uint64_t)((req->n_steps + refr) / (refr + 1.0));
    q.r.params.spike_log_capacity = std::min(bound, kLogCapMax);
  } else {
    q.r.params.spike_log_capacity = 0;
  }
  if (q.r.params.tile_width == 0) q.r.params.tile_width = serve_tile_width(q.r);
  q.est = estimate_bytes(q.r, sv->fmt);
  SREQ(q.est <= sv->budget, SNN_E_ARG,
       "request needs about %llu bytes, above the server budget",
       (unsigned long long)q.est);
  std::lock_guard<std::mutex> lk(sv->mu);
  q.id = sv->next_id++;
  q.res.id = q.id;
  q.res.user_tag = req->user_tag;
  q.res.state = SNN_REQ_QUEUED;
  q.res.n_neurons = (uint64_t)req->params.n_exc + req->params.n_inh;
  q.res.n_steps = req->n_steps;
  q.res.t_submit = now_s() - sv->t0;
  q.res.t_admit = q.res.t_start = q.res.t_done = -1;
  q.res.bytes = q.est;
  *id = q.id;
  sv->reqs.emplace(q.id, std::move(q));
  sv->queue.push_back(*id);
  sv->submitted += 1;
  sv->cv.notify_all();
  return SNN_OK;
}

int snn_server_step(snn_server* sv, int32_t* n_active) {
  SREQ(sv, SNN_E_ARG, "null server");
  SCK(cudaSetDevice(sv->device));
  // fold in the GPU time of finished steps, oldest first; the pair this
  // step reuses must be finished
  int rc;
  for (int k = 0; k < 2; ++k) {
    const int slot = sv->ev_cur ^ k;
    if ((rc = fold_step_time(sv, slot, k == 0)) != SNN_OK) return rc;
  }
  // admit nets the builder finished
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    for (Req* q : sv->ready) {
      q->res.state = SNN_REQ_RUNNING;
      q->res.t_start = now_s() - sv->t0;
      sv->active.push_back(q);
      sv->active_steps.push_back(-1);
      sv->dirty = true;
    }
    sv->ready.clear();
  }
  if (sv->active.empty()) {
    if (n_active) *n_active = 0;
    return SNN_OK;
  }
  // this step's intervals: m if every net has m full intervals left
  int m = sv->ips;
  for (size_t k = 0; k < sv->active.size(); ++k) {
    const Req& q = *sv->active[k];
    const int iv = q.net->interval;
    const int next = (int)std::min<int64_t>(iv, q.steps_left);
    if (q.steps_left < (int64_t)m * iv) m = 1;
    if (sv->active_steps[k] != next) {
      sv->active_steps[k] = next;
      sv->dirty = true;
    }
  }
  if (sv->dirty && (rc = rebuild_tables(sv)) != SNN_OK) return rc;
  if (m > 1 && (!sv->graph || sv->graph_m != m) &&
      (rc = capture(sv, m)) != SNN_OK)
    return rc;
  const int slot = sv->ev_cur;
  SCK(cudaEventRecord(sv->ev[slot][0], sv->stream));
  if (m > 1) {
    SCK(cudaGraphLaunch(sv->graph, sv->stream));
  } else {
    if ((rc = launch_intervals(sv, 1)) != SNN_OK) return rc;
  }
  SCK(cudaEventRecord(sv->ev[slot][1], sv->stream));
  sv->ev_pending[slot] = true;
  sv->ev_m[slot] = m;
  sv->ev_cur ^= 1;
  sv->steps += 1;
  sv->intervals += m;
  sv->launches += 2ull * m;
  // bookkeeping; retire nets that finished
  std::vector<Req*> finished, keep;
  std::vector<int> keep_steps;
  for (size_t k = 0; k < sv->active.size(); ++k) {
    Req& q = *sv->active[k];
    q.steps_left -= (int64_t)m * sv->active_steps[k];
    if (q.steps_left <= 0) {
      finished.push_back(sv->active[k]);
    } else {
      keep.push_back(sv->active[k]);
      keep_steps.push_back(sv->active_steps[k]);
    }
  }
  if (!finished.empty()) {
    sv->active.swap(keep);
    sv->active_steps.swap(keep_steps);
    sv->dirty = true;
    if ((rc = retire(sv, finished)) != SNN_OK) return rc;
  }
  if (n_active) *n_active = (int32_t)sv->active.size();
  return SNN_OK;
}

int snn_server_poll(snn_server* sv, uint64_t id, snn_result* out) {
  SREQ(sv && out, SNN_E_ARG, "null argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(id);
  SREQ(it != sv->reqs.end(), SNN_E_ARG, "unknown request %llu",
       (unsigned long long)id);
  *out = it->second.res;
  return SNN_OK;
}

int snn_server_spikes(snn_server* sv, uint64_t id, uint32_t* src, int32_t* t,
                      uint64_t cap, uint64_t* n) {
  SREQ(sv && n, SNN_E_ARG, "null argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(id);
  SREQ(it != sv->reqs.end(), SNN_E_ARG, "unknown request");
  const Req& q = it->second;
  SREQ(q.res.state == SNN_REQ_DONE, SNN_E_STATE, "request not finished");
  *n = q.sp_src.size();
  const uint64_t k = std::min<uint64_t>(cap, q.sp_src.size());
  if (k) {
    SREQ(src && t, SNN_E_ARG, "null output arrays");
    memcpy(src, q.sp_src.data(), k * 4);
    memcpy(t, q.sp_t.data(), k * 4);
  }
  return k < q.sp_src.size() ? sfail(SNN_E_OVERFLOW, "%llu spikes recorded",
                                     (unsigned long long)q.sp_src.size())
                             : SNN_OK;
}

int snn_server_release(snn_server* sv, uint64_t id) {
  SREQ(sv, SNN_E_ARG, "null server");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(id);
  SREQ(it != sv->reqs.end(), SNN_E_ARG, "unknown request");
  SREQ(it->second.res.state == SNN_REQ_DONE ||
           it->second.res.state == SNN_REQ_FAILED,
       SNN_E_STATE, "request not finished");
  sv->reqs.erase(it);
  return SNN_OK;
}

int snn_server_get_stats(snn_server* sv, snn_server_stats* out) {
  SREQ(sv && out, SNN_E_ARG, "null argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  memset(out, 0, sizeof *out);
  out->submitted = sv->submitted;
  out->done = sv->done;
  out->failed = sv->failed;
  out->active = sv->active.size();
  out->queued = sv->queue.size();
  out->steps = sv->steps;
  out->intervals = sv->intervals;
  out->kernel_launches = sv->launches;
  out->events = sv->events;
  out->spikes = sv->spikes;
  out->mem_budget = sv->budget;
  out->mem_used = sv->used;
  out->intervals_per_step = sv->ips;
  out->tuned = sv->tuned;
  out->gpu_ms = sv->gpu_ms;
  return SNN_OK;
}

int snn_server_destroy(snn_server* sv) {
  if (!sv) return SNN_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  if (sv->builder.joinable()) sv->builder.join();
  cudaSetDevice(sv->device);
  if (sv->stream) cudaStreamSynchronize(sv->stream);
  for (auto& kv : sv->reqs)
    if (kv.second.net) snn_destroy(kv.second.net);
  if (sv->graph) cudaGraphExecDestroy(sv->graph);
  for (auto& pair : sv->ev)
    for (cudaEvent_t e : pair)
      if (e) cudaEventDestroy(e);
  pool_free(sv->d_nets, sv->stream);
  pool_free(sv->d_umap, sv->stream);
  pool_free(sv->d_dmap, sv->stream);
  if (sv->stream) cudaStreamSynchronize(sv->stream);
  if (sv->own_stream) cudaStreamDestroy(sv->stream);
  delete sv;
  return SNN_OK;
}

}  // extern "C"
