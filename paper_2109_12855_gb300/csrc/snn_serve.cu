// snn_serve.cu -- continuous batching of independent simulation requests
// (the serving entry points of include/snn.h).
//
// Requests queue in arrival order.  A builder thread admits the head request
// when its estimated device footprint fits the budget and builds its net
// (store construction on the net's own stream) while the admitted nets keep
// running.  Running nets are grouped into lanes by size (synapse count); a
// lane is a batch with its own stream: a step advances every net of a lane
// by its next interval with one batched update launch and one batched
// tiled-delivery launch for all of them (k_update_batch /
// k_deliver_tiled_batch: a device table holds each net's view, update
// constants and step count, and a block map sends every CTA to its (net,
// block) or (net, tile)).  Lanes run concurrently, so a small net does not
// advance at the pace of the largest one.  While a lane's batch is unchanged
// a step may run several intervals captured as one CUDA graph; a small
// autotuner per lane picks that number from measured GPU time per interval.
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

constexpr int kTuneCandidates[] = {1, 2, 4, 8, 16};  // 2^0 .. 2^kMaxGraphLog
constexpr int kTuneStepsPerCandidate = 4;
constexpr uint64_t kLogCapMax = 1ull << 22;  // recorded spikes per request
// Served nets share each delivery launch, so a net gets tiles in proportion
// to its synapses (one per kSynPerTile, at most one per SM) rather than one
// per SM: small nets then add few CTAs of fixed per-CTA cost to the batch.
constexpr uint64_t kSynPerTile = 1ull << 22;
// At most this many tiles per served net, so that other lanes keep SMs.
constexpr uint64_t kServeMaxTiles = 120;
// Graphs cached per lane for steps of 2^1 .. 2^kMaxGraphLog intervals.
constexpr int kMaxGraphLog = 4;
// Lanes by synapse count: below 2^24, below 2^27, and the rest.
constexpr int kLanes = 3;
constexpr uint64_t kLaneBound[kLanes - 1] = {1ull << 24, 1ull << 27};

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

// One lane: a batch of running nets advanced together on its own stream.
struct Lane {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<Req*> active;
  std::vector<int> active_steps;       // n_steps per net in the tables
  BatchNet* d_nets = nullptr;
  uint2* d_umap = nullptr;
  uint2* d_dmap = nullptr;
  size_t cap_nets = 0, cap_umap = 0, cap_dmap = 0;
  uint32_t n_ublocks = 0, n_dctas = 0;
  size_t dsmem = 0;
  bool dirty = true;
  // captured steps of 2, 4, 8 and 16 intervals for the current tables
  cudaGraphExec_t graph[kMaxGraphLog + 1] = {};
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
  double t_last = 0;      // wall time of the lane's previous step (0: idle)
  int m_last = 0;         // intervals of that step
};

struct snn_server {
  uint64_t budget = 0, used = 0;
  int fmt = 0;
  int device = 0;
  double t0 = 0;

  std::mutex mu;                       // guards everything below it
  std::condition_variable cv;          // builder wake-ups
  std::deque<uint64_t> queue[2];       // ids waiting for admission, by
                                       // size class (small, large)
  std::map<uint64_t, Req> reqs;
  std::vector<Req*> ready;             // built, not yet in a lane
  uint64_t next_id = 1;
  bool stop = false;
  uint64_t submitted = 0, done = 0, failed = 0, events = 0, spikes = 0;

  // used by the stepping thread only (map nodes are stable: a request is
  // erased only after it finished)
  Lane lanes[kLanes];
  uint64_t steps = 0;

  std::thread builder[2];
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
  tiles = std::min<uint64_t>(std::max<uint64_t>(tiles, 1),
                             std::min<uint64_t>(kServeMaxTiles, std::max(sms, 1)));
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

// Builder thread for one size class (0: small requests, 1: large): admits
// the oldest queued request of its class when its footprint fits the budget
// and builds it on the net's own stream, at the lowest stream priority so
// that the running nets' kernels are served first.  Small requests thus never
// wait behind the build of a large one.
void builder_main(snn_server* sv, int cls) {
  cudaSetDevice(sv->device);
  int prio_least = 0, prio_greatest = 0;
  cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  std::deque<uint64_t>& queue = sv->queue[cls];
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    sv->cv.wait(lk, [&] {
      if (sv->stop) return true;
      if (queue.empty()) return false;
      const Req& h = sv->reqs[queue.front()];
      return sv->used + h.est <= sv->budget;
    });
    if (sv->stop) return;
    const uint64_t id = queue.front();
    queue.pop_front();
    Req& q = sv->reqs[id];
    q.res.state = SNN_REQ_BUILDING;
    q.res.t_admit = now_s() - sv->t0;
    sv->used += q.est;
    snn_request r = q.r;
    r.params.stream_priority = prio_least;
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

int lane_of(const snn_net* net) {
  int k = 0;
  while (k < kLanes - 1 && net->n_syn >= kLaneBound[k]) ++k;
  return k;
}

// Rebuild a lane's batch table and block maps for its active nets.
int rebuild_tables(Lane* ln) {
  // earlier steps may still read the tables: finish them first
  SCK(cudaStreamSynchronize(ln->stream));
  std::vector<BatchNet> nets(ln->active.size());
  std::vector<uint2> umap, dmap;
  size_t smem = 0;
  const uint32_t ut = update_threads();
  for (size_t k = 0; k < ln->active.size(); ++k) {
    snn_net* net = ln->active[k]->net;
    nets[k].v = net->view();
    nets[k].c = net->uc;
    nets[k].n_steps = ln->active_steps[k];
    nets[k].pad_ = 0;
    const uint32_t nb = (net->n + ut - 1) / ut;
    for (uint32_t b = 0; b < nb; ++b) umap.push_back(make_uint2((uint32_t)k, b));
    for (uint32_t t = 0; t < net->n_tiles; ++t)
      dmap.push_back(make_uint2((uint32_t)k, t));
    smem = std::max(smem, tiled_smem_bytes(nets[k].v));
  }
  int rc;
  if ((rc = ensure_dev(&ln->d_nets, &ln->cap_nets, nets.size(), ln->stream)) != SNN_OK)
    return rc;
  if ((rc = ensure_dev(&ln->d_umap, &ln->cap_umap, umap.size(), ln->stream)) != SNN_OK)
    return rc;
  if ((rc = ensure_dev(&ln->d_dmap, &ln->cap_dmap, dmap.size(), ln->stream)) != SNN_OK)
    return rc;
  SCK(cudaMemcpyAsync(ln->d_nets, nets.data(), nets.size() * sizeof(BatchNet),
                      cudaMemcpyHostToDevice, ln->stream));
  SCK(cudaMemcpyAsync(ln->d_umap, umap.data(), umap.size() * sizeof(uint2),
                      cudaMemcpyHostToDevice, ln->stream));
  SCK(cudaMemcpyAsync(ln->d_dmap, dmap.data(), dmap.size() * sizeof(uint2),
                      cudaMemcpyHostToDevice, ln->stream));
  SCK(cudaStreamSynchronize(ln->stream));  // host vectors go out of scope
  ln->n_ublocks = (uint32_t)umap.size();
  ln->n_dctas = (uint32_t)dmap.size();
  ln->dsmem = smem;
  for (cudaGraphExec_t& g : ln->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  ln->dirty = false;
  return SNN_OK;
}

int launch_intervals(Lane* ln, int fmt, int m) {
  for (int i = 0; i < m; ++i) {
    SCK(launch_update_batch(ln->d_nets, ln->d_umap, ln->n_ublocks, ln->stream));
    SCK(launch_deliver_tiled_batch(fmt, ln->d_nets, ln->d_dmap, ln->n_dctas,
                                   ln->dsmem, ln->stream));
  }
  return SNN_OK;
}

int log2_of(int m) {
  int l = 0;
  while ((1 << (l + 1)) <= m) ++l;
  return l;
}

// The lane's graph of m intervals (m a power of two, 2 .. 2^kMaxGraphLog),
// captured on first use for the current tables.
int graph_for(Lane* ln, int fmt, int m, cudaGraphExec_t* out) {
  const int l = log2_of(m);
  if (!ln->graph[l]) {
    cudaGraph_t g;
    SCK(cudaStreamBeginCapture(ln->stream, cudaStreamCaptureModeThreadLocal));
    int rc = launch_intervals(ln, fmt, m);
    cudaError_t e = cudaStreamEndCapture(ln->stream, &g);
    if (rc != SNN_OK) return rc;
    SCK(e);
    e = cudaGraphInstantiate(&ln->graph[l], g, 0);
    cudaGraphDestroy(g);
    SCK(e);
  }
  *out = ln->graph[l];
  return SNN_OK;
}

// Feed a lane's autotuner with the wall time of one of its steps (from its
// start to the start of the next: what the stepping loop, host overheads
// included, spends per interval).
void tune_observe(Lane* ln, double ms, int m) {
  if (ln->tuned || m != kTuneCandidates[ln->tune_idx]) return;
  ln->tune_ms += ms / m;
  if (++ln->tune_count < kTuneStepsPerCandidate) return;
  const double avg = ln->tune_ms / ln->tune_count;
  if (avg < ln->tune_best) {
    ln->tune_best = avg;
    ln->tune_best_m = m;
  }
  ln->tune_ms = 0;
  ln->tune_count = 0;
  if (++ln->tune_idx == (int)(sizeof(kTuneCandidates) / sizeof(int))) {
    ln->tuned = 1;
    ln->ips = ln->tune_best_m;
  } else {
    ln->ips = kTuneCandidates[ln->tune_idx];
  }
}

// Add the GPU time of the step recorded in event pair `slot` if it has
// finished (or wait for it when `wait`).
int fold_step_time(Lane* ln, int slot, bool wait) {
  if (!ln->ev_pending[slot]) return SNN_OK;
  if (wait) {
    SCK(cudaEventSynchronize(ln->ev[slot][1]));
  } else {
    const cudaError_t q = cudaEventQuery(ln->ev[slot][1]);
    if (q == cudaErrorNotReady) return SNN_OK;
    SCK(q);
  }
  float ms = 0;
  SCK(cudaEventElapsedTime(&ms, ln->ev[slot][0], ln->ev[slot][1]));
  ln->gpu_ms += ms;
  ln->ev_pending[slot] = false;
  return SNN_OK;
}

int retire(snn_server* sv, Lane* ln, std::vector<Req*>& finished) {
  if (finished.empty()) return SNN_OK;
  SCK(cudaStreamSynchronize(ln->stream));
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

// One step of one lane: launch its nets' next intervals (several in one
// graph when the autotuner chose so), then retire the nets that finished.
int lane_step(snn_server* sv, Lane* ln, bool* launched) {
  *launched = false;
  int rc;
  // fold in the GPU time of finished steps, oldest first; the pair this
  // step reuses must be finished
  for (int k = 0; k < 2; ++k) {
    const int slot = ln->ev_cur ^ k;
    if ((rc = fold_step_time(ln, slot, k == 0)) != SNN_OK) return rc;
  }
  const double now = now_s();
  if (ln->t_last > 0 && ln->m_last > 0)
    tune_observe(ln, 1e3 * (now - ln->t_last), ln->m_last);
  ln->t_last = 0;
  if (ln->active.empty()) return SNN_OK;
  // this step's intervals: the largest power of two up to the tuned number
  // that every net can fill with whole intervals (1 for a net's last,
  // possibly short, interval)
  int m = ln->ips;
  for (size_t k = 0; k < ln->active.size(); ++k) {
    const Req& q = *ln->active[k];
    const int iv = q.net->interval;
    const int next = (int)std::min<int64_t>(iv, q.steps_left);
    while (m > 1 && q.steps_left < (int64_t)m * iv) m >>= 1;
    if (ln->active_steps[k] != next) {
      ln->active_steps[k] = next;
      ln->dirty = true;
    }
  }
  if (ln->dirty && (rc = rebuild_tables(ln)) != SNN_OK) return rc;
  cudaGraphExec_t gx = nullptr;
  if (m > 1 && (rc = graph_for(ln, sv->fmt, m, &gx)) != SNN_OK) return rc;
  const int slot = ln->ev_cur;
  SCK(cudaEventRecord(ln->ev[slot][0], ln->stream));
  if (m > 1) {
    SCK(cudaGraphLaunch(gx, ln->stream));
  } else {
    if ((rc = launch_intervals(ln, sv->fmt, 1)) != SNN_OK) return rc;
  }
  SCK(cudaEventRecord(ln->ev[slot][1], ln->stream));
  ln->ev_pending[slot] = true;
  ln->ev_m[slot] = m;
  ln->ev_cur ^= 1;
  ln->t_last = now;
  ln->m_last = m;
  ln->steps += 1;
  ln->intervals += m;
  ln->launches += 2ull * m;
  *launched = true;
  // bookkeeping; retire nets that finished
  std::vector<Req*> finished, keep;
  std::vector<int> keep_steps;
  for (size_t k = 0; k < ln->active.size(); ++k) {
    Req& q = *ln->active[k];
    q.steps_left -= (int64_t)m * ln->active_steps[k];
    if (q.steps_left <= 0) {
      finished.push_back(ln->active[k]);
    } else {
      keep.push_back(ln->active[k]);
      keep_steps.push_back(ln->active_steps[k]);
    }
  }
  if (!finished.empty()) {
    ln->active.swap(keep);
    ln->active_steps.swap(keep_steps);
    ln->dirty = true;
    ln->t_last = 0;  // retiring (a synchronisation) is not a steady step
    if ((rc = retire(sv, ln, finished)) != SNN_OK) return rc;
  }
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
  // smaller nets get higher stream priority: when SMs free up, the CTA
  // scheduler serves the short intervals of small nets first and the large
  // nets take the remaining capacity
  int prio_least = 0, prio_greatest = 0;
  cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  for (int k = 0; k < kLanes; ++k) {
    Lane& ln = sv->lanes[k];
    const int prio = prio_greatest + (prio_least - prio_greatest) * k / (kLanes - 1);
    if (k == 0 && stream) {
      ln.stream = static_cast<cudaStream_t>(stream);
    } else if (cudaStreamCreateWithPriority(&ln.stream, cudaStreamDefault, prio) !=
               cudaSuccess) {
      snn_server_destroy(sv);
      return sfail(SNN_E_CUDA, "stream creation failed");
    } else {
      ln.own_stream = true;
    }
    for (auto& pair : ln.ev)
      for (cudaEvent_t& e : pair)
        if (cudaEventCreate(&e) != cudaSuccess) {
          snn_server_destroy(sv);
          return sfail(SNN_E_CUDA, "event creation failed");
        }
    ln.ips = kTuneCandidates[0];
  }
  sv->builder[0] = std::thread(builder_main, sv, 0);
  sv->builder[1] = std::thread(builder_main, sv, 1);
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
  const uint64_t n_syn = ((uint64_t)req->params.n_exc + req->params.n_inh) *
                         ((uint64_t)req->conn.k_exc + req->conn.k_inh);
  sv->reqs.emplace(q.id, std::move(q));
  sv->queue[n_syn >= kLaneBound[0] ? 1 : 0].push_back(*id);
  sv->submitted += 1;
  sv->cv.notify_all();
  return SNN_OK;
}

int snn_server_step(snn_server* sv, int32_t* n_active) {
  SREQ(sv, SNN_E_ARG, "null server");
  SCK(cudaSetDevice(sv->device));
  // admit nets the builder finished, each into the lane of its size
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    for (Req* q : sv->ready) {
      q->res.state = SNN_REQ_RUNNING;
      q->res.t_start = now_s() - sv->t0;
      Lane& ln = sv->lanes[lane_of(q->net)];
      ln.active.push_back(q);
      ln.active_steps.push_back(-1);
      ln.dirty = true;
    }
    sv->ready.clear();
  }
  bool any = false;
  int32_t act = 0;
  for (int k = 0; k < kLanes; ++k) {
    bool launched = false;
    int rc = lane_step(sv, &sv->lanes[k], &launched);
    if (rc != SNN_OK) return rc;
    any = any || launched;
    act += (int32_t)sv->lanes[k].active.size();
  }
  if (any) sv->steps += 1;
  if (n_active) *n_active = act;
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
  out->queued = sv->queue[0].size() + sv->queue[1].size();
  out->steps = sv->steps;
  int tuned = 1, busiest = 0;
  for (int k = 0; k < kLanes; ++k) {
    const Lane& ln = sv->lanes[k];
    out->active += ln.active.size();
    out->intervals += ln.intervals;
    out->kernel_launches += ln.launches;
    out->gpu_ms += ln.gpu_ms;
    if (ln.steps && !ln.tuned) tuned = 0;
    if (ln.intervals > sv->lanes[busiest].intervals) busiest = k;
  }
  out->events = sv->events;
  out->spikes = sv->spikes;
  out->mem_budget = sv->budget;
  out->mem_used = sv->used;
  out->intervals_per_step = sv->lanes[busiest].ips;
  out->tuned = tuned && sv->steps > 0;
  return SNN_OK;
}

int snn_server_destroy(snn_server* sv) {
  if (!sv) return SNN_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  for (std::thread& b : sv->builder)
    if (b.joinable()) b.join();
  cudaSetDevice(sv->device);
  for (Lane& ln : sv->lanes)
    if (ln.stream) cudaStreamSynchronize(ln.stream);
  for (auto& kv : sv->reqs)
    if (kv.second.net) snn_destroy(kv.second.net);
  for (Lane& ln : sv->lanes) {
    for (cudaGraphExec_t g : ln.graph)
      if (g) cudaGraphExecDestroy(g);
    for (auto& pair : ln.ev)
      for (cudaEvent_t e : pair)
        if (e) cudaEventDestroy(e);
    if (ln.stream) {
      pool_free(ln.d_nets, ln.stream);
      pool_free(ln.d_umap, ln.stream);
      pool_free(ln.d_dmap, ln.stream);
      cudaStreamSynchronize(ln.stream);
      if (ln.own_stream) cudaStreamDestroy(ln.stream);
    }
  }
  delete sv;
  return SNN_OK;
}

}  // extern "C"
