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
#include <atomic>
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
// Device memory mapped into the pool when a server is created (at most its
// budget).
constexpr uint64_t kPoolWarmBytes = 64ull << 30;
// Persistent mode: the target GPU time of one step (one launch of the
// persistent kernel), candidates of its autotuner in microseconds, polls of
// a CTA that finds no ready item before it reports a timeout (32 to 256 ns
// apart: a fraction of a second), and the SMs left to large builds while
// one is in flight.
constexpr double kStepUsCandidates[] = {250.0, 500.0, 1000.0, 2000.0};
constexpr int kStepTuneSteps = 3;
constexpr unsigned long long kSpinLimit = 1ull << 20;
constexpr int kBuildReserveSms = 16;
// Nets one persistent step runs at most (sizes its pinned host records).
constexpr size_t kServeMaxNets = 4096;
// Exclusive mode: the target GPU time of one step of the chosen net, the
// intervals of a net's first step (before its time per interval is known),
// and the steps in flight on the GPU at most (the next one is queued while
// the current one runs, so the GPU never idles between steps).
constexpr double kExclusiveStepUs = 1000.0;
constexpr int kExclusiveFirstIntervals = 16;
constexpr int kExclusiveInFlight = 2;
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
  double iv_us = 0;      // persistent / exclusive mode: measured time per
                         // interval
  int fail_code = 0;     // non-zero: retire as failed (e.g. SNN_E_TIMEOUT)
  bool cancel = false;   // snn_server_cancel asked (guarded by the mutex)
};

// fail_code of a cancelled request
constexpr int kCancelled = 1;

}  // namespace

// Device tables of one batch shape: each net's view and constants, and the
// block maps of the batched update and delivery launches; with the graphs
// captured for them.  A lane keeps two, so that it rewrites one while steps
// that read the other may still run.
struct LaneTables {
  BatchNet* d_nets = nullptr;
  uint2* d_umap = nullptr;
  uint2* d_dmap = nullptr;
  size_t cap_nets = 0, cap_umap = 0, cap_dmap = 0;
  uint32_t n_ublocks = 0, n_dctas = 0;
  size_t dsmem = 0;
  // host copies, kept until the next rewrite (the copies to the device are
  // asynchronous)
  std::vector<BatchNet> h_nets;
  std::vector<uint2> h_umap, h_dmap;
  // captured steps of 2, 4, 8 and 16 intervals for these tables
  cudaGraphExec_t graph[kMaxGraphLog + 1] = {};
  cudaEvent_t last_use = nullptr;  // after the last step that read them
  bool used = false;
  std::vector<uint32_t> ub, nt;    // persistent mode: items per interval
};

// One lane: a batch of running nets advanced together on its own stream.
// Nothing in a lane's step waits for the GPU: a lane whose earlier work is
// still needed (an event pair to reuse, tables to rewrite) is skipped for
// that step, and finished nets are retired once the event recorded after
// their last interval has completed.  One slow lane therefore never holds
// up the stepping of the others.
struct Lane {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<Req*> active;
  std::vector<int> active_steps;       // n_steps per net in the tables
  LaneTables tab[2];
  int cur = 0;                         // tables of the current batch shape
  bool dirty = true;
  // nets whose last interval is launched, with the event after it
  std::vector<std::pair<Req*, cudaEvent_t>> retiring;
  std::vector<cudaEvent_t> spare_events;
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
  // persistent mode, per event-pair slot: the per-net launch records (host
  // copy sent before the launch, device copy read back after it), the
  // launch's error word, and the nets (with their interval counts) it ran
  ServeNet* h_sn[2] = {nullptr, nullptr};
  ServeNet* h_sn_back[2] = {nullptr, nullptr};
  ServeCtl* h_ctl[2] = {nullptr, nullptr};
  std::vector<std::pair<Req*, uint32_t>> step_nets[2];
  ServeNet* d_sn = nullptr;
  size_t cap_sn = 0;
  ServeCtl* d_ctl = nullptr;
  // exclusive mode: steps in flight (net, intervals, start and end events)
  struct XStep {
    Req* q;
    int intervals;
    cudaEvent_t e0, e1;
  };
  std::deque<XStep> x_inflight;
  std::vector<cudaEvent_t> x_spare;  // timing events for reuse
  // autotuner of the step's target GPU time
  double step_us = kStepUsCandidates[0];
  int st_idx = 0, st_count = 0, st_tuned = 0;
  double st_gpu = 0, st_wall = 0, st_best = -1;
  double st_util[sizeof(kStepUsCandidates) / sizeof(double)] = {};
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
  bool holds_pool = false;
  // builds in flight: while any runs, the stepping thread instantiates no
  // CUDA graph (instantiation waits for the build's kernels; it launches
  // the intervals directly meanwhile, or replays a graph it already has)
  std::atomic<int> building{0};
  std::atomic<int> building_large{0};  // of which large requests
  bool persistent = false;              // one persistent launch per step
  bool exclusive = false;               // one net per step, least work first
  unsigned long long spin_limit = kSpinLimit;
  double step_us_fixed = 0;             // > 0: no autotuning
  int sms = 1;
};

namespace {

// Device bytes a request will hold (the store with its build keys, tile
// index, ring buffer, state, interval list, spike log), plus slack for the
// allocator's granularity.
int32_t serve_tile_width(const snn_request& r, bool persistent) {
  const uint64_t n = (uint64_t)r.params.n_exc + r.params.n_inh;
  const uint64_t n_syn = n * ((uint64_t)r.conn.k_exc + r.conn.k_inh);
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t tiles = (n_syn + kSynPerTile - 1) / kSynPerTile;
  // the persistent kernel claims tiles one by one: a small net gets at
  // least a few (of 32 neurons or more), so that its delivery spreads over
  // several CTAs when the GPU has room
  if (persistent) tiles = std::max<uint64_t>(tiles, std::min<uint64_t>(8, (n + 31) / 32));
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
    // small builds (a few ms) run at the highest priority, so that small
    // requests start at once; large builds at the lowest, below the lanes
    r.params.stream_priority = cls == 0 ? prio_greatest : prio_least;
    // builds hand SMs back to the running nets every few microseconds
    r.params.build_yield = 1;
    sv->building.fetch_add(1);
    if (cls == 1) sv->building_large.fetch_add(1);
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
    sv->building.fetch_sub(1);
    if (cls == 1) sv->building_large.fetch_sub(1);
    lk.lock();
    Req& q2 = sv->reqs[id];
    if (rc == SNN_OK && q2.cancel) {
      snn_destroy(net);
      sv->used -= q2.est;
      q2.res.state = SNN_REQ_CANCELLED;
      q2.res.t_done = now_s() - sv->t0;
    } else if (rc == SNN_OK) {
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

// Whether the GPU work recorded by event e (nullptr: none) has completed.
int event_done(cudaEvent_t e, bool* done) {
  *done = true;
  if (!e) return SNN_OK;
  const cudaError_t q = cudaEventQuery(e);
  if (q == cudaErrorNotReady) {
    *done = false;
    return SNN_OK;
  }
  SCK(q);
  return SNN_OK;
}

// Write the lane's active nets into its other table set (if no running step
// still reads that set; else *busy = true and nothing changes).
int rebuild_tables(Lane* ln, bool* busy) {
  LaneTables& t = ln->tab[ln->cur ^ 1];
  int rc;
  bool done = true;
  if (t.used && (rc = event_done(t.last_use, &done)) != SNN_OK) return rc;
  *busy = !done;
  if (!done) return SNN_OK;
  t.h_nets.assign(ln->active.size(), BatchNet{});
  t.h_umap.clear();
  t.h_dmap.clear();
  size_t smem = 0;
  const uint32_t ut = update_threads();
  for (size_t k = 0; k < ln->active.size(); ++k) {
    snn_net* net = ln->active[k]->net;
    t.h_nets[k].v = net->view();
    t.h_nets[k].c = net->uc;
    t.h_nets[k].n_steps = ln->active_steps[k];
    t.h_nets[k].pad_ = 0;
    const uint32_t nb = (net->n + ut - 1) / ut;
    for (uint32_t b = 0; b < nb; ++b) t.h_umap.push_back(make_uint2((uint32_t)k, b));
    for (uint32_t tl = 0; tl < net->n_tiles; ++tl)
      t.h_dmap.push_back(make_uint2((uint32_t)k, tl));
    smem = std::max(smem, tiled_smem_bytes(t.h_nets[k].v));
  }
  t.ub.resize(ln->active.size());
  t.nt.resize(ln->active.size());
  for (size_t k = 0; k < ln->active.size(); ++k) {
    const snn_net* net = ln->active[k]->net;
    t.ub[k] = (net->n + serve_threads() - 1) / serve_threads();
    t.nt[k] = net->n_tiles;
  }
  if ((rc = ensure_dev(&t.d_nets, &t.cap_nets, t.h_nets.size(), ln->stream)) != SNN_OK)
    return rc;
  if ((rc = ensure_dev(&t.d_umap, &t.cap_umap, t.h_umap.size(), ln->stream)) != SNN_OK)
    return rc;
  if ((rc = ensure_dev(&t.d_dmap, &t.cap_dmap, t.h_dmap.size(), ln->stream)) != SNN_OK)
    return rc;
  SCK(cudaMemcpyAsync(t.d_nets, t.h_nets.data(), t.h_nets.size() * sizeof(BatchNet),
                      cudaMemcpyHostToDevice, ln->stream));
  SCK(cudaMemcpyAsync(t.d_umap, t.h_umap.data(), t.h_umap.size() * sizeof(uint2),
                      cudaMemcpyHostToDevice, ln->stream));
  SCK(cudaMemcpyAsync(t.d_dmap, t.h_dmap.data(), t.h_dmap.size() * sizeof(uint2),
                      cudaMemcpyHostToDevice, ln->stream));
  t.n_ublocks = (uint32_t)t.h_umap.size();
  t.n_dctas = (uint32_t)t.h_dmap.size();
  t.dsmem = smem;
  for (cudaGraphExec_t& g : t.graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  ln->cur ^= 1;
  ln->dirty = false;
  return SNN_OK;
}

int launch_intervals(Lane* ln, int fmt, int m) {
  const LaneTables& t = ln->tab[ln->cur];
  for (int i = 0; i < m; ++i) {
    SCK(launch_update_batch(t.d_nets, t.d_umap, t.n_ublocks, ln->stream));
    SCK(launch_deliver_tiled_batch(fmt, t.d_nets, t.d_dmap, t.n_dctas, t.dsmem,
                                   ln->stream));
  }
  return SNN_OK;
}

int log2_of(int m) {
  int l = 0;
  while ((1 << (l + 1)) <= m) ++l;
  return l;
}

// The lane's graph of m intervals (m a power of two, 2 .. 2^kMaxGraphLog),
// captured on first use for the current tables; *out = nullptr (launch the
// intervals directly) when it is not there yet and may_instantiate is false.
int graph_for(Lane* ln, int fmt, int m, bool may_instantiate,
              cudaGraphExec_t* out) {
  const int l = log2_of(m);
  cudaGraphExec_t* slot = &ln->tab[ln->cur].graph[l];
  *out = nullptr;
  if (!*slot && !may_instantiate) return SNN_OK;
  if (!*slot) {
    cudaGraph_t g;
    SCK(cudaStreamBeginCapture(ln->stream, cudaStreamCaptureModeThreadLocal));
    int rc = launch_intervals(ln, fmt, m);
    cudaError_t e = cudaStreamEndCapture(ln->stream, &g);
    if (rc != SNN_OK) return rc;
    SCK(e);
    e = cudaGraphInstantiate(slot, g, 0);
    cudaGraphDestroy(g);
    SCK(e);
  }
  *out = *slot;
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

// Add the GPU time of the step recorded in event pair `slot` once it has
// finished; *done = false while it runs.
int fold_step_time(Lane* ln, int slot, bool* done) {
  *done = true;
  if (!ln->ev_pending[slot]) return SNN_OK;
  int rc;
  if ((rc = event_done(ln->ev[slot][1], done)) != SNN_OK || !*done) return rc;
  float ms = 0;
  SCK(cudaEventElapsedTime(&ms, ln->ev[slot][0], ln->ev[slot][1]));
  ln->gpu_ms += ms;
  ln->ev_pending[slot] = false;
  return SNN_OK;
}

// Retire the lane's finished nets whose last interval has completed: read
// their counters and spikes, free them, publish the results.
int retire_done(snn_server* sv, Lane* ln) {
  std::vector<std::pair<Req*, cudaEvent_t>> keep;
  for (auto& fe : ln->retiring) {
    bool done = true;
    int rc = event_done(fe.second, &done);
    if (rc != SNN_OK) return rc;
    if (!done) {
      keep.push_back(fe);
      continue;
    }
    ln->spare_events.push_back(fe.second);
    Req* q = fe.first;
    snn_net* net = q->net;
    const bool rec = q->r.record_spikes != 0;
    snn_stats st;
    rc = q->fail_code ? q->fail_code : snn_get_stats(net, &st);
    if (q->fail_code == kCancelled) {
      snn_destroy(net);
      std::lock_guard<std::mutex> lk(sv->mu);
      q->net = nullptr;
      sv->used -= q->est;
      q->res.t_done = now_s() - sv->t0;
      q->res.state = SNN_REQ_CANCELLED;
      sv->cv.notify_all();
      continue;
    }
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
    sv->cv.notify_all();
  }
  ln->retiring.swap(keep);
  return SNN_OK;
}

// Nets of the lane whose cancellation was asked leave the batch and retire
// (as cancelled) once the work already launched for them has completed.
int drop_cancelled(snn_server* sv, Lane* ln) {
  std::vector<Req*> gone;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    for (Req* q : ln->active)
      if (q->cancel) gone.push_back(q);
  }
  if (gone.empty()) return SNN_OK;
  std::vector<Req*> keep;
  std::vector<int> keep_steps;
  for (size_t k = 0; k < ln->active.size(); ++k) {
    Req* q = ln->active[k];
    if (std::find(gone.begin(), gone.end(), q) != gone.end()) {
      q->fail_code = kCancelled;
      cudaEvent_t e = nullptr;
      SCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      // (exclusive mode runs each net on its own stream)
      SCK(cudaEventRecord(e, sv->exclusive ? q->net->stream : ln->stream));
      ln->retiring.emplace_back(q, e);
    } else {
      keep.push_back(q);
      keep_steps.push_back(ln->active_steps[k]);
    }
  }
  ln->active.swap(keep);
  ln->active_steps.swap(keep_steps);
  ln->dirty = true;
  ln->t_last = 0;
  return SNN_OK;
}

// One step of one lane: retire what finished, then launch its nets' next
// intervals (several in one graph when the autotuner chose so) unless the
// GPU still needs the lane's event pair or its other table set.
int lane_step(snn_server* sv, Lane* ln, bool* launched) {
  *launched = false;
  int rc;
  if ((rc = drop_cancelled(sv, ln)) != SNN_OK) return rc;
  if ((rc = retire_done(sv, ln)) != SNN_OK) return rc;
  // fold in the GPU time of finished steps, oldest first; the pair this
  // step reuses must be finished, else the lane sits this step out
  bool reuse_done = true;
  for (int k = 0; k < 2; ++k) {
    const int slot = ln->ev_cur ^ k;
    bool done = true;
    if ((rc = fold_step_time(ln, slot, &done)) != SNN_OK) return rc;
    if (k == 0) reuse_done = done;
  }
  if (!reuse_done) return SNN_OK;
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
  if (ln->dirty) {
    bool busy = false;
    if ((rc = rebuild_tables(ln, &busy)) != SNN_OK) return rc;
    if (busy) return SNN_OK;
  }
  cudaGraphExec_t gx = nullptr;
  if (m > 1 && (rc = graph_for(ln, sv->fmt, m, sv->building.load() == 0,
                               &gx)) != SNN_OK)
    return rc;
  const int slot = ln->ev_cur;
  SCK(cudaEventRecord(ln->ev[slot][0], ln->stream));
  if (gx) {
    SCK(cudaGraphLaunch(gx, ln->stream));
  } else {
    if ((rc = launch_intervals(ln, sv->fmt, m)) != SNN_OK) return rc;
  }
  SCK(cudaEventRecord(ln->ev[slot][1], ln->stream));
  LaneTables& tb = ln->tab[ln->cur];
  if (!tb.last_use) SCK(cudaEventCreateWithFlags(&tb.last_use, cudaEventDisableTiming));
  SCK(cudaEventRecord(tb.last_use, ln->stream));
  tb.used = true;
  ln->ev_pending[slot] = true;
  ln->ev_m[slot] = m;
  ln->ev_cur ^= 1;
  ln->t_last = now;
  ln->m_last = m;
  ln->steps += 1;
  ln->intervals += m;
  ln->launches += 2ull * m;
  *launched = true;
  // bookkeeping; nets that finished leave the batch and retire once this
  // step has completed
  std::vector<Req*> keep;
  std::vector<int> keep_steps;
  bool any_done = false;
  for (size_t k = 0; k < ln->active.size(); ++k) {
    Req& q = *ln->active[k];
    q.steps_left -= (int64_t)m * ln->active_steps[k];
    if (q.steps_left <= 0) {
      cudaEvent_t e = nullptr;
      if (!ln->spare_events.empty()) {
        e = ln->spare_events.back();
        ln->spare_events.pop_back();
      } else {
        SCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      }
      SCK(cudaEventRecord(e, ln->stream));
      ln->retiring.emplace_back(ln->active[k], e);
      any_done = true;
    } else {
      keep.push_back(ln->active[k]);
      keep_steps.push_back(ln->active_steps[k]);
    }
  }
  if (any_done) {
    ln->active.swap(keep);
    ln->active_steps.swap(keep_steps);
    ln->dirty = true;
    ln->t_last = 0;  // a change of batch is not a steady step
  }
  return SNN_OK;
}

// Exclusive mode: one step runs one net alone -- the running net with the
// least remaining work (steps left x synapses: shortest remaining processing
// time first, so that a small request is never slowed by a large one) --
// for about kExclusiveStepUs of GPU time, with the single-net kernels on the
// net's own stream (its captured interval graphs, or direct launches while a
// build runs).  Up to kExclusiveInFlight steps are queued on the GPU; the
// choice is made again at every step, so a newly admitted smaller request
// preempts a larger one within a step or two.
int lane_step_exclusive(snn_server* sv, Lane* ln, bool* launched) {
  *launched = false;
  int rc;
  if ((rc = drop_cancelled(sv, ln)) != SNN_OK) return rc;
  if ((rc = retire_done(sv, ln)) != SNN_OK) return rc;
  // steps of nets retired just now keep no pointer to their request (the
  // caller may release it once it has seen the result)
  for (Lane::XStep& x : ln->x_inflight)
    if (x.q && !x.q->net) x.q = nullptr;
  // fold in the GPU time of completed steps, oldest first
  while (!ln->x_inflight.empty()) {
    Lane::XStep& x = ln->x_inflight.front();
    bool done = true;
    if ((rc = event_done(x.e1, &done)) != SNN_OK) return rc;
    if (!done) break;
    float ms = 0;
    SCK(cudaEventElapsedTime(&ms, x.e0, x.e1));
    ln->gpu_ms += ms;
    const double us = 1e3 * ms / std::max(x.intervals, 1);
    if (x.q) x.q->iv_us = x.q->iv_us > 0 ? 0.5 * (x.q->iv_us + us) : us;
    ln->x_spare.push_back(x.e0);
    ln->x_spare.push_back(x.e1);
    ln->x_inflight.pop_front();
  }
  if (ln->active.empty() || ln->x_inflight.size() >= (size_t)kExclusiveInFlight)
    return SNN_OK;
  size_t pick = 0;
  double best = 1e300;
  for (size_t k = 0; k < ln->active.size(); ++k) {
    const Req& q = *ln->active[k];
    const double work = (double)q.steps_left * (double)q.net->n_syn;
    if (work < best) {
      best = work;
      pick = k;
    }
  }
  Req& q = *ln->active[pick];
  const int iv = q.net->interval;
  int m = kExclusiveFirstIntervals;
  if (q.iv_us > 0)
    m = (int)std::min(4096.0, std::max(8.0, kExclusiveStepUs / q.iv_us));
  const int64_t steps = std::min<int64_t>((int64_t)m * iv, q.steps_left);
  cudaEvent_t e[2];
  for (int k = 0; k < 2; ++k) {
    if (!ln->x_spare.empty()) {
      e[k] = ln->x_spare.back();
      ln->x_spare.pop_back();
    } else {
      SCK(cudaEventCreate(&e[k]));
    }
  }
  cudaStream_t s = q.net->stream;
  SCK(cudaEventRecord(e[0], s));
  if ((rc = simulate_async(q.net, steps, sv->building.load() == 0)) != SNN_OK) {
    ln->x_spare.push_back(e[0]);
    ln->x_spare.push_back(e[1]);
    return rc;
  }
  SCK(cudaEventRecord(e[1], s));
  const int n_iv = (int)((steps + iv - 1) / iv);
  ln->x_inflight.push_back({&q, n_iv, e[0], e[1]});
  ln->steps += 1;
  ln->intervals += n_iv;
  ln->launches += 2ull * n_iv;
  *launched = true;
  q.steps_left -= steps;
  if (q.steps_left <= 0) {  // retire once this last step has completed
    cudaEvent_t d = nullptr;
    if (!ln->spare_events.empty()) {
      d = ln->spare_events.back();
      ln->spare_events.pop_back();
    } else {
      SCK(cudaEventCreateWithFlags(&d, cudaEventDisableTiming));
    }
    SCK(cudaEventRecord(d, s));
    ln->retiring.emplace_back(&q, d);
    ln->active.erase(ln->active.begin() + pick);
    ln->active_steps.erase(ln->active_steps.begin() + pick);
  }
  return SNN_OK;
}

// Persistent mode: observe the GPU time of a finished step for the step
// length autotuner (steady steps only), and move to the next candidate or
// settle on the shortest step whose GPU utilisation (GPU time over wall
// time) is within 5 % of the best.
void tune_step_length(Lane* ln, double gpu_ms) {
  if (ln->st_tuned) return;
  const double now = now_s();
  if (ln->st_count == 0) {
    ln->st_wall = now;  // window start
    ln->st_gpu = 0;
  } else {
    ln->st_gpu += gpu_ms;
  }
  if (++ln->st_count <= kStepTuneSteps) return;
  const double util = ln->st_gpu / (1e3 * std::max(now - ln->st_wall, 1e-9));
  constexpr int nc = (int)(sizeof(kStepUsCandidates) / sizeof(double));
  if (ln->st_best < 0 || util > ln->st_best) ln->st_best = util;
  ln->st_util[ln->st_idx] = util;
  ln->st_count = 0;
  if (++ln->st_idx < nc) {
    ln->step_us = kStepUsCandidates[ln->st_idx];
    return;
  }
  for (int c = 0; c < nc; ++c)
    if (ln->st_util[c] >= 0.95 * ln->st_best) {
      ln->step_us = kStepUsCandidates[c];
      break;
    }
  ln->st_tuned = 1;
}

// Persistent mode: fold a finished step (GPU time; each net's measured time
// per interval; a timeout fails the nets it ran).  *done = false while the
// step runs.
int fold_persistent(snn_server* sv, Lane* ln, int slot, bool* done) {
  *done = true;
  if (!ln->ev_pending[slot]) return SNN_OK;
  int rc;
  if ((rc = event_done(ln->ev[slot][1], done)) != SNN_OK || !*done) return rc;
  float ms = 0;
  SCK(cudaEventElapsedTime(&ms, ln->ev[slot][0], ln->ev[slot][1]));
  ln->gpu_ms += ms;
  ln->ev_pending[slot] = false;
  const bool timeout = ln->h_ctl[slot]->error != 0;
  auto& sn = ln->step_nets[slot];
  for (size_t k = 0; k < sn.size(); ++k) {
    Req* q = sn[k].first;
    const ServeNet& b = ln->h_sn_back[slot][k];
    if (b.iv && b.t_last > b.t_first) {
      const double us = 1e-3 * (double)(b.t_last - b.t_first) / b.iv;
      q->iv_us = q->iv_us > 0 ? 0.5 * (q->iv_us + us) : us;
    }
    if (timeout) q->fail_code = SNN_E_TIMEOUT;
  }
  if (timeout) {
    // the nets of that step leave the batch and retire as failed
    std::vector<Req*> keep;
    std::vector<int> keep_steps;
    for (size_t k = 0; k < ln->active.size(); ++k) {
      Req* q = ln->active[k];
      if (q->fail_code) {
        cudaEvent_t e = nullptr;
        SCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        SCK(cudaEventRecord(e, ln->stream));
        ln->retiring.emplace_back(q, e);
      } else {
        keep.push_back(q);
        keep_steps.push_back(ln->active_steps[k]);
      }
    }
    ln->active.swap(keep);
    ln->active_steps.swap(keep_steps);
    ln->dirty = true;
  } else if (ln->t_last > 0) {
    tune_step_length(ln, ms);
  }
  sn.clear();
  return SNN_OK;
}

// Persistent mode: one step = one launch of the persistent kernel that runs
// every net's next intervals: as many as fit the target step time at the
// net's measured time per interval (so small nets take many intervals while
// a large net takes a few), all of one length (a net's last, shorter
// interval runs alone in its step).  Nothing here waits for the GPU.
int lane_step_persistent(snn_server* sv, Lane* ln, bool* launched) {
  *launched = false;
  int rc;
  if ((rc = drop_cancelled(sv, ln)) != SNN_OK) return rc;
  if ((rc = retire_done(sv, ln)) != SNN_OK) return rc;
  bool reuse_done = true;
  for (int k = 0; k < 2; ++k) {
    const int slot = ln->ev_cur ^ k;
    bool done = true;
    if ((rc = fold_persistent(sv, ln, slot, &done)) != SNN_OK) return rc;
    if (k == 0) reuse_done = done;
  }
  if (!reuse_done) return SNN_OK;
  if (ln->active.empty()) {
    ln->t_last = 0;
    return SNN_OK;
  }
  const size_t n = ln->active.size();
  SREQ(n <= kServeMaxNets, SNN_E_STATE, "more than %d running nets",
       (int)kServeMaxNets);
  std::vector<uint32_t> iv(n);
  for (size_t k = 0; k < n; ++k) {
    const Req& q = *ln->active[k];
    const int D = q.net->interval;
    int next = D;
    if (q.steps_left < D) {
      iv[k] = 1;
      next = (int)q.steps_left;
    } else {
      const double est = q.iv_us > 0 ? q.iv_us
                                     : 20.0 + 40.0 * (double)q.net->n_syn / 1.27e9;
      const double want = std::max(1.0, std::floor(ln->step_us / est + 0.5));
      iv[k] = (uint32_t)std::min<double>(want, (double)(q.steps_left / D));
    }
    if (ln->active_steps[k] != next) {
      ln->active_steps[k] = next;
      ln->dirty = true;
    }
  }
  if (ln->dirty) {
    bool busy = false;
    if ((rc = rebuild_tables(ln, &busy)) != SNN_OK) return rc;
    if (busy) return SNN_OK;
  }
  LaneTables& tb = ln->tab[ln->cur];
  if (n > ln->cap_sn) {
    pool_free(ln->d_sn, ln->stream);
    ln->d_sn = nullptr;
    ln->cap_sn = 0;
    SCK(pool_alloc(reinterpret_cast<void**>(&ln->d_sn), kServeMaxNets * sizeof(ServeNet),
                   ln->stream));
    ln->cap_sn = kServeMaxNets;
  }
  const int slot = ln->ev_cur;
  ServeNet* h = ln->h_sn[slot];
  auto& sn = ln->step_nets[slot];
  sn.clear();
  for (size_t k = 0; k < n; ++k) {
    ServeNet e{};
    e.ub = tb.ub[k];
    e.nt = tb.nt[k];
    e.iv = iv[k];
    e.n_items = iv[k] * (e.ub + e.nt);
    h[k] = e;
    sn.emplace_back(ln->active[k], iv[k]);
  }
  SCK(cudaMemcpyAsync(ln->d_sn, h, n * sizeof(ServeNet), cudaMemcpyHostToDevice,
                      ln->stream));
  SCK(cudaMemsetAsync(ln->d_ctl, 0, sizeof(ServeCtl), ln->stream));
  SCK(cudaEventRecord(ln->ev[slot][0], ln->stream));
  // while a large build runs, some SMs stay free for its kernels (small
  // builds run at a higher priority and need no reserve)
  const int ctas =
      std::max(1, sv->sms - (sv->building_large.load() ? kBuildReserveSms : 0));
  SCK(launch_serve(sv->fmt, tb.d_nets, ln->d_sn, ln->d_ctl, (uint32_t)n,
                   (uint32_t)ctas, tb.dsmem, sv->spin_limit, ln->stream));
  SCK(cudaMemcpyAsync(ln->h_sn_back[slot], ln->d_sn, n * sizeof(ServeNet),
                      cudaMemcpyDeviceToHost, ln->stream));
  SCK(cudaMemcpyAsync(ln->h_ctl[slot], ln->d_ctl, sizeof(ServeCtl),
                      cudaMemcpyDeviceToHost, ln->stream));
  SCK(cudaEventRecord(ln->ev[slot][1], ln->stream));
  if (!tb.last_use) SCK(cudaEventCreateWithFlags(&tb.last_use, cudaEventDisableTiming));
  SCK(cudaEventRecord(tb.last_use, ln->stream));
  tb.used = true;
  ln->ev_pending[slot] = true;
  ln->ev_m[slot] = 1;
  ln->ev_cur ^= 1;
  if (ln->t_last == 0) ln->t_last = now_s();
  ln->steps += 1;
  ln->launches += 1;
  *launched = true;
  // bookkeeping: intervals counted, finished nets retire after this step
  std::vector<Req*> keep;
  std::vector<int> keep_steps;
  bool any_done = false;
  for (size_t k = 0; k < n; ++k) {
    Req& q = *ln->active[k];
    ln->intervals += iv[k];
    q.steps_left -= (int64_t)iv[k] * ln->active_steps[k];
    if (q.steps_left <= 0) {
      cudaEvent_t e = nullptr;
      if (!ln->spare_events.empty()) {
        e = ln->spare_events.back();
        ln->spare_events.pop_back();
      } else {
        SCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      }
      SCK(cudaEventRecord(e, ln->stream));
      ln->retiring.emplace_back(ln->active[k], e);
      any_done = true;
    } else {
      keep.push_back(ln->active[k]);
      keep_steps.push_back(ln->active_steps[k]);
    }
  }
  if (any_done) {
    ln->active.swap(keep);
    ln->active_steps.swap(keep_steps);
    ln->dirty = true;
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
  pool_hold(sv->device, +1);
  sv->holds_pool = true;
  cudaDeviceGetAttribute(&sv->sms, cudaDevAttrMultiProcessorCount, sv->device);
  if (sv->sms < 1) sv->sms = 1;
  {
    // map the pool's memory up front (an allocation of the budget, freed at
    // once, stays in the pool): growing it later, while requests are built,
    // maps memory under the driver's locks and stalls the stepping thread's
    // launches for the duration
    const uint64_t warm = std::min<uint64_t>(mem_budget, kPoolWarmBytes);
    void* p = nullptr;
    if (pool_alloc(&p, warm, nullptr) == cudaSuccess) {
      pool_free(p, nullptr);
      cudaStreamSynchronize(nullptr);
    } else {
      cudaGetLastError();
    }
  }
  // smaller nets get higher stream priority: when SMs free up, the CTA
  // scheduler serves the short intervals of small nets first and the large
  // nets take the remaining capacity
  int prio_least = 0, prio_greatest = 0;
  cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  // (the builders take the least priority; every lane is above it)
  const int lane_least = prio_greatest < prio_least ? prio_least - 1 : prio_least;
  for (int k = 0; k < kLanes; ++k) {
    Lane& ln = sv->lanes[k];
    const int prio = prio_greatest + (lane_least - prio_greatest) * k / (kLanes - 1);
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
    if (k == 0) {
      // persistent-mode records (page-locked: copied asynchronously)
      for (int sl = 0; sl < 2; ++sl)
        if (cudaHostAlloc(&ln.h_sn[sl], kServeMaxNets * sizeof(ServeNet), 0) != cudaSuccess ||
            cudaHostAlloc(&ln.h_sn_back[sl], kServeMaxNets * sizeof(ServeNet), 0) != cudaSuccess ||
            cudaHostAlloc(&ln.h_ctl[sl], sizeof(ServeCtl), 0) != cudaSuccess) {
          snn_server_destroy(sv);
          return sfail(SNN_E_OOM, "page-locked host allocation failed");
        }
      if (pool_alloc(reinterpret_cast<void**>(&ln.d_ctl), sizeof(ServeCtl), ln.stream) !=
          cudaSuccess) {
        snn_server_destroy(sv);
        return sfail(SNN_E_OOM, "device allocation failed");
      }
    }
  }
  sv->builder[0] = std::thread(builder_main, sv, 0);
  sv->builder[1] = std::thread(builder_main, sv, 1);
  *out = sv;
  return SNN_OK;
}

int snn_server_set_option(snn_server* sv, int32_t option, double value) {
  SREQ(sv, SNN_E_ARG, "null server");
  switch (option) {
    case SNN_SERVE_OPT_PERSISTENT: {
      std::lock_guard<std::mutex> lk(sv->mu);
      bool idle = sv->ready.empty();
      for (const Lane& ln : sv->lanes)
        idle = idle && ln.active.empty() && ln.retiring.empty();
      SREQ(idle, SNN_E_STATE, "the serving mode changes only while no net runs");
      SREQ(value == 0 || value == 1, SNN_E_ARG, "persistent must be 0 or 1");
      sv->persistent = value != 0;
      if (sv->persistent) sv->exclusive = false;
      return SNN_OK;
    }
    case SNN_SERVE_OPT_EXCLUSIVE: {
      std::lock_guard<std::mutex> lk(sv->mu);
      bool idle = sv->ready.empty();
      for (const Lane& ln : sv->lanes)
        idle = idle && ln.active.empty() && ln.retiring.empty() &&
               ln.x_inflight.empty();
      SREQ(idle, SNN_E_STATE, "the serving mode changes only while no net runs");
      SREQ(value == 0 || value == 1, SNN_E_ARG, "exclusive must be 0 or 1");
      sv->exclusive = value != 0;
      if (sv->exclusive) sv->persistent = false;
      return SNN_OK;
    }
    case SNN_SERVE_OPT_SPIN_LIMIT:
      SREQ(value >= 1 && value <= 1e15, SNN_E_ARG, "spin limit out of range");
      sv->spin_limit = (unsigned long long)value;
      return SNN_OK;
    case SNN_SERVE_OPT_STEP_US:
      SREQ(value >= 0 && value <= 1e6, SNN_E_ARG, "step length out of range");
      sv->step_us_fixed = value;
      for (Lane& ln : sv->lanes) {
        if (value > 0) {
          ln.step_us = value;
          ln.st_tuned = 1;
        } else {
          ln.st_tuned = 0;
          ln.st_idx = 0;
          ln.st_count = 0;
          ln.step_us = kStepUsCandidates[0];
        }
      }
      return SNN_OK;
    default:
      return sfail(SNN_E_ARG, "unknown server option %d", option);
  }
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
  // (exclusive mode: the single-net tiles, about one per SM, for a net that
  // runs alone)
  if (q.r.params.tile_width == 0 && !sv->exclusive)
    q.r.params.tile_width = serve_tile_width(q.r, sv->persistent);
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
      if (q->cancel) {  // cancelled after its build: nothing launched yet
        snn_destroy(q->net);
        q->net = nullptr;
        sv->used -= q->est;
        q->res.state = SNN_REQ_CANCELLED;
        q->res.t_done = now_s() - sv->t0;
        sv->cv.notify_all();
        continue;
      }
      q->res.state = SNN_REQ_RUNNING;
      q->res.t_start = now_s() - sv->t0;
      Lane& ln = sv->lanes[sv->persistent || sv->exclusive ? 0 : lane_of(q->net)];
      // (smallest nets first: the persistent kernel serves them first)
      size_t at = ln.active.size();
      if (sv->persistent)
        while (at > 0 && ln.active[at - 1]->net->n_syn > q->net->n_syn) --at;
      ln.active.insert(ln.active.begin() + at, q);
      ln.active_steps.insert(ln.active_steps.begin() + at, -1);
      ln.dirty = true;
    }
    sv->ready.clear();
  }
  bool any = false;
  int32_t act = 0;
  for (int k = 0; k < kLanes; ++k) {
    bool launched = false;
    int rc = sv->persistent ? (k == 0 ? lane_step_persistent(sv, &sv->lanes[k], &launched)
                                      : SNN_OK)
             : sv->exclusive ? (k == 0 ? lane_step_exclusive(sv, &sv->lanes[k], &launched)
                                       : SNN_OK)
                             : lane_step(sv, &sv->lanes[k], &launched);
    if (rc != SNN_OK) return rc;
    any = any || launched;
    act += (int32_t)(sv->lanes[k].active.size() + sv->lanes[k].retiring.size());
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
           it->second.res.state == SNN_REQ_FAILED ||
           it->second.res.state == SNN_REQ_CANCELLED,
       SNN_E_STATE, "request not finished");
  sv->reqs.erase(it);
  return SNN_OK;
}

int snn_server_cancel(snn_server* sv, uint64_t id) {
  SREQ(sv, SNN_E_ARG, "null server");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(id);
  SREQ(it != sv->reqs.end(), SNN_E_ARG, "unknown request %llu",
       (unsigned long long)id);
  Req& q = it->second;
  const int st = q.res.state;
  SREQ(st == SNN_REQ_QUEUED || st == SNN_REQ_BUILDING || st == SNN_REQ_RUNNING,
       SNN_E_STATE, "request %llu already ended", (unsigned long long)id);
  SREQ(!q.cancel, SNN_E_STATE, "request %llu already cancelled",
       (unsigned long long)id);
  q.cancel = true;
  if (st == SNN_REQ_QUEUED) {
    for (auto& qu : sv->queue) {
      auto pos = std::find(qu.begin(), qu.end(), id);
      if (pos != qu.end()) qu.erase(pos);
    }
    q.res.state = SNN_REQ_CANCELLED;
    q.res.t_done = now_s() - sv->t0;
    sv->cv.notify_all();
  }
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
    out->active += ln.active.size() + ln.retiring.size();
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
  if (sv->persistent || sv->exclusive) {
    // one lane; its intervals per launch on average, and the step tuner
    const Lane& ln = sv->lanes[0];
    out->intervals_per_step =
        ln.steps ? (int32_t)((ln.intervals + ln.steps / 2) / ln.steps) : 0;
    out->tuned = sv->exclusive ? 1 : ln.st_tuned;
  }
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
    for (LaneTables& t : ln.tab) {
      for (cudaGraphExec_t g : t.graph)
        if (g) cudaGraphExecDestroy(g);
      if (t.last_use) cudaEventDestroy(t.last_use);
      if (ln.stream) {
        pool_free(t.d_nets, ln.stream);
        pool_free(t.d_umap, ln.stream);
        pool_free(t.d_dmap, ln.stream);
      }
    }
    for (auto& fe : ln.retiring) cudaEventDestroy(fe.second);
    for (auto& x : ln.x_inflight) {
      cudaEventDestroy(x.e0);
      cudaEventDestroy(x.e1);
    }
    for (cudaEvent_t e : ln.x_spare) cudaEventDestroy(e);
    for (int sl = 0; sl < 2; ++sl) {
      if (ln.h_sn[sl]) cudaFreeHost(ln.h_sn[sl]);
      if (ln.h_sn_back[sl]) cudaFreeHost(ln.h_sn_back[sl]);
      if (ln.h_ctl[sl]) cudaFreeHost(ln.h_ctl[sl]);
    }
    if (ln.stream) {
      pool_free(ln.d_sn, ln.stream);
      pool_free(ln.d_ctl, ln.stream);
    }
    for (cudaEvent_t e : ln.spare_events) cudaEventDestroy(e);
    for (auto& pair : ln.ev)
      for (cudaEvent_t e : pair)
        if (e) cudaEventDestroy(e);
    if (ln.stream) {
      cudaStreamSynchronize(ln.stream);
      if (ln.own_stream) cudaStreamDestroy(ln.stream);
    }
  }
  if (sv->holds_pool) pool_hold(sv->device, -1);
  delete sv;
  return SNN_OK;
}

}  // extern "C"
