// snn_api.cu -- host side of the libsnn C ABI (declared in include/snn.h).
//
// Owns every device allocation of a net, drives the construction pipeline
// (snn_build.cu) and the interval loop update -> deliver (snn_kernels.cu),
// captures full intervals into CUDA graphs, and implements the read-back,
// state and statistics calls.
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "snn_internal.cuh"

using namespace snn;

namespace snn {
// (snn_probe.cu)
cudaError_t launch_red_probe(float* buf, uint32_t n_cells, uint64_t n_ops,
                             int pattern, cudaStream_t s);
}  // namespace snn

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(call)                                                            \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess)                                                  \
      return fail(e_ == cudaErrorMemoryAllocation ? SNN_E_OOM : SNN_E_CUDA, \
                  "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),   \
                  __FILE__, __LINE__);                                      \
  } while (0)

#define REQ(cond, code, ...)                  \
  do {                                        \
    if (!(cond)) return fail(code, __VA_ARGS__); \
  } while (0)

constexpr int kGraphIntervals = 8;
constexpr size_t kTileSmemBudget = 200 * 1024;  // accumulator bytes per CTA

// ---------------------------------------------------------------------------
// Neuron constants, computed in FP64.
// ---------------------------------------------------------------------------
// exp(M) of a 3x3 matrix by scaling and squaring with a Taylor series.
void expm3(const double A[3][3], double E[3][3]) {
  double norm = 0;
  for (int c = 0; c < 3; ++c) {
    double s = 0;
    for (int r = 0; r < 3; ++r) s += fabs(A[r][c]);
    norm = std::max(norm, s);
  }
  int sq = 0;
  while (norm / ldexp(1.0, sq) > 0.25) ++sq;
  double B[3][3], T[3][3], S[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      B[r][c] = ldexp(A[r][c], -sq);
      T[r][c] = (r == c) ? 1.0 : 0.0;   // current term B^k / k!
      S[r][c] = T[r][c];
    }
  for (int k = 1; k < 30; ++k) {
    double N[3][3] = {};
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        double acc = 0;
        for (int q = 0; q < 3; ++q) acc += T[r][q] * B[q][c];
        N[r][c] = acc / k;
      }
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        T[r][c] = N[r][c];
        S[r][c] += N[r][c];
      }
  }
  for (int i = 0; i < sq; ++i) {
    double N[3][3] = {};
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        for (int q = 0; q < 3; ++q) N[r][c] += S[r][q] * S[q][c];
    memcpy(S, N, sizeof S);
  }
  memcpy(E, S, sizeof S);
}

// Poisson(lam) inversion thresholds floor(F_k 2^32) for k = 0, 1, ... up to
// the first that reaches 2^32 - 1; that outcome takes the rest of the unit
// interval (its threshold is implicit on the device).  Returns the number of
// outcomes (thresholds + 1), or -1 if more than cap are needed.
int poisson_thresholds(double lam, uint32_t* thr, int cap) {
  double pk = exp(-lam), F = pk;
  for (int k = 0; k < cap; ++k) {
    double T = floor(F * 4294967296.0);
    if (T >= 4294967295.0) return k + 1;
    thr[k] = (uint32_t)T;
    pk *= lam / (double)(k + 1);
    F += pk;
  }
  return -1;
}

int make_upd_const(const snn_params& p, UpdConst* c) {
  memset(c, 0, sizeof *c);
  const double a = 1.0 / p.tau_syn, b = 1.0 / p.tau_m;
  // state (J, I, V): J' = -a J; I' = J - a I; V' = I / C - b V
  double A[3][3] = {{-a * p.h, 0, 0}, {p.h, -a * p.h, 0},
                    {0, p.h / p.c_m, -b * p.h}};
  double E[3][3];
  expm3(A, E);
  c->p11 = (float)E[0][0];
  c->p21 = (float)E[1][0];
  c->p22 = (float)E[1][1];
  c->p31 = (float)E[2][0];
  c->p32 = (float)E[2][1];
  c->p33 = (float)E[2][2];
  c->psc = (float)(M_E / p.tau_syn);
  c->v_th = (float)p.v_th;
  c->v_reset = (float)p.v_reset;
  c->w_ext = (float)p.w_ext;
  c->refr_steps = (int)llround(p.t_ref / p.h);
  c->seed = p.seed;
  c->n_thr = 0;
  if (p.nu_ext > 0.0 && p.w_ext != 0.0) {
    int n = poisson_thresholds(p.nu_ext * p.h * 1e-3, c->thr, kMaxPoisson);
    if (n < 0) return -1;
    c->n_thr = n;
    for (int j = 0; j < 256; ++j) {
      const uint32_t lo = (uint32_t)j << 24;
      int k = 0;
      while (k < n - 1 && c->thr[k] <= lo) ++k;
      c->guide[j] = (uint8_t)k;
    }
  }
  return 0;
}

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

}  // namespace

#include "snn_net.cuh"

void snn::set_last_error(const char* msg) { g_err = msg; }

namespace {

// Device memory of the library comes from one stream-ordered pool per
// device (allocations and frees are ordered on the net's stream, so freeing
// never synchronises the device); freed blocks stay in the pool for the next
// net and are returned to the device when the last net is destroyed.
struct DevicePools {
  std::mutex mu;
  cudaMemPool_t pool[64] = {};
  int live[64] = {};
};
DevicePools& pools() {
  static DevicePools p;
  return p;
}

cudaMemPool_t device_pool(int dev) {
  if (dev < 0 || dev >= 64) return nullptr;
  DevicePools& P = pools();
  std::lock_guard<std::mutex> lk(P.mu);
  if (!P.pool[dev]) {
    cudaMemPoolProps pr;
    memset(&pr, 0, sizeof pr);
    pr.allocType = cudaMemAllocationTypePinned;
    pr.handleTypes = cudaMemHandleTypeNone;
    pr.location.type = cudaMemLocationTypeDevice;
    pr.location.id = dev;
    cudaMemPool_t mp = nullptr;
    if (cudaMemPoolCreate(&mp, &pr) != cudaSuccess) return nullptr;
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &keep);
    P.pool[dev] = mp;
  }
  return P.pool[dev];
}

// Nets (and servers, which hold the pool for their lifetime) alive per
// device; the pool's unused memory goes back to the device when the count
// reaches zero.  The wait and the trim happen outside the lock, so that
// other threads' allocations never queue behind them (a trim releases only
// unused memory and may run beside allocations).
void count_net(int dev, int delta, cudaStream_t s) {
  if (dev < 0 || dev >= 64) return;
  DevicePools& P = pools();
  cudaMemPool_t trim = nullptr;
  {
    std::lock_guard<std::mutex> lk(P.mu);
    P.live[dev] += delta;
    if (P.live[dev] == 0) trim = P.pool[dev];
  }
  if (trim) {
    cudaStreamSynchronize(s);  // its frees are done
    cudaMemPoolTrimTo(trim, 0);
  }
}

}  // namespace

// Host-side fault injection (snn_debug_fail_allocations): after g_fail_after
// more allocations succeed, the next g_fail_count fail.
std::atomic<long long> g_fail_after{-1};
std::atomic<long long> g_fail_count{0};

bool injected_failure() {
  long long a = g_fail_after.load(std::memory_order_relaxed);
  while (a > 0) {
    if (g_fail_after.compare_exchange_weak(a, a - 1)) return false;
  }
  if (a < 0) return false;
  long long c = g_fail_count.load(std::memory_order_relaxed);
  while (c > 0) {
    if (g_fail_count.compare_exchange_weak(c, c - 1)) return true;
  }
  return false;
}

cudaError_t snn::pool_alloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (injected_failure()) return cudaErrorMemoryAllocation;
  if (bytes == 0) bytes = 16;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaMemPool_t mp = device_pool(dev);
  if (!mp) return cudaErrorMemoryAllocation;
  return cudaMallocFromPoolAsync(p, bytes, mp, s);
}

void snn::pool_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

void snn::pool_hold(int dev, int delta) { count_net(dev, delta, nullptr); }

namespace {

template <class T>
cudaError_t dalloc(T** p, size_t bytes, cudaStream_t s) {
  return snn::pool_alloc(reinterpret_cast<void**>(p), bytes, s);
}

void dfree(void* p, cudaStream_t s) { snn::pool_free(p, s); }

cudaMemcpyKind kind_to(int mem) {
  return mem == SNN_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
}
cudaMemcpyKind kind_from(int mem) {
  return mem == SNN_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
}

int check_mem(int mem) {
  return mem == SNN_MEM_HOST || mem == SNN_MEM_DEVICE;
}

int set_device(snn_net* net) {
  CK(cudaSetDevice(net->device));
  return SNN_OK;
}

// Tile geometry for the tiled delivery: the fewest tiles that are a
// multiple of the SM count and whose ring-buffer window (window steps x
// tile width cells of two int32 accumulators) fits the shared-memory budget.  The sort key holds the
// tile and the position in it in 24 bits; when a non-power-of-two width
// would not fit them, the width is rounded up to a power of two.
// per_target: shared-memory bytes a tile needs per target beyond its
// accumulator (the post-spike rings of a plastic net)
// acc_words: int32 words per accumulator cell (1 or 2).
void choose_tiles(uint32_t n, int window, int32_t hint, size_t per_target,
                  int acc_words, uint32_t* tile_w, int* lo_bits,
                  uint32_t* n_tiles) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms < 1) sms = 1;
  const uint64_t tw_max = std::max<uint64_t>(
      32, kTileSmemBudget /
              (4ull * acc_words * std::max(window, 1) + per_target));
  uint64_t tw = n;
  for (uint64_t k = 1; k <= 4096; ++k) {
    tw = (n + k * sms - 1) / (k * sms);
    if (tw <= tw_max) break;
  }
  if (hint > 0) tw = std::min<uint64_t>((uint64_t)hint, tw_max);
  tw = std::max<uint64_t>(tw, std::min<uint64_t>(64, n));
  tw = std::min<uint64_t>(tw, n);
  int lb = 1;
  while ((1ull << lb) < tw) ++lb;
  uint64_t nt = (n + tw - 1) / tw;
  if (nt > (1ull << (24 - lb))) {
    tw = 1ull << lb;
    nt = (n + tw - 1) / tw;
  }
  *tile_w = (uint32_t)tw;
  *lo_bits = lb;
  *n_tiles = (uint32_t)nt;
}

// Plastic nets: a tile of excitatory targets applies the weight rule to its
// E->E events, about four times the work of a static tile of the same width
// on the benchmark network, and every tile takes a whole SM.  The static
// tiles after the plastic ones therefore go kStaticTilesPerCta to a CTA, and
// the width becomes the smallest in [max(64, ceil(n_exc / SMs)), chosen
// width] whose CTAs still fit one wave, so that the plastic tiles are as
// narrow as the SM count allows.  Nets already needing more than one wave
// keep their geometry, one tile per CTA.
constexpr uint32_t kStaticTilesPerCta = 4;
void balance_plastic_tiles(uint32_t n, uint32_t n_exc, uint32_t* tile_w,
                           int* lo_bits, uint32_t* n_tiles, uint32_t* pl_tiles,
                           uint32_t* tile_grp) {
  const uint32_t tw0 = *tile_w;
  *pl_tiles = std::min<uint32_t>(*n_tiles, (n_exc + tw0 - 1) / tw0);
  *tile_grp = 1;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms < 1 || n_exc == 0 || n_exc >= n) return;
  const uint32_t k = kStaticTilesPerCta;
  for (uint64_t tw = std::min<uint64_t>(std::max<uint64_t>(64, (n_exc + sms - 1) / sms), tw0);
       tw <= tw0; ++tw) {
    const uint64_t nt = (n + tw - 1) / tw, pt = (n_exc + tw - 1) / tw;
    if (pt + (nt - pt + k - 1) / k > (uint64_t)sms) continue;
    int lb = 1;
    while ((1ull << lb) < tw) ++lb;
    if (nt > (1ull << (24 - lb))) return;  // (the sort key's tile field)
    *tile_w = (uint32_t)tw;
    *lo_bits = lb;
    *n_tiles = (uint32_t)nt;
    *pl_tiles = (uint32_t)pt;
    *tile_grp = k;
    return;
  }
}

}  // namespace

void snn::tile_geometry(uint32_t n, int window, int32_t hint, uint32_t* tile_w,
                        int* lo_bits, uint32_t* n_tiles) {
  choose_tiles(n, window, hint, 0, 2, tile_w, lo_bits, n_tiles);
}

namespace {

// shared-memory bytes per target of the plastic delivery beyond the
// accumulator: spike-time ring, spike count, post trace at each of the
// window's horizons
size_t stdp_bytes_per_target(const snn_net* net, int window) {
  return net->stdp_on ? (size_t)net->stdp.history * 4 + 4 + 4 * (size_t)window : 0;
}

bool use_tiled(const snn_net* net) {
  return net->p.deliver_mode == SNN_DELIVER_TILED && net->n_syn > 0 &&
         net->tile_off &&
         (size_t)net->tile_w *
                 ((size_t)net->window * 4 * net->acc_words +
                  stdp_bytes_per_target(net, net->window)) <=
             kTileSmemBudget;
}

// ---- one-word accumulator cells -----------------------------------------
// The tiled delivery sums x = w 2^(q-s) split as hi = rint(x) and
// lo = rint((x - hi) 2^s).  When every stored weight is a multiple of 2^-g
// and q - s >= g, x is an integer and lo = 0: a cell needs one word.  The
// scales of a launch follow from its event bound E and max|w| (the kernel's
// fix_scale); q - s only grows as E or max|w| shrink, so the bounds of the
// interval lists (E <= max in-degree x spikes per neuron per interval) and
// an upper bound of max|w| give the smallest q - s any interval can get.

// Exponent of the lowest set bit of a nonzero double (exact for the float
// and bfloat16 values the store holds).
int lowbit_exp(double v) {
  int e = 0;
  const double m = frexp(fabs(v), &e);           // |v| = m 2^e, m in [0.5, 1)
  uint64_t i = (uint64_t)ldexp(m, 53);           // integer, exact
  return e - 53 + __builtin_ctzll(i);
}

// The value a weight is stored as.
double stored_weight(double w, int fmt) {
  if (fmt == SNN_W_FP32_12B) return (double)(float)w;
  return (double)bf16_to_f32(bf16_bits_rne(w));
}

// Bounds of the stored weights: every nonzero one is a multiple of 2^g_min
// (g_min = INT_MAX: all zero) and at most w_max in magnitude.
struct WeightBounds {
  int g_min = INT_MAX;
  double w_max = 0.0;
  bool ok = true;  // false: no useful bound (weights may come near zero)
  void add_value(double stored) {
    if (stored == 0.0) return;
    g_min = std::min(g_min, lowbit_exp(stored));
    w_max = std::max(w_max, fabs(stored));
  }
};

// One population of the fixed-in-degree rule: mean + sd z, |z| <= 6.7 for
// the Box-Muller draw of two 32-bit uniforms (u1 >= 2^-32), clipped at 0 on
// the side the rule clips.
void add_population(WeightBounds* b, double mean, double sd, bool clip_neg,
                    bool clip_pos, int fmt) {
  if (sd == 0.0) {
    double x = mean;
    if (clip_neg && x < 0.0) x = 0.0;
    if (clip_pos && x > 0.0) x = 0.0;
    b->add_value(stored_weight(x, fmt));
    return;
  }
  const double span = 6.7 * fabs(sd);
  if (!(fabs(mean) > span)) {  // the draws can come arbitrarily near zero
    b->ok = false;
    return;
  }
  const double lo = (fabs(mean) - span) * (1.0 - 0x1p-7);  // after rounding
  const double hi = (fabs(mean) + span) * (1.0 + 0x1p-7);
  int e = 0;
  frexp(lo, &e);  // 2^(e-1) <= lo: a stored value >= lo has its lowest set
                  // bit at or above 2^(e - 1 - fraction bits)
  b->g_min = std::min(b->g_min, e - 1 - (fmt == SNN_W_FP32_12B ? 23 : 7));
  b->w_max = std::max(b->w_max, hi);
}

// Decide the accumulator cells of a net about to build its store.
void decide_acc_words(snn_net* net, const WeightBounds& b, uint32_t k_in_max,
                      int max_interval) {
  net->acc_words = 2;
  net->acc_qs_min = 0;
  if (net->p.acc_words == 2 || net->stdp_on || !b.ok ||
      net->fmt != SNN_W_BF16_8B)
    return;
  if (b.g_min == INT_MAX) {  // every weight is zero
    net->acc_words = 1;
    return;
  }
  const uint32_t refr = (uint32_t)net->uc.refr_steps;
  const uint64_t spikes = ((uint64_t)max_interval + refr) / (refr + 1u);
  const int qs = fixed_qs_host((uint64_t)k_in_max * std::max<uint64_t>(spikes, 1),
                               b.w_max);
  if (qs >= 0 && qs >= -b.g_min) {
    net->acc_words = 1;
    net->acc_qs_min = -b.g_min;
  }
}

cudaError_t launch_deliver_any(snn_net* net, unsigned long long* pair,
                               unsigned int* done, const SpikeEntry* list,
                               int from_list_range, int advance_time) {
  NetView v = net->view();
  if (use_tiled(net))
    return launch_deliver_tiled(v, pair, done, list, from_list_range,
                                advance_time, net->stream);
  return launch_deliver(v, pair, done, list, advance_time, net->stream);
}

// Build the store from per-row key arrays: host row offsets from the device
// out-degrees, scatter (callback), sort and pack.
template <class Scatter>
int build_store(snn_net* net, uint32_t* d_deg, Scatter scatter,
                const BuildFixed* bf, const double* d_edge_w, int d_lo,
                int d_hi) {
  cudaStream_t s = net->stream;
  const uint32_t n = net->n_src;  // rows: every source of the population
  std::vector<uint32_t> deg(n);
  CK(cudaMemcpyAsync(deg.data(), d_deg, n * sizeof(uint32_t),
                     cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<uint64_t> rp(n + 1, 0);
  uint32_t max_row = 0;
  std::vector<uint32_t> long_rows;
  std::vector<uint64_t> long_off;
  uint64_t scratch = 0;
  for (uint32_t i = 0; i < n; ++i) {
    rp[i + 1] = rp[i] + deg[i];
    max_row = std::max(max_row, deg[i]);
    if (deg[i] > kSortCap) {
      long_rows.push_back(i);
      long_off.push_back(scratch);
      uint64_t P = 1;
      while (P < deg[i]) P <<= 1;
      scratch += P;
    }
  }
  const uint64_t n_syn = rp[n];
  const uint32_t ch = (uint32_t)chunk_records(net->fmt);
  const uint64_t padded = (n_syn + ch - 1) / ch * ch + ch;
  const int rec_bytes = net->fmt == SNN_W_FP32_12B ? 12 : 8;
  CK(dalloc(&net->row_ptr, (n + 1) * sizeof(uint64_t), net->stream));
  CK(cudaMemcpyAsync(net->row_ptr, rp.data(), (n + 1) * sizeof(uint64_t),
                     cudaMemcpyHostToDevice, s));
  // tiles sized for the widest window the interval can reach
  const int iv = net->p.interval ? net->p.interval : d_lo;
  choose_tiles(net->n, iv + (d_hi - d_lo), net->p.tile_width,
               stdp_bytes_per_target(net, iv + (d_hi - d_lo)), net->acc_words,
               &net->tile_w, &net->lo_bits, &net->n_tiles);
  net->pl_tiles = net->n_tiles;
  net->tile_grp = 1;
  if (net->stdp_on && net->p.tile_width == 0)
    balance_plastic_tiles(net->n, net->p.n_exc, &net->tile_w, &net->lo_bits,
                          &net->n_tiles, &net->pl_tiles, &net->tile_grp);
  CK(dalloc(&net->tile_off, (uint64_t)n * (net->n_tiles + 1) * sizeof(uint32_t), net->stream));
  // keys; for 8-byte records the key array becomes the record array
  uint64_t* keys = nullptr;
  CK(dalloc(&keys, padded * sizeof(uint64_t), net->stream));
  uint32_t* cursor = d_deg;  // reuse as the scatter cursor
  CK(cudaMemsetAsync(cursor, 0, n * sizeof(uint32_t), s));
  CK(scatter(net->row_ptr, cursor, keys, net->tile_w, net->lo_bits));
  void* recs = nullptr;
  if (rec_bytes == 8) {
    recs = keys;
  } else {
    cudaError_t e = dalloc(&recs, padded * rec_bytes, net->stream);
    if (e != cudaSuccess) {
      dfree(keys, net->stream);
      return fail(SNN_E_OOM, "store allocation of %llu bytes failed",
                  (unsigned long long)(padded * rec_bytes));
    }
  }
  // zero the padding records once (target 0, weight 0; never delivered)
  CK(cudaMemsetAsync(static_cast<char*>(recs) + n_syn * rec_bytes, 0,
                     (padded - n_syn) * rec_bytes, s));
  uint32_t* d_long = nullptr;
  uint64_t *d_loff = nullptr, *d_scr = nullptr;
  if (!long_rows.empty()) {
    CK(dalloc(&d_long, long_rows.size() * sizeof(uint32_t), net->stream));
    CK(dalloc(&d_loff, long_off.size() * sizeof(uint64_t), net->stream));
    CK(dalloc(&d_scr, scratch * sizeof(uint64_t), net->stream));
    CK(cudaMemcpyAsync(d_long, long_rows.data(),
                       long_rows.size() * sizeof(uint32_t),
                       cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_loff, long_off.data(),
                       long_off.size() * sizeof(uint64_t),
                       cudaMemcpyHostToDevice, s));
  }
  uint32_t* d_stats = nullptr;
  CK(dalloc(&d_stats, 2 * sizeof(uint32_t), net->stream));
  CK(cudaMemsetAsync(d_stats, 0, 2 * sizeof(uint32_t), s));
  CK(build_sort_pack(net->fmt, n, net->row_ptr, keys, recs, bf, d_edge_w,
                     max_row, d_long, (uint32_t)long_rows.size(), d_scr,
                     d_loff, net->tile_w, net->lo_bits, net->n_tiles,
                     net->tile_off, d_stats, s));
  uint32_t h_stats[2] = {0, 0};
  CK(cudaMemcpyAsync(h_stats, d_stats, sizeof h_stats, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  dfree(d_stats, net->stream);
  net->mult_max = h_stats[0];
  memcpy(&net->max_abs_w, &h_stats[1], sizeof(float));
  if (recs != keys) dfree(keys, net->stream);
  dfree(d_long, net->stream);
  dfree(d_loff, net->stream);
  dfree(d_scr, net->stream);
  net->recs = recs;
  net->n_syn = n_syn;
  net->recs_bytes = padded * rec_bytes;
  net->connected = true;
  return SNN_OK;
}

int ensure_ext(snn_net* net, uint64_t n) {
  if (n <= net->ext_cap) return SNN_OK;
  uint64_t cap = std::max<uint64_t>(n, 2 * net->ext_cap);
  dfree(net->ext_list, net->stream);
  dfree(net->ext_src, net->stream);
  dfree(net->ext_t, net->stream);
  net->ext_list = nullptr;
  net->ext_src = nullptr;
  net->ext_t = nullptr;
  net->ext_cap = 0;
  CK(dalloc(&net->ext_list, cap * sizeof(SpikeEntry), net->stream));
  CK(dalloc(&net->ext_src, cap * sizeof(uint32_t), net->stream));
  CK(dalloc(&net->ext_t, cap * sizeof(int32_t), net->stream));
  net->ext_cap = cap;
  return SNN_OK;
}

cudaEvent_t pool_event(snn_net* net, size_t k) {
  while (net->ev.size() <= k) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    net->ev.push_back(e);
  }
  return net->ev[k];
}

// One interval: update (time from the control block) then deliver.
int launch_interval(snn_net* net, int steps) {
  NetView v = net->view();
  CK(launch_update(v, net->uc, steps, 1, 0, net->stream));
  CK(launch_deliver_any(net, &net->ctl->pair, &net->ctl->done, net->list, 0,
                        1));
  net->launches += 2;
  net->upd_launches += 1;
  net->del_launches += 1;
  return SNN_OK;
}

// kGraphIntervals intervals captured as one graph.  prof: the profiling form,
// with an event recorded (as a graph node) before each update, between it and
// its delivery, and after the delivery (events 3k, 3k+1, 3k+2), so that the
// kernels are timed in the launch context of the production graph.
int capture_graph(snn_net* net, bool prof) {
  cudaGraphExec_t* out = prof ? &net->graph_prof : &net->graph;
  if (*out) return SNN_OK;
  if (prof)
    for (int k = 0; k < 3 * kGraphIntervals; ++k)
      REQ(pool_event(net, (size_t)k), SNN_E_CUDA, "event creation failed");
  cudaGraph_t g;
  CK(cudaStreamBeginCapture(net->stream, cudaStreamCaptureModeThreadLocal));
  NetView v = net->view();
  for (int k = 0; k < kGraphIntervals; ++k) {
    cudaError_t e0 = cudaSuccess, e3 = cudaSuccess, e4 = cudaSuccess;
    if (prof)
      e0 = cudaEventRecordWithFlags(net->ev[3 * k], net->stream,
                                    cudaEventRecordExternal);
    cudaError_t e1 = launch_update(v, net->uc, net->interval, 1, 0, net->stream);
    if (prof)
      e3 = cudaEventRecordWithFlags(net->ev[3 * k + 1], net->stream,
                                    cudaEventRecordExternal);
    cudaError_t e2 = launch_deliver_any(net, &net->ctl->pair, &net->ctl->done,
                                        net->list, 0, 1);
    if (prof)
      e4 = cudaEventRecordWithFlags(net->ev[3 * k + 2], net->stream,
                                    cudaEventRecordExternal);
    const cudaError_t e = e0 != cudaSuccess ? e0 : e1 != cudaSuccess ? e1
                        : e2 != cudaSuccess ? e2 : e3 != cudaSuccess ? e3 : e4;
    if (e != cudaSuccess) {
      cudaStreamEndCapture(net->stream, &g);
      return fail(SNN_E_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    }
  }
  CK(cudaStreamEndCapture(net->stream, &g));
  cudaError_t e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  CK(e);
  return SNN_OK;
}

// Captured graphs hold the net's view and constants: drop them when those
// change.
void drop_graphs(snn_net* net) {
  if (net->graph) cudaGraphExecDestroy(net->graph);
  if (net->graph_prof) cudaGraphExecDestroy(net->graph_prof);
  net->graph = nullptr;
  net->graph_prof = nullptr;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
// Bounds-checked builds: nets seen with SNN_ERRF_CHECK (counted once each).
static std::atomic<uint64_t> g_check_failures{0};
static void note_check_failure(snn_net* net, unsigned flags) {
  if (kChecked && (flags & SNN_ERRF_CHECK) && !net->check_noted) {
    net->check_noted = true;
    g_check_failures.fetch_add(1, std::memory_order_relaxed);
  }
}

extern "C" {

int snn_abi_version(void) { return SNN_ABI_VERSION; }

int snn_debug_fail_allocations(int64_t after, int64_t count) {
  REQ(count >= 0, SNN_E_ARG, "negative count");
  g_fail_count.store(count);
  g_fail_after.store(after < 0 ? -1 : after);
  return SNN_OK;
}

const char* snn_last_error(void) { return g_err.c_str(); }

int snn_default_params(snn_params* p) {
  REQ(p, SNN_E_ARG, "null params");
  memset(p, 0, sizeof *p);
  p->n_exc = 1000;
  p->n_inh = 250;
  p->h = 0.1;
  p->tau_m = 10.0;
  p->c_m = 250.0;
  p->v_th = 20.0;
  p->v_reset = 0.0;
  p->t_ref = 2.0;
  p->tau_syn = 0.5;
  p->nu_ext = 0.0;
  p->w_ext = 0.0;
  p->seed = 1;
  p->weight_format = SNN_W_FP32_12B;
  p->n_slots = 32;
  p->interval = 0;
  p->init_v_random = 1;
  p->count_events = 0;
  p->spike_log_capacity = 0;
  return SNN_OK;
}

int snn_psc_weight_for_psp(const snn_params* p, double psp_mv, double* w_pa) {
  REQ(p && w_pa, SNN_E_ARG, "null argument");
  REQ(p->tau_syn > 0 && p->tau_m > 0 && p->c_m > 0 && p->tau_syn != p->tau_m,
      SNN_E_ARG, "bad time constants");
  // Membrane response to a unit PSC: (e/tau_s)/C * f(t)/c^2 with
  // f(t) = e^{-bt} - e^{-at}(1 + ct), a = 1/tau_s, b = 1/tau_m, c = a - b.
  // Its maximum solves b e^{ct} = b + a c t (t > 0): g(t) = b e^{ct} - b -
  // a c t is negative just after 0 and grows without bound; bisect it.
  const double a = 1.0 / p->tau_syn, b = 1.0 / p->tau_m, c = a - b;
  auto g = [&](double t) { return b * expm1(c * t) - a * c * t; };
  double lo = 1e-12 * p->tau_syn, hi = 1e-3 * p->tau_syn;
  while (g(hi) < 0.0) hi *= 2.0;
  for (int it = 0; it < 400 && hi - lo > 1e-15 * hi; ++it) {
    double mid = 0.5 * (lo + hi);
    if (g(mid) < 0.0) lo = mid; else hi = mid;
  }
  const double t = 0.5 * (lo + hi);
  const double f = exp(-b * t) - exp(-a * t) * (1.0 + c * t);
  const double peak = (M_E / p->tau_syn) / p->c_m * f / (c * c);
  *w_pa = psp_mv / peak;
  return SNN_OK;
}

int snn_create(const snn_params* p, void* stream, snn_net** out) {
  REQ(p && out, SNN_E_ARG, "null argument");
  *out = nullptr;
  const uint64_t n = (uint64_t)p->n_exc + p->n_inh;
  REQ(n >= 1 && n < (1u << 24), SNN_E_ARG, "N = %llu outside [1, 2^24)",
      (unsigned long long)n);
  REQ(p->h > 0 && p->tau_m > 0 && p->c_m > 0 && p->tau_syn > 0 &&
          p->tau_syn != p->tau_m && p->t_ref >= 0 && p->nu_ext >= 0,
      SNN_E_ARG, "bad neuron parameters");
  REQ(p->weight_format == SNN_W_FP32_12B || p->weight_format == SNN_W_BF16_8B,
      SNN_E_ARG, "bad weight format %d", p->weight_format);
  REQ(is_pow2(p->n_slots) && p->n_slots >= 2 && p->n_slots <= 256, SNN_E_ARG,
      "n_slots must be a power of two in [2, 256]");
  REQ(p->interval >= 0 && p->interval <= p->n_slots, SNN_E_ARG,
      "bad interval");
  REQ(p->deliver_mode == SNN_DELIVER_TILED || p->deliver_mode == SNN_DELIVER_ATOMIC,
      SNN_E_ARG, "bad deliver_mode %d", p->deliver_mode);
  REQ(p->tile_width >= 0, SNN_E_ARG, "bad tile_width %d", p->tile_width);
  REQ(p->acc_words == 0 || p->acc_words == 2, SNN_E_ARG,
      "acc_words must be 0 (automatic) or 2, not %d", p->acc_words);
  REQ(p->build_yield == 0 || p->build_yield == 1, SNN_E_ARG,
      "build_yield must be 0 or 1, not %d", p->build_yield);
  const bool part = p->part_hi != 0 || p->part_lo != 0;
  REQ(!part || (p->part_lo < p->part_hi && p->part_hi <= n), SNN_E_ARG,
      "partition [%u, %u) outside [0, %llu)", p->part_lo, p->part_hi,
      (unsigned long long)n);
  const uint64_t n_loc = part ? (uint64_t)(p->part_hi - p->part_lo) : n;
  snn_net* net = new snn_net();
  net->p = *p;
  net->n = (uint32_t)n_loc;
  net->n_src = (uint32_t)n;
  net->g0 = part ? p->part_lo : 0u;
  net->pitch = (uint32_t)((n_loc + 31) / 32 * 32);
  net->fmt = p->weight_format;
  net->n_slots = p->n_slots;
  if (make_upd_const(*p, &net->uc) != 0) {
    delete net;
    return fail(SNN_E_ARG, "Poisson drive rate too high for the inversion table");
  }
  int rc = SNN_OK;
  auto bail = [&](int code) {
    snn_destroy(net);
    return code;
  };
  if (cudaGetDevice(&net->device) != cudaSuccess)
    return bail(fail(SNN_E_CUDA, "no CUDA device"));
  count_net(net->device, +1, nullptr);
  net->counted = true;
  if (stream) {
    net->stream = static_cast<cudaStream_t>(stream);
  } else {
    // a blocking stream stays ordered with the legacy default stream and,
    // unlike it, can be captured into graphs
    if (cudaStreamCreateWithPriority(&net->stream, cudaStreamDefault,
                                     p->stream_priority) != cudaSuccess)
      return bail(fail(SNN_E_CUDA, "stream creation failed"));
    net->own_stream = true;
  }
  cudaStream_t s = net->stream;
  const size_t rb_bytes = (size_t)net->n_slots * net->pitch * sizeof(float);
#define ALLOC(ptr, bytes)                                                   \
  do {                                                                      \
    if (dalloc(&(ptr), (bytes), net->stream) != cudaSuccess)                  \
      return bail(fail(SNN_E_OOM, "allocation of %zu bytes failed",        \
                       (size_t)(bytes)));                                   \
  } while (0)
  ALLOC(net->V, n * sizeof(float));
  ALLOC(net->I, n * sizeof(float));
  ALLOC(net->J, n * sizeof(float));
  ALLOC(net->refr, n * sizeof(int32_t));
  ALLOC(net->rb, rb_bytes);
  ALLOC(net->ctl, sizeof(Ctl));
  if (p->count_events) ALLOC(net->counts, rb_bytes);
  ALLOC(net->isi_last, n * sizeof(int32_t));
  ALLOC(net->isi_spikes, n * sizeof(uint32_t));
  ALLOC(net->isi_n, n * sizeof(uint32_t));
  ALLOC(net->isi_sum, n * sizeof(double));
  ALLOC(net->isi_sq, n * sizeof(double));
  if (p->spike_log_capacity) {
    ALLOC(net->log_src, p->spike_log_capacity * sizeof(uint32_t));
    ALLOC(net->log_t, p->spike_log_capacity * sizeof(int32_t));
    net->log_cap = p->spike_log_capacity;
  }
#undef ALLOC
  if (cudaMemsetAsync(net->rb, 0, rb_bytes, s) != cudaSuccess ||
      cudaMemsetAsync(net->ctl, 0, sizeof(Ctl), s) != cudaSuccess ||
      (net->counts && cudaMemsetAsync(net->counts, 0, rb_bytes, s) != cudaSuccess))
    return bail(fail(SNN_E_CUDA, "memset failed"));
  if (launch_fill_i32(net->isi_last, kNoSpike, n, s) != cudaSuccess ||
      cudaMemsetAsync(net->isi_spikes, 0, n * sizeof(uint32_t), s) != cudaSuccess ||
      cudaMemsetAsync(net->isi_n, 0, n * sizeof(uint32_t), s) != cudaSuccess ||
      cudaMemsetAsync(net->isi_sum, 0, n * sizeof(double), s) != cudaSuccess ||
      cudaMemsetAsync(net->isi_sq, 0, n * sizeof(double), s) != cudaSuccess)
    return bail(fail(SNN_E_CUDA, "statistics initialisation failed"));
  NetView v = net->view();
  if (launch_init_v(v, &net->uc, p->init_v_random, s) != cudaSuccess)
    return bail(fail(SNN_E_CUDA, "init kernel launch failed"));
  net->launches += 1;
  if ((rc = snn_sync(net)) != SNN_OK) return bail(rc);
  *out = net;
  return SNN_OK;
}

// The build kernels of the calling thread take the net's build_yield shape
// while this object lives.
struct BuildShapeScope {
  explicit BuildShapeScope(const snn_net* net) {
    set_build_yield(net->p.build_yield != 0 ? 1u : 0u);
  }
  ~BuildShapeScope() { set_build_yield(0); }
};

int snn_connect_fixed_indegree(snn_net* net, const snn_conn_params* c) {
  REQ(net && c, SNN_E_ARG, "null argument");
  REQ(!net->connected && !net->finalized, SNN_E_STATE, "net already connected");
  BuildShapeScope confine(net);
  const snn_params& p = net->p;
  REQ(c->d_lo >= 1 && c->d_hi >= c->d_lo && c->d_hi <= net->n_slots &&
          c->d_hi <= 255,
      SNN_E_ARG, "delays [%d, %d] outside [1, min(n_slots, 255)]", c->d_lo,
      c->d_hi);
  REQ(c->k_exc == 0 || p.n_exc > 0, SNN_E_ARG, "k_exc > 0 without E neurons");
  REQ(c->k_inh == 0 || p.n_inh > 0, SNN_E_ARG, "k_inh > 0 without I neurons");
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  BuildFixed b;
  b.n_e = p.n_exc;
  b.n_i = p.n_inh;
  b.k_e = c->k_exc;
  b.k_i = c->k_inh;
  b.w_e = c->w_exc;
  b.w_i = c->w_inh;
  b.sd_e = c->sd_exc;
  b.sd_i = c->sd_inh;
  b.d_lo = c->d_lo;
  b.d_hi = c->d_hi;
  b.seed = c->seed;
  b.clip_e = c->clip_exc;
  b.clip_i = c->clip_inh;
  b.n_tgt = net->n;
  b.tgt0 = net->g0;
  uint32_t* deg = nullptr;
  CK(dalloc(&deg, net->n_src * sizeof(uint32_t), net->stream));
  CK(cudaMemsetAsync(deg, 0, net->n_src * sizeof(uint32_t), net->stream));
  cudaError_t e = build_count_fixed(b, deg, net->stream);
  if (e != cudaSuccess) {
    dfree(deg, net->stream);
    CK(e);
  }
  cudaStream_t s = net->stream;
  {
    WeightBounds wb;
    if (c->k_exc) add_population(&wb, c->w_exc, c->sd_exc, c->clip_exc != 0, false, net->fmt);
    if (c->k_inh) add_population(&wb, c->w_inh, c->sd_inh, false, c->clip_inh != 0, net->fmt);
    decide_acc_words(net, wb, c->k_exc + c->k_inh,
                     net->p.interval ? net->p.interval : c->d_hi);
  }
  rc = build_store(
      net, deg,
      [&](const uint64_t* rp, uint32_t* cur, uint64_t* keys, uint32_t tw,
          int lb) { return build_scatter_fixed(b, rp, cur, keys, tw, lb, s); },
      &b, nullptr, c->d_lo, c->d_hi);
  dfree(deg, net->stream);
  net->launches += 3;
  net->k_in_max = c->k_exc + c->k_inh;
  return rc;
}

int snn_connect_edges(snn_net* net, const uint32_t* src, const uint32_t* tgt,
                      const uint8_t* delay, const double* w, uint64_t n,
                      int mem) {
  REQ(net && net->g0 == 0 && net->n == net->n_src, SNN_E_ARG,
      "explicit edge lists are not supported for target partitions");
  REQ(net, SNN_E_ARG, "null net");
  REQ(!net->connected && !net->finalized, SNN_E_STATE, "net already connected");
  REQ(check_mem(mem), SNN_E_ARG, "bad mem kind");
  REQ(n < (1ull << 32), SNN_E_ARG, "too many edges");
  REQ(n == 0 || (src && tgt && delay && w), SNN_E_ARG, "null edge array");
  BuildShapeScope confine(net);
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  cudaStream_t s = net->stream;
  // validate on the host
  std::vector<uint32_t> hs, ht;
  std::vector<uint8_t> hd;
  std::vector<double> hw;
  const uint32_t *ps = src, *pt = tgt;
  const uint8_t* pd = delay;
  const double* pw = w;
  if (mem == SNN_MEM_DEVICE && n) {
    hs.resize(n);
    ht.resize(n);
    hd.resize(n);
    hw.resize(n);
    CK(cudaMemcpyAsync(hs.data(), src, n * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ht.data(), tgt, n * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hd.data(), delay, n, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hw.data(), w, n * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ps = hs.data();
    pt = ht.data();
    pd = hd.data();
    pw = hw.data();
  }
  const int dmax = std::min(net->n_slots, 255);
  int e_lo = 255, e_hi = 1;
  std::vector<uint32_t> indeg(net->n, 0);
  for (uint64_t e = 0; e < n; ++e) {
    e_lo = std::min<int>(e_lo, pd[e]);
    e_hi = std::max<int>(e_hi, pd[e]);
    REQ(ps[e] < net->n && pt[e] < net->n, SNN_E_ARG,
        "edge %llu: index out of range", (unsigned long long)e);
    REQ(pd[e] >= 1 && pd[e] <= dmax, SNN_E_ARG,
        "edge %llu: delay %d outside [1, %d]", (unsigned long long)e,
        (int)pd[e], dmax);
    REQ(isfinite(pw[e]), SNN_E_ARG, "edge %llu: weight not finite",
        (unsigned long long)e);
    ++indeg[pt[e]];
  }
  const uint32_t k_in_max =
      indeg.empty() ? 0u : *std::max_element(indeg.begin(), indeg.end());
  uint32_t *d_src = nullptr, *d_tgt = nullptr, *deg = nullptr;
  uint8_t* d_del = nullptr;
  double* d_w = nullptr;
  CK(dalloc(&d_src, n * 4, net->stream));
  CK(dalloc(&d_tgt, n * 4, net->stream));
  CK(dalloc(&d_del, n, net->stream));
  CK(dalloc(&d_w, n * 8, net->stream));
  CK(dalloc(&deg, net->n * sizeof(uint32_t), net->stream));
  if (n) {
    CK(cudaMemcpyAsync(d_src, ps, n * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_tgt, pt, n * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_del, pd, n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_w, pw, n * 8, cudaMemcpyHostToDevice, s));
  }
  CK(cudaMemsetAsync(deg, 0, net->n * sizeof(uint32_t), s));
  CK(build_count_edges(d_src, n, deg, s));
  {
    WeightBounds wb;
    for (uint64_t e = 0; e < n; ++e) wb.add_value(stored_weight(pw[e], net->fmt));
    decide_acc_words(net, wb, k_in_max, net->p.interval ? net->p.interval : e_hi);
  }
  rc = build_store(
      net, deg,
      [&](const uint64_t* rp, uint32_t* cur, uint64_t* keys, uint32_t tw,
          int lb) {
        return build_scatter_edges(d_src, d_tgt, d_del, n, rp, cur, keys, tw,
                                   lb, s);
      },
      nullptr, d_w, e_lo, e_hi);
  dfree(d_src, net->stream);
  dfree(d_tgt, net->stream);
  dfree(d_del, net->stream);
  dfree(d_w, net->stream);
  dfree(deg, net->stream);
  net->launches += 3;
  net->k_in_max = k_in_max;
  return rc;
}

// Plasticity state of a finalized store (snn_set_stdp): plastic weights
// start at the stored weights; traces and post-spike rings start empty.
int setup_stdp(snn_net* net) {
  REQ(use_tiled(net), SNN_E_ARG,
      "STDP needs the tiled delivery (deliver_mode SNN_DELIVER_TILED, and a "
      "tile that fits shared memory)");
  REQ(net->uc.refr_steps + 1 >= net->interval, SNN_E_ARG,
      "STDP needs at most one spike per neuron per interval: refractory "
      "steps + 1 = %d < interval %d", net->uc.refr_steps + 1, net->interval);
  cudaStream_t s = net->stream;
  const snn_stdp_params& q = net->stdp;
  StdpView& sp = net->sp;
  const uint64_t n = net->n, H = (uint64_t)q.history;
  const uint64_t n_rec = net->recs_bytes / (net->fmt == SNN_W_FP32_12B ? 12 : 8);
  CK(dalloc(&sp.wp, std::max<uint64_t>(n_rec, 1) * sizeof(float), s));
  CK(cudaMemsetAsync(sp.wp, 0, std::max<uint64_t>(n_rec, 1) * sizeof(float), s));
  CK(unpack_store(net->fmt, net->recs, net->n_syn, nullptr, nullptr, sp.wp, s));
  CK(dalloc(&sp.pre_t, n * sizeof(int32_t), s));
  CK(dalloc(&sp.prev_t, n * sizeof(int32_t), s));
  CK(dalloc(&sp.pre_k, n * sizeof(float), s));
  CK(dalloc(&sp.prev_k, n * sizeof(float), s));
  CK(dalloc(&sp.ring_t, H * net->pitch * sizeof(int32_t), s));
  CK(dalloc(&sp.ring_k, H * net->pitch * sizeof(float), s));
  CK(dalloc(&sp.ring_n, n * sizeof(uint32_t), s));
  CK(launch_fill_i32(sp.pre_t, kNoSpike, n, s));
  CK(launch_fill_i32(sp.prev_t, kNoSpike, n, s));
  CK(cudaMemsetAsync(sp.pre_k, 0, n * sizeof(float), s));
  CK(cudaMemsetAsync(sp.prev_k, 0, n * sizeof(float), s));
  CK(cudaMemsetAsync(sp.ring_n, 0, n * sizeof(uint32_t), s));
  CK(cudaMemsetAsync(sp.ring_t, 0, H * net->pitch * sizeof(int32_t), s));
  CK(cudaMemsetAsync(sp.ring_k, 0, H * net->pitch * sizeof(float), s));
  sp.n_exc = net->p.n_exc;
  sp.hist = (uint32_t)H;
  sp.l2_plus = (float)(M_LOG2E * net->p.h / q.tau_plus);
  sp.l2_minus = (float)(M_LOG2E * net->p.h / q.tau_minus);
  sp.c_pot = (float)(q.lambda * pow(q.w0, 1.0 - q.mu));
  sp.c_dep = (float)(q.lambda * q.alpha);
  sp.mu = (float)q.mu;
  sp.w_max = (float)q.w_max;
  // the exact accumulation bounds every delivered weight by max|w|
  net->max_abs_w = std::max(net->max_abs_w, sp.w_max);
  net->launches += 3;
  return SNN_OK;
}

int snn_finalize(snn_net* net) {
  REQ(net, SNN_E_ARG, "null net");
  REQ(!net->finalized, SNN_E_STATE, "already finalized");
  BuildShapeScope confine(net);
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  cudaStream_t s = net->stream;
  if (!net->connected) {
    // a net without synapses: empty store
    CK(dalloc(&net->row_ptr, (net->n_src + 1) * sizeof(uint64_t), net->stream));
    CK(cudaMemsetAsync(net->row_ptr, 0, (net->n_src + 1) * sizeof(uint64_t), s));
    CK(dalloc(&net->recs, 4096, net->stream));
    CK(cudaMemsetAsync(net->recs, 0, 4096, s));
    net->n_syn = 0;
    net->connected = true;
  }
  unsigned* dd = nullptr;
  unsigned h[2] = {0xFFFFFFFFu, 0u};
  CK(dalloc(&dd, 2 * sizeof(unsigned), net->stream));
  CK(cudaMemcpyAsync(dd, h, sizeof h, cudaMemcpyHostToDevice, s));
  CK(delay_range(net->fmt, net->recs, net->n_syn, dd, s));
  CK(cudaMemcpyAsync(h, dd, sizeof h, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  dfree(dd, net->stream);
  net->dmin = net->n_syn ? (int)h[0] : 0;
  net->dmax = net->n_syn ? (int)h[1] : 0;
  int iv = net->p.interval;
  if (iv == 0) iv = net->n_syn ? net->dmin : net->n_slots;
  REQ(iv >= 1 && (net->n_syn == 0 || iv <= net->dmin), SNN_E_ARG,
      "interval %d exceeds the minimum delay %d", iv, net->dmin);
  REQ(net->dmax <= net->n_slots, SNN_E_ARG, "max delay %d exceeds n_slots %d",
      net->dmax, net->n_slots);
  net->interval = iv;
  net->window = net->n_syn ? iv + (net->dmax - net->dmin) : iv;
  // a neuron fires at most once per refractory period plus one step
  net->spikes_per_iv =
      (uint32_t)((iv + net->uc.refr_steps) / (net->uc.refr_steps + 1));
  // a partition also takes the gathered list of the whole population
  net->list_cap = (uint64_t)net->n_src * iv;
  CK(dalloc(&net->list, net->list_cap * sizeof(SpikeEntry), net->stream));
  if (net->stdp_on) {
    int rc2;
    if ((rc2 = setup_stdp(net)) != SNN_OK) return rc2;
  }
  (void)deliver_grid_size(net->fmt);
  CK(cudaGetLastError());
  net->finalized = true;
  return SNN_OK;
}

int snn_update(snn_net* net, int64_t t0, int32_t n_steps) {
  REQ(net, SNN_E_ARG, "null net");
  REQ(net->finalized, SNN_E_STATE, "net not finalized");
  REQ(!net->pending, SNN_E_STATE, "spikes of the previous update are pending");
  REQ(n_steps >= 1 && n_steps <= net->interval, SNN_E_ARG,
      "n_steps %d outside [1, interval %d]", n_steps, net->interval);
  const bool dev_clock = t0 == SNN_T_DEVICE;
  REQ(dev_clock || (t0 >= 0 && t0 + n_steps < (1ll << 31)), SNN_E_ARG,
      "t0 out of range");
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  CK(launch_update(net->view(), net->uc, n_steps, dev_clock ? 1 : 0,
                   dev_clock ? 0 : t0, net->stream));
  net->launches += 1;
  net->upd_launches += 1;
  net->pending = true;
  net->t_host = dev_clock ? net->t_host + n_steps : t0 + n_steps;
  return SNN_OK;
}

int snn_deliver_pending(snn_net* net) {
  REQ(net, SNN_E_ARG, "null net");
  REQ(net->finalized, SNN_E_STATE, "net not finalized");
  if (!net->pending) return SNN_OK;
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  CK(launch_deliver_any(net, &net->ctl->pair, &net->ctl->done, net->list, 0,
                        1));
  net->launches += 1;
  net->del_launches += 1;
  net->pending = false;
  return SNN_OK;
}

int snn_discard_pending(snn_net* net) {
  REQ(net, SNN_E_ARG, "null net");
  if (!net->pending) return SNN_OK;
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  CK(cudaMemsetAsync(&net->ctl->pair, 0, sizeof(unsigned long long),
                     net->stream));
  CK(cudaMemsetAsync(&net->ctl->pending_events, 0, sizeof(unsigned long long),
                     net->stream));
  if (net->xbuf)  // no delivery will clear the discarded spikes
    CK(cudaMemsetAsync(net->xbuf, 0, sizeof(uint32_t), net->stream));
  CK(cudaMemcpyAsync(&net->ctl->t_now, &net->t_host, sizeof(long long),
                     cudaMemcpyHostToDevice, net->stream));
  CK(cudaStreamSynchronize(net->stream));
  net->pending = false;
  return SNN_OK;
}

int snn_deliver(snn_net* net, const uint32_t* src, const int32_t* t_emit,
                uint32_t n_spikes, int mem, uint64_t* n_events_out) {
  REQ(net, SNN_E_ARG, "null net");
  REQ(net->finalized, SNN_E_STATE, "net not finalized");
  REQ(!net->stdp_on, SNN_E_STATE,
      "plastic nets deliver only their own spikes (traces kept by the update)");
  REQ(check_mem(mem), SNN_E_ARG, "bad mem kind");
  REQ(n_spikes == 0 || (src && t_emit), SNN_E_ARG, "null spike arrays");
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  cudaStream_t s = net->stream;
  if (n_spikes == 0) {
    if (n_events_out) *n_events_out = 0;
    return SNN_OK;
  }
  if ((rc = ensure_ext(net, n_spikes)) != SNN_OK) return rc;
  const uint32_t* d_src = src;
  const int32_t* d_t = t_emit;
  if (mem == SNN_MEM_HOST) {
    for (uint32_t k = 0; k < n_spikes; ++k)
      REQ(src[k] < net->n_src, SNN_E_ARG, "spike %u: source %u >= N", k, src[k]);
    CK(cudaMemcpyAsync(net->ext_src, src, n_spikes * 4ull,
                       cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(net->ext_t, t_emit, n_spikes * 4ull,
                       cudaMemcpyHostToDevice, s));
    d_src = net->ext_src;
    d_t = net->ext_t;
  }
  unsigned long long ev0 = 0, ev1 = 0;
  if (n_events_out) {
    CK(cudaMemcpyAsync(&ev0, &net->ctl->events, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  NetView v = net->view();
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (net->profiling) {
    e0 = pool_event(net, 0);
    e1 = pool_event(net, 1);
  }
  CK(launch_prepare_external(v, d_src, d_t, n_spikes, net->ext_list,
                             &net->ctl->ext_pair, s));
  if (e0) CK(cudaEventRecord(e0, s));
  CK(launch_deliver_any(net, &net->ctl->ext_pair, &net->ctl->ext_done,
                        net->ext_list, 1, 0));
  if (e1) CK(cudaEventRecord(e1, s));
  net->launches += 2;
  net->del_launches += 1;
  if (e1) {
    float ms = 0;
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    net->ms_deliver += ms;
  }
  if (n_events_out) {
    CK(cudaMemcpyAsync(&ev1, &net->ctl->events, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *n_events_out = ev1 - ev0;
  }
  return SNN_OK;
}

int snn_deliver_gathered(snn_net* net, const uint32_t* src,
                         const int32_t* t_emit, uint32_t n_spikes, int mem,
                         uint64_t* n_events_out) {
  REQ(net, SNN_E_ARG, "null net");
  REQ(net->finalized, SNN_E_STATE, "net not finalized");
  REQ(net->pending, SNN_E_STATE, "no pending interval (call snn_update first)");
  REQ(!net->stdp_on, SNN_E_STATE, "plastic nets deliver their own spikes");
  REQ(check_mem(mem), SNN_E_ARG, "bad mem kind");
  REQ(n_spikes == 0 || (src && t_emit), SNN_E_ARG, "null spike arrays");
  REQ(n_spikes <= net->list_cap, SNN_E_OVERFLOW,
      "%u gathered spikes exceed the interval list (%llu)", n_spikes,
      (unsigned long long)net->list_cap);
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  cudaStream_t s = net->stream;
  const uint32_t* d_src = src;
  const int32_t* d_t = t_emit;
  if (n_spikes && mem == SNN_MEM_HOST) {
    if ((rc = ensure_ext(net, n_spikes)) != SNN_OK) return rc;
    for (uint32_t k = 0; k < n_spikes; ++k)
      REQ(src[k] < net->n_src, SNN_E_ARG, "spike %u: source %u >= N", k, src[k]);
    CK(cudaMemcpyAsync(net->ext_src, src, n_spikes * 4ull,
                       cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(net->ext_t, t_emit, n_spikes * 4ull,
                       cudaMemcpyHostToDevice, s));
    d_src = net->ext_src;
    d_t = net->ext_t;
  }
  unsigned long long ev0 = 0, ev1 = 0;
  if (n_events_out) {
    CK(cudaMemcpyAsync(&ev0, &net->ctl->events, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  // the gathered list replaces the update's own list (and its events)
  CK(cudaMemsetAsync(&net->ctl->pair, 0, sizeof(unsigned long long), s));
  CK(cudaMemsetAsync(&net->ctl->pending_events, 0, sizeof(unsigned long long), s));
  NetView v = net->view();
  if (n_spikes) {
    CK(launch_prepare_external(v, d_src, d_t, n_spikes, net->list,
                               &net->ctl->pair, s));
    net->launches += 1;
  }
  CK(launch_deliver_any(net, &net->ctl->pair, &net->ctl->done, net->list, 0, 1));
  net->launches += 1;
  net->del_launches += 1;
  net->pending = false;
  if (n_events_out) {
    CK(cudaMemcpyAsync(&ev1, &net->ctl->events, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *n_events_out = ev1 - ev0;
  }
  return SNN_OK;
}

// Device (or managed) memory of the net's device, 16-byte aligned: the
// exchange buffers are read and written by the kernels directly.
static int check_exchange_ptr(snn_net* net, const void* p, const char* what) {
  REQ(((uintptr_t)p & 15u) == 0, SNN_E_ARG, "%s is not 16-byte aligned", what);
  cudaPointerAttributes pa;
  const cudaError_t pe = cudaPointerGetAttributes(&pa, p);
  if (pe != cudaSuccess) cudaGetLastError();
  REQ(pe == cudaSuccess, SNN_E_ARG, "%s: not a CUDA pointer (%s)", what,
      cudaGetErrorString(pe));
  REQ((pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged) &&
          pa.device == net->device,
      SNN_E_ARG, "%s must be device memory of the net's device", what);
  return SNN_OK;
}

int snn_exchange_capacity(snn_net* net, uint64_t* cap_entries) {
  REQ(net && cap_entries, SNN_E_ARG, "null argument");
  REQ(net->finalized, SNN_E_STATE, "net not finalized");
  *cap_entries = (uint64_t)net->n * std::max<uint32_t>(net->spikes_per_iv, 1u);
  return SNN_OK;
}

int snn_set_exchange(snn_net* net, void* buf, uint64_t cap_entries) {
  REQ(net, SNN_E_ARG, "null net");
  REQ(net->finalized, SNN_E_STATE, "net not finalized");
  REQ(!net->pending, SNN_E_STATE, "spikes of an update are pending");
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  if (buf) {
    REQ(cap_entries >= 1 && cap_entries <= 0xFFFFFFFFull, SNN_E_ARG,
        "exchange capacity %llu outside [1, 2^32 - 1]",
        (unsigned long long)cap_entries);
    if ((rc = check_exchange_ptr(net, buf, "exchange buffer")) != SNN_OK)
      return rc;
  }
  // the captured intervals hold the old view; the stream's queued work may
  // still write the old buffer, so the caller's reuse waits for it
  CK(cudaStreamSynchronize(net->stream));
  drop_graphs(net);
  if (buf) {  // an empty list until the first update
    CK(cudaMemsetAsync(buf, 0, 16, net->stream));
    CK(cudaStreamSynchronize(net->stream));
  }
  net->xbuf = static_cast<uint32_t*>(buf);
  net->xcap = buf ? (uint32_t)cap_entries : 0u;
  net->x_parts_ok = nullptr;
  return SNN_OK;
}

int snn_deliver_exchanged(snn_net* net, const void* parts, uint32_t n_parts,
                          uint64_t stride_bytes) {
  REQ(net, SNN_E_ARG, "null net");
  REQ(net->finalized, SNN_E_STATE, "net not finalized");
  REQ(net->pending, SNN_E_STATE, "no pending interval (call snn_update first)");
  REQ(!net->stdp_on, SNN_E_STATE, "plastic nets deliver their own spikes");
  REQ(use_tiled(net), SNN_E_STATE,
      "exchanged lists need the tiled delivery (deliver_mode TILED with a "
      "window that fits a tile)");
  REQ(n_parts >= 1 && n_parts <= kMaxGatherParts, SNN_E_ARG,
      "n_parts %u outside [1, %u]", n_parts, kMaxGatherParts);
  REQ(stride_bytes >= 16 && stride_bytes % 16 == 0, SNN_E_ARG,
      "stride %llu is not a multiple of 16 bytes of at least 16",
      (unsigned long long)stride_bytes);
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  // validated once per pointer (no runtime query inside a stream capture
  // that replays the same buffers)
  if (parts != net->x_parts_ok) {
    if ((rc = check_exchange_ptr(net, parts, "parts")) != SNN_OK) return rc;
    net->x_parts_ok = parts;
  }
  cudaStream_t s = net->stream;
  // the union's events are counted by the delivery itself (the update's
  // count covers only the local sources' synapses and is dropped)
  NetView v = net->view();
  v.gx = static_cast<const uint32_t*>(parts);
  v.gx_parts = n_parts;
  v.gx_stride = stride_bytes / 4;
  v.gx_cap = (uint32_t)std::min<uint64_t>((stride_bytes - 16) / 8, 0xFFFFFFFFull);
  CK(launch_deliver_tiled(v, &net->ctl->pair, &net->ctl->done, net->list, 0, 1,
                          s));
  net->launches += 1;
  net->del_launches += 1;
  net->pending = false;
  return SNN_OK;
}

int snn_deliver_noalloc(snn_net* net, const uint32_t* src,
                        const int32_t* t_emit, uint32_t n_spikes,
                        uint64_t* n_events_out) {
  REQ(net, SNN_E_ARG, "null net");
  REQ(net->finalized, SNN_E_STATE, "net not finalized");
  REQ(!net->stdp_on, SNN_E_STATE,
      "plastic nets deliver only their own spikes (traces kept by the update)");
  REQ(n_spikes <= SNN_NOALLOC_MAX_SPIKES, SNN_E_ARG,
      "%u spikes exceed the allocation-free scratch of %u spikes", n_spikes,
      (unsigned)SNN_NOALLOC_MAX_SPIKES);
  REQ(n_spikes == 0 || (src && t_emit), SNN_E_ARG, "null spike arrays");
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  cudaStream_t s = net->stream;
  if (n_spikes == 0) {
    if (n_events_out) *n_events_out = 0;
    return SNN_OK;
  }
  // the kernels read the lists directly: a host pointer would fault on the
  // device, so only device (or managed) memory of the net's device passes
  // (cudaPointerGetAttributes allocates nothing)
  const void* lists[2] = {src, t_emit};
  for (int k = 0; k < 2; ++k) {
    cudaPointerAttributes pa;
    const cudaError_t pe = cudaPointerGetAttributes(&pa, lists[k]);
    if (pe != cudaSuccess) cudaGetLastError();  // not left for later checks
    REQ(pe == cudaSuccess, SNN_E_ARG, "%s: not a CUDA pointer (%s)",
        k ? "t_emit" : "src", cudaGetErrorString(pe));
    REQ((pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged) &&
            pa.device == net->device,
        SNN_E_ARG, "%s must be device memory of the net's device",
        k ? "t_emit" : "src");
  }
  unsigned long long ev0 = 0, ev1 = 0;
  if (n_events_out) {
    CK(cudaMemcpyAsync(&ev0, &net->ctl->events, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  CK(launch_deliver_noalloc(net->view(), src, t_emit, n_spikes, s));
  net->launches += 2;
  net->del_launches += 1;
  if (n_events_out) {
    CK(cudaMemcpyAsync(&ev1, &net->ctl->events, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *n_events_out = ev1 - ev0;
  }
  return SNN_OK;
}

}  // extern "C"

// The production path of snn_simulate: whole intervals as replays of the
// net's captured graph (captured now if may_capture, else launched one by
// one while none exists: instantiation waits for other streams' work), the
// rest launched directly; asynchronous.
int snn::simulate_async(snn_net* net, int64_t n_steps, bool may_capture) {
  const int D = net->interval;
  int64_t full = n_steps / D;
  const int rem = (int)(n_steps % D);
  cudaStream_t s = net->stream;
  int rc;
  if (full >= kGraphIntervals && (net->graph || may_capture)) {
    if ((rc = capture_graph(net, false)) != SNN_OK) return rc;
    for (; full >= kGraphIntervals; full -= kGraphIntervals) {
      CK(cudaGraphLaunch(net->graph, s));
      net->launches += 2 * kGraphIntervals;
      net->upd_launches += kGraphIntervals;
      net->del_launches += kGraphIntervals;
    }
  }
  for (; full > 0; --full)
    if ((rc = launch_interval(net, D)) != SNN_OK) return rc;
  if (rem)
    if ((rc = launch_interval(net, rem)) != SNN_OK) return rc;
  net->t_host += n_steps;
  return SNN_OK;
}

extern "C" {

int snn_simulate(snn_net* net, int64_t n_steps) {
  REQ(net, SNN_E_ARG, "null net");
  REQ(net->finalized, SNN_E_STATE, "net not finalized");
  REQ(!net->pending, SNN_E_STATE, "spikes of an update are pending");
  REQ(n_steps >= 0 && net->t_host + n_steps < (1ll << 31), SNN_E_ARG,
      "n_steps out of range");
  if (n_steps == 0) return SNN_OK;
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  const int D = net->interval;
  int64_t full = n_steps / D;
  const int rem = (int)(n_steps % D);
  cudaStream_t s = net->stream;
  if (net->profiling) {
    // whole graphs of intervals with their timing events, read after each
    // replay; the remaining intervals one by one between events
    auto add_times = [&](int64_t n) -> int {
      for (int64_t k = 0; k < n; ++k) {
        float mu = 0, md = 0;
        CK(cudaEventElapsedTime(&mu, net->ev[3 * k], net->ev[3 * k + 1]));
        CK(cudaEventElapsedTime(&md, net->ev[3 * k + 1], net->ev[3 * k + 2]));
        net->ms_update += mu;
        net->ms_deliver += md;
      }
      return SNN_OK;
    };
    if (full >= kGraphIntervals) {
      if ((rc = capture_graph(net, true)) != SNN_OK) return rc;
      for (; full >= kGraphIntervals; full -= kGraphIntervals) {
        CK(cudaGraphLaunch(net->graph_prof, s));
        CK(cudaStreamSynchronize(s));
        if ((rc = add_times(kGraphIntervals)) != SNN_OK) return rc;
        net->launches += 2 * kGraphIntervals;
        net->upd_launches += kGraphIntervals;
        net->del_launches += kGraphIntervals;
      }
    }
    const int64_t n_iv = full + (rem ? 1 : 0);
    for (int64_t k = 0; k < n_iv; ++k) {
      const int steps = k < full ? D : rem;
      cudaEvent_t a = pool_event(net, 3 * (size_t)k);
      cudaEvent_t b = pool_event(net, 3 * (size_t)k + 1);
      cudaEvent_t c = pool_event(net, 3 * (size_t)k + 2);
      REQ(a && b && c, SNN_E_CUDA, "event creation failed");
      NetView v = net->view();
      CK(cudaEventRecord(a, s));
      CK(launch_update(v, net->uc, steps, 1, 0, s));
      CK(cudaEventRecord(b, s));
      CK(launch_deliver_any(net, &net->ctl->pair, &net->ctl->done, net->list, 0,
                            1));
      CK(cudaEventRecord(c, s));
      net->launches += 2;
      net->upd_launches += 1;
      net->del_launches += 1;
    }
    CK(cudaStreamSynchronize(s));
    if ((rc = add_times(n_iv)) != SNN_OK) return rc;
  } else {
    if ((rc = simulate_async(net, n_steps, true)) != SNN_OK) return rc;
    return SNN_OK;
  }
  net->t_host += n_steps;
  return SNN_OK;
}

int snn_read_spikes(snn_net* net, uint32_t* src, int32_t* t, uint64_t cap,
                    uint64_t* n, int mem) {
  REQ(net && n, SNN_E_ARG, "null argument");
  REQ(check_mem(mem), SNN_E_ARG, "bad mem kind");
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  cudaStream_t s = net->stream;
  unsigned long long cnt = 0;
  CK(cudaMemcpyAsync(&cnt, &net->ctl->log_count, 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *n = cnt;
  uint64_t kept = std::min<uint64_t>(std::min<uint64_t>(cnt, net->log_cap), cap);
  if (kept) {
    REQ(src && t, SNN_E_ARG, "null output arrays");
    CK(cudaMemcpyAsync(src, net->log_src, kept * 4, kind_to(mem), s));
    CK(cudaMemcpyAsync(t, net->log_t, kept * 4, kind_to(mem), s));
  }
  CK(cudaMemsetAsync(&net->ctl->log_count, 0, 8, s));
  CK(cudaStreamSynchronize(s));
  if (cnt > kept)
    return fail(SNN_E_OVERFLOW, "%llu spikes logged, %llu returned",
                (unsigned long long)cnt, (unsigned long long)kept);
  return SNN_OK;
}

static int copy_slots(snn_net* net, void* host_or_dev, const void* dev_base,
                      int to_caller, int mem, size_t elem) {
  REQ(check_mem(mem), SNN_E_ARG, "bad mem kind");
  cudaStream_t s = net->stream;
  const size_t w = (size_t)net->n * elem, pitch = (size_t)net->pitch * elem;
  if (to_caller)
    CK(cudaMemcpy2DAsync(host_or_dev, w, dev_base, pitch, w, net->n_slots,
                         kind_to(mem), s));
  else
    CK(cudaMemcpy2DAsync(const_cast<void*>(dev_base), pitch, host_or_dev, w, w,
                         net->n_slots, kind_from(mem), s));
  if (mem == SNN_MEM_HOST) CK(cudaStreamSynchronize(s));
  return SNN_OK;
}

int snn_read_rb(snn_net* net, float* dst, int mem) {
  REQ(net && dst, SNN_E_ARG, "null argument");
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  return copy_slots(net, dst, net->rb, 1, mem, sizeof(float));
}

int snn_write_rb(snn_net* net, const float* src, int mem) {
  REQ(net && src, SNN_E_ARG, "null argument");
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  return copy_slots(net, const_cast<float*>(src), net->rb, 0, mem,
                    sizeof(float));
}

int snn_read_counts(snn_net* net, uint32_t* dst, int mem) {
  REQ(net && dst, SNN_E_ARG, "null argument");
  REQ(net->counts, SNN_E_STATE, "net created without count_events");
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  return copy_slots(net, dst, net->counts, 1, mem, sizeof(uint32_t));
}

int snn_clear_rb(snn_net* net) {
  REQ(net, SNN_E_ARG, "null net");
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  const size_t bytes = (size_t)net->n_slots * net->pitch * 4;
  CK(cudaMemsetAsync(net->rb, 0, bytes, net->stream));
  if (net->counts) CK(cudaMemsetAsync(net->counts, 0, bytes, net->stream));
  return SNN_OK;
}

int snn_read_state(snn_net* net, float* V, float* I, float* J, int32_t* refr,
                   int mem) {
  REQ(net, SNN_E_ARG, "null net");
  REQ(check_mem(mem), SNN_E_ARG, "bad mem kind");
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  cudaStream_t s = net->stream;
  const size_t b = (size_t)net->n * 4;
  if (V) CK(cudaMemcpyAsync(V, net->V, b, kind_to(mem), s));
  if (I) CK(cudaMemcpyAsync(I, net->I, b, kind_to(mem), s));
  if (J) CK(cudaMemcpyAsync(J, net->J, b, kind_to(mem), s));
  if (refr) CK(cudaMemcpyAsync(refr, net->refr, b, kind_to(mem), s));
  if (mem == SNN_MEM_HOST) CK(cudaStreamSynchronize(s));
  return SNN_OK;
}

int snn_write_state(snn_net* net, const float* V, const float* I,
                    const float* J, const int32_t* refr, int mem) {
  REQ(net, SNN_E_ARG, "null net");
  REQ(check_mem(mem), SNN_E_ARG, "bad mem kind");
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  cudaStream_t s = net->stream;
  const size_t b = (size_t)net->n * 4;
  if (V) CK(cudaMemcpyAsync(net->V, V, b, kind_from(mem), s));
  if (I) CK(cudaMemcpyAsync(net->I, I, b, kind_from(mem), s));
  if (J) CK(cudaMemcpyAsync(net->J, J, b, kind_from(mem), s));
  if (refr) CK(cudaMemcpyAsync(net->refr, refr, b, kind_from(mem), s));
  if (mem == SNN_MEM_HOST) CK(cudaStreamSynchronize(s));
  return SNN_OK;
}

int snn_read_store(snn_net* net, uint64_t* row_ptr, uint32_t* tgt,
                   uint8_t* delay, float* w, int mem) {
  REQ(net, SNN_E_ARG, "null net");
  REQ(net->connected, SNN_E_STATE, "net has no store");
  REQ(check_mem(mem), SNN_E_ARG, "bad mem kind");
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  cudaStream_t s = net->stream;
  if (row_ptr)
    CK(cudaMemcpyAsync(row_ptr, net->row_ptr, (net->n_src + 1) * 8ull,
                       kind_to(mem), s));
  const uint64_t m = net->n_syn;
  if (m && (tgt || delay || w)) {
    if (mem == SNN_MEM_DEVICE) {
      CK(unpack_store(net->fmt, net->recs, m, tgt, delay, w, s));
    } else {
      uint32_t* dt = nullptr;
      uint8_t* dd = nullptr;
      float* dw = nullptr;
      CK(dalloc(&dt, m * 4, net->stream));
      CK(dalloc(&dd, m, net->stream));
      CK(dalloc(&dw, m * 4, net->stream));
      CK(unpack_store(net->fmt, net->recs, m, dt, dd, dw, s));
      if (tgt) CK(cudaMemcpyAsync(tgt, dt, m * 4, cudaMemcpyDeviceToHost, s));
      if (delay) CK(cudaMemcpyAsync(delay, dd, m, cudaMemcpyDeviceToHost, s));
      if (w) CK(cudaMemcpyAsync(w, dw, m * 4, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      dfree(dt, net->stream);
      dfree(dd, net->stream);
      dfree(dw, net->stream);
    }
    net->launches += 1;
  }
  if (mem == SNN_MEM_HOST) CK(cudaStreamSynchronize(s));
  return SNN_OK;
}

namespace {
struct StateHeader {
  char magic[8];     // "SNNSTATE"
  uint32_t version;  // 1
  uint32_t n;
  int32_t n_slots;
  int32_t pad_;
  int64_t t_now;
  char reserved[32];
};
static_assert(sizeof(StateHeader) == 64, "state header is 64 bytes");

uint64_t state_bytes(const snn_net* net) {
  return sizeof(StateHeader) + 4ull * net->n * 4 +
         4ull * net->n * (uint64_t)net->n_slots;
}
}  // namespace

int snn_state_size(snn_net* net, uint64_t* bytes) {
  REQ(net && bytes, SNN_E_ARG, "null argument");
  *bytes = state_bytes(net);
  return SNN_OK;
}

int snn_save_state(snn_net* net, void* host_buf, uint64_t cap) {
  REQ(net && host_buf, SNN_E_ARG, "null argument");
  REQ(cap >= state_bytes(net), SNN_E_OVERFLOW, "state needs %llu bytes",
      (unsigned long long)state_bytes(net));
  REQ(!net->stdp_on, SNN_E_STATE, "checkpoints of plastic nets are not supported");
  REQ(!net->pending, SNN_E_STATE, "spikes of an update are pending");
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  long long t_now = 0;
  CK(cudaMemcpyAsync(&t_now, &net->ctl->t_now, sizeof t_now,
                     cudaMemcpyDeviceToHost, net->stream));
  CK(cudaStreamSynchronize(net->stream));
  StateHeader h{};
  memcpy(h.magic, "SNNSTATE", 8);
  h.version = 1;
  h.n = net->n;
  h.n_slots = net->n_slots;
  h.t_now = t_now;
  char* out = static_cast<char*>(host_buf);
  memcpy(out, &h, sizeof h);
  char* p = out + sizeof h;
  const size_t b = (size_t)net->n * 4;
  if ((rc = snn_read_state(net, reinterpret_cast<float*>(p),
                           reinterpret_cast<float*>(p + b),
                           reinterpret_cast<float*>(p + 2 * b),
                           reinterpret_cast<int32_t*>(p + 3 * b),
                           SNN_MEM_HOST)) != SNN_OK)
    return rc;
  return snn_read_rb(net, reinterpret_cast<float*>(p + 4 * b), SNN_MEM_HOST);
}

int snn_load_state(snn_net* net, const void* host_buf, uint64_t size) {
  REQ(net && host_buf, SNN_E_ARG, "null argument");
  REQ(size >= state_bytes(net), SNN_E_ARG, "state image too short");
  REQ(!net->stdp_on, SNN_E_STATE, "checkpoints of plastic nets are not supported");
  REQ(!net->pending, SNN_E_STATE, "spikes of an update are pending");
  StateHeader h;
  memcpy(&h, host_buf, sizeof h);
  REQ(memcmp(h.magic, "SNNSTATE", 8) == 0 && h.version == 1, SNN_E_ARG,
      "not a state image");
  REQ(h.n == net->n && h.n_slots == net->n_slots, SNN_E_ARG,
      "state image of a different net (N %u, slots %d)", h.n, h.n_slots);
  REQ(h.t_now >= 0 && h.t_now < (1ll << 31), SNN_E_ARG, "bad clock");
  const char* p = static_cast<const char*>(host_buf) + sizeof h;
  const size_t b = (size_t)net->n * 4;
  int rc;
  if ((rc = snn_write_state(net, reinterpret_cast<const float*>(p),
                            reinterpret_cast<const float*>(p + b),
                            reinterpret_cast<const float*>(p + 2 * b),
                            reinterpret_cast<const int32_t*>(p + 3 * b),
                            SNN_MEM_HOST)) != SNN_OK)
    return rc;
  if ((rc = snn_write_rb(net, reinterpret_cast<const float*>(p + 4 * b),
                         SNN_MEM_HOST)) != SNN_OK)
    return rc;
  return snn_set_time(net, h.t_now);
}

int snn_set_drive(snn_net* net, double nu_ext, double w_ext) {
  REQ(net, SNN_E_ARG, "null net");
  REQ(nu_ext >= 0 && isfinite(nu_ext) && isfinite(w_ext), SNN_E_ARG,
      "bad drive");
  REQ(!net->pending, SNN_E_STATE, "spikes of an update are pending");
  snn_params p = net->p;
  p.nu_ext = nu_ext;
  p.w_ext = w_ext;
  UpdConst uc;
  REQ(make_upd_const(p, &uc) == 0, SNN_E_ARG,
      "Poisson drive rate too high for the inversion table");
  net->p = p;
  net->uc = uc;
  drop_graphs(net);  // the captured graphs hold the old constants
  return SNN_OK;
}

int snn_set_time(snn_net* net, int64_t t) {
  REQ(net, SNN_E_ARG, "null net");
  REQ(t >= 0 && t < (1ll << 31), SNN_E_ARG, "t out of range");
  REQ(!net->pending, SNN_E_STATE, "spikes of an update are pending");
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  net->t_host = t;
  CK(cudaMemcpyAsync(&net->ctl->t_now, &net->t_host, sizeof(long long),
                     cudaMemcpyHostToDevice, net->stream));
  CK(cudaStreamSynchronize(net->stream));
  return SNN_OK;
}

int snn_set_profiling(snn_net* net, int on) {
  REQ(net, SNN_E_ARG, "null net");
  net->profiling = on != 0;
  return SNN_OK;
}

int snn_get_stats(snn_net* net, snn_stats* out) {
  REQ(net && out, SNN_E_ARG, "null argument");
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  Ctl c;
  CK(cudaMemcpyAsync(&c, net->ctl, sizeof c, cudaMemcpyDeviceToHost,
                     net->stream));
  CK(cudaStreamSynchronize(net->stream));
  memset(out, 0, sizeof *out);
  out->events_delivered = c.events;
  out->spikes = c.spikes;
  out->n_synapses = net->n_syn;
  out->t_now = c.t_now;
  out->interval = net->interval;
  out->min_delay = net->dmin;
  out->max_delay = net->dmax;
  out->error_flags = c.error_flags;
  out->kernel_launches = net->launches;
  out->update_launches = net->upd_launches;
  out->deliver_launches = net->del_launches;
  out->ms_update = net->ms_update;
  out->ms_deliver = net->ms_deliver;
  out->bytes_per_record = net->fmt == SNN_W_FP32_12B ? 12 : 8;
  out->store_bytes = net->recs_bytes;
  out->n_tiles = net->n_tiles;
  out->tile_width = net->tile_w;
  out->window = net->window;
  out->deliver_mode = use_tiled(net) ? SNN_DELIVER_TILED : SNN_DELIVER_ATOMIC;
  out->plastic_events = c.plastic_events;
  out->stdp_truncated = c.stdp_truncated;
  out->first_neuron = net->g0;
  out->n_sources = net->n_src;
  out->acc_words = net->acc_words;
  // replayed captures advance the device clock only: resynchronise
  if (!net->pending) net->t_host = c.t_now;
  note_check_failure(net, c.error_flags);
  return SNN_OK;
}

int snn_read_pending(snn_net* net, uint32_t* src, int32_t* t, uint64_t cap,
                     uint64_t* n, int32_t mem) {
  REQ(net && n, SNN_E_ARG, "null argument");
  REQ(net->pending, SNN_E_STATE, "no pending interval list");
  REQ(check_mem(mem), SNN_E_ARG, "bad mem kind");
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  cudaStream_t s = net->stream;
  unsigned long long pair = 0;
  CK(cudaMemcpyAsync(&pair, &net->ctl->pair, sizeof pair, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const uint64_t cnt = std::min<uint64_t>(pair >> 32, net->list_cap);
  *n = cnt;
  const uint64_t k = std::min(cap, cnt);
  if (k) {
    REQ(src && t, SNN_E_ARG, "null output arrays");
    if (mem == SNN_MEM_DEVICE) {
      CK(launch_list_to_arrays(net->list, k, src, t, s));
    } else {
      std::vector<SpikeEntry> h(k);
      CK(cudaMemcpyAsync(h.data(), net->list, k * sizeof(SpikeEntry),
                         cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (uint64_t q = 0; q < k; ++q) {
        src[q] = h[q].src;
        t[q] = h[q].t;
      }
    }
    CK(cudaStreamSynchronize(s));
  }
  return k < cnt ? fail(SNN_E_OVERFLOW, "%llu pending spikes", (unsigned long long)cnt)
                 : SNN_OK;
}

int snn_get_bounds(snn_net* net, snn_bounds* out) {
  REQ(net && out, SNN_E_ARG, "null argument");
  REQ(net->connected, SNN_E_STATE, "net not connected");
  memset(out, 0, sizeof *out);
  out->mult_max = net->mult_max;
  out->k_in_max = net->k_in_max;
  out->max_abs_w = net->max_abs_w;
  return SNN_OK;
}

int snn_set_bounds(snn_net* net, const snn_bounds* b) {
  REQ(net && b, SNN_E_ARG, "null argument");
  REQ(net->connected, SNN_E_STATE, "net not connected");
  REQ(isfinite(b->max_abs_w) && b->max_abs_w >= 0.f, SNN_E_ARG, "bad max |w|");
  net->mult_max = std::max(net->mult_max, b->mult_max);
  net->k_in_max = std::max(net->k_in_max, b->k_in_max);
  net->max_abs_w = std::max(net->max_abs_w, b->max_abs_w);
  drop_graphs(net);  // the captured intervals hold the old view
  return SNN_OK;
}

int snn_set_stdp(snn_net* net, const snn_stdp_params* q) {
  REQ(net && q, SNN_E_ARG, "null argument");
  REQ(!net->connected && !net->finalized, SNN_E_STATE,
      "snn_set_stdp must come before connecting");
  REQ(q->tau_plus > 0 && q->tau_minus > 0 && q->lambda >= 0 && q->alpha >= 0 &&
          q->mu >= 0 && q->mu <= 1 && q->w0 > 0 && q->w_max > 0 &&
          isfinite(q->lambda) && isfinite(q->alpha) && isfinite(q->w_max),
      SNN_E_ARG, "bad STDP parameters");
  REQ(q->history >= 2 && q->history <= kMaxStdpHistory &&
          (q->history & (q->history - 1)) == 0,
      SNN_E_ARG, "STDP history %d is not a power of two in [2, %d]",
      q->history, kMaxStdpHistory);
  REQ(net->p.deliver_mode == SNN_DELIVER_TILED, SNN_E_ARG,
      "STDP needs deliver_mode SNN_DELIVER_TILED");
  REQ(net->n == net->n_src, SNN_E_ARG, "STDP is not supported for partitions");
  net->stdp = *q;
  net->stdp_on = true;
  return SNN_OK;
}

int snn_read_spike_stats(snn_net* net, uint32_t* n_spikes, uint32_t* n_isi,
                         double* isi_sum, double* isi_sq) {
  REQ(net, SNN_E_ARG, "null net");
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  cudaStream_t s = net->stream;
  const size_t n = net->n;
  if (n_spikes)
    CK(cudaMemcpyAsync(n_spikes, net->isi_spikes, n * 4, cudaMemcpyDeviceToHost, s));
  if (n_isi) CK(cudaMemcpyAsync(n_isi, net->isi_n, n * 4, cudaMemcpyDeviceToHost, s));
  if (isi_sum)
    CK(cudaMemcpyAsync(isi_sum, net->isi_sum, n * 8, cudaMemcpyDeviceToHost, s));
  if (isi_sq) CK(cudaMemcpyAsync(isi_sq, net->isi_sq, n * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return SNN_OK;
}

int snn_clear_spike_stats(snn_net* net) {
  REQ(net, SNN_E_ARG, "null net");
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  cudaStream_t s = net->stream;
  const size_t n = net->n;
  CK(cudaMemsetAsync(net->isi_spikes, 0, n * 4, s));
  CK(cudaMemsetAsync(net->isi_n, 0, n * 4, s));
  CK(cudaMemsetAsync(net->isi_sum, 0, n * 8, s));
  CK(cudaMemsetAsync(net->isi_sq, 0, n * 8, s));
  return SNN_OK;
}

int snn_read_weights(snn_net* net, float* w, int32_t mem) {
  REQ(net && w, SNN_E_ARG, "null argument");
  REQ(net->finalized, SNN_E_STATE, "net not finalized");
  REQ(check_mem(mem), SNN_E_ARG, "bad mem kind");
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  cudaStream_t s = net->stream;
  const uint64_t m = net->n_syn;
  if (m == 0) return SNN_OK;
  if (net->sp.wp) {
    CK(cudaMemcpyAsync(w, net->sp.wp, m * sizeof(float), kind_to(mem), s));
  } else if (mem == SNN_MEM_DEVICE) {
    CK(unpack_store(net->fmt, net->recs, m, nullptr, nullptr, w, s));
  } else {
    float* dw = nullptr;
    CK(dalloc(&dw, m * sizeof(float), s));
    CK(unpack_store(net->fmt, net->recs, m, nullptr, nullptr, dw, s));
    CK(cudaMemcpyAsync(w, dw, m * sizeof(float), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    dfree(dw, s);
  }
  if (mem == SNN_MEM_HOST) CK(cudaStreamSynchronize(s));
  return SNN_OK;
}

int snn_clear_errors(snn_net* net) {
  REQ(net, SNN_E_ARG, "null net");
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  CK(cudaMemsetAsync(&net->ctl->error_flags, 0, sizeof(unsigned),
                     net->stream));
  CK(cudaStreamSynchronize(net->stream));
  return SNN_OK;
}

int snn_sync(snn_net* net) {
  REQ(net, SNN_E_ARG, "null net");
  CK(cudaStreamSynchronize(net->stream));
  CK(cudaGetLastError());
  return SNN_OK;
}

int snn_probe_reductions(float* buf, uint64_t n_cells, uint64_t n_ops,
                         int pattern, void* stream, float* ms) {
  REQ(buf && ms, SNN_E_ARG, "null argument");
  REQ(n_cells >= 1 && n_cells < (1ull << 32), SNN_E_ARG,
      "n_cells %llu outside [1, 2^32)", (unsigned long long)n_cells);
  REQ(n_ops >= 1, SNN_E_ARG, "n_ops is 0");
  REQ(pattern == SNN_PROBE_SCATTER || pattern == SNN_PROBE_SWEEP, SNN_E_ARG,
      "unknown pattern %d", pattern);
  cudaPointerAttributes pa;
  const cudaError_t pe = cudaPointerGetAttributes(&pa, buf);
  if (pe != cudaSuccess) cudaGetLastError();
  REQ(pe == cudaSuccess && (pa.type == cudaMemoryTypeDevice ||
                            pa.type == cudaMemoryTypeManaged),
      SNN_E_ARG, "buf is not device memory");
  int prev = 0;
  CK(cudaGetDevice(&prev));
  CK(cudaSetDevice(pa.device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = cudaEventRecord(a, s);
  if (e == cudaSuccess)
    e = snn::launch_red_probe(buf, (uint32_t)n_cells, n_ops, pattern, s);
  if (e == cudaSuccess) e = cudaEventRecord(b, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaSetDevice(prev);  // the caller's current device, as it was
  CK(e);
  return SNN_OK;
}

int snn_get_stream(snn_net* net, void** stream) {
  REQ(net && stream, SNN_E_ARG, "null argument");
  *stream = static_cast<void*>(net->stream);
  return SNN_OK;
}

int snn_checked(void) { return kChecked ? 1 : 0; }

uint64_t snn_debug_check_failures(void) {
  return g_check_failures.load(std::memory_order_relaxed);
}

int snn_debug_poke_record(snn_net* net, uint64_t index, int field,
                          uint32_t value) {
  REQ(net, SNN_E_ARG, "null net");
  REQ(kChecked, SNN_E_STATE,
      "store corruption is only accepted by bounds-checked builds");
  REQ(net->finalized, SNN_E_STATE, "net not finalized");
  REQ(index < net->n_syn, SNN_E_ARG, "record %llu outside the store",
      (unsigned long long)index);
  REQ(field == 0 || (field == 1 && value <= 0xFFu), SNN_E_ARG,
      "field %d / value %u", field, value);
  int rc;
  if ((rc = set_device(net)) != SNN_OK) return rc;
  // target: word 0 of both formats; delay: low byte of word 2 (FP32
  // records) or of word 1 (BF16 records)
  const size_t rb = net->fmt == SNN_W_FP32_12B ? 12 : 8;
  const size_t off = field == 0 ? 0 : (net->fmt == SNN_W_FP32_12B ? 8 : 4);
  char* p = static_cast<char*>(net->recs) + index * rb + off;
  uint32_t word = 0;
  CK(cudaMemcpyAsync(&word, p, 4, cudaMemcpyDeviceToHost, net->stream));
  CK(cudaStreamSynchronize(net->stream));
  word = field == 0 ? value : ((word & ~0xFFu) | value);
  CK(cudaMemcpyAsync(p, &word, 4, cudaMemcpyHostToDevice, net->stream));
  CK(cudaStreamSynchronize(net->stream));
  return SNN_OK;
}

int snn_destroy(snn_net* net) {
  if (!net) return SNN_OK;
  cudaSetDevice(net->device);
  if (net->stream) cudaStreamSynchronize(net->stream);
  if (kChecked && net->ctl) {
    unsigned flags = 0;
    if (cudaMemcpy(&flags, &net->ctl->error_flags, sizeof flags,
                   cudaMemcpyDeviceToHost) == cudaSuccess)
      note_check_failure(net, flags);
    cudaGetLastError();
  }
  drop_graphs(net);
  for (cudaEvent_t e : net->ev) cudaEventDestroy(e);
  void* bufs[] = {net->V,        net->I,        net->J,       net->refr,
                  net->rb,       net->counts,   net->ctl,     net->row_ptr,
                  net->recs,     net->list,     net->ext_list, net->ext_src,
                  net->ext_t,    net->log_src,  net->log_t,   net->tile_off};
  for (void* b : bufs) dfree(b, net->stream);
  void* ibufs[] = {net->isi_last, net->isi_spikes, net->isi_n, net->isi_sum,
                   net->isi_sq};
  for (void* b : ibufs) dfree(b, net->stream);
  void* sbufs[] = {net->sp.wp,     net->sp.pre_t,  net->sp.prev_t,
                   net->sp.pre_k,  net->sp.prev_k, net->sp.ring_t,
                   net->sp.ring_k, net->sp.ring_n};
  for (void* b : sbufs) dfree(b, net->stream);
  if (net->counted) count_net(net->device, -1, net->stream);
  if (net->own_stream) cudaStreamDestroy(net->stream);
  delete net;
  return SNN_OK;
}

}  // extern "C"
