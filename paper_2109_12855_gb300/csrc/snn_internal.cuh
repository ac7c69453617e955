// snn_internal.cuh -- device-side definitions shared by the libsnn CUDA
// translation units: record formats, the per-net control block, the
// counter-based generator and small warp helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <limits.h>
#include <string.h>

#include "../../include/snn.h"

namespace snn {

// ---------------------------------------------------------------------------
// Connection store records.  A target segment (Section 3.1 of the paper) is
// a contiguous run of records; the store is source-major with row offsets.
// Chunking: every row is processed in chunks aligned to absolute record
// indices that are multiples of kChunk, so that each lane of a warp issues
// naturally aligned 16-byte loads; records of a chunk outside the row are
// loaded and ignored.  The record array is padded to whole chunks.
// ---------------------------------------------------------------------------
struct RecF32 {       // 12 bytes
  uint32_t target;
  float weight;
  uint32_t delay;     // low 8 bits; upper 24 bits are zero padding
};
struct RecBF16 {      // 8 bytes
  uint32_t target;
  uint32_t meta;      // bits 0-7 delay, 8-15 pad, 16-31 bfloat16 weight
};

template <int FMT> struct Fmt;
template <> struct Fmt<SNN_W_FP32_12B> {
  static constexpr int kRecBytes = 12;
  static constexpr int kPerLane = 4;            // 48 bytes = 3 x 16 B
  static constexpr int kChunk = 32 * kPerLane;  // 128 records, 1,536 B
};
template <> struct Fmt<SNN_W_BF16_8B> {
  static constexpr int kRecBytes = 8;
  static constexpr int kPerLane = 2;            // 16 bytes
  static constexpr int kChunk = 32 * kPerLane;  // 64 records, 512 B
};

__host__ __device__ inline int chunk_records(int fmt) {
  return fmt == SNN_W_FP32_12B ? Fmt<SNN_W_FP32_12B>::kChunk
                               : Fmt<SNN_W_BF16_8B>::kChunk;
}

// Number of aligned chunks that cover records [beg, end).
__host__ __device__ inline uint32_t row_chunks(uint64_t beg, uint64_t end,
                                               uint32_t ch) {
  return end > beg ? (uint32_t)((end - 1) / ch - beg / ch + 1) : 0u;
}

// ---------------------------------------------------------------------------
// Interval spike list entry (the GPU counterpart of the spike-receive
// register): source, emission step and the entry's first chunk in the
// interval's chunk space (an exclusive prefix sum of row chunk counts).
// ---------------------------------------------------------------------------
struct SpikeEntry {
  uint32_t src;
  int32_t t;
  uint32_t choff;
  uint32_t pad;
};

// Per-net control block in device memory.
// The four counters that every update block adds to (pair, spikes,
// log_count, pending_events) sit on separate 128-byte lines: atomics on one
// line are serialised in its L2 slice, and hundreds of blocks reach them at
// the same moment.
struct Ctl {
  alignas(128) unsigned long long pair;  // (spikes << 32) | chunks of the
                                         // pending list
  unsigned int done;            // CTAs finished in the current delivery
  unsigned int error_flags;     // SNN_ERRF_*
  unsigned long long events;    // events delivered (accumulated)
  alignas(128) unsigned long long spikes;     // spikes emitted (accumulated)
  alignas(128) unsigned long long log_count;  // entries in the spike log
  alignas(128) unsigned long long pending_events;  // events of the pending
                                // list (moved to events when that list is
                                // delivered)
  alignas(128) long long t_now; // next step to update
  int iv_steps;                 // steps of the pending interval
  unsigned int ext_done;        // CTAs finished delivering an external list
  unsigned long long ext_pair;  // (spikes << 32) | chunks of an external list
  int ext_tmin, ext_tmax;       // emission-step range of an external list
  unsigned long long plastic_events;  // plastic synapse updates (accumulated)
  unsigned long long stdp_truncated;  // updates whose post-spike window
                                      // reached past the kept history
  unsigned long long gx_events;  // events of a gathered list, counted by the
                                 // delivery's CTAs (replace pending_events)
};

// "No spike yet" for the spike-time fields of the plasticity state.
constexpr int32_t kNoSpike = INT32_MIN;
constexpr int kMaxStdpHistory = 32;
constexpr uint32_t kMaxGatherParts = 64;  // exchange buffers of one delivery
// SNN_CHECK builds (-DSNN_CHECK=1) compile bounds checks into the kernels:
// a record whose target or delay lies outside the store's ranges, a tile
// index entry outside its row, or a spike list whose chunk offsets are not
// non-decreasing is skipped and raises SNN_ERRF_CHECK instead of being used.
#ifndef SNN_CHECK
#define SNN_CHECK 0
#endif
constexpr bool kChecked = SNN_CHECK != 0;

// Plasticity state of a net with STDP on its E->E synapses (see
// snn_kernels.cu); all pointers null for a static net.
struct StdpView {
  float* wp;            // plastic weight of every record (store order)
  int32_t* pre_t;       // [n] latest spike step (kNoSpike if none)
  float* pre_k;         // [n] presynaptic trace right after it
  int32_t* prev_t;      // [n] the two values before the latest spike
  float* prev_k;
  int32_t* ring_t;      // [hist][pitch] steps of the last hist spikes
  float* ring_k;        // [hist][pitch] postsynaptic trace right after each
  uint32_t* ring_n;     // [n] spikes so far (ring position = count mod hist)
  uint32_t n_exc;       // plastic: source < n_exc and target < n_exc
  uint32_t hist;        // a power of two
  float l2_plus, l2_minus;  // log2(e) h / tau_plus, log2(e) h / tau_minus
  float c_pot;              // lambda w0^(1 - mu)
  float c_dep;              // lambda alpha
  float mu, w_max;
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32->64-bit multiplications, the high halves xor-ed with the other
// counter words and the round key; the key advances by the golden-ratio
// Weyl increments between rounds.
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__host__ __device__ inline U4 philox10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint64_t m0 = (uint64_t)0xD2511F53u * c.x;
    uint64_t m1 = (uint64_t)0xCD9E8D57u * c.z;
    U4 n;
    n.x = (uint32_t)(m1 >> 32) ^ c.y ^ k0;
    n.y = (uint32_t)m1;
    n.z = (uint32_t)(m0 >> 32) ^ c.w ^ k1;
    n.w = (uint32_t)m0;
    c = n;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Random streams of the model: 0 connection (target, k), 1 initial
// potential (neuron, 0), 2 Poisson drive (neuron, step).
__host__ __device__ inline U4 draw(uint64_t seed, uint32_t a, uint64_t b,
                                   uint32_t stream) {
  U4 c{a, (uint32_t)b, (uint32_t)(b >> 32), stream};
  return philox10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// floor(u * n / 2^32)
__host__ __device__ inline uint32_t scale_u32(uint32_t u, uint32_t n) {
  return (uint32_t)(((uint64_t)u * n) >> 32);
}

// FP64 -> bfloat16 bits, round to nearest even in one step (finite inputs
// of normal float range; values below the smallest normal float flush to
// a signed zero).
__host__ __device__ inline uint16_t bf16_bits_rne(double x) {
  uint64_t b;
  memcpy(&b, &x, 8);
  uint32_t sign = (uint32_t)(b >> 63);
  int e = (int)((b >> 52) & 0x7FF);
  uint64_t mant = b & 0xFFFFFFFFFFFFFull;
  if (e == 0) return (uint16_t)(sign << 15);             // zero / subnormal
  int ef = e - 1023 + 127;                               // float exponent
  if (ef <= 0) return (uint16_t)(sign << 15);
  if (ef >= 255 || e == 0x7FF) return (uint16_t)((sign << 15) | 0x7F80u);
  // keep 7 explicit mantissa bits; 45 bits are rounded away
  uint64_t keep = mant >> 45;
  uint64_t rest = mant & ((1ull << 45) - 1);
  uint64_t half = 1ull << 44;
  if (rest > half || (rest == half && (keep & 1))) ++keep;
  uint32_t v = ((uint32_t)ef << 7) + (uint32_t)keep;     // carry may bump ef
  if (v >= 0x7F80u) v = 0x7F80u;
  return (uint16_t)((sign << 15) | v);
}

__host__ __device__ inline float bf16_to_f32(uint32_t bits16) {
  uint32_t u = bits16 << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

// ---------------------------------------------------------------------------
// Neuron update constants (FP64 on the host, rounded to float32 once).
// ---------------------------------------------------------------------------
constexpr int kMaxPoisson = 128;
struct UpdConst {
  float p11, p21, p22, p31, p32, p33;
  float psc;       // e / tau_syn
  float v_th, v_reset, w_ext;
  int refr_steps;
  int n_thr;       // 0: no drive
  uint64_t seed;
  uint32_t thr[kMaxPoisson];  // Poisson inversion thresholds (last = 2^32-1
                              // sentinel handled by n_thr)
  // guide[j] = number of thresholds thr[m] (m < n_thr - 1) with
  // thr[m] <= j * 2^24: the inversion of a word in [j 2^24, (j+1) 2^24)
  // starts its search there (the result is that of the plain search)
  uint8_t guide[256];
};

// Device view of one net.
struct NetView {
  uint32_t n;               // local neurons (targets)
  uint32_t n_src;           // store rows: sources (the whole population)
  uint32_t g0;              // global index of local neuron 0
  uint32_t pitch;           // ring-buffer row pitch (floats)
  uint32_t slot_mask;       // n_slots - 1
  uint32_t chunk;           // records per chunk
  int fmt;
  float* V;
  float* I;
  float* J;
  int32_t* refr;
  float* rb;                // [n_slots][pitch]
  uint32_t* counts;         // [n_slots][pitch] or null
  const uint64_t* row_ptr;  // [n+1]
  const void* recs;
  const uint32_t* tile_off; // [n][n_tiles + 1] row-relative tile starts
  uint32_t tile_w;          // targets per tile (tile tau: [tau tile_w, ...))
  uint32_t n_tiles;
  // plastic nets: tiles [0, pl_tiles) hold the excitatory (plastic) targets
  // and take one CTA each; the static tiles after them go tile_grp to a CTA
  uint32_t pl_tiles;
  uint32_t tile_grp;
  int d_min, d_max;         // delay range of the store
  int window;               // ring steps one interval's spikes can reach
  // bounds for the exact fixed-point accumulation of k_deliver_tiled
  uint32_t mult_max;        // most synapses sharing (source, target, delay)
  uint32_t k_in_max;        // largest in-degree
  uint32_t spikes_per_iv;   // most spikes one neuron emits per interval
  float max_abs_w;          // largest |stored weight|
  // words per accumulator cell: 2 (hi, lo), or 1 (hi only) when every
  // stored weight is a multiple of 2^-acc_qs_min, so that a launch whose
  // scale has q - s >= acc_qs_min has lo = 0 for every event
  int acc_words;
  int acc_qs_min;
  float mean_run;           // synapses per (source, tile): the mean run length
  SpikeEntry* list;         // interval list, capacity list_cap
  uint64_t list_cap;
  // partition exchange: the update also writes its spikes as {src, t} pairs
  // into xbuf (word 0: count; entries from word 4; capacity xcap).  A
  // delivery with gx set takes its list from gx_parts such buffers (gx_stride
  // words apart, capacity gx_cap entries each) instead of `list`.
  uint32_t* xbuf;
  uint32_t xcap;
  uint32_t gx_parts;
  const uint32_t* gx;
  uint64_t gx_stride;
  uint32_t gx_cap;
  uint32_t* log_src;        // spike log, capacity log_cap
  int32_t* log_t;
  uint64_t log_cap;
  Ctl* ctl;
  int plastic;              // STDP on (state in sp)
  StdpView sp;
  // long-run spike statistics (FP64 sums of integer inter-spike intervals)
  int32_t* isi_last;        // [n] latest spike step (kNoSpike if none)
  uint32_t* isi_spikes;     // [n] spikes counted
  uint32_t* isi_n;          // [n] intervals counted
  double* isi_sum;          // [n] sum of intervals (steps)
  double* isi_sq;           // [n] sum of squared intervals
};

// One net of a batch advanced by the batched kernels (device table entry).
struct BatchNet {
  NetView v;
  UpdConst c;
  int n_steps;   // steps of this net's next interval
  int pad_;
};

// Progress of one net in one launch of the persistent serving kernel
// (written by the host before the launch, counters zero).  The launch runs
// iv intervals of the net; interval r is ub update items (blocks of the
// update's threads) then nt delivery items (tiles); items are claimed in
// order through `next`, an update item of interval r once del_done >= r nt,
// a delivery item once upd_done >= (r + 1) ub.
struct alignas(128) ServeNet {  // one cache line per net (polled by CTAs)
  unsigned int next;          // next item to claim
  unsigned int upd_done;      // update items finished
  unsigned int del_done;      // delivery items finished
  unsigned int n_items;       // iv (ub + nt)
  unsigned int ub, nt, iv;
  unsigned int pad_;
  unsigned long long t_first; // globaltimer ns at the first claim
  unsigned long long t_last;  // and at the latest completion
};

// Launch-wide state of the persistent serving kernel.
struct ServeCtl {
  unsigned int error;         // SNN_ERRF_TIMEOUT when a wait gave up
  unsigned int pad_[31];
};

__device__ inline unsigned lane_id() { return threadIdx.x & 31u; }

}  // namespace snn

// Launchers implemented in the .cu files (host side).
namespace snn {
cudaError_t launch_init_v(const NetView& v, const UpdConst* c, int random,
                          cudaStream_t s);
cudaError_t launch_update(const NetView& v, const UpdConst& c, int n_steps,
                          int from_ctl_time, long long t0, cudaStream_t s);
cudaError_t launch_deliver(const NetView& v, unsigned long long* pair,
                           unsigned int* done, const SpikeEntry* list,
                           int advance_time, cudaStream_t s);
cudaError_t launch_prepare_external(const NetView& v, const uint32_t* src,
                                    const int32_t* t, uint32_t n,
                                    SpikeEntry* list,
                                    unsigned long long* pair, cudaStream_t s);
int deliver_grid_size(int fmt);
// Tile-binned delivery (see k_deliver_tiled).  from_list_range: the window
// starts at the external list's minimum emission step (ctl->ext_tmin) rather
// than at the interval start ctl->t_now.
// q - s of the delivery kernel's fixed-point scales for event bound e and
// max|w| (-1: no fixed point; the kernel sums in FP32).
int fixed_qs_host(uint64_t e, double max_abs_w);
cudaError_t launch_deliver_tiled(const NetView& v, unsigned long long* pair,
                                 unsigned int* done, const SpikeEntry* list,
                                 int from_list_range, int advance_time,
                                 cudaStream_t s);
size_t tiled_smem_bytes(const NetView& v);
// Batched kernels (serving): bmap entries are (net index, block or tile).
cudaError_t launch_update_batch(const BatchNet* nets, const uint2* bmap,
                                uint32_t n_blocks, cudaStream_t s);
cudaError_t launch_deliver_tiled_batch(int fmt, const BatchNet* nets,
                                       const uint2* bmap, uint32_t n_ctas,
                                       size_t smem, cudaStream_t s);
uint32_t update_threads();
// Threads of a persistent serving CTA (= neurons of one update item).
uint32_t serve_threads();
// The persistent serving kernel: every net of the table advances by its
// ServeNet intervals; CTAs claim ready items until none is left.  A CTA that
// finds nothing ready polls again up to spin_limit times (about 100 ns
// apart), then sets ServeCtl.error and leaves, as do all others.  n_ctas:
// the grid; smem: the largest accumulator of the nets.
cudaError_t launch_serve(int fmt, const BatchNet* nets, ServeNet* sn,
                         ServeCtl* ctl, uint32_t n_nets, uint32_t n_ctas,
                         size_t smem, unsigned long long spin_limit,
                         cudaStream_t s);
cudaError_t launch_deliver_noalloc(const NetView& v, const uint32_t* src,
                                   const int32_t* t, uint32_t n,
                                   cudaStream_t s);

// store construction
struct BuildFixed {
  uint32_t n_e, n_i, k_e, k_i;  // source populations, in-degrees
  uint32_t n_tgt, tgt0;         // local targets; global index of the first
  double w_e, w_i, sd_e, sd_i;
  int d_lo, d_hi;
  uint64_t seed;
  int clip_e, clip_i;
};
// Build kernels launched by the calling thread run as short whole-SM CTAs
// (1) or in their normal shape (0); see snn_params.build_yield.
void set_build_yield(unsigned on);
cudaError_t build_count_fixed(const BuildFixed& b, uint32_t* deg,
                              cudaStream_t s);
cudaError_t build_scatter_fixed(const BuildFixed& b, const uint64_t* row_ptr,
                                uint32_t* cursor, uint64_t* keys,
                                uint32_t tile_w, int lo_bits, cudaStream_t s);
cudaError_t build_count_edges(const uint32_t* src, uint64_t n, uint32_t* deg,
                              cudaStream_t s);
cudaError_t build_scatter_edges(const uint32_t* src, const uint32_t* tgt,
                                const uint8_t* delay, uint64_t n,
                                const uint64_t* row_ptr, uint32_t* cursor,
                                uint64_t* keys, uint32_t tile_w, int lo_bits,
                                cudaStream_t s);
// Sort every row's keys by value, pack records and write the tile index
// (n rows of n_tiles + 1 entries).  weights: either the
// fixed-rule parameters (edge_w == null) or per-edge FP64 weights.
constexpr uint32_t kSortCap = 16384;  // keys sorted in shared memory (128 KiB)
// stats (device, 2 words, zeroed by the caller): [0] = largest number of
// synapses sharing (source, target, delay); [1] = bits of the largest
// |stored weight| (a non-negative float, ordered as an unsigned integer).
cudaError_t build_sort_pack(int fmt, uint32_t n, const uint64_t* row_ptr,
                            uint64_t* keys, void* recs, const BuildFixed* b,
                            const double* edge_w, uint32_t max_row,
                            const uint32_t* long_rows, uint32_t n_long,
                            uint64_t* long_scratch,
                            const uint64_t* long_scratch_off, uint32_t tile_w,
                            int lo_bits, uint32_t n_tiles, uint32_t* tile_off,
                            uint32_t* stats, cudaStream_t s);
cudaError_t launch_fill_i32(int32_t* p, int32_t value, uint64_t n,
                            cudaStream_t s);
cudaError_t launch_list_to_arrays(const SpikeEntry* list, uint64_t n,
                                  uint32_t* src, int32_t* t, cudaStream_t s);
cudaError_t unpack_store(int fmt, const void* recs, uint64_t n_syn,
                         uint32_t* tgt, uint8_t* delay, float* w,
                         cudaStream_t s);
cudaError_t delay_range(int fmt, const void* recs, uint64_t n_syn,
                        unsigned int* dmin_dmax, cudaStream_t s);
}  // namespace snn
