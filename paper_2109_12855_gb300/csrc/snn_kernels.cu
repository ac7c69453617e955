// snn_kernels.cu -- the simulation hot path on sm_103a.
//
//  k_update   fused neuron update for one min-delay interval (Section 2.1 of
//             arXiv 2109.12855: exact integration of the linear
//             subthreshold dynamics on the 0.1 ms grid), ring-buffer slot
//             read-and-clear, Poisson drive, threshold/reset/refractoriness,
//             and warp-ballot compaction of the spikes into the interval
//             list.  Each compacted spike also reserves its source row's
//             chunks with the same 64-bit atomic, so the list carries an
//             exclusive prefix sum of chunk counts in list order (the
//             degree scan of the load-balanced expansion) with no extra pass.
//  k_deliver  spike delivery (Section 3.2, Algorithm REF): every spike's
//             target segment is expanded and each synapse adds its weight
//             into rb[(t + delay) mod S][target].  Load balance is a
//             merge-path split of the interval's chunk space: warp w takes
//             chunks [w C / W, (w+1) C / W), finds its first spike by a
//             32-ary search of the prefix sums, then walks spikes and
//             chunks.  Each lane reads its records with 16-byte loads
//             (streaming cache hint); additions are red.global.add.f32.
//  k_deliver_tiled  the default delivery (Section 3.2's target-ordered
//             access, made tile-local): one CTA per tile of targets sums
//             the interval's events for its targets in shared memory in
//             exact fixed point, then adds them into its window of the ring
//             buffer with plain coalesced read-modify-writes.
//  k_update_batch, k_deliver_tiled_batch  the same for all nets of a served
//             batch in one launch each.
//  k_prepare_external  prefix sum of chunk counts for a caller's list.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "snn_internal.cuh"

namespace snn {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kUpdThreads = 256;
constexpr int kDelThreads = 256;

__device__ __forceinline__ void red_add_f32(float* p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

__device__ __forceinline__ uint4 ld_stream16(const void* p) {
  return __ldcs(reinterpret_cast<const uint4*>(p));
}

// ---------------------------------------------------------------------------
// Initial state.
// ---------------------------------------------------------------------------
__global__ void k_init_state(NetView v, float v_reset, float v_span,
                            uint64_t seed, int random) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  float V0 = 0.0f;
  if (random) {
    U4 r = draw(seed, v.g0 + i, 0, 1u);  // keyed by the global index
    double u = (double)r.x * 0x1p-32;
    V0 = (float)((double)v_reset + (double)v_span * u);
  }
  v.V[i] = V0;
  v.I[i] = 0.0f;
  v.J[i] = 0.0f;
  v.refr[i] = 0;
}

__global__ void k_list_to_arrays(const SpikeEntry* list, uint64_t n,
                                 uint32_t* src, int32_t* t) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n;
       k += (uint64_t)gridDim.x * blockDim.x) {
    src[k] = list[k].src;
    t[k] = list[k].t;
  }
}

__global__ void k_fill_i32(int32_t* p, int32_t value, uint64_t n) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n;
       k += (uint64_t)gridDim.x * blockDim.x)
    p[k] = value;
}

// ---------------------------------------------------------------------------
// Fused update.
//
// One thread per neuron integrates its state for the interval's steps.  The
// ring-buffer values of a step are loaded in groups of eight independent
// loads ahead of use (one memory round trip per eight steps instead of one
// per step).  Spikes are kept as a per-thread bit mask of step indices and
// compacted once per warp for up to 32 steps: a warp scan of the per-thread
// counts, then one set of global atomics per warp with spikes reserves its
// list entries and chunk ranges.
// ---------------------------------------------------------------------------
constexpr int kPrefetch = 8;


// Plasticity state at a spike of excitatory neuron i at step t: the
// presynaptic trace (kept with the values before this spike, which its own
// delivery needs) and the postsynaptic ring of the last hist spikes with the
// trace right after each.  Traces decay by exp(-steps h / tau) and jump by 1.
__device__ __forceinline__ void stdp_on_spike(const StdpView& sp, uint32_t i,
                                              int32_t t, uint32_t pitch) {
  const int32_t tl = sp.pre_t[i];
  const float kl = sp.pre_k[i];
  sp.prev_t[i] = tl;
  sp.prev_k[i] = kl;
  sp.pre_k[i] =
      (tl == kNoSpike ? 0.f : kl * exp2f(-(float)(t - tl) * sp.l2_plus)) + 1.f;
  sp.pre_t[i] = t;
  const uint32_t n = sp.ring_n[i];
  const uint32_t hm = sp.hist - 1u;
  float km = 0.f;
  if (n) {
    const size_t last = (size_t)((n - 1u) & hm) * pitch + i;
    km = sp.ring_k[last] * exp2f(-(float)(t - sp.ring_t[last]) * sp.l2_minus);
  }
  const size_t slot = (size_t)(n & hm) * pitch + i;
  sp.ring_t[slot] = t;
  sp.ring_k[slot] = km + 1.f;
  sp.ring_n[i] = n + 1u;
}

// L2 prefetch of source src's row of the tile index, line by line.
__device__ __forceinline__ void prefetch_row_l2(const NetView& v, uint32_t src) {
  const char* a = reinterpret_cast<const char*>(
      v.tile_off + (uint64_t)src * (v.n_tiles + 1u));
  const char* e = a + 4ull * (v.n_tiles + 1u);
  for (const char* p = reinterpret_cast<const char*>(
           reinterpret_cast<uintptr_t>(a) & ~(uintptr_t)127);
       p < e; p += 128)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Body of the update for neuron block `block` of net v (one thread per
// neuron); shared by the single-net and the batched kernels.
// PL: the single-net update, which also keeps the plasticity state and the
// long-run spike statistics (the batched serving update does neither).
template <bool PL>
__device__ __forceinline__ void update_body(const NetView& v, const UpdConst& c,
                                            int n_steps, int from_ctl,
                                            long long t0_arg, uint32_t block) {
  __shared__ uint32_t s_thr[kMaxPoisson];
  __shared__ uint8_t s_guide[256];
  for (int k = threadIdx.x; k < c.n_thr; k += blockDim.x) s_thr[k] = c.thr[k];
  for (int k = threadIdx.x; k < 256; k += blockDim.x) s_guide[k] = c.guide[k];

  const uint32_t i = block * blockDim.x + threadIdx.x;
  const bool live = i < v.n;
  float V = 0.f, I = 0.f, J = 0.f;
  int refr = 0;
  uint32_t nch = 0;
  unsigned long long deg = 0;
  if (live) {
    V = v.V[i];
    I = v.I[i];
    J = v.J[i];
    refr = v.refr[i];
    // the neuron's own row (rows are indexed by global source)
    uint64_t beg = v.row_ptr[v.g0 + i], end = v.row_ptr[v.g0 + i + 1];
    nch = row_chunks(beg, end, v.chunk);
    deg = end - beg;
  }
  // long-run spike statistics of this neuron, read now so that their
  // latency overlaps the integration; written back once if it fired
  const bool isi = PL && v.isi_spikes && live;
  int32_t isi_last = kNoSpike;
  uint32_t isi_spk = 0, isi_cnt = 0;
  double isi_s1 = 0.0, isi_s2 = 0.0;
  bool isi_dirty = false;
  if (isi) {
    isi_last = v.isi_last[i];
    isi_spk = v.isi_spikes[i];
    isi_cnt = v.isi_n[i];
    isi_s1 = v.isi_sum[i];
    isi_s2 = v.isi_sq[i];
  }
  // the single-net update may start while the previous delivery's last
  // CTAs run (programmatic dependent launch): everything above reads only
  // what the previous update wrote; from here on the delivery's ring-buffer
  // additions, clock and counters must be complete
  if constexpr (PL) asm volatile("griddepcontrol.wait;" ::: "memory");
  const long long t0 = from_ctl ? v.ctl->t_now : t0_arg;
  if (block == 0 && threadIdx.x == 0) {
    v.ctl->iv_steps = n_steps;
    if (!from_ctl) v.ctl->t_now = t0;
  }
  __syncthreads();
  U4 rnd{0, 0, 0, 0};
  long long rnd_block = -1;
  float* const rb_i = v.rb + i;  // slot s of neuron i at rb_i[s * pitch]

  for (int s0 = 0; s0 < n_steps; s0 += 32) {
    const int ns = n_steps - s0 < 32 ? n_steps - s0 : 32;
    uint32_t mask = 0;
    for (int sb = 0; sb < ns; sb += kPrefetch) {
      // ring-buffer values and drive counts of up to eight steps, computed
      // before the (sequential) integration so they do not lengthen it
      float buf[kPrefetch];
      const long long tf = t0 + s0 + sb;  // first step of this group
      const int ng = ns - sb < kPrefetch ? ns - sb : kPrefetch;
#pragma unroll
      for (int q = 0; q < kPrefetch; ++q) {
        buf[q] = 0.f;
        if (live && q < ng)
          buf[q] = rb_i[((uint32_t)(tf + q) & v.slot_mask) * v.pitch];
      }
      if (c.n_thr > 0 && live) {
        // the group's steps lie in the 4-step draw blocks b0 .. b0 + 2;
        // the draws are independent of one another (issued together), and
        // the block drawn last is kept for the next group
        const long long b0 = tf >> 2, bl = (tf + ng - 1) >> 2;
        const uint32_t ig = v.g0 + i;  // drive keyed by the global index
        const U4 r0 = b0 == rnd_block ? rnd : draw(c.seed, ig, (uint64_t)b0, 2u);
        U4 r1 = r0, r2 = r0;
        if (bl >= b0 + 1) r1 = draw(c.seed, ig, (uint64_t)(b0 + 1), 2u);
        if (bl >= b0 + 2) r2 = draw(c.seed, ig, (uint64_t)(b0 + 2), 2u);
        rnd = bl == b0 ? r0 : bl == b0 + 1 ? r1 : r2;
        rnd_block = bl;
        const uint32_t wd[12] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y,
                                 r1.z, r1.w, r2.x, r2.y, r2.z, r2.w};
        const int a = (int)(tf & 3);
        // inversion of each step's word: the group's guide and first
        // threshold lookups are issued together (independent shared-memory
        // loads); the search goes on only where the word passes the first
        // threshold (a threshold inside its guide bucket), as the plain
        // search would
        uint32_t wq[kPrefetch];
        int kq[kPrefetch];
        uint32_t tq[kPrefetch];
#pragma unroll
        for (int q = 0; q < kPrefetch; ++q) {
          // word (tf + q) mod 4 of block (tf + q) / 4: wd[a + q]
          wq[q] = a == 0 ? wd[q] : a == 1 ? wd[q + 1]
                : a == 2 ? wd[q + 2] : wd[q + 3];
          kq[q] = s_guide[wq[q] >> 24];
        }
#pragma unroll
        for (int q = 0; q < kPrefetch; ++q) tq[q] = s_thr[kq[q]];
#pragma unroll
        for (int q = 0; q < kPrefetch; ++q) {
          if (q >= ng) continue;
          int k = kq[q];
          if (k < c.n_thr - 1 && wq[q] >= tq[q]) {
            ++k;
            while (k < c.n_thr - 1 && wq[q] >= s_thr[k]) ++k;
          }
          buf[q] += c.w_ext * (float)k;
        }
      }
#pragma unroll
      for (int q = 0; q < kPrefetch; ++q) {
        if (!live || sb + q >= ns) continue;
        const long long t = t0 + s0 + sb + q;
        // (1) membrane, unless refractory
        if (refr == 0) V = c.p31 * J + c.p32 * I + c.p33 * V;
        else refr -= 1;
        // (2) synaptic current and its derivative
        I = c.p21 * J + c.p22 * I;
        J = c.p11 * J;
        // (3) this step's ring-buffer input (read above; the slot is
        // cleared here) plus drive
        rb_i[((uint32_t)t & v.slot_mask) * v.pitch] = 0.0f;
        J += c.psc * buf[q];
        // (4) threshold
        if (V >= c.v_th) {
          V = c.v_reset;
          refr = c.refr_steps;
          mask |= 1u << (sb + q);
        }
      }
    }
    // warp compaction of this chunk's spikes: a warp with spikes scans its
    // lanes' counts and reserves its list entries, chunk ranges and log
    // slots with one set of global atomics; warps without spikes (most of
    // them at a few Hz) go on without waiting for anyone
    const uint32_t cnt = __popc(mask);
    if (__ballot_sync(kFull, cnt != 0)) {
      const unsigned lane = threadIdx.x & 31u;
      uint32_t inc_cnt = cnt, inc_ch = cnt * nch;
      unsigned long long inc_deg = (unsigned long long)cnt * deg;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t ya = __shfl_up_sync(kFull, inc_cnt, o);
        const uint32_t yb = __shfl_up_sync(kFull, inc_ch, o);
        const unsigned long long yc = __shfl_up_sync(kFull, inc_deg, o);
        if (lane >= (unsigned)o) {
          inc_cnt += ya;
          inc_ch += yb;
          inc_deg += yc;
        }
      }
      const uint32_t ex_cnt = inc_cnt - cnt, ex_ch = inc_ch - cnt * nch;
      unsigned long long old = 0ull, logb = 0ull;
      uint32_t xbase = 0u;
      if (lane == 31u) {  // the warp's totals
        // all counters first (separate lines, the returning atomics in
        // flight together), then the overflow check on the list's one
        old = atomicAdd(&v.ctl->pair, ((unsigned long long)inc_cnt << 32) | inc_ch);
        logb = v.log_cap ? atomicAdd(&v.ctl->log_count, (unsigned long long)inc_cnt)
                         : 0ull;
        xbase = v.xbuf ? atomicAdd(v.xbuf, inc_cnt) : 0u;
        atomicAdd(&v.ctl->pending_events, inc_deg);
        atomicAdd(&v.ctl->spikes, (unsigned long long)inc_cnt);
        if ((uint32_t)old + (unsigned long long)inc_ch > 0xFFFFFFFFull)
          atomicOr(&v.ctl->error_flags, (unsigned)SNN_ERRF_CHUNKS);
      }
      old = __shfl_sync(kFull, old, 31);
      logb = __shfl_sync(kFull, logb, 31);
      xbase = __shfl_sync(kFull, xbase, 31);
      uint32_t m = mask, k = 0;
      while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1u;
        const long long t = t0 + s0 + b;
        const unsigned long long idx = (old >> 32) + ex_cnt + k;
        if (idx < v.list_cap) {
          SpikeEntry e;
          e.src = v.g0 + i;
          e.t = (int32_t)t;
          e.choff = (uint32_t)old + ex_ch + k * nch;
          e.pad = 0;
          v.list[idx] = e;
          // the tiled delivery that follows reads this source's row of the
          // tile index (two words per CTA): bring the row into L2 now
          if (v.tile_off && k == 0) prefetch_row_l2(v, v.g0 + i);
        } else {
          atomicOr(&v.ctl->error_flags, (unsigned)SNN_ERRF_SPIKE_LIST);
        }
        if (v.xbuf) {  // the partition exchange's copy of the list
          const uint32_t xi = xbase + ex_cnt + k;
          if (xi < v.xcap) {
            reinterpret_cast<uint2*>(v.xbuf + 4)[xi] =
                make_uint2(v.g0 + i, (uint32_t)(int32_t)t);
          } else {
            atomicOr(&v.ctl->error_flags, (unsigned)SNN_ERRF_SPIKE_LIST);
          }
        }
        if (v.log_cap) {
          const unsigned long long li = logb + ex_cnt + k;
          if (li < v.log_cap) {
            v.log_src[li] = v.g0 + i;
            v.log_t[li] = (int32_t)t;
          } else {
            atomicOr(&v.ctl->error_flags, (unsigned)SNN_ERRF_SPIKE_LOG);
          }
        }
        if (PL && v.plastic && i < v.sp.n_exc)
          stdp_on_spike(v.sp, i, (int32_t)t, v.pitch);
        if (isi) {
          if (isi_last != kNoSpike) {
            const double d = (double)((int32_t)t - isi_last);  // exact in FP64
            isi_s1 += d;
            isi_s2 += d * d;
            isi_cnt += 1u;
          }
          isi_last = (int32_t)t;
          isi_spk += 1u;
          isi_dirty = true;
        }
        ++k;
      }
    }
  }
  if (live) {
    v.V[i] = V;
    v.I[i] = I;
    v.J[i] = J;
    v.refr[i] = refr;
  }
  if (isi_dirty) {
    v.isi_last[i] = isi_last;
    v.isi_spikes[i] = isi_spk;
    v.isi_n[i] = isi_cnt;
    v.isi_sum[i] = isi_s1;
    v.isi_sq[i] = isi_s2;
  }
}

// MINB blocks per SM: 3 leaves room for spill-free registers (a
// 112,500-neuron net's 440 blocks run in one wave); nets that need several
// waves anyway take 4, for more warps per SM.
template <int MINB>
__global__ void __launch_bounds__(kUpdThreads, MINB)
k_update(NetView v, UpdConst c, int n_steps, int from_ctl, long long t0_arg) {
  update_body<true>(v, c, n_steps, from_ctl, t0_arg, blockIdx.x);
}

// All nets of a batch in one launch: block b updates neuron block bmap[b].y
// of net bmap[b].x, from that net's clock.
__global__ void __launch_bounds__(kUpdThreads, 3)
k_update_batch(const BatchNet* __restrict__ nets, const uint2* __restrict__ bmap) {
  __shared__ UpdConst s_c;
  const uint2 m = bmap[blockIdx.x];
  const BatchNet& bn = nets[m.x];
  const uint32_t* src = reinterpret_cast<const uint32_t*>(&bn.c);
  uint32_t* dst = reinterpret_cast<uint32_t*>(&s_c);
  for (uint32_t k = threadIdx.x; k < sizeof(UpdConst) / 4; k += blockDim.x)
    dst[k] = src[k];
  const NetView v = bn.v;
  const int n_steps = bn.n_steps;
  __syncthreads();
  update_body<false>(v, s_c, n_steps, 1, 0, m.y);  // served nets are static
}

// ---------------------------------------------------------------------------
// Delivery.
// ---------------------------------------------------------------------------
template <int FMT> struct Loaded;
template <> struct Loaded<SNN_W_FP32_12B> { uint4 a, b, c; };
template <> struct Loaded<SNN_W_BF16_8B> { uint4 a; };

template <int FMT>
__device__ __forceinline__ Loaded<FMT> load_lane(const void* recs,
                                                 uint64_t rec_index);
template <>
__device__ __forceinline__ Loaded<SNN_W_FP32_12B> load_lane<SNN_W_FP32_12B>(
    const void* recs, uint64_t r) {
  const char* p = reinterpret_cast<const char*>(recs) + r * 12u;
  Loaded<SNN_W_FP32_12B> x;
  x.a = ld_stream16(p);
  x.b = ld_stream16(p + 16);
  x.c = ld_stream16(p + 32);
  return x;
}
template <>
__device__ __forceinline__ Loaded<SNN_W_BF16_8B> load_lane<SNN_W_BF16_8B>(
    const void* recs, uint64_t r) {
  Loaded<SNN_W_BF16_8B> x;
  x.a = ld_stream16(reinterpret_cast<const char*>(recs) + r * 8u);
  return x;
}

// Record q (0 .. kPerLane-1) of a lane's loaded bytes.
template <int FMT>
__device__ __forceinline__ void unpack(const Loaded<FMT>& x, int q,
                                       uint32_t& tgt, uint32_t& d, float& w);
template <>
__device__ __forceinline__ void unpack<SNN_W_FP32_12B>(
    const Loaded<SNN_W_FP32_12B>& x, int q, uint32_t& tgt, uint32_t& d,
    float& w) {
  // 48 bytes = words a.x a.y a.z a.w b.x ... c.w; record q = words 3q..3q+2
  uint32_t wd[12] = {x.a.x, x.a.y, x.a.z, x.a.w, x.b.x, x.b.y,
                     x.b.z, x.b.w, x.c.x, x.c.y, x.c.z, x.c.w};
  tgt = wd[3 * q];
  w = __uint_as_float(wd[3 * q + 1]);
  d = wd[3 * q + 2] & 0xFFu;
}
template <>
__device__ __forceinline__ void unpack<SNN_W_BF16_8B>(
    const Loaded<SNN_W_BF16_8B>& x, int q, uint32_t& tgt, uint32_t& d,
    float& w) {
  uint32_t t0 = q == 0 ? x.a.x : x.a.z;
  uint32_t m0 = q == 0 ? x.a.y : x.a.w;
  tgt = t0;
  d = m0 & 0xFFu;
  w = __uint_as_float(m0 & 0xFFFF0000u);
}

// Bounds-checked builds: a record whose target lies outside [lo, lo + width)
// (or the net) or whose delay lies outside the store's range is skipped
// and flagged.  Production builds compile this to `true`.
__device__ __forceinline__ bool rec_in_bounds(const NetView& v, uint32_t tgt,
                                              uint32_t d, uint32_t lo,
                                              uint32_t width) {
  if (!kChecked) return true;
  const bool ok = tgt - lo < width && tgt < v.n && d >= (uint32_t)v.d_min &&
                  d <= (uint32_t)v.d_max;
  if (!ok) atomicOr(&v.ctl->error_flags, (unsigned)SNN_ERRF_CHECK);
  return ok;
}

template <int FMT, bool COUNT>
__global__ void __launch_bounds__(kDelThreads)
k_deliver(NetView v, unsigned long long* pair_p, unsigned int* done_p,
          const SpikeEntry* __restrict__ list, int advance_time) {
  constexpr int CH = Fmt<FMT>::kChunk;
  constexpr int PL = Fmt<FMT>::kPerLane;
  constexpr int G = FMT == SNN_W_FP32_12B ? 4 : 8;  // chunks in flight / warp
  __shared__ unsigned long long s_pair;
  if (threadIdx.x == 0) s_pair = *reinterpret_cast<volatile unsigned long long*>(pair_p);
  __syncthreads();
  const uint32_t n_sp = (uint32_t)(s_pair >> 32);
  const uint64_t n_ch = (uint32_t)s_pair;
  const unsigned lane = threadIdx.x & 31u;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t c_begin = warp * n_ch / n_warps;
  const uint64_t c_end = (warp + 1) * n_ch / n_warps;

  if (c_begin < c_end) {
    // last spike j with choff[j] <= c_begin (choff is non-decreasing)
    uint32_t lo = 0, hi = n_sp;
    while (hi - lo > 32) {
      uint32_t p = lo + (uint32_t)(((uint64_t)(hi - lo) * lane) >> 5);
      bool le = list[p].choff <= c_begin;
      unsigned m = __ballot_sync(kFull, le);
      int last = 31 - __clz(m);
      uint32_t nlo = __shfl_sync(kFull, p, last);
      uint32_t nhi = __shfl_sync(kFull, p, last < 31 ? last + 1 : 31);
      lo = nlo;
      hi = last < 31 ? nhi : hi;
    }
    {
      uint32_t p = lo + lane;
      bool le = p < hi && list[p].choff <= c_begin;
      unsigned m = __ballot_sync(kFull, le);
      lo = lo + (31 - __clz(m));
    }
    uint32_t j = lo;
    uint64_t c = c_begin;
    uint32_t prev_choff = 0u;
    while (c < c_end && j < n_sp) {
      const SpikeEntry e = list[j];
      ++j;
      if (kChecked) {  // the merge-path split needs non-decreasing offsets
        if (e.choff < prev_choff) {
          atomicOr(&v.ctl->error_flags, (unsigned)SNN_ERRF_CHECK);
          break;
        }
        prev_choff = e.choff;
      }
      if (e.src >= v.n_src) continue;
      const uint64_t beg = v.row_ptr[e.src], end = v.row_ptr[e.src + 1];
      const uint64_t last = (uint64_t)e.choff + row_chunks(beg, end, CH);
      const uint64_t stop = last < c_end ? last : c_end;
      if (c < e.choff) c = e.choff;   // (only if entries were skipped)
      const int64_t abs0 = (int64_t)(beg / CH) - (int64_t)e.choff;
      const int32_t t = e.t;
      for (; c < stop; c += G) {
        Loaded<FMT> x[G];
#pragma unroll
        for (int g = 0; g < G; ++g)
          if (c + g < stop)
            x[g] = load_lane<FMT>(v.recs,
                                  (uint64_t)(abs0 + (int64_t)(c + g)) * CH +
                                      lane * PL);
#pragma unroll
        for (int g = 0; g < G; ++g) {
          if (c + g < stop) {
            const uint64_t r0 =
                (uint64_t)(abs0 + (int64_t)(c + g)) * CH + lane * PL;
#pragma unroll
            for (int q = 0; q < PL; ++q) {
              const uint64_t r = r0 + q;
              if (r >= beg && r < end) {
                uint32_t tgt, d;
                float w;
                unpack<FMT>(x[g], q, tgt, d, w);
                if (!rec_in_bounds(v, tgt, d, 0u, v.n)) continue;
                const size_t cell =
                    (size_t)(((uint32_t)t + d) & v.slot_mask) * v.pitch + tgt;
                red_add_f32(v.rb + cell, w);
                if (COUNT) atomicAdd(v.counts + cell, 1u);
              }
            }
          }
        }
      }
      c = stop;
    }
  }

  // The last CTA to finish clears the list counters for the next interval
  // (every CTA read them before arriving here) and advances the clock.
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned prev = atomicAdd(done_p, 1u);
    if (prev == gridDim.x - 1) {
      *pair_p = 0ull;
      *done_p = 0u;
      if (advance_time) {  // the interval's own list: commit its events
        if (v.xbuf) *v.xbuf = 0u;  // the next update refills the exchange list
        v.ctl->t_now += v.ctl->iv_steps;
        v.ctl->events += v.ctl->pending_events;
        v.ctl->pending_events = 0ull;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Tile-binned delivery.
//
// CTA tau owns the targets [tau TW, (tau+1) TW) and accumulates, in shared
// memory, every event of the list aimed at them for the ring steps
// base .. base + window - 1 that one interval can reach (base = interval
// start + min delay).  Rows are sorted by target tile, so the records of
// spike j for tile tau are one contiguous run, located by the row's tile
// index.  (A) the CTA describes a batch of runs in shared memory; (B) its 32
// warps take U runs at a time from a shared counter and load up to PER
// records per lane of each before adding any (independent loads in flight).
// (Staging the runs through shared memory, with bulk copies or per-lane
// asynchronous copies, was measured slower: each record then passes through
// shared memory twice beside its two atomics, and every run of ~74 records
// pays a copy and a wait.)
//
// Accumulation is exact fixed point: a weight w becomes x = w 2^(q-s),
// split into hi = rint(x) and lo = rint((x - hi) 2^s) in [-2^(s-1), 2^(s-1)]
// (hi 2^s + lo = rint(w 2^q)); hi and lo are summed in two int32 arrays
// with shared-memory integer atomics, so the sum is order-independent and
// the cell value is (H 2^s + L) 2^-q.  The scales come from bounds on one
// launch: a cell receives at most E = min(spikes x max synapse
// multiplicity, max in-degree x spikes per neuron per interval) events of
// magnitude <= max|w|; s makes E 2^s < 2^31 and q makes
// E max|w| 2^(q-s) + E < 2^31, so neither sum can overflow, and the
// rounding error (<= 2^-(q+1) per event) is below that of FP32
// accumulation.  If no such scales exist the CTA falls back to FP32
// shared-memory atomics.  The CTA then adds its cells into the ring buffer
// with plain coalesced read-modify-writes: no other CTA touches them.
// An external list whose emission steps span more than the window is
// delivered by the same CTAs with global atomics instead.
// ---------------------------------------------------------------------------
constexpr int kTileThreads = 1024;
constexpr int kTileWarps = kTileThreads / 32;

template <int FMT> struct Rec1;
template <> struct Rec1<SNN_W_FP32_12B> { uint32_t a, b, c; };
template <> struct Rec1<SNN_W_BF16_8B> { uint32_t a, b; };

template <int FMT>
__device__ __forceinline__ Rec1<FMT> load_rec(const void* recs, uint64_t r);
template <>
__device__ __forceinline__ Rec1<SNN_W_FP32_12B> load_rec<SNN_W_FP32_12B>(
    const void* recs, uint64_t r) {
  const uint32_t* p = reinterpret_cast<const uint32_t*>(recs) + r * 3u;
  Rec1<SNN_W_FP32_12B> x;
  x.a = __ldcs(p);
  x.b = __ldcs(p + 1);
  x.c = __ldcs(p + 2);
  return x;
}
template <>
__device__ __forceinline__ Rec1<SNN_W_BF16_8B> load_rec<SNN_W_BF16_8B>(
    const void* recs, uint64_t r) {
  const uint2 u = __ldcs(reinterpret_cast<const uint2*>(recs) + r);
  Rec1<SNN_W_BF16_8B> x;
  x.a = u.x;
  x.b = u.y;
  return x;
}
// FP32 records, interval-list launches: only the weight and the delay word,
// whose upper 24 bits hold the record's cell in its tile's window,
// d TW + (target - first target of the tile), written by the store build.
__device__ __forceinline__ Rec1<SNN_W_FP32_12B> load_rec_wc(const void* recs,
                                                           uint64_t r) {
  const uint32_t* p = reinterpret_cast<const uint32_t*>(recs) + r * 3u;
  Rec1<SNN_W_FP32_12B> x;
  x.a = 0u;
  x.b = __ldcs(p + 1);
  x.c = __ldcs(p + 2);
  return x;
}
__device__ __forceinline__ void rec_fields(const Rec1<SNN_W_FP32_12B>& x,
                                           uint32_t& tgt, uint32_t& d,
                                           float& w) {
  tgt = x.a;
  w = __uint_as_float(x.b);
  d = x.c & 0xFFu;
}
__device__ __forceinline__ void rec_fields(const Rec1<SNN_W_BF16_8B>& x,
                                           uint32_t& tgt, uint32_t& d,
                                           float& w) {
  tgt = x.a;
  d = x.b & 0xFFu;
  w = __uint_as_float(x.b & 0xFFFF0000u);
}

// Per-spike run of records for this CTA's tile.
struct SegDesc {
  uint64_t beg;
  uint32_t len;
  int32_t t;
};

// Fixed-point scales of one launch (see above); fixed = 0: use FP32.
struct FixScale {
  int fixed;
  int sh;          // s
  float scale_hs;  // 2^(q - s)
  float scale_s;   // 2^s
  float inv_q;     // 2^-q (q <= 123: a normal float)
  float scale_sq;  // 2^(s-q)
};

// 2^k from the exponent bits (k inside the normal range of the type), and
// floor(log2 x) of a positive normal double.
__device__ __forceinline__ float pow2f(int k) {
  return __int_as_float((k + 127) << 23);
}
__device__ __forceinline__ double pow2d(int k) {
  return __longlong_as_double((long long)(k + 1023) << 52);
}
__device__ __forceinline__ int ilog2d(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF) - 1023;
}

// Largest s <= 23 and q - s <= 21 - ceil(log2 max|w|): a scaled weight
// x = w 2^(q-s) then has |x| < 2^22 and |(x - rint x) 2^s| <= 2^22, the
// range in which adding 1.5 2^23 rounds to an integer (fixed_split).
constexpr int kFixMaxShift = 23;

__device__ FixScale fix_scale(const NetView& v, uint64_t n_sp,
                              bool per_interval) {
  FixScale f{0, 0, 1.f, 1.f, 1.f, 1.f};
  uint64_t e = n_sp * (uint64_t)(v.mult_max ? v.mult_max : 1u);
  if (per_interval) {
    const uint64_t e2 = (uint64_t)v.k_in_max * (v.spikes_per_iv ? v.spikes_per_iv : 1u);
    if (e2 < e) e = e2;
  }
  if (e == 0 || e >= (1ull << 30) || !(v.max_abs_w > 0.f) ||
      !(v.max_abs_w <= 3.0e38f))
    return f;
  const int lg = 63 - __clzll((long long)e);  // 2^lg <= e < 2^(lg+1)
  const int sh = min(30 - lg, kFixMaxShift);  // e 2^sh < 2^31
  // largest qs with e max|w| 2^qs <= 2^31 - 1 - e: the hi sums (each
  // |hi| <= |x| + 1/2) cannot overflow
  const double A = 2147483647.0 - (double)e;
  const double B = (double)e * (double)v.max_abs_w;
  int qs = ilog2d(A) - ilog2d(B);  // floor(log2(A / B)) is qs or qs - 1
  if (B * pow2d(qs) > A) --qs;
  const uint32_t wb = __float_as_uint(v.max_abs_w);
  const int wexp = (int)((wb >> 23) & 0xFFu) - 127 + ((wb & 0x7FFFFFu) ? 1 : 0);
  qs = min(qs, 21 - wexp);
  if (qs < 0) return f;
  qs = min(qs, 100);
  // one-word cells hold hi only: lo must be zero for every weight
  if (v.acc_words == 1 && qs < v.acc_qs_min) return f;
  const int q = sh + qs;
  f.fixed = 1;
  f.sh = sh;
  f.scale_hs = pow2f(qs);
  f.scale_s = pow2f(sh);
  f.inv_q = pow2f(-q);
  f.scale_sq = pow2f(-qs);
  return f;
}

// Exact split of x = w 2^(q-s) (|x| < 2^22, s <= 23): hi = rint(x),
// lo = rint((x - hi) 2^s), so hi 2^s + lo = rint(w 2^q).  Adding
// M = 1.5 2^23 puts a value of magnitude <= 2^22 into [2^23, 2^24], where
// the float spacing is 1: the sum is rounded to an integer (to nearest,
// ties to even) whose value is the bit pattern minus M's.  Only FMA-pipe
// arithmetic and integer subtractions; x - hi is exact.
__device__ __forceinline__ void fixed_split(float w, const FixScale& fx,
                                            int& hi, int& lo) {
  constexpr float kM = 12582912.0f;  // 1.5 * 2^23
  const float x = __fmul_rn(w, fx.scale_hs);
  const float y = __fadd_rn(x, kM);
  hi = __float_as_int(y) - __float_as_int(kM);
  const float fr = __fsub_rn(x, __fsub_rn(y, kM));
  lo = __float_as_int(__fmaf_rn(fr, fx.scale_s, kM)) - __float_as_int(kM);
}

// Plastic weight of an E->E synapse at its presynaptic spike t with delay
// d (pair-based power-law STDP, all pairs, the whole delay dendritic): the
// potentiation owed to the post spikes seen since the previous pre spike,
// in time order, then the depression by the post trace at t; weights stay in
// [0, w_max].  tprev / kprev: the previous pre spike and the presynaptic
// trace right after it.  The post spikes of target j come from the CTA's
// copy of its last hist spike times (rt: [hist][TW]; n: spikes so far); km
// is its post trace at t - d (from the CTA's table).
// Compiled once (not inlined into every unrolled record slot: the code would
// no longer fit the instruction cache).  .trunc = 1 when the potentiation
// window reached past the kept spikes.
struct StdpConst {
  float c_pot, c_dep, mu, w_max, l2_plus, l2_minus;
  uint32_t hmask;
};
struct StdpOut {
  float w;
  uint32_t trunc;
};

__device__ __noinline__ StdpOut stdp_weight(float w, int32_t t, uint32_t d,
                                            int32_t tprev, float kprev,
                                            uint32_t j, uint32_t TW,
                                            const int32_t* rt, float km,
                                            uint32_t n, StdpConst c) {
  StdpOut o;
  o.trunc = 0u;
  if (tprev != kNoSpike) {
    // post spikes seen in (previous pre spike, t]: newest first to find
    // the window, then applied oldest first
    const uint32_t H = c.hmask + 1u;
    const int32_t horizon = t - (int32_t)d;
    const int32_t after = tprev - (int32_t)d;
    const int32_t k_min = n > H ? (int32_t)(n - H) : 0;
    int32_t k_hi = -1, k_lo = -1, k = (int32_t)n - 1;
    for (; k >= k_min; --k) {
      const int32_t tp = rt[((uint32_t)k & c.hmask) * TW + j];
      if (tp > horizon) continue;
      if (tp <= after) break;
      if (k_hi < 0) k_hi = k;
      k_lo = k;
    }
    o.trunc = (k < k_min && n > H) ? 1u : 0u;
    if (k_lo >= 0) {
      for (int32_t q = k_lo; q <= k_hi; ++q) {
        const int32_t tp = rt[((uint32_t)q & c.hmask) * TW + j];
        const float kp =
            kprev * exp2f(-(float)(tp + (int32_t)d - tprev) * c.l2_plus);
        const float wm = w > 0.f ? exp2f(c.mu * log2f(w)) : 0.f;
        w = fminf(w + c.c_pot * wm * kp, c.w_max);
      }
    }
  }
  // depression by the post trace at t (from the CTA's table)
  o.w = fmaxf(w - c.c_dep * w * km, 0.f);
  return o;
}

// FAST: an interval's own list (inside the window) whose fixed-point scales
// the host has shown to exist for every spike count: no per-event test of
// either.
// ONE: one-word cells known at compile time (BF16 stores).  SHORT: runs of
// a few dozen records (BF16, static): eight runs per warp pass, each on half
// a warp (48 record slots per run instead of 96).
template <int FMT, bool COUNT, bool PL, bool FAST = false, bool ONE = false,
          bool SHORT = false, bool GX = false>
__device__ __forceinline__ void deliver_tile_body(
    const NetView& v, unsigned long long* pair_p, unsigned int* done_p,
    const SpikeEntry* __restrict__ list, int from_list_range, int advance_time,
    uint32_t tile, int* acc_mem, uint32_t desc_off, uint32_t desc_cap) {
  // U runs per warp pass, PER records per lane of each loaded before use
  // (plastic nets also hold each record's plastic weight: fewer runs)
  constexpr int U = PL ? (FMT == SNN_W_FP32_12B ? 1 : 2)
                       : (FMT == SNN_W_FP32_12B ? 2 : (SHORT ? 8 : 4));
  constexpr int PER = 3;
  // lanes per run: short runs take half a warp each, two side by side (48
  // record slots per run instead of a whole warp's)
  constexpr int LG = SHORT ? 16 : 32;
  constexpr int G = 32 / LG;   // runs side by side in a warp
  constexpr int UR = U / G;    // run slots of a lane per pass
  static_assert(U % G == 0, "runs per pass must fill the warp");
  // FP32 interval lists: each record's cell comes precomputed in its delay
  // word (no target load, no d TW + target arithmetic); bounds-checked
  // builds keep the checked form
  constexpr bool CELL = FAST && FMT == SNN_W_FP32_12B && !PL && !COUNT && !kChecked;
  // run descriptors of one batch (desc_cap spikes), after the accumulator
  SegDesc* const s_desc =
      reinterpret_cast<SegDesc*>(reinterpret_cast<char*>(acc_mem) + desc_off);
  int32_t* const s_tprev = reinterpret_cast<int32_t*>(s_desc + desc_cap);  // PL
  float* const s_kprev = reinterpret_cast<float*>(s_tprev + desc_cap);     // PL
  __shared__ unsigned long long s_pl[2];             // plastic updates, truncations
  __shared__ uint32_t s_next;                        // next run of the batch
  __shared__ FixScale s_fx;
  const uint32_t TW = v.tile_w;
  const uint32_t W = (uint32_t)v.window;
  const uint32_t cells = W * TW;
  // hi and lo words per cell (FP32 stores always use two: their 24-bit
  // significands never sit on a grid as coarse as a launch's step)
  const bool two = FMT == SNN_W_FP32_12B || (!ONE && v.acc_words == 2);
  const uint32_t acc_len = two ? 2 * cells : cells;
  const uint32_t tgt_lo = tile * TW;
  const unsigned lane = threadIdx.x & 31u;
  const uint32_t warp = threadIdx.x >> 5;
  // An interval's own list (capacity list_cap): this thread's first list
  // entries are read together with the list's length, not after it (one
  // memory round trip fewer before the runs can be described); entries past
  // the length are never used.
  constexpr int kDU = PL ? 1 : 4;
  // GX: the list is gathered from the partitions' exchange buffers (v.gx)
  constexpr bool gathered = GX;
  SpikeEntry pre[GX ? 1 : kDU];
  uint2 pre_g[GX ? kDU : 1];
  const bool spec = !from_list_range;
  if (spec) {
#pragma unroll
    for (int u = 0; u < kDU; ++u) {
      const uint32_t k = threadIdx.x + u * blockDim.x;
      if constexpr (GX) {  // part 0's first entries (its count comes next)
        if (k < desc_cap && k < v.gx_cap)
          pre_g[u] = reinterpret_cast<const uint2*>(v.gx + 4)[k];
      } else {
        if (k < desc_cap && k < v.list_cap) pre[u] = list[k];
      }
    }
  }
  // every thread reads the launch's list size and window (same addresses);
  // thread 0 derives the fixed-point scales meanwhile
  uint32_t n_sp;
  // a list gathered from the partitions: the parts' counts (each at most
  // its capacity) and their starts in the union, in part order; every
  // thread computes them (same values, no barrier) from the same words
  __shared__ uint32_t s_gstart[kMaxGatherParts + 1];
  if constexpr (GX) {
    uint32_t run = 0;
    for (uint32_t p = 0; p < v.gx_parts; ++p) {
      s_gstart[p] = run;
      run += min(*reinterpret_cast<const volatile uint32_t*>(
                     v.gx + (uint64_t)p * v.gx_stride),
                 v.gx_cap);
    }
    s_gstart[v.gx_parts] = run;
    n_sp = run;
  } else {
    const unsigned long long pr =
        *reinterpret_cast<volatile unsigned long long*>(pair_p);
    n_sp = (uint32_t)(pr >> 32);
  }
  long long base;
  bool inwin;
  // gathered lists: steps of this interval lie in [t_now, t_now + iv_span)
  const long long t_now = gathered ? v.ctl->t_now : 0ll;
  const uint32_t iv_span = (uint32_t)(W - (uint32_t)(v.d_max - v.d_min));
  if (from_list_range) {
    const long long tmin = v.ctl->ext_tmin, tmax = v.ctl->ext_tmax;
    base = tmin + v.d_min;
    inwin = (tmax - tmin) + (v.d_max - v.d_min) + 1 <= (long long)W;
  } else {
    base = v.ctl->t_now + v.d_min;
    inwin = true;
  }
  if (threadIdx.x == 0) {
    s_fx = fix_scale(v, n_sp, !from_list_range);
    s_next = 0u;
  }
  int* accH = acc_mem;                                // fixed: hi parts
  int* accL = acc_mem + cells;                        // fixed: lo parts (two)
  float* accF = reinterpret_cast<float*>(acc_mem);    // FP32 fallback
  for (uint32_t x = threadIdx.x; x < acc_len; x += blockDim.x) acc_mem[x] = 0;
  // plastic nets: the post-spike times of this tile's targets (rings) and
  // their post traces at the W horizons (t - d) this interval can ask for
  int32_t* s_rt = acc_mem + acc_len;                             // [hist][TW]
  uint32_t* s_rn = reinterpret_cast<uint32_t*>(s_rt + (PL ? v.sp.hist * TW : 0));
  float* s_km = reinterpret_cast<float*>(s_rn + (PL ? TW : 0));  // [W][TW]
  const bool tile_plastic = PL && tgt_lo < v.sp.n_exc;
  uint32_t my_pl = 0, my_trunc = 0;
  // first horizon: (interval start) - d_max
  const long long h_lo = base - v.d_min - v.d_max;
  if (PL) {
    if (threadIdx.x < 2) s_pl[threadIdx.x] = 0ull;
    if (tile_plastic) {
      for (uint32_t x = threadIdx.x; x < TW; x += blockDim.x)
        s_rn[x] = tgt_lo + x < v.n ? v.sp.ring_n[tgt_lo + x] : 0u;
      for (uint32_t x = threadIdx.x; x < v.sp.hist * TW; x += blockDim.x) {
        const uint32_t q = x / TW, jj = x - q * TW;
        if (tgt_lo + jj < v.n)
          s_rt[x] = v.sp.ring_t[(size_t)q * v.pitch + tgt_lo + jj];
      }
      __syncthreads();
      // post trace of target j at horizon h: the trace right after its
      // latest spike at or before h, decayed to h (0 if it never fired)
      const uint32_t hm = v.sp.hist - 1u;
      for (uint32_t x = threadIdx.x; x < W * TW; x += blockDim.x) {
        const uint32_t hi = x / TW, jj = x - hi * TW;
        const int32_t h = (int32_t)(h_lo + hi);
        const uint32_t n = s_rn[jj];
        const int32_t k_min = n > v.sp.hist ? (int32_t)(n - v.sp.hist) : 0;
        float km = 0.f;
        int32_t k = (int32_t)n - 1;
        for (; k >= k_min; --k) {
          const int32_t tp = s_rt[((uint32_t)k & hm) * TW + jj];
          if (tp <= h) {
            km = v.sp.ring_k[(size_t)((uint32_t)k & hm) * v.pitch + tgt_lo + jj] *
                 exp2f(-(float)(h - tp) * v.sp.l2_minus);
            break;
          }
        }
        // every kept spike is after h but older ones were dropped: the
        // trace at h is unknown (-1; an update that needs it is counted
        // with the truncated windows)
        s_km[x] = (k < k_min && n > v.sp.hist) ? -1.f : km;
      }
    }
  }
  const uint32_t row_stride = v.n_tiles + 1;
  FixScale fx{};  // thread 0's s_fx, read after the first barrier
  __shared__ unsigned long long s_events;  // gathered lists: this CTA's events
  if (gathered && threadIdx.x == 0) s_events = 0ull;

  // one event: cell = d TW + tgt + off, off = (t - base) TW - tgt_lo per run
  auto add = [&](uint32_t tgt, int32_t t, int32_t off, uint32_t d, float w) {
    if (FAST || inwin) {
      const uint32_t cell = d * TW + tgt + (uint32_t)off;
      if (FAST || fx.fixed) {
        int hi, lo;
        fixed_split(w, fx, hi, lo);
        atomicAdd(&accH[cell], hi);
        // BF16 weights have 8 significant bits: their scaled value is
        // usually an integer, and a zero low part needs no addition (with
        // one-word cells it is zero for every event)
        if (two && (FMT == SNN_W_FP32_12B || lo != 0)) atomicAdd(&accL[cell], lo);
      } else {
        atomicAdd(&accF[cell], w);
      }
    } else {
      const uint32_t step = (uint32_t)t + d;
      red_add_f32(v.rb + (size_t)(step & v.slot_mask) * v.pitch + tgt, w);
    }
    if (COUNT)
      atomicAdd(v.counts + (size_t)(((uint32_t)t + d) & v.slot_mask) * v.pitch + tgt,
                1u);
  };
  // one event of an interval list (in the window, fixed point) by its cell
  auto add_cell = [&](uint32_t cell, float w) {
    int hi, lo;
    fixed_split(w, fx, hi, lo);
    atomicAdd(&accH[cell], hi);
    atomicAdd(&accL[cell], lo);
  };

  // plastic E->E synapse: update its weight (record index r), store it
  StdpConst sc{};
  if (PL) {
    sc.c_pot = v.sp.c_pot;
    sc.c_dep = v.sp.c_dep;
    sc.mu = v.sp.mu;
    sc.w_max = v.sp.w_max;
    sc.l2_plus = v.sp.l2_plus;
    sc.l2_minus = v.sp.l2_minus;
    sc.hmask = v.sp.hist - 1u;
  }
  auto plastic = [&](uint32_t tgt, uint32_t k_run, int32_t t, uint32_t d,
                     float w, uint64_t r) -> float {
    const uint32_t j = tgt - tgt_lo;
    const float km = s_km[(uint32_t)((long long)t - (long long)d - h_lo) * TW + j];
    const StdpOut o = stdp_weight(w, t, d, s_tprev[k_run], s_kprev[k_run], j,
                                  TW, s_rt, fmaxf(km, 0.f), s_rn[j], sc);
    v.sp.wp[r] = o.w;
    ++my_pl;
    my_trunc += o.trunc | (km < 0.f ? 1u : 0u);
    return o.w;
  };
  const uint32_t sub = lane & (uint32_t)(LG - 1);  // lane within its run
  const uint32_t grp = lane / (uint32_t)LG;         // run side of the warp
  auto load_pass = [&](Rec1<FMT> (&r)[UR][PER], float (&wv)[UR][PER], uint32_t k0,
                       uint32_t nb) {
#pragma unroll
    for (int u = 0; u < UR; ++u) {
      const uint32_t j = k0 + (uint32_t)(G * u) + grp;
      const bool ok = j < nb;
      const uint64_t beg = ok ? s_desc[j].beg : 0ull;
      const uint32_t len = ok ? s_desc[j].len : 0u;
      const bool pl = PL && tile_plastic && ok && s_kprev[j] >= 0.f;
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const uint32_t idx = sub + (uint32_t)LG * q;
        if (idx < len) {
          if constexpr (CELL)
            r[u][q] = load_rec_wc(v.recs, beg + idx);
          else
            r[u][q] = load_rec<FMT>(v.recs, beg + idx);
          if (pl) wv[u][q] = __ldcs(v.sp.wp + beg + idx);
        }
      }
    }
  };
  auto add_pass = [&](const Rec1<FMT> (&r)[UR][PER], const float (&wv)[UR][PER],
                      uint32_t k0, uint32_t nb) {
#pragma unroll
    for (int u = 0; u < UR; ++u) {
      const uint32_t j = k0 + (uint32_t)(G * u) + grp;
      if (j >= nb) {
        if constexpr (G == 1) break;  // (uniform across the warp)
        else continue;
      }
      const SegDesc sd = s_desc[j];
      const int32_t roff = (int32_t)(((long long)sd.t - base) * (long long)TW);
      const int32_t off = roff - (int32_t)tgt_lo;
      const bool pl = PL && tile_plastic && s_kprev[j] >= 0.f;
      if constexpr (CELL) {
#pragma unroll
        for (int q = 0; q < PER; ++q) {
          const uint32_t idx = sub + (uint32_t)LG * q;
          if (idx < sd.len)
            add_cell((r[u][q].c >> 8) + (uint32_t)roff, __uint_as_float(r[u][q].b));
        }
        for (uint32_t idx = (uint32_t)LG * PER + sub; idx < sd.len; idx += (uint32_t)LG) {
          const Rec1<FMT> x = load_rec_wc(v.recs, sd.beg + idx);
          add_cell((x.c >> 8) + (uint32_t)roff, __uint_as_float(x.b));
        }
        continue;
      }
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const uint32_t idx = sub + (uint32_t)LG * q;
        if (idx < sd.len) {
          uint32_t tgt, d;
          float w;
          rec_fields(r[u][q], tgt, d, w);
          if (!rec_in_bounds(v, tgt, d, tgt_lo, TW)) continue;
          if (pl && tgt < v.sp.n_exc)
            w = plastic(tgt, j, sd.t, d, wv[u][q], sd.beg + idx);
          add(tgt, sd.t, off, d, w);
        }
      }
      for (uint32_t idx = (uint32_t)LG * PER + sub; idx < sd.len; idx += (uint32_t)LG) {
        uint32_t tgt, d;
        float w;
        rec_fields(load_rec<FMT>(v.recs, sd.beg + idx), tgt, d, w);
        if (!rec_in_bounds(v, tgt, d, tgt_lo, TW)) continue;
        if (pl && tgt < v.sp.n_exc)
          w = plastic(tgt, j, sd.t, d, __ldcs(v.sp.wp + sd.beg + idx),
                      sd.beg + idx);
        add(tgt, sd.t, off, d, w);
      }
    }
  };

  // (A) describe the runs of spikes [j0, j0 + nb): kDU list entries per
  // thread in flight (the first ones already read), then their tile-index
  // words and row starts
  auto describe = [&](uint32_t j0, uint32_t nb) {
    unsigned long long my_events = 0;
    for (uint32_t k0 = threadIdx.x; k0 < nb; k0 += kDU * blockDim.x) {
      SpikeEntry e[kDU];
      const bool have = spec && j0 == 0 && k0 == threadIdx.x;
#pragma unroll
      for (int u = 0; u < kDU; ++u) {
        const uint32_t k = k0 + u * blockDim.x;
        if (k < nb) {
          if constexpr (GX) {
            const uint32_t g = j0 + k;
            uint32_t p = 0;
            while (s_gstart[p + 1] <= g) ++p;
            const uint2 x = (have && p == 0)
                ? pre_g[u]
                : reinterpret_cast<const uint2*>(
                      v.gx + (uint64_t)p * v.gx_stride + 4)[g - s_gstart[p]];
            // entries come from the caller's buffers: a source outside the
            // store or a step outside this interval is skipped and flagged
            // (its cells would lie outside the tile's window)
            const bool ok = x.x < v.n_src &&
                            (uint32_t)((int32_t)x.y - (int32_t)t_now) < iv_span;
            if (!ok) atomicOr(&v.ctl->error_flags, (unsigned)SNN_ERRF_BAD_SOURCE);
            e[u].src = ok ? x.x : 0xFFFFFFFFu;
            e[u].t = (int32_t)x.y;
            e[u].choff = 0;
            e[u].pad = 0;
          } else {
            e[u] = have ? pre[u] : list[j0 + k];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kDU; ++u) {
        const uint32_t k = k0 + u * blockDim.x;
        if (k < nb) {
          SegDesc sd{0, 0u, e[u].t};
          if (e[u].src < v.n_src) {
            const uint32_t* to = v.tile_off + (uint64_t)e[u].src * row_stride + tile;
            const uint32_t a = to[0], b = to[1];
            sd.beg = v.row_ptr[e[u].src] + a;
            sd.len = b - a;
            if (kChecked && (b < a || sd.beg + sd.len > v.row_ptr[e[u].src + 1])) {
              atomicOr(&v.ctl->error_flags, (unsigned)SNN_ERRF_CHECK);
              sd.len = 0;
            }
            if (gathered) my_events += sd.len;
          }
          s_desc[k] = sd;
          if (PL) {
            const bool exc = e[u].src < v.sp.n_exc;
            s_tprev[k] = exc ? v.sp.prev_t[e[u].src] : kNoSpike;
            s_kprev[k] = exc ? v.sp.prev_k[e[u].src] : -1.f;
          }
        }
      }
    }
    // gathered lists: the warp's events (all threads of the CTA reach this)
    if (gathered) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) my_events += __shfl_xor_sync(kFull, my_events, o);
    }
    return my_events;
  };
  // next U runs for this warp (shared counter: warps that met short runs or
  // fast loads take more)
  auto grab = [&]() {
    uint32_t k = 0u;
    if (lane == 0) k = atomicAdd(&s_next, (uint32_t)U);
    return __shfl_sync(kFull, k, 0);
  };

  uint32_t j0 = 0;
  do {
    const uint32_t nb = min(desc_cap, n_sp - j0);
    const unsigned long long warp_events = describe(j0, nb);
    if (threadIdx.x == 0) s_next = 0u;
    __syncthreads();
    // (after the barrier: s_events was cleared before it)
    if (gathered && lane == 0 && warp_events) atomicAdd(&s_events, warp_events);
    fx = s_fx;
    if (FAST && !fx.fixed && n_sp > 0 && j0 == 0 && threadIdx.x == 0)
      atomicOr(&v.ctl->error_flags, (unsigned)SNN_ERRF_SCALES);
    // (B) each warp takes U runs at a time: all loads first, then the adds
    // (plastic nets: a fixed share per warp, the registers being spent on
    // the weight update)
    if constexpr (PL) {
      for (uint32_t k = warp * U; k < nb; k += kTileWarps * U) {
        Rec1<FMT> r[UR][PER];
        float wv[UR][PER];
        load_pass(r, wv, k, nb);
        add_pass(r, wv, k, nb);
      }
    } else {
      uint32_t k = grab();
      while (k < nb) {
        Rec1<FMT> r[UR][PER];
        float wv[UR][PER];
        load_pass(r, wv, k, nb);
        const uint32_t k_next = grab();
        add_pass(r, wv, k, nb);
        k = k_next;
      }
    }
    j0 += nb;
    __syncthreads();  // s_desc is rewritten by the next batch
  } while (j0 < n_sp);
  if (inwin) {
    // Every cell of the window belongs to this CTA alone, so its sum goes
    // into the ring buffer as a fire-and-forget global reduction: the one
    // addition rb + sum that a read-modify-write would make, without a
    // memory round trip.  The exact sum (H 2^s + L) 2^-q becomes
    // H 2^(s-q) + L 2^-q in FP32: both products are exact while |H| and |L|
    // are below 2^24 (then only the addition rounds, so the result is the
    // correctly rounded sum; larger words round once more), no 64-bit
    // conversion or FP64 arithmetic, whose rate is low on this part.
    // (the slots of a column are independent: unrolled, so that their
    // shared-memory reads and conversions overlap)
    const uint32_t x_end = tgt_lo < v.n ? min(TW, v.n - tgt_lo) : 0u;
    for (uint32_t x = threadIdx.x; x < x_end; x += blockDim.x) {
      float* const col = v.rb + tgt_lo + x;
#pragma unroll 4
      for (uint32_t sl = 0; sl < W; ++sl) {
        const uint32_t c = sl * TW + x;
        float a;
        if (fx.fixed) {
          a = __fmul_rn(__int2float_rn(accH[c]), fx.scale_sq);
          if (two) a = __fadd_rn(a, __fmul_rn(__int2float_rn(accL[c]), fx.inv_q));
        } else {
          a = accF[c];
        }
        if (a != 0.f)
          red_add_f32(col + (size_t)((uint32_t)(base + sl) & v.slot_mask) * v.pitch, a);
      }
    }
  }
  if (PL) {
    // one pair of atomics per warp, one per CTA
    unsigned long long a = my_pl, b = my_trunc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(kFull, a, o);
      b += __shfl_xor_sync(kFull, b, o);
    }
    if (lane == 0 && (a | b)) {
      atomicAdd(&s_pl[0], a);
      atomicAdd(&s_pl[1], b);
    }
    __syncthreads();
    if (threadIdx.x == 0 && (s_pl[0] | s_pl[1])) {
      atomicAdd(&v.ctl->plastic_events, s_pl[0]);
      atomicAdd(&v.ctl->stdp_truncated, s_pl[1]);
    }
  }
  // The last CTA to finish clears the list counters and advances the clock
  // (a gathered list's events -- its spikes' runs onto this partition's
  // targets -- are counted by the CTAs themselves).
  __syncthreads();
  if (threadIdx.x == 0) {
    if (gathered && s_events) atomicAdd(&v.ctl->gx_events, s_events);
    __threadfence();
    unsigned prev = atomicAdd(done_p, 1u);
    if (prev == v.n_tiles - 1) {
      *pair_p = 0ull;
      *done_p = 0u;
      if (advance_time) {  // the interval's own list: commit its events
        // this net's exchange list has been read (by the collective before
        // this delivery, or by this delivery itself): the next update
        // refills it
        if (v.xbuf) *v.xbuf = 0u;
        v.ctl->t_now += v.ctl->iv_steps;
        const unsigned long long own = atomicExch(&v.ctl->pending_events, 0ull);
        v.ctl->events += gathered ? atomicExch(&v.ctl->gx_events, 0ull) : own;
      }
    }
  }
}

template <int FMT, bool COUNT, bool PL, bool FAST, bool ONE, bool SHORT,
          bool GX>
__global__ void __launch_bounds__(kTileThreads, 1)
k_deliver_tiled(NetView v, unsigned long long* pair_p, unsigned int* done_p,
                const SpikeEntry* __restrict__ list, int from_list_range,
                int advance_time, uint32_t desc_off, uint32_t desc_cap) {
  extern __shared__ __align__(16) int acc_mem[];
  if constexpr (PL) {
    // one tile of plastic targets, or up to tile_grp static tiles one
    // after another in the same shared memory
    uint32_t t0 = blockIdx.x, t1 = blockIdx.x + 1u;
    if (blockIdx.x >= v.pl_tiles) {
      t0 = v.pl_tiles + (blockIdx.x - v.pl_tiles) * v.tile_grp;
      t1 = min(t0 + v.tile_grp, v.n_tiles);
    }
    for (uint32_t t = t0; t < t1; ++t) {
      if (t > t0) __syncthreads();  // the previous tile's last reads
      deliver_tile_body<FMT, COUNT, PL, FAST, ONE, SHORT, GX>(
          v, pair_p, done_p, list, from_list_range, advance_time, t, acc_mem,
          desc_off, desc_cap);
    }
  } else {
    deliver_tile_body<FMT, COUNT, PL, FAST, ONE, SHORT, GX>(
        v, pair_p, done_p, list, from_list_range, advance_time, blockIdx.x,
        acc_mem, desc_off, desc_cap);
  }
  // the next update may be scheduled once every CTA got here
  asm volatile("griddepcontrol.launch_dependents;");
}

// All nets of a batch in one launch: CTA b delivers tile bmap[b].y of net
// bmap[b].x (its pending interval list, advancing that net's clock).
template <int FMT>
__global__ void __launch_bounds__(kTileThreads, 1)
k_deliver_tiled_batch(const BatchNet* __restrict__ nets,
                      const uint2* __restrict__ bmap, uint32_t desc_off,
                      uint32_t desc_cap) {
  extern __shared__ __align__(16) int acc_mem[];
  const uint2 m = bmap[blockIdx.x];
  const NetView v = nets[m.x].v;
  deliver_tile_body<FMT, false, false>(v, &v.ctl->pair, &v.ctl->done, v.list,
                                       0, 1, m.y, acc_mem, desc_off, desc_cap);
}

// ---------------------------------------------------------------------------
// Persistent serving kernel: one launch advances every admitted net by its
// own number of intervals.  Each net is a chain of items -- per interval its
// update blocks, then its delivery tiles -- with the dependencies of the
// time-driven cycle (Section 2.1): an interval's delivery reads the spike
// list its update wrote, and the next update reads the ring buffer that
// delivery filled.  A CTA claims the first ready item of the first net
// (nets are ordered by size, smallest first) and runs it; so small nets
// keep advancing while large ones take the remaining CTAs, and no net waits
// for the pace of another.  Deadlock-free: an item is claimed only when its
// dependencies have completed, and no item waits inside.  The only wait is
// a CTA polling for a ready item; it gives up after spin_limit polls
// (ServeCtl.error = SNN_ERRF_TIMEOUT), and every CTA then leaves.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned x;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(x) : "l"(p) : "memory");
  return x;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// The two kinds of item, compiled out of line (each keeps its own register
// allocation instead of sharing one with the other and the claim loop).
__device__ __noinline__ void serve_update(const NetView& v, const UpdConst& c,
                                          int n_steps, uint32_t block) {
  update_body<false>(v, c, n_steps, 1, 0, block);
}
template <int FMT>
__device__ __noinline__ void serve_deliver(const NetView& v, uint32_t tile,
                                           int* acc_mem, uint32_t desc_off,
                                           uint32_t desc_cap) {
  deliver_tile_body<FMT, false, false>(v, &v.ctl->pair, &v.ctl->done, v.list, 0,
                                       1, tile, acc_mem, desc_off, desc_cap);
}

template <int FMT>
__global__ void __launch_bounds__(kTileThreads, 1)
k_serve(const BatchNet* __restrict__ nets, ServeNet* sn, ServeCtl* ctl,
        uint32_t n_nets, uint32_t desc_off, uint32_t desc_cap,
        unsigned long long spin_limit) {
  extern __shared__ __align__(16) int acc_mem[];
  __shared__ UpdConst s_c;
  __shared__ int s_state;      // 0: run s_net/s_item, 1: all claimed, 2: error
  __shared__ uint32_t s_net, s_item;
  for (;;) {
    if (threadIdx.x == 0) {
      int st = 1;
      unsigned long long polls = 0;
      unsigned nap = 32;  // ns between polls, doubling up to 256 while idle
      for (;;) {
        if (*reinterpret_cast<volatile unsigned*>(&ctl->error)) {
          st = 2;
          break;
        }
        bool left = false, got = false;
        for (uint32_t j = 0; j < n_nets && !got; ++j) {
          volatile ServeNet& q = sn[j];
          const unsigned per = q.ub + q.nt, n_items = q.n_items;
          for (;;) {
            const unsigned k = q.next;
            if (k >= n_items) break;
            left = true;
            const unsigned r = k / per, w = k - r * per;
            const bool ready = w < q.ub ? q.del_done >= r * q.nt
                                        : q.upd_done >= (r + 1) * q.ub;
            if (!ready) break;
            if (atomicCAS(&sn[j].next, k, k + 1) == k) {
              if (k == 0) sn[j].t_first = global_ns();
              s_net = j;
              s_item = k;
              got = true;
              break;
            }
          }
        }
        if (got) {
          st = 0;
          break;
        }
        if (!left) break;  // every item of every net is claimed
        if (++polls > spin_limit) {
          atomicOr(&ctl->error, (unsigned)SNN_ERRF_TIMEOUT);
          st = 2;
          break;
        }
        __nanosleep(nap);
        nap = nap < 256 ? 2 * nap : 256;
      }
      s_state = st;
    }
    __syncthreads();
    if (s_state != 0) break;
    const uint32_t j = s_net, k = s_item;
    ServeNet& q = sn[j];
    const unsigned per = q.ub + q.nt, r = k / per, w = k - r * per;
    const bool upd = w < q.ub;
    // every thread acquires what the item depends on (its writers released
    // it with a fence before counting their item done)
    ld_acquire_u32(upd ? &q.del_done : &q.upd_done);
    const NetView& v = nets[j].v;
    if (upd) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(&nets[j].c);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&s_c);
      for (uint32_t x = threadIdx.x; x < sizeof(UpdConst) / 4; x += blockDim.x)
        dst[x] = src[x];
      __syncthreads();
      serve_update(v, s_c, nets[j].n_steps, w);
    } else {
      serve_deliver<FMT>(v, w - q.ub, acc_mem, desc_off, desc_cap);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      atomicAdd(upd ? &q.upd_done : &q.del_done, 1u);
      atomicMax(&q.t_last, global_ns());
    }
  }
}

// ---------------------------------------------------------------------------
// Caller's spike list -> entries with chunk prefix sums (one CTA).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
k_prepare_external(NetView v, const uint32_t* __restrict__ src,
                   const int32_t* __restrict__ tt, uint32_t n,
                   SpikeEntry* out, unsigned long long* pair_p) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_carry;
  __shared__ int s_tmin, s_tmax;
  const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    s_carry = 0;
    s_tmin = 0x7FFFFFFF;
    s_tmax = -0x7FFFFFFF - 1;
  }
  unsigned long long deg_sum = 0;
  int tmin = 0x7FFFFFFF, tmax = -0x7FFFFFFF - 1;
  bool bad = false;
  __syncthreads();
  for (uint32_t base = 0; base < n; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    uint32_t s = 0xFFFFFFFFu, nch = 0;
    int32_t t = 0;
    if (i < n) {
      s = src[i];
      t = tt[i];
      tmin = min(tmin, t);
      tmax = max(tmax, t);
      if (s < v.n_src) {
        uint64_t b = v.row_ptr[s], e = v.row_ptr[s + 1];
        nch = row_chunks(b, e, v.chunk);
        deg_sum += e - b;
      } else {
        s = 0xFFFFFFFFu;
        bad = true;
      }
    }
    uint32_t incl = nch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(kFull, incl, o);
      if (lane >= (unsigned)o) incl += y;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      uint32_t x = lane < (blockDim.x >> 5) ? s_warp[lane] : 0u;
      uint32_t xi = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, xi, o);
        if (lane >= (unsigned)o) xi += y;
      }
      s_warp[lane] = xi - x;  // exclusive over warps
    }
    __syncthreads();
    const uint32_t carry = s_carry;
    if (i < n) {
      SpikeEntry en;
      en.src = s;
      en.t = t;
      en.choff = carry + s_warp[wid] + incl - nch;
      en.pad = 0;
      out[i] = en;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_carry = carry + s_warp[wid] + incl;
    __syncthreads();
  }
  // block reduction of deg_sum
  for (int o = 16; o > 0; o >>= 1) deg_sum += __shfl_xor_sync(kFull, deg_sum, o);
  if (lane == 0 && deg_sum) atomicAdd(&v.ctl->events, deg_sum);
  atomicMin(&s_tmin, tmin);
  atomicMax(&s_tmax, tmax);
  if (__syncthreads_or(bad) && threadIdx.x == 0)
    atomicOr(&v.ctl->error_flags, (unsigned)SNN_ERRF_BAD_SOURCE);
  if (threadIdx.x == 0) {
    *pair_p = ((unsigned long long)n << 32) | (unsigned long long)s_carry;
    v.ctl->ext_tmin = s_tmin;
    v.ctl->ext_tmax = s_tmax;
  }
}

// grid of the atomic delivery (SMs x resident blocks), computed on first use
std::atomic<int> g_deliver_blocks[2];

template <int FMT>
int deliver_blocks_for() {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_deliver<FMT, false>,
                                                kDelThreads, 0);
  if (per < 1) per = 1;
  return sms * per;
}

}  // namespace

// q - s of the kernel's fix_scale for event bound e and max|w| (-1: FP32),
// computed on the host with the same steps.
int fixed_qs_host(uint64_t e, double max_abs_w) {
  const float mw = (float)max_abs_w;
  if (e == 0 || e >= (1ull << 30) || !(mw > 0.f) || !(mw <= 3.0e38f)) return -1;
  const double A = 2147483647.0 - (double)e;
  const double B = (double)e * (double)mw;
  int qs = ilogb(A) - ilogb(B);
  if (B * ldexp(1.0, qs) > A) --qs;
  uint32_t wb;
  memcpy(&wb, &mw, 4);
  const int wexp = (int)((wb >> 23) & 0xFFu) - 127 + ((wb & 0x7FFFFFu) ? 1 : 0);
  qs = std::min(qs, 21 - wexp);
  if (qs < 0) return -1;
  return std::min(qs, 100);
}

int deliver_grid_size(int fmt) {
  const int k = fmt == SNN_W_FP32_12B ? 0 : 1;
  int b = g_deliver_blocks[k].load(std::memory_order_relaxed);
  if (b == 0) {
    b = fmt == SNN_W_FP32_12B ? deliver_blocks_for<SNN_W_FP32_12B>()
                              : deliver_blocks_for<SNN_W_BF16_8B>();
    g_deliver_blocks[k].store(b, std::memory_order_relaxed);
  }
  return b;
}

cudaError_t launch_init_v(const NetView& v, const UpdConst* c, int random,
                          cudaStream_t s) {
  if (v.n == 0) return cudaSuccess;
  unsigned blocks = (v.n + 255) / 256;
  k_init_state<<<blocks, 256, 0, s>>>(v, c->v_reset, c->v_th - c->v_reset,
                                      c->seed, random);
  return cudaGetLastError();
}

cudaError_t launch_update(const NetView& v, const UpdConst& c, int n_steps,
                          int from_ctl_time, long long t0, cudaStream_t s) {
  unsigned blocks = (v.n + kUpdThreads - 1) / kUpdThreads;
  if (blocks == 0) blocks = 1;
  static std::atomic<int> sms{0};
  if (sms.load(std::memory_order_relaxed) == 0) {
    int dev = 0, m = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      sms.store(m, std::memory_order_relaxed);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kUpdThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (blocks > 3u * (unsigned)std::max(sms.load(std::memory_order_relaxed), 1))
    return cudaLaunchKernelEx(&cfg, k_update<4>, v, c, n_steps, from_ctl_time, t0);
  return cudaLaunchKernelEx(&cfg, k_update<3>, v, c, n_steps, from_ctl_time, t0);
}

cudaError_t launch_deliver(const NetView& v, unsigned long long* pair,
                           unsigned int* done, const SpikeEntry* list,
                           int advance_time, cudaStream_t s) {
  int blocks = deliver_grid_size(v.fmt);
  if (v.fmt == SNN_W_FP32_12B) {
    if (v.counts)
      k_deliver<SNN_W_FP32_12B, true>
          <<<blocks, kDelThreads, 0, s>>>(v, pair, done, list, advance_time);
    else
      k_deliver<SNN_W_FP32_12B, false>
          <<<blocks, kDelThreads, 0, s>>>(v, pair, done, list, advance_time);
  } else {
    if (v.counts)
      k_deliver<SNN_W_BF16_8B, true>
          <<<blocks, kDelThreads, 0, s>>>(v, pair, done, list, advance_time);
    else
      k_deliver<SNN_W_BF16_8B, false>
          <<<blocks, kDelThreads, 0, s>>>(v, pair, done, list, advance_time);
  }
  return cudaGetLastError();
}

size_t tiled_smem_bytes(const NetView& v) {
  // accumulator; plastic nets: spike-time rings, counts, post-trace table
  return (size_t)v.tile_w *
         ((size_t)v.acc_words * v.window * sizeof(int) +
          (v.plastic ? (size_t)v.sp.hist * 4 + 4 + (size_t)v.window * 4 : 0));
}

// Raise a tiled-delivery kernel's dynamic shared-memory limit to all that
// its static shared memory leaves, once per device (the attribute belongs to
// the kernel on the current device); returns that limit.  `lim` holds one
// entry per device and is safe to fill from several threads.
template <class Kernel>
cudaError_t allow_tile_smem(Kernel kernel, std::atomic<uint32_t>* lim,
                            size_t* dyn_max) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::atomic<uint32_t>& slot = lim[dev & 63];
  const uint32_t have = slot.load(std::memory_order_acquire);
  if (have) {
    *dyn_max = have;
    return cudaSuccess;
  }
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  const int dyn = optin - (int)fa.sharedSizeBytes;
  if (dyn <= 0) return cudaErrorInvalidConfiguration;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
  if (e != cudaSuccess) return e;
  slot.store((uint32_t)dyn, std::memory_order_release);
  *dyn_max = (size_t)dyn;
  return cudaSuccess;
}

// Run descriptors go after the accumulator (and the plastic state): as
// many as the remaining shared memory holds, within kDescBytes (a larger
// shared-memory carve-out would take L1 capacity from the record loads).
constexpr size_t kDescBytes = 32 * 1024;
struct DescLayout {
  uint32_t off, cap;
  size_t smem;
};
cudaError_t desc_layout(size_t used, size_t dyn_max, bool plastic,
                        DescLayout* out) {
  const size_t per = sizeof(SegDesc) + (plastic ? 8u : 0u);
  const size_t off = (used + 15u) & ~(size_t)15u;
  if (dyn_max < off + 32u * per) return cudaErrorInvalidConfiguration;
  const size_t cap = std::min(kDescBytes, dyn_max - off) / per;
  out->off = (uint32_t)off;
  out->cap = (uint32_t)cap;
  out->smem = off + cap * per;
  return cudaSuccess;
}

template <int FMT, bool COUNT, bool PL, bool FAST = false, bool ONE = false,
          bool SHORT = false, bool GX = false>
cudaError_t launch_tiled_t(const NetView& v, unsigned long long* pair,
                           unsigned int* done, const SpikeEntry* list,
                           int from_list_range, int advance_time,
                           cudaStream_t s) {
  static std::atomic<uint32_t> lim[64];
  size_t dm = 0;
  cudaError_t e = allow_tile_smem(
      k_deliver_tiled<FMT, COUNT, PL, FAST, ONE, SHORT, GX>, lim, &dm);
  if (e != cudaSuccess) return e;
  DescLayout dl;
  e = desc_layout(tiled_smem_bytes(v), dm, PL, &dl);
  if (e != cudaSuccess) return e;
  // plastic nets: a CTA per plastic tile, then one per tile_grp static ones
  const uint32_t ctas =
      PL ? v.pl_tiles + (v.n_tiles - v.pl_tiles + v.tile_grp - 1u) / v.tile_grp
         : v.n_tiles;
  k_deliver_tiled<FMT, COUNT, PL, FAST, ONE, SHORT, GX>
      <<<ctas, kTileThreads, dl.smem, s>>>(
      v, pair, done, list, from_list_range, advance_time, dl.off, dl.cap);
  return cudaGetLastError();
}

template <bool GX>
cudaError_t launch_deliver_tiled_gx(const NetView& v, unsigned long long* pair,
                                    unsigned int* done, const SpikeEntry* list,
                                    int from_list_range, int advance_time,
                                    cudaStream_t s) {
#define SNN_TILED(F, C, P)                                                   \
  launch_tiled_t<F, C, P, false, false, false, GX>(v, pair, done, list,     \
                                                   from_list_range,         \
                                                   advance_time, s)
  // an interval's own list: the scales exist for every spike count when
  // they exist for the largest (E = max in-degree x spikes per neuron)
  bool interval_exact = false;
  if (!from_list_range && !v.counts) {
    const int qs = fixed_qs_host(
        (uint64_t)v.k_in_max * (v.spikes_per_iv ? v.spikes_per_iv : 1u), v.max_abs_w);
    interval_exact = qs >= 0 && (v.acc_words == 2 || qs >= v.acc_qs_min);
  }
  if constexpr (GX) {  // gathered lists: static nets only
    if (v.plastic) return cudaErrorNotSupported;
  } else if (v.plastic) {
    if (interval_exact)
      return v.fmt == SNN_W_FP32_12B
                 ? launch_tiled_t<SNN_W_FP32_12B, false, true, true>(
                       v, pair, done, list, 0, advance_time, s)
                 : launch_tiled_t<SNN_W_BF16_8B, false, true, true>(
                       v, pair, done, list, 0, advance_time, s);
    if (v.fmt == SNN_W_FP32_12B)
      return v.counts ? SNN_TILED(SNN_W_FP32_12B, true, true)
                      : SNN_TILED(SNN_W_FP32_12B, false, true);
    return v.counts ? SNN_TILED(SNN_W_BF16_8B, true, true)
                    : SNN_TILED(SNN_W_BF16_8B, false, true);
  }
  {
    if (interval_exact) {
      if (v.fmt == SNN_W_FP32_12B) {
        // (the records' precomputed cells exist for tiles below 2^16
        // targets; wider tiles take the general form below)
        if (v.tile_w < (1u << 16))
          return launch_tiled_t<SNN_W_FP32_12B, false, false, true, false,
                                false, GX>(v, pair, done, list, 0, advance_time, s);
      } else if (v.acc_words == 1) {
        // runs of a few dozen records: half a warp per run, eight per pass
        return v.mean_run < 48.f
                   ? launch_tiled_t<SNN_W_BF16_8B, false, false, true, true,
                                    true, GX>(v, pair, done, list, 0,
                                              advance_time, s)
                   : launch_tiled_t<SNN_W_BF16_8B, false, false, true, true,
                                    false, GX>(v, pair, done, list, 0,
                                               advance_time, s);
      } else {
        return launch_tiled_t<SNN_W_BF16_8B, false, false, true, false, false,
                              GX>(v, pair, done, list, 0, advance_time, s);
      }
    }
  }
  if (v.fmt == SNN_W_FP32_12B)
    return v.counts ? SNN_TILED(SNN_W_FP32_12B, true, false)
                    : SNN_TILED(SNN_W_FP32_12B, false, false);
  return v.counts ? SNN_TILED(SNN_W_BF16_8B, true, false)
                  : SNN_TILED(SNN_W_BF16_8B, false, false);
#undef SNN_TILED
}

cudaError_t launch_deliver_tiled(const NetView& v, unsigned long long* pair,
                                 unsigned int* done, const SpikeEntry* list,
                                 int from_list_range, int advance_time,
                                 cudaStream_t s) {
  if (v.gx) {
    if (from_list_range) return cudaErrorInvalidValue;
    return launch_deliver_tiled_gx<true>(v, pair, done, list, 0, advance_time, s);
  }
  return launch_deliver_tiled_gx<false>(v, pair, done, list, from_list_range,
                                        advance_time, s);
}

cudaError_t launch_fill_i32(int32_t* p, int32_t value, uint64_t n,
                            cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const uint64_t blocks = std::min<uint64_t>((n + 255) / 256, 4096);
  k_fill_i32<<<(unsigned)blocks, 256, 0, s>>>(p, value, n);
  return cudaGetLastError();
}

cudaError_t launch_list_to_arrays(const SpikeEntry* list, uint64_t n,
                                  uint32_t* src, int32_t* t, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const uint64_t blocks = std::min<uint64_t>((n + 255) / 256, 4096);
  k_list_to_arrays<<<(unsigned)blocks, 256, 0, s>>>(list, n, src, t);
  return cudaGetLastError();
}

cudaError_t launch_update_batch(const BatchNet* nets, const uint2* bmap,
                                uint32_t n_blocks, cudaStream_t s) {
  if (n_blocks == 0) return cudaSuccess;
  k_update_batch<<<n_blocks, kUpdThreads, 0, s>>>(nets, bmap);
  return cudaGetLastError();
}

cudaError_t launch_deliver_tiled_batch(int fmt, const BatchNet* nets,
                                       const uint2* bmap, uint32_t n_ctas,
                                       size_t smem, cudaStream_t s) {
  if (n_ctas == 0) return cudaSuccess;
  static std::atomic<uint32_t> lim[2][64];
  const int k = fmt == SNN_W_FP32_12B ? 0 : 1;
  size_t dm = 0;
  cudaError_t e = k == 0
      ? allow_tile_smem(k_deliver_tiled_batch<SNN_W_FP32_12B>, lim[0], &dm)
      : allow_tile_smem(k_deliver_tiled_batch<SNN_W_BF16_8B>, lim[1], &dm);
  if (e != cudaSuccess) return e;
  DescLayout dl;  // after the largest accumulator of the batch
  e = desc_layout(smem, dm, false, &dl);
  if (e != cudaSuccess) return e;
  if (k == 0)
    k_deliver_tiled_batch<SNN_W_FP32_12B><<<n_ctas, kTileThreads, dl.smem, s>>>(
        nets, bmap, dl.off, dl.cap);
  else
    k_deliver_tiled_batch<SNN_W_BF16_8B><<<n_ctas, kTileThreads, dl.smem, s>>>(
        nets, bmap, dl.off, dl.cap);
  return cudaGetLastError();
}

uint32_t update_threads() { return kUpdThreads; }

uint32_t serve_threads() { return kTileThreads; }

cudaError_t launch_serve(int fmt, const BatchNet* nets, ServeNet* sn,
                         ServeCtl* ctl, uint32_t n_nets, uint32_t n_ctas,
                         size_t smem, unsigned long long spin_limit,
                         cudaStream_t s) {
  if (n_nets == 0 || n_ctas == 0) return cudaSuccess;
  static std::atomic<uint32_t> lim[2][64];
  const int k = fmt == SNN_W_FP32_12B ? 0 : 1;
  size_t dm = 0;
  cudaError_t e = k == 0 ? allow_tile_smem(k_serve<SNN_W_FP32_12B>, lim[0], &dm)
                         : allow_tile_smem(k_serve<SNN_W_BF16_8B>, lim[1], &dm);
  if (e != cudaSuccess) return e;
  DescLayout dl;  // after the largest accumulator of the nets
  e = desc_layout(smem, dm, false, &dl);
  if (e != cudaSuccess) return e;
  if (k == 0)
    k_serve<SNN_W_FP32_12B><<<n_ctas, kTileThreads, dl.smem, s>>>(
        nets, sn, ctl, n_nets, dl.off, dl.cap, spin_limit);
  else
    k_serve<SNN_W_BF16_8B><<<n_ctas, kTileThreads, dl.smem, s>>>(
        nets, sn, ctl, n_nets, dl.off, dl.cap, spin_limit);
  return cudaGetLastError();
}

cudaError_t launch_prepare_external(const NetView& v, const uint32_t* src,
                                    const int32_t* t, uint32_t n,
                                    SpikeEntry* list,
                                    unsigned long long* pair, cudaStream_t s) {
  k_prepare_external<<<1, 1024, 0, s>>>(v, src, t, n, list, pair);
  return cudaGetLastError();
}

}  // namespace snn

// ---------------------------------------------------------------------------
// Allocation-free delivery of a caller's spike list.
//
// snn_deliver stages a caller's list in a buffer the library grows with
// cudaMalloc.  Some callers cannot let a library allocate: processes whose
// device memory is fully reserved by another allocator (a framework's caching
// allocator holding all of HBM), and latency-critical loops where cudaMalloc's
// implicit device synchronisation is not acceptable.  For them the list is
// staged in this file-scope device array instead: a fixed 4 MiB (2^18
// entries) held by every GPU that loads the library until the process exits.
// All calls share it, so calls whose work overlaps on the GPU race; the
// counters that must start at zero are cleared by every call.
// ---------------------------------------------------------------------------
namespace snn {
namespace {
struct NoAllocScratch {
  SpikeEntry list[SNN_NOALLOC_MAX_SPIKES];
  unsigned long long pair;
  unsigned int done;
  unsigned int pad_;
};
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
NoAllocScratch* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (in host code the symbol is only a stand-in for that address).
cudaError_t noalloc_scratch(NoAllocScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<NoAllocScratch*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}
}  // namespace

cudaError_t launch_deliver_noalloc(const NetView& v, const uint32_t* src,
                                   const int32_t* t, uint32_t n,
                                   cudaStream_t s) {
  if (n > SNN_NOALLOC_MAX_SPIKES) return cudaErrorInvalidValue;
  NoAllocScratch* sc = nullptr;
  cudaError_t e = noalloc_scratch(&sc);
  if (e != cudaSuccess) return e;
  // the list counters must start at zero: clear them on every call
  e = cudaMemsetAsync(&sc->pair, 0, sizeof(unsigned long long) + 2 * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  e = launch_prepare_external(v, src, t, n, sc->list, &sc->pair, s);
  if (e != cudaSuccess) return e;
  return launch_deliver(v, &sc->pair, &sc->done, sc->list, 0, s);
}
}  // namespace snn
