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
//  k_prepare_external  prefix sum of chunk counts for a caller's list.
#include <cuda_runtime.h>
#include <stdint.h>

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
    U4 r = draw(seed, i, 0, 1u);
    double u = (double)r.x * 0x1p-32;
    V0 = (float)((double)v_reset + (double)v_span * u);
  }
  v.V[i] = V0;
  v.I[i] = 0.0f;
  v.J[i] = 0.0f;
  v.refr[i] = 0;
}

// ---------------------------------------------------------------------------
// Fused update.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kUpdThreads)
k_update(NetView v, UpdConst c, int n_steps, int from_ctl, long long t0_arg) {
  __shared__ uint32_t s_thr[kMaxPoisson];
  for (int k = threadIdx.x; k < c.n_thr; k += blockDim.x) s_thr[k] = c.thr[k];
  const long long t0 = from_ctl ? v.ctl->t_now : t0_arg;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    v.ctl->iv_steps = n_steps;
    if (!from_ctl) v.ctl->t_now = t0;
  }
  __syncthreads();

  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < v.n;
  const unsigned lane = threadIdx.x & 31u;
  float V = 0.f, I = 0.f, J = 0.f;
  int refr = 0;
  uint32_t nch = 0;
  unsigned long long deg = 0;
  if (live) {
    V = v.V[i];
    I = v.I[i];
    J = v.J[i];
    refr = v.refr[i];
    uint64_t beg = v.row_ptr[i], end = v.row_ptr[i + 1];
    nch = row_chunks(beg, end, v.chunk);
    deg = end - beg;
  }
  // warp-constant prefix data of the chunk reservation, recomputed on use
  U4 rnd{0, 0, 0, 0};
  long long rnd_block = -1;

  for (int s = 0; s < n_steps; ++s) {
    const long long t = t0 + s;
    bool spike = false;
    if (live) {
      // (1) membrane, unless refractory
      if (refr == 0) V = c.p31 * J + c.p32 * I + c.p33 * V;
      else refr -= 1;
      // (2) synaptic current and its derivative
      I = c.p21 * J + c.p22 * I;
      J = c.p11 * J;
      // (3) ring-buffer slot of this step (read and clear) and drive
      float* cell = v.rb + (size_t)((uint32_t)t & v.slot_mask) * v.pitch + i;
      float in = *cell;
      *cell = 0.0f;
      if (c.n_thr > 0) {
        long long blk = t >> 2;
        if (blk != rnd_block) {
          rnd = draw(c.seed, i, (uint64_t)blk, 2u);
          rnd_block = blk;
        }
        uint32_t w = (t & 3) == 0 ? rnd.x : (t & 3) == 1 ? rnd.y
                   : (t & 3) == 2 ? rnd.z : rnd.w;
        int k = 0;
        while (k < c.n_thr - 1 && w >= s_thr[k]) ++k;
        in += c.w_ext * (float)k;
      }
      J += c.psc * in;
      // (4) threshold
      if (V >= c.v_th) {
        V = c.v_reset;
        refr = c.refr_steps;
        spike = true;
      }
    }
    const unsigned m = __ballot_sync(kFull, spike);
    if (m) {
      // warp-inclusive scan of chunk counts of the spiking lanes
      uint32_t my = spike ? nch : 0u;
      uint32_t incl = my;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= (unsigned)o) incl += y;
      }
      const uint32_t tot = __shfl_sync(kFull, incl, 31);
      unsigned long long dsum = spike ? deg : 0ull;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(kFull, dsum, o);
      const int leader = __ffs(m) - 1;
      const unsigned cnt = __popc(m);
      unsigned long long old = 0, logb = 0;
      if ((int)lane == leader) {
        old = atomicAdd(&v.ctl->pair, ((unsigned long long)cnt << 32) | tot);
        atomicAdd(&v.ctl->events, dsum);
        atomicAdd(&v.ctl->spikes, (unsigned long long)cnt);
        if (v.log_cap) logb = atomicAdd(&v.ctl->log_count, (unsigned long long)cnt);
        if ((uint32_t)old + (unsigned long long)tot > 0xFFFFFFFFull)
          atomicOr(&v.ctl->error_flags, (unsigned)SNN_ERRF_CHUNKS);
      }
      old = __shfl_sync(kFull, old, leader);
      logb = __shfl_sync(kFull, logb, leader);
      if (spike) {
        const unsigned rank = __popc(m & ((1u << lane) - 1u));
        const unsigned long long idx = (old >> 32) + rank;
        if (idx < v.list_cap) {
          SpikeEntry e;
          e.src = i;
          e.t = (int32_t)t;
          e.choff = (uint32_t)old + incl - my;
          e.pad = 0;
          v.list[idx] = e;
        } else {
          atomicOr(&v.ctl->error_flags, (unsigned)SNN_ERRF_SPIKE_LIST);
        }
        if (v.log_cap) {
          const unsigned long long li = logb + rank;
          if (li < v.log_cap) {
            v.log_src[li] = i;
            v.log_t[li] = (int32_t)t;
          } else {
            atomicOr(&v.ctl->error_flags, (unsigned)SNN_ERRF_SPIKE_LOG);
          }
        }
      }
    }
  }
  if (live) {
    v.V[i] = V;
    v.I[i] = I;
    v.J[i] = J;
    v.refr[i] = refr;
  }
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
    while (c < c_end && j < n_sp) {
      const SpikeEntry e = list[j];
      ++j;
      if (e.src >= v.n) continue;
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
    unsigned prev = atomicAdd(done_p, 1u);
    if (prev == gridDim.x - 1) {
      *pair_p = 0ull;
      *done_p = 0u;
      if (advance_time) v.ctl->t_now += v.ctl->iv_steps;
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
  const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  unsigned long long deg_sum = 0;
  bool bad = false;
  __syncthreads();
  for (uint32_t base = 0; base < n; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    uint32_t s = 0xFFFFFFFFu, nch = 0;
    int32_t t = 0;
    if (i < n) {
      s = src[i];
      t = tt[i];
      if (s < v.n) {
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
  if (__syncthreads_or(bad) && threadIdx.x == 0)
    atomicOr(&v.ctl->error_flags, (unsigned)SNN_ERRF_BAD_SOURCE);
  if (threadIdx.x == 0)
    *pair_p = ((unsigned long long)n << 32) | (unsigned long long)s_carry;
}

int g_deliver_blocks[2] = {0, 0};

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

int deliver_grid_size(int fmt) {
  int k = fmt == SNN_W_FP32_12B ? 0 : 1;
  if (g_deliver_blocks[k] == 0)
    g_deliver_blocks[k] = fmt == SNN_W_FP32_12B
                              ? deliver_blocks_for<SNN_W_FP32_12B>()
                              : deliver_blocks_for<SNN_W_BF16_8B>();
  return g_deliver_blocks[k];
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
  k_update<<<blocks, kUpdThreads, 0, s>>>(v, c, n_steps, from_ctl_time, t0);
  return cudaGetLastError();
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
