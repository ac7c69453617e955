// snn_build.cu -- construction of the source-major connection store on the
// device (network construction is outside the paper's measurements, Section
// 2.2; the store layout follows its Section 3.1: source-specific target
// segments).
//
// Pipeline: (1) count out-degrees with one generator call per synapse,
// (2) the host turns them into row offsets, (3) scatter one 64-bit sort key
// per synapse into its row, (4) sort every row by key in shared memory
// (bitonic network; rows longer than the shared-memory capacity are sorted
// in a global scratch buffer), pack the records (regenerating the weight from
// the key's tie field) and write the row's target-tile index.
//
// Sort key, for target tiles of TW neurons (tile = target / TW, position in
// the tile lo = target - tile TW < 2^B with B = lo_bits):
//   tile (24 - B bits) | delay (8) | lo (B) | tie (32)
// so a row is ordered by (target tile, delay, target, tie), where tie is the
// draw index k (fixed in-degree rule) or the edge index.  Sorting by the full
// key makes the store independent of the scatter's atomic order.  Within a
// tile a row is sorted by (delay, target); the tile index tile_off[row][tau]
// is the offset (relative to the row) of the first record of tile tau, for
// tau = 0 .. n_tiles (the last entry is the row length).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "snn_internal.cuh"

namespace snn {
namespace {

struct TileGeom {
  uint32_t tw;  // targets per tile
  int lb;       // bits of the position within a tile
};

__device__ __forceinline__ uint64_t make_key(uint32_t d, uint32_t tgt,
                                             uint32_t tie, TileGeom g) {
  const uint32_t tile = tgt / g.tw, lo = tgt - tile * g.tw;
  return ((uint64_t)tile << (40 + g.lb)) | ((uint64_t)(d & 0xFFu) << (32 + g.lb)) |
         ((uint64_t)lo << 32) | tie;
}
__device__ __forceinline__ uint32_t key_target(uint64_t key, TileGeom g) {
  return (uint32_t)(key >> (40 + g.lb)) * g.tw +
         ((uint32_t)(key >> 32) & ((1u << g.lb) - 1u));
}
__device__ __forceinline__ uint32_t key_delay(uint64_t key, TileGeom g) {
  return (uint32_t)(key >> (32 + g.lb)) & 0xFFu;
}

__device__ __forceinline__ uint32_t fixed_source(const BuildFixed& b,
                                                 uint32_t k, uint32_t u) {
  return k < b.k_e ? scale_u32(u, b.n_e) : b.n_e + scale_u32(u, b.n_i);
}

// One block per local target (the draws use its global index); a grid
// smaller than the targets walks them in strides (a build confined to some
// SMs, see BuildShape).
__global__ void __launch_bounds__(1024) k_count_fixed(BuildFixed b, uint32_t* deg) {
  const uint32_t kk = b.k_e + b.k_i;
  for (uint32_t tgt = blockIdx.x; tgt < b.n_tgt; tgt += gridDim.x)
    for (uint32_t k = threadIdx.x; k < kk; k += blockDim.x) {
      U4 r = draw(b.seed, b.tgt0 + tgt, k, 0u);
      atomicAdd(&deg[fixed_source(b, k, r.x)], 1u);
    }
}

__global__ void __launch_bounds__(1024) k_scatter_fixed(BuildFixed b, const uint64_t* row_ptr,
                                uint32_t* cursor, uint64_t* keys, TileGeom g) {
  const uint32_t kk = b.k_e + b.k_i;
  const uint32_t span = (uint32_t)(b.d_hi - b.d_lo + 1);
  for (uint32_t tgt = blockIdx.x; tgt < b.n_tgt; tgt += gridDim.x)
    for (uint32_t k = threadIdx.x; k < kk; k += blockDim.x) {
      U4 r = draw(b.seed, b.tgt0 + tgt, k, 0u);
      uint32_t src = fixed_source(b, k, r.x);
      uint32_t d = (uint32_t)b.d_lo + scale_u32(r.y, span);
      uint32_t pos = atomicAdd(&cursor[src], 1u);
      keys[row_ptr[src] + pos] = make_key(d, tgt, k, g);
    }
}

__global__ void k_count_edges(const uint32_t* src, uint64_t n, uint32_t* deg) {
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < n;
       e += (uint64_t)gridDim.x * blockDim.x)
    atomicAdd(&deg[src[e]], 1u);
}

__global__ void k_scatter_edges(const uint32_t* src, const uint32_t* tgt,
                                const uint8_t* delay, uint64_t n,
                                const uint64_t* row_ptr, uint32_t* cursor,
                                uint64_t* keys, TileGeom g) {
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < n;
       e += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t s = src[e];
    uint32_t pos = atomicAdd(&cursor[s], 1u);
    keys[row_ptr[s] + pos] = make_key(delay[e], tgt[e], (uint32_t)e, g);
  }
}

// Weight of a synapse, FP64: per-edge value, or the fixed rule's mean plus
// a Box-Muller normal from words 2 and 3 of the synapse's draw.
template <int WMODE>
__device__ double weight_of(const BuildFixed& b, const double* edge_w,
                            bool exc, uint32_t tgt, uint32_t tie) {
  if (WMODE == 1) return edge_w[tie];
  double mean = exc ? b.w_e : b.w_i, sd = exc ? b.sd_e : b.sd_i;
  double x = mean;
  if (sd != 0.0) {
    U4 r = draw(b.seed, b.tgt0 + tgt, tie, 0u);
    double u1 = ((double)r.z + 1.0) * 0x1p-32;
    double u2 = (double)r.w * 0x1p-32;
    double z = sqrt(-2.0 * log(u1)) * cos(2.0 * 3.14159265358979323846 * u2);
    x = mean + sd * z;
  }
  if (exc && b.clip_e && x < 0.0) x = 0.0;
  if (!exc && b.clip_i && x > 0.0) x = 0.0;
  return x;
}

// BF16 bits of a fixed-rule weight.  The rounding to 8 significant bits is
// decided from an FP32 evaluation of the same Box-Muller normal whenever the
// FP32 value's error bound lies inside one rounding interval, and only
// otherwise (about 0.2 % of the draws) from the FP64 evaluation: rounding is
// monotonic, so if both ends of [x - e, x + e] round to the same BF16 value,
// the FP64 value does too.  The result equals the FP64 path's, at a small
// fraction of its cost (FP64 arithmetic is a small share of this GPU's
// throughput).  Bound: with the CUDA math library's documented maximum
// errors (1 ulp for logf, log1pf and cospif; sqrtf correctly rounded) and
// the conversions of the draw words to float, |s| <= 6.67 and
// |dz| <= 14 2^-21 < 2^-16; the conversions of mean and sd and the final
// fused multiply-add add at most 2^-23 (|mean| + 7 |sd|).
__device__ uint16_t bf16_weight_bits(const BuildFixed& b, bool exc,
                                     uint32_t tgt, uint32_t tie) {
  const double mean = exc ? b.w_e : b.w_i, sd = exc ? b.sd_e : b.sd_i;
  const bool clip_lo = exc && b.clip_e, clip_hi = !exc && b.clip_i;
  if (sd == 0.0) {
    double x = mean;
    if (clip_lo && x < 0.0) x = 0.0;
    if (clip_hi && x > 0.0) x = 0.0;
    return bf16_bits_rne(x);
  }
  const U4 r = draw(b.seed, b.tgt0 + tgt, tie, 0u);
  // ln u1 for u1 = (z + 1) 2^-32: directly below 1/2; above it as
  // log1p(u1 - 1) with u1 - 1 = -(2^32 - 1 - z) 2^-32 (no cancellation)
  const float ln = r.z < 0x7FFFFFFFu ? logf(((float)r.z + 1.0f) * 0x1p-32f)
                                     : log1pf(-(float)(~r.z) * 0x1p-32f);
  const float sv = sqrtf(-2.0f * ln);
  const float cv = cospif(2.0f * ((float)r.w * 0x1p-32f));
  const float sdf = (float)sd, meanf = (float)mean;
  const float xf = fmaf(sdf, sv * cv, meanf);
  const float e = fabsf(sdf) * 0x1p-16f +
                  (fabsf(meanf) + 7.0f * fabsf(sdf)) * 0x1p-20f;
  float lo = __fsub_rd(xf, e), hi = __fadd_ru(xf, e);
  if (clip_lo) {
    lo = fmaxf(lo, 0.0f);
    hi = fmaxf(hi, 0.0f);
  }
  if (clip_hi) {
    lo = fminf(lo, 0.0f);
    hi = fminf(hi, 0.0f);
  }
  const uint16_t a = bf16_bits_rne((double)lo);
  if (a == bf16_bits_rne((double)hi)) return a;
  return bf16_bits_rne(weight_of<0>(b, nullptr, exc, tgt, tie));
}

// Writes a record; returns |stored weight| (as stored, widened to float).
// FP32 records also carry, above the delay byte, the record's cell in its
// tile's ring-buffer window (d TW + position in the tile; below 2^24 for
// tiles narrower than 2^16 targets, else 0), so that interval-list
// deliveries need neither the target word nor the index arithmetic.
template <int FMT>
__device__ __forceinline__ float store_rec(void* recs, uint64_t idx,
                                           uint32_t tgt, uint32_t d, double w,
                                           uint32_t cell = 0u) {
  if (FMT == SNN_W_FP32_12B) {
    uint32_t* p = reinterpret_cast<uint32_t*>(recs) + idx * 3u;
    const float wf = __double2float_rn(w);
    p[0] = tgt;
    p[1] = __float_as_uint(wf);
    p[2] = (d & 0xFFu) | (cell < (1u << 24) ? cell << 8 : 0u);
    return fabsf(wf);
  } else {
    uint2 r;
    const uint16_t bits = bf16_bits_rne(w);
    r.x = tgt;
    r.y = (d & 0xFFu) | ((uint32_t)bits << 16);
    reinterpret_cast<uint2*>(recs)[idx] = r;
    return fabsf(bf16_to_f32(bits));
  }
}

template <int FMT, int WMODE>
__device__ void pack_row(const uint64_t* sorted, uint32_t len, uint32_t row,
                         uint64_t beg, void* recs, const BuildFixed& b,
                         const double* edge_w, TileGeom g, uint32_t n_tiles,
                         uint32_t* tile_off, uint32_t* stats) {
  const bool exc = row < b.n_e;
  float wmax = 0.f;
  uint32_t run_max = 0;
  for (uint32_t p = threadIdx.x; p < len; p += blockDim.x) {
    uint64_t key = sorted[p];
    uint32_t d = key_delay(key, g);
    uint32_t tgt = key_target(key, g);
    uint32_t tie = (uint32_t)key;
    if (FMT == SNN_W_BF16_8B && WMODE == 0) {
      const uint16_t bits = bf16_weight_bits(b, exc, tgt, tie);
      uint2 rec;
      rec.x = tgt;
      rec.y = (d & 0xFFu) | ((uint32_t)bits << 16);
      reinterpret_cast<uint2*>(recs)[beg + p] = rec;
      wmax = fmaxf(wmax, fabsf(bf16_to_f32(bits)));
    } else {
      const uint32_t in_tile = (uint32_t)(key >> 32) & ((1u << g.lb) - 1u);
      const uint32_t cell = g.tw < (1u << 16) ? d * g.tw + in_tile : (1u << 24);
      wmax = fmaxf(wmax, store_rec<FMT>(recs, beg + p, tgt, d,
                                        weight_of<WMODE>(b, edge_w, exc, tgt, tie),
                                        cell));
    }
    // multiplicity of (target, delay): length of the run of equal keys
    // (ignoring the tie field) that starts here
    if (p == 0 || (sorted[p - 1] >> 32) != (key >> 32)) {
      uint32_t r = 1;
      while (p + r < len && (sorted[p + r] >> 32) == (key >> 32)) ++r;
      run_max = max(run_max, r);
    }
  }
  // |w| >= 0 orders like its bit pattern as an unsigned integer
  const uint32_t wbits = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(wmax));
  run_max = __reduce_max_sync(0xFFFFFFFFu, run_max);
  if ((threadIdx.x & 31u) == 0) {
    if (run_max) atomicMax(&stats[0], run_max);
    if (wbits) atomicMax(&stats[1], wbits);
  }
  // tile index: first position whose tile is >= tau (lower bound)
  uint32_t* out = tile_off + (uint64_t)row * (n_tiles + 1);
  for (uint32_t tau = threadIdx.x; tau <= n_tiles; tau += blockDim.x) {
    if (tau == n_tiles) {  // every key's tile is below n_tiles
      out[tau] = len;
      continue;
    }
    const uint64_t probe = (uint64_t)tau << (40 + g.lb);
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
      uint32_t mid = (lo + hi) >> 1;
      if (sorted[mid] < probe) lo = mid + 1; else hi = mid;
    }
    out[tau] = lo;
  }
}

// In-place ascending bitonic sort of P (a power of two) keys.
__device__ void bitonic(uint64_t* a, uint32_t P) {
  for (uint32_t k = 2; k <= P; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
        uint32_t l = i ^ j;
        if (l > i) {
          uint64_t x = a[i], y = a[l];
          bool up = (i & k) == 0;
          if ((x > y) == up) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

__device__ __forceinline__ uint32_t pow2_ceil(uint32_t x) {
  uint32_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Segments (keys of one target tile) up to this long are rank-sorted by a
// warp in registers; a row with a longer one is sorted whole (bitonic).
constexpr uint32_t kWarpSegMax = 256;
// Rows of stores with more tiles than this are sorted whole.
constexpr uint32_t kBucketTilesMax = 4096;

// Sort one row of keys in shared memory (len keys at a[0..len), room for the
// next power of two; cnt: n_tiles + 1 words): bucket by target tile
// (histogram, exclusive scan, scatter from registers), then every warp
// rank-sorts the short segments of the tiles it takes.  Keys are distinct,
// so a key's rank in its segment is its position, and the result equals a
// full sort of the row.  Falls back to the bitonic network when a segment
// is longer than kWarpSegMax or the store has too many tiles.
__device__ void sort_row(uint64_t* a, uint32_t len, uint32_t* cnt,
                         uint32_t n_tiles, int lb) {
  const uint32_t P = pow2_ceil(len);
  bool whole = n_tiles > kBucketTilesMax || len > 16u * blockDim.x;
  if (!whole) {
    for (uint32_t t = threadIdx.x; t <= n_tiles; t += blockDim.x) cnt[t] = 0;
    __syncthreads();
    // keys of this thread (at most 16) into registers, tiles counted
    uint64_t r[16];
#pragma unroll
    for (uint32_t q = 0; q < 16; ++q) {
      const uint32_t i = threadIdx.x + q * blockDim.x;
      if (i < len) {
        r[q] = a[i];
        atomicAdd(&cnt[(uint32_t)(r[q] >> (40 + lb))], 1u);
      }
    }
    __syncthreads();
    // longest segment, then the exclusive scan of the counts (one thread
    // per block of counts: n_tiles is small)
    __shared__ uint32_t s_max;
    if (threadIdx.x == 0) {
      uint32_t run = 0, mx = 0;
      for (uint32_t t = 0; t <= n_tiles; ++t) {
        const uint32_t c = cnt[t];
        cnt[t] = run;
        run += c;
        mx = max(mx, c);
      }
      s_max = mx;
    }
    __syncthreads();
    whole = s_max > kWarpSegMax;
    // scatter into the buckets (cnt becomes each bucket's end)
#pragma unroll
    for (uint32_t q = 0; q < 16; ++q) {
      const uint32_t i = threadIdx.x + q * blockDim.x;
      if (i < len) {
        const uint32_t pos = atomicAdd(&cnt[(uint32_t)(r[q] >> (40 + lb))], 1u);
        a[pos] = r[q];
      }
    }
    __syncthreads();
    if (!whole) {
      const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
      const uint32_t n_warps = blockDim.x >> 5;
      for (uint32_t t = warp; t < n_tiles; t += n_warps) {
        const uint32_t end = cnt[t];
        const uint32_t beg = t == 0 ? 0u : cnt[t - 1];
        const uint32_t c = end - beg;
        if (c < 2) continue;
        uint64_t key[kWarpSegMax / 32];
        uint32_t rank[kWarpSegMax / 32];
#pragma unroll
        for (uint32_t q = 0; q < kWarpSegMax / 32; ++q) {
          rank[q] = 0;
          key[q] = lane + 32u * q < c ? a[beg + lane + 32u * q] : ~0ull;
        }
        for (uint32_t i = 0; i < c; ++i) {
          const uint64_t y = a[beg + i];  // the same word for every lane
#pragma unroll
          for (uint32_t q = 0; q < kWarpSegMax / 32; ++q) rank[q] += y < key[q];
        }
        __syncwarp();
#pragma unroll
        for (uint32_t q = 0; q < kWarpSegMax / 32; ++q)
          if (lane + 32u * q < c) a[beg + rank[q]] = key[q];
        __syncwarp();
      }
      __syncthreads();
      return;
    }
  }
  for (uint32_t i = len + threadIdx.x; i < P; i += blockDim.x) a[i] = ~0ull;
  __syncthreads();
  if (P > 1) bitonic(a, P);
}

template <int FMT, int WMODE>
__global__ void __launch_bounds__(1024) k_sort_pack(uint32_t n, const uint64_t* row_ptr,
                            uint64_t* keys, void* recs, BuildFixed b,
                            const double* edge_w, uint32_t cap, TileGeom g,
                            uint32_t n_tiles, uint32_t* tile_off,
                            uint32_t* stats) {
  extern __shared__ uint64_t sk[];
  uint32_t* cnt = reinterpret_cast<uint32_t*>(sk + cap);
  for (uint32_t row = blockIdx.x; row < n; row += gridDim.x) {
    const uint64_t beg = row_ptr[row];
    const uint32_t len = (uint32_t)(row_ptr[row + 1] - beg);
    if (len > cap) continue;                 // uniform per block
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) sk[i] = keys[beg + i];
    __syncthreads();
    if (len > 1) sort_row(sk, len, cnt, n_tiles, g.lb);
    pack_row<FMT, WMODE>(sk, len, row, beg, recs, b, edge_w, g, n_tiles,
                         tile_off, stats);
    __syncthreads();
  }
}

template <int FMT, int WMODE>
__global__ void __launch_bounds__(1024) k_sort_long(const uint32_t* rows, uint32_t n_long,
                            const uint64_t* row_ptr,
                            uint64_t* keys, void* recs, BuildFixed b,
                            const double* edge_w, uint64_t* scratch,
                            const uint64_t* scratch_off, TileGeom g,
                            uint32_t n_tiles, uint32_t* tile_off,
                            uint32_t* stats) {
  for (uint32_t j = blockIdx.x; j < n_long; j += gridDim.x) {
    const uint32_t row = rows[j];
    const uint64_t beg = row_ptr[row];
    const uint32_t len = (uint32_t)(row_ptr[row + 1] - beg);
    uint64_t* a = scratch + scratch_off[j];
    const uint32_t P = pow2_ceil(len);
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x)
      a[i] = i < len ? keys[beg + i] : ~0ull;
    __syncthreads();
    bitonic(a, P);
    pack_row<FMT, WMODE>(a, len, row, beg, recs, b, edge_w, g, n_tiles,
                         tile_off, stats);
    __syncthreads();
  }
}

template <int FMT>
__global__ void k_unpack(const void* recs, uint64_t n, uint32_t* tgt,
                         uint8_t* delay, float* w) {
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n;
       s += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t t, d;
    float x;
    if (FMT == SNN_W_FP32_12B) {
      const uint32_t* p = reinterpret_cast<const uint32_t*>(recs) + s * 3u;
      t = p[0];
      x = __uint_as_float(p[1]);
      d = p[2] & 0xFFu;
    } else {
      uint2 r = reinterpret_cast<const uint2*>(recs)[s];
      t = r.x;
      d = r.y & 0xFFu;
      x = bf16_to_f32(r.y >> 16);
    }
    if (tgt) tgt[s] = t;
    if (delay) delay[s] = (uint8_t)d;
    if (w) w[s] = x;
  }
}

template <int FMT>
__global__ void __launch_bounds__(1024) k_delay_range(const void* recs, uint64_t n, unsigned* out) {
  __shared__ unsigned s_lo, s_hi;
  if (threadIdx.x == 0) {
    s_lo = 0xFFFFFFFFu;
    s_hi = 0u;
  }
  __syncthreads();
  unsigned lo = 0xFFFFFFFFu, hi = 0u;
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n;
       s += (uint64_t)gridDim.x * blockDim.x) {
    unsigned d = FMT == SNN_W_FP32_12B
                     ? reinterpret_cast<const uint32_t*>(recs)[s * 3u + 2u] & 0xFFu
                     : reinterpret_cast<const uint2*>(recs)[s].y & 0xFFu;
    lo = min(lo, d);
    hi = max(hi, d);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xFFFFFFFFu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xFFFFFFFFu, hi, o));
  }
  // one pair of global atomics per block (not per warp: every warp would
  // hit the same two words)
  if ((threadIdx.x & 31u) == 0) {
    atomicMin(&s_lo, lo);
    atomicMax(&s_hi, hi);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicMin(&out[0], s_lo);
    atomicMax(&out[1], s_hi);
  }
}

unsigned grid_for(uint64_t n, unsigned threads) {
  uint64_t b = (n + threads - 1) / threads;
  if (b > 65536u * 8u) b = 65536u * 8u;
  return b ? (unsigned)b : 1u;
}

// Build mode of the calling thread, set around a build by the API
// (snn_params.build_yield).
thread_local unsigned t_build_yield = 0;

// Launch shape of a build kernel.  Normal: the kernel's own grid.
// Yielding: the same grid of short CTAs (one target or one row each), but of
// 1024 threads and with more than half of an SM's shared memory, so that no
// two share an SM.  Each SM then becomes entirely free whenever one of its
// build CTAs ends (every few to a few hundred microseconds), and the CTA
// scheduler hands it to pending work of higher-priority streams first: the
// kernels of running nets, whose delivery CTAs need a whole SM and would
// otherwise wait for the build to end, since small build CTAs keep refilling
// partly free SMs.
struct BuildShape {
  unsigned blocks, threads;
  size_t smem;
};

template <class Kernel>
cudaError_t build_shape(Kernel kernel, unsigned blocks, unsigned threads,
                        size_t smem, BuildShape* out) {
  *out = BuildShape{blocks, threads, smem};
  int dev = 0, per_sm = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  // the kernel's dynamic shared-memory limit is always raised to all that
  // its static shared memory leaves of the opt-in amount: one value for
  // every caller, so that builds on several host threads never lower it
  // under one another's launch
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, kernel)) != cudaSuccess) return e;
  const int dyn_max = optin - (int)fa.sharedSizeBytes;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           dyn_max);
  if (e != cudaSuccess) return e;
  if (!t_build_yield) return cudaSuccess;
  const size_t excl = std::min<size_t>((size_t)per_sm / 2 + 2048, (size_t)dyn_max);
  out->threads = threads > 1024 ? threads : 1024;
  out->smem = std::max(smem, excl);
  return cudaSuccess;
}

template <int FMT, int WMODE>
cudaError_t sort_pack_t(uint32_t n, const uint64_t* row_ptr, uint64_t* keys,
                        void* recs, const BuildFixed* b, const double* edge_w,
                        uint32_t max_row, const uint32_t* long_rows,
                        uint32_t n_long, uint64_t* long_scratch,
                        const uint64_t* long_off, TileGeom g, uint32_t n_tiles,
                        uint32_t* tile_off, uint32_t* stats, cudaStream_t s) {
  BuildFixed bb = b ? *b : BuildFixed{};
  uint32_t cap = max_row < kSortCap ? max_row : kSortCap;
  uint32_t P = 1;
  while (P < cap) P <<= 1;
  // keys (room for the next power of two) and the tile buckets
  size_t smem = (size_t)P * sizeof(uint64_t) +
                (size_t)(std::min(n_tiles, kBucketTilesMax) + 1) * sizeof(uint32_t);
  cudaError_t e;
  unsigned threads = P >= 1024 ? 1024 : (P >= 128 ? P : 128);
  unsigned blocks = n < (1u << 20) ? n : (1u << 20);
  BuildShape sh;
  if (blocks) {
    if ((e = build_shape(k_sort_pack<FMT, WMODE>, blocks, threads, smem, &sh)) !=
        cudaSuccess)
      return e;
    k_sort_pack<FMT, WMODE><<<sh.blocks, sh.threads, sh.smem, s>>>(
        n, row_ptr, keys, recs, bb, edge_w, P, g, n_tiles, tile_off, stats);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (n_long) {
    if ((e = build_shape(k_sort_long<FMT, WMODE>, n_long, 1024, 0, &sh)) !=
        cudaSuccess)
      return e;
    k_sort_long<FMT, WMODE><<<sh.blocks, sh.threads, sh.smem, s>>>(
        long_rows, n_long, row_ptr, keys, recs, bb, edge_w, long_scratch,
        long_off, g, n_tiles, tile_off, stats);
  }
  return cudaGetLastError();
}

}  // namespace

void set_build_yield(unsigned on) { t_build_yield = on; }

cudaError_t build_count_fixed(const BuildFixed& b, uint32_t* deg,
                              cudaStream_t s) {
  if (b.n_tgt == 0 || b.k_e + b.k_i == 0) return cudaSuccess;
  BuildShape sh;
  cudaError_t e = build_shape(k_count_fixed, b.n_tgt, 256, 0, &sh);
  if (e != cudaSuccess) return e;
  k_count_fixed<<<sh.blocks, sh.threads, sh.smem, s>>>(b, deg);
  return cudaGetLastError();
}

cudaError_t build_scatter_fixed(const BuildFixed& b, const uint64_t* row_ptr,
                                uint32_t* cursor, uint64_t* keys,
                                uint32_t tile_w, int lo_bits, cudaStream_t s) {
  if (b.n_tgt == 0 || b.k_e + b.k_i == 0) return cudaSuccess;
  BuildShape sh;
  cudaError_t e = build_shape(k_scatter_fixed, b.n_tgt, 256, 0, &sh);
  if (e != cudaSuccess) return e;
  k_scatter_fixed<<<sh.blocks, sh.threads, sh.smem, s>>>(
      b, row_ptr, cursor, keys, TileGeom{tile_w, lo_bits});
  return cudaGetLastError();
}

cudaError_t build_count_edges(const uint32_t* src, uint64_t n, uint32_t* deg,
                              cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_count_edges<<<grid_for(n, 256), 256, 0, s>>>(src, n, deg);
  return cudaGetLastError();
}

cudaError_t build_scatter_edges(const uint32_t* src, const uint32_t* tgt,
                                const uint8_t* delay, uint64_t n,
                                const uint64_t* row_ptr, uint32_t* cursor,
                                uint64_t* keys, uint32_t tile_w, int lo_bits,
                                cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_scatter_edges<<<grid_for(n, 256), 256, 0, s>>>(
      src, tgt, delay, n, row_ptr, cursor, keys, TileGeom{tile_w, lo_bits});
  return cudaGetLastError();
}

cudaError_t build_sort_pack(int fmt, uint32_t n, const uint64_t* row_ptr,
                            uint64_t* keys, void* recs, const BuildFixed* b,
                            const double* edge_w, uint32_t max_row,
                            const uint32_t* long_rows, uint32_t n_long,
                            uint64_t* long_scratch,
                            const uint64_t* long_scratch_off, uint32_t tile_w,
                            int lo_bits, uint32_t n_tiles, uint32_t* tile_off,
                            uint32_t* stats, cudaStream_t s) {
  const TileGeom g{tile_w, lo_bits};
#define SNN_SORT_ARGS                                                       \
  n, row_ptr, keys, recs, b, edge_w, max_row, long_rows, n_long,           \
      long_scratch, long_scratch_off, g, n_tiles, tile_off, stats, s
  if (fmt == SNN_W_FP32_12B)
    return edge_w ? sort_pack_t<SNN_W_FP32_12B, 1>(SNN_SORT_ARGS)
                  : sort_pack_t<SNN_W_FP32_12B, 0>(SNN_SORT_ARGS);
  return edge_w ? sort_pack_t<SNN_W_BF16_8B, 1>(SNN_SORT_ARGS)
                : sort_pack_t<SNN_W_BF16_8B, 0>(SNN_SORT_ARGS);
#undef SNN_SORT_ARGS
}

cudaError_t unpack_store(int fmt, const void* recs, uint64_t n_syn,
                         uint32_t* tgt, uint8_t* delay, float* w,
                         cudaStream_t s) {
  if (n_syn == 0) return cudaSuccess;
  if (fmt == SNN_W_FP32_12B)
    k_unpack<SNN_W_FP32_12B><<<grid_for(n_syn, 256), 256, 0, s>>>(recs, n_syn,
                                                                  tgt, delay, w);
  else
    k_unpack<SNN_W_BF16_8B><<<grid_for(n_syn, 256), 256, 0, s>>>(recs, n_syn,
                                                                 tgt, delay, w);
  return cudaGetLastError();
}

cudaError_t delay_range(int fmt, const void* recs, uint64_t n_syn,
                        unsigned int* dmin_dmax, cudaStream_t s) {
  if (n_syn == 0) return cudaSuccess;
  BuildShape sh;
  cudaError_t e;
  if (fmt == SNN_W_FP32_12B) {
    if ((e = build_shape(k_delay_range<SNN_W_FP32_12B>, std::min(grid_for(n_syn, 256), 4096u), 256,
                         0, &sh)) != cudaSuccess)
      return e;
    k_delay_range<SNN_W_FP32_12B><<<sh.blocks, sh.threads, sh.smem, s>>>(
        recs, n_syn, dmin_dmax);
  } else {
    if ((e = build_shape(k_delay_range<SNN_W_BF16_8B>, std::min(grid_for(n_syn, 256), 4096u), 256,
                         0, &sh)) != cudaSuccess)
      return e;
    k_delay_range<SNN_W_BF16_8B><<<sh.blocks, sh.threads, sh.smem, s>>>(
        recs, n_syn, dmin_dmax);
  }
  return cudaGetLastError();
}

}  // namespace snn
