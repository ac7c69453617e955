// snn_probe.cu -- throughput probe of the L2 reductions that the delivery's
// ring-buffer additions use (red.global.add.f32): the secondary bound of the
// atomic delivery (one reduction per synaptic event) and of the tiled
// delivery's flush (one per nonzero cell of a tile's window).
#include <cuda_runtime.h>
#include <cstdint>

namespace snn {
namespace {

// An integer hash (xor-shift-multiply finalizer): spreads consecutive
// operation numbers over the cells.
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// Operation k adds 1.0f to cell c(k) of buf[n_cells]: pattern 0, c = a hash
// of k scaled to [0, n_cells) (scattered, like the atomic delivery's
// targets); pattern 1, c = k mod n_cells (a warp covers 32 consecutive
// cells, like the flush of a tile's window).
__global__ void k_red_probe(float* __restrict__ buf, uint32_t n_cells,
                            uint64_t n_ops, int pattern) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_ops;
       k += stride) {
    const uint32_t c =
        pattern == 0
            ? (uint32_t)(((uint64_t)mix32((uint32_t)k ^ (uint32_t)(k >> 32)) * n_cells) >> 32)
            : (uint32_t)(k % n_cells);
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(buf + c), "f"(1.0f) : "memory");
  }
}

}  // namespace

cudaError_t launch_red_probe(float* buf, uint32_t n_cells, uint64_t n_ops,
                             int pattern, cudaStream_t s) {
  int dev = 0, sms = 1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  k_red_probe<<<8u * (unsigned)sms, 256, 0, s>>>(buf, n_cells, n_ops, pattern);
  return cudaGetLastError();
}

}  // namespace snn
