// One bit per cell: conversions between the uint8 interface layout and the
// packed storage of CAT_STORE_BIT1 instances (8 cells per byte, cell x in bit
// x % 8 of byte x / 8).  Used by cat_set_state / cat_get_state and when an
// instance changes storage; the step kernel reads and writes the packed rows
// itself.
#include <cuda_runtime.h>

#include <cstdint>

#include "cat_internal.h"

namespace cat {
namespace {

// One thread per packed byte: bit k = (cell 8b + k == 1); bits past W are 0.
__global__ void pack_bits_kernel(const uint8_t *src, int64_t spitch, uint8_t *dst, int64_t dpitch, int64_t rows,
                                 int64_t W) {
  const int64_t nb = (W + 7) / 8, n = rows * nb;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = i / nb, b = i - y * nb;
    const uint8_t *row = src + y * spitch;
    uint32_t bits = 0;
    for (int k = 0; k < 8; ++k) {
      const int64_t x = 8 * b + k;
      if (x < W && row[x] == 1) bits |= 1u << k;
    }
    dst[y * dpitch + b] = (uint8_t)bits;
  }
}

// One thread per cell.
__global__ void unpack_bits_kernel(const uint8_t *src, int64_t spitch, uint8_t *dst, int64_t dpitch, int64_t rows,
                                   int64_t W) {
  const int64_t n = rows * W;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = i / W, x = i - y * W;
    dst[y * dpitch + x] = (src[y * spitch + x / 8] >> (x % 8)) & 1u;
  }
}

int blocks_for(int64_t n) {
  const int64_t want = (n + 255) / 256;
  return (int)(want < 8192 ? (want > 0 ? want : 1) : 8192);
}

}  // namespace

cudaError_t pack_bits_launch(const uint8_t *src, int64_t spitch, uint8_t *dst, int64_t dpitch, int64_t rows,
                             int64_t W, cudaStream_t s) {
  pack_bits_kernel<<<blocks_for(rows * ((W + 7) / 8)), 256, 0, s>>>(src, spitch, dst, dpitch, rows, W);
  return cudaGetLastError();
}

cudaError_t unpack_bits_launch(const uint8_t *src, int64_t spitch, uint8_t *dst, int64_t dpitch, int64_t rows,
                               int64_t W, cudaStream_t s) {
  unpack_bits_kernel<<<blocks_for(rows * W), 256, 0, s>>>(src, spitch, dst, dpitch, rows, W);
  return cudaGetLastError();
}

}  // namespace cat
