// Packed storage: conversions between the uint8 interface layout and the
// packed rows of CAT_STORE_BIT1 instances (8 cells per byte, cell x in bit
// x % 8 of byte x / 8) and CAT_STORE_NIB4 instances (2 cells per byte, cell x
// in nibble x % 2 of byte x / 2).  Used by cat_set_state / cat_get_state and when an
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

// One thread per packed byte of four-bit storage: low nibble = cell 2b, high
// nibble = cell 2b + 1 (0 past W); states above 15 are not representable.
__global__ void pack_nib_kernel(const uint8_t *src, int64_t spitch, uint8_t *dst, int64_t dpitch, int64_t rows,
                                int64_t W) {
  const int64_t nb = (W + 1) / 2, n = rows * nb;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = i / nb, b = i - y * nb;
    const uint8_t *row = src + y * spitch;
    const uint32_t lo = row[2 * b] & 0xFu, hi = 2 * b + 1 < W ? row[2 * b + 1] & 0xFu : 0u;
    dst[y * dpitch + b] = (uint8_t)(lo | (hi << 4));
  }
}

__global__ void unpack_nib_kernel(const uint8_t *src, int64_t spitch, uint8_t *dst, int64_t dpitch, int64_t rows,
                                  int64_t W) {
  const int64_t n = rows * W;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = i / W, x = i - y * W;
    dst[y * dpitch + x] = (src[y * spitch + x / 2] >> (4 * (x & 1))) & 0xFu;
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

namespace cat {

cudaError_t pack_nib_launch(const uint8_t *src, int64_t spitch, uint8_t *dst, int64_t dpitch, int64_t rows,
                            int64_t W, cudaStream_t s) {
  pack_nib_kernel<<<blocks_for(rows * ((W + 1) / 2)), 256, 0, s>>>(src, spitch, dst, dpitch, rows, W);
  return cudaGetLastError();
}

cudaError_t unpack_nib_launch(const uint8_t *src, int64_t spitch, uint8_t *dst, int64_t dpitch, int64_t rows,
                              int64_t W, cudaStream_t s) {
  unpack_nib_kernel<<<blocks_for(rows * W), 256, 0, s>>>(src, spitch, dst, dpitch, rows, W);
  return cudaGetLastError();
}

}  // namespace cat
