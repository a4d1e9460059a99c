// Periodic boundary: the ghost frame.
//
// A periodic instance keeps its H x W grid inside a frame of G = 16 ghost cells
// on every side (G >= r for every served radius).  Before each step this kernel
// writes every ghost cell with the grid cell it wraps to, ((y mod H), (x mod W))
// in grid coordinates, so the step kernel can treat the framed grid like any
// other: its windows read real neighbours across every edge (the paper's own
// boundary, Sec. V), and its tiles start at TMA coordinate (x0 + G, y0 + G),
// which keeps every TMA x-coordinate 16-byte aligned.  The frame is 2G(W + 2G)
// + 2GH cells: 1.05 M cells for a 16384^2 grid, against 268 M in the grid.
#include <cuda_runtime.h>

#include <cstdint>

#include "cat_internal.h"

namespace cat {
namespace {

__device__ __forceinline__ int64_t wrap(int64_t v, int64_t n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// One thread per ghost cell, grid-stride.  Cells 0 .. 2G(W+2G)-1 are the G top
// and G bottom frame rows (full width); the rest are the left and right frame
// columns of the H grid rows.
__global__ void ghost_fill_kernel(uint8_t *base, int64_t pitch, int64_t H, int64_t W, int G) {
  const int64_t WP = W + 2 * G;
  const int64_t n_rows = 2 * (int64_t)G * WP, n_all = n_rows + 2 * (int64_t)G * H;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_all;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t py, px;                                  // framed coordinates
    if (i < n_rows) {
      const int64_t r = i / WP;
      px = i - r * WP;
      py = r < G ? r : H + r;                        // rows 0..G-1 and H+G..H+2G-1
    } else {
      const int64_t k = i - n_rows, r = k / (2 * G), c = k - r * (2 * G);
      py = G + r;
      px = c < G ? c : W + c;                        // columns 0..G-1 and W+G..W+2G-1
    }
    const int64_t sy = wrap(py - G, H) + G, sx = wrap(px - G, W) + G;
    base[py * pitch + px] = base[sy * pitch + sx];
  }
}

}  // namespace

cudaError_t ghost_fill_launch(uint8_t *base, int64_t pitch, int64_t H, int64_t W, int G, cudaStream_t s) {
  const int64_t n = 2 * (int64_t)G * (W + 2 * G) + 2 * (int64_t)G * H;
  const int threads = 256;
  const int64_t want = (n + threads - 1) / threads;
  const int blocks = (int)(want < 4096 ? want : 4096);
  ghost_fill_kernel<<<blocks, threads, 0, s>>>(base, pitch, H, W, G);
  return cudaGetLastError();
}

}  // namespace cat
