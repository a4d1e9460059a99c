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

__device__ __forceinline__ int wrap32(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// The frame in three kinds of items, none of which reads a ghost cell, so
// they need no order among themselves:
//   rows     the grid columns of the 2G frame rows, 16 bytes per item (the
//            framed row and its source share the offset G = 16, so full
//            chunks are aligned 16-byte copies);
//   columns  the G left and G right frame cells of one grid row (two aligned
//            16-byte copies when W is a multiple of 16, else per byte);
//   corners  the 4 G x G corner cells, one per item.
// Grid-stride over rows, then columns, then corners.  The kernel lets the
// next kernel in the stream start its set-up and reads the grid only after
// the previous kernel (the step that wrote it) has completed.
__global__ void ghost_fill_kernel(uint8_t *base, int64_t pitch, int H, int W, int G) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int chunks = (W + 15) / 16;
  const int64_t n_rows = 2 * (int64_t)G * chunks, n_cols = 2 * (int64_t)H, n_corners = 4 * (int64_t)G * G;
  const int64_t n_all = n_rows + n_cols + n_corners;
  const bool vec_cols = (W % 16) == 0 && W >= G;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_all; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n_rows) {
      const int fr = (int)(i / chunks), ch = (int)(i - (int64_t)fr * chunks);
      const int py = fr < G ? fr : H + fr;                       // rows 0..G-1 and H+G..H+2G-1
      const int sy = wrap32(py - G, H) + G;
      uint8_t *dst = base + (int64_t)py * pitch + G + 16 * ch;
      const uint8_t *src = base + (int64_t)sy * pitch + G + 16 * ch;
      if (16 * ch + 16 <= W) {
        *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(src);
      } else {
        for (int b = 0; b < W - 16 * ch; ++b) dst[b] = src[b];
      }
    } else if (i < n_rows + n_cols) {
      const int64_t k = i - n_rows;
      const int y = (int)(k >> 1), side = (int)(k & 1);
      uint8_t *row = base + (int64_t)(G + y) * pitch;
      const int px0 = side ? W + G : 0;                          // first frame column of this side
      if (vec_cols && G == 16) {
        // left: grid columns W-16..W-1 (framed W..W+15); right: grid 0..15 (framed 16..31)
        *reinterpret_cast<uint4 *>(row + px0) = *reinterpret_cast<const uint4 *>(row + (side ? G : W));
      } else {
        for (int b = 0; b < G; ++b) row[px0 + b] = row[wrap32(px0 + b - G, W) + G];
      }
    } else {
      const int k = (int)(i - n_rows - n_cols), corner = k / (G * G), c = k - corner * G * G;
      const int py = (corner & 1 ? H + G : 0) + c / G, px = (corner & 2 ? W + G : 0) + c % G;
      base[(int64_t)py * pitch + px] = base[(int64_t)(wrap32(py - G, H) + G) * pitch + wrap32(px - G, W) + G];
    }
  }
}

}  // namespace

// Launched programmatically dependent on the previous kernel in the stream
// (see ghost_fill_kernel); the tcgen05 step launched after it is in turn
// dependent on it.
cudaError_t ghost_fill_launch(uint8_t *base, int64_t pitch, int64_t H, int64_t W, int G, cudaStream_t s) {
  const int64_t n = 2 * (int64_t)G * ((W + 15) / 16) + 2 * H + 4 * (int64_t)G * G;
  const int threads = 256;
  const int64_t want = (n + threads - 1) / threads;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(want < 4096 ? want : 4096));
  cfg.blockDim = dim3(threads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, ghost_fill_kernel, base, pitch, (int)H, (int)W, G);
}

}  // namespace cat
