// Classical shared-memory CUDA-core stencil (the out-halo SHARED approach the
// paper compares against, Sec. V-A Table V): a CTA stages its (B + 2r)^2
// window of states in shared memory and every thread sums the (2r+1)^2 box of
// each of its cells directly, then applies the LTL rule.  O(r^2) work per cell.
// With the simplified von Neumann neighbourhood (Eq. 3) it sums the vertical
// and the horizontal segment instead (the centre on both), O(r) per cell.
#include "cat_internal.h"

namespace cat {
namespace stencil {

constexpr int BX = 32, BY = 32;           // output tile
constexpr int kThreads = 256;             // 32 x 8 threads, 4 rows each
constexpr int kMaxR = 32;
constexpr int SW = BX + 2 * kMaxR, SH = BY + 2 * kMaxR;

__device__ __forceinline__ uint32_t next_state(int s, uint32_t c, const RuleDev &R) {
  if (c == 0) return (uint32_t)(s - R.b_lo) <= (uint32_t)R.b_w;
  if (c == 1) return ((uint32_t)(s - R.s_lo) <= (uint32_t)R.s_w) ? 1u : (R.C > 2 ? 2u : 0u);
  return (c + 1 == (uint32_t)R.C) ? 0u : c + 1;
}

__global__ void __launch_bounds__(kThreads) smem_stencil_kernel(const SimpleParams p) {
  __shared__ uint8_t win[SH * SW];
  __shared__ uint8_t ctr[BY * BX];
  const int r = p.rule.r;
  const int ww = BX + 2 * r, wh = BY + 2 * r;
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
  for (int i = threadIdx.x; i < wh * ww; i += kThreads) {
    const int y = i / ww, x = i - y * ww;
    const int gy = y0 - r + y, gx = x0 - r + x;
    uint8_t s = 0;
    if (gy >= 0 && gy < p.H && gx >= 0 && gx < p.W) s = p.in[(int64_t)gy * p.pitch + gx];
    win[y * SW + x] = s == 1;
    if (y >= r && y < r + BY && x >= r && x < r + BX) ctr[(y - r) * BX + (x - r)] = s;
  }
  __syncthreads();
  const int tx = threadIdx.x & 31, ty0 = threadIdx.x >> 5;
  for (int ty = ty0; ty < BY; ty += kThreads / 32) {
    const int gy = y0 + ty, gx = x0 + tx;
    if (gy >= p.H || gx >= p.W) continue;
    int s = 0;
    if (p.rule.nbhd) {
      for (int d = 0; d <= 2 * r; ++d) s += win[(ty + d) * SW + tx + r] + win[(ty + r) * SW + tx + d];
    } else {
      for (int dy = 0; dy <= 2 * r; ++dy) {
        const uint8_t *row = win + (ty + dy) * SW + tx;
        for (int dx = 0; dx <= 2 * r; ++dx) s += row[dx];
      }
    }
    if (p.sums) p.sums[(int64_t)gy * p.sums_ld + gx] = s;
    else p.out[(int64_t)gy * p.pitch + gx] = (uint8_t)next_state(s, ctr[ty * BX + tx], p.rule);
  }
}

}  // namespace stencil

cudaError_t stencil_launch(const SimpleParams &p, cudaStream_t s) {
  dim3 grid((p.W + stencil::BX - 1) / stencil::BX, (p.H + stencil::BY - 1) / stencil::BY);
  stencil::smem_stencil_kernel<<<grid, stencil::kThreads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace cat
