// CUDA-core comparators for the tensor-core step.
//
// STENCIL: the classical shared-memory stencil the paper compares against
// (the out-halo SHARED approach, Sec. V-A, Table V): a CTA stages its haloed
// window of states in shared memory and every cell's (2r+1)^2 box is summed
// directly, O(r^2) per cell.  Four cells per 32-bit word: for every row and
// column offset of the box, the word of four shifted flags is added in
// packed bytes (each row's partial sums stay below 256) and then widened to
// 16-bit pairs.  With the simplified von Neumann neighbourhood (Eq. 3) it
// sums the vertical and the horizontal segment instead (the centre on both).
//
// RUNSUM: a separable running-sum kernel, O(1) per cell in r: vertical box
// sums V = sum of 2r+1 rows, kept as running sums down each column four
// columns per word (one add and one subtract per four cells and row), then
// horizontal box sums of V as running sums along each row (one add, one
// subtract per cell).  The counts are the same box sums as the band products
// of Sec. IV (Eqs. 1-2) compute, so it is the honest CUDA-core reference
// point for the tensor-core kernels at every r.
//
// Both stage 16-byte chunks of the input with vector loads; the window spans
// columns x0 - 32 .. x0 + 159 (a 32-cell halo for every r <= 32, so chunk
// loads stay aligned) and rows y0 - r .. y0 + BY + r - 1; cells outside the
// grid and bytes past W count as dead.  Both apply the rule of every C.
#include "cat_internal.h"

namespace cat {
namespace stencil {

constexpr int BX = 128, BY = 64;          // output tile
constexpr int kThreads = 256;
constexpr int kMaxR = 32;
constexpr int WX = BX + 64;               // window columns: 12 chunks of 16 bytes
constexpr int WY = BY + 2 * kMaxR;        // window rows (at most)
constexpr int VX = WX + 4;                // row stride of the vertical sums (bank spread)

__device__ __forceinline__ uint32_t next_state(int s, uint32_t c, const RuleDev &R) {
  if (c == 0) return (uint32_t)(s - R.b_lo) <= (uint32_t)R.b_w;
  if (c == 1) return ((uint32_t)(s - R.s_lo) <= (uint32_t)R.s_w) ? 1u : (R.C > 2 ? 2u : 0u);
  return (c + 1 == (uint32_t)R.C) ? 0u : c + 1;
}

// 0x01 in each byte of w holding state 1 (borrow-free byte test).
__device__ __forceinline__ uint32_t alive4(uint32_t w) {
  const uint32_t x = w ^ 0x01010101u;
  const uint32_t nonzero = ((((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x) >> 7) & 0x01010101u;
  return nonzero ^ 0x01010101u;
}

// Stages alive flags of window rows [y0 - r, y0 + BY + r) x columns
// [x0 - 32, x0 + 160) into A (row stride WX) and the raw centre tile into ctr
// (row stride CS: BX, or BX + 4 so that threads reading down a column of
// rows hit different banks).
template <int CS>
__device__ __forceinline__ void stage(const SimpleParams &p, int x0, int y0, int r, uint8_t *A, uint8_t *ctr) {
  const int rows = BY + 2 * r;
  for (int i = threadIdx.x; i < rows * (WX / 16); i += kThreads) {
    const int wy = i / (WX / 16), c = i - wy * (WX / 16);
    const int gy = y0 - r + wy, gx = x0 - 32 + 16 * c;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (gy >= 0 && gy < p.H && gx >= 0 && gx < p.W) {
      v = *reinterpret_cast<const uint4 *>(p.in + (int64_t)gy * p.pitch + gx);
      const int lim = p.W - gx;   // bytes of the chunk inside the grid
      if (lim < 16) {
        uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int keep = lim - 4 * k;
          w[k] = keep >= 4 ? w[k] : keep <= 0 ? 0u : w[k] & ((1u << (8 * keep)) - 1u);
        }
        v = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    if (wy >= r && wy < r + BY && c >= 2 && c < 10) {
      uint8_t *dst = ctr + (wy - r) * CS + 16 * (c - 2);
      if constexpr (CS % 16 == 0) {
        *reinterpret_cast<uint4 *>(dst) = v;
      } else {
        uint32_t *d4 = reinterpret_cast<uint32_t *>(dst);
        d4[0] = v.x; d4[1] = v.y; d4[2] = v.z; d4[3] = v.w;
      }
    }
    if (p.rule.C > 2) v = make_uint4(alive4(v.x), alive4(v.y), alive4(v.z), alive4(v.w));
    *reinterpret_cast<uint4 *>(A + wy * WX + 16 * c) = v;
  }
}

// Writes 32 next states (packed four per word) of row gy from column gx on.
__device__ __forceinline__ void store32(const SimpleParams &p, int gy, int gx, const uint32_t (&o)[8]) {
  uint8_t *dst = p.out + (int64_t)gy * p.pitch + gx;
  if (gx + 32 <= p.W) {
    reinterpret_cast<uint4 *>(dst)[0] = make_uint4(o[0], o[1], o[2], o[3]);
    reinterpret_cast<uint4 *>(dst)[1] = make_uint4(o[4], o[5], o[6], o[7]);
  } else {
    for (int t = 0; t < 32 && gx + t < p.W; ++t) dst[t] = (uint8_t)(o[t >> 2] >> (8 * (t & 3)));
  }
}

__global__ void __launch_bounds__(kThreads) smem_stencil_kernel(const SimpleParams p) {
  __shared__ __align__(16) uint8_t A[WY * WX + 16];   // + the word a shift by 0 loads past the last row
  __shared__ __align__(16) uint8_t ctr[BY * BX];
  const int r = p.rule.r;
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
  stage<BX>(p, x0, y0, r, A, ctr);
  __syncthreads();
  // lane q: the word of four cells 4q .. 4q + 3 of a row (consecutive lanes
  // read consecutive words, so no bank conflicts); warp w: rows w, w + 8, ...
  const int q = threadIdx.x & 31, w8 = threadIdx.x >> 5;
  const int gx = x0 + 4 * q;
  if (gx >= p.W) return;
  const int xw = 32 + 4 * q;              // window column of the word's first cell
  for (int y = w8; y < BY; y += kThreads / 32) {
    const int gy = y0 + y;
    if (gy >= p.H) break;
    uint32_t s01 = 0, s23 = 0;            // counts of cells 0,1 and 2,3 as 16-bit pairs
    if (p.rule.nbhd) {                    // Eq. 3: vertical and horizontal segment
      uint32_t h = 0;
      const uint32_t *row = reinterpret_cast<const uint32_t *>(A + (y + r) * WX);
      for (int d = 0; d <= 2 * r; ++d) {
        h += *reinterpret_cast<const uint32_t *>(A + (y + d) * WX + xw);
        const int b = xw - r + d, j = b >> 2;
        h += __funnelshift_r(row[j], row[j + 1], 8 * (b & 3));
      }
      s01 = __byte_perm(h, 0, 0x4140);
      s23 = __byte_perm(h, 0, 0x4342);
    } else {
      for (int dy = 0; dy <= 2 * r; ++dy) {
        const uint32_t *row = reinterpret_cast<const uint32_t *>(A + (y + dy) * WX);
        uint32_t h = 0;                   // this row's part of the four box sums (<= 65 per byte)
        for (int dx = 0; dx <= 2 * r; ++dx) {
          const int b = xw - r + dx, j = b >> 2;
          h += __funnelshift_r(row[j], row[j + 1], 8 * (b & 3));
        }
        s01 += __byte_perm(h, 0, 0x4140);
        s23 += __byte_perm(h, 0, 0x4342);
      }
    }
    const int sv[4] = {(int)(s01 & 0xFFFF), (int)(s01 >> 16), (int)(s23 & 0xFFFF), (int)(s23 >> 16)};
    if (p.sums) {
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (gx + t < p.W) p.sums[(int64_t)gy * p.sums_ld + gx + t] = sv[t];
      continue;
    }
    const uint32_t cw = *reinterpret_cast<const uint32_t *>(ctr + y * BX + 4 * q);
    uint32_t w = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) w |= next_state(sv[t], (cw >> (8 * t)) & 0xFFu, p.rule) << (8 * t);
    uint8_t *dst = p.out + (int64_t)gy * p.pitch + gx;
    if (gx + 4 <= p.W) {
      *reinterpret_cast<uint32_t *>(dst) = w;
    } else {
      for (int t = 0; gx + t < p.W; ++t) dst[t] = (uint8_t)(w >> (8 * t));
    }
  }
}

__global__ void __launch_bounds__(kThreads) runsum_kernel(const SimpleParams p) {
  constexpr int CS = BX + 4;   // centre rows 132 bytes apart: the 32 lanes' byte reads hit 32 banks
  __shared__ __align__(16) uint8_t A[WY * WX];
  __shared__ __align__(16) uint8_t ctr[BY * CS];
  __shared__ __align__(16) uint8_t V[BY * VX];
  const int r = p.rule.r;
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
  stage<CS>(p, x0, y0, r, A, ctr);
  __syncthreads();
  // vertical running sums, four columns per word: 48 word columns x 4 segments of 16 rows
  if (threadIdx.x < (WX / 4) * (BY / 16)) {
    const int wc = threadIdx.x % (WX / 4), seg = threadIdx.x / (WX / 4);
    const uint32_t *a = reinterpret_cast<const uint32_t *>(A) + wc;
    uint32_t *v = reinterpret_cast<uint32_t *>(V) + wc;
    const int yb = 16 * seg;                  // V row yb sums window rows yb .. yb + 2r
    uint32_t s = 0;
    for (int d = 0; d <= 2 * r; ++d) s += a[(yb + d) * (WX / 4)];
    v[yb * (VX / 4)] = s;
#pragma unroll 4
    for (int y = yb + 1; y < yb + 16; ++y) {
      s += a[(y + 2 * r) * (WX / 4)] - a[(y - 1) * (WX / 4)];   // no byte borrows: the removed flag was added
      v[y * (VX / 4)] = s;
    }
  }
  __syncthreads();
  // horizontal running sums along a 32-cell segment of a row
  const int k = threadIdx.x & 3, y = threadIdx.x >> 2;
  const int gy = y0 + y, gx = x0 + 32 * k;
  if (gy >= p.H || gx >= p.W) return;
  const uint8_t *vr = V + y * VX + 32 + 32 * k;   // V of the segment's first cell
  int s = 0;
  for (int d = -r; d <= r; ++d) s += vr[d];
  uint32_t o[8];
  const uint8_t *cr = ctr + y * CS + 32 * k;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    uint32_t w = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int x = 4 * q + t;
      if (x > 0) s += (int)vr[x + r] - (int)vr[x - 1 - r];
      if (p.sums) {
        if (gx + x < p.W) p.sums[(int64_t)gy * p.sums_ld + gx + x] = s;
      } else {
        w |= next_state(s, cr[x], p.rule) << (8 * t);
      }
    }
    o[q] = w;
  }
  if (!p.sums) store32(p, gy, gx, o);
}

}  // namespace stencil

cudaError_t stencil_launch(const SimpleParams &p, cudaStream_t s) {
  dim3 grid((p.W + stencil::BX - 1) / stencil::BX, (p.H + stencil::BY - 1) / stencil::BY);
  stencil::smem_stencil_kernel<<<grid, stencil::kThreads, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t runsum_launch(const SimpleParams &p, cudaStream_t s) {
  dim3 grid((p.W + stencil::BX - 1) / stencil::BX, (p.H + stencil::BY - 1) / stencil::BY);
  stencil::runsum_kernel<<<grid, stencil::kThreads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace cat
