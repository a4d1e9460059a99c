// The paper's own fragment scheme (Sec. IV, Eqs. 4-5, Alg. 1) on warp-level
// tensor-core MMAs, as the "plain FP16 CAT" comparator.
//
// A CTA owns a tile of FH x FW output fragments of 16 x 16 cells plus one halo
// fragment on every side.  The band matrix Pi is represented by three 16 x 16
// fragments (Sec. IV):
//   pi1[a][b] = [a - b >= 16 - r]  (block below the diagonal block)
//   pi2[a][b] = [|a - b| <= r]     (diagonal block)
//   pi3[a][b] = [b - a >= 16 - r]  (block above the diagonal block)
// Step 1 (Eq. 4): F^H_{i,j} = F_{i,j-1} pi1 + F_{i,j} pi2 + F_{i,j+1} pi3 for
// every fragment row i including the halo rows; H stays in shared memory.
// Step 2 (Eq. 5, with F^H in all three terms, as in Alg. 1):
// F^R_{i,j} = pi3 F^H_{i-1,j} + pi2 F^H_{i,j} + pi1 F^H_{i+1,j}.
// Then every thread applies the LTL rule to its cells (Alg. 1, last loop).
// Simplified von Neumann neighbourhood (Eq. 3, R = Pi x Lambda + H), FP16 path:
// step 2 takes the Lambda fragments instead of F^H and starts from the
// accumulator F^H_{i,j} instead of zero (the MMA's C operand).
//
// FP16 path: nvcuda::wmma 16x16x16 with FP16 accumulation.  Every partial sum
// is an integer <= (2r+1)^2 <= 1089 < 2^11, so FP16 holds it exactly (Sec. V-A).
// INT8 path: the same three-fragment scheme on mma.sync m16n8k32 u8 x u8 -> s32
// (sm_103a has no tcgen05 kind::i8), with the K extent of a fragment triple
// (48) padded to 64.
#include <mma.h>

#include "cat_internal.h"

namespace cat {
namespace frag {

using namespace nvcuda;

constexpr int FW = 4, FH = 4;                  // tile of 4 x 4 fragments (64 x 64 cells)
constexpr int TW = 16 * FW, TH = 16 * FH;
constexpr int WW = TW + 32, WH = TH + 32;      // window with one halo fragment per side
constexpr int kThreads = 256;

__device__ __forceinline__ uint32_t next_state(int s, uint32_t c, const RuleDev &R) {
  if (c == 0) return (uint32_t)(s - R.b_lo) <= (uint32_t)R.b_w;
  if (c == 1) return ((uint32_t)(s - R.s_lo) <= (uint32_t)R.s_w) ? 1u : (R.C > 2 ? 2u : 0u);
  return (c + 1 == (uint32_t)R.C) ? 0u : c + 1;
}

__device__ __forceinline__ bool band_entry(int which, int a, int b, int r) {
  if (which == 0) return a - b >= 16 - r;
  if (which == 1) return (a - b <= r) && (b - a <= r);
  return b - a >= 16 - r;
}

__global__ void __launch_bounds__(kThreads) cat_wmma_f16_kernel(const SimpleParams p) {
  __shared__ __align__(32) half lam[WH * WW];
  __shared__ __align__(32) half qh[WH * TW];
  __shared__ __align__(32) half qr[TH * TW];
  __shared__ __align__(32) half pis[3][256];
  __shared__ uint8_t cst[TH * TW];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
  const RuleDev R = p.rule;

  for (int i = tid; i < WH * WW; i += kThreads) {
    const int y = i / WW, x = i - y * WW;
    const int gy = y0 - 16 + y, gx = x0 - 16 + x;
    uint8_t s = 0;
    if (gy >= 0 && gy < p.H && gx >= 0 && gx < p.W) s = p.in[(int64_t)gy * p.pitch + gx];
    lam[i] = __float2half(s == 1 ? 1.0f : 0.0f);
    if (y >= 16 && y < 16 + TH && x >= 16 && x < 16 + TW) cst[(y - 16) * TW + (x - 16)] = s;
  }
  for (int i = tid; i < 3 * 256; i += kThreads) {
    const int w = i >> 8, a = (i >> 4) & 15, b = i & 15;
    pis[w][a * 16 + b] = __float2half(band_entry(w, a, b, R.r) ? 1.0f : 0.0f);
  }
  __syncthreads();

  // Step 1: horizontal reduction for the interior fragment columns, all rows.
  for (int k = warp; k < (FH + 2) * FW; k += kThreads / 32) {
    const int i = k / FW, j = k - i * FW + 1;
    wmma::fragment<wmma::accumulator, 16, 16, 16, half> F;
    wmma::fill_fragment(F, __float2half(0.0f));
    wmma::fragment<wmma::matrix_a, 16, 16, 16, half, wmma::row_major> A;
    wmma::fragment<wmma::matrix_b, 16, 16, 16, half, wmma::row_major> B;
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
      wmma::load_matrix_sync(A, lam + (16 * i) * WW + 16 * (j + d), WW);
      wmma::load_matrix_sync(B, pis[d + 1], 16);
      wmma::mma_sync(F, A, B, F);
    }
    wmma::store_matrix_sync(qh + (16 * i) * TW + 16 * (j - 1), F, TW, wmma::mem_row_major);
  }
  __syncthreads();

  // Step 2: vertical reduction for the interior fragments.
  for (int k = warp; k < FH * FW; k += kThreads / 32) {
    const int i = k / FW + 1, j = k - (i - 1) * FW;
    wmma::fragment<wmma::accumulator, 16, 16, 16, half> F;
    wmma::fragment<wmma::matrix_a, 16, 16, 16, half, wmma::row_major> A;
    wmma::fragment<wmma::matrix_b, 16, 16, 16, half, wmma::row_major> B;
    if (R.nbhd) {  // Eq. 3: C = F^H_{i,j}, B = Lambda fragments
      wmma::load_matrix_sync(F, qh + (16 * i) * TW + 16 * j, TW, wmma::mem_row_major);
#pragma unroll
      for (int d = -1; d <= 1; ++d) {
        wmma::load_matrix_sync(A, pis[1 - d], 16);
        wmma::load_matrix_sync(B, lam + (16 * (i + d)) * WW + 16 * (j + 1), WW);
        wmma::mma_sync(F, A, B, F);
      }
    } else {
      wmma::fill_fragment(F, __float2half(0.0f));
#pragma unroll
      for (int d = -1; d <= 1; ++d) {
        wmma::load_matrix_sync(A, pis[1 - d], 16);  // pi3 for i-1, pi2 for i, pi1 for i+1
        wmma::load_matrix_sync(B, qh + (16 * (i + d)) * TW + 16 * j, TW);
        wmma::mma_sync(F, A, B, F);
      }
    }
    wmma::store_matrix_sync(qr + (16 * (i - 1)) * TW + 16 * j, F, TW, wmma::mem_row_major);
  }
  __syncthreads();

  // Transition, one thread per cell.
  for (int i = tid; i < TH * TW; i += kThreads) {
    const int y = i / TW, x = i - y * TW;
    const int gy = y0 + y, gx = x0 + x;
    if (gy >= p.H || gx >= p.W) continue;
    const int s = __half2int_rn(qr[i]);
    if (p.sums) p.sums[(int64_t)gy * p.sums_ld + gx] = s;
    else p.out[(int64_t)gy * p.pitch + gx] = (uint8_t)next_state(s, cst[i], R);
  }
}

// ------------------------------------------------------------------- INT8
// mma.sync.m16n8k32 u8: A 16x32 row-major, B 32x8 column-major, D 16x8 s32.
// Fragment ownership (lane = 4g + t): a0 = A[g][4t..4t+3], a1 = A[g+8][4t..],
// a2 = A[g][16+4t..], a3 = A[g+8][16+4t..]; b0 = B[4t..4t+3][g], b1 = B[16+4t..][g];
// d0,d1 = D[g][2t, 2t+1], d2,d3 = D[g+8][2t, 2t+1].
__device__ __forceinline__ void mma_u8(int (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

constexpr int kPad = 16;  // extra columns so every 64-wide K window stays in bounds
constexpr int WWI = WW + kPad;

// Band rows for one output fragment: Bq[n][k] = 1 iff (k - 16) - n in [-r, r],
// n < 16 outputs, k < 64 inputs starting one fragment to the left / above.
__global__ void __launch_bounds__(kThreads) cat_mma_i8_kernel(const SimpleParams p) {
  __shared__ __align__(16) uint8_t lam[WH * WWI];   // window, row-major (rows y', cols x')
  __shared__ __align__(16) uint8_t hT[TW * (WH + kPad)];  // H^T: rows x, cols y'
  __shared__ __align__(16) uint8_t bq[16 * 64];      // band as K-contiguous rows
  __shared__ __align__(16) int qr[TH * TW];
  __shared__ uint8_t cst[TH * TW];
  constexpr int LDH = WH + kPad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
  const RuleDev R = p.rule;

  for (int i = tid; i < WH * WWI; i += kThreads) {
    const int y = i / WWI, x = i - y * WWI;
    const int gy = y0 - 16 + y, gx = x0 - 16 + x;
    uint8_t s = 0;
    if (x < WW && gy >= 0 && gy < p.H && gx >= 0 && gx < p.W) s = p.in[(int64_t)gy * p.pitch + gx];
    lam[i] = s == 1;
    if (y >= 16 && y < 16 + TH && x >= 16 && x < 16 + TW) cst[(y - 16) * TW + (x - 16)] = s;
  }
  for (int i = tid; i < TW * LDH; i += kThreads) hT[i] = 0;
  for (int i = tid; i < 16 * 64; i += kThreads) {
    const int n = i >> 6, k = i & 63;
    const int d = (k - 16) - n;
    bq[i] = (d >= -R.r && d <= R.r) ? 1 : 0;
  }
  __syncthreads();

  // Step 1: H[y'][x] for all window rows y' and interior columns x.
  // Per (16-row block i, 16-col output block j): D(16 x 16) = X[rows][16j .. 16j+64) x Bq^T.
  for (int k = warp; k < (FH + 2) * FW; k += kThreads / 32) {
    const int i = k / FW, j = k - i * FW;
#pragma unroll
    for (int nh = 0; nh < 2; ++nh) {
      int d[4] = {0, 0, 0, 0};
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const uint8_t *A0 = lam + (16 * i) * WWI + 16 * j + 32 * ks;
        uint32_t a[4], b[2];
        a[0] = *reinterpret_cast<const uint32_t *>(A0 + g * WWI + 4 * t);
        a[1] = *reinterpret_cast<const uint32_t *>(A0 + (g + 8) * WWI + 4 * t);
        a[2] = *reinterpret_cast<const uint32_t *>(A0 + g * WWI + 16 + 4 * t);
        a[3] = *reinterpret_cast<const uint32_t *>(A0 + (g + 8) * WWI + 16 + 4 * t);
        const uint8_t *B0 = bq + (8 * nh + g) * 64 + 32 * ks;
        b[0] = *reinterpret_cast<const uint32_t *>(B0 + 4 * t);
        b[1] = *reinterpret_cast<const uint32_t *>(B0 + 16 + 4 * t);
        mma_u8(d, a, b);
      }
      // D[row][n] = H[16i + row][16j + 8nh + n] -> hT[x][y']
      const int xa = 16 * j + 8 * nh + 2 * t;
      hT[(xa)*LDH + 16 * i + g] = (uint8_t)d[0];
      hT[(xa + 1) * LDH + 16 * i + g] = (uint8_t)d[1];
      hT[(xa)*LDH + 16 * i + g + 8] = (uint8_t)d[2];
      hT[(xa + 1) * LDH + 16 * i + g + 8] = (uint8_t)d[3];
    }
  }
  __syncthreads();

  // Step 2: S[y][x] = sum_y' Band[y][y'] H[y'][x]; A = Bq (rows y, K = y'), B = H^T (col-major).
  for (int k = warp; k < FH * FW; k += kThreads / 32) {
    const int i = k / FW, j = k - i * FW;
#pragma unroll
    for (int nh = 0; nh < 2; ++nh) {
      int d[4] = {0, 0, 0, 0};
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        uint32_t a[4], b[2];
        const uint8_t *A0 = bq + 32 * ks;
        a[0] = *reinterpret_cast<const uint32_t *>(A0 + g * 64 + 4 * t);
        a[1] = *reinterpret_cast<const uint32_t *>(A0 + (g + 8) * 64 + 4 * t);
        a[2] = *reinterpret_cast<const uint32_t *>(A0 + g * 64 + 16 + 4 * t);
        a[3] = *reinterpret_cast<const uint32_t *>(A0 + (g + 8) * 64 + 16 + 4 * t);
        const uint8_t *B0 = hT + (16 * j + 8 * nh + g) * LDH + 16 * i + 32 * ks;
        b[0] = *reinterpret_cast<const uint32_t *>(B0 + 4 * t);
        b[1] = *reinterpret_cast<const uint32_t *>(B0 + 16 + 4 * t);
        mma_u8(d, a, b);
      }
      const int xa = 16 * j + 8 * nh + 2 * t, ya = 16 * i + g;
      qr[ya * TW + xa] = d[0];
      qr[ya * TW + xa + 1] = d[1];
      qr[(ya + 8) * TW + xa] = d[2];
      qr[(ya + 8) * TW + xa + 1] = d[3];
    }
  }
  __syncthreads();

  for (int i = tid; i < TH * TW; i += kThreads) {
    const int y = i / TW, x = i - y * TW;
    const int gy = y0 + y, gx = x0 + x;
    if (gy >= p.H || gx >= p.W) continue;
    if (p.sums) p.sums[(int64_t)gy * p.sums_ld + gx] = qr[i];
    else p.out[(int64_t)gy * p.pitch + gx] = (uint8_t)next_state(qr[i], cst[i], R);
  }
}

// ------------------------------------------------------- 16 < r <= 32, FP16
// The extension the paper describes beyond the fragment size (Sec. VII): the
// neighbours of a fragment reach two fragments away, so each reduction takes
// five band fragments (offsets -2 .. 2) and the window carries a halo of two
// fragments.  H <= 65 stays exact in FP16; the counts reach 65^2 = 4225 >
// 2^11, so step 2 accumulates in FP32 (the paper's remark that FP16 stops
// being precise enough at such radii).
constexpr int kWideHF = 2;                          // halo fragments per side
constexpr int WWX = TW + 32 * kWideHF, WHX = TH + 32 * kWideHF;
constexpr size_t kWideSmem = (size_t)WHX * WWX * 2 + (size_t)WHX * TW * 2 + (size_t)TH * TW * 4 +
                             2 * 5 * 256 * 2 + (size_t)TH * TW;

__global__ void __launch_bounds__(kThreads) cat_wmma_f16_wide_kernel(const SimpleParams p) {
  extern __shared__ __align__(128) uint8_t wide_smem[];
  half *lam = reinterpret_cast<half *>(wide_smem);                 // WHX x WWX
  half *qh = lam + WHX * WWX;                                       // WHX x TW  (H, all window rows)
  float *qr = reinterpret_cast<float *>(qh + WHX * TW);             // TH x TW   (counts)
  half *pk = reinterpret_cast<half *>(qr + TH * TW);                // step 1: P_d[k][n] = [|16d + k - n| <= r]
  half *pm = pk + 5 * 256;                                          // step 2: A_d[m][k] = [|16d + k - m| <= r]
  uint8_t *cst = reinterpret_cast<uint8_t *>(pm + 5 * 256);         // TH x TW centre states
  const int tid = threadIdx.x, warp = tid >> 5;
  const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
  const RuleDev R = p.rule;
  constexpr int H0 = 16 * kWideHF;                                  // halo width in cells

  for (int i = tid; i < WHX * WWX; i += kThreads) {
    const int y = i / WWX, x = i - y * WWX;
    const int gy = y0 - H0 + y, gx = x0 - H0 + x;
    uint8_t s = 0;
    if (gy >= 0 && gy < p.H && gx >= 0 && gx < p.W) s = p.in[(int64_t)gy * p.pitch + gx];
    lam[i] = __float2half(s == 1 ? 1.0f : 0.0f);
    if (y >= H0 && y < H0 + TH && x >= H0 && x < H0 + TW) cst[(y - H0) * TW + (x - H0)] = s;
  }
  for (int i = tid; i < 5 * 256; i += kThreads) {
    const int d = i / 256 - kWideHF, a = (i >> 4) & 15, b = i & 15;
    const int e1 = 16 * d + a - b, e2 = 16 * d + b - a;
    pk[i] = __float2half(e1 >= -R.r && e1 <= R.r ? 1.0f : 0.0f);   // a = k, b = n
    pm[i] = __float2half(e2 >= -R.r && e2 <= R.r ? 1.0f : 0.0f);   // a = m, b = k
  }
  __syncthreads();

  // Step 1: F^H_{i,j} = sum_d F_{i, j+d} P_d, every fragment row of the window.
  for (int k = warp; k < (FH + 2 * kWideHF) * FW; k += kThreads / 32) {
    const int i = k / FW, j = k - i * FW;
    wmma::fragment<wmma::accumulator, 16, 16, 16, half> F;
    wmma::fill_fragment(F, __float2half(0.0f));
    wmma::fragment<wmma::matrix_a, 16, 16, 16, half, wmma::row_major> A;
    wmma::fragment<wmma::matrix_b, 16, 16, 16, half, wmma::row_major> B;
#pragma unroll
    for (int d = -kWideHF; d <= kWideHF; ++d) {
      wmma::load_matrix_sync(A, lam + (16 * i) * WWX + 16 * (j + kWideHF + d), WWX);
      wmma::load_matrix_sync(B, pk + (d + kWideHF) * 256, 16);
      wmma::mma_sync(F, A, B, F);
    }
    wmma::store_matrix_sync(qh + (16 * i) * TW + 16 * j, F, TW, wmma::mem_row_major);
  }
  __syncthreads();

  // Step 2: F^R_{i,j} = sum_d A_d F^H_{i+d, j}, FP32 accumulation.
  for (int k = warp; k < FH * FW; k += kThreads / 32) {
    const int i = k / FW, j = k - i * FW;
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> F;
    wmma::fill_fragment(F, 0.0f);
    wmma::fragment<wmma::matrix_a, 16, 16, 16, half, wmma::row_major> A;
    wmma::fragment<wmma::matrix_b, 16, 16, 16, half, wmma::row_major> B;
#pragma unroll
    for (int d = -kWideHF; d <= kWideHF; ++d) {
      wmma::load_matrix_sync(A, pm + (d + kWideHF) * 256, 16);
      wmma::load_matrix_sync(B, qh + (16 * (i + kWideHF + d)) * TW + 16 * j, TW);
      wmma::mma_sync(F, A, B, F);
    }
    wmma::store_matrix_sync(qr + (16 * i) * TW + 16 * j, F, TW, wmma::mem_row_major);
  }
  __syncthreads();

  for (int i = tid; i < TH * TW; i += kThreads) {
    const int y = i / TW, x = i - y * TW;
    const int gy = y0 + y, gx = x0 + x;
    if (gy >= p.H || gx >= p.W) continue;
    const int s = __float2int_rn(qr[i]);
    if (p.sums) p.sums[(int64_t)gy * p.sums_ld + gx] = s;
    else p.out[(int64_t)gy * p.pitch + gx] = (uint8_t)next_state(s, cst[i], R);
  }
}

}  // namespace frag

// dt follows cat.h: 1 = FP16, 3 = INT8.  FP16 with r > 16 runs the wide kernel.
cudaError_t mma_launch(const SimpleParams &p, int dt, cudaStream_t s) {
  dim3 grid((p.W + frag::TW - 1) / frag::TW, (p.H + frag::TH - 1) / frag::TH);
  if (dt == 3) {
    frag::cat_mma_i8_kernel<<<grid, frag::kThreads, 0, s>>>(p);
  } else if (p.rule.r > 16) {
    static bool configured = false;
    if (!configured) {
      cudaError_t e = cudaFuncSetAttribute(frag::cat_wmma_f16_wide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)frag::kWideSmem);
      if (e != cudaSuccess) return e;
      configured = true;
    }
    frag::cat_wmma_f16_wide_kernel<<<grid, frag::kThreads, frag::kWideSmem, s>>>(p);
  } else {
    frag::cat_wmma_f16_kernel<<<grid, frag::kThreads, 0, s>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace cat
