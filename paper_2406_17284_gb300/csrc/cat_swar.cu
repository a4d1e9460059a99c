// Bit-sliced (SWAR) Larger-than-Life step on one-bit storage, radii 1..3.
//
// At the smallest radii the paper finds its packed-cell comparator faster
// than the tensor-core method (Sec. V-B: at r = 1 the packed program beats
// CAT by 2.3x; CAT wins from r = 3): a (2r+1)^2 box of one-bit cells is a few
// additions, and the tensor cores' fixed cost per tile no longer pays.  This
// kernel is that regime's design for GB300, on CUDA cores: every 32-bit word
// of a packed row holds 32 cells, and the counts of all 32 are computed at
// once as bit planes (bit b of every cell's count in one word), with full
// adders made of bitwise operations.
//
//   horizontal  h(y, x) = sum_{|d| <= r} cell(y, x + d): the 2r + 1 shifted
//               copies of a row word (funnel shifts with the neighbouring
//               words, fetched by warp shuffles) added as 1-bit numbers;
//   vertical    S(y, x) = sum_{|d| <= r} h(y + d, x): 2r + 1 bit-sliced
//               numbers added (the horizontal sums of a thread's rows are
//               kept in registers while it walks down its strip);
//   rule        S in [lo, lo + w] for the survival and birth ranges of the
//               reduced rule, each bound a bit-serial comparison with a
//               constant; the centre bit picks survival or birth.
//
// S is the Moore box count with the centre (Sec. IV, Eqs. 1-2 compute the
// same number as band products); the reduced rule's survival bounds already
// account for the M flag.  Cells past W stay 0.  One thread per word column
// and strip of kRows output rows; a warp covers 32 consecutive words of a row.
#include <cuda_runtime.h>

#include <cstdint>

#include "cat_internal.h"

namespace cat {
namespace {

constexpr int kRows = 32;        // output rows per thread
constexpr int kBlock = 256;      // threads: 8 warps side by side, 256 words

template <int R>
struct Bits {
  static constexpr int kH = 2 * R + 1 <= 3 ? 2 : 3;                         // bits of a horizontal sum
  static constexpr int kS = (2 * R + 1) * (2 * R + 1) < 16 ? 4 : (2 * R + 1) * (2 * R + 1) < 32 ? 5 : 6;
};

// acc += x (bit-sliced, NX-bit x into an NB-bit accumulator).
template <int NB, int NX>
__device__ __forceinline__ void bs_add(uint32_t (&acc)[NB], const uint32_t (&x)[NX]) {
  uint32_t c = 0;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const uint32_t xb = b < NX ? x[b] : 0u;
    const uint32_t a = acc[b];
    acc[b] = a ^ xb ^ c;
    c = (a & xb) | (c & (a ^ xb));
  }
}

// Plane of the cells whose count S >= K (K uniform across the grid).
template <int NB>
__device__ __forceinline__ uint32_t bs_ge(const uint32_t (&S)[NB], int K) {
  if (K <= 0) return ~0u;
  if (K >= (1 << NB)) return 0u;
  uint32_t gt = 0, eq = ~0u;
#pragma unroll
  for (int b = NB - 1; b >= 0; --b) {
    if ((K >> b) & 1) {
      eq &= S[b];
    } else {
      gt |= eq & S[b];
      eq &= ~S[b];
    }
  }
  return gt | eq;
}

// Plane of the cells whose count lies in [lo, lo + w].
template <int NB>
__device__ __forceinline__ uint32_t bs_in(const uint32_t (&S)[NB], int lo, int w) {
  if (lo >= (1 << NB)) return 0u;
  const int64_t end = (int64_t)lo + w + 1;                     // first count above the range
  return bs_ge<NB>(S, lo) & (end >= (1 << NB) ? ~0u : ~bs_ge<NB>(S, (int)end));
}

struct SwarParams {
  const uint32_t *in;
  uint32_t *out;
  int64_t pitch_words;   // 32-bit words between rows
  int32_t H, W, words;   // rows, cells per row, words holding them
  RuleDev rule;
  int32_t *sums;
  int64_t sums_ld;
};

template <int R>
__global__ void __launch_bounds__(kBlock) ltl_swar_kernel(const SwarParams p) {
  constexpr int NH = Bits<R>::kH, NS = Bits<R>::kS, WIN = 2 * R + 1;
  const int lane = threadIdx.x & 31;
  const int wi = blockIdx.x * kBlock + threadIdx.x;             // word column
  const bool col = wi < p.words;
  const int last_bits = p.W - 32 * (p.words - 1);                 // valid bits of the last word
  const uint32_t mask = (wi == p.words - 1 && last_bits < 32) ? (1u << last_bits) - 1u : ~0u;

  // the word of row y at column c, 0 outside the grid
  auto word = [&](int y, int c) -> uint32_t {
    if (y < 0 || y >= p.H || c < 0 || c >= p.words) return 0u;
    const uint32_t v = __ldg(p.in + (int64_t)y * p.pitch_words + c);
    return c == p.words - 1 && last_bits < 32 ? v & ((1u << last_bits) - 1u) : v;
  };
  // horizontal sums of row y for this thread's 32 cells (every lane takes part)
  auto hsum = [&](int y, uint32_t (&h)[NH], uint32_t &centre) {
    const uint32_t w = col ? word(y, wi) : 0u;
    uint32_t left = __shfl_up_sync(0xffffffffu, w, 1), right = __shfl_down_sync(0xffffffffu, w, 1);
    if (lane == 0) left = word(y, wi - 1);
    if (lane == 31) right = word(y, wi + 1);
#pragma unroll
    for (int b = 0; b < NH; ++b) h[b] = 0u;
    const uint32_t w1[1] = {w};
    bs_add<NH, 1>(h, w1);
#pragma unroll
    for (int d = 1; d <= R; ++d) {
      const uint32_t l[1] = {__funnelshift_l(left, w, d)};    // cell x - d at bit x
      const uint32_t r[1] = {__funnelshift_r(w, right, d)};   // cell x + d at bit x
      bs_add<NH, 1>(h, l);
      bs_add<NH, 1>(h, r);
    }
    centre = w;
  };

  const RuleDev &rd = p.rule;
  // strips of kRows rows, grid-stride in y (grids taller than 65535 strips)
  for (int64_t y0 = (int64_t)blockIdx.y * kRows; y0 < p.H; y0 += (int64_t)gridDim.y * kRows) {
  uint32_t hs[WIN][NH], cs[WIN];
#pragma unroll
  for (int k = 0; k < WIN - 1; ++k) hsum((int)y0 - R + k, hs[k + 1], cs[k + 1]);
  for (int i = 0; i < kRows; ++i) {
    const int y = (int)y0 + i;
    if (y >= p.H) break;                                          // uniform across the block
#pragma unroll
    for (int k = 0; k < WIN - 1; ++k) {
#pragma unroll
      for (int b = 0; b < NH; ++b) hs[k][b] = hs[k + 1][b];
      cs[k] = cs[k + 1];
    }
    hsum(y + R, hs[WIN - 1], cs[WIN - 1]);
    uint32_t S[NS];
#pragma unroll
    for (int b = 0; b < NS; ++b) S[b] = b < NH ? hs[0][b] : 0u;
#pragma unroll
    for (int k = 1; k < WIN; ++k) bs_add<NS, NH>(S, hs[k]);
    if (!col) continue;
    const uint32_t c = cs[R];
    if (p.sums) {
      int32_t *row = p.sums + (int64_t)y * p.sums_ld;
      for (int t = 0; t < 32 && 32 * wi + t < p.W; ++t) {
        int v = 0;
#pragma unroll
        for (int b = 0; b < NS; ++b) v |= (int)((S[b] >> t) & 1u) << b;
        row[32 * wi + t] = v;
      }
      continue;
    }
    const uint32_t surv = bs_in<NS>(S, rd.s_lo, rd.s_w), born = bs_in<NS>(S, rd.b_lo, rd.b_w);
    p.out[(int64_t)y * p.pitch_words + wi] = ((c & surv) | (~c & born)) & mask;
  }
  }
}

}  // namespace

cudaError_t swar_launch(const uint8_t *in, uint8_t *out, int64_t pitch, int64_t H, int64_t W, const RuleDev &rule,
                        int32_t *sums, int64_t sums_ld, cudaStream_t s) {
  SwarParams p;
  p.in = reinterpret_cast<const uint32_t *>(in);
  p.out = reinterpret_cast<uint32_t *>(out);
  p.pitch_words = pitch / 4;
  p.H = (int32_t)H;
  p.W = (int32_t)W;
  p.words = (int32_t)((W + 31) / 32);
  p.rule = rule;
  p.sums = sums;
  p.sums_ld = sums_ld;
  const int64_t strips = (H + kRows - 1) / kRows;
  const dim3 grid((unsigned)((p.words + kBlock - 1) / kBlock), (unsigned)(strips < 65535 ? strips : 65535));
  switch (rule.r) {
    case 1: ltl_swar_kernel<1><<<grid, kBlock, 0, s>>>(p); break;
    case 2: ltl_swar_kernel<2><<<grid, kBlock, 0, s>>>(p); break;
    case 3: ltl_swar_kernel<3><<<grid, kBlock, 0, s>>>(p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace cat
