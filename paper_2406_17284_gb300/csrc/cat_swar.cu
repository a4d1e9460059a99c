// Bit-sliced (SWAR) Larger-than-Life step on one-bit storage, radii 1..5.
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
//               reduced rule, each bound the carry chain of a bit-sliced
//               addition of a constant; the centre bit picks survival or birth.
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

// Bits needed for a value up to n.
constexpr int bits_for(int n) { return n < 2 ? 1 : 1 + bits_for(n / 2); }

template <int R>
struct Bits {
  static constexpr int kH = bits_for(2 * R + 1);                 // bits of a horizontal sum
  static constexpr int kS = bits_for((2 * R + 1) * (2 * R + 1));  // bits of a box count
};
static_assert(Bits<1>::kH == 2 && Bits<1>::kS == 4 && Bits<2>::kS == 5 && Bits<3>::kS == 6 && Bits<5>::kS == 7,
              "plane counts");

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

// S >= K for every cell of a word, as the carry out of the bit-sliced sum
// S + (2^NB - K): one majority function per bit, carry = maj(S_b, carry, k_b),
// where k_b is bit b of 2^NB - K replicated over a word (0 or ~0).  K <= 0 and
// K >= 2^NB are settled by the caller.
template <int NB>
__device__ __forceinline__ uint32_t bs_ge(const uint32_t (&S)[NB], const uint32_t (&k)[NB]) {
  uint32_t carry = 0;
#pragma unroll
  for (int b = 0; b < NB; ++b) carry = (S[b] & carry) | (k[b] & (S[b] | carry));
  return carry;
}

// One range [lo, lo + w] of the reduced rule as the constants of two carry
// chains: in range iff S >= lo and not S >= lo + w + 1, with the chains that
// can never or must always carry replaced by fixed words.
template <int NB>
struct RangeBits {
  uint32_t klo[NB], khi[NB];
  uint32_t lo_fix_and, lo_fix_or, hi_fix_and, hi_fix_or;
};

template <int NB>
__device__ __forceinline__ void bound_bits(int64_t K, uint32_t (&k)[NB], uint32_t &fix_and, uint32_t &fix_or) {
  // K <= 0: always >= K (or 1); K >= 2^NB: never (and 0); else the chain
  const int64_t c = (int64_t(1) << NB) - K;
#pragma unroll
  for (int b = 0; b < NB; ++b) k[b] = (K > 0 && K < (int64_t(1) << NB) && ((c >> b) & 1)) ? ~0u : 0u;
  fix_and = (K > 0 && K < (int64_t(1) << NB)) ? ~0u : 0u;
  fix_or = K <= 0 ? ~0u : 0u;
}

template <int NB>
__device__ __forceinline__ RangeBits<NB> range_bits(int lo, int w) {
  RangeBits<NB> rb;
  bound_bits<NB>(lo, rb.klo, rb.lo_fix_and, rb.lo_fix_or);
  bound_bits<NB>((int64_t)lo + w + 1, rb.khi, rb.hi_fix_and, rb.hi_fix_or);
  return rb;
}

template <int NB>
__device__ __forceinline__ uint32_t bs_in(const uint32_t (&S)[NB], const RangeBits<NB> &rb) {
  const uint32_t ge_lo = (bs_ge<NB>(S, rb.klo) & rb.lo_fix_and) | rb.lo_fix_or;
  const uint32_t ge_hi = (bs_ge<NB>(S, rb.khi) & rb.hi_fix_and) | rb.hi_fix_or;
  return ge_lo & ~ge_hi;
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
  const uint32_t last_mask = last_bits < 32 ? (1u << last_bits) - 1u : ~0u;
  const uint32_t mask = wi == p.words - 1 ? last_mask : ~0u;
  // the neighbour word this lane loads besides its own: lane 0 the one to the
  // left of the warp, lane 31 the one to the right (a warp covers 32 words)
  const int nc = lane == 0 ? wi - 1 : lane == 31 ? wi + 1 : wi;
  const bool nc_ok = nc >= 0 && nc < p.words;
  const uint32_t nmask = nc == p.words - 1 ? last_mask : ~0u;
  const uint32_t *in_c = p.in + (col ? wi : 0), *in_n = p.in + (nc_ok ? nc : 0);
  const RangeBits<NS> surv = range_bits<NS>(p.rule.s_lo, p.rule.s_w), born = range_bits<NS>(p.rule.b_lo, p.rule.b_w);
  // programmatic dependent launch: the next kernel may be scheduled, and the
  // grid is read only once the previous kernel (the step that wrote it) is done
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");

  // horizontal sums of row y for this thread's 32 cells (every lane takes part)
  auto hsum = [&](int y, uint32_t (&h)[NH], uint32_t &centre) {
    const bool row_ok = y >= 0 && y < p.H;
    const int64_t ro = row_ok ? (int64_t)y * p.pitch_words : 0;
    const uint32_t w = (row_ok && col) ? __ldg(in_c + ro) & mask : 0u;
    const uint32_t x = (row_ok && nc_ok) ? __ldg(in_n + ro) & nmask : 0u;
    uint32_t left = __shfl_up_sync(0xffffffffu, w, 1), right = __shfl_down_sync(0xffffffffu, w, 1);
    if (lane == 0) left = x;
    if (lane == 31) right = x;
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

  // strips of kRows rows, grid-stride in y (grids taller than 65535 strips)
  for (int64_t y0 = (int64_t)blockIdx.y * kRows; y0 < p.H; y0 += (int64_t)gridDim.y * kRows) {
    uint32_t hs[WIN][NH], cs[WIN];
#pragma unroll
    for (int k = 0; k < WIN - 1; ++k) hsum((int)y0 - R + k, hs[k + 1], cs[k + 1]);
    for (int i = 0; i < kRows; ++i) {
      const int y = (int)y0 + i;
      if (y >= p.H) break;                                        // uniform across the block
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
      p.out[(int64_t)y * p.pitch_words + wi] = ((c & bs_in<NS>(S, surv)) | (~c & bs_in<NS>(S, born))) & mask;
    }
  }
}

// ---------------------------------------------------------------------------
// Temporal blocking: k steps per launch on a tile kept in shared memory.  A
// block holds 128 word columns (the 126 of its tile and one on each side) of
// rows y0 - kR .. y0 + 32 + kR - 1; step s computes the rows whose 2R + 1-row
// neighbourhood is still valid after s - 1 steps (the stale halo grows by R
// rows, and R cells into the side words, per step), from one buffer into the
// other, and after k steps the tile's 32 x 126 words are written out.  Cells
// outside the grid are forced back to 0 after every step.  k R <= 8: two
// buffers of 48 rows x 128 words (48 KiB of dynamic shared memory).
constexpr int kTbThreads = 128, kTbTile = kTbThreads - 2, kTbRows = 32, kTbMaxHalo = 8;
constexpr int kTbBufRows = kTbRows + 2 * kTbMaxHalo;
constexpr int kTbSmem = 2 * kTbBufRows * kTbThreads * 4;

template <int R>
__global__ void __launch_bounds__(kTbThreads) ltl_swar_tb_kernel(const SwarParams p, int k) {
  constexpr int NH = Bits<R>::kH, NS = Bits<R>::kS, WIN = 2 * R + 1;
  extern __shared__ uint32_t tb_smem[];
  uint32_t(*buf)[kTbBufRows][kTbThreads] = reinterpret_cast<uint32_t(*)[kTbBufRows][kTbThreads]>(tb_smem);
  const int c = threadIdx.x;                                   // column in the block
  const int wi = blockIdx.x * kTbTile - 1 + c;                 // word column in the grid
  const int halo = k * R, rows = kTbRows + 2 * halo;
  const int64_t y0 = (int64_t)blockIdx.y * kTbRows;
  const int last_bits = p.W - 32 * (p.words - 1);
  const bool col = wi >= 0 && wi < p.words;
  const uint32_t mask = !col ? 0u : (wi == p.words - 1 && last_bits < 32) ? (1u << last_bits) - 1u : ~0u;
  const RangeBits<NS> surv = range_bits<NS>(p.rule.s_lo, p.rule.s_w), born = range_bits<NS>(p.rule.b_lo, p.rule.b_w);
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");   // as in ltl_swar_kernel
  asm volatile("griddepcontrol.wait;" ::: "memory");
  for (int i = 0; i < rows; ++i) {
    const int64_t y = y0 - halo + i;
    buf[0][i][c] = (col && y >= 0 && y < p.H) ? __ldg(p.in + y * p.pitch_words + wi) & mask : 0u;
  }
  __syncthreads();
  int cur = 0;
  for (int s = 1; s <= k; ++s) {
    const uint32_t(*A)[kTbThreads] = buf[cur];
    uint32_t(*B)[kTbThreads] = buf[cur ^ 1];
    auto hsum = [&](int i, uint32_t (&h)[NH], uint32_t &centre) {
      const uint32_t w = A[i][c];
      const uint32_t left = c > 0 ? A[i][c - 1] : 0u, right = c < kTbThreads - 1 ? A[i][c + 1] : 0u;
#pragma unroll
      for (int b = 0; b < NH; ++b) h[b] = 0u;
      const uint32_t w1[1] = {w};
      bs_add<NH, 1>(h, w1);
#pragma unroll
      for (int d = 1; d <= R; ++d) {
        const uint32_t l[1] = {__funnelshift_l(left, w, d)};
        const uint32_t r[1] = {__funnelshift_r(w, right, d)};
        bs_add<NH, 1>(h, l);
        bs_add<NH, 1>(h, r);
      }
      centre = w;
    };
    // rows lo .. hi - 1 of the buffer are computed in this step
    const int lo = s * R, hi = rows - s * R;
    uint32_t hs[WIN][NH], cs[WIN];
#pragma unroll
    for (int q = 0; q < WIN - 1; ++q) hsum(lo - R + q, hs[q + 1], cs[q + 1]);
    for (int i = lo; i < hi; ++i) {
#pragma unroll
      for (int q = 0; q < WIN - 1; ++q) {
#pragma unroll
        for (int b = 0; b < NH; ++b) hs[q][b] = hs[q + 1][b];
        cs[q] = cs[q + 1];
      }
      hsum(i + R, hs[WIN - 1], cs[WIN - 1]);
      uint32_t S[NS];
#pragma unroll
      for (int b = 0; b < NS; ++b) S[b] = b < NH ? hs[0][b] : 0u;
#pragma unroll
      for (int q = 1; q < WIN; ++q) bs_add<NS, NH>(S, hs[q]);
      const int64_t y = y0 - halo + i;
      const uint32_t cc = cs[R];
      const uint32_t nxt = (cc & bs_in<NS>(S, surv)) | (~cc & bs_in<NS>(S, born));
      B[i][c] = (y >= 0 && y < p.H) ? nxt & mask : 0u;   // cells outside the grid stay dead
    }
    __syncthreads();
    cur ^= 1;
  }
  if (c == 0 || c == kTbThreads - 1 || !col) return;
  for (int i = 0; i < kTbRows; ++i) {
    const int64_t y = y0 + i;
    if (y >= p.H) break;
    p.out[y * p.pitch_words + wi] = buf[cur][halo + i][c];
  }
}

// Launch configuration with programmatic stream serialization: the kernels
// above wait for the previous kernel in the stream before reading the grid.
cudaLaunchConfig_t pdl_config(dim3 grid, int threads, size_t smem, cudaStream_t s) {
  static cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

}  // namespace

cudaError_t swar_tb_launch(const uint8_t *in, uint8_t *out, int64_t pitch, int64_t H, int64_t W, const RuleDev &rule,
                           int k, cudaStream_t s) {
  if (k < 1 || k * rule.r > kTbMaxHalo) return cudaErrorInvalidValue;
  SwarParams p;
  p.in = reinterpret_cast<const uint32_t *>(in);
  p.out = reinterpret_cast<uint32_t *>(out);
  p.pitch_words = pitch / 4;
  p.H = (int32_t)H;
  p.W = (int32_t)W;
  p.words = (int32_t)((W + 31) / 32);
  p.rule = rule;
  p.sums = nullptr;
  p.sums_ld = 0;
  const int64_t strips = (H + kTbRows - 1) / kTbRows;
  if (strips > 65535) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)((p.words + kTbTile - 1) / kTbTile), (unsigned)strips);
  void (*kern)(SwarParams, int) = nullptr;
  switch (rule.r) {
    case 1: kern = ltl_swar_tb_kernel<1>; break;
    case 2: kern = ltl_swar_tb_kernel<2>; break;
    case 3: kern = ltl_swar_tb_kernel<3>; break;
    case 4: kern = ltl_swar_tb_kernel<4>; break;
    case 5: kern = ltl_swar_tb_kernel<5>; break;
    default: return cudaErrorInvalidValue;
  }
  static bool configured[6] = {false, false, false, false, false, false};
  if (!configured[rule.r]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kTbSmem);
    if (e != cudaSuccess) return e;
    configured[rule.r] = true;
  }
  cudaLaunchConfig_t cfg = pdl_config(grid, kTbThreads, kTbSmem, s);
  return cudaLaunchKernelEx(&cfg, kern, p, k);
}

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
  void (*kern)(SwarParams) = nullptr;
  switch (rule.r) {
    case 1: kern = ltl_swar_kernel<1>; break;
    case 2: kern = ltl_swar_kernel<2>; break;
    case 3: kern = ltl_swar_kernel<3>; break;
    case 4: kern = ltl_swar_kernel<4>; break;
    case 5: kern = ltl_swar_kernel<5>; break;
    default: return cudaErrorInvalidValue;
  }
  cudaLaunchConfig_t cfg = pdl_config(grid, kBlock, 0, s);
  return cudaLaunchKernelEx(&cfg, kern, p);
}

}  // namespace cat
