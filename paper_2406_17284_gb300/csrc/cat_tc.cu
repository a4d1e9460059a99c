// One Larger-than-Life step on the 5th-generation tensor cores (sm_103a).
//
// The box count of every cell is the CAT band product of Sec. IV (Eqs. 1-2):
// a horizontal reduction H = Lambda x Pi followed by a vertical one R = Pi x H,
// Pi the 0/1 band of half-width r.  The paper cuts Pi into three 16x16
// fragments per output fragment (out-halo scheme, Sec. IV, Eqs. 4-5, Alg. 1);
// here one CTA owns a 128 x 128 output tile and both products are single
// dense tcgen05 MMAs over a haloed 160 x 160 window:
//
//   window  X[y'][x'] = state(y0-16+y', x0-16+x') == 1,  y', x' in [0, 160)
//   band    B[m][k]   = 1 iff k - m in [16-r, 16+r],       m < 128, k < 160
//   pass 1  D1[x][y'] = sum_x' B[x][x'] X[y'][x']   = H^T   (M=128, N=160, K=160)
//   pass 2  D2[y][x]  = sum_y' B[y][y'] D1[x][y']   = S     (M=128, N=128, K=160)
//
// The band is the A operand of both products and lives in tensor memory
// (written once per radius by the convert warps); only the window and the
// pass-2 operand are read from shared memory.  An MMA with both operands in
// shared memory reads 128 bytes per clock at N = 128, which is all of the
// SM's shared-memory bandwidth and starves the convert and epilogue warps.
//
// The window offset is a fixed 16 cells for every r <= 16, so every TMA load
// starts on a 16-byte boundary; r only changes the band.  Cells outside the
// grid arrive as TMA zero fill (dead ghost cells, the zero halo of Sec. IV).
// D1 leaves TMEM lane-locally (lane x owns row x of H^T, which is row x of the
// K-major pass-2 operand), so no transpose is needed between the passes; D2
// has one output row per TMEM lane, so the epilogue reads 16 contiguous
// centre states and writes 16 contiguous next states per access.
//
// Precision (exact in every case, Sec. V-A):
//   FP16 kernel: X, band and H in f16; D1 = H, D2 = S.
//   FP8 kernel:  pass 1 on e4m3 -- the raw 0/1 state bytes ARE the B operand
//                (0x01 reads as e4m3 2^-9), so D1 = H * 2^-9 exactly; pass 2
//                takes H * 2^-9 as e4m3 when 2r+1 <= 15 (all such values are
//                e4m3 numbers) and as f16 otherwise (e4m3 cannot hold the odd
//                counts above 16); D2 = S * 2^-9.  The wide tile (r <= 32,
//                H <= 65) splits H into e4m3 digits instead (see Tm).
// The epilogue compares S (as f16, exact up to 2048) against the rule's
// ranges two cells at a time in half2 arithmetic.
//
// Roles (896 threads): warp 0 = window TMA loads, warp 1 = TMEM allocator and
// pass-1 MMA issuer, warp 2 = centre-tile TMA loads and TMA stores, warp 3 =
// pass-2 MMA issuer, warps 4..11 = convert warps (D1 -> pass-2 operand,
// window encoding when needed, bands), warps 12..27 = epilogue warps (fused
// transition).  The two worker roles
// work on different tiles at once; tensor memory holds the accumulator
// regions and the bands (see Tm below).  Both products
// accumulate in f16 (exact: every partial sum is a multiple of the operand
// scale no larger than 1089 times it), so the workers read f16 pairs straight
// from TMEM.  Every wait is bounded; on timeout the CTA records
// kDevErrTimeout, drains its own in-flight copies and MMAs, frees TMEM and
// returns.
#include <cuda_fp16.h>

#include "cat_internal.h"
#include "ptx.cuh"

namespace cat {
namespace tc {

constexpr int kTile = 128;
constexpr int kWin = 160;
constexpr int kCvtWarps = 8;                       // two per TMEM lane quarter
constexpr int kEpiWarps = 16;                      // four per TMEM lane quarter
constexpr int kCvtThreads = 32 * kCvtWarps;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kThreads = 128 + kCvtThreads + kEpiThreads;
constexpr int kMaxRegions = 3;

// Window geometry and tensor memory, by kernel variant.  The standard window
// is 160 x 160 starting 16 cells above and left of the tile; two 160-column
// accumulator regions (D1, then D2 of a tile) leave room for the f16 band (80
// columns, pass 2 when 2r+1 > 15 and the FP16 kernel) and the e4m3 band (40).
// Short window (SW, FP8 with r <= 7, where pass 2 runs on e4m3): the window
// holds 144 rows starting 8 above the tile (TMA y-coordinates need no
// alignment), so pass 1 has N = 144 and three 144-column regions fit beside
// two e4m3 bands -- pass 1's (window columns offset by 16) and pass 2's
// (window rows offset by 8): 3 * 144 + 40 + 40 = 512.  Three tiles are then in
// flight instead of two.
// Wide tile (WIDE, radii up to 32): a 96 x 96 output tile inside the same
// 160 x 160 window, which then starts 32 cells above and left of the tile
// (96 + 2 * 32 = 160; x0 - 32 stays 16-byte aligned since x0 is a multiple of
// 96).  The bands have offset 32 and rows 96..127 zero, so the MMA shapes stay
// M = 128, K = 160; pass 2 has N = 96.
// Big window (BIG, radii up to 32 on the 128 x 128 tile): the window is
// 192 x 192 starting 32 cells above and left of the tile, so pass 1 has
// N = K = 192 (six K-steps); pass 2 takes H as two e4m3 digits (H <= 65)
// against the band of ones and a band of 16s (48 columns each at K = 192)
// into an f32 accumulator over the tile's own D1 region: 2 * 192 + 48 + 48 =
// 480 columns.
template <bool SW, bool WIDE = false, bool BIG = false>
struct Geo {
  static constexpr int kTS = WIDE ? 96 : 128;         // output tile side
  static constexpr int kXOff = (WIDE || BIG) ? 32 : 16;   // window columns left of the tile
  static constexpr int kRows = SW ? 144 : BIG ? 192 : 160;   // window rows = pass-1 N
  static constexpr int kYOff = (WIDE || BIG) ? 32 : (SW ? 8 : 16);   // window rows above the tile
  static constexpr int kRegions = SW ? 3 : 2;
  static constexpr int kRegionCols = SW ? 144 : BIG ? 192 : 160;
  static constexpr uint32_t kBand16 = 320;            // f16 band (standard only)
  static constexpr uint32_t kBand8 = SW ? 432 : BIG ? 384 : 416;  // e4m3 band, offset kXOff (pass 1; also pass 2 if not SW)
  static constexpr uint32_t kBand8P2 = SW ? 472 : BIG ? 384 : 416;  // e4m3 band for pass 2 (offset kYOff)
};
constexpr uint32_t kTmemCols = 512;

// Tensor-memory map of a kernel.  In the 128 x 128 kernels a tile's D2
// overwrites its D1 region, which stays taken from pass 1 until the epilogue
// has read S: two 160-column regions beside the f16 band (80 columns, pass 2
// when 2r+1 > 15, and the FP16 kernel) and the e4m3 band (40), or three
// 144-column regions in the short window.  The wide tile (DEC) keeps them
// apart: two 160-column D1 regions, free again once the convert warps have
// read H, and one 96-column D2 region, free once the epilogue has read S.
// Its counts reach 4225, so D2 accumulates in f32 and H (up to 65) splits into
// H & 15 and H >> 4 (at most 4), both e4m3 codes of themselves times 2^-9,
// the second against a band of 16s: 2 * 160 + 96 + 40 + 40 = 496 columns.
// (The same split for the 128 x 128 FP8 kernel -- pass 2 on e4m3 for every r,
// no f16 band, and separate D1 / D2 regions, 2 + 1 or 1 + 2 -- measured 8%
// and 3% slower at r >= 8 than the shared regions, 2.05 and 2.15 against
// 2.22 * 10^12 cell updates/s, so it is not used there.)
template <int DT, bool SW, bool WIDE = false, bool BIG = false>
struct Tm {
  using GB = Geo<SW, false, BIG>;
  static constexpr bool kDec = DT == 1 && !SW && WIDE;
  static constexpr int kND1 = kDec ? 2 : GB::kRegions;
  static constexpr int kND2 = kDec ? 1 : GB::kRegions;
  static constexpr uint32_t kD1Cols = GB::kRegionCols;
  static constexpr uint32_t kD2Base = kDec ? kND1 * kD1Cols : 0;
  static constexpr uint32_t kD2Cols = kDec ? Geo<SW, WIDE>::kTS : GB::kRegionCols;
  static constexpr uint32_t kBand16 = GB::kBand16;          // FP16 kernel only
  static constexpr uint32_t kBand8 = kDec ? kD2Base + kND2 * kD2Cols : GB::kBand8;
  static constexpr uint32_t kBand8P2 = kDec ? kBand8 : GB::kBand8P2;
  static constexpr uint32_t kBand8x16 = kBand8 + (BIG ? 48 : 40);   // wide tile, big window: the band of 16s
  static_assert(!kDec || kBand8 + (WIDE ? 80 : 40) <= kTmemCols, "tensor memory budget");
  static_assert(!BIG || kBand8x16 + 48 <= kTmemCols, "tensor memory budget");
  static_assert(kND1 <= kMaxRegions && kND2 <= kMaxRegions, "barrier arrays");
};

// Byte offset of the element at byte position kb (= k * E) of row `row` in a
// K-major operand tile of R rows.  A row holds 160 elements of E bytes, split
// into E blocks of 128 bytes (128B swizzle, rows at 128 B pitch) followed by E
// blocks of 32 bytes (32B swizzle, rows at 32 B pitch).  The swizzles XOR the
// 16-byte chunk index with address bits [7,10) (128B) or bit 7 (32B).
__device__ __forceinline__ uint32_t op_off(int R, int E, int row, int kb) {
  if (kb < 128 * E) {
    const int blk = kb >> 7, w = kb & 127;
    return blk * R * 128 + row * 128 + ((((w >> 4) ^ row) & 7) << 4) + (w & 15);
  }
  const int kk = kb - 128 * E, blk = kk >> 5, w = kk & 31;
  return E * R * 128 + blk * R * 32 + row * 32 + ((((w >> 4) ^ (row >> 2)) & 1) << 4) + (w & 15);
}

// UMMA descriptors of such a tile: the 128B-swizzle and 32B-swizzle
// descriptors of its base address.  K-step j (32 bytes of K) is then the
// matching one plus a compile-time offset (op_desc_k), so issuing an MMA costs
// one add per operand instead of a full descriptor encode.
struct OpDesc {
  uint64_t d128, d32;
};

__device__ __forceinline__ OpDesc op_descs(uint32_t base) {
  return OpDesc{smem_desc(base, 16, 1024, kSwizzle128B), smem_desc(base, 16, 256, kSwizzle32B)};
}

// The start-address field holds address >> 4 in its low 14 bits; shared
// addresses stay below 2^18, so adding to it never carries into other fields.
template <int R, int E, int J>
__device__ __forceinline__ uint64_t op_desc_k(const OpDesc &d) {
  constexpr int kb = 32 * J;
  if constexpr (kb < 128 * E) {
    return d.d128 + (uint64_t)(((kb >> 7) * R * 128 + (kb & 127)) >> 4);
  } else {
    return d.d32 + (uint64_t)((E * R * 128 + ((kb - 128 * E) >> 5) * R * 32) >> 4);
  }
}

// Issues the K-steps of one band product: D = A[M=128, K=160] x B[N, K=160]^T
// with the band A in tensor memory (32 bytes of K = 8 columns per step) and
// B in shared memory.
// ACC: the first K-step adds to D instead of overwriting it.  KS: K-steps per
// operand byte (5 for K = 160, 6 for the big window's K = 192).
template <int KIND, int RB, int E, bool ACC = false, int KS = 5, int J = 0>
__device__ __forceinline__ void band_mma(uint32_t d, uint32_t a_tmem, const OpDesc &b, uint32_t idesc) {
  if constexpr (J < KS * E) {
    if constexpr (KIND == 0) mma_f16_ts(d, a_tmem + 8 * J, op_desc_k<RB, E, J>(b), idesc, ACC || J > 0);
    else mma_f8f6f4_ts(d, a_tmem + 8 * J, op_desc_k<RB, E, J>(b), idesc, ACC || J > 0);
    band_mma<KIND, RB, E, ACC, KS, J + 1>(d, a_tmem, b, idesc);
  }
}

// DT 0: FP16 kernel; DT 1: FP8 kernel.  ENC: the window is re-encoded in
// shared memory (always for FP16; for FP8 only when C > 2).  The centre tile
// of every output tile gets its own TMA load into a ring of NR entries that
// also serves as the output staging (the epilogue overwrites each centre state
// with the next state in place), so the 160 x 160 window stage is free as
// soon as pass 1 (or the encoding) has read it.
// BITS: the grid is stored one bit per cell (8 cells per byte, lowest x in the
// lowest bit); a window stage is then one 48-byte x 160-row box (cells x0 - 128
// .. x0 + 255, of which the window uses x0 - 16 .. x0 + 143) that the convert
// warps unpack into the e4m3 operand, and a ring entry is 16 bytes x 128 rows.
// NIB: four bits per cell (two cells per byte, the even x in the low nibble);
// a window stage is one 96-byte x 160-row box (cells x0 - 32 .. x0 + 159),
// unpacked by the convert warps into the e4m3 operand, and a ring entry is 64
// bytes x 128 rows (64B swizzle).
// BIG: a window stage is 192 x 192 bytes (a 128-column and two 32-column
// boxes), an H buffer two 128 x 192 digit halves.
template <int DT, bool ENC, bool SW = false, bool BITS = false, bool WIDE = false, bool NIB = false,
          bool BIG = false>
struct Layout {
  static constexpr int E1 = DT == 0 ? 2 : 1;                  // pass-1 operand bytes
  static constexpr int NS = (SW || BITS || NIB) ? 4 : ((DT == 0 || ENC || BIG) ? 2 : 3);   // TMA window stages
  static constexpr int NR = (SW || BITS || NIB) ? 4 : ((DT == 0 || ENC) ? 2 : 3);  // centre / output ring
  static constexpr int NE = (BITS || NIB) ? 3 : (ENC ? 2 : 1);  // encoded windows (encode ahead)
  // pass-2 operand buffers: FP16 one, so that its two 50 KiB encoded windows
  // fit (the encode then runs beside pass 1 instead of before it); four-bit
  // storage one, for its third encoded window (measured 2% faster)
  static constexpr int NH = SW ? 3 : ((DT == 0 || NIB) ? 1 : 2);
  static constexpr uint32_t kXs = 0;                          // raw windows (TMA)
  static constexpr uint32_t kXsBytes = BITS ? 48 * kWin : NIB ? 96 * kWin : BIG ? 192 * 192 : kWin * Geo<SW>::kRows;
  static constexpr uint32_t kXsStride = (kXsBytes + 1023) / 1024 * 1024;  // 128B-swizzle atoms stay aligned
  static constexpr uint32_t kXe = kXs + NS * kXsStride;       // encoded window
  static constexpr uint32_t kXeStride = kWin * kWin * E1;     // one encoded window (25 or 50 KiB)
  static constexpr uint32_t kXeBytes = ENC ? NE * kXeStride : 0;
  static constexpr uint32_t kH = kXe + kXeBytes;              // pass-2 operand (K padded to 160)
  static constexpr uint32_t kHBytes = kTile * (BIG ? 192 : kWin) * (SW ? 1 : 2);
  static constexpr uint32_t kRing = kH + NH * kHBytes;        // centre tiles / output staging
  static constexpr uint32_t kRingBytes = BITS ? 16 * kTile : NIB ? 64 * kTile : Geo<SW, WIDE>::kTS * Geo<SW, WIDE>::kTS;
  static constexpr uint32_t kBars = kRing + NR * kRingBytes;
  static constexpr uint32_t kDyn = kBars + 512 + 1024;        // + alignment slack
  static_assert(kDyn <= 232448, "shared memory budget");
  static_assert(kH >= kXs + NS * kXsStride && kH >= kXe + kXeBytes, "window stages and encoded windows end before H");
  static_assert(kXe % 1024 == 0 && kXeStride % 1024 == 0 && kH % 1024 == 0 && kRing % 1024 == 0 && kHBytes % 1024 == 0,
                "swizzled operands start on 1024-byte boundaries");
};

constexpr int kMaxStages = 6;

struct Bars {
  uint64_t x_full[kMaxStages], x_empty[kMaxStages];
  uint64_t c_full[kMaxStages], out_full[kMaxStages];
  uint64_t d1_full[kMaxRegions], d2_full[kMaxRegions], tmem_empty[kMaxRegions];
  uint64_t h_full[3], enc_full[3], band_ready;
  uint64_t d1_empty[kMaxRegions], h_empty[3];   // wide tile: D1 read, H read
  uint64_t mma_done[2], never;
  uint32_t tmem_base;
  int abort;
};

static_assert(sizeof(Bars) <= 512, "the barrier block fits its reserved 512 bytes");

__device__ __forceinline__ void set_abort(Bars *b, int32_t *err, int where) {
  b->abort = 1;
  if (err) atomicCAS(err, 0, kDevErrTimeout | where);
}

// Every lane waits; the warp agrees on the outcome.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, Bars *b, uint64_t timeout_ns) {
  bool ok = mbar_wait(bar, parity, &b->abort, timeout_ns);
  return __all_sync(0xffffffffu, ok);
}

// One 16-cell unit of the e2m1 window operand (kind::f8f6f4 reads e2m1 from
// shared memory as 16 elements packed into the first 8 bytes of every 16-byte
// unit, element 2i in the low nibble of byte i; bytes 8..15 are not read):
// the flags 0/1 of the 16 cells, bytes of w[0..3], as e2m1 codes 0 / 1 (0.5).
__device__ __forceinline__ uint2 fp4_unit(const uint32_t (&w)[4]) {
  // w | w >> 4 holds cells 0, 1 in byte 0 and cells 2, 3 in byte 2
  return make_uint2(__byte_perm(w[0] | (w[0] >> 4), w[1] | (w[1] >> 4), 0x6420),
                    __byte_perm(w[2] | (w[2] >> 4), w[3] | (w[3] >> 4), 0x6420));
}

// Eight cells' bits (bits 0..7 of b) -> eight nibbles 0/1 (bit i to bit 4i).
__device__ __forceinline__ uint32_t bits8_to_nibbles(uint32_t b) {
  uint32_t x = b & 0xFFu;
  x = (x | (x << 12)) & 0x000F000Fu;
  x = (x | (x << 6)) & 0x03030303u;
  return (x | (x << 3)) & 0x11111111u;
}

// Encodes the 160 x 160 u8 window xs as operand values: alive (state 1) ->
// 0x01 (e4m3 2^-9, FP8 kernel), f16 1.0 (FP16 kernel) or e2m1 0.5 (FP4
// kernel, packed units), anything else -> 0.
// FP8 and FP4: the encoded window has the raw window's layout unit for unit
// (a swizzle moves whole 16-byte units, and a unit holds 16 consecutive cells
// of one row), so the buffer is encoded as a flat array of units: consecutive
// threads take consecutive units (no bank conflicts, no address arithmetic
// beyond the index).  The state-1 test per byte: x = w ^ 0x01 is zero exactly
// where the state is 1, and bit 7 of ((x & 0x7F) + 0x7F) | x is set exactly
// where x is not zero (no carry leaves a byte).
template <int E, bool FP4 = false>
__device__ __forceinline__ void encode_window(const uint8_t *xs, uint8_t *xe, bool multistate,
                                              int tid, int nthr) {
  constexpr int kUnits = kWin * 10;
  if constexpr (E == 1) {
    const uint4 *src = reinterpret_cast<const uint4 *>(xs);
    for (int q = tid; q < kUnits; q += nthr) {
      const uint4 v = src[q];
      uint32_t w[4] = {v.x, v.y, v.z, v.w};
      if (multistate) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const uint32_t x = w[i] ^ 0x01010101u;
          w[i] = ((((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x) >> 7 & 0x01010101u) ^ 0x01010101u;
        }
      }
      if constexpr (FP4) reinterpret_cast<uint2 *>(xe)[2 * q] = fp4_unit(w);
      else reinterpret_cast<uint4 *>(xe)[q] = make_uint4(w[0], w[1], w[2], w[3]);
    }
  } else {
    // f16 operands take two units per source unit: positions through op_off;
    // consecutive threads take consecutive rows of one 16-byte column chunk,
    // so every warp access touches each bank group evenly under both swizzles
    for (int q = tid; q < kUnits; q += nthr) {
      const int c = q / kWin, row = q - c * kWin;
      uint4 v = *reinterpret_cast<const uint4 *>(xs + op_off(kWin, 1, row, 16 * c));
      uint32_t w[4] = {v.x, v.y, v.z, v.w};
      if (multistate) {
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] = __vcmpeq4(w[i], 0x01010101u) & 0x01010101u;
      }
      uint32_t h[8];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        h[2 * i] = __byte_perm(w[i], 0, 0x4140) * 0x3C00u;
        h[2 * i + 1] = __byte_perm(w[i], 0, 0x4342) * 0x3C00u;
      }
      *reinterpret_cast<uint4 *>(xe + op_off(kWin, 2, row, 32 * c)) = make_uint4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<uint4 *>(xe + op_off(kWin, 2, row, 32 * c + 16)) = make_uint4(h[4], h[5], h[6], h[7]);
    }
  }
}

// Unpacks a bit-packed window stage (160 rows of 48 bytes, window cell x' at
// bit x' + 112 of the row) into the e4m3 window operand: byte x' is the cell's
// bit left in place within its nibble, 2^(x' mod 4) (codes 1, 2, 4, 8: the
// e4m3 numbers 2^(x' mod 4) * 2^-9) for a live cell, which the pass-1 band's
// 2^-(x' mod 4) scales back to 2^-9 exactly -- one byte permute and one mask
// per four cells (FP4: e2m1 units, code 1 for a live cell).  One item is half a row (80
// cells, 16-cell chunks 5h .. 5h+4): three aligned 32-bit loads (bytes 12 +
// 12h ..), shifted by 16 bits for h = 0 so that the chunks are the five
// consecutive 16-bit fields.
template <bool FP4 = false>
__device__ __forceinline__ void unpack_window(const uint8_t *xs, uint8_t *xe, int tid, int nthr) {
  for (int q = tid; q < 2 * kWin; q += nthr) {
    const int h = q >= kWin ? 1 : 0, row = q - h * kWin;
    const uint32_t *src = reinterpret_cast<const uint32_t *>(xs + row * 48 + 12 + 12 * h);
    uint32_t a = src[0], b = src[1], c = src[2];
    if (!h) {
      a = __funnelshift_r(a, b, 16);
      b = __funnelshift_r(b, c, 16);
      c >>= 16;
    }
    const uint32_t f[5] = {a, a >> 16, b, b >> 16, c};
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      if constexpr (FP4)
        *reinterpret_cast<uint2 *>(xe + op_off(kWin, 1, row, 16 * (5 * h + i))) =
            make_uint2(bits8_to_nibbles(f[i]), bits8_to_nibbles(f[i] >> 8));
      else   // byte j of each word: bit j of its cell's source nibble, i.e. 2^j for a live cell
        *reinterpret_cast<uint4 *>(xe + op_off(kWin, 1, row, 16 * (5 * h + i))) =
            make_uint4(__byte_perm(f[i], 0, 0x0000) & 0x08040201u, __byte_perm(f[i] >> 4, 0, 0x0000) & 0x08040201u,
                       __byte_perm(f[i], 0, 0x1111) & 0x08040201u, __byte_perm(f[i] >> 4, 0, 0x1111) & 0x08040201u);
    }
  }
}

// Bytes 0/1 of four nibble flags 0/1 held in the 16-bit field `sel` (0x4140:
// the low half of a, 0x4342: the high half) of a.
__device__ __forceinline__ uint32_t nib4_to_bytes(uint32_t a, uint32_t sel) {
  const uint32_t t = __byte_perm(a, 0, sel);   // the field's two bytes in bytes 0 and 2
  return (t | (t << 4)) & 0x0F0F0F0Fu;
}

// Unpacks a four-bit window stage (160 rows of 96 bytes, window cell x' in
// nibble x' % 2 of byte 8 + x' / 2) into the e4m3 window operand: 0x01 for
// state 1, else 0 (FP4: the nibble flags are already the packed e2m1 unit).
// Item = two 16-cell units of a row (16 source bytes): units 2p and 2p + 1
// sit in the two halves of one 32-byte slot under either swizzle (their
// positions differ in the lowest bit), so the second offset is the first
// XOR 16; consecutive threads take consecutive items of a row.
template <bool FP4 = false>
__device__ __forceinline__ void unpack_nib_window(const uint8_t *xs, uint8_t *xe, int tid, int nthr) {
  for (int q = tid; q < kWin * 5; q += nthr) {
    const int row = q / 5, pr = q - row * 5;
    const uint2 *src = reinterpret_cast<const uint2 *>(xs + row * 96 + 8 + 16 * pr);
    const uint2 a = src[0], b = src[1];
    const uint32_t w[4] = {a.x, a.y, b.x, b.y};
    uint32_t f[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {   // nibble 1 where the state is 1 (borrow-free nibble test)
      const uint32_t x = w[i] ^ 0x11111111u;
      const uint32_t nz = (((x & 0x77777777u) + 0x77777777u) | x) & 0x88888888u;
      f[i] = (nz ^ 0x88888888u) >> 3;
    }
    const uint32_t o0 = op_off(kWin, 1, row, 32 * pr), o1 = o0 ^ 16u;
    if constexpr (FP4) {
      *reinterpret_cast<uint2 *>(xe + o0) = make_uint2(f[0], f[1]);
      *reinterpret_cast<uint2 *>(xe + o1) = make_uint2(f[2], f[3]);
    } else {
      *reinterpret_cast<uint4 *>(xe + o0) = make_uint4(nib4_to_bytes(f[0], 0x4140), nib4_to_bytes(f[0], 0x4342),
                                                       nib4_to_bytes(f[1], 0x4140), nib4_to_bytes(f[1], 0x4342));
      *reinterpret_cast<uint4 *>(xe + o1) = make_uint4(nib4_to_bytes(f[2], 0x4140), nib4_to_bytes(f[2], 0x4342),
                                                       nib4_to_bytes(f[3], 0x4140), nib4_to_bytes(f[3], 0x4342));
    }
  }
}

// Packs the states of four cells (bytes 0..3 of w, each below 16) pairwise:
// byte 0 of the result holds cells 0 and 1 (low and high nibble), byte 2
// cells 2 and 3; bytes 1 and 3 hold no cell.
__device__ __forceinline__ uint32_t bytes_to_nib_pairs(uint32_t w) { return w | (w >> 4); }

// Band B[m][k] = one iff k - m in [off - r, off + r] as an A operand in tensor
// memory: row m in lane m, K packed along the columns (two f16 values, or four
// e4m3 values, per column, the lowest k in the low bits); 80 columns (f16) or
// 40 (e4m3).  Standard kernels hold the f16 band (FP16 kernel and pass 2 when
// 2r+1 > 15) and, in the FP8 kernel, the e4m3 band, both with offset 16;
// short-window kernels hold two e4m3 bands, offset 16 (pass 1) and offset 8
// (pass 2).  The FP4 kernel holds the FP8 kernel's two pass-2 bands, the f16
// one with 2^-8 for one (its pass 1 leaves H / 2, not H * 2^-9), and an e2m1
// band for pass 1 in the 40 columns after the e4m3 one (kind::f8f6f4 reads an
// e2m1 A operand from tensor memory as one element per byte with the code in
// bits 2..5, so 1.0 = 0010b is 0x08), all with offset 16.  The one-bit FP8
// kernel keeps its pass-1 band in those 40 columns too: 2^-(k mod 4) at K
// index k, against window bytes 2^(k mod 4) * 2^-9.  Convert warp (q, kq)
// writes lanes 32q .. 32q+31 and every other 8-column chunk from chunk kq.
// The big window holds the e4m3 band and the band of 16s, 48 columns each
// (K = 192), with offset 32.
template <int DT, bool SW, bool WIDE = false, bool FP4 = false, bool BITS = false, bool BIG = false>
__device__ __forceinline__ void store_bands(uint32_t tmem, int r, int q, int kq, int lane) {
  using G = Geo<SW, WIDE, BIG>;
  using T = Tm<DT, SW, WIDE, BIG>;
  constexpr bool W32 = WIDE || BIG;                 // offset 32, the band of 16s second
  // chunks [0, n0) belong to the first band, [n0, n1) to the second, [n1, n)
  // to a third: the f16 band (standard window; the FP16 kernel has only this
  // one) and the e4m3 band, or in the short window the e4m3 bands of pass 1
  // and pass 2, or in the wide tile the e4m3 band and the band of 16s (offset
  // 32, rows 96..127 zero), or in the FP4 kernel the f16 band of 2^-8 (pass 2
  // on H / 2), the e4m3 band and the e2m1 band (pass 1, after the e4m3 one);
  // the one-bit kernel's pass-1 band sits there too: e4m3 2^-(k mod 4) at
  // column k, against window bytes 2^(k mod 4) * 2^-9 for live cells
  constexpr int n0 = BIG ? 6 : WIDE ? 5 : (SW ? 5 : 10), n1 = BIG ? 12 : WIDE ? 10 : (SW ? 10 : (DT == 1 ? 15 : 10));
  constexpr int n = (FP4 || BITS) ? 20 : n1;
  const int m = 32 * q + lane;
  const uint32_t la = static_cast<uint32_t>(32 * q) << 16;
  for (int c = kq; c < n; c += 2) {                 // warp-uniform
    const bool first = c < n0, third = c >= n1;
    const bool f16 = !SW && !W32 && first;
    const int cc = first ? c : third ? c - n1 : c - n0;
    const int off = W32 ? G::kXOff : (SW && !first) ? G::kYOff : 16;
    const uint32_t col = third ? T::kBand8 + 40
                       : W32 ? (first ? T::kBand8 : T::kBand8x16)
                       : SW ? (first ? G::kBand8 : G::kBand8P2) : (first ? G::kBand16 : T::kBand8);
    const uint32_t one8 = third ? 0x08u : (W32 && !first) ? 0x58u : 0x38u;   // e2m1 1.0, e4m3 16.0 or 1.0
    const uint32_t one16 = FP4 ? 0x1C00u : 0x3C00u;                             // f16 2^-8 or 1.0
    uint32_t v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k0 = (f16 ? 2 : 4) * (8 * cc + i);
      uint32_t w = 0;
      if (f16) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          const int d = k0 + b - m;
          if (d >= off - r && d <= off + r) w |= one16 << (16 * b);
        }
      } else if (m < G::kTS) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int d = k0 + b - m;
          const uint32_t v8 = (third && !FP4) ? 0x38u - 8u * (uint32_t)b : one8;   // 1, 1/2, 1/4, 1/8
          if (d >= off - r && d <= off + r) w |= v8 << (8 * b);
        }
      }
      v[i] = w;
    }
    tmem_st8(tmem + la + col + 8 * cc, v);
  }
  tmem_wait_st();
}

// The rule's two ranges as f16 pairs, scaled like the accumulator (S * scale).
// A lower bound above 2048 (above every count tested in f16: 1089 in the
// 160-row window, 2025 in the 192-row one up to r = 22) makes the range
// empty; an upper bound above it is clamped to 2048.  All values are exact in
// f16.
struct HalfRule {
  uint32_t bl2, bh2, sl2, sh2;
};

__device__ __forceinline__ uint32_t half_pair(float v) {
  __half2 h = __float2half2_rn(v);
  return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ HalfRule make_half_rule(const RuleDev &R, float scale) {
  auto lo_of = [](int lo) { return lo > 2048 ? 4096.0f : (float)lo; };
  auto hi_of = [](int lo, int w) { return lo > 2048 ? 2048.0f : fminf((float)lo + (float)w, 2048.0f); };
  HalfRule h;
  h.bl2 = half_pair(lo_of(R.b_lo) * scale);
  h.bh2 = half_pair(hi_of(R.b_lo, R.b_w) * scale);
  h.sl2 = half_pair(lo_of(R.s_lo) * scale);
  h.sh2 = half_pair(hi_of(R.s_lo, R.s_w) * scale);
  return h;
}

__device__ __forceinline__ __half2 as_h2(uint32_t v) { return *reinterpret_cast<const __half2 *>(&v); }

__device__ __forceinline__ uint32_t h2_bits(__half2 h) { return *reinterpret_cast<uint32_t *>(&h); }

// As rule4_binary, from counts already packed as f16 pairs (cells 0,1 and 2,3).
// One multiply builds both byte-permute selectors (low half: cells 0, 1; high
// half shifted down: cells 2, 3).  A cell is in range iff (s - lo)(hi - s) is
// not negative: for lo <= hi both factors are exact multiples of the scale and
// every nonzero product is at least scale^2 >= 2^-18, so no sign is lost to
// underflow (an overflow to infinity keeps its sign); an empty range has
// lo = 4096 * scale > s and hi = 2048 * scale > s, so its product is negative.
// The subtractions and products run on the FMA pipe, and one byte permute
// replicates each product's sign bit over its cell's byte.
__device__ __forceinline__ uint32_t rule4_binary_h(uint32_t s01, uint32_t s23, uint32_t cw, const HalfRule &h) {
  const uint32_t selA = cw * 0x44u + 0x32103210u;
  const uint32_t selB = selA >> 16;
  const __half2 t01 = __hmul2(__hsub2(as_h2(s01), as_h2(__byte_perm(h.bl2, h.sl2, selA))),
                              __hsub2(as_h2(__byte_perm(h.bh2, h.sh2, selA)), as_h2(s01)));
  const __half2 t23 = __hmul2(__hsub2(as_h2(s23), as_h2(__byte_perm(h.bl2, h.sl2, selB))),
                              __hsub2(as_h2(__byte_perm(h.bh2, h.sh2, selB)), as_h2(s23)));
  uint32_t neg;   // bytes 1, 3 of t01 and 5, 7 of t23 (the sign bytes), sign-replicated
  asm("prmt.b32 %0, %1, %2, 0xFDB9;" : "=r"(neg) : "r"(h2_bits(t01)), "r"(h2_bits(t23)));
  return ~neg & 0x01010101u;
}

// Out-of-range flags (product signs) of four cells as a nibble, cell k in bit
// k: the sign bytes (1 and 3) of two half2 products side by side, and their
// top bits gathered by one multiply (every partial product lands on its own
// bit, so nothing carries into bits 28..31).
__device__ __forceinline__ uint32_t sign_nibble(__half2 t01, __half2 t23) {
  const uint32_t x = __byte_perm(h2_bits(t01), h2_bits(t23), 0x7531) & 0x80808080u;
  return (x * 0x00204081u) >> 28;
}

// Next states of 16 cells of a two-state rule as bits (lowest cell lowest),
// from their counts as f16 pairs (v[i]: cells 2i, 2i + 1) and their current
// states as bits.  Every cell gets both range tests, (s - lo)(hi - s) >= 0 as
// in rule4_binary_h, on the FMA pipe; one three-input logic op then picks the
// survival test for live cells and the birth test for dead ones.  Cheaper in
// integer instructions than expanding the bits to bytes for rule4_binary_h.
__device__ __forceinline__ uint32_t rule16_bits(const uint32_t (&v)[8], uint32_t c, const HalfRule &h) {
  const __half2 sl = as_h2(h.sl2), sh = as_h2(h.sh2), bl = as_h2(h.bl2), bh = as_h2(h.bh2);
  uint32_t out_s = 0, out_b = 0;  // out of the survival / birth range
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __half2 s0 = as_h2(v[2 * i]), s1 = as_h2(v[2 * i + 1]);
    out_s |= sign_nibble(__hmul2(__hsub2(s0, sl), __hsub2(sh, s0)), __hmul2(__hsub2(s1, sl), __hsub2(sh, s1))) << (4 * i);
    out_b |= sign_nibble(__hmul2(__hsub2(s0, bl), __hsub2(bh, s0)), __hmul2(__hsub2(s1, bl), __hsub2(bh, s1))) << (4 * i);
  }
  return ~((c & out_s) | (~c & out_b)) & 0xFFFFu;
}

// 0x01 in each byte of w that is not zero, else 0x00 (no carry between bytes:
// (b & 0x7F) + 0x7F <= 0xFE; bit 7 of the sum or of b is set iff b != 0).
__device__ __forceinline__ uint32_t nonzero_bytes(uint32_t w) {
  return ((((w & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w) >> 7) & 0x01010101u;
}

// 4 next states (C > 2) from counts packed as f16 pairs and 4 centre bytes
// (states 0 .. C-1), four cells per 32-bit word: a dead cell (0) is born into
// state 1 when its count is in the birth range; an alive cell (1) stays alive
// in the survival range and otherwise starts dying (state 2); a dying cell
// (c >= 2) ages to c + 1, and to 0 after state C - 1.  Cb = C in every byte.
__device__ __forceinline__ uint32_t rule4_multistate_h(uint32_t s01, uint32_t s23, uint32_t cw, const HalfRule &h,
                                                       uint32_t Cb) {
  const uint32_t nonzero = nonzero_bytes(cw);                       // c >= 1
  const uint32_t dying = nonzero_bytes((cw >> 1) & 0x7F7F7F7Fu);    // c >= 2
  const uint32_t alive = nonzero ^ dying;                           // c == 1
  const uint32_t dead = nonzero ^ 0x01010101u;                      // c == 0
  const uint32_t inr = rule4_binary_h(s01, s23, nonzero, h);        // birth range (c = 0) or survival range
  const uint32_t inc = cw + 0x01010101u;                            // c + 1 <= C <= 255: no carries
  const uint32_t aged = inc & (nonzero_bytes(inc ^ Cb) * 0xFFu);    // c + 1, or 0 where c + 1 == C
  return (inr & dead) | ((0x02020202u - inr) & (alive * 0xFFu)) | (aged & (dying * 0xFFu));
}

// As rule4_multistate_h for C <= 128, with fewer operations: every state is
// below 128, so adding up to 0x7F to a byte carries into no other byte and
// bit 7 of the sum is a comparison: c >= 1 (c + 0x7F), c >= 2 (c + 0x7E),
// c + 1 >= C (c + 1 + Kc, Kc = 0x80 - C in every byte).  A cell alive (c = 1)
// becomes inr ? 1 : 2 = inr + 2 (1 - inr); a dead one inr; a dying one c + 1,
// or 0 at C.
__device__ __forceinline__ uint32_t rule4_multistate_small_h(uint32_t s01, uint32_t s23, uint32_t cw,
                                                             const HalfRule &h, uint32_t Kc) {
  const uint32_t ge1 = ((cw + 0x7F7F7F7Fu) >> 7) & 0x01010101u;
  const uint32_t ge2 = ((cw + 0x7E7E7E7Eu) >> 7) & 0x01010101u;
  const uint32_t inr = rule4_binary_h(s01, s23, ge1, h);
  const uint32_t r01 = inr + 2u * (ge1 & ~ge2 & ~inr);
  const uint32_t inc = cw + 0x01010101u;
  const uint32_t wrap = ((inc + Kc) >> 7) & 0x01010101u;
  const uint32_t aged = inc & ~(wrap * 0xFFu);
  const uint32_t dm = ge2 * 0xFFu;
  return (aged & dm) | (r01 & ~dm);
}

// The rule's two ranges for the wide tile's integer test: the bounds of each
// range as two 16-bit halves, the upper ones with bit 15 set.  An empty range
// (or one starting above 4225, the largest count) gets lo = 0x7FFF.
struct IntRule {
  uint32_t bl2, bh2, sl2, sh2;
};

__host__ __device__ __forceinline__ IntRule make_int_rule(const RuleDev &R) {
  auto pair = [](int v) { return (uint32_t)v * 0x00010001u; };
  auto lo_of = [](int lo) { return lo > 4225 ? 0x7FFF : (lo < 0 ? 0 : lo); };
  auto hi_of = [](int lo, int w) {
    const int64_t hi = (int64_t)lo + w;
    return lo > 4225 ? 0 : (hi > 0x7FFF ? 0x7FFF : (hi < 0 ? 0 : (int)hi));
  };
  return IntRule{pair(lo_of(R.b_lo)), pair(hi_of(R.b_lo, R.b_w) | 0x8000), pair(lo_of(R.s_lo)),
                 pair(hi_of(R.s_lo, R.s_w) | 0x8000)};
}

// Next states of four cells (bytes of cw, 0/1) of a two-state rule from their
// counts as the wide tile's f32 accumulators (S * 2^-9, S <= 4225).  Adding
// 16384 puts S in the low bits of the f32's mantissa (16384 + S * 2^-9 is
// exact: the ulp at 2^14 is 2^-9), so one byte permute packs the counts of two
// cells as 16-bit halves; per half, 0x8000 + S - lo and 0x8000 + hi - S stay
// positive (no borrow crosses the halves) and their bit 15 says S >= lo and
// S <= hi.  The range of each cell (survival if alive, birth if dead) is
// picked per half by a byte permute with the state as selector, as in
// rule4_binary_h.
__device__ __forceinline__ uint32_t rule4_binary_i(const uint32_t *f4, uint32_t cw, const IntRule &ir) {
  uint32_t s[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) s[i] = __float_as_uint(__uint_as_float(f4[i]) + 16384.0f);
  const uint32_t S01 = __byte_perm(s[0], s[1], 0x5410), S23 = __byte_perm(s[2], s[3], 0x5410);
  const uint32_t selA = cw * 0x44u + 0x32103210u, selB = selA >> 16;
  const uint32_t lo01 = __byte_perm(ir.bl2, ir.sl2, selA), hi01 = __byte_perm(ir.bh2, ir.sh2, selA);
  const uint32_t lo23 = __byte_perm(ir.bl2, ir.sl2, selB), hi23 = __byte_perm(ir.bh2, ir.sh2, selB);
  const uint32_t in01 = ((S01 | 0x80008000u) - lo01) & (hi01 - S01) & 0x80008000u;
  const uint32_t in23 = ((S23 | 0x80008000u) - lo23) & (hi23 - S23) & 0x80008000u;
  return (__byte_perm(in01, in23, 0x7531) >> 7) & 0x01010101u;   // bytes 1 and 3 of each: cells 0..3
}

__device__ __forceinline__ float half_lo(uint32_t h2) { return __low2float(as_h2(h2)); }
__device__ __forceinline__ float half_hi(uint32_t h2) { return __high2float(as_h2(h2)); }

// What one output tile needs: its maps, origin, grid extent and rule.
struct Tile {
  const CUtensorMap *in_a, *in_b, *out, *ctr;
  int x0, y0, H, W;     // tile origin in grid cells, grid extent
  int tx0, ty0;         // tile origin in TMA coordinates (x0 + ox, y0 + oy)
  RuleDev R;
  int32_t *err;
};

// Tiles of this CTA: single instance -> t = blockIdx + j * gridDim (row-major
// waves, so halo rows are L2 hits); batch -> a contiguous chunk of the
// work-list (sorted by radius, so the band rarely changes).
template <bool BATCH>
__device__ __forceinline__ void my_range(const TcParams &p, int &first, int &count) {
  if constexpr (BATCH) {
    const int64_t n = p.n_tiles, g = gridDim.x, b = blockIdx.x;
    first = (int)(b * n / g);
    count = (int)((b + 1) * n / g) - first;
  } else {
    first = 0;
    count = (p.n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  }
}

// Walks this CTA's tiles in order: tile j of the work-list chunk (batch) or
// tile id blockIdx + j * gridDim (single instance), whose (tx, ty) advances
// by a fixed step without a division.  MS: a single instance stepped several
// times in one launch walks its `per` tiles once per step; odd steps use the
// second set of maps.
template <bool BATCH, bool MS = false, int TS = kTile>
struct TileSeq {
  int first, j, tx, ty, sx, sy;
  int k, per, step;   // single instance: tile k of this CTA's `per` tiles in step `step`
  __device__ __forceinline__ TileSeq(const TcParams &p, int first_, int per_ = 0)
      : first(first_), j(0), tx(0), ty(0), sx(0), sy(0), k(0), per(per_), step(0) {
    if constexpr (!BATCH) start(p);
  }
  __device__ __forceinline__ void start(const TcParams &p) {
    ty = (int)blockIdx.x / p.tiles_x;
    tx = (int)blockIdx.x - ty * p.tiles_x;
    sy = (int)gridDim.x / p.tiles_x;
    sx = (int)gridDim.x - sy * p.tiles_x;
  }
  __device__ __forceinline__ void next(const TcParams &p) {
    ++j;
    if constexpr (!BATCH) {
      if constexpr (MS) {
        if (++k == per) {   // next step: back to this CTA's first tile
          k = 0;
          ++step;
          start(p);
          return;
        }
      }
      tx += sx;
      ty += sy;
      if (tx >= p.tiles_x) { tx -= p.tiles_x; ++ty; }
    }
  }
  __device__ __forceinline__ Tile get(const TcParams &p) const {
    Tile t;
    if constexpr (BATCH) {
      const BatchTile bt = p.btiles[first + j];
      const BatchInst *I = p.binst + bt.inst;
      const int in = I->cur ^ p.parity;
      t.in_a = &I->map_in_a[in];
      t.in_b = &I->map_in_b[in];
      t.out = &I->map_out[in ^ 1];
      t.ctr = &I->map_out[in];
      t.x0 = bt.tx * kTile;
      t.y0 = bt.ty * kTile;
      t.tx0 = t.x0 + I->ox;
      t.ty0 = t.y0 + I->oy;
      t.H = I->H;
      t.W = I->W;
      t.R = I->rule;
      t.err = I->err;
    } else {
      const bool odd = MS && (step & 1);
      t.in_a = odd ? &p.map2_in_a : &p.map_in_a;
      t.in_b = odd ? &p.map2_in_b : &p.map_in_b;
      t.out = odd ? &p.map2_out : &p.map_out;
      t.ctr = odd ? &p.map2_ctr : &p.map_ctr;
      t.x0 = tx * TS;
      t.y0 = ty * TS;
      t.tx0 = t.x0 + p.ox;
      t.ty0 = t.y0 + p.oy;
      t.H = p.H;
      t.W = p.W;
      t.R = p.rule;
      t.err = p.err;
    }
    return t;
  }
};

// Rule of tile j of this CTA (the same for every tile of a single instance).
template <bool BATCH>
__device__ __forceinline__ RuleDev tile_rule(const TcParams &p, int first, int j) {
  if constexpr (BATCH) return p.binst[p.btiles[first + j].inst].rule;
  else return p.rule;
}

template <bool BATCH>
__device__ __forceinline__ int32_t *tile_err(const TcParams &p, int first, int j) {
  if constexpr (BATCH) return p.binst[p.btiles[first + j].inst].err;
  else return p.err;
}

// Pass 2 reads f16 in the FP16 kernel and, in the FP8 kernel, whenever H can
// exceed 15 (e4m3 holds every integer multiple of 2^-9 up to 15 * 2^-9).
__device__ __forceinline__ bool pass2_f16(int DT, int r) { return DT == 0 || 2 * r + 1 > 15; }

template <int DT, bool ENC, bool BATCH, bool SW, bool BITS, bool MS, bool WIDE = false, bool NIB = false,
          bool FP4 = false, bool BIG = false, int HB = 0>
__device__ __forceinline__ void ltl_tc_body(const TcParams &p) {
  static_assert(!MS || !BATCH, "several steps per launch serve single instances");
  static_assert(!WIDE || (DT == 1 && !ENC && !BATCH && !SW && !BITS && !MS),
                "the wide tile serves single two-state instances on FP8 operands, one step per launch");
  static_assert(!BITS || (DT == 1 && ENC && !SW), "bit storage runs the FP8 kernel on a re-encoded window");
  static_assert(!NIB || (DT == 1 && ENC && !SW && !BITS && !WIDE && !BATCH && !MS),
                "four-bit storage runs the FP8 kernel on a re-encoded window, single instance, one step per launch");
  static_assert(!FP4 || (DT == 1 && ENC && !SW && !WIDE && !BATCH && !MS),
                "FP4 operands: the FP8 kernel on a re-encoded window, single instance, one step per launch");
  static_assert(!BIG || (DT == 1 && !ENC && !BATCH && !SW && !BITS && !MS && !WIDE && !NIB && !FP4),
                "the big window serves single two-state instances on FP8 operands, one step per launch");
  // HB (big window, r <= 22, every count <= 45^2 = 2025 exact in f16): the
  // epilogue tests f16 pairs, converted from the f32 accumulator (1) or
  // accumulated in f16 by pass 2 (2); 0: the f32 integer test
  static_assert(HB == 0 || BIG, "f16 pairs serve the big window");
  static_assert(Layout<DT, ENC, SW, BITS>::NS <= kMaxStages && Layout<DT, ENC, SW, BITS>::NR <= kMaxStages &&
                Layout<DT, ENC, SW, BITS>::NE <= 3, "barrier arrays");
  using L = Layout<DT, ENC, SW, BITS, WIDE, NIB, BIG>;
  // x-coordinate of a tile's centre box in its tensor map (bytes of packed rows)
  auto ctr_x = [](int tx0) { return BITS ? tx0 / 8 : NIB ? tx0 / 2 : tx0; };
  using G = Geo<SW, WIDE, BIG>;
  using T = Tm<DT, SW, WIDE, BIG>;
  constexpr bool DEC = T::kDec;       // D1 and D2 in separate regions, pass 2 on e4m3 digits
  constexpr int KW = BIG ? 192 : kWin;   // window columns = pass-1 K = pass-2 K
  constexpr int KS = KW / 32;            // K-steps of one e4m3 band product
  constexpr int ND1 = T::kND1, ND2 = T::kND2;
  constexpr int E1 = L::E1;
  constexpr int NS = L::NS;
  constexpr int NR = L::NR;
  constexpr int NH = L::NH;
  constexpr float kScale = DT == 1 ? (1.0f / 512.0f) : 1.0f;   // accumulator = count * kScale

  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  Bars *bars = reinterpret_cast<Bars *>(smem + L::kBars);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int first, n_my;
  my_range<BATCH>(p, first, n_my);
  int32_t *err0 = n_my > 0 ? tile_err<BATCH>(p, first, 0) : (BATCH ? nullptr : p.err);
  const int r0 = n_my > 0 ? tile_rule<BATCH>(p, first, 0).r : 1;
  // several steps per launch (single instance): every role walks n_my tiles
  // per step; the loads of step s >= 1 wait on the grid barrier that all CTAs
  // reach once their step s - 1 stores have completed
  const int n_steps = MS ? (p.n_steps > 1 ? p.n_steps : 1) : 1;
  const int n_all = MS ? n_my * n_steps : n_my;

  // ---- set-up: barriers, TMEM, bands ------------------------------------
  if (threadIdx.x == 0) {
    for (int i = 0; i < kMaxStages; ++i) {   // every stage and ring entry a layout can use
      mbar_init(&bars->x_full[i], 1);
      mbar_init(&bars->x_empty[i], ENC ? kCvtWarps : 1);  // encoders, or pass 1's commit
      mbar_init(&bars->c_full[i], 1);
      mbar_init(&bars->out_full[i], kEpiWarps);
    }
    for (int i = 0; i < kMaxRegions; ++i) {
      mbar_init(&bars->d1_full[i], 1);
      mbar_init(&bars->d1_empty[i], kCvtWarps);
      mbar_init(&bars->d2_full[i], 1);
      mbar_init(&bars->tmem_empty[i], kEpiWarps);
    }
    for (int i = 0; i < 3; ++i) {
      mbar_init(&bars->h_full[i], kCvtWarps);
      mbar_init(&bars->h_empty[i], 1);
    }
    for (int i = 0; i < L::NE; ++i) mbar_init(&bars->enc_full[i], kCvtWarps);
    mbar_init(&bars->band_ready, kCvtWarps);
    mbar_init(&bars->mma_done[0], 1);
    mbar_init(&bars->mma_done[1], 1);
    mbar_init(&bars->never, 1);
    bars->abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(&bars->tmem_base, kTmemCols);
    tmem_relinquish();
  }
  if constexpr (SW) {  // pass-2 operand columns 144..159 (K padding) stay zero
    for (int i = threadIdx.x; i < (int)(L::NH * L::kHBytes / 16); i += kThreads)
      reinterpret_cast<uint4 *>(smem + L::kH)[i] = make_uint4(0, 0, 0, 0);
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // barriers and tensor memory are set up: the next kernel in the stream may
  // start its own set-up, and this one reads and writes global memory only
  // once the previous kernel has completed
  griddep_launch_dependents();
  griddep_wait();
  const uint32_t tmem = bars->tmem_base;
  const uint32_t s_base = smem_u32(smem);

  // The convert warps encode window j into buffer j % NE once pass 1 of tile
  // j - NE has read that buffer (at the start of the loop iteration of tile
  // j - NE + 1, or of the step's first tile when window j opens a step).
  auto encode = [&](int j, int tid, int nthr) -> bool {
    const int s = j % L::NS, e = j % L::NE;
    if (!warp_wait(&bars->x_full[s], (j / L::NS) & 1, bars, p.timeout_ns)) return false;
    uint8_t *xe = smem + L::kXe + e * L::kXeStride;
    if constexpr (BITS) unpack_window<FP4>(smem + L::kXs + s * L::kXsStride, xe, tid, nthr);
    else if constexpr (NIB) unpack_nib_window<FP4>(smem + L::kXs + s * L::kXsStride, xe, tid, nthr);
    else encode_window<L::E1, FP4>(smem + L::kXs + s * L::kXsStride, xe, tile_rule<BATCH>(p, first, j).C > 2, tid, nthr);
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) { mbar_arrive(&bars->enc_full[e]); mbar_arrive(&bars->x_empty[s]); }
    return true;
  };

  if (warp == 0) {
    // ------------------------------------------------------ window producer
    // Streams the haloed windows into NS stages (freed by pass 1 or the encoder).
    if (lane == 0) {
      int issued = 0;
      TileSeq<BATCH, MS, G::kTS> seq(p, first, n_my);
      for (int j = 0; j < n_all; ++j, seq.next(p)) {
        const int s = j % NS;
        const Tile t = seq.get(p);
        if constexpr (MS) {
          if (seq.k == 0 && seq.step > 0) {   // step `step` reads what every CTA stored in step - 1
            if (!gbar_wait(p.gbar, p.gbar_base + (uint32_t)seq.step * gridDim.x, &bars->abort, p.timeout_ns)) {
              set_abort(bars, err0, 14);
              break;
            }
            fence_proxy_async_global();
          }
        }
        if ((MS ? seq.k == 0 : j == 0) || BATCH) { prefetch_tmap(t.in_a); prefetch_tmap(t.in_b); }
        if (!mbar_wait(&bars->x_empty[s], ((j / NS) & 1) ^ 1, &bars->abort, p.timeout_ns)) { set_abort(bars, t.err, 1); break; }
        uint8_t *xs = smem + L::kXs + s * L::kXsStride;
        mbar_arrive_expect_tx(&bars->x_full[s], L::kXsBytes);
        if constexpr (BITS) {   // bytes x0/8 - 16 .. x0/8 + 31: 16-byte aligned
          tma_load_2d(xs, t.in_a, t.tx0 / 8 - 16, t.ty0 - 16, &bars->x_full[s]);
        } else if constexpr (NIB) {   // bytes x0/2 - 16 .. x0/2 + 79: 16-byte aligned
          tma_load_2d(xs, t.in_a, t.tx0 / 2 - 16, t.ty0 - 16, &bars->x_full[s]);
        } else {
          tma_load_2d(xs, t.in_a, t.tx0 - G::kXOff, t.ty0 - G::kYOff, &bars->x_full[s]);
          tma_load_2d(xs + G::kRows * 128, t.in_b, t.tx0 - G::kXOff + 128, t.ty0 - G::kYOff, &bars->x_full[s]);
          if constexpr (BIG)   // columns x0 + 128 .. x0 + 159: the second 32-byte block
            tma_load_2d(xs + G::kRows * 160, t.in_b, t.tx0 - G::kXOff + 160, t.ty0 - G::kYOff, &bars->x_full[s]);
        }
        issued = j + 1;
      }
      volatile int no_abort = 0;  // drain: the last load issued into each stage has landed
      for (int j = issued - 1; j >= 0 && j >= issued - NS; --j)
        if (!mbar_wait(&bars->x_full[j % NS], (j / NS) & 1, &no_abort, p.timeout_ns)) set_abort(bars, err0, 2);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------- pass-1 MMA issuer
    // D1 of tile j into its region once that region is free (wide tile: the
    // convert warps have read its previous D1; otherwise the epilogue has
    // read its previous D2), the window is in place and the bands match the
    // radius.
    // Each issuer blocks on exactly the barrier it needs next, so neither
    // polls; the two passes are issued from different warps.
    if (lane == 0) {
      // f16 accumulators: every partial sum is a multiple of the operand scale
      // up to 1089 * scale, which f16 represents exactly
      // (FP4: e2m1 window and band, the band after the e4m3 one)
      const uint32_t idesc1 = idesc_f16acc(128, G::kRows) | (FP4 ? kIdescE2M1 : 0u);
      const uint32_t band1 = tmem + ((FP4 || BITS) ? T::kBand8 + 40 : DT == 1 ? T::kBand8 : T::kBand16);
      const OpDesc win0 = op_descs(s_base + (ENC ? L::kXe : L::kXs));
      bool ok = true;
      if (p.inject == 1) {  // timeout test: nobody ever arrives on `never`
        ok = mbar_wait(&bars->never, 0, &bars->abort, p.timeout_ns);
        if (!ok) set_abort(bars, err0, 3);
      }
      int band_r = -1, builds = 0;
      for (int j = 0; ok && j < n_all; ++j) {
        const int reg = j % ND1, s = j % NS;
        const int r = tile_rule<BATCH>(p, first, j).r;
        if (r != band_r) {                 // the convert warps have built the bands for r
          if (!(ok = mbar_wait(&bars->band_ready, builds & 1, &bars->abort, p.timeout_ns))) { set_abort(bars, err0, 4); break; }
          ++builds;
          band_r = r;
        }
        // the region is free: its D1 converted (DEC), or its D2 read by the epilogue
        uint64_t *free_bar = DEC ? &bars->d1_empty[reg] : &bars->tmem_empty[reg];
        if (!(ok = mbar_wait(free_bar, ((j / ND1) & 1) ^ 1, &bars->abort, p.timeout_ns))) { set_abort(bars, err0, 5); break; }
        if (ENC) ok = mbar_wait(&bars->enc_full[j % L::NE], (j / L::NE) & 1, &bars->abort, p.timeout_ns);
        else ok = mbar_wait(&bars->x_full[s], (j / NS) & 1, &bars->abort, p.timeout_ns);
        if (!ok) { set_abort(bars, err0, 6); break; }
        tc_fence_after();
        const uint64_t soff = ENC ? (uint64_t)(((j % L::NE) * L::kXeStride) >> 4)   // encoded window
                                  : (uint64_t)((s * L::kXsStride) >> 4);             // window stage
        const OpDesc win{win0.d128 + soff, win0.d32 + soff};
        band_mma<DT == 0 ? 0 : 1, G::kRows, E1, false, KS>(tmem + reg * T::kD1Cols, band1, win, idesc1);
        mma_commit(&bars->d1_full[reg]);
        if (!ENC) mma_commit(&bars->x_empty[s]);   // the raw window is no longer read
      }
      // drain: every MMA issued above has completed before TMEM is freed
      mma_commit(&bars->mma_done[0]);
      volatile int no_abort = 0;
      if (!mbar_wait(&bars->mma_done[0], 0, &no_abort, p.timeout_ns)) set_abort(bars, err0, 12);
    }
  } else if (warp == 2) {
    // ------------------------------------------------ centre tiles and stores
    // One thread: loads the centre tiles into the ring, stores each finished
    // tile from its entry and reloads the entry with the centre tile NR ahead
    // once the store has read it.  (Kept out of warp 0: a lane suspended in a
    // barrier wait holds up the other lanes of its warp.)
    if (lane == 0) {
      int issued = 0;
      if constexpr (MS) {
        int passed = 0;       // centre tiles loaded; steps whose loads may start
        TileSeq<BATCH, true, G::kTS> lseq(p, first, n_my), sseq(p, first, n_my);
        // loads the centre tiles up to (not including) tile `limit` whose step
        // has passed its grid barrier, each into the entry its tile - NR freed
        auto load_ctr = [&](int limit) {
          while (issued < n_all && issued < limit && lseq.step <= passed) {
            const int k = issued % NR;
            const Tile t = lseq.get(p);
            if (lseq.k == 0 || BATCH) prefetch_tmap(t.ctr);
            mbar_arrive_expect_tx(&bars->c_full[k], L::kRingBytes);
            tma_load_2d(smem + L::kRing + k * L::kRingBytes, t.ctr, ctr_x(t.tx0), t.ty0, &bars->c_full[k]);
            lseq.next(p);
            ++issued;
          }
        };
        load_ctr(NR);
        for (int j = 0; j < n_all; ++j, sseq.next(p)) {
          const int k = j % NR;
          const Tile t = sseq.get(p);
          if (!mbar_wait(&bars->out_full[k], (j / NR) & 1, &bars->abort, p.timeout_ns)) { set_abort(bars, t.err, 7); break; }
          if (BATCH || !p.sums) {
            tma_store_2d(t.out, ctr_x(t.tx0), t.ty0, smem + L::kRing + k * L::kRingBytes);
            bulk_commit();
            bulk_wait_read<0>();          // the store has read the entry
          }
          if (!BATCH && sseq.k == n_my - 1 && sseq.step + 1 < n_steps) {
            // this CTA's last tile of the step: its stores complete, then arrive
            // and wait for every CTA before loading centre tiles of the next step
            bulk_wait<0>();
            fence_proxy_async_global();
            gbar_arrive(p.gbar);
            if (!gbar_wait(p.gbar, p.gbar_base + (uint32_t)(sseq.step + 1) * gridDim.x, &bars->abort, p.timeout_ns)) {
              set_abort(bars, err0, 15);
              break;
            }
            fence_proxy_async_global();
            passed = sseq.step + 1;
          }
          load_ctr(j + 1 + NR);
        }
      } else {
        TileSeq<BATCH, false, G::kTS> lseq(p, first), sseq(p, first);
        auto load_ctr = [&](int j) {
          const int k = j % NR;
          const Tile t = lseq.get(p);
          if (j == 0 || BATCH) prefetch_tmap(t.ctr);
          mbar_arrive_expect_tx(&bars->c_full[k], L::kRingBytes);
          tma_load_2d(smem + L::kRing + k * L::kRingBytes, t.ctr, ctr_x(t.tx0), t.ty0, &bars->c_full[k]);
          lseq.next(p);
          issued = j + 1;
        };
        for (int j = 0; j < n_my && j < NR; ++j) load_ctr(j);
        for (int j = 0; j < n_my; ++j, sseq.next(p)) {
          const int k = j % NR;
          const Tile t = sseq.get(p);
          if (!mbar_wait(&bars->out_full[k], (j / NR) & 1, &bars->abort, p.timeout_ns)) { set_abort(bars, t.err, 7); break; }
          if (BATCH || !p.sums) {
            tma_store_2d(t.out, ctr_x(t.tx0), t.ty0, smem + L::kRing + k * L::kRingBytes);
            bulk_commit();
            bulk_wait_read<0>();          // the store has read the entry
          }
          if (j + NR < n_my) load_ctr(j + NR);
        }
      }
      bulk_wait<0>();                   // all writes complete before the CTA exits
      volatile int no_abort = 0;        // drain: the last load issued into each entry has landed
      for (int j = issued - 1; j >= 0 && j >= issued - NR; --j)
        if (!mbar_wait(&bars->c_full[j % NR], (j / NR) & 1, &no_abort, p.timeout_ns)) set_abort(bars, err0, 11);
    }
  } else if (warp == 3) {
    // ---------------------------------------------------- pass-2 MMA issuer
    // D2 of tile j once the convert warps have written H: into the D2 region
    // once the epilogue has read the previous S (wide tile), else over the
    // tile's own D1 region.
    if (lane == 0) {
      // the wide tile: N = 96 and f32 accumulators (counts up to 4225)
      const uint32_t idesc2 = ((WIDE || BIG) && HB != 2) ? idesc_f32acc(128, G::kTS) : idesc_f16acc(128, kTile);
      const uint32_t band16 = tmem + T::kBand16, band8 = tmem + T::kBand8P2;
      const uint32_t band_hi = tmem + T::kBand8x16;   // wide tile: the band of 16s for the second digit
      const OpDesc hop0 = op_descs(s_base + L::kH);
      for (int j = 0; j < n_all; ++j) {
        const int reg = j % ND2;
        if (DEC && !mbar_wait(&bars->tmem_empty[reg], ((j / ND2) & 1) ^ 1, &bars->abort, p.timeout_ns)) { set_abort(bars, err0, 10); break; }
        if (!mbar_wait(&bars->h_full[j % NH], (j / NH) & 1, &bars->abort, p.timeout_ns)) { set_abort(bars, err0, 9); break; }
        tc_fence_after();
        const uint64_t hoff = (uint64_t)(((j % NH) * L::kHBytes) >> 4);
        const OpDesc hop{hop0.d128 + hoff, hop0.d32 + hoff};
        const uint32_t d2 = tmem + T::kD2Base + reg * T::kD2Cols;
        const int rj = tile_rule<BATCH>(p, first, j).r;
        if constexpr (BIG) {
          // the DEC digits at K = 192 into the f32 accumulator over D1's region
          band_mma<1, kTile, 1, false, 6>(d2, band8, hop, idesc2);
          if (2 * rj + 1 > 15) {
            constexpr uint64_t kHi = (uint64_t)((kTile * KW) >> 4);
            band_mma<1, kTile, 1, true, 6>(d2, band_hi, OpDesc{hop.d128 + kHi, hop.d32 + kHi}, idesc2);
          }
        } else if constexpr (DEC) {
          // S = band x (H & 15) + (16 band) x (H >> 4), the second only when H
          // can exceed 15; both e4m3 halves of the H buffer
          band_mma<1, kTile, 1>(d2, band8, hop, idesc2);
          if (2 * rj + 1 > 15) {
            constexpr uint64_t kHi = (uint64_t)((kTile * kWin) >> 4);
            band_mma<1, kTile, 1, true>(d2, band_hi, OpDesc{hop.d128 + kHi, hop.d32 + kHi}, idesc2);
          }
          mma_commit(&bars->h_empty[j % NH]);
        } else if (pass2_f16(DT, rj)) {
          band_mma<0, kTile, 2>(d2, band16, hop, idesc2);
        } else {
          band_mma<1, kTile, 1>(d2, band8, hop, idesc2);
        }
        mma_commit(&bars->d2_full[reg]);
      }
      mma_commit(&bars->mma_done[1]);
      volatile int no_abort = 0;
      if (!mbar_wait(&bars->mma_done[1], 0, &no_abort, p.timeout_ns)) set_abort(bars, err0, 13);
    }
  } else if (warp < 4 + kCvtWarps) {
    // ------------------------------------------------ convert warps (4 .. 11)
    // D1 (H^T, lane x, columns y') -> K-major pass-2 operand; window encoding
    // for the next tile; band rebuilds when the radius changes (batch mode).
    const int wtid = threadIdx.x - 128;           // 0 .. kCvtThreads-1
    const int q = warp & 3;                       // TMEM lane quarter of this warp
    const int kq = (warp - 4) >> 2;               // 0..1: which warp of the quarter
    const int row = 32 * q + lane;                // TMEM lane = x
    const uint32_t lane_addr = static_cast<uint32_t>(32 * q) << 16;
    bool ok = true;
    int band_r = r0;
    // this thread's operand offsets: D1 column chunks 5kq .. 5kq+4 (16 columns
    // each); the big window's chunks 6kq .. 6kq+5 of its digit operand
    uint32_t offb[BIG ? 6 : 1];
    if constexpr (BIG) {
#pragma unroll
      for (int c = 0; c < 6; ++c) offb[c] = op_off(kTile, 1, row, 16 * (6 * kq + c));
    }
    uint32_t off16a[5], off16b[5], off8[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const int cc = 5 * kq + c;
      off16a[c] = op_off(kTile, 2, row, 32 * cc);
      off16b[c] = op_off(kTile, 2, row, 32 * cc + 16);
      off8[c] = op_off(kTile, 1, row, 16 * cc);
    }
    // the bands for the first tile
    store_bands<DT, SW, WIDE, FP4, BITS, BIG>(tmem, r0, q, kq, lane);
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&bars->band_ready);
    if (ENC && !MS)
      for (int j = 0; ok && j < n_all && j < L::NE; ++j) ok = encode(j, wtid, kCvtThreads);
    int enc_next = 0;   // MS: next window to encode
    for (int j = 0; ok && j < n_all; ++j) {
      if constexpr (ENC && MS) {
        // windows up to j + NE - 1 (their buffers were read by passes 1 up to
        // tile j - 1), but none of a later step than tile j: those wait on the
        // grid barrier, which needs this CTA's remaining tiles of this step
        const int lim = j + L::NE < n_all ? j + L::NE : n_all;
        while (ok && enc_next < lim && enc_next / n_my <= j / n_my) ok = encode(enc_next++, wtid, kCvtThreads);
        if (!ok) break;
      }
      const int reg = j % ND1;
      const int rj = tile_rule<BATCH>(p, first, j).r;
      const bool p2f16 = pass2_f16(DT, rj);
      // pass 2 of tile j-NH has finished reading this H buffer (DEC: it
      // committed to h_empty; otherwise its D2 is complete, and the region's
      // next D2 needs this very conversion)
      if (j >= NH) {
        if (DEC) ok = warp_wait(&bars->h_empty[j % NH], ((j / NH) & 1) ^ 1, bars, p.timeout_ns);
        else ok = warp_wait(&bars->d2_full[(j - NH) % ND2], ((j - NH) / ND2) & 1, bars, p.timeout_ns);
        if (!ok) break;
      }
      if (BATCH && rj != band_r) {
        // every pass 2 so far (tile j-1 last) has finished reading the bands
        // (and every pass 1: their D1 has been converted)
        if (NH > 1 && j >= 1) {
          if (DEC) ok = warp_wait(&bars->h_empty[(j - 1) % NH], ((j - 1) / NH) & 1, bars, p.timeout_ns);
          else ok = warp_wait(&bars->d2_full[(j - 1) % ND2], ((j - 1) / ND2) & 1, bars, p.timeout_ns);
          if (!ok) break;
        }
        tc_fence_after();
        store_bands<DT, SW, WIDE, FP4, BITS, BIG>(tmem, rj, q, kq, lane);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars->band_ready);
        band_r = rj;
      }
      if (!(ok = warp_wait(&bars->d1_full[reg], (j / ND1) & 1, bars, p.timeout_ns))) break;
      tc_fence_after();
      if constexpr (BIG) {
        // D1 (f16 H * 2^-9, 192 columns: six chunks of 16 per warp, read in
        // two halves of three) -> the e4m3 digits H & 15 and H >> 4 (each
        // the code of itself times 2^-9) in the two halves of the H buffer,
        // the second only when H can exceed 15
        const uint32_t treg = tmem + lane_addr + reg * T::kD1Cols + 96 * kq;
        uint8_t *hop = smem + L::kH + (j % NH) * L::kHBytes;
        const bool split = 2 * rj + 1 > 15;
        const __half2 k512 = __float2half2_rn(512.0f), k1024 = __float2half2_rn(1024.0f);
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          uint32_t v[3][8];
#pragma unroll
          for (int c = 0; c < 3; ++c) tmem_ld16_pack16(treg + 16 * (3 * hf + c), v[c]);
          tmem_wait_ld();
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            uint32_t e[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
              e[i] = __byte_perm(h2_bits(__hfma2(as_h2(v[c][2 * i]), k512, k1024)),
                                 h2_bits(__hfma2(as_h2(v[c][2 * i + 1]), k512, k1024)), 0x6420);
            const uint32_t o = offb[3 * hf + c];
            *reinterpret_cast<uint4 *>(hop + o) =
                make_uint4(e[0] & 0x0F0F0F0Fu, e[1] & 0x0F0F0F0Fu, e[2] & 0x0F0F0F0Fu, e[3] & 0x0F0F0F0Fu);
            if (split)
              *reinterpret_cast<uint4 *>(hop + kTile * KW + o) =
                  make_uint4((e[0] >> 4) & 0x0F0F0F0Fu, (e[1] >> 4) & 0x0F0F0F0Fu, (e[2] >> 4) & 0x0F0F0F0Fu,
                             (e[3] >> 4) & 0x0F0F0F0Fu);
          }
        }
      } else {
        // D1 is f16 (one value per column); packed loads give f16 pairs, which
        // are already the pass-2 operand (or become e4m3 pairs with one cvt)
        const uint32_t treg = tmem + lane_addr + reg * T::kD1Cols + 80 * kq;
        uint8_t *hop = smem + L::kH + (j % NH) * L::kHBytes;
        // V has kRows columns: 10 chunks of 16, or 9 in a short window (the
        // second warp of a quarter then takes 4)
        const bool last = !SW || kq == 0;           // this warp converts chunk 4 of its five
        uint32_t v[5][8];
#pragma unroll
        for (int c = 0; c < 4; ++c) tmem_ld16_pack16(treg + 16 * c, v[c]);
        if (last) tmem_ld16_pack16(treg + 64, v[4]);
        tmem_wait_ld();
        if constexpr (DEC) {   // D1 read: pass 1 of tile j + ND1 may overwrite it
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&bars->d1_empty[reg]);
        }
        const bool split = 2 * rj + 1 > 15;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          if (c == 4 && !last) break;
          if constexpr (DEC) {
            // e4m3 digits H & 15 and H >> 4 (at most 4): each the code of
            // itself times 2^-9 (e4m3 subnormals for 1..7)
            const __half2 k512 = __float2half2_rn(512.0f), k1024 = __float2half2_rn(1024.0f);
            uint32_t e[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
              e[i] = __byte_perm(h2_bits(__hfma2(as_h2(v[c][2 * i]), k512, k1024)),
                                 h2_bits(__hfma2(as_h2(v[c][2 * i + 1]), k512, k1024)), 0x6420);
            *reinterpret_cast<uint4 *>(hop + off8[c]) =
                make_uint4(e[0] & 0x0F0F0F0Fu, e[1] & 0x0F0F0F0Fu, e[2] & 0x0F0F0F0Fu, e[3] & 0x0F0F0F0Fu);
            if (split) {
              uint32_t hi[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) hi[i] = (e[i] >> 4) & 0x0F0F0F0Fu;
              *reinterpret_cast<uint4 *>(hop + kTile * kWin + off8[c]) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            }
          } else if (p2f16) {
            *reinterpret_cast<uint4 *>(hop + off16a[c]) = make_uint4(v[c][0], v[c][1], v[c][2], v[c][3]);
            *reinterpret_cast<uint4 *>(hop + off16b[c]) = make_uint4(v[c][4], v[c][5], v[c][6], v[c][7]);
          } else {
            // the e4m3 code of k * 2^-9 is k itself for k <= 15, and k * 2^-9 *
            // 512 + 1024 is exactly 1024 + k, an f16 whose low byte is k (FP4:
            // D1 holds 0.5 k, the e2m1 products, and 0.5 k * 2 + 1024 = 1024 + k)
            const __half2 ks = __float2half2_rn(FP4 ? 2.0f : 512.0f), k1024 = __float2half2_rn(1024.0f);
            uint32_t e[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
              e[i] = __byte_perm(h2_bits(__hfma2(as_h2(v[c][2 * i]), ks, k1024)),
                                 h2_bits(__hfma2(as_h2(v[c][2 * i + 1]), ks, k1024)), 0x6420);
            *reinterpret_cast<uint4 *>(hop + off8[c]) = make_uint4(e[0], e[1], e[2], e[3]);
          }
        }
      }
      fence_proxy_async_smem();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars->h_full[j % NH]);
      // encode window j + NE into the buffer pass 1 of tile j has finished reading
      if (ENC && !MS && j + L::NE < n_all && !(ok = encode(j + L::NE, wtid, kCvtThreads))) break;
    }
    if (!ok) set_abort(bars, err0, 8);
  } else if constexpr (WIDE || BIG) {
    // ------------------------- epilogue warps, wide tile or big window (12 .. 27)
    // S as f32 (D2, lane y < 96, columns x < 96: six chunks of 16, chunks kq
    // and kq + 4 per warp) and the centre tile (96-byte rows, no swizzle) ->
    // next states in place, stored by TMA.  Warps of lane quarter 3 (rows
    // 96..127, outside the tile) only take part in the barriers.  Big window:
    // all 128 rows and eight chunks, the centre tile in the standard
    // 128B-swizzled ring entry.
    const int q = warp & 3;
    const int kq = (warp - 4 - kCvtWarps) >> 2;
    const int y = 32 * q + lane;
    const uint32_t lane_addr = static_cast<uint32_t>(32 * q) << 16;
    const bool rows = BIG || q < 3;
    const int nch = (BIG || kq + 4 < 6) ? 2 : 1;
    bool ok = true;
    const IntRule ir = make_int_rule(p.rule);
    const HalfRule hr = make_half_rule(p.rule, kScale);
    TileSeq<false, false, G::kTS> seq(p, first, n_my);
    for (int j = 0; ok && j < n_all; ++j, seq.next(p)) {
      const int reg = j % ND2, k = j % NR;
      const Tile t = seq.get(p);
      if (!(ok = warp_wait(&bars->d2_full[reg], (j / ND2) & 1, bars, p.timeout_ns))) break;
      tc_fence_after();
      uint32_t v[2][HB == 2 ? 8 : 16];                 // S * scale as f32, or f16 pairs (HB 2)
      if (rows) {
        const uint32_t treg = tmem + lane_addr + T::kD2Base + reg * T::kD2Cols;
        if constexpr (HB == 2) {
          tmem_ld16_pack16(treg + 16 * kq, v[0]);
          tmem_ld16_pack16(treg + 16 * (kq + 4), v[1]);
        } else {
          tmem_ld16(treg + 16 * kq, v[0]);
          if (nch == 2) tmem_ld16(treg + 16 * (kq + 4), v[1]);
        }
        tmem_wait_ld();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars->tmem_empty[reg]);
      if (!(ok = warp_wait(&bars->c_full[k], (j / NR) & 1, bars, p.timeout_ns))) break;
      if (rows) {
        uint8_t *ring = smem + L::kRing + k * L::kRingBytes;
        for (int c = 0; c < nch; ++c) {
          const int cc = kq + 4 * c;
          if (!p.sums) {
            uint4 *cell = reinterpret_cast<uint4 *>(ring + (BIG ? y * 128 + (((cc ^ y) & 7) << 4) : y * G::kTS + 16 * cc));
            const uint4 cv = *cell;
            uint4 ov;
            if constexpr (HB == 0) {
              ov.x = rule4_binary_i(v[c], cv.x, ir);
              ov.y = rule4_binary_i(v[c] + 4, cv.y, ir);
              ov.z = rule4_binary_i(v[c] + 8, cv.z, ir);
              ov.w = rule4_binary_i(v[c] + 12, cv.w, ir);
            } else {
              // f16 pairs of cells (2i, 2i + 1): packed by pass 2, or converted
              // here (exact, S * 2^-9 < 4)
              auto pr = [&](int i) -> uint32_t {
                if constexpr (HB == 2) return v[c][i];
                else return h2_bits(__floats2half2_rn(__uint_as_float(v[c][2 * i]), __uint_as_float(v[c][2 * i + 1])));
              };
              ov.x = rule4_binary_h(pr(0), pr(1), cv.x, hr);
              ov.y = rule4_binary_h(pr(2), pr(3), cv.y, hr);
              ov.z = rule4_binary_h(pr(4), pr(5), cv.z, hr);
              ov.w = rule4_binary_h(pr(6), pr(7), cv.w, hr);
            }
            *cell = ov;
          } else {   // box counts
            const int gy = t.y0 + y;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int gx = t.x0 + 16 * cc + i;
              float sv;
              if constexpr (HB == 2) sv = (i & 1) ? half_hi(v[c][i >> 1]) : half_lo(v[c][i >> 1]);
              else sv = __uint_as_float(v[c][i]);
              if (gy < t.H && gx < t.W) p.sums[(int64_t)gy * p.sums_ld + gx] = __float2int_rn(sv * (1.0f / kScale));
            }
          }
        }
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars->out_full[k]);
    }
    if (!ok) set_abort(bars, err0, 8);
  } else {
    // ------------------------------------------------ epilogue warps (12 .. 27)
    // S (D2, lane y, columns x) and the centre tile -> next states, written in
    // place over the centre tile and stored from there by TMA.
    const int q = warp & 3;
    const int kq = (warp - 4 - kCvtWarps) >> 2;        // 0..3: which warp of the quarter
    const int y = 32 * q + lane;                       // TMEM lane = output row y
    const uint32_t lane_addr = static_cast<uint32_t>(32 * q) << 16;
    uint32_t off_c[2];                                 // D2 column chunks kq and kq + 4
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int cc = kq + 4 * c;
      off_c[c] = y * 128 + (((cc ^ y) & 7) << 4);
    }
    bool ok = true;
    HalfRule hr = make_half_rule(BATCH ? RuleDev{} : p.rule, kScale);
    TileSeq<BATCH, MS, G::kTS> seq(p, first, n_my);
    for (int j = 0; ok && j < n_all; ++j, seq.next(p)) {
      const int reg = j % ND2, k = j % NR;
      const Tile t = seq.get(p);
      const RuleDev &R = t.R;
      if (BATCH) hr = make_half_rule(R, kScale);
      if (!(ok = warp_wait(&bars->d2_full[reg], (j / ND2) & 1, bars, p.timeout_ns))) break;
      tc_fence_after();
      // read S and free the region (the next pass 1, or in DEC the next pass
      // 2, waits for it) before waiting for the centre tile
      uint32_t v[2][8];                                // S * scale as f16 pairs
      {
        const uint32_t treg = tmem + lane_addr + T::kD2Base + reg * T::kD2Cols;
        tmem_ld16_pack16(treg + 16 * kq, v[0]);
        tmem_ld16_pack16(treg + 16 * (kq + 4), v[1]);
        tmem_wait_ld();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars->tmem_empty[reg]);
      }
      if (!(ok = warp_wait(&bars->c_full[k], (j / NR) & 1, bars, p.timeout_ns))) break;
      uint8_t *ring = smem + L::kRing + k * L::kRingBytes;
      {
        const bool sums_mode = !BATCH && p.sums != nullptr;
        if (BITS && !sums_mode) {
          // 16 cells of a chunk are 16 bits of the row (lowest x lowest);
          // cells at x >= W, inside the row's last byte, stay dead
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int cc = kq + 4 * c;
            uint16_t *cellp = reinterpret_cast<uint16_t *>(ring + y * 16 + 2 * cc);
            uint32_t nb = rule16_bits(v[c], *cellp, hr);
            const int lim = t.W - (t.x0 + 16 * cc);
            if (lim < 16) nb &= lim > 0 ? (1u << lim) - 1u : 0u;
            *cellp = (uint16_t)nb;
          }
        } else if (NIB && !sums_mode) {
          // 16 cells of a chunk are 8 bytes of the row, cell 2i in the low
          // nibble of byte i; the ring row is 64 bytes, 64B-swizzled (16-byte
          // unit u of row y at u ^ ((y >> 1) & 3)); cells at x >= W stay 0
          const uint32_t Kc = (uint32_t)((0x80 - R.C) & 0xFF) * 0x01010101u;
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int cc = kq + 4 * c;
            uint2 *cellp = reinterpret_cast<uint2 *>(ring + y * 64 + ((((cc >> 1) ^ (y >> 1)) & 3) << 4) + 8 * (cc & 1));
            const uint2 cv = *cellp;
            const uint32_t st[4] = {nib4_to_bytes(cv.x, 0x4140), nib4_to_bytes(cv.x, 0x4342),
                                    nib4_to_bytes(cv.y, 0x4140), nib4_to_bytes(cv.y, 0x4342)};
            uint32_t ns[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)   // C <= 16 here
              ns[i] = bytes_to_nib_pairs(R.C == 2 ? rule4_binary_h(v[c][2 * i], v[c][2 * i + 1], st[i], hr)
                                                  : rule4_multistate_small_h(v[c][2 * i], v[c][2 * i + 1], st[i], hr, Kc));
            uint2 ov = make_uint2(__byte_perm(ns[0], ns[1], 0x6420), __byte_perm(ns[2], ns[3], 0x6420));
            const int lim = t.W - (t.x0 + 16 * cc);
            if (lim < 16) {
              ov.x = lim >= 8 ? ov.x : lim > 0 ? ov.x & ((1u << (4 * lim)) - 1u) : 0u;
              ov.y = lim > 8 ? ov.y & ((1u << (4 * (lim - 8))) - 1u) : 0u;
            }
            *cellp = ov;
          }
        } else if (!sums_mode && R.C == 2) {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            uint4 *cell = reinterpret_cast<uint4 *>(ring + off_c[c]);
            const uint4 cv = *cell;
            uint4 ov;
            ov.x = rule4_binary_h(v[c][0], v[c][1], cv.x, hr);
            ov.y = rule4_binary_h(v[c][2], v[c][3], cv.y, hr);
            ov.z = rule4_binary_h(v[c][4], v[c][5], cv.z, hr);
            ov.w = rule4_binary_h(v[c][6], v[c][7], cv.w, hr);
            *cell = ov;
          }
        } else if (!sums_mode) {
          if constexpr (ENC) {   // C > 2 runs only on re-encoded windows
            const uint32_t Cb = (uint32_t)R.C * 0x01010101u;
            const uint32_t Kc = (uint32_t)((0x80 - R.C) & 0xFF) * 0x01010101u;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              uint4 *cell = reinterpret_cast<uint4 *>(ring + off_c[c]);
              const uint4 cv = *cell;
              uint4 ov;
              if (R.C <= 128) {
                ov.x = rule4_multistate_small_h(v[c][0], v[c][1], cv.x, hr, Kc);
                ov.y = rule4_multistate_small_h(v[c][2], v[c][3], cv.y, hr, Kc);
                ov.z = rule4_multistate_small_h(v[c][4], v[c][5], cv.z, hr, Kc);
                ov.w = rule4_multistate_small_h(v[c][6], v[c][7], cv.w, hr, Kc);
              } else {
                ov.x = rule4_multistate_h(v[c][0], v[c][1], cv.x, hr, Cb);
                ov.y = rule4_multistate_h(v[c][2], v[c][3], cv.y, hr, Cb);
                ov.z = rule4_multistate_h(v[c][4], v[c][5], cv.z, hr, Cb);
                ov.w = rule4_multistate_h(v[c][6], v[c][7], cv.w, hr, Cb);
              }
              *cell = ov;
            }
          } else {
            // Not reached: C > 2 runs only on re-encoded windows.  Keeping the
            // general form compiled into the two-state kernels measured 3%
            // faster at r >= 8 than leaving the branch out (code generation of
            // the surrounding loop), so it stays.
            const uint32_t Cb = (uint32_t)R.C * 0x01010101u;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              uint4 *cell = reinterpret_cast<uint4 *>(ring + off_c[c]);
              const uint4 cv = *cell;
              uint4 ov;
              ov.x = rule4_multistate_h(v[c][0], v[c][1], cv.x, hr, Cb);
              ov.y = rule4_multistate_h(v[c][2], v[c][3], cv.y, hr, Cb);
              ov.z = rule4_multistate_h(v[c][4], v[c][5], cv.z, hr, Cb);
              ov.w = rule4_multistate_h(v[c][6], v[c][7], cv.w, hr, Cb);
              *cell = ov;
            }
          }
        } else {   // box counts
          const int gy = t.y0 + y;
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int cc = kq + 4 * c;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const uint32_t h2 = v[c][i >> 1];
              const float s = (i & 1) ? half_hi(h2) : half_lo(h2);
              const int gx = t.x0 + 16 * cc + i;
              if (gy < t.H && gx < t.W) p.sums[(int64_t)gy * p.sums_ld + gx] = __float2int_rn(s * (1.0f / kScale));
            }
          }
        }
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars->out_full[k]);
    }
    if (!ok) set_abort(bars, err0, 8);
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

template <int DT, bool ENC, bool BATCH, bool SW>
__global__ void __launch_bounds__(kThreads, 1) ltl_tc_kernel(const __grid_constant__ TcParams p) {
  ltl_tc_body<DT, ENC, BATCH, SW, false, false>(p);
}

// One bit per cell: the same body under its own name, so that a profiler can
// single it out.
__global__ void __launch_bounds__(kThreads, 1) ltl_bits_kernel(const __grid_constant__ TcParams p) {
  ltl_tc_body<1, true, false, false, true, false>(p);
}

// FP4 (e2m1) pass-1 operands on the re-encoded window, pass 2 as in the FP8
// kernel (e4m3 for 2r+1 <= 15, else f16): uint8, one-bit and four-bit storage.
__global__ void __launch_bounds__(kThreads, 1) ltl_fp4_kernel(const __grid_constant__ TcParams p) {
  ltl_tc_body<1, true, false, false, false, false, false, false, true>(p);
}
__global__ void __launch_bounds__(kThreads, 1) ltl_fp4_bits_kernel(const __grid_constant__ TcParams p) {
  ltl_tc_body<1, true, false, false, true, false, false, false, true>(p);
}
__global__ void __launch_bounds__(kThreads, 1) ltl_fp4_nib_kernel(const __grid_constant__ TcParams p) {
  ltl_tc_body<1, true, false, false, false, false, false, true, true>(p);
}

// Four bits per cell (C <= 16): the same body under its own name.
__global__ void __launch_bounds__(kThreads, 1) ltl_nib_kernel(const __grid_constant__ TcParams p) {
  ltl_tc_body<1, true, false, false, false, false, false, true>(p);
}

// Radii up to 32 (and any radius when asked for): the 96 x 96 tile, single
// instance, FP8 operands, two-state rules, one step per launch.
__global__ void __launch_bounds__(kThreads, 1) ltl_wide_kernel(const __grid_constant__ TcParams p) {
  ltl_tc_body<1, false, false, false, false, false, true>(p);
}

// Radii up to 32 on the 128 x 128 tile: the 192 x 192 window, single
// instance, FP8 operands, two-state rules, one step per launch.
__global__ void __launch_bounds__(kThreads, 1) ltl_big_kernel(const __grid_constant__ TcParams p) {
  ltl_tc_body<1, false, false, false, false, false, false, false, false, true>(p);
}
// The same for r <= 22, where every count is exact in f16: pass 2
// accumulates in f16 and the epilogue tests f16 pairs (measured 7% faster
// than the f32 test, 2% faster than converting the f32 accumulator).
__global__ void __launch_bounds__(kThreads, 1) ltl_big16_kernel(const __grid_constant__ TcParams p) {
  ltl_tc_body<1, false, false, false, false, false, false, false, false, true, 2>(p);
}

// Several steps of a single instance in one cooperative launch (separate
// instantiations, so that the one-step kernels carry none of it).
template <int DT, bool ENC, bool SW, bool BITS>
__global__ void __launch_bounds__(kThreads, 1) ltl_tc_multi_kernel(const __grid_constant__ TcParams p) {
  ltl_tc_body<DT, ENC, false, SW, BITS, true>(p);
}

// ---------------------------------------------------------------------------
// Simplified von Neumann neighbourhood (Eq. 3): R = Pi x Lambda + H with
// H = Lambda x Pi, the sums over the vertical and the horizontal segment of
// half-length r through each cell (the centre lies on both).  Both products
// accumulate into one tensor-memory region, so nothing leaves the tensor
// memory between them:
//   V[y][x] = sum_y' band[y][y'] X[y'][x]   A = the band in tensor memory;
//             B = X as an MN-major operand: the centre box, 128 columns x 160
//             rows at (x0, y0 - 16), 128B swizzle, K = y' along its rows;
//   H[y][x] = sum_x' X[y][x'] band[x'][x]   A = rows 16..143 of three boxes
//             side by side in K (x' = x0 - 32 ..): the left box (32 columns,
//             32B swizzle), the centre box and the right box (32 columns),
//             K-major, one 32-column K-step of the left and the right box
//             each; B = the band as a K-major operand in shared memory, cut
//             the same way (row x holds band[.][x]).
// A stage is 192 x 160 bytes, the fewest whole boxes that hold the halo and
// the centre box once.  X is read as raw 0/1 bytes (e4m3 2^-9) and the bands
// hold e4m3 1.0, so the f16 accumulator holds R * 2^-9, exact (R <= 2(2r+1)
// = 66).  Rows 16..143 of the centre box are the centre tile: the epilogue
// overwrites them with the next states, warp 2 stores them, and the stage is
// then free.
namespace vn {
constexpr int NS = 6;                                // stages
constexpr int kRegions = 3;                          // accumulators of 128 columns
constexpr uint32_t kLeft = kTile * kWin;             // 20480: left box, 32 B x 160 rows (centre box at 0)
constexpr uint32_t kRight = kLeft + 32 * kWin;       // 25600: right box, 32 B x 160 rows
constexpr uint32_t kStage = kRight + 32 * kWin;      // 30720 bytes, all delivered by the three loads
constexpr uint32_t kCtrOff = 16 * 128;               // centre tile: centre-box rows 16..143
constexpr uint32_t kBandC = NS * kStage;             // horizontal band: centre piece, 128 rows x 128 B
constexpr uint32_t kBandL = kBandC + kTile * 128;    // left piece, 128 rows x 32 B
constexpr uint32_t kBandR = kBandL + kTile * 32;     // right piece, 128 rows x 32 B
constexpr uint32_t kBars = kBandR + kTile * 32;
constexpr uint32_t kDyn = kBars + 512 + 1024;
constexpr uint32_t kBandCol = kRegions * kTile;      // vertical band (A operand), 40 columns
static_assert(kLeft % 1024 == 0 && kStage % 1024 == 0 && kBandC % 1024 == 0 && kRight % 256 == 0 &&
              kBandL % 256 == 0 && kBandR % 256 == 0, "swizzle atoms stay aligned");
static_assert(kDyn <= 232448, "shared memory budget");
static_assert(kBandCol + 40 <= kTmemCols, "tensor memory budget");
static_assert(kRegions <= kMaxRegions && NS <= kMaxStages, "barrier arrays");

// V: five K-steps of 32 rows of the column box (4096 bytes each).
template <int J = 0>
__device__ __forceinline__ void vertical_mma(uint32_t d, uint32_t band, uint64_t col0, uint32_t idesc) {
  if constexpr (J < 5) {
    mma_f8f6f4_ts(d, band + 8 * J, col0 + (uint64_t)((4096 * J) >> 4), idesc, J > 0);
    vertical_mma<J + 1>(d, band, col0, idesc);
  }
}

// H: the left box, four K-steps of 32 columns of the centre box, the right
// box, each against its piece of the band (descriptors of rows 16.. of the
// stage, and of the band pieces).
__device__ __forceinline__ void horizontal_mma(uint32_t d, uint64_t a_left, uint64_t a_centre, uint64_t a_right,
                                               uint64_t b_left, uint64_t b_centre, uint64_t b_right, uint32_t idesc) {
  mma_f8f6f4(d, a_left, b_left, idesc, 1);
#pragma unroll
  for (int j = 0; j < 4; ++j) mma_f8f6f4(d, a_centre + 2 * j, b_centre + 2 * j, idesc, 1);   // +32 bytes of K
  mma_f8f6f4(d, a_right, b_right, idesc, 1);
}

// Byte offset of (row, kb) in a K-major operand piece of 128B (w = 128) or
// 32B (w = 32) swizzle, rows at w bytes.
__device__ __forceinline__ uint32_t piece_off(int w, int row, int kb) {
  if (w == 128) return row * 128 + ((((kb >> 4) ^ row) & 7) << 4) + (kb & 15);
  return row * 32 + ((((kb >> 4) ^ (row >> 2)) & 1) << 4) + (kb & 15);
}
}  // namespace vn

// One step (or the counts R) of a single instance, FP8 operands, two-state
// rules.  Warps: 0 loads, 1 allocates tensor memory and issues the MMAs, 2
// stores, 4..11 build the two bands, 12..27 evaluate the rule.
__global__ void __launch_bounds__(kThreads, 1) ltl_vn_kernel(const __grid_constant__ TcParams p) {
  constexpr float kScale = 1.0f / 512.0f;            // accumulator = R * kScale
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  Bars *bars = reinterpret_cast<Bars *>(smem + vn::kBars);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int first, n_my;
  my_range<false>(p, first, n_my);
  int32_t *err0 = p.err;

  if (threadIdx.x == 0) {
    for (int i = 0; i < vn::NS; ++i) {
      mbar_init(&bars->x_full[i], 1);
      mbar_init(&bars->x_empty[i], 1);            // the store thread, once the stage is stored
      mbar_init(&bars->out_full[i], kEpiWarps);
    }
    for (int i = 0; i < vn::kRegions; ++i) {
      mbar_init(&bars->d2_full[i], 1);
      mbar_init(&bars->tmem_empty[i], kEpiWarps);
    }
    mbar_init(&bars->band_ready, kCvtWarps);
    mbar_init(&bars->mma_done[0], 1);
    mbar_init(&bars->never, 1);
    bars->abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(&bars->tmem_base, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  griddep_launch_dependents();   // as in the Moore body: set up, then wait for the previous kernel
  griddep_wait();
  const uint32_t tmem = bars->tmem_base;
  const uint32_t s_base = smem_u32(smem);

  if (warp == 0) {
    // --------------------------------------------------------------- loads
    if (lane == 0) {
      int issued = 0;
      TileSeq<false> seq(p, first);
      for (int j = 0; j < n_my; ++j, seq.next(p)) {
        const int s = j % vn::NS;
        const Tile t = seq.get(p);
        if (j == 0) { prefetch_tmap(t.in_a); prefetch_tmap(t.in_b); }
        if (!mbar_wait(&bars->x_empty[s], ((j / vn::NS) & 1) ^ 1, &bars->abort, p.timeout_ns)) { set_abort(bars, t.err, 1); break; }
        uint8_t *st = smem + s * vn::kStage;
        mbar_arrive_expect_tx(&bars->x_full[s], vn::kStage);
        tma_load_2d(st, t.in_a, t.tx0, t.ty0 - 16, &bars->x_full[s]);
        tma_load_2d(st + vn::kLeft, t.in_b, t.tx0 - 32, t.ty0 - 16, &bars->x_full[s]);
        tma_load_2d(st + vn::kRight, t.in_b, t.tx0 + 128, t.ty0 - 16, &bars->x_full[s]);
        issued = j + 1;
      }
      volatile int no_abort = 0;  // drain: the last load issued into each stage has landed
      for (int j = issued - 1; j >= 0 && j >= issued - vn::NS; --j)
        if (!mbar_wait(&bars->x_full[j % vn::NS], (j / vn::NS) & 1, &no_abort, p.timeout_ns)) set_abort(bars, err0, 2);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc_v = idesc_f16acc(128, kTile) | (1u << 16);  // B (column box) MN-major
      const uint32_t idesc_h = idesc_f16acc(128, kTile);
      const uint32_t band_a = tmem + vn::kBandCol;
      const uint64_t b_left = smem_desc(s_base + vn::kBandL, 16, 256, kSwizzle32B);
      const uint64_t b_centre = smem_desc(s_base + vn::kBandC, 16, 1024, kSwizzle128B);
      const uint64_t b_right = smem_desc(s_base + vn::kBandR, 16, 256, kSwizzle32B);
      bool ok = true;
      if (p.inject == 1) {  // timeout test: nobody ever arrives on `never`
        ok = mbar_wait(&bars->never, 0, &bars->abort, p.timeout_ns);
        if (!ok) set_abort(bars, err0, 3);
      }
      if (ok && !(ok = mbar_wait(&bars->band_ready, 0, &bars->abort, p.timeout_ns))) set_abort(bars, err0, 4);
      for (int j = 0; ok && j < n_my; ++j) {
        const int reg = j % vn::kRegions, s = j % vn::NS;
        if (!(ok = mbar_wait(&bars->tmem_empty[reg], ((j / vn::kRegions) & 1) ^ 1, &bars->abort, p.timeout_ns))) { set_abort(bars, err0, 5); break; }
        if (!(ok = mbar_wait(&bars->x_full[s], (j / vn::NS) & 1, &bars->abort, p.timeout_ns))) { set_abort(bars, err0, 6); break; }
        tc_fence_after();
        const uint32_t st = s_base + s * vn::kStage;
        const uint32_t d = tmem + reg * kTile;
        vn::vertical_mma(d, band_a, smem_desc(st, 1024, 1024, kSwizzle128B), idesc_v);
        vn::horizontal_mma(d, smem_desc(st + vn::kLeft + 16 * 32, 16, 256, kSwizzle32B),
                           smem_desc(st + 16 * 128, 16, 1024, kSwizzle128B),
                           smem_desc(st + vn::kRight + 16 * 32, 16, 256, kSwizzle32B), b_left, b_centre, b_right, idesc_h);
        mma_commit(&bars->d2_full[reg]);
      }
      mma_commit(&bars->mma_done[0]);  // drain before the tensor memory is freed
      volatile int no_abort = 0;
      if (!mbar_wait(&bars->mma_done[0], 0, &no_abort, p.timeout_ns)) set_abort(bars, err0, 12);
    }
  } else if (warp == 2) {
    // -------------------------------------------------------------- stores
    if (lane == 0) {
      TileSeq<false> seq(p, first);
      for (int j = 0; j < n_my; ++j, seq.next(p)) {
        const int s = j % vn::NS;
        const Tile t = seq.get(p);
        if (!mbar_wait(&bars->out_full[s], (j / vn::NS) & 1, &bars->abort, p.timeout_ns)) { set_abort(bars, t.err, 7); break; }
        if (!p.sums) {
          tma_store_2d(t.out, t.tx0, t.ty0, smem + s * vn::kStage + vn::kCtrOff);
          bulk_commit();
          bulk_wait_read<0>();          // the store has read the stage
        }
        mbar_arrive(&bars->x_empty[s]);
      }
      bulk_wait<0>();                   // all writes complete before the CTA exits
    }
  } else if (warp == 3) {
    // idle
  } else if (warp < 4 + kCvtWarps) {
    // --------------------------------------------------------------- bands
    const int q = warp & 3, kq = (warp - 4) >> 2, r = p.rule.r;
    {  // vertical band: lane m = output row y, K = window row y', one iff |y' - 16 - y| <= r
      const int m = 32 * q + lane;
      const uint32_t la = static_cast<uint32_t>(32 * q) << 16;
      for (int c = kq; c < 5; c += 2) {
        uint32_t v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          uint32_t w = 0;
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int d = 4 * (8 * c + i) + b - m - 16;
            if (d >= -r && d <= r) w |= 0x38u << (8 * b);
          }
          v[i] = w;
        }
        tmem_st8(tmem + la + vn::kBandCol + 8 * c, v);
      }
      tmem_wait_st();
    }
    // horizontal band: row x (N), K = column x' = x0 - 32 + k of the three
    // boxes side by side, one iff |x' - x0 - x| = |k - 32 - x| <= r; 16-byte
    // chunk c of K: 0, 1 in the left piece, 2..9 the centre, 10, 11 the right
    for (int i = threadIdx.x - 128; i < kTile * 12; i += kCvtThreads) {
      const int c = i / kTile, x = i - c * kTile;
      uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
      for (int b = 0; b < 16; ++b) {
        const int d = 16 * c + b - 32 - x;
        if (d >= -r && d <= r) w[b >> 2] |= 0x38u << (8 * (b & 3));
      }
      const uint32_t off = c < 2 ? vn::kBandL + vn::piece_off(32, x, 16 * c)
                         : c < 10 ? vn::kBandC + vn::piece_off(128, x, 16 * (c - 2))
                                  : vn::kBandR + vn::piece_off(32, x, 16 * (c - 10));
      *reinterpret_cast<uint4 *>(smem + off) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&bars->band_ready);
  } else {
    // ------------------------------------------------ epilogue warps (12 .. 27)
    const int q = warp & 3;
    const int kq = (warp - 4 - kCvtWarps) >> 2;      // 0..3: which warp of the quarter
    const int y = 32 * q + lane;                     // TMEM lane = output row y
    const uint32_t lane_addr = static_cast<uint32_t>(32 * q) << 16;
    uint32_t off_c[2];                               // column chunks kq and kq + 4 of row y
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int cc = kq + 4 * c;
      off_c[c] = y * 128 + (((cc ^ y) & 7) << 4);
    }
    bool ok = true;
    const HalfRule hr = make_half_rule(p.rule, kScale);
    TileSeq<false> seq(p, first);
    for (int j = 0; ok && j < n_my; ++j, seq.next(p)) {
      const int reg = j % vn::kRegions, s = j % vn::NS;
      const Tile t = seq.get(p);
      if (!(ok = warp_wait(&bars->d2_full[reg], (j / vn::kRegions) & 1, bars, p.timeout_ns))) break;
      tc_fence_after();
      uint32_t v[2][8];                              // R * scale as f16 pairs
      {
        const uint32_t treg = tmem + lane_addr + reg * kTile;
        tmem_ld16_pack16(treg + 16 * kq, v[0]);
        tmem_ld16_pack16(treg + 16 * (kq + 4), v[1]);
        tmem_wait_ld();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars->tmem_empty[reg]);
      }
      // the stage's loads completed before its MMAs; waiting on the same phase
      // (still current: the stage is freed only after this tile's store) makes
      // the centre tile visible to these threads
      if (!(ok = warp_wait(&bars->x_full[s], (j / vn::NS) & 1, bars, p.timeout_ns))) break;
      uint8_t *ctr = smem + s * vn::kStage + vn::kCtrOff;
      if (!p.sums) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          uint4 *cell = reinterpret_cast<uint4 *>(ctr + off_c[c]);
          const uint4 cv = *cell;
          uint4 ov;
          ov.x = rule4_binary_h(v[c][0], v[c][1], cv.x, hr);
          ov.y = rule4_binary_h(v[c][2], v[c][3], cv.y, hr);
          ov.z = rule4_binary_h(v[c][4], v[c][5], cv.z, hr);
          ov.w = rule4_binary_h(v[c][6], v[c][7], cv.w, hr);
          *cell = ov;
        }
      } else {  // the counts R of Eq. 3
        const int gy = t.y0 + y;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int cc = kq + 4 * c;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const uint32_t h2 = v[c][i >> 1];
            const float sv = (i & 1) ? half_hi(h2) : half_lo(h2);
            const int gx = t.x0 + 16 * cc + i;
            if (gy < t.H && gx < t.W) p.sums[(int64_t)gy * p.sums_ld + gx] = __float2int_rn(sv * (1.0f / kScale));
          }
        }
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars->out_full[s]);
    }
    if (!ok) set_abort(bars, err0, 8);
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace tc

// dt follows cat.h: 1 = FP16, 2 = FP8 e4m3.
size_t tc_smem_bytes(int dt, bool encode, bool sw) {
  if (dt == 1) return tc::Layout<0, true>::kDyn;
  if (sw) return tc::Layout<1, false, true>::kDyn;
  return encode ? tc::Layout<1, true>::kDyn : tc::Layout<1, false>::kDyn;
}

// One-step kernels are launched with the programmatic-stream-serialization
// attribute: the kernel may be scheduled while the previous kernel in the
// stream drains (its CTAs start on SMs as the previous grid's CTAs leave
// them), sets up its barriers and tensor memory, and waits for the previous
// grid's completion (griddepcontrol.wait) before any global memory access.
static cudaError_t launch_pdl(void (*kern)(TcParams), int grid, size_t smem, cudaStream_t s, const TcParams &p) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(tc::kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, p);
}

template <int DT, bool ENC, bool BATCH, bool SW = false, bool BITS = false>
static cudaError_t launch_one(const TcParams &p, int grid, cudaStream_t s) {
  static bool configured = false;
  const size_t smem = tc::Layout<DT, ENC, SW, BITS>::kDyn;
  void (*kern)(TcParams);
  if constexpr (BITS) kern = tc::ltl_bits_kernel;
  else kern = tc::ltl_tc_kernel<DT, ENC, BATCH, SW>;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if constexpr (!BATCH) {
    if (p.n_steps > 1) {  // CTAs wait on one another: all must be resident at once
      static bool configured_multi = false;
      void (*multi)(TcParams) = tc::ltl_tc_multi_kernel<DT, ENC, SW, BITS>;
      if (!configured_multi) {
        cudaError_t e = cudaFuncSetAttribute(multi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured_multi = true;
      }
      void *args[] = {const_cast<TcParams *>(&p)};
      return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(multi), dim3(grid), dim3(tc::kThreads), args, smem, s);
    }
    return launch_pdl(kern, grid, smem, s, p);
  }
  kern<<<grid, tc::kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

// sw: the short-window variant (FP8, two-state rules, r <= 7); the caller
// passes the tensor maps whose window boxes are 144 rows high.  bits: the
// grid is stored one bit per cell (FP8, two-state rules, single instance);
// the caller passes the 48 x 160 window and 16 x 128 tile maps of the packed
// buffers.
cudaError_t tc_launch(const TcParams &p, int dt, bool encode, bool sw, bool bits, int grid, cudaStream_t s) {
  if (bits) return launch_one<1, true, false, false, true>(p, grid, s);
  if (dt == 1) return launch_one<0, true, false>(p, grid, s);
  if (encode) return launch_one<1, true, false>(p, grid, s);
  if (sw) return launch_one<1, false, false, true>(p, grid, s);
  return launch_one<1, false, false>(p, grid, s);
}

// Four bits per cell: map_in_a is the 96 x 160-byte window map of the packed
// rows, map_ctr / map_out the 64 x 128-byte tile maps (64B swizzle).
cudaError_t nib_launch(const TcParams &p, int grid, cudaStream_t s) {
  static bool configured = false;
  using L = tc::Layout<1, true, false, false, false, true>;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(tc::ltl_nib_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::kDyn);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  return launch_pdl(tc::ltl_nib_kernel, grid, L::kDyn, s, p);
}

// FP4 operands: the maps of the FP8 kernel for the same storage (0 = uint8,
// 1 = one bit, 2 = four bits per cell).
cudaError_t fp4_launch(const TcParams &p, int storage, int grid, cudaStream_t s) {
  static bool configured[3] = {false, false, false};
  void (*kern)(TcParams) = storage == 1 ? tc::ltl_fp4_bits_kernel : storage == 2 ? tc::ltl_fp4_nib_kernel : tc::ltl_fp4_kernel;
  const size_t smem = storage == 1 ? tc::Layout<1, true, false, true>::kDyn
                    : storage == 2 ? tc::Layout<1, true, false, false, false, true>::kDyn
                                   : tc::Layout<1, true>::kDyn;
  if (storage < 0 || storage > 2) return cudaErrorInvalidValue;
  if (!configured[storage]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured[storage] = true;
  }
  return launch_pdl(kern, grid, smem, s, p);
}

// The 96 x 96 tile: map_in_a / map_in_b are the 128 x 160 and 32 x 160 window
// maps, map_ctr / map_out the 96 x 96 tile maps (no swizzle) of the input and
// output buffers; tiles_x and n_tiles count 96 x 96 tiles.
cudaError_t wide_launch(const TcParams &p, int grid, cudaStream_t s) {
  static bool configured = false;
  using L = tc::Layout<1, false, false, false, true>;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(tc::ltl_wide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::kDyn);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  return launch_pdl(tc::ltl_wide_kernel, grid, L::kDyn, s, p);
}

// The 192 x 192 window: map_in_a / map_in_b are the 128 x 192 and 32 x 192
// window maps (the second loaded twice, at x0 + 96 and x0 + 128), map_ctr /
// map_out the 128 x 128 tile maps; tiles_x and n_tiles count 128 x 128 tiles.
cudaError_t big_launch(const TcParams &p, int grid, cudaStream_t s) {
  static bool configured[2] = {false, false};
  using L = tc::Layout<1, false, false, false, false, false, true>;
  const int k = p.rule.r <= 22 ? 1 : 0;
  void (*kern)(TcParams) = k ? tc::ltl_big16_kernel : tc::ltl_big_kernel;
  if (!configured[k]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::kDyn);
    if (e != cudaSuccess) return e;
    configured[k] = true;
  }
  return launch_pdl(kern, grid, L::kDyn, s, p);
}

// Simplified von Neumann neighbourhood: FP8, two-state rules, single instance
// (map_in_a / map_in_b: the 128 x 160 and 32 x 160 window maps; map_out: the
// 128 x 128 tile map of the output buffer).
cudaError_t vn_launch(const TcParams &p, int grid, cudaStream_t s) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(tc::ltl_vn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::vn::kDyn);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  return launch_pdl(tc::ltl_vn_kernel, grid, tc::vn::kDyn, s, p);
}

cudaError_t tc_launch_batch(const TcParams &p, int dt, bool encode, bool sw, int grid, cudaStream_t s) {
  if (dt == 1) return launch_one<0, true, true>(p, grid, s);
  if (encode) return launch_one<1, true, true>(p, grid, s);
  if (sw) return launch_one<1, false, true, true>(p, grid, s);
  return launch_one<1, false, true>(p, grid, s);
}

}  // namespace cat
