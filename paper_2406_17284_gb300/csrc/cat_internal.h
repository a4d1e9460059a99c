// Host/device structures shared by the C ABI (cat_api.cu) and the kernels.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/cat.h"

namespace cat {

// LTL rule reduced to range tests on the box count S (centre included).
//   state 0 : born  iff (uint32)(S - b_lo) <= b_w
//   state 1 : kept  iff (uint32)(S - s_lo) <= s_w   (s_lo = s1 + [M == 0])
//   state >= 2 : decays to state + 1 (0 when state + 1 == C)
// An empty range is encoded as lo = 1 << 24, w = 0 (no count reaches it).
struct RuleDev {
  int32_t r, C, M;
  int32_t s_lo, s_w, b_lo, b_w;
  int32_t nbhd;  // 0: Moore box; 1: simplified von Neumann cross (centre counted twice)
};

// One instance of a batched launch (global memory, read by the kernel).
// Buffer b of the instance is read through map_in_a[b] / map_in_b[b] and
// written through map_out[b]; the state of step t lives in buffer cur ^ (t & 1).
struct BatchInst {
  CUtensorMap map_in_a[2];
  CUtensorMap map_in_b[2];
  CUtensorMap map_out[2];
  RuleDev rule;
  int32_t H, W, cur, pad;
  int32_t *err;
  int32_t ox, oy, pad2[2];  // TMA coordinates of grid cell (0, 0) (the ghost-frame width)
};

// One 128 x 128 output tile of a batched launch.
struct BatchTile {
  int32_t inst;
  int16_t ty, tx;
};

// Parameters of the tcgen05 step kernel (passed as a __grid_constant__ so the
// tensor maps of a single instance live in parameter space).  In batch mode
// the tiles come from `btiles` (each CTA takes a contiguous chunk) and the
// per-instance maps and rules from `binst`; the single-instance fields are unused.
struct TcParams {
  CUtensorMap map_in_a;  // input buffer, box 128 x 160 bytes, 128B swizzle
  CUtensorMap map_in_b;  // input buffer, box  32 x 160 bytes,  32B swizzle
  CUtensorMap map_out;   // output buffer, box 128 x 128 bytes, 128B swizzle
  CUtensorMap map_ctr;   // input buffer, box 128 x 128 bytes, 128B swizzle (centre tile)
  int32_t H, W, tiles_x, n_tiles;
  int32_t ox, oy;   // TMA coordinates of grid cell (0, 0): 16 with a periodic ghost frame, else 0
  RuleDev rule;
  int32_t *err;     // device status word (0 = ok)
  int32_t *sums;    // non-null: write box counts here instead of stepping
  int64_t sums_ld;  // row stride of sums (elements)
  uint64_t timeout_ns;
  int32_t inject;   // 1: wait on a barrier nobody arrives at (timeout test)
  int32_t parity;   // batch mode: step index & 1
  const BatchInst *binst;
  const BatchTile *btiles;
  // several steps in one cooperative launch (single instance, n_steps > 1):
  // odd steps read and write through the second set of maps (buffers
  // swapped), and all CTAs meet on a grid barrier between steps
  CUtensorMap map2_in_a, map2_in_b, map2_out, map2_ctr;
  int32_t n_steps;       // steps in this launch (1 unless cooperative)
  uint32_t gbar_base;    // barrier counter value when the launch starts
  uint32_t *gbar;        // barrier counter (global memory)
};

// Parameters of the warp-level kernels (mma.sync fragments, CUDA-core stencil).
struct SimpleParams {
  const uint8_t *in;
  uint8_t *out;
  int64_t pitch;
  int32_t H, W;
  RuleDev rule;
  int32_t *sums;
  int64_t sums_ld;
};

enum : int32_t { kDevErrTimeout = 0x100 };

// tcgen05 kernel launchers (cat_tc.cu).  dt: CAT_DTYPE_FP16 or CAT_DTYPE_FP8_E4M3.
// encode: FP8 only -- stage the operand through an encoded copy of the window
// (needed when C > 2; otherwise the raw 0/1 bytes are used as e4m3 operands).
// sw: short-window variant (FP8 operands, C = 2, r <= 7): map_in_a / map_in_b
// must then be the maps with 144-row window boxes.
// bits: one bit per cell (FP8, C = 2, single instance): map_in_a is the 48 x
// 160-byte window map and map_out / map_ctr the 16 x 128-byte tile maps.
cudaError_t tc_launch(const TcParams &p, int dt, bool encode, bool sw, bool bits, int grid, cudaStream_t s);
// Simplified von Neumann neighbourhood (FP8, C = 2, single instance).
cudaError_t vn_launch(const TcParams &p, int grid, cudaStream_t s);
// The 96 x 96 tile with a 32-cell halo, radii up to 32 (FP8, C = 2, single
// instance): map_in_a / map_in_b the 128 x 160 and 32 x 160 window maps,
// map_ctr / map_out the 96 x 96 tile maps; tiles_x, n_tiles in 96 x 96 tiles.
cudaError_t wide_launch(const TcParams &p, int grid, cudaStream_t s);
// The 128 x 128 tile in a 192 x 192 window (32-cell halo), radii up to 32
// (FP8, C = 2, single instance): map_in_a / map_in_b the 128 x 192 and
// 32 x 192 window maps, map_ctr / map_out the 128 x 128 tile maps.
cudaError_t big_launch(const TcParams &p, int grid, cudaStream_t s);
// FP4 (e2m1) pass-1 operands, pass 2 as in the FP8 kernel, on the re-encoded window
// of uint8 (storage 0), one-bit (1) or four-bit (2) grids: the maps of the
// FP8 kernel for that storage.
cudaError_t fp4_launch(const TcParams &p, int storage, int grid, cudaStream_t s);
// Four bits per cell (FP8 on a re-encoded window, C <= 16, single instance):
// map_in_a the 96 x 160-byte window map, map_ctr / map_out the 64 x 128-byte
// tile maps (64B swizzle) of the packed buffers.
cudaError_t nib_launch(const TcParams &p, int grid, cudaStream_t s);
cudaError_t tc_launch_batch(const TcParams &p, int dt, bool encode, bool sw, int grid, cudaStream_t s);
size_t tc_smem_bytes(int dt, bool encode, bool sw);

// What the autotuner needs to know about an instance (cat_api.cu).
struct InstanceInfo {
  int64_t H, W;
  cat_rule_t rule;
  int32_t boundary, storage, kernel, dtype, tile, window, steps_per_launch;
};
int host_instance_info(cat_handle_t h, InstanceInfo *out);
// The autotuner's cached choice for an instance from the JSON-lines file named
// by the environment variable CAT_AUTOTUNE_CACHE (cat_tune.cu); false when
// the variable is unset or the file holds no entry for the instance.
bool tune_cache_lookup_env(const InstanceInfo &info, int32_t *kernel, int32_t *dtype, int32_t *tile,
                           int32_t *window, int32_t *spl);

// Host helpers defined in cat_api.cu (error message of the calling thread,
// rule checks, TMA descriptor encoding of a uint8 grid).
int host_fail(int code, const char *msg);
int host_validate_rule(const cat_rule_t *r);
RuleDev host_reduce_rule(const cat_rule_t &r);
int host_make_map(CUtensorMap *m, void *base, int64_t H, int64_t W, int64_t pitch, uint32_t box_x,
                  uint32_t box_y, int swizzle128);

// One bit per cell (cat_bits.cu): rows of W cells <-> rows of (W + 7) / 8
// bytes, cell x in bit x % 8 of byte x / 8; pack writes bit 1 for state 1 and
// zeros past W in each row's last byte.
cudaError_t pack_bits_launch(const uint8_t *src, int64_t spitch, uint8_t *dst, int64_t dpitch, int64_t rows,
                             int64_t W, cudaStream_t s);
cudaError_t unpack_bits_launch(const uint8_t *src, int64_t spitch, uint8_t *dst, int64_t dpitch, int64_t rows,
                               int64_t W, cudaStream_t s);
// Four bits per cell (cat_bits.cu): rows of W cells <-> rows of (W + 1) / 2
// bytes, cell x in nibble x % 2 of byte x / 2 (states 0..15; the nibble past
// an odd W is 0).
cudaError_t pack_nib_launch(const uint8_t *src, int64_t spitch, uint8_t *dst, int64_t dpitch, int64_t rows,
                            int64_t W, cudaStream_t s);
cudaError_t unpack_nib_launch(const uint8_t *src, int64_t spitch, uint8_t *dst, int64_t dpitch, int64_t rows,
                              int64_t W, cudaStream_t s);

// Periodic boundary (cat_halo.cu): fills the G-cell ghost frame around the
// H x W grid whose cell (0, 0) is at base + G * pitch + G with the cells the
// frame wraps to.
cudaError_t ghost_fill_launch(uint8_t *base, int64_t pitch, int64_t H, int64_t W, int G, cudaStream_t s);

// Paper-style fragment kernels (cat_mma.cu).  dt: FP16 or INT8.
cudaError_t mma_launch(const SimpleParams &p, int dt, cudaStream_t s);
// Shared-memory CUDA-core stencil, and the separable running-sum kernel
// (cat_stencil.cu).
cudaError_t stencil_launch(const SimpleParams &p, cudaStream_t s);
cudaError_t runsum_launch(const SimpleParams &p, cudaStream_t s);
// Bit-sliced CUDA-core step on one-bit storage, r <= 5 (cat_swar.cu): in/out
// are packed rows at `pitch` bytes (a multiple of 4); sums: counts instead.
cudaError_t swar_launch(const uint8_t *in, uint8_t *out, int64_t pitch, int64_t H, int64_t W, const RuleDev &rule,
                        int32_t *sums, int64_t sums_ld, cudaStream_t s);
// The same rule, k steps per launch on tiles held in shared memory (temporal
// blocking, a k r-cell stale halo; k r <= 8); reads `in`, writes the state
// after k steps to `out`.
cudaError_t swar_tb_launch(const uint8_t *in, uint8_t *out, int64_t pitch, int64_t H, int64_t W, const RuleDev &rule,
                           int k, cudaStream_t s);

}  // namespace cat
