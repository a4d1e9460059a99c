/*
 * cat.h -- C ABI of the GB300 (sm_103a) Larger-than-Life step library.
 *
 * The library advances 2-D cellular automata of the Larger-than-Life (LTL)
 * family, R_r C_c M_m S_{s1..s2} B_{b1..b2} N_M, by the method of
 * "CAT: Cellular Automata on Tensor cores" (Navarro et al., arXiv 2406.17284):
 * the Moore box count of every cell is computed as two products with a banded
 * 0/1 matrix (Sec. IV, Eqs. 1-2: H = Lambda x Pi, R = Pi x H), and the LTL
 * transition of Sec. V-A is applied to the count.
 *
 * Conventions shared by every entry point
 *  - Grids are H rows x W columns of uint8 cell states in [0, C), row-major,
 *    row y starting at byte y * pitch.  Cell (y, x) is byte y*pitch + x.
 *  - Only state 1 ("alive") is counted.  The count of a cell is
 *        L(y,x) = #{ (dy,dx) in [-r,r]^2 : state(y+dy, x+dx) == 1 },
 *    centre included; k = L - (M == 0 ? [state(y,x) == 1] : 0); then
 *        state 0      -> 1 if b1 <= k <= b2 else 0
 *        state 1      -> 1 if s1 <= k <= s2 else (C > 2 ? 2 : 0)
 *        2 <= state   -> state + 1, or 0 when state + 1 == C.
 *    All cells update synchronously (ping-pong buffers, Sec. IV-C).
 *  - Boundary: CAT_BOUNDARY_ZERO treats cells outside the grid as dead ghost
 *    cells (the global halo of Sec. IV filled with zeros).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Every call that takes a stream only enqueues work on it and returns; work
 *    enqueued by cat_step / cat_batch_step may be captured into a CUDA graph.
 *  - Return value: CAT_OK (0) or a negative CAT_ERR_* code; cat_last_error()
 *    returns a message for the calling thread's last failure.
 *  - States outside [0, C) give unspecified (but memory-safe) results.
 */
#ifndef CAT_H
#define CAT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CAT_API __attribute__((visibility("default")))
#else
#define CAT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define CAT_OK 0
#define CAT_ERR_INVALID_ARG (-1) /* bad size, rule, pointer, option or pitch         */
#define CAT_ERR_UNSUPPORTED (-2) /* valid request this build cannot serve            */
#define CAT_ERR_OOM (-3)         /* device or host allocation failed                 */
#define CAT_ERR_CUDA (-4)        /* a CUDA runtime/driver call failed (see message)  */
#define CAT_ERR_TIMEOUT (-5)     /* a device-side bounded wait gave up               */
#define CAT_ERR_STATE (-6)       /* call out of order (e.g. stepping before a state) */

/* LTL rule in the R C M S B N notation of Sec. V-A (Table IV lists instances).
 *   r      neighbourhood radius, 1 <= r <= 32.  Up to 16 (the fragment size,
 *          Sec. IV-A) every kernel serves it; 17..32 (the extension to a
 *          second halo fragment that Sec. VII describes) is served with uint8
 *          storage and the zero boundary by TCGEN05 on 128 x 128 tiles in a
 *          192 x 192 window or 96 x 96 tiles in a 160 x 160 one (FP8, C = 2,
 *          Moore; CAT_KERNEL_AUTO picks the first), by the FP16 fragment
 *          kernel (MMA_SYNC, Moore, every C) and by the stencil.
 *   C      number of states, 2 <= C <= 255
 *   M      1: the centre cell counts towards k; 0: it does not
 *   s1,s2  survival range for state-1 cells (inclusive; s1 > s2 means empty)
 *   b1,b2  birth range for state-0 cells (inclusive; b1 > b2 means empty)
 *   nbhd   'M': Moore box of (2r+1)^2 cells (Eqs. 1-2);
 *          'N': simplified von Neumann cross (Eq. 3, R = Pi*Lambda + H): the
 *          vertical and the horizontal segment of half-length r, 4r + 1 cells.
 *          R holds the centre twice; k = R - 2c for M = 0 and R - c for M = 1,
 *          so k counts the live neighbours (plus the cell itself when M = 1)
 *          as with the Moore box.  Served by TCGEN05 with FP8 operands for
 *          C = 2, by MMA_SYNC with FP16 operands and by STENCIL for every C
 *          (CAT_KERNEL_AUTO picks the stencil when C > 2); not by MMA_SYNC
 *          with INT8 operands, BIT1 storage or cat_batch_step_static.
 * Negative range bounds are rejected; nbhd other than 'M' / 'N' is
 * INVALID_ARG.                                                              */
typedef struct cat_rule {
  int32_t r, C, M, s1, s2, b1, b2;
  int32_t nbhd;
} cat_rule_t;

enum { CAT_BOUNDARY_ZERO = 0, CAT_BOUNDARY_PERIODIC = 1 };

/* Operand precision of the two band products (Sec. V-A uses FP16; the others
 * are the lower-precision types Sec. VI names).  Counts are exact in all of
 * them, so every dtype gives the same next states:
 *   FP16      holds every integer <= 2048: the cell states, the band and the
 *             horizontal sums H <= 2r+1 are exact, and so is every partial sum.
 *   FP8_E4M3  a state byte 0x01 read as e4m3 is 2^-9, so the raw bytes are the
 *             pass-1 operand; H * 2^-9 is an e4m3 number while H <= 15
 *             (2r+1 <= 15).  Beyond that the TCGEN05 kernel passes H to the
 *             second product as f16 operands in the 160-row window, and with
 *             a 32-cell halo (H <= 65) as two e4m3 digits, H & 15 against the
 *             band and H >> 4 against a band of 16s (f32 accumulation).
 *   INT8      H <= 65 < 127; served by MMA_SYNC (sm_103a has no tcgen05 kind::i8).
 *   FP4_E2M1  TCGEN05, Moore, r <= 16, one step per launch, uint8 / one-bit /
 *             four-bit storage, any C: the window is re-encoded as e2m1 (a
 *             state-1 cell 0.5; kind::f8f6f4 reads e2m1 from shared memory as
 *             16 elements packed into the first 8 bytes of each 16-byte unit)
 *             against an e2m1 band of ones, so pass 1 gives H / 2 exactly.
 *             H <= 33 is not an e2m1 number (the largest is 6), so pass 2
 *             runs as in FP8_E4M3: H as e4m3 for 2r+1 <= 15 (the e2m1 /
 *             e4m3 mix of kind::f8f6f4), else H / 2 in f16 against an f16
 *             band of 2^-8. */
enum {
  CAT_DTYPE_AUTO = 0,
  CAT_DTYPE_FP16 = 1,
  CAT_DTYPE_FP8_E4M3 = 2,
  CAT_DTYPE_INT8 = 3,
  CAT_DTYPE_FP4_E2M1 = 4
};

/* How the instance stores its grid in device memory.
 *   U8    one byte per cell (the cell's state), W bytes per row.
 *   BIT1  one bit per cell, for two-state rules (C = 2): cell x of a row is
 *         bit x % 8 of byte x / 8 (lowest x in the lowest bit), so a row takes
 *         ceil(W / 8) bytes and the bits past W in the last byte stay 0.  An
 *         eighth of the HBM traffic of U8.  Stepped by the TCGEN05 kernel on
 *         FP8 or FP4 operands, or by BITSLICE for r <= 5, with the zero boundary
 *         (Moore neighbourhood); cat_batch_step advances BIT1
 *         instances one launch per instance and step.  The state is still
 *         passed in and out one byte per cell (cat_set_state/cat_get_state
 *         convert on the device); cat_state_ptr exposes the packed rows.
 *   NIB4  four bits per cell, for rules with C <= 16 (the multi-state rules
 *         of the Generations reading): cell x of a row is nibble x % 2 of
 *         byte x / 2 (even x in the low nibble), so a row takes ceil(W / 2)
 *         bytes and the nibble past an odd W stays 0.  Half the HBM traffic
 *         of U8.  Stepped by the TCGEN05 kernel on FP8 or FP4 operands (the
 *         window unpacked to state-1 flags in shared memory), r <= 16, Moore, the
 *         zero boundary, one step per launch; cat_batch_step advances NIB4
 *         instances one launch per instance and step.  State in and out as
 *         with BIT1.                                                        */
enum { CAT_STORE_U8 = 0, CAT_STORE_BIT1 = 1, CAT_STORE_NIB4 = 2 };

/* Which kernel advances the grid.
 *   TCGEN05   TMA-staged haloed 128x128 tiles (a 32-cell halo for r > 16, or
 *             96x96 tiles), both band products on the 5th-generation tensor cores
 *             (tcgen05.mma, TMEM accumulators), transition fused into the
 *             epilogue (FP16 or FP8 operands).
 *   MMA_SYNC  the paper's own fragment scheme (Alg. 1: three 16x16 band
 *             fragments, 6 MMAs per fragment) on warp-level mma.sync
 *             (FP16 operands, or INT8 operands for CAT_DTYPE_INT8).
 *   STENCIL   classical shared-memory CUDA-core stencil (the out-halo SHARED
 *             design of Sec. V-A, Table V), one (2r+1)^2 loop per cell.
 *   BITSLICE  bit-sliced CUDA-core kernel on one-bit storage for r <= 5, the
 *             packed-cell regime where Sec. V-B finds packing faster than
 *             tensor cores: the counts of 32 cells per 32-bit word are added
 *             as bit planes by bitwise full adders, and the rule is a
 *             bit-serial range comparison (CAT_STORE_BIT1, C = 2, Moore, zero
 *             boundary; no operand dtype).
 *   RUNSUM    separable running-sum CUDA-core kernel, O(1) work per cell in
 *             r: vertical box sums as running sums down columns (four cells
 *             per 32-bit word), then horizontal running sums along rows
 *             (Moore neighbourhood, every C, uint8 storage, zero boundary,
 *             r <= 32): the strongest CUDA-core reference point.           */
enum {
  CAT_KERNEL_AUTO = 0,
  CAT_KERNEL_TCGEN05 = 1,
  CAT_KERNEL_MMA_SYNC = 2,
  CAT_KERNEL_STENCIL = 3,
  CAT_KERNEL_BITSLICE = 4,
  CAT_KERNEL_RUNSUM = 5
};

typedef struct cat_instance *cat_handle_t;

/* Creates an instance: validates the rule and the shape, allocates two
 * pitch-padded device buffers (ping-pong, Sec. IV-C; pitch = W rounded up to a
 * multiple of 16 bytes) and builds the TMA descriptors.  boundary:
 * CAT_BOUNDARY_ZERO (cells outside the grid are dead) or CAT_BOUNDARY_PERIODIC
 * (the grid wraps around in both directions, the paper's setting, Sec. V); a
 * periodic grid sits inside a 16-cell ghost frame (pitch = W + 32 rounded up to
 * 16), refreshed by a small kernel before every step, and is stepped by the
 * tcgen05 kernel only.  The state is all zero until cat_set_state.  The
 * instance owns its buffers; cat_destroy frees them.  Uses the current CUDA
 * device.  The kernel defaults to TCGEN05 with FP8 operands; r > 16 with C > 2
 * selects MMA_SYNC with FP16 operands, the simplified von Neumann cross with
 * C > 2 or r > 16 the STENCIL, and one-bit storage with r <= 5 BITSLICE
 * (cat_set_options changes them).  Errors:
 * INVALID_ARG (H or W < 1, H or W > 2^31 - 256, H * pitch > 2^40, bad rule,
 * unknown boundary), UNSUPPORTED (r > 16 with a periodic boundary), OOM,
 * CUDA.                                                                     */
CAT_API int cat_create(int64_t H, int64_t W, const cat_rule_t *rule, int32_t boundary,
               cat_handle_t *out);

/* cat_create with the storage chosen up front, so that a one-bit grid never
 * holds the byte-per-cell buffers (a CAT_STORE_BIT1 grid of 2^40 cells takes
 * 2 x 128 GiB).  storage is CAT_STORE_U8 (same as cat_create) or
 * CAT_STORE_BIT1 (C = 2 and the zero boundary; options default to TCGEN05 +
 * FP8_E4M3).  Errors: as cat_create, INVALID_ARG for an unknown storage,
 * UNSUPPORTED for BIT1 with C != 2 or a periodic boundary.                  */
CAT_API int cat_create_ex(int64_t H, int64_t W, const cat_rule_t *rule, int32_t boundary,
                  int32_t storage, cat_handle_t *out);

/* Chooses the kernel, operand dtype and storage used by later steps
 * (defaults: CAT_KERNEL_AUTO -> TCGEN05, CAT_DTYPE_AUTO -> FP8_E4M3 for
 * TCGEN05 (FP4_E2M1 on NIB4 storage), FP16 for
 * MMA_SYNC; instances start with CAT_STORE_U8).  A change
 * of storage reallocates both buffers and converts the current grid (the
 * device is synchronised; earlier cat_state_ptr addresses become invalid).
 * CAT_STORE_BIT1 needs C = 2, the zero boundary and TCGEN05 with FP8_E4M3 or
 * FP4_E2M1, or BITSLICE (r <= 5).  CAT_STORE_NIB4 needs TCGEN05 with
 * FP8_E4M3 or FP4_E2M1.
 * steps_per_launch = k > 1 makes cat_step run k steps per kernel launch: one
 * cooperative launch (all CTAs resident, one per SM) whose CTAs meet on a
 * grid-wide barrier between steps, so small grids stop paying a launch per
 * step; served by TCGEN05 for the Moore neighbourhood with the zero boundary
 * (any dtype and C; uint8 or one-bit storage).  With BITSLICE, k steps per
 * launch with k r <= 8 run as temporal blocking: each block keeps its tile
 * and a k r-row, k r-cell stale halo in shared memory and advances it k steps
 * before writing it back (small grids then pay one launch per k steps).  A
 * tcgen05 launch that gives up on a barrier wait sets
 * the status word like any other bounded wait; cat_status then also resets
 * the barrier counter.  Errors: INVALID_ARG for unknown values,
 * UNSUPPORTED for combinations this build does not serve (e.g. TCGEN05 +
 * INT8: sm_103a has no tcgen05 kind::i8; FP4_E2M1 with r > 16, the von
 * Neumann cross or k > 1), OOM, CUDA.  After INVALID_ARG,
 * UNSUPPORTED or OOM the instance keeps its previous options and state.     */
CAT_API int cat_set_options(cat_handle_t h, int32_t kernel, int32_t dtype, int32_t storage,
                    int32_t steps_per_launch);

/* Tile shape and window of the TCGEN05 Moore kernel (the ty, tx tile options;
 * the step's results do not depend on them, only its speed).
 *   ty x tx  0 x 0 or 128 x 128: the 128 x 128 tile (its window chosen
 *            below); 96 x 96: the tile of a 160 x 160 window with a 32-cell
 *            halo (any r <= 32; FP8 operands, C = 2, uint8 storage, the zero
 *            boundary, one step per launch).
 *   window_rows  0: chosen by the rule (144 for FP8 operands, C = 2, r <= 7;
 *            192 for r > 16; else 160); 144: the short window (FP8, C = 2,
 *            r <= 7, uint8 storage); 160: the 160 x 160 window with a
 *            16-cell halo (r <= 16); 192: the 192 x 192 window with a 32-cell
 *            halo (any r <= 32; FP8 operands, C = 2, uint8 storage, the zero
 *            boundary, one step per launch; pass 2 on two e4m3 digits of H
 *            into f32).
 * The autotuner (cat_autotune) drives this call.  Later changes of
 * kernel, dtype or storage that a chosen tile does not serve are rejected by
 * cat_set_options.  Errors: INVALID_ARG (other shapes), UNSUPPORTED (a shape
 * the instance's kernel, dtype, storage, boundary or rule does not serve). */
CAT_API int cat_set_tile(cat_handle_t h, int32_t ty, int32_t tx, int32_t window_rows);

/* The options in force: kernel, operand dtype (CAT_DTYPE_AUTO for kernels
 * without one), storage, steps per launch, and for the TCGEN05 Moore kernel
 * the tile side (128 or 96) and window rows (144, 160 or 192; 0 for the
 * 96 x 96 tile); 0 where they do not apply.  Any pointer may be NULL.  Errors:
 * INVALID_ARG (NULL handle).                                                */
CAT_API int cat_get_options(cat_handle_t h, int32_t *kernel, int32_t *dtype, int32_t *storage,
                            int32_t *steps_per_launch, int32_t *tile, int32_t *window_rows);

/* Autotuner (the paper tunes its tile shape by hand, Sec. V-B; every
 * candidate computes the same states, so only speed is at stake).  Times
 * every configuration the instance can run -- kernel x operand dtype x tile
 * shape x window x steps per launch (1, 4, 16), keeping its storage -- with
 * n_steps steps each from its current state (CUDA events on `stream`), then
 * applies the fastest and restores the state.  The choice is appended to the
 * JSON-lines file cache_path (NULL: no file), one object per line:
 *   {"key": "H=.. W=.. r=.. C=.. nbhd=.. boundary=.. storage=.. gpu=<name>/<SMs>",
 *    "kernel": k, "dtype": d, "tile": t, "window": w, "steps_per_launch": s,
 *    "cell_updates_per_s": v}
 * and when the file already holds an entry for the instance, that entry is
 * applied without timing (unless flags has CAT_TUNE_REMEASURE).  With the
 * environment variable CAT_AUTOTUNE_CACHE naming such a file,
 * cat_set_options(CAT_KERNEL_AUTO, ...) takes the cached choice (kernel,
 * dtype, steps per launch, tile, window) in place of its fixed rule.
 * Synchronises `stream`; allocates a temporary copy of the state.  Errors:
 * INVALID_ARG, UNSUPPORTED (no candidate ran), OOM/CUDA.                    */
#define CAT_TUNE_REMEASURE 1 /* ignore a cached entry and time again         */
#define CAT_TUNE_NO_WRITE 2  /* do not append the choice to the cache file   */
CAT_API int cat_autotune(cat_handle_t h, int32_t n_steps, const char *cache_path, int32_t flags, void *stream);

/* Autotuner for a batch: one configuration for all instances (a batched
 * launch shares kernel and dtype) -- TCGEN05 with FP8 or FP16 operands, the
 * window chosen by the rule or the full one -- each timed over n_steps steps
 * of cat_batch_step after one untimed call; applies the fastest, restores
 * every state and reports its dtype in *chosen_dtype (may be NULL).
 * Synchronises `stream`.  Errors: as cat_batch_step, UNSUPPORTED.           */
CAT_API int cat_autotune_batch(const cat_handle_t *hs, int32_t count, int32_t n_steps, int32_t *chosen_dtype,
                               void *stream);

/* Copies a grid into the instance's current buffer: the state Lambda that the
 * next step reads (Sec. IV-C, Alg. 1: the grid the ping-pong loop starts
 * from).  src holds H rows of W bytes at `pitch` (>= W) bytes, states in
 * [0, C); it is device memory when src_on_device != 0, else host memory
 * (pageable or pinned).  Enqueued on `stream`; a pageable host source is
 * copied synchronously.  The caller keeps ownership of src.  Errors:
 * INVALID_ARG (NULL, pitch < W), CUDA.                                      */
CAT_API int cat_set_state(cat_handle_t h, const uint8_t *src, int64_t pitch, int32_t src_on_device,
                  void *stream);

/* Copies the current grid out: the state after the steps taken so far (the
 * buffer the last step of the Sec. IV-C ping-pong wrote).  Same layout,
 * ownership and error rules as cat_set_state; dst is written, H rows of W
 * bytes at `pitch`.                                                          */
CAT_API int cat_get_state(cat_handle_t h, uint8_t *dst, int64_t pitch, int32_t dst_on_device,
                  void *stream);

/* Device address of grid cell (0, 0) of the current buffer and the buffer's
 * pitch (valid until the next step, set_state or destroy).  For zero-copy
 * inspection; the library owns it.  With a periodic boundary the address lies
 * inside the ghost frame's allocation, 16 rows and 16 bytes past its start.
 * With CAT_STORE_BIT1 it holds the packed rows (pitch = ceil(W / 8) rounded
 * up to 16 bytes).                                                          */
CAT_API int cat_state_ptr(cat_handle_t h, void **dptr, int64_t *pitch);

/* Makes the instance step two caller-owned device buffers instead of its own
 * (for a framework whose allocator owns the memory, e.g. two torch tensors):
 * a and b hold H rows of W cells at `pitch` bytes (pitch >= W and a multiple
 * of 16; both 16-byte aligned, device memory, distinct).  The current state
 * is taken from a as it is (no copy); after a step the state is in b, then a
 * again, as cat_state_ptr reports.  The instance's own buffers are freed; the
 * library never frees bound ones (cat_destroy leaves them to the caller, who
 * must keep them alive while the instance uses them).  Synchronises the
 * device.  Zero boundary and uint8 storage only (UNSUPPORTED otherwise, and
 * for a later change to one-bit storage).  Errors: INVALID_ARG, UNSUPPORTED,
 * CUDA.                                                                     */
CAT_API int cat_bind(cat_handle_t h, uint8_t *a, uint8_t *b, int64_t pitch);

/* Advances the instance by n_steps >= 0 synchronous LTL steps on `stream`:
 * the host loop of Sec. IV-C (Alg. 1), one launch reading buffer A and
 * writing buffer B, then the two swap (with steps_per_launch = k > 1, k steps
 * per launch, the swap inside it).  Each step computes the band products of
 * Sec. IV (Eqs. 1-2) and the rule of Sec. V-A for every cell.  Errors:
 * INVALID_ARG (NULL, n_steps < 0), CUDA (launch failure); device-side
 * timeouts are reported by cat_status.                                     */
CAT_API int cat_step(cat_handle_t h, int64_t n_steps, void *stream);

/* Advances `count` independent instances by n_steps each.  The instances may
 * differ in size, radius and rule.  When all of them run the tcgen05 kernel
 * on the Moore neighbourhood with r <= 16 (128 x 128 tiles), the zero
 * boundary and uint8 storage, and share the dtype, each step is ONE
 * persistent launch over a flat tile work-list of all instances, and when
 * `stream` is not capturing the n_steps launches are replayed from a CUDA
 * graph cached for this handle list; otherwise every instance is stepped by
 * its own launches, one step at a time.  Errors: INVALID_ARG (NULL or
 * repeated handles, instances on different devices, mixed dtypes in a
 * batched launch), UNSUPPORTED (a batched instance above 4194176 cells per
 * side), OOM, CUDA.                                                        */
CAT_API int cat_batch_step(const cat_handle_t *hs, int32_t count, int64_t n_steps, void *stream);

/* Debug/verification: writes the counts of the current state, computed by
 * the selected kernel's band products, to dst (device memory, int32, row
 * stride ld >= W elements): the Moore box count L(y,x) (centre once), or for
 * nbhd 'N' the cross count R(y,x) of Eq. 3 (centre twice).  Does not advance
 * the state.                                                                */
CAT_API int cat_box_sums(cat_handle_t h, int32_t *dst, int64_t ld, void *stream);

/* Synchronises `stream` and reports device-side failures of this instance's
 * earlier launches: CAT_ERR_TIMEOUT if a bounded wait gave up (the kernel
 * then skipped its remaining tiles), else CAT_OK.  Clears the flag.         */
CAT_API int cat_status(cat_handle_t h, void *stream);

/* ---------------------------------------------------------------------------
 * Allocation-free batched step.  The paper has no counterpart to this call.
 *
 * cat_batch_step allocates device memory for its descriptor table and tile
 * work-list.  Some callers cannot allow that: a framework whose caching
 * allocator already owns the whole device-memory budget, a service whose
 * memory footprint is fixed when it starts, or code that must not call
 * cudaMalloc/cudaFree because those calls can synchronise the device.
 * cat_batch_step_static advances `count` independent grids by ONE step in one
 * persistent tcgen05 launch and allocates nothing: the caller passes the input
 * and output buffers (device memory, e.g. from its own allocator), and the
 * table and work-list go into one fixed array compiled into the library
 * (753,664 bytes = 736 KiB of device memory, held on every GPU that loads the
 * library until the process exits).
 *
 *  - Limits: at most CAT_STATIC_MAX_GRIDS grids and CAT_STATIC_MAX_TILES tiles
 *    of 128 x 128 cells in total; larger batches get CAT_ERR_INVALID_ARG and
 *    nothing is launched.  Each grid: 1 <= H, W <= 4194176, pitch >= W and a
 *    multiple of 16 bytes, 16-byte aligned buffers, r <= 16, Moore
 *    neighbourhood, zero boundary.
 *  - Buffers: all grids advance in one launch, so a grid's `out` bytes (rows
 *    0..H-1 at `pitch`, W bytes each) may overlap no other grid's `in` or
 *    `out` and not its own `in`; inputs may share memory.  Overlaps are
 *    rejected with CAT_ERR_INVALID_ARG.
 *  - dtype: CAT_DTYPE_FP8_E4M3 (or AUTO) or CAT_DTYPE_FP16.
 *  - d_status: required device int32 (NULL is CAT_ERR_INVALID_ARG).  It is
 *    zeroed at the start of the call and receives a non-zero code if a
 *    bounded device wait timed out, in which case the kernel skipped its
 *    remaining tiles and `out` is incomplete.  The call itself returns before
 *    the launch completes, so only d_status reports such a timeout.
 *  - The table is staged from host memory that the next call reuses, so the
 *    call must not be captured into a CUDA graph: on a capturing stream it
 *    returns CAT_ERR_INVALID_ARG without enqueueing anything.
 *  - The first call on a device finds the array's device address
 *    (cudaGetSymbolAddress) with that device current.
 *  - Every call reuses the same array, which keeps the last call's contents.
 *    Calls whose launches overlap on the GPU (e.g. on two streams without an
 *    ordering between them) race on it: order them on one stream.
 *  - The next states are written to `out`; swap `in` and `out` to continue.
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA.                                    */
#define CAT_STATIC_MAX_GRIDS 256
#define CAT_STATIC_MAX_TILES 65536

typedef struct cat_grid_desc {
  const uint8_t *in; /* current states (device memory), H rows at `pitch` bytes */
  uint8_t *out;      /* next states (device memory), same layout               */
  int64_t H, W;      /* rows and columns                                      */
  int64_t pitch;     /* bytes between consecutive rows of both buffers        */
  cat_rule_t rule;
} cat_grid_desc_t;

CAT_API int cat_batch_step_static(const cat_grid_desc_t *grids, int32_t count, int32_t dtype,
                                  int32_t *d_status, void *stream);

/* Measurement: the dense tcgen05 MMA rate of the current GPU, the denominator
 * of the roofline's tensor term (the paper has no counterpart; its cost model,
 * Sec. IV-D, uses the vendor's peak).  Launches one CTA per SM, each issuing
 * mmas_per_sm back-to-back MMAs of M = 128, N = 256 with zero operands in
 * shared memory and f32 accumulators in tensor memory; dtype
 * CAT_DTYPE_FP8_E4M3 or CAT_DTYPE_FP4_E2M1 (K = 32, kind::f8f6f4) or
 * CAT_DTYPE_FP16 (K = 16, kind::f16).  The caller times the launch on
 * `stream`; it performs
 * SMs x mmas_per_sm x 2 x 128 x 256 x K flops.  d_status (device int32,
 * required) receives a non-zero code if the bounded wait for the MMAs gave
 * up; the caller zeroes it.  Errors: INVALID_ARG (mmas_per_sm outside
 * [1, 2^30], NULL d_status), UNSUPPORTED (another dtype or device), CUDA.   */
CAT_API int cat_tensor_probe(int32_t dtype, int64_t mmas_per_sm, int32_t *d_status, void *stream);

/* Test hook for the failure-detection path; not needed in normal use.
 *   what = 1: value 1 makes the next tcgen05 launches wait on a barrier that
 *             nothing arrives at, so the bounded wait runs out (value 0 clears);
 *   what = 2: bounded-wait limit in milliseconds (default 2000).
 * Errors: INVALID_ARG.                                                      */
CAT_API int cat_debug_control(cat_handle_t h, int32_t what, int64_t value);

/* Frees the instance (synchronises the device first).  NULL is accepted.    */
CAT_API int cat_destroy(cat_handle_t h);

/* Message describing the calling thread's most recent failure ("" if none). */
CAT_API const char *cat_last_error(void);

/* Library version string and the compute capability it was built for.      */
CAT_API const char *cat_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CAT_H */
