// C ABI (include/cat.h): instance management, TMA descriptors, dispatch.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/cat.h"
#include "cat_internal.h"

using cat::RuleDev;

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  return fail(CAT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CAT_CUDA(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

struct DeviceInfo {
  int id = -1, sms = 0, major = 0, minor = 0;
};

int device_info(DeviceInfo *di) {
  int dev = 0;
  CAT_CUDA(cudaGetDevice(&dev));
  CAT_CUDA(cudaDeviceGetAttribute(&di->sms, cudaDevAttrMultiProcessorCount, dev));
  CAT_CUDA(cudaDeviceGetAttribute(&di->major, cudaDevAttrComputeCapabilityMajor, dev));
  CAT_CUDA(cudaDeviceGetAttribute(&di->minor, cudaDevAttrComputeCapabilityMinor, dev));
  di->id = dev;
  if (di->major != 10 || di->minor != 3)
    return fail(CAT_ERR_UNSUPPORTED, "device %d is sm_%d%d; this library is built for sm_103a", dev,
                di->major, di->minor);
  return CAT_OK;
}

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

}  // namespace

struct cat_instance {
  int64_t H = 0, W = 0, pitch = 0;
  cat_rule_t rule{};
  RuleDev rd{};
  int32_t boundary = 0;
  int32_t ghost = 0;       // periodic: ghost-frame width around the grid (16), else 0
  int32_t storage = CAT_STORE_U8;  // BIT1: one bit per cell, (W + 7) / 8 bytes per row
  int32_t kernel = CAT_KERNEL_TCGEN05, dtype = CAT_DTYPE_FP8_E4M3;
  uint8_t *buf[2] = {nullptr, nullptr};
  int cur = 0;
  int32_t *d_err = nullptr;
  // per buffer: window boxes 128 x 160 and 32 x 160, the 128 x 128 tile box,
  // the window boxes of the short-window kernel, 128 x 144 and 32 x 144, and
  // the 96 x 96 tile box (no swizzle) of the wide-tile kernel
  CUtensorMap maps[2][8];
  int32_t tile = 0;     // cat_set_tile: 0 chosen by the radius, 128 or 96
  int32_t window = 0;   // cat_set_tile: 0 chosen by the rule, 144 or 160
  DeviceInfo dev;
  int32_t inject = 0;
  uint64_t timeout_ns = 2000000000ull;
  int32_t steps_per_launch = 1;  // > 1: cooperative launches of several steps
  bool owns_buffers = true;      // false after cat_bind: the caller owns buf[0], buf[1]
  uint32_t gbar_count = 0;       // arrivals on the grid-barrier counter (d_err[1]) so far
  // grid cell (0, 0) of buffer b (past the ghost frame when there is one)
  uint8_t *origin(int b) const { return buf[b] + ghost * pitch + ghost; }
};

namespace {

int validate_rule(const cat_rule_t *r) {
  if (!r) return fail(CAT_ERR_INVALID_ARG, "rule is NULL");
  if (r->r < 1 || r->r > 32) return fail(CAT_ERR_INVALID_ARG, "radius %d outside [1, 32]", r->r);
  if (r->C < 2 || r->C > 255) return fail(CAT_ERR_INVALID_ARG, "C = %d outside [2, 255]", r->C);
  if (r->M != 0 && r->M != 1) return fail(CAT_ERR_INVALID_ARG, "M must be 0 or 1");
  if (r->s1 < 0 || r->s2 < 0 || r->b1 < 0 || r->b2 < 0)
    return fail(CAT_ERR_INVALID_ARG, "negative range bound");
  if (r->nbhd != 'M' && r->nbhd != 'N')
    return fail(CAT_ERR_INVALID_ARG, "neighbourhood must be 'M' (Moore) or 'N' (simplified von Neumann)");
  return CAT_OK;
}

// Range tests on the box count S (centre included), see RuleDev.
RuleDev reduce_rule(const cat_rule_t &r) {
  RuleDev d{};
  d.r = r.r;
  d.C = r.C;
  d.M = r.M;
  d.nbhd = r.nbhd == 'N' ? 1 : 0;
  // a live cell's own state is in S once (Moore) or twice (the cross of
  // Eq. 3); the rule's count keeps it once when M = 1, drops it when M = 0
  const int own = (d.nbhd ? 2 : 1) - r.M;
  const int empty_lo = 1 << 24;
  if (r.s1 > r.s2) { d.s_lo = empty_lo; d.s_w = 0; }
  else { d.s_lo = r.s1 + own; d.s_w = r.s2 - r.s1; }
  if (r.b1 > r.b2) { d.b_lo = empty_lo; d.b_w = 0; }
  else { d.b_lo = r.b1; d.b_w = r.b2 - r.b1; }
  return d;
}

int make_map(CUtensorMap *m, void *base, int64_t H, int64_t W, int64_t pitch, uint32_t box_x,
             uint32_t box_y, CUtensorMapSwizzle sw) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return fail(CAT_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
  cuuint64_t strides[1] = {(cuuint64_t)pitch};
  cuuint32_t box[2] = {box_x, box_y};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(CAT_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return CAT_OK;
}

int build_maps(cat_instance *h) {
  if (h->storage == CAT_STORE_NIB4) {  // packed rows: 96 x 160-byte windows, 64 x 128-byte tiles (64B swizzle)
    for (int b = 0; b < 2; ++b) {
      int rc;
      const int64_t wb = (h->W + 1) / 2;
      if ((rc = make_map(&h->maps[b][0], h->buf[b], h->H, wb, h->pitch, 96, 160, CU_TENSOR_MAP_SWIZZLE_NONE))) return rc;
      if ((rc = make_map(&h->maps[b][2], h->buf[b], h->H, wb, h->pitch, 64, 128, CU_TENSOR_MAP_SWIZZLE_64B))) return rc;
      h->maps[b][1] = h->maps[b][3] = h->maps[b][4] = h->maps[b][5] = h->maps[b][6] = h->maps[b][7] = h->maps[b][0];
    }
    return CAT_OK;
  }
  if (h->storage == CAT_STORE_BIT1) {  // packed rows: 48 x 160-byte windows, 16 x 128-byte tiles
    for (int b = 0; b < 2; ++b) {
      int rc;
      const int64_t wb = (h->W + 7) / 8;
      if ((rc = make_map(&h->maps[b][0], h->buf[b], h->H, wb, h->pitch, 48, 160, CU_TENSOR_MAP_SWIZZLE_NONE))) return rc;
      if ((rc = make_map(&h->maps[b][2], h->buf[b], h->H, wb, h->pitch, 16, 128, CU_TENSOR_MAP_SWIZZLE_NONE))) return rc;
      h->maps[b][1] = h->maps[b][3] = h->maps[b][4] = h->maps[b][5] = h->maps[b][6] = h->maps[b][7] = h->maps[b][0];
    }
    return CAT_OK;
  }
  for (int b = 0; b < 2; ++b) {
    int rc;
    // the maps span the buffer including any ghost frame
    const int64_t H = h->H + 2 * h->ghost, W = h->W + 2 * h->ghost;
    if ((rc = make_map(&h->maps[b][0], h->buf[b], H, W, h->pitch, 128, 160, CU_TENSOR_MAP_SWIZZLE_128B))) return rc;
    if ((rc = make_map(&h->maps[b][1], h->buf[b], H, W, h->pitch, 32, 160, CU_TENSOR_MAP_SWIZZLE_32B))) return rc;
    if ((rc = make_map(&h->maps[b][2], h->buf[b], H, W, h->pitch, 128, 128, CU_TENSOR_MAP_SWIZZLE_128B))) return rc;
    if ((rc = make_map(&h->maps[b][3], h->buf[b], H, W, h->pitch, 128, 144, CU_TENSOR_MAP_SWIZZLE_128B))) return rc;
    if ((rc = make_map(&h->maps[b][4], h->buf[b], H, W, h->pitch, 32, 144, CU_TENSOR_MAP_SWIZZLE_32B))) return rc;
    if ((rc = make_map(&h->maps[b][5], h->buf[b], H, W, h->pitch, 96, 96, CU_TENSOR_MAP_SWIZZLE_NONE))) return rc;
    if ((rc = make_map(&h->maps[b][6], h->buf[b], H, W, h->pitch, 128, 192, CU_TENSOR_MAP_SWIZZLE_128B))) return rc;
    if ((rc = make_map(&h->maps[b][7], h->buf[b], H, W, h->pitch, 32, 192, CU_TENSOR_MAP_SWIZZLE_32B))) return rc;
  }
  return CAT_OK;
}

// The kernels with a 32-cell halo serve radii above 16 on tcgen05, and any
// radius when cat_set_tile asks for one of them: the 128 x 128 tile in a
// 192 x 192 window (radii above 16 by default, or window 192), or the
// 96 x 96 tile in the 160 x 160 window (tile 96).
bool wide_tile(const cat_instance *h) {
  return h->kernel == CAT_KERNEL_TCGEN05 && h->rule.nbhd == 'M' &&
         (h->rule.r > 16 || h->tile == 96 || h->window == 192);
}
bool big_window(const cat_instance *h) { return wide_tile(h) && h->tile != 96; }

// The short-window kernel serves FP8 operands on two-state rules with r <= 7
// (pass 2 then runs on e4m3, and 128 + 2r window rows fit in 144), unless
// cat_set_tile asked for the 160-row window.
bool short_window(const cat_instance *h) {
  return h->kernel == CAT_KERNEL_TCGEN05 && h->dtype == CAT_DTYPE_FP8_E4M3 && h->rule.C == 2 && h->rule.r <= 7 &&
         h->window != 160 && !wide_tile(h);
}

// n_steps steps of instance h from buffer `in` (into buffer 1 - in after an
// odd count), or the box sums of buffer `in` into `sums`.  n_steps > 1 is one
// cooperative launch of the tcgen05 Moore kernel (zero boundary).
int launch_step(cat_instance *h, int in, int32_t *sums, int64_t sums_ld, cudaStream_t s, int n_steps = 1) {
  cudaError_t e;
  if (h->kernel == CAT_KERNEL_TCGEN05) {
    if (h->ghost) {  // periodic: refresh the input's ghost frame first
      e = cat::ghost_fill_launch(h->buf[in], h->pitch, h->H, h->W, h->ghost, s);
      if (e != cudaSuccess) return cuda_fail(e, "ghost-frame launch");
    }
    cat::TcParams p;
    memset(&p, 0, sizeof(p));
    p.ox = p.oy = h->ghost;
    const bool vn = h->rule.nbhd == 'N';
    const bool bits = h->storage == CAT_STORE_BIT1;
    const bool nib = h->storage == CAT_STORE_NIB4;
    const bool sw = !vn && !bits && !nib && short_window(h);
    const bool wide = !vn && wide_tile(h);
    const bool big = wide && big_window(h);   // 128 x 128 tiles in the 192 x 192 window
    p.map_in_a = h->maps[in][big ? 6 : sw ? 3 : 0];
    p.map_in_b = h->maps[in][big ? 7 : sw ? 4 : 1];
    p.map_out = h->maps[1 - in][2];
    p.map_ctr = h->maps[in][2];
    p.n_steps = n_steps;
    if (n_steps > 1) {  // odd steps: buffers swapped; the grid barrier counter sits after the status word
      p.map2_in_a = h->maps[1 - in][sw ? 3 : 0];
      p.map2_in_b = h->maps[1 - in][sw ? 4 : 1];
      p.map2_out = h->maps[in][2];
      p.map2_ctr = h->maps[1 - in][2];
      p.gbar = reinterpret_cast<uint32_t *>(h->d_err) + 1;
      p.gbar_base = h->gbar_count;
    }
    const int ts = wide && !big ? 96 : 128;
    if (wide && !big) {   // 96 x 96 centre and output tiles
      p.map_out = h->maps[1 - in][5];
      p.map_ctr = h->maps[in][5];
    }
    p.H = (int32_t)h->H;
    p.W = (int32_t)h->W;
    p.tiles_x = (int32_t)((h->W + ts - 1) / ts);
    p.n_tiles = p.tiles_x * (int32_t)((h->H + ts - 1) / ts);
    p.rule = h->rd;
    p.err = h->d_err;
    p.sums = sums;
    p.sums_ld = sums_ld;
    p.timeout_ns = h->timeout_ns;
    p.inject = h->inject;
    const int grid = p.n_tiles < h->dev.sms ? p.n_tiles : h->dev.sms;
    const bool fp4 = h->dtype == CAT_DTYPE_FP4_E2M1;
    e = vn ? cat::vn_launch(p, grid, s)
           : big  ? cat::big_launch(p, grid, s)
           : wide ? cat::wide_launch(p, grid, s)
           : fp4  ? cat::fp4_launch(p, bits ? 1 : nib ? 2 : 0, grid, s)
           : nib  ? cat::nib_launch(p, grid, s)
                  : cat::tc_launch(p, h->dtype, bits || h->rule.C > 2, sw, bits, grid, s);
    if (e == cudaSuccess && n_steps > 1) h->gbar_count += (uint32_t)grid * (uint32_t)(n_steps - 1);
  } else {
    if (h->ghost) return fail(CAT_ERR_UNSUPPORTED, "the periodic boundary is served by the tcgen05 kernel only");
    cat::SimpleParams p;
    memset(&p, 0, sizeof(p));
    p.in = h->buf[in];
    p.out = h->buf[1 - in];
    p.pitch = h->pitch;
    p.H = (int32_t)h->H;
    p.W = (int32_t)h->W;
    p.rule = h->rd;
    p.sums = sums;
    p.sums_ld = sums_ld;
    if (h->kernel == CAT_KERNEL_BITSLICE && n_steps > 1)   // temporal blocking: n_steps in one launch
      e = cat::swar_tb_launch(h->buf[in], h->buf[1 - in], h->pitch, h->H, h->W, h->rd, n_steps, s);
    else if (h->kernel == CAT_KERNEL_BITSLICE)
      e = cat::swar_launch(h->buf[in], h->buf[1 - in], h->pitch, h->H, h->W, h->rd, sums, sums_ld, s);
    else if (h->kernel == CAT_KERNEL_RUNSUM)
      e = cat::runsum_launch(p, s);
    else
      e = h->kernel == CAT_KERNEL_MMA_SYNC ? cat::mma_launch(p, h->dtype, s) : cat::stencil_launch(p, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return CAT_OK;
}

// ---------------------------------------------------------------- batches
// A batch plan: the per-instance descriptor table and the tile work-list of
// one handle list, kept on the device, plus cached CUDA graphs of n launches.
struct BatchPlan {
  std::vector<cat_instance *> hs;
  std::vector<int> cur0;      // each instance's current buffer when the table was built
  int64_t steps_done = 0;     // steps advanced through this plan since then
  int32_t dtype = 0;
  bool encode = false;
  bool sw = false;            // every instance qualifies for the short-window kernel
  cat::BatchInst *d_inst = nullptr;
  cat::BatchTile *d_tiles = nullptr;
  int n_tiles = 0, grid = 0;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};  // by start parity
  int64_t exec_steps[2] = {0, 0};
  cudaStream_t capture_stream = nullptr;
};

std::mutex g_plan_mu;
std::vector<BatchPlan *> g_plans;

void free_plan(BatchPlan *pl) {
  for (int i = 0; i < 2; ++i)
    if (pl->exec[i]) cudaGraphExecDestroy(pl->exec[i]);
  if (pl->capture_stream) cudaStreamDestroy(pl->capture_stream);
  cudaFree(pl->d_inst);
  cudaFree(pl->d_tiles);
  delete pl;
}

void drop_plans_with(cat_instance *h) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  for (auto it = g_plans.begin(); it != g_plans.end();) {
    if (std::find((*it)->hs.begin(), (*it)->hs.end(), h) != (*it)->hs.end()) {
      free_plan(*it);
      it = g_plans.erase(it);
    } else {
      ++it;
    }
  }
}

// (Re)writes the instance table of a plan from the handles' current state.
int upload_instances(BatchPlan *pl) {
  CAT_CUDA(cudaDeviceSynchronize());  // earlier launches of this plan may still read the table
  std::vector<cat::BatchInst> inst(pl->hs.size());
  memset(inst.data(), 0, inst.size() * sizeof(cat::BatchInst));
  pl->cur0.resize(pl->hs.size());
  for (size_t i = 0; i < pl->hs.size(); ++i) {
    const cat_instance *h = pl->hs[i];
    for (int b = 0; b < 2; ++b) {
      inst[i].map_in_a[b] = h->maps[b][pl->sw ? 3 : 0];
      inst[i].map_in_b[b] = h->maps[b][pl->sw ? 4 : 1];
      inst[i].map_out[b] = h->maps[b][2];
    }
    inst[i].rule = h->rd;
    inst[i].H = (int32_t)h->H;
    inst[i].W = (int32_t)h->W;
    inst[i].cur = h->cur;
    inst[i].err = h->d_err;
    pl->cur0[i] = h->cur;
  }
  CAT_CUDA(cudaMemcpy(pl->d_inst, inst.data(), inst.size() * sizeof(cat::BatchInst), cudaMemcpyHostToDevice));
  pl->steps_done = 0;
  for (int i = 0; i < 2; ++i) {
    if (pl->exec[i]) cudaGraphExecDestroy(pl->exec[i]);
    pl->exec[i] = nullptr;
    pl->exec_steps[i] = 0;
  }
  return CAT_OK;
}

int build_plan(const cat_handle_t *hs, int32_t count, BatchPlan **out) {
  BatchPlan *pl = new (std::nothrow) BatchPlan();
  if (!pl) return fail(CAT_ERR_OOM, "host allocation failed");
  pl->hs.assign(hs, hs + count);
  pl->dtype = hs[0]->dtype;
  pl->encode = false;
  for (int32_t i = 0; i < count; ++i) pl->encode |= hs[i]->rule.C > 2;
  pl->sw = true;
  for (int32_t i = 0; i < count; ++i) pl->sw &= short_window(hs[i]);
  // work-list: instances ordered by radius, tiles row-major within an instance
  std::vector<int> order(count);
  for (int32_t i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hs[a]->rule.r < hs[b]->rule.r; });
  std::vector<cat::BatchTile> tiles;
  for (int i : order) {
    const int64_t ty = (hs[i]->H + 127) / 128, tx = (hs[i]->W + 127) / 128;
    for (int64_t y = 0; y < ty; ++y)
      for (int64_t x = 0; x < tx; ++x) tiles.push_back(cat::BatchTile{i, (int16_t)y, (int16_t)x});
  }
  if (tiles.size() > (size_t)INT32_MAX) { delete pl; return fail(CAT_ERR_UNSUPPORTED, "batch too large"); }
  pl->n_tiles = (int)tiles.size();
  pl->grid = std::min(pl->n_tiles, hs[0]->dev.sms);
  cudaError_t e = cudaMalloc(&pl->d_inst, sizeof(cat::BatchInst) * count);
  if (e == cudaSuccess) e = cudaMalloc(&pl->d_tiles, sizeof(cat::BatchTile) * tiles.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(pl->d_tiles, tiles.data(), sizeof(cat::BatchTile) * tiles.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&pl->capture_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) { free_plan(pl); return cuda_fail(e, "batch plan"); }
  int rc = upload_instances(pl);
  if (rc) { free_plan(pl); return rc; }
  *out = pl;
  return CAT_OK;
}

int launch_batch_steps(BatchPlan *pl, int64_t n_steps, int64_t start, cudaStream_t s) {
  cat::TcParams p;
  memset(&p, 0, sizeof(p));
  p.n_tiles = pl->n_tiles;
  p.timeout_ns = pl->hs[0]->timeout_ns;
  p.binst = pl->d_inst;
  p.btiles = pl->d_tiles;
  for (int64_t t = 0; t < n_steps; ++t) {
    p.parity = (int32_t)((start + t) & 1);
    cudaError_t e = cat::tc_launch_batch(p, pl->dtype, pl->encode, pl->sw, pl->grid, s);
    if (e != cudaSuccess) return cuda_fail(e, "batched launch");
  }
  return CAT_OK;
}

}  // namespace

// Host helpers shared with the allocation-free entry point (cat_static.cu).
namespace cat {
int host_fail(int code, const char *msg) { return fail(code, "%s", msg); }
int host_validate_rule(const cat_rule_t *r) { return validate_rule(r); }
RuleDev host_reduce_rule(const cat_rule_t &r) { return reduce_rule(r); }
int host_make_map(CUtensorMap *m, void *base, int64_t H, int64_t W, int64_t pitch, uint32_t box_x,
                  uint32_t box_y, int swizzle128) {
  return make_map(m, base, H, W, pitch, box_x, box_y,
                  swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_32B);
}
int host_instance_info(cat_handle_t h, InstanceInfo *f) {
  if (!h || !f) return fail(CAT_ERR_INVALID_ARG, "NULL handle");
  f->H = h->H;
  f->W = h->W;
  f->rule = h->rule;
  f->boundary = h->boundary;
  f->storage = h->storage;
  f->kernel = h->kernel;
  f->dtype = h->dtype;
  f->tile = h->tile;
  f->window = h->window;
  f->steps_per_launch = h->steps_per_launch;
  return CAT_OK;
}
}  // namespace cat

namespace {

// Rows per chunk when a uint8 grid passes through a temporary device buffer
// on its way to or from one-bit storage (64 MiB at most).
int64_t chunk_rows(int64_t W) { return std::max<int64_t>(1, std::min<int64_t>(4096, (64ll << 20) / W)); }

int64_t storage_pitch(int32_t storage, int64_t W) {
  return storage == CAT_STORE_BIT1 ? round_up((W + 7) / 8, 16) : storage == CAT_STORE_NIB4 ? round_up((W + 1) / 2, 16)
                                                                                           : round_up(W, 16);
}

// Packs uint8 rows into `storage` (BIT1 or NIB4) or unpacks them back.
cudaError_t pack_rows(int32_t storage, const uint8_t *src, int64_t spitch, uint8_t *dst, int64_t dpitch, int64_t rows,
                      int64_t W, cudaStream_t s) {
  return storage == CAT_STORE_BIT1 ? cat::pack_bits_launch(src, spitch, dst, dpitch, rows, W, s)
                                   : cat::pack_nib_launch(src, spitch, dst, dpitch, rows, W, s);
}
cudaError_t unpack_rows(int32_t storage, const uint8_t *src, int64_t spitch, uint8_t *dst, int64_t dpitch,
                        int64_t rows, int64_t W, cudaStream_t s) {
  return storage == CAT_STORE_BIT1 ? cat::unpack_bits_launch(src, spitch, dst, dpitch, rows, W, s)
                                   : cat::unpack_nib_launch(src, spitch, dst, dpitch, rows, W, s);
}

// Reallocates the state of h in `storage`, converting the current grid
// (through a temporary uint8 copy when neither storage is uint8).
int change_storage(cat_instance *h, int32_t storage) {
  const int64_t pitch = storage_pitch(storage, h->W);
  const size_t bytes = (size_t)(pitch * h->H);
  uint8_t *nb[2] = {nullptr, nullptr}, *tmp = nullptr;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMalloc(&nb[0], bytes);
  if (e == cudaSuccess) e = cudaMalloc(&nb[1], bytes);
  if (e == cudaSuccess) e = cudaMemset(nb[0], 0, bytes);
  if (e == cudaSuccess) e = cudaMemset(nb[1], 0, bytes);
  const uint8_t *u8 = h->origin(h->cur);   // the grid one byte per cell
  int64_t u8_pitch = h->pitch;
  if (e == cudaSuccess && h->storage != CAT_STORE_U8) {
    if (storage == CAT_STORE_U8) {
      e = unpack_rows(h->storage, h->origin(h->cur), h->pitch, nb[0], pitch, h->H, h->W, 0);
    } else {
      e = cudaMalloc(&tmp, (size_t)(h->H * h->W));
      if (e == cudaSuccess) e = unpack_rows(h->storage, h->origin(h->cur), h->pitch, tmp, h->W, h->H, h->W, 0);
      u8 = tmp;
      u8_pitch = h->W;
    }
  }
  if (e == cudaSuccess && storage != CAT_STORE_U8) e = pack_rows(storage, u8, u8_pitch, nb[0], pitch, h->H, h->W, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(tmp);
  if (e != cudaSuccess) {
    cudaFree(nb[0]);
    cudaFree(nb[1]);
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? fail(CAT_ERR_OOM, "device allocation of %zu bytes failed", bytes)
                                          : cuda_fail(e, "storage change");
  }
  drop_plans_with(h);
  cudaFree(h->buf[0]);
  cudaFree(h->buf[1]);
  h->buf[0] = nb[0];
  h->buf[1] = nb[1];
  h->cur = 0;
  h->pitch = pitch;
  h->storage = storage;
  return build_maps(h);
}

// uint8 rows <-> packed storage through a temporary device buffer.
int bits_set_state(cat_instance *h, const uint8_t *src, int64_t pitch, cudaStream_t s) {
  const int64_t R = chunk_rows(h->W);
  uint8_t *tmp = nullptr;
  CAT_CUDA(cudaMalloc(&tmp, (size_t)(R * h->W)));
  cudaError_t e = cudaSuccess;
  for (int64_t y = 0; y < h->H && e == cudaSuccess; y += R) {
    const int64_t n = std::min(R, h->H - y);
    e = cudaMemcpy2DAsync(tmp, (size_t)h->W, src + y * pitch, (size_t)pitch, (size_t)h->W, (size_t)n, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = pack_rows(h->storage, tmp, h->W, h->buf[h->cur] + y * h->pitch, h->pitch, n, h->W, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(e, "cat_set_state (packed storage)");
  return CAT_OK;
}

int bits_get_state(cat_instance *h, uint8_t *dst, int64_t pitch, cudaStream_t s) {
  const int64_t R = chunk_rows(h->W);
  uint8_t *tmp = nullptr;
  CAT_CUDA(cudaMalloc(&tmp, (size_t)(R * h->W)));
  cudaError_t e = cudaSuccess;
  for (int64_t y = 0; y < h->H && e == cudaSuccess; y += R) {
    const int64_t n = std::min(R, h->H - y);
    e = unpack_rows(h->storage, h->buf[h->cur] + y * h->pitch, h->pitch, tmp, h->W, n, h->W, s);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(dst + y * pitch, (size_t)pitch, tmp, (size_t)h->W, (size_t)h->W, (size_t)n, cudaMemcpyDefault, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(e, "cat_get_state (packed storage)");
  return CAT_OK;
}

}  // namespace

extern "C" {

const char *cat_last_error(void) { return g_err; }

const char *cat_version(void) { return "cat-gb300 0.1 (sm_103a)"; }

int cat_create(int64_t H, int64_t W, const cat_rule_t *rule, int32_t boundary, cat_handle_t *out) {
  return cat_create_ex(H, W, rule, boundary, CAT_STORE_U8, out);
}

int cat_create_ex(int64_t H, int64_t W, const cat_rule_t *rule, int32_t boundary, int32_t storage,
                  cat_handle_t *out) {
  if (!out) return fail(CAT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (H < 1 || W < 1) return fail(CAT_ERR_INVALID_ARG, "grid %lld x %lld is empty", (long long)H, (long long)W);
  if (H > (1ll << 31) - 256 || W > (1ll << 31) - 256 || H * round_up(W, 16) > (1ll << 40))
    return fail(CAT_ERR_INVALID_ARG, "grid %lld x %lld is too large", (long long)H, (long long)W);
  int rc = validate_rule(rule);
  if (rc) return rc;
  if (boundary != CAT_BOUNDARY_ZERO && boundary != CAT_BOUNDARY_PERIODIC)
    return fail(CAT_ERR_INVALID_ARG, "unknown boundary %d", boundary);
  if (storage != CAT_STORE_U8 && storage != CAT_STORE_BIT1 && storage != CAT_STORE_NIB4)
    return fail(CAT_ERR_INVALID_ARG, "unknown storage %d", storage);
  if (storage == CAT_STORE_BIT1 && rule->C != 2) return fail(CAT_ERR_UNSUPPORTED, "one-bit storage holds two-state rules only");
  if (storage == CAT_STORE_NIB4 && (rule->C > 16 || boundary != CAT_BOUNDARY_ZERO || rule->nbhd != 'M' || rule->r > 16))
    return fail(CAT_ERR_UNSUPPORTED, "four-bit storage holds rules with C <= 16, r <= 16, the Moore "
                                     "neighbourhood and the zero boundary");
  if (storage == CAT_STORE_BIT1 && boundary != CAT_BOUNDARY_ZERO)
    return fail(CAT_ERR_UNSUPPORTED, "one-bit storage is served with the zero boundary only");
  if (storage == CAT_STORE_BIT1 && rule->nbhd != 'M')
    return fail(CAT_ERR_UNSUPPORTED, "one-bit storage is served for the Moore neighbourhood only");
  if (rule->r > 16 && (storage == CAT_STORE_BIT1 || boundary != CAT_BOUNDARY_ZERO))
    return fail(CAT_ERR_UNSUPPORTED, "radii above 16 are served with uint8 storage and the zero boundary");
  cat_instance *h = new (std::nothrow) cat_instance();
  if (!h) return fail(CAT_ERR_OOM, "host allocation failed");
  if ((rc = device_info(&h->dev))) { delete h; return rc; }
  h->H = H;
  h->W = W;
  h->boundary = boundary;
  h->ghost = boundary == CAT_BOUNDARY_PERIODIC ? 16 : 0;
  h->storage = storage;
  h->pitch = storage == CAT_STORE_U8 ? round_up(W + 2 * h->ghost, 16) : storage_pitch(storage, W);
  h->rule = *rule;
  h->rd = reduce_rule(*rule);
  if (rule->nbhd == 'N' && (rule->C > 2 || rule->r > 16)) {  // the cross with C > 2 or r > 16: CUDA-core stencil
    h->kernel = CAT_KERNEL_STENCIL;
    h->dtype = CAT_DTYPE_INT8;
  } else if (rule->r > 16 && rule->C > 2) {  // the paper's fragment scheme with two halo fragments
    h->kernel = CAT_KERNEL_MMA_SYNC;
    h->dtype = CAT_DTYPE_FP16;
  } else if (storage == CAT_STORE_BIT1 && rule->r <= 5) {  // packed cells at small r: bit planes on CUDA cores
    h->kernel = CAT_KERNEL_BITSLICE;
    h->dtype = CAT_DTYPE_AUTO;
  }   // r > 16 with C = 2: the tcgen05 wide tile
  const size_t bytes = (size_t)(h->pitch * (H + 2 * h->ghost));
  cudaError_t e = cudaMalloc(&h->buf[0], bytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->buf[1], bytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_err, 256);
  if (e == cudaSuccess) e = cudaMemset(h->buf[0], 0, bytes);
  if (e == cudaSuccess) e = cudaMemset(h->buf[1], 0, bytes);
  if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, 256);
  if (e != cudaSuccess) {
    cudaFree(h->buf[0]); cudaFree(h->buf[1]); cudaFree(h->d_err);
    delete h;
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? fail(CAT_ERR_OOM, "device allocation of %zu bytes failed", bytes)
                                          : cuda_fail(e, "cat_create");
  }
  if ((rc = build_maps(h))) { cat_destroy(h); return rc; }
  *out = h;
  return CAT_OK;
}

int cat_set_options(cat_handle_t h, int32_t kernel, int32_t dtype, int32_t storage, int32_t steps_per_launch) {
  if (!h) return fail(CAT_ERR_INVALID_ARG, "handle is NULL");
  if (kernel < CAT_KERNEL_AUTO || kernel > CAT_KERNEL_RUNSUM) return fail(CAT_ERR_INVALID_ARG, "unknown kernel %d", kernel);
  if (dtype < CAT_DTYPE_AUTO || dtype > CAT_DTYPE_FP4_E2M1) return fail(CAT_ERR_INVALID_ARG, "unknown dtype %d", dtype);
  if (storage != CAT_STORE_U8 && storage != CAT_STORE_BIT1 && storage != CAT_STORE_NIB4)
    return fail(CAT_ERR_INVALID_ARG, "unknown storage %d", storage);
  if (steps_per_launch < 1) return fail(CAT_ERR_INVALID_ARG, "steps_per_launch must be >= 1");
  const bool vn = h->rule.nbhd == 'N';
  const bool wide = h->rule.r > 16;
  // AUTO: the autotuner's cached choice when CAT_AUTOTUNE_CACHE names a file
  // holding one for this instance (with the storage asked for), else a fixed rule
  int32_t tuned_tile = -1, tuned_window = 0;
  if (kernel == CAT_KERNEL_AUTO && storage == h->storage) {
    cat::InstanceInfo f{};
    cat::host_instance_info(h, &f);
    int32_t k = 0, d = 0, t = 0, w = 0, spl = 0;
    if (cat::tune_cache_lookup_env(f, &k, &d, &t, &w, &spl) && k >= CAT_KERNEL_TCGEN05 && k <= CAT_KERNEL_RUNSUM &&
        d >= CAT_DTYPE_AUTO && d <= CAT_DTYPE_FP4_E2M1 && spl >= 1) {
      kernel = k;
      dtype = d;
      steps_per_launch = spl;
      tuned_tile = t;
      tuned_window = w;
    }
  }
  if (kernel == CAT_KERNEL_AUTO)
    kernel = vn && (h->rule.C > 2 || wide)                                ? CAT_KERNEL_STENCIL
           : wide && h->rule.C > 2                                        ? CAT_KERNEL_MMA_SYNC
           : storage == CAT_STORE_BIT1 && h->rule.r <= 5 && h->rule.C == 2 ? CAT_KERNEL_BITSLICE
                                                                          : CAT_KERNEL_TCGEN05;
  const int32_t cur_tile = tuned_tile >= 0 ? 0 : h->tile;   // a cached choice brings its own tile
  const int32_t cur_window = tuned_tile >= 0 ? 0 : h->window;
  // AUTO: FP8 on tcgen05 (FP4 on four-bit storage, whose state-1 nibble
  // flags are the e2m1 operand as they stand: measured faster at every radius
  // and state count), FP16 on the fragment kernel
  if (dtype == CAT_DTYPE_AUTO)
    dtype = kernel != CAT_KERNEL_TCGEN05 ? CAT_DTYPE_FP16
          : (storage == CAT_STORE_NIB4 && !vn && !wide) ? CAT_DTYPE_FP4_E2M1
                                                          : CAT_DTYPE_FP8_E4M3;
  if (kernel == CAT_KERNEL_TCGEN05 && dtype == CAT_DTYPE_INT8)
    return fail(CAT_ERR_UNSUPPORTED, "sm_103a has no tcgen05 kind::i8; INT8 runs on CAT_KERNEL_MMA_SYNC");
  if (kernel == CAT_KERNEL_TCGEN05 && dtype == CAT_DTYPE_FP4_E2M1 &&
      (vn || wide || cur_tile == 96 || cur_window == 192 || steps_per_launch > 1))
    return fail(CAT_ERR_UNSUPPORTED, "FP4 operands are served by the 128 x 128 tcgen05 Moore kernel (r <= 16), "
                                     "one step per launch");
  if (kernel == CAT_KERNEL_MMA_SYNC && dtype != CAT_DTYPE_FP16 && dtype != CAT_DTYPE_INT8)
    return fail(CAT_ERR_UNSUPPORTED, "the mma.sync kernel serves FP16 and INT8 operands");
  if (kernel == CAT_KERNEL_STENCIL || kernel == CAT_KERNEL_RUNSUM) dtype = CAT_DTYPE_INT8;  // integer counts on CUDA cores
  if (kernel == CAT_KERNEL_RUNSUM && vn)
    return fail(CAT_ERR_UNSUPPORTED, "the running-sum kernel serves the Moore neighbourhood");
  if (kernel == CAT_KERNEL_BITSLICE) {   // bitwise adders on CUDA cores: no operand dtype
    if (storage != CAT_STORE_BIT1 || h->rule.C != 2 || vn || h->ghost || h->rule.r > 5)
      return fail(CAT_ERR_UNSUPPORTED, "the bit-sliced kernel serves one-bit storage, two-state Moore rules, "
                                       "the zero boundary and r <= 5");
    dtype = CAT_DTYPE_AUTO;
  }
  // the 32-cell-halo kernels: radii above 16 on tcgen05, or any radius after
  // cat_set_tile(96, 96) or a 192-row window
  const bool wide_tc = kernel == CAT_KERNEL_TCGEN05 && !vn && (wide || cur_tile == 96 || cur_window == 192);
  if (wide_tc && (dtype != CAT_DTYPE_FP8_E4M3 || h->rule.C != 2 || storage != CAT_STORE_U8 || steps_per_launch > 1))
    return fail(CAT_ERR_UNSUPPORTED,
                "the tcgen05 kernels for r > 16 (192-row window, 96 x 96 tile) serve FP8 operands, two-state rules, "
                "uint8 storage, one step per launch");
  if (wide && kernel == CAT_KERNEL_TCGEN05 && vn)
    return fail(CAT_ERR_UNSUPPORTED, "the simplified von Neumann cross with r > 16 is served by the stencil");
  if (wide && kernel == CAT_KERNEL_MMA_SYNC && (dtype != CAT_DTYPE_FP16 || vn))
    return fail(CAT_ERR_UNSUPPORTED, "radii above 16 on MMA_SYNC are served with FP16 operands (Moore)");
  if (h->ghost && kernel != CAT_KERNEL_TCGEN05)
    return fail(CAT_ERR_UNSUPPORTED, "the periodic boundary is served by the tcgen05 kernel only");
  if (vn) {
    if (kernel == CAT_KERNEL_MMA_SYNC && dtype != CAT_DTYPE_FP16)
      return fail(CAT_ERR_UNSUPPORTED, "the mma.sync kernel serves the simplified von Neumann neighbourhood with FP16 operands");
    if (kernel == CAT_KERNEL_TCGEN05 && (dtype != CAT_DTYPE_FP8_E4M3 || h->rule.C != 2))
      return fail(CAT_ERR_UNSUPPORTED, "the tcgen05 von Neumann kernel serves FP8 operands and two-state rules");
    if (storage == CAT_STORE_BIT1)
      return fail(CAT_ERR_UNSUPPORTED, "one-bit storage is served for the Moore neighbourhood only");
  }
  if (storage == CAT_STORE_BIT1) {
    if (h->rule.C != 2) return fail(CAT_ERR_UNSUPPORTED, "one-bit storage holds two-state rules only");
    if (h->ghost) return fail(CAT_ERR_UNSUPPORTED, "one-bit storage is served with the zero boundary only");
    if ((kernel != CAT_KERNEL_TCGEN05 || dtype == CAT_DTYPE_FP16) && kernel != CAT_KERNEL_BITSLICE)
      return fail(CAT_ERR_UNSUPPORTED, "one-bit storage is served by the tcgen05 kernel with FP8 or FP4 operands "
                                       "and by the bit-sliced kernel");
  }
  if (storage == CAT_STORE_NIB4) {
    if (h->rule.C > 16 || h->ghost || vn || wide)
      return fail(CAT_ERR_UNSUPPORTED, "four-bit storage holds rules with C <= 16, r <= 16, the Moore "
                                       "neighbourhood and the zero boundary");
    if (kernel != CAT_KERNEL_TCGEN05 || dtype == CAT_DTYPE_FP16 || steps_per_launch > 1)
      return fail(CAT_ERR_UNSUPPORTED, "four-bit storage is served by the tcgen05 kernel with FP8 or FP4 operands, "
                                       "one step per launch");
  }
  if (steps_per_launch > 1 && kernel == CAT_KERNEL_BITSLICE) {
    if ((int64_t)steps_per_launch * h->rule.r > 8 || h->H > 65535ll * 32)
      return fail(CAT_ERR_UNSUPPORTED, "the bit-sliced kernel runs k steps per launch for k r <= 8 "
                                       "(and at most 2097120 rows)");
  } else if (steps_per_launch > 1 && (kernel != CAT_KERNEL_TCGEN05 || vn || h->ghost))
    return fail(CAT_ERR_UNSUPPORTED, "several steps per launch are served by the tcgen05 Moore kernel with the zero boundary");
  if (storage != h->storage && !h->owns_buffers)
    return fail(CAT_ERR_UNSUPPORTED, "an instance on bound buffers keeps uint8 storage");
  if (storage != h->storage) {
    int rc = change_storage(h, storage);
    if (rc) return rc;
  }
  h->kernel = kernel;
  h->dtype = dtype;
  h->steps_per_launch = steps_per_launch;
  if (tuned_tile >= 0) {
    h->tile = 0;
    h->window = 0;
    cat_set_tile(h, tuned_tile, tuned_tile, tuned_window);   // a stale entry keeps the radius's own tile
  }
  return CAT_OK;
}

int cat_get_options(cat_handle_t h, int32_t *kernel, int32_t *dtype, int32_t *storage, int32_t *steps_per_launch,
                    int32_t *tile, int32_t *window_rows) {
  if (!h) return fail(CAT_ERR_INVALID_ARG, "handle is NULL");
  if (kernel) *kernel = h->kernel;
  if (dtype) *dtype = h->dtype;
  if (storage) *storage = h->storage;
  if (steps_per_launch) *steps_per_launch = h->steps_per_launch;
  if (tile) *tile = h->kernel == CAT_KERNEL_TCGEN05 && h->rule.nbhd == 'M' ? (wide_tile(h) && !big_window(h) ? 96 : 128) : 0;
  if (window_rows) *window_rows = h->kernel != CAT_KERNEL_TCGEN05 || h->rule.nbhd != 'M' ? 0
                                  : big_window(h) ? 192 : wide_tile(h) ? 0 : short_window(h) ? 144 : 160;
  return CAT_OK;
}

int cat_set_tile(cat_handle_t h, int32_t ty, int32_t tx, int32_t window_rows) {
  if (!h) return fail(CAT_ERR_INVALID_ARG, "handle is NULL");
  const bool t0 = ty == 0 && tx == 0, t128 = ty == 128 && tx == 128, t96 = ty == 96 && tx == 96;
  if (!t0 && !t128 && !t96) return fail(CAT_ERR_INVALID_ARG, "tile %d x %d: choose 0 x 0, 128 x 128 or 96 x 96", ty, tx);
  if (window_rows != 0 && window_rows != 144 && window_rows != 160 && window_rows != 192)
    return fail(CAT_ERR_INVALID_ARG, "window of %d rows: choose 0, 144, 160 or 192", window_rows);
  const bool vn = h->rule.nbhd == 'N';
  if (window_rows == 160 && !t96 && h->rule.r > 16)
    return fail(CAT_ERR_UNSUPPORTED, "the 160-row window serves radii up to 16 on the 128 x 128 tile");
  if (window_rows == 192 && (t96 || h->kernel != CAT_KERNEL_TCGEN05 || vn || h->dtype != CAT_DTYPE_FP8_E4M3 ||
                             h->rule.C != 2 || h->storage != CAT_STORE_U8 || h->ghost || h->steps_per_launch > 1))
    return fail(CAT_ERR_UNSUPPORTED, "the 192-row window serves the 128 x 128 tcgen05 Moore kernel with FP8 operands, "
                                     "two-state rules, uint8 storage, the zero boundary and one step per launch");
  if (t96 && (h->kernel != CAT_KERNEL_TCGEN05 || vn || h->dtype != CAT_DTYPE_FP8_E4M3 || h->rule.C != 2 ||
              h->storage != CAT_STORE_U8 || h->ghost || h->steps_per_launch > 1))
    return fail(CAT_ERR_UNSUPPORTED, "the 96 x 96 tile serves the tcgen05 Moore kernel with FP8 operands, two-state "
                                     "rules, uint8 storage, the zero boundary and one step per launch");
  if (window_rows == 144 && (t96 || h->rule.r > 7 || h->kernel != CAT_KERNEL_TCGEN05 || vn ||
                             h->dtype != CAT_DTYPE_FP8_E4M3 || h->rule.C != 2 || h->storage != CAT_STORE_U8))
    return fail(CAT_ERR_UNSUPPORTED, "the 144-row window serves the 128 x 128 tcgen05 Moore kernel with FP8 "
                                     "operands, two-state rules, uint8 storage and r <= 7");
  if (h->tile != (t0 ? 0 : ty) || h->window != window_rows) drop_plans_with(h);
  h->tile = t0 ? 0 : ty;
  h->window = window_rows;
  return CAT_OK;
}

static int copy2d(void *dst, int64_t dpitch, const void *src, int64_t spitch, int64_t W, int64_t H, cudaStream_t s) {
  if (dpitch == W && spitch == W) {  // both sides contiguous: one linear copy
    CAT_CUDA(cudaMemcpyAsync(dst, src, (size_t)(W * H), cudaMemcpyDefault, s));
  } else {
    CAT_CUDA(cudaMemcpy2DAsync(dst, (size_t)dpitch, src, (size_t)spitch, (size_t)W, (size_t)H, cudaMemcpyDefault, s));
  }
  return CAT_OK;
}

int cat_set_state(cat_handle_t h, const uint8_t *src, int64_t pitch, int32_t src_on_device, void *stream) {
  (void)src_on_device;  // unified addressing tells host and device memory apart
  if (!h || !src) return fail(CAT_ERR_INVALID_ARG, "NULL handle or source");
  if (pitch < h->W) return fail(CAT_ERR_INVALID_ARG, "pitch %lld < W %lld", (long long)pitch, (long long)h->W);
  if (h->storage != CAT_STORE_U8) return bits_set_state(h, src, pitch, (cudaStream_t)stream);
  return copy2d(h->origin(h->cur), h->pitch, src, pitch, h->W, h->H, (cudaStream_t)stream);
}

int cat_get_state(cat_handle_t h, uint8_t *dst, int64_t pitch, int32_t dst_on_device, void *stream) {
  (void)dst_on_device;
  if (!h || !dst) return fail(CAT_ERR_INVALID_ARG, "NULL handle or destination");
  if (pitch < h->W) return fail(CAT_ERR_INVALID_ARG, "pitch %lld < W %lld", (long long)pitch, (long long)h->W);
  if (h->storage != CAT_STORE_U8) return bits_get_state(h, dst, pitch, (cudaStream_t)stream);
  return copy2d(dst, pitch, h->origin(h->cur), h->pitch, h->W, h->H, (cudaStream_t)stream);
}

int cat_state_ptr(cat_handle_t h, void **dptr, int64_t *pitch) {
  if (!h || !dptr || !pitch) return fail(CAT_ERR_INVALID_ARG, "NULL argument");
  *dptr = h->origin(h->cur);
  *pitch = h->pitch;
  return CAT_OK;
}

int cat_step(cat_handle_t h, int64_t n_steps, void *stream) {
  if (!h) return fail(CAT_ERR_INVALID_ARG, "handle is NULL");
  if (n_steps < 0) return fail(CAT_ERR_INVALID_ARG, "n_steps < 0");
  for (int64_t t = 0; t < n_steps;) {
    const int m = (int)std::min<int64_t>(h->steps_per_launch, n_steps - t);
    int rc = launch_step(h, h->cur, nullptr, 0, (cudaStream_t)stream, m);
    if (rc) return rc;
    // the tcgen05 multi-step launch alternates buffers step by step; the
    // blocked bit-sliced launch writes its last step to the other buffer
    h->cur ^= h->kernel == CAT_KERNEL_BITSLICE ? 1 : (m & 1);
    t += m;
  }
  return CAT_OK;
}

int cat_batch_step(const cat_handle_t *hs, int32_t count, int64_t n_steps, void *stream) {
  if (!hs || count < 0 || n_steps < 0) return fail(CAT_ERR_INVALID_ARG, "bad batch arguments");
  for (int32_t i = 0; i < count; ++i) {
    if (!hs[i]) return fail(CAT_ERR_INVALID_ARG, "instance %d is NULL", i);
    for (int32_t k = 0; k < i; ++k)
      if (hs[k] == hs[i]) return fail(CAT_ERR_INVALID_ARG, "instance %d appears twice", i);
  }
  if (count == 0 || n_steps == 0) return CAT_OK;
  cudaStream_t s = (cudaStream_t)stream;
  bool all_tc = true;   // Moore, zero boundary, uint8 storage, no FP4: other instances step one by one
  for (int32_t i = 0; i < count; ++i) {
    all_tc &= hs[i]->kernel == CAT_KERNEL_TCGEN05 && hs[i]->ghost == 0 && hs[i]->storage == CAT_STORE_U8 &&
              hs[i]->rule.nbhd == 'M' && !wide_tile(hs[i]) && hs[i]->dtype != CAT_DTYPE_FP4_E2M1;
    if (hs[i]->dev.id != hs[0]->dev.id) return fail(CAT_ERR_INVALID_ARG, "instances of a batch must share the device");
  }
  if (all_tc) {   // one persistent launch over every instance: one kernel instantiation
    for (int32_t i = 0; i < count; ++i) {
      if (hs[i]->dtype != hs[0]->dtype)
        return fail(CAT_ERR_INVALID_ARG, "instances of a batched tcgen05 launch must share the dtype");
      if (hs[i]->H > 128 * 32767 || hs[i]->W > 128 * 32767)
        return fail(CAT_ERR_UNSUPPORTED, "batched instances are limited to 4194176 x 4194176 cells");
    }
  }
  if (!all_tc) {  // the comparator kernels have no batched launch: one launch per instance and step
    for (int64_t t = 0; t < n_steps; ++t)
      for (int32_t i = 0; i < count; ++i) {
        int rc = launch_step(hs[i], hs[i]->cur, nullptr, 0, s);
        if (rc) return rc;
        hs[i]->cur ^= 1;
      }
    return CAT_OK;
  }
  std::lock_guard<std::mutex> lk(g_plan_mu);
  BatchPlan *pl = nullptr;
  for (BatchPlan *c : g_plans)
    if ((int32_t)c->hs.size() == count && std::equal(c->hs.begin(), c->hs.end(), hs) && c->dtype == hs[0]->dtype) {
      pl = c;
      break;
    }
  int rc;
  if (!pl) {
    if ((rc = build_plan(hs, count, &pl))) return rc;
    g_plans.push_back(pl);
  }
  bool in_sync = true;
  for (int32_t i = 0; i < count; ++i) in_sync &= hs[i]->cur == (pl->cur0[i] ^ (int)(pl->steps_done & 1));
  if (!in_sync && (rc = upload_instances(pl))) return rc;
  const int par = (int)(pl->steps_done & 1);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CAT_CUDA(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone) {
    if ((rc = launch_batch_steps(pl, n_steps, pl->steps_done, s))) return rc;
  } else {
    if (!pl->exec[par] || pl->exec_steps[par] != n_steps) {
      if (pl->exec[par]) cudaGraphExecDestroy(pl->exec[par]);
      pl->exec[par] = nullptr;
      cudaGraph_t g = nullptr;
      CAT_CUDA(cudaStreamBeginCapture(pl->capture_stream, cudaStreamCaptureModeThreadLocal));
      rc = launch_batch_steps(pl, n_steps, pl->steps_done, pl->capture_stream);
      cudaError_t e = cudaStreamEndCapture(pl->capture_stream, &g);
      if (rc) { if (g) cudaGraphDestroy(g); return rc; }
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&pl->exec[par], g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
      pl->exec_steps[par] = n_steps;
    }
    CAT_CUDA(cudaGraphLaunch(pl->exec[par], s));
  }
  pl->steps_done += n_steps;
  for (int32_t i = 0; i < count; ++i) hs[i]->cur ^= (int)(n_steps & 1);
  return CAT_OK;
}

int cat_box_sums(cat_handle_t h, int32_t *dst, int64_t ld, void *stream) {
  if (!h || !dst) return fail(CAT_ERR_INVALID_ARG, "NULL handle or destination");
  if (ld < h->W) return fail(CAT_ERR_INVALID_ARG, "ld < W");
  return launch_step(h, h->cur, dst, ld, (cudaStream_t)stream);
}

int cat_status(cat_handle_t h, void *stream) {
  if (!h) return fail(CAT_ERR_INVALID_ARG, "handle is NULL");
  CAT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  int32_t v = 0;
  CAT_CUDA(cudaMemcpy(&v, h->d_err, sizeof(v), cudaMemcpyDeviceToHost));
  if (v != 0) {
    // the status word and the grid-barrier counter (a launch that gave up
    // left it short of its last target)
    CAT_CUDA(cudaMemset(h->d_err, 0, 2 * sizeof(v)));
    h->gbar_count = 0;
    return fail(CAT_ERR_TIMEOUT, "a device-side wait timed out (code 0x%x)", v);
  }
  return CAT_OK;
}

int cat_debug_control(cat_handle_t h, int32_t what, int64_t value) {
  if (!h) return fail(CAT_ERR_INVALID_ARG, "handle is NULL");
  switch (what) {
    case 1: h->inject = (int32_t)value; return CAT_OK;
    case 2:
      if (value < 1) return fail(CAT_ERR_INVALID_ARG, "timeout must be >= 1 ms");
      h->timeout_ns = (uint64_t)value * 1000000ull;
      return CAT_OK;
    default: return fail(CAT_ERR_INVALID_ARG, "unknown debug control %d", what);
  }
}

int cat_bind(cat_handle_t h, uint8_t *a, uint8_t *b, int64_t pitch) {
  if (!h || !a || !b || a == b) return fail(CAT_ERR_INVALID_ARG, "NULL handle or buffers, or a == b");
  if (pitch < h->W || pitch % 16 != 0) return fail(CAT_ERR_INVALID_ARG, "pitch must be >= W and a multiple of 16");
  if (((uintptr_t)a | (uintptr_t)b) % 16 != 0) return fail(CAT_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
  if (h->ghost || h->storage != CAT_STORE_U8)
    return fail(CAT_ERR_UNSUPPORTED, "bound buffers are served with the zero boundary and uint8 storage");
  cudaPointerAttributes at{}, bt{};
  if (cudaPointerGetAttributes(&at, a) != cudaSuccess || cudaPointerGetAttributes(&bt, b) != cudaSuccess ||
      at.type != cudaMemoryTypeDevice || bt.type != cudaMemoryTypeDevice) {
    (void)cudaGetLastError();
    return fail(CAT_ERR_INVALID_ARG, "buffers must be device memory");
  }
  CAT_CUDA(cudaDeviceSynchronize());
  drop_plans_with(h);
  if (h->owns_buffers) {
    cudaFree(h->buf[0]);
    cudaFree(h->buf[1]);
  }
  h->buf[0] = a;
  h->buf[1] = b;
  h->pitch = pitch;
  h->cur = 0;
  h->owns_buffers = false;
  return build_maps(h);
}

int cat_destroy(cat_handle_t h) {
  if (!h) return CAT_OK;
  cudaDeviceSynchronize();
  drop_plans_with(h);
  if (h->owns_buffers) {
    cudaFree(h->buf[0]);
    cudaFree(h->buf[1]);
  }
  cudaFree(h->d_err);
  delete h;
  return CAT_OK;
}

}  // extern "C"
