// Allocation-free batched step: cat_batch_step_static (include/cat.h).
//
// The batched tcgen05 kernel needs a per-grid descriptor table and a tile
// work-list in device memory.  cat_batch_step keeps them in memory it
// allocates; this entry point keeps them instead in one file-scope
// __device__ array of fixed size, so that callers who cannot allocate device
// memory can still run a batch.  Every call reuses the same array.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/cat.h"
#include "cat_internal.h"

namespace {

struct StaticScratch {
  cat::BatchInst inst[CAT_STATIC_MAX_GRIDS];
  cat::BatchTile tiles[CAT_STATIC_MAX_TILES];
};
static_assert(sizeof(StaticScratch) == 753664, "the size include/cat.h states");

// The scratch lives in device memory for as long as the library is loaded.
// In host code `g_scratch` only names the symbol; its device address comes
// from cudaGetSymbolAddress (done once per device in scratch_address).
static __device__ __align__(256) StaticScratch g_scratch;

constexpr int kMaxDevices = 64;

struct DeviceSlot {
  StaticScratch *ptr = nullptr;
  int sms = 0;
};

std::mutex g_mu;  // guards g_slots and the host staging copy below
DeviceSlot g_slots[kMaxDevices];
StaticScratch g_host_stage;  // host image of the table, copied before each launch

int err(int code, const char *fmt, long long a = 0, long long b = 0) {
  char buf[256];
  snprintf(buf, sizeof(buf), fmt, a, b);
  return cat::host_fail(code, buf);
}

// Device address of the scratch on the current device (set up on first use).
int scratch_address(DeviceSlot **slot) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return err(CAT_ERR_CUDA, "cudaGetDevice failed");
  if (dev < 0 || dev >= kMaxDevices) return err(CAT_ERR_UNSUPPORTED, "device index %lld out of range", dev);
  DeviceSlot &s = g_slots[dev];
  if (!s.ptr) {
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3)
      return err(CAT_ERR_UNSUPPORTED, "device is sm_%lld%lld; this library is built for sm_103a", major, minor);
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) return err(CAT_ERR_CUDA, "cudaGetSymbolAddress failed (%lld)", (long long)e);
    e = cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return err(CAT_ERR_CUDA, "cudaDeviceGetAttribute failed (%lld)", (long long)e);
    s.ptr = static_cast<StaticScratch *>(p);
  }
  *slot = &s;
  return CAT_OK;
}

// Bytes of grid memory a descriptor's buffer spans: rows 0 .. H-1 at `pitch`.
uintptr_t span(int64_t H, int64_t W, int64_t pitch) { return (uintptr_t)((H - 1) * pitch + W); }

bool overlap(uintptr_t a, uintptr_t na, uintptr_t b, uintptr_t nb) { return a < b + nb && b < a + na; }

}  // namespace

extern "C" CAT_API int cat_batch_step_static(const cat_grid_desc_t *grids, int32_t count, int32_t dtype,
                                             int32_t *d_status, void *stream) {
  if (!grids || count < 1) return err(CAT_ERR_INVALID_ARG, "need at least one grid");
  if (count > CAT_STATIC_MAX_GRIDS)
    return err(CAT_ERR_INVALID_ARG, "%lld grids exceed the static limit of %lld", count, CAT_STATIC_MAX_GRIDS);
  if (!d_status) return err(CAT_ERR_INVALID_ARG, "d_status is NULL: a timed-out launch could not be reported");
  if (dtype == CAT_DTYPE_AUTO) dtype = CAT_DTYPE_FP8_E4M3;
  if (dtype != CAT_DTYPE_FP8_E4M3 && dtype != CAT_DTYPE_FP16)
    return err(CAT_ERR_UNSUPPORTED, "dtype %lld: only FP8 and FP16 operands are served here", dtype);
  int64_t n_tiles = 0;
  bool encode = false;
  for (int32_t i = 0; i < count; ++i) {
    const cat_grid_desc_t &g = grids[i];
    if (!g.in || !g.out || g.in == g.out) return err(CAT_ERR_INVALID_ARG, "grid %lld: NULL or aliased buffers", i);
    if (g.H < 1 || g.W < 1 || g.H > 128 * 32767 || g.W > 128 * 32767)
      return err(CAT_ERR_INVALID_ARG, "grid %lld: size outside [1, 4194176]", i);
    if (g.pitch < g.W || g.pitch % 16 != 0)
      return err(CAT_ERR_INVALID_ARG, "grid %lld: pitch must be >= W and a multiple of 16", i);
    if (((uintptr_t)g.in | (uintptr_t)g.out) % 16 != 0)
      return err(CAT_ERR_INVALID_ARG, "grid %lld: buffers must be 16-byte aligned", i);
    int rc = cat::host_validate_rule(&g.rule);
    if (rc) return rc;
    if (g.rule.nbhd != 'M') return err(CAT_ERR_UNSUPPORTED, "grid %lld: the static batch serves the Moore neighbourhood", i);
    if (g.rule.r > 16) return err(CAT_ERR_UNSUPPORTED, "grid %lld: the static batch serves radii up to 16", i);
    encode |= g.rule.C > 2;
    n_tiles += ((g.H + 127) / 128) * ((g.W + 127) / 128);
  }
  if (n_tiles > CAT_STATIC_MAX_TILES)
    return err(CAT_ERR_INVALID_ARG, "%lld tiles of 128 x 128 cells exceed the static limit of %lld", n_tiles,
               CAT_STATIC_MAX_TILES);
  // one persistent launch steps every grid at once: a grid's output may share
  // no byte with another grid's input or output (inputs may share bytes)
  for (int32_t i = 0; i < count; ++i) {
    const cat_grid_desc_t &g = grids[i];
    const uintptr_t o = (uintptr_t)g.out, no = span(g.H, g.W, g.pitch);
    for (int32_t j = 0; j < count; ++j) {
      const cat_grid_desc_t &k = grids[j];
      const uintptr_t nk = span(k.H, k.W, k.pitch);
      if (overlap(o, no, (uintptr_t)k.in, nk) || (j != i && overlap(o, no, (uintptr_t)k.out, nk)))
        return err(CAT_ERR_INVALID_ARG, "grid %lld writes memory that grid %lld also uses", i, j);
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  {
    // the table is staged from host memory that the next call overwrites, so
    // a captured copy would replay stale contents: refuse capture
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return err(CAT_ERR_CUDA, "cudaStreamIsCapturing failed (%lld)", (long long)e);
    if (cs != cudaStreamCaptureStatusNone)
      return err(CAT_ERR_INVALID_ARG, "cat_batch_step_static may not be captured into a CUDA graph");
  }

  std::lock_guard<std::mutex> lk(g_mu);
  DeviceSlot *slot = nullptr;
  int rc = scratch_address(&slot);
  if (rc) return rc;
  StaticScratch &h = g_host_stage;
  int32_t *status = d_status;
  int64_t t = 0;
  // work-list ordered by radius (the kernel rebuilds its band when r changes)
  for (int r = 1; r <= 16; ++r)
    for (int32_t i = 0; i < count; ++i) {
      if (grids[i].rule.r != r) continue;
      const int64_t ty = (grids[i].H + 127) / 128, tx = (grids[i].W + 127) / 128;
      for (int64_t y = 0; y < ty; ++y)
        for (int64_t x = 0; x < tx; ++x) h.tiles[t++] = cat::BatchTile{i, (int16_t)y, (int16_t)x};
    }
  for (int32_t i = 0; i < count; ++i) {
    const cat_grid_desc_t &g = grids[i];
    cat::BatchInst &I = h.inst[i];
    memset(&I, 0, sizeof(I));
    // buffer 0 = g.in (read, also as centre tiles), buffer 1 = g.out (written): cur = 0, parity 0
    if ((rc = cat::host_make_map(&I.map_in_a[0], (void *)g.in, g.H, g.W, g.pitch, 128, 160, 1))) return rc;
    if ((rc = cat::host_make_map(&I.map_in_b[0], (void *)g.in, g.H, g.W, g.pitch, 32, 160, 0))) return rc;
    if ((rc = cat::host_make_map(&I.map_out[0], (void *)g.in, g.H, g.W, g.pitch, 128, 128, 1))) return rc;
    if ((rc = cat::host_make_map(&I.map_out[1], g.out, g.H, g.W, g.pitch, 128, 128, 1))) return rc;
    I.rule = cat::host_reduce_rule(g.rule);
    I.H = (int32_t)g.H;
    I.W = (int32_t)g.W;
    I.cur = 0;
    I.err = status;
  }
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(slot->ptr->inst, h.inst, sizeof(cat::BatchInst) * count, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(slot->ptr->tiles, h.tiles, sizeof(cat::BatchTile) * n_tiles, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return err(CAT_ERR_CUDA, "staging the batch table failed (%lld)", (long long)e);
  cat::TcParams p;
  memset(&p, 0, sizeof(p));
  p.n_tiles = (int32_t)n_tiles;
  p.timeout_ns = 2000000000ull;
  p.parity = 0;
  p.binst = slot->ptr->inst;
  p.btiles = slot->ptr->tiles;
  const int grid = (int)(n_tiles < slot->sms ? n_tiles : slot->sms);
  e = cat::tc_launch_batch(p, dtype, encode, false, grid, s);
  if (e != cudaSuccess) return err(CAT_ERR_CUDA, "batched launch failed (%lld)", (long long)e);
  // the host image is copied from pageable memory: the copies have consumed it
  // before cudaMemcpyAsync returned, so the next call may overwrite it
  return CAT_OK;
}
