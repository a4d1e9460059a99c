// Autotuner: chooses the kernel, operand dtype, tile shape, window and steps
// per launch of an instance (or of a batch) by timing the candidates the
// instance's rule, storage and boundary allow, on its own state, with CUDA
// events; the choice is kept in a JSON-lines cache file keyed by the grid's
// shape, radius, number of states, neighbourhood, boundary, storage and GPU.
//
// Every candidate computes the same next states (all kernels are exact), so
// the choice only affects speed.  The tuner is a client of the C ABI: it sets
// options with cat_set_options / cat_set_tile, saves and restores the state
// with cat_get_state / cat_set_state, and steps with cat_step /
// cat_batch_step.  The paper tunes its tile shape by hand (Sec. V-B); this is
// the GB300 build's measured replacement.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cat.h"
#include "cat_internal.h"

namespace cat {
namespace {

struct Cand {
  int32_t kernel, dtype, tile, window, spl;
};

std::string cache_key(const InstanceInfo &f) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, dev);
  for (char *c = prop.name; *c; ++c)
    if (*c == '"' || *c == '\\') *c = '_';
  char buf[384];
  snprintf(buf, sizeof(buf), "H=%lld W=%lld r=%d C=%d nbhd=%c boundary=%d storage=%d gpu=%s/%d",
           (long long)f.H, (long long)f.W, f.rule.r, f.rule.C, (char)f.rule.nbhd, f.boundary, f.storage, prop.name,
           prop.multiProcessorCount);
  return buf;
}

// The last entry for `key` in the JSON-lines file at `path`.
bool cache_read(const char *path, const std::string &key, Cand *out, double *rate) {
  FILE *fp = path ? fopen(path, "r") : nullptr;
  if (!fp) return false;
  const std::string pat = "\"key\": \"" + key + "\"";
  char line[1024];
  bool found = false;
  while (fgets(line, sizeof(line), fp)) {
    const char *k = strstr(line, pat.c_str());
    if (!k) continue;
    Cand c{};
    double v = 0;
    const char *o = strstr(k, "\"kernel\"");
    if (o && sscanf(o, "\"kernel\": %d, \"dtype\": %d, \"tile\": %d, \"window\": %d, \"steps_per_launch\": %d, "
                       "\"cell_updates_per_s\": %lf",
                    &c.kernel, &c.dtype, &c.tile, &c.window, &c.spl, &v) == 6) {
      *out = c;
      if (rate) *rate = v;
      found = true;
    }
  }
  fclose(fp);
  return found;
}

void cache_write(const char *path, const std::string &key, const Cand &c, double rate) {
  FILE *fp = path ? fopen(path, "a") : nullptr;
  if (!fp) return;
  fprintf(fp,
          "{\"key\": \"%s\", \"kernel\": %d, \"dtype\": %d, \"tile\": %d, \"window\": %d, \"steps_per_launch\": %d, "
          "\"cell_updates_per_s\": %.6e}\n",
          key.c_str(), c.kernel, c.dtype, c.tile, c.window, c.spl, rate);
  fclose(fp);
}

// Sets every option of `h` to candidate c; false (options left unspecified)
// when the instance cannot run it.
bool apply(cat_handle_t h, const InstanceInfo &f, const Cand &c) {
  if (cat_set_tile(h, 0, 0, 0) != CAT_OK) return false;
  if (cat_set_options(h, c.kernel, c.dtype, f.storage, c.spl) != CAT_OK) return false;
  return cat_set_tile(h, c.tile, c.tile, c.window) == CAT_OK;
}

std::vector<Cand> candidates(const InstanceInfo &f) {
  std::vector<Cand> out;
  for (int spl : {1, 4, 16}) {
    for (int dt : {CAT_DTYPE_FP8_E4M3, CAT_DTYPE_FP16}) {
      out.push_back({CAT_KERNEL_TCGEN05, dt, 128, 160, spl});
      if (f.rule.r <= 7) out.push_back({CAT_KERNEL_TCGEN05, dt, 128, 144, spl});
      out.push_back({CAT_KERNEL_TCGEN05, dt, 96, 0, spl});
      out.push_back({CAT_KERNEL_TCGEN05, dt, 128, 192, spl});
    }
  }
  out.push_back({CAT_KERNEL_TCGEN05, CAT_DTYPE_FP4_E2M1, 128, 160, 1});
  out.push_back({CAT_KERNEL_MMA_SYNC, CAT_DTYPE_FP16, 0, 0, 1});
  out.push_back({CAT_KERNEL_MMA_SYNC, CAT_DTYPE_INT8, 0, 0, 1});
  out.push_back({CAT_KERNEL_STENCIL, CAT_DTYPE_AUTO, 0, 0, 1});
  out.push_back({CAT_KERNEL_RUNSUM, CAT_DTYPE_AUTO, 0, 0, 1});
  for (int spl : {1, 2, 4, 8}) out.push_back({CAT_KERNEL_BITSLICE, CAT_DTYPE_AUTO, 0, 0, spl});
  return out;
}

int cuda_err(cudaError_t e, const char *what) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  return host_fail(CAT_ERR_CUDA, buf);
}

}  // namespace

bool tune_cache_lookup_env(const InstanceInfo &info, int32_t *kernel, int32_t *dtype, int32_t *tile, int32_t *window,
                           int32_t *spl) {
  const char *path = getenv("CAT_AUTOTUNE_CACHE");
  Cand c{};
  if (!path || !*path || !cache_read(path, cache_key(info), &c, nullptr)) return false;
  *kernel = c.kernel;
  *dtype = c.dtype;
  *tile = c.tile;
  *window = c.window;
  *spl = c.spl;
  return true;
}

}  // namespace cat

using cat::Cand;

extern "C" CAT_API int cat_autotune(cat_handle_t h, int32_t n_steps, const char *cache_path, int32_t flags,
                                    void *stream) {
  if (!h) return cat::host_fail(CAT_ERR_INVALID_ARG, "handle is NULL");
  if (n_steps < 1 || n_steps > 1 << 20) return cat::host_fail(CAT_ERR_INVALID_ARG, "n_steps must be in [1, 2^20]");
  cat::InstanceInfo f{};
  int rc = cat::host_instance_info(h, &f);
  if (rc) return rc;
  const std::string key = cat::cache_key(f);
  Cand best{};
  double best_rate = 0;
  if (!(flags & CAT_TUNE_REMEASURE) && cat::cache_read(cache_path, key, &best, &best_rate) &&
      cat::apply(h, f, best))
    return CAT_OK;
  const Cand before{f.kernel, f.dtype, f.tile, f.window, f.steps_per_launch};
  cudaStream_t s = (cudaStream_t)stream;
  // the state is saved once and restored before every candidate and at the end
  uint8_t *saved = nullptr;
  cudaError_t e = cudaMalloc(&saved, (size_t)(f.H * f.W));
  if (e != cudaSuccess) return cat::cuda_err(e, "cat_autotune");
  if ((rc = cat_get_state(h, saved, f.W, 1, stream))) { cudaFree(saved); return rc; }
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  bool any = false;
  for (const Cand &c : cat::candidates(f)) {
    if (!cat::apply(h, f, c)) continue;
    const int64_t steps = (n_steps + c.spl - 1) / c.spl * c.spl;
    if (cat_set_state(h, saved, f.W, 1, stream) || cat_step(h, c.spl, stream) || cudaEventRecord(a, s) ||
        cat_step(h, steps, stream) || cudaEventRecord(b, s) || cudaEventSynchronize(b))
      continue;
    float ms = 0;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess || ms <= 0 || cat_status(h, stream) != CAT_OK) continue;
    const double rate = (double)f.H * (double)f.W * (double)steps / (ms * 1e-3);
    if (rate > best_rate) {
      best_rate = rate;
      best = c;
      any = true;
    }
  }
  (void)cudaGetLastError();
  rc = CAT_OK;
  if (!any) rc = cat::host_fail(CAT_ERR_UNSUPPORTED, "no candidate configuration ran");
  if (!cat::apply(h, f, any ? best : before)) rc = rc ? rc : cat::host_fail(CAT_ERR_STATE, "restoring options failed");
  const int rs = cat_set_state(h, saved, f.W, 1, stream);
  e = cudaStreamSynchronize(s);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(saved);
  if (rs) return rs;
  if (e != cudaSuccess) return cat::cuda_err(e, "cat_autotune");
  if (rc == CAT_OK && !(flags & CAT_TUNE_NO_WRITE)) cat::cache_write(cache_path, key, best, best_rate);
  return rc;
}

extern "C" CAT_API int cat_autotune_batch(const cat_handle_t *hs, int32_t count, int32_t n_steps, int32_t *chosen_dtype,
                                          void *stream) {
  if (!hs || count < 1 || n_steps < 1) return cat::host_fail(CAT_ERR_INVALID_ARG, "bad batch arguments");
  std::vector<cat::InstanceInfo> fs(count);
  size_t total = 0;
  for (int32_t i = 0; i < count; ++i) {
    int rc = cat::host_instance_info(hs[i], &fs[i]);
    if (rc) return rc;
    total += (size_t)(fs[i].H * fs[i].W);
  }
  cudaStream_t s = (cudaStream_t)stream;
  uint8_t *saved = nullptr;
  cudaError_t e = cudaMalloc(&saved, total);
  if (e != cudaSuccess) return cat::cuda_err(e, "cat_autotune_batch");
  auto each_state = [&](bool save) -> int {
    size_t off = 0;
    for (int32_t i = 0; i < count; ++i) {
      int rc = save ? cat_get_state(hs[i], saved + off, fs[i].W, 1, stream)
                    : cat_set_state(hs[i], saved + off, fs[i].W, 1, stream);
      if (rc) return rc;
      off += (size_t)(fs[i].H * fs[i].W);
    }
    return CAT_OK;
  };
  int rc = each_state(true);
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  Cand best{};
  double best_ms = 0;
  bool any = false;
  // one configuration for every instance: a batch shares kernel and dtype
  const Cand cands[] = {{CAT_KERNEL_TCGEN05, CAT_DTYPE_FP8_E4M3, 0, 0, 1},
                        {CAT_KERNEL_TCGEN05, CAT_DTYPE_FP8_E4M3, 0, 160, 1},
                        {CAT_KERNEL_TCGEN05, CAT_DTYPE_FP16, 0, 0, 1}};
  for (const Cand &c : cands) {
    if (rc) break;
    bool ok = true;
    for (int32_t i = 0; i < count && ok; ++i) ok = cat::apply(hs[i], fs[i], c);
    if (!ok || each_state(false) || cat_batch_step(hs, count, n_steps, stream) || cudaEventRecord(a, s) ||
        cat_batch_step(hs, count, n_steps, stream) || cudaEventRecord(b, s) || cudaEventSynchronize(b))
      continue;
    float ms = 0;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess || ms <= 0) continue;
    if (!any || ms < best_ms) {
      best_ms = ms;
      best = c;
      any = true;
    }
  }
  (void)cudaGetLastError();
  if (!rc && !any) rc = cat::host_fail(CAT_ERR_UNSUPPORTED, "no candidate configuration ran");
  if (any)
    for (int32_t i = 0; i < count; ++i)
      if (!cat::apply(hs[i], fs[i], best) && !rc) rc = cat::host_fail(CAT_ERR_STATE, "applying the choice failed");
  const int rs = each_state(false);
  e = cudaStreamSynchronize(s);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(saved);
  if (rc) return rc;
  if (rs) return rs;
  if (e != cudaSuccess) return cat::cuda_err(e, "cat_autotune_batch");
  if (chosen_dtype) *chosen_dtype = best.dtype;
  return CAT_OK;
}
