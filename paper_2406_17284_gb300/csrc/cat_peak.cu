// Dense tcgen05 MMA throughput probe: the denominator of the roofline's
// tensor term.
//
// The roofline of a step is the slower of two bounds: the state bytes at the
// HBM copy rate, and the band products' flops at the operand dtype's dense
// tensor rate.  The second needs the e4m3 and f16 rates of this GPU's
// tcgen05 MMAs as this library issues them, so this kernel measures them: one
// CTA per SM, one thread issuing back-to-back M = 128, N = 256 MMAs (K = 32
// e4m3 or K = 16 f16 elements, f32 accumulators in tensor memory, both
// operands in shared memory, K-major, 128B swizzle), the largest shape a
// single CTA issues.  The operands are zero: only the rate matters.  The
// caller times the launch; one launch performs
//   SMs x mmas_per_sm x 2 x 128 x 256 x K   flops.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/cat.h"
#include "cat_internal.h"
#include "ptx.cuh"

namespace cat {
namespace {

constexpr int kProbeN = 256;
constexpr uint32_t kProbeA = 128 * 128;                 // 128 rows x 128 bytes
constexpr uint32_t kProbeB = kProbeN * 128;             // 256 rows x 128 bytes
// more shared memory than two CTAs could share, so that every SM runs one CTA
constexpr uint32_t kProbeDyn = 150 * 1024;
static_assert(kProbeA + kProbeB + 64 + 1024 <= kProbeDyn, "probe layout");

template <int KIND>
__device__ __forceinline__ void probe_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (KIND == 0) mma_f16(d, a, b, idesc, acc);
  else mma_f8f6f4(d, a, b, idesc, acc);
}

// KIND 0: kind::f16 (f16 operands, K = 16); KIND 1: kind::f8f6f4 (e4m3, K = 32);
// KIND 2: kind::f8f6f4 with e2m1 operands (K = 32).
template <int KIND>
__global__ void __launch_bounds__(128, 1) mma_probe_kernel(int64_t n_mma, uint64_t timeout_ns, int32_t *err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *done = reinterpret_cast<uint64_t *>(smem + kProbeA + kProbeB);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
  int *abort = reinterpret_cast<int *>(done + 2);
  for (uint32_t i = threadIdx.x; i < (kProbeA + kProbeB) / 16; i += blockDim.x)
    reinterpret_cast<uint4 *>(smem)[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    mbar_init(done, 1);
    *abort = 0;
    fence_mbar_init();
  }
  if (threadIdx.x < 32) {
    tmem_alloc(tmem_slot, kProbeN);
    tmem_relinquish();
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  if (threadIdx.x == 0) {
    const uint32_t base = smem_u32(smem);
    const uint64_t a = smem_desc(base, 16, 1024, kSwizzle128B);
    const uint64_t b = smem_desc(base + kProbeA, 16, 1024, kSwizzle128B);
    const uint32_t idesc = idesc_f32acc(128, kProbeN) | (KIND == 2 ? kIdescE2M1 : 0u);
    probe_mma<KIND>(tmem, a, b, idesc, 0);
    int64_t i = 1;
    for (; i + 8 <= n_mma; i += 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) probe_mma<KIND>(tmem, a, b, idesc, 1);
    }
    for (; i < n_mma; ++i) probe_mma<KIND>(tmem, a, b, idesc, 1);
    mma_commit(done);
  }
  __syncwarp();   // warp 0 waits as one warp once its lane 0 has issued
  // every thread waits for the MMAs before the tensor memory is freed
  const bool ok = mbar_wait(done, 0, abort, timeout_ns);
  if (!ok && err) atomicCAS(err, 0, kDevErrTimeout | 16);
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tmem_dealloc(tmem, kProbeN);
  }
}

}  // namespace
}  // namespace cat

extern "C" CAT_API int cat_tensor_probe(int32_t dtype, int64_t mmas_per_sm, int32_t *d_status, void *stream) {
  if (dtype != CAT_DTYPE_FP8_E4M3 && dtype != CAT_DTYPE_FP16 && dtype != CAT_DTYPE_FP4_E2M1)
    return cat::host_fail(CAT_ERR_UNSUPPORTED, "the tensor probe measures FP8 e4m3, FP4 e2m1 and FP16 MMAs");
  if (mmas_per_sm < 1 || mmas_per_sm > (int64_t)1 << 30)
    return cat::host_fail(CAT_ERR_INVALID_ARG, "mmas_per_sm must be in [1, 2^30]");
  if (!d_status) return cat::host_fail(CAT_ERR_INVALID_ARG, "d_status is NULL");
  int dev = 0, sms = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
    return cat::host_fail(CAT_ERR_CUDA, "device query failed");
  if (major != 10 || minor != 3) return cat::host_fail(CAT_ERR_UNSUPPORTED, "this library is built for sm_103a");
  cudaStream_t s = (cudaStream_t)stream;
  void (*kern)(int64_t, uint64_t, int32_t *) =
      dtype == CAT_DTYPE_FP16 ? cat::mma_probe_kernel<0>
    : dtype == CAT_DTYPE_FP4_E2M1 ? cat::mma_probe_kernel<2> : cat::mma_probe_kernel<1>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cat::kProbeDyn);
  // the bounded wait: 1 us per MMA (over ten times its duration) plus 1 s
  const uint64_t timeout_ns = 1000000000ull + (uint64_t)mmas_per_sm * 1000ull;
  if (e == cudaSuccess) {
    kern<<<sms, 128, cat::kProbeDyn, s>>>(mmas_per_sm, timeout_ns, d_status);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cat::host_fail(CAT_ERR_CUDA, cudaGetErrorString(e));
  return CAT_OK;
}
