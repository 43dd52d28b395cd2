// Test-only translation unit: the bulk asynchronous copy into shared memory and its bounded mbarrier
// wait (mhd_kernels.cuh, used by the FP32 x sweep's row staging), on the GPU.
// tests/test_gpu_xstage.py builds it into a temporary directory; it is not part of libmhd.so.
#include <cuda_runtime.h>

#include "mhd_kernels.cuh"

namespace {
// One block: thread 0 announces n floats plus `extra` bytes on the barrier and copies the n floats
// of src into shared memory; every thread waits (bounded).  status[0] = 1 where the phase completed
// (then out = the copied floats), 2 where the wait gave up.  With extra > 0 no copy can complete
// the phase, so the wait runs out.
__global__ void k_bulk(const float* __restrict__ src, int n, int extra, float* __restrict__ out, int* status) {
  extern __shared__ __align__(16) unsigned char raw[];
  float* buf = reinterpret_cast<float*>(raw + 16);
  const unsigned bar = mhd::smem_u32(raw);
  if (threadIdx.x == 0) mhd::mbar_init(bar);
  __syncthreads();
  if (threadIdx.x == 0) {
    mhd::mbar_arrive_expect(bar, (unsigned)n * 4u + (unsigned)extra);
    mhd::bulk_copy_g2s(mhd::smem_u32(buf), src, (unsigned)n * 4u, bar);
  }
  const bool ok = mhd::mbar_wait_bounded(bar, 0);
  const bool any_timeout = __syncthreads_or(!ok);
  if (threadIdx.x == 0) status[0] = any_timeout ? 2 : 1;
  if (any_timeout) return;
  for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = buf[i];
}
}  // namespace

extern "C" int selftest_bulk(const float* src, int n, int extra, float* out, int* status) {
  if (n <= 0 || n % 4 != 0 || extra < 0 || extra % 16 != 0) return -1;
  const size_t smem = 16 + (size_t)n * 4;
  if (cudaFuncSetAttribute(k_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -2;
  k_bulk<<<1, 128, smem>>>(src, n, extra, out, status);
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : -3;
}
