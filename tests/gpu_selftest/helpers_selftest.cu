// Test-only translation unit: runs the FP64 path's arithmetic helpers (mhd_device.cuh) over an
// array of doubles on the GPU, so that tests/test_gpu_helpers.py can check them element by element
// against their definitions.  Built by that test with nvcc into a temporary directory; it is not
// part of libmhd.so.
#include <cuda_runtime.h>

#include "mhd_device.cuh"

namespace {
// out[8 i + k]: k = 0 |x|, 1 -x, 2 x / 2, 3 x / 4, 4 the ordered key of x (its bits), 5 1/x,
// 6 1/sqrt(|x|), 7 sqrt(|x|)
__global__ void k_selftest_helpers(const double* __restrict__ x, int n, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i], a = fabs(v);
  double* o = out + 8 * (size_t)i;
  o[0] = mhd::abs_b(v);
  o[1] = mhd::neg_b(v);
  o[2] = mhd::scale_down_b<1>(v);
  o[3] = mhd::scale_down_b<2>(v);
  o[4] = __longlong_as_double(mhd::okey(v));
  o[5] = mhd::rcp_nr(v);
  o[6] = mhd::rsqrt_nr(a);
  o[7] = mhd::sqrt_nr(a);
}
}  // namespace

// x and out are device pointers (n and 8 n doubles); synchronises; 0 on success, else the CUDA
// error code
extern "C" int selftest_helpers(const double* x, int n, double* out) {
  if (n <= 0) return 0;
  k_selftest_helpers<<<(n + 255) / 256, 256>>>(x, n, out);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return (int)e;
}
