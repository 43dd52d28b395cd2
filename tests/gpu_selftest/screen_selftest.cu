// Test-only translation unit: the chemistry's table-driven exponential and the CFL screen's FP32
// estimate (mhd_device.cuh) on the GPU, next to the library exp and the FP64 denominator of the
// same inputs.  tests/test_gpu_screen.py builds it twice, with the FP64 path's compile flags and
// with the FP32-bulk path's (flush to zero, approximate division and square root), into a temporary
// directory; it is not part of libmhd.so.
#include <cuda_runtime.h>

#include "mhd_device.cuh"

namespace {
// out[2 i] = exp_tang(x), out[2 i + 1] = exp(x)
__global__ void k_selftest_exp(const double* __restrict__ x, int n, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[2 * (size_t)i] = mhd::exp_tang(x[i]);
  out[2 * (size_t)i + 1] = exp(x[i]);
}

// in[12 i + k]: rho, m_x, m_y, m_z, B_x, B_y, B_z, rho eps, rho_H2, rho_H+, gamma, chem (0 or 1);
// out[2 i] = the FP32 estimate (+inf where a guard fails), out[2 i + 1] = the FP64 denominator
__global__ void k_selftest_screen(const double* __restrict__ in, int n, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* w = in + 12 * (size_t)i;
  const bool chem = w[11] != 0.0;
  const float gm1 = mhd::gamma_minus_one_f32(chem, w[10], (float)w[0], (float)w[8], (float)w[9]);
  out[2 * (size_t)i] = mhd::cfl_estimate_f32((float)w[0], (float)w[1], (float)w[2], (float)w[3], (float)w[4],
                                             (float)w[5], (float)w[6], (float)w[7], gm1);
  const double gm = chem ? mhd::gamma_eff(w[0], w[8], w[9]) : w[10];
  out[2 * (size_t)i + 1] = mhd::cfl_denominator(w[0], w[1], w[2], w[3], w[4], w[5], w[6], gm * ((gm - 1.0) * w[7]));
}

int finish() {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return (int)e;
}
}  // namespace

// device pointers: x (n doubles), out (2 n doubles); synchronises; 0 on success, else the CUDA
// error code
extern "C" int selftest_exp(const double* x, int n, double* out) {
  if (n <= 0) return 0;
  k_selftest_exp<<<(n + 255) / 256, 256>>>(x, n, out);
  return finish();
}

// device pointers: in (12 n doubles), out (2 n doubles); synchronises; 0 on success, else the CUDA
// error code
extern "C" int selftest_screen(const double* in, int n, double* out) {
  if (n <= 0) return 0;
  k_selftest_screen<<<(n + 255) / 256, 256>>>(in, n, out);
  return finish();
}
