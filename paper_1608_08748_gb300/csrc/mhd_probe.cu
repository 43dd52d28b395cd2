// mhd_probe.cu -- measured arithmetic peaks of the current GPU, for the roofline denominators of
// the kernels whose bound is an arithmetic pipe rather than HBM (the FP64 faces of the FP64 step,
// the FP32 faces of the FP32-bulk step).  A grid of independent FMA chains, timed with CUDA events.
#include <cuda_runtime.h>

#include <string>

#include "mhd.h"

namespace mhd_rt {
int set_error(int code, const std::string& msg);  // mhd.cu: message returned by mhd_last_error()
}

namespace {

// CHAINS independent dependent-FMA chains per thread; every chain's value is stored, so none can
// be dropped.  a * x + b with |a| < 1 keeps the values finite for any iteration count.
template <typename T, int CHAINS>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T a, T b, T* out) {
  T x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = fma(a, x[c], b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int probe(int iters, double* tflops) {
  constexpr int CHAINS = 8, THREADS = 256;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return mhd_rt::set_error(MHD_ECUDA, std::string("probe: ") + cudaGetErrorString(e));
  const int blocks = nsm * 8;  // eight blocks of 256 per SM: enough warps to hide the FMA latency
  T* out = nullptr;
  if ((e = cudaMalloc(&out, sizeof(T) * (size_t)blocks * THREADS)) != cudaSuccess)
    return mhd_rt::set_error(MHD_ENOMEM, std::string("probe: ") + cudaGetErrorString(e));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {  // the first launch warms up; the best of the rest counts
    cudaEventRecord(e0);
    k_fma_chains<T, CHAINS><<<blocks, THREADS>>>(iters, (T)0.999, (T)1e-3, out);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return mhd_rt::set_error(MHD_ECUDA, std::string("probe: ") + cudaGetErrorString(e));
  const double flops = 2.0 * CHAINS * (double)iters * THREADS * blocks;
  *tflops = flops / (best * 1e-3) / 1e12;
  return MHD_OK;
}

}  // namespace

extern "C" int mhd_probe_fma_peak(int fp64, int iters, double* tflops) {
  if (!tflops || iters < 1 || (fp64 != 0 && fp64 != 1))
    return mhd_rt::set_error(MHD_EINVAL, "mhd_probe_fma_peak: need fp64 in {0, 1}, iters >= 1, tflops");
  return fp64 ? probe<double>(iters, tflops) : probe<float>(iters, tflops);
}
