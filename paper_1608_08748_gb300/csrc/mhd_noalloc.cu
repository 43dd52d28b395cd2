// mhd_noalloc.cu -- FP64 diagnostics over caller-owned device arrays with no device allocation.
//
// Some callers cannot allocate device memory at the moment they want the diagnostics:
//   * code that runs while another component is capturing its stream into a CUDA graph in global
//     capture mode, where cudaMalloc / cudaFree are illegal calls that invalidate the capture;
//   * a serving process that has committed its whole HBM budget to resident simulation state and
//     must not take memory from under the admission controller;
//   * monitors embedded in another application's time loop that share (and must not fragment or
//     synchronise) that application's caching allocator.
// For them this file keeps the block partials of the reduction in a fixed file-scope device array,
// so the call below only launches two kernels.
#include <cuda.h>  // types of the two driver entry points fetched at run time (no libcuda link)
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "mhd.h"
#include "mhd_device.cuh"

namespace mhd_rt {
int set_error(int code, const std::string& msg);  // mhd.cu: message returned by mhd_last_error()
}

namespace {

constexpr int NA_THREADS = 256;
// One 9-value partial per block of 256 cells: MHD_NOALLOC_MAX_CELLS / 256 blocks.
constexpr long long NA_MAX_BLOCKS = MHD_NOALLOC_MAX_CELLS / NA_THREADS;

// Shared by every call on a device and kept between calls (each call rewrites the partials it
// reads, so nothing has to start at zero).  Calls that overlap on the GPU race on this array.
static __device__ __align__(256) double g_partials[NA_MAX_BLOCKS * 9];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_mutex;
// Per device: the address of g_partials and the id of the context it was looked up in.  A device
// reset destroys that context and loads the module again at another address, so the address is
// only reused while the same context (by its process-unique id) is current.
double* g_ptr[NA_MAX_DEVICES] = {nullptr};
unsigned long long g_ctx_id[NA_MAX_DEVICES] = {0};

// cuCtxGetCurrent and cuCtxGetId, fetched from the driver through the runtime, so that the library
// does not link libcuda itself (it still loads on a machine without a driver)
typedef CUresult (*ctx_get_current_fn)(CUcontext*);
typedef CUresult (*ctx_get_id_fn)(CUcontext, unsigned long long*);
ctx_get_current_fn g_ctx_get_current = nullptr;
ctx_get_id_fn g_ctx_get_id = nullptr;

// id of the current context (0 if none is current or the driver does not tell)
unsigned long long current_context_id() {
  if (!g_ctx_get_current || !g_ctx_get_id) {
    cudaDriverEntryPointQueryResult q1, q2;
    void* f1 = nullptr;
    void* f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
      cudaGetLastError();
      return 0;
    }
    g_ctx_get_current = (ctx_get_current_fn)f1;
    g_ctx_get_id = (ctx_get_id_fn)f2;
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}


__device__ __forceinline__ long long na_up(int i, int j, int k, int d, const int n[3], const int bc[3]) {
  int c[3] = {i, j, k};
  c[d] += 1;
  int a = mhd::wrap(c[0], n[0], bc[0]), b = mhd::wrap(c[1], n[1], bc[1]), e = mhd::wrap(c[2], n[2], bc[2]);
  return ((long long)e * n[1] + b) * n[0] + a;
}

// Same arithmetic and block tree as the diagnostics of a simulation, on raw FP64 arrays.
__global__ void __launch_bounds__(NA_THREADS)
k_na_partial(const double* rho, const double* mx, const double* my, const double* mz, const double* E,
             const double* bx, const double* by, const double* bz, int nx, int ny, int nz, int bcx,
             int bcy, int bcz, double* part) {
  __shared__ double sh[9][NA_THREADS];
  const int n[3] = {nx, ny, nz}, bc[3] = {bcx, bcy, bcz};
  const long long N = (long long)nx * ny * nz;
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (c < N) {
    int i = (int)(c % nx);
    long long r = c / nx;
    int j = (int)(r % ny);
    int k = (int)(r / ny);
    v[0] = rho[c];
    v[1] = mx[c];
    v[2] = my[c];
    v[3] = mz[c];
    v[4] = E[c];
    v[5] = bx[c];
    v[6] = by[c];
    v[7] = bz[c];
    double div = (bx[na_up(i, j, k, 0, n, bc)] - bx[c]) + (by[na_up(i, j, k, 1, n, bc)] - by[c]) +
                 (bz[na_up(i, j, k, 2, n, bc)] - bz[c]);
    v[8] = fabs(div);
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) sh[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int w = NA_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
#pragma unroll
      for (int q = 0; q < 8; ++q) sh[q][threadIdx.x] = sh[q][threadIdx.x] + sh[q][threadIdx.x + w];
      sh[8][threadIdx.x] = fmax(sh[8][threadIdx.x], sh[8][threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x < 9) part[(long long)blockIdx.x * 9 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(NA_THREADS) k_na_final(const double* part, int nblocks, double* out) {
  __shared__ double sh[9][NA_THREADS];
  double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblocks; b += NA_THREADS) {
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = v[q] + part[(long long)b * 9 + q];
    v[8] = fmax(v[8], part[(long long)b * 9 + 8]);
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) sh[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int w = NA_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
#pragma unroll
      for (int q = 0; q < 8; ++q) sh[q][threadIdx.x] = sh[q][threadIdx.x] + sh[q][threadIdx.x + w];
      sh[8][threadIdx.x] = fmax(sh[8][threadIdx.x], sh[8][threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x < 9) out[threadIdx.x] = sh[threadIdx.x][0];
}

// Device address of g_partials on the current device, looked up once per device (and again after
// the device's context was replaced, as by cudaDeviceReset).  In host code the name g_partials is
// only a host-side stand-in, never a device address.
int scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return mhd_rt::set_error(MHD_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= NA_MAX_DEVICES) return mhd_rt::set_error(MHD_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mutex);
  const unsigned long long id = current_context_id();
  if (!g_ptr[dev] || id == 0 || id != g_ctx_id[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_partials);  // creates the context if none is current yet
    if (e != cudaSuccess || p == nullptr)
      return mhd_rt::set_error(MHD_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_ptr[dev] = p;
    g_ctx_id[dev] = current_context_id();
  }
  *out = g_ptr[dev];
  return MHD_OK;
}

}  // namespace

extern "C" int mhd_diagnostics_noalloc(const double* rho, const double* mx, const double* my,
                                       const double* mz, const double* E, const double* bx,
                                       const double* by, const double* bz, int nx, int ny, int nz,
                                       int bc_x, int bc_y, int bc_z, double* out, void* stream) {
  if (!rho || !mx || !my || !mz || !E || !bx || !by || !bz || !out)
    return mhd_rt::set_error(MHD_EINVAL, "mhd_diagnostics_noalloc: null pointer");
  if (nx < 1 || ny < 1 || nz < 1)
    return mhd_rt::set_error(MHD_EINVAL, "mhd_diagnostics_noalloc: need nx, ny, nz >= 1");
  const long long N = (long long)nx * ny * nz;
  if (N > MHD_NOALLOC_MAX_CELLS)
    return mhd_rt::set_error(MHD_EINVAL, "mhd_diagnostics_noalloc: " + std::to_string(N) +
                                             " cells exceed the fixed maximum of " +
                                             std::to_string((long long)MHD_NOALLOC_MAX_CELLS));
  if ((bc_x != 0 && bc_x != 1) || (bc_y != 0 && bc_y != 1) || (bc_z != 0 && bc_z != 1))
    return mhd_rt::set_error(MHD_EINVAL, "mhd_diagnostics_noalloc: boundary flags must be 0 or 1");
  double* part = nullptr;
  int rc = scratch_for_current_device(&part);
  if (rc != MHD_OK) return rc;
  const int nblocks = (int)((N + NA_THREADS - 1) / NA_THREADS);
  cudaStream_t st = (cudaStream_t)stream;
  k_na_partial<<<nblocks, NA_THREADS, 0, st>>>(rho, mx, my, mz, E, bx, by, bz, nx, ny, nz, bc_x, bc_y,
                                               bc_z, part);
  k_na_final<<<1, NA_THREADS, 0, st>>>(part, nblocks, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return mhd_rt::set_error(MHD_ECUDA, std::string("mhd_diagnostics_noalloc launch: ") + cudaGetErrorString(e));
  return MHD_OK;
}
