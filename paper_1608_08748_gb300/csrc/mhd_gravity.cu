// mhd_gravity.cu -- self-gravity of a periodic box: the Sec. 2.10 solution of the Poisson equation
// Delta Phi = 4 pi G rho in harmonic space with the 27-point scheme,
//   Phi_jmn = -(2/3) pi G h^2 rho_jmn / (1 - c_j c_m c_n),  c_j = (3 - 2 sin^2(pi j / N)) / 3,
// the mean mode set to zero (the potential of the periodic box), by cuFFT real-to-complex and
// complex-to-real transforms on the sim's stream.  The Eulerian update takes -grad Phi by central
// differences (mhd_kernels.cuh).
#include <cufft.h>

#include <cmath>
#include <string>
#include <vector>

#include "mhd_runtime.cuh"

namespace mhd_rt {
// index-check flags of the Poisson-solve kernels (MHD_CHECK builds)
unsigned check_flags_gravity(bool clear) { return check_flags_of_this_unit(clear); }
}  // namespace mhd_rt

using namespace mhd;
using namespace mhd_rt;

namespace mhd_rt {
int set_error(int code, const std::string& msg);  // mhd.cu: message returned by mhd_last_error()
}

namespace {

struct Gravity {
  int precision = -1;
  int n[3] = {0, 0, 0};
  cufftHandle fwd = 0, inv = 0;
  bool plans = false;
  void* spec = nullptr;    // nz x ny x (nx/2 + 1) complex
  void* phi = nullptr;     // nz x ny x nx real potential
  double* tab = nullptr;   // c_j of the three axes: nx/2 + 1, ny, nz values
};

void release(Gravity* G) {
  if (G->plans) {
    cufftDestroy(G->fwd);
    cufftDestroy(G->inv);
  }
  G->plans = false;
  if (G->spec) cudaFree(G->spec);
  if (G->phi) cudaFree(G->phi);
  if (G->tab) cudaFree(G->tab);
  G->spec = G->phi = nullptr;
  G->tab = nullptr;
}

// spectrum x= coef / (1 - c_i c_j c_k), the (0, 0, 0) mode zero; coef = -(2/3) pi G h^2 / N (the
// 1/N of the unnormalised inverse transform folded in)
template <typename C>
__global__ void k_poisson_symbol(C* spec, const double* tab, int nxh, int ny, int nz, double coef) {
  const long long total = (long long)nxh * ny * nz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % nxh);
    const int j = (int)((t / nxh) % ny);
    const int k = (int)(t / ((long long)nxh * ny));
    double f = 0.0;
    if (i != 0 || j != 0 || k != 0) {
      const double cc = (tab[i] * tab[nxh + j]) * tab[nxh + ny + k];
      f = coef / (1.0 - cc);
    }
    spec[t].x = spec[t].x * f;
    spec[t].y = spec[t].y * f;
  }
}

int gfail(int code, const std::string& msg) { return mhd_rt::set_error(code, msg); }

}  // namespace

namespace mhd_rt {

// allocate the transforms and buffers of a sim with self-gravity on (idempotent) and point its box
// descriptor at the potential; returns MHD_OK or an error code
int grav_prepare(mhd_sim* S) {
  Gravity* G = static_cast<Gravity*>(S->grav);
  if (!G) {
    G = new Gravity();
    S->grav = G;
  }
  const int nx = S->g.n[0], ny = S->g.n[1], nz = S->g.n[2];
  if (G->plans && G->precision == S->precision && G->n[0] == nx && G->n[1] == ny && G->n[2] == nz) {
    const void* want = G->phi;
    const void* have = S->precision ? (const void*)S->b32.phi : (const void*)S->b64.phi;
    if (want == have) return MHD_OK;
  }
  release(G);
  const size_t N = (size_t)nx * ny * nz, NC = (size_t)(nx / 2 + 1) * ny * nz;
  const size_t es = S->precision ? sizeof(float) : sizeof(double);
  if (cudaMalloc(&G->spec, NC * 2 * es) != cudaSuccess || cudaMalloc(&G->phi, N * es) != cudaSuccess ||
      cudaMalloc(&G->tab, sizeof(double) * (size_t)(nx / 2 + 1 + ny + nz)) != cudaSuccess) {
    cudaGetLastError();
    release(G);
    return gfail(MHD_ENOMEM, "self-gravity: device allocation failed");
  }
  if (cufftPlan3d(&G->fwd, nz, ny, nx, S->precision ? CUFFT_R2C : CUFFT_D2Z) != CUFFT_SUCCESS) {
    release(G);
    return gfail(MHD_ECUDA, "self-gravity: cufftPlan3d (forward) failed");
  }
  if (cufftPlan3d(&G->inv, nz, ny, nx, S->precision ? CUFFT_C2R : CUFFT_Z2D) != CUFFT_SUCCESS) {
    cufftDestroy(G->fwd);
    release(G);
    return gfail(MHD_ECUDA, "self-gravity: cufftPlan3d (inverse) failed");
  }
  G->plans = true;
  // c_j = (3 - 2 sin^2(pi j / N)) / 3 of each axis (x: the j <= nx/2 of the half spectrum)
  std::vector<double> h;
  for (int j = 0; j <= nx / 2; ++j) {
    const double s = std::sin(M_PI * j / nx);
    h.push_back((3.0 - 2.0 * s * s) / 3.0);
  }
  for (int j = 0; j < ny; ++j) {
    const double s = std::sin(M_PI * j / ny);
    h.push_back((3.0 - 2.0 * s * s) / 3.0);
  }
  for (int j = 0; j < nz; ++j) {
    const double s = std::sin(M_PI * j / nz);
    h.push_back((3.0 - 2.0 * s * s) / 3.0);
  }
  if (cudaMemcpy(G->tab, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return gfail(MHD_ECUDA, "self-gravity: table upload failed");
  G->precision = S->precision;
  G->n[0] = nx;
  G->n[1] = ny;
  G->n[2] = nz;
  if (S->precision)
    S->b32.phi = static_cast<const float*>(G->phi);
  else
    S->b64.phi = static_cast<const double*>(G->phi);
  S->exec_valid = false;  // the box descriptor changed
  S->graph_valid = false;
  return MHD_OK;
}

// enqueue the potential of the current density on the sim's stream
int grav_solve(mhd_sim* S) {
  Gravity* G = static_cast<Gravity*>(S->grav);
  if (!G || !G->plans) return gfail(MHD_EINVAL, "self-gravity: not prepared");
  const int nx = S->g.n[0], ny = S->g.n[1], nz = S->g.n[2];
  const double N = (double)nx * ny * nz;
  const double coef = -(2.0 / 3.0) * M_PI * S->ph.grav_g * S->ph.dx * S->ph.dx / N;
  if (cufftSetStream(G->fwd, S->stream) != CUFFT_SUCCESS || cufftSetStream(G->inv, S->stream) != CUFFT_SUCCESS)
    return gfail(MHD_ECUDA, "self-gravity: cufftSetStream failed");
  const long long total = (long long)(nx / 2 + 1) * ny * nz;
  const unsigned blocks = (unsigned)std::min<long long>((total + 255) / 256, 4096);
  if (S->precision) {
    if (cufftExecR2C(G->fwd, S->b32.s.rho, static_cast<cufftComplex*>(G->spec)) != CUFFT_SUCCESS)
      return gfail(MHD_ECUDA, "self-gravity: forward transform failed");
    k_poisson_symbol<<<blocks, 256, 0, S->stream>>>(static_cast<cufftComplex*>(G->spec), G->tab, nx / 2 + 1, ny,
                                                   nz, coef);
    if (cufftExecC2R(G->inv, static_cast<cufftComplex*>(G->spec), static_cast<float*>(G->phi)) != CUFFT_SUCCESS)
      return gfail(MHD_ECUDA, "self-gravity: inverse transform failed");
  } else {
    if (cufftExecD2Z(G->fwd, S->b64.s.rho, static_cast<cufftDoubleComplex*>(G->spec)) != CUFFT_SUCCESS)
      return gfail(MHD_ECUDA, "self-gravity: forward transform failed");
    k_poisson_symbol<<<blocks, 256, 0, S->stream>>>(static_cast<cufftDoubleComplex*>(G->spec), G->tab, nx / 2 + 1,
                                                   ny, nz, coef);
    if (cufftExecZ2D(G->inv, static_cast<cufftDoubleComplex*>(G->spec), static_cast<double*>(G->phi)) != CUFFT_SUCCESS)
      return gfail(MHD_ECUDA, "self-gravity: inverse transform failed");
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return gfail(MHD_ECUDA, std::string("self-gravity: ") + cudaGetErrorString(e));
  return MHD_OK;
}

// copy the potential of the last solve out (interior cells, x fastest), host or device pointer
int grav_copy(mhd_sim* S, double* out) {
  Gravity* G = static_cast<Gravity*>(S->grav);
  if (!G || !G->plans) return gfail(MHD_EINVAL, "self-gravity: not prepared");
  const size_t N = (size_t)S->g.N;
  if (S->precision) {
    std::vector<float> f(N);
    if (cudaMemcpyAsync(f.data(), G->phi, N * sizeof(float), cudaMemcpyDeviceToHost, S->stream) != cudaSuccess ||
        cudaStreamSynchronize(S->stream) != cudaSuccess)
      return gfail(MHD_ECUDA, "self-gravity: potential read-back failed");
    for (size_t i = 0; i < N; ++i) out[i] = f[i];
  } else {
    if (cudaMemcpyAsync(out, G->phi, N * sizeof(double), cudaMemcpyDefault, S->stream) != cudaSuccess ||
        cudaStreamSynchronize(S->stream) != cudaSuccess)
      return gfail(MHD_ECUDA, "self-gravity: potential read-back failed");
  }
  return MHD_OK;
}

void grav_free(mhd_sim* S) {
  Gravity* G = static_cast<Gravity*>(S->grav);
  if (!G) return;
  release(G);
  delete G;
  S->grav = nullptr;
}

}  // namespace mhd_rt
