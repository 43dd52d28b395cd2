// mhd.cu -- C ABI (include/mhd.h) and host runtime of the GB300 MHD + H/H2 chemistry step.
// The host only allocates, enqueues and (optionally) captures the launches of a step into a CUDA
// graph; tau, t and all per-step scalars live in device memory.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mhd.h"
#include "mhd_runtime.cuh"

using namespace mhd;
using namespace mhd_rt;

namespace {

thread_local std::string g_err;
thread_local int g_err_code = MHD_OK;

int fail(int code, const std::string& msg) {
  g_err = msg;
  g_err_code = code;
  return code;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) return fail(MHD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

namespace mhd_rt {
unsigned check_flags_f32(bool clear);      // mhd_f32.cu
unsigned check_flags_gravity(bool clear);  // mhd_gravity.cu
// record the message mhd_last_error() returns on this thread; returns code
int set_error(int code, const std::string& msg) { return fail(code, msg); }
// the code of the last failure recorded on this thread (for calls that return a pointer)
int last_error_code() { return g_err_code; }
}  // namespace mhd_rt

namespace {

size_t pool_size(const Geom& g, int precision, int chem) {
  (void)chem;
  size_t es = precision ? sizeof(float) : sizeof(double);
  size_t cells = (size_t)g.N, faces = (size_t)g.NF;
  // state 11, Q^n 11, primitives 9 (cells); face outputs 3 x 8 and edges 3 (lattice)
  return es * (cells * 31 + faces * 27) + 64 * 64;
}

// lay the box's arrays out in the pool and fill its descriptor
template <typename T>
void carve(mhd_sim* S, Box<T>& B) {
  char* p = S->pool;
  auto take = [&](size_t n) {
    T* r = reinterpret_cast<T*>(p);
    size_t bytes = (n * sizeof(T) + 255) & ~size_t(255);
    p += bytes;
    return r;
  };
  const size_t N = (size_t)S->g.N, NF = (size_t)S->g.NF;
  State<T>* st[2] = {&B.s, &B.s0};
  for (State<T>* s : st) {
    s->rho = take(N);
    for (int d = 0; d < 3; ++d) s->m[d] = take(N);
    s->E = take(N);
    s->eint = take(N);
    s->rh2 = take(N);
    s->rhp = take(N);
    for (int d = 0; d < 3; ++d) s->b[d] = take(N);
  }
  for (int d = 0; d < 3; ++d) B.w.v[d] = take(N);
  for (int d = 0; d < 3; ++d) B.w.B[d] = take(N);
  B.w.p = take(N);
  B.w.g = take(N);
  B.w.sr = take(N);
  for (int d = 0; d < 3; ++d)
    for (int v = 0; v < 8; ++v) B.fo[d].f[v] = take(NF);
  for (int d = 0; d < 3; ++d) B.e[d] = take(NF);
  B.phi = nullptr;
  B.hflags = S->hflags_dev;
  B.g = S->g;
  B.ph = S->ph;
  B.sc = S->sc;
  B.nv = S->ph.chem ? (S->ph.ions ? 8 : 7) : 6;
}

// (re)build the single-box executor after a change of options
template <typename T>
int rebuild_exec(mhd_sim* S, Box<T>& B, Exec<T>& X) {
  B.g = S->g;
  B.ph = S->ph;
  B.sc = S->sc;
  B.nv = S->ph.chem ? (S->ph.ions ? 8 : 7) : 6;
  exec_free(X);
  X.prof = &S->prof;
  cudaError_t e = exec_init(X, std::vector<Box<T>>{B});
  X.x_stage = S->x_stage != 0;
  if (e != cudaSuccess) return fail(MHD_ECUDA, std::string("executor set-up: ") + cudaGetErrorString(e));
  return MHD_OK;
}

int ensure_exec(mhd_sim* S) {
  if (S->exec_valid) return MHD_OK;
  int rc = S->precision ? rebuild_exec(S, S->b32, S->x32) : rebuild_exec(S, S->b64, S->x64);
  if (rc == MHD_OK) S->exec_valid = true;
  S->graph_valid = false;
  return rc;
}

int alloc_pool(mhd_sim* S) {
  if (S->pool) cudaFree(S->pool);
  S->pool = nullptr;
  size_t bytes = pool_size(S->g, S->precision, S->ph.chem) + 256 * 64;
  if (cudaMalloc(&S->pool, bytes) != cudaSuccess) {
    cudaGetLastError();
    S->pool = nullptr;
    return fail(MHD_ENOMEM, "cudaMalloc of the field pool failed (" + std::to_string(bytes) + " bytes)");
  }
  S->pool_bytes = bytes;
  CK(cudaMemsetAsync(S->pool, 0, bytes, S->stream));
  if (S->precision)
    carve(S, S->b32);
  else
    carve(S, S->b64);
  S->graph_valid = false;
  S->exec_valid = false;
  S->has_state = false;
  return ensure_exec(S);
}

void drop_graph(mhd_sim* S) {
  if (S->gexec) cudaGraphExecDestroy(S->gexec);
  S->gexec = nullptr;
  S->graph_valid = false;
}

void launch_sim_step(mhd_sim* S) {
  if (S->precision)
    launch_step(S->x32, S->stream);
  else
    launch_step(S->x64, S->stream);
}

int enqueue_step(mhd_sim* S) {
  int rc;
  const bool grav = S->ph.grav_g > 0.0;
  if (grav) {
    if (S->g.bc[0] || S->g.bc[1] || S->g.bc[2]) return fail(MHD_EINVAL, "self-gravity needs periodic boundaries");
    if ((rc = grav_prepare(S)) != MHD_OK) return rc;
  }
  rc = ensure_exec(S);
  if (rc != MHD_OK) return rc;
  if (grav) {
    // the potential of rho^n (stage 7 of the previous step), then the step; launched directly, so
    // the cuFFT transforms stay outside a captured graph
    if ((rc = grav_solve(S)) != MHD_OK) return rc;
    launch_sim_step(S);
    CK(cudaGetLastError());
    return MHD_OK;
  }
  if (S->use_graph) {
    if (!S->graph_valid) {
      drop_graph(S);
      cudaGraph_t graph;
      CK(cudaStreamBeginCapture(S->stream, cudaStreamCaptureModeThreadLocal));
      launch_sim_step(S);
      cudaError_t e = cudaStreamEndCapture(S->stream, &graph);
      if (e != cudaSuccess) return fail(MHD_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      e = cudaGraphInstantiate(&S->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return fail(MHD_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
      S->graph_valid = true;
    }
    CK(cudaGraphLaunch(S->gexec, S->stream));
  } else {
    launch_sim_step(S);
    CK(cudaGetLastError());
  }
  return MHD_OK;
}

int set_params(mhd_sim* S, double cfl, double t_end, int fixed_tau, double tau) {
  int rc = ensure_exec(S);
  if (rc != MHD_OK) return rc;
  CK(S->precision ? launch_set_params(S->x32, S->stream, cfl, t_end, fixed_tau, tau)
                  : launch_set_params(S->x64, S->stream, cfl, t_end, fixed_tau, tau));
  return MHD_OK;
}

int read_scalars(mhd_sim* S) {
  CK(cudaMemcpyAsync(S->sc_host, S->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  return MHD_OK;
}

int refresh_cfl(mhd_sim* S) {
  int rc = ensure_exec(S);
  if (rc != MHD_OK) return rc;
  CK(S->precision ? launch_cfl(S->x32, S->stream) : launch_cfl(S->x64, S->stream));
  return MHD_OK;
}

size_t dtype_size(int dt) { return dt == MHD_F32 ? 4 : 8; }

// The device address of a host buffer that kernels can read and write in place: page-locked
// memory (cudaMallocHost, cudaHostAlloc) or memory registered with cudaHostRegister; nullptr for
// pageable memory.  On GB300 the GPU reaches such memory over NVLink-C2C, so the load and store
// kernels take it directly instead of a copy through the staging buffer.
const void* mapped_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  return a.devicePointer;
}

int reset_scalars(mhd_sim* S) {
  CK(cudaMemsetAsync(S->sc, 0, sizeof(Scalars), S->stream));
  S->params_dirty = true;
  return MHD_OK;
}

bool valid(const mhd_sim* S) { return S != nullptr && S->pool != nullptr; }

}  // namespace

// ================================================================================================
extern "C" {

const char* mhd_last_error(void) { return g_err.c_str(); }

size_t mhd_bytes_needed(int nx, int ny, int nz, int precision, int chem) {
  Geom g;
  g.n[0] = nx;
  g.n[1] = ny;
  g.n[2] = nz;
  g.N = (long long)nx * ny * nz;
  g.NF = (long long)(nx + 1) * (ny + 1) * (nz + 1);
  set_divisors(g);
  return pool_size(g, precision, chem) + (size_t)g.N * 10 * 8 + sizeof(Scalars) +
         ((size_t)g.N / 256 + 2) * 9 * 8;
}

mhd_sim* mhd_create(int nx, int ny, int nz, double gamma, double dx) {
  if (nx < 1 || ny < 1 || nz < 1 || !(gamma > 1.0) || !(dx > 0.0)) {
    fail(MHD_EINVAL, "mhd_create: need nx, ny, nz >= 1, gamma > 1, dx > 0");
    return nullptr;
  }
  if ((long long)(nx + 1) * (ny + 1) * (nz + 1) >= (1ll << 31)) {
    fail(MHD_EINVAL, "mhd_create: grid too large (the (nx+1)(ny+1)(nz+1) lattice must stay below 2^31)");
    return nullptr;
  }
  mhd_sim* S = new (std::nothrow) mhd_sim();
  if (!S) {
    fail(MHD_ENOMEM, "mhd_create: host allocation failed");
    return nullptr;
  }
  S->g.n[0] = nx;
  S->g.n[1] = ny;
  S->g.n[2] = nz;
  S->g.bc[0] = S->g.bc[1] = S->g.bc[2] = 0;
  S->g.N = (long long)nx * ny * nz;
  S->g.NF = (long long)(nx + 1) * (ny + 1) * (nz + 1);
  set_divisors(S->g);
  S->ph.gamma = gamma;
  S->ph.dx = dx;
  S->ph.ih = 1.0 / dx;
  S->ph.chem = 0;
  S->ph.regul_mode = 0;
  S->ph.lshield = 0.0;
  S->ph.bdop = 3.0;
  S->ph.xnorm = 5e14;
  S->ph.ibdop = 1.0 / 3.0;
  S->ph.ixnorm = 1.0 / 5e14;
  S->ph.taud = 1e-21;
  mhd::set_shielding(S->ph);
  S->ph.heatcool = 0;
  S->ph.grav_g = 0.0;
  S->ph.ions = 0;
  auto bail = [&](const char* what, cudaError_t e) {
    fail(e == cudaErrorMemoryAllocation ? MHD_ENOMEM : MHD_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    mhd_destroy(S);
    return (mhd_sim*)nullptr;
  };
  cudaError_t e;
  if ((e = cudaGetDevice(&S->device)) != cudaSuccess) return bail("cudaGetDevice", e);
  if ((e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking)) != cudaSuccess)
    return bail("cudaStreamCreate", e);
  S->own_stream = true;
  if ((e = cudaMalloc(&S->sc, sizeof(Scalars))) != cudaSuccess) return bail("cudaMalloc(scalars)", e);
  if ((e = cudaMallocHost(&S->sc_host, sizeof(Scalars))) != cudaSuccess) return bail("cudaMallocHost", e);
  S->diag_blocks = (int)nblk(S->g.N, DIAG_THREADS);
  if ((e = cudaMalloc(&S->diag_part, (size_t)S->diag_blocks * 9 * sizeof(double) + 16 * sizeof(double))) != cudaSuccess)
    return bail("cudaMalloc(diag)", e);
  S->diag_out = S->diag_part + (size_t)S->diag_blocks * 9;
  if ((e = cudaMallocHost(&S->diag_host, 16 * sizeof(double))) != cudaSuccess) return bail("cudaMallocHost(diag)", e);
  if ((e = cudaMalloc(&S->staging, (size_t)S->g.N * 10 * 8)) != cudaSuccess) return bail("cudaMalloc(staging)", e);
  if ((e = cudaHostAlloc((void**)&S->hflags_host, sizeof(int), cudaHostAllocMapped)) != cudaSuccess)
    return bail("cudaHostAlloc(flags)", e);
  *(volatile int*)S->hflags_host = 0;
  if ((e = cudaHostGetDevicePointer((void**)&S->hflags_dev, S->hflags_host, 0)) != cudaSuccess)
    return bail("cudaHostGetDevicePointer(flags)", e);
  if (alloc_pool(S) != MHD_OK) {
    std::string msg = g_err;
    const int code = g_err_code;
    mhd_destroy(S);
    g_err = msg;
    g_err_code = code;
    return nullptr;
  }
  if (reset_scalars(S) != MHD_OK || cudaStreamSynchronize(S->stream) != cudaSuccess) {
    mhd_destroy(S);
    return nullptr;
  }
  return S;
}

void mhd_destroy(mhd_sim* S) {
  if (!S) return;
  if (S->stream) cudaStreamSynchronize(S->stream);
  drop_graph(S);
  exec_free(S->x64);
  exec_free(S->x32);
  grav_free(S);
  if (S->pool) cudaFree(S->pool);
  if (S->staging) cudaFree(S->staging);
  if (S->sc) cudaFree(S->sc);
  if (S->sc_host) cudaFreeHost(S->sc_host);
  if (S->diag_part) cudaFree(S->diag_part);
  if (S->diag_host) cudaFreeHost(S->diag_host);
  if (S->hflags_host) cudaFreeHost(S->hflags_host);
  if (S->own_stream && S->stream) cudaStreamDestroy(S->stream);
  delete S;
}

int mhd_set_option(mhd_sim* S, int key, double v) {
  if (!valid(S)) return fail(MHD_EINVAL, "mhd_set_option: null sim");
  switch (key) {
    case MHD_OPT_BC_X:
    case MHD_OPT_BC_Y:
    case MHD_OPT_BC_Z:
      if (v != 0.0 && v != 1.0) return fail(MHD_EINVAL, "boundary must be 0 (periodic) or 1 (outflow)");
      S->g.bc[key - MHD_OPT_BC_X] = (int)v;
      break;
    case MHD_OPT_CHEM:
      S->ph.chem = v != 0.0;
      break;
    case MHD_OPT_PRECISION:
      if (v != 0.0 && v != 1.0) return fail(MHD_EINVAL, "precision must be 0 (FP64) or 1 (FP32 bulk)");
      if ((int)v != S->precision) {
        S->precision = (int)v;
        int rc = alloc_pool(S);
        if (rc != MHD_OK) return rc;
      }
      break;
    case MHD_OPT_REGUL_MODE:
      if (v != 0.0 && v != 1.0 && v != 2.0) return fail(MHD_EINVAL, "regularisation mode must be 0, 1 or 2");
      S->ph.regul_mode = (int)v;
      break;
    case MHD_OPT_CHEM_LSHIELD:
      if (v < 0.0) return fail(MHD_EINVAL, "shielding length must be >= 0");
      S->ph.lshield = v;
      mhd::set_shielding(S->ph);
      break;
    case MHD_OPT_CHEM_BDOP:
      if (!(v > 0.0)) return fail(MHD_EINVAL, "Doppler parameter must be > 0");
      S->ph.bdop = v;
      S->ph.ibdop = 1.0 / v;
      break;
    case MHD_OPT_CHEM_XNORM:
      if (!(v > 0.0)) return fail(MHD_EINVAL, "x normaliser must be > 0");
      S->ph.xnorm = v;
      S->ph.ixnorm = 1.0 / v;
      mhd::set_shielding(S->ph);
      break;
    case MHD_OPT_CHEM_TAUD:
      if (v < 0.0) return fail(MHD_EINVAL, "dust opacity must be >= 0");
      S->ph.taud = v;
      mhd::set_shielding(S->ph);
      break;
    case MHD_OPT_GRAPH:
      S->use_graph = v != 0.0;
      break;
    case MHD_OPT_HEATCOOL:
      if (v != 0.0 && v != 1.0) return fail(MHD_EINVAL, "heating/cooling must be 0 (off) or 1 (on)");
      S->ph.heatcool = (int)v;
      break;
    case MHD_OPT_GRAV_G:
      if (!(v >= 0.0)) return fail(MHD_EINVAL, "the gravitational constant must be >= 0");
      S->ph.grav_g = v;
      break;
    case MHD_OPT_IONS:
      if (v != 0.0 && v != 1.0) return fail(MHD_EINVAL, "ions must be 0 (off) or 1 (on)");
      S->ph.ions = (int)v;
      break;
    case MHD_OPT_X_STAGE:
      if (v != 0.0 && v != 1.0) return fail(MHD_EINVAL, "x staging must be 0 (off) or 1 (on)");
      S->x_stage = (int)v;
      break;
    default:
      return fail(MHD_EINVAL, "unknown option key " + std::to_string(key));
  }
  S->graph_valid = false;  // kernel arguments are baked into the captured graph
  S->exec_valid = false;   // and the box descriptor into the executor
  return MHD_OK;
}

int mhd_set_stream(mhd_sim* S, void* stream) {
  if (!valid(S)) return fail(MHD_EINVAL, "mhd_set_stream: null sim");
  CK(cudaStreamSynchronize(S->stream));
  if (S->own_stream) cudaStreamDestroy(S->stream);
  S->stream = (cudaStream_t)stream;
  S->own_stream = false;
  return MHD_OK;
}

int mhd_set_state(mhd_sim* S, const mhd_fields* in) {
  if (!valid(S) || !in) return fail(MHD_EINVAL, "mhd_set_state: null argument");
  if (in->dtype != MHD_F64 && in->dtype != MHD_F32) return fail(MHD_EINVAL, "mhd_set_state: bad dtype");
  const void* src[9] = {in->rho, in->mom[0], in->mom[1], in->mom[2], in->E, in->B[0], in->B[1], in->B[2], in->rho_h2};
  for (int q = 0; q < 8; ++q)
    if (!src[q]) return fail(MHD_EINVAL, "mhd_set_state: rho, mom[3], E and B[3] are required");
  const size_t es = dtype_size(in->dtype), bytes = (size_t)S->g.N * es;
  const void* dev[9];
  for (int q = 0; q < 9; ++q) {
    if (!src[q]) {
      dev[q] = nullptr;
      continue;
    }
    if (in->on_device) {
      dev[q] = src[q];
    } else if (const void* m = mapped_host(src[q])) {
      dev[q] = m;  // page-locked: the load kernels read it in place
    } else {
      void* dst = S->staging + (size_t)q * S->g.N * 8;
      CK(cudaMemcpyAsync(dst, src[q], bytes, cudaMemcpyHostToDevice, S->stream));
      dev[q] = dst;
    }
  }
  int rc;
  if (in->dtype == MHD_F64) {
    const double* p[9];
    for (int q = 0; q < 9; ++q) p[q] = (const double*)dev[q];
    CK(S->precision ? load_state(S, S->b32, p) : load_state(S, S->b64, p));
  } else {
    const float* p[9];
    for (int q = 0; q < 9; ++q) p[q] = (const float*)dev[q];
    CK(S->precision ? load_state(S, S->b32, p) : load_state(S, S->b64, p));
  }
  if ((rc = reset_scalars(S)) != MHD_OK) return rc;
  if ((rc = refresh_cfl(S)) != MHD_OK) return rc;
  CK(cudaStreamSynchronize(S->stream));
  *(volatile int*)S->hflags_host = 0;  // the steps before this load are finished
  S->has_state = true;
  return MHD_OK;
}

int mhd_set_face_B(mhd_sim* S, const double* bx, const double* by, const double* bz, int on_device) {
  if (!valid(S) || !bx || !by || !bz) return fail(MHD_EINVAL, "mhd_set_face_B: null argument");
  const size_t bytes = (size_t)S->g.N * 8;
  const double* src[3] = {bx, by, bz};
  const double* dev[3];
  for (int q = 0; q < 3; ++q) {
    if (on_device) {
      dev[q] = src[q];
    } else {
      double* dst = (double*)(S->staging + (size_t)q * bytes);
      CK(cudaMemcpyAsync(dst, src[q], bytes, cudaMemcpyHostToDevice, S->stream));
      dev[q] = dst;
    }
  }
  CK(S->precision ? set_faces(S, S->b32, dev) : set_faces(S, S->b64, dev));
  int rc = refresh_cfl(S);
  if (rc != MHD_OK) return rc;
  CK(cudaStreamSynchronize(S->stream));
  return MHD_OK;
}

int mhd_get_state(mhd_sim* S, mhd_fields* out) {
  if (!valid(S) || !out) return fail(MHD_EINVAL, "mhd_get_state: null argument");
  if (out->dtype != MHD_F64 && out->dtype != MHD_F32) return fail(MHD_EINVAL, "mhd_get_state: bad dtype");
  void* dst[9] = {out->rho, out->mom[0], out->mom[1], out->mom[2], out->E, out->B[0], out->B[1], out->B[2], out->rho_h2};
  for (int q = 0; q < 8; ++q)
    if (!dst[q]) return fail(MHD_EINVAL, "mhd_get_state: rho, mom[3], E and B[3] are required");
  const size_t es = dtype_size(out->dtype), bytes = (size_t)S->g.N * es;
  void* dev[9];
  bool in_place[9];
  for (int q = 0; q < 9; ++q) {
    in_place[q] = false;
    if (!dst[q]) {
      dev[q] = nullptr;
    } else if (out->on_device) {
      dev[q] = dst[q];
    } else if (const void* m = mapped_host(dst[q])) {
      dev[q] = const_cast<void*>(m);  // page-locked: the store kernel writes it in place
      in_place[q] = true;
    } else {
      dev[q] = (void*)(S->staging + (size_t)q * S->g.N * 8);
    }
  }
  if (out->dtype == MHD_F64) {
    double* p[9];
    for (int q = 0; q < 9; ++q) p[q] = (double*)dev[q];
    CK(S->precision ? store_state(S, S->b32, p) : store_state(S, S->b64, p));
  } else {
    float* p[9];
    for (int q = 0; q < 9; ++q) p[q] = (float*)dev[q];
    CK(S->precision ? store_state(S, S->b32, p) : store_state(S, S->b64, p));
  }
  if (!out->on_device)
    for (int q = 0; q < 9; ++q)
      if (dst[q] && !in_place[q]) CK(cudaMemcpyAsync(dst[q], dev[q], bytes, cudaMemcpyDeviceToHost, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  return MHD_OK;
}

int mhd_get_full(mhd_sim* S, double* eint, double* bx, double* by, double* bz, int on_device) {
  if (!valid(S) || !eint || !bx || !by || !bz) return fail(MHD_EINVAL, "mhd_get_full: null argument");
  const size_t bytes = (size_t)S->g.N * 8;
  double* dst[4] = {eint, bx, by, bz};
  double* dev[4];
  for (int q = 0; q < 4; ++q) dev[q] = on_device ? dst[q] : (double*)(S->staging + q * bytes);
  CK(S->precision ? store_full(S, S->b32, dev) : store_full(S, S->b64, dev));
  if (!on_device)
    for (int q = 0; q < 4; ++q) CK(cudaMemcpyAsync(dst[q], dev[q], bytes, cudaMemcpyDeviceToHost, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  return MHD_OK;
}

int mhd_get_ions(mhd_sim* S, double* rho_hp, int on_device) {
  if (!valid(S) || !rho_hp) return fail(MHD_EINVAL, "mhd_get_ions: null argument");
  const size_t bytes = (size_t)S->g.N * 8;
  double* dev = on_device ? rho_hp : (double*)S->staging;
  CK(S->precision ? store_ions(S, S->b32, dev) : store_ions(S, S->b64, dev));
  if (!on_device) CK(cudaMemcpyAsync(rho_hp, dev, bytes, cudaMemcpyDeviceToHost, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  return MHD_OK;
}

int mhd_set_ions(mhd_sim* S, const double* rho_hp, int on_device) {
  if (!valid(S) || !rho_hp) return fail(MHD_EINVAL, "mhd_set_ions: null argument");
  if (!S->has_state) return fail(MHD_EINVAL, "mhd_set_ions: load a state first (mhd_set_state zeroes rho_H+)");
  const size_t bytes = (size_t)S->g.N * 8;
  const double* dev = rho_hp;
  if (!on_device) {
    CK(cudaMemcpyAsync(S->staging, rho_hp, bytes, cudaMemcpyHostToDevice, S->stream));
    dev = (const double*)S->staging;
  }
  CK(S->precision ? load_ions(S, S->b32, dev) : load_ions(S, S->b64, dev));
  int rc = refresh_cfl(S);  // gamma_eff, hence the sound speed, depends on rho_H+
  if (rc != MHD_OK) return rc;
  CK(cudaStreamSynchronize(S->stream));
  return MHD_OK;
}

int mhd_set_full(mhd_sim* S, const double* eint, const double* bx, const double* by, const double* bz,
                 int on_device) {
  if (!valid(S) || !eint || !bx || !by || !bz) return fail(MHD_EINVAL, "mhd_set_full: null argument");
  const size_t bytes = (size_t)S->g.N * 8;
  const double* src[4] = {eint, bx, by, bz};
  const double* dev[4];
  for (int q = 0; q < 4; ++q) {
    if (on_device) {
      dev[q] = src[q];
    } else {
      double* d = (double*)(S->staging + q * bytes);
      CK(cudaMemcpyAsync(d, src[q], bytes, cudaMemcpyHostToDevice, S->stream));
      dev[q] = d;
    }
  }
  CK(S->precision ? load_full(S, S->b32, dev) : load_full(S, S->b64, dev));
  int rc = refresh_cfl(S);
  if (rc != MHD_OK) return rc;
  CK(cudaStreamSynchronize(S->stream));
  return MHD_OK;
}

int mhd_step(mhd_sim* S, double cfl, double* dt_taken) {
  if (!valid(S)) return fail(MHD_EINVAL, "mhd_step: null sim");
  if (!S->has_state) return fail(MHD_EINVAL, "mhd_step: no state loaded");
  if (!(cfl > 0.0)) return fail(MHD_EINVAL, "mhd_step: cfl must be > 0");
  int rc;
  if (S->params_dirty || cfl != S->last_cfl || S->last_tend != 0.0) {
    if ((rc = set_params(S, cfl, 0.0, 0, 0.0)) != MHD_OK) return rc;
    S->last_cfl = cfl;
    S->last_tend = 0.0;
    S->params_dirty = false;
  }
  if (!dt_taken) {
    // an earlier step flagged by the device and finished by now (no synchronisation here)
    const int hf = *(volatile int*)S->hflags_host;
    if (hf & 1) return fail(MHD_ENONPHYS, "non-physical state after an earlier step (rho, rho eps <= 0 or non-finite)");
    if (hf & 2) return fail(MHD_EINVAL, "tau <= 0 in an earlier step");
    if (hf & 4) return fail(MHD_ECUDA, "a bulk copy into shared memory did not complete in an earlier step");
  }
  if ((rc = enqueue_step(S)) != MHD_OK) return rc;
  if (dt_taken) {
    if ((rc = read_scalars(S)) != MHD_OK) return rc;
    *dt_taken = S->sc_host->tau;
    if (S->sc_host->flags & 1) return fail(MHD_ENONPHYS, "non-physical state (rho, rho eps <= 0 or non-finite)");
    if (S->sc_host->flags & 2) return fail(MHD_EINVAL, "tau <= 0");
    if (S->sc_host->flags & 4) return fail(MHD_ECUDA, "a bulk copy into shared memory did not complete");
  }
  return MHD_OK;
}

int mhd_advance(mhd_sim* S, double cfl, double t_end, int max_steps, int* steps_done) {
  if (!valid(S)) return fail(MHD_EINVAL, "mhd_advance: null sim");
  if (!S->has_state) return fail(MHD_EINVAL, "mhd_advance: no state loaded");
  if (!(cfl > 0.0) || !(t_end > 0.0)) return fail(MHD_EINVAL, "mhd_advance: need cfl > 0, t_end > 0");
  int rc;
  if ((rc = set_params(S, cfl, t_end, 0, 0.0)) != MHD_OK) return rc;
  S->last_cfl = cfl;
  S->last_tend = t_end;
  S->params_dirty = false;
  if ((rc = read_scalars(S)) != MHD_OK) return rc;
  int k = 0;
  while (k < max_steps && S->sc_host->t < t_end) {
    if ((rc = enqueue_step(S)) != MHD_OK) break;
    ++k;
    if ((rc = read_scalars(S)) != MHD_OK) break;
    if (S->sc_host->flags & 1) {
      rc = fail(MHD_ENONPHYS, "non-physical state (rho, rho eps <= 0 or non-finite)");
      break;
    }
    if (S->sc_host->flags & 2) {
      rc = fail(MHD_EINVAL, "tau <= 0");
      break;
    }
    if (S->sc_host->flags & 4) {
      rc = fail(MHD_ECUDA, "a bulk copy into shared memory did not complete");
      break;
    }
  }
  if (steps_done) *steps_done = k;
  return rc;
}

int mhd_sync(mhd_sim* S) {
  if (!valid(S)) return fail(MHD_EINVAL, "mhd_sync: null sim");
  int rc = read_scalars(S);
  if (rc != MHD_OK) return rc;
  if (S->sc_host->flags & 1) return fail(MHD_ENONPHYS, "non-physical state (rho, rho eps <= 0 or non-finite)");
  if (S->sc_host->flags & 4) return fail(MHD_ECUDA, "a bulk copy into shared memory did not complete");
  return MHD_OK;
}

int mhd_stage(mhd_sim* S, int which, double tau) {
  if (!valid(S)) return fail(MHD_EINVAL, "mhd_stage: null sim");
  if (which < 1 || which > 5 || !(tau > 0.0)) return fail(MHD_EINVAL, "mhd_stage: which in 1..5, tau > 0");
  const int cell_stages = which == 3 ? 1 : (which == 5 ? 2 : 0);
  int rc;
  const bool grav = which == 1 && S->ph.grav_g > 0.0;
  if (grav) {
    if (S->g.bc[0] || S->g.bc[1] || S->g.bc[2]) return fail(MHD_EINVAL, "self-gravity needs periodic boundaries");
    if ((rc = grav_prepare(S)) != MHD_OK) return rc;
  }
  if ((rc = set_params(S, 1.0, 0.0, 1, tau)) != MHD_OK) return rc;
  if (grav && (rc = grav_solve(S)) != MHD_OK) return rc;
  S->params_dirty = true;
  if (S->precision) {
    launch_small(S->x32, S->stream, 0);
    if (which == 1) launch_euler_stage(S->x32, S->stream);
    if (which == 2) launch_lag_stage(S->x32, S->stream, false);
    if (which >= 3) launch_post(S->x32, S->stream, cell_stages, which == 4, 1);
  } else {
    launch_small(S->x64, S->stream, 0);
    if (which == 1) launch_euler_stage(S->x64, S->stream);
    if (which == 2) launch_lag_stage(S->x64, S->stream, false);
    if (which >= 3) launch_post(S->x64, S->stream, cell_stages, which == 4, 1);
  }
  CK(cudaGetLastError());
  if ((rc = refresh_cfl(S)) != MHD_OK) return rc;
  if ((rc = set_params(S, 1.0, 0.0, 0, 0.0)) != MHD_OK) return rc;
  return mhd_sync(S);
}

int mhd_get_potential(mhd_sim* S, double* out) {
  if (!valid(S) || !out) return fail(MHD_EINVAL, "mhd_get_potential: null argument");
  if (!(S->ph.grav_g > 0.0)) return fail(MHD_EINVAL, "mhd_get_potential: self-gravity is off");
  if (!S->has_state) return fail(MHD_EINVAL, "mhd_get_potential: no state loaded");
  if (S->g.bc[0] || S->g.bc[1] || S->g.bc[2]) return fail(MHD_EINVAL, "self-gravity needs periodic boundaries");
  int rc;
  if ((rc = grav_prepare(S)) != MHD_OK) return rc;
  if ((rc = ensure_exec(S)) != MHD_OK) return rc;
  if ((rc = grav_solve(S)) != MHD_OK) return rc;
  return grav_copy(S, out);
}

int mhd_check_flags(int clear, unsigned* flags) {
  if (!flags || (clear != 0 && clear != 1)) return fail(MHD_EINVAL, "mhd_check_flags: need flags and clear in {0, 1}");
#ifdef MHD_CHECK
  CK(cudaDeviceSynchronize());
  *flags = check_flags_of_this_unit(clear != 0) | check_flags_f32(clear != 0) | check_flags_gravity(clear != 0);
  return MHD_OK;
#else
  *flags = 0;
  return fail(MHD_EINVAL, "mhd_check_flags: this library was built without index checks");
#endif
}

int mhd_launches_per_step(mhd_sim* S) {
  if (!valid(S)) return fail(MHD_EINVAL, "mhd_launches_per_step: null sim");
  // begin + 3 x (primitives, 3 faces, edges, update) + 3 x (3 faces) + 2 updates + the last
  // update with the post stage + end (the first update of each stage stores its RK register Q^n)
  return 1 + 3 * 6 + 3 * 3 + 2 + 1 + 1;
}

int mhd_profile(mhd_sim* S, double cfl, int steps, double* out_ms, int64_t* out_launches) {
  if (!valid(S) || !out_ms || !out_launches || steps < 1) return fail(MHD_EINVAL, "mhd_profile: bad argument");
  if (!S->has_state) return fail(MHD_EINVAL, "mhd_profile: no state loaded");
  int rc = set_params(S, cfl, 0.0, 0, 0.0);
  if (rc != MHD_OK) return rc;
  S->last_cfl = cfl;
  S->last_tend = 0.0;
  S->params_dirty = false;
  S->prof.on = true;
  for (int k = 0; k < steps; ++k) launch_sim_step(S);
  S->prof.on = false;
  cudaError_t e = cudaStreamSynchronize(S->stream);
  for (int c = 0; c < MHD_K_NCLASSES; ++c) {
    out_ms[c] = 0.0;
    out_launches[c] = 0;
  }
  for (size_t q = 0; q < S->prof.cls.size(); ++q) {
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, S->prof.ev[2 * q], S->prof.ev[2 * q + 1]);
    out_ms[report_class(S->prof.cls[q])] += ms;
    out_launches[report_class(S->prof.cls[q])] += 1;
  }
  for (cudaEvent_t ev : S->prof.ev) cudaEventDestroy(ev);
  S->prof.ev.clear();
  S->prof.cls.clear();
  if (e != cudaSuccess) return fail(MHD_ECUDA, std::string("mhd_profile: ") + cudaGetErrorString(e));
  return mhd_sync(S);
}

int mhd_diagnostics(mhd_sim* S, mhd_diag* out) {
  if (!valid(S) || !out) return fail(MHD_EINVAL, "mhd_diagnostics: null argument");
  CK(S->precision ? diag_partial(S, S->b32) : diag_partial(S, S->b64));
  k_diag_final<<<1, DIAG_THREADS, 0, S->stream>>>(S->diag_part, S->diag_blocks, S->diag_out);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(S->diag_host, S->diag_out, 9 * sizeof(double), cudaMemcpyDeviceToHost, S->stream));
  int rc = read_scalars(S);
  if (rc != MHD_OK) return rc;
  const double* d = S->diag_host;
  out->sum_rho = d[0];
  for (int q = 0; q < 3; ++q) out->sum_mom[q] = d[1 + q];
  out->sum_E = d[4];
  for (int q = 0; q < 3; ++q) out->sum_b[q] = d[5 + q];
  out->max_div_b_h = d[8];
  out->t = S->sc_host->t;
  double Dm;
  unsigned long long bits = S->sc_host->dmax;
  std::memcpy(&Dm, &bits, sizeof(Dm));
  out->tau_next = Dm > 0.0 ? S->ph.dx / Dm : 0.0;
  out->steps = S->sc_host->steps;
  out->vel_branch = (int64_t)S->sc_host->vel_branch;
  out->error_flags = S->sc_host->flags;
  return MHD_OK;
}

}  // extern "C"

// ================================================================================================
// Batches: many boxes, one launch per kernel class
struct mhd_batch {
  std::vector<mhd_sim*> sims;
  int precision = 0;
  cudaStream_t stream = nullptr;
  Exec<double> x64;
  Exec<float> x32;
  Profiler prof;
  cudaGraphExec_t gexec = nullptr;
  bool graph_valid = false;
  double last_cfl = -1.0;
};

namespace {

void batch_drop_graph(mhd_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  b->graph_valid = false;
}

template <typename T>
Exec<T>& bexec(mhd_batch* b);
template <>
Exec<double>& bexec<double>(mhd_batch* b) { return b->x64; }
template <>
Exec<float>& bexec<float>(mhd_batch* b) { return b->x32; }

template <typename T>
const Box<T>& sim_box(mhd_sim* S);
template <>
const Box<double>& sim_box<double>(mhd_sim* S) { return S->b64; }
template <>
const Box<float>& sim_box<float>(mhd_sim* S) { return S->b32; }

template <typename T>
int batch_init(mhd_batch* b) {
  std::vector<Box<T>> boxes;
  for (mhd_sim* S : b->sims) boxes.push_back(sim_box<T>(S));
  Exec<T>& X = bexec<T>(b);
  X.prof = &b->prof;
  cudaError_t e = exec_init(X, boxes);
  if (e != cudaSuccess) return fail(MHD_ECUDA, std::string("batch set-up: ") + cudaGetErrorString(e));
  X.x_stage = !b->sims.empty();
  for (mhd_sim* S : b->sims) X.x_stage = X.x_stage && S->x_stage != 0;
  return MHD_OK;
}

template <typename T>
void batch_launch_step(mhd_batch* b) {
  launch_step(bexec<T>(b), b->stream);
}

int batch_enqueue(mhd_batch* b) {
  if (!b->graph_valid) {
    batch_drop_graph(b);
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    if (b->precision)
      batch_launch_step<float>(b);
    else
      batch_launch_step<double>(b);
    cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    if (e != cudaSuccess) return fail(MHD_ECUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(MHD_ECUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
    b->graph_valid = true;
  }
  CK(cudaGraphLaunch(b->gexec, b->stream));
  return MHD_OK;
}

int batch_set_params(mhd_batch* b, double cfl) {
  if (cfl != b->last_cfl) {
    CK(b->precision ? launch_set_params(b->x32, b->stream, cfl, 0.0, 0, 0.0)
                    : launch_set_params(b->x64, b->stream, cfl, 0.0, 0, 0.0));
    b->last_cfl = cfl;
  }
  for (mhd_sim* S : b->sims) S->params_dirty = true;  // members' cached parameters are stale
  return MHD_OK;
}

// state snapshot of every member (10 state arrays into its staging buffer, scalars on the host)
template <typename T>
int batch_snapshot(mhd_batch* b, std::vector<Scalars>& sc, bool restore) {
  sc.resize(b->sims.size());
  for (size_t i = 0; i < b->sims.size(); ++i) {
    mhd_sim* S = b->sims[i];
    const Box<T>& B = sim_box<T>(S);
    T* arrs[10] = {B.s.rho, B.s.m[0], B.s.m[1], B.s.m[2], B.s.E, B.s.eint, B.s.rh2, B.s.b[0], B.s.b[1], B.s.b[2]};
    const size_t bytes = (size_t)S->g.N * sizeof(T);
    for (int q = 0; q < 10; ++q) {
      char* snap = S->staging + (size_t)q * S->g.N * 8;
      if (restore)
        CK(cudaMemcpyAsync(arrs[q], snap, bytes, cudaMemcpyDeviceToDevice, b->stream));
      else
        CK(cudaMemcpyAsync(snap, arrs[q], bytes, cudaMemcpyDeviceToDevice, b->stream));
    }
    if (restore)
      CK(cudaMemcpyAsync(S->sc, &sc[i], sizeof(Scalars), cudaMemcpyHostToDevice, b->stream));
    else
      CK(cudaMemcpyAsync(&sc[i], S->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
  }
  return MHD_OK;
}

// run `steps` launched steps with event pairs; per-tag milliseconds
template <typename T>
int batch_timed(mhd_batch* b, int steps, std::vector<double>& ms_per_tag, std::vector<long long>& n_per_tag) {
  Exec<T>& X = bexec<T>(b);
  b->prof.on = true;
  for (int k = 0; k < steps; ++k) launch_step(X, b->stream);
  b->prof.on = false;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  ms_per_tag.assign(PROF_KC_BASE + NKC, 0.0);
  n_per_tag.assign(PROF_KC_BASE + NKC, 0);
  for (size_t q = 0; q < b->prof.cls.size(); ++q) {
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, b->prof.ev[2 * q], b->prof.ev[2 * q + 1]);
    ms_per_tag[b->prof.cls[q]] += ms;
    n_per_tag[b->prof.cls[q]] += 1;
  }
  for (cudaEvent_t ev : b->prof.ev) cudaEventDestroy(ev);
  b->prof.ev.clear();
  b->prof.cls.clear();
  if (e != cudaSuccess) return fail(MHD_ECUDA, std::string("batch timing: ") + cudaGetErrorString(e));
  return MHD_OK;
}

bool is_face_class(int kc) { return kc == KC_EFACE || kc == KC_LFACE; }

template <typename T>
int batch_tune(mhd_batch* b, double cfl, int reps, double* best_ms) {
  Exec<T>& X = bexec<T>(b);
  std::vector<Scalars> snap;
  int rc = batch_snapshot<T>(b, snap, false);
  if (rc != MHD_OK) return rc;
  const int face_blocks[3] = {64, 128, 256}, cell_blocks[3] = {128, 256, 512}, mults[3] = {0, 4, 16};
  double best[NKC];
  LaunchCfg bestc[NKC];
  for (int kc = 0; kc < NKC; ++kc) {
    best[kc] = 1e300;
    bestc[kc] = X.cfg[kc];
  }
  std::vector<double> ms;
  std::vector<long long> nl;
  for (int bi = 0; bi < 3; ++bi)
    for (int mi = 0; mi < 3; ++mi) {
      for (int kc = 0; kc < NKC; ++kc) X.cfg[kc] = LaunchCfg{is_face_class(kc) ? face_blocks[bi] : cell_blocks[bi], mults[mi]};
      cudaError_t e = ensure_tables(X);
      if (e != cudaSuccess) return fail(MHD_ECUDA, std::string("tile tables: ") + cudaGetErrorString(e));
      if ((rc = batch_snapshot<T>(b, snap, true)) != MHD_OK) return rc;
      CK(launch_set_params(X, b->stream, cfl, 0.0, 0, 0.0));
      if ((rc = batch_timed<T>(b, reps, ms, nl)) != MHD_OK) return rc;
      for (int kc = 0; kc < NKC; ++kc)
        if (ms[PROF_KC_BASE + kc] < best[kc]) {
          best[kc] = ms[PROF_KC_BASE + kc];
          bestc[kc] = X.cfg[kc];
        }
    }
  for (int kc = 0; kc < NKC; ++kc) X.cfg[kc] = bestc[kc];
  cudaError_t e = ensure_tables(X);
  if (e != cudaSuccess) return fail(MHD_ECUDA, std::string("tile tables: ") + cudaGetErrorString(e));
  if (best_ms) {
    double tot = 0.0;
    for (int kc = 0; kc < NKC; ++kc) tot += best[kc];
    *best_ms = tot / reps;
  }
  if ((rc = batch_snapshot<T>(b, snap, true)) != MHD_OK) return rc;
  b->last_cfl = -1.0;
  batch_drop_graph(b);
  return MHD_OK;
}

}  // namespace

extern "C" {

mhd_batch* mhd_batch_create(mhd_sim* const* sims, int n) {
  if (!sims || n < 1) {
    fail(MHD_EINVAL, "mhd_batch_create: need at least one sim");
    return nullptr;
  }
  for (int i = 0; i < n; ++i) {
    if (!valid(sims[i]) || !sims[i]->has_state) {
      fail(MHD_EINVAL, "mhd_batch_create: every sim needs a loaded state");
      return nullptr;
    }
    if (sims[i]->precision != sims[0]->precision || sims[i]->device != sims[0]->device) {
      fail(MHD_EINVAL, "mhd_batch_create: sims differ in precision or device");
      return nullptr;
    }
    if (sims[i]->ph.grav_g > 0.0) {
      fail(MHD_EINVAL, "mhd_batch_create: self-gravity sims step alone (one Poisson solve per box)");
      return nullptr;
    }
  }
  mhd_batch* b = new (std::nothrow) mhd_batch();
  if (!b) {
    fail(MHD_ENOMEM, "mhd_batch_create: host allocation failed");
    return nullptr;
  }
  b->precision = sims[0]->precision;
  for (int i = 0; i < n; ++i) {
    if (ensure_exec(sims[i]) != MHD_OK || cudaStreamSynchronize(sims[i]->stream) != cudaSuccess) {
      fail(MHD_ECUDA, "mhd_batch_create: member not ready");
      delete b;
      return nullptr;
    }
    b->sims.push_back(sims[i]);
  }
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
    fail(MHD_ECUDA, "mhd_batch_create: stream");
    delete b;
    return nullptr;
  }
  int rc = b->precision ? batch_init<float>(b) : batch_init<double>(b);
  if (rc != MHD_OK) {
    mhd_batch_destroy(b);
    return nullptr;
  }
  for (mhd_sim* S : b->sims) S->batched += 1;
  return b;
}

void mhd_batch_destroy(mhd_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_drop_graph(b);
  exec_free(b->x64);
  exec_free(b->x32);
  for (mhd_sim* S : b->sims) S->batched -= 1;
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

int mhd_batch_step(mhd_batch* b, double cfl) {
  if (!b) return fail(MHD_EINVAL, "mhd_batch_step: null batch");
  if (!(cfl > 0.0)) return fail(MHD_EINVAL, "mhd_batch_step: cfl must be > 0");
  int rc = batch_set_params(b, cfl);
  if (rc != MHD_OK) return rc;
  return batch_enqueue(b);
}

int mhd_batch_sync(mhd_batch* b) {
  if (!b) return fail(MHD_EINVAL, "mhd_batch_sync: null batch");
  CK(cudaStreamSynchronize(b->stream));
  int bad = 0;
  for (mhd_sim* S : b->sims) {
    CK(cudaMemcpy(S->sc_host, S->sc, sizeof(Scalars), cudaMemcpyDeviceToHost));
    if (S->sc_host->flags & 1) bad |= 1;
    if (S->sc_host->flags & 4) bad |= 4;
  }
  if (bad & 4) return fail(MHD_ECUDA, "a bulk copy into shared memory did not complete in a batch member");
  if (bad) return fail(MHD_ENONPHYS, "non-physical state in a batch member");
  return MHD_OK;
}

int mhd_batch_query(mhd_batch* b) {
  if (!b) return fail(MHD_EINVAL, "mhd_batch_query: null batch");
  cudaError_t e = cudaStreamQuery(b->stream);
  if (e == cudaErrorNotReady) return MHD_PENDING;
  CK(e);
  return mhd_batch_sync(b);
}

int mhd_batch_set_priority(mhd_batch* b, int high) {
  if (!b || (high != 0 && high != 1)) return fail(MHD_EINVAL, "mhd_batch_set_priority: high must be 0 or 1");
  int least = 0, greatest = 0;
  CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  cudaStream_t st = nullptr;
  CK(cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, high ? greatest : least));
  CK(cudaStreamSynchronize(b->stream));
  cudaStreamDestroy(b->stream);
  b->stream = st;
  return MHD_OK;
}

int mhd_batch_tune(mhd_batch* b, double cfl, int reps, double* best_ms) {
  if (!b || reps < 1 || !(cfl > 0.0)) return fail(MHD_EINVAL, "mhd_batch_tune: bad argument");
  CK(cudaStreamSynchronize(b->stream));
  return b->precision ? batch_tune<float>(b, cfl, reps, best_ms) : batch_tune<double>(b, cfl, reps, best_ms);
}

static int kc_of_profile_class(int cls) {
  for (int kc = 0; kc < NKC; ++kc)
    if (profile_class(kc) == cls) return kc;
  return -1;
}

int mhd_batch_get_shape(mhd_batch* b, int cls, int* block, int* grid_mult) {
  int kc = kc_of_profile_class(cls);
  if (!b || kc < 0 || !block || !grid_mult) return fail(MHD_EINVAL, "mhd_batch_get_shape: bad argument");
  const LaunchCfg& c = b->precision ? b->x32.cfg[kc] : b->x64.cfg[kc];
  *block = c.block;
  *grid_mult = c.grid_mult;
  return MHD_OK;
}

int mhd_batch_set_shape(mhd_batch* b, int cls, int block, int grid_mult) {
  int kc = kc_of_profile_class(cls);
  if (!b || kc < 0) return fail(MHD_EINVAL, "mhd_batch_set_shape: bad kernel class");
  if ((block != 64 && block != 128 && block != 256 && block != 512) || grid_mult < 0)
    return fail(MHD_EINVAL, "mhd_batch_set_shape: block in {64, 128, 256, 512}, grid_mult >= 0");
  if (is_face_class(kc) && block > 256) return fail(MHD_EINVAL, "face kernels take at most 256 threads");
  CK(cudaStreamSynchronize(b->stream));
  cudaError_t e;
  if (b->precision) {
    b->x32.cfg[kc] = LaunchCfg{block, grid_mult};
    e = ensure_tables(b->x32);
  } else {
    b->x64.cfg[kc] = LaunchCfg{block, grid_mult};
    e = ensure_tables(b->x64);
  }
  if (e != cudaSuccess) return fail(MHD_ECUDA, std::string("tile tables: ") + cudaGetErrorString(e));
  batch_drop_graph(b);
  return MHD_OK;
}

int mhd_batch_profile(mhd_batch* b, double cfl, int steps, double* out_ms, int64_t* out_launches) {
  if (!b || steps < 1 || !out_ms || !out_launches) return fail(MHD_EINVAL, "mhd_batch_profile: bad argument");
  int rc = batch_set_params(b, cfl);
  if (rc != MHD_OK) return rc;
  std::vector<double> ms;
  std::vector<long long> nl;
  rc = b->precision ? batch_timed<float>(b, steps, ms, nl) : batch_timed<double>(b, steps, ms, nl);
  if (rc != MHD_OK) return rc;
  for (int c = 0; c < MHD_K_NCLASSES; ++c) {
    out_ms[c] = 0.0;
    out_launches[c] = 0;
  }
  for (int tag = 0; tag < (int)ms.size(); ++tag) {
    if (nl[tag] == 0) continue;
    out_ms[report_class(tag)] += ms[tag];
    out_launches[report_class(tag)] += nl[tag];
  }
  return mhd_batch_sync(b);
}

}  // extern "C"
