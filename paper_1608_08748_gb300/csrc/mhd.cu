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
#include "mhd_kernels.cuh"

using namespace mhd;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) return fail(MHD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// SSP-RK3 (Sec. 2.2): Q = a Q^n + b Q + g tau R
const double RK_A[3] = {0.0, 0.75, 1.0 / 3.0};
const double RK_B[3] = {1.0, 0.25, 2.0 / 3.0};
const double RK_G[3] = {1.0, 0.25, 2.0 / 3.0};

template <typename T>
struct Buffers {
  State<T> s, s0;
  Prim<T> w;
  FaceOut<T> fo[3];  // Eulerian face outputs; the Lagrangian fluxes reuse the same memory
  T* e[3];
  LagFlux<T> lf[3];
};

}  // namespace

namespace mhd_rt {
// record the message mhd_last_error() returns on this thread; returns code
int set_error(int code, const std::string& msg) { return fail(code, msg); }
}  // namespace mhd_rt

struct mhd_sim {
  Geom g;
  Phys ph;
  int precision = 0;
  int use_graph = 1;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  char* pool = nullptr;
  size_t pool_bytes = 0;
  char* staging = nullptr;  // 10 * N * 8 bytes for host transfers / dtype conversion
  Scalars* sc = nullptr;
  Scalars* sc_host = nullptr;  // pinned mirror
  double* diag_part = nullptr;
  double* diag_out = nullptr;
  double* diag_host = nullptr;  // pinned, 9 doubles
  int diag_blocks = 0;
  Buffers<double> b64;
  Buffers<float> b32;
  cudaGraphExec_t gexec = nullptr;
  bool graph_valid = false;
  bool params_dirty = true;
  double last_cfl = -1.0, last_tend = -1.0;
  bool has_state = false;
  // profiling: event pairs around every launch while mhd_profile runs
  bool profiling = false;
  std::vector<cudaEvent_t> prof_ev;
  std::vector<int> prof_cls;
};

namespace {

size_t pool_size(const Geom& g, int precision, int chem) {
  (void)chem;
  size_t es = precision ? sizeof(float) : sizeof(double);
  size_t cells = (size_t)g.N, faces = (size_t)g.NF;
  // state 10, Q^n 10, primitives 9 (cells); face outputs 3 x 7 and edges 3 (lattice)
  return es * (cells * 29 + faces * 24) + 64 * 64;
}

template <typename T>
void carve(mhd_sim* S, Buffers<T>& B) {
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
    for (int d = 0; d < 3; ++d) s->b[d] = take(N);
  }
  for (int d = 0; d < 3; ++d) B.w.v[d] = take(N);
  for (int d = 0; d < 3; ++d) B.w.B[d] = take(N);
  B.w.p = take(N);
  B.w.g = take(N);
  B.w.sr = take(N);
  for (int d = 0; d < 3; ++d)
    for (int v = 0; v < 7; ++v) {
      B.fo[d].f[v] = take(NF);
      B.lf[d].f[v] = B.fo[d].f[v];
    }
  for (int d = 0; d < 3; ++d) B.e[d] = take(NF);
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
  S->has_state = false;
  return MHD_OK;
}

// CUDA event pair around one launch (only while profiling)
struct PScope {
  mhd_sim* S;
  PScope(mhd_sim* s_, int cls) : S(s_) {
    if (!S->profiling) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, S->stream);
    S->prof_ev.push_back(e);
    S->prof_cls.push_back(cls);
  }
  ~PScope() {
    if (!S->profiling) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, S->stream);
    S->prof_ev.push_back(e);
  }
};

void drop_graph(mhd_sim* S) {
  if (S->gexec) cudaGraphExecDestroy(S->gexec);
  S->gexec = nullptr;
  S->graph_valid = false;
}

// ------------------------------------------------------------------------------------------------
// stage launchers
template <typename T>
void launch_euler_stage(mhd_sim* S, Buffers<T>& B) {
  const Geom& g = S->g;
  cudaStream_t st = S->stream;
  const size_t bytes = (size_t)g.N * sizeof(T);
  for (int d = 0; d < 3; ++d) cudaMemcpyAsync(B.s0.m[d], B.s.m[d], bytes, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(B.s0.E, B.s.E, bytes, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(B.s0.eint, B.s.eint, bytes, cudaMemcpyDeviceToDevice, st);
  for (int d = 0; d < 3; ++d) cudaMemcpyAsync(B.s0.b[d], B.s.b[d], bytes, cudaMemcpyDeviceToDevice, st);
  const long long fx = (long long)(g.n[0] + 1) * g.n[1] * g.n[2];
  const long long fy = (long long)g.n[0] * (g.n[1] + 1) * g.n[2];
  const long long fz = (long long)g.n[0] * g.n[1] * (g.n[2] + 1);
  for (int r = 0; r < 3; ++r) {
    { PScope p(S, MHD_K_PRIM); k_prim<T><<<nblk(g.N, 256), 256, 0, st>>>(g, S->ph, B.s, B.w); }
    { PScope p(S, MHD_K_EULER_FACE); k_euler_face<T, 0><<<nblk(fx, 128), 128, 0, st>>>(g, S->sc, B.s, B.w, B.fo[0]); }
    { PScope p(S, MHD_K_EULER_FACE); k_euler_face<T, 1><<<nblk(fy, 128), 128, 0, st>>>(g, S->sc, B.s, B.w, B.fo[1]); }
    { PScope p(S, MHD_K_EULER_FACE); k_euler_face<T, 2><<<nblk(fz, 128), 128, 0, st>>>(g, S->sc, B.s, B.w, B.fo[2]); }
    { PScope p(S, MHD_K_EDGES);
      k_edges<T><<<nblk(g.NF, 256), 256, 0, st>>>(g, B.fo[0], B.fo[1], B.fo[2], B.e[0], B.e[1], B.e[2]); }
    { PScope p(S, MHD_K_EULER_UPDATE);
      k_euler_update<T><<<nblk(g.N, 256), 256, 0, st>>>(g, S->ph, S->sc, B.s, B.s0, B.w, B.fo[0], B.fo[1],
                                                        B.fo[2], B.e[0], B.e[1], B.e[2], (T)RK_A[r],
                                                        (T)RK_B[r], (T)RK_G[r]); }
  }
}

template <typename T>
void launch_lag_stage(mhd_sim* S, Buffers<T>& B) {
  const Geom& g = S->g;
  cudaStream_t st = S->stream;
  const size_t bytes = (size_t)g.N * sizeof(T);
  const int nv = S->ph.chem ? 7 : 6;
  cudaMemcpyAsync(B.s0.rho, B.s.rho, bytes, cudaMemcpyDeviceToDevice, st);
  for (int d = 0; d < 3; ++d) cudaMemcpyAsync(B.s0.m[d], B.s.m[d], bytes, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(B.s0.E, B.s.E, bytes, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(B.s0.eint, B.s.eint, bytes, cudaMemcpyDeviceToDevice, st);
  if (S->ph.chem) cudaMemcpyAsync(B.s0.rh2, B.s.rh2, bytes, cudaMemcpyDeviceToDevice, st);
  const long long fx = (long long)(g.n[0] + 1) * g.n[1] * g.n[2];
  const long long fy = (long long)g.n[0] * (g.n[1] + 1) * g.n[2];
  const long long fz = (long long)g.n[0] * g.n[1] * (g.n[2] + 1);
  for (int r = 0; r < 3; ++r) {
    { PScope p(S, MHD_K_LAG_FACE); k_lag_face<T, 0><<<nblk(fx, 128), 128, 0, st>>>(g, S->sc, B.s, nv, B.lf[0]); }
    { PScope p(S, MHD_K_LAG_FACE); k_lag_face<T, 1><<<nblk(fy, 128), 128, 0, st>>>(g, S->sc, B.s, nv, B.lf[1]); }
    { PScope p(S, MHD_K_LAG_FACE); k_lag_face<T, 2><<<nblk(fz, 128), 128, 0, st>>>(g, S->sc, B.s, nv, B.lf[2]); }
    { PScope p(S, MHD_K_LAG_UPDATE);
      k_lag_update<T><<<nblk(g.N, 256), 256, 0, st>>>(g, S->ph, S->sc, B.s, B.s0, nv, B.lf[0], B.lf[1],
                                                      B.lf[2], (T)RK_A[r], (T)RK_B[r], (T)RK_G[r]); }
  }
}

template <typename T>
void launch_step(mhd_sim* S, Buffers<T>& B) {
  cudaStream_t st = S->stream;
  { PScope p(S, MHD_K_SMALL); k_begin_step<<<1, 32, 0, st>>>(S->ph, S->sc); }
  launch_euler_stage(S, B);
  launch_lag_stage(S, B);
  { PScope p(S, MHD_K_POST); k_post<T><<<nblk(S->g.N, 256), 256, 0, st>>>(S->g, S->ph, S->sc, B.s, 1, 1); }
  { PScope p(S, MHD_K_SMALL); k_end_step<<<1, 32, 0, st>>>(S->sc); }
}

int enqueue_step(mhd_sim* S) {
  if (S->use_graph) {
    if (!S->graph_valid) {
      drop_graph(S);
      cudaGraph_t graph;
      CK(cudaStreamBeginCapture(S->stream, cudaStreamCaptureModeThreadLocal));
      if (S->precision)
        launch_step(S, S->b32);
      else
        launch_step(S, S->b64);
      cudaError_t e = cudaStreamEndCapture(S->stream, &graph);
      if (e != cudaSuccess) return fail(MHD_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      e = cudaGraphInstantiate(&S->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return fail(MHD_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
      S->graph_valid = true;
    }
    CK(cudaGraphLaunch(S->gexec, S->stream));
  } else {
    if (S->precision)
      launch_step(S, S->b32);
    else
      launch_step(S, S->b64);
    CK(cudaGetLastError());
  }
  return MHD_OK;
}

int set_params(mhd_sim* S, double cfl, double t_end, int fixed_tau, double tau) {
  k_set_params<<<1, 32, 0, S->stream>>>(S->sc, cfl, t_end, fixed_tau, tau);
  CK(cudaGetLastError());
  return MHD_OK;
}

int read_scalars(mhd_sim* S) {
  CK(cudaMemcpyAsync(S->sc_host, S->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  return MHD_OK;
}

template <typename T>
int launch_cfl(mhd_sim* S, Buffers<T>& B) {
  CK(cudaMemsetAsync(&S->sc->dmax, 0, sizeof(unsigned long long), S->stream));
  k_cfl<T><<<nblk(S->g.N, 256), 256, 0, S->stream>>>(S->g, S->ph, S->sc, B.s);
  CK(cudaGetLastError());
  return MHD_OK;
}

int refresh_cfl(mhd_sim* S) { return S->precision ? launch_cfl(S, S->b32) : launch_cfl(S, S->b64); }

size_t dtype_size(int dt) { return dt == MHD_F32 ? 4 : 8; }

template <typename T, typename In>
int load_state(mhd_sim* S, Buffers<T>& B, const In* p[9]) {
  const Geom& g = S->g;
  k_load_cells<T, In><<<nblk(g.N, 256), 256, 0, S->stream>>>(g, B.s, p[0], p[1], p[2], p[3], p[4], p[8]);
  k_faces_from_cells<T, In><<<nblk(g.N, 256), 256, 0, S->stream>>>(g, B.s, p[5], p[6], p[7]);
  k_derive_eint<T><<<nblk(g.N, 256), 256, 0, S->stream>>>(g, B.s);
  CK(cudaGetLastError());
  return MHD_OK;
}

template <typename T, typename Out>
int store_state(mhd_sim* S, Buffers<T>& B, Out* p[9]) {
  const Geom& g = S->g;
  k_store_state<T, Out><<<nblk(g.N, 256), 256, 0, S->stream>>>(g, B.s, p[0], p[1], p[2], p[3], p[4], p[5],
                                                                p[6], p[7], p[8]);
  CK(cudaGetLastError());
  return MHD_OK;
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
  return pool_size(g, precision, chem) + (size_t)g.N * 10 * 8 + sizeof(Scalars) +
         ((size_t)g.N / 256 + 2) * 9 * 8;
}

mhd_sim* mhd_create(int nx, int ny, int nz, double gamma, double dx) {
  if (nx < 1 || ny < 1 || nz < 1 || !(gamma > 1.0) || !(dx > 0.0)) {
    fail(MHD_EINVAL, "mhd_create: need nx, ny, nz >= 1, gamma > 1, dx > 0");
    return nullptr;
  }
  if ((long long)(nx + 1) * (ny + 1) * (nz + 1) > (1ll << 40)) {
    fail(MHD_EINVAL, "mhd_create: grid too large");
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
  S->ph.gamma = gamma;
  S->ph.dx = dx;
  S->ph.ih = 1.0 / dx;
  S->ph.chem = 0;
  S->ph.regul_mode = 0;
  S->ph.lshield = 0.0;
  S->ph.bdop = 3.0;
  S->ph.xnorm = 5e14;
  S->ph.taud = 1e-21;
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
  if (alloc_pool(S) != MHD_OK) {
    std::string msg = g_err;
    mhd_destroy(S);
    g_err = msg;
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
  if (S->pool) cudaFree(S->pool);
  if (S->staging) cudaFree(S->staging);
  if (S->sc) cudaFree(S->sc);
  if (S->sc_host) cudaFreeHost(S->sc_host);
  if (S->diag_part) cudaFree(S->diag_part);
  if (S->diag_host) cudaFreeHost(S->diag_host);
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
      break;
    case MHD_OPT_CHEM_BDOP:
      if (!(v > 0.0)) return fail(MHD_EINVAL, "Doppler parameter must be > 0");
      S->ph.bdop = v;
      break;
    case MHD_OPT_CHEM_XNORM:
      if (!(v > 0.0)) return fail(MHD_EINVAL, "x normaliser must be > 0");
      S->ph.xnorm = v;
      break;
    case MHD_OPT_CHEM_TAUD:
      if (v < 0.0) return fail(MHD_EINVAL, "dust opacity must be >= 0");
      S->ph.taud = v;
      break;
    case MHD_OPT_GRAPH:
      S->use_graph = v != 0.0;
      break;
    default:
      return fail(MHD_EINVAL, "unknown option key " + std::to_string(key));
  }
  S->graph_valid = false;  // kernel arguments are baked into the captured graph
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
    rc = S->precision ? load_state(S, S->b32, p) : load_state(S, S->b64, p);
  } else {
    const float* p[9];
    for (int q = 0; q < 9; ++q) p[q] = (const float*)dev[q];
    rc = S->precision ? load_state(S, S->b32, p) : load_state(S, S->b64, p);
  }
  if (rc != MHD_OK) return rc;
  if ((rc = reset_scalars(S)) != MHD_OK) return rc;
  if ((rc = refresh_cfl(S)) != MHD_OK) return rc;
  CK(cudaStreamSynchronize(S->stream));
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
  const Geom& g = S->g;
  if (S->precision) {
    k_faces_copy<float><<<nblk(g.N, 256), 256, 0, S->stream>>>(g, S->b32.s, dev[0], dev[1], dev[2]);
    k_derive_eint<float><<<nblk(g.N, 256), 256, 0, S->stream>>>(g, S->b32.s);
  } else {
    k_faces_copy<double><<<nblk(g.N, 256), 256, 0, S->stream>>>(g, S->b64.s, dev[0], dev[1], dev[2]);
    k_derive_eint<double><<<nblk(g.N, 256), 256, 0, S->stream>>>(g, S->b64.s);
  }
  CK(cudaGetLastError());
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
  for (int q = 0; q < 9; ++q) {
    if (!dst[q])
      dev[q] = nullptr;
    else
      dev[q] = out->on_device ? dst[q] : (void*)(S->staging + (size_t)q * S->g.N * 8);
  }
  int rc;
  if (out->dtype == MHD_F64) {
    double* p[9];
    for (int q = 0; q < 9; ++q) p[q] = (double*)dev[q];
    rc = S->precision ? store_state(S, S->b32, p) : store_state(S, S->b64, p);
  } else {
    float* p[9];
    for (int q = 0; q < 9; ++q) p[q] = (float*)dev[q];
    rc = S->precision ? store_state(S, S->b32, p) : store_state(S, S->b64, p);
  }
  if (rc != MHD_OK) return rc;
  if (!out->on_device)
    for (int q = 0; q < 9; ++q)
      if (dst[q]) CK(cudaMemcpyAsync(dst[q], dev[q], bytes, cudaMemcpyDeviceToHost, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  return MHD_OK;
}

int mhd_get_full(mhd_sim* S, double* eint, double* bx, double* by, double* bz, int on_device) {
  if (!valid(S) || !eint || !bx || !by || !bz) return fail(MHD_EINVAL, "mhd_get_full: null argument");
  const size_t bytes = (size_t)S->g.N * 8;
  double* dst[4] = {eint, bx, by, bz};
  double* dev[4];
  for (int q = 0; q < 4; ++q) dev[q] = on_device ? dst[q] : (double*)(S->staging + q * bytes);
  const Geom& g = S->g;
  if (S->precision)
    k_store_full<float><<<nblk(g.N, 256), 256, 0, S->stream>>>(g, S->b32.s, dev[0], dev[1], dev[2], dev[3]);
  else
    k_store_full<double><<<nblk(g.N, 256), 256, 0, S->stream>>>(g, S->b64.s, dev[0], dev[1], dev[2], dev[3]);
  CK(cudaGetLastError());
  if (!on_device)
    for (int q = 0; q < 4; ++q) CK(cudaMemcpyAsync(dst[q], dev[q], bytes, cudaMemcpyDeviceToHost, S->stream));
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
  const Geom& g = S->g;
  if (S->precision)
    k_load_full<float><<<nblk(g.N, 256), 256, 0, S->stream>>>(g, S->b32.s, dev[0], dev[1], dev[2], dev[3]);
  else
    k_load_full<double><<<nblk(g.N, 256), 256, 0, S->stream>>>(g, S->b64.s, dev[0], dev[1], dev[2], dev[3]);
  CK(cudaGetLastError());
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
  if ((rc = enqueue_step(S)) != MHD_OK) return rc;
  if (dt_taken) {
    if ((rc = read_scalars(S)) != MHD_OK) return rc;
    *dt_taken = S->sc_host->tau;
    if (S->sc_host->flags & 1) return fail(MHD_ENONPHYS, "non-physical state (rho, rho eps <= 0 or non-finite)");
    if (S->sc_host->flags & 2) return fail(MHD_EINVAL, "tau <= 0");
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
  }
  if (steps_done) *steps_done = k;
  return rc;
}

int mhd_sync(mhd_sim* S) {
  if (!valid(S)) return fail(MHD_EINVAL, "mhd_sync: null sim");
  int rc = read_scalars(S);
  if (rc != MHD_OK) return rc;
  if (S->sc_host->flags & 1) return fail(MHD_ENONPHYS, "non-physical state (rho, rho eps <= 0 or non-finite)");
  return MHD_OK;
}

int mhd_stage(mhd_sim* S, int which, double tau) {
  if (!valid(S)) return fail(MHD_EINVAL, "mhd_stage: null sim");
  if (which < 1 || which > 4 || !(tau > 0.0)) return fail(MHD_EINVAL, "mhd_stage: which in 1..4, tau > 0");
  int rc;
  if ((rc = set_params(S, 1.0, 0.0, 1, tau)) != MHD_OK) return rc;
  S->params_dirty = true;
  k_begin_step<<<1, 32, 0, S->stream>>>(S->ph, S->sc);
  const Geom& g = S->g;
  if (S->precision) {
    if (which == 1) launch_euler_stage(S, S->b32);
    if (which == 2) launch_lag_stage(S, S->b32);
    if (which >= 3) k_post<float><<<nblk(g.N, 256), 256, 0, S->stream>>>(g, S->ph, S->sc, S->b32.s, which == 3, which == 4);
  } else {
    if (which == 1) launch_euler_stage(S, S->b64);
    if (which == 2) launch_lag_stage(S, S->b64);
    if (which >= 3) k_post<double><<<nblk(g.N, 256), 256, 0, S->stream>>>(g, S->ph, S->sc, S->b64.s, which == 3, which == 4);
  }
  CK(cudaGetLastError());
  if ((rc = refresh_cfl(S)) != MHD_OK) return rc;
  if ((rc = set_params(S, 1.0, 0.0, 0, 0.0)) != MHD_OK) return rc;
  return mhd_sync(S);
}

int mhd_launches_per_step(mhd_sim* S) {
  if (!valid(S)) return fail(MHD_EINVAL, "mhd_launches_per_step: null sim");
  // begin + 3 x (primitives, 3 faces, edges, update) + 3 x (3 faces, update) + post + end
  return 1 + 3 * 6 + 3 * 4 + 1 + 1;
}

int mhd_profile(mhd_sim* S, double cfl, int steps, double* out_ms, int64_t* out_launches) {
  if (!valid(S) || !out_ms || !out_launches || steps < 1) return fail(MHD_EINVAL, "mhd_profile: bad argument");
  if (!S->has_state) return fail(MHD_EINVAL, "mhd_profile: no state loaded");
  int rc = set_params(S, cfl, 0.0, 0, 0.0);
  if (rc != MHD_OK) return rc;
  S->last_cfl = cfl;
  S->last_tend = 0.0;
  S->params_dirty = false;
  S->profiling = true;
  for (int k = 0; k < steps; ++k) {
    if (S->precision)
      launch_step(S, S->b32);
    else
      launch_step(S, S->b64);
  }
  S->profiling = false;
  cudaError_t e = cudaStreamSynchronize(S->stream);
  for (int c = 0; c < MHD_K_NCLASSES; ++c) {
    out_ms[c] = 0.0;
    out_launches[c] = 0;
  }
  for (size_t q = 0; q < S->prof_cls.size(); ++q) {
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, S->prof_ev[2 * q], S->prof_ev[2 * q + 1]);
    out_ms[S->prof_cls[q]] += ms;
    out_launches[S->prof_cls[q]] += 1;
  }
  for (cudaEvent_t ev : S->prof_ev) cudaEventDestroy(ev);
  S->prof_ev.clear();
  S->prof_cls.clear();
  if (e != cudaSuccess) return fail(MHD_ECUDA, std::string("mhd_profile: ") + cudaGetErrorString(e));
  return mhd_sync(S);
}

int mhd_diagnostics(mhd_sim* S, mhd_diag* out) {
  if (!valid(S) || !out) return fail(MHD_EINVAL, "mhd_diagnostics: null argument");
  const Geom& g = S->g;
  if (S->precision)
    k_diag_partial<float><<<S->diag_blocks, DIAG_THREADS, 0, S->stream>>>(g, S->b32.s, S->diag_part);
  else
    k_diag_partial<double><<<S->diag_blocks, DIAG_THREADS, 0, S->stream>>>(g, S->b64.s, S->diag_part);
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
