// mhd_runtime.cuh -- internal runtime of libmhd.so shared by its translation units: the simulation
// object, the executor that steps a set of boxes with one launch per kernel class, and the
// templated launchers.  The FP64 instances are compiled in mhd.cu (no contraction: every product
// and sum rounded as written); the FP32-bulk instances in mhd_f32.cu (contraction allowed).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>  // header-only; ranges cost nothing unless a profiler is attached

#include <vector>

#include "mhd.h"
#include "mhd_kernels.cuh"

namespace mhd_rt {
using namespace mhd;

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// The index-check flags of the translation unit that includes this header (MHD_CHECK builds; 0
// otherwise), read and optionally cleared.  Each translation unit has its own device word.
static inline unsigned check_flags_of_this_unit(bool clear) {
#ifdef MHD_CHECK
  unsigned v = 0;
  if (cudaMemcpyFromSymbol(&v, ::mhd::g_check_flags, sizeof(v)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (clear) {
    const unsigned z = 0;
    cudaMemcpyToSymbol(::mhd::g_check_flags, &z, sizeof(z));
  }
  return v;
#else
  (void)clear;
  return 0;
#endif
}

// An NVTX range around the enqueueing of one stage of the step, so that a profiler can attribute
// and filter the kernels by the paper's stages (ncu --nvtx --nvtx-include "Lagrangian stage/").
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// kernel classes with their own launch shape
enum KClass { KC_PRIM = 0, KC_EFACE, KC_EDGES, KC_EUPD, KC_LFACE, KC_LUPD, KC_POST, NKC };
// profile class of each kernel class (include/mhd.h, enum mhd_kernel_class)
inline int profile_class(int kc) {
  const int m[NKC] = {MHD_K_PRIM, MHD_K_EULER_FACE, MHD_K_EDGES, MHD_K_EULER_UPDATE,
                      MHD_K_LAG_FACE, MHD_K_LAG_UPDATE, MHD_K_POST};
  return m[kc];
}
// profiler tags: PROF_KC_BASE + kernel class for the tiled kernels, MHD_K_SMALL for the rest
constexpr int PROF_KC_BASE = 100;
inline int report_class(int tag) { return tag >= PROF_KC_BASE ? profile_class(tag - PROF_KC_BASE) : tag; }
// domain of the tiles of each kernel class (per-direction kernels: first of three domains)
// The Lagrangian faces run in pencils (kb_lag_pencil) where the parabolas are FP64: sharing the
// differences, slopes and edge values of neighbouring cells saves FP64 instructions, the bound of
// that path; the FP32 path keeps one thread per face (kb_lag_face).
template <typename T>
constexpr bool lag_in_pencils() { return sizeof(T) == 8; }

// shared memory per thread of the Eulerian pencils: six PPMStreams where they stream
template <typename T>
constexpr size_t euler_pencil_smem() { return euler_streams<T>() ? 6 * 9 * sizeof(T) : 0; }

template <typename T>
inline int class_domain(int kc) {
  const int lag = lag_in_pencils<T>() ? DOM_PENCIL_X : DOM_FACE_X;
  const int m[NKC] = {DOM_CELLS, DOM_PENCIL_X, DOM_LATTICE, DOM_CELLS, lag, DOM_CELLS, DOM_CELLS};
  return m[kc];
}

// launch shape: threads per block (= tile size) and grid = min(tiles, grid_mult x SMs), or one
// block per tile when grid_mult == 0
struct LaunchCfg {
  int block = 256;
  int grid_mult = 0;
};
constexpr int NTILE_SIZES = 4;  // 64, 128, 256, 512
inline int tile_slot(int block) { return block == 64 ? 0 : block == 128 ? 1 : block == 256 ? 2 : 3; }

struct TileTable {
  int* d = nullptr;  // [box..., start...] in one allocation
  int n = 0;
};

// CUDA event pairs around launches while profiling
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> cls;
};

struct PScope {
  Profiler* P;
  cudaStream_t st;
  PScope(Profiler* p, cudaStream_t s, int cls) : P(p), st(s) {
    if (!P || !P->on) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, st);
    P->ev.push_back(e);
    P->cls.push_back(cls);
  }
  ~PScope() {
    if (!P || !P->on) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, st);
    P->ev.push_back(e);
  }
};

// A set of boxes advanced together: one launch per kernel class covers every box.
template <typename T>
struct Exec {
  std::vector<Box<T>> h;  // host copies of the descriptors
  Box<T>* d = nullptr;    // device table
  int nb = 0;
  TileTable tab[NDOM][NTILE_SIZES];
  LaunchCfg cfg[NKC];
  int nsm = 152;
  Profiler* prof = nullptr;
  bool ions = false;      // some box has H+ (reactions 5-8): the kernels with the ion code
  bool x_stage = false;   // the FP32 x sweep may stage its rows in shared memory (kb_euler_x_staged)
  // The three directional sweeps of a stage are independent (each reads the cells and writes its
  // own face arrays): the y and z sweeps run on two side streams forked from and joined to the
  // launching stream, so that each sweep's tail overlaps the others' work.  In a captured step the
  // fork and join become graph edges.
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t fork_ev = nullptr, join_ev[2] = {nullptr, nullptr};
};

template <typename T>
long long domain_size(const Box<T>& B, int dom) {
  const Geom& g = B.g;
  switch (dom) {
    case DOM_CELLS: return g.N;
    case DOM_FACE_X: return (long long)(g.n[0] + 1) * g.n[1] * g.n[2];
    case DOM_FACE_Y: return (long long)g.n[0] * (g.n[1] + 1) * g.n[2];
    case DOM_FACE_Z: return (long long)g.n[0] * g.n[1] * (g.n[2] + 1);
    case DOM_PENCIL_X: return (long long)pencil_segments<T>(g.n[0]) * g.n[1] * g.n[2];
    case DOM_PENCIL_Y: return (long long)g.n[0] * pencil_segments<T>(g.n[1]) * g.n[2];
    case DOM_PENCIL_Z: return (long long)g.n[0] * g.n[1] * pencil_segments<T>(g.n[2]);
    default: return g.NF;
  }
}

template <typename T>
cudaError_t ensure_table(Exec<T>& X, int dom, int block) {
  TileTable& t = X.tab[dom][tile_slot(block)];
  if (t.d) return cudaSuccess;
  std::vector<int> bx, st;
  for (int b = 0; b < X.nb; ++b) {
    long long n = domain_size(X.h[b], dom);
    for (long long s = 0; s < n; s += block) {
      bx.push_back(b);
      st.push_back((int)s);
    }
  }
  t.n = (int)bx.size();
  if (t.n == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(&t.d, sizeof(int) * 2 * (size_t)t.n);
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(t.d, bx.data(), sizeof(int) * t.n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(t.d + t.n, st.data(), sizeof(int) * t.n, cudaMemcpyHostToDevice);
}

template <typename T>
cudaError_t ensure_tables(Exec<T>& X) {
  for (int kc = 0; kc < NKC; ++kc) {
    int dom = class_domain<T>(kc);
    int ndom = (dom == DOM_FACE_X || dom == DOM_PENCIL_X) ? 3 : 1;
    for (int q = 0; q < ndom; ++q) {
      cudaError_t e = ensure_table(X, dom + q, X.cfg[kc].block);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

template <typename T>
Tiles tiles_of(const Exec<T>& X, int dom, int block) {
  const TileTable& t = X.tab[dom][tile_slot(block)];
  Tiles r;
  r.box = t.d;
  r.start = t.d + t.n;
  r.n = t.n;
  return r;
}

inline unsigned grid_of(const Tiles& t, const LaunchCfg& c, int nsm) {
  long long g = t.n;
  if (c.grid_mult > 0 && (long long)c.grid_mult * nsm < g) g = (long long)c.grid_mult * nsm;
  return (unsigned)(g > 0 ? g : 1);
}

// default launch shapes: the face kernels are register heavy (150-230 registers), so 128-thread
// blocks let two or three blocks share an SM; the rest 256, one block per tile.  The FP32 path's
// HBM-bound cell kernels (primitives, edge EMFs, the two updates) run grid-stride over their tiles
// with a few blocks per SM: on the 256^3 box that takes 0.04, 0.11, 0.15 and 0.24 ms per step off
// one block per tile (measured over 128-512 threads and 2-8 blocks per SM).
template <typename T>
void default_cfgs(Exec<T>& X) {
  for (int kc = 0; kc < NKC; ++kc) X.cfg[kc] = LaunchCfg{256, 0};
  X.cfg[KC_EFACE].block = 128;
  X.cfg[KC_LFACE].block = 128;
  if constexpr (sizeof(T) == 4) {
    X.cfg[KC_PRIM] = LaunchCfg{512, 4};
    X.cfg[KC_EDGES] = LaunchCfg{512, 4};
    X.cfg[KC_EUPD] = LaunchCfg{128, 8};
    X.cfg[KC_LUPD] = LaunchCfg{128, 8};
  }
}

// The FP32 x sweep stages the window primitives of its tiles' rows in dynamic shared memory
// (kb_euler_x_staged): 16 bytes of barrier and six primitives of at most (block - 1) / S + 2 rows
// of n_x cells (S pencils per row).  It needs every box's n_x to be a multiple of 4 and the largest
// box's rows to fit in kXStageMax; 0 otherwise, and the launch takes the direct kernel.
constexpr size_t kXStageMax = 200 * 1024;
template <typename T>
size_t euler_x_stage_bytes(const Exec<T>& X, int block) {
  size_t m = 0;
  for (int b = 0; b < X.nb; ++b) {
    const int nx = X.h[b].g.n[0];
    if (nx % 4 != 0) return 0;
    const size_t rows = (size_t)((block - 1) / pencil_segments<T>(nx) + 2);
    const size_t need = 16 + rows * 6 * (size_t)nx * sizeof(T);
    m = need > m ? need : m;
  }
  return m <= kXStageMax ? m : 0;
}

// Kernel attributes of the current device: dynamic shared memory above the 48 KB default for the
// Eulerian pencils that stream their parabolas (up to 256 threads per block).  A kernel template
// instantiated in two translation units is two kernels, so this is instantiated where the launches
// of T are (the float launchers live in their own translation unit).
template <typename T>
cudaError_t prepare_kernels() {
  if constexpr (euler_pencil_smem<T>() == 0)
    return cudaFuncSetAttribute(kb_euler_x_staged<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kXStageMax);
  if constexpr (euler_pencil_smem<T>() > 0) {
    const int bytes = (int)(256 * euler_pencil_smem<T>());
    cudaError_t e = cudaFuncSetAttribute(kb_euler_pencil<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kb_euler_pencil<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kb_euler_pencil<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t exec_init(Exec<T>& X, const std::vector<Box<T>>& boxes) {
  X.h = boxes;
  X.nb = (int)boxes.size();
  X.ions = false;
  for (const Box<T>& b : boxes) X.ions = X.ions || (b.ph.chem && b.ph.ions);
  if (!X.side[0]) {
    for (int k = 0; k < 2; ++k) {
      cudaError_t es = cudaStreamCreateWithFlags(&X.side[k], cudaStreamNonBlocking);
      if (es != cudaSuccess) return es;
      es = cudaEventCreateWithFlags(&X.join_ev[k], cudaEventDisableTiming);
      if (es != cudaSuccess) return es;
    }
    cudaError_t es = cudaEventCreateWithFlags(&X.fork_ev, cudaEventDisableTiming);
    if (es != cudaSuccess) return es;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&X.nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = prepare_kernels<T>();
  if (e != cudaSuccess) return e;
  default_cfgs(X);
  e = cudaMalloc(&X.d, sizeof(Box<T>) * (size_t)X.nb);
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(X.d, X.h.data(), sizeof(Box<T>) * (size_t)X.nb, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  return ensure_tables(X);
}

template <typename T>
void exec_free(Exec<T>& X) {
  for (int d = 0; d < NDOM; ++d)
    for (int q = 0; q < NTILE_SIZES; ++q) {
      if (X.tab[d][q].d) cudaFree(X.tab[d][q].d);
      X.tab[d][q].d = nullptr;
      X.tab[d][q].n = 0;
    }
  if (X.d) cudaFree(X.d);
  X.d = nullptr;
  X.nb = 0;
  X.h.clear();
  for (int k = 0; k < 2; ++k) {
    if (X.side[k]) cudaStreamDestroy(X.side[k]);
    if (X.join_ev[k]) cudaEventDestroy(X.join_ev[k]);
    X.side[k] = nullptr;
    X.join_ev[k] = nullptr;
  }
  if (X.fork_ev) cudaEventDestroy(X.fork_ev);
  X.fork_ev = nullptr;
}

// ------------------------------------------------------------------------------------------------
// launchers
template <typename T, typename K, typename... A>
void launch_ks(Exec<T>& X, cudaStream_t st, int kc, int dom, size_t smem_per_thread, K kernel, A... args) {
  const LaunchCfg& c = X.cfg[kc];
  Tiles t = tiles_of(X, dom, c.block);
  PScope p(X.prof, st, PROF_KC_BASE + kc);  // the profiler records the kernel class
  kernel<<<grid_of(t, c, X.nsm), c.block, smem_per_thread * c.block, st>>>(X.d, t, args...);
}
// the same with the block's dynamic shared memory given in bytes
template <typename T, typename K, typename... A>
void launch_kb(Exec<T>& X, cudaStream_t st, int kc, int dom, size_t bytes, K kernel, A... args) {
  const LaunchCfg& c = X.cfg[kc];
  Tiles t = tiles_of(X, dom, c.block);
  PScope p(X.prof, st, PROF_KC_BASE + kc);
  kernel<<<grid_of(t, c, X.nsm), c.block, bytes, st>>>(X.d, t, args...);
}
template <typename T, typename K, typename... A>
void launch_k(Exec<T>& X, cudaStream_t st, int kc, int dom, K kernel, A... args) {
  launch_ks(X, st, kc, dom, 0, kernel, args...);
}


template <typename T>
void launch_small(Exec<T>& X, cudaStream_t st, int which, double cfl = 0, double t_end = 0,
                  int fixed = 0, double tau = 0) {
  PScope p_(X.prof, st, MHD_K_SMALL);
  unsigned g = nblk(X.nb, 128);
  if (which == 0) kb_begin_step<T><<<g, 128, 0, st>>>(X.d, X.nb);
  if (which == 1) kb_end_step<T><<<g, 128, 0, st>>>(X.d, X.nb);
  if (which == 2) kb_set_params<T><<<g, 128, 0, st>>>(X.d, X.nb, cfl, t_end, fixed, tau);
  if (which == 3) kb_zero_dmax<T><<<g, 128, 0, st>>>(X.d, X.nb);
}

// the x, y, z sweeps sw(dir, stream): forked onto the side streams, or in order on st while the
// per-class profiler runs (its events bracket launches on st)
template <typename T, typename F>
void launch_sweeps(Exec<T>& X, cudaStream_t st, F sw) {
  if (!X.side[0] || (X.prof && X.prof->on)) {
    for (int d = 0; d < 3; ++d) sw(d, st);
    return;
  }
  cudaEventRecord(X.fork_ev, st);
  cudaStreamWaitEvent(X.side[0], X.fork_ev, 0);
  cudaStreamWaitEvent(X.side[1], X.fork_ev, 0);
  sw(0, st);
  sw(1, X.side[0]);
  sw(2, X.side[1]);
  for (int k = 0; k < 2; ++k) {
    cudaEventRecord(X.join_ev[k], X.side[k]);
    cudaStreamWaitEvent(st, X.join_ev[k], 0);
  }
}

template <typename T>
void launch_euler_stage(Exec<T>& X, cudaStream_t st) {
  NvtxRange range("Eulerian stage with Flux-CT (Sec. 2.4, 2.5)");
  // self-gravity: a box with a potential (such sims step alone, never in a batch)
  const bool grav = X.nb == 1 && X.h[0].phi != nullptr;
  for (int r = 0; r < 3; ++r) {
    if (X.ions)
      launch_k(X, st, KC_PRIM, DOM_CELLS, kb_prim<T, true>);
    else
      launch_k(X, st, KC_PRIM, DOM_CELLS, kb_prim<T, false>);
    launch_sweeps(X, st, [&](int d, cudaStream_t s) {
      if (d == 0) {
        if constexpr (!euler_streams<T>()) {
          const size_t xs = X.x_stage ? euler_x_stage_bytes(X, X.cfg[KC_EFACE].block) : 0;
          if (xs > 0) {
            launch_kb(X, s, KC_EFACE, DOM_PENCIL_X, xs, kb_euler_x_staged<T>);
            return;
          }
        }
        launch_ks(X, s, KC_EFACE, DOM_PENCIL_X, euler_pencil_smem<T>(), kb_euler_pencil<T, 0>);
      }
      if (d == 1) launch_ks(X, s, KC_EFACE, DOM_PENCIL_Y, euler_pencil_smem<T>(), kb_euler_pencil<T, 1>);
      if (d == 2) launch_ks(X, s, KC_EFACE, DOM_PENCIL_Z, euler_pencil_smem<T>(), kb_euler_pencil<T, 2>);
    });
    launch_k(X, st, KC_EDGES, DOM_LATTICE, kb_edges<T>);
    if (grav)
      launch_k(X, st, KC_EUPD, DOM_CELLS, kb_euler_update<T, true>, r);
    else
      launch_k(X, st, KC_EUPD, DOM_CELLS, kb_euler_update<T, false>, r);
  }
}

// fuse_last: the last substage's update is left to the fused update and post stage of the step
// (launch_lag_post)
template <typename T>
void launch_lag_stage(Exec<T>& X, cudaStream_t st, bool fuse_last) {
  NvtxRange range("Lagrangian stage (Sec. 2.6)");
  for (int r = 0; r < 3; ++r) {
    launch_sweeps(X, st, [&](int d, cudaStream_t s) {
      if constexpr (lag_in_pencils<T>()) {
        const int dom = DOM_PENCIL_X + d;
        if (X.ions) {
          if (d == 0) launch_k(X, s, KC_LFACE, dom, kb_lag_pencil<T, 0, true>);
          if (d == 1) launch_k(X, s, KC_LFACE, dom, kb_lag_pencil<T, 1, true>);
          if (d == 2) launch_k(X, s, KC_LFACE, dom, kb_lag_pencil<T, 2, true>);
        } else {
          if (d == 0) launch_k(X, s, KC_LFACE, dom, kb_lag_pencil<T, 0, false>);
          if (d == 1) launch_k(X, s, KC_LFACE, dom, kb_lag_pencil<T, 1, false>);
          if (d == 2) launch_k(X, s, KC_LFACE, dom, kb_lag_pencil<T, 2, false>);
        }
      } else {
        const int dom = DOM_FACE_X + d;
        if (X.ions) {
          if (d == 0) launch_k(X, s, KC_LFACE, dom, kb_lag_face<T, 0, true>);
          if (d == 1) launch_k(X, s, KC_LFACE, dom, kb_lag_face<T, 1, true>);
          if (d == 2) launch_k(X, s, KC_LFACE, dom, kb_lag_face<T, 2, true>);
        } else {
          if (d == 0) launch_k(X, s, KC_LFACE, dom, kb_lag_face<T, 0, false>);
          if (d == 1) launch_k(X, s, KC_LFACE, dom, kb_lag_face<T, 1, false>);
          if (d == 2) launch_k(X, s, KC_LFACE, dom, kb_lag_face<T, 2, false>);
        }
      }
    });
    if (r == 2 && fuse_last) break;
    if (X.ions)
      launch_k(X, st, KC_LUPD, DOM_CELLS, kb_lag_update<T, true>, r);
    else
      launch_k(X, st, KC_LUPD, DOM_CELLS, kb_lag_update<T, false>, r);
  }
}

// per-cell stages (bit 0 chemistry, bit 1 heating/cooling) / regularisation / check / CFL of the
// new state (cell_stages = do_reg = check = 0: only the CFL denominator)
template <typename T>
void launch_post(Exec<T>& X, cudaStream_t st, int cell_stages, int do_reg, int check) {
  NvtxRange range("chemistry, heating/cooling, regularisation, CFL (Sec. 2.7-2.9, 2.3)");
  if (X.ions)
    launch_k(X, st, KC_POST, DOM_CELLS, kb_post<T, true>, cell_stages, do_reg, check);
  else
    launch_k(X, st, KC_POST, DOM_CELLS, kb_post<T, false>, cell_stages, do_reg, check);
}

// the last Lagrangian update with the post stage (kb_lag_update_post; the post stage's launch
// shape)
template <typename T>
void launch_lag_post(Exec<T>& X, cudaStream_t st, int cell_stages, int do_reg, int check) {
  NvtxRange range("last Lagrangian update + chemistry, heating/cooling, regularisation, CFL");
  if (X.ions)
    launch_k(X, st, KC_POST, DOM_CELLS, kb_lag_update_post<T, true>, cell_stages, do_reg, check);
  else
    launch_k(X, st, KC_POST, DOM_CELLS, kb_lag_update_post<T, false>, cell_stages, do_reg, check);
}

template <typename T>
void launch_step(Exec<T>& X, cudaStream_t st) {
  NvtxRange range("mhd step");
  launch_small(X, st, 0);
  launch_euler_stage(X, st);
  launch_lag_stage(X, st, true);
  launch_lag_post(X, st, 3, 1, 1);
  launch_small(X, st, 1);
}

// the max CFL denominator of the current state of every box
template <typename T>
cudaError_t launch_cfl(Exec<T>& X, cudaStream_t st) {
  launch_small(X, st, 3);
  launch_post(X, st, 0, 0, 0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_set_params(Exec<T>& X, cudaStream_t st, double cfl, double t_end, int fixed, double tau) {
  launch_small(X, st, 2, cfl, t_end, fixed, tau);
  return cudaGetLastError();
}

}  // namespace mhd_rt

// ------------------------------------------------------------------------------------------------
struct mhd_sim {
  using Geom = mhd::Geom;
  using Phys = mhd::Phys;
  using Scalars = mhd::Scalars;
  Geom g;
  Phys ph;
  int precision = 0;
  int use_graph = 1;
  int x_stage = 0;  // MHD_OPT_X_STAGE
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  char* pool = nullptr;
  size_t pool_bytes = 0;
  char* staging = nullptr;  // 10 * N * 8 bytes for host transfers / dtype conversion
  Scalars* sc = nullptr;
  Scalars* sc_host = nullptr;  // pinned mirror
  int* hflags_host = nullptr;  // host-mapped error flags of the last finished step
  int* hflags_dev = nullptr;   // its device address
  double* diag_part = nullptr;
  double* diag_out = nullptr;
  double* diag_host = nullptr;  // pinned, 9 doubles
  int diag_blocks = 0;
  mhd::Box<double> b64;  // descriptors of this box (one of the two is used)
  mhd::Box<float> b32;
  mhd_rt::Exec<double> x64;  // executor of this box alone
  mhd_rt::Exec<float> x32;
  mhd_rt::Profiler prof;
  cudaGraphExec_t gexec = nullptr;
  bool graph_valid = false;
  bool exec_valid = false;
  bool params_dirty = true;
  double last_cfl = -1.0, last_tend = -1.0;
  bool has_state = false;
  int batched = 0;  // number of batches that reference this sim
  void* grav = nullptr;  // self-gravity resources (mhd_gravity.cu), allocated on first use
};

namespace mhd_rt {

// ------------------------------------------------------------------------------------------------
// self-gravity (mhd_gravity.cu): allocate and point the box at the potential; enqueue the Poisson
// solve of the current density; copy the potential out; release
int grav_prepare(mhd_sim* S);
int grav_solve(mhd_sim* S);
int grav_copy(mhd_sim* S, double* out);
void grav_free(mhd_sim* S);

// per-sim (non-batched) helpers: state transfer and diagnostics.  They take the sim's geometry
// (S->g), not the box descriptor's copy: that copy is refreshed only when the executor is rebuilt,
// so after a boundary option changes it still holds the old boundaries until the next step.
template <typename T, typename In>
cudaError_t load_state(mhd_sim* S, Box<T>& B, const In* const* p) {
  const Geom& g = S->g;
  k_load_cells<T, In><<<nblk(g.N, 256), 256, 0, S->stream>>>(g, B.s, p[0], p[1], p[2], p[3], p[4], p[8]);
  k_faces_from_cells<T, In><<<nblk(g.N, 256), 256, 0, S->stream>>>(g, B.s, p[5], p[6], p[7]);
  k_derive_eint<T><<<nblk(g.N, 256), 256, 0, S->stream>>>(g, B.s);
  return cudaGetLastError();
}

template <typename T, typename Out>
cudaError_t store_state(mhd_sim* S, Box<T>& B, Out* const* p) {
  const Geom& g = S->g;
  k_store_state<T, Out><<<nblk(g.N, 256), 256, 0, S->stream>>>(g, B.s, p[0], p[1], p[2], p[3], p[4], p[5],
                                                                p[6], p[7], p[8]);
  return cudaGetLastError();
}

template <typename T>
cudaError_t set_faces(mhd_sim* S, Box<T>& B, const double* const* b) {
  const Geom& g = S->g;
  k_faces_copy<T><<<nblk(g.N, 256), 256, 0, S->stream>>>(g, B.s, b[0], b[1], b[2]);
  k_derive_eint<T><<<nblk(g.N, 256), 256, 0, S->stream>>>(g, B.s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t store_full(mhd_sim* S, Box<T>& B, double* const* d) {
  k_store_full<T><<<nblk(S->g.N, 256), 256, 0, S->stream>>>(S->g, B.s, d[0], d[1], d[2], d[3]);
  return cudaGetLastError();
}

template <typename T>
cudaError_t load_full(mhd_sim* S, Box<T>& B, const double* const* d) {
  k_load_full<T><<<nblk(S->g.N, 256), 256, 0, S->stream>>>(S->g, B.s, d[0], d[1], d[2], d[3]);
  return cudaGetLastError();
}

template <typename T>
cudaError_t store_ions(mhd_sim* S, Box<T>& B, double* d) {
  k_store_ions<T><<<nblk(S->g.N, 256), 256, 0, S->stream>>>(S->g, B.s, d);
  return cudaGetLastError();
}

template <typename T>
cudaError_t load_ions(mhd_sim* S, Box<T>& B, const double* d) {
  k_load_ions<T><<<nblk(S->g.N, 256), 256, 0, S->stream>>>(S->g, B.s, d);
  return cudaGetLastError();
}

template <typename T>
cudaError_t diag_partial(mhd_sim* S, Box<T>& B) {
  k_diag_partial<T><<<S->diag_blocks, DIAG_THREADS, 0, S->stream>>>(S->g, B.s, S->diag_part);
  return cudaGetLastError();
}

// The FP32 instances live in mhd_f32.cu.
#ifndef MHD_RT_F32_TU
extern template cudaError_t prepare_kernels<float>();
extern template void launch_euler_stage<float>(Exec<float>&, cudaStream_t);
extern template void launch_lag_stage<float>(Exec<float>&, cudaStream_t, bool);
extern template void launch_step<float>(Exec<float>&, cudaStream_t);
extern template void launch_post<float>(Exec<float>&, cudaStream_t, int, int, int);
extern template cudaError_t launch_cfl<float>(Exec<float>&, cudaStream_t);
extern template cudaError_t launch_set_params<float>(Exec<float>&, cudaStream_t, double, double, int, double);
extern template void launch_small<float>(Exec<float>&, cudaStream_t, int, double, double, int, double);
extern template cudaError_t load_state<float, double>(mhd_sim*, Box<float>&, const double* const*);
extern template cudaError_t load_state<float, float>(mhd_sim*, Box<float>&, const float* const*);
extern template cudaError_t store_state<float, double>(mhd_sim*, Box<float>&, double* const*);
extern template cudaError_t store_state<float, float>(mhd_sim*, Box<float>&, float* const*);
extern template cudaError_t set_faces<float>(mhd_sim*, Box<float>&, const double* const*);
extern template cudaError_t store_full<float>(mhd_sim*, Box<float>&, double* const*);
extern template cudaError_t load_full<float>(mhd_sim*, Box<float>&, const double* const*);
extern template cudaError_t diag_partial<float>(mhd_sim*, Box<float>&);
extern template cudaError_t store_ions<float>(mhd_sim*, Box<float>&, double*);
extern template cudaError_t load_ions<float>(mhd_sim*, Box<float>&, const double*);
#endif

}  // namespace mhd_rt
