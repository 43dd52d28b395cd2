// mhd_kernels.cuh -- CUDA kernels of one time step (arXiv:1608.08748, Sec. 2), templated on the
// bulk type T.  Every kernel maps threadIdx.x to the x index so that all loads along any axis are
// coalesced; boundary cells are reached through the periodic / zero-gradient index map.
#pragma once
#include "mhd_device.cuh"

namespace mhd {

// SSP-RK3 (Sec. 2.2): Q = a Q^n + b Q + g tau R for the substages r = 0, 1, 2
__host__ __device__ __forceinline__ double RK3_A(int r) { return r == 0 ? 0.0 : (r == 1 ? 0.75 : 1.0 / 3.0); }
__host__ __device__ __forceinline__ double RK3_B(int r) { return r == 0 ? 1.0 : (r == 1 ? 0.25 : 2.0 / 3.0); }
__host__ __device__ __forceinline__ double RK3_G(int r) { return r == 0 ? 1.0 : (r == 1 ? 0.25 : 2.0 / 3.0); }

// primitives W of every cell: v (3), cell-centred B (3), p, gamma, sqrt(rho)   [Sec. 2 closure,
// Sec. 2.5 centring of B, Sec. 4.3 gamma_eff]
template <typename T>
struct Prim {
  T* v[3];
  T* B[3];
  T* p;
  T* g;
  T* sr;
};

// Eulerian face outputs of one direction: F_mn, F_mt1, F_mt2, F_E, V_n, eA, eB   (Sec. 2.4, 2.5)
template <typename T>
struct FaceOut {
  T* f[8];  // the Lagrangian fluxes use f[0..nv-1]
};

// ------------------------------------------------------------------------------------------------
// Batched execution.  Every step kernel walks a table of tiles; a tile is blockDim.x consecutive
// elements (cells, faces of one direction, or lattice points) of one box, so a warp never spans
// two boxes.  Grid-stride over tiles: a grid smaller than the tile count makes the launch
// persistent.  A single simulation is a table of one box.
template <typename T>
struct Box {
  Geom g;
  Phys ph;
  Scalars* sc;
  State<T> s, s0;
  Prim<T> w;
  FaceOut<T> fo[3];  // Eulerian face outputs; the Lagrangian fluxes reuse fo[d].f[0..nv-1]
  T* e[3];
  int nv;            // advected fields of the Lagrangian stage (6; 7 with rho_H2; 8 with rho_H+)
  const T* phi;      // gravitational potential of the step (nullptr: no self-gravity)
  int* hflags;       // host-mapped copy of the error flags, written at the end of every step
};

struct Tiles {
  const int* box;    // box of tile t
  const int* start;  // first element of tile t inside its box
  int n;             // number of tiles
};

// domains of the tile tables
enum { DOM_CELLS = 0, DOM_FACE_X = 1, DOM_FACE_Y = 2, DOM_FACE_Z = 3, DOM_LATTICE = 4,
       DOM_PENCIL_X = 5, DOM_PENCIL_Y = 6, DOM_PENCIL_Z = 7, NDOM = 8 };

// Faces are solved in pencils of pencil_len<T>() consecutive faces along the sweep direction: the
// thread carries the parabolas (or the stencil) of the left cell from one face to the next, so
// every cell's parabolas are built once per direction (plus one extra cell per pencil).  Measured
// on the 256^3 FP32 and 128^3 FP64 steps: 12 faces for the float pencils (Eulerian faces 7.10 ms
// against 7.40 with 8 and 7.15 with 16), 8 for the double ones (16.6 ms against 17.0 with 12 and
// 17.6 with 16; their register files hold the stream of each face).
template <typename T>
__host__ __device__ constexpr int pencil_len() { return sizeof(T) == 4 ? 12 : 8; }
template <typename T>
__host__ __device__ __forceinline__ int pencil_segments(int n) { return (n + 1 + pencil_len<T>() - 1) / pencil_len<T>(); }

// decode a cell index / a face index of direction D / a lattice index
__device__ __forceinline__ void decode(idx_t t, int e0, int e1, int c[3]) {
  c[0] = t % e0;
  idx_t r = t / e0;
  c[1] = (int)(r % e1);
  c[2] = (int)(r / e1);
}
// the same with the grid's precomputed divisors (t >= 0): a cell index (cells), a face index of
// direction D (D = 0, 1, 2) or a lattice index (D = 3)
template <int D>
__device__ __forceinline__ void decode_fast(const Geom& g, idx_t t, int c[3]) {
  const FastDiv f0 = D == 0 || D == 3 ? g.dn1[0] : g.dn[0];
  const FastDiv f1 = D == 1 || D == 3 ? g.dn1[1] : g.dn[1];
  const unsigned r = fdiv((unsigned)t, f0);
  c[0] = (int)((unsigned)t - r * f0.d);
  const unsigned q = fdiv(r, f1);
  c[1] = (int)(r - q * f1.d);
  c[2] = (int)q;
}
// a cell index with the precomputed divisors of n_x and n_y
__device__ __forceinline__ void decode_cell(const Geom& g, idx_t t, int c[3]) {
  const unsigned r = fdiv((unsigned)t, g.dn[0]);
  c[0] = (int)((unsigned)t - r * g.dn[0].d);
  const unsigned q = fdiv(r, g.dn[1]);
  c[1] = (int)(r - q * g.dn[1].d);
  c[2] = (int)q;
}

// pencil p of direction D -> (segment along D, the other two indices) in c.  In the FP64 x sweep
// the y index runs fastest, so the threads of a warp share one segment and its face count (the last
// segment of a row is shorter; the FP64 pipe, not the memory system, bounds those kernels); the
// FP32 x sweep keeps the segment fastest for coalescing (the y-fastest order measured 12.9 against
// 8.1 ms per 256^3 step there), and the y and z sweeps run x fastest as the cells do.
template <typename T, int D>
__device__ __forceinline__ void decode_pencil(idx_t p, const int ext[3], int c[3]) {
  if (D == 0 && sizeof(T) == 8) {
    c[1] = p % ext[1];
    const idx_t r = p / ext[1];
    c[0] = (int)(r % ext[0]);
    c[2] = (int)(r / ext[0]);
  } else {
    decode(p, ext[0], ext[1], c);
  }
}

#define MHD_TILE_LOOP(tl) for (int t_ = blockIdx.x; t_ < (tl).n; t_ += gridDim.x)

// Bulk asynchronous copies from global into shared memory (the copy engine moves the bytes; the
// issuing thread spends one instruction per copy) completed on an mbarrier.  Both addresses are
// 16-byte aligned and the size a multiple of 16 bytes; every wait on the barrier is bounded.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned dynamic_smem_bytes() {
  unsigned r;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void mbar_init(unsigned bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// the one arrival of a phase, announcing the bytes its copies will deliver
__device__ __forceinline__ void mbar_arrive_expect(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
               "selp.u32 %0, 1, 0, p;\n\t}"
               : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}
// waits for the phase of the given parity, for about a second at most; false if it gave up
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity) {
  const long long t0 = clock64();
  for (unsigned it = 0; it < (1u << 26); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > 2000000000ll) break;
  }
  return false;
}
// the error flag of a bulk copy that did not complete in time (bit 2 of Scalars::flags)
constexpr int FLAG_COPY_TIMEOUT = 4;

// ------------------------------------------------------------------------------------------------
// primitives of one cell (IONS: the kernel may see boxes with H+, whose gamma_eff counts it)
template <typename T, bool IONS>
__device__ __forceinline__ void prim_cell(const Box<T>& B, idx_t c) {
  const Geom& g = B.g;
  int q[3];
  decode_cell(g, c, q);
  const T rho = B.s.rho[c];
  idx_t up[3] = {cmap(g, q[0] + 1, q[1], q[2]), cmap(g, q[0], q[1] + 1, q[2]), cmap(g, q[0], q[1], q[2] + 1)};
  T Bc[3], m[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    Bc[d] = T(0.5) * (B.s.b[d][c] + B.s.b[d][up[d]]);
    m[d] = B.s.m[d][c];
  }
  const T eint = B.s.eint[c];
  // gamma_eff in the bulk type: the FP32-bulk path's fluxes are FP32
  T gmt = !B.ph.chem ? (T)B.ph.gamma
          : (IONS && B.ph.ions) ? gamma_eff(rho, B.s.rh2[c], B.s.rhp[c]) : gamma_eff(rho, B.s.rh2[c]);
  const T irho = rcp_t(rho);  // one reciprocal for the three velocities
#pragma unroll
  for (int d = 0; d < 3; ++d) B.w.B[d][c] = Bc[d];
#pragma unroll
  for (int d = 0; d < 3; ++d) B.w.v[d][c] = m[d] * irho;
  B.w.p[c] = (gmt - T(1)) * eint;
  B.w.g[c] = gmt;
  B.w.sr[c] = sqrt_t(rho);
}

template <typename T, bool IONS>
__global__ void __launch_bounds__(512) kb_prim(const Box<T>* __restrict__ boxes, Tiles tl) {
  MHD_TILE_LOOP(tl) {
    const Box<T>& B = boxes[tl.box[t_]];
    idx_t c = tl.start[t_] + (idx_t)threadIdx.x;
    if (c < B.g.N) prim_cell<T, IONS>(B, c);
  }
}

// ------------------------------------------------------------------------------------------------
// Eulerian pencils that stream their parabolas (the FP64 path: its bound is FP64 instructions)
template <typename T>
__host__ __device__ constexpr bool euler_streams() { return sizeof(T) == 8; }

// The Eulerian pencils that stream their parabolas keep each primitive's PPMStream in this thread's
// slots of dynamic shared memory between faces (9 values x 6 primitives; value k of primitive v at
// [(9 v + k) blockDim.x + threadIdx.x], so a warp's accesses are consecutive).
template <typename T>
__device__ __forceinline__ T& stream_slot(int v, int k) {
  extern __shared__ __align__(16) unsigned char stream_smem_raw[];
  T* sm = reinterpret_cast<T*>(stream_smem_raw);
  return sm[(9 * v + k) * blockDim.x + threadIdx.x];
}
template <typename T>
__device__ __forceinline__ void stream_save(const PPMStream<T>& S, int v) {
  stream_slot<T>(v, 0) = S.qm;
  stream_slot<T>(v, 1) = S.q0;
  stream_slot<T>(v, 2) = S.qp;
  stream_slot<T>(v, 3) = S.dp;
  stream_slot<T>(v, 4) = S.h0;
  stream_slot<T>(v, 5) = S.eL;
  stream_slot<T>(v, 6) = S.Cm;
  stream_slot<T>(v, 7) = S.C0;
  stream_slot<T>(v, 8) = S.s0;
}
template <typename T>
__device__ __forceinline__ PPMStream<T> stream_load(int v) {
  PPMStream<T> S;
  S.qm = stream_slot<T>(v, 0);
  S.q0 = stream_slot<T>(v, 1);
  S.qp = stream_slot<T>(v, 2);
  S.dp = stream_slot<T>(v, 3);
  S.h0 = stream_slot<T>(v, 4);
  S.eL = stream_slot<T>(v, 5);
  S.Cm = stream_slot<T>(v, 6);
  S.C0 = stream_slot<T>(v, 7);
  S.s0 = stream_slot<T>(v, 8);
  return S;
}

// The fluxes of one Eulerian face f of direction D from its Riemann solution q* = (V_n, V_t1, V_t2,
// B_t1, B_t2, P) and the face field B_n (the non-advective parts of Sec. 2, reading A12), and the
// two EMF contributions E = B x U of Sec. 2.5.
template <typename T>
__device__ __forceinline__ void store_face_fluxes(const FaceOut<T>& fo, idx_t f, T Bn, const T qs[6]) {
  T Vn = qs[0], Vt1 = qs[1], Vt2 = qs[2], Bt1 = qs[3], Bt2 = qs[4], P = qs[5];
  T pstar = P + T(0.5) * (Bn * Bn + Bt1 * Bt1 + Bt2 * Bt2);
  fo.f[0][f] = pstar - Bn * Bn;
  fo.f[1][f] = -(Bn * Bt1);
  fo.f[2][f] = -(Bn * Bt2);
  fo.f[3][f] = pstar * Vn - Bn * (Bn * Vn + Bt1 * Vt1 + Bt2 * Vt2);
  fo.f[4][f] = Vn;
  fo.f[5][f] = Bn * Vt1 - Bt1 * Vn;
  fo.f[6][f] = Bt2 * Vn - Bn * Vt2;
}

// The FP32 Eulerian pencil: the five-cell stencil of each of the six primitives slides along the
// pencil in registers (register moves; the loop over the faces stays rolled, since eight unrolled
// copies of the Riemann solve overflow the instruction cache), and the left cell's density, gamma
// and sqrt(rho) are carried from the previous face: ten loads per face instead of forty-three.
// Each cell's limited slope is formed once and carried to the parabolas of the next two cells
// (ppm_carried; the same operations on the same numbers as the five-point ppm_direct).  Where all
// cells f0 - 3 .. f1 + 1 of the pencil lie inside the grid they are addressed as base + i * stride
// without the boundary map.
//
// STG (the x sweep only): the six window primitives of the pencil's row are read from shared memory,
// srow[v * fs + x] for x in [0, n_x), where the block staged them (kb_euler_x_staged); the boundary map
// then only wraps or clamps x within the row.
template <typename T, int D, bool STG = false>
__device__ __forceinline__ void euler_pencil_window(const Box<T>& B, idx_t p, const T* srow = nullptr,
                                                    int fs = 0) {
  static_assert(!STG || D == 0, "rows are staged for the x sweep only");
  constexpr int D1 = (D + 1) % 3, D2 = (D + 2) % 3;
  const Geom& g = B.g;
  int ext[3] = {g.n[0], g.n[1], g.n[2]};
  const int n = g.n[D], nf = n + 1;
  ext[D] = pencil_segments<T>(n);
  int c[3];
  decode_pencil<T, D>(p, ext, c);
  const int f0 = c[D] * pencil_len<T>();
  const int nfp = (f0 + pencil_len<T>() < nf ? f0 + pencil_len<T>() : nf) - f0;
  const T tau_h = (T)B.sc->tau_h;
  const bool inside = f0 >= 3 && f0 + nfp + 2 <= n;
  int c0[3] = {c[0], c[1], c[2]};
  c0[D] = 0;
  const idx_t base = cidx(g, c0[0], c0[1], c0[2]);
  const idx_t stride = D == 0 ? 1 : (D == 1 ? g.n[0] : g.n[0] * g.n[1]);
  auto cell_at = [&](int i) -> idx_t {
    if (inside) return MHD_CELL(g, base + i * stride);
    int cc[3] = {c[0], c[1], c[2]};
    cc[D] = i;
    return cmap(g, cc[0], cc[1], cc[2]);
  };
  int cf[3] = {c[0], c[1], c[2]};
  cf[D] = f0;
  const idx_t fbase = fidx(g, cf[0], cf[1], cf[2]);
  const idx_t fstride = D == 0 ? 1 : (D == 1 ? (idx_t)(g.n[0] + 1) : (idx_t)(g.n[0] + 1) * (g.n[1] + 1));
  const T* qv[6] = {B.w.v[D], B.w.v[D1], B.w.v[D2], B.w.B[D1], B.w.B[D2], B.w.p};
  // the six window primitives of cell i along the pencil
  auto load6 = [&](int i, T out[6]) {
    if constexpr (STG) {
      const int x = inside ? i : wrap(i, n, g.bc[0]);
#pragma unroll
      for (int v = 0; v < 6; ++v) out[v] = srow[v * fs + x];
    } else {
      const idx_t q = cell_at(i);
#pragma unroll
      for (int v = 0; v < 6; ++v) out[v] = qv[v][q];
    }
  };
  T w[6][5];  // cells j - 2 .. j + 2 of the parabola of cell j
#pragma unroll
  for (int o = 0; o < 5; ++o) {
    T col[6];
    load6(f0 - 3 + o, col);
#pragma unroll
    for (int v = 0; v < 6; ++v) w[v][o] = col[v];
  }
  Para<T> pl[6], pr[6];
  T sa[6], sb[6];  // the slopes of cells i - 1 and i, carried to the parabola of cell i
#pragma unroll
  for (int v = 0; v < 6; ++v) {
    pl[v] = ppm_direct(w[v][0], w[v][1], w[v][2], w[v][3], w[v][4]);  // cell f0 - 1
    sa[v] = slope_m(w[v][1], w[v][2], w[v][3]);
    sb[v] = slope_m(w[v][2], w[v][3], w[v][4]);
  }
  T rl, gl, sl;  // density, gamma and sqrt(rho) of the face's left cell
  {
    const idx_t q = cell_at(f0 - 1);
    rl = B.s.rho[q];
    gl = B.w.g[q];
    sl = B.w.sr[q];
  }
  // the loads of a face are issued one face ahead, so that their latency overlaps the previous
  // face's Riemann solve: the new stencil cell i + 2 and the right cell i (density, gamma,
  // sqrt(rho), face field)
  T nq[6], nr, ng, ns, nb;
  {
    const idx_t cr = cell_at(f0);
    load6(f0 + 2, nq);
    nr = B.s.rho[cr];
    ng = B.w.g[cr];
    ns = B.w.sr[cr];
    nb = B.s.b[D][cr];
  }
#pragma unroll 1
  for (int k = 0; k < pencil_len<T>(); ++k) {
    if (k < nfp) {
      const int i = f0 + k;
      // the left cell's p, B_t1, B_t2 are the centre of the window before it slides
      const T pL = w[5][2], b1L = w[3][2], b2L = w[4][2];
#pragma unroll
      for (int v = 0; v < 6; ++v) {
        w[v][0] = w[v][1];
        w[v][1] = w[v][2];
        w[v][2] = w[v][3];
        w[v][3] = w[v][4];
        w[v][4] = nq[v];
      }
      const T rr = nr, gr = ng, sr = ns, Bn = nb;
      if (k + 1 < nfp) {
        const idx_t cr = cell_at(i + 1);
        load6(i + 3, nq);
        nr = B.s.rho[cr];
        ng = B.w.g[cr];
        ns = B.w.sr[cr];
        nb = B.s.b[D][cr];
      }
#pragma unroll
      for (int v = 0; v < 6; ++v) {  // cell i
        const T sc = slope_m(w[v][2], w[v][3], w[v][4]);
        pr[v] = ppm_carried(w[v][1], w[v][2], w[v][3], sa[v], sb[v], sc, w[v][4] - T(2) * w[v][3] + w[v][2],
                            w[v][2] - T(2) * w[v][1] + w[v][0]);
        sa[v] = sb[v];
        sb[v] = sc;
      }
      const T wl[6] = {rl, pL, gl, b1L, b2L, sl};
      const T wr[6] = {rr, w[5][2], gr, w[3][2], w[4][2], sr};
      T qs[6];
      riemann(wl, wr, Bn, pl, pr, tau_h, qs);
      store_face_fluxes(B.fo[D], MHD_LATTICE(g, fbase + k * fstride), Bn, qs);
#pragma unroll
      for (int v = 0; v < 6; ++v) {
        pl[v].R = pr[v].L + pr[v].d;  // q^R of cell i again, so that it need not live across the solve
        pl[v].d = pr[v].d;
        pl[v].q6 = pr[v].q6;
      }
      rl = rr;
      gl = gr;
      sl = sr;
    }
  }
}

// Eulerian faces of direction D (Sec. 2.4): the face i_D - 1/2 lies between cells i_D - 1 and i_D.
// One thread takes the faces i_D in [s P, min((s+1) P, n_D + 1)), P = pencil_len<T>(), of one pencil s (the
// other two indices in [0, n)); each cell's parabolas are built once and serve both its faces.
// Per face: the PPM parabolas of (v_n, v_t1, v_t2, B_t1, B_t2, p) of the two cells, the Riemann
// solve, and the non-advective fluxes with the two EMF contributions E = B x U (Sec. 2.5).  The
// FP64 form streams the parabolas (PPMStream in shared memory); the FP32 form slides the stencil.
template <typename T, int D>
__device__ __forceinline__ void euler_pencil(const Box<T>& B, idx_t p) {
  if constexpr (!euler_streams<T>()) {
    euler_pencil_window<T, D>(B, p);
    return;
  }
  constexpr int D1 = (D + 1) % 3, D2 = (D + 2) % 3;
  const Geom& g = B.g;
  int ext[3] = {g.n[0], g.n[1], g.n[2]};
  const int nf = g.n[D] + 1;
  ext[D] = pencil_segments<T>(g.n[D]);
  int c[3];
  decode_pencil<T, D>(p, ext, c);
  const int f0 = c[D] * pencil_len<T>();
  const int f1 = f0 + pencil_len<T>() < nf ? f0 + pencil_len<T>() : nf;
  const T tau_h = (T)B.sc->tau_h;
  const T* qv[6] = {B.w.v[D], B.w.v[D1], B.w.v[D2], B.w.B[D1], B.w.B[D2], B.w.p};
  auto cell_at = [&](int i) {
    int cc[3] = {c[0], c[1], c[2]};
    cc[D] = i;
    return cmap(g, cc[0], cc[1], cc[2]);
  };
  Para<T> pl[6], pr[6];
  {
    idx_t cell[5];
#pragma unroll
    for (int o = 0; o < 5; ++o) cell[o] = cell_at(f0 - 3 + o);
#pragma unroll
    for (int v = 0; v < 6; ++v) {
      PPMStream<T> S;
      S.prime(qv[v][cell[0]], qv[v][cell[1]], qv[v][cell[2]], qv[v][cell[3]]);
      pl[v] = S.next(qv[v][cell[4]]);  // cell f0 - 1
      stream_save(S, v);
    }
  }
  for (int i = f0; i < f1; ++i) {
    idx_t cell[5];
#pragma unroll
    for (int o = 0; o < 5; ++o) cell[o] = cell_at(i - 2 + o);
#pragma unroll
    for (int v = 0; v < 6; ++v) {
      PPMStream<T> S = stream_load<T>(v);
      pr[v] = S.next(qv[v][cell[4]]);  // cell i
      stream_save(S, v);
    }
    idx_t cl = cell[1], cr = cell[2];
    T wl[6] = {B.s.rho[cl], B.w.p[cl], B.w.g[cl], B.w.B[D1][cl], B.w.B[D2][cl], B.w.sr[cl]};
    T wr[6] = {B.s.rho[cr], B.w.p[cr], B.w.g[cr], B.w.B[D1][cr], B.w.B[D2][cr], B.w.sr[cr]};
    T Bn = B.s.b[D][cr];
    T qs[6];
    riemann(wl, wr, Bn, pl, pr, tau_h, qs);
    T Vn = qs[0], Vt1 = qs[1], Vt2 = qs[2], Bt1 = qs[3], Bt2 = qs[4], P = qs[5];
    T pstar = P + T(0.5) * (Bn * Bn + Bt1 * Bt1 + Bt2 * Bt2);
    int cf[3] = {c[0], c[1], c[2]};
    cf[D] = i;
    idx_t f = fidx(g, cf[0], cf[1], cf[2]);
    const FaceOut<T>& fo = B.fo[D];
    fo.f[0][f] = pstar - Bn * Bn;
    fo.f[1][f] = -(Bn * Bt1);
    fo.f[2][f] = -(Bn * Bt2);
    fo.f[3][f] = pstar * Vn - Bn * (Bn * Vn + Bt1 * Vt1 + Bt2 * Vt2);
    fo.f[4][f] = Vn;
    fo.f[5][f] = Bn * Vt1 - Bt1 * Vn;
    fo.f[6][f] = Bt2 * Vn - Bn * Vt2;
#pragma unroll
    for (int v = 0; v < 6; ++v) pl[v] = pr[v];
  }
}

// The FP32 x sweep with the window primitives of its rows staged in shared memory.  A tile is
// blockDim.x consecutive x pencils (the segments of a row fastest), so its pencils lie in rows
// r_lo .. r_hi of the box (row r = k n_y + j, the cells r n_x .. r n_x + n_x - 1).  The six window
// primitives of those rows are brought into shared memory by bulk copies, one per row and
// primitive, issued by the lanes of the first warp; the threads then read their windows there
// instead of with global loads whose lanes lie 12 cells apart (12 cache lines per warp load).  Rows
// need n_x a multiple of 4 (16-byte rows) and the launch's dynamic shared memory to hold them
// (16 bytes of barrier, then [primitive][row][x]): the launcher takes this kernel only where every
// box qualifies, and a tile that does not (which the launcher rules out) is flagged, not solved.
// The results are those of kb_euler_pencil<T, 0> bit for bit.  It is opt-in (MHD_OPT_X_STAGE): on
// GB300 the x sweep measured slower with it (119 against 111 us per 128^3 launch), since the shared
// memory takes L1 capacity from the sweep's other strided accesses (L1 hit rate 38 -> 16 %), and
// staging all ten input fields as well (72 KB per block) kept the concurrent y and z sweeps' blocks
// off the SMs.
template <typename T>
__global__ void __launch_bounds__(256, 2) kb_euler_x_staged(const Box<T>* __restrict__ boxes, Tiles tl) {
  extern __shared__ __align__(16) unsigned char stream_smem_raw[];
  T* rows = reinterpret_cast<T*>(stream_smem_raw + 16);
  const unsigned bar = smem_u32(stream_smem_raw), rows_s = smem_u32(rows);
  const unsigned cap = dynamic_smem_bytes();
  if (threadIdx.x == 0 && cap >= 16) mbar_init(bar);
  __syncthreads();
  unsigned parity = 0;
  MHD_TILE_LOOP(tl) {
    const Box<T>& B = boxes[tl.box[t_]];
    const int nx = B.g.n[0], S = pencil_segments<T>(nx);
    const idx_t total = (idx_t)S * B.g.n[1] * B.g.n[2];
    const idx_t p0 = tl.start[t_], p = p0 + (idx_t)threadIdx.x;
    const idx_t pe = p0 + (idx_t)blockDim.x < total ? p0 + (idx_t)blockDim.x : total;
    const int r_lo = p0 / S, nrows = (int)((pe - 1) / S) - r_lo + 1;
    const unsigned bytes = (unsigned)nrows * 6u * (unsigned)nx * (unsigned)sizeof(T);
    if (nx % 4 != 0 || 16u + bytes > cap) {  // the same for every thread of the block
      if (threadIdx.x == 0) atomicOr(&B.sc->flags, FLAG_COPY_TIMEOUT);
      continue;
    }
    __syncthreads();  // every thread is done with the previous tile's rows
    if (threadIdx.x < 32) {
      if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect(bar, bytes);
      }
      const T* src[6] = {B.w.v[0], B.w.v[1], B.w.v[2], B.w.B[1], B.w.B[2], B.w.p};
      for (int q = (int)threadIdx.x; q < 6 * nrows; q += 32) {
        const int v = q / nrows, lr = q - v * nrows;
        bulk_copy_g2s(rows_s + (unsigned)((v * nrows + lr) * nx) * (unsigned)sizeof(T),
                      src[v] + (size_t)(r_lo + lr) * nx, (unsigned)nx * (unsigned)sizeof(T), bar);
      }
    }
    const unsigned phase = parity;
    parity ^= 1u;
    const bool ok = mbar_wait_bounded(bar, phase);
    if (__syncthreads_or(!ok)) {
      // a copy did not arrive in time: flag it, give the copies in flight one more bounded wait,
      // and leave
      if (threadIdx.x == 0) atomicOr(&B.sc->flags, FLAG_COPY_TIMEOUT);
      mbar_wait_bounded(bar, phase);
      return;
    }
    if (p < total) euler_pencil_window<T, 0, true>(B, p, rows + (int)(p / S - r_lo) * nx, nrows * nx);
  }
}

template <typename T, int D>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) kb_euler_pencil(const Box<T>* __restrict__ boxes, Tiles tl) {
  MHD_TILE_LOOP(tl) {
    const Box<T>& B = boxes[tl.box[t_]];
    idx_t p = tl.start[t_] + (idx_t)threadIdx.x;
    idx_t total = (idx_t)(D == 0 ? pencil_segments<T>(B.g.n[0]) : B.g.n[0]) *
                      (D == 1 ? pencil_segments<T>(B.g.n[1]) : B.g.n[1]) *
                      (D == 2 ? pencil_segments<T>(B.g.n[2]) : B.g.n[2]);
    if (p < total) euler_pencil<T, D>(B, p);
  }
}

// App. C: edge EMFs.  E_d at the corner (i_{d+1} - 1/2, i_{d+2} - 1/2) of lattice point c, for
// c_d in [0, n_d) and c_{d+1}, c_{d+2} in [0, n]: the mean of the two faces of direction d+1 and
// the two of direction d+2 that share the edge.
template <typename T>
__device__ __forceinline__ void edges_point(const Box<T>& B, idx_t t) {
  const Geom& g = B.g;
  int c[3];
  decode_fast<3>(g, t, c);
  T e[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
    e[d] = T(0);
    if (c[d] >= g.n[d]) continue;
    int a[3] = {c[0], c[1], c[2]};
    a[d2] = wrap(c[d2], g.n[d2], g.bc[d2]);
    int alo[3] = {c[0], c[1], c[2]};
    alo[d2] = wrap(c[d2] - 1, g.n[d2], g.bc[d2]);
    T f1 = B.fo[d1].f[5][fidx(g, alo[0], alo[1], alo[2])] + B.fo[d1].f[5][fidx(g, a[0], a[1], a[2])];
    int b[3] = {c[0], c[1], c[2]};
    b[d1] = wrap(c[d1], g.n[d1], g.bc[d1]);
    int blo[3] = {c[0], c[1], c[2]};
    blo[d1] = wrap(c[d1] - 1, g.n[d1], g.bc[d1]);
    T f2 = B.fo[d2].f[6][fidx(g, blo[0], blo[1], blo[2])] + B.fo[d2].f[6][fidx(g, b[0], b[1], b[2])];
    e[d] = T(0.25) * (f1 + f2);
  }
#pragma unroll
  for (int d = 0; d < 3; ++d)
    if (c[d] < g.n[d]) B.e[d][t] = e[d];
}

template <typename T>
__global__ void __launch_bounds__(512) kb_edges(const Box<T>* __restrict__ boxes, Tiles tl) {
  MHD_TILE_LOOP(tl) {
    const Box<T>& B = boxes[tl.box[t_]];
    idx_t t = tl.start[t_] + (idx_t)threadIdx.x;
    if (t < B.g.NF) edges_point(B, t);
  }
}

// SSP-RK3 combination of Sec. 2.2 for one value: a Q^n + b Q + g tau R, with g tau R = gth S for a
// flux-difference sum S (R = S / h, gth = g tau / h once per thread).  The first substage has
// a = 0, b = g = 1 and returns Q + gth S; its caller stores Q^n (the stage's start value, the Q it
// read) in the RK register, which later substages read as q0.  (The FP64 update kernels are bound
// by the FP64 pipe, so the constants are folded.)
template <typename T>
__device__ __forceinline__ T rk_value(T q, T q0, T a, T b, T gthS, int r) {
  return r == 0 ? q + gthS : (a * q0 + b * q) + gthS;
}

// The cell kernels (primitives, edge EMFs, and the two updates in FP32) issue every load of a cell
// before its first store.  A thread stores only its own cell (or edge), which no load of the kernel
// reads, so the order is free; the compiler cannot prove that (all fields are plain pointers), and
// a store between two loads costs the thread one DRAM latency per stored field.  The FP64 updates
// keep the order field by field: holding all their loads would double their registers and halve
// the resident warps, and at the FP64 path's sizes that costs more than the latencies.
template <typename T>
__host__ __device__ constexpr bool update_loads_first() { return sizeof(T) == 4; }
// g tau / h of substage r
template <typename T>
__device__ __forceinline__ T rk_gth(const Box<T>& B, int r) {
  return (T)(RK3_G(r) * B.sc->tau * B.ph.ih);
}

// Eulerian update of one cell: finite-volume R of m, rho E, rho eps (Sec. 2.4 + A12), Flux-CT of
// the cell's three faces (Sec. 2.5), SSP-RK3 combination (Sec. 2.2) with stage r.
template <typename T, bool GRAV>
__device__ __forceinline__ void euler_update_cell(const Box<T>& B, idx_t c, int r) {
  const Geom& g = B.g;
  int q[3];
  decode_cell(g, c, q);
  const T a = (T)RK3_A(r), bb = (T)RK3_B(r), gth = rk_gth(B, r);
  idx_t f0 = fidx(g, q[0], q[1], q[2]);
  idx_t fup[3] = {fidx(g, q[0] + 1, q[1], q[2]), fidx(g, q[0], q[1] + 1, q[2]), fidx(g, q[0], q[1], q[2] + 1)};
  // -0 + x is x for every x, so the first addition to each sum folds away
  T acc[5] = {T(-0.0), T(-0.0), T(-0.0), T(-0.0), T(-0.0)};  // m_x, m_y, m_z, rho E, -h div V
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
    const FaceOut<T>& o = B.fo[d];
    acc[d] = acc[d] + (o.f[0][f0] - o.f[0][fup[d]]);
    acc[d1] = acc[d1] + (o.f[1][f0] - o.f[1][fup[d]]);
    acc[d2] = acc[d2] + (o.f[2][f0] - o.f[2][fup[d]]);
    acc[3] = acc[3] + (o.f[3][f0] - o.f[3][fup[d]]);
    acc[4] = acc[4] + (o.f[4][f0] - o.f[4][fup[d]]);
  }
  T Rv[5];  // h R: the flux-difference sums, and -(gamma - 1) rho eps h div V
#pragma unroll
  for (int v = 0; v < 4; ++v) Rv[v] = acc[v];
  Rv[4] = ((B.w.g[c] - T(1)) * B.s.eint[c]) * acc[4];
  if (GRAV) {
    // self-gravity (Sec. 2): -rho grad Phi and -rho v . grad Phi, central differences of the
    // potential of the step (periodic box); a separate instance, so that the update without
    // gravity keeps its registers
    const idx_t dn[3] = {cmap(g, q[0] - 1, q[1], q[2]), cmap(g, q[0], q[1] - 1, q[2]), cmap(g, q[0], q[1], q[2] - 1)};
    const idx_t upc[3] = {cmap(g, q[0] + 1, q[1], q[2]), cmap(g, q[0], q[1] + 1, q[2]), cmap(g, q[0], q[1], q[2] + 1)};
    const T rho = B.s.rho[c];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T gd = -(B.phi[upc[d]] - B.phi[dn[d]]) * T(0.5);  // h (-d Phi / dx_d)
      Rv[d] = Rv[d] + rho * gd;
      Rv[3] = Rv[3] + B.s.m[d][c] * gd;
    }
  }
  T* qq[5] = {B.s.m[0], B.s.m[1], B.s.m[2], B.s.E, B.s.eint};
  T* q0[5] = {B.s0.m[0], B.s0.m[1], B.s0.m[2], B.s0.E, B.s0.eint};
  // Flux-CT: d b_d / dt = -(curl E)_d on the face i_d - 1/2 of this cell
  auto curl_of = [&](int d) {
    const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
    return (B.e[d1][fup[d2]] - B.e[d1][f0]) - (B.e[d2][fup[d1]] - B.e[d2][f0]);
  };
  if constexpr (update_loads_first<T>()) {
    T qv[5], q0v[5], bv[3], b0v[3], curl[3];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      qv[v] = qq[v][c];
      q0v[v] = r ? q0[v][c] : T(0);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      bv[d] = B.s.b[d][c];
      b0v[d] = r ? B.s0.b[d][c] : T(0);
      curl[d] = curl_of(d);
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      if (r == 0) q0[v][c] = qv[v];
      qq[v][c] = rk_value(qv[v], q0v[v], a, bb, gth * Rv[v], r);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (r == 0) B.s0.b[d][c] = bv[d];
      B.s.b[d][c] = rk_value(bv[d], b0v[d], a, bb, gth * curl[d], r);
    }
  } else {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const T qv = qq[v][c], q0v = r ? q0[v][c] : T(0);
      if (r == 0) q0[v][c] = qv;
      qq[v][c] = rk_value(qv, q0v, a, bb, gth * Rv[v], r);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T curl = curl_of(d);
      const T bv = B.s.b[d][c], b0v = r ? B.s0.b[d][c] : T(0);
      if (r == 0) B.s0.b[d][c] = bv;
      B.s.b[d][c] = rk_value(bv, b0v, a, bb, gth * curl, r);
    }
  }
}

template <typename T, bool GRAV>
__global__ void __launch_bounds__(512) kb_euler_update(const Box<T>* __restrict__ boxes, Tiles tl, int r) {
  MHD_TILE_LOOP(tl) {
    const Box<T>& B = boxes[tl.box[t_]];
    idx_t c = tl.start[t_] + (idx_t)threadIdx.x;
    if (c < B.g.N) euler_update_cell<T, GRAV>(B, c, r);
  }
}

// ------------------------------------------------------------------------------------------------
// Sec. 2.6 Lagrangian face flux for direction D: F = v_n q(-|v_n| tau) (v_n >= 0, left cell) or
// v_n q(|v_n| tau) (right cell) with v_n the sqrt(rho)-weighted mean of the cell velocities.
template <typename T, int D, bool IONS>
__device__ __forceinline__ void lag_face(const Box<T>& B, idx_t t) {
  const Geom& g = B.g;
  int c[3];
  decode_fast<D>(g, t, c);
  const T tau_h = (T)B.sc->tau_h;
  idx_t cell[6];
  if (c[D] >= 3 && c[D] + 2 < g.n[D]) {
    // the whole stencil inside the grid: a stride from this face's right cell, no boundary map
    const idx_t stride = D == 0 ? 1 : (D == 1 ? g.n[0] : g.n[0] * g.n[1]);
    const idx_t cc = cidx(g, c[0], c[1], c[2]);
#pragma unroll
    for (int o = 0; o < 6; ++o) cell[o] = MHD_CELL(g, cc + (o - 3) * stride);
  } else {
#pragma unroll
    for (int o = 0; o < 6; ++o) {
      int cc[3] = {c[0], c[1], c[2]};
      cc[D] += o - 3;
      cell[o] = cmap(g, cc[0], cc[1], cc[2]);
    }
  }
  idx_t cl = cell[2], cr = cell[3];
  // v_l sqrt(rho_l) = m_l / sqrt(rho_l) and sqrt(rho) = rho / sqrt(rho): two 1/sqrt and a division
  T rl = B.s.rho[cl], rr = B.s.rho[cr];
  T isl = rsqrt_t(rl), isr = rsqrt_t(rr);
  T vn = (B.s.m[D][cl] * isl + B.s.m[D][cr] * isr) * rcp_t(rl * isl + rr * isr);
  T y = fabs(vn) * tau_h;
  const T* q[7] = {B.s.rho, B.s.m[0], B.s.m[1], B.s.m[2], B.s.E, B.s.eint, B.s.rh2};
  idx_t f = fidx(g, c[0], c[1], c[2]);
  const int o0 = vn >= T(0) ? 0 : 1;  // upwind cell: stencil cells o0 .. o0 + 4
  const int nv = B.nv;
  idx_t st[5];
#pragma unroll
  for (int o = 0; o < 5; ++o) st[o] = o0 == 0 ? cell[o] : cell[o + 1];
  auto flux = [&](const T* a, int v) {
    Para<T> P = ppm_lean(a[st[0]], a[st[1]], a[st[2]], a[st[3]], a[st[4]]);
    T qb = o0 == 0 ? avg_right_end(P, y) : avg_left_end(P, y);
    B.fo[D].f[v][f] = vn * qb;
  };
#pragma unroll
  for (int v = 0; v < 7; ++v) {
    if (v >= nv) break;
    flux(q[v], v);
  }
  if (IONS) {
#pragma unroll 1
    for (int v = 7; v < nv; ++v) flux(B.s.rhp, v);  // rho_H+ (ions on)
  }
}

template <typename T, int D, bool IONS>
__global__ void __launch_bounds__(256) kb_lag_face(const Box<T>* __restrict__ boxes, Tiles tl) {
  MHD_TILE_LOOP(tl) {
    const Box<T>& B = boxes[tl.box[t_]];
    idx_t t = tl.start[t_] + (idx_t)threadIdx.x;
    idx_t total = (idx_t)(B.g.n[0] + (D == 0)) * (B.g.n[1] + (D == 1)) * (B.g.n[2] + (D == 2));
    if (t < total) lag_face<T, D, IONS>(B, t);
  }
}

// The same fluxes for the faces i_D - 1/2, i_D in [s P, min((s+1) P, n_D + 1)), of one
// pencil s: the face velocities first, then field by field the parabolas of the pencil's cells in
// one PPMStream along D, each face taking the average of its upwind cell.
template <typename T, int D, bool IONS>
__device__ __forceinline__ void lag_pencil(const Box<T>& B, idx_t p) {
  const Geom& g = B.g;
  int ext[3] = {g.n[0], g.n[1], g.n[2]};
  const int nf = g.n[D] + 1;
  ext[D] = pencil_segments<T>(g.n[D]);
  int c[3];
  decode_pencil<T, D>(p, ext, c);
  const int f0 = c[D] * pencil_len<T>();
  const int nfp = (f0 + pencil_len<T>() < nf ? f0 + pencil_len<T>() : nf) - f0;
  const T tau_h = (T)B.sc->tau_h;
  const T TWO_THIRDS = T(2.0 / 3.0);
  auto cell_at = [&](int i) {
    int cc[3] = {c[0], c[1], c[2]};
    cc[D] = i;
    return cmap(g, cc[0], cc[1], cc[2]);
  };
  int cf[3] = {c[0], c[1], c[2]};
  cf[D] = f0;
  const idx_t fbase = fidx(g, cf[0], cf[1], cf[2]);
  const idx_t fstride = D == 0 ? 1 : (D == 1 ? (idx_t)(g.n[0] + 1) : (idx_t)(g.n[0] + 1) * (g.n[1] + 1));
  // per face: v_n, and the average over the upwind fraction y = |v_n| tau / h written as
  // E + shy (d + sgn q6 w) with E = q^R of the left cell (v_n >= 0, sgn = -1) or q^L of the right
  // cell (sgn = +1), shy = sgn y / 2 and w = 1 - 2y/3 (the two forms of Sec. 2.4)
  T vn[pencil_len<T>()], shy[pencil_len<T>()], w[pencil_len<T>()];
  // v_n = (v_l sqrt(rho_l) + v_r sqrt(rho_r)) / (sqrt(rho_l) + sqrt(rho_r)) from the per-cell
  // m / sqrt(rho) and rho / sqrt(rho) = sqrt(rho), each formed once and carried to the next face
  T al, bl;
  {
    const idx_t c0 = cell_at(f0 - 1);
    const T r0 = B.s.rho[c0], is0 = rsqrt_t(r0);
    al = B.s.m[D][c0] * is0;
    bl = r0 * is0;
  }
#pragma unroll
  for (int k = 0; k < pencil_len<T>(); ++k) {
    vn[k] = T(0);
    shy[k] = T(0);
    w[k] = T(1);
    if (k < nfp) {
      const idx_t cr = cell_at(f0 + k);
      const T rr = B.s.rho[cr], isr = rsqrt_t(rr);
      const T ar = B.s.m[D][cr] * isr, br = rr * isr;
      vn[k] = (al + ar) * rcp_t(bl + br);
      al = ar;
      bl = br;
      const T y = abs_b(vn[k]) * tau_h;
      const T hy = scale_down_b<1>(y);
      shy[k] = sign_bit_b(vn[k]) ? hy : neg_b(hy);  // v_n = -0 has y = 0
      w[k] = T(1) - TWO_THIRDS * y;
    }
  }
  const int nv = B.nv;
#pragma unroll 1
  for (int v = 0; v < nv; ++v) {
    const T* a = v == 0 ? B.s.rho : v < 4 ? B.s.m[v - 1] : v == 4 ? B.s.E : v == 5 ? B.s.eint
                 : (IONS && v == 7) ? B.s.rhp : B.s.rh2;
    T* out = B.fo[D].f[v] + fbase;
    PPMStream<T> S;
    S.prime(a[cell_at(f0 - 3)], a[cell_at(f0 - 2)], a[cell_at(f0 - 1)], a[cell_at(f0)]);
    Para<T> Pl = S.next(a[cell_at(f0 + 1)]);  // cell f0 - 1
#pragma unroll
    for (int k = 0; k < pencil_len<T>(); ++k) {
      if (k < nfp) {
        const Para<T> Pr = S.next(a[cell_at(f0 + k + 2)]);  // cell f0 + k
        const bool left = !sign_bit_b(vn[k]);  // v_n = -0: a zero flux either way
        const T E = left ? Pl.R : Pr.L;
        const T d = left ? Pl.d : Pr.d;
        const T q6 = left ? neg_b(Pl.q6) : Pr.q6;
        out[MHD_LATTICE(g, fbase + k * fstride) - fbase] = vn[k] * (E + shy[k] * (d + q6 * w[k]));
        Pl = Pr;
      }
    }
  }
}

template <typename T, int D, bool IONS>
__global__ void __launch_bounds__(256, 1) kb_lag_pencil(const Box<T>* __restrict__ boxes, Tiles tl) {
  MHD_TILE_LOOP(tl) {
    const Box<T>& B = boxes[tl.box[t_]];
    idx_t p = tl.start[t_] + (idx_t)threadIdx.x;
    idx_t total = (idx_t)(D == 0 ? pencil_segments<T>(B.g.n[0]) : B.g.n[0]) *
                      (D == 1 ? pencil_segments<T>(B.g.n[1]) : B.g.n[1]) *
                      (D == 2 ? pencil_segments<T>(B.g.n[2]) : B.g.n[2]);
    if (p < total) lag_pencil<T, D, IONS>(B, p);
  }
}

// IONS: up to 8 advected fields (rho_H+ last), else up to 7
template <typename T, bool IONS>
__device__ __forceinline__ void lag_update_cell(const Box<T>& B, idx_t c, int r) {
  const Geom& g = B.g;
  int q[3];
  decode_cell(g, c, q);
  const T a = (T)RK3_A(r), bb = (T)RK3_B(r), gth = rk_gth(B, r);
  idx_t f0 = fidx(g, q[0], q[1], q[2]);
  idx_t fup[3] = {fidx(g, q[0] + 1, q[1], q[2]), fidx(g, q[0], q[1] + 1, q[2]), fidx(g, q[0], q[1], q[2] + 1)};
  T* qq[8] = {B.s.rho, B.s.m[0], B.s.m[1], B.s.m[2], B.s.E, B.s.eint, B.s.rh2, B.s.rhp};
  T* q0[8] = {B.s0.rho, B.s0.m[0], B.s0.m[1], B.s0.m[2], B.s0.E, B.s0.eint, B.s0.rh2, B.s0.rhp};
  const int nv = B.nv;
  constexpr int NV = IONS ? 8 : 7;
  auto sum_of = [&](int v) {
    T acc = T(-0.0);  // -0 + x is x: the first addition folds away
#pragma unroll
    for (int d = 0; d < 3; ++d) acc = acc + (B.fo[d].f[v][f0] - B.fo[d].f[v][fup[d]]);
    return acc;
  };
  if constexpr (update_loads_first<T>()) {
    // the fields in two halves, each with its loads before its stores: all seven at once kept 21
    // values and the flux sums live at the 64 registers the compiler chose, and measured slower
    // (1.34 against 1.25 ms per 256^3 step)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      constexpr int H = (NV + 1) / 2;
      T acc[H], qv[H], q0v[H];
#pragma unroll
      for (int i = 0; i < H; ++i) {
        const int v = h * H + i;
        acc[i] = qv[i] = q0v[i] = T(0);
        if (v < NV && v < nv) {
          acc[i] = sum_of(v);
          qv[i] = qq[v][c];
          if (r) q0v[i] = q0[v][c];
        }
      }
#pragma unroll
      for (int i = 0; i < H; ++i) {
        const int v = h * H + i;
        if (v < NV && v < nv) {
          if (r == 0) q0[v][c] = qv[i];
          qq[v][c] = rk_value(qv[i], q0v[i], a, bb, gth * acc[i], r);
        }
      }
    }
  } else {

#pragma unroll
    for (int v = 0; v < NV; ++v) {
      if (v >= nv) break;
      const T acc = sum_of(v);
      const T qv = qq[v][c], q0v = r ? q0[v][c] : T(0);
      if (r == 0) q0[v][c] = qv;
      qq[v][c] = rk_value(qv, q0v, a, bb, gth * acc, r);
    }
  }
}

template <typename T, bool IONS>
__global__ void __launch_bounds__(512) kb_lag_update(const Box<T>* __restrict__ boxes, Tiles tl, int r) {
  MHD_TILE_LOOP(tl) {
    const Box<T>& B = boxes[tl.box[t_]];
    idx_t c = tl.start[t_] + (idx_t)threadIdx.x;
    if (c < B.g.N) lag_update_cell<T, IONS>(B, c, r);
  }
}

// ------------------------------------------------------------------------------------------------
// warp-aggregated helpers
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Per cell, after the Lagrangian stage: chemistry (Sec. 2.7, FP64), heating/cooling (Sec. 2.8,
// FP64, when on), regularisation (Sec. 2.9), the non-physical check, and the CFL denominator of the
// new state for the next tau (Sec. 2.3).  cell_stages selects the per-cell stages (bit 0
// chemistry, bit 1 heating/cooling; the full step runs both), do_reg the regularisation;
// cell_stages = do_reg = 0 computes only the CFL denominator.  All lanes of the warp call it (valid
// marks those with a cell): the FP64 denominator is evaluated only where the FP32 screen
// (cfl_estimate_f32) cannot exclude the cell from the maximum, against the largest estimate of the
// warp and the FP64 maximum the box has reached so far; D stays 0 elsewhere.  Returns the flags via
// the warp-aggregated atomics of the caller.
template <typename T, bool IONS>
__device__ __forceinline__ void post_cell(const Box<T>& B, idx_t c, bool valid, int cell_stages,
                                          int do_reg, double& D, int& bad, unsigned& vb) {
  const Geom& g = B.g;
  const Phys& ph = B.ph;
  const bool ions = IONS && ph.ions;
  const State<T>& s = B.s;
  T rho = T(0), m[3] = {T(0), T(0), T(0)}, Bc[3] = {T(0), T(0), T(0)}, eint = T(0), rh2 = T(0), rhp = T(0);
  float D32 = 0.0f;  // 0: no candidate
  if (valid) {
    int q[3];
    decode_cell(g, c, q);
    const double tau = B.sc->tau;
    if ((cell_stages & 1) && ph.chem) {
      const ChemOut co = chem_cell<IONS>(ph, (double)s.rho[c], (double)s.eint[c], (double)s.rh2[c],
                                         ions ? (double)s.rhp[c] : 0.0, tau);
      s.rh2[c] = (T)co.rh2;
      if (ions) s.rhp[c] = (T)co.rhp;
    }
    if ((cell_stages & 2) && ph.chem && ph.heatcool) {
      const double d = heatcool_delta<IONS>(ph, (double)s.rho[c], (double)s.eint[c], (double)s.rh2[c],
                                            ions ? (double)s.rhp[c] : 0.0, tau);
      s.E[c] = (T)((double)s.E[c] + d);
      s.eint[c] = (T)((double)s.eint[c] + d);
    }
    idx_t up[3] = {cmap(g, q[0] + 1, q[1], q[2]), cmap(g, q[0], q[1] + 1, q[2]),
                   cmap(g, q[0], q[1], q[2] + 1)};
#pragma unroll
    for (int d = 0; d < 3; ++d) Bc[d] = T(0.5) * (s.b[d][c] + s.b[d][up[d]]);
    rho = s.rho[c];
#pragma unroll
    for (int d = 0; d < 3; ++d) m[d] = s.m[d][c];
    T E = s.E[c];
    eint = s.eint[c];
    if (do_reg) {
      T m2 = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
      T kin = T(0.5) * m2 / rho;
      T mag = T(0.5) * (Bc[0] * Bc[0] + Bc[1] * Bc[1] + Bc[2] * Bc[2]);
      T e = E - kin - mag;
      T f = e / E;
      bool entropy_branch = f >= T(1e-3);
      if (ph.regul_mode == 2) entropy_branch = !entropy_branch;
      if (entropy_branch) {
        if (ph.regul_mode != 0 || e > eint) eint = e;
      } else {
        T v2 = T(2) * (E - eint - mag) / rho;
        if (v2 < T(0)) v2 = T(0);
        T vnew = sqrt(v2);
        T vold = sqrt(m2) / rho;
        if (vold > T(0)) {
          T scl = vnew / vold;
#pragma unroll
          for (int d = 0; d < 3; ++d) m[d] = m[d] * scl;
        }
        vb = 1;
      }
      s.eint[c] = eint;
#pragma unroll
      for (int d = 0; d < 3; ++d) s.m[d][c] = m[d];
    }
    if (ph.chem) rh2 = s.rh2[c];
    if (ions) rhp = s.rhp[c];
    T vals[11] = {rho, m[0], m[1], m[2], E, eint, rh2, s.b[0][c], s.b[1][c], s.b[2][c], rhp};
#pragma unroll
    for (int k = 0; k < 11; ++k)
      if (!isfinite(vals[k])) bad = 1;
    if (!(rho > T(0)) || !(eint > T(0))) bad = 1;
    if (!bad)
      D32 = cfl_estimate_f32((float)rho, (float)m[0], (float)m[1], (float)m[2], (float)Bc[0], (float)Bc[1],
                             (float)Bc[2], (float)eint,
                             gamma_minus_one_f32(ph.chem, ph.gamma, (float)rho, (float)rh2, (float)rhp));
  }
  // the screen: a finite estimate raised by 2^-12 below the largest finite estimate of the warp
  // lowered by 2^-12 (whose cell is evaluated unless it is excluded too), or below the FP64 maximum
  // reached so far, excludes the cell
  const float wmax = warp_max_f(D32 <= 3.0e38f ? D32 : 0.0f);
  const double reached = __longlong_as_double(*(volatile long long*)&B.sc->dmax);
  const float bound = fmaxf(__double2float_rd(reached), wmax * (1.0f - 0x1p-12f));
  if (valid && !bad && !(D32 * (1.0f + 0x1p-12f) < bound)) {
    // FP64 CFL of the new state (FP32 fields widened)
    double gm = ph.chem ? gamma_eff((double)rho, (double)rh2) : ph.gamma;
    if (ions) gm = gamma_eff((double)rho, (double)rh2, (double)rhp);
    D = cfl_denominator((double)rho, (double)m[0], (double)m[1], (double)m[2], (double)Bc[0],
                        (double)Bc[1], (double)Bc[2], gm * ((gm - 1.0) * (double)eint));
  }
}

// the warp's share of the post stage's box scalars: the largest FP64 CFL denominator, the
// non-physical flag and the count of velocity-branch regularisations
template <typename T>
__device__ __forceinline__ void post_warp_reduce(const Box<T>& B, double D, int bad, unsigned vb, int check) {
  if (!check) bad = 0;
  if (__any_sync(0xffffffffu, D > 0.0)) D = warp_max(D);
  int anybad = __any_sync(0xffffffffu, bad);
  unsigned nvb = __popc(__ballot_sync(0xffffffffu, vb));
  if ((threadIdx.x & 31) == 0) {
    if (D > 0.0) atomicMax(&B.sc->dmax, (unsigned long long)__double_as_longlong(D));
    if (anybad) atomicOr(&B.sc->flags, 1);
    if (nvb) atomicAdd(&B.sc->vel_branch, (unsigned long long)nvb);
  }
}

template <typename T, bool IONS>
__global__ void __launch_bounds__(512) kb_post(const Box<T>* __restrict__ boxes, Tiles tl, int cell_stages,
                                               int do_reg, int check) {
  MHD_TILE_LOOP(tl) {
    const Box<T>& B = boxes[tl.box[t_]];
    idx_t c = tl.start[t_] + (idx_t)threadIdx.x;
    double D = 0.0;
    int bad = 0;
    unsigned vb = 0;
    post_cell<T, IONS>(B, c, c < B.g.N, cell_stages, do_reg, D, bad, vb);
    post_warp_reduce(B, D, bad, vb, check);
  }
}

// The last Lagrangian substage (r = 2) and the post stage of a step in one pass.  A cell's update
// reads the face fluxes and the cell's own fields, and its post stage reads only the cell's own
// fields and the face field b, which neither changes; so one thread takes both, in program order,
// and the update's HBM traffic overlaps the post stage's FP64 work.
template <typename T, bool IONS>
__global__ void __launch_bounds__(512) kb_lag_update_post(const Box<T>* __restrict__ boxes, Tiles tl,
                                                          int cell_stages, int do_reg, int check) {
  MHD_TILE_LOOP(tl) {
    const Box<T>& B = boxes[tl.box[t_]];
    idx_t c = tl.start[t_] + (idx_t)threadIdx.x;
    const bool valid = c < B.g.N;
    if (valid) lag_update_cell<T, IONS>(B, c, 2);
    double D = 0.0;
    int bad = 0;
    unsigned vb = 0;
    post_cell<T, IONS>(B, c, valid, cell_stages, do_reg, D, bad, vb);
    post_warp_reduce(B, D, bad, vb, check);
  }
}

// tau of the step from the device-resident max denominator (Sec. 2.3; min over cells of
// CFL h / D equals CFL h / max D since rounding is monotone), truncated at t_end (A18).
template <typename T>
__global__ void kb_begin_step(const Box<T>* __restrict__ boxes, int nb) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  Scalars* sc = boxes[b].sc;
  const double dx = boxes[b].ph.dx;
  if (!sc->fixed_tau) {
    double Dm = __longlong_as_double((long long)sc->dmax);
    double tau = sc->cfl * dx / Dm;
    if (sc->t_end > 0.0 && tau > sc->t_end - sc->t) tau = sc->t_end - sc->t;
    sc->tau = tau;
  }
  sc->tau_h = sc->tau / dx;
  if (!(sc->tau > 0.0)) sc->flags |= 2;
  sc->dmax = 0ull;  // the post kernel of this step accumulates the next state's denominator
}

template <typename T>
__global__ void kb_end_step(const Box<T>* __restrict__ boxes, int nb) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  Scalars* sc = boxes[b].sc;
  sc->t = sc->t + sc->tau;
  sc->steps += 1;
  // the host reads this word without synchronising (mhd_step with dt = NULL)
  if (boxes[b].hflags) *(volatile int*)boxes[b].hflags = sc->flags;
}

template <typename T>
__global__ void kb_set_params(const Box<T>* __restrict__ boxes, int nb, double cfl, double t_end,
                              int fixed_tau, double tau) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  Scalars* sc = boxes[b].sc;
  sc->cfl = cfl;
  sc->t_end = t_end;
  sc->fixed_tau = fixed_tau;
  if (fixed_tau) sc->tau = tau;
}

template <typename T>
__global__ void kb_zero_dmax(const Box<T>* __restrict__ boxes, int nb) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nb) boxes[b].sc->dmax = 0ull;
}

// ------------------------------------------------------------------------------------------------
// set_state helpers
template <typename T, typename In>
__global__ void k_load_cells(Geom g, State<T> s, const In* rho, const In* mx, const In* my,
                             const In* mz, const In* E, const In* rh2) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  s.rho[c] = (T)rho[c];
  s.m[0][c] = (T)mx[c];
  s.m[1][c] = (T)my[c];
  s.m[2][c] = (T)mz[c];
  s.E[c] = (T)E[c];
  if (s.rh2) s.rh2[c] = rh2 ? (T)rh2[c] : T(0);
  if (s.rhp) s.rhp[c] = T(0);
}

// A17: face b_d(i_d - 1/2) = (B_d(i_d - 1) + B_d(i_d)) / 2 from cell-centred input (in FP64)
template <typename T, typename In>
__global__ void k_faces_from_cells(Geom g, State<T> s, const In* Bx, const In* By, const In* Bz) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  int i = (int)(c % g.n[0]);
  long long r = c / g.n[0];
  int j = (int)(r % g.n[1]);
  int k = (int)(r / g.n[1]);
  const In* B[3] = {Bx, By, Bz};
  long long lo[3] = {cmap(g, i - 1, j, k), cmap(g, i, j - 1, k), cmap(g, i, j, k - 1)};
#pragma unroll
  for (int d = 0; d < 3; ++d) s.b[d][c] = (T)(0.5 * ((double)B[d][lo[d]] + (double)B[d][c]));
}

template <typename T>
__global__ void k_faces_copy(Geom g, State<T> s, const double* bx, const double* by, const double* bz) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  s.b[0][c] = (T)bx[c];
  s.b[1][c] = (T)by[c];
  s.b[2][c] = (T)bz[c];
}

// rho eps = rho E - |m|^2 / (2 rho) - |B_cell|^2 / 2 with B_cell from the faces
template <typename T>
__global__ void k_derive_eint(Geom g, State<T> s) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  int i = (int)(c % g.n[0]);
  long long r = c / g.n[0];
  int j = (int)(r % g.n[1]);
  int k = (int)(r / g.n[1]);
  long long up[3] = {cmap(g, i + 1, j, k), cmap(g, i, j + 1, k), cmap(g, i, j, k + 1)};
  T B[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) B[d] = T(0.5) * (s.b[d][c] + s.b[d][up[d]]);
  T rho = s.rho[c];
  T kin = T(0.5) * (s.m[0][c] * s.m[0][c] + s.m[1][c] * s.m[1][c] + s.m[2][c] * s.m[2][c]) / rho;
  T mag = T(0.5) * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
  s.eint[c] = s.E[c] - kin - mag;
}

template <typename T, typename Out>
__global__ void k_store_state(Geom g, State<T> s, Out* rho, Out* mx, Out* my, Out* mz, Out* E,
                              Out* Bx, Out* By, Out* Bz, Out* rh2) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  int i = (int)(c % g.n[0]);
  long long r = c / g.n[0];
  int j = (int)(r % g.n[1]);
  int k = (int)(r / g.n[1]);
  long long up[3] = {cmap(g, i + 1, j, k), cmap(g, i, j + 1, k), cmap(g, i, j, k + 1)};
  Out* B[3] = {Bx, By, Bz};
#pragma unroll
  for (int d = 0; d < 3; ++d) B[d][c] = (Out)(T(0.5) * (s.b[d][c] + s.b[d][up[d]]));
  rho[c] = (Out)s.rho[c];
  mx[c] = (Out)s.m[0][c];
  my[c] = (Out)s.m[1][c];
  mz[c] = (Out)s.m[2][c];
  E[c] = (Out)s.E[c];
  if (rh2) rh2[c] = s.rh2 ? (Out)s.rh2[c] : Out(0);
}

template <typename T>
__global__ void k_store_full(Geom g, State<T> s, double* eint, double* bx, double* by, double* bz) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  eint[c] = (double)s.eint[c];
  bx[c] = (double)s.b[0][c];
  by[c] = (double)s.b[1][c];
  bz[c] = (double)s.b[2][c];
}

// rho_H+ in and out (FP64 interface)
template <typename T>
__global__ void k_load_ions(Geom g, State<T> s, const double* rhp) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c < g.N) s.rhp[c] = (T)rhp[c];
}

template <typename T>
__global__ void k_store_ions(Geom g, State<T> s, double* rhp) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c < g.N) rhp[c] = (double)s.rhp[c];
}

template <typename T>
__global__ void k_load_full(Geom g, State<T> s, const double* eint, const double* bx,
                            const double* by, const double* bz) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  s.eint[c] = (T)eint[c];
  s.b[0][c] = (T)bx[c];
  s.b[1][c] = (T)by[c];
  s.b[2][c] = (T)bz[c];
}

// ------------------------------------------------------------------------------------------------
// FP64 diagnostics: fixed-shape tree reduction (block partials, then one block) -> deterministic.
// Partial layout per block: 8 sums + 1 max.
constexpr int DIAG_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(DIAG_THREADS) k_diag_partial(Geom g, State<T> s, double* part) {
  __shared__ double sh[9][DIAG_THREADS];
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (c < g.N) {
    int i = (int)(c % g.n[0]);
    long long r = c / g.n[0];
    int j = (int)(r % g.n[1]);
    int k = (int)(r / g.n[1]);
    long long up[3] = {cmap(g, i + 1, j, k), cmap(g, i, j + 1, k), cmap(g, i, j, k + 1)};
    v[0] = (double)s.rho[c];
    v[1] = (double)s.m[0][c];
    v[2] = (double)s.m[1][c];
    v[3] = (double)s.m[2][c];
    v[4] = (double)s.E[c];
    v[5] = (double)s.b[0][c];
    v[6] = (double)s.b[1][c];
    v[7] = (double)s.b[2][c];
    double div = ((double)s.b[0][up[0]] - (double)s.b[0][c]) + ((double)s.b[1][up[1]] - (double)s.b[1][c]) +
                 ((double)s.b[2][up[2]] - (double)s.b[2][c]);
    v[8] = fabs(div);
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) sh[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int w = DIAG_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
#pragma unroll
      for (int q = 0; q < 8; ++q) sh[q][threadIdx.x] = sh[q][threadIdx.x] + sh[q][threadIdx.x + w];
      sh[8][threadIdx.x] = fmax(sh[8][threadIdx.x], sh[8][threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x < 9) part[(long long)blockIdx.x * 9 + threadIdx.x] = sh[threadIdx.x][0];
}

static __global__ void __launch_bounds__(DIAG_THREADS) k_diag_final(const double* part, int nblocks, double* out) {
  __shared__ double sh[9][DIAG_THREADS];
  double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblocks; b += DIAG_THREADS) {
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = v[q] + part[(long long)b * 9 + q];
    v[8] = fmax(v[8], part[(long long)b * 9 + 8]);
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) sh[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int w = DIAG_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
#pragma unroll
      for (int q = 0; q < 8; ++q) sh[q][threadIdx.x] = sh[q][threadIdx.x] + sh[q][threadIdx.x + w];
      sh[8][threadIdx.x] = fmax(sh[8][threadIdx.x], sh[8][threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x < 9) out[threadIdx.x] = sh[threadIdx.x][0];
}

}  // namespace mhd
