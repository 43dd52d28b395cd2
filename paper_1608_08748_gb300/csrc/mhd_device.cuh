// mhd_device.cuh -- device arithmetic of one time step of the MHD + H/H2 chemistry method of
// arXiv:1608.08748 (Kulikov, Chernykh & Protasov).  Templated on the bulk type T (double for the
// FP64 path, float for the FP32-bulk path); the CFL reduction and the chemistry are FP64 always.
//
// The formulas follow the paper section by section.  On GB300 the FP64 pipe is the bound of the FP64
// path, so the work that need not be FP64 arithmetic leaves it: the limiter's sign tests, minima,
// orderings and power-of-two scalings run on the integer pipes (inline PTX on the halves of the
// doubles), quotients and roots take one Newton-Raphson step from the hardware seeds, and the
// Riemann solver forms its speeds and eigenvector rows with few divisions and square roots.  The
// PPM keeps the plain evaluation's edge values bit for bit outside the Step 4 blend (q6 is formed as
// 6 q_c - 3 (q_L + q_R)); the FP64 build contracts a*b+c into one FMA.  The FP64 path agrees with a
// plain evaluation to a few ulp per operation (about 1e-15 relative L1 after 50 steps of the 128^3
// turbulence box).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace mhd {

// ------------------------------------------------------------------------------------------------
// Geometry and parameters (passed by value to every kernel)
// Division of a non-negative 32-bit index by an invariant divisor d >= 1 with a multiply-high, two
// shifts and two additions instead of the integer division's dozen-odd instructions (the
// round-up method with an add indicator of Granlund & Montgomery, 1994): l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1 (below 2^32), and for every t < 2^32 the quotient is
// (hi + ((t - hi) >> min(l, 1))) >> max(l - 1, 0) with hi = floor(m t / 2^32).
struct FastDiv {
  unsigned d, m;
  int s1, s2;
};
inline FastDiv make_fastdiv(unsigned d) {
  int l = 0;
  while ((1ull << l) < d) ++l;
  const unsigned long long m = (((1ull << 32) * ((1ull << l) - d)) / d) + 1;
  return FastDiv{d, (unsigned)m, l < 1 ? l : 1, l > 1 ? l - 1 : 0};
}

struct Geom {
  int n[3];          // cells per axis
  int bc[3];         // 0 periodic, 1 outflow (zero-gradient)
  long long N;       // cells
  long long NF;      // (nx+1)(ny+1)(nz+1): size of face / edge scratch arrays
  FastDiv dn[2];     // division by n_x, n_y (cell indices)
  FastDiv dn1[2];    // division by n_x + 1, n_y + 1 (face and lattice indices)
};

// the divisors of a grid of nx x ny x nz cells
inline void set_divisors(Geom& g) {
  for (int d = 0; d < 2; ++d) {
    g.dn[d] = make_fastdiv((unsigned)g.n[d]);
    g.dn1[d] = make_fastdiv((unsigned)g.n[d] + 1u);
  }
}

struct Phys {
  double gamma;      // scalar adiabatic index (chemistry off)
  double dx, ih;     // cell width and 1/dx
  int chem;          // H/H2 network on
  int regul_mode;    // Sec. 2.9 reading: 0 max form, 1 unconditional, 2 literal branch order
  double lshield;    // shielding length, code units
  double bdop, xnorm, taud;
  double ibdop, ixnorm;  // 1 / bdop, 1 / xnorm
  double taud_ls, ls_ixnorm;  // taud L_s and L_s / xnorm, L_s the shielding length in cm (set_shielding)
  int heatcool;          // Sec. 2.8 heating/cooling stage on (needs chem)
  double grav_g;         // gravitational constant in code units (0: no self-gravity)
  int ions;              // reactions 5-8 with H+ and electrons on (needs chem)
};

// Device-resident scalars of a simulation: tau never crosses to the host inside a step.
struct Scalars {
  double cfl, t_end;       // set by the host with a kernel launch (graph-safe)
  double tau, tau_h;       // this step's tau and tau / dx
  double t;                // simulated time
  unsigned long long dmax; // bits of max CFL denominator of the current state (positive double)
  unsigned long long vel_branch;
  long long steps;
  int flags;               // bit 0: non-physical state, bit 1: tau <= 0
  int fixed_tau;           // 1: tau was given by the host (stage calls)
};

template <typename T>
struct State {
  T* rho;
  T* m[3];
  T* E;
  T* eint;
  T* rh2;  // may be unused when chemistry is off
  T* rhp;  // rho_H+ = n_H+ = n_e; used when the ions are on
  T* b[3];
};

// ------------------------------------------------------------------------------------------------
// indexing: cells [k][j][i]; face / edge scratch arrays on the (n+1)^3 lattice
__device__ __forceinline__ int wrap(int i, int n, int bc) {
  if ((unsigned)i < (unsigned)n) return i;  // interior: no integer division
  if (bc == 0) {
    int r = i % n;
    return r < 0 ? r + n : r;
  }
  return i < 0 ? 0 : n - 1;
}
// Cell, face and lattice indices are 32-bit: mhd_create rejects grids whose (n+1)^3 lattice does
// not fit (512^3 needs 1.35e8).
typedef int idx_t;

// Index-checked build (compiled with -DMHD_CHECK; build.build(check=True) makes libmhd_check.so):
// every computed cell index is tested against the cells [0, N) and every face or lattice index
// against [0, NF); a bad one sets a bit of this translation unit's flag word (1: cell, 2: lattice)
// and is replaced by 0, so that the access stays inside its array.  mhd_check_flags reads the
// words.  The plain build compiles the checks away.
#ifdef MHD_CHECK
static __device__ unsigned int g_check_flags;
__device__ __forceinline__ idx_t checked_index(idx_t i, long long n, unsigned bit) {
  if (i < 0 || (long long)i >= n) {
    atomicOr(&g_check_flags, bit);
    return 0;
  }
  return i;
}
#define MHD_CELL(g, i) ::mhd::checked_index((i), (g).N, 1u)
#define MHD_LATTICE(g, i) ::mhd::checked_index((i), (g).NF, 2u)
#else
#define MHD_CELL(g, i) (i)
#define MHD_LATTICE(g, i) (i)
#endif

__device__ __forceinline__ idx_t cidx(const Geom& g, int i, int j, int k) {
  return MHD_CELL(g, (k * g.n[1] + j) * g.n[0] + i);
}
__device__ __forceinline__ idx_t fidx(const Geom& g, int i, int j, int k) {
  return MHD_LATTICE(g, (k * (g.n[1] + 1) + j) * (g.n[0] + 1) + i);
}
// cell index of (c[0], c[1], c[2]) after the boundary map on each axis
__device__ __forceinline__ idx_t cmap(const Geom& g, int c0, int c1, int c2) {
  return cidx(g, wrap(c0, g.n[0], g.bc[0]), wrap(c1, g.n[1], g.bc[1]), wrap(c2, g.n[2], g.bc[2]));
}

// ------------------------------------------------------------------------------------------------
// Sec. 2.1: local parabola.  Delta q = q^R - q^L (the parabola's endpoints q(0) = q^L, q(1) = q^R).
template <typename T>
struct Para {
  T L, R, d, q6;
};

// The limited slope of Sec. 2.1 Step 1 (the FP32 Eulerian pencils).  Selects, not branches, and
// fmin for the minima (the operands are never NaN): the FP32 pencils are bound by instruction issue.
template <typename T>
__device__ __forceinline__ T slope_m(T qm, T q0, T qp) {
  T dq = T(0.5) * (qp - qm);
  T dp = qp - q0, dn = q0 - qm;
  const T mn = fmin(fmin(fabs(dq), T(2) * fabs(dp)), T(2) * fabs(dn));
  return dp * dn > T(0) ? copysign(mn, dq) : T(0);
}

// Steps 1-5 for cell i, evaluated as written, from q_{i-1}, q_i, q_{i+1}, the slopes of cells i - 1,
// i, i + 1 and the second differences D+ = q_{i+2} - 2 q_{i+1} + q_i, D- = q_i - 2 q_{i-1} + q_{i-2}:
// the FP32 Eulerian pencils take this form, carrying each slope to the next two cells (their bound
// is instruction issue, and the form has no branches: the tests of Steps 2 and 4 are selects, the
// division of eta is taken where it is not used, and the blend is q + hbar (q' - q)); ppm_lean
// below serves the other parabolas.
template <typename T>
__device__ __forceinline__ Para<T> ppm_carried(T qm1, T qc, T qp1, T dmm, T dm0, T dmp, T Dp, T Dm) {
  const T SIXTH = T(1.0 / 6.0);
  T qL = T(0.5) * (qm1 + qc) - (dm0 - dmm) * SIXTH;
  T qR = T(0.5) * (qc + qp1) - (dmp - dm0) * SIXTH;
  T dq = qR - qL;
  T q6 = T(6) * (qc - T(0.5) * (qL + qR));
  {
    const bool ext = (qL - qc) * (qc - qR) <= T(0);
    const bool up = dq * q6 > dq * dq, dn = dq * q6 < -(dq * dq);
    const T cL = T(3) * qc - T(2) * qR, cR = T(3) * qc - T(2) * qL;
    const T nL = ext ? qc : (up ? cL : qL);
    qR = ext ? qc : (!up && dn ? cR : qR);
    qL = nL;
  }
  T qLp = qc - T(0.25) * dm0, qRp = qc + T(0.25) * dm0;
  T dq2 = qp1 - qm1;
  // min(|q_{i+1}|, |q_{i-1}|, |q_{i+1}| + |q_{i-1}|) is the smaller of the first two
  const T mn = fmin(fabs(qp1), fabs(qm1));
  const bool det = !(fabs(dq2) - T(0.01) * mn <= T(0) || Dp * Dm > T(0));
  const T eta = (Dm - Dp) / (T(3) * dq2);  // discarded where det is false (dq2 may be 0 there)
  const T hb = det ? fmax(fmin(T(20) * (eta - T(0.05)), T(1)), T(0)) : T(0);
  qL = fma(hb, qLp - qL, qL);
  qR = fma(hb, qRp - qR, qR);
  Para<T> P;
  P.L = qL;
  P.R = qR;
  P.d = qR - qL;
  P.q6 = T(6) * (qc - T(0.5) * (qL + qR));
  return P;
}
// the same parabola from q_{i-2} .. q_{i+2}
template <typename T>
__device__ __forceinline__ Para<T> ppm_direct(T qm2, T qm1, T qc, T qp1, T qp2) {
  return ppm_carried(qm1, qc, qp1, slope_m(qm2, qm1, qc), slope_m(qm1, qc, qp1), slope_m(qc, qp1, qp2),
                     qp2 - T(2) * qp1 + qc, qc - T(2) * qm1 + qm2);
}

// 2^(j/32) for j = 0 .. 31, correctly rounded (the table of the exponential exp_tang below)
__device__ const double kExp2Frac32[32] = {
    0x1.0000000000000p+0, 0x1.059b0d3158574p+0, 0x1.0b5586cf9890fp+0, 0x1.11301d0125b51p+0,
    0x1.172b83c7d517bp+0, 0x1.1d4873168b9aap+0, 0x1.2387a6e756238p+0, 0x1.29e9df51fdee1p+0,
    0x1.306fe0a31b715p+0, 0x1.371a7373aa9cbp+0, 0x1.3dea64c123422p+0, 0x1.44e086061892dp+0,
    0x1.4bfdad5362a27p+0, 0x1.5342b569d4f82p+0, 0x1.5ab07dd485429p+0, 0x1.6247eb03a5585p+0,
    0x1.6a09e667f3bcdp+0, 0x1.71f75e8ec5f74p+0, 0x1.7a11473eb0187p+0, 0x1.82589994cce13p+0,
    0x1.8ace5422aa0dbp+0, 0x1.93737b0cdc5e5p+0, 0x1.9c49182a3f090p+0, 0x1.a5503b23e255dp+0,
    0x1.ae89f995ad3adp+0, 0x1.b7f76f2fb5e47p+0, 0x1.c199bdd85529cp+0, 0x1.cb720dcef9069p+0,
    0x1.d5818dcfba487p+0, 0x1.dfc97337b9b5fp+0, 0x1.ea4afa2a490dap+0, 0x1.f50765b6e4540p+0};

// ---- begin inline-PTX helpers ----
// Sign tests, absolute values, minima and comparisons of doubles on the integer pipes.  On sm_103
// the FP64 pipe issues two instructions per clock per SM and the integer pipes 64, and the PPM
// limiter is mostly such tests.  They work on the two 32-bit halves in inline PTX, so that the
// compiler does not turn them back into floating-point negations, absolute values or compares.
// For non-NaN operands they give the IEEE answer, with two exceptions that cannot change a
// limited value: -0 and +0 are told apart, and a product of two differences that underflows to
// zero is not formed (the test "a b > 0" is taken on the signs).  The float overloads are the plain
// operations.
__device__ __forceinline__ double abs_b(double x) {
  double r;
  asm("{\n\t.reg .b32 lo, hi;\n\tmov.b64 {lo, hi}, %1;\n\tand.b32 hi, hi, 0x7fffffff;\n\t"
      "mov.b64 %0, {lo, hi};\n\t}" : "=d"(r) : "d"(x));
  return r;
}
__device__ __forceinline__ float abs_b(float x) { return fabsf(x); }
__device__ __forceinline__ double neg_b(double x) {
  double r;
  asm("{\n\t.reg .b32 lo, hi;\n\tmov.b64 {lo, hi}, %1;\n\txor.b32 hi, hi, 0x80000000;\n\t"
      "mov.b64 %0, {lo, hi};\n\t}" : "=d"(r) : "d"(x));
  return r;
}
__device__ __forceinline__ float neg_b(float x) { return -x; }
// m (>= 0) with the sign of s
__device__ __forceinline__ double with_sign_b(double m, double s) {
  double r;
  asm("{\n\t.reg .b32 lo, hi, hs, ls;\n\tmov.b64 {lo, hi}, %1;\n\tmov.b64 {ls, hs}, %2;\n\t"
      "and.b32 hs, hs, 0x80000000;\n\tor.b32 hi, hi, hs;\n\tmov.b64 %0, {lo, hi};\n\t}"
      : "=d"(r) : "d"(m), "d"(s));
  return r;
}
__device__ __forceinline__ float with_sign_b(float m, float s) { return copysignf(m, s); }
// the smaller of a, b >= 0
__device__ __forceinline__ double min_nn(double a, double b) {
  double r;
  asm("{\n\t.reg .s64 ia, ib;\n\t.reg .pred p;\n\tmov.b64 ia, %1;\n\tmov.b64 ib, %2;\n\t"
      "setp.lt.s64 p, ia, ib;\n\tselp.b64 %0, %1, %2, p;\n\t}" : "=d"(r) : "d"(a), "d"(b));
  return r;
}
__device__ __forceinline__ float min_nn(float a, float b) { return fminf(a, b); }  // one FMNMX
// the larger of a, b >= 0
__device__ __forceinline__ double max_nn(double a, double b) {
  double r;
  asm("{\n\t.reg .s64 ia, ib;\n\t.reg .pred p;\n\tmov.b64 ia, %1;\n\tmov.b64 ib, %2;\n\t"
      "setp.gt.s64 p, ia, ib;\n\tselp.b64 %0, %1, %2, p;\n\t}" : "=d"(r) : "d"(a), "d"(b));
  return r;
}
__device__ __forceinline__ float max_nn(float a, float b) { return a > b ? a : b; }
// a > b for b >= 0
__device__ __forceinline__ bool gt_nn(double a, double b) {
  unsigned r;
  asm("{\n\t.reg .s64 ia, ib;\n\t.reg .pred p;\n\tmov.b64 ia, %1;\n\tmov.b64 ib, %2;\n\t"
      "setp.gt.s64 p, ia, ib;\n\tselp.u32 %0, 1, 0, p;\n\t}" : "=r"(r) : "d"(a), "d"(b));
  return r != 0;
}
__device__ __forceinline__ bool gt_nn(float a, float b) { return a > b; }
// a b > 0: both nonzero, one sign
__device__ __forceinline__ bool same_sign(double a, double b) {
  unsigned r;
  asm("{\n\t.reg .b32 la, ha, lb, hb, t;\n\t.reg .pred p;\n\t"
      "mov.b64 {la, ha}, %1;\n\tmov.b64 {lb, hb}, %2;\n\t"
      "and.b32 t, ha, 0x7fffffff;\n\tor.b32 t, t, la;\n\tsetp.ne.u32 p, t, 0;\n\t"
      "and.b32 t, hb, 0x7fffffff;\n\tor.b32 t, t, lb;\n\tsetp.ne.and.u32 p, t, 0, p;\n\t"
      "xor.b32 t, ha, hb;\n\tsetp.ge.and.s32 p, t, 0, p;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r) : "d"(a), "d"(b));
  return r != 0;
}
__device__ __forceinline__ bool same_sign(float a, float b) { return a * b > 0.f; }
// the sign bit
__device__ __forceinline__ bool sign_bit_b(double x) {
  unsigned r;
  asm("{\n\t.reg .b32 lo, hi;\n\tmov.b64 {lo, hi}, %1;\n\tshr.u32 %0, hi, 31;\n\t}" : "=r"(r) : "d"(x));
  return r != 0;
}
__device__ __forceinline__ bool sign_bit_b(float x) { return signbit(x); }

// Ordered key of a double: the signed 64-bit order of the keys is the order of the values, with
// -0 below +0 (the magnitude bits of a negative value flipped).  Comparisons of keys run on the
// integer pipe.
__device__ __forceinline__ long long okey(double x) {
  long long k;
  asm("{\n\t.reg .s64 m;\n\tmov.b64 %0, %1;\n\tshr.s64 m, %0, 63;\n\t"
      "and.b64 m, m, 0x7fffffffffffffff;\n\txor.b64 %0, %0, m;\n\t}" : "=l"(k) : "d"(x));
  return k;
}

// x 2^-K (K = 1, 2) on the integer pipe: the exponent field lowered by K.  Equal to the FP64
// product wherever that is a normal double, a zero, an infinity or a NaN; a product below the
// normal range (|x| < 2^(K-1021)) is taken as the zero of the sign of x.
template <int K>
__device__ __forceinline__ double scale_down_b(double x) {
  double r;
  asm("{\n\t.reg .b32 lo, hi, e, s, t, l;\n\t.reg .pred p, q;\n\tmov.b64 {lo, hi}, %1;\n\t"
      "bfe.u32 e, hi, 20, 11;\n\tsetp.gt.u32 p, e, %2;\n\tsetp.eq.u32 q, e, 2047;\n\t"
      "and.b32 s, hi, 0x80000000;\n\tsub.u32 t, hi, %3;\n\tselp.b32 t, t, s, p;\n\t"
      "selp.b32 l, lo, 0, p;\n\tselp.b32 t, hi, t, q;\n\tselp.b32 l, lo, l, q;\n\t"
      "mov.b64 %0, {l, t};\n\t}"
      : "=d"(r) : "d"(x), "n"(K), "n"(K << 20));
  return r;
}
template <int K>
__device__ __forceinline__ float scale_down_b(float x) { return x * (1.0f / (float)(1 << K)); }

// Approximate reciprocal and reciprocal square root of a double (PTX rcp.approx.ftz.f64,
// rsqrt.approx.ftz.f64): seeds for the Newton-Raphson steps below.  Subnormal arguments count as 0.
__device__ __forceinline__ double rcp_seed(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}
__device__ __forceinline__ double rsqrt_seed(double x) {
  double r;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}

// high 32 bits of the 64-bit product (the fast index divisions)
__device__ __forceinline__ unsigned umulhi32(unsigned a, unsigned b) { return __umulhi(a, b); }

// Device intrinsics, grouped here with the other device-only helpers.  The pieces of exp_tang below
// that act on bit patterns: the range test of its argument (-707 <= x
// <= -0 or +0 <= x < 707; NaNs and infinities fail), the low word of a double, 2^m y for y in
// [0.5, 4) and |m| <= 1020 by an addition to the exponent field, and the table read.
__device__ __forceinline__ bool exp_fast_range(double x) {
  const unsigned long long ux = (unsigned long long)__double_as_longlong(x);
  return ux <= 0xc086180000000000ull && (ux >= 0x8000000000000000ull || ux < 0x4086180000000000ull);
}
__device__ __forceinline__ int lo_word(double x) { return __double2loint(x); }
__device__ __forceinline__ double scale_pow2(double y, int m) {
  return __hiloint2double(__double2hiint(y) + (int)((unsigned)m << 20), __double2loint(y));
}
__device__ __forceinline__ double exp2_frac32(int j) { return __ldg(&kExp2Frac32[j]); }

// FP32 operations rounded to nearest whatever the build's FP32 flags (the CFL screen's error bound
// assumes them), and +inf
__device__ __forceinline__ float fsqrt_rn(float x) { return __fsqrt_rn(x); }
__device__ __forceinline__ float frsqrt_rn(float x) { return __frsqrt_rn(x); }
__device__ __forceinline__ float fdiv_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fmul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float f_inf() { return __int_as_float(0x7f800000); }

// ---- end inline-PTX helpers ----

// t / f.d for t < 2^32 (FastDiv)
__device__ __forceinline__ unsigned fdiv(unsigned t, const FastDiv& f) {
  const unsigned hi = umulhi32(f.m, t);
  return (hi + ((t - hi) >> f.s1)) >> f.s2;
}

__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }

// FP64 reciprocal, quotient and square root in few FP64 instructions, by one third-order
// Newton-Raphson step (the series of the inverse function) from the seeds above; a correctly
// rounded FP64 division or square root takes about twice the FP64-pipe slots.
//   1/x: with e = 1 - x r0, 1/x = r0 / (1 - e) = r0 (1 + e + e^2 + e^3 + ...); keeping 1 + e + e^2
//        leaves a relative error of about e^3, below the double's rounding for the seed's error.
//   1/sqrt(x): with e = 1 - x y0^2, 1/sqrt(x) = y0 (1 - e)^(-1/2) = y0 (1 + e/2 + 3 e^2 / 8 + ...).
//   sqrt(x) = x (1/sqrt(x)).
// Each is within 2 ulp of the correctly rounded value for finite normal arguments (x != 0); sqrt_nr
// takes 0 and subnormal arguments through the library square root.
__device__ __forceinline__ double rcp_nr(double x) {
  const double r = rcp_seed(x);
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}
__device__ __forceinline__ double rsqrt_nr(double x) {
  const double y = rsqrt_seed(x);
  const double e = fma(-x, y * y, 1.0);
  return fma(y, e * fma(0.375, e, 0.5), y);
}
__device__ __forceinline__ double sqrt_nr(double x) {
  // the range test on the integer pipe (x >= 0 or NaN here; -0 and negative x take the library)
  if (__builtin_expect(!gt_nn(2.2250738585072014e-308, x), 1)) return x * rsqrt_nr(x);
  return sqrt(x);
}
// bulk-type forms: FP64 by the steps above; FP32 by the plain operations (the FP32 build already
// takes the hardware-approximate division and square root)
__device__ __forceinline__ double rcp_t(double x) { return rcp_nr(x); }
__device__ __forceinline__ float rcp_t(float x) { return 1.0f / x; }
__device__ __forceinline__ double sqrt_t(double x) { return sqrt_nr(x); }
__device__ __forceinline__ float sqrt_t(float x) { return sqrtf(x); }

// e^x in FP64 by the table-driven method of P. T. P. Tang (ACM TOMS 15, 144-157, 1989), for the
// arguments of the H/H2 rates (x <= 0).  With k the integer nearest to 32 x / ln 2, k = 32 m + j
// (0 <= j < 32) and r = x - k ln2/32 (|r| <= ln2/64), e^x = 2^m 2^(j/32) e^r; e^r - 1 is its
// Taylor polynomial of degree 6 (the remainder r^7/7! stays below 4e-18), 2^(j/32) comes from a
// table of correctly rounded doubles, and 2^m is added to the exponent field on the integer pipe.
// ln2/32 is split in a 36-bit head, whose products with |k| < 2^15 are exact, and a tail.  The
// result lies within 1.01 ulp of e^x (half an ulp of the table entry, scaled by e^r, and half an ulp
// of the last rounding); it takes 11 FP64-pipe instructions.  Arguments outside
// [-707, 707] (where 2^m or the result leaves the normal range), infinities and NaNs take the
// library exp; the range test runs on the integer pipe.
__device__ __forceinline__ double exp_tang(double x) {
  if (!exp_fast_range(x)) return exp(x);
  const double INV_L = 0x1.71547652b82fep+5;                 // 32 / ln 2
  const double L_HI = 0x1.62e42fefa0000p-6, L_LO = 0x1.cf79abc9e3b3ap-45;  // ln2/32 = L_HI + L_LO
  const double SHIFTER = 0x1.8p52;                           // adding it rounds to an integer
  const double t = fma(x, INV_L, SHIFTER);
  const double kd = t - SHIFTER;
  const int k = lo_word(t);                                  // k in the low word, two's complement
  const double r = fma(-kd, L_LO, fma(-kd, L_HI, x));
  double p = fma(r, 1.0 / 720.0, 1.0 / 120.0);
  p = fma(r, p, 1.0 / 24.0);
  p = fma(r, p, 1.0 / 6.0);
  p = fma(r, p, 0.5);
  p = fma(r, p, 1.0);
  p = r * p;                                                 // e^r - 1
  const double tj = exp2_frac32(k & 31);
  const double y = fma(tj, p, tj);                           // 2^(j/32) e^r, in [0.98, 2.03)
  return scale_pow2(y, k >> 5);
}

// Half the limited slope of Sec. 2.1 Step 1 for a cell with differences dn = q_0 - q_-1,
// dp = q_1 - q_0 and s = q_1 - q_-1: the slope is min(|s|/2, 2|dp|, 2|dn|) with the sign of s where
// dn and dp have one sign, else 0; halving it is exact, and saves the doublings.
template <typename T>
__device__ __forceinline__ T half_slope(T s, T dn, T dp) {
  if (!same_sign(dn, dp)) return T(0);
  T m = min_nn(min_nn(scale_down_b<2>(abs_b(s)), abs_b(dp)), abs_b(dn));
  return with_sign_b(m, s);
}

// Steps 2-5 from the Step 1 edge values qL, qR of cell i (value qc, halved slope h0), the second
// differences D+ and D-, s0 = q_{i+1} - q_{i-1} and q_{i+1}, q_{i-1}.  Steps 2 and 5 are taken by
// selects, not branches: partly taken branches leave FP64 lanes idle, and the FP64 pipe is the
// bound.
template <typename T>
__device__ __forceinline__ Para<T> ppm_limit(T qL, T qR, T qc, T h0, T Dp, T Dm, T s0, T qp1, T qm1) {
  // 6 q_c once per parabola (FP64); 3 q_c = (6 q_c) / 2 exactly
  const T six_qc = T(6) * qc;
  // Step 2: monotonicity
  {
    const T dq = qR - qL;
    const T q6 = six_qc - T(3) * (qL + qR);
    bool ext, up, dn;
    if constexpr (sizeof(T) == 8) {
      // the tests as orderings of the values on the integer pipe: (q_L - q_c)(q_c - q_R) > 0 is q_c
      // strictly between q_L and q_R; dq q6 > dq^2 is q6 beyond dq on the side of its sign, and
      // -dq q6 > dq^2 is q6 beyond -dq on the other side (exact comparisons instead of rounded
      // products: the fixes are continuous at the ties, q_L = 3 q_c - 2 q_R there)
      const long long kL = okey(qL), kc = okey(qc), kR = okey(qR);
      ext = !((kL > kc && kc > kR) || (kL < kc && kc < kR));
      const long long kd = okey(dq), k6 = okey(q6), kmd = okey(neg_b(dq));
      const bool dpos = kd > 0, dneg = kd < -1;  // dq > 0, dq < 0 (keys of +0 and -0: 0 and -1)
      up = (dpos && k6 > kd) || (dneg && k6 < kd);
      dn = (dpos && k6 < kmd) || (dneg && k6 > kmd);
    } else {
      ext = !same_sign(qL - qc, qc - qR);
      const T a = dq * q6, b = dq * dq;
      up = gt_nn(a, b);
      dn = !up && gt_nn(neg_b(a), b);
    }
    // the two overshoot fixes are exclusive: one candidate 3 qc - 2 q from the opposite edge
    const T cand = scale_down_b<1>(six_qc) - T(2) * (up ? qR : qL);
    const T qLm = ext ? qc : (up ? cand : qL);
    const T qRm = ext ? qc : (dn ? cand : qR);
    qL = qLm;
    qR = qRm;
  }
  // Step 4: discontinuity detector
  const T mn = min_nn(abs_b(qp1), abs_b(qm1));
  if constexpr (sizeof(T) == 4) {
    // FP32 (bound by instruction issue): selects, not branches; eta is divided out everywhere and
    // discarded where the detector is off (s0 may be 0 there), and the blend is q + hbar (q' - q)
    const bool det = gt_nn(abs_b(s0), T(0.01) * mn) && !same_sign(Dp, Dm);
    const T eta = (Dm - Dp) / (T(3) * s0);
    const T hb = det ? fmaxf(fminf(T(20) * (eta - T(0.05)), T(1)), T(0)) : T(0);
    qL = fma(hb, (qc - T(0.5) * h0) - qL, qL);
    qR = fma(hb, (qc + T(0.5) * h0) - qR, qR);
  } else if (gt_nn(abs_b(s0), T(0.01) * mn) && !same_sign(Dp, Dm)) {
    // eta = num / den with den = 3 s0 != 0 here; num_s = num sgn(den)
    const T num = Dm - Dp;
    const T num_s = sign_bit_b(s0) ? neg_b(num) : num;
    const T qLp = qc - T(0.5) * h0, qRp = qc + T(0.5) * h0;
    // eta > 1/20 as num_s > |den| / 20 = 0.15 |s0| and eta > 1/10 as num_s / 2 > 0.15 |s0| (halving is
    // exact): one product serves both tests (at the two thresholds hbar is continuous, so their
    // rounding cannot move the result)
    const T ad20 = T(0.15) * abs_b(s0);
    if (sizeof(T) == 8 && gt_nn(scale_down_b<1>(num_s), ad20)) {
      // eta > 1/10: hbar = 1, the flattened values themselves (no FP64 division; in FP32 the
      // division is cheaper than the branch)
      qL = qLp;
      qR = qRp;
    } else if (gt_nn(num_s, ad20)) {
      if constexpr (sizeof(T) == 8) {
        // hbar = 20 (eta - 1/20) = 20 num / (3 s0) - 1 by the Newton-Raphson reciprocal (den is
        // nonzero here).  hbar lies in (0, 1] here up to rounding: the clamp and the test compare
        // on the integer pipe (a negative hbar orders below both 1 and 0), and the blend
        // hbar q' + (1 - hbar) q is taken as q + hbar (q' - q)
        T hb = fma(T(20) * num, rcp_nr(T(3) * s0), T(-1));
        hb = min_nn(hb, T(1));
        if (gt_nn(hb, T(0))) {
          qL = fma(hb, qLp - qL, qL);
          qR = fma(hb, qRp - qR, qR);
        }
      } else {
        const T eta = num / (T(3) * s0);
        T hb = T(20) * (eta - T(0.05));
        hb = hb < T(1) ? hb : T(1);
        if (hb > T(0)) {
          qL = hb * qLp + (T(1) - hb) * qL;
          qR = hb * qRp + (T(1) - hb) * qR;
        }
      }
    }
  }
  // Step 5
  Para<T> P;
  P.L = qL;
  P.R = qR;
  P.d = qR - qL;
  P.q6 = six_qc - T(3) * (qL + qR);
  return P;
}

// Sec. 2.1 Steps 1-5 for cell i from q_{i-2} .. q_{i+2}, with the Step 4 weights in the reading
// where hbar weighs the flattened values q -+ delta_m q / 4 (the amendment acts in
// discontinuities).  Written for few FP64 operations: the slopes are carried halved, the
// differences q_{i+1} - q_{i-1} and the second differences are formed once, min(|q_{i+1}|,
// |q_{i-1}|, |q_{i+1}| + |q_{i-1}|) is min(|q_{i+1}|, |q_{i-1}|), and eta = -(D+ - D-) / (3 dq) is
// divided out only where it lies between 1/20 and 1/10 (below, hbar = 0 and Step 4 changes
// nothing; above, hbar = 1 and the flattened values replace the edges; hbar = 20 (eta - 1/20)
// clamped to [0, 1] is continuous at both ends, so the tests' rounding cannot move the result).
template <typename T>
__device__ __forceinline__ Para<T> ppm_lean(T qm2, T qm1, T qc, T qp1, T qp2) {
  const T THIRD = T(1.0 / 3.0);  // twice 1/6, exactly
  const T d0 = qm1 - qm2, d1 = qc - qm1, d2 = qp1 - qc, d3 = qp2 - qp1;
  const T sm = qc - qm2, s0 = qp1 - qm1, sp = qp2 - qc;
  const T hm = half_slope(sm, d0, d1), h0 = half_slope(s0, d1, d2), hp = half_slope(sp, d2, d3);
  // Step 1: edge values (dm0 - dmm) / 6 = (h0 - hm) / 3
  const T qL = scale_down_b<1>(qm1 + qc) - (h0 - hm) * THIRD;
  const T qR = scale_down_b<1>(qc + qp1) - (hp - h0) * THIRD;
  // second differences D+ = q_{i+2} - 2 q_{i+1} + q_i, D- = q_i - 2 q_{i-1} + q_{i-2}: in FP64 as
  // differences of the first differences (one instruction each, as the stream forms them)
  T Dp, Dm;
  if constexpr (sizeof(T) == 8) {
    Dp = d3 - d2;
    Dm = d1 - d0;
  } else {
    Dp = (qp2 - T(2) * qp1) + qc;
    Dm = (qc - T(2) * qm1) + qm2;
  }
  return ppm_limit(qL, qR, qc, h0, Dp, Dm, s0, qp1, qm1);
}

// The parabolas of consecutive cells j, j+1, ... along a line, each from the quantities ppm_lean
// forms for it (so bit for bit the same), where the difference q_{j+1} - q_j, the halved slope, the
// edge value between two cells and the second difference centred on a cell are formed once and
// shared by the neighbours that use them.  Prime with q_{J-2} .. q_{J+1}; each next(q_{j+2}) then
// returns the parabola of the next cell j = J, J+1, ...
template <typename T>
struct PPMStream {
  T qm, q0, qp;  // q_{j-1}, q_j, q_{j+1}
  T dp;          // q_{j+1} - q_j
  T h0;          // halved slope of cell j
  T eL;          // edge value between j-1 and j
  T Cm, C0;      // second differences centred on j-1 and j
  T s0;          // q_{j+1} - q_{j-1}

  __device__ __forceinline__ void prime(T qa, T qb, T qc, T qd) {  // q_{J-2} .. q_{J+1}
    const T THIRD = T(1.0 / 3.0);
    const T d0 = qb - qa, d1 = qc - qb, d2 = qd - qc;
    const T hm = half_slope(qc - qa, d0, d1);
    s0 = qd - qb;
    h0 = half_slope(s0, d1, d2);
    eL = scale_down_b<1>(qb + qc) - (h0 - hm) * THIRD;
    Cm = d1 - d0;
    C0 = d2 - d1;
    qm = qb;
    q0 = qc;
    qp = qd;
    dp = d2;
  }
  __device__ __forceinline__ Para<T> next(T qn) {  // qn = q_{j+2}
    const T THIRD = T(1.0 / 3.0);
    const T d2 = qn - qp;
    const T s1 = qn - q0;
    const T h1 = half_slope(s1, dp, d2);
    const T C1 = d2 - dp;
    const T eR = scale_down_b<1>(q0 + qp) - (h1 - h0) * THIRD;
    Para<T> P = ppm_limit(eL, eR, q0, h0, C1, Cm, s0, qp, qm);
    qm = q0;
    q0 = qp;
    qp = qn;
    dp = d2;
    h0 = h1;
    eL = eR;
    Cm = C0;
    C0 = C1;
    s0 = s1;
    return P;
  }
};

// Sec. 2.4: parabola averages over the domain of dependence of a wave of |speed| y h / tau
template <typename T>
__device__ __forceinline__ T avg_right_end(const Para<T>& P, T y) {
  const T TWO_THIRDS = T(2.0 / 3.0);
  return P.R - T(0.5) * y * (P.d - P.q6 * (T(1) - TWO_THIRDS * y));
}
template <typename T>
__device__ __forceinline__ T avg_left_end(const Para<T>& P, T y) {
  const T TWO_THIRDS = T(2.0 / 3.0);
  return P.L + T(0.5) * y * (P.d + P.q6 * (T(1) - TWO_THIRDS * y));
}

// ------------------------------------------------------------------------------------------------
// Sec. 2.4 + App. A: Roe-type face state, eigenvectors and the characteristic Riemann solution.
// wl/wr = (rho, p, gamma, B_t1, B_t2, sqrt(rho)) of the left/right cell; Bn the face field.
// qs = (V_n, V_t1, V_t2, B_t1, B_t2, P).
//
// The speeds, alpha factors and eigenvector entries are those of App. A with 10 divisions and
// square roots instead of 29: one reciprocal of the weight sum, 1/sqrt(rho) (giving 1/rho,
// sqrt(rho), c_a = |B_n| / sqrt(rho) and the 1/sqrt(2 rho) of the Alfven rows), 1/c (giving c and
// the 1/(2c^2), 1/(2 sqrt(rho) c) factors of L), 1/c_f (giving c_f and c_s = c c_a / c_f, from
// c_f^2 c_s^2 = c^2 c_a^2) and 1/|B_perp|.  The left and right waves of each pair share their
// rows up to the sign of the velocity components, so the rows are formed once.
template <typename T>
__device__ __forceinline__ void riemann(const T wl[6], const T wr[6], T Bn, const Para<T> pl[6],
                                        const Para<T> pr[6], T tau_h, T qs[6]) {
  const T INV_SQRT2 = T(0.70710678118654752440);
  const T sl = wl[5], sr = wr[5];
  const T iden = rcp_t(sl + sr);
  const T al = sl * iden, ar = sr * iden;  // the normalised weights
  const T rho = al * wl[0] + ar * wr[0];
  const T p = al * wl[1] + ar * wr[1];
  const T gam = al * wl[2] + ar * wr[2];
  const T Bt1 = al * wr[3] + ar * wl[3];  // crossed weights for B
  const T Bt2 = al * wr[4] + ar * wl[4];

  const T rs = rsqrt_t(rho);  // 1 / sqrt(rho)
  const T irho = rs * rs;
  const T gp = gam * p;
  const T c2 = gp * irho;
  const T ca2 = (Bn * Bn) * irho;
  const T bp2 = Bt1 * Bt1 + Bt2 * Bt2;
  const T bp2r = bp2 * irho;
  const T s = c2 + (ca2 + bp2r);
  // fast and slow speeds without cancellation: with X = c^2 - c_a^2 and b_perp^2 = B_perp^2 / rho,
  //   c_f^2 - c_s^2 = sqrt(X^2 + b_perp^2 (2 c^2 + 2 c_a^2 + b_perp^2)),
  //   (c^2 - c_s^2)(c_f^2 - c^2) = c^2 b_perp^2,
  // so alpha_s (or alpha_f) is exactly 0 where B_perp = 0; dcs = c^2 - c_s^2, dfc = c_f^2 - c^2
  const T X = c2 - ca2;
  const T sq = sqrt_t(X * X + bp2r * ((T(2) * c2 + T(2) * ca2) + bp2r));
  // the larger of the two differences from the sum, the other from their product
  T dcs, dfc;
  if constexpr (sizeof(T) == 8) {
    // one FP64 division for both signs of X, so a warp with both signs does not take two
    const bool xpos = !sign_bit_b(X);  // at X = 0 either form holds
    // (|X| + sq - bp2r) / 2 for X >= 0, (|X| + sq + bp2r) / 2 for X < 0
    T big = scale_down_b<1>((abs_b(X) + sq) - (xpos ? bp2r : neg_b(bp2r)));
    big = sign_bit_b(big) ? T(0) : big;
    const T other = !gt_nn(T(2.2250738585072014e-308), big) ? (c2 * bp2r) * rcp_t(big)
                    : gt_nn(big, T(0)) ? c2 * bp2r / big : T(0);
    dcs = xpos ? big : other;
    dfc = xpos ? other : big;
  } else {
    // the same selects in FP32, where they save the branch
    const bool xpos = X >= T(0);
    T big = T(0.5) * ((fabs(X) + sq) - (xpos ? bp2r : -bp2r));
    big = fmax(big, T(0));
    const T other = big > T(0) ? c2 * bp2r / big : T(0);
    dcs = xpos ? big : other;
    dfc = xpos ? other : big;
  }
  const T cf2 = c2 + dfc;
  const T rc = rsqrt_t(c2), rcf = rsqrt_t(cf2);
  const T c = c2 * rc, cf = cf2 * rcf, ca = abs_b(Bn) * rs;
  const T cs = (c * ca) * rcf;
  T af, as;
  if (gt_nn(sq, T(1e-12) * s)) {
    const T isq = rcp_t(sq);
    af = sqrt_t(dcs * isq);
    as = sqrt_t(dfc * isq);
  } else {
    af = INV_SQRT2;
    as = INV_SQRT2;
  }
  T by, bz;
  if (gt_nn(bp2, T(1e-24) * rho * s)) {
    const T ibp = rsqrt_t(bp2);
    by = Bt1 * ibp;
    bz = Bt2 * ibp;
  } else {
    by = INV_SQRT2;
    bz = INV_SQRT2;
  }
  const T sg = (sign_bit_b(Bn) && gt_nn(abs_b(Bn), T(0))) ? T(-1) : T(1);  // sign(0) = +1
  const T sqr = rho * rs, sc = sqr * c, sr2 = sqr * INV_SQRT2;
  const T i2c2 = scale_down_b<1>(rc * rc), i2sc = scale_down_b<1>(rs * rc), i2rc2 = i2c2 * irho;
  const T isr2 = rs * INV_SQRT2;

  // App. A rows of the +c_f and +c_s waves; the -c waves negate the v_n, v_t1, v_t2 entries
  const T afcf = af * cf, ascs = as * cs, bys = by * sg, bzs = bz * sg;
  const T Rf[6] = {afcf, -(ascs * bys), -(ascs * bzs), as * sc * by, as * sc * bz, af * gp};
  const T Lf[6] = {afcf * i2c2, -(ascs * bys) * i2c2, -(ascs * bzs) * i2c2, as * by * i2sc,
                   as * bz * i2sc, af * i2rc2};
  const T Rs[6] = {ascs, afcf * bys, afcf * bzs, -(af * sc * by), -(af * sc * bz), as * gp};
  const T Ls[6] = {ascs * i2c2, afcf * bys * i2c2, afcf * bzs * i2c2, -(af * by * i2sc),
                   -(af * bz * i2sc), as * i2rc2};
  // Alfven rows: v_t1, v_t2 entries shared, B_t1, B_t2 entries negated for the -c_a wave
  const T Av[2] = {-(bzs * INV_SQRT2), bys * INV_SQRT2};
  const T AL[2] = {bz * isr2, -(by * isr2)};
  const T AR[2] = {sr2 * bz, -(sr2 * by)};

#pragma unroll
  for (int m = 0; m < 6; ++m) qs[m] = T(0);
  const T TWO_THIRDS = T(2.0 / 3.0);
  // s_k = L_k . qbar_k (qbar_k the domain-of-dependence average on the upwind side), q* = sum R_k s_k.
  // The +c and -c waves of a pair share y, and their rows up to the sign S of the velocity entries:
  // with s_+ = L . qbar_+ (left cell, right end) and s_- = (S L) . qbar_- (right cell, left end),
  // R s_+ + (S R) s_- is R (s_+ - s_-) on v_n, v_t1, v_t2 and R (s_+ + s_-) on B_t1, B_t2, P.
  auto magnetosonic_pair = [&](const T L[6], const T R[6], T speed) {
    const T y = speed * tau_h;
    const T hy = scale_down_b<1>(y), w = T(1) - TWO_THIRDS * y;
    T pa = T(0), pb = T(0), ma = T(0), mb = T(0);
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      // avg_right_end of the left cell, avg_left_end of the right cell (Sec. 2.4)
      const T qp = pl[m].R - hy * (pl[m].d - pl[m].q6 * w);
      const T qm = pr[m].L + hy * (pr[m].d + pr[m].q6 * w);
      if (m < 3) {
        pa = pa + L[m] * qp;
        ma = ma + L[m] * qm;
      } else {
        pb = pb + L[m] * qp;
        mb = mb + L[m] * qm;
      }
    }
    const T sp = pa + pb, sm = mb - ma;
    const T dif = sp - sm, sum = sp + sm;
#pragma unroll
    for (int m = 0; m < 6; ++m) qs[m] = qs[m] + R[m] * (m < 3 ? dif : sum);
  };
  // Alfven pair: the v_t rows are shared, the B_t rows change sign
  auto alfven_pair = [&]() {
    const T y = ca * tau_h;
    const T hy = scale_down_b<1>(y), w = T(1) - TWO_THIRDS * y;
    T qp[5], qm[5];
#pragma unroll
    for (int m = 1; m < 5; ++m) {
      qp[m] = pl[m].R - hy * (pl[m].d - pl[m].q6 * w);
      qm[m] = pr[m].L + hy * (pr[m].d + pr[m].q6 * w);
    }
    const T sp = (Av[0] * qp[1] + Av[1] * qp[2]) + (AL[0] * qp[3] + AL[1] * qp[4]);
    const T sm = (Av[0] * qm[1] + Av[1] * qm[2]) - (AL[0] * qm[3] + AL[1] * qm[4]);
    const T sum = sp + sm, dif = sp - sm;
    qs[1] = qs[1] + Av[0] * sum;
    qs[2] = qs[2] + Av[1] * sum;
    qs[3] = qs[3] + AR[0] * dif;
    qs[4] = qs[4] + AR[1] * dif;
  };
  magnetosonic_pair(Lf, Rf, cf);  // waves 1, 2: +-c_f
  magnetosonic_pair(Ls, Rs, cs);  // waves 3, 4: +-c_s
  alfven_pair();                  // waves 5, 6: +-c_a
}

// ------------------------------------------------------------------------------------------------
// Sec. 2.3: CFL denominator |v| + b + c + c_a + c_s + c_f, the largest over the three choices of
// the longitudinal axis (b^2 = B^2 / rho), in FP64.  With c_f^2 + c_s^2 = c^2 + b^2 and
// c_f c_s = c c_a, c_f + c_s = sqrt(c^2 + b^2 + 2 c c_a); the denominator grows with c_a = |B_d| /
// sqrt(rho), so the largest one is that of the axis of the largest |B_d|.  Takes the momenta and
// gamma p; 1/sqrt(rho) is the one reciprocal: |v| = |m| / rho, b = |B| / sqrt(rho),
// c = sqrt(gamma p) / sqrt(rho) and c_f + c_s = sqrt(gamma p + B^2 + 2 sqrt(gamma p) |B_d|) / sqrt(rho).
__device__ __forceinline__ double cfl_denominator(double rho, double mx, double my, double mz,
                                                  double Bx, double By, double Bz, double gp) {
  const double irs = rsqrt(rho);
  const double irho = irs * irs;
  const double sgp = sqrt_nr(gp);
  const double B2 = Bx * Bx + By * By + Bz * Bz;
  const double sB = sqrt_nr(B2);
  const double v = sqrt_nr(mx * mx + my * my + mz * mz) * irho;
  const double Bm = max_nn(abs_b(Bx), max_nn(abs_b(By), abs_b(Bz)));
  const double fs = sqrt_nr((gp + B2) + 2.0 * sgp * Bm);
  return v + ((sB + sgp + Bm) + fs) * irs;
}

// The screen of the CFL maximum.  tau takes only the largest FP64 denominator over the cells, so a
// cell whose denominator provably lies below an FP64 denominator already reached by another cell
// cannot set it and need not be evaluated in FP64: tau stays bit for bit that of evaluating every
// cell.  The proof is the FP32 estimate below, the same formula from FP32-rounded inputs (square
// roots and 1/sqrt correctly rounded, sums and products rounded to nearest).  With u = 2^-24 a
// first-order count of its relative error gives about 30 u: up to 23 u in gamma - 1 (the
// cancellation in n_H = rho - rho_H2 - rho_H+ stays below 5 u rho, against numerator and
// denominator of at least rho / 2 and 2 rho), 35 u in gamma p, half of that through the square
// roots, 1.5 u through 1/sqrt(rho) and its square, a few u of sums.  FP32 squares that flush to
// zero or lose bits below the normal range move |m| or |B| by less than 2^-62, which is below 2^-22
// of the denominator (>= sqrt(gamma p / rho)) while rho >= 2^-40 and gamma p >= 2^-40.  The
// screen allows 2^-12 (4096 u).  A cell outside those guards, or whose estimate overflows, gets
// +inf and is always evaluated in FP64.
__device__ __forceinline__ float cfl_estimate_f32(float rho, float mx, float my, float mz, float Bx,
                                                  float By, float Bz, float eint, float gm1) {
  const float gp = fmul_rn(fmul_rn(1.0f + gm1, gm1), eint);
  if (!(rho >= 0x1p-40f) || !(gp >= 0x1p-40f)) return f_inf();
  const float irs = frsqrt_rn(rho);
  const float irho = irs * irs;
  const float sgp = fsqrt_rn(gp);
  const float B2 = Bx * Bx + By * By + Bz * Bz;
  const float sB = fsqrt_rn(B2);
  const float v = fsqrt_rn(mx * mx + my * my + mz * mz) * irho;
  const float Bm = fmaxf(fabsf(Bx), fmaxf(fabsf(By), fabsf(Bz)));
  const float fs = fsqrt_rn((gp + B2) + 2.0f * sgp * Bm);
  return v + ((sB + sgp + Bm) + fs) * irs;
}

// gamma - 1 of the cell in FP32 for the screen: that of the ideal gas, or of the H/H2 (+ H+, e-)
// mixture as (2 n_1 + 2 n_H2) / (3 n_1 + 5 n_H2) (gamma_eff below minus one); -1 where the
// numerator falls below rho / 2 or the denominator below 2 rho (3 rho - rho_H2 / 2 + 3 rho_H+ for
// physical abundances), which fails the screen's guard.
__device__ __forceinline__ float gamma_minus_one_f32(bool chem, double gamma, float rho, float rh2, float rhp) {
  if (!chem) return (float)(gamma - 1.0);
  const float n1 = (rho - rh2 - rhp) + 2.0f * rhp, nH2 = 0.5f * rh2;
  const float num = 2.0f * (n1 + nH2), den = 3.0f * n1 + 5.0f * nH2;
  return (num >= 0.5f * rho && den >= 2.0f * rho) ? fdiv_rn(num, den) : -1.0f;
}

// Sec. 4.3 effective adiabatic index of the H/H2 mixture (no electrons)
template <typename T>
__device__ __forceinline__ T gamma_eff(T rho, T rh2) {
  T nH = rho - rh2, nH2 = T(0.5) * rh2;
  return (T(5) * nH + T(7) * nH2) * rcp_t(T(3) * nH + T(5) * nH2);
}

// ... and with H+ and electrons: the monatomic particles n_1 = n_H + n_H+ + n_e replace n_H, with
// the neutral atoms n_H = rho - rho_H2 - rho_H+ and n_H+ = n_e = rho_H+ (rho_H+ = 0: the form above)
template <typename T>
__device__ __forceinline__ T gamma_eff(T rho, T rh2, T rhp) {
  T n1 = (rho - rh2 - rhp) + T(2) * rhp, nH2 = T(0.5) * rh2;
  return (T(5) * n1 + T(7) * nH2) * rcp_t(T(3) * n1 + T(5) * nH2);
}

// ------------------------------------------------------------------------------------------------
// Sec. 2.7 + App. D: one cell of the H/H2 network (reactions 1-4), backward-differentiation
// update of n_H2 with rates frozen over the step; returns the new rho_H2.  FP64.
struct ChemConst {
  static constexpr double KB = 1.380649e-16;         // erg / K
  static constexpr double MH = 1.6735575e-24;        // g
  static constexpr double PC = 3.0856775814913673e18; // cm
  static constexpr double KMS = 1.0e5;               // cm / s
};

// the per-box products of the shielding length L_s = (lshield > 0 ? lshield : dx) pc (App. D column
// densities N = n L_s): set on the host whenever lshield, xnorm, taud or dx change
inline void set_shielding(Phys& ph) {
  const double Ls = (ph.lshield > 0.0 ? ph.lshield : ph.dx) * ChemConst::PC;
  ph.taud_ls = ph.taud * Ls;
  ph.ls_ixnorm = Ls * ph.ixnorm;
}

// The App. D formulas in FP64 with few FP64 instructions (the rates agree with a term-by-term
// evaluation to about 1e-14 relative):
//   T = (gamma - 1) rho eps P0 / (n_particles k_B) with gamma - 1 = 2 n_particles / (3 n_1 + 5 n_H2)
//     = (2 P0 / k_B) rho eps / (3 n_1 + 5 n_H2), n_1 = n_H + n_H+ + n_e, and T, 1/T and sqrt(T)
//     from one reciprocal square root of the product;
//   1/sqrt(1 + x) from one reciprocal square root; 1/x_norm, 1/b_doppler and the products with the
//   shielding length precomputed; one reciprocal for k1' and 1/u^2 (of their denominators' product);
//   the exponentials of the H/H2 rates by exp_tang (their arguments are <= 0); the arguments of
//   reactions 2 and 3 not formed in gas cold enough for their exponentials to be 0.
struct ChemOut {
  double rh2, rhp;  // new rho_H2 and rho_H+
};

// App. D rates of reactions 5-8 at T (ln T given): k5 = 6e-18 s^-1 per atom, k6 = exp(poly(ln T_eV))
// (Horner), k7 = 10^(P(x) / Q(x)) with x = log10 T, k8 the grain-recombination fit with
// T^0.01586 10^(-4.4e-5 log10 T) = T^(0.01586 - 4.4e-5).
struct IonRates {
  double k5, k6, k7, k8;
};
__device__ __forceinline__ IonRates ion_rates(double lnT) {
  const double LN_KB_EV = -9.359149794515579;  // ln(8.617333262e-5 eV/K)
  const double INV_LN10 = 0.43429448190325176;
  IonRates r;
  r.k5 = 6e-18;
  const double L = lnT + LN_KB_EV;
  double p = -2.1e-6;
  p = fma(p, L, 1.1e-4);
  p = fma(p, L, -2.6e-3);
  p = fma(p, L, 3.4e-2);
  p = fma(p, L, -0.3);
  p = fma(p, L, 1.5);
  p = fma(p, L, -5.7);
  p = fma(p, L, 13.5);
  p = fma(p, L, -32.7);
  r.k6 = exp(p);
  const double x = lnT * INV_LN10;
  const double P = fma(fma(fma(fma(-3.87e-3, x, 0.08), x, -0.87), x, 4.68), x, -10.78);
  const double Q = fma(fma(fma(fma(2.4e-4, x, -5.1e-3), x, 0.06), x, -0.38), x, 1.0);
  r.k7 = exp10(P / Q);
  const double A = 8.074e-6 * 570.1642722807472;  // 8.074e-6 10^2.756
  const double Bc = 5.087e2 * 0.012906247820605376;  // 5.087e2 10^-1.8892
  r.k8 = 12.25e-14 / (1.0 + A * (1.0 + Bc * exp((1.586e-2 - 4.4e-5) * lnT)));
  return r;
}

// IONS: the kernel may see boxes with the ions on (ph.ions decides per box); without it the ion
// code is compiled out and rhp must be 0.
template <bool IONS>
__device__ __forceinline__ ChemOut chem_cell(const Phys& ph, double rho, double eint, double rh2,
                                             double rhp, double tau) {
  const double P0 = ChemConst::MH * ChemConst::KMS * ChemConst::KMS;  // code pressure, erg cm^-3
  const double T0 = ChemConst::PC / ChemConst::KMS;                  // code time, s
  // the ion terms are added to the H/H2 expressions with explicit FMAs, so that a box without ions
  // gets the same bits from either instance (rhp = 0 then adds exactly nothing)
  double nH = rho - rh2;
  if (IONS) nH = nH - rhp;
  const double nH2 = scale_down_b<1>(rh2), n = rho;
  const double num = (2.0 * P0 / ChemConst::KB) * eint;
  double den3 = fma(3.0, nH, 5.0 * nH2);  // 3 n_1 + 5 n_H2 with n_1 = n_H + n_H+ + n_e
  if (IONS) den3 = fma(6.0, rhp, den3);
  // T = num / den3 and its square root from one reciprocal square root q = 1 / sqrt(num den3):
  // sqrt(T) = num q, T = (num q)^2, 1/T = (den3 q)^2
  const double q = rsqrt_nr(num * den3);
  const double sT = num * q, dq = den3 * q;
  const double T = sT * sT, iT = dq * dq;
  // App. D rates; the branch tests and clamps compare on the integer pipe (T >= 0; a2, a3 < 0)
  const bool hot2 = gt_nn(T, 7390.0), hot3 = gt_nn(T, 7291.0);
  // reactions 2 and 3: exp of an argument below -746 is exactly 0 in double, and the cold branches'
  // arguments -(6750 / T)^2 and -4060 / T - (7500 / T)^2 lie below -746.6 for T <= 247 and below
  // -747 for T <= 277, so there the rates are 0 without forming them (warps of cold cells skip)
  double k2 = 0.0, k3 = 0.0;
  if (gt_nn(T, 247.0)) {
    const double a2 = hot2 ? -2.93e4 * iT : -((6750.0 * iT) * (6750.0 * iT));
    if (!gt_nn(neg_b(a2), 746.0)) k2 = (hot2 ? 6.11e-14 : 2.67e-15) * exp_tang(a2);
  }
  if (gt_nn(T, 277.0)) {
    const double a3 = hot3 ? -3.22e4 * iT : -(4060.0 * iT) - (7500.0 * iT) * (7500.0 * iT);
    if (!gt_nn(neg_b(a3), 746.0)) k3 = (hot3 ? 5.22e-14 : 3.17e-15) * exp_tang(a3);
  }
  // shielding: f_dust = exp(-taud (N_H + N_H2)), x = N_H2 / x_norm, N = n L_s
  const double fdust = exp_tang(-(ph.taud_ls * (nH + nH2)));
  const double x = nH2 * ph.ls_ixnorm;
  const double u = 1.0 + x * ph.ibdop;
  const double isx = rsqrt_nr(1.0 + x);
  const double sx = (1.0 + x) * isx;
  // k1' = 3e-17 s / (1 + 0.4 s + 0.2 t + 0.08 t^2) with t = T / 100, s = sqrt(t) = sqrt(T) / 10
  const double d1 = fma(fma(0.08 * 1e-4, T, 0.2 * 1e-2), T, fma(0.4 * 0.1, sT, 1.0)), u2 = u * u;
  const double rd = rcp_nr(d1 * u2);  // 1 / (d1 u^2): d1, u^2 >= 1
  const double k1p = (3e-17 * 0.1 * sT) * (u2 * rd);
  // k4 = 3.3 1.7e-11 f_sh f_dust with f_sh = 0.965 / u^2 + 0.035 exp(-8.5e-4 sqrt(1 + x)) / sqrt(1 + x)
  const double k4 = fdust * fma(3.3 * 1.7e-11 * 0.965, d1 * rd,
                                ((3.3 * 1.7e-11 * 0.035) * isx) * exp_tang(-8.5e-4 * sx));
  const double C = k1p * n * nH;
  const double D = (k2 * nH + k3 * nH2) + k4;
  const double ts = tau * T0;
  double nH2n = nH2 + (ts * (C - D * nH2)) * rcp_nr(1.0 + ts * D);
  if (sign_bit_b(nH2n)) nH2n = 0.0;
  const double half_n = scale_down_b<1>(n);
  if (gt_nn(nH2n, half_n)) nH2n = half_n;
  ChemOut out;
  out.rh2 = 2.0 * nH2n;
  out.rhp = rhp;
  if (IONS && ph.ions) {
    // reactions 5-8: creation k5 n_H + k6 n_H n_e, destruction (k7 n_e + k8 n) n_H+, the same
    // semi-implicit update from the stage-start densities; n_H+ <= n - 2 n_H2 (n_H >= 0)
    const double ne = rhp;
    const IonRates q = ion_rates(log(T));
    const double Ci = (q.k5 + q.k6 * ne) * nH;
    const double Di = q.k7 * ne + q.k8 * n;
    double nHpn = rhp + ts * (Ci - Di * rhp) / (1.0 + ts * Di);
    if (nHpn < 0.0) nHpn = 0.0;
    if (nHpn > n - 2.0 * nH2n) nHpn = n - 2.0 * nH2n;
    out.rhp = nHpn;
  }
  return out;
}

// ------------------------------------------------------------------------------------------------
// Sec. 2.8 + App. D: heating and cooling of one cell, d(rho E)/dt = d(rho eps)/dt = Gamma - Lambda by
// one Euler step; returns the change of rho E and rho eps in code units.  FP64.  Readings:
//   Gamma_1 = 7.2e-12 erg (k1' n n_H) / (1 + n_cr / n), n_cr = 10^(4 - 0.416 x - 0.327 x^2) (the H2
//     formation heating: the printed numerator read as the formation rate, the printed polynomial
//     over n as the critical density);
//   Lambda_2 = n_H2 L_H / (1 + L_H / L_L) with the printed two-branch L_H, L_L;
//   Lambda_3 = n_H2 L_H / (1 + L_H / L_L), L_H = 1.1e-13 exp(-6744 / T),
//     L_L = 8.18e-13 (n_H + n_H2) k_H2 (k_H, undefined in the paper, read as k_H2),
//     k_H2 = 6.29e-15 1.38 f(T) / f(4500), f(T) = sqrt(T) a e^a, a = 1 + 1 / (k_B T), k_B in eV/K;
//   Gamma_4 = 6.4e-13 erg k4 n_H2;
//   x = log10(T / 1e4); T, k1' and k4 as in chem_cell, from the state after the chemistry update;
//   the change is limited to at most half of rho eps (the explicit step of a cooling time shorter
//   than tau would drive rho eps negative).
template <bool IONS>
__device__ __forceinline__ double heatcool_delta(const Phys& ph, double rho, double eint, double rh2,
                                                 double rhp, double tau) {
  const double P0 = ChemConst::MH * ChemConst::KMS * ChemConst::KMS;  // erg cm^-3
  const double T0 = ChemConst::PC / ChemConst::KMS;                  // s
  const double KB_EV = 8.617333262e-5;                               // eV / K
  double nH = rho - rh2;
  if (IONS) nH = nH - rhp;
  const double nH2 = 0.5 * rh2, n = rho;
  double den3 = fma(3.0, nH, 5.0 * nH2);
  if (IONS) den3 = fma(6.0, rhp, den3);
  const double T = ((2.0 * P0) * eint) / (den3 * ChemConst::KB);
  const double x = log10(T * 1e-4);
  // k1' and k4 (App. D, as in chem_cell)
  const double t2 = T * 0.01, s2 = sqrt(t2);
  const double k1p = 3e-17 * s2 / (((1.0 + 0.4 * s2) + 0.2 * t2) + 0.08 * (t2 * t2));
  const double Ls = (ph.lshield > 0.0 ? ph.lshield : ph.dx) * ChemConst::PC;
  const double NH = nH * Ls, NH2 = nH2 * Ls;
  const double fdust = exp(-(ph.taud * (NH + NH2)));
  const double xs = NH2 * ph.ixnorm;
  const double u = 1.0 + xs * ph.ibdop;
  const double isx = rsqrt(1.0 + xs);
  const double fsh = 0.965 / (u * u) + (0.035 * isx) * exp(-8.5e-4 * ((1.0 + xs) * isx));
  const double k4 = (3.3 * 1.7e-11) * fsh * fdust;
  // Gamma_1
  const double ncr = exp10(4.0 - 0.416 * x - 0.327 * x * x);
  const double G1 = 7.2e-12 * (k1p * n * nH) / (1.0 + ncr / n);
  // Lambda_2
  const double LH2 = T > 1087.0 ? 3.9e-19 * exp(-6118.0 / T) : exp10(-19.24 + 0.474 * x - 1.247 * x * x);
  const double LL2 = (pow(nH2, 0.77) + 1.2 * pow(nH, 0.77)) *
                     (T > 4031.0 ? 1.38e-22 * exp(-9243.0 / T) : exp10(-22.9 - 0.553 * x - 1.148 * x * x));
  const double L2 = nH2 * LH2 / (1.0 + LH2 / LL2);
  // Lambda_3
  const double LH3 = 1.1e-13 * exp(-6744.0 / T);
  const double a = 1.0 + 1.0 / (KB_EV * T), a0 = 1.0 + 1.0 / (KB_EV * 4500.0);
  const double lnf = (0.5 * log(T) + log(a)) + a, lnf0 = (0.5 * log(4500.0) + log(a0)) + a0;
  const double kH2 = (6.29e-15 * 1.38) * exp(lnf - lnf0);
  const double LL3 = 8.18e-13 * ((nH + nH2) * kH2);
  const double L3 = nH2 * LH3 / (1.0 + LH3 / LL3);
  // Gamma_4
  const double G4 = 6.4e-13 * k4 * nH2;
  double net = (G1 + G4) - (L2 + L3);
  if (IONS && ph.ions) {
    // Gamma_5 = 1.92e-28 n; Lambda_6 = 2.18e-11 k6 n_H n_e; Lambda_7 = 4.65e-30 T^0.94 psi^beta n_e n_H+
    // with psi = exp(-0.75e-20 (N_H + N_H2)) sqrt(T) / n_e and beta = 0.74 / T^0.068 (0 where
    // n_e = 0); Lambda_8 = 5.7e-26 (T / 1e4)^0.8 n_e n_H+
    const double ne = rhp, lnT = log(T);
    const IonRates q = ion_rates(lnT);
    const double G5 = 1.92e-28 * n;
    const double L6 = 2.18e-11 * q.k6 * nH * ne;
    double L7 = 0.0;
    if (ne > 0.0) {
      const double lnpsi = (-0.75e-20 * (NH + NH2) + 0.5 * lnT) - log(ne);
      const double beta = 0.74 * exp(-0.068 * lnT);
      L7 = 4.65e-30 * exp(0.94 * lnT + beta * lnpsi) * ne * rhp;
    }
    const double L8 = 5.7e-26 * exp(0.8 * (lnT - 9.210340371976184)) * ne * rhp;  // ln 1e4
    net = (net + G5) - ((L6 + L7) + L8);
  }
  double d = (tau * T0) * net / P0;
  if (d < -0.5 * eint) d = -0.5 * eint;
  return d;
}

}  // namespace mhd
