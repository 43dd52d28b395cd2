// The CUDA path's per-face and per-cell arithmetic (mhd_device.cuh) compiled for the host and
// compared with the oracle's unit entry points on seeded random and adversarial inputs.  The test
// that builds this file gives it a copy of the header in which the inline-PTX helpers
// are replaced by portable C++ with the same definitions (MHD_DEVICE_HOST_COPY).  Prints one line
// per check: "<name> <cases> <worst relative difference> <cases beyond the bound>".
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <random>
#include <vector>

static inline double rsqrt(double x) { return 1.0 / std::sqrt(x); }
static inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }
#include MHD_DEVICE_HOST_COPY

extern "C" {
struct osim;
osim* osim_create(int nx, int ny, int nz, double gamma, double dx);
void osim_destroy(osim* s);
void osim_chem_cell(const osim* s, double rho, double eint, double rh2, double tau, double out[8]);
void osim_heatcool_cell(const osim* s, double rho, double eint, double rh2, double tau, double out[7]);
void osim_chem_cell_ions(const osim* s, double rho, double eint, double rh2, double rhp, double tau,
                         double out[15]);
void osim_heatcool_cell_ions(const osim* s, double rho, double eint, double rh2, double rhp, double tau,
                             double out[11]);
int osim_set_option(osim* s, int key, double v);
void o_ppm(const double q[5], int step4_as_written, double out[4]);
void o_face_solve(const double wl[5], const double wr[5], double Bn, const double sl[30], const double sr[30],
                  double tau_h, int edge, int step4_as_written, double out[6]);
double o_cfl_denominator(const double w[9]);
}

using namespace mhd;

static void report(const char* name, long n, double worst, long beyond) {
  std::printf("%s %ld %.6e %ld\n", name, n, worst, beyond);
}

// stencils of five values: rough, smooth, jumps, oscillating, and on a coarse lattice (ties, zeros)
static void stencil(std::mt19937_64& g, long it, double q[5]) {
  std::uniform_real_distribution<double> U(-1, 1);
  const int kind = (int)(it % 5);
  for (int i = 0; i < 5; ++i) {
    if (kind == 0) q[i] = U(g);
    else if (kind == 1) q[i] = 1.0 + 0.01 * i + 1e-3 * U(g) * (i == 2);
    else if (kind == 2) q[i] = (i < 2 + (it / 5) % 3) ? 1.0 : 0.125 + 1e-6 * U(g);
    else if (kind == 3) q[i] = std::sin(0.3 * i + U(g)) * (1 + 0.1 * U(g));
    else q[i] = std::round(4 * U(g)) / 4;
  }
}

int main() {
  std::mt19937_64 g(20160829);
  std::uniform_real_distribution<double> U(-1, 1), U01(0, 1);

  // 1. FP64 parabolas: the oracle's Steps 1-5 exactly (equal values)
  {
    const long n = 400000;
    long bad = 0;
    double worst = 0;
    for (long it = 0; it < n; ++it) {
      double q[5], o[4];
      stencil(g, it, q);
      o_ppm(q, 0, o);
      const Para<double> P = ppm_lean(q[0], q[1], q[2], q[3], q[4]);
      const double d[4] = {P.L, P.R, P.d, P.q6};
      // within 3e-15 of the largest |q| of the stencil: q6 is formed as 6 q_c - 3 (q_L + q_R), two
      // roundings of values up to 6 max|q| on each side (at most 4 ulp of 6 max|q|, 2.7e-15), and the
      // Step 4 blend's eta comes from the Newton-Raphson reciprocal; q_L, q_R and Delta q outside the
      // blend are the oracle's bits
      double sc = 0;
      for (int i = 0; i < 5; ++i) sc = std::max(sc, std::fabs(q[i]));
      double e = 0;
      for (int k = 0; k < 4; ++k) e = std::max(e, std::fabs(d[k] - o[k]) / (sc + 1e-300));
      worst = std::max(worst, e);
      if (e > 3e-15) ++bad;
    }
    report("ppm_lean_close", n, worst, bad);
  }
  // 2. the streamed parabolas equal the five-point ones bit for bit
  {
    long n = 0, bad = 0;
    for (int line = 0; line < 5000; ++line) {
      double q[40];
      const int kind = line % 4;
      for (int i = 0; i < 40; ++i)
        q[i] = kind == 0 ? U(g) : kind == 1 ? std::sin(0.2 * i + line) :
               kind == 2 ? (i < 20 ? 1.0 : 0.125) + 1e-3 * U(g) : std::round(3 * U(g)) / 3;
      PPMStream<double> S;
      S.prime(q[0], q[1], q[2], q[3]);
      for (int j = 2; j < 38; ++j) {
        const Para<double> a = S.next(q[j + 2]);
        const Para<double> b = ppm_lean(q[j - 2], q[j - 1], q[j], q[j + 1], q[j + 2]);
        ++n;
        if (std::memcmp(&a, &b, sizeof(a)) != 0) ++bad;
      }
    }
    report("ppm_stream_bits", n, 0.0, bad);
  }
  // 2b. the FP32 pencils' parabolas with each cell's slope carried to the next two cells (the order
  // of the Eulerian window) equal the five-point ppm_direct bit for bit
  {
    long n = 0, bad = 0;
    for (int line = 0; line < 5000; ++line) {
      float q[40];
      const int kind = line % 4;
      for (int i = 0; i < 40; ++i)
        q[i] = (float)(kind == 0 ? U(g) : kind == 1 ? std::sin(0.2 * i + line) :
                       kind == 2 ? (i < 20 ? 1.0 : 0.125) + 1e-3 * U(g) : std::round(3 * U(g)) / 3);
      float sa = slope_m(q[0], q[1], q[2]), sb = slope_m(q[1], q[2], q[3]);  // cells 1 and 2
      for (int j = 2; j < 38; ++j) {
        const float sc = slope_m(q[j], q[j + 1], q[j + 2]);
        const Para<float> a = ppm_carried(q[j - 1], q[j], q[j + 1], sa, sb, sc,
                                          q[j + 2] - 2.0f * q[j + 1] + q[j], q[j] - 2.0f * q[j - 1] + q[j - 2]);
        const Para<float> b = ppm_direct(q[j - 2], q[j - 1], q[j], q[j + 1], q[j + 2]);
        sa = sb;
        sb = sc;
        ++n;
        if (std::memcmp(&a, &b, sizeof(a)) != 0) ++bad;
      }
    }
    report("ppm_carried_bits", n, 0.0, bad);
  }
  // 3. FP32 parabolas of the FP32-bulk path against the FP64 oracle
  {
    const long n = 200000;
    long bad = 0;
    double worst = 0;
    for (long it = 0; it < n; ++it) {
      double q[5], o[4];
      stencil(g, it, q);
      for (int i = 0; i < 5; ++i) q[i] = (double)(float)q[i];
      o_ppm(q, 0, o);
      const Para<float> a = ppm_direct<float>(q[0], q[1], q[2], q[3], q[4]);
      const Para<float> b = ppm_lean<float>(q[0], q[1], q[2], q[3], q[4]);
      double sc = 0;
      for (int i = 0; i < 5; ++i) sc = std::max(sc, std::fabs(q[i]));
      const double da[4] = {a.L, a.R, a.d, a.q6}, db[4] = {b.L, b.R, b.d, b.q6};
      for (int k = 0; k < 4; ++k) {
        const double e = std::max(std::fabs(da[k] - o[k]), std::fabs(db[k] - o[k])) / (sc + 1e-300);
        worst = std::max(worst, e);
        if (e > 1e-5) ++bad;
      }
    }
    report("ppm_fp32", n, worst, bad);
  }
  // 4. Riemann solve at a face (both precisions) against the oracle's face solve
  {
    const long n = 200000;
    long bad64 = 0, bad32 = 0;
    double w64 = 0, w32 = 0;
    for (long it = 0; it < n; ++it) {
      double wl5[5], wr5[5], sl[30], sr[30];
      auto state = [&](double* w) {
        w[0] = std::exp(2 * U(g));
        w[1] = std::exp(2 * U(g));
        w[2] = 1.4 + 0.3 * U(g);
        const bool no_perp = it % 4 == 1;
        w[3] = no_perp ? 0.0 : U(g);
        w[4] = no_perp ? 0.0 : U(g);
      };
      state(wl5);
      state(wr5);
      const double Bn = (it % 7 == 0) ? 0.0 : 2 * U(g);
      for (int i = 0; i < 30; ++i) {
        sl[i] = U(g);
        sr[i] = U(g);
      }
      const double tau_h = 0.05 * (1 + U(g));
      double o[6];
      o_face_solve(wl5, wr5, Bn, sl, sr, tau_h, 0, 0, o);
      double sc = 0;
      for (int m = 0; m < 6; ++m) sc = std::max(sc, std::fabs(o[m]));
      {
        double wl[6], wr[6], qs[6];
        for (int i = 0; i < 5; ++i) {
          wl[i] = wl5[i];
          wr[i] = wr5[i];
        }
        wl[5] = std::sqrt(wl5[0]);
        wr[5] = std::sqrt(wr5[0]);
        Para<double> pl[6], pr[6];
        for (int v = 0; v < 6; ++v) {
          pl[v] = ppm_lean(sl[5 * v], sl[5 * v + 1], sl[5 * v + 2], sl[5 * v + 3], sl[5 * v + 4]);
          pr[v] = ppm_lean(sr[5 * v], sr[5 * v + 1], sr[5 * v + 2], sr[5 * v + 3], sr[5 * v + 4]);
        }
        riemann(wl, wr, Bn, pl, pr, tau_h, qs);
        for (int m = 0; m < 6; ++m) {
          const double e = std::fabs(qs[m] - o[m]) / (sc + 1e-300);
          w64 = std::max(w64, e);
          if (e > 1e-12) ++bad64;
        }
      }
      {
        float wl[6], wr[6], qs[6];
        for (int i = 0; i < 5; ++i) {
          wl[i] = (float)wl5[i];
          wr[i] = (float)wr5[i];
        }
        wl[5] = std::sqrt(wl[0]);
        wr[5] = std::sqrt(wr[0]);
        Para<float> pl[6], pr[6];
        for (int v = 0; v < 6; ++v) {
          pl[v] = ppm_direct<float>(sl[5 * v], sl[5 * v + 1], sl[5 * v + 2], sl[5 * v + 3], sl[5 * v + 4]);
          pr[v] = ppm_direct<float>(sr[5 * v], sr[5 * v + 1], sr[5 * v + 2], sr[5 * v + 3], sr[5 * v + 4]);
        }
        riemann<float>(wl, wr, (float)Bn, pl, pr, (float)tau_h, qs);
        for (int m = 0; m < 6; ++m) {
          const double e = std::fabs(qs[m] - o[m]) / (sc + 1e-300);
          w32 = std::max(w32, e);
          if (e > 1e-4) ++bad32;
        }
      }
    }
    report("riemann_fp64", n, w64, bad64);
    report("riemann_fp32", n, w32, bad32);
  }
  // 5. chemistry of one cell (FP64) against the oracle's
  {
    const double dx = 2.0;
    osim* s = osim_create(4, 4, 4, 5.0 / 3.0, dx);
    Phys ph{};
    ph.dx = dx;
    ph.ih = 1.0 / dx;
    ph.chem = 1;
    ph.lshield = 0.0;
    ph.bdop = 3.0;
    ph.xnorm = 5e14;
    ph.taud = 1e-21;
    ph.ibdop = 1.0 / ph.bdop;
    ph.ixnorm = 1.0 / ph.xnorm;
    set_shielding(ph);
    ph.heatcool = 1;
    const long n = 300000;
    long bad = 0;
    double worst = 0;
    for (long it = 0; it < n; ++it) {
      const double rho = std::exp(10 * U01(g) - 3);
      const double rh2 = rho * U01(g) * (it % 3 ? 1.0 : 1e-6);
      const double eint = rho * std::exp(14 * U01(g) - 6);
      const double tau = std::exp(10 * U01(g) - 12);
      double o[8];
      osim_chem_cell(s, rho, eint, rh2, tau, o);
      const double a = chem_cell<false>(ph, rho, eint, rh2, 0.0, tau).rh2;
      const double e = std::fabs(a - o[0]) / std::max(std::fabs(o[0]), 1e-12 * rho);
      worst = std::max(worst, e);
      if (e > 1e-12) ++bad;
    }
    report("chemistry", n, worst, bad);
    // 5b. heating/cooling of one cell (FP64, Sec. 2.8) against the oracle's
    osim_set_option(s, 13, 1.0);
    long badh = 0;
    double worsth = 0;
    for (long it = 0; it < n; ++it) {
      const double rho = std::exp(12 * U01(g) - 4);
      const double rh2 = rho * U01(g) * (it % 3 ? 1.0 : 1e-6) * (it % 11 == 0 ? 0.0 : 1.0);
      const double eint = rho * std::exp(14 * U01(g) - 8);
      const double tau = std::exp(10 * U01(g) - 12);
      double o[7];
      osim_heatcool_cell(s, rho, eint, rh2, tau, o);
      const double a = heatcool_delta<false>(ph, rho, eint, rh2, 0.0, tau);
      // relative to the gross exchange tau (Gamma_1 + Gamma_4 + Lambda_2 + Lambda_3) in code units:
      // the net change cancels near equilibrium
      const double gross = tau * (3.0856775814913673e18 / 1e5) * (o[2] + o[3] + o[4] + o[5]) / (1.6735575e-24 * 1e10);
      const double e = std::fabs(a - o[0]) / std::max(std::max(std::fabs(o[0]), gross), 1e-300);
      worsth = std::max(worsth, e);
      if (e > 1e-12) ++badh;
    }
    report("heatcool", n, worsth, badh);
    // 5c. with H+ and electrons (reactions 5-8): the new rho_H2 and rho_H+, and the heating/cooling
    // change with Gamma_5, Lambda_6-8, over cold to hot, neutral to fully ionised cells
    osim_set_option(s, 15, 1.0);
    ph.ions = 1;
    long badi = 0, badhi = 0;
    double worsti = 0, worsthi = 0;
    for (long it = 0; it < n; ++it) {
      const double rho = std::exp(12 * U01(g) - 4);
      const double f2 = U01(g) * (it % 3 ? 1.0 : 1e-6) * (it % 13 == 0 ? 0.0 : 1.0);
      const double fp = (1.0 - f2) * U01(g) * (it % 5 ? 1.0 : 1e-6) * (it % 17 == 0 ? 0.0 : 1.0);
      const double rh2 = rho * f2, rhp = rho * fp;
      const double eint = rho * std::exp(16 * U01(g) - 8);
      const double tau = std::exp(10 * U01(g) - 12);
      double o[15];
      osim_chem_cell_ions(s, rho, eint, rh2, rhp, tau, o);
      const ChemOut a = chem_cell<true>(ph, rho, eint, rh2, rhp, tau);
      // relative to the largest density the update adds or subtracts: the printed form n + tau (C -
      // D n) / (1 + tau D) cancels where recombination removes nearly all of n_H+, leaving a rounding
      // error of order eps n_H+(start) on both sides
      const double e = std::max(std::fabs(a.rh2 - o[0]), std::fabs(a.rhp - o[1])) /
                       std::max({std::fabs(o[0]), std::fabs(o[1]), rh2, rhp, 1e-12 * rho});
      worsti = std::max(worsti, e);
      if (e > 1e-12) ++badi;
      double h[11];
      osim_heatcool_cell_ions(s, rho, eint, rh2, rhp, tau, h);
      const double d = heatcool_delta<true>(ph, rho, eint, rh2, rhp, tau);
      double gross_rate = 0.0;
      for (int k = 2; k <= 9; ++k) gross_rate += std::fabs(h[k]);
      const double gross = tau * (3.0856775814913673e18 / 1e5) * gross_rate / (1.6735575e-24 * 1e10);
      const double eh = std::fabs(d - h[0]) / std::max(std::max(std::fabs(h[0]), gross), 1e-300);
      worsthi = std::max(worsthi, eh);
      if (eh > 1e-12) ++badhi;
    }
    // 5d. the instances with the ion code, on a box without ions (rho_H+ = 0), give the bits of the
    // instances without it (a batch that mixes such boxes runs the former for all of them)
    ph.ions = 0;
    long badsame = 0;
    for (long it = 0; it < n / 10; ++it) {
      const double rho = std::exp(12 * U01(g) - 4);
      const double rh2 = rho * U01(g) * (it % 3 ? 1.0 : 1e-6);
      const double eint = rho * std::exp(16 * U01(g) - 8);
      const double tau = std::exp(10 * U01(g) - 12);
      const ChemOut a1 = chem_cell<true>(ph, rho, eint, rh2, 0.0, tau);
      const ChemOut a0 = chem_cell<false>(ph, rho, eint, rh2, 0.0, tau);
      const double h1 = heatcool_delta<true>(ph, rho, eint, rh2, 0.0, tau);
      const double h0 = heatcool_delta<false>(ph, rho, eint, rh2, 0.0, tau);
      if (std::memcmp(&a1.rh2, &a0.rh2, 8) != 0 || std::memcmp(&h1, &h0, 8) != 0) ++badsame;
    }
    osim_destroy(s);
    report("chemistry_ions", n, worsti, badi);
    report("heatcool_ions", n, worsthi, badhi);
    report("ion_instances_without_ions_same_bits", n / 10, 0.0, badsame);
  }
  // 5d. the Newton-Raphson reciprocal, reciprocal square root and square root against the correctly
  // rounded library values: within 2 ulp over the normal range
  {
    const long n = 1000000;
    long bad = 0;
    double worst = 0;
    for (long it = 0; it < n; ++it) {
      const double x = std::ldexp(1.0 + U01(g), (int)(2040 * U01(g)) - 1020) * (it % 2 ? 1.0 : -1.0);
      const double ax = std::fabs(x);
      const double e1 = std::fabs(rcp_nr(x) - 1.0 / x) / std::fabs(1.0 / x);
      const double e2 = std::fabs(rsqrt_nr(ax) - 1.0 / std::sqrt(ax)) * std::sqrt(ax);
      const double e3 = std::fabs(sqrt_nr(ax) - std::sqrt(ax)) / std::sqrt(ax);
      const double e = std::max(e1, std::max(e2, e3)) / 2.220446049250313e-16;
      worst = std::max(worst, e);
      if (e > 2.0) ++bad;
    }
    report("newton_raphson_ulp", n, worst, bad);
  }
  // 5e. the table-driven exponential of the chemistry rates (Tang's method) against e^x in long
  // double: within 1.01 ulp (half an ulp of the table entry, scaled by e^r <= 1.011, and half an ulp
  // of the last rounding) over the rates' argument range [-746, 0] (dense near 0 and over whole
  // decades of small arguments), the ends of its fast range and the library tail below it
  {
    const long n = 2000000;
    long bad = 0;
    double worst = 0;
    auto ulp_err = [](double y, long double e) -> double {
      if (e == 0.0L) return y == 0.0 ? 0.0 : 1e300;
      const double ulp = std::ldexp(1.0, std::max(std::ilogb((double)e), -1022) - 52);
      return (double)(std::fabs((long double)y - e) / ulp);
    };
    const double special[] = {0.0, -0.0, -5e-324, -1e-300, -1e-17, -0.010830424696249145,
                              -0.010830424696249146, -0.5, -1.0, -707.0, -706.9999999999999,
                              -707.0000000000001, -708.0, -708.4, -745.0, -745.13, -746.0, 1.0, 706.9};
    long cases = 0;
    for (double x : special) {
      const double e = ulp_err(exp_tang(x), expl((long double)x));
      worst = std::max(worst, e);
      if (e > 1.01) ++bad;
      ++cases;
    }
    for (long it = 0; it < n; ++it) {
      const int kind = (int)(it % 4);
      const double x = kind == 0 ? -746.0 * U01(g)
                     : kind == 1 ? -U01(g)
                     : kind == 2 ? -std::ldexp(1.0 + U01(g), -(int)(60 * U01(g)))
                                 : -20.0 * U01(g);
      const double e = ulp_err(exp_tang(x), expl((long double)x));
      worst = std::max(worst, e);
      if (e > 1.01) ++bad;
      ++cases;
    }
    report("exp_tang_ulp", cases, worst, bad);
  }
  // 5f. the FP32 estimate of the CFL screen against the FP64 denominator of the same cell: within
  // 64 u (u = 2^-24; the screen allows 4096 u) wherever the guards pass, on densities, momenta,
  // fields and internal energies over many decades, zero components, the ideal gas with gamma - 1
  // down to 1e-4, and the H/H2 (+ H+) mixture with some unphysical abundances; the guards must pass
  // on at least half of the cases
  {
    const long n = 1000000;
    long bad = 0, passed = 0;
    double worst = 0;
    auto logu = [&](double lo, double hi) { return std::exp(std::log(lo) + (std::log(hi) - std::log(lo)) * U01(g)); };
    for (long it = 0; it < n; ++it) {
      const int kind = (int)(it % 4);
      const bool chem = (it / 4) % 2;
      const double rho = kind == 0 ? logu(1e-13, 1e13) : logu(1e-3, 1e3);
      double m[3], Bv[3];
      for (int d = 0; d < 3; ++d) {
        m[d] = U01(g) < 0.1 ? 0.0 : U(g) * (kind == 1 ? logu(1e-30, 1e10) : logu(1e-3, 1e3));
        Bv[d] = U01(g) < 0.2 ? 0.0 : U(g) * (kind == 2 ? logu(1e-30, 1e10) : logu(1e-3, 1e3));
      }
      const double eint = rho * (kind == 3 ? logu(1e-16, 1e8) : logu(1e-4, 1e4));
      const double fhp = it % 3 == 0 ? 0.0 : 0.1 * U01(g);
      double rh2 = rho * U01(g) * (1.0 - fhp);
      const double rhp = rho * fhp;
      if (it % 97 == 0) rh2 = rho * (1.0 + 0.5 * U01(g));  // more H2 than gas
      const double gamma = chem ? 5.0 / 3.0 : 1.0 + logu(1e-4, 0.67);
      const float gm1 = gamma_minus_one_f32(chem, gamma, (float)rho, (float)rh2, (float)rhp);
      const float D32 = cfl_estimate_f32((float)rho, (float)m[0], (float)m[1], (float)m[2], (float)Bv[0],
                                         (float)Bv[1], (float)Bv[2], (float)eint, gm1);
      if (!(D32 <= 3.0e38f)) continue;
      ++passed;
      const double gm = chem ? gamma_eff(rho, rh2, rhp) : gamma;
      const double D = cfl_denominator(rho, m[0], m[1], m[2], Bv[0], Bv[1], Bv[2], gm * ((gm - 1.0) * eint));
      const double e = (std::isfinite(D) && D > 0.0) ? std::fabs((double)D32 - D) / D : 1e300;
      worst = std::max(worst, e);
      if (e > 0x1p-18) ++bad;
    }
    report("cfl_screen_bound", passed, worst, bad);
    report("cfl_screen_guard_share", n, (double)passed / n, passed < n / 2 ? 1 : 0);
  }
  // 6. CFL denominator (FP64) against the oracle's
  {
    const long n = 300000;
    long bad = 0;
    double worst = 0;
    for (long it = 0; it < n; ++it) {
      const double rho = std::exp(4 * U(g));
      const double m[3] = {10 * U(g), 10 * U(g), 10 * U(g)};
      const double Bv[3] = {3 * U(g), (it % 5 == 0) ? 0.0 : 3 * U(g), (it % 7 == 0) ? 0.0 : 3 * U(g)};
      const double gam = 1.4 + 0.3 * U01(g), p = std::exp(4 * U(g));
      const double w[9] = {rho, m[0] / rho, m[1] / rho, m[2] / rho, Bv[0], Bv[1], Bv[2], p, gam};
      const double o = o_cfl_denominator(w);
      const double a = cfl_denominator(rho, m[0], m[1], m[2], Bv[0], Bv[1], Bv[2], gam * p);
      const double e = std::fabs(a - o) / o;
      worst = std::max(worst, e);
      if (e > 1e-13) ++bad;
    }
    report("cfl", n, worst, bad);
  }
  // the index decoding's division by an invariant divisor (FastDiv, Granlund-Montgomery) against
  // the integer division: every divisor up to 4096 and a spread of larger ones, with quotient
  // boundaries, small and large dividends and random ones up to 2^32 - 1
  {
    long n = 0, bad = 0;
    std::uniform_int_distribution<unsigned> Ut(0u, 0xffffffffu);
    std::vector<unsigned> divs;
    for (unsigned d = 1; d <= 4096; ++d) divs.push_back(d);
    for (int k = 0; k < 2000; ++k) divs.push_back(1u + (unsigned)(g() % 0x7fffffffu));
    for (unsigned d : {65535u, 65536u, 65537u, 1u << 20, (1u << 31) - 1u, 1u << 31, 0xffffffffu}) divs.push_back(d);
    for (unsigned d : divs) {
      const mhd::FastDiv f = mhd::make_fastdiv(d);
      auto check = [&](unsigned t) {
        ++n;
        if (mhd::fdiv(t, f) != t / d) ++bad;
      };
      for (unsigned t = 0; t < 300; ++t) check(t);
      for (unsigned k = 1; k < 40; ++k) {
        const unsigned long long b = (unsigned long long)k * d;
        if (b <= 0xffffffffull) {
          check((unsigned)b);
          if (b > 0) check((unsigned)(b - 1));
        }
      }
      check(0xffffffffu);
      check(0x7fffffffu);
      for (int k = 0; k < 64; ++k) check(Ut(g));
    }
    report("fast_index_division", n, 0.0, bad);
  }
  return 0;
}
