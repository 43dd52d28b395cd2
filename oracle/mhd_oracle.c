/*
 * mhd_oracle.c -- plain FP64 CPU oracle for the MHD + H/H2 chemistry time step of
 * Kulikov, Chernykh & Protasov, "A new code for numerical simulation of MHD astrophysical
 * flows with chemistry" (arXiv:1608.08748).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load this file.  It shares no code with the CUDA library: it keeps explicit ghost
 * layers, loops over (k, j, i) in plain order and stores intermediate results in full-grid
 * arrays.  It is compiled with -O2 -ffp-contract=off so that every a*b+c is rounded twice, the
 * way the formulas are written.
 *
 * What it computes (paper section / equation in brackets):
 *   state          rho, m = rho v, rho E, rho eps, rho_H2 cell-centred; b_x, b_y, b_z on faces
 *                  [Sec. 2 closure: p = (gamma-1) rho eps, rho E = rho eps + rho v^2/2 + B^2/2]
 *   one step       tau from the CFL rule [Sec. 2.3] (truncated at t_end when asked),
 *                  Eulerian stage with Flux-CT inside each SSP-RK3 substage [Sec. 2.2, 2.4, 2.5,
 *                  App. A, App. C], Lagrangian stage with SSP-RK3 [Sec. 2.6], H/H2 chemistry
 *                  [Sec. 2.7, App. D reactions 1-4; with the ion option also reactions 5-8 with
 *                  H+ and e], heating/cooling when on [Sec. 2.8], regularisation [Sec. 2.9];
 *                  self-gravity when on [Sec. 2.10].
 *   PPM            local parabola, Steps 1-5 [Sec. 2.1]; domain-of-dependence averages [Sec. 2.4].
 *
 * Readings taken where the paper is garbled or silent (each documented at its use):
 *   A1  Delta q = q^R - q^L (the parabola's endpoints and the averages of Sec. 2.4 need it).
 *   A2  delta^2 q_j = (q_{j+1} - 2 q_j + q_{j-1}) / (3 h^2), so eta = -(D_{i+1}-D_{i-1}) /
 *       (3 (q_{i+1}-q_{i-1})) with D the undivided second difference.
 *   A3  eta := 0 when |q_{i+1}-q_{i-1}| <= min(|q_{i+1}|,|q_{i-1}|)/100 or D_{i+1} D_{i-1} > 0.
 *   A4  weights of Step 4 swapped: q_final = hbar q^{+} + (1 - hbar) q (flag: as written).
 *   A5  b^2 = B^2/rho; c_a, c_s, c_f with B_d longitudinal for each d; max over d.
 *   A6  v = |v|, h = dx.
 *   A7  face rho as written; p and gamma with the velocity weights; B_n = staggered face value.
 *   A8  degenerate alpha when c_f^2 - c_s^2 <= 1e-12 (c^2 + b^2); degenerate beta when
 *       B_perp^2 <= 1e-24 rho (c^2 + b^2); sign(0) = +1; speeds and alpha evaluated in a
 *       cancellation-free form of the same formulas (mhd_speeds).
 *   A9  row k of R^T is the right eigenvector for (+c_f, -c_f, +c_s, -c_s, +c_a, -c_a).
 *   A10 Flux-CT inside each Eulerian RK substage; tau fixed for the whole step.
 *   A11 domain-of-dependence averages (flag: edge values, i.e. the tau -> 0 limit).
 *   A12 Eulerian fluxes: momentum p* n - B_n B, energy p* V_n - B_n (B.V), rho eps source
 *       -(gamma-1) rho eps div V.
 *   A13 Lagrangian face velocity from the two cell-centre normal velocities; v >= 0 takes the
 *       left parabola; conserved densities are reconstructed.
 *   A14 regularisation: f >= 1e-3 -> rho eps := max(rho eps, rho E - rho v^2/2 - B^2/2), the
 *       form that never lowers the entropy; else rescale |v| keeping its direction (flags:
 *       unconditional overwrite; the sentence's literal branch order).
 *   A15 H2 updated by the Sec. 2.7 formula with C = k1' n n_H, D = k2 n_H + k3 n_H2 + k4;
 *       n_H := n - 2 n_H2; column densities N_X = n_X L_shield.
 *   A16 outflow = zero-gradient copy of ghost cells (their primitives, cell-centred B included)
 *       and of ghost faces; periodic otherwise.
 *   A17 set_state builds faces as the mean of the two neighbouring cell-centred values.
 *   A18 tau = min(tau_CFL, t_end - t) when a target time is given.
 *   A19 code units: 1 pc, m_H cm^-3, 1 km/s.
 *   A23 no positivity floors; rho <= 0, p <= 0 or a non-finite value is reported.
 *   A24-A31 heating/cooling and self-gravity readings (at their use).
 *   A32 ions: one more advected density rho_H+ = n_H+ (proton mass = m_H), n_e = n_H+ (charge
 *       neutrality of pure hydrogen), neutral atoms n_H = rho - rho_H2 - rho_H+.
 *   A33 gamma_eff of Sec. 4.3 with electrons: its n_H counts every nucleus outside H2 (n_H +
 *       n_H+), so gamma = (5 n_1 + 7 n_H2) / (3 n_1 + 5 n_H2), n_1 = n_H + n_H+ + n_e; T counts
 *       every particle, p = (n_H + n_H2 + n_H+ + n_e) k_B T.
 *   A34-A37 rates of reactions 5-8 (at ion_rates_at); A38 the H+ update; A39 Gamma_5, Lambda_6-8.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NG 4 /* ghost layers: 3 for the PPM stencil of a face, 1 more for the CT edges */

/* option keys of the oracle (its own numbering) */
enum {
  O_BC_X = 1, O_BC_Y = 2, O_BC_Z = 3, /* 0 periodic, 1 outflow */
  O_CHEM = 4,                         /* 0 off, 1 H/H2 network on */
  O_STEP4_AS_WRITTEN = 5,             /* A4 flag */
  O_IFACE_EDGE = 6,                   /* A11 flag */
  O_REGUL_MODE = 7,                   /* A14: 0 max form (default), 1 unconditional, 2 literal */
  O_CHEM_LSHIELD = 8,                 /* shielding length in code length units (0: dx) */
  O_CHEM_BDOP = 9,                    /* Doppler parameter b in km/s */
  O_CHEM_XNORM = 10,                  /* N_H2 normaliser of f_shield, cm^-2 */
  O_CHEM_TAUD = 11,                   /* dust optical depth per column, cm^2 */
  O_THREADS = 12,
  O_HEATCOOL = 13,                    /* 0 off (default), 1 Sec. 2.8 heating/cooling (needs chemistry) */
  O_GRAV_G = 14,                      /* G in code units for self-gravity (0: off, the default; periodic) */
  O_IONS = 15                         /* 0 off (default), 1 reactions 5-8 with H+ and e (needs chemistry) */
};

enum { O_OK = 0, O_EINVAL = -1, O_ENOMEM = -2, O_ENONPHYS = -4 };

/* physical constants (CGS) and code units (A19) */
static const double KB_CGS = 1.380649e-16;
static const double MH_CGS = 1.6735575e-24;
static const double PC_CGS = 3.0856775814913673e18;
static const double KMS_CGS = 1.0e5;
static const double KB_EV = 8.617333262e-5; /* Boltzmann constant in eV/K (A27) */

typedef struct {
  int n[3];   /* nx, ny, nz */
  int ne[3];  /* extended sizes n + 2 NG */
  size_t next; /* extended cell count */
  int bc[3];
  double gamma, dx;
  int chem, step4_as_written, iface_edge, regul_mode, threads, heatcool, ions;
  double lshield, bdop, xnorm, taud;
  double grav_g;     /* gravitational constant in code units (0: no self-gravity) */
  double t;
  long nsteps, nvel_branch;
  /* state on the extended grid */
  double *rho, *m[3], *E, *eint, *rh2, *rhp, *b[3]; /* rhp: rho_H+ = n_H+ (A32) */
  /* RK register Q^n and scratch */
  double *rho0, *m0[3], *E0, *eint0, *rh20, *rhp0, *b0[3];
  double *w[9];      /* primitives: rho, v0, v1, v2, B0, B1, B2, p, gamma */
  double *fo[8];     /* face outputs of the current direction */
  double *acc[6];    /* accumulated flux differences: m0, m1, m2, E, div v, (rho_H2 / rho) */
  double *accL[8];   /* Lagrangian accumulators */
  double *eA[3], *eB[3]; /* per-direction EMF contributions of the faces */
  double *edge[3];   /* edge EMFs E_x, E_y, E_z */
  double *phi;       /* gravitational potential (extended grid) */
} osim;

/* ---------------------------------------------------------------- indexing */
static inline size_t IX(const osim* s, int ie, int je, int ke) {
  return ((size_t)ke * s->ne[1] + je) * s->ne[0] + ie;
}
/* step of one cell along axis d in the extended layout */
static inline ptrdiff_t ST(const osim* s, int d) {
  return d == 0 ? 1 : (d == 1 ? (ptrdiff_t)s->ne[0] : (ptrdiff_t)s->ne[0] * s->ne[1]);
}

static int map_index(int i, int n, int bc) {
  if (bc == 0) { int r = i % n; return r < 0 ? r + n : r; }
  return i < 0 ? 0 : (i >= n ? n - 1 : i); /* A16: zero-gradient copy */
}

/* fill the ghost layers of one extended array from its interior (cells and faces alike:
   face index i stands for the face i - 1/2, so the same map gives the nearest stored face) */
static void fill_ghosts(const osim* s, double* a) {
  const int nx = s->n[0], ny = s->n[1], nz = s->n[2];
#pragma omp parallel for schedule(static) num_threads(s->threads)
  for (int ke = 0; ke < s->ne[2]; ++ke)
    for (int je = 0; je < s->ne[1]; ++je)
      for (int ie = 0; ie < s->ne[0]; ++ie) {
        int i = ie - NG, j = je - NG, k = ke - NG;
        if (i >= 0 && i < nx && j >= 0 && j < ny && k >= 0 && k < nz) continue;
        int si = map_index(i, nx, s->bc[0]) + NG, sj = map_index(j, ny, s->bc[1]) + NG,
            sk = map_index(k, nz, s->bc[2]) + NG;
        a[IX(s, ie, je, ke)] = a[IX(s, si, sj, sk)];
      }
}

/* ---------------------------------------------------------------- Sec. 2.1 local parabola */
typedef struct { double L, R, d, q6; } para; /* q^L, q^R, Delta q = q^R - q^L (A1), q^(6) */

static const double SIXTH = 1.0 / 6.0;
static const double TWO_THIRDS = 2.0 / 3.0;

/* Step 1: limited slope delta_m q_j from q_{j-1}, q_j, q_{j+1} */
static double slope_m(double qm, double q0, double qp) {
  double dq = 0.5 * (qp - qm);
  double dp = qp - q0, dn = q0 - qm;
  if (dp * dn > 0.0) {
    double a = fabs(dq), b = 2.0 * fabs(dp), c = 2.0 * fabs(dn);
    double mn = a < b ? a : b;
    mn = mn < c ? mn : c;
    return copysign(mn, dq);
  }
  return 0.0;
}

/* Step 4 discontinuity detector for cell i from q[0..4] = q_{i-2}..q_{i+2}: the criterion eta
   with D the undivided second difference (A2), zeroed by the two conditions (A3), and the weight
   hbar = max(min(20 (eta - 0.05), 1), 0) of the flattened edge values.  eta_out may be NULL. */
static double step4_weight(const double q[5], double* eta_out) {
  double Dp = q[4] - 2.0 * q[3] + q[2];
  double Dm = q[2] - 2.0 * q[1] + q[0];
  double dq2 = q[3] - q[1];
  double ap = fabs(q[3]), am = fabs(q[1]);
  double mn = ap < am ? ap : am;
  double sum = ap + am;
  mn = mn < sum ? mn : sum;
  double eta;
  if (fabs(dq2) - 0.01 * mn <= 0.0 || Dp * Dm > 0.0)
    eta = 0.0;
  else
    eta = -(Dp - Dm) / (3.0 * dq2);
  double hb = 20.0 * (eta - 0.05);
  hb = hb < 1.0 ? hb : 1.0;
  hb = hb > 0.0 ? hb : 0.0;
  if (eta_out) *eta_out = eta;
  return hb;
}

/* Steps 1-5 for cell i from q[0..4] = q_{i-2}..q_{i+2} */
static para ppm_cell(const double q[5], int step4_as_written) {
  const double qc = q[2];
  double dmm = slope_m(q[0], q[1], q[2]);
  double dm0 = slope_m(q[1], q[2], q[3]);
  double dmp = slope_m(q[2], q[3], q[4]);
  /* Step 1: fourth-order edge values from the limited slopes */
  double qL = 0.5 * (q[1] + q[2]) - (dm0 - dmm) * SIXTH;
  double qR = 0.5 * (q[2] + q[3]) - (dmp - dm0) * SIXTH;
  /* Step 2: monotonise (extremum -> flat; else the two overshoot fixes, mutually exclusive) */
  double dq = qR - qL;
  double q6 = 6.0 * (qc - 0.5 * (qL + qR));
  if ((qL - qc) * (qc - qR) <= 0.0) {
    qL = qc;
    qR = qc;
  } else if (dq * q6 > dq * dq) {
    qL = 3.0 * qc - 2.0 * qR;
  } else if (dq * q6 < -(dq * dq)) {
    qR = 3.0 * qc - 2.0 * qL;
  }
  /* Step 3 recomputes Delta q and q6; Step 4 only needs q^L, q^R, so they are recomputed in
     Step 5 below. */
  /* Step 4: flattened edge values q -+ delta_m q / 4, weighted by hbar (A2, A3, A4) */
  double qLp = qc - 0.25 * dm0, qRp = qc + 0.25 * dm0;
  double hb = step4_weight(q, NULL);
  if (step4_as_written) {
    qL = (1.0 - hb) * qLp + hb * qL;
    qR = (1.0 - hb) * qRp + hb * qR;
  } else {
    qL = hb * qLp + (1.0 - hb) * qL;
    qR = hb * qRp + (1.0 - hb) * qR;
  }
  /* Step 5 */
  para P;
  P.L = qL;
  P.R = qR;
  P.d = qR - qL;
  P.q6 = 6.0 * (qc - 0.5 * (qL + qR));
  return P;
}

/* Sec. 2.4: average of the parabola over the last fraction y = nu tau / h of the cell
   (q(-nu t), a wave leaving through the right face) and over the first fraction (q(nu t)). */
static double avg_right_end(para P, double y) {
  return P.R - 0.5 * y * (P.d - P.q6 * (1.0 - TWO_THIRDS * y));
}
static double avg_left_end(para P, double y) {
  return P.L + 0.5 * y * (P.d + P.q6 * (1.0 - TWO_THIRDS * y));
}

/* ---------------------------------------------------------------- Sec. 2.4 / App. A eigensystem */
typedef struct {
  double rho, p, gam, Bn, Bt1, Bt2; /* face-averaged state */
  double c, cf, cs, ca, af, as, by, bz, sg, sqr;
  double R[6][6]; /* R[m][k]: component m of right eigenvector k */
  double L[6][6]; /* L[k][m]: component m of left eigenvector k */
  double lam[6];
} eig;

static const double INV_SQRT2 = 0.70710678118654752440;

/* Fast and slow magnetosonic speeds (Sec. 2.3) and the differences the alpha factors of Sec. 2.4
   need, from c^2, c_a^2 = B_n^2/rho and b_perp^2 = B_perp^2/rho, evaluated without cancellation
   (A8): with X = c^2 - c_a^2,
     c_f^2 - c_s^2 = sqrt((c^2 + b^2)^2 - 4 c^2 c_a^2) = sqrt(X^2 + b_perp^2 (2c^2 + 2c_a^2 + b_perp^2)),
     (c^2 - c_s^2)(c_f^2 - c^2) = c^2 b_perp^2,   c_f^2 c_s^2 = c^2 c_a^2.
   The literal form takes the square root of rounding noise where B_perp -> 0; this one gives
   alpha_s = 0 (or alpha_f = 0) exactly there, as the formula intends. */
typedef struct { double cf2, cs2, sq, dcs, dfc; } speeds; /* dcs = c^2 - c_s^2, dfc = c_f^2 - c^2 */

static speeds mhd_speeds(double c2, double ca2, double bp2) {
  speeds r;
  double X = c2 - ca2;
  double W = bp2 * ((2.0 * c2 + 2.0 * ca2) + bp2);
  r.sq = sqrt(X * X + W);
  if (X >= 0.0) {
    r.dcs = 0.5 * ((X + r.sq) - bp2);
    if (r.dcs < 0.0) r.dcs = 0.0;
    r.dfc = r.dcs > 0.0 ? c2 * bp2 / r.dcs : 0.0;
  } else {
    r.dfc = 0.5 * ((bp2 - X) + r.sq);
    r.dcs = r.dfc > 0.0 ? c2 * bp2 / r.dfc : 0.0;
  }
  r.cf2 = c2 + r.dfc;
  r.cs2 = r.cf2 > 0.0 ? c2 * ca2 / r.cf2 : 0.0;
  return r;
}

/* Build R, L and the eigenvalues for the face state (A5, A8, A9). */
static void build_eigen(eig* e) {
  const double rho = e->rho, p = e->p, gam = e->gam, Bn = e->Bn, Bt1 = e->Bt1, Bt2 = e->Bt2;
  double c2 = gam * p / rho;
  double ca2 = Bn * Bn / rho;
  double bp2r = (Bt1 * Bt1 + Bt2 * Bt2) / rho;
  double s = c2 + (ca2 + bp2r);
  speeds sp = mhd_speeds(c2, ca2, bp2r);
  double c = sqrt(c2), cf = sqrt(sp.cf2), cs = sqrt(sp.cs2), ca = sqrt(ca2);
  double af, as;
  if (sp.sq > 1e-12 * s) {
    af = sqrt(sp.dcs / sp.sq);
    as = sqrt(sp.dfc / sp.sq);
  } else {
    af = INV_SQRT2;
    as = INV_SQRT2;
  }
  double bp2 = Bt1 * Bt1 + Bt2 * Bt2;
  double by, bz;
  if (bp2 > 1e-24 * rho * s) {
    double bp = sqrt(bp2);
    by = Bt1 / bp;
    bz = Bt2 / bp;
  } else {
    by = INV_SQRT2;
    bz = INV_SQRT2;
  }
  double sg = Bn >= 0.0 ? 1.0 : -1.0;
  double sqr = sqrt(rho);
  e->c = c; e->cf = cf; e->cs = cs; e->ca = ca; e->af = af; e->as = as;
  e->by = by; e->bz = bz; e->sg = sg; e->sqr = sqr;
  e->lam[0] = cf; e->lam[1] = -cf; e->lam[2] = cs; e->lam[3] = -cs; e->lam[4] = ca; e->lam[5] = -ca;

  /* App. A, R^T: row k = right eigenvector k over q = (v_n, v_t1, v_t2, B_t1, B_t2, p) */
  double gp = gam * p, sc = sqr * c, sr2 = sqrt(0.5 * rho);
  double rk[6][6] = {
      {af * cf, -as * cs * by * sg, -as * cs * bz * sg, as * sc * by, as * sc * bz, af * gp},
      {-af * cf, as * cs * by * sg, as * cs * bz * sg, as * sc * by, as * sc * bz, af * gp},
      {as * cs, af * cf * by * sg, af * cf * bz * sg, -af * sc * by, -af * sc * bz, as * gp},
      {-as * cs, -af * cf * by * sg, -af * cf * bz * sg, -af * sc * by, -af * sc * bz, as * gp},
      {0.0, -bz * INV_SQRT2 * sg, by * INV_SQRT2 * sg, sr2 * bz, -sr2 * by, 0.0},
      {0.0, -bz * INV_SQRT2 * sg, by * INV_SQRT2 * sg, -sr2 * bz, sr2 * by, 0.0}};
  /* App. A, L: row k = left eigenvector k */
  double i2c2 = 1.0 / (2.0 * c2), i2sc = 1.0 / (2.0 * sc), i2rc2 = 1.0 / (2.0 * rho * c2);
  double isr2 = 1.0 / sqrt(2.0 * rho);
  double lk[6][6] = {
      {af * cf * i2c2, -as * cs * by * sg * i2c2, -as * cs * bz * sg * i2c2, as * by * i2sc,
       as * bz * i2sc, af * i2rc2},
      {-af * cf * i2c2, as * cs * by * sg * i2c2, as * cs * bz * sg * i2c2, as * by * i2sc,
       as * bz * i2sc, af * i2rc2},
      {as * cs * i2c2, af * cf * by * sg * i2c2, af * cf * bz * sg * i2c2, -af * by * i2sc,
       -af * bz * i2sc, as * i2rc2},
      {-as * cs * i2c2, -af * cf * by * sg * i2c2, -af * cf * bz * sg * i2c2, -af * by * i2sc,
       -af * bz * i2sc, as * i2rc2},
      {0.0, -bz * sg * INV_SQRT2, by * sg * INV_SQRT2, bz * isr2, -by * isr2, 0.0},
      {0.0, -bz * sg * INV_SQRT2, by * sg * INV_SQRT2, -bz * isr2, by * isr2, 0.0}};
  for (int k = 0; k < 6; ++k)
    for (int m = 0; m < 6; ++m) {
      e->R[m][k] = rk[k][m];
      e->L[k][m] = lk[k][m];
    }
}

/* Sec. 2.4 averaging of the two cells' values at a face (A7). wl/wr hold rho, p, gamma, B_t1,
   B_t2 of the left/right cell. */
static void face_average(const double wl[5], const double wr[5], double Bn, eig* e) {
  double sl = sqrt(wl[0]), sr = sqrt(wr[0]);
  double den = sl + sr;
  e->rho = (sl * wl[0] + sr * wr[0]) / den;
  e->p = (sl * wl[1] + sr * wr[1]) / den;
  e->gam = (sl * wl[2] + sr * wr[2]) / den;
  e->Bt1 = (sl * wr[3] + sr * wl[3]) / den; /* crossed weights for B */
  e->Bt2 = (sl * wr[4] + sr * wl[4]) / den;
  e->Bn = Bn;
}

/* Characteristic Riemann solution at a face (Sec. 2.4): s_k = L_k q_k, where q_k is the vector
   of the six parabola averages over the domain of dependence of wave k (odd k: left cell, right
   end; even k: right cell, left end), then q* = R s.  tau_h = tau / h; edge != 0 takes the
   tau -> 0 limit (A11 flag). */
static void riemann_solve(const eig* e, const para pl[6], const para pr[6], double tau_h, int edge,
                          double qs[6]) {
  const double speed[6] = {e->cf, e->cf, e->cs, e->cs, e->ca, e->ca};
  double s[6];
  for (int k = 0; k < 6; ++k) {
    double y = edge ? 0.0 : speed[k] * tau_h;
    double acc = 0.0;
    for (int m = 0; m < 6; ++m) {
      double qb = (k % 2 == 0) ? avg_right_end(pl[m], y) : avg_left_end(pr[m], y);
      acc = acc + e->L[k][m] * qb;
    }
    s[k] = acc;
  }
  for (int m = 0; m < 6; ++m) {
    double acc = 0.0;
    for (int k = 0; k < 6; ++k) acc = acc + e->R[m][k] * s[k];
    qs[m] = acc;
  }
}

/* ---------------------------------------------------------------- Sec. 2.3 CFL */
static double cfl_denominator(double rho, double vx, double vy, double vz, double Bx, double By,
                              double Bz, double p, double gam) {
  double c2 = gam * p / rho;
  double b2 = (Bx * Bx + By * By + Bz * Bz) / rho;
  double v = sqrt(vx * vx + vy * vy + vz * vz);
  double b = sqrt(b2), c = sqrt(c2);
  const double Bd[3] = {Bx, By, Bz};
  double Dmax = 0.0;
  for (int d = 0; d < 3; ++d) {
    double ca2 = Bd[d] * Bd[d] / rho;
    double bp2r = (Bd[(d + 1) % 3] * Bd[(d + 1) % 3] + Bd[(d + 2) % 3] * Bd[(d + 2) % 3]) / rho;
    speeds sp = mhd_speeds(c2, ca2, bp2r);
    double cf = sqrt(sp.cf2), cs = sqrt(sp.cs2), ca = sqrt(ca2);
    double D = v + b + c + ca + cs + cf;
    if (D > Dmax) Dmax = D;
  }
  return Dmax;
}

/* ---------------------------------------------------------------- Sec. 2 closure + App. D gamma */
/* effective adiabatic index of the mixture (Sec. 4.3): gamma = (5 n_1 + 7 n_H2) / (3 n_1 + 5 n_H2)
   with n_1 the monatomic particles.  With H+ and electrons (A33) n_1 = n_H + n_H+ + n_e, where
   n_H = rho - rho_H2 - rho_H+ are the neutral atoms, n_H+ = n_e = rho_H+; without them
   (rho_H+ = 0) n_1 = n_H = rho - rho_H2. */
static double gamma_eff(double rho, double rh2, double rhp) {
  double n1 = (rho - rh2 - rhp) + 2.0 * rhp, nH2 = 0.5 * rh2;
  return (5.0 * n1 + 7.0 * nH2) / (3.0 * n1 + 5.0 * nH2);
}

static double cell_rhp(const osim* s, size_t c) { return s->ions ? s->rhp[c] : 0.0; }

static double cell_gamma(const osim* s, size_t c) {
  return s->chem ? gamma_eff(s->rho[c], s->rh2[c], cell_rhp(s, c)) : s->gamma;
}

/* temperature of the gas (K) from rho eps (code units) and the composition: p = (gamma - 1) rho eps
   P0 = (n_H + n_H2 + n_H+ + n_e) k_B T (A15 v, A33) */
static double temperature(double rho, double eint, double rh2, double rhp) {
  const double P0 = MH_CGS * KMS_CGS * KMS_CGS; /* code pressure unit, erg cm^-3 */
  double nH = rho - rh2 - rhp, nH2 = 0.5 * rh2, nHp = rhp, ne = rhp;
  double g = gamma_eff(rho, rh2, rhp);
  double p = (g - 1.0) * eint * P0;
  return p / ((((nH + nH2) + nHp) + ne) * KB_CGS);
}

/* ---------------------------------------------------------------- allocation */
static double* xalloc(size_t n) { return (double*)calloc(n, sizeof(double)); }

osim* osim_create(int nx, int ny, int nz, double gamma, double dx) {
  if (nx < 1 || ny < 1 || nz < 1 || !(gamma > 1.0) || !(dx > 0.0)) return NULL;
  osim* s = (osim*)calloc(1, sizeof(osim));
  if (!s) return NULL;
  s->n[0] = nx; s->n[1] = ny; s->n[2] = nz;
  for (int d = 0; d < 3; ++d) s->ne[d] = s->n[d] + 2 * NG;
  s->next = (size_t)s->ne[0] * s->ne[1] * s->ne[2];
  s->gamma = gamma;
  s->dx = dx;
  s->lshield = 0.0;
  s->bdop = 3.0;
  s->xnorm = 5e14;
  s->taud = 1e-21;
  s->threads = 1;
#ifdef _OPENMP
  s->threads = omp_get_max_threads();
#endif
  size_t n = s->next;
  double** all[] = {&s->rho, &s->m[0], &s->m[1], &s->m[2], &s->E, &s->eint, &s->rh2, &s->rhp,
                    &s->b[0], &s->b[1], &s->b[2], &s->rho0, &s->m0[0], &s->m0[1], &s->m0[2],
                    &s->E0, &s->eint0, &s->rh20, &s->rhp0, &s->b0[0], &s->b0[1], &s->b0[2]};
  for (size_t i = 0; i < sizeof(all) / sizeof(all[0]); ++i)
    if (!(*all[i] = xalloc(n))) goto fail;
  for (int i = 0; i < 9; ++i) if (!(s->w[i] = xalloc(n))) goto fail;
  for (int i = 0; i < 8; ++i) if (!(s->fo[i] = xalloc(n))) goto fail;
  for (int i = 0; i < 6; ++i) if (!(s->acc[i] = xalloc(n))) goto fail;
  for (int i = 0; i < 8; ++i) if (!(s->accL[i] = xalloc(n))) goto fail;
  for (int i = 0; i < 3; ++i)
    if (!(s->eA[i] = xalloc(n)) || !(s->eB[i] = xalloc(n)) || !(s->edge[i] = xalloc(n))) goto fail;
  if (!(s->phi = xalloc(n))) goto fail;
  return s;
fail:;
  extern void osim_destroy(osim*);
  osim_destroy(s);
  return NULL;
}

void osim_destroy(osim* s) {
  if (!s) return;
  double* all[] = {s->rho, s->m[0], s->m[1], s->m[2], s->E, s->eint, s->rh2, s->rhp, s->b[0],
                   s->b[1], s->b[2], s->rho0, s->m0[0], s->m0[1], s->m0[2], s->E0, s->eint0,
                   s->rh20, s->rhp0, s->b0[0], s->b0[1], s->b0[2]};
  for (size_t i = 0; i < sizeof(all) / sizeof(all[0]); ++i) free(all[i]);
  for (int i = 0; i < 9; ++i) free(s->w[i]);
  for (int i = 0; i < 8; ++i) free(s->fo[i]);
  for (int i = 0; i < 6; ++i) free(s->acc[i]);
  for (int i = 0; i < 8; ++i) free(s->accL[i]);
  for (int i = 0; i < 3; ++i) { free(s->eA[i]); free(s->eB[i]); free(s->edge[i]); }
  free(s->phi);
  free(s);
}

int osim_set_option(osim* s, int key, double v) {
  switch (key) {
    case O_BC_X: case O_BC_Y: case O_BC_Z:
      if (v != 0.0 && v != 1.0) return O_EINVAL;
      s->bc[key - O_BC_X] = (int)v;
      return O_OK;
    case O_CHEM: s->chem = v != 0.0; return O_OK;
    case O_STEP4_AS_WRITTEN: s->step4_as_written = v != 0.0; return O_OK;
    case O_IFACE_EDGE: s->iface_edge = v != 0.0; return O_OK;
    case O_REGUL_MODE:
      if (v != 0.0 && v != 1.0 && v != 2.0) return O_EINVAL;
      s->regul_mode = (int)v;
      return O_OK;
    case O_CHEM_LSHIELD: if (v < 0.0) return O_EINVAL; s->lshield = v; return O_OK;
    case O_CHEM_BDOP: if (!(v > 0.0)) return O_EINVAL; s->bdop = v; return O_OK;
    case O_CHEM_XNORM: if (!(v > 0.0)) return O_EINVAL; s->xnorm = v; return O_OK;
    case O_CHEM_TAUD: if (v < 0.0) return O_EINVAL; s->taud = v; return O_OK;
    case O_THREADS: if (v < 1.0) return O_EINVAL; s->threads = (int)v; return O_OK;
    case O_HEATCOOL: if (v != 0.0 && v != 1.0) return O_EINVAL; s->heatcool = (int)v; return O_OK;
    case O_GRAV_G: if (v < 0.0) return O_EINVAL; s->grav_g = v; return O_OK;
    case O_IONS: if (v != 0.0 && v != 1.0) return O_EINVAL; s->ions = (int)v; return O_OK;
    default: return O_EINVAL;
  }
}

/* cell-centred B from the faces (Sec. 2.5, last three equations); ghost faces must be valid */
static void cell_B(const osim* s, size_t c, double B[3]) {
  for (int d = 0; d < 3; ++d) B[d] = 0.5 * (s->b[d][c] + s->b[d][c + ST(s, d)]);
}

/* rho eps from the conserved energy (Sec. 2 closure) using the face-centred B */
static void derive_eint(osim* s) {
  const int nx = s->n[0], ny = s->n[1], nz = s->n[2];
  for (int d = 0; d < 3; ++d) fill_ghosts(s, s->b[d]);
#pragma omp parallel for schedule(static) num_threads(s->threads)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t c = IX(s, i + NG, j + NG, k + NG);
        double B[3];
        cell_B(s, c, B);
        double r = s->rho[c];
        double kin = 0.5 * (s->m[0][c] * s->m[0][c] + s->m[1][c] * s->m[1][c] + s->m[2][c] * s->m[2][c]) / r;
        double mag = 0.5 * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
        s->eint[c] = s->E[c] - kin - mag;
      }
}

/* state in: C-order [k][j][i] arrays of n cells; B cell-centred (A17 builds the faces) */
int osim_set_state(osim* s, const double* rho, const double* mx, const double* my,
                   const double* mz, const double* E, const double* Bx, const double* By,
                   const double* Bz, const double* rh2) {
  const int nx = s->n[0], ny = s->n[1], nz = s->n[2];
  const double* Bc[3] = {Bx, By, Bz};
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t src = ((size_t)k * ny + j) * nx + i;
        size_t c = IX(s, i + NG, j + NG, k + NG);
        s->rho[c] = rho[src];
        s->m[0][c] = mx[src];
        s->m[1][c] = my[src];
        s->m[2][c] = mz[src];
        s->E[c] = E[src];
        s->rh2[c] = rh2 ? rh2[src] : 0.0;
        s->rhp[c] = 0.0;
        const int ii[3] = {i, j, k};
        for (int d = 0; d < 3; ++d) {
          /* face d at index ii[d] sits between cells ii[d]-1 and ii[d] */
          int lo[3] = {i, j, k};
          lo[d] = map_index(ii[d] - 1, s->n[d], s->bc[d]);
          size_t srclo = ((size_t)lo[2] * ny + lo[1]) * nx + lo[0];
          s->b[d][c] = 0.5 * (Bc[d][srclo] + Bc[d][src]);
        }
      }
  derive_eint(s);
  s->t = 0.0;
  s->nsteps = 0;
  s->nvel_branch = 0;
  return O_OK;
}

/* exact face values (b_d at face i_d - 1/2), e.g. a divergence-free initial field */
int osim_set_face_B(osim* s, const double* bx, const double* by, const double* bz) {
  const int nx = s->n[0], ny = s->n[1], nz = s->n[2];
  const double* bf[3] = {bx, by, bz};
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t src = ((size_t)k * ny + j) * nx + i;
        size_t c = IX(s, i + NG, j + NG, k + NG);
        for (int d = 0; d < 3; ++d) s->b[d][c] = bf[d][src];
      }
  derive_eint(s);
  return O_OK;
}

/* set rho eps and the face fields directly (checkpoint / restart), float64 C order */
int osim_set_full(osim* s, const double* eint, const double* bx, const double* by, const double* bz) {
  const int nx = s->n[0], ny = s->n[1], nz = s->n[2];
  const double* bf[3] = {bx, by, bz};
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t src = ((size_t)k * ny + j) * nx + i;
        size_t c = IX(s, i + NG, j + NG, k + NG);
        s->eint[c] = eint[src];
        for (int d = 0; d < 3; ++d) s->b[d][c] = bf[d][src];
      }
  return O_OK;
}

int osim_get_state(osim* s, double* rho, double* mx, double* my, double* mz, double* E,
                   double* Bx, double* By, double* Bz, double* rh2) {
  const int nx = s->n[0], ny = s->n[1], nz = s->n[2];
  for (int d = 0; d < 3; ++d) fill_ghosts(s, s->b[d]);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t dst = ((size_t)k * ny + j) * nx + i;
        size_t c = IX(s, i + NG, j + NG, k + NG);
        double B[3];
        cell_B(s, c, B);
        rho[dst] = s->rho[c];
        mx[dst] = s->m[0][c];
        my[dst] = s->m[1][c];
        mz[dst] = s->m[2][c];
        E[dst] = s->E[c];
        Bx[dst] = B[0];
        By[dst] = B[1];
        Bz[dst] = B[2];
        if (rh2) rh2[dst] = s->rh2[c];
      }
  return O_OK;
}

/* rho eps and the face fields (b_d at face i_d - 1/2) */
int osim_get_full(osim* s, double* eint, double* bx, double* by, double* bz) {
  const int nx = s->n[0], ny = s->n[1], nz = s->n[2];
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t dst = ((size_t)k * ny + j) * nx + i;
        size_t c = IX(s, i + NG, j + NG, k + NG);
        eint[dst] = s->eint[c];
        bx[dst] = s->b[0][c];
        by[dst] = s->b[1][c];
        bz[dst] = s->b[2][c];
      }
  return O_OK;
}

/* rho_H+ (A32) of every cell, C order: set after set_state, which zeroes it */
int osim_set_ions(osim* s, const double* rhp) {
  const int nx = s->n[0], ny = s->n[1], nz = s->n[2];
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) s->rhp[IX(s, i + NG, j + NG, k + NG)] = rhp[((size_t)k * ny + j) * nx + i];
  return O_OK;
}

int osim_get_ions(osim* s, double* rhp) {
  const int nx = s->n[0], ny = s->n[1], nz = s->n[2];
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) rhp[((size_t)k * ny + j) * nx + i] = s->rhp[IX(s, i + NG, j + NG, k + NG)];
  return O_OK;
}

/* ---------------------------------------------------------------- primitives on the ext. grid */
/* primitives of the interior cells (needs valid ghost faces for the cell-centred B), then the
   ghost layers as zero-gradient / periodic copies of the cell-centred primitives (A16) */
static void compute_primitives(osim* s) {
  const int* n = s->n;
#pragma omp parallel for schedule(static) num_threads(s->threads)
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        size_t c = IX(s, i + NG, j + NG, k + NG);
        double r = s->rho[c];
        double B[3];
        cell_B(s, c, B);
        double g = cell_gamma(s, c);
        s->w[0][c] = r;
        s->w[1][c] = s->m[0][c] / r;
        s->w[2][c] = s->m[1][c] / r;
        s->w[3][c] = s->m[2][c] / r;
        s->w[4][c] = B[0];
        s->w[5][c] = B[1];
        s->w[6][c] = B[2];
        s->w[7][c] = (g - 1.0) * s->eint[c];
        s->w[8][c] = g;
      }
  for (int q = 0; q < 9; ++q) fill_ghosts(s, s->w[q]);
}

/* ---------------------------------------------------------------- Sec. 2.3 */
double osim_tau(osim* s, double cfl) {
  for (int f = 0; f < 3; ++f) fill_ghosts(s, s->b[f]);
  const int nx = s->n[0], ny = s->n[1], nz = s->n[2];
  double tau = INFINITY;
#pragma omp parallel for schedule(static) reduction(min : tau) num_threads(s->threads)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t c = IX(s, i + NG, j + NG, k + NG);
        double r = s->rho[c];
        double B[3];
        cell_B(s, c, B);
        double g = cell_gamma(s, c);
        double p = (g - 1.0) * s->eint[c];
        double D = cfl_denominator(r, s->m[0][c] / r, s->m[1][c] / r, s->m[2][c] / r, B[0], B[1],
                                   B[2], p, g);
        double tc = cfl * s->dx / D;
        if (tc < tau) tau = tc;
      }
  return tau;
}

/* ---------------------------------------------------------------- Sec. 2.4 / 2.5 right-hand side */
/* Eulerian R for m, rho E, rho eps (in acc[0..4]: flux sums before the 1/h factor) and the
   edge EMFs (edge[0..2]) for the current state. */
static void eulerian_rhs(osim* s, double tau_h) {
  const int* n = s->n;
  double* cells[] = {s->rho, s->m[0], s->m[1], s->m[2], s->eint, s->rh2, s->b[0], s->b[1], s->b[2]};
  for (size_t f = 0; f < sizeof(cells) / sizeof(cells[0]); ++f) fill_ghosts(s, cells[f]);
  compute_primitives(s);
  for (int a = 0; a < 5; ++a) memset(s->acc[a], 0, s->next * sizeof(double));

  for (int d = 0; d < 3; ++d) {
    const int d1 = (d + 1) % 3, d2 = (d + 2) % 3; /* cyclic frame (n, t1, t2) */
    const ptrdiff_t sd = ST(s, d);
    /* faces: normal index [0, n_d], transverse [-1, n_t] */
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = -1;
      hi[a] = n[a];
    }
    lo[d] = 0;
    hi[d] = n[d];
    const double* qv[6] = {s->w[1 + d], s->w[1 + d1], s->w[1 + d2], s->w[4 + d1], s->w[4 + d2], s->w[7]};
#pragma omp parallel for schedule(static) num_threads(s->threads)
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          size_t cr = IX(s, i + NG, j + NG, k + NG);
          size_t cl = cr - sd;
          para pl[6], pr[6];
          for (int v = 0; v < 6; ++v) {
            double ql[5], qr[5];
            for (int o = 0; o < 5; ++o) {
              ql[o] = qv[v][cl + (o - 2) * sd];
              qr[o] = qv[v][cr + (o - 2) * sd];
            }
            pl[v] = ppm_cell(ql, s->step4_as_written);
            pr[v] = ppm_cell(qr, s->step4_as_written);
          }
          double wl[5] = {s->w[0][cl], s->w[7][cl], s->w[8][cl], s->w[4 + d1][cl], s->w[4 + d2][cl]};
          double wr[5] = {s->w[0][cr], s->w[7][cr], s->w[8][cr], s->w[4 + d1][cr], s->w[4 + d2][cr]};
          eig e;
          face_average(wl, wr, s->b[d][cr], &e);
          build_eigen(&e);
          double qs[6];
          riemann_solve(&e, pl, pr, tau_h, s->iface_edge, qs);
          /* A12 fluxes from the face solution (V_n, V_t1, V_t2, B_t1, B_t2, P) */
          double Bn = e.Bn, Vn = qs[0], Vt1 = qs[1], Vt2 = qs[2], Bt1 = qs[3], Bt2 = qs[4], P = qs[5];
          double pstar = P + 0.5 * (Bn * Bn + Bt1 * Bt1 + Bt2 * Bt2);
          s->fo[0][cr] = pstar - Bn * Bn;
          s->fo[1][cr] = -(Bn * Bt1);
          s->fo[2][cr] = -(Bn * Bt2);
          s->fo[3][cr] = pstar * Vn - Bn * (Bn * Vn + Bt1 * Vt1 + Bt2 * Vt2);
          s->fo[4][cr] = Vn;
          /* E = B x U at the face (Sec. 2.5): component along t2 and along t1 */
          s->eA[d][cr] = Bn * Vt1 - Bt1 * Vn;
          s->eB[d][cr] = Bt2 * Vn - Bn * Vt2;
        }
    /* flux differences of interior cells, accumulated direction by direction */
    double* accm[3] = {s->acc[0], s->acc[1], s->acc[2]};
    double* tgt[5] = {accm[d], accm[d1], accm[d2], s->acc[3], s->acc[4]};
#pragma omp parallel for schedule(static) num_threads(s->threads)
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
          size_t c = IX(s, i + NG, j + NG, k + NG);
          for (int v = 0; v < 5; ++v) tgt[v][c] = tgt[v][c] + (s->fo[v][c] - s->fo[v][c + sd]);
        }
  }

  /* App. C edge EMFs: E_d at the corner (i_{d+1} - 1/2, i_{d+2} - 1/2) of cell index c, the mean
     of the contributions of the two faces of direction d+1 and the two of direction d+2 */
  for (int d = 0; d < 3; ++d) {
    const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
    const ptrdiff_t s1 = ST(s, d1), s2 = ST(s, d2);
#pragma omp parallel for schedule(static) num_threads(s->threads)
    for (int k = 0; k <= n[2]; ++k)
      for (int j = 0; j <= n[1]; ++j)
        for (int i = 0; i <= n[0]; ++i) {
          size_t c = IX(s, i + NG, j + NG, k + NG);
          double f1 = s->eA[d1][c - s2] + s->eA[d1][c];
          double f2 = s->eB[d2][c - s1] + s->eB[d2][c];
          s->edge[d][c] = 0.25 * (f1 + f2);
        }
  }
}

/* Eulerian SSP-RK3 substage combination: Q = a Q^n + b Q + g tau R (Sec. 2.2) */
static void eulerian_update(osim* s, double a, double bb, double g, double tau) {
  const int* n = s->n;
  const double ih = 1.0 / s->dx;
#pragma omp parallel for schedule(static) num_threads(s->threads)
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        size_t c = IX(s, i + NG, j + NG, k + NG);
        double g_cell = s->w[8][c];
        double R[5];
        for (int v = 0; v < 3; ++v) R[v] = s->acc[v][c] * ih;
        R[3] = s->acc[3][c] * ih;
        /* rho eps source -(gamma - 1) rho eps div V (A12); acc[4] * ih = -div V */
        R[4] = ((g_cell - 1.0) * s->eint[c]) * (s->acc[4][c] * ih);
        if (s->grav_g > 0.0) {
          /* Sec. 2.4: the gravity terms -rho grad Phi and -rho v . grad Phi by central differences
             of the potential of the step (A31) */
          for (int d = 0; d < 3; ++d) {
            double gd = -(s->phi[c + ST(s, d)] - s->phi[c - ST(s, d)]) * (0.5 * ih);
            R[d] = R[d] + s->rho[c] * gd;
            R[3] = R[3] + s->m[d][c] * gd;
          }
        }
        double* q[5] = {s->m[0], s->m[1], s->m[2], s->E, s->eint};
        double* q0[5] = {s->m0[0], s->m0[1], s->m0[2], s->E0, s->eint0};
        for (int v = 0; v < 5; ++v) q[v][c] = (a * q0[v][c] + bb * q[v][c]) + g * (tau * R[v]);
        /* Flux-CT (Sec. 2.5): d b_d / dt = -(curl E)_d on the face d of this cell */
        for (int d = 0; d < 3; ++d) {
          const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
          double curl = (s->edge[d1][c + ST(s, d2)] - s->edge[d1][c]) -
                        (s->edge[d2][c + ST(s, d1)] - s->edge[d2][c]);
          double Rb = curl * ih;
          s->b[d][c] = (a * s->b0[d][c] + bb * s->b[d][c]) + g * (tau * Rb);
        }
      }
}

/* ---------------------------------------------------------------- Sec. 2.6 Lagrangian stage */
/* advected conserved densities q in {rho, m_x, m_y, m_z, rho E, rho eps, rho_H2, rho_H+} */
static int lag_fields(osim* s, double** q, double** q0) {
  double* a[8] = {s->rho, s->m[0], s->m[1], s->m[2], s->E, s->eint, s->rh2, s->rhp};
  double* a0[8] = {s->rho0, s->m0[0], s->m0[1], s->m0[2], s->E0, s->eint0, s->rh20, s->rhp0};
  int nv = s->chem ? (s->ions ? 8 : 7) : 6;
  for (int v = 0; v < nv; ++v) {
    q[v] = a[v];
    q0[v] = a0[v];
  }
  return nv;
}

static void lagrangian_rhs(osim* s, double tau_h) {
  const int* n = s->n;
  double *q[8], *q0[8];
  const int nv = lag_fields(s, q, q0);
  for (int v = 0; v < nv; ++v) fill_ghosts(s, q[v]);
  for (int v = 0; v < nv; ++v) memset(s->accL[v], 0, s->next * sizeof(double));
  for (int d = 0; d < 3; ++d) {
    const ptrdiff_t sd = ST(s, d);
    int hi[3] = {n[0] - 1, n[1] - 1, n[2] - 1};
    hi[d] = n[d]; /* faces 0..n_d along d */
#pragma omp parallel for schedule(static) num_threads(s->threads)
    for (int k = 0; k <= hi[2]; ++k)
      for (int j = 0; j <= hi[1]; ++j)
        for (int i = 0; i <= hi[0]; ++i) {
          size_t cr = IX(s, i + NG, j + NG, k + NG);
          size_t cl = cr - sd;
          /* face velocity: sqrt(rho)-weighted mean of the two normal velocities (A13) */
          double vl = s->m[d][cl] / s->rho[cl], vr = s->m[d][cr] / s->rho[cr];
          double sl = sqrt(s->rho[cl]), sr = sqrt(s->rho[cr]);
          double vn = (vl * sl + vr * sr) / (sl + sr);
          double y = s->iface_edge ? 0.0 : fabs(vn) * tau_h;
          for (int v = 0; v < nv; ++v) {
            double st[5];
            double qb;
            if (vn >= 0.0) {
              for (int o = 0; o < 5; ++o) st[o] = q[v][cl + (o - 2) * sd];
              qb = avg_right_end(ppm_cell(st, s->step4_as_written), y);
            } else {
              for (int o = 0; o < 5; ++o) st[o] = q[v][cr + (o - 2) * sd];
              qb = avg_left_end(ppm_cell(st, s->step4_as_written), y);
            }
            s->fo[v][cr] = vn * qb;
          }
        }
#pragma omp parallel for schedule(static) num_threads(s->threads)
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
          size_t c = IX(s, i + NG, j + NG, k + NG);
          for (int v = 0; v < nv; ++v) s->accL[v][c] = s->accL[v][c] + (s->fo[v][c] - s->fo[v][c + sd]);
        }
  }
}

static void lagrangian_update(osim* s, double a, double bb, double g, double tau) {
  const int* n = s->n;
  const double ih = 1.0 / s->dx;
  double *q[8], *q0[8];
  const int nv = lag_fields(s, q, q0);
#pragma omp parallel for schedule(static) num_threads(s->threads)
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        size_t c = IX(s, i + NG, j + NG, k + NG);
        for (int v = 0; v < nv; ++v) {
          double R = s->accL[v][c] * ih;
          q[v][c] = (a * q0[v][c] + bb * q[v][c]) + g * (tau * R);
        }
      }
}

/* ---------------------------------------------------------------- Sec. 2.7 + App. D chemistry */
typedef struct { double T, k1p, k2, k3, k4, C, D; } chem_rates;

/* App. D rates of reactions 1-4 at temperature T (K) for number densities (cm^-3); A15 readings:
   C = k1' n n_H (k1 carries the factor n/n_H), column densities N_X = n_X L_shield. */
static chem_rates chem_rates_at(const osim* s, double T, double nH, double nH2, double n) {
  chem_rates r;
  r.T = T;
  double t2 = T / 100.0;
  double s2 = sqrt(t2);
  r.k1p = 3e-17 * s2 / (((1.0 + 0.4 * s2) + 0.2 * t2) + 0.08 * (t2 * t2));
  if (T > 7390.0)
    r.k2 = 6.11e-14 * exp(-2.93e4 / T);
  else
    r.k2 = 2.67e-15 * exp(-((6750.0 / T) * (6750.0 / T)));
  if (T > 7291.0)
    r.k3 = 5.22e-14 * exp(-3.22e4 / T);
  else
    r.k3 = 3.17e-15 * exp(-(4060.0 / T) - (7500.0 / T) * (7500.0 / T));
  double Ls = (s->lshield > 0.0 ? s->lshield : s->dx) * PC_CGS;
  double NH = nH * Ls, NH2 = nH2 * Ls;
  double fdust = exp(-(s->taud * (NH + NH2)));
  double x = NH2 / s->xnorm;
  double u = 1.0 + x / s->bdop;
  double sx = sqrt(1.0 + x);
  double fsh = 0.965 / (u * u) + 0.035 / sx * exp(-8.5e-4 * sx);
  r.k4 = (3.3 * 1.7e-11) * fsh * fdust;
  r.C = r.k1p * n * nH;
  r.D = (r.k2 * nH + r.k3 * nH2) + r.k4;
  return r;
}

/* App. D rates of reactions 5-8 (H+ and e) at temperature T (K), readings A34-A37:
   k5 = 6e-18 s^-1 per H atom (cosmic-ray ionisation; the printed density factor read as a stray,
        as Gamma_5 = 1.92e-28 n = k5 x 20 eV x n shows);
   k6 = exp(sum_j c_j (ln T_eV)^j), j = 0..8, the collisional ionisation fit in the natural logarithm
        of the temperature in eV;
   k7 = 10^(P(x) / Q(x)), x = log10 T, the printed quartics;
   k8 = the printed grain-recombination fit, log = log10, "a(-b)" = a 10^-b;
   creation and destruction of H+ per unit volume: C = k5 n_H + k6 n_H n_e, D n_H+ with
   D = k7 n_e + k8 n (A38). */
typedef struct { double k5, k6, k7, k8, C, D; } ion_rates;

static ion_rates ion_rates_at(double T, double nH, double ne, double n) {
  static const double c6[9] = {-32.7, 13.5, -5.7, 1.5, -0.3, 3.4e-2, -2.6e-3, 1.1e-4, -2.1e-6};
  ion_rates r;
  r.k5 = 6e-18;
  double L = log(T * KB_EV), acc = 0.0, Lj = 1.0;
  for (int j = 0; j < 9; ++j) {
    acc += c6[j] * Lj;
    Lj *= L;
  }
  r.k6 = exp(acc);
  double x = log10(T);
  double P = -10.78 + 4.68 * x - 0.87 * x * x + 0.08 * x * x * x - 3.87e-3 * x * x * x * x;
  double Q = 1.0 - 0.38 * x + 0.06 * x * x - 5.1e-3 * x * x * x + 2.4e-4 * x * x * x * x;
  r.k7 = pow(10.0, P / Q);
  r.k8 = 12.25e-14 / (1.0 + 8.074e-6 * pow(10.0, 2.756) *
                                (1.0 + 5.087e2 * pow(T, 1.586e-2) * pow(10.0, -1.8892 - 4.4e-5 * log10(T))));
  r.C = r.k5 * nH + r.k6 * nH * ne;
  r.D = r.k7 * ne + r.k8 * n;
  return r;
}

/* one cell (Sec. 2.7): returns the new rho_H2 and, with the ions on, stores the new rho_H+ in
   *rhp_new.  The rates are evaluated once from the state at stage start (A15, A38); each species
   takes the printed semi-implicit update n' = n + tau (C - D n) / (1 + tau D): H2 first, then H+ from
   the stage-start n_H and n_e; n_H = n - 2 n_H2 - n_H+ and n_e = n_H+ close the composition. */
static double chem_cell(const osim* s, double rho, double eint, double rh2, double rhp, double tau,
                        chem_rates* out, ion_rates* iout, double* rhp_new) {
  const double T0 = PC_CGS / KMS_CGS; /* code time unit, s */
  double nH = rho - rh2 - rhp, nH2 = 0.5 * rh2, n = rho;
  double T = temperature(rho, eint, rh2, rhp);
  chem_rates r = chem_rates_at(s, T, nH, nH2, n);
  double ts = tau * T0;
  double nH2n = nH2 + ts * (r.C - r.D * nH2) / (1.0 + ts * r.D);
  if (nH2n < 0.0) nH2n = 0.0;
  if (nH2n > 0.5 * n) nH2n = 0.5 * n;
  if (out) *out = r;
  if (s->ions) {
    double nHp = rhp, ne = rhp;
    ion_rates q = ion_rates_at(T, nH, ne, n);
    double nHpn = nHp + ts * (q.C - q.D * nHp) / (1.0 + ts * q.D);
    if (nHpn < 0.0) nHpn = 0.0;
    if (nHpn > n - 2.0 * nH2n) nHpn = n - 2.0 * nH2n;
    if (iout) *iout = q;
    if (rhp_new) *rhp_new = nHpn;
  } else if (rhp_new) {
    *rhp_new = rhp;
  }
  return 2.0 * nH2n;
}

static void chemistry(osim* s, double tau) {
  const int* n = s->n;
#pragma omp parallel for schedule(static) num_threads(s->threads)
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        size_t c = IX(s, i + NG, j + NG, k + NG);
        double rhp = cell_rhp(s, c);
        s->rh2[c] = chem_cell(s, s->rho[c], s->eint[c], s->rh2[c], rhp, tau, NULL, NULL, &rhp);
        if (s->ions) s->rhp[c] = rhp;
      }
}

/* ---------------------------------------------------------------- Sec. 2.8 + App. D heating/cooling */
/* Heating and cooling of the H/H2 gas, erg cm^-3 s^-1, at the state (rho, rho eps, rho_H2) in code
   units (readings A24-A29):
   - T from the composition as in the chemistry (n_H = rho - rho_H2, n_H2 = rho_H2 / 2, n = rho);
   - Gamma_1 = 7.2e-12 erg x (k1' n n_H) / (1 + n_cr / n), n_cr = 10^(4 - 0.416 x - 0.327 x^2): the
     H2 formation heating, the printed numerator read as the formation rate of reaction 1 and the
     printed polynomial over n as the critical density (A25);
   - Lambda_2 = n_H2 L_H / (1 + L_H / L_L) with the two-branch L_H and L_L as printed (A26);
   - Lambda_3 = n_H2 L_H / (1 + L_H / L_L), L_H = 1.1e-13 exp(-6744 / T),
     L_L = 8.18e-13 (n_H k_H + n_H2 k_H2), k_H2 = 6.29e-15 x 1.38 f(T) / f(4500),
     f(T) = sqrt(T) a exp(a), a = 1 + 1 / (k_B T) with k_B in eV/K, and k_H = k_H2 (A27);
   - Gamma_4 = 6.4e-13 erg x k4 n_H2 (A28);
   with the ions on (A39), also
   - Gamma_5 = 1.92e-28 n (cosmic-ray heating, as printed);
   - Lambda_6 = 2.18e-11 erg x k6 n_H n_e (13.6 eV per collisional ionisation);
   - Lambda_7 = 4.65e-30 T^0.94 psi^(0.74 / T^0.068) n_e n_H+, psi = exp(-0.75e-20 (N_H + N_H2))
     sqrt(T) / n_e (the printed sqrt(t) read as sqrt(T)), 0 where n_e = 0;
   - Lambda_8 = 5.7e-26 (T / 1e4)^0.8 n_e n_H+;
   x = log10(T / 1e4) throughout (A15 iv); n_H the neutral atoms. */
typedef struct { double T, G1, L2, L3, G4, G5, L6, L7, L8, net; } heatcool_terms;

static double log_f_A27(double T) {
  double a = 1.0 + 1.0 / (KB_EV * T);
  return 0.5 * log(T) + log(a) + a;
}

static heatcool_terms heatcool_at(const osim* s, double rho, double eint, double rh2, double rhp) {
  double nH = rho - rh2 - rhp, nH2 = 0.5 * rh2, n = rho;
  double T = temperature(rho, eint, rh2, rhp);
  chem_rates r = chem_rates_at(s, T, nH, nH2, n);
  double x = log10(T / 1e4);
  heatcool_terms h;
  h.T = T;
  /* Gamma_1 (A25) */
  double ncr = pow(10.0, 4.0 - 0.416 * x - 0.327 * x * x);
  h.G1 = 7.2e-12 * r.C / (1.0 + ncr / n);
  /* Lambda_2 (A26) */
  double LH2 = T > 1087.0 ? 3.9e-19 * exp(-6118.0 / T) : pow(10.0, -19.24 + 0.474 * x - 1.247 * x * x);
  double LL2 = (pow(nH2, 0.77) + 1.2 * pow(nH, 0.77)) *
               (T > 4031.0 ? 1.38e-22 * exp(-9243.0 / T) : pow(10.0, -22.9 - 0.553 * x - 1.148 * x * x));
  h.L2 = nH2 * LH2 / (1.0 + LH2 / LL2);
  /* Lambda_3 (A27) */
  double LH3 = 1.1e-13 * exp(-6744.0 / T);
  double kH2 = 6.29e-15 * 1.38 * exp(log_f_A27(T) - log_f_A27(4500.0));
  double LL3 = 8.18e-13 * (nH * kH2 + nH2 * kH2);
  h.L3 = nH2 * LH3 / (1.0 + LH3 / LL3);
  /* Gamma_4 (A28) */
  h.G4 = 6.4e-13 * r.k4 * nH2;
  h.G5 = h.L6 = h.L7 = h.L8 = 0.0;
  if (s->ions) {
    double nHp = rhp, ne = rhp;
    ion_rates q = ion_rates_at(T, nH, ne, n);
    h.G5 = 1.92e-28 * n;
    h.L6 = 2.18e-11 * q.k6 * nH * ne;
    if (ne > 0.0) {
      double Ls = (s->lshield > 0.0 ? s->lshield : s->dx) * PC_CGS;
      double psi = exp(-0.75e-20 * (nH * Ls + nH2 * Ls)) * sqrt(T) / ne;
      h.L7 = 4.65e-30 * pow(T, 0.94) * pow(psi, 0.74 / pow(T, 0.068)) * ne * nHp;
    }
    h.L8 = 5.7e-26 * pow(T / 1e4, 0.8) * ne * nHp;
  }
  h.net = (h.G1 + h.G4 + h.G5) - (h.L2 + h.L3 + h.L6 + h.L7 + h.L8);
  return h;
}

/* Sec. 2.8: d(rho E)/dt = d(rho eps)/dt = Gamma - Lambda by one Euler step; returns the change of
   rho E and rho eps in code units, limited so that rho eps keeps at least half its value (A29) */
static double heatcool_delta(const osim* s, double rho, double eint, double rh2, double rhp,
                             double tau, heatcool_terms* out) {
  const double P0 = MH_CGS * KMS_CGS * KMS_CGS; /* code energy density unit, erg cm^-3 */
  const double T0 = PC_CGS / KMS_CGS;           /* code time unit, s */
  heatcool_terms h = heatcool_at(s, rho, eint, rh2, rhp);
  double d = tau * T0 * h.net / P0;
  if (d < -0.5 * eint) d = -0.5 * eint;
  if (out) *out = h;
  return d;
}

static void heatcool(osim* s, double tau) {
  const int* n = s->n;
#pragma omp parallel for schedule(static) num_threads(s->threads)
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        size_t c = IX(s, i + NG, j + NG, k + NG);
        double d = heatcool_delta(s, s->rho[c], s->eint[c], s->rh2[c], cell_rhp(s, c), tau, NULL);
        s->E[c] = s->E[c] + d;
        s->eint[c] = s->eint[c] + d;
      }
}

/* ---------------------------------------------------------------- Sec. 2.9 regularisation */
static long regularise(osim* s) {
  const int* n = s->n;
  for (int d = 0; d < 3; ++d) fill_ghosts(s, s->b[d]);
  long count = 0;
#pragma omp parallel for schedule(static) reduction(+ : count) num_threads(s->threads)
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        size_t c = IX(s, i + NG, j + NG, k + NG);
        double B[3];
        cell_B(s, c, B);
        double r = s->rho[c];
        double m2 = s->m[0][c] * s->m[0][c] + s->m[1][c] * s->m[1][c] + s->m[2][c] * s->m[2][c];
        double kin = 0.5 * m2 / r;
        double mag = 0.5 * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
        double e = s->E[c] - kin - mag;
        double f = e / s->E[c];
        int entropy_branch = f >= 1e-3;
        if (s->regul_mode == 2) entropy_branch = !entropy_branch; /* the sentence's literal order */
        if (entropy_branch) {
          /* the correction "guarantees non-decreasing of entropy": at fixed rho it may only raise
             rho eps (mode 0); mode 1 overwrites unconditionally */
          if (s->regul_mode != 0 || e > s->eint[c]) s->eint[c] = e;
        } else {
          double v2 = 2.0 * (s->E[c] - s->eint[c] - mag) / r;
          if (v2 < 0.0) v2 = 0.0;
          double vnew = sqrt(v2);
          double vold = sqrt(m2) / r;
          if (vold > 0.0) {
            double sc = vnew / vold;
            for (int d = 0; d < 3; ++d) s->m[d][c] = s->m[d][c] * sc;
          }
          count += 1;
        }
      }
  return count;
}

/* ---------------------------------------------------------------- the step */
static void save_Qn(osim* s, int lagrangian) {
  size_t bytes = s->next * sizeof(double);
  for (int d = 0; d < 3; ++d) memcpy(s->m0[d], s->m[d], bytes);
  memcpy(s->E0, s->E, bytes);
  memcpy(s->eint0, s->eint, bytes);
  if (lagrangian) {
    memcpy(s->rho0, s->rho, bytes);
    memcpy(s->rh20, s->rh2, bytes);
    memcpy(s->rhp0, s->rhp, bytes);
  } else {
    for (int d = 0; d < 3; ++d) memcpy(s->b0[d], s->b[d], bytes);
  }
}

static const double RK_A[3] = {0.0, 0.75, 1.0 / 3.0};
static const double RK_B[3] = {1.0, 0.25, 2.0 / 3.0};
static const double RK_G[3] = {1.0, 0.25, 2.0 / 3.0};

/* Eulerian stage with Flux-CT inside each RK substage (A10) */
/* ---------------------------------------------------------------- Sec. 2.10 Poisson equation */
/* One-dimensional discrete Fourier transform along axis d of the complex field (re, im) on the
   interior grid (x fastest): X_k = sum_j x_j exp(sign 2 pi i j k / N), plain O(N^2) sums with the
   phase of (j k mod N) from a table. */
static void dft_axis(const osim* s, double* re, double* im, int d, int sign) {
  const int nx = s->n[0], ny = s->n[1], nz = s->n[2];
  const int N = s->n[d];
  const size_t stride = d == 0 ? 1 : (d == 1 ? (size_t)nx : (size_t)nx * ny);
  const int lines = nx * ny * nz / N;
  double* cs = (double*)malloc(sizeof(double) * N);
  double* sn = (double*)malloc(sizeof(double) * N);
  for (int m = 0; m < N; ++m) {
    cs[m] = cos(2.0 * M_PI * m / N);
    sn[m] = sign * sin(2.0 * M_PI * m / N);
  }
#pragma omp parallel for schedule(static) num_threads(s->threads)
  for (int l = 0; l < lines; ++l) {
    /* first element of line l: the other two indices enumerate the lines */
    size_t base;
    if (d == 0) base = (size_t)l * nx;
    else if (d == 1) base = (size_t)(l / nx) * nx * ny + (size_t)(l % nx);
    else base = (size_t)l;
    double* xr = (double*)malloc(sizeof(double) * N);
    double* xi = (double*)malloc(sizeof(double) * N);
    for (int j = 0; j < N; ++j) {
      xr[j] = re[base + j * stride];
      xi[j] = im[base + j * stride];
    }
    for (int k = 0; k < N; ++k) {
      double sr = 0.0, si = 0.0;
      for (int j = 0; j < N; ++j) {
        int m = (int)(((long)j * k) % N);
        sr += xr[j] * cs[m] - xi[j] * sn[m];
        si += xr[j] * sn[m] + xi[j] * cs[m];
      }
      re[base + k * stride] = sr;
      im[base + k * stride] = si;
    }
    free(xr);
    free(xi);
  }
  free(cs);
  free(sn);
}

/* Sec. 2.10: the potential of the 27-point scheme in harmonic space,
   Phi_jmn = -(2/3) pi G h^2 rho_jmn / (1 - c_j c_m c_n), c_j = (3 - 2 sin^2(pi j / N)) / 3, the mean
   (j = m = n = 0) mode zero (A30); the potential of the periodic box. */
static void poisson(osim* s) {
  const int nx = s->n[0], ny = s->n[1], nz = s->n[2];
  const size_t N = (size_t)nx * ny * nz;
  double* re = (double*)malloc(sizeof(double) * N);
  double* im = (double*)calloc(N, sizeof(double));
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) re[((size_t)k * ny + j) * nx + i] = s->rho[IX(s, i + NG, j + NG, k + NG)];
  for (int d = 0; d < 3; ++d) dft_axis(s, re, im, d, -1);
  const double h = s->dx;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t c = ((size_t)k * ny + j) * nx + i;
        if (i == 0 && j == 0 && k == 0) {
          re[c] = 0.0;
          im[c] = 0.0;
          continue;
        }
        double si = sin(M_PI * i / nx), sj = sin(M_PI * j / ny), sk = sin(M_PI * k / nz);
        double cx = (3.0 - 2.0 * si * si) / 3.0, cy = (3.0 - 2.0 * sj * sj) / 3.0, cz = (3.0 - 2.0 * sk * sk) / 3.0;
        double f = -(2.0 / 3.0) * M_PI * s->grav_g * h * h / (1.0 - cx * cy * cz);
        re[c] *= f;
        im[c] *= f;
      }
  for (int d = 0; d < 3; ++d) dft_axis(s, re, im, d, +1);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) s->phi[IX(s, i + NG, j + NG, k + NG)] = re[((size_t)k * ny + j) * nx + i] / (double)N;
  fill_ghosts(s, s->phi);
  free(re);
  free(im);
}

static void eulerian_stage(osim* s, double tau) {
  const double tau_h = tau / s->dx;
  save_Qn(s, 0);
  for (int r = 0; r < 3; ++r) {
    eulerian_rhs(s, tau_h);
    eulerian_update(s, RK_A[r], RK_B[r], RK_G[r], tau);
  }
}

static void lagrangian_stage(osim* s, double tau) {
  const double tau_h = tau / s->dx;
  save_Qn(s, 1);
  for (int r = 0; r < 3; ++r) {
    lagrangian_rhs(s, tau_h);
    lagrangian_update(s, RK_A[r], RK_B[r], RK_G[r], tau);
  }
}

static int check_physical(osim* s) {
  const int* n = s->n;
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad) num_threads(s->threads)
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        size_t c = IX(s, i + NG, j + NG, k + NG);
        double v[] = {s->rho[c], s->m[0][c], s->m[1][c], s->m[2][c], s->E[c], s->eint[c], s->rh2[c],
                      s->rhp[c], s->b[0][c], s->b[1][c], s->b[2][c]};
        for (size_t q = 0; q < sizeof(v) / sizeof(v[0]); ++q)
          if (!isfinite(v[q])) bad = 1;
        if (!(s->rho[c] > 0.0) || !(s->eint[c] > 0.0)) bad = 1;
      }
  return bad ? O_ENONPHYS : O_OK;
}

/* run one stage alone (debugging and per-stage parity): 1 Eulerian, 2 Lagrangian,
   3 chemistry, 4 regularisation, 5 heating/cooling */
int osim_stage(osim* s, int which, double tau) {
  switch (which) {
    case 1:
      if (s->grav_g > 0.0) poisson(s);
      eulerian_stage(s, tau);
      break;
    case 2: lagrangian_stage(s, tau); break;
    case 3: if (s->chem) chemistry(s, tau); break;
    case 4: s->nvel_branch += regularise(s); break;
    case 5: if (s->chem && s->heatcool) heatcool(s, tau); break;
    default: return O_EINVAL;
  }
  return check_physical(s);
}

/* one full step (Sec. 2 stage order, stages 1-6 without gravity; stage 5 only with the option on);
   t_end > 0 truncates tau (A18) */
int osim_step(osim* s, double cfl, double t_end, double* dt) {
  double tau = osim_tau(s, cfl);
  if (t_end > 0.0 && tau > t_end - s->t) tau = t_end - s->t;
  if (!(tau > 0.0)) return O_EINVAL;
  if (s->grav_g > 0.0) {
    if (s->bc[0] || s->bc[1] || s->bc[2]) return O_EINVAL; /* self-gravity of a periodic box */
    poisson(s); /* stage 7 of the previous step: the potential of rho^n (A31) */
  }
  eulerian_stage(s, tau);
  lagrangian_stage(s, tau);
  if (s->chem) chemistry(s, tau);
  if (s->chem && s->heatcool) heatcool(s, tau);
  s->nvel_branch += regularise(s);
  s->t += tau;
  s->nsteps += 1;
  if (dt) *dt = tau;
  return check_physical(s);
}

/* steps until t_end (or max_steps); returns the status of the last step */
int osim_advance(osim* s, double cfl, double t_end, int max_steps, int* steps_done) {
  int k = 0, rc = O_OK;
  while (k < max_steps && s->t < t_end) {
    rc = osim_step(s, cfl, t_end, NULL);
    ++k;
    if (rc != O_OK) break;
  }
  if (steps_done) *steps_done = k;
  return rc;
}

double osim_time(const osim* s) { return s->t; }
long osim_nsteps(const osim* s) { return s->nsteps; }

/* FP64 diagnostics: sums of rho, m_x, m_y, m_z, rho E, b_x, b_y, b_z, max |div b| * h, count of
   velocity-branch regularisations */
void osim_diag(osim* s, double out[10]) {
  const int* n = s->n;
  for (int d = 0; d < 3; ++d) fill_ghosts(s, s->b[d]);
  double sums[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  double dmax = 0.0;
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        size_t c = IX(s, i + NG, j + NG, k + NG);
        sums[0] += s->rho[c];
        sums[1] += s->m[0][c];
        sums[2] += s->m[1][c];
        sums[3] += s->m[2][c];
        sums[4] += s->E[c];
        sums[5] += s->b[0][c];
        sums[6] += s->b[1][c];
        sums[7] += s->b[2][c];
        double div = (s->b[0][c + ST(s, 0)] - s->b[0][c]) + (s->b[1][c + ST(s, 1)] - s->b[1][c]) +
                     (s->b[2][c + ST(s, 2)] - s->b[2][c]);
        if (fabs(div) > dmax) dmax = fabs(div);
      }
  for (int q = 0; q < 8; ++q) out[q] = sums[q];
  out[8] = dmax;
  out[9] = (double)s->nvel_branch;
}

/* ---------------------------------------------------------------- unit-level entry points */
/* PPM of one cell: q[0..4] = q_{i-2}..q_{i+2} -> out = (q^L, q^R, Delta q, q^(6)) */
void o_ppm(const double q[5], int step4_as_written, double out[4]) {
  para P = ppm_cell(q, step4_as_written);
  out[0] = P.L;
  out[1] = P.R;
  out[2] = P.d;
  out[3] = P.q6;
}

/* Step 4 detector of one cell: q[0..4] = q_{i-2}..q_{i+2} -> out = (eta, hbar) */
void o_step4(const double q[5], double out[2]) {
  double eta = 0.0;
  out[1] = step4_weight(q, &eta);
  out[0] = eta;
}

/* domain-of-dependence average of a parabola P = (q^L, q^R, Delta q, q^(6)) over the fraction y
   at the right end (right_end != 0) or the left end */
double o_avg(const double P[4], double y, int right_end) {
  para p = {P[0], P[1], P[2], P[3]};
  return right_end ? avg_right_end(p, y) : avg_left_end(p, y);
}

/* eigensystem for the face state st = (rho, p, gamma, B_n, B_t1, B_t2); R row-major [m][k],
   L row-major [k][m]; info = (c, c_f, c_s, c_a, alpha_f, alpha_s, beta_y, beta_z, sign) */
void o_eigen(const double st[6], double R[36], double L[36], double lam[6], double info[9]) {
  eig e;
  e.rho = st[0]; e.p = st[1]; e.gam = st[2]; e.Bn = st[3]; e.Bt1 = st[4]; e.Bt2 = st[5];
  build_eigen(&e);
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) {
      R[a * 6 + b] = e.R[a][b];
      L[a * 6 + b] = e.L[a][b];
    }
  for (int k = 0; k < 6; ++k) lam[k] = e.lam[k];
  double in[9] = {e.c, e.cf, e.cs, e.ca, e.af, e.as, e.by, e.bz, e.sg};
  for (int k = 0; k < 9; ++k) info[k] = in[k];
}

/* face Riemann solution from cell states and stencils:
   wl, wr = (rho, p, gamma, B_t1, B_t2) of the two cells; Bn the face field;
   sl, sr = 6 x 5 stencils (variable-major) of (v_n, v_t1, v_t2, B_t1, B_t2, p) around each cell;
   out = (V_n, V_t1, V_t2, B_t1, B_t2, P) */
void o_face_solve(const double wl[5], const double wr[5], double Bn, const double sl[30],
                  const double sr[30], double tau_h, int edge, int step4_as_written, double out[6]) {
  para pl[6], pr[6];
  for (int v = 0; v < 6; ++v) {
    pl[v] = ppm_cell(sl + 5 * v, step4_as_written);
    pr[v] = ppm_cell(sr + 5 * v, step4_as_written);
  }
  eig e;
  face_average(wl, wr, Bn, &e);
  build_eigen(&e);
  riemann_solve(&e, pl, pr, tau_h, edge, out);
}

double o_cfl_denominator(const double w[9]) {
  return cfl_denominator(w[0], w[1], w[2], w[3], w[4], w[5], w[6], w[7], w[8]);
}

double o_gamma_eff(double rho, double rh2) { return gamma_eff(rho, rh2, 0.0); }
double o_gamma_eff_ions(double rho, double rh2, double rhp) { return gamma_eff(rho, rh2, rhp); }
double o_temperature(double rho, double eint, double rh2, double rhp) {
  return temperature(rho, eint, rh2, rhp);
}

/* chemistry of one cell with the simulation's parameters:
   out = (rho_H2 new, T, k1', k2, k3, k4, C, D) */
void osim_chem_cell(const osim* s, double rho, double eint, double rh2, double tau, double out[8]) {
  chem_rates r;
  out[0] = chem_cell(s, rho, eint, rh2, 0.0, tau, &r, NULL, NULL);
  out[1] = r.T;
  out[2] = r.k1p;
  out[3] = r.k2;
  out[4] = r.k3;
  out[5] = r.k4;
  out[6] = r.C;
  out[7] = r.D;
}

/* the gravitational potential of the current density (Sec. 2.10), interior cells, x fastest */
int osim_potential(osim* s, double* out) {
  if (!(s->grav_g > 0.0)) return O_EINVAL;
  poisson(s);
  for (int k = 0; k < s->n[2]; ++k)
    for (int j = 0; j < s->n[1]; ++j)
      for (int i = 0; i < s->n[0]; ++i)
        out[((size_t)k * s->n[1] + j) * s->n[0] + i] = s->phi[IX(s, i + NG, j + NG, k + NG)];
  return O_OK;
}

/* heating/cooling of one cell with the simulation's parameters:
   out = (change of rho E and rho eps in code units, T, Gamma_1, Lambda_2, Lambda_3, Gamma_4, net) */
void osim_heatcool_cell(const osim* s, double rho, double eint, double rh2, double tau, double out[7]) {
  heatcool_terms h;
  out[0] = heatcool_delta(s, rho, eint, rh2, 0.0, tau, &h);
  out[1] = h.T;
  out[2] = h.G1;
  out[3] = h.L2;
  out[4] = h.L3;
  out[5] = h.G4;
  out[6] = h.net;
}

/* App. D rates at a given temperature and composition (for the rate pins) */
void osim_chem_rates(const osim* s, double T, double nH, double nH2, double out[7]) {
  chem_rates r = chem_rates_at(s, T, nH, nH2, nH + 2.0 * nH2);
  double v[7] = {r.k1p, r.k2, r.k3, r.k4, r.C, r.D, r.T};
  for (int k = 0; k < 7; ++k) out[k] = v[k];
}

/* chemistry of one cell with H+ (the sim's ion option decides whether reactions 5-8 run):
   out = (rho_H2 new, rho_H+ new, T, k1', k2, k3, k4, C, D, k5, k6, k7, k8, C_H+, D_H+) */
void osim_chem_cell_ions(const osim* s, double rho, double eint, double rh2, double rhp, double tau,
                         double out[15]) {
  chem_rates r;
  ion_rates q = {0, 0, 0, 0, 0, 0};
  double rhpn = rhp;
  out[0] = chem_cell(s, rho, eint, rh2, rhp, tau, &r, &q, &rhpn);
  double v[14] = {rhpn, r.T, r.k1p, r.k2, r.k3, r.k4, r.C, r.D, q.k5, q.k6, q.k7, q.k8, q.C, q.D};
  for (int k = 0; k < 14; ++k) out[k + 1] = v[k];
}

/* App. D rates of reactions 5-8 at a given temperature and composition: out = (k5, k6, k7, k8, C, D) */
void o_ion_rates(double T, double nH, double ne, double n, double out[6]) {
  ion_rates q = ion_rates_at(T, nH, ne, n);
  double v[6] = {q.k5, q.k6, q.k7, q.k8, q.C, q.D};
  for (int k = 0; k < 6; ++k) out[k] = v[k];
}

/* heating/cooling of one cell with H+: out = (change of rho E and rho eps in code units, T, Gamma_1,
   Lambda_2, Lambda_3, Gamma_4, Gamma_5, Lambda_6, Lambda_7, Lambda_8, net) */
void osim_heatcool_cell_ions(const osim* s, double rho, double eint, double rh2, double rhp,
                             double tau, double out[11]) {
  heatcool_terms h;
  out[0] = heatcool_delta(s, rho, eint, rh2, rhp, tau, &h);
  double v[10] = {h.T, h.G1, h.L2, h.L3, h.G4, h.G5, h.L6, h.L7, h.L8, h.net};
  for (int k = 0; k < 10; ++k) out[k + 1] = v[k];
}
