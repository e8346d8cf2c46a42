/*
 * Oracle for the quasi-conservative two-phase finite-volume scheme of
 * Wang, Xiang, Zhang & Hu, "An incremental-stencil WENO reconstruction for
 * simulation of compressible two-phase flows" (arXiv 1707.00592).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, FP64 CPU restatement of
 * the method, written from the paper, that the CUDA path is checked against.
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * load it.  It shares no code with the CUDA library and never calls it.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp (no fast-math), so every
 * operation is one IEEE-754 binary64 operation in the order written here.
 *
 * Steps, in the paper's order (section / equation of the paper):
 *   Sec. 2, Eqs. (governing-equation), (eos), (material-equation),
 *           (material-properties): state U = (rho, rho u_i, E, Gamma, Pi),
 *           rho e = Gamma p + Pi with Gamma = 1/(gamma-1), Pi = gamma P_inf/(gamma-1).
 *   Sec. 3.1, Eqs. (semi-discrezization-euler), (semi-discrezization-material):
 *           L(U) = -(F_{i+1/2} - F_{i-1/2})/dx, plus phi_i (u_{i+1/2}-u_{i-1/2})/dx
 *           for Gamma and Pi; SSP-RK3 of Shu & Osher in time.
 *   Sec. 3.2, Eqs. (primitive-variable), (eigen-vectors),
 *           (characteristic-decompsoition), (back-projected): projection of
 *           the stencil's primitives with L_{i+1/2}, back-projection with R.
 *   Sec. 3.2.1, Eqs. (hllc-flux), (flux-function), (wave-speed),
 *           (wave-speeds), (velocities): stiffened-gas HLLC flux and face velocity.
 *   Sec. 3.3.1-3.3.2, Eqs. (final-weighting), (candidates), (weight-new),
 *           (smoothness-indicator), (tau-5), (weighting-modification): WENO-IS.
 *   Sec. 3.4, Eq. (upwind): MOOD-type positivity cascade 5th -> 3rd -> 1st.
 *   Sec. 5, Sec. 6: the comparison scheme WENO-JS (Jiang & Shu 1996), as an
 *           option of the reconstruction.
 *
 * Readings where the paper is silent or garbled (each one is applied here,
 * in the CUDA path and in the tests):
 *   - candidate 1 is q_i/2 + q_{i+1}/2 (the printed minus sign cannot
 *     recover the 5th-order linear scheme with d = (4,2,3,1)/10);
 *   - the candidates are evaluated in increment form about q_i and the
 *     weighted sum as q_i + sum(alpha_k delta_k)/sum(alpha_k): algebraically
 *     Eq. (final-weighting) with Eq. (weighting-modification), and it keeps
 *     a constant stencil exactly constant;
 *   - linear weights are held as the integers (4,2,3,1); the normalisation by
 *     sum(alpha) makes the common factor 1/10 irrelevant;
 *   - S_12 = {i-1, i, i+1}, matching the printed beta_12;
 *   - L_{i+1/2} and R_{i+1/2} are both built from rho_bar = (rho_i+rho_{i+1})/2
 *     and c_bar = (c_i+c_{i+1})/2, so that L R = I;
 *   - epsilon is a parameter (1e-40 by default in FP64; WENO-JS: 1e-6 and
 *     the power 2 of Jiang & Shu, which the paper does not restate);
 *   - WENO-JS under MOOD: its 3rd-order level is the scheme's own (the
 *     2-point candidates with the modified weights), since WENO-JS has no
 *     smaller candidates;
 *   - the MOOD check is rho > 0, Gamma > 0 and (Gamma+1) p + Pi > 0, done per
 *     face and per side; the 3rd-order retry keeps tau_5 and the modified
 *     alpha_1, alpha_2 and sets d_3 = d_4 = 0; the 1st-order level takes the
 *     primitive state of the upwind cell itself;
 *   - HLLC: the Roe average of u uses sqrt(rho_r) u_r and the averaged c^2
 *     uses sqrt(rho_r) c_r^2 (printed typos); sign(0) = 0; where S_k == S*
 *     the star state of that side is its own flux and velocity;
 *   - dt = CFL / max_cells sum_d (|u_d| + c)/dx_d, taken once per step at U^n;
 *   - multi-dimensional: dimension by dimension, directions summed x, y, z.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NG 3   /* ghost layers per side */
#define MAXV 7 /* rho, 3 momenta, E, Gamma, Pi */

enum { OR_BC_TRANSMISSIVE = 0, OR_BC_PERIODIC = 1, OR_BC_REFLECTIVE = 2 };
enum { OR_W_MODIFIED = 0, OR_W_BASIC = 1, OR_W_JS = 2 };

typedef struct {
  int ndim;        /* 1, 2 or 3 */
  int n[3];        /* interior cells per direction (unused dims: 1) */
  double dx[3];    /* cell size per direction */
  int bc[3][2];    /* boundary kind per direction and side */
  double eps;      /* WENO epsilon */
  int mood;        /* 1: MOOD positivity cascade on */
  int weights;     /* OR_W_MODIFIED (the scheme), OR_W_BASIC (Eq. weight-new) or OR_W_JS (WENO-JS) */
} or_grid;

/* ------------------------------------------------------------------ */
/* layout: conservative field f, padded extents P[d] = n[d]+2*NG for active
 * directions and 1 otherwise, x fastest.                              */

static int nvars(const or_grid *g) { return g->ndim + 4; }

static void padded(const or_grid *g, int64_t P[3]) {
  for (int d = 0; d < 3; ++d) P[d] = (d < g->ndim) ? (int64_t)g->n[d] + 2 * NG : 1;
}

static int64_t cells_padded(const or_grid *g) {
  int64_t P[3];
  padded(g, P);
  return P[0] * P[1] * P[2];
}

/* linear index of padded coordinates (x, y, z) */
static int64_t lin(const int64_t P[3], int64_t x, int64_t y, int64_t z) {
  return (z * P[1] + y) * P[0] + x;
}

/* ------------------------------------------------------------------ */
/* Sec. 2, Eq. (eos): conservative <-> primitive for one cell.  The
 * primitive vector is (rho, u_1..u_ndim, p, Gamma, Pi) in axis order.  */

static void cons_to_prim(int ndim, const double *U, double *q) {
  double rho = U[0];
  double usq = 0.0;
  q[0] = rho;
  for (int d = 0; d < ndim; ++d) {
    q[1 + d] = U[1 + d] / rho;
    usq = usq + q[1 + d] * q[1 + d];
  }
  double ke = (0.5 * rho) * usq;
  double E = U[1 + ndim], Gam = U[2 + ndim], Pi = U[3 + ndim];
  q[1 + ndim] = ((E - ke) - Pi) / Gam; /* p from rho e = Gamma p + Pi */
  q[2 + ndim] = Gam;
  q[3 + ndim] = Pi;
}

static void prim_to_cons(int ndim, const double *q, double *U) {
  double rho = q[0];
  double usq = 0.0;
  U[0] = rho;
  for (int d = 0; d < ndim; ++d) {
    U[1 + d] = rho * q[1 + d];
    usq = usq + q[1 + d] * q[1 + d];
  }
  double ke = (0.5 * rho) * usq;
  double p = q[1 + ndim], Gam = q[2 + ndim], Pi = q[3 + ndim];
  U[1 + ndim] = ((Gam * p) + Pi) + ke;
  U[2 + ndim] = Gam;
  U[3 + ndim] = Pi;
}

/* squared sound speed of the stiffened gas, gamma (p + P_inf)/rho written
 * with Gamma and Pi: ((Gamma+1) p + Pi)/(Gamma rho). */
static double sound_speed2(double rho, double p, double Gam, double Pi) {
  return (((Gam + 1.0) * p) + Pi) / (Gam * rho);
}

/* ------------------------------------------------------------------ */
/* Sec. 3.3.1-3.3.2: WENO-IS reconstruction of the left face value at
 * x_{i+1/2} from v[0..4] = q_{i-2}, q_{i-1}, q_i, q_{i+1}, q_{i+2}.
 * order 5: all four candidates; order 3: d_3 = d_4 = 0 (end of Sec. 3.3.1).
 * dbg (nullable) receives beta_1..beta_4, beta_12, tau_5, alpha_1..alpha_4;
 * for WENO-JS at order 5: beta_0..beta_2, 0, 0, tau_5, alpha_0..alpha_2, 0. */
double or_weno_is(const double v[5], double eps, int order, int weights, double *dbg) {
  const double qm2 = v[0], qm1 = v[1], q0 = v[2], qp1 = v[3], qp2 = v[4];
  const double c13_12 = 13.0 / 12.0;

  /* Eq. (candidates), increment form about q_i:
   *   q^(1) = q_i/2 + q_{i+1}/2        = q_i + (1/2)(q_{i+1} - q_i)
   *   q^(2) = -q_{i-1}/2 + 3 q_i/2     = q_i + (1/2)(q_i - q_{i-1})
   *   q^(3) = q_i/3 + 5q_{i+1}/6 - q_{i+2}/6 = q_i + (5/6)(q_{i+1}-q_i) - (1/6)(q_{i+2}-q_i)
   *   q^(4) = q_{i-2}/3 - 7q_{i-1}/6 + 11q_i/6 = q_i + (1/3)(q_{i-2}-q_i) - (7/6)(q_{i-1}-q_i) */
  double delta1 = 0.5 * (qp1 - q0);
  double delta2 = 0.5 * (q0 - qm1);
  double delta3 = ((5.0 / 6.0) * (qp1 - q0)) - ((1.0 / 6.0) * (qp2 - q0));
  double delta4 = ((1.0 / 3.0) * (qm2 - q0)) - ((7.0 / 6.0) * (qm1 - q0));

  /* Eq. (smoothness-indicator) */
  double a, b;
  a = qp1 - q0;
  double beta1 = a * a;
  a = q0 - qm1;
  double beta2 = a * a;
  a = (q0 - 2.0 * qp1) + qp2;
  b = ((3.0 * q0) - (4.0 * qp1)) + qp2;
  double beta3 = (c13_12 * (a * a)) + (0.25 * (b * b));
  a = (qm2 - 2.0 * qm1) + q0;
  b = (qm2 - (4.0 * qm1)) + (3.0 * q0);
  double beta4 = (c13_12 * (a * a)) + (0.25 * (b * b));
  /* beta_12 on S_12 = {i-1, i, i+1} (Sec. 3.3.2) */
  a = (qm1 - 2.0 * q0) + qp1;
  b = qm1 - qp1;
  double beta12 = (c13_12 * (a * a)) + (0.25 * (b * b));
  /* Eq. (tau-5) */
  a = ((qp2 - 2.0 * qp1) + 2.0 * qm1) - qm2;
  b = ((((qp2 - 4.0 * qp1) + 6.0 * q0) - 4.0 * qm1) + qm2);
  double tau5 = (0.25 * (a * a)) + (c13_12 * (b * b));

  if (weights == OR_W_JS && order == 5) {
    /* Classical WENO-JS (Jiang & Shu 1996), the paper's comparison scheme:
     * three 3-point candidates S_0 = {i-2,i-1,i}, S_1 = {i-1,i,i+1},
     * S_2 = {i,i+1,i+2} with linear weights (1,6,3)/10 and
     * alpha_k = d_k / (eps + beta_k)^2.  S_0 and S_2 are the paper's S_4 and
     * S_3 (candidates q^(4), q^(3), indicators beta_4, beta_3); S_1 is S_12
     * (indicator beta_12), whose 3rd-order candidate is
     *   -q_{i-1}/6 + 5q_i/6 + q_{i+1}/3 = q_i + (1/3)(q_{i+1}-q_i) - (1/6)(q_{i-1}-q_i). */
    double deltaC = ((1.0 / 3.0) * (qp1 - q0)) - ((1.0 / 6.0) * (qm1 - q0));
    double e0 = eps + beta4, e1 = eps + beta12, e2 = eps + beta3;
    double a0 = 1.0 / (e0 * e0);
    double a1 = 6.0 / (e1 * e1);
    double a2 = 3.0 / (e2 * e2);
    if (dbg) {
      dbg[0] = beta4; dbg[1] = beta12; dbg[2] = beta3;
      dbg[3] = 0.0; dbg[4] = 0.0; dbg[5] = tau5;
      dbg[6] = a0; dbg[7] = a1; dbg[8] = a2; dbg[9] = 0.0;
    }
    double numJ = ((a0 * delta4) + (a1 * deltaC)) + (a2 * delta3);
    double denJ = (a0 + a1) + a2;
    return q0 + numJ / denJ;
  }

  /* Eq. (weighting-modification) (or Eq. (weight-new) with q = 1).  The
   * 3rd-order level of WENO-JS is the one of the scheme (modified weights,
   * d_3 = d_4 = 0): WENO-JS has no 2-point candidates of its own. */
  double r1 = tau5 / (beta1 + eps);
  double r2 = tau5 / (beta2 + eps);
  double r3 = tau5 / (beta3 + eps);
  double r4 = tau5 / (beta4 + eps);
  double alpha1, alpha2;
  if (weights != OR_W_BASIC) {
    double r12 = tau5 / (beta12 + eps);
    alpha1 = 4.0 * (1.0 + r1 * r12);
    alpha2 = 2.0 * (1.0 + r2 * r12);
  } else {
    alpha1 = 4.0 * (1.0 + r1);
    alpha2 = 2.0 * (1.0 + r2);
  }
  double alpha3 = 3.0 * (1.0 + r3);
  double alpha4 = 1.0 * (1.0 + r4);
  if (order == 3) { /* d_3 = d_4 = 0 */
    alpha3 = 0.0;
    alpha4 = 0.0;
  }
  if (dbg) {
    dbg[0] = beta1; dbg[1] = beta2; dbg[2] = beta3; dbg[3] = beta4;
    dbg[4] = beta12; dbg[5] = tau5;
    dbg[6] = alpha1; dbg[7] = alpha2; dbg[8] = alpha3; dbg[9] = alpha4;
  }
  /* Eq. (final-weighting): sum_k omega_k q^(k), omega_k = alpha_k / sum alpha */
  double num = (((alpha1 * delta1) + (alpha2 * delta2)) + (alpha3 * delta3)) + (alpha4 * delta4);
  double den = ((alpha1 + alpha2) + alpha3) + alpha4;
  return q0 + num / den;
}

/* ------------------------------------------------------------------ */
/* Sec. 3.2, Eq. (eigen-vectors) generalised to nq = ndim + 4 primitive
 * variables in the frame of the sweep direction:
 *   q = (rho, u_n, u_t1, [u_t2], p, Gamma, Pi)
 * rows of L / columns of R: (u-c), entropy, shear(s), Gamma, Pi, (u+c). */
void or_char_matrices(int nq, double rho_bar, double c_bar, double *Lm, double *Rm) {
  int nt = nq - 5;         /* tangential velocities */
  int ip = 2 + nt;         /* column of p in q */
  int iG = ip + 1, iP = ip + 2;
  int last = nq - 1;
  memset(Lm, 0, sizeof(double) * nq * nq);
  memset(Rm, 0, sizeof(double) * nq * nq);
  double rc = rho_bar * c_bar;
  double c2 = c_bar * c_bar;
  /* L */
  Lm[0 * nq + 1] = -rc / 2.0;
  Lm[0 * nq + ip] = 1.0 / 2.0;
  Lm[1 * nq + 0] = 1.0;
  Lm[1 * nq + ip] = -1.0 / c2;
  for (int t = 0; t < nt; ++t) Lm[(2 + t) * nq + (2 + t)] = 1.0;
  Lm[(2 + nt) * nq + iG] = 1.0;
  Lm[(3 + nt) * nq + iP] = 1.0;
  Lm[last * nq + 1] = rc / 2.0;
  Lm[last * nq + ip] = 1.0 / 2.0;
  /* R */
  Rm[0 * nq + 0] = 1.0 / c2;
  Rm[0 * nq + 1] = 1.0;
  Rm[0 * nq + last] = 1.0 / c2;
  Rm[1 * nq + 0] = -1.0 / rc;
  Rm[1 * nq + last] = 1.0 / rc;
  for (int t = 0; t < nt; ++t) Rm[(2 + t) * nq + (2 + t)] = 1.0;
  Rm[ip * nq + 0] = 1.0;
  Rm[ip * nq + last] = 1.0;
  Rm[iG * nq + (2 + nt)] = 1.0;
  Rm[iP * nq + (3 + nt)] = 1.0;
}

static void matvec(int nq, const double *M, const double *x, double *y) {
  for (int r = 0; r < nq; ++r) {
    double acc = 0.0;
    for (int k = 0; k < nq; ++k) acc = acc + M[r * nq + k] * x[k];
    y[r] = acc;
  }
}

/* Sec. 3.4 (with the strict reading): a reconstructed primitive state is
 * admissible when rho > 0, Gamma > 0 and (Gamma+1) p + Pi > 0. */
static int admissible(int nq, const double *q) {
  double rho = q[0], p = q[nq - 3], Gam = q[nq - 2], Pi = q[nq - 1];
  return (rho > 0.0) && (Gam > 0.0) && ((((Gam + 1.0) * p) + Pi) > 0.0);
}

/* ------------------------------------------------------------------ */
/* Sec. 3.2.1: HLLC flux of the stiffened-gas mixture in the sweep frame.
 * ql, qr: (rho, u_n, u_t.., p, Gamma, Pi).  Fhat receives the nq flux
 * components of (rho, rho u_n, rho u_t.., E, Gamma, Pi); *ustar the face
 * velocity of Eq. (velocities). */
static void hllc_core(int nq, const double *ql, const double *qr, double *Fhat, double *ustar, double *waves) {
  int nt = nq - 5;
  const double *qs[2] = {ql, qr};
  double U[2][MAXV], F[2][MAXV], c2[2], cc[2];
  for (int k = 0; k < 2; ++k) {
    const double *q = qs[k];
    double rho = q[0], un = q[1], p = q[2 + nt], Gam = q[3 + nt], Pi = q[4 + nt];
    double usq = un * un;
    for (int t = 0; t < nt; ++t) usq = usq + q[2 + t] * q[2 + t];
    double E = ((Gam * p) + Pi) + (0.5 * rho) * usq;
    double mn = rho * un;
    U[k][0] = rho;
    U[k][1] = mn;
    F[k][0] = mn;
    F[k][1] = (mn * un) + p;
    for (int t = 0; t < nt; ++t) {
      U[k][2 + t] = rho * q[2 + t];
      F[k][2 + t] = mn * q[2 + t];
    }
    U[k][2 + nt] = E;
    F[k][2 + nt] = (E + p) * un;
    U[k][3 + nt] = Gam;
    F[k][3 + nt] = Gam * un;
    U[k][4 + nt] = Pi;
    F[k][4 + nt] = Pi * un;
    c2[k] = sound_speed2(rho, p, Gam, Pi);
    cc[k] = sqrt(c2[k]);
  }
  double rl = ql[0], ul = ql[1], pl = ql[2 + nt];
  double rr = qr[0], ur = qr[1], pr = qr[2 + nt];
  /* Eq. (wave-speeds): Roe-averaged u and Einfeldt-type c^2 */
  double sl = sqrt(rl), sr = sqrt(rr);
  double den = sl + sr;
  double ubar = ((sl * ul) + (sr * ur)) / den;
  double du = ur - ul;
  double c2bar = (((sl * c2[0]) + (sr * c2[1])) / den) + (((0.5 * (sl * sr)) / (den * den)) * (du * du));
  double cbar = sqrt(c2bar);
  double Sl = fmin(fmin(ubar - cbar, ul - cc[0]), 0.0);
  double Sr = fmax(fmax(ubar + cbar, ur + cc[1]), 0.0);
  /* Eq. (wave-speed): middle wave */
  double num = ((pr - pl) + ((rl * ul) * (Sl - ul))) - ((rr * ur) * (Sr - ur));
  double dd = (rl * (Sl - ul)) - (rr * (Sr - ur));
  double Ss = num / dd;
  if (waves) {
    waves[0] = ubar; waves[1] = c2bar; waves[2] = Sl; waves[3] = Sr; waves[4] = Ss;
  }
  /* Eq. (flux-function) with D* = (0, 1, 0.., S*, 0, 0) */
  double Fs[2][MAXV], us[2];
  double Sk[2] = {Sl, Sr};
  for (int k = 0; k < 2; ++k) {
    const double *q = qs[k];
    double S = Sk[k], rho = q[0], un = q[1], p = q[2 + nt];
    if (S == Ss) {
      for (int m = 0; m < nq; ++m) Fs[k][m] = F[k][m];
      us[k] = un;
      continue;
    }
    double Pk = p + ((rho * (S - un)) * (Ss - un));
    for (int m = 0; m < nq; ++m) {
      double D = 0.0;
      if (m == 1) D = 1.0;
      if (m == 2 + nt) D = Ss;
      double t = (Ss * ((S * U[k][m]) - F[k][m])) + ((S * Pk) * D);
      Fs[k][m] = t / (S - Ss);
    }
    us[k] = (Ss * (S - un)) / (S - Ss); /* Eq. (velocities) */
  }
  /* Eq. (hllc-flux) and Eq. (velocities): blend by sign(S*) */
  double s = (Ss > 0.0) ? 1.0 : ((Ss < 0.0) ? -1.0 : 0.0);
  double wl = (1.0 + s) / 2.0, wr = (1.0 - s) / 2.0;
  for (int m = 0; m < nq; ++m) Fhat[m] = (wl * Fs[0][m]) + (wr * Fs[1][m]);
  *ustar = (wl * us[0]) + (wr * us[1]);
}

void or_hllc(int nq, const double *ql, const double *qr, double *Fhat, double *ustar) {
  hllc_core(nq, ql, qr, Fhat, ustar, NULL);
}

/* or_hllc that also reports the wave-speed estimates of Eq. (wave-speeds)
 * and Eq. (wave-speed): waves = (u_bar, c2_bar, S_l, S_r, S*). */
void or_hllc_waves(int nq, const double *ql, const double *qr, double *Fhat, double *ustar, double *waves) {
  hllc_core(nq, ql, qr, Fhat, ustar, waves);
}

/* ------------------------------------------------------------------ */
/* One face i+1/2: qc[j] (j = 0..5) are the sweep-frame primitives of
 * cells i-2..i+3 and cc[j] their sound speeds.  Sec. 3.2 projection,
 * Sec. 3.3 reconstruction of both sides, Sec. 3.2 back-projection,
 * Sec. 3.4 MOOD cascade, Sec. 3.2.1 HLLC.  lev receives the order used on
 * the left and right side (5, 3 or 1). */
void or_face(int nq, const double *qc /* [6][nq] */, const double *cc /* [6] */, double eps,
             int mood, int weights, double *Fhat, double *ustar, int lev[2], double *qlr /* nullable [2][nq] */) {
  double rho_bar = 0.5 * (qc[2 * nq + 0] + qc[3 * nq + 0]);
  double c_bar = 0.5 * (cc[2] + cc[3]);
  double Lm[MAXV * MAXV], Rm[MAXV * MAXV];
  or_char_matrices(nq, rho_bar, c_bar, Lm, Rm);
  double w[6][MAXV];
  for (int j = 0; j < 6; ++j) matvec(nq, Lm, &qc[j * nq], w[j]);

  double q[2][MAXV];
  for (int side = 0; side < 2; ++side) {
    /* left: cells i-2..i+2; right: the mirror i+3..i-1 */
    int order = 5;
    for (;;) {
      double wt[MAXV];
      for (int r = 0; r < nq; ++r) {
        double v[5];
        for (int k = 0; k < 5; ++k) v[k] = (side == 0) ? w[k][r] : w[5 - k][r];
        wt[r] = or_weno_is(v, eps, order, weights, NULL);
      }
      matvec(nq, Rm, wt, q[side]);
      if (!mood || admissible(nq, q[side])) break;
      if (order == 5) {
        order = 3;
        continue;
      }
      /* Eq. (upwind): first order, the primitive state of the upwind cell */
      order = 1;
      const double *src = &qc[(side == 0 ? 2 : 3) * nq];
      for (int r = 0; r < nq; ++r) q[side][r] = src[r];
      break;
    }
    lev[side] = order;
  }
  if (qlr) {
    for (int r = 0; r < nq; ++r) {
      qlr[r] = q[0][r];
      qlr[nq + r] = q[1][r];
    }
  }
  hllc_core(nq, q[0], q[1], Fhat, ustar, NULL);
}

/* ------------------------------------------------------------------ */
/* ghost layers of direction d (Sec. 4: periodic; Sec. 6: constant
 * extrapolation / non-reflecting; reflective walls).  Only cells whose other
 * coordinates are interior are filled: the sweeps never read the corners. */
static void fill_ghosts_dir(const or_grid *g, double *Ufull, int d) {
  int64_t P[3];
  padded(g, P);
  int64_t N = cells_padded(g);
  int nv = nvars(g);
  int64_t lo[3], hi[3];
  for (int e = 0; e < 3; ++e) {
    lo[e] = (e < g->ndim) ? NG : 0;
    hi[e] = (e < g->ndim) ? NG + g->n[e] : 1;
  }
  int n = g->n[d];
  int64_t a[3];
  for (a[2] = lo[2]; a[2] < hi[2]; ++a[2])
    for (a[1] = lo[1]; a[1] < hi[1]; ++a[1])
      for (a[0] = lo[0]; a[0] < hi[0]; ++a[0]) {
        if (a[d] != NG) continue; /* one pencil per transverse position */
        for (int side = 0; side < 2; ++side) {
          int kind = g->bc[d][side];
          for (int gI = 1; gI <= NG; ++gI) {
            int64_t dst = (side == 0) ? (NG - gI) : (NG + n - 1 + gI);
            int64_t src;
            if (kind == OR_BC_PERIODIC)
              src = (side == 0) ? (NG + n - gI) : (NG + gI - 1);
            else if (kind == OR_BC_REFLECTIVE)
              src = (side == 0) ? (NG + gI - 1) : (NG + n - gI);
            else
              src = (side == 0) ? NG : (NG + n - 1);
            int64_t b[3] = {a[0], a[1], a[2]}, s[3] = {a[0], a[1], a[2]};
            b[d] = dst;
            s[d] = src;
            int64_t id = lin(P, b[0], b[1], b[2]), is = lin(P, s[0], s[1], s[2]);
            for (int f = 0; f < nv; ++f) {
              double val = Ufull[f * N + is];
              if (kind == OR_BC_REFLECTIVE && f == 1 + d) val = -val;
              Ufull[f * N + id] = val;
            }
          }
        }
      }
}

void or_fill_ghosts(const or_grid *g, double *U) {
  for (int d = 0; d < g->ndim; ++d) fill_ghosts_dir(g, U, d);
}

/* ------------------------------------------------------------------ */
/* Sec. 3.1: L(U) on the interior.  U must have its ghosts filled.
 * L receives the nv fields on the padded layout (ghosts untouched).
 * mask (nullable): per direction d, faces i+1/2 for i = -1..n_d-1 at every
 * interior transverse position, laid out [z][y][x] with extent n_d+1 along d;
 * byte = code(left) | code(right) << 2, code 0/1/2 for order 5/3/1. */
void or_rhs(const or_grid *g, const double *U, double *L, uint8_t *mask[3]) {
  int64_t P[3];
  padded(g, P);
  int64_t N = cells_padded(g);
  int nv = nvars(g), nq = nv, ndim = g->ndim;
  int64_t lo[3], hi[3];
  for (int e = 0; e < 3; ++e) {
    lo[e] = (e < ndim) ? NG : 0;
    hi[e] = (e < ndim) ? NG + g->n[e] : 1;
  }
  /* L starts at zero on the interior */
  for (int64_t z = lo[2]; z < hi[2]; ++z)
    for (int64_t y = lo[1]; y < hi[1]; ++y)
      for (int64_t x = lo[0]; x < hi[0]; ++x)
        for (int f = 0; f < nv; ++f) L[f * N + lin(P, x, y, z)] = 0.0;

  for (int d = 0; d < ndim; ++d) {
    /* transverse axes of direction d, in increasing axis order */
    int t1 = -1, t2 = -1;
    for (int e = 0; e < ndim; ++e)
      if (e != d) {
        if (t1 < 0) t1 = e; else t2 = e;
      }
    /* sweep-frame primitive order: rho, u_d, u_t1, u_t2, p, Gamma, Pi */
    int perm[MAXV];
    perm[0] = 0;
    perm[1] = 1 + d;
    int k = 2;
    if (t1 >= 0) perm[k++] = 1 + t1;
    if (t2 >= 0) perm[k++] = 1 + t2;
    perm[k++] = 1 + ndim;
    perm[k++] = 2 + ndim;
    perm[k++] = 3 + ndim;
    int n = g->n[d];
    int64_t ext[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
    int64_t mext[3] = {ext[0], ext[1], ext[2]};
    mext[d] = n + 1;

    int64_t npencil = ext[0] * ext[1] * ext[2] / n;
#pragma omp parallel for schedule(static)
    for (int64_t pid = 0; pid < npencil; ++pid) {
      /* transverse coordinates of this pencil */
      int64_t a[3];
      int64_t rem = pid;
      for (int e = 0; e < 3; ++e) {
        if (e == d) { a[e] = 0; continue; }
        a[e] = rem % ext[e];
        rem /= ext[e];
      }
      double *Fh = (double *)malloc(sizeof(double) * (size_t)(n + 1) * nq);
      double *us = (double *)malloc(sizeof(double) * (size_t)(n + 1));
      for (int i = -1; i < n; ++i) { /* face i+1/2 */
        double qc[6 * MAXV], cc[6], qg[MAXV], Uc[MAXV];
        for (int j = 0; j < 6; ++j) {
          int64_t c[3] = {lo[0] + a[0], lo[1] + a[1], lo[2] + a[2]};
          c[d] = NG + i - 2 + j;
          int64_t id = lin(P, c[0], c[1], c[2]);
          for (int f = 0; f < nv; ++f) Uc[f] = U[f * N + id];
          cons_to_prim(ndim, Uc, qg);
          for (int r = 0; r < nq; ++r) qc[j * nq + r] = qg[perm[r]];
          cc[j] = sqrt(sound_speed2(qg[0], qg[1 + ndim], qg[2 + ndim], qg[3 + ndim]));
        }
        int lev[2];
        or_face(nq, qc, cc, g->eps, g->mood, g->weights, &Fh[(i + 1) * nq], &us[i + 1], lev, NULL);
        if (mask && mask[d]) {
          int64_t m[3] = {a[0], a[1], a[2]};
          m[d] = i + 1;
          int code_l = lev[0] == 5 ? 0 : (lev[0] == 3 ? 1 : 2);
          int code_r = lev[1] == 5 ? 0 : (lev[1] == 3 ? 1 : 2);
          mask[d][(m[2] * mext[1] + m[1]) * mext[0] + m[0]] = (uint8_t)(code_l | (code_r << 2));
        }
      }
      /* Eqs. (semi-discrezization-euler), (semi-discrezization-material) */
      double dx = g->dx[d];
      for (int i = 0; i < n; ++i) {
        int64_t c[3] = {lo[0] + a[0], lo[1] + a[1], lo[2] + a[2]};
        c[d] = NG + i;
        int64_t id = lin(P, c[0], c[1], c[2]);
        for (int r = 0; r < nq; ++r) {
          int f = perm[r];
          double dF = Fh[(i + 1) * nq + r] - Fh[i * nq + r];
          double term = -(dF / dx);
          if (f >= 2 + ndim) { /* Gamma, Pi: add phi_i (u_{i+1/2} - u_{i-1/2})/dx */
            double phi = U[f * N + id];
            term = term + phi * ((us[i + 1] - us[i]) / dx);
          }
          L[f * N + id] = L[f * N + id] + term;
        }
      }
      free(Fh);
      free(us);
    }
  }
}

/* ------------------------------------------------------------------ */
/* CFL step size at U (ghosts not needed):
 * dt = cfl / max_cells sum_d (|u_d| + c)/dx_d. */
double or_cfl_dt(const or_grid *g, const double *U, double cfl) {
  int64_t P[3];
  padded(g, P);
  int64_t N = cells_padded(g);
  int nv = nvars(g), ndim = g->ndim;
  int64_t lo[3], hi[3];
  for (int e = 0; e < 3; ++e) {
    lo[e] = (e < ndim) ? NG : 0;
    hi[e] = (e < ndim) ? NG + g->n[e] : 1;
  }
  double lmax = 0.0;
  for (int64_t z = lo[2]; z < hi[2]; ++z)
    for (int64_t y = lo[1]; y < hi[1]; ++y)
      for (int64_t x = lo[0]; x < hi[0]; ++x) {
        double Uc[MAXV], q[MAXV];
        int64_t id = lin(P, x, y, z);
        for (int f = 0; f < nv; ++f) Uc[f] = U[f * N + id];
        cons_to_prim(ndim, Uc, q);
        double c = sqrt(sound_speed2(q[0], q[1 + ndim], q[2 + ndim], q[3 + ndim]));
        double lam = 0.0;
        for (int d = 0; d < ndim; ++d) lam = lam + (fabs(q[1 + d]) + c) / g->dx[d];
        if (lam > lmax) lmax = lam;
      }
  return cfl / lmax;
}

/* number of interior cells with rho <= 0 or (Gamma+1) p + Pi <= 0 (or NaN) */
int64_t or_count_nonphysical(const or_grid *g, const double *U) {
  int64_t P[3];
  padded(g, P);
  int64_t N = cells_padded(g);
  int nv = nvars(g), ndim = g->ndim;
  int64_t lo[3], hi[3], bad = 0;
  for (int e = 0; e < 3; ++e) {
    lo[e] = (e < ndim) ? NG : 0;
    hi[e] = (e < ndim) ? NG + g->n[e] : 1;
  }
  for (int64_t z = lo[2]; z < hi[2]; ++z)
    for (int64_t y = lo[1]; y < hi[1]; ++y)
      for (int64_t x = lo[0]; x < hi[0]; ++x) {
        double Uc[MAXV], q[MAXV];
        int64_t id = lin(P, x, y, z);
        for (int f = 0; f < nv; ++f) Uc[f] = U[f * N + id];
        cons_to_prim(ndim, Uc, q);
        if (!admissible(nv, &q[0] /* axis-order q ends with p, Gamma, Pi too */)) ++bad;
      }
  return bad;
}

/* ------------------------------------------------------------------ */
/* One SSP-RK3 step of Shu & Osher (Sec. 3.1):
 *   U1 = Un + dt L(Un)
 *   U2 = 3/4 Un + 1/4 (U1 + dt L(U1))
 *   Un+1 = 1/3 Un + 2/3 (U2 + dt L(U2))
 * U (padded) is advanced in place.  dt <= 0 takes the CFL step at Un.
 * masks (nullable): 3 stages x ndim direction arrays, as in or_rhs.
 * Returns the dt used. */
double or_step(const or_grid *g, double *U, double dt, double cfl, uint8_t *masks[3][3]) {
  int64_t N = cells_padded(g);
  int nv = nvars(g);
  if (dt <= 0.0) dt = or_cfl_dt(g, U, cfl);
  size_t bytes = sizeof(double) * (size_t)N * nv;
  double *Un = (double *)malloc(bytes);
  double *Us = (double *)malloc(bytes);
  double *L = (double *)malloc(bytes);
  memcpy(Un, U, bytes);
  memcpy(Us, U, bytes);
  int64_t P[3];
  padded(g, P);
  int ndim = g->ndim;
  int64_t lo[3], hi[3];
  for (int e = 0; e < 3; ++e) {
    lo[e] = (e < ndim) ? NG : 0;
    hi[e] = (e < ndim) ? NG + g->n[e] : 1;
  }
  const double c13 = 1.0 / 3.0, c23 = 2.0 / 3.0;
  for (int s = 0; s < 3; ++s) {
    or_fill_ghosts(g, Us);
    or_rhs(g, Us, L, masks ? masks[s] : NULL);
    for (int f = 0; f < nv; ++f)
      for (int64_t z = lo[2]; z < hi[2]; ++z)
        for (int64_t y = lo[1]; y < hi[1]; ++y)
          for (int64_t x = lo[0]; x < hi[0]; ++x) {
            int64_t id = f * N + lin(P, x, y, z);
            double un = Un[id], us = Us[id], l = L[id];
            double out;
            if (s == 0)
              out = un + dt * l;
            else if (s == 1)
              out = (0.75 * un) + (0.25 * (us + dt * l));
            else
              out = (c13 * un) + (c23 * (us + dt * l));
            Us[id] = out;
          }
  }
  memcpy(U, Us, bytes);
  free(Un);
  free(Us);
  free(L);
  return dt;
}

/* ------------------------------------------------------------------ */
/* helpers exported for the pins and the drivers */
void or_cons_to_prim(int ndim, const double *U, double *q) { cons_to_prim(ndim, U, q); }
void or_prim_to_cons(int ndim, const double *q, double *U) { prim_to_cons(ndim, q, U); }
double or_sound_speed(double rho, double p, double Gam, double Pi) {
  return sqrt(sound_speed2(rho, p, Gam, Pi));
}

/* prim -> cons over a whole padded array (fields in axis order) */
void or_prim_to_cons_array(int ndim, int64_t ncell, const double *Q, double *U) {
  int nv = ndim + 4;
  for (int64_t i = 0; i < ncell; ++i) {
    double q[MAXV] = {0}, u[MAXV] = {0};
    for (int f = 0; f < nv; ++f) q[f] = Q[f * ncell + i];
    prim_to_cons(ndim, q, u);
    for (int f = 0; f < nv; ++f) U[f * ncell + i] = u[f];
  }
}

void or_cons_to_prim_array(int ndim, int64_t ncell, const double *U, double *Q) {
  int nv = ndim + 4;
  for (int64_t i = 0; i < ncell; ++i) {
    double q[MAXV] = {0}, u[MAXV] = {0};
    for (int f = 0; f < nv; ++f) u[f] = U[f * ncell + i];
    cons_to_prim(ndim, u, q);
    for (int f = 0; f < nv; ++f) Q[f * ncell + i] = q[f];
  }
}

/* ------------------------------------------------------------------ */
/* Batched independent 1D tubes: tube t occupies padded cells
 * [off[t], off[t+1]) of every field (3 ghosts each side), dx = 1/len,
 * transmissive ends, its own CFL dt.  dts (nullable) receives the dt used. */
void or_tubes_step(int64_t ntubes, const int64_t *off, int64_t total, double *U, double cfl, double eps,
                   int mood, int weights, double *dts) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t t = 0; t < ntubes; ++t) {
    int64_t len = off[t + 1] - off[t] - 2 * NG;
    or_grid g;
    memset(&g, 0, sizeof g);
    g.ndim = 1;
    g.n[0] = (int)len;
    g.n[1] = g.n[2] = 1;
    g.dx[0] = 1.0 / (double)len;
    g.dx[1] = g.dx[2] = 1.0;
    g.eps = eps;
    g.mood = mood;
    g.weights = weights;
    int64_t P = len + 2 * NG;
    double *Ut = (double *)malloc(sizeof(double) * 5 * (size_t)P);
    for (int f = 0; f < 5; ++f) memcpy(&Ut[f * P], &U[f * total + off[t]], sizeof(double) * (size_t)P);
    double dt = or_step(&g, Ut, 0.0, cfl, NULL);
    for (int f = 0; f < 5; ++f) memcpy(&U[f * total + off[t]], &Ut[f * P], sizeof(double) * (size_t)P);
    if (dts) dts[t] = dt;
    free(Ut);
  }
}

/* ------------------------------------------------------------------ */
/* ctypes-friendly constructor of the grid struct */
void or_grid_set(or_grid *g, int ndim, const int *n, const double *dx, const int *bc, double eps, int mood,
                 int weights) {
  memset(g, 0, sizeof *g);
  g->ndim = ndim;
  for (int d = 0; d < 3; ++d) {
    g->n[d] = (d < ndim) ? n[d] : 1;
    g->dx[d] = (d < ndim) ? dx[d] : 1.0;
    g->bc[d][0] = (d < ndim) ? bc[2 * d] : 0;
    g->bc[d][1] = (d < ndim) ? bc[2 * d + 1] : 0;
  }
  g->eps = eps;
  g->mood = mood;
  g->weights = weights;
}

int or_grid_sizeof(void) { return (int)sizeof(or_grid); }

#ifdef _OPENMP
#include <omp.h>
void or_set_threads(int n) { omp_set_num_threads(n); }
int or_get_threads(void) { return omp_get_max_threads(); }
#else
void or_set_threads(int n) { (void)n; }
int or_get_threads(void) { return 1; }
#endif
