// FP64 arithmetic of one face i+1/2 (shared by the grid sweep and the
// batched-tube sweep; both translation units are built with -fmad=false):
// characteristic projection (Sec. 3.2), WENO-IS reconstruction of both sides
// (Secs. 3.3.1, 3.3.2), back-projection, MOOD positivity cascade (Sec. 3.4)
// and the stiffened-gas HLLC flux and face velocity (Sec. 3.2.1).  Each
// operation is one IEEE binary64 operation in the order written, the order of
// the plain evaluation of the same formulas; the characteristic matrices are
// applied through their non-zero entries only (the skipped terms are exact
// zeros).
#pragma once

#include "ws_internal.h"

namespace ws {
namespace fp64 {

// WENO-JS (Jiang & Shu 1996), the paper's comparison scheme: candidates on
// S_0 = {i-2,i-1,i}, S_1 = {i-1,i,i+1}, S_2 = {i,i+1,i+2} (the paper's S_4,
// S_12, S_3) with linear weights (1,6,3)/10 and alpha_k = d_k/(eps+beta_k)^2.
__device__ __forceinline__ double weno_js(double qm2, double qm1, double q0, double qp1, double qp2, double eps) {
  const double c13_12 = 13.0 / 12.0;
  double delta3 = ((5.0 / 6.0) * (qp1 - q0)) - ((1.0 / 6.0) * (qp2 - q0));
  double delta4 = ((1.0 / 3.0) * (qm2 - q0)) - ((7.0 / 6.0) * (qm1 - q0));
  double deltaC = ((1.0 / 3.0) * (qp1 - q0)) - ((1.0 / 6.0) * (qm1 - q0));
  double a, b;
  a = (q0 - 2.0 * qp1) + qp2;
  b = ((3.0 * q0) - (4.0 * qp1)) + qp2;
  double beta3 = (c13_12 * (a * a)) + (0.25 * (b * b));
  a = (qm2 - 2.0 * qm1) + q0;
  b = (qm2 - (4.0 * qm1)) + (3.0 * q0);
  double beta4 = (c13_12 * (a * a)) + (0.25 * (b * b));
  a = (qm1 - 2.0 * q0) + qp1;
  b = qm1 - qp1;
  double beta12 = (c13_12 * (a * a)) + (0.25 * (b * b));
  double e0 = eps + beta4, e1 = eps + beta12, e2 = eps + beta3;
  double a0 = 1.0 / (e0 * e0);
  double a1 = 6.0 / (e1 * e1);
  double a2 = 3.0 / (e2 * e2);
  double num = ((a0 * delta4) + (a1 * deltaC)) + (a2 * delta3);
  double den = (a0 + a1) + a2;
  return q0 + num / den;
}

// Sec. 3.3.1-3.3.2: left value at x_{i+1/2} from q_{i-2..i+2}.
// order 5: all four candidates; order 3: d3 = d4 = 0.  JS (the WENO-JS
// instantiation): order 5 goes to weno_js, and the 3rd-order MOOD level is
// the scheme's own (modified weights).
template <bool JS>
__device__ __forceinline__ double weno_is(double qm2, double qm1, double q0, double qp1, double qp2, double eps,
                                          int order, int weights) {
  if (JS) {
    if (order == 5) return weno_js(qm2, qm1, q0, qp1, qp2, eps);
    weights = WS_W_MODIFIED;
  }
  const double c13_12 = 13.0 / 12.0;
  // Eq. (candidates) as increments about q_i
  double delta1 = 0.5 * (qp1 - q0);
  double delta2 = 0.5 * (q0 - qm1);
  double delta3 = ((5.0 / 6.0) * (qp1 - q0)) - ((1.0 / 6.0) * (qp2 - q0));
  double delta4 = ((1.0 / 3.0) * (qm2 - q0)) - ((7.0 / 6.0) * (qm1 - q0));
  // Eq. (smoothness-indicator), beta_12 and Eq. (tau-5)
  double a, b;
  a = qp1 - q0;
  double beta1 = a * a;
  a = q0 - qm1;
  double beta2 = a * a;
  a = (qm1 - 2.0 * q0) + qp1;
  b = qm1 - qp1;
  double beta12 = (c13_12 * (a * a)) + (0.25 * (b * b));
  a = ((qp2 - 2.0 * qp1) + 2.0 * qm1) - qm2;
  b = ((((qp2 - 4.0 * qp1) + 6.0 * q0) - 4.0 * qm1) + qm2);
  double tau5 = (0.25 * (a * a)) + (c13_12 * (b * b));
  // Eq. (weighting-modification) / Eq. (weight-new) with q = 1
  double r1 = tau5 / (beta1 + eps);
  double r2 = tau5 / (beta2 + eps);
  double alpha1, alpha2;
  if (weights != WS_W_BASIC) {
    double r12 = tau5 / (beta12 + eps);
    alpha1 = 4.0 * (1.0 + r1 * r12);
    alpha2 = 2.0 * (1.0 + r2 * r12);
  } else {
    alpha1 = 4.0 * (1.0 + r1);
    alpha2 = 2.0 * (1.0 + r2);
  }
  double num = (alpha1 * delta1) + (alpha2 * delta2);
  double den = alpha1 + alpha2;
  if (order == 5) {
    a = (q0 - 2.0 * qp1) + qp2;
    b = ((3.0 * q0) - (4.0 * qp1)) + qp2;
    double beta3 = (c13_12 * (a * a)) + (0.25 * (b * b));
    a = (qm2 - 2.0 * qm1) + q0;
    b = (qm2 - (4.0 * qm1)) + (3.0 * q0);
    double beta4 = (c13_12 * (a * a)) + (0.25 * (b * b));
    double alpha3 = 3.0 * (1.0 + tau5 / (beta3 + eps));
    double alpha4 = 1.0 * (1.0 + tau5 / (beta4 + eps));
    num = (num + (alpha3 * delta3)) + (alpha4 * delta4);
    den = (den + alpha3) + alpha4;
  }
  // Eq. (final-weighting) with omega_k = alpha_k / sum(alpha)
  return q0 + num / den;
}

__device__ __forceinline__ double sound_speed2(double rho, double p, double Gam, double Pi) {
  return (((Gam + 1.0) * p) + Pi) / (Gam * rho);
}

// Characteristic variable r of the sweep-frame primitive q
// (rho, u_n, u_t.., p, Gamma, Pi): row r of L_{i+1/2} in Eq. (eigen-vectors).
template <int NQ>
__device__ __forceinline__ double project(const double* q, int r, double L01, double L1p, double L51) {
  constexpr int NT = NQ - 5, IP = 2 + NT;
  if (r == 0) return (L01 * q[1]) + (0.5 * q[IP]);
  if (r == 1) return q[0] + (L1p * q[IP]);
  if (r == NQ - 1) return (L51 * q[1]) + (0.5 * q[IP]);
  if (r < IP) return q[r];      // shear
  return q[r + 1];              // Gamma, Pi
}

// q = R_{i+1/2} w (Eq. back-projected)
template <int NQ>
__device__ __forceinline__ void back_project(const double* w, double R00, double R10, double R1l, double* q) {
  constexpr int NT = NQ - 5, IP = 2 + NT;
  q[0] = ((R00 * w[0]) + w[1]) + (R00 * w[NQ - 1]);
  q[1] = (R10 * w[0]) + (R1l * w[NQ - 1]);
#pragma unroll
  for (int t = 0; t < NT; ++t) q[2 + t] = w[2 + t];
  q[IP] = w[0] + w[NQ - 1];
  q[IP + 1] = w[IP];
  q[IP + 2] = w[IP + 1];
}

template <int NQ>
__device__ __forceinline__ bool admissible(const double* q) {
  double rho = q[0], p = q[NQ - 3], Gam = q[NQ - 2], Pi = q[NQ - 1];
  return (rho > 0.0) && (Gam > 0.0) && ((((Gam + 1.0) * p) + Pi) > 0.0);
}

// Sec. 3.2.1: HLLC flux (nq components) and face velocity.
template <int NQ>
__device__ __forceinline__ void hllc(const double* ql, const double* qr, double* Fhat, double& ustar) {
  constexpr int NT = NQ - 5;
  double U[2][NQ], F[2][NQ], c2[2], cc[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const double* q = k == 0 ? ql : qr;
    double rho = q[0], un = q[1], p = q[2 + NT], Gam = q[3 + NT], Pi = q[4 + NT];
    double usq = un * un;
#pragma unroll
    for (int t = 0; t < NT; ++t) usq = usq + q[2 + t] * q[2 + t];
    double E = ((Gam * p) + Pi) + (0.5 * rho) * usq;
    double mn = rho * un;
    U[k][0] = rho;
    U[k][1] = mn;
    F[k][0] = mn;
    F[k][1] = (mn * un) + p;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      U[k][2 + t] = rho * q[2 + t];
      F[k][2 + t] = mn * q[2 + t];
    }
    U[k][2 + NT] = E;
    F[k][2 + NT] = (E + p) * un;
    U[k][3 + NT] = Gam;
    F[k][3 + NT] = Gam * un;
    U[k][4 + NT] = Pi;
    F[k][4 + NT] = Pi * un;
    c2[k] = sound_speed2(rho, p, Gam, Pi);
    cc[k] = sqrt(c2[k]);
  }
  double rl = ql[0], ul = ql[1], pl = ql[2 + NT];
  double rr = qr[0], ur = qr[1], pr = qr[2 + NT];
  // Eq. (wave-speeds)
  double sl = sqrt(rl), sr = sqrt(rr);
  double den = sl + sr;
  double ubar = ((sl * ul) + (sr * ur)) / den;
  double du = ur - ul;
  double c2bar = (((sl * c2[0]) + (sr * c2[1])) / den) + (((0.5 * (sl * sr)) / (den * den)) * (du * du));
  double cbar = sqrt(c2bar);
  double Sl = fmin(fmin(ubar - cbar, ul - cc[0]), 0.0);
  double Sr = fmax(fmax(ubar + cbar, ur + cc[1]), 0.0);
  // Eq. (wave-speed)
  double num = ((pr - pl) + ((rl * ul) * (Sl - ul))) - ((rr * ur) * (Sr - ur));
  double dd = (rl * (Sl - ul)) - (rr * (Sr - ur));
  double Ss = num / dd;
  double s = (Ss > 0.0) ? 1.0 : ((Ss < 0.0) ? -1.0 : 0.0);
  double wl = (1.0 + s) / 2.0, wr = (1.0 - s) / 2.0;
  // Eq. (flux-function), D* = (0, 1, 0.., S*, 0, 0), and Eq. (velocities)
  double Fs[2][NQ], us[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const double* q = k == 0 ? ql : qr;
    double S = k == 0 ? Sl : Sr;
    double rho = q[0], un = q[1], p = q[2 + NT];
    if (S == Ss) {
#pragma unroll
      for (int m = 0; m < NQ; ++m) Fs[k][m] = F[k][m];
      us[k] = un;
    } else {
      double Pk = p + ((rho * (S - un)) * (Ss - un));
      double SP = S * Pk;
      double dS = S - Ss;
#pragma unroll
      for (int m = 0; m < NQ; ++m) {
        double t = Ss * ((S * U[k][m]) - F[k][m]);
        if (m == 1) t = t + SP;
        if (m == 2 + NT) t = t + SP * Ss;
        Fs[k][m] = t / dS;
      }
      us[k] = (Ss * (S - un)) / dS;
    }
  }
  // Eq. (hllc-flux)
#pragma unroll
  for (int m = 0; m < NQ; ++m) Fhat[m] = (wl * Fs[0][m]) + (wr * Fs[1][m]);
  ustar = (wl * us[0]) + (wr * us[1]);
}

// One face from the sweep-frame primitives of cells i-2..i+3.
template <int NQ, bool JS>
__device__ __forceinline__ void face(const double (&qc)[6][NQ], const double (&cc)[6], double eps, int mood,
                                     int weights, double* Fhat, double& ustar, int& code_l, int& code_r) {
  double rho_bar = 0.5 * (qc[2][0] + qc[3][0]);
  double c_bar = 0.5 * (cc[2] + cc[3]);
  double rc = rho_bar * c_bar;
  double c2 = c_bar * c_bar;
  // non-zero entries of L and R (Eq. eigen-vectors)
  double L01 = -rc / 2.0, L51 = rc / 2.0, L1p = -1.0 / c2;
  double R00 = 1.0 / c2, R10 = -1.0 / rc, R1l = 1.0 / rc;
  double q[2][NQ];
  int code[2];
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    int order = 5;
    code[side] = 0;
    for (int pass = 0; pass < 2; ++pass) {
      double wt[NQ];
#pragma unroll
      for (int r = 0; r < NQ; ++r) {
        double v[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) v[k] = project<NQ>(qc[side == 0 ? k : 5 - k], r, L01, L1p, L51);
        wt[r] = weno_is<JS>(v[0], v[1], v[2], v[3], v[4], eps, order, weights);
      }
      back_project<NQ>(wt, R00, R10, R1l, q[side]);
      if (!mood || admissible<NQ>(q[side])) break;
      if (pass == 0) {
        order = 3;
        code[side] = 1;
        continue;
      }
      // Eq. (upwind): the upwind cell's primitive state
#pragma unroll
      for (int r = 0; r < NQ; ++r) q[side][r] = qc[2 + side][r];
      code[side] = 2;
    }
  }
  code_l = code[0];
  code_r = code[1];
  hllc<NQ>(q[0], q[1], Fhat, ustar);
}

}  // namespace fp64
}  // namespace ws
