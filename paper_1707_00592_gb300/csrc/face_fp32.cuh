// Mixed-precision arithmetic of one face i+1/2: characteristic projection
// (Sec. 3.2), WENO-IS of both sides (Secs. 3.3.1, 3.3.2), back-projection,
// MOOD cascade (Sec. 3.4) and stiffened-gas HLLC (Sec. 3.2.1) in FP32 with
// FMA, except the MOOD admissibility test, whose sign is decided exactly
// (as an FP64 evaluation on the FP32 operands would decide it).
//
// FP32-specific choices (the method itself is unchanged):
//  - WENO epsilon is relative: eps_eff = eps_rel * (beta1 + beta2 + tau5) +
//    eps_abs, which keeps tau5/(beta+eps) and its products inside the FP32
//    range for dimensional variables (p ~ 1e9) while acting, like the FP64
//    epsilon, only where a smoothness indicator vanishes;
//  - divisions and square roots use the hardware approximations (about 1 ulp).
#pragma once

#include "ws_internal.h"

namespace ws {
namespace fp32 {

struct WenoParams {
  float eps_rel;  // relative epsilon of WENO-IS
  float eps_abs;  // absolute floor (keeps 0/0 away on flat stencils)
  int weights;    // WS_W_MODIFIED, WS_W_BASIC or WS_W_JS
  float eps_js;   // WS_W_JS: the absolute epsilon of WENO-JS (> 0)
};

// eps: the context's epsilon option (already defaulted).  With WENO-JS it is
// the JS epsilon, and the 3rd-order MOOD level (the scheme's own) takes the
// default relative epsilon of WENO-IS.
inline WenoParams weno_params(float eps, int weights) {
  if (weights == WS_W_JS) return WenoParams{1e-10f, 1e-30f, weights, eps};
  return WenoParams{eps, 1e-30f, weights, 0.0f};
}

// hardware approximations (MUFU): rcp and sqrt to about 1 ulp, no IEEE
// special-case sequences; subnormals flush to zero
__device__ __forceinline__ float frcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float fsqrt(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float fdiv(float a, float b) { return a * frcp(b); }

// FP64 <-> FP32 conversions on the integer pipe (GB300 runs FP64-pipe
// instructions at 1/64 of the FP32 rate).  f64_to_f32: round to nearest
// even in the FP32 normal range, +-0 below it, +-inf above it, NaN kept.
// f32_to_f64: exact (+-0 for zero and subnormal inputs; inf and NaN kept).
__device__ __forceinline__ float f64_to_f32(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  unsigned sign = hi & 0x80000000u, mag = hi & 0x7fffffffu;
  unsigned f = ((mag - (896u << 20)) << 3) | (lo >> 29);
  unsigned rb = (lo >> 28) & 1u, sticky = lo & 0x0fffffffu;
  f += rb & ((sticky != 0u) | (f & 1u));
  f = mag < (897u << 20) ? 0u : f;
  // beyond the FP32 range: +-inf; NaN stays NaN
  f = mag >= (1151u << 20) ? (0x7f800000u | (mag > 0x7ff00000u || (mag == 0x7ff00000u && lo) ? 0x400000u : 0u)) : f;
  return __uint_as_float(sign | f);
}
__device__ __forceinline__ double f32_to_f64(float v) {
  unsigned f = __float_as_uint(v);
  unsigned mag = f & 0x7fffffffu;
  unsigned hi = (f & 0x80000000u) | ((mag >> 3) + (896u << 20));
  unsigned lo = f << 29;
  hi = mag < 0x00800000u ? (f & 0x80000000u) : hi;
  lo = mag < 0x00800000u ? 0u : lo;
  // +-inf and NaN keep their class
  hi = mag >= 0x7f800000u ? ((f & 0x80000000u) | 0x7ff00000u | (mag > 0x7f800000u ? 0x80000u : 0u)) : hi;
  lo = mag >= 0x7f800000u ? 0u : lo;
  return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

// WENO-JS of Jiang & Shu (1996), the paper's comparison scheme: candidates on
// S_0 = {i-2,i-1,i}, S_1 = {i-1,i,i+1}, S_2 = {i,i+1,i+2} (the paper's S_4,
// S_12, S_3), d = (1,6,3)/10, alpha_k = d_k/(eps + beta_k)^2.  In FP32 the
// weights are scaled by (eps + beta_min)^2, which cancels in the
// normalisation and keeps every alpha_k in [0, d_k] for any magnitude of beta.
__device__ __forceinline__ float weno_js(float qm2, float qm1, float q0, float qp1, float qp2, float eps) {
  const float c13_12 = 13.0f / 12.0f;
  float dp1 = qp1 - q0, dm1 = q0 - qm1;
  float a = (q0 - 2.0f * qp1) + qp2;
  float b = ((3.0f * q0) - (4.0f * qp1)) + qp2;
  float e2 = fmaf(c13_12, a * a, fmaf(0.25f, b * b, eps));
  a = (qm2 - 2.0f * qm1) + q0;
  b = (qm2 - (4.0f * qm1)) + (3.0f * q0);
  float e0 = fmaf(c13_12, a * a, fmaf(0.25f, b * b, eps));
  a = (qm1 - 2.0f * q0) + qp1;
  b = qm1 - qp1;
  float e1 = fmaf(c13_12, a * a, fmaf(0.25f, b * b, eps));
  float em = fminf(fminf(e0, e1), e2);
  float r0 = em * frcp(e0), r1 = em * frcp(e1), r2 = em * frcp(e2);
  float a0 = r0 * r0, a1 = 6.0f * (r1 * r1), a2 = 3.0f * (r2 * r2);
  float delta0 = fmaf(1.0f / 3.0f, qm2 - q0, (7.0f / 6.0f) * dm1);
  float delta1 = fmaf(1.0f / 3.0f, dp1, (1.0f / 6.0f) * dm1);
  float delta2 = fmaf(5.0f / 6.0f, dp1, -(1.0f / 6.0f) * (qp2 - q0));
  float num = fmaf(a0, delta0, fmaf(a1, delta1, a2 * delta2));
  return fmaf(num, frcp((a0 + a1) + a2), q0);
}

// Sec. 3.3.1-3.3.2: left value at x_{i+1/2} from q_{i-2..i+2}; order 5 or 3.
// WENO-JS at order 5 goes to weno_js; its 3rd-order level is the scheme's.
__device__ __forceinline__ float weno_is(float qm2, float qm1, float q0, float qp1, float qp2, const WenoParams& P,
                                         int order) {
  if (P.weights == WS_W_JS && order == 5) return weno_js(qm2, qm1, q0, qp1, qp2, P.eps_js);
  const float c13_12 = 13.0f / 12.0f;
  float dp1 = qp1 - q0, dm1 = q0 - qm1;
  float delta1 = 0.5f * dp1;
  float delta2 = 0.5f * dm1;
  float beta1 = dp1 * dp1;
  float beta2 = dm1 * dm1;
  float a = (qm1 - 2.0f * q0) + qp1;
  float b = qm1 - qp1;
  float beta12 = fmaf(c13_12, a * a, 0.25f * (b * b));
  a = ((qp2 - 2.0f * qp1) + 2.0f * qm1) - qm2;
  b = ((((qp2 - 4.0f * qp1) + 6.0f * q0) - 4.0f * qm1) + qm2);
  float tau5 = fmaf(0.25f, a * a, c13_12 * (b * b));
  float eps = fmaf(P.eps_rel, (beta1 + beta2) + tau5, P.eps_abs);
  float r1 = fdiv(tau5, beta1 + eps);
  float r2 = fdiv(tau5, beta2 + eps);
  float alpha1, alpha2;
  if (P.weights != WS_W_BASIC) {
    float r12 = fdiv(tau5, beta12 + eps);
    alpha1 = 4.0f * fmaf(r1, r12, 1.0f);
    alpha2 = 2.0f * fmaf(r2, r12, 1.0f);
  } else {
    alpha1 = 4.0f * (1.0f + r1);
    alpha2 = 2.0f * (1.0f + r2);
  }
  float num = fmaf(alpha1, delta1, alpha2 * delta2);
  float den = alpha1 + alpha2;
  if (order == 5) {
    float d3 = qp2 - q0, d4 = qm2 - q0;
    float delta3 = fmaf(5.0f / 6.0f, dp1, -(1.0f / 6.0f) * d3);
    float delta4 = fmaf(1.0f / 3.0f, d4, (7.0f / 6.0f) * dm1);  // -(7/6)(q_{i-1}-q_i) = (7/6) dm1
    a = (q0 - 2.0f * qp1) + qp2;
    b = ((3.0f * q0) - (4.0f * qp1)) + qp2;
    float beta3 = fmaf(c13_12, a * a, 0.25f * (b * b));
    a = (qm2 - 2.0f * qm1) + q0;
    b = (qm2 - (4.0f * qm1)) + (3.0f * q0);
    float beta4 = fmaf(c13_12, a * a, 0.25f * (b * b));
    float alpha3 = 3.0f * (1.0f + fdiv(tau5, beta3 + eps));
    float alpha4 = 1.0f + fdiv(tau5, beta4 + eps);
    num = fmaf(alpha3, delta3, fmaf(alpha4, delta4, num));
    den = (den + alpha3) + alpha4;
  }
  return fmaf(num, frcp(den), q0);
}

// 5th-order reconstruction with the linear weights d = (4,2,3,1)/10, i.e.
// (2 q_{i-2} - 13 q_{i-1} + 47 q_i + 27 q_{i+1} - 3 q_{i+2})/60, in increment
// form about q_i (a constant stencil reconstructs exactly)
__device__ __forceinline__ float linear5(float qm2, float qm1, float q0, float qp1, float qp2) {
  float t = fmaf(2.0f, qm2 - q0, -13.0f * (qm1 - q0));
  t = fmaf(27.0f, qp1 - q0, t);
  t = fmaf(-3.0f, qp2 - q0, t);
  return fmaf(t, 1.0f / 60.0f, q0);
}

// Paired FP32 arithmetic: one sm_100-family instruction computes both lanes,
// each rounded exactly as its scalar counterpart.  The two sides of a face
// run the same WENO-IS arithmetic on mirrored stencils, so a face
// reconstructs both as one float2 (x: left state, y: right state), which
// halves the issued FP32 instructions of the reconstruction.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }  // exact -b
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(frcp(a.x), frcp(a.y)); }

// weno_js on both lanes
__device__ __forceinline__ float2 js5_pair(float2 qm2, float2 qm1, float2 q0, float2 qp1, float2 qp2, float eps) {
  const float2 c13 = f2(13.0f / 12.0f), half = f2(0.5f), ep = f2(eps);
  float2 dp1 = sub2(qp1, q0), dm1 = sub2(q0, qm1);
  float2 a = add2(fma2(qp1, f2(-2.0f), q0), qp2);
  float2 b = mul2(add2(fma2(qp1, f2(-4.0f), mul2(f2(3.0f), q0)), qp2), half);
  float2 e2 = fma2(c13, mul2(a, a), fma2(b, b, ep));
  a = add2(fma2(qm1, f2(-2.0f), qm2), q0);
  b = mul2(fma2(q0, f2(3.0f), fma2(qm1, f2(-4.0f), qm2)), half);
  float2 e0 = fma2(c13, mul2(a, a), fma2(b, b, ep));
  a = add2(fma2(q0, f2(-2.0f), qm1), qp1);
  b = mul2(sub2(qm1, qp1), half);
  float2 e1 = fma2(c13, mul2(a, a), fma2(b, b, ep));
  float2 em = make_float2(fminf(fminf(e0.x, e1.x), e2.x), fminf(fminf(e0.y, e1.y), e2.y));
  float2 r0 = mul2(em, rcp2(e0)), r1 = mul2(em, rcp2(e1)), r2 = mul2(em, rcp2(e2));
  float2 a0 = mul2(r0, r0), a1 = mul2(f2(6.0f), mul2(r1, r1)), a2 = mul2(f2(3.0f), mul2(r2, r2));
  float2 delta0 = fma2(f2(1.0f / 3.0f), sub2(qm2, q0), mul2(f2(7.0f / 6.0f), dm1));
  float2 delta1 = fma2(f2(1.0f / 3.0f), dp1, mul2(f2(1.0f / 6.0f), dm1));
  float2 delta2 = fma2(f2(5.0f / 6.0f), dp1, mul2(f2(-1.0f / 6.0f), sub2(qp2, q0)));
  float2 num = fma2(a0, delta0, fma2(a1, delta1, mul2(a2, delta2)));
  return fma2(num, rcp2(add2(add2(a0, a1), a2)), q0);
}

// weno_is(..., 5) on both lanes.  Factors of 1/2 and 4 are moved between
// products where the scaling is exact (powers of two), and 3 (1 + r3) is
// formed as one fused multiply-add.
__device__ __forceinline__ float2 weno5_pair(float2 qm2, float2 qm1, float2 q0, float2 qp1, float2 qp2,
                                             const WenoParams& P) {
  if (P.weights == WS_W_JS) return js5_pair(qm2, qm1, q0, qp1, qp2, P.eps_js);
  const float2 c13 = f2(13.0f / 12.0f), one = f2(1.0f), half = f2(0.5f);
  float2 dp1 = sub2(qp1, q0), dm1 = sub2(q0, qm1);
  float2 beta1 = mul2(dp1, dp1);
  float2 beta2 = mul2(dm1, dm1);
  float2 a = add2(fma2(q0, f2(-2.0f), qm1), qp1);  // (q_{i-1} - 2 q_i) + q_{i+1}
  float2 b = mul2(sub2(qm1, qp1), half);
  float2 beta12 = fma2(c13, mul2(a, a), mul2(b, b));
  a = mul2(sub2(fma2(qm1, f2(2.0f), fma2(qp1, f2(-2.0f), qp2)), qm2), half);
  b = add2(fma2(qm1, f2(-4.0f), fma2(q0, f2(6.0f), fma2(qp1, f2(-4.0f), qp2))), qm2);
  float2 tau5 = fma2(a, a, mul2(c13, mul2(b, b)));  // a holds half the scalar form's a
  float2 eps = fma2(f2(P.eps_rel), add2(add2(beta1, beta2), tau5), f2(P.eps_abs));
  float2 r1 = mul2(tau5, rcp2(add2(beta1, eps)));
  float2 r2 = mul2(tau5, rcp2(add2(beta2, eps)));
  float2 alpha1, alpha2;
  if (P.weights != WS_W_BASIC) {
    float2 r12 = mul2(tau5, rcp2(add2(beta12, eps)));
    alpha1 = fma2(mul2(r1, f2(4.0f)), r12, f2(4.0f));  // 4 (1 + r1 r12)
    alpha2 = fma2(add2(r2, r2), r12, f2(2.0f));        // 2 (1 + r2 r12)
  } else {
    alpha1 = fma2(r1, f2(4.0f), f2(4.0f));
    alpha2 = fma2(r2, f2(2.0f), f2(2.0f));
  }
  float2 num = mul2(fma2(alpha1, dp1, mul2(alpha2, dm1)), half);  // alpha1 delta1 + alpha2 delta2
  float2 den = add2(alpha1, alpha2);
  float2 delta3 = fma2(f2(5.0f / 6.0f), dp1, mul2(f2(-1.0f / 6.0f), sub2(qp2, q0)));
  float2 delta4 = fma2(f2(1.0f / 3.0f), sub2(qm2, q0), mul2(f2(7.0f / 6.0f), dm1));
  a = add2(fma2(qp1, f2(-2.0f), q0), qp2);
  b = mul2(add2(fma2(qp1, f2(-4.0f), mul2(f2(3.0f), q0)), qp2), half);
  float2 beta3 = fma2(c13, mul2(a, a), mul2(b, b));
  a = add2(fma2(qm1, f2(-2.0f), qm2), q0);
  b = mul2(fma2(q0, f2(3.0f), fma2(qm1, f2(-4.0f), qm2)), half);
  float2 beta4 = fma2(c13, mul2(a, a), mul2(b, b));
  float2 alpha3 = fma2(mul2(tau5, rcp2(add2(beta3, eps))), f2(3.0f), f2(3.0f));
  float2 alpha4 = fma2(tau5, rcp2(add2(beta4, eps)), one);
  num = fma2(alpha3, delta3, fma2(alpha4, delta4, num));
  den = add2(add2(den, alpha3), alpha4);
  return fma2(num, rcp2(den), q0);
}

// linear5 on both lanes
__device__ __forceinline__ float2 linear5_pair(float2 qm2, float2 qm1, float2 q0, float2 qp1, float2 qp2) {
  float2 t = fma2(f2(2.0f), sub2(qm2, q0), mul2(f2(-13.0f), sub2(qm1, q0)));
  t = fma2(f2(27.0f), sub2(qp1, q0), t);
  t = fma2(f2(-3.0f), sub2(qp2, q0), t);
  return fma2(t, f2(1.0f / 60.0f), q0);
}

__device__ __forceinline__ float sound_speed2(float rho, float p, float Gam, float Pi) {
  return fdiv(fmaf(Gam + 1.0f, p, Pi), Gam * rho);
}

// Exact sign test of (Gamma+1) p + Pi > 0 on FP32 operands: the FP32 value is
// trusted when it clears its rounding-error bound, otherwise the expression
// is evaluated in FP64 (exact for these operands up to the final rounding,
// which preserves the sign).
__device__ __forceinline__ bool pressure_admissible(float Gam, float p, float Pi) {
  float g1 = Gam + 1.0f;
  float t = fmaf(g1, p, Pi);
  float bound = fmaf(4.0e-7f, fabsf(g1 * p) + fabsf(Pi), 1e-37f);
  if (t > bound) return true;
  if (t < -bound) return false;
  double e = ((double)Gam + 1.0) * (double)p + (double)Pi;
  return e > 0.0;
}

template <int NQ>
__device__ __forceinline__ bool admissible(const float* q) {
  return (q[0] > 0.0f) && (q[NQ - 2] > 0.0f) && pressure_admissible(q[NQ - 2], q[NQ - 3], q[NQ - 1]);
}

// admissible<NQ> of both sides of a face at once (sweep-frame primitives,
// x: left state, y: right state): the pressure test as paired FP32 and
// without branches; only a side within the rounding bound goes to FP64.
// The verdicts are those of admissible<NQ> on each side.
template <int NQ>
__device__ __forceinline__ void admissible_pair(const float2 (&Q)[NQ], bool& ok0, bool& ok1) {
  const float2 p = Q[NQ - 3], G = Q[NQ - 2], Pi = Q[NQ - 1];
  const float2 g1 = add2(G, f2(1.0f));
  const float2 t = fma2(g1, p, Pi);
  const float2 gp = mul2(g1, p);
  const float b0 = fmaf(4.0e-7f, fabsf(gp.x) + fabsf(Pi.x), 1e-37f);
  const float b1 = fmaf(4.0e-7f, fabsf(gp.y) + fabsf(Pi.y), 1e-37f);
  bool s0 = t.x > b0, s1 = t.y > b1;
  const bool u0 = !s0 && !(t.x < -b0), u1 = !s1 && !(t.y < -b1);  // within the bound, or NaN
  if (u0 || u1) {
    if (u0) s0 = ((double)G.x + 1.0) * (double)p.x + (double)Pi.x > 0.0;
    if (u1) s1 = ((double)G.y + 1.0) * (double)p.y + (double)Pi.y > 0.0;
  }
  ok0 = (Q[0].x > 0.0f) & (G.x > 0.0f) & s0;
  ok1 = (Q[0].y > 0.0f) & (G.y > 0.0f) & s1;
}

// Characteristic variable r of the sweep-frame primitive q (Eq. eigen-vectors).
template <int NQ>
__device__ __forceinline__ float project(const float* q, int r, float hrc, float ic2) {
  constexpr int NT = NQ - 5, IP = 2 + NT;
  if (r == 0) return 0.5f * fmaf(-2.0f * hrc, q[1], q[IP]) ;
  if (r == 1) return fmaf(-ic2, q[IP], q[0]);
  if (r == NQ - 1) return 0.5f * fmaf(2.0f * hrc, q[1], q[IP]);
  if (r < IP) return q[r];
  return q[r + 1];
}

template <int NQ>
__device__ __forceinline__ void back_project(const float* w, float ic2, float irc, float* q) {
  constexpr int NT = NQ - 5, IP = 2 + NT;
  q[0] = fmaf(ic2, w[0] + w[NQ - 1], w[1]);
  q[1] = irc * (w[NQ - 1] - w[0]);
#pragma unroll
  for (int t = 0; t < NT; ++t) q[2 + t] = w[2 + t];
  q[IP] = w[0] + w[NQ - 1];
  q[IP + 1] = w[IP];
  q[IP + 2] = w[IP + 1];
}

// Sec. 3.2.1 HLLC in FP32.
template <int NQ>
__device__ __forceinline__ void hllc(const float* ql, const float* qr, float* Fhat, float& ustar) {
  constexpr int NT = NQ - 5;
  float U[2][NQ], F[2][NQ], c2[2], cc[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float* q = k == 0 ? ql : qr;
    float rho = q[0], un = q[1], p = q[2 + NT], Gam = q[3 + NT], Pi = q[4 + NT];
    float usq = un * un;
#pragma unroll
    for (int t = 0; t < NT; ++t) usq = fmaf(q[2 + t], q[2 + t], usq);
    float E = fmaf(Gam, p, Pi) + (0.5f * rho) * usq;
    float mn = rho * un;
    U[k][0] = rho;
    U[k][1] = mn;
    F[k][0] = mn;
    F[k][1] = fmaf(mn, un, p);
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
    cc[k] = fsqrt(c2[k]);
  }
  float rl = ql[0], ul = ql[1], pl = ql[2 + NT];
  float rr = qr[0], ur = qr[1], pr = qr[2 + NT];
  float sl = fsqrt(rl), sr = fsqrt(rr);
  float iden = frcp(sl + sr);
  float ubar = fmaf(sl, ul, sr * ur) * iden;
  float du = ur - ul;
  float c2bar = fmaf(sl, c2[0], sr * c2[1]) * iden + (0.5f * (sl * sr) * (iden * iden)) * (du * du);
  float cbar = fsqrt(c2bar);
  float Sl = fminf(fminf(ubar - cbar, ul - cc[0]), 0.0f);
  float Sr = fmaxf(fmaxf(ubar + cbar, ur + cc[1]), 0.0f);
  float ml = rl * (Sl - ul), mr = rr * (Sr - ur);
  float Ss = fdiv(fmaf(ml, ul, pr - pl) - mr * ur, ml - mr);
  float s = (Ss > 0.0f) ? 1.0f : ((Ss < 0.0f) ? -1.0f : 0.0f);
  float wl = 0.5f * (1.0f + s), wr = 0.5f * (1.0f - s);
  float Fs[2][NQ], us[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float* q = k == 0 ? ql : qr;
    float S = k == 0 ? Sl : Sr;
    float rho = q[0], un = q[1], p = q[2 + NT];
    if (S == Ss) {
#pragma unroll
      for (int m = 0; m < NQ; ++m) Fs[k][m] = F[k][m];
      us[k] = un;
    } else {
      float Pk = fmaf(rho * (S - un), Ss - un, p);
      float SP = S * Pk;
      float idS = frcp(S - Ss);
#pragma unroll
      for (int m = 0; m < NQ; ++m) {
        float t = Ss * fmaf(S, U[k][m], -F[k][m]);
        if (m == 1) t += SP;
        if (m == 2 + NT) t = fmaf(SP, Ss, t);
        Fs[k][m] = t * idS;
      }
      us[k] = Ss * (S - un) * idS;
    }
  }
#pragma unroll
  for (int m = 0; m < NQ; ++m) Fhat[m] = fmaf(wl, Fs[0][m], wr * Fs[1][m]);
  ustar = fmaf(wl, us[0], wr * us[1]);
}

// three-operand minimum and maximum (sm_100 family; NaN operands are
// ignored as by fminf / fmaxf)
__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// back_project<NQ> of both sides at once: W[r] = (left, right) characteristic r
template <int NQ>
__device__ __forceinline__ void back_project_pair(const float2 (&W)[NQ], float ic2, float irc, float2 (&Q)[NQ]) {
  constexpr int NT = NQ - 5, IP = 2 + NT;
  float2 s0 = add2(W[0], W[NQ - 1]);
  Q[0] = fma2(f2(ic2), s0, W[1]);
  Q[1] = mul2(f2(irc), sub2(W[NQ - 1], W[0]));
#pragma unroll
  for (int t = 0; t < NT; ++t) Q[2 + t] = W[2 + t];
  Q[IP] = s0;
  Q[IP + 1] = W[IP];
  Q[IP + 2] = W[IP + 1];
}

// hllc<NQ> with the states of both sides in the lanes of Q (x: left, y:
// right).  The per-side quantities (conserved state, physical flux, sound
// speed, star flux) are computed for both sides in paired instructions; the
// wave-speed estimates and the contact speed are scalar.
template <int NQ>
__device__ __forceinline__ void hllc_pair(const float2 (&Q)[NQ], float* Fhat, float& ustar) {
  constexpr int NT = NQ - 5;
  const float2 rho = Q[0], un = Q[1], p = Q[2 + NT], Gam = Q[3 + NT], Pi = Q[4 + NT];
  float2 usq = mul2(un, un);
#pragma unroll
  for (int t = 0; t < NT; ++t) usq = fma2(Q[2 + t], Q[2 + t], usq);
  float2 E = fma2(mul2(f2(0.5f), rho), usq, fma2(Gam, p, Pi));
  float2 mn = mul2(rho, un);
  float2 U[NQ], F[NQ];
  U[0] = rho;
  U[1] = mn;
  F[0] = mn;
  F[1] = fma2(mn, un, p);
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    U[2 + t] = mul2(rho, Q[2 + t]);
    F[2 + t] = mul2(mn, Q[2 + t]);
  }
  U[2 + NT] = E;
  F[2 + NT] = mul2(add2(E, p), un);
  U[3 + NT] = Gam;
  F[3 + NT] = mul2(Gam, un);
  U[4 + NT] = Pi;
  F[4 + NT] = mul2(Pi, un);
  float2 c2 = mul2(fma2(add2(Gam, f2(1.0f)), p, Pi), rcp2(mul2(Gam, rho)));
  float2 cc = make_float2(fsqrt(c2.x), fsqrt(c2.y));
  float sl = fsqrt(rho.x), sr = fsqrt(rho.y);
  float iden = frcp(sl + sr);
  float ubar = fmaf(sl, un.x, sr * un.y) * iden;
  float du = un.y - un.x;
  float c2bar = fmaf(sl, c2.x, sr * c2.y) * iden + (0.5f * (sl * sr) * (iden * iden)) * (du * du);
  float cbar = fsqrt(c2bar);
  float Sl = fmin3(ubar - cbar, un.x - cc.x, 0.0f);
  float Sr = fmax3(ubar + cbar, un.y + cc.y, 0.0f);
  float2 S = make_float2(Sl, Sr);
  float2 Sm = sub2(S, un);
  float2 m = mul2(rho, Sm);
  float Ss = fdiv(fmaf(m.x, un.x, p.y - p.x) - m.y * un.y, m.x - m.y);
  float s = (Ss > 0.0f) ? 1.0f : ((Ss < 0.0f) ? -1.0f : 0.0f);
  float wl = 0.5f * (1.0f + s), wr = 0.5f * (1.0f - s);
  const float2 SS = f2(Ss);
  float2 Pk = fma2(m, sub2(SS, un), p);
  float2 SP = mul2(S, Pk);
  float2 idS = rcp2(sub2(S, SS));
  float2 Fs[NQ];
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    float2 t = mul2(SS, fma2(S, U[k], mul2(F[k], f2(-1.0f))));
    if (k == 1) t = add2(t, SP);
    if (k == 2 + NT) t = fma2(SP, SS, t);
    Fs[k] = mul2(t, idS);
  }
  float2 us = mul2(mul2(SS, Sm), idS);
  if (Sl == Ss || Sr == Ss) {  // a wave speed equal to the contact: that side's flux is its physical flux
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      if (Sl == Ss) Fs[k].x = F[k].x;
      if (Sr == Ss) Fs[k].y = F[k].y;
    }
    if (Sl == Ss) us.x = un.x;
    if (Sr == Ss) us.y = un.y;
  }
#pragma unroll
  for (int k = 0; k < NQ; ++k) Fhat[k] = fmaf(wl, Fs[k].x, wr * Fs[k].y);
  ustar = fmaf(wl, us.x, wr * us.y);
}

// One face from sweep-frame FP32 primitives of cells i-2..i+3 and their sound
// speeds.  code_l / code_r: 0, 1, 2 for 5th, 3rd, 1st order.
template <int NQ>
__device__ __forceinline__ void face(const float (&qc)[6][NQ], const float (&cc)[6], const WenoParams& P, int mood,
                                     float* Fhat, float& ustar, int& code_l, int& code_r) {
  float rho_bar = 0.5f * (qc[2][0] + qc[3][0]);
  float c_bar = 0.5f * (cc[2] + cc[3]);
  float rc = rho_bar * c_bar;
  float hrc = 0.5f * rc;
  float ic2 = frcp(c_bar * c_bar);
  float irc = frcp(rc);
  float q[2][NQ];
  int code[2];
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    int order = 5;
    code[side] = 0;
    for (int pass = 0; pass < 2; ++pass) {
      float wt[NQ];
#pragma unroll
      for (int r = 0; r < NQ; ++r) {
        float v[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) v[k] = project<NQ>(qc[side == 0 ? k : 5 - k], r, hrc, ic2);
        wt[r] = weno_is(v[0], v[1], v[2], v[3], v[4], P, order);
      }
      back_project<NQ>(wt, ic2, irc, q[side]);
      if (!mood || admissible<NQ>(q[side])) break;
      if (pass == 0) {
        order = 3;
        code[side] = 1;
        continue;
      }
#pragma unroll
      for (int r = 0; r < NQ; ++r) q[side][r] = qc[2 + side][r];
      code[side] = 2;
    }
  }
  code_l = code[0];
  code_r = code[1];
  hllc<NQ>(q[0], q[1], Fhat, ustar);
}

}  // namespace fp32
}  // namespace ws
