// Op-counting build of the FP64 oracle.
//
// TEST INFRASTRUCTURE ONLY (the measurement's flop count and its tests use
// it; the CUDA library never does).  weno_is_oracle.c is compiled a second
// time, as C++, with its `double` replaced by Real, a double that counts the
// arithmetic performed on it.  Nothing of the oracle is re-typed here: the
// counts are those of the oracle's own code paths.
//
// What counts as one flop: an add, subtract, multiply, divide, square root,
// min, max or comparison of floating-point values.  Not counted: sign changes
// and absolute values (bit operations), constant expressions the compiler
// folds (13.0/12.0), and operations with a trivial operand -- an add or
// subtract with an exact zero, a multiply by an exact zero or +-1.  The
// trivial ones are the products with the structural zeros and ones of the
// characteristic matrices and of the HLLC selection vectors, which the
// oracle applies as dense products; on generic data (no exact zeros or ones
// among the states) they are exactly the operations the method does not need.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <type_traits>

namespace fc {

enum { ADD, MUL, DIV, SQRT, MINMAX, CMP, NKIND };
static long long g_n[NKIND];

struct Real {
  double v;
  Real() = default;
  template <class T, class = typename std::enable_if<std::is_arithmetic<T>::value>::type>
  Real(T x) : v((double)x) {}
  explicit operator double() const { return v; }
  explicit operator int() const { return (int)v; }
};

static inline bool zero(double x) { return x == 0.0; }
static inline bool unit(double x) { return x == 1.0 || x == -1.0; }

static inline Real operator+(Real a, Real b) {
  if (!zero(a.v) && !zero(b.v)) ++g_n[ADD];
  return Real(a.v + b.v);
}
static inline Real operator-(Real a, Real b) {
  if (!zero(a.v) && !zero(b.v)) ++g_n[ADD];
  return Real(a.v - b.v);
}
static inline Real operator*(Real a, Real b) {
  if (!zero(a.v) && !zero(b.v) && !unit(a.v) && !unit(b.v)) ++g_n[MUL];
  return Real(a.v * b.v);
}
static inline Real operator/(Real a, Real b) {
  ++g_n[DIV];
  return Real(a.v / b.v);
}
static inline Real operator-(Real a) { return Real(-a.v); }
static inline Real& operator+=(Real& a, Real b) { return a = a + b; }
static inline Real& operator-=(Real& a, Real b) { return a = a - b; }
static inline Real& operator*=(Real& a, Real b) { return a = a * b; }
#define FC_CMP(op)                                        \
  static inline bool operator op(Real a, Real b) {        \
    ++g_n[CMP];                                           \
    return a.v op b.v;                                    \
  }
FC_CMP(<)
FC_CMP(>)
FC_CMP(<=)
FC_CMP(>=)
FC_CMP(==)
FC_CMP(!=)
#undef FC_CMP
static inline Real sqrt(Real a) {
  ++g_n[SQRT];
  return Real(::sqrt(a.v));
}
static inline Real fabs(Real a) { return Real(::fabs(a.v)); }
static inline Real fmin(Real a, Real b) {
  ++g_n[MINMAX];
  return Real(::fmin(a.v, b.v));
}
static inline Real fmax(Real a, Real b) {
  ++g_n[MINMAX];
  return Real(::fmax(a.v, b.v));
}

#define double Real
#include "weno_is_oracle.c"
#undef double

static void take(long long* out) {
  for (int k = 0; k < NKIND; ++k) {
    out[k] = g_n[k];
    g_n[k] = 0;
  }
}

}  // namespace fc

extern "C" {

// Counts (add, mul, div, sqrt, min/max, compare) of one oracle face
// (projection, reconstruction of both sides, back-projection, MOOD check,
// HLLC) from the sweep-frame primitives qc[6][nq] and sound speeds cc[6].
// levels receives the MOOD orders used (5, 3 or 1) of the two sides.
void fc_face(int nq, const double* qc, const double* cc, double eps, int mood, int weights, long long* counts,
             int* levels) {
  using fc::Real;
  Real q[6 * MAXV], c[6], F[MAXV], us;
  for (int i = 0; i < 6 * nq; ++i) q[i] = Real(qc[i]);
  for (int i = 0; i < 6; ++i) c[i] = Real(cc[i]);
  fc::take(counts);
  fc::or_face(nq, q, c, Real(eps), mood, weights, F, &us, levels, nullptr);
  fc::take(counts);
}

// Counts of one reconstruction (one variable, one side) from v[5].
void fc_weno(const double* v, double eps, int order, int weights, long long* counts) {
  using fc::Real;
  Real w[5];
  for (int i = 0; i < 5; ++i) w[i] = Real(v[i]);
  fc::take(counts);
  fc::or_weno_is(w, Real(eps), order, weights, nullptr);
  fc::take(counts);
}

// Counts of one HLLC flux (Sec. 3.2.1) between the sweep-frame states ql, qr.
void fc_hllc(int nq, const double* ql, const double* qr, long long* counts) {
  using fc::Real;
  Real a[MAXV], b[MAXV], F[MAXV], us;
  for (int i = 0; i < nq; ++i) {
    a[i] = Real(ql[i]);
    b[i] = Real(qr[i]);
  }
  fc::take(counts);
  fc::or_hllc(nq, a, b, F, &us);
  fc::take(counts);
}

// Counts of the per-cell conservative -> primitive recovery and sound speed
// (Sec. 2, Eq. eos) of one cell U[ndim + 4].
void fc_cell_prim(int ndim, const double* U, long long* counts) {
  using fc::Real;
  Real u[MAXV], q[MAXV];
  for (int i = 0; i < ndim + 4; ++i) u[i] = Real(U[i]);
  fc::take(counts);
  fc::or_cons_to_prim(ndim, u, q);
  fc::or_sound_speed(q[0], q[1 + ndim], q[2 + ndim], q[3 + ndim]);
  fc::take(counts);
}

// Counts of a whole oracle flux divergence (or_rhs) and of a whole SSP-RK3
// step (or_step, CFL step included) on a grid of padded state U.  The
// oracle recomputes each stencil cell's primitives for every face; the
// caller separates the per-face, per-cell and per-stage parts.
void fc_rhs_step(int ndim, const int* n, const double* dx, const int* bc, double eps, int mood, int weights,
                 const double* U, long long* rhs_counts, long long* step_counts) {
  using fc::Real;
  fc::or_grid g;
  Real dxr[3] = {Real(dx[0]), Real(ndim > 1 ? dx[1] : 1.0), Real(ndim > 2 ? dx[2] : 1.0)};
  fc::or_grid_set(&g, ndim, n, dxr, bc, Real(eps), mood, weights);
  int64_t N = fc::cells_padded(&g) * (ndim + 4);
  Real* u = (Real*)malloc(sizeof(Real) * (size_t)N);
  Real* L = (Real*)malloc(sizeof(Real) * (size_t)N);
  for (int64_t i = 0; i < N; ++i) u[i] = Real(U[i]);
  fc::or_fill_ghosts(&g, u);
  fc::take(rhs_counts);
  fc::or_rhs(&g, u, L, nullptr);
  fc::take(rhs_counts);
  for (int64_t i = 0; i < N; ++i) u[i] = Real(U[i]);
  fc::take(step_counts);
  fc::or_step(&g, u, Real(0.0), Real(0.5), nullptr);
  fc::take(step_counts);
  free(u);
  free(L);
}

}  // extern "C"
