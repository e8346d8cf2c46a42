// Cell-wise kernels of the solver: ghost layers, conservative <-> primitive
// conversion, the CFL reduction, the flux-divergence + SSP-RK3 update and the
// MOOD counters.  Built with -fmad=false: every FP64 operation rounds once,
// in the order written, so that the FP64 path reproduces a plain IEEE
// evaluation of the same formulas bit for bit.
#include <cuda_runtime.h>

#include "ws_internal.h"

namespace ws {

namespace {

constexpr int BS = 256;

inline int blocks_for(int64_t n, int bs = BS) {
  int64_t b = (n + bs - 1) / bs;
  if (b > (1LL << 30)) b = 1LL << 30;
  return (int)(b < 1 ? 1 : b);
}

// Sec. 2, Eq. (eos): rho e = Gamma p + Pi.
__device__ __forceinline__ void cons_to_prim(int ndim, const double* U, double* q) {
  double rho = U[0];
  double usq = 0.0;
  q[0] = rho;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (d < ndim) {
      double u = U[1 + d] / rho;
      q[1 + d] = u;
      usq = usq + u * u;
    }
  }
  double ke = (0.5 * rho) * usq;
  double E = U[1 + ndim], Gam = U[2 + ndim], Pi = U[3 + ndim];
  q[1 + ndim] = ((E - ke) - Pi) / Gam;
  q[2 + ndim] = Gam;
  q[3 + ndim] = Pi;
}

__device__ __forceinline__ double sound_speed2(double rho, double p, double Gam, double Pi) {
  return (((Gam + 1.0) * p) + Pi) / (Gam * rho);
}

__device__ __forceinline__ bool admissible(double rho, double p, double Gam, double Pi) {
  return (rho > 0.0) && (Gam > 0.0) && ((((Gam + 1.0) * p) + Pi) > 0.0);
}

// padded coordinates of linear index i
__device__ __forceinline__ void coords(const GridDev& g, int64_t i, int64_t c[3]) {
  c[0] = i % g.P[0];
  int64_t r = i / g.P[0];
  c[1] = r % g.P[1];
  c[2] = r / g.P[1];
}

// ---------------------------------------------------------------------------
// ghost layers of direction d at interior transverse positions
__global__ void k_ghost(GridDev g, double* __restrict__ U, int d) {
  int e1 = (d == 0) ? 1 : 0;
  int e2 = (d == 2) ? 1 : 2;
  int64_t T1 = g.n[e1], T2 = g.n[e2];
  int64_t total = T1 * T2 * 2 * NG;
  int n = g.n[d];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t a1 = t % T1;
    int64_t r = t / T1;
    int64_t a2 = r % T2;
    r /= T2;
    int gI = (int)(r % NG) + 1;
    int side = (int)(r / NG);
    int kind = g.bc[d][side];
    int64_t dst = side == 0 ? (NG - gI) : (NG + n - 1 + gI);
    int64_t src;
    if (kind == WS_BC_PERIODIC)
      src = side == 0 ? (NG + n - gI) : (NG + gI - 1);
    else if (kind == WS_BC_REFLECTIVE)
      src = side == 0 ? (NG + gI - 1) : (NG + n - gI);
    else
      src = side == 0 ? NG : (NG + n - 1);
    // unused axes have extent 1 and ghost offset 0, so they add nothing
    int64_t base = (g.G[e1] + a1) * g.st[e1] + (g.G[e2] + a2) * g.st[e2];
    int64_t id = base + dst * g.st[d], is = base + src * g.st[d];
    for (int f = 0; f < g.nv; ++f) {
      double v = U[f * g.N + is];
      if (kind == WS_BC_REFLECTIVE && f == 1 + d) v = -v;
      U[f * g.N + id] = v;
    }
  }
}

// primitives + sound speed of every cell the sweeps read (at most one
// coordinate outside the interior)
__global__ void k_prim(GridDev g, const double* __restrict__ U, double* __restrict__ Q) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t c[3];
    coords(g, i, c);
    int out = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (d < g.ndim && (c[d] < NG || c[d] >= NG + g.n[d])) ++out;
    if (out > 1) continue;
    double u[MAXV], q[MAXV];
    for (int f = 0; f < g.nv; ++f) u[f] = U[f * g.N + i];
    cons_to_prim(g.ndim, u, q);
    for (int f = 0; f < g.nv; ++f) Q[f * g.N + i] = q[f];
    int nd = g.ndim;
    Q[g.nv * g.N + i] = sqrt(sound_speed2(q[0], q[1 + nd], q[2 + nd], q[3 + nd]));
  }
}

__global__ void k_prim_to_cons(GridDev g, const double* __restrict__ Q, double* __restrict__ U) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N; i += (int64_t)gridDim.x * blockDim.x) {
    int nd = g.ndim;
    double rho = Q[i];
    double usq = 0.0;
    U[i] = rho;
    for (int d = 0; d < nd; ++d) {
      double u = Q[(1 + d) * g.N + i];
      U[(1 + d) * g.N + i] = rho * u;
      usq = usq + u * u;
    }
    double ke = (0.5 * rho) * usq;
    double p = Q[(1 + nd) * g.N + i], Gam = Q[(2 + nd) * g.N + i], Pi = Q[(3 + nd) * g.N + i];
    U[(1 + nd) * g.N + i] = ((Gam * p) + Pi) + ke;
    U[(2 + nd) * g.N + i] = Gam;
    U[(3 + nd) * g.N + i] = Pi;
  }
}

__global__ void k_cons_to_prim_all(GridDev g, const double* __restrict__ U, double* __restrict__ Q) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N; i += (int64_t)gridDim.x * blockDim.x) {
    double u[MAXV], q[MAXV];
    for (int f = 0; f < g.nv; ++f) u[f] = U[f * g.N + i];
    cons_to_prim(g.ndim, u, q);
    for (int f = 0; f < g.nv; ++f) Q[f * g.N + i] = q[f];
  }
}

// max over interior cells of sum_d (|u_d| + c)/dx_d; non-negative doubles
// order like their bit patterns, so the max is an integer atomicMax.
__global__ void k_cfl(GridDev g, const double* __restrict__ Q, unsigned long long* lmax) {
  double best = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < g.ncell; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t x = t % g.n[0];
    int64_t r = t / g.n[0];
    int64_t y = r % g.n[1];
    int64_t z = r / g.n[1];
    int64_t i = (g.G[0] + x) * g.st[0] + (g.G[1] + y) * g.st[1] + (g.G[2] + z) * g.st[2];
    double c = Q[g.nv * g.N + i];
    double lam = 0.0;
    for (int d = 0; d < g.ndim; ++d) lam = lam + (fabs(Q[(1 + d) * g.N + i]) + c) / g.dx[d];
    // NaN propagates (it orders above +inf as bits)
    if (!(lam <= best)) best = lam;
  }
  unsigned long long b = (unsigned long long)__double_as_longlong(best);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long v = __shfl_xor_sync(0xffffffffu, b, o);
    b = v > b ? v : b;
  }
  __shared__ unsigned long long sm[32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sm[w] = b;
  __syncthreads();
  if (w == 0) {
    b = lane < (int)(blockDim.x >> 5) ? sm[lane] : 0ULL;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long v = __shfl_xor_sync(0xffffffffu, b, o);
      b = v > b ? v : b;
    }
    if (lane == 0) atomicMax(lmax, b);
  }
}

__global__ void k_set_dt(double dt_fixed, double cfl, const unsigned long long* __restrict__ lmax,
                         double* __restrict__ dt, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (dt_fixed > 0.0)
      dt[i] = dt_fixed;
    else
      dt[i] = cfl / __longlong_as_double((long long)lmax[i]);
  }
}

// Sec. 3.1: L(U) summed over x, y, z, then the SSP-RK3 stage.
// stage -1: write L itself; 0, 1, 2: the three Shu-Osher stages.  Uout may
// alias Un or Us (each thread reads its cell before writing it).
template <typename FT>
__global__ void k_update(GridDev g, int stage, const double* Un, const double* Us, double* Uout, const FT* __restrict__ F0, const FT* __restrict__ F1,
                         const FT* __restrict__ F2, const FT* __restrict__ u0, const FT* __restrict__ u1,
                         const FT* __restrict__ u2, const double* __restrict__ dtp, unsigned long long* nbad) {
  const FT* Fd[3] = {F0, F1, F2};
  const FT* ud[3] = {u0, u1, u2};
  const double c13 = 1.0 / 3.0, c23 = 2.0 / 3.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < g.ncell; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t a[3];
    a[0] = t % g.n[0];
    int64_t r = t / g.n[0];
    a[1] = r % g.n[1];
    a[2] = r / g.n[1];
    int64_t i = (g.G[0] + a[0]) * g.st[0] + (g.G[1] + a[1]) * g.st[1] + (g.G[2] + a[2]) * g.st[2];
    int64_t fl[3], fr[3];
    double du[3];
    for (int d = 0; d < g.ndim; ++d) {
      int64_t b[3] = {a[0], a[1], a[2]};
      fl[d] = (b[2] * g.fe[d][1] + b[1]) * g.fe[d][0] + b[0];
      b[d] += 1;
      fr[d] = (b[2] * g.fe[d][1] + b[1]) * g.fe[d][0] + b[0];
      du[d] = (double)ud[d][fr[d]] - (double)ud[d][fl[d]];
    }
    double dt = stage >= 0 ? dtp[0] : 0.0;
    double out[MAXV];
    for (int f = 0; f < g.nv; ++f) {
      double L = 0.0;
      double phi = Us[f * g.N + i];
      for (int d = 0; d < g.ndim; ++d) {
        int64_t nf = g.nfaces[d];
        double dF = (double)Fd[d][f * nf + fr[d]] - (double)Fd[d][f * nf + fl[d]];
        double term = -(dF / g.dx[d]);
        if (f >= 2 + g.ndim) term = term + phi * (du[d] / g.dx[d]);
        L = L + term;
      }
      double o;
      if (stage < 0) {
        o = L;
      } else {
        double un = Un[f * g.N + i];
        if (stage == 0)
          o = un + dt * L;
        else if (stage == 1)
          o = (0.75 * un) + (0.25 * (phi + dt * L));
        else
          o = (c13 * un) + (c23 * (phi + dt * L));
      }
      out[f] = o;
    }
    for (int f = 0; f < g.nv; ++f) Uout[f * g.N + i] = out[f];
    if (stage == 2) {
      double q[MAXV];
      cons_to_prim(g.ndim, out, q);
      int nd = g.ndim;
      if (!admissible(q[0], q[1 + nd], q[2 + nd], q[3 + nd])) atomicAdd(nbad, 1ULL);
    }
  }
}

__global__ void k_mood_count(const uint8_t* __restrict__ mask, int64_t n, int64_t nstage,
                             const int64_t* __restrict__ dir_off, int ndim, unsigned long long* counts) {
  __shared__ unsigned long long sc[9];
  if (threadIdx.x < 9) sc[threadIdx.x] = 0;
  __syncthreads();
  unsigned long long loc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  int64_t total = n * nstage;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t k = t % n;
    int d = 0;
    for (int e = 1; e < ndim; ++e)
      if (k >= dir_off[e]) d = e;
    uint8_t m = mask[t];
    int cl = m & 3, cr = (m >> 2) & 3;
    if (cl < 3) loc[3 * d + cl]++;
    if (cr < 3) loc[3 * d + cr]++;
  }
  for (int j = 0; j < 9; ++j)
    if (loc[j]) atomicAdd(&sc[j], loc[j]);
  __syncthreads();
  if (threadIdx.x < 9 && sc[threadIdx.x]) atomicAdd(&counts[threadIdx.x], sc[threadIdx.x]);
}

}  // namespace

void launch_ghost(const GridDev& g, double* U, int d, cudaStream_t s) {
  int e1 = (d == 0) ? 1 : 0, e2 = (d == 2) ? 1 : 2;
  int64_t total = (int64_t)g.n[e1] * g.n[e2] * 2 * NG;
  k_ghost<<<blocks_for(total), BS, 0, s>>>(g, U, d);
}

void launch_prim(const GridDev& g, const double* U, double* Q, cudaStream_t s) {
  k_prim<<<blocks_for(g.N), BS, 0, s>>>(g, U, Q);
}

void launch_prim_to_cons(const GridDev& g, const double* Q, double* U, cudaStream_t s) {
  k_prim_to_cons<<<blocks_for(g.N), BS, 0, s>>>(g, Q, U);
}

void launch_cons_to_prim_all(const GridDev& g, const double* U, double* Q, cudaStream_t s) {
  k_cons_to_prim_all<<<blocks_for(g.N), BS, 0, s>>>(g, U, Q);
}

void launch_cfl(const GridDev& g, const double* Q, unsigned long long* lmax, cudaStream_t s) {
  int b = blocks_for(g.ncell);
  if (b > 152 * 8) b = 152 * 8;
  k_cfl<<<b, BS, 0, s>>>(g, Q, lmax);
}

void launch_set_dt(const double*, double dt_fixed, double cfl, const unsigned long long* lmax, double* dt_dev,
                   int64_t n, cudaStream_t s) {
  k_set_dt<<<blocks_for(n), BS, 0, s>>>(dt_fixed, cfl, lmax, dt_dev, n);
}

void launch_update(const GridDev& g, int stage, const double* Un, const double* Us, double* Uout,
                   double* const Fh[3], double* const us[3], const double* dt_dev, unsigned long long* nbad,
                   cudaStream_t s) {
  k_update<double><<<blocks_for(g.ncell), BS, 0, s>>>(g, stage, Un, Us, Uout, Fh[0], Fh[1], Fh[2], us[0], us[1],
                                                      us[2], dt_dev, nbad);
}

void launch_mood_count(const uint8_t* mask, int64_t n, int64_t nstage, const int64_t* dir_off, int ndim,
                       unsigned long long* counts, cudaStream_t s) {
  int b = blocks_for(n * nstage);
  if (b > 152 * 4) b = 152 * 4;
  k_mood_count<<<b, BS, 0, s>>>(mask, n, nstage, dir_off, ndim, counts);
}

}  // namespace ws
