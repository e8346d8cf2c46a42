// Mixed-precision sweep: FP32 projection, WENO-IS and HLLC (face_fp32.cuh),
// FP64 where accuracy needs it -- the pressure recovery's E - Pi
// cancellation, the sign of the MOOD admissibility test, and the
// conservative SSP-RK3 accumulation of the FP64 state.
//
// Generic form (any dimension): primitive cache in FP32 (k_prim32), one face
// sweep per direction (k_face32) writing FP32 fluxes, and the update
// (k_update_mixed) that forms L(U) in FP32 and accumulates the RK stage in
// FP64.
#include <cuda_runtime.h>

#include "face_fp32.cuh"
#include "ws_internal.h"

namespace ws {

namespace {

using namespace fp32;

constexpr int BS = 256;

inline int blocks_for(int64_t n, int bs = BS) {
  int64_t b = (n + bs - 1) / bs;
  if (b > (1LL << 30)) b = 1LL << 30;
  return (int)(b < 1 ? 1 : b);
}

// Conservative FP64 -> FP32 primitives: the internal energy E - Pi is formed
// in FP64 (for water Pi ~ 7.8e8 dwarfs Gamma p at p ~ 1e5), the rest in FP32.
template <int NDIM>
__device__ __forceinline__ void cons_to_prim32(const double* U, float* q, float& c) {
  float rho = (float)U[0];
  float irho = frcp(rho);
  float usq = 0.0f;
  q[0] = rho;
#pragma unroll
  for (int d = 0; d < NDIM; ++d) {
    float u = (float)U[1 + d] * irho;
    q[1 + d] = u;
    usq = fmaf(u, u, usq);
  }
  float Gam = (float)U[2 + NDIM], Pi = (float)U[3 + NDIM];
  float eint = (float)(U[1 + NDIM] - U[3 + NDIM]);  // E - Pi in FP64
  float p = fmaf(-0.5f * rho, usq, eint) * frcp(Gam);
  q[1 + NDIM] = p;
  q[2 + NDIM] = Gam;
  q[3 + NDIM] = Pi;
  c = fsqrt(sound_speed2(rho, p, Gam, Pi));
}

template <int NDIM>
__global__ void k_prim32(GridDev g, const double* __restrict__ U, float* __restrict__ Q) {
  constexpr int NV = NDIM + 4;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t c3[3];
    c3[0] = i % g.P[0];
    int64_t r = i / g.P[0];
    c3[1] = r % g.P[1];
    c3[2] = r / g.P[1];
    int out = 0;
#pragma unroll
    for (int d = 0; d < NDIM; ++d)
      if (c3[d] < NG || c3[d] >= NG + g.n[d]) ++out;
    if (out > 1) continue;
    double u[NV];
#pragma unroll
    for (int f = 0; f < NV; ++f) u[f] = U[f * g.N + i];
    float q[NV], c;
    cons_to_prim32<NDIM>(u, q, c);
#pragma unroll
    for (int f = 0; f < NV; ++f) Q[f * g.N + i] = q[f];
    Q[NV * g.N + i] = c;
  }
}

template <int NDIM>
__global__ void __launch_bounds__(128) k_face32(GridDev g, int d, const float* __restrict__ Q, float* __restrict__ Fh,
                                                float* __restrict__ us, uint8_t* __restrict__ mask, WenoParams P,
                                                int mood) {
  constexpr int NQ = NDIM + 4;
  const int64_t nf = g.nfaces[d];
  const int64_t fe0 = g.fe[d][0], fe1 = g.fe[d][1];
  const int64_t N = g.N;
  int fld[NQ];
  fld[0] = 0;
  fld[1] = 1 + d;
  {
    int k = 2;
#pragma unroll
    for (int e = 0; e < NDIM; ++e)
      if (e != d) fld[k++] = 1 + e;
  }
  fld[NQ - 3] = 1 + NDIM;
  fld[NQ - 2] = 2 + NDIM;
  fld[NQ - 1] = 3 + NDIM;
  const int64_t sd = g.st[d];
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
    int64_t c[3];
    c[0] = f % fe0;
    int64_t r = f / fe0;
    c[1] = r % fe1;
    c[2] = r / fe1;
    c[d] -= 1;
    int64_t base = (g.G[0] + c[0]) * g.st[0] + (g.G[1] + c[1]) * g.st[1] + (g.G[2] + c[2]) * g.st[2];
    float qc[6][NQ], cc[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      int64_t idx = base + (j - 2) * sd;
#pragma unroll
      for (int m = 0; m < NQ; ++m) qc[j][m] = Q[fld[m] * N + idx];
      cc[j] = Q[NQ * N + idx];
    }
    float Fhat[NQ], ustar;
    int cl, cr;
    face<NQ>(qc, cc, P, mood, Fhat, ustar, cl, cr);
#pragma unroll
    for (int m = 0; m < NQ; ++m) Fh[fld[m] * nf + f] = Fhat[m];
    us[f] = ustar;
    if (mask) mask[f] = (uint8_t)(cl | (cr << 2));
  }
}

// RK stage of one cell from its L in FP32: FP64 accumulation.
__device__ __forceinline__ double rk_stage(int stage, double un, double us, float incr) {
  double di = (double)incr;
  if (stage == 0) return un + di;
  if (stage == 1) return fma(0.75, un, 0.25 * (us + di));
  return fma(1.0 / 3.0, un, (2.0 / 3.0) * (us + di));
}

// division-free FP64 admissibility of a conservative state:
// rho > 0, Gamma > 0 and (Gamma+1)(rho E - |m|^2/2) - rho Pi > 0
template <int NDIM>
__device__ __forceinline__ bool admissible_cons(const double* o) {
  double rho = o[0], Gam = o[2 + NDIM], Pi = o[3 + NDIM];
  double m2 = 0.0;
#pragma unroll
  for (int d = 0; d < NDIM; ++d) m2 = fma(o[1 + d], o[1 + d], m2);
  double t = fma(rho, o[1 + NDIM], -0.5 * m2);
  return rho > 0.0 && Gam > 0.0 && fma(Gam + 1.0, t, -rho * Pi) > 0.0;
}

template <int NDIM>
__global__ void k_update_mixed(GridDev g, int stage, const double* Un, const double* Us, double* Uout,
                               const float* __restrict__ F0, const float* __restrict__ F1,
                               const float* __restrict__ F2, const float* __restrict__ u0,
                               const float* __restrict__ u1, const float* __restrict__ u2,
                               const float* __restrict__ Q, const double* __restrict__ dtp,
                               unsigned long long* nbad) {
  constexpr int NV = NDIM + 4;
  const float* Fd[3] = {F0, F1, F2};
  const float* ud[3] = {u0, u1, u2};
  float idx_[3];
#pragma unroll
  for (int d = 0; d < NDIM; ++d) idx_[d] = (float)(1.0 / g.dx[d]);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < g.ncell; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t a[3];
    a[0] = t % g.n[0];
    int64_t r = t / g.n[0];
    a[1] = r % g.n[1];
    a[2] = r / g.n[1];
    int64_t i = (g.G[0] + a[0]) * g.st[0] + (g.G[1] + a[1]) * g.st[1] + (g.G[2] + a[2]) * g.st[2];
    int64_t fl[3], fr[3];
    float du[3];
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
      int64_t b[3] = {a[0], a[1], a[2]};
      fl[d] = (b[2] * g.fe[d][1] + b[1]) * g.fe[d][0] + b[0];
      b[d] += 1;
      fr[d] = (b[2] * g.fe[d][1] + b[1]) * g.fe[d][0] + b[0];
      du[d] = (ud[d][fr[d]] - ud[d][fl[d]]) * idx_[d];
    }
    float dt = stage >= 0 ? (float)dtp[0] : 1.0f;
    double out[NV];
#pragma unroll
    for (int f = 0; f < NV; ++f) {
      float L = 0.0f;
#pragma unroll
      for (int d = 0; d < NDIM; ++d) {
        int64_t nf = g.nfaces[d];
        L = fmaf(-(Fd[d][f * nf + fr[d]] - Fd[d][f * nf + fl[d]]), idx_[d], L);
      }
      if (f >= 2 + NDIM) {
        float phi = Q[f * g.N + i];
        float s = 0.0f;
#pragma unroll
        for (int d = 0; d < NDIM; ++d) s += du[d];
        L = fmaf(phi, s, L);
      }
      if (stage < 0)
        out[f] = (double)L;
      else
        out[f] = rk_stage(stage, Un[f * g.N + i], Us[f * g.N + i], dt * L);
    }
#pragma unroll
    for (int f = 0; f < NV; ++f) Uout[f * g.N + i] = out[f];
    if (stage == 2 && !admissible_cons<NDIM>(out)) atomicAdd(nbad, 1ULL);
  }
}

// max over interior cells of sum_d (|u_d| + c)/dx_d from the FP32 cache
template <int NDIM>
__global__ void k_cfl32(GridDev g, const float* __restrict__ Q, unsigned long long* lmax) {
  constexpr int NV = NDIM + 4;
  float idx_[3];
#pragma unroll
  for (int d = 0; d < NDIM; ++d) idx_[d] = (float)(1.0 / g.dx[d]);
  float best = 0.0f;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < g.ncell; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t x = t % g.n[0];
    int64_t r = t / g.n[0];
    int64_t y = r % g.n[1];
    int64_t z = r / g.n[1];
    int64_t i = (g.G[0] + x) * g.st[0] + (g.G[1] + y) * g.st[1] + (g.G[2] + z) * g.st[2];
    float c = Q[NV * g.N + i];
    float lam = 0.0f;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) lam = fmaf(fabsf(Q[(1 + d) * g.N + i]) + c, idx_[d], lam);
    if (!(lam <= best)) best = lam;  // NaN propagates
  }
  unsigned long long b = (unsigned long long)__double_as_longlong((double)best);
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

// CFL reduction straight from the FP64 state (no primitive cache)
template <int NDIM>
__global__ void k_cfl_u(GridDev g, const double* __restrict__ U, unsigned long long* lmax) {
  constexpr int NV = NDIM + 4;
  float idx_[3];
#pragma unroll
  for (int d = 0; d < NDIM; ++d) idx_[d] = (float)(1.0 / g.dx[d]);
  float best = 0.0f;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < g.ncell; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t x = t % g.n[0];
    int64_t r = t / g.n[0];
    int64_t y = r % g.n[1];
    int64_t z = r / g.n[1];
    int64_t i = (g.G[0] + x) * g.st[0] + (g.G[1] + y) * g.st[1] + (g.G[2] + z) * g.st[2];
    double u[NV];
#pragma unroll
    for (int f = 0; f < NV; ++f) u[f] = U[f * g.N + i];
    float q[NV], c;
    cons_to_prim32<NDIM>(u, q, c);
    float lam = 0.0f;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) lam = fmaf(fabsf(q[1 + d]) + c, idx_[d], lam);
    if (!(lam <= best)) best = lam;
  }
  unsigned long long b = (unsigned long long)__double_as_longlong((double)best);
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

}  // namespace

void launch_cfl_u(const GridDev& g, const double* U, unsigned long long* lmax, cudaStream_t s) {
  int b = blocks_for(g.ncell);
  if (b > 152 * 8) b = 152 * 8;
  switch (g.ndim) {
    case 1: k_cfl_u<1><<<b, BS, 0, s>>>(g, U, lmax); break;
    case 2: k_cfl_u<2><<<b, BS, 0, s>>>(g, U, lmax); break;
    default: k_cfl_u<3><<<b, BS, 0, s>>>(g, U, lmax); break;
  }
}

void launch_cfl32(const GridDev& g, const float* Q, unsigned long long* lmax, cudaStream_t s) {
  int b = blocks_for(g.ncell);
  if (b > 152 * 8) b = 152 * 8;
  switch (g.ndim) {
    case 1: k_cfl32<1><<<b, BS, 0, s>>>(g, Q, lmax); break;
    case 2: k_cfl32<2><<<b, BS, 0, s>>>(g, Q, lmax); break;
    default: k_cfl32<3><<<b, BS, 0, s>>>(g, Q, lmax); break;
  }
}

void launch_prim32(const GridDev& g, const double* U, float* Q, cudaStream_t s) {
  int b = blocks_for(g.N);
  switch (g.ndim) {
    case 1: k_prim32<1><<<b, BS, 0, s>>>(g, U, Q); break;
    case 2: k_prim32<2><<<b, BS, 0, s>>>(g, U, Q); break;
    default: k_prim32<3><<<b, BS, 0, s>>>(g, U, Q); break;
  }
}

void launch_face_mixed(const GridDev& g, int d, const float* Q, float* Fh, float* us, uint8_t* mask, float eps_rel,
                       int mood, int weights, cudaStream_t s) {
  WenoParams P = weno_params(eps_rel, weights);
  int b = blocks_for(g.nfaces[d], 128);
  switch (g.ndim) {
    case 1: k_face32<1><<<b, 128, 0, s>>>(g, d, Q, Fh, us, mask, P, mood); break;
    case 2: k_face32<2><<<b, 128, 0, s>>>(g, d, Q, Fh, us, mask, P, mood); break;
    default: k_face32<3><<<b, 128, 0, s>>>(g, d, Q, Fh, us, mask, P, mood); break;
  }
}

void launch_update_mixed(const GridDev& g, int stage, const double* Un, const double* Us, double* Uout,
                         float* const Fh[3], float* const us[3], const float* Q, const double* dt_dev,
                         unsigned long long* nbad, cudaStream_t s) {
  int b = blocks_for(g.ncell);
  switch (g.ndim) {
    case 1:
      k_update_mixed<1><<<b, BS, 0, s>>>(g, stage, Un, Us, Uout, Fh[0], Fh[1], Fh[2], us[0], us[1], us[2], Q, dt_dev,
                                         nbad);
      break;
    case 2:
      k_update_mixed<2><<<b, BS, 0, s>>>(g, stage, Un, Us, Uout, Fh[0], Fh[1], Fh[2], us[0], us[1], us[2], Q, dt_dev,
                                         nbad);
      break;
    default:
      k_update_mixed<3><<<b, BS, 0, s>>>(g, stage, Un, Us, Uout, Fh[0], Fh[1], Fh[2], us[0], us[1], us[2], Q, dt_dev,
                                         nbad);
      break;
  }
}

}  // namespace ws
