// Batched independent 1D Riemann tubes of uneven length in single launches.
// Tube t owns padded cells [off[t], off[t+1]) of every field (3 ghost cells
// at each end, transmissive), has len = off[t+1]-off[t]-6 interior cells,
// dx = 1/len and its own CFL step.  Every kernel maps one thread to one padded
// cell of the concatenation, so uneven lengths cost no idle lanes beyond the
// 6 ghost cells of each tube.  Built with -fmad=false; the face arithmetic is
// the FP64 face of the grid sweep.
#include <cuda_runtime.h>

#include "face_fp64.cuh"
#include "ws_internal.h"

namespace ws {

namespace {

using namespace fp64;

constexpr int BS = 256;

inline int blocks_for(int64_t n, int bs = BS) {
  int64_t b = (n + bs - 1) / bs;
  if (b > (1LL << 30)) b = 1LL << 30;
  return (int)(b < 1 ? 1 : b);
}

__global__ void k_tubes_ghost(TubesDev t, double* __restrict__ U) {
  int64_t total = t.ntubes * 2 * NG;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t tube = k / (2 * NG);
    int r = (int)(k % (2 * NG));
    int side = r / NG, gI = r % NG + 1;
    int64_t a = t.off[tube], b = t.off[tube + 1];
    int64_t dst = side == 0 ? a + NG - gI : b - NG - 1 + gI;
    int64_t src = side == 0 ? a + NG : b - NG - 1;
    for (int f = 0; f < 5; ++f) U[f * t.total + dst] = U[f * t.total + src];
  }
}

__global__ void k_tubes_prim(TubesDev t, const double* __restrict__ U, double* __restrict__ Q) {
  const int64_t N = t.total;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double rho = U[i];
    double u = U[N + i] / rho;
    double usq = 0.0;
    usq = usq + u * u;
    double ke = (0.5 * rho) * usq;
    double E = U[2 * N + i], Gam = U[3 * N + i], Pi = U[4 * N + i];
    double p = ((E - ke) - Pi) / Gam;
    Q[i] = rho;
    Q[N + i] = u;
    Q[2 * N + i] = p;
    Q[3 * N + i] = Gam;
    Q[4 * N + i] = Pi;
    Q[5 * N + i] = sqrt(sound_speed2(rho, p, Gam, Pi));
  }
}

// per-tube max of (|u| + c)/dx: one atomic per warp when the warp lies in one tube
__global__ void k_tubes_cfl(TubesDev t, const double* __restrict__ Q, unsigned long long* lmax) {
  const int64_t N = t.total;
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x; i0 < N; i0 += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = i0 + threadIdx.x;
    int tube = -1;
    unsigned long long b = 0;
    if (i < N) {
      tube = t.cell_tube[i];
      int64_t a = t.off[tube], e = t.off[tube + 1];
      if (i >= a + NG && i < e - NG) {
        double dx = 1.0 / (double)(e - a - 2 * NG);
        double lam = 0.0;
        lam = lam + (fabs(Q[N + i]) + Q[5 * N + i]) / dx;
        b = (unsigned long long)__double_as_longlong(lam);
      }
    }
    unsigned active = __activemask();
    int t0 = __shfl_sync(active, tube, 0);
    bool same = __all_sync(active, tube == t0);
    if (same) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        unsigned long long v = __shfl_xor_sync(active, b, o);
        b = v > b ? v : b;
      }
      if ((threadIdx.x & 31) == 0 && tube >= 0 && b) atomicMax(&lmax[tube], b);
    } else if (tube >= 0 && b) {
      atomicMax(&lmax[tube], b);
    }
  }
}

// face i+1/2 of a tube stored at padded cell i (faces -1/2 .. len-1/2 sit on
// the cells off+2 .. off+len+2); other cells get the mask byte 0xff.
template <bool JS>
__global__ void __launch_bounds__(128) k_tubes_face(TubesDev t, const double* __restrict__ Q, double* __restrict__ Fh,
                                                    double* __restrict__ us, uint8_t* __restrict__ mask, double eps,
                                                    int mood, int weights) {
  const int64_t N = t.total;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    int tube = t.cell_tube[i];
    int64_t a = t.off[tube], e = t.off[tube + 1];
    if (i < a + NG - 1 || i > e - NG - 1) {
      if (mask) mask[i] = 0xff;
      continue;
    }
    double qc[6][5], cc[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      int64_t idx = i + (j - 2);
#pragma unroll
      for (int m = 0; m < 5; ++m) qc[j][m] = Q[m * N + idx];
      cc[j] = Q[5 * N + idx];
    }
    double Fhat[5], ustar;
    int cl, cr;
    face<5, JS>(qc, cc, eps, mood, weights, Fhat, ustar, cl, cr);
#pragma unroll
    for (int m = 0; m < 5; ++m) Fh[m * N + i] = Fhat[m];
    us[i] = ustar;
    if (mask) mask[i] = (uint8_t)(cl | (cr << 2));
  }
}

__global__ void k_tubes_update(TubesDev t, int stage, const double* Un, const double* Us, double* Uout,
                               const double* __restrict__ Fh, const double* __restrict__ us,
                               const double* __restrict__ dtp, unsigned long long* nbad) {
  const int64_t N = t.total;
  const double c13 = 1.0 / 3.0, c23 = 2.0 / 3.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    int tube = t.cell_tube[i];
    int64_t a = t.off[tube], e = t.off[tube + 1];
    if (i < a + NG || i >= e - NG) continue;
    double dx = 1.0 / (double)(e - a - 2 * NG);
    double dt = dtp[tube];
    double du = us[i] - us[i - 1];
    double out[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      double phi = Us[f * N + i];
      double dF = Fh[f * N + i] - Fh[f * N + i - 1];
      double term = -(dF / dx);
      if (f >= 3) term = term + phi * (du / dx);
      double L = 0.0;
      L = L + term;
      double un = Un[f * N + i];
      double o;
      if (stage == 0)
        o = un + dt * L;
      else if (stage == 1)
        o = (0.75 * un) + (0.25 * (phi + dt * L));
      else
        o = (c13 * un) + (c23 * (phi + dt * L));
      out[f] = o;
    }
#pragma unroll
    for (int f = 0; f < 5; ++f) Uout[f * N + i] = out[f];
    if (stage == 2) {
      double rho = out[0];
      double u = out[1] / rho;
      double usq = 0.0;
      usq = usq + u * u;
      double p = ((out[2] - (0.5 * rho) * usq) - out[4]) / out[3];
      bool ok = (rho > 0.0) && (out[3] > 0.0) && ((((out[3] + 1.0) * p) + out[4]) > 0.0);
      if (!ok) atomicAdd(nbad, 1ULL);
    }
  }
}

}  // namespace

void launch_tubes_ghost(const TubesDev& t, double* U, cudaStream_t s) {
  k_tubes_ghost<<<blocks_for(t.ntubes * 2 * NG), BS, 0, s>>>(t, U);
}
void launch_tubes_prim(const TubesDev& t, const double* U, double* Q, cudaStream_t s) {
  k_tubes_prim<<<blocks_for(t.total), BS, 0, s>>>(t, U, Q);
}
void launch_tubes_cfl(const TubesDev& t, const double* Q, unsigned long long* lmax, cudaStream_t s) {
  k_tubes_cfl<<<blocks_for(t.total), BS, 0, s>>>(t, Q, lmax);
}
void launch_tubes_face_fp64(const TubesDev& t, const double* Q, double* Fh, double* us, uint8_t* mask, double eps,
                            int mood, int weights, cudaStream_t s) {
  if (weights == WS_W_JS)
    k_tubes_face<true><<<blocks_for(t.total, 128), 128, 0, s>>>(t, Q, Fh, us, mask, eps, mood, weights);
  else
    k_tubes_face<false><<<blocks_for(t.total, 128), 128, 0, s>>>(t, Q, Fh, us, mask, eps, mood, weights);
}
void launch_tubes_update(const TubesDev& t, int stage, const double* Un, const double* Us, double* Uout,
                         const double* Fh, const double* us, const double* dt_dev, unsigned long long* nbad,
                         cudaStream_t s) {
  k_tubes_update<<<blocks_for(t.total), BS, 0, s>>>(t, stage, Un, Us, Uout, Fh, us, dt_dev, nbad);
}

}  // namespace ws
