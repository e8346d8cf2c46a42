// FP64 face sweep of one direction over the grid: one thread per face
// i+1/2 gathers the cached primitives of cells i-2..i+3 and evaluates the
// face (face_fp64.cuh).  Built with -fmad=false.
#include <cuda_runtime.h>

#include "face_fp64.cuh"
#include "ws_internal.h"

namespace ws {

namespace {

using namespace fp64;

template <int NDIM, bool JS>
__global__ void __launch_bounds__(128) k_face(GridDev g, int d, const double* __restrict__ Q, double* __restrict__ Fh,
                                              double* __restrict__ us, uint8_t* __restrict__ mask, double eps,
                                              int mood, int weights) {
  constexpr int NQ = NDIM + 4;
  const int64_t nf = g.nfaces[d];
  const int64_t fe0 = g.fe[d][0], fe1 = g.fe[d][1];
  const int64_t N = g.N;
  // sweep-frame order of the cached primitive fields: rho, u_d, u_t.., p, Gamma, Pi
  int64_t foff[NQ];
  foff[0] = 0;
  foff[1] = (int64_t)(1 + d) * N;
  {
    int k = 2;
#pragma unroll
    for (int e = 0; e < NDIM; ++e)
      if (e != d) foff[k++] = (int64_t)(1 + e) * N;
  }
  foff[NQ - 3] = (int64_t)(1 + NDIM) * N;
  foff[NQ - 2] = (int64_t)(2 + NDIM) * N;
  foff[NQ - 1] = (int64_t)(3 + NDIM) * N;
  const int64_t coff = (int64_t)(NDIM + 4) * N;
  const int64_t sd = g.st[d];
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
    int64_t c[3];
    c[0] = f % fe0;
    int64_t r = f / fe0;
    c[1] = r % fe1;
    c[2] = r / fe1;
    c[d] -= 1;  // face i+1/2 with i = f_d - 1
    int64_t base = (g.G[0] + c[0]) * g.st[0] + (g.G[1] + c[1]) * g.st[1] + (g.G[2] + c[2]) * g.st[2];
    double qc[6][NQ], cc[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      int64_t idx = base + (j - 2) * sd;
#pragma unroll
      for (int m = 0; m < NQ; ++m) qc[j][m] = Q[foff[m] + idx];
      cc[j] = Q[coff + idx];
    }
    double Fhat[NQ], ustar;
    int cl, cr;
    face<NQ, JS>(qc, cc, eps, mood, weights, Fhat, ustar, cl, cr);
    // fluxes stored in the global field order (rho, rho u_1.., E, Gamma, Pi)
#pragma unroll
    for (int m = 0; m < NQ; ++m) Fh[(foff[m] / N) * nf + f] = Fhat[m];
    us[f] = ustar;
    if (mask) mask[f] = (uint8_t)(cl | (cr << 2));
  }
}

}  // namespace

void launch_face_fp64(const GridDev& g, int d, const double* Q, double* Fh, double* us, uint8_t* mask, double eps,
                      int mood, int weights, cudaStream_t s) {
  int64_t nf = g.nfaces[d];
  int bs = 128;
  int64_t b = (nf + bs - 1) / bs;
  if (b > (1LL << 30)) b = 1LL << 30;
  if (b < 1) b = 1;
  const bool js = weights == WS_W_JS;
  switch (g.ndim) {
    case 1:
      if (js) k_face<1, true><<<(int)b, bs, 0, s>>>(g, d, Q, Fh, us, mask, eps, mood, weights);
      else k_face<1, false><<<(int)b, bs, 0, s>>>(g, d, Q, Fh, us, mask, eps, mood, weights);
      break;
    case 2:
      if (js) k_face<2, true><<<(int)b, bs, 0, s>>>(g, d, Q, Fh, us, mask, eps, mood, weights);
      else k_face<2, false><<<(int)b, bs, 0, s>>>(g, d, Q, Fh, us, mask, eps, mood, weights);
      break;
    default:
      if (js) k_face<3, true><<<(int)b, bs, 0, s>>>(g, d, Q, Fh, us, mask, eps, mood, weights);
      else k_face<3, false><<<(int)b, bs, 0, s>>>(g, d, Q, Fh, us, mask, eps, mood, weights);
      break;
  }
}

}  // namespace ws
