// Learned smooth-face gate: training-data sampling and the MLP's training
// kernels (forward, backward, Adam), hand-written in FP32.
//
// The gate is a 24 -> 32 -> 32 -> 1 MLP (ReLU, ReLU, sigmoid) that reads, for
// one face i+1/2, the characteristic variables w1 (u-c), w2 (entropy), w6
// (u+c) and w_Gamma of the six stencil cells i-2..i+3, each normalised over
// the stencil as (w - mean)/(max - min + 1e-30), or zero when the stencil is
// flat to 1e-6 of its magnitude (below FP32 resolution of the variable).  A
// face is labelled "needs WENO-IS" (1) when MOOD lowers either side below 5th
// order or when, for any characteristic variable with a non-flat stencil and
// either side, the WENO-IS value differs from the 5th-order linear-weight
// value by more than 1e-6 (max - min); faces labelled 0 may take the linear
// weights d = (4,2,3,1)/10 for w1, w2, w6, w_Gamma and w_Pi (Pi is affine in
// Gamma across a two-material interface, so w_Gamma's inputs speak for it);
// shear variables always keep WENO-IS and are not part of the label.
// Parameter layout (FP32, WS_MLP_NPARAM floats): W1[32][24], b1[32],
// W2[32][32], b2[32], W3[32], b3.
#include <cuda_runtime.h>

#include "face_fp32.cuh"
#include "ws_internal.h"

namespace ws {

namespace {

using namespace fp32;

constexpr int NIN = 24, NH = 32;
constexpr int OW1 = 0, OB1 = OW1 + NH * NIN, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NH, NPARAM = OB3 + 1;
static_assert(NPARAM == WS_MLP_NPARAM, "parameter count");

inline int blocks_for(int64_t n, int bs) {
  int64_t b = (n + bs - 1) / bs;
  if (b > (1LL << 30)) b = 1LL << 30;
  return (int)(b < 1 ? 1 : b);
}

// features and label of one face from sweep-frame FP32 primitives
template <int NQ>
__device__ void face_features(const float (&qc)[6][NQ], const float (&cc)[6], const WenoParams& P, float* feat,
                              uint8_t& label) {
  constexpr int NT = NQ - 5, IP = 2 + NT;
  float rho_bar = 0.5f * (qc[2][0] + qc[3][0]);
  float c_bar = 0.5f * (cc[2] + cc[3]);
  float rc = rho_bar * c_bar, hrc = 0.5f * rc;
  float ic2 = frcp(c_bar * c_bar), irc = frcp(rc);
  bool rough = false;
  bool flat_gamma = false;
  float wt5[2][NQ];
#pragma unroll
  for (int r = 0; r < NQ; ++r) {
    float w[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) w[k] = project<NQ>(qc[k], r, hrc, ic2);
    float mn = w[0], mx = w[0], sum = w[0];
#pragma unroll
    for (int k = 1; k < 6; ++k) {
      mn = fminf(mn, w[k]);
      mx = fmaxf(mx, w[k]);
      sum += w[k];
    }
    float range = (mx - mn) + 1e-30f;
    // features: w1 (r = 0), w2 (r = 1), w6 (r = NQ-1), w_Gamma (r = IP); a
    // stencil flat to 1e-6 of its magnitude gives zero features
    int slot = r == 0 ? 0 : (r == 1 ? 1 : (r == NQ - 1 ? 2 : (r == IP ? 3 : -1)));
    if (slot >= 0) {
      float mean = sum * (1.0f / 6.0f);
      float inv = (mx - mn) > 1e-6f * fmaxf(fabsf(mx), fabsf(mn)) ? frcp(range) : 0.0f;
#pragma unroll
      for (int k = 0; k < 6; ++k) feat[slot * 6 + k] = (w[k] - mean) * inv;
    }
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      float v0 = side == 0 ? w[0] : w[5], v1 = side == 0 ? w[1] : w[4], v2 = side == 0 ? w[2] : w[3];
      float v3 = side == 0 ? w[3] : w[2], v4 = side == 0 ? w[4] : w[1];
      float full = weno_is(v0, v1, v2, v3, v4, P, 5);
      float lin = linear5(v0, v1, v2, v3, v4);
      // a stencil flat to 1e-6 of its magnitude (FP32 noise level) counts as
      // smooth; shear variables always keep WENO-IS, so they do not count
      bool flat = (mx - mn) <= 1e-6f * fmaxf(fabsf(mx), fabsf(mn));
      if (r == IP) flat_gamma = flat;
      if (r == IP + 1) flat = flat || flat_gamma;  // Pi follows Gamma (affine across the interface)
      bool shear = r >= 2 && r < IP;
      if (!shear && !flat && fabsf(full - lin) > 1e-6f * range) rough = true;
      wt5[side][r] = full;
    }
  }
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    float q[NQ];
    back_project<NQ>(wt5[side], ic2, irc, q);
    if (!admissible<NQ>(q)) rough = true;
  }
  label = rough ? 1 : 0;
}

template <int NDIM>
__global__ void k_face_samples(GridDev g, int d, const float* __restrict__ Q, int64_t stride, int64_t out0,
                               int64_t max_out, float* __restrict__ feats, uint8_t* __restrict__ labels,
                               WenoParams P) {
  constexpr int NQ = NDIM + 4;
  const int64_t nf = g.nfaces[d];
  const int64_t ns = (nf + stride - 1) / stride;
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
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
    int64_t o = out0 + s;
    if (o >= max_out) break;
    int64_t f = s * stride;
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
      int64_t idx = base + (j - 2) * g.st[d];
#pragma unroll
      for (int m = 0; m < NQ; ++m) qc[j][m] = Q[fld[m] * N + idx];
      cc[j] = Q[NQ * N + idx];
    }
    float feat[NIN];
    uint8_t lab;
    face_features<NQ>(qc, cc, P, feat, lab);
#pragma unroll
    for (int k = 0; k < NIN; ++k) feats[o * NIN + k] = feat[k];
    labels[o] = lab;
  }
}

// ---- MLP in FP32 ----
__device__ __forceinline__ void mlp_forward(const float* __restrict__ W, const float* x, float* h1, float* h2,
                                            float& z) {
#pragma unroll 4
  for (int j = 0; j < NH; ++j) {
    float a = W[OB1 + j];
#pragma unroll
    for (int k = 0; k < NIN; ++k) a = fmaf(W[OW1 + j * NIN + k], x[k], a);
    h1[j] = fmaxf(a, 0.0f);
  }
#pragma unroll 4
  for (int j = 0; j < NH; ++j) {
    float a = W[OB2 + j];
#pragma unroll
    for (int k = 0; k < NH; ++k) a = fmaf(W[OW2 + j * NH + k], h1[k], a);
    h2[j] = fmaxf(a, 0.0f);
  }
  float a = W[OB3];
#pragma unroll
  for (int k = 0; k < NH; ++k) a = fmaf(W[OW3 + k], h2[k], a);
  z = a;
}

__global__ void k_mlp_forward(const float* __restrict__ params, const float* __restrict__ X, int64_t n,
                              float* __restrict__ logits) {
  __shared__ float W[NPARAM];
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) W[i] = params[i];
  __syncthreads();
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    float x[NIN], h1[NH], h2[NH], z;
#pragma unroll
    for (int k = 0; k < NIN; ++k) x[k] = X[s * NIN + k];
    mlp_forward(W, x, h1, h2, z);
    logits[s] = z;
  }
}

// The gradient is summed in 64-bit fixed point (units of 2^-48): integer
// additions commute, so the sums -- within a block through shared-memory
// atomics, across blocks through global ones -- do not depend on the order in
// which threads arrive, and a gradient is the same on every run.  Each
// contribution is rounded to the unit once (|contributions| < 3e4).
constexpr float kFixScale = 281474976710656.0f;  // 2^48
__device__ unsigned long long g_mlp_acc[NPARAM + 1];  // the sums; [NPARAM]: the loss

__device__ __forceinline__ void fix_add(unsigned long long* a, float v) {
  float s = fminf(fmaxf(v * kFixScale, -9.0e18f), 9.0e18f);  // exact scaling by a power of two
  atomicAdd(a, (unsigned long long)__float2ll_rn(s));
}

__global__ void k_mlp_acc_zero() {
  for (int i = threadIdx.x; i <= NPARAM; i += blockDim.x) g_mlp_acc[i] = 0ULL;
}

__global__ void k_mlp_acc_out(float* __restrict__ grad, float* __restrict__ loss) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= NPARAM; i += gridDim.x * blockDim.x) {
    float v = (float)((double)(long long)g_mlp_acc[i] * (1.0 / 281474976710656.0));
    if (i < NPARAM)
      grad[i] = v;
    else
      *loss = v;
  }
}

// mean binary cross-entropy (positives weighted by pos_weight) and its
// gradient over n samples, into g_mlp_acc (zeroed before the launch)
__global__ void k_mlp_grad(const float* __restrict__ params, const float* __restrict__ X,
                           const uint8_t* __restrict__ y, int64_t n, float pos_weight, float inv_n) {
  __shared__ float W[NPARAM];
  __shared__ unsigned long long G[NPARAM];
  __shared__ unsigned long long Ls;
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) {
    W[i] = params[i];
    G[i] = 0ULL;
  }
  if (threadIdx.x == 0) Ls = 0ULL;
  __syncthreads();
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    float x[NIN], h1[NH], h2[NH], z;
#pragma unroll
    for (int k = 0; k < NIN; ++k) x[k] = X[s * NIN + k];
    mlp_forward(W, x, h1, h2, z);
    float t = y[s] ? 1.0f : 0.0f;
    float wgt = (y[s] ? pos_weight : 1.0f) * inv_n;
    // BCE with logits: softplus(z) - t z, computed stably
    float sp = fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z)));
    fix_add(&Ls, wgt * (sp - t * z));
    float p = 1.0f / (1.0f + expf(-z));
    float dz = wgt * (p - t);
    float dh2[NH];
#pragma unroll
    for (int k = 0; k < NH; ++k) {
      fix_add(&G[OW3 + k], dz * h2[k]);
      dh2[k] = h2[k] > 0.0f ? dz * W[OW3 + k] : 0.0f;
    }
    fix_add(&G[OB3], dz);
    float dh1[NH];
#pragma unroll
    for (int k = 0; k < NH; ++k) dh1[k] = 0.0f;
    for (int j = 0; j < NH; ++j) {
      float g2 = dh2[j];
      if (g2 == 0.0f) continue;
      fix_add(&G[OB2 + j], g2);
#pragma unroll
      for (int k = 0; k < NH; ++k) {
        fix_add(&G[OW2 + j * NH + k], g2 * h1[k]);
        dh1[k] = fmaf(W[OW2 + j * NH + k], g2, dh1[k]);
      }
    }
    for (int j = 0; j < NH; ++j) {
      float g1 = h1[j] > 0.0f ? dh1[j] : 0.0f;
      if (g1 == 0.0f) continue;
      fix_add(&G[OB1 + j], g1);
#pragma unroll
      for (int k = 0; k < NIN; ++k) fix_add(&G[OW1 + j * NIN + k], g1 * x[k]);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x)
    if (G[i] != 0ULL) atomicAdd(&g_mlp_acc[i], G[i]);
  if (threadIdx.x == 0) atomicAdd(&g_mlp_acc[NPARAM], Ls);
}

__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  float gi = g[i];
  float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
  float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

}  // namespace

void launch_face_samples(const GridDev& g, int d, const float* Q, int64_t stride, int64_t out0, int64_t max_out,
                         float* feats, uint8_t* labels, float eps_rel, int weights, cudaStream_t s) {
  WenoParams P = weno_params(eps_rel, weights);
  int64_t ns = (g.nfaces[d] + stride - 1) / stride;
  int b = blocks_for(ns, 128);
  switch (g.ndim) {
    case 1: k_face_samples<1><<<b, 128, 0, s>>>(g, d, Q, stride, out0, max_out, feats, labels, P); break;
    case 2: k_face_samples<2><<<b, 128, 0, s>>>(g, d, Q, stride, out0, max_out, feats, labels, P); break;
    default: k_face_samples<3><<<b, 128, 0, s>>>(g, d, Q, stride, out0, max_out, feats, labels, P); break;
  }
}

}  // namespace ws

using namespace ws;

extern "C" WS_API int ws_mlp_forward(const float* params, const float* X, int64_t n, float* logits, void* stream) {
  if (n < 0 || !params || (n > 0 && (!X || !logits))) return WS_EINVAL;
  if (n == 0) return WS_OK;
  int b = blocks_for(n, 256);
  if (b > 152 * 16) b = 152 * 16;
  k_mlp_forward<<<b, 256, 0, (cudaStream_t)stream>>>(params, X, n, logits);
  return cudaGetLastError() == cudaSuccess ? WS_OK : WS_ECUDA;
}

extern "C" WS_API int ws_mlp_grad(const float* params, const float* X, const uint8_t* y, int64_t n, float pos_weight,
                                  float* grad, float* loss, void* stream) {
  if (n <= 0 || !params || !X || !y || !grad || !loss) return WS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int b = blocks_for(n, 256);
  if (b > 152 * 2) b = 152 * 2;
  k_mlp_acc_zero<<<1, 1024, 0, s>>>();
  k_mlp_grad<<<b, 256, 0, s>>>(params, X, y, n, pos_weight, 1.0f / (float)n);
  k_mlp_acc_out<<<(NPARAM + 256) / 256, 256, 0, s>>>(grad, loss);
  return cudaGetLastError() == cudaSuccess ? WS_OK : WS_ECUDA;
}

extern "C" WS_API int ws_mlp_adam(float* params, float* m, float* v, const float* grad, int64_t step, float lr,
                                  void* stream) {
  if (!params || !m || !v || !grad || step < 1) return WS_EINVAL;
  const float b1 = 0.9f, b2 = 0.999f;
  float c1 = 1.0f / (1.0f - powf(b1, (float)step)), c2 = 1.0f / (1.0f - powf(b2, (float)step));
  k_adam<<<(NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, m, v, grad, lr, b1, b2, 1e-8f, c1, c2);
  return cudaGetLastError() == cudaSuccess ? WS_OK : WS_ECUDA;
}
