// Batched independent 1D tubes, mixed precision, one persistent launch per RK
// stage.  Work items are chunks of CH cells of one tube; CTAs (a few per SM,
// for the whole launch) pull items from an atomic counter until none is left,
// so tubes of very different lengths balance across the GPU.  Per chunk the
// phases mirror the 2D fused stage: FP32 primitives of the chunk plus a
// 3-cell halo in shared memory (transmissive tube ends applied on load, E - Pi
// in FP64); one loop over the faces, each thread taking a face through
// WENO-IS of its characteristic variables (the linear weights for stencils
// flat to 1e-6), back-projection, MOOD and HLLC; and the increment-form
// SSP-RK3 with FP64 accumulation (see ws_fused.cu).  A chunk of CH = 2^k - 1
// cells has 2^k faces, a whole number per thread.
// Stage 0 also reduces each tube's CFL rate (atomicMax per tube); stages 1
// and 2 take dt = CFL / max per tube.
#include <cuda_runtime.h>

#include "face_fp32.cuh"
#include "ws_internal.h"

namespace ws {

namespace {

using namespace fp32;

constexpr int NQ = 5;  // rho, u, p, Gamma, Pi

template <int CH>
struct TSmem {
  float q[NQ + 1][CH + 2 * NG];  // primitives + sound speed
  float F[NQ + 1][CH + 1];       // face fluxes + face velocity
  int item;
  float dt;
  unsigned long long red[32];
};

struct TubeArgs {
  TubesDev t;
  int stage;
  double* U;
  float* U32;
  const float* Kin;
  float* Kout;
  double dt_fixed;
  float cfl;
  unsigned long long* lmax;  // per tube
  double* dt_out;            // per tube (written in stage 1)
  const int64_t* chunk_tube; // work item -> tube
  const int* chunk_start;    // work item -> first interior cell of the chunk (tube-local)
  int64_t nitems;
  unsigned* counter;         // work counter (zeroed before the launch)
  uint8_t* mask;             // per padded cell, nullable
  WenoParams P;
  int mood;
  unsigned long long* nbad;
};

template <int CH, int NTH>
__global__ void __launch_bounds__(NTH, 1024 / NTH) k_tube_stage(TubeArgs a) {  // 64 registers
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TSmem<CH>& S = *reinterpret_cast<TSmem<CH>*>(smem_raw);
  constexpr int HW = CH + 2 * NG;
  const int tid = threadIdx.x;
  const int64_t N = a.t.total;
  for (;;) {
    if (tid == 0) S.item = (int)atomicAdd(a.counter, 1u);
    __syncthreads();
    const int item = S.item;
    if (item >= a.nitems) break;
    const int64_t tube = a.chunk_tube[item];
    const int64_t off = a.t.off[tube];
    const int len = (int)(a.t.off[tube + 1] - off - 2 * NG);
    const int c0 = a.chunk_start[item];
    const int nc = min(CH, len - c0);  // cells of this chunk
    const float idx = (float)len;      // 1/dx, dx = 1/len
    if (a.stage > 0 && tid == 0) {
      double d = a.dt_fixed > 0.0 ? a.dt_fixed : (double)a.cfl / __longlong_as_double((long long)a.lmax[tube]);
      if (a.stage == 1 && c0 == 0) a.dt_out[tube] = d;
      S.dt = f64_to_f32(d);
    }
    __syncthreads();
    // ---- phase A ----
    float lam = 0.0f;
    for (int h = tid; h < nc + 2 * NG; h += NTH) {
      int gc = c0 + h - NG;  // tube-local interior index
      int mc = gc < 0 ? 0 : (gc >= len ? len - 1 : gc);
      int64_t i = off + NG + mc;
      float rho, mu, eint, Gam, Pi;
      if (a.stage == 0) {
        rho = f64_to_f32(a.U[i]);
        mu = f64_to_f32(a.U[N + i]);
        eint = f64_to_f32(a.U[2 * N + i] - a.U[4 * N + i]);
        Gam = f64_to_f32(a.U[3 * N + i]);
        Pi = f64_to_f32(a.U[4 * N + i]);
        if (h >= NG && h < NG + nc) {
          a.U32[i] = rho;
          a.U32[N + i] = mu;
          a.U32[2 * N + i] = eint;
          a.U32[3 * N + i] = Gam;
          a.U32[4 * N + i] = Pi;
        }
      } else {
        float coef = a.stage == 1 ? S.dt : 0.25f * S.dt;
        const float* V = a.U32;
        const float* K = a.Kin;
        rho = fmaf(coef, K[i], V[i]);
        mu = fmaf(coef, K[N + i], V[N + i]);
        eint = fmaf(coef, K[2 * N + i] - K[4 * N + i], V[2 * N + i]);
        Gam = fmaf(coef, K[3 * N + i], V[3 * N + i]);
        Pi = fmaf(coef, K[4 * N + i], V[4 * N + i]);
      }
      float u = mu * frcp(rho);
      float p = fmaf(-0.5f * rho, u * u, eint) * frcp(Gam);
      float c = fsqrt(sound_speed2(rho, p, Gam, Pi));
      S.q[0][h] = rho;
      S.q[1][h] = u;
      S.q[2][h] = p;
      S.q[3][h] = Gam;
      S.q[4][h] = Pi;
      S.q[5][h] = c;
      if (a.stage == 0 && h >= NG && h < NG + nc) {
        float l = (fabsf(u) + c) * idx;
        if (!(l <= lam)) lam = l;
      }
    }
    if (a.stage == 0) {
      unsigned long long b = (unsigned long long)__double_as_longlong(f32_to_f64(lam));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        unsigned long long v = __shfl_xor_sync(0xffffffffu, b, o);
        b = v > b ? v : b;
      }
      if ((tid & 31) == 0) S.red[tid >> 5] = b;
    }
    __syncthreads();
    if (a.stage == 0 && tid == 0) {
      unsigned long long b = 0;
      for (int w = 0; w < NTH / 32; ++w) b = S.red[w] > b ? S.red[w] : b;
      if (b) atomicMax(&a.lmax[tube], b);
    }
    // ---- phase B: faces f = 0..nc (face f between chunk cells f-1 and f) ----
    const int nf = nc + 1;
    for (int f = tid; f < nf; f += NTH) {
      const int ha = f + 2, hb = f + 3, h0 = f;  // stencil cell 0 = chunk cell f-3 -> halo index f
      float rho_bar = 0.5f * (S.q[0][ha] + S.q[0][hb]);
      float c_bar = 0.5f * (S.q[5][ha] + S.q[5][hb]);
      float c2 = c_bar * c_bar, rc = rho_bar * c_bar;
      float inv = frcp(c2 * rc);
      float ic2 = rc * inv, irc = c2 * inv;
      const float mic2 = -frcp(c2);
      float2 W[NQ], Q[NQ];  // (left, right) characteristics, then primitives
#pragma unroll
      for (int r = 0; r < NQ; ++r) {
        float w[6];
        if (r == 0 || r == NQ - 1) {
          const float rcs = r == 0 ? -rc : rc;
#pragma unroll
          for (int k = 0; k < 6; ++k) w[k] = 0.5f * fmaf(rcs, S.q[1][h0 + k], S.q[2][h0 + k]);
        } else if (r == 1) {
#pragma unroll
          for (int k = 0; k < 6; ++k) w[k] = fmaf(mic2, S.q[2][h0 + k], S.q[0][h0 + k]);
        } else {
#pragma unroll
          for (int k = 0; k < 6; ++k) w[k] = S.q[r + 1][h0 + k];  // Gamma (r = 2), Pi (r = 3)
        }
        float mn = fminf(fmin3(w[0], w[1], w[2]), fmin3(w[3], w[4], w[5]));
        float mx = fmaxf(fmax3(w[0], w[1], w[2]), fmax3(w[3], w[4], w[5]));
        // both sides at once: lanes (left, right) of the mirrored stencils
        float2 p0 = make_float2(w[0], w[5]), p1 = make_float2(w[1], w[4]), p2 = make_float2(w[2], w[3]);
        float2 p3 = make_float2(w[3], w[2]), p4 = make_float2(w[4], w[1]);
        if (mx - mn <= 1e-6f * fmaxf(fabsf(mx), fabsf(mn)))
          W[r] = linear5_pair(p0, p1, p2, p3, p4);
        else
          W[r] = weno5_pair(p0, p1, p2, p3, p4, a.P);
      }
      back_project_pair<NQ>(W, ic2, irc, Q);
      int code[2] = {0, 0};
      if (a.mood) {
        float qs[2][NQ];
#pragma unroll
        for (int r = 0; r < NQ; ++r) {
          qs[0][r] = Q[r].x;
          qs[1][r] = Q[r].y;
        }
        const bool ok0 = admissible<NQ>(qs[0]), ok1 = admissible<NQ>(qs[1]);
        if (!ok0 || !ok1) {  // MOOD cascade of the failing side(s): rare
#pragma unroll 1
          for (int side = 0; side < 2; ++side) {
            if (side == 0 ? ok0 : ok1) continue;
            // 3rd-order retry (d3 = d4 = 0) of this side
            float qc[6][NQ];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
#pragma unroll
              for (int m = 0; m < NQ; ++m) qc[k][m] = S.q[m][f + k];
            }
            float hrc = 0.5f * rc, wt[NQ], q3[NQ];
#pragma unroll
            for (int r = 0; r < NQ; ++r) {
              float v[5];
#pragma unroll
              for (int k = 0; k < 5; ++k) v[k] = project<NQ>(qc[side == 0 ? k : 5 - k], r, hrc, ic2);
              wt[r] = weno_is(v[0], v[1], v[2], v[3], v[4], a.P, 3);
            }
            back_project<NQ>(wt, ic2, irc, q3);
            code[side] = 1;
            if (!admissible<NQ>(q3)) {
              int hh = side == 0 ? ha : hb;
#pragma unroll
              for (int m = 0; m < NQ; ++m) q3[m] = S.q[m][hh];
              code[side] = 2;
            }
#pragma unroll
            for (int r = 0; r < NQ; ++r) {
              if (side == 0)
                Q[r].x = q3[r];
              else
                Q[r].y = q3[r];
            }
          }
        }
      }
      float Fh[NQ], us;
      hllc_pair<NQ>(Q, Fh, us);
#pragma unroll
      for (int m = 0; m < NQ; ++m) S.F[m][f] = Fh[m];
      S.F[NQ][f] = us;
      // face f sits at padded cell off + NG + c0 + f - 1 (faces -1/2 .. len-1/2 on cells off+2 .. off+len+2)
      if (a.mask) a.mask[off + NG + c0 + f - 1] = (uint8_t)(code[0] | (code[1] << 2));
    }
    __syncthreads();
    // ---- phase C ----
    const float dt = S.dt;
    for (int cc_ = tid; cc_ < nc; cc_ += NTH) {
      int64_t gi = off + NG + c0 + cc_;
      float du = (S.F[NQ][cc_ + 1] - S.F[NQ][cc_]) * idx;
      float inc[NQ];
#pragma unroll
      for (int m = 0; m < NQ; ++m) {
        float L = -(S.F[m][cc_ + 1] - S.F[m][cc_]) * idx;
        if (m >= 3) L = fmaf(S.q[m][cc_ + NG], du, L);
        inc[m] = L;
      }
      if (a.stage == 0) {
#pragma unroll
        for (int m = 0; m < NQ; ++m) a.Kout[m * N + gi] = inc[m];
      } else if (a.stage == 1) {
#pragma unroll
        for (int m = 0; m < NQ; ++m) a.Kout[m * N + gi] = a.Kin[m * N + gi] + inc[m];
      } else {
        float d[NQ];
#pragma unroll
        for (int m = 0; m < NQ; ++m) {
          d[m] = dt * fmaf(1.0f / 6.0f, a.Kin[m * N + gi], (2.0f / 3.0f) * inc[m]);
          a.U[m * N + gi] = a.U[m * N + gi] + f32_to_f64(d[m]);
        }
        const float* V = a.U32;
        float rho = V[gi] + d[0], mu = V[N + gi] + d[1];
        float eint = V[2 * N + gi] + (d[2] - d[4]), Gam = V[3 * N + gi] + d[3], Pi = V[4 * N + gi] + d[4];
        float pe = fmaf(-0.5f, mu * mu * frcp(rho), eint);
        bool ok = rho > 0.0f && Gam > 0.0f && fmaf(Gam + 1.0f, pe * frcp(Gam), Pi) > 0.0f;
        if (!ok) atomicAdd(a.nbad, 1ULL);
      }
    }
    __syncthreads();  // shared memory is reused by the next item
  }
}

template <int CH, int NTH>
void launch_one(const TubeArgs& a, int ctas_per_sm, cudaStream_t s) {
  static bool prepared = false;
  if (!prepared) {
    cudaFuncSetAttribute(k_tube_stage<CH, NTH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(TSmem<CH>));
    prepared = true;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t grid = (int64_t)sms * ctas_per_sm;
  if (grid > a.nitems) grid = a.nitems > 0 ? a.nitems : 1;
  k_tube_stage<CH, NTH><<<(int)grid, NTH, sizeof(TSmem<CH>), s>>>(a);
}

}  // namespace

// configurations the autotuner chooses from: chunk size x threads (a chunk of
// 2^k - 1 cells has 2^k faces)
const int kTubeConfigs[][2] = {{255, 128}, {255, 256}, {511, 256}, {511, 512}, {1023, 512}};
const int kNumTubeConfigs = 5;

int tube_chunk_size(int config) { return kTubeConfigs[config][0]; }

void launch_tubes_stage_mixed(const TubesDev& t, int config, int stage, double* U, float* U32, const float* Kin,
                              float* Kout, double dt_fixed, double cfl, unsigned long long* lmax, double* dt_out,
                              const int64_t* chunk_tube, const int* chunk_start, int64_t nitems, unsigned* counter,
                              uint8_t* mask, float eps_rel, int mood, int weights, unsigned long long* nbad,
                              cudaStream_t s) {
  TubeArgs a;
  a.t = t;
  a.stage = stage;
  a.U = U;
  a.U32 = U32;
  a.Kin = Kin;
  a.Kout = Kout;
  a.dt_fixed = dt_fixed;
  a.cfl = (float)cfl;
  a.lmax = lmax;
  a.dt_out = dt_out;
  a.chunk_tube = chunk_tube;
  a.chunk_start = chunk_start;
  a.nitems = nitems;
  a.counter = counter;
  a.mask = mask;
  a.P = weno_params(eps_rel, weights);
  a.mood = mood;
  a.nbad = nbad;
  switch (config) {
    case 0: launch_one<255, 128>(a, 8, s); break;
    case 1: launch_one<255, 256>(a, 4, s); break;
    case 2: launch_one<511, 256>(a, 4, s); break;
    case 3: launch_one<511, 512>(a, 2, s); break;
    default: launch_one<1023, 512>(a, 2, s); break;
  }
}

}  // namespace ws
