// Fused mixed-precision RK stage for 2D grids: one kernel per SSP-RK3 stage.
//
// A CTA owns a TX x TY tile of cells and works through five phases separated
// by barriers, all in shared memory:
//   A  stage-state FP32 primitives of the tile plus a 3-cell halo; boundary
//      conditions are applied while loading (no ghost kernel), E - Pi in FP64;
//   B1 per (face, characteristic variable): projection of the six stencil
//      cells with L_{i+1/2} and 5th-order WENO-IS of both sides;
//   B2 one thread per face: back-projection, MOOD cascade (a side that fails
//      is reconstructed again at 3rd order from the staged primitives), HLLC;
//   C  one thread per cell: flux divergence with the Gamma/Pi source and the
//      RK stage.
// Splitting the face into (face, variable) work items keeps the register
// count low; with only 5th-order values staged, two 512-thread CTAs fit per
// SM, so one CTA's memory phases overlap the other's arithmetic.
//
// The Shu-Osher SSP-RK3 is carried in increment form, algebraically
// identical to U1 = U + dt L0, U2 = 3/4 U + 1/4 (U1 + dt L1),
// U' = 1/3 U + 2/3 (U2 + dt L2) with L_s = L(U_s):
//   U1 = U + dt K0,  K0 = L0
//   U2 = U + dt K1/4,  K1 = L0 + L1
//   U' = U + dt (K1/6 + 2 L2/3)
// Stage 0 needs no dt: it also reduces the CFL wave rate max sum_d
// (|u_d| + c)/dx_d over its cells (atomicMax), and stage 1 derives
// dt = CFL / max from it, so a step needs no separate CFL kernel.
// The FP64 state U is converted to FP32 once, in stage 0 (E - Pi formed in
// FP64 first), into a scratch image that stages 1 and 2 read together with
// the FP32 increments K; stage 2 adds its increment to U in FP64, in place,
// since no tile reads U's FP64 values after stage 0.  K0 and K1 live in
// separate buffers because neighbouring tiles read K in their halos.
#include <cuda_runtime.h>

#include "face_fp32.cuh"
#include "ws_internal.h"

namespace ws {

namespace {

using namespace fp32;

constexpr int TX = 32, TY = 15;
constexpr int HX = TX + 2 * NG, HY = TY + 2 * NG;
constexpr int NQ = 6;  // rho, u, v, p, Gamma, Pi
constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1), NF = NFX + NFY;
constexpr int NT = 512;

struct Smem {
  float q[NQ + 1][HY][HX];        // primitives + sound speed of tile and halo
  float w[2][NQ][NF];             // [side l/r][variable][face] 5th-order reconstructed characteristics
  float fx[NQ + 1][TY][TX + 1];   // x-face fluxes (global field order) + face velocity
  float fy[NQ + 1][TY + 1][TX];   // y-face fluxes + face velocity
  unsigned long long red[NT / 32];  // per-warp CFL maxima
  float dt;                         // the step, broadcast from thread 0
};

struct StageArgs {
  GridDev g;
  int stage;
  float idx, idy;     // 1/dx, 1/dy
  float cfl;
  double dt_fixed;    // > 0: use this step; otherwise CFL
  unsigned long long* lmax;  // stage 0: max wave rate (FP64 bits)
  double* dt_out;     // stage 1 (block 0): the dt used
  double* U;          // state at t^n; stage 2 replaces it with t^{n+1}
  float* U32;         // FP32 image of U^n (rho, m_x, m_y, E - Pi, Gamma, Pi): written in stage 0
  const float* Kin;   // stages 1, 2: accumulated increments
  float* Kout;        // stages 0, 1
  uint8_t* mask_x;    // nullable
  uint8_t* mask_y;
  WenoParams P;
  int mood;
  unsigned long long* nbad;
};

// interior index along an axis of n cells for a (possibly out-of-range)
// coordinate, with the boundary kinds of the two ends; flip: reflective image
__device__ __forceinline__ int map_bc(int x, int n, int lo, int hi, bool& flip) {
  if (x >= 0 && x < n) return x;
  int kind = x < 0 ? lo : hi;
  if (kind == WS_BC_PERIODIC) {
    int m = x % n;
    return m < 0 ? m + n : m;
  }
  if (kind == WS_BC_REFLECTIVE) {
    flip = !flip;
    int m = x < 0 ? -1 - x : 2 * n - 1 - x;
    return m < 0 ? 0 : (m >= n ? n - 1 : m);
  }
  return x < 0 ? 0 : n - 1;
}

// halo-tile coordinates of stencil cell k (0..5 = i-2..i+3) of face f, and
// whether the face is an x face; false if the face lies outside the grid
// x faces are numbered row by row for tile faces 0..TX-1 (warp = one row,
// no shared-memory bank conflicts), then the TY right-most faces.
__device__ __forceinline__ bool face_geom(int f, int x0, int y0, int nx, int ny, bool& isx, int& hx, int& hy,
                                          int& dhx, int& dhy) {
  if (f < NFX) {
    int j, i;
    if (f < TX * TY) {
      j = f / TX;
      i = f - j * TX;
    } else {
      j = f - TX * TY;
      i = TX;
    }
    isx = true;
    hx = i;  // cell k at hx + k
    hy = j + NG;
    dhx = 1;
    dhy = 0;
    return (x0 + i - 1 <= nx - 1) && (y0 + j < ny);
  }
  int ff = f - NFX;
  int j = ff / TX, i = ff - j * TX;
  isx = false;
  hx = i + NG;
  hy = j;
  dhx = 0;
  dhy = 1;
  return (x0 + i < nx) && (y0 + j - 1 <= ny - 1);
}

// Characteristic variable R of the face's six stencil cells (qb points at
// cell 0 in the halo tile; cells are D-strided).  D = 0: x face (frame
// rho, u, v, ...); D = 1: y face (rho, v, u, ...).  All shared-memory offsets
// are compile-time constants.
template <int D, int R>
__device__ __forceinline__ void project6(const float* qb, float (&w)[6]) {
  constexpr int ST = D == 0 ? 1 : HX;  // stride between stencil cells
  constexpr int FS = HY * HX;          // stride between fields
  constexpr int UN = D == 0 ? 1 : 2, UT = D == 0 ? 2 : 1;
  if (R == 0 || R == NQ - 1) {
    float rho_bar = 0.5f * (qb[2 * ST] + qb[3 * ST]);
    float c_bar = 0.5f * (qb[6 * FS + 2 * ST] + qb[6 * FS + 3 * ST]);
    float rc = R == 0 ? -(rho_bar * c_bar) : rho_bar * c_bar;
#pragma unroll
    for (int k = 0; k < 6; ++k) w[k] = 0.5f * fmaf(rc, qb[UN * FS + k * ST], qb[3 * FS + k * ST]);
  } else if (R == 1) {
    float c_bar = 0.5f * (qb[6 * FS + 2 * ST] + qb[6 * FS + 3 * ST]);
    float mic2 = -frcp(c_bar * c_bar);
#pragma unroll
    for (int k = 0; k < 6; ++k) w[k] = fmaf(mic2, qb[3 * FS + k * ST], qb[k * ST]);
  } else {
    constexpr int F = R == 2 ? UT : R + 1;  // shear, Gamma, Pi
#pragma unroll
    for (int k = 0; k < 6; ++k) w[k] = qb[F * FS + k * ST];
  }
}

// 5th-order reconstruction of variable R on both sides of a face
template <int D, int R>
__device__ __forceinline__ void weno_item(const float* qb, const WenoParams& P, float& l5, float& r5) {
  float w[6];
  project6<D, R>(qb, w);
  l5 = weno_is(w[0], w[1], w[2], w[3], w[4], P, 5);
  r5 = weno_is(w[5], w[4], w[3], w[2], w[1], P, 5);
}

// 3rd-order reconstruction (d3 = d4 = 0) of all variables of one side:
// the MOOD retry, taken only by faces whose 5th-order state is inadmissible
template <int D>
__device__ __noinline__ void weno_side3(const float* qb, int side, const WenoParams& P, float* wt) {
  float w[6];
#define WS_SIDE3(R)                                                                                   \
  project6<D, R>(qb, w);                                                                             \
  wt[R] = side == 0 ? weno_is(w[0], w[1], w[2], w[3], w[4], P, 3) : weno_is(w[5], w[4], w[3], w[2], w[1], P, 3);
  WS_SIDE3(0)
  WS_SIDE3(1)
  WS_SIDE3(2)
  WS_SIDE3(3)
  WS_SIDE3(4)
  WS_SIDE3(5)
#undef WS_SIDE3
}

// the (at most FPT) faces a thread owns in phase B1
constexpr int FPT = (NF + NT - 1) / NT;

__global__ void __launch_bounds__(NT, 2) k_stage2d(StageArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  const GridDev& g = a.g;
  const int nx = g.n[0], ny = g.n[1];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int64_t N = g.N, P0 = g.P[0];
  const int tid = threadIdx.x;
  if (a.stage > 0) {
    if (tid == 0) {  // one FP64 division per CTA
      double d = a.dt_fixed > 0.0 ? a.dt_fixed : (double)a.cfl / __longlong_as_double((long long)*a.lmax);
      if (a.stage == 1 && blockIdx.x == 0 && blockIdx.y == 0) *a.dt_out = d;
      S.dt = f64_to_f32(d);
    }
    __syncthreads();
  }
  const float dt = a.stage > 0 ? S.dt : 0.0f;
  const float coef = a.stage == 0 ? 0.0f : (a.stage == 1 ? dt : 0.25f * dt);
  float lam_max = 0.0f;

  // ---- phase A: stage-state primitives of tile + halo ----
  for (int h = tid; h < HX * HY; h += NT) {
    int hy = h / HX, hx = h - hy * HX;
    int gx = x0 + hx - NG, gy = y0 + hy - NG;
    bool outx = gx < 0 || gx >= nx, outy = gy < 0 || gy >= ny;
    if (outx && outy) continue;  // corners are never read
    bool fx = false, fy = false;
    int mx = map_bc(gx, nx, g.bc[0][0], g.bc[0][1], fx);
    int my = map_bc(gy, ny, g.bc[1][0], g.bc[1][1], fy);
    int64_t i = (int64_t)(NG + my) * P0 + (NG + mx);
    float rho, mu, mv, eint, Gam, Pi;
    if (a.stage == 0) {
      const double* U = a.U;
      rho = f64_to_f32(U[i]);
      mu = f64_to_f32(U[N + i]);
      mv = f64_to_f32(U[2 * N + i]);
      eint = f64_to_f32(U[3 * N + i] - U[5 * N + i]);  // E - Pi in FP64
      Gam = f64_to_f32(U[4 * N + i]);
      Pi = f64_to_f32(U[5 * N + i]);
      bool own = hx >= NG && hx < NG + TX && hy >= NG && hy < NG + TY && !outx && !outy;
      if (own) {
        a.U32[i] = rho;
        a.U32[N + i] = mu;
        a.U32[2 * N + i] = mv;
        a.U32[3 * N + i] = eint;
        a.U32[4 * N + i] = Gam;
        a.U32[5 * N + i] = Pi;
      }
    } else {
      const float* V = a.U32;
      const float* K = a.Kin;
      rho = fmaf(coef, K[i], V[i]);
      mu = fmaf(coef, K[N + i], V[N + i]);
      mv = fmaf(coef, K[2 * N + i], V[2 * N + i]);
      eint = fmaf(coef, K[3 * N + i] - K[5 * N + i], V[3 * N + i]);
      Gam = fmaf(coef, K[4 * N + i], V[4 * N + i]);
      Pi = fmaf(coef, K[5 * N + i], V[5 * N + i]);
    }
    float irho = frcp(rho);
    float u = mu * irho, v = mv * irho;
    if (fx) u = -u;
    if (fy) v = -v;
    float p = fmaf(-0.5f * rho, fmaf(u, u, v * v), eint) * frcp(Gam);
    S.q[0][hy][hx] = rho;
    S.q[1][hy][hx] = u;
    S.q[2][hy][hx] = v;
    S.q[3][hy][hx] = p;
    S.q[4][hy][hx] = Gam;
    S.q[5][hy][hx] = Pi;
    float c = fsqrt(sound_speed2(rho, p, Gam, Pi));
    S.q[6][hy][hx] = c;
    if (a.stage == 0 && hx >= NG && hx < NG + TX && hy >= NG && hy < NG + TY && !outx && !outy) {
      float lam = fmaf(fabsf(u) + c, a.idx, (fabsf(v) + c) * a.idy);
      if (!(lam <= lam_max)) lam_max = lam;  // NaN propagates
    }
  }
  if (a.stage == 0) {
    unsigned long long b = (unsigned long long)__double_as_longlong(f32_to_f64(lam_max));
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
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) b = S.red[w] > b ? S.red[w] : b;
    if (b) atomicMax(a.lmax, b);
  }

  // ---- phase B1: WENO-IS per (face, characteristic variable) ----
  {
    int fo[FPT];       // face index, or -1
    int qo[FPT];       // offset of stencil cell 0 in the halo tile
    bool fxd[FPT];     // x face?
#pragma unroll
    for (int t = 0; t < FPT; ++t) {
      int f = tid + t * NT;
      bool isx = false;
      int hx = 0, hy = 0, dhx, dhy;
      bool ok = f < NF && face_geom(f, x0, y0, nx, ny, isx, hx, hy, dhx, dhy);
      fo[t] = ok ? f : -1;
      qo[t] = hy * HX + hx;
      fxd[t] = isx;
    }
    const float* q0 = &S.q[0][0][0];
#define WS_B1(R)                                                              \
    _Pragma("unroll") for (int t = 0; t < FPT; ++t) {                         \
      if (fo[t] < 0) continue;                                                \
      float l5, r5;                                                           \
      if (fxd[t])                                                             \
        weno_item<0, R>(q0 + qo[t], a.P, l5, r5);                             \
      else                                                                    \
        weno_item<1, R>(q0 + qo[t], a.P, l5, r5);                             \
      S.w[0][R][fo[t]] = l5;                                                  \
      S.w[1][R][fo[t]] = r5;                                                  \
    }
    WS_B1(0)
    WS_B1(1)
    WS_B1(2)
    WS_B1(3)
    WS_B1(4)
    WS_B1(5)
#undef WS_B1
  }
  __syncthreads();

  // ---- phase B2: back-projection, MOOD, HLLC per face ----
  for (int f = tid; f < NF; f += NT) {
    bool isx;
    int hx, hy, dhx, dhy;
    if (!face_geom(f, x0, y0, nx, ny, isx, hx, hy, dhx, dhy)) continue;
    const int un = isx ? 1 : 2, ut = isx ? 2 : 1;
    int ya = hy + 2 * dhy, xa = hx + 2 * dhx, yb = hy + 3 * dhy, xb = hx + 3 * dhx;
    float rho_bar = 0.5f * (S.q[0][ya][xa] + S.q[0][yb][xb]);
    float c_bar = 0.5f * (S.q[6][ya][xa] + S.q[6][yb][xb]);
    float c2 = c_bar * c_bar, rc = rho_bar * c_bar;
    float inv = frcp(c2 * rc);
    float ic2 = rc * inv, irc = c2 * inv;
    float q[2][NQ];
    int code[2];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      float wt[NQ];
#pragma unroll
      for (int r = 0; r < NQ; ++r) wt[r] = S.w[side][r][f];
      back_project<NQ>(wt, ic2, irc, q[side]);
      code[side] = 0;
      if (a.mood && !admissible<NQ>(q[side])) {
        const float* qb = &S.q[0][hy][hx];
        if (isx)
          weno_side3<0>(qb, side, a.P, wt);
        else
          weno_side3<1>(qb, side, a.P, wt);
        back_project<NQ>(wt, ic2, irc, q[side]);
        code[side] = 1;
        if (!admissible<NQ>(q[side])) {
          int yy = side == 0 ? ya : yb, xx = side == 0 ? xa : xb;
          q[side][0] = S.q[0][yy][xx];
          q[side][1] = S.q[un][yy][xx];
          q[side][2] = S.q[ut][yy][xx];
          q[side][3] = S.q[3][yy][xx];
          q[side][4] = S.q[4][yy][xx];
          q[side][5] = S.q[5][yy][xx];
          code[side] = 2;
        }
      }
    }
    float Fh[NQ], us;
    hllc<NQ>(q[0], q[1], Fh, us);
    uint8_t mb = (uint8_t)(code[0] | (code[1] << 2));
    if (isx) {
      int j = hy - NG, i = hx;
#pragma unroll
      for (int m = 0; m < NQ; ++m) S.fx[m][j][i] = Fh[m];
      S.fx[NQ][j][i] = us;
      if (a.mask_x) a.mask_x[(int64_t)(y0 + j) * (nx + 1) + (x0 + i)] = mb;
    } else {
      int j = hy, i = hx - NG;
      S.fy[0][j][i] = Fh[0];
      S.fy[1][j][i] = Fh[2];  // rho u
      S.fy[2][j][i] = Fh[1];  // rho v
      S.fy[3][j][i] = Fh[3];
      S.fy[4][j][i] = Fh[4];
      S.fy[5][j][i] = Fh[5];
      S.fy[NQ][j][i] = us;
      if (a.mask_y) a.mask_y[(int64_t)(y0 + j) * nx + (x0 + i)] = mb;
    }
  }
  __syncthreads();

  // ---- phase C: flux divergence and RK stage ----
  const float idx = a.idx, idy = a.idy;
  for (int c = tid; c < TX * TY; c += NT) {
    int j = c / TX, i = c - j * TX;
    int gx = x0 + i, gy = y0 + j;
    if (gx >= nx || gy >= ny) continue;
    int64_t gi = (int64_t)(NG + gy) * P0 + (NG + gx);
    float div_u = (S.fx[NQ][j][i + 1] - S.fx[NQ][j][i]) * idx + (S.fy[NQ][j + 1][i] - S.fy[NQ][j][i]) * idy;
    float inc[NQ];
#pragma unroll
    for (int m = 0; m < NQ; ++m) {
      float L = -(S.fx[m][j][i + 1] - S.fx[m][j][i]) * idx;
      L = fmaf(-(S.fy[m][j + 1][i] - S.fy[m][j][i]), idy, L);
      if (m >= 4) L = fmaf(S.q[m][j + NG][i + NG], div_u, L);
      inc[m] = L;
    }
    if (a.stage == 0) {
#pragma unroll
      for (int m = 0; m < NQ; ++m) a.Kout[m * N + gi] = inc[m];
    } else if (a.stage == 1) {
#pragma unroll
      for (int m = 0; m < NQ; ++m) a.Kout[m * N + gi] = a.Kin[m * N + gi] + inc[m];
    } else {
      // this cell's U^n is read only here, by this thread, so U is updated in place
      float d[NQ];
#pragma unroll
      for (int m = 0; m < NQ; ++m) {
        d[m] = dt * fmaf(1.0f / 6.0f, a.Kin[m * N + gi], (2.0f / 3.0f) * inc[m]);
        a.U[m * N + gi] = a.U[m * N + gi] + f32_to_f64(d[m]);  // FP64 accumulation
      }
      // admissibility of the new state (rho > 0, Gamma > 0, (Gamma+1) p + Pi > 0)
      // from its FP32 image: a diagnostic, not part of the update
      const float* V = a.U32;
      float rho = V[gi] + d[0], mu = V[N + gi] + d[1], mv = V[2 * N + gi] + d[2];
      float eint = V[3 * N + gi] + (d[3] - d[5]), Gam = V[4 * N + gi] + d[4], Pi = V[5 * N + gi] + d[5];
      float pe = fmaf(-0.5f, (mu * mu + mv * mv) * frcp(rho), eint);  // Gamma p
      bool ok = rho > 0.0f && Gam > 0.0f && fmaf(Gam + 1.0f, pe * frcp(Gam), Pi) > 0.0f;
      if (!ok) atomicAdd(a.nbad, 1ULL);
    }
  }
}

}  // namespace

int fused2d_smem_bytes() { return (int)sizeof(Smem); }

cudaError_t fused2d_prepare() {
  return cudaFuncSetAttribute(k_stage2d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
}

void launch_stage2d(const GridDev& g, int stage, double* U, float* U32, const float* Kin, float* Kout,
                    double dt_fixed, double cfl, unsigned long long* lmax, double* dt_out, uint8_t* mask_x,
                    uint8_t* mask_y, float eps_rel, int mood, int weights, unsigned long long* nbad,
                    cudaStream_t s) {
  StageArgs a;
  a.g = g;
  a.stage = stage;
  a.idx = (float)(1.0 / g.dx[0]);
  a.idy = (float)(1.0 / g.dx[1]);
  a.cfl = (float)cfl;
  a.dt_fixed = dt_fixed;
  a.lmax = lmax;
  a.dt_out = dt_out;
  a.U = U;
  a.U32 = U32;
  a.Kin = Kin;
  a.Kout = Kout;
  a.mask_x = mask_x;
  a.mask_y = mask_y;
  a.P = WenoParams{eps_rel, 1e-30f, weights};
  a.mood = mood;
  a.nbad = nbad;
  dim3 grid((g.n[0] + TX - 1) / TX, (g.n[1] + TY - 1) / TY);
  k_stage2d<<<grid, NT, sizeof(Smem), s>>>(a);
}

}  // namespace ws
