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

#include <cuda_bf16.h>

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

// learned gate: BF16 MMA fragments of the MLP weights (m16n8k16, 32 lanes)
constexpr int NFRAG1 = 2 * 4, NFRAG2 = 2 * 4, NFRAG3 = 2;  // (k-step, n-tile) pairs per layer
constexpr int NFRAG = NFRAG1 + NFRAG2 + NFRAG3;
constexpr int NMT = (NF + 15) / 16;  // 16-face M tiles

template <bool LEARNED>
struct Smem {
  float q[NQ + 1][HY][HX];        // primitives + sound speed of tile and halo
  float fx[NQ + 1][TY][TX + 1];   // x-face fluxes (global field order) + face velocity
  float fy[NQ + 1][TY + 1][TX];   // y-face fluxes + face velocity
  union {
    struct {                      // plain kernel: this tile's own cells, for phase C
      double u[NQ][TY][TX];       // stage 2: FP64 state, copied in asynchronously from the start
      float k[NQ][TY][TX];        // stages 1, 2: accumulated increments (kept from the phase-A loads)
      float v[NQ][TY][TX];        // stage 2: FP32 image of U^n (kept from the phase-A loads)
    } own;
    __nv_bfloat16 feat[NF][24];   // learned kernel: gate inputs (read before the reconstruction)
  };
  unsigned long long red[NT / 32];  // per-warp CFL maxima
  float dt;                         // the step, broadcast from thread 0
};

struct SmemGate {
  uint2 frag[NFRAG][32];            // weight fragments
  float b1[32], b2[32], b3;         // biases
  uint8_t smooth[NF];               // 1: the face takes the linear weights
  float red[4][NT / 32];             // per-warp sums: |linear - WENO-IS|, |WENO-IS|, smooth faces, faces
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
  // learned gate
  const uint2* mlp_frag;   // NFRAG x 32 fragments, then biases (as floats) -- see ws_set_mlp
  const float* mlp_bias;   // b1[32], b2[32], b3
  float thr;               // logit threshold: smooth when logit < thr
  int drift_tile;          // tiles with (tile id % 64) == drift_tile run the drift check
  double* Ubackup;         // stage 0: copy of U (for a plain redo)
  float* lstat;            // [0] gated faces failing MOOD, [1] drift |lin - full|, [2] drift |full|,
                           // [3] smooth-gated faces, [4] gated faces examined
  const int* run_if;       // nullable: the CTA returns at once when *run_if == 0
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
// whether the face is an x face; false if the face lies outside the grid.
// Faces are numbered so that every 32-face chunk (a warp's share) is one row
// of one orientation: x faces 0..TX-1 of the TY rows, then the TY+1 rows of y
// faces, then the TY right-most x faces.
__device__ __forceinline__ bool face_geom(int f, int x0, int y0, int nx, int ny, bool& isx, int& hx, int& hy,
                                          int& dhx, int& dhy) {
  if (f < TX * TY || f >= TX * TY + NFY) {
    int j, i;
    if (f < TX * TY) {
      j = f / TX;
      i = f - j * TX;
    } else {
      j = f - TX * TY - NFY;
      i = TX;
    }
    isx = true;
    hx = i;  // cell k at hx + k
    hy = j + NG;
    dhx = 1;
    dhy = 0;
    return (x0 + i - 1 <= nx - 1) && (y0 + j < ny);
  }
  int ff = f - TX * TY;
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

// Per-face averages of the characteristic projection: rho c and -1/c^2 at
// the face (arithmetic means of cells i and i+1), shared by all variables.
struct FaceAvg {
  float rc;    // rho_bar c_bar
  float mic2;  // -1 / c_bar^2
};

// Orientation of a face, resolved at run time so that x and y faces share one
// copy of the reconstruction code: offsets of the six stencil cells in the
// halo tile and the normal / tangential velocity fields.
struct FaceGeo {
  int off[6];
  int un, ut;
};

// Characteristic variable R of the six stencil cells as mirrored pairs
// p[k] = (w_k, w_{5-k}), k = 0..4: the .x lanes are the left stencil
// w_0..w_4, the .y lanes the right stencil w_5..w_1.
template <int R>
__device__ __forceinline__ void project_pairs(const float* qb, const FaceGeo& fg, const FaceAvg& fa, float2 (&p)[5]) {
  constexpr int FS = HY * HX;
  auto cell = [&](const float* b, int k) { return make_float2(b[fg.off[k]], b[fg.off[5 - k]]); };
  if (R == 0 || R == NQ - 1) {
    float2 rc = f2(R == 0 ? -fa.rc : fa.rc);
#pragma unroll
    for (int k = 0; k < 5; ++k) p[k] = mul2(f2(0.5f), fma2(rc, cell(qb + fg.un * FS, k), cell(qb + 3 * FS, k)));
  } else if (R == 1) {
#pragma unroll
    for (int k = 0; k < 5; ++k) p[k] = fma2(f2(fa.mic2), cell(qb + 3 * FS, k), cell(qb, k));
  } else if (R == 2) {  // shear
#pragma unroll
    for (int k = 0; k < 5; ++k) p[k] = cell(qb + fg.ut * FS, k);
  } else {  // Gamma, Pi
#pragma unroll
    for (int k = 0; k < 5; ++k) p[k] = cell(qb + (R + 1) * FS, k);
  }
}

// 5th-order reconstruction of variable R on both sides of a face.  A
// stencil flat to 1e-6 of its magnitude (a few FP32 ulps: rounding noise)
// takes the linear weights, from which WENO-IS differs there by less than
// the stencil's range; elsewhere WENO-IS.
template <int R>
__device__ __forceinline__ void weno_item(const float* qb, const FaceGeo& fg, const FaceAvg& fa, const WenoParams& P,
                                          float& l5, float& r5) {
  float2 p[5];
  project_pairs<R>(qb, fg, fa, p);
  float mn = fminf(fmin3(p[0].x, p[1].x, p[2].x), fmin3(p[2].y, p[1].y, p[0].y));
  float mx = fmaxf(fmax3(p[0].x, p[1].x, p[2].x), fmax3(p[2].y, p[1].y, p[0].y));
  float2 v;
  if (mx - mn <= 1e-6f * fmaxf(fabsf(mx), fabsf(mn)))
    v = linear5_pair(p[0], p[1], p[2], p[3], p[4]);
  else
    v = weno5_pair(p[0], p[1], p[2], p[3], p[4], P);
  l5 = v.x;
  r5 = v.y;
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

// the (at most HPT) halo cells a thread owns in phase A
constexpr int HPT = (HX * HY + NT - 1) / NT;

__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint2 b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b.x), "r"(b.y));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// gate inputs of one face: w1, w2, w6, w_Gamma of the six stencil cells, each
// normalised over the stencil (zero for a stencil flat to 1e-6)
template <int D>
__device__ __forceinline__ void gate_features(const float* qb, __nv_bfloat16* out) {
  constexpr int ST = D == 0 ? 1 : HX;
  constexpr int FS = HY * HX;
  constexpr int UN = D == 0 ? 1 : 2;
  float rho_bar = 0.5f * (qb[2 * ST] + qb[3 * ST]);
  float c_bar = 0.5f * (qb[6 * FS + 2 * ST] + qb[6 * FS + 3 * ST]);
  float rc = rho_bar * c_bar, mic2 = -frcp(c_bar * c_bar);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    float w[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float p = qb[3 * FS + k * ST];
      if (v == 0) w[k] = 0.5f * fmaf(-rc, qb[UN * FS + k * ST], p);
      else if (v == 1) w[k] = fmaf(mic2, p, qb[k * ST]);
      else if (v == 2) w[k] = 0.5f * fmaf(rc, qb[UN * FS + k * ST], p);
      else w[k] = qb[4 * FS + k * ST];
    }
    float mn = w[0], mx = w[0], sum = w[0];
#pragma unroll
    for (int k = 1; k < 6; ++k) {
      mn = fminf(mn, w[k]);
      mx = fmaxf(mx, w[k]);
      sum += w[k];
    }
    float mean = sum * (1.0f / 6.0f);
    float inv = (mx - mn) > 1e-6f * fmaxf(fabsf(mx), fabsf(mn)) ? frcp((mx - mn) + 1e-30f) : 0.0f;
#pragma unroll
    for (int k = 0; k < 6; k += 2) {
      __nv_bfloat162 pr = __floats2bfloat162_rn((w[k] - mean) * inv, (w[k + 1] - mean) * inv);
      *reinterpret_cast<__nv_bfloat162*>(&out[v * 6 + k]) = pr;
    }
  }
}

// 5th-order linear-weight reconstruction of variable R on both sides
template <int R>
__device__ __forceinline__ void linear_item(const float* qb, const FaceGeo& fg, const FaceAvg& fa, float& l5,
                                            float& r5) {
  float2 p[5];
  project_pairs<R>(qb, fg, fa, p);
  float2 v = linear5_pair(p[0], p[1], p[2], p[3], p[4]);
  l5 = v.x;
  r5 = v.y;
}

// Asynchronous 8-byte global -> shared copy (holds no register while in flight)
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <bool LEARNED>
__global__ void __launch_bounds__(NT, 2) k_stage2d(StageArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<LEARNED>& S = *reinterpret_cast<Smem<LEARNED>*>(smem_raw);
  SmemGate& SG = *reinterpret_cast<SmemGate*>(smem_raw + sizeof(Smem<LEARNED>));
  if (a.run_if && *a.run_if == 0) return;  // a conditional redo that is not needed
  const GridDev& g = a.g;
  const int nx = g.n[0], ny = g.n[1];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int64_t N = g.N, P0 = g.P[0];
  const int tid = threadIdx.x;
  if (a.stage == 1 || a.stage == 2) {
    if (tid == 0) {  // one FP64 division per CTA
      double d = a.dt_fixed > 0.0 ? a.dt_fixed : (double)a.cfl / __longlong_as_double((long long)*a.lmax);
      if (a.stage == 1 && blockIdx.x == 0 && blockIdx.y == 0) *a.dt_out = d;
      S.dt = f64_to_f32(d);
    }
    __syncthreads();
  }
  // plain kernel, stage 2: the own cells' FP64 state, needed only in phase C,
  // is copied into shared memory while phases A and B run
  constexpr bool CACHE = !LEARNED;
  if (CACHE && a.stage == 2) {
    for (int c = tid; c < TX * TY; c += NT) {
      int j = c / TX, i = c - j * TX;
      if (x0 + i >= nx || y0 + j >= ny) continue;
      int64_t gi = (int64_t)(NG + y0 + j) * P0 + (NG + x0 + i);
#pragma unroll
      for (int m = 0; m < NQ; ++m) cp_async8(&S.own.u[m][j][i], &a.U[m * N + gi]);
    }
    cp_async_commit();
  }
  const float dt = (a.stage == 1 || a.stage == 2) ? S.dt : 0.0f;
  const float coef = a.stage == 0 ? 0.0f : (a.stage == 1 ? dt : 0.25f * dt);
  float lam_max = 0.0f;

  // ---- phase A: stage-state primitives of tile + halo ----
  // A thread owns up to HPT halo cells; all their global loads are issued
  // before any of them is used, so that a CTA has its whole halo in flight.
  {
    float ld[HPT][NQ];
    float rk[HPT][NQ], rv[HPT][NQ];  // stages 1, 2: increment and FP32 image as loaded
    int hh[HPT];
    bool flx[HPT], fly[HPT], own[HPT];
#pragma unroll
    for (int t = 0; t < HPT; ++t) {
      int h = tid + t * NT;
      int hy = h / HX, hx = h - hy * HX;
      int gx = x0 + hx - NG, gy = y0 + hy - NG;
      bool outx = gx < 0 || gx >= nx, outy = gy < 0 || gy >= ny;
      hh[t] = (h < HX * HY && !(outx && outy)) ? h : -1;  // corners are never read
      if (hh[t] < 0) continue;
      bool fx = false, fy = false;
      int mx = map_bc(gx, nx, g.bc[0][0], g.bc[0][1], fx);
      int my = map_bc(gy, ny, g.bc[1][0], g.bc[1][1], fy);
      flx[t] = fx;
      fly[t] = fy;
      int64_t i = (int64_t)(NG + my) * P0 + (NG + mx);
      if (a.stage == 0 || a.stage == 3) {
        const double* U = a.U;
        ld[t][0] = f64_to_f32(U[i]);
        ld[t][1] = f64_to_f32(U[N + i]);
        ld[t][2] = f64_to_f32(U[2 * N + i]);
        ld[t][3] = f64_to_f32(U[3 * N + i] - U[5 * N + i]);  // E - Pi in FP64
        ld[t][4] = f64_to_f32(U[4 * N + i]);
        ld[t][5] = f64_to_f32(U[5 * N + i]);
        own[t] = a.stage == 0 && hx >= NG && hx < NG + TX && hy >= NG && hy < NG + TY && !outx && !outy;
        if (LEARNED && own[t]) {
#pragma unroll
          for (int m = 0; m < NQ; ++m) a.Ubackup[m * N + i] = U[m * N + i];
        }
        if (own[t]) {
#pragma unroll
          for (int m = 0; m < NQ; ++m) a.U32[m * N + i] = ld[t][m];
        }
      } else {
        own[t] = hx >= NG && hx < NG + TX && hy >= NG && hy < NG + TY && !outx && !outy;
#pragma unroll
        for (int m = 0; m < NQ; ++m) {
          rk[t][m] = __ldg(&a.Kin[m * N + i]);
          rv[t][m] = __ldg(&a.U32[m * N + i]);
        }
      }
    }
    if (a.stage == 1 || a.stage == 2) {
#pragma unroll
      for (int t = 0; t < HPT; ++t) {
        if (hh[t] < 0) continue;
        ld[t][0] = fmaf(coef, rk[t][0], rv[t][0]);
        ld[t][1] = fmaf(coef, rk[t][1], rv[t][1]);
        ld[t][2] = fmaf(coef, rk[t][2], rv[t][2]);
        ld[t][3] = fmaf(coef, rk[t][3] - rk[t][5], rv[t][3]);
        ld[t][4] = fmaf(coef, rk[t][4], rv[t][4]);
        ld[t][5] = fmaf(coef, rk[t][5], rv[t][5]);
        if (CACHE && own[t]) {  // phase C reads these instead of global memory
          int j = hh[t] / HX - NG, i = hh[t] % HX - NG;
#pragma unroll
          for (int m = 0; m < NQ; ++m) {
            S.own.k[m][j][i] = rk[t][m];
            if (a.stage == 2) S.own.v[m][j][i] = rv[t][m];
          }
        }
      }
    }
#pragma unroll
    for (int t = 0; t < HPT; ++t) {
      if (hh[t] < 0) continue;
      int hy = hh[t] / HX, hx = hh[t] - hy * HX;
      float rho = ld[t][0], eint = ld[t][3], Gam = ld[t][4], Pi = ld[t][5];
      float irho = frcp(rho);
      float u = ld[t][1] * irho, v = ld[t][2] * irho;
      if (flx[t]) u = -u;
      if (fly[t]) v = -v;
      float p = fmaf(-0.5f * rho, fmaf(u, u, v * v), eint) * frcp(Gam);
      S.q[0][hy][hx] = rho;
      S.q[1][hy][hx] = u;
      S.q[2][hy][hx] = v;
      S.q[3][hy][hx] = p;
      S.q[4][hy][hx] = Gam;
      S.q[5][hy][hx] = Pi;
      float c = fsqrt(sound_speed2(rho, p, Gam, Pi));
      S.q[6][hy][hx] = c;
      int gx = x0 + hx - NG, gy = y0 + hy - NG;
      if (a.stage == 0 && hx >= NG && hx < NG + TX && hy >= NG && hy < NG + TY && gx < nx && gy < ny) {
        float lam = fmaf(fabsf(u) + c, a.idx, (fabsf(v) + c) * a.idy);
        if (!(lam <= lam_max)) lam_max = lam;  // NaN propagates
      }
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

  // ---- phases G1, G2 (learned gate): features, then the BF16 tensor-core MLP ----
  if (LEARNED) {
    for (int i = tid; i < NFRAG * 32; i += NT) SG.frag[i / 32][i % 32] = a.mlp_frag[i];
    for (int i = tid; i < 65; i += NT) {
      float b = a.mlp_bias[i];
      if (i < 32) SG.b1[i] = b;
      else if (i < 64) SG.b2[i - 32] = b;
      else SG.b3 = b;
    }
    for (int f = tid; f < NF; f += NT) {
      bool isx;
      int hx, hy, dhx, dhy;
      SG.smooth[f] = 0;
      if (!face_geom(f, x0, y0, nx, ny, isx, hx, hy, dhx, dhy)) continue;
      const float* qb = &S.q[0][hy][hx];
      if (isx)
        gate_features<0>(qb, S.feat[f]);
      else
        gate_features<1>(qb, S.feat[f]);
    }
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5, g8 = lane >> 2, t4 = lane & 3;
    for (int mt = warp; mt < NMT; mt += NT / 32) {
      int r0 = min(mt * 16 + g8, NF - 1), r1 = min(mt * 16 + g8 + 8, NF - 1);
      const uint32_t* x0p = reinterpret_cast<const uint32_t*>(S.feat[r0]);
      const uint32_t* x1p = reinterpret_cast<const uint32_t*>(S.feat[r1]);
      // layer 1: [16 x 24(32)] x [24(32) x 32]
      float h[4][4];
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        h[nt][0] = h[nt][1] = h[nt][2] = h[nt][3] = 0.0f;
        mma16816(h[nt], x0p[t4], x1p[t4], x0p[t4 + 4], x1p[t4 + 4], SG.frag[nt][lane]);
        mma16816(h[nt], x0p[t4 + 8], x1p[t4 + 8], 0u, 0u, SG.frag[4 + nt][lane]);
      }
      uint32_t A[2][4];
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        float b0 = SG.b1[nt * 8 + 2 * t4], b1 = SG.b1[nt * 8 + 2 * t4 + 1];
        uint32_t lo = pack_bf16(fmaxf(h[nt][0] + b0, 0.0f), fmaxf(h[nt][1] + b1, 0.0f));
        uint32_t hi = pack_bf16(fmaxf(h[nt][2] + b0, 0.0f), fmaxf(h[nt][3] + b1, 0.0f));
        A[nt >> 1][(nt & 1) * 2 + 0] = lo;
        A[nt >> 1][(nt & 1) * 2 + 1] = hi;
      }
      // layer 2: [16 x 32] x [32 x 32]
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        h[nt][0] = h[nt][1] = h[nt][2] = h[nt][3] = 0.0f;
        mma16816(h[nt], A[0][0], A[0][1], A[0][2], A[0][3], SG.frag[NFRAG1 + nt][lane]);
        mma16816(h[nt], A[1][0], A[1][1], A[1][2], A[1][3], SG.frag[NFRAG1 + 4 + nt][lane]);
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        float b0 = SG.b2[nt * 8 + 2 * t4], b1 = SG.b2[nt * 8 + 2 * t4 + 1];
        uint32_t lo = pack_bf16(fmaxf(h[nt][0] + b0, 0.0f), fmaxf(h[nt][1] + b1, 0.0f));
        uint32_t hi = pack_bf16(fmaxf(h[nt][2] + b0, 0.0f), fmaxf(h[nt][3] + b1, 0.0f));
        A[nt >> 1][(nt & 1) * 2 + 0] = lo;
        A[nt >> 1][(nt & 1) * 2 + 1] = hi;
      }
      // layer 3: [16 x 32] x [32 x 1 (8)]
      float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      mma16816(z, A[0][0], A[0][1], A[0][2], A[0][3], SG.frag[NFRAG1 + NFRAG2][lane]);
      mma16816(z, A[1][0], A[1][1], A[1][2], A[1][3], SG.frag[NFRAG1 + NFRAG2 + 1][lane]);
      if (t4 == 0) {
        int f0 = mt * 16 + g8, f1 = f0 + 8;
        if (f0 < NF && (z[0] + SG.b3) < a.thr) SG.smooth[f0] = 1;
        if (f1 < NF && (z[2] + SG.b3) < a.thr) SG.smooth[f1] = 1;
      }
    }
    __syncthreads();
    if (a.stage == 3) {  // gate evaluation only: the decisions go to the mask arrays
      for (int f = tid; f < NF; f += NT) {
        bool isx;
        int hx, hy, dhx, dhy;
        if (!face_geom(f, x0, y0, nx, ny, isx, hx, hy, dhx, dhy)) continue;
        if (isx)
          a.mask_x[(int64_t)(y0 + hy - NG) * (nx + 1) + (x0 + hx)] = SG.smooth[f];
        else
          a.mask_y[(int64_t)(y0 + hy) * nx + (x0 + hx - NG)] = SG.smooth[f];
      }
      return;
    }
  }

  // ---- phase B: per face, WENO-IS per characteristic variable (B1), then
  // back-projection, MOOD and HLLC (B2).  The thread that reconstructs a face
  // also solves its Riemann problem, so no barrier separates the two and the
  // reconstructed characteristics stay in registers.
  const bool drift = LEARNED && ((int)((blockIdx.y * gridDim.x + blockIdx.x) & 63) == a.drift_tile);
  float dnum = 0.0f, dden = 0.0f, nsm = 0.0f, nval = 0.0f;
  const float* q0 = &S.q[0][0][0];
#pragma unroll 1
  for (int f = tid; f < NF; f += NT) {
    bool isx;
    int hx, hy, dhx, dhy;
    if (!face_geom(f, x0, y0, nx, ny, isx, hx, hy, dhx, dhy)) continue;
    const int qo = hy * HX + hx;  // stencil cell 0 in the halo tile
    const bool sm = LEARNED && SG.smooth[f];
    float wl[NQ], wr[NQ];  // reconstructed characteristics, left and right
    const int un = isx ? 1 : 2, ut = isx ? 2 : 1;
    int ya = hy + 2 * dhy, xa = hx + 2 * dhx, yb = hy + 3 * dhy, xb = hx + 3 * dhx;
    float rho_bar = 0.5f * (S.q[0][ya][xa] + S.q[0][yb][xb]);
    float c_bar = 0.5f * (S.q[6][ya][xa] + S.q[6][yb][xb]);
    float c2 = c_bar * c_bar, rc = rho_bar * c_bar;
    float inv = frcp(c2 * rc);
    float ic2 = rc * inv, irc = c2 * inv;  // 1/c^2, 1/(rho c)
    const FaceAvg fa{rc, -ic2};
    FaceGeo fg;
    {
      const int st = isx ? 1 : HX;
#pragma unroll
      for (int k = 0; k < 6; ++k) fg.off[k] = k * st;
      fg.un = un;
      fg.ut = ut;
    }
    if (LEARNED) {
      nval += 1.0f;
      nsm += sm ? 1.0f : 0.0f;
    }
#define WS_B1(R)                                                          \
    {                                                                     \
      float l5, r5;                                                       \
      bool lin = LEARNED && R != 2 && sm; /* shear: always WENO-IS */     \
      if (lin) {                                                          \
        linear_item<R>(q0 + qo, fg, fa, l5, r5);                             \
      }                                                                   \
      if (!lin || drift) {                                                \
        float fl, fr;                                                     \
        weno_item<R>(q0 + qo, fg, fa, a.P, fl, fr);                          \
        if (lin) {                                                        \
          dnum += fabsf(l5 - fl) + fabsf(r5 - fr);                        \
          dden += fabsf(fl) + fabsf(fr);                                  \
        } else {                                                          \
          l5 = fl;                                                        \
          r5 = fr;                                                        \
        }                                                                 \
      }                                                                   \
      wl[R] = l5;                                                         \
      wr[R] = r5;                                                         \
    }
    WS_B1(0)
    WS_B1(1)
    WS_B1(2)
    WS_B1(3)
    WS_B1(4)
    WS_B1(5)
#undef WS_B1

    float2 W[NQ], Q[NQ];  // (left, right) characteristics, then primitives
#pragma unroll
    for (int r = 0; r < NQ; ++r) W[r] = make_float2(wl[r], wr[r]);
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
          if (LEARNED && sm) atomicAdd(&a.lstat[0], 1.0f);
          float wt[NQ];
          const float* qb = &S.q[0][hy][hx];
          if (isx)
            weno_side3<0>(qb, side, a.P, wt);
          else
            weno_side3<1>(qb, side, a.P, wt);
          float q3[NQ];
          back_project<NQ>(wt, ic2, irc, q3);
          code[side] = 1;
          if (!admissible<NQ>(q3)) {
            int yy = side == 0 ? ya : yb, xx = side == 0 ? xa : xb;
            q3[0] = S.q[0][yy][xx];
            q3[1] = S.q[un][yy][xx];
            q3[2] = S.q[ut][yy][xx];
            q3[3] = S.q[3][yy][xx];
            q3[4] = S.q[4][yy][xx];
            q3[5] = S.q[5][yy][xx];
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
  if (LEARNED) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dnum += __shfl_xor_sync(0xffffffffu, dnum, o);
      dden += __shfl_xor_sync(0xffffffffu, dden, o);
      nsm += __shfl_xor_sync(0xffffffffu, nsm, o);
      nval += __shfl_xor_sync(0xffffffffu, nval, o);
    }
    if ((tid & 31) == 0) {
      SG.red[0][tid >> 5] = dnum;
      SG.red[1][tid >> 5] = dden;
      SG.red[2][tid >> 5] = nsm;
      SG.red[3][tid >> 5] = nval;
    }
  }
  if (CACHE && a.stage == 2) cp_async_wait_all();  // own FP64 state, visible after the barrier
  __syncthreads();
  if (LEARNED && tid < 4) {
    float sum = 0.0f;
    for (int w = 0; w < NT / 32; ++w) sum += SG.red[tid][w];
    if (tid >= 2 || drift) atomicAdd(&a.lstat[1 + tid], sum);
  }

  // ---- phase C: flux divergence and RK stage (variables in pairs) ----
  const float2 idx = f2(a.idx), idy = f2(a.idy);
  for (int c = tid; c < TX * TY; c += NT) {
    int j = c / TX, i = c - j * TX;
    int gx = x0 + i, gy = y0 + j;
    if (gx >= nx || gy >= ny) continue;
    int64_t gi = (int64_t)(NG + gy) * P0 + (NG + gx);
    float div_u = (S.fx[NQ][j][i + 1] - S.fx[NQ][j][i]) * a.idx + (S.fy[NQ][j + 1][i] - S.fy[NQ][j][i]) * a.idy;
    float2 inc[NQ / 2];
#pragma unroll
    for (int k = 0; k < NQ / 2; ++k) {
      const int m = 2 * k;
      float2 L = mul2(sub2(make_float2(S.fx[m][j][i], S.fx[m + 1][j][i]),
                           make_float2(S.fx[m][j][i + 1], S.fx[m + 1][j][i + 1])), idx);
      L = fma2(sub2(make_float2(S.fy[m][j][i], S.fy[m + 1][j][i]), make_float2(S.fy[m][j + 1][i], S.fy[m + 1][j + 1][i])),
               idy, L);
      if (m >= 4) L = fma2(make_float2(S.q[m][j + NG][i + NG], S.q[m + 1][j + NG][i + NG]), f2(div_u), L);
      inc[k] = L;
    }
    auto kin = [&](int m) { return CACHE ? S.own.k[m][j][i] : a.Kin[m * N + gi]; };
    if (a.stage == 0) {
#pragma unroll
      for (int k = 0; k < NQ / 2; ++k) {
        a.Kout[2 * k * N + gi] = inc[k].x;
        a.Kout[(2 * k + 1) * N + gi] = inc[k].y;
      }
    } else if (a.stage == 1) {
#pragma unroll
      for (int k = 0; k < NQ / 2; ++k) {
        float2 K1 = add2(make_float2(kin(2 * k), kin(2 * k + 1)), inc[k]);
        a.Kout[2 * k * N + gi] = K1.x;
        a.Kout[(2 * k + 1) * N + gi] = K1.y;
      }
    } else {
      // this cell's U^n is read only here, by this thread, so U is updated in place
      float d[NQ];
#pragma unroll
      for (int k = 0; k < NQ / 2; ++k) {
        float2 dd = mul2(f2(dt), fma2(f2(1.0f / 6.0f), make_float2(kin(2 * k), kin(2 * k + 1)),
                                      mul2(f2(2.0f / 3.0f), inc[k])));
        d[2 * k] = dd.x;
        d[2 * k + 1] = dd.y;
      }
#pragma unroll
      for (int m = 0; m < NQ; ++m) {
        double u = CACHE ? S.own.u[m][j][i] : a.U[m * N + gi];
        a.U[m * N + gi] = u + f32_to_f64(d[m]);  // FP64 accumulation
      }
      // admissibility of the new state (rho > 0, Gamma > 0, (Gamma+1) p + Pi > 0)
      // from its FP32 image: a diagnostic, not part of the update
      auto v = [&](int m) { return CACHE ? S.own.v[m][j][i] : a.U32[m * N + gi]; };
      float rho = v(0) + d[0], mu = v(1) + d[1], mv = v(2) + d[2];
      float eint = v(3) + (d[3] - d[5]), Gam = v(4) + d[4], Pi = v(5) + d[5];
      float pe = fmaf(-0.5f, (mu * mu + mv * mv) * frcp(rho), eint);  // Gamma p
      bool ok = rho > 0.0f && Gam > 0.0f && fmaf(Gam + 1.0f, pe * frcp(Gam), Pi) > 0.0f;
      if (!ok) atomicAdd(a.nbad, 1ULL);
    }
  }
}

}  // namespace

// After a gated step: decide on the device whether to redo it without the gate
// (no host round trip), and keep the gate statistics.
static __global__ void k_gate_decide(const float* __restrict__ lstat, unsigned long long* nbad, unsigned long long* lmax,
                              int flags, int* redo, double* stats) {
  bool r = false;
  double drift = lstat[2] > 0.0f ? (double)lstat[1] / (double)lstat[2] : 0.0;
  if ((flags & WS_GATE_REDO_MOOD) && lstat[0] > 0.0f) r = true;
  if ((flags & WS_GATE_REDO_DRIFT) && drift > 1e-6) r = true;
  if ((flags & WS_GATE_REDO_NONPHYS) && *nbad > 0ULL) r = true;
  *redo = r ? 1 : 0;
  stats[0] += 1.0;
  stats[1] += r ? 1.0 : 0.0;
  stats[2] += lstat[3];
  stats[3] += lstat[4];
  stats[4] = drift > stats[4] ? drift : stats[4];
  stats[5] += lstat[5];
  if (r) {
    *nbad = 0ULL;
    *lmax = 0ULL;
  }
}

static __global__ void k_restore(const int* __restrict__ redo, const double* __restrict__ src, double* __restrict__ dst,
                          int64_t n) {
  if (*redo == 0) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

void launch_gate_decide(const float* lstat, unsigned long long* nbad, unsigned long long* lmax, int flags, int* redo,
                        double* stats, cudaStream_t s) {
  k_gate_decide<<<1, 1, 0, s>>>(lstat, nbad, lmax, flags, redo, stats);
}

void launch_restore(const int* redo, const double* src, double* dst, int64_t n, cudaStream_t s) {
  k_restore<<<152 * 4, 256, 0, s>>>(redo, src, dst, n);
}

int fused2d_smem_bytes() { return (int)(sizeof(Smem<true>) + sizeof(SmemGate)); }

cudaError_t fused2d_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_stage2d<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(Smem<false>));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_stage2d<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(sizeof(Smem<true>) + sizeof(SmemGate)));
}

void launch_stage2d(const GridDev& g, int stage, double* U, float* U32, const float* Kin, float* Kout,
                    double dt_fixed, double cfl, unsigned long long* lmax, double* dt_out, uint8_t* mask_x,
                    uint8_t* mask_y, float eps_rel, int mood, int weights, unsigned long long* nbad,
                    const GateArgs* gate, const int* run_if, cudaStream_t s) {
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
  a.run_if = run_if;
  if (gate) {
    a.mlp_frag = gate->frag;
    a.mlp_bias = gate->bias;
    a.thr = gate->thr;
    a.drift_tile = gate->drift_tile;
    a.Ubackup = gate->Ubackup;
    a.lstat = gate->lstat;
    k_stage2d<true><<<grid, NT, sizeof(Smem<true>) + sizeof(SmemGate), s>>>(a);
  } else {
    a.mlp_frag = nullptr;
    a.mlp_bias = nullptr;
    a.thr = 0.0f;
    a.drift_tile = -1;
    a.Ubackup = nullptr;
    a.lstat = nullptr;
    k_stage2d<false><<<grid, NT, sizeof(Smem<false>), s>>>(a);
  }
}

}  // namespace ws
