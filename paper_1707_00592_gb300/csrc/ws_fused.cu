// Fused mixed-precision RK stage: one kernel per SSP-RK3 stage in 2D, two in
// 3D.
//
// A CTA owns a TX x TY tile of cells and works through three phases separated
// by barriers, all in shared memory:
//   A  stage-state FP32 primitives of the tile plus a 3-cell halo; boundary
//      conditions are applied while loading (no ghost kernel), E - Pi in FP64;
//   B  per face: projection of the six stencil cells with L_{i+1/2}, 5th-order
//      WENO-IS of both sides (as the two lanes of paired FP32 instructions),
//      back-projection, MOOD cascade (a side that fails is reconstructed again
//      at 3rd order from the staged primitives), HLLC;
//   C  one thread per cell: flux divergence with the Gamma/Pi source and the
//      RK stage.
// Two 512-thread CTAs fit per SM, so one CTA's memory phases overlap the
// other's arithmetic.
//
// Passes (MODE):
//   0  2D: the tile spans x and y; x and y faces; phase C ends the stage.
//   1  3D, first pass: one z plane per CTA row (blockIdx.z); x and y faces;
//      phase C writes the x + y part of the divergence (with the Gamma/Pi
//      source of the x and y face velocities) to a scratch buffer.
//   2  3D, second pass: an x-z tile of one y plane; z faces only; phase C adds
//      the z part to the scratch and ends the stage.
// The directions are summed x, y, z, as Sec. 3.1 states the dimension-by-
// dimension divergence.
//
// Gate modes (GATE): 0 plain; 1 and 2 the learned smooth-face gate (the MLP
// evaluated in this launch, or decisions stored by an earlier stage of the
// step); 3 the census: the plain stage, bit for bit, that also counts per
// face-variable whether the stencil was flat (linear weights) or took
// WENO-IS, and per warp whether the WENO-IS branch ran.
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
//
// The FP32 buffers (image, K, the 3D partial divergence) have a layout of
// their own (GridDev st32, N32): their rows are padded to a multiple of four
// floats, so that the halo of every tile starts on a 16-byte boundary (padded
// column x0 - 3 + 3 = x0, a multiple of 32).  A tile whose halo lies inside
// the grid (in the second 3D pass: whose z halo does) then loads the image
// and K of tile and halo as two TMA boxes (cp.async.bulk.tensor, completion
// on an mbarrier) straight into shared memory, with no per-cell address
// arithmetic; tiles on the boundary and the FP64 loads of a first stage 0
// load cell by cell and apply the boundary conditions while loading.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <functional>
#include <queue>
#include <vector>

#include <cuda_bf16.h>

#include "face_fp32.cuh"
#include "ws_internal.h"

namespace ws {

namespace {

using namespace fp32;

// Tile shape and CTA size of a launch: TX x TY cells per CTA of NT threads.
// The per-face arithmetic does not depend on the tile (faces on tile edges
// are evaluated by both tiles, with the same operands), so every tile gives
// bit-identical results; ws_autotune chooses among them.
template <int TX_, int TY_, int NT_>
struct Tile {
  static constexpr int TX = TX_, TY = TY_, NT = NT_;
  static constexpr int HX = TX + 2 * NG, HY = TY + 2 * NG;
  static constexpr int HXP = (HX + 7) / 8 * 8;  // row pitch of the halo tile in shared memory (a TMA box row)
  static constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1), NF = NFX + NFY;
  static constexpr int NMT = (NF + 15) / 16;  // 16-face M tiles of the gate's MLP
};
using TileA = Tile<32, 15, 512>;   // two CTAs per SM (the default)
using TileB = Tile<32, 31, 1024>;  // one CTA per SM, 15 % fewer halo cells per cell
using TileC = Tile<32, 7, 256>;    // four CTAs per SM
using TileH = Tile<32, 7, 512>;    // the closing rows of a tail-filled launch (TileA's CTA size)

// Per-pass constants.  NQ: fields (rho, velocities, E or p, Gamma, Pi), 6 in
// 2D and 7 in 3D; the q tile holds them as primitives plus the sound speed.
template <int NQ_, int MODE, class TL>
struct Tr {
  static constexpr int TX = TL::TX, TY = TL::TY, NT = TL::NT, HX = TL::HX, HY = TL::HY;
  static constexpr int NFX = TL::NFX, NFY = TL::NFY, NF = TL::NF;
  static constexpr int NQ = NQ_;
  static constexpr int ND = NQ - 4;                 // velocity components
  static constexpr int NTG = NQ - 5;                // tangential components at a face
  static constexpr bool XF = MODE != 2;             // the pass has x faces (and an x halo)
  static constexpr int QW = XF ? HX : TX;           // cells of a q row that phase A fills
  static constexpr int QP = TL::HXP;                // row pitch of the q tile (a TMA box row)
  static constexpr int QX = NG;                     // q column of the tile's first cell
  static constexpr int QL = XF ? 0 : NG;            // q column of the first cell phase A fills
  static constexpr int NH = QW * HY;                // q tile cells
  static constexpr int FS = QP * HY;                // field stride in the q tile
  static constexpr int NFP = (XF ? NFX : 0) + NFY;  // faces of the pass
  static constexpr int HPT = (NH + NT - 1) / NT;    // q tile cells per thread in phase A
  static constexpr int IP = NQ - 3, IG = NQ - 2, IPI = NQ - 1, IC = NQ;  // q fields p, Gamma, Pi, c
  static constexpr bool RK = MODE != 1;             // phase C ends the stage
};

// learned gate (2D): BF16 MMA fragments of the MLP weights (m16n8k16, 32 lanes)
constexpr int NFRAG1 = 2 * 4, NFRAG2 = 2 * 4, NFRAG3 = 2;  // (k-step, n-tile) pairs per layer
constexpr int NFRAG = NFRAG1 + NFRAG2 + NFRAG3;

// GATE: 0 plain; 1 the learned gate evaluates the MLP in this launch; 2 the
// launch applies decisions stored by an earlier stage of the same step; 3 a
// plain launch that also counts the flat-stencil decisions (census).
template <int GATE, int NQ_, int MODE, class TL>
struct Smem {
  using T = Tr<NQ_, MODE, TL>;
  static constexpr int TX = TL::TX, TY = TL::TY, NT = TL::NT, HY = TL::HY, NF = TL::NF;
  static constexpr bool CACHE = GATE != 1 && T::RK;  // own cells staged for phase C
  // primitives + sound speed of tile and halo; in a TMA load, fields 0..NQ-1
  // first receive the stage's FP32 image, converted in place
  alignas(128) float q[NQ_ + 1][HY][T::QP];
  // x-face fluxes (global field order) + face velocity; in a TMA load, fx and
  // fy first receive the increments K of tile and halo (read in phase A)
  alignas(128) float fx[T::XF ? NQ_ + 1 : 1][TY][TX + 1];
  float fy[NQ_ + 1][TY + 1][TX];              // fluxes + face velocity of the faces along the tile's 2nd axis
  static constexpr bool OWNV = CACHE && MODE != 2;  // the own cells' image kept (the second 3D pass reads it)
  // the second pass's K box lies over k, v, l and this padding, not over u,
  // so that u can be copied in while the box is still being read
  static constexpr int KBOX = MODE == 2 ? (int)sizeof(float) * NQ_ * HY * T::QP : 0;
  static constexpr int KVL = (int)sizeof(float) * TY * TX * ((CACHE ? NQ_ : 1) + (OWNV ? NQ_ : 1)) +
                             (int)sizeof(float) * (MODE == 2 ? NQ_ * TY * TX : 1);
  static constexpr int PAD = KBOX > KVL ? (KBOX - KVL + 7) / 8 * 8 : 8;
  union alignas(128) {
    struct {                                     // this tile's own cells, for phase C
      float k[CACHE ? NQ_ : 1][TY][TX];          // stages 1, 2: accumulated increments (kept from the phase-A loads)
      float v[OWNV ? NQ_ : 1][TY][TX];           // stage 2: FP32 image of U^n (kept from the phase-A loads)
      // 3D second pass: x + y part of the divergence (asynchronous copy)
      float l[MODE == 2 ? NQ_ : 1][MODE == 2 ? TY : 1][MODE == 2 ? TX : 1];
      alignas(8) char pad[PAD];
      double u[CACHE ? NQ_ : 1][TY][TX];         // stage 2: FP64 state, copied in asynchronously
    } own;
    __nv_bfloat16 feat[GATE == 1 ? NF : 1][24];  // gate inputs (read before the reconstruction)
    // 3D second pass, TMA load: the increments K of tile and z halo, read in
    // phase A before the own cells' arrays are filled
    float kbox[MODE == 2 ? NQ_ : 1][MODE == 2 ? HY : 1][MODE == 2 ? T::QP : 1];
  };
  unsigned long long red[NT / 32];  // per-warp CFL maxima
  unsigned long long mbar;          // completion of the TMA loads
  float dt;                         // the step, broadcast from thread 0
};

// Two 2D stage CTAs of the default tile, with the 1 KiB the hardware keeps
// per CTA, fit the 196 KiB shared-memory carveout of an SM: the next larger
// carveout would leave the halo loads of boundary tiles 28 KiB of L1 instead
// of 60 (measured: 10 % slower per-thread loads).
static_assert(2 * (sizeof(Smem<0, 6, 0, Tile<32, 15, 512>>) + 1024) <= 196 * 1024,
              "the default 2D stage no longer leaves room for L1");
// The 3D passes keep their CTAs per SM: four of 32 x 7 cells, two of 32 x 15
// (228 KiB of shared memory per SM at most).
static_assert(4 * (sizeof(Smem<0, 7, 2, Tile<32, 7, 256>>) + 1024) <= 228 * 1024 &&
                  4 * (sizeof(Smem<0, 7, 1, Tile<32, 7, 256>>) + 1024) <= 228 * 1024,
              "a 32 x 7 3D pass no longer fits four CTAs per SM");
static_assert(2 * (sizeof(Smem<0, 7, 2, Tile<32, 15, 512>>) + 1024) <= 228 * 1024 &&
                  2 * (sizeof(Smem<0, 7, 1, Tile<32, 15, 512>>) + 1024) <= 228 * 1024,
              "a 32 x 15 3D pass no longer fits two CTAs per SM");

template <class TL>
struct SmemGate {
  static constexpr int NT = TL::NT, NF = TL::NF;
  uint2 frag[NFRAG][32];            // weight fragments
  float b1[32], b2[32], b3;         // biases
  uint8_t smooth[NF];               // 1: the face takes the linear weights
  float red[4][NT / 32];             // per-warp sums: |linear - WENO-IS|, |WENO-IS|, smooth faces, faces
  float dpart[2][NT];                // drift check, per thread: sum |linear - WENO-IS|, sum |WENO-IS|
};

struct StageArgs {
  GridDev g;
  int stage;
  float idx, idy, idz;  // 1/dx, 1/dy, 1/dz
  float cfl;
  double dt_fixed;    // > 0: use this step; otherwise CFL
  unsigned long long* lmax;  // stage 0: max wave rate (FP64 bits)
  double* dt_out;     // stage 1 (block 0): the dt used
  double* U;          // state at t^n; stage 2 replaces it with t^{n+1}
  float* U32;         // FP32 image of U^n (rho, momenta, E - Pi, Gamma, Pi): written in stage 0
  const float* Kin;   // stages 1, 2: accumulated increments
  float* Kout;        // stages 0, 1
  float* Lp;          // 3D: x + y part of the divergence (first pass writes, second reads)
  uint8_t* mask_x;    // nullable: MOOD levels of the pass's x faces
  uint8_t* mask_a;    // nullable: MOOD levels of the faces along the tile's 2nd axis (y, or z in pass 2)
  WenoParams P;
  int mood;
  unsigned long long* nbad;
  // learned gate
  const uint2* mlp_frag;   // NFRAG x 32 fragments, then biases (as floats) -- see ws_set_mlp
  const float* mlp_bias;   // b1[32], b2[32], b3
  float thr;               // logit threshold: smooth when logit < thr
  int drift_tile;          // tiles with (tile id % 64) == drift_tile run the drift check
  const int* drift_dev;    // nullable: the drift tile residue in device memory (overrides drift_tile)
  double* Ubackup;         // stage 0: copy of U (for a plain redo)
  float* lstat;            // [0] gated faces failing MOOD, [1] drift |lin - full|, [2] drift |full|,
                           // [3] smooth-gated faces, [4] gated faces examined
  const int* run_if;       // nullable: the CTA returns at once when *run_if == 0
  uint8_t* gflags;         // nullable: per-tile gate decisions (NF bytes per tile), written when the
                           // MLP runs, read by launches that reuse them
  int row0;                // first tile row of the launch (a launch may cover a band of tile rows)
  int img_in;              // stage 0: U32 already holds the FP32 image of U (carried from the previous step)
  float* img_out;          // nullable, stage 2 (the pass that ends it): receives the FP32 image of the new state
  unsigned long long* census;  // census launches: [0] face-variables, [1] those with a flat stencil,
                               // [2] warp passes over a variable, [3] those in which a face took WENO-IS
  // 2D: TMA descriptors of the stage's K (Kin) and FP32 image (U32) over the
  // FP32 layout, boxes of one tile's halo (all fields); tma = 0: every tile
  // loads cell by cell
  int tma;
  alignas(64) CUtensorMap tm_k;
  alignas(64) CUtensorMap tm_v;
  // a tail-filled 2D launch: tile rows of the first tile shape, and the
  // descriptors of the closing rows' boxes
  int rows_full;
  alignas(64) CUtensorMap tm_k2;
  alignas(64) CUtensorMap tm_v2;
  // nullable: slots block (0, 0, 0) clears once the previous grid has
  // completed (a step's last launch clears the next step's CFL maximum and
  // inadmissible-cell count, so consecutive steps need no memset between them)
  unsigned long long* clear0;
  unsigned long long* clear1;
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

// q-tile coordinates of stencil cell 0 (cells i-2..i+3 follow at stride 1 or
// one q row) of face f, and whether the face is an x face; false if the face
// lies outside the grid (n1: cells along the tile's 2nd axis).  Faces are
// numbered so that every 32-face chunk (a warp's share) is one row of one
// orientation: x faces 0..TX-1 of the TY rows, then the TY+1 rows of faces
// along the 2nd axis, then the TY right-most x faces.  A pass without x
// faces numbers only the 2nd-axis rows.
template <bool XF, class TL>
__device__ __forceinline__ bool face_geom(int f, int x0, int y0, int nx, int n1, bool& isx, int& hx, int& hy) {
  constexpr int TX = TL::TX, TY = TL::TY, NFY = TL::NFY;
  if (XF && (f < TX * TY || f >= TX * TY + NFY)) {
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
    return (x0 + i - 1 <= nx - 1) && (y0 + j < n1);
  }
  int ff = XF ? f - TX * TY : f;
  int j = ff / TX, i = ff - j * TX;
  isx = false;
  hx = i + NG;
  hy = j;  // cell k at row hy + k
  return (x0 + i < nx) && (y0 + j - 1 <= n1 - 1);
}

// Per-face averages of the characteristic projection: rho c and -1/c^2 at
// the face (arithmetic means of cells i and i+1), shared by all variables.
struct FaceAvg {
  float rc;    // rho_bar c_bar
  float mic2;  // -1 / c_bar^2
};

// Orientation of a face, resolved at run time so that the faces of both
// directions of a pass share one copy of the reconstruction code: offsets of
// the six stencil cells in the q tile and the q fields of the normal and
// tangential velocities.
template <int NTG>
struct FaceGeo {
  int off[6];
  int un;
  int ut[NTG];
};

// Characteristic variable R of the six stencil cells as mirrored pairs
// p[k] = (w_k, w_{5-k}), k = 0..4: the .x lanes are the left stencil
// w_0..w_4, the .y lanes the right stencil w_5..w_1.  Variables: 0 w1,
// 1 w2 (entropy), 2 .. 1+NTG tangential velocities, NQ-3 Gamma, NQ-2 Pi,
// NQ-1 w6.
template <class T, int R>
__device__ __forceinline__ void project_pairs(const float* qb, const FaceGeo<T::NTG>& fg, const FaceAvg& fa,
                                              float2 (&p)[5]) {
  constexpr int FS = T::FS;
  auto cell = [&](const float* b, int k) { return make_float2(b[fg.off[k]], b[fg.off[5 - k]]); };
  if constexpr (R == 0 || R == T::NQ - 1) {
    float2 rc = f2(R == 0 ? -fa.rc : fa.rc);
#pragma unroll
    for (int k = 0; k < 5; ++k) p[k] = mul2(f2(0.5f), fma2(rc, cell(qb + fg.un * FS, k), cell(qb + T::IP * FS, k)));
  } else if constexpr (R == 1) {
#pragma unroll
    for (int k = 0; k < 5; ++k) p[k] = fma2(f2(fa.mic2), cell(qb + T::IP * FS, k), cell(qb, k));
  } else if constexpr (R < 2 + T::NTG) {  // tangential velocities
#pragma unroll
    for (int k = 0; k < 5; ++k) p[k] = cell(qb + fg.ut[R - 2] * FS, k);
  } else {  // Gamma, Pi
#pragma unroll
    for (int k = 0; k < 5; ++k) p[k] = cell(qb + (R + 1) * FS, k);
  }
}

// 5th-order reconstruction of variable R on both sides of a face.  A
// stencil flat to 1e-6 of its magnitude (a few FP32 ulps: rounding noise)
// takes the linear weights, from which WENO-IS differs there by less than
// the stencil's range; elsewhere WENO-IS.  linear: the learned gate sent the
// face to the linear weights (one branch serves both reasons).
template <class T, int R>
__device__ __forceinline__ void weno_item(const float* qb, const FaceGeo<T::NTG>& fg, const FaceAvg& fa,
                                          const WenoParams& P, float& l5, float& r5, bool linear = false) {
  float2 p[5];
  project_pairs<T, R>(qb, fg, fa, p);
  float mn = fminf(fmin3(p[0].x, p[1].x, p[2].x), fmin3(p[2].y, p[1].y, p[0].y));
  float mx = fmaxf(fmax3(p[0].x, p[1].x, p[2].x), fmax3(p[2].y, p[1].y, p[0].y));
  float2 v;
  if (linear || mx - mn <= 1e-6f * fmaxf(fabsf(mx), fabsf(mn)))
    v = linear5_pair(p[0], p[1], p[2], p[3], p[4]);
  else
    v = weno5_pair(p[0], p[1], p[2], p[3], p[4], P);
  l5 = v.x;
  r5 = v.y;
}

// Census of variable R at a face: the flat-stencil test of weno_item on the
// same projected values.  cnt: [0] face-variables, [1] flat ones (linear
// weights), [2] warp passes, [3] warp passes in which some active lane has a
// non-flat stencil, so that the warp runs the WENO-IS branch.
template <class T, int R>
__device__ __forceinline__ void census_item(const float* qb, const FaceGeo<T::NTG>& fg, const FaceAvg& fa,
                                            unsigned (&cnt)[4]) {
  float2 p[5];
  project_pairs<T, R>(qb, fg, fa, p);
  float mn = fminf(fmin3(p[0].x, p[1].x, p[2].x), fmin3(p[2].y, p[1].y, p[0].y));
  float mx = fmaxf(fmax3(p[0].x, p[1].x, p[2].x), fmax3(p[2].y, p[1].y, p[0].y));
  const bool flat = mx - mn <= 1e-6f * fmaxf(fabsf(mx), fabsf(mn));
  const unsigned act = __activemask();
  const unsigned rough = __ballot_sync(act, !flat);
  cnt[0] += 1u;
  cnt[1] += flat ? 1u : 0u;
  if ((threadIdx.x & 31) == __ffs(act) - 1) {
    cnt[2] += 1u;
    cnt[3] += rough ? 1u : 0u;
  }
}

// A gated variable on a drift-check tile: the linear-weight values (which
// the face uses) and WENO-IS, whose difference is added to acc[0] and the
// WENO-IS magnitude to acc[NT] (the calling thread's own shared-memory
// slots).  Out of line, so that the common path keeps its registers.
template <class T, int R>
__device__ __noinline__ void drift_item(const float* qb, const FaceGeo<T::NTG> fg, const FaceAvg fa,
                                        const WenoParams P, float* acc, float& l5, float& r5) {
  float2 p[5];
  project_pairs<T, R>(qb, fg, fa, p);
  float2 lin = linear5_pair(p[0], p[1], p[2], p[3], p[4]);
  float fl, fr;
  weno_item<T, R>(qb, fg, fa, P, fl, fr);
  acc[0] += fabsf(lin.x - fl) + fabsf(lin.y - fr);
  acc[T::NT] += fabsf(fl) + fabsf(fr);
  l5 = lin.x;
  r5 = lin.y;
}

// Characteristic variable R of the six stencil cells, one value per cell
// (the MOOD retry's projection, with its own face averages)
template <class T, int R>
__device__ __forceinline__ void project6(const float* qb, const FaceGeo<T::NTG>& fg, float (&w)[6]) {
  constexpr int FS = T::FS;
  if constexpr (R == 0 || R == T::NQ - 1) {
    float rho_bar = 0.5f * (qb[fg.off[2]] + qb[fg.off[3]]);
    float c_bar = 0.5f * (qb[T::IC * FS + fg.off[2]] + qb[T::IC * FS + fg.off[3]]);
    float rc = R == 0 ? -(rho_bar * c_bar) : rho_bar * c_bar;
#pragma unroll
    for (int k = 0; k < 6; ++k) w[k] = 0.5f * fmaf(rc, qb[fg.un * FS + fg.off[k]], qb[T::IP * FS + fg.off[k]]);
  } else if constexpr (R == 1) {
    float c_bar = 0.5f * (qb[T::IC * FS + fg.off[2]] + qb[T::IC * FS + fg.off[3]]);
    float mic2 = -frcp(c_bar * c_bar);
#pragma unroll
    for (int k = 0; k < 6; ++k) w[k] = fmaf(mic2, qb[T::IP * FS + fg.off[k]], qb[fg.off[k]]);
  } else if constexpr (R < 2 + T::NTG) {
#pragma unroll
    for (int k = 0; k < 6; ++k) w[k] = qb[fg.ut[R - 2] * FS + fg.off[k]];
  } else {
#pragma unroll
    for (int k = 0; k < 6; ++k) w[k] = qb[(R + 1) * FS + fg.off[k]];
  }
}

// 3rd-order reconstruction (d3 = d4 = 0) of all variables of one side:
// the MOOD retry, taken only by faces whose 5th-order state is inadmissible
template <class T>
__device__ __noinline__ void weno_side3(const float* qb, const FaceGeo<T::NTG> fg, int side, const WenoParams P,
                                        float* wt) {
#define WS_SIDE3(R)                                                                                        \
  if constexpr (R < T::NQ) {                                                                              \
    float w[6];                                                                                           \
    project6<T, R>(qb, fg, w);                                                                            \
    wt[R] = side == 0 ? weno_is(w[0], w[1], w[2], w[3], w[4], P, 3) : weno_is(w[5], w[4], w[3], w[2], w[1], P, 3); \
  }
  WS_SIDE3(0)
  WS_SIDE3(1)
  WS_SIDE3(2)
  WS_SIDE3(3)
  WS_SIDE3(4)
  WS_SIDE3(5)
  WS_SIDE3(6)
#undef WS_SIDE3
}

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

// gate inputs of one face (2D): w1, w2, w6, w_Gamma of the six stencil cells,
// each normalised over the stencil (zero for a stencil flat to 1e-6)
template <int D, class TL>
__device__ __forceinline__ void gate_features(const float* qb, __nv_bfloat16* out) {
  constexpr int ST = D == 0 ? 1 : TL::HXP;
  constexpr int FS = TL::HY * TL::HXP;
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

// Asynchronous global -> shared copies (hold no register while in flight)
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// TMA: a tiled 3D box (x, row, field) of an FP32 buffer into shared memory,
// completing on an mbarrier that expects its bytes
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  unsigned b = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(b), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  unsigned b = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(b), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int f,
                                            unsigned long long* bar) {
  unsigned d = (unsigned)__cvta_generic_to_shared(dst), b = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cta.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(d),
      "l"(map), "r"(x), "r"(y), "r"(f), "r"(b)
      : "memory");
}
// The same for a 4D box (x, row, plane, field) of a 3D grid's FP32 buffer.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int f,
                                            unsigned long long* bar) {
  unsigned d = (unsigned)__cvta_generic_to_shared(dst), b = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cta.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];\n" ::"r"(d),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(f), "r"(b)
      : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Waits for phase 0 of the barrier, at most `limit_ns` nanoseconds; false if
// it gave up.  Each try suspends the thread until the phase completes or up
// to a millisecond passes, so waiting warps issue nothing meanwhile (a plain
// poll would take issue slots from the co-resident CTA).
__device__ __forceinline__ bool mbar_wait0(unsigned long long* bar, unsigned long long limit_ns) {
  unsigned b = (unsigned)__cvta_generic_to_shared(bar);
  const unsigned long long t0 = global_ns();
  for (;;) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0, %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(b), "r"(1000000u)
        : "memory");
    if (ok) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// One CTA's work: the tile in tile row `trow` of tiles TL starting at grid row
// `ybase`.  MAP 1 takes the second pair of TMA descriptors (boxes of TL).
template <int GATE, int NQ_, int MODE, class TL, int MAP>
__device__ __forceinline__ void stage_body(const StageArgs& a, const int trow, const int ybase) {
  using T = Tr<NQ_, MODE, TL>;
  using SM = Smem<GATE, NQ_, MODE, TL>;
  constexpr int TX = TL::TX, TY = TL::TY, NT = TL::NT, NF = TL::NF, NMT = TL::NMT;
  constexpr bool LEARNED = GATE == 1 || GATE == 2;  // faces may take the linear weights by the gate's decision
  constexpr bool CENSUS = GATE == 3;
  constexpr int NQ = NQ_, ND = T::ND, FS = T::FS;
  constexpr bool CACHE = SM::CACHE;
  // axes: x, the tile's 2nd axis (y; z in pass 2), the plane axis (z; y in pass 2; none in 2D)
  constexpr int AX1 = MODE == 2 ? 2 : 1, AXP = MODE == 2 ? 1 : 2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  SM& S = *reinterpret_cast<SM*>(smem_raw);
  // a TMA load stages K of tile and halo in fx and fy, and the image in q
  static_assert(MODE == 2 || (sizeof(S.fx) + sizeof(S.fy) >= sizeof(float) * NQ_ * T::HY * T::QP &&
                              offsetof(SM, fy) == offsetof(SM, fx) + sizeof(S.fx)),
                "the K box does not fit the flux arrays");
  static_assert(T::QP * sizeof(float) % 16 == 0, "TMA box rows are multiples of 16 bytes");
  static_assert(offsetof(SM, q) % 128 == 0 && offsetof(SM, fx) % 128 == 0 && offsetof(SM, kbox) % 128 == 0,
                "TMA destinations start on 128-byte boundaries");
  static_assert(MODE != 2 || offsetof(decltype(S.own), u) >= sizeof(S.kbox), "the K box reaches the FP64 copies");
  SmemGate<TL>& SG = *reinterpret_cast<SmemGate<TL>*>(smem_raw + sizeof(SM));
  // Launched with programmatic stream serialization (the plain 2D stage), a
  // CTA may become resident while the previous stage is still finishing: it
  // waits here until that grid has completed and its writes are visible, and
  // lets the next stage's CTAs be scheduled as this grid's CTAs retire.
  // Without the launch attribute both instructions return at once.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (a.run_if && *a.run_if == 0) return;  // a conditional redo that is not needed
  if (a.clear0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) {
    *a.clear0 = 0ULL;
    if (a.clear1) *a.clear1 = 0ULL;
  }
  const GridDev& g = a.g;
  const int nx = g.n[0], n1 = g.n[AX1];
  const int tile = trow * gridDim.x + blockIdx.x;
  const int x0 = blockIdx.x * TX, y0 = ybase + trow * TY, plane = blockIdx.z;
  const int64_t N = g.N, S1 = g.st[AX1];
  const int64_t pbase = (int64_t)(g.G[AXP] + plane) * g.st[AXP] + g.G[0];  // cell (x, a) at pbase + (G1 + a) S1 + x
  const int tid = threadIdx.x;
  // index in the FP32 buffers (image, K, the 3D partial divergence) of cell
  // (x, a) of the tile's plane, computed where it is used
  // (3D: the plane's base and the row stride are formed once, like pbase and S1)
  const int64_t pbase32 = MODE == 0 ? 0 : (int64_t)(g.G[AXP] + plane) * g.st32[AXP] + g.G[0];
  const int64_t S1f = MODE == 0 ? 0 : g.st32[AX1];
  auto idx32 = [&](int a_, int x_) -> int64_t {
    if constexpr (MODE == 0)
      return (int64_t)(g.G[1] + a_) * g.st32[1] + g.G[0] + x_;
    else
      return pbase32 + (int64_t)(g.G[AX1] + a_) * S1f + x_;
  };
  const int64_t N32 = g.N32;
  // A tile of the 2D stage or of the first 3D pass whose halo lies inside the
  // grid, in a stage that reads the FP32 image (and K), takes both as TMA
  // boxes: no boundary mapping, one instruction per array.  They are issued
  // first thing and land while the CTA sets up.
  // (The second 3D pass has a z halo only; its boxes also cover the x halo
  // columns, which it does not read.)
  const bool tma = a.tma && (a.stage == 1 || a.stage == 2 || (a.stage == 0 && a.img_in)) && y0 >= NG &&
                   y0 + TY + NG <= n1 && (MODE == 2 || (x0 >= NG && x0 + TX + NG <= nx));
  if (tma && tid == 0) {
    mbar_init(&S.mbar, 1);
    // boxes of the halo: padded column x0 - NG + NG, padded row y0, all fields
    constexpr unsigned box = (unsigned)(NQ_ * T::HY * T::QP * sizeof(float));
    mbar_expect_tx(&S.mbar, a.stage == 0 ? box : 2 * box);
    if constexpr (MODE == 0) {
      tma_load_3d(&S.q[0][0][0], MAP ? &a.tm_v2 : &a.tm_v, x0, y0, 0, &S.mbar);
      if (a.stage != 0) tma_load_3d(&S.fx[0][0][0], MAP ? &a.tm_k2 : &a.tm_k, x0, y0, 0, &S.mbar);
    } else if constexpr (MODE == 1) {  // the tile's z plane
      tma_load_4d(&S.q[0][0][0], &a.tm_v, x0, y0, g.G[2] + plane, 0, &S.mbar);
      if (a.stage != 0) tma_load_4d(&S.fx[0][0][0], &a.tm_k, x0, y0, g.G[2] + plane, 0, &S.mbar);
    } else {  // the tile's y plane: boxes of x, one y, z rows and all fields
      tma_load_4d(&S.q[0][0][0], &a.tm_v, x0, g.G[1] + plane, y0, 0, &S.mbar);
      if (a.stage != 0) tma_load_4d(&S.kbox[0][0][0], &a.tm_k, x0, g.G[1] + plane, y0, 0, &S.mbar);
    }
  }
  if (a.stage == 1 || a.stage == 2 || tma) {
    if (tid == 0) {
      if (a.stage == 1 || a.stage == 2) {  // one FP64 division per CTA
        double d = a.dt_fixed > 0.0 ? a.dt_fixed : (double)a.cfl / __longlong_as_double((long long)*a.lmax);
        if (a.stage == 1 && MODE != 2 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) *a.dt_out = d;
        S.dt = f64_to_f32(d);
      }
      // The boxes: this thread, which set the mbarrier up, waits for them; the
      // other warps wait at the barrier below, where they issue nothing.  A
      // copy that never lands is reported as an impossible count of
      // inadmissible cells (the results of the launch are then void).
      if (tma && !mbar_wait0(&S.mbar, 1000000000ULL)) atomicAdd(a.nbad, 1ULL << 40);
    }
    __syncthreads();
  }
  // The own cells' FP64 state (stage 2) and, in the second 3D pass, the x + y
  // part of their divergence are needed only in phase C: they are copied into
  // shared memory while phases A and B run (a second-pass tile that took its
  // K as a box, which shares their memory, copies them once phase A has read
  // it).
  auto own_copies = [&](bool u, bool l) {
    for (int c = tid; c < TX * TY; c += NT) {
      int j = c / TX, i = c - j * TX;
      if (x0 + i >= nx || y0 + j >= n1) continue;
      if (u) {
        const int64_t gi = pbase + (int64_t)(g.G[AX1] + y0 + j) * S1 + x0 + i;
#pragma unroll
        for (int m = 0; m < NQ; ++m) cp_async8(&S.own.u[m][j][i], &a.U[m * N + gi]);
      }
      if (MODE == 2 && l) {
        const int64_t gf = idx32(y0 + j, x0 + i);
#pragma unroll
        for (int m = 0; m < NQ; ++m) cp_async4(&S.own.l[m][j][i], &a.Lp[m * N32 + gf]);
      }
    }
    cp_async_commit();
  };
  if (CACHE && (a.stage == 2 || MODE == 2)) own_copies(a.stage == 2, !(MODE == 2 && tma));
  const float dt = (a.stage == 1 || a.stage == 2) ? S.dt : 0.0f;
  const float coef = a.stage == 0 ? 0.0f : (a.stage == 1 ? dt : 0.25f * dt);
  float lam_max = 0.0f;

  if (LEARNED) {  // this thread's drift sums (only it touches them until after phase B)
    SG.dpart[0][tid] = 0.0f;
    SG.dpart[1][tid] = 0.0f;
  }
  if constexpr (GATE == 2) {  // this step's decisions, stored by its stage 0
    const uint8_t* fl = a.gflags + (int64_t)tile * NF;
    for (int f = tid; f < NF; f += NT) SG.smooth[f] = fl[f];
  }

  // ---- phase A: stage-state primitives of tile + halo ----
  // A TMA tile (above) reads image and K from shared memory once its boxes
  // land and takes its cells one at a time.  Otherwise a thread owns up to HPT
  // q-tile cells and issues all their global loads before any of them is
  // used, so that a CTA has its whole halo in flight.
  {
    // stages 1, 2: the stage state from the image and the increments (E - Pi
    // with Pi's increment); the own cells' values are kept for phase C
    auto stage_state = [&](float (&ld)[NQ], const float (&rk)[NQ], const float (&rv)[NQ], int hy, int hx,
                           bool ownc) {
#pragma unroll
      for (int m = 0; m < NQ; ++m) {
        if (m == NQ - 3)
          ld[m] = fmaf(coef, rk[m] - rk[NQ - 1], rv[m]);
        else
          ld[m] = fmaf(coef, rk[m], rv[m]);
      }
      if (CACHE && ownc) {  // phase C reads these instead of global memory
        const int j = hy - NG, i = hx - T::QX;
#pragma unroll
        for (int m = 0; m < NQ; ++m) {
          S.own.k[m][j][i] = rk[m];
          if (SM::OWNV && a.stage == 2) S.own.v[m][j][i] = rv[m];
        }
      }
    };
    // primitives and sound speed into the q tile; stage 0: the CFL rate
    auto primitives = [&](const float (&ld)[NQ], int hy, int hx, bool fx, bool fa, bool ownc) {
      float rho = ld[0], eint = ld[NQ - 3], Gam = ld[NQ - 2], Pi = ld[NQ - 1];
      float irho = frcp(rho);
      float vel[ND];
#pragma unroll
      for (int d = 0; d < ND; ++d) vel[d] = ld[1 + d] * irho;
      if (fx) vel[0] = -vel[0];
      if (fa) vel[AX1] = -vel[AX1];
      float ksq = ND == 2 ? fmaf(vel[0], vel[0], vel[1] * vel[1])
                          : fmaf(vel[0], vel[0], fmaf(vel[1], vel[1], vel[ND - 1] * vel[ND - 1]));
      float p = fmaf(-0.5f * rho, ksq, eint) * frcp(Gam);
      S.q[0][hy][hx] = rho;
#pragma unroll
      for (int d = 0; d < ND; ++d) S.q[1 + d][hy][hx] = vel[d];
      S.q[T::IP][hy][hx] = p;
      S.q[T::IG][hy][hx] = Gam;
      S.q[T::IPI][hy][hx] = Pi;
      float c = fsqrt(sound_speed2(rho, p, Gam, Pi));
      S.q[T::IC][hy][hx] = c;
      if (a.stage == 0 && MODE != 2 && ownc) {
        float lam = fmaf(fabsf(vel[0]) + c, a.idx, (fabsf(vel[1]) + c) * a.idy);
        if (ND == 3) lam = fmaf(fabsf(vel[ND - 1]) + c, a.idz, lam);
        if (!(lam <= lam_max)) lam_max = lam;  // NaN propagates
      }
    };
    if (tma && MODE == 2) {  // the boxes have landed (barrier above)
      // K lies in the own cells' arrays: every thread reads its cells' values
      // before any of those arrays is written
      const float* kst = &S.kbox[0][0][0];
      float rk[T::HPT][NQ], rv[T::HPT][NQ];
#pragma unroll
      for (int t = 0; t < T::HPT; ++t) {
        const int h = tid + t * NT;
        if (h >= T::NH) continue;
        const int hy = h / T::QW, hx = h - hy * T::QW + T::QL;
#pragma unroll
        for (int m = 0; m < NQ; ++m) {
          rv[t][m] = S.q[m][hy][hx];
          if (a.stage != 0) rk[t][m] = kst[(m * T::HY + hy) * T::QP + hx];
        }
      }
      __syncthreads();
      if (CACHE) own_copies(false, true);
#pragma unroll
      for (int t = 0; t < T::HPT; ++t) {
        const int h = tid + t * NT;
        if (h >= T::NH) continue;
        const int hy = h / T::QW, hx = h - hy * T::QW + T::QL;
        const bool ownc = hy >= NG && hy < NG + TY;
        float ld[NQ];
        if (a.stage == 0) {
#pragma unroll
          for (int m = 0; m < NQ; ++m) ld[m] = rv[t][m];
        } else {
          stage_state(ld, rk[t], rv[t], hy, hx, ownc);
        }
        primitives(ld, hy, hx, false, false, ownc);
      }
    } else if (tma) {  // the boxes have landed (barrier above)
      const float* kst = &S.fx[0][0][0];  // K of tile and halo, [field][row][column] like q
#pragma unroll
      for (int t = 0; t < T::HPT; ++t) {
        const int h = tid + t * NT;
        if (h >= T::NH) continue;
        const int hy = h / T::QW, hx = h - hy * T::QW + T::QL;
        const bool ownc = hx >= T::QX && hx < T::QX + TX && hy >= NG && hy < NG + TY;
        float ld[NQ];
        if (a.stage == 0) {
#pragma unroll
          for (int m = 0; m < NQ; ++m) ld[m] = S.q[m][hy][hx];
        } else {
          float rk[NQ], rv[NQ];
#pragma unroll
          for (int m = 0; m < NQ; ++m) {
            rv[m] = S.q[m][hy][hx];
            rk[m] = kst[(m * T::HY + hy) * T::QP + hx];
          }
          stage_state(ld, rk, rv, hy, hx, ownc);
        }
        primitives(ld, hy, hx, false, false, ownc);
      }
    } else {
      float ld[T::HPT][NQ];
      float rk[T::HPT][NQ], rv[T::HPT][NQ];  // stages 1, 2: increment and FP32 image as loaded
      int hh[T::HPT];
      bool flx[T::HPT], fla[T::HPT], own[T::HPT];
#pragma unroll
      for (int t = 0; t < T::HPT; ++t) {
        int h = tid + t * NT;
        int hy = h / T::QW, hx = h - hy * T::QW + T::QL;
        int gx = x0 + hx - T::QX, ga = y0 + hy - NG;
        bool outx = gx < 0 || gx >= nx, outa = ga < 0 || ga >= n1;
        // corners are never read, nor (without x faces) columns past the grid
        bool skip = h >= T::NH || (outx && outa) || (!T::XF && outx);
        hh[t] = skip ? -1 : h;
        if (skip) continue;
        bool fx = false, fa = false;
        int mx = map_bc(gx, nx, g.bc[0][0], g.bc[0][1], fx);
        int ma = map_bc(ga, n1, g.bc[AX1][0], g.bc[AX1][1], fa);
        flx[t] = fx;
        fla[t] = fa;
        own[t] = hx >= T::QX && hx < T::QX + TX && hy >= NG && hy < NG + TY && !outx && !outa;
        if (a.stage == 0 && a.img_in) {  // the image the previous step's stage 2 left
          const int64_t i32 = idx32(ma, mx);
#pragma unroll
          for (int m = 0; m < NQ; ++m) ld[t][m] = __ldg(&a.U32[m * N32 + i32]);
        } else if (a.stage == 0 || a.stage == 3) {
          const int64_t i = pbase + (int64_t)(g.G[AX1] + ma) * S1 + mx;  // FP64 state
          const double* U = a.U;
#pragma unroll
          for (int m = 0; m < NQ; ++m) {
            if (m == NQ - 3)
              ld[t][m] = f64_to_f32(U[m * N + i] - U[(NQ - 1) * N + i]);  // E - Pi in FP64
            else
              ld[t][m] = f64_to_f32(U[m * N + i]);
          }
          if (a.stage == 0 && MODE != 2 && own[t]) {
            if (LEARNED) {
#pragma unroll
              for (int m = 0; m < NQ; ++m) a.Ubackup[m * N + i] = U[m * N + i];
            }
            const int64_t i32 = idx32(ma, mx);
#pragma unroll
            for (int m = 0; m < NQ; ++m) a.U32[m * N32 + i32] = ld[t][m];
          }
        } else {
          const int64_t i32 = idx32(ma, mx);
#pragma unroll
          for (int m = 0; m < NQ; ++m) {
            rk[t][m] = __ldg(&a.Kin[m * N32 + i32]);
            rv[t][m] = __ldg(&a.U32[m * N32 + i32]);
          }
        }
      }
#pragma unroll
      for (int t = 0; t < T::HPT; ++t) {
        if (hh[t] < 0) continue;
        const int hy = hh[t] / T::QW, hx = hh[t] - hy * T::QW + T::QL;
        if (a.stage == 1 || a.stage == 2) stage_state(ld[t], rk[t], rv[t], hy, hx, own[t]);
        primitives(ld[t], hy, hx, flx[t], fla[t], own[t]);
      }
    }
  }
  if (a.stage == 0 && MODE != 2) {
    unsigned long long b = (unsigned long long)__double_as_longlong(f32_to_f64(lam_max));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long v = __shfl_xor_sync(0xffffffffu, b, o);
      b = v > b ? v : b;
    }
    if ((tid & 31) == 0) S.red[tid >> 5] = b;
  }
  __syncthreads();
  if (a.stage == 0 && MODE != 2 && tid == 0) {
    unsigned long long b = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) b = S.red[w] > b ? S.red[w] : b;
    if (b) atomicMax(a.lmax, b);
  }

  // ---- phases G1, G2 (learned gate, 2D): features, then the BF16 tensor-core MLP ----
  if constexpr (GATE == 1) {
    for (int i = tid; i < NFRAG * 32; i += NT) SG.frag[i / 32][i % 32] = a.mlp_frag[i];
    for (int i = tid; i < 65; i += NT) {
      float b = a.mlp_bias[i];
      if (i < 32) SG.b1[i] = b;
      else if (i < 64) SG.b2[i - 32] = b;
      else SG.b3 = b;
    }
    for (int f = tid; f < NF; f += NT) {
      bool isx;
      int hx, hy;
      SG.smooth[f] = 0;
      if (!face_geom<true, TL>(f, x0, y0, nx, n1, isx, hx, hy)) continue;
      const float* qb = &S.q[0][hy][hx];
      if (isx)
        gate_features<0, TL>(qb, S.feat[f]);
      else
        gate_features<1, TL>(qb, S.feat[f]);
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
    if (a.gflags) {  // kept for the step's later stages
      uint8_t* fl = a.gflags + (int64_t)tile * NF;
      for (int f = tid; f < NF; f += NT) fl[f] = SG.smooth[f];
    }
    if (a.stage == 3) {  // gate evaluation only: the decisions go to the mask arrays
      for (int f = tid; f < NF; f += NT) {
        bool isx;
        int hx, hy;
        if (!face_geom<true, TL>(f, x0, y0, nx, n1, isx, hx, hy)) continue;
        if (isx)
          a.mask_x[(int64_t)(y0 + hy - NG) * (nx + 1) + (x0 + hx)] = SG.smooth[f];
        else
          a.mask_a[(int64_t)(y0 + hy) * nx + (x0 + hx - NG)] = SG.smooth[f];
      }
      return;
    }
  }

  // ---- phase B: per face, WENO-IS per characteristic variable, then
  // back-projection, MOOD and HLLC.  The thread that reconstructs a face also
  // solves its Riemann problem, so no barrier separates the two and the
  // reconstructed characteristics stay in registers.
  const bool drift = LEARNED && ((tile & 63) ==
                                  (a.drift_dev ? *a.drift_dev : a.drift_tile));
  const float* q0 = &S.q[0][0][0];
  unsigned cnt[4] = {0u, 0u, 0u, 0u};  // census counts of this thread (GATE 3)
#pragma unroll 1
  for (int f = tid; f < T::NFP; f += NT) {
    bool isx;
    int hx, hy;
    if (!face_geom<T::XF, TL>(f, x0, y0, nx, n1, isx, hx, hy)) continue;
    const float* qb = q0 + hy * T::QP + hx;  // stencil cell 0 in the q tile
    const bool sm = LEARNED && SG.smooth[f];
    FaceGeo<T::NTG> fg;
    {
      const int st = isx ? 1 : T::QP;
#pragma unroll
      for (int k = 0; k < 6; ++k) fg.off[k] = k * st;
      fg.un = isx ? 1 : 1 + AX1;
      fg.ut[0] = isx ? 2 : 1;  // tangential velocities in increasing axis order
      if constexpr (T::NTG == 2) fg.ut[1] = isx ? 3 : (AX1 == 1 ? 3 : 2);
    }
    float rho_bar = 0.5f * (qb[fg.off[2]] + qb[fg.off[3]]);
    float c_bar = 0.5f * (qb[T::IC * FS + fg.off[2]] + qb[T::IC * FS + fg.off[3]]);
    float c2 = c_bar * c_bar, rc = rho_bar * c_bar;
    float inv = frcp(c2 * rc);
    float ic2 = rc * inv, irc = c2 * inv;  // 1/c^2, 1/(rho c)
    const FaceAvg fa{rc, -ic2};
    float wl[NQ], wr[NQ];  // reconstructed characteristics, left and right
#define WS_RECON(R)                                                                 \
    if constexpr (R < NQ) {                                                      \
      if constexpr (CENSUS) census_item<T, R>(qb, fg, fa, cnt);                  \
      bool lin = LEARNED && R != 2 && sm; /* shear: always WENO-IS */            \
      if (LEARNED && lin && drift)                                               \
        drift_item<T, R>(qb, fg, fa, a.P, &SG.dpart[0][tid], wl[R], wr[R]);      \
      else                                                                       \
        weno_item<T, R>(qb, fg, fa, a.P, wl[R], wr[R], lin);                     \
    }
    WS_RECON(0)
    WS_RECON(1)
    WS_RECON(2)
    WS_RECON(3)
    WS_RECON(4)
    WS_RECON(5)
    WS_RECON(6)
#undef WS_RECON

    float2 W[NQ], Q[NQ];  // (left, right) characteristics, then primitives
#pragma unroll
    for (int r = 0; r < NQ; ++r) W[r] = make_float2(wl[r], wr[r]);
    back_project_pair<NQ>(W, ic2, irc, Q);
    int code[2] = {0, 0};
    if (a.mood) {
      bool ok0, ok1;
      admissible_pair<NQ>(Q, ok0, ok1);
      if (!ok0 || !ok1) {  // MOOD cascade of the failing side(s): rare
#pragma unroll 1
        for (int side = 0; side < 2; ++side) {
          if (side == 0 ? ok0 : ok1) continue;
          if (LEARNED && sm) atomicAdd(&a.lstat[0], 1.0f);
          float wt[NQ];
          weno_side3<T>(qb, fg, side, a.P, wt);
          float q3[NQ];
          back_project<NQ>(wt, ic2, irc, q3);
          code[side] = 1;
          if (!admissible<NQ>(q3)) {  // 1st order: the cell's own primitive state
            const int oc = side == 0 ? fg.off[2] : fg.off[3];
            q3[0] = qb[oc];
            q3[1] = qb[fg.un * FS + oc];
#pragma unroll
            for (int t = 0; t < T::NTG; ++t) q3[2 + t] = qb[fg.ut[t] * FS + oc];
            q3[T::IP] = qb[T::IP * FS + oc];
            q3[T::IP + 1] = qb[T::IG * FS + oc];
            q3[T::IP + 2] = qb[T::IPI * FS + oc];
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
    bool stored = false;
    if constexpr (T::XF) {
      if (isx) {  // x faces: the sweep frame is the global field order
        int j = hy - NG, i = hx;
#pragma unroll
        for (int m = 0; m < NQ; ++m) S.fx[m][j][i] = Fh[m];
        S.fx[NQ][j][i] = us;
        if (a.mask_x) a.mask_x[((int64_t)plane * n1 + (y0 + j)) * (nx + 1) + (x0 + i)] = mb;
        stored = true;
      }
    }
    if (!stored) {
      int j = hy, i = hx - T::QX;
      S.fy[0][j][i] = Fh[0];
      S.fy[fg.un][j][i] = Fh[1];  // normal momentum
#pragma unroll
      for (int t = 0; t < T::NTG; ++t) S.fy[fg.ut[t]][j][i] = Fh[2 + t];
#pragma unroll
      for (int m = NQ - 3; m < NQ; ++m) S.fy[m][j][i] = Fh[m];
      S.fy[NQ][j][i] = us;
      if (a.mask_a) {
        int64_t mi = MODE == 2 ? ((int64_t)(y0 + j) * g.n[1] + plane) * nx + (x0 + i)
                               : ((int64_t)plane * (n1 + 1) + (y0 + j)) * nx + (x0 + i);
        a.mask_a[mi] = mb;
      }
    }
  }
  if constexpr (CENSUS) {  // every lane is back from the face loop
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      unsigned v = __reduce_add_sync(0xffffffffu, cnt[k]);
      if ((tid & 31) == 0 && v) atomicAdd(&a.census[k], (unsigned long long)v);
    }
  }
  if (LEARNED) {  // drift sums, faces examined, faces the gate sent to the linear weights
    float nsm = 0.0f, nval = 0.0f;
    for (int f = tid; f < T::NFP; f += NT) {
      bool isx;
      int hx, hy;
      if (!face_geom<T::XF, TL>(f, x0, y0, nx, n1, isx, hx, hy)) continue;
      nval += 1.0f;
      nsm += SG.smooth[f] ? 1.0f : 0.0f;
    }
    float dnum = SG.dpart[0][tid], dden = SG.dpart[1][tid];
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
  if (CACHE && (a.stage == 2 || MODE == 2)) cp_async_wait_all();  // own-cell copies, visible after the barrier
  __syncthreads();
  if (LEARNED && tid < 4) {
    float sum = 0.0f;
    for (int w = 0; w < NT / 32; ++w) sum += SG.red[tid][w];
    if (tid >= 2 || drift) atomicAdd(&a.lstat[1 + tid], sum);
  }

  // ---- phase C: flux divergence and RK stage ----
  constexpr int M0 = NQ % 2;  // with an odd field count, field 0 goes alone ahead of the pairs
  for (int c = tid; c < TX * TY; c += NT) {
    int j = c / TX, i = c - j * TX;
    if (x0 + i >= nx || y0 + j >= n1) continue;
    const int64_t gi = pbase + (int64_t)(g.G[AX1] + y0 + j) * S1 + x0 + i;  // FP64 state
    const int64_t gf = idx32(y0 + j, x0 + i);                              // FP32 buffers
    const int qj = j + NG, qi = i + T::QX;
    float inc[NQ];
    auto fy2 = [&](int m, int jj) { return make_float2(S.fy[m][jj][i], S.fy[m + 1][jj][i]); };
    if constexpr (MODE != 2) {  // x then y faces
      const float2 idx = f2(a.idx), idy = f2(a.idy);
      float div_u = (S.fx[NQ][j][i + 1] - S.fx[NQ][j][i]) * a.idx + (S.fy[NQ][j + 1][i] - S.fy[NQ][j][i]) * a.idy;
      if constexpr (M0 == 1) inc[0] = fmaf(S.fy[0][j][i] - S.fy[0][j + 1][i], a.idy, (S.fx[0][j][i] - S.fx[0][j][i + 1]) * a.idx);
#pragma unroll
      for (int m = M0; m < NQ; m += 2) {
        float2 L = mul2(sub2(make_float2(S.fx[m][j][i], S.fx[m + 1][j][i]),
                             make_float2(S.fx[m][j][i + 1], S.fx[m + 1][j][i + 1])), idx);
        L = fma2(sub2(fy2(m, j), fy2(m, j + 1)), idy, L);
        if (m == NQ - 2) L = fma2(make_float2(S.q[m][qj][qi], S.q[m + 1][qj][qi]), f2(div_u), L);
        inc[m] = L.x;
        inc[m + 1] = L.y;
      }
    } else {  // z faces, added to the x + y part
      const float2 idz = f2(a.idz);
      float div_u = (S.fy[NQ][j + 1][i] - S.fy[NQ][j][i]) * a.idz;
      if constexpr (M0 == 1) inc[0] = fmaf(S.fy[0][j][i] - S.fy[0][j + 1][i], a.idz, S.own.l[0][j][i]);
#pragma unroll
      for (int m = M0; m < NQ; m += 2) {
        float2 L = fma2(sub2(fy2(m, j), fy2(m, j + 1)), idz, make_float2(S.own.l[m][j][i], S.own.l[m + 1][j][i]));
        if (m == NQ - 2) L = fma2(make_float2(S.q[m][qj][qi], S.q[m + 1][qj][qi]), f2(div_u), L);
        inc[m] = L.x;
        inc[m + 1] = L.y;
      }
    }
    if constexpr (MODE == 1) {
#pragma unroll
      for (int m = 0; m < NQ; ++m) a.Lp[m * N32 + gf] = inc[m];
    } else {
      auto kin = [&](int m) { return CACHE ? S.own.k[m][j][i] : a.Kin[m * N32 + gf]; };
      if (a.stage == 0) {
#pragma unroll
        for (int m = 0; m < NQ; ++m) a.Kout[m * N32 + gf] = inc[m];
      } else if (a.stage == 1) {
#pragma unroll
        for (int m = 0; m < NQ; ++m) a.Kout[m * N32 + gf] = kin(m) + inc[m];
      } else {
        // this cell's U^n is read only here, by this thread, so U is updated in place
        float d[NQ];
        double uE = 0.0, uPi = 0.0;
#pragma unroll
        for (int m = 0; m < NQ; ++m) {
          d[m] = dt * fmaf(1.0f / 6.0f, kin(m), (2.0f / 3.0f) * inc[m]);
          double u = CACHE ? S.own.u[m][j][i] : a.U[m * N + gi];
          const double un = u + f32_to_f64(d[m]);  // FP64 accumulation
          a.U[m * N + gi] = un;
          if (m == NQ - 3) uE = un;
          if (m == NQ - 1) uPi = un;
          // the FP32 image of the new state for the next step's stage 0: the
          // values its phase A would form from U (E - Pi in FP64), bit for bit
          if (a.img_out && m != NQ - 3) a.img_out[m * N32 + gf] = f64_to_f32(un);
        }
        if (a.img_out) a.img_out[(NQ - 3) * N32 + gf] = f64_to_f32(uE - uPi);
        // admissibility of the new state (rho > 0, Gamma > 0, (Gamma+1) p + Pi > 0)
        // from its FP32 image: a diagnostic, not part of the update
        auto v = [&](int m) { return SM::OWNV ? S.own.v[m][j][i] : a.U32[m * N32 + gf]; };
        float rho = v(0) + d[0];
        float msq = 0.0f;
#pragma unroll
        for (int e = 0; e < ND; ++e) {
          float me = v(1 + e) + d[1 + e];
          msq = fmaf(me, me, msq);
        }
        float eint = v(NQ - 3) + (d[NQ - 3] - d[NQ - 1]), Gam = v(NQ - 2) + d[NQ - 2], Pi = v(NQ - 1) + d[NQ - 1];
        float pe = fmaf(-0.5f, msq * frcp(rho), eint);  // Gamma p
        bool ok = rho > 0.0f && Gam > 0.0f && fmaf(Gam + 1.0f, pe * frcp(Gam), Pi) > 0.0f;
        if (!ok) atomicAdd(a.nbad, 1ULL);
      }
    }
  }
}

template <int GATE, int NQ_, int MODE, class TL>
__global__ void __launch_bounds__(TL::NT, 1024 / TL::NT) k_stage(const __grid_constant__ StageArgs a) {  // 64 registers
  stage_body<GATE, NQ_, MODE, TL, 0>(a, blockIdx.y + a.row0, 0);
}

// A 2D stage whose first a.rows_full tile rows are tiles TL and whose closing
// rows are the lower tiles TH of the same CTA size: a CTA of TH costs about
// 0.6 of one of TL, so the launch's last wave of CTAs ends more evenly across
// the SMs (the CTAs are scheduled in launch order, the TH rows last).
template <int NQ_, class TL, class TH>
__global__ void __launch_bounds__(TL::NT, 1024 / TL::NT) k_stage_tail(const __grid_constant__ StageArgs a) {
  static_assert(TL::NT == TH::NT && TL::TX == TH::TX, "one CTA shape");
  if ((int)blockIdx.y < a.rows_full)
    stage_body<0, NQ_, 0, TL, 0>(a, blockIdx.y, 0);
  else
    stage_body<0, NQ_, 0, TH, 1>(a, blockIdx.y - a.rows_full, a.rows_full * TL::TY);
}

}  // namespace

// After a gated step: decide on the device whether to redo it without the gate
// (no host round trip), keep the gate statistics, advance the drift-check tile
// and, inside a step graph, set the condition of the graph's redo branch.
static __global__ void k_gate_decide(const float* __restrict__ lstat, unsigned long long* nbad, unsigned long long* lmax,
                              int flags, int* redo, double* stats, int* drift_dev, cudaGraphConditionalHandle cond) {
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
  if (drift_dev) *drift_dev = (*drift_dev + 1) & 63;
  if (cond) cudaGraphSetConditional(cond, r ? 1u : 0u);
}

static __global__ void k_restore(const int* __restrict__ redo, const double* __restrict__ src, double* __restrict__ dst,
                          int64_t n) {
  if (*redo == 0) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

void launch_gate_decide(const float* lstat, unsigned long long* nbad, unsigned long long* lmax, int flags, int* redo,
                        double* stats, int* drift_dev, cudaGraphConditionalHandle cond, cudaStream_t s) {
  k_gate_decide<<<1, 1, 0, s>>>(lstat, nbad, lmax, flags, redo, stats, drift_dev, cond);
}

void launch_restore(const int* redo, const double* src, double* dst, int64_t n, cudaStream_t s) {
  k_restore<<<152 * 4, 256, 0, s>>>(redo, src, dst, n);
}

// dynamic shared memory of each instantiation
template <int GATE, int NQ, int MODE, class TL>
constexpr int smem_of() {
  return (int)(sizeof(Smem<GATE, NQ, MODE, TL>) + ((GATE == 1 || GATE == 2) ? sizeof(SmemGate<TL>) : 0));
}

// the tail-filled 2D launch: room for either tile shape
constexpr int tail_smem() {
  return smem_of<0, 6, 0, TileA>() > smem_of<0, 6, 0, TileH>() ? smem_of<0, 6, 0, TileA>() : smem_of<0, 6, 0, TileH>();
}

template <int GATE, int NQ, int MODE, class TL>
static cudaError_t allow_smem() {
  return cudaFuncSetAttribute(k_stage<GATE, NQ, MODE, TL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_of<GATE, NQ, MODE, TL>());
}

int fused2d_smem_bytes() { return smem_of<1, 6, 0, TileA>(); }

cudaError_t fused2d_prepare() {
  cudaError_t e;
  if ((e = allow_smem<0, 6, 0, TileA>()) || (e = allow_smem<1, 6, 0, TileA>()) || (e = allow_smem<2, 6, 0, TileA>()) ||
      (e = allow_smem<3, 6, 0, TileA>()) || (e = allow_smem<0, 6, 0, TileB>()) || (e = allow_smem<3, 6, 0, TileB>()) ||
      (e = allow_smem<0, 6, 0, TileC>()) || (e = allow_smem<3, 6, 0, TileC>()))
    return e;
  return cudaFuncSetAttribute(k_stage_tail<6, TileA, TileH>, cudaFuncAttributeMaxDynamicSharedMemorySize, tail_smem());
}

// Tile rows of a tail-filled 2D launch (tile 3): the number R of TileA rows,
// the rest of the grid's rows in TileH rows, chosen by a list schedule of the
// launch's CTAs, in launch order, on `slots` CTA slots.  A TileA CTA counts 1,
// a TileH CTA 0.6 (per-CTA times measured on the shock-bubble: the load
// latency is the same, the face work halves), a CTA of a partial row by the
// fraction of its rows it holds.  R = all rows (no tail) when no split is
// expected to end sooner.
int fused2d_tail_rows(const GridDev& g, int slots) {
  const int n1 = g.n[1], ncol = (g.n[0] + TileA::TX - 1) / TileA::TX;
  const int rows = (n1 + TileA::TY - 1) / TileA::TY;
  if (slots < 1) return rows;
  std::vector<double> fin((size_t)slots);
  auto makespan = [&](int R) {
    std::fill(fin.begin(), fin.end(), 0.0);
    std::priority_queue<double, std::vector<double>, std::greater<double>> q(fin.begin(), fin.end());
    auto put = [&](double cost, int n) {
      for (int k = 0; k < n; ++k) {
        double t = q.top();
        q.pop();
        q.push(t + cost);
      }
    };
    auto cost = [](double full, int held, int ty) { return full * (0.4 + 0.6 * held / ty); };
    const int rem = n1 - R * TileA::TY;
    if (rem <= 0) {  // TileA rows only, the last one possibly partial
      put(1.0, ncol * (rows - 1));
      put(cost(1.0, n1 - (rows - 1) * TileA::TY, TileA::TY), ncol);
    } else {
      const int H = (rem + TileH::TY - 1) / TileH::TY;
      put(1.0, ncol * R);
      put(0.6, ncol * (H - 1));
      put(cost(0.6, rem - (H - 1) * TileH::TY, TileH::TY), ncol);
    }
    double m = 0.0;
    while (!q.empty()) {
      m = std::max(m, q.top());
      q.pop();
    }
    return m;
  };
  int best = rows;
  double bm = makespan(rows);
  for (int R = rows - 1; R >= 0 && R >= rows - 64; --R) {
    const double m = makespan(R);
    if (m < bm * 0.999) {
      bm = m;
      best = R;
    }
  }
  return best;
}

int64_t fused2d_gate_flag_bytes(const GridDev& g) {
  return (int64_t)((g.n[0] + TileA::TX - 1) / TileA::TX) * ((g.n[1] + TileA::TY - 1) / TileA::TY) * TileA::NF;
}

int fused3d_smem_bytes() {
  int a = smem_of<0, 7, 1, TileA>(), b = smem_of<0, 7, 2, TileA>();
  return a > b ? a : b;
}

cudaError_t fused3d_prepare() {
  cudaError_t e;
  if ((e = allow_smem<0, 7, 1, TileA>()) || (e = allow_smem<0, 7, 2, TileA>()) || (e = allow_smem<3, 7, 1, TileA>()) ||
      (e = allow_smem<3, 7, 2, TileA>()) || (e = allow_smem<0, 7, 1, TileC>()) || (e = allow_smem<0, 7, 2, TileC>()) ||
      (e = allow_smem<3, 7, 1, TileC>()) || (e = allow_smem<3, 7, 2, TileC>()))
    return e;
  return cudaSuccess;
}

// Launch with programmatic stream serialization (pdl): the stage's CTAs may
// be scheduled before the previous kernel on the stream has finished and wait
// in griddepcontrol.wait, which hides the launch latency between the stages.
static void launch_kernel(void (*k)(StageArgs), int nt, int smem, dim3 grid, bool pdl, cudaStream_t s,
                          const StageArgs& a) {
  if (!pdl) {
    k<<<grid, nt, smem, s>>>(a);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(nt);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, a);
}

template <int GATE, int NQ, int MODE, class TL>
static void launch_k(dim3 grid, bool pdl, cudaStream_t s, const StageArgs& a) {
  launch_kernel(k_stage<GATE, NQ, MODE, TL>, TL::NT, smem_of<GATE, NQ, MODE, TL>(), grid, pdl, s, a);
}


template <class TL>
static dim3 grid2d(const GridDev& g, int nrows = -1) {
  return dim3((g.n[0] + TL::TX - 1) / TL::TX, nrows >= 0 ? nrows : (g.n[1] + TL::TY - 1) / TL::TY);
}

static StageArgs stage_args(const GridDev& g, int stage, double* U, float* U32, const float* Kin, float* Kout,
                            double dt_fixed, double cfl, unsigned long long* lmax, double* dt_out, float eps_rel,
                            int mood, int weights, unsigned long long* nbad) {
  StageArgs a;
  a.g = g;
  a.stage = stage;
  a.idx = (float)(1.0 / g.dx[0]);
  a.idy = (float)(1.0 / g.dx[1]);
  a.idz = (float)(1.0 / g.dx[2]);
  a.cfl = (float)cfl;
  a.dt_fixed = dt_fixed;
  a.lmax = lmax;
  a.dt_out = dt_out;
  a.U = U;
  a.U32 = U32;
  a.Kin = Kin;
  a.Kout = Kout;
  a.Lp = nullptr;
  a.mask_x = nullptr;
  a.mask_a = nullptr;
  a.P = weno_params(eps_rel, weights);
  a.mood = mood;
  a.nbad = nbad;
  a.tma = 0;
  a.clear0 = a.clear1 = nullptr;
  a.mlp_frag = nullptr;
  a.mlp_bias = nullptr;
  a.thr = 0.0f;
  a.drift_tile = -1;
  a.drift_dev = nullptr;
  a.Ubackup = nullptr;
  a.lstat = nullptr;
  a.run_if = nullptr;
  a.gflags = nullptr;
  a.row0 = 0;
  a.census = nullptr;
  a.img_in = 0;
  a.img_out = nullptr;
  a.rows_full = 0;
  return a;
}

// The stage configurations ws_autotune chooses among: tile (0 TileA, 1 TileB,
// 2 TileC, 3 TileA rows closed by TileH rows) and whether consecutive stages are launched with programmatic
// dependent launch.  3D launches take TileA or TileC (TileB's shared memory
// exceeds a CTA's limit with 7 fields).
int fused_num_tiles(int ndim) { return ndim == 3 ? 2 : 4; }
int fused_tile_index(int ndim, int k) { return ndim == 3 ? (k == 0 ? 0 : 2) : k; }

void launch_stage2d(const GridDev& g, int stage, double* U, float* U32, const float* Kin, float* Kout,
                    double dt_fixed, double cfl, unsigned long long* lmax, double* dt_out, uint8_t* mask_x,
                    uint8_t* mask_y, float eps_rel, int mood, int weights, unsigned long long* nbad,
                    const GateArgs* gate, const int* run_if, unsigned long long* census, int tile, bool pdl,
                    bool img_in, float* img_out, const CUtensorMap* tmk, const CUtensorMap* tmv,
                    unsigned long long* clear0, unsigned long long* clear1, int rows_full, const CUtensorMap* tmk2,
                    const CUtensorMap* tmv2, cudaStream_t s) {
  StageArgs a = stage_args(g, stage, U, U32, Kin, Kout, dt_fixed, cfl, lmax, dt_out, eps_rel, mood, weights, nbad);
  a.clear0 = clear0;
  a.clear1 = clear1;
  if (tmk && tmv && !gate) {
    a.tma = 1;
    a.tm_k = *tmk;
    a.tm_v = *tmv;
  }
  a.img_in = img_in ? 1 : 0;
  a.img_out = img_out;
  a.mask_x = mask_x;
  a.mask_a = mask_y;
  a.run_if = run_if;
  a.census = census;
  if (gate) {  // the learned gate runs on the default tile
    a.mlp_frag = gate->frag;
    a.mlp_bias = gate->bias;
    a.thr = gate->thr;
    a.drift_tile = gate->drift_tile;
    a.drift_dev = gate->drift_dev;
    a.Ubackup = gate->Ubackup;
    a.lstat = gate->lstat;
    a.gflags = gate->flags;
    if (gate->flags && (stage == 1 || stage == 2))  // decisions of this step's stage 0
      launch_k<2, 6, 0, TileA>(grid2d<TileA>(g), false, s, a);
    else
      launch_k<1, 6, 0, TileA>(grid2d<TileA>(g), false, s, a);
    return;
  }
  if (run_if) pdl = false;  // inside a conditional graph body: plain launches
  if (census) {
    switch (tile) {
      case 1: launch_k<3, 6, 0, TileB>(grid2d<TileB>(g), false, s, a); break;
      case 2: launch_k<3, 6, 0, TileC>(grid2d<TileC>(g), false, s, a); break;
      default: launch_k<3, 6, 0, TileA>(grid2d<TileA>(g), false, s, a); break;
    }
    return;
  }
  if (tile == 3 && rows_full >= 0 && rows_full * TileA::TY < g.n[1]) {
    a.rows_full = rows_full;
    if (a.tma) {
      if (tmk2 && tmv2) {
        a.tm_k2 = *tmk2;
        a.tm_v2 = *tmv2;
      } else {
        a.tma = 0;
      }
    }
    const int hrows = (g.n[1] - rows_full * TileA::TY + TileH::TY - 1) / TileH::TY;
    launch_kernel(k_stage_tail<6, TileA, TileH>, TileA::NT, tail_smem(), dim3(grid2d<TileA>(g).x, rows_full + hrows),
                  pdl, s, a);
    return;
  }
  switch (tile) {
    case 1: launch_k<0, 6, 0, TileB>(grid2d<TileB>(g), pdl, s, a); break;
    case 2: launch_k<0, 6, 0, TileC>(grid2d<TileC>(g), pdl, s, a); break;
    default: launch_k<0, 6, 0, TileA>(grid2d<TileA>(g), pdl, s, a); break;
  }
}

// cuTensorMapEncodeTiled, from the driver through the runtime (the library
// does not link the driver library itself)
static PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// pass2 (3D): boxes of the second pass's tile -- HXP columns x one y plane x
// HY z rows x all fields
template <class TL>
static bool encode_map(const GridDev& g, const float* buf, CUtensorMap* out, bool pass2 = false) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled();
  if (!enc || !buf) return false;
  // 2D (padded column, padded row, field), 3D (padded column, padded row,
  // padded plane, field); a box is the q tile of one CTA: HXP columns (the
  // halo's HX and the pitch's padding) x HY rows (x one plane) x all fields
  const cuuint32_t rank = g.ndim == 3 ? 4 : 3;
  cuuint64_t dims[4] = {(cuuint64_t)g.st32[1], (cuuint64_t)g.P[1], (cuuint64_t)g.nv, 1};
  cuuint64_t strides[3] = {(cuuint64_t)g.st32[1] * sizeof(float), (cuuint64_t)g.N32 * sizeof(float), 0};
  cuuint32_t box[4] = {(cuuint32_t)TL::HXP, (cuuint32_t)TL::HY, (cuuint32_t)g.nv, 1};
  if (rank == 4) {
    dims[2] = (cuuint64_t)g.P[2];
    dims[3] = (cuuint64_t)g.nv;
    strides[1] = (cuuint64_t)g.st32[2] * sizeof(float);
    strides[2] = (cuuint64_t)g.N32 * sizeof(float);
    box[2] = 1;
    box[3] = (cuuint32_t)g.nv;
    if (pass2) {
      box[1] = 1;
      box[2] = (cuuint32_t)TL::HY;
    }
  }
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, const_cast<float*>(buf), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool fused2d_encode_map(const GridDev& g, int tile, const float* buf, CUtensorMap* out) {
  // the 16-byte rules of TMA: row, plane and field pitches, and the first
  // column of every box (x0 - NG + NG = x0, a multiple of 32) as a multiple
  // of 4 floats
  if ((g.ndim != 2 && g.ndim != 3) || g.G[0] != NG || g.st32[1] % 4 != 0 || g.st32[2] % 4 != 0 ||
      g.N32 % 4 != 0 || reinterpret_cast<uintptr_t>(buf) % 16 != 0)
    return false;
  switch (tile) {
    case 1: return encode_map<TileB>(g, buf, out);
    case 2: return encode_map<TileC>(g, buf, out);
    case 4: return g.ndim == 2 && encode_map<TileH>(g, buf, out);  // the closing rows of tile 3
    case 6: return g.ndim == 3 && encode_map<TileA>(g, buf, out, true);  // second 3D pass, tile 0
    case 7: return g.ndim == 3 && encode_map<TileC>(g, buf, out, true);  // second 3D pass, tile 2
    default: return encode_map<TileA>(g, buf, out);
  }
}

// tile 3 reports its first tile shape (the one its bands and gated launches use)
int fused2d_tile_height(int tile) {
  const int ty[4] = {TileA::TY, TileB::TY, TileC::TY, TileA::TY};
  return ty[tile >= 0 && tile < 4 ? tile : 0];
}

int fused_tile_threads(int tile) {
  const int nt[4] = {TileA::NT, TileB::NT, TileC::NT, TileA::NT};
  return nt[tile >= 0 && tile < 4 ? tile : 0];
}

void launch_stage2d_band(const GridDev& g, int stage, double* U, float* U32, const float* Kin, float* Kout,
                         double dt_fixed, double cfl, unsigned long long* lmax, double* dt_out, uint8_t* mask_x,
                         uint8_t* mask_y, float eps_rel, int mood, int weights, unsigned long long* nbad, int row0,
                         int nrows, int tile, const CUtensorMap* tmk, const CUtensorMap* tmv, cudaStream_t s) {
  StageArgs a = stage_args(g, stage, U, U32, Kin, Kout, dt_fixed, cfl, lmax, dt_out, eps_rel, mood, weights, nbad);
  if (tmk && tmv) {
    a.tma = 1;
    a.tm_k = *tmk;
    a.tm_v = *tmv;
  }
  a.mask_x = mask_x;
  a.mask_a = mask_y;
  a.row0 = row0;
  switch (tile) {
    case 1: launch_k<0, 6, 0, TileB>(grid2d<TileB>(g, nrows), false, s, a); break;
    case 2: launch_k<0, 6, 0, TileC>(grid2d<TileC>(g, nrows), false, s, a); break;
    default: launch_k<0, 6, 0, TileA>(grid2d<TileA>(g, nrows), false, s, a); break;
  }
}

template <class TL>
static void stage3d_passes(const GridDev& g, const StageArgs& a0, uint8_t* mask_x, uint8_t* mask_y, uint8_t* mask_z,
                           bool census, bool pdl, const CUtensorMap* tmk2, const CUtensorMap* tmv2, cudaStream_t s) {
  StageArgs a = a0;
  // pass 1: x and y faces of every z plane -> x + y part of the divergence
  // (interior tiles by TMA when a0 carries the descriptors)
  a.mask_x = mask_x;
  a.mask_a = mask_y;
  a.clear0 = a.clear1 = nullptr;  // the stage's last pass clears
  dim3 g1((g.n[0] + TL::TX - 1) / TL::TX, (g.n[1] + TL::TY - 1) / TL::TY, g.n[2]);
  if (census)
    launch_k<3, 7, 1, TL>(g1, false, s, a);
  else
    launch_k<0, 7, 1, TL>(g1, pdl, s, a);
  // pass 2: z faces of every y plane, the whole divergence and the RK stage
  // (interior z rows by TMA with the second pair of descriptors)
  a.mask_x = nullptr;
  a.mask_a = mask_z;
  if (a0.tma && tmk2 && tmv2) {
    a.tm_k = *tmk2;
    a.tm_v = *tmv2;
  } else {
    a.tma = 0;
  }
  a.clear0 = a0.clear0;
  a.clear1 = a0.clear1;
  dim3 g2((g.n[0] + TL::TX - 1) / TL::TX, (g.n[2] + TL::TY - 1) / TL::TY, g.n[1]);
  if (census)
    launch_k<3, 7, 2, TL>(g2, false, s, a);
  else
    launch_k<0, 7, 2, TL>(g2, pdl, s, a);
}

void launch_stage3d(const GridDev& g, int stage, double* U, float* U32, const float* Kin, float* Kout, float* Lp,
                    double dt_fixed, double cfl, unsigned long long* lmax, double* dt_out, uint8_t* mask_x,
                    uint8_t* mask_y, uint8_t* mask_z, float eps_rel, int mood, int weights, unsigned long long* nbad,
                    unsigned long long* census, int tile, bool pdl, bool img_in, float* img_out,
                    unsigned long long* clear0, unsigned long long* clear1, const CUtensorMap* tmk,
                    const CUtensorMap* tmv, const CUtensorMap* tmk2, const CUtensorMap* tmv2, cudaStream_t s) {
  StageArgs a = stage_args(g, stage, U, U32, Kin, Kout, dt_fixed, cfl, lmax, dt_out, eps_rel, mood, weights, nbad);
  a.clear0 = clear0;
  a.clear1 = clear1;
  if (tmk && tmv && !census) {
    a.tma = 1;
    a.tm_k = *tmk;
    a.tm_v = *tmv;
  }
  a.Lp = Lp;
  a.census = census;
  a.img_in = img_in ? 1 : 0;
  a.img_out = img_out;
  if (tile == 2)
    stage3d_passes<TileC>(g, a, mask_x, mask_y, mask_z, census != nullptr, pdl, tmk2, tmv2, s);
  else
    stage3d_passes<TileA>(g, a, mask_x, mask_y, mask_z, census != nullptr, pdl, tmk2, tmv2, s);
}

}  // namespace ws
