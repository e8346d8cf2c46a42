// Internal declarations shared by the library's translation units (never
// installed; the public surface is include/ws.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "ws.h"

namespace ws {

constexpr int NG = 3;    // ghost layers per side
constexpr int MAXV = 7;  // rho, 3 momenta, E, Gamma, Pi

// Grid description passed by value to every kernel.
struct GridDev {
  int ndim, nv;
  int n[3];          // interior cells (1 for unused dims)
  int G[3];          // ghost offset (NG for active dims, 0 otherwise)
  int64_t P[3];      // padded extents
  int64_t st[3];     // strides of x, y, z in a field
  int64_t N;         // padded cells per field
  // layout of the fused path's FP32 buffers (stage image, increments K, 3D
  // partial divergence): the same ghost offsets G, strides and cells per
  // field of their own (2D: rows padded to a multiple of four floats, so that
  // TMA boxes of tile halos start on 16-byte boundaries; otherwise st, N)
  int64_t st32[3];
  int64_t N32;
  double dx[3];
  int bc[3][2];
  int64_t fe[3][3];  // face-array extents per direction: n[e], n[d]+1 along d
  int64_t nfaces[3];
  int64_t ncell;     // interior cells
};

// Batched 1D tubes (independent Riemann problems of uneven length).
struct TubesDev {
  int64_t ntubes;
  int64_t total;        // padded cells per field
  const int64_t* off;   // device, ntubes+1
  const int* cell_tube; // device, tube index of every padded cell
};

}  // namespace ws

struct ws_ctx {
  int dev = 0;
  cudaStream_t stream = nullptr;
  ws_grid grid{};
  ws_opts opts{};
  ws::GridDev gd{};
  int64_t nstate = 0;   // doubles per state buffer
  int64_t nmask = 0;    // mask bytes per RHS evaluation
  int64_t mask_off[3] = {0, 0, 0};
  // scratch (device)
  double* S1 = nullptr;         // RK stage state
  double* Q = nullptr;          // primitives + sound speed, nv+1 fields
  float* Q32 = nullptr;         // mixed precision: FP32 primitives + sound speed
  float* Ka = nullptr;          // fused: RK increments K0 (stage 0 -> 1)
  float* Kb = nullptr;          // fused: RK increments K1 (stage 1 -> 2)
  float* Lp = nullptr;          // fused 3D: x + y part of the divergence (first pass -> second)
  bool fused = false;           // fused mixed-precision stage kernels in use (2D or 3D)
  int stage_tile = 0;           // fused: tile shape of the stage launches (ws_autotune)
  int stage_sched = 0;          // fused: 0 stage launches with programmatic dependent launch, 1 plain
                                // stage launches (ws_autotune)
  int stage_tma = 0;            // fused 2D: 1 interior tiles load image and K as TMA boxes (ws_autotune)
  // fused plain steps: CFL maxima [0, 1] and inadmissible-cell counts [2, 3]
  // of two consecutive steps (step n uses slots n % 2 and clears those of
  // step n + 1 in its last launch, so steps follow one another with no
  // memset); the step count; the counter the last step used
  unsigned long long* chain = nullptr;
  int64_t chain_n = 0;
  unsigned long long* nbad_last = nullptr;
  bool capturing = false;       // a step is being captured into a graph (no chained slots)
  // fused 2D: TMA descriptors of Ka, Kb, Q32, img[0], img[1] for the current
  // tile shape, and [5..9] the same for the closing rows of tile 3; tmap_ok
  // bit k: descriptors k (and k + 5 for tile 3) are valid
  CUtensorMap tmap[10];
  unsigned tmap_ok = 0;
  int tail_rows = 0;            // fused 2D, tile 3: tile rows of the first shape (fused2d_tail_rows)
  bool resident = false;        // fused 2D/3D: carry the FP32 image of U between steps (ws_set_resident)
  float* img[2] = {nullptr, nullptr};  // the two image buffers (one read by a step, one written)
  int img_cur = -1;             // image valid for the next step on img_U, or -1
  const double* img_U = nullptr;
  double* Fh[3] = {nullptr, nullptr, nullptr};  // face fluxes per direction (nv fields)
  double* us[3] = {nullptr, nullptr, nullptr};  // face velocities per direction
  float* Fh32[3] = {nullptr, nullptr, nullptr}; // mixed precision face fluxes
  float* us32[3] = {nullptr, nullptr, nullptr};
  uint8_t* mask = nullptr;      // 3 stages x nmask
  double* dt_dev = nullptr;     // 1 (grid) or ntubes
  unsigned long long* lmax = nullptr;  // 1 or ntubes, max wave rate as ordered bits
  unsigned long long* nbad = nullptr;  // inadmissible cells of the last step
  unsigned long long* census = nullptr;  // fused paths: the counts of ws_census_step
  double* Uhost_dev = nullptr;  // device state for ws_run_host
  cudaStream_t cp_in = nullptr, cp_out = nullptr;  // ws_run_host: copy streams of the banded copies
  std::vector<cudaEvent_t> band_ev;                 // ws_run_host: one event per band and direction
  int last_stages = 0;
  // batched tubes
  ws::TubesDev td{};
  int64_t* off_dev = nullptr;
  int* cell_tube = nullptr;
  std::vector<int64_t> off_host;   // tube offsets
  int tube_config = 2;             // mixed tubes: autotuned (chunk, threads) configuration
  int64_t* chunk_tube = nullptr;   // device: work item -> tube
  int* chunk_start = nullptr;      // device: work item -> first cell of the chunk
  int64_t nchunks = 0;
  unsigned* counters = nullptr;    // device: 3 work counters (one per stage)
  // measurement: event pairs around launches, launch counts per kernel class
  bool prof_on = false;
  std::vector<cudaEvent_t> ev;  // 2 per recorded launch
  std::vector<int> ev_cls;
  size_t ev_used = 0;
  int64_t nlaunch[WS_NKERNEL] = {0};
  // learned smooth-face gate (ws_set_mlp)
  bool learned_on = false;
  uint2* mlp_frag = nullptr;     // device, 18 x 32
  float* mlp_bias = nullptr;     // device, 65
  float mlp_thr = 0.0f;
  int gate_flags = 6;
  float* lstat = nullptr;        // device gate statistics of the current step
  int* gate_redo = nullptr;      // device: redo flag of the current step
  double* gate_stats = nullptr;  // device: steps, redone, gated faces, faces, max drift, constant faces
  int* gate_drift = nullptr;     // device: drift-check tile residue, advanced after every gated step
  uint8_t* gate_tile_flags = nullptr;     // WS_GATE_PER_STEP: stage-0 decisions per tile
  cudaGraphExec_t ggraph_exec = nullptr;  // the gated step as a graph with a conditional redo branch
  const double* ggraph_U = nullptr;
  double ggraph_dt = 0.0;
  // CUDA graph of one CFL step (ws_set_graph)
  bool graph_on = false;
  cudaGraphExec_t graph_exec = nullptr;
  const double* graph_U = nullptr;
  // ws_get_mood scratch
  unsigned long long* mood_counts = nullptr;
  int64_t* mask_off_dev = nullptr;
  char err[512] = {0};
};

namespace ws {

// ---- launchers (ws_common.cu, built with -fmad=false) ----
void launch_ghost(const GridDev& g, double* U, int d, cudaStream_t s);
void launch_prim(const GridDev& g, const double* U, double* Q, cudaStream_t s);
void launch_prim_to_cons(const GridDev& g, const double* Q, double* U, cudaStream_t s);
void launch_cons_to_prim_all(const GridDev& g, const double* U, double* Q, cudaStream_t s);
void launch_cfl(const GridDev& g, const double* Q, unsigned long long* lmax, cudaStream_t s);
void launch_set_dt(const double* dt_fixed_or_null, double dt_fixed, double cfl, const unsigned long long* lmax,
                   double* dt_dev, int64_t n, cudaStream_t s);
void launch_update(const GridDev& g, int stage, const double* Un, const double* Us, double* Uout,
                   double* const Fh[3], double* const us[3], const double* dt_dev, unsigned long long* nbad,
                   cudaStream_t s);
void launch_mood_count(const uint8_t* mask, int64_t n, int64_t nstage, const int64_t* dir_off, int ndim,
                       unsigned long long* counts, cudaStream_t s);

// ---- FP64 sweep (ws_fp64.cu, built with -fmad=false) ----
void launch_face_fp64(const GridDev& g, int d, const double* Q, double* Fh, double* us, uint8_t* mask,
                      double eps, int mood, int weights, cudaStream_t s);

// ---- mixed-precision sweep (ws_mixed.cu, FMA allowed) ----
void launch_prim32(const GridDev& g, const double* U, float* Q, cudaStream_t s);
void launch_cfl32(const GridDev& g, const float* Q, unsigned long long* lmax, cudaStream_t s);
void launch_face_mixed(const GridDev& g, int d, const float* Q, float* Fh, float* us, uint8_t* mask, float eps_rel,
                       int mood, int weights, cudaStream_t s);
void launch_update_mixed(const GridDev& g, int stage, const double* Un, const double* Us, double* Uout,
                         float* const Fh[3], float* const us[3], const float* Q, const double* dt_dev,
                         unsigned long long* nbad, cudaStream_t s);

void launch_cfl_u(const GridDev& g, const double* U, unsigned long long* lmax, cudaStream_t s);

// ---- fused mixed-precision RK stage, 2D and 3D (ws_fused.cu) ----
struct GateArgs {
  const uint2* frag;   // BF16 MMA fragments of W1, W2, W3 (18 x 32 lanes)
  const float* bias;   // b1[32], b2[32], b3
  float thr;           // logit threshold (smooth when below)
  int drift_tile;      // tile residue (mod 64) of this step's drift check
  double* Ubackup;     // stage 0 copies U here
  float* lstat;        // gate statistics, see k_stage
  uint8_t* flags;      // nullable: per-tile decisions of stage 0, reused by stages 1 and 2
  const int* drift_dev;  // nullable: drift tile residue in device memory (overrides drift_tile)
};
int64_t fused2d_gate_flag_bytes(const GridDev& g);
// plain 2D stage over the tile rows [row0, row0 + nrows) only
// tile shapes of the fused stages (index 0, 1, 2: 32 x 15 cells per CTA of
// 512 threads, 32 x 31 of 1024, 32 x 7 of 256; 3, 2D only: rows of 32 x 15
// closed by rows of 32 x 7, both on 512 threads); 3D takes 0 and 2
int fused_num_tiles(int ndim);
int fused_tile_index(int ndim, int k);
int fused2d_tile_height(int tile);
int fused_tile_threads(int tile);
// tile 3: the number of 32 x 15 tile rows for `slots` resident CTAs
int fused2d_tail_rows(const GridDev& g, int slots);

void launch_stage2d_band(const GridDev& g, int stage, double* U, float* U32, const float* Kin, float* Kout,
                         double dt_fixed, double cfl, unsigned long long* lmax, double* dt_out, uint8_t* mask_x,
                         uint8_t* mask_y, float eps_rel, int mood, int weights, unsigned long long* nbad, int row0,
                         int nrows, int tile, const CUtensorMap* tmk, const CUtensorMap* tmv, cudaStream_t s);
int fused2d_smem_bytes();
cudaError_t fused2d_prepare();
void launch_stage2d(const GridDev& g, int stage, double* U, float* U32, const float* Kin, float* Kout,
                    double dt_fixed, double cfl, unsigned long long* lmax, double* dt_out, uint8_t* mask_x,
                    uint8_t* mask_y, float eps_rel, int mood, int weights, unsigned long long* nbad,
                    const GateArgs* gate, const int* run_if, unsigned long long* census, int tile, bool pdl,
                    bool img_in, float* img_out, const CUtensorMap* tmk, const CUtensorMap* tmv,
                    unsigned long long* clear0, unsigned long long* clear1, int rows_full, const CUtensorMap* tmk2,
                    const CUtensorMap* tmv2, cudaStream_t s);
// rows_full, tmk2, tmv2 (tile 3): the tile rows of the first shape and the
// descriptors (tile code 4) of the closing rows' boxes
// clear0, clear1 (nullable): device slots the launch sets to zero once the
// previous grid has completed (before any of its CTAs reads them)
// tmk, tmv (nullable, both or neither; plain and census launches): TMA
// descriptors of Kin and U32 from fused2d_encode_map for the launch's tile;
// interior tiles then load both as boxes.
// Describes an FP32 buffer of the fused 2D or 3D layout (g.st32, g.N32, g.nv
// fields) with boxes of one tile's halo (of one z plane in 3D); false if the
// driver refuses.  3D: tile 0 or 2 (the first pass's tiles), and 6 or 7
// for the second pass's boxes of those tiles; 2D: 0..3, and 4 for the boxes
// of tile 3's closing rows.
bool fused2d_encode_map(const GridDev& g, int tile, const float* buf, CUtensorMap* out);
// census (nullable, without a gate): the same stage, also counting the
// flat-stencil decisions into census[4] (face-variables, flat ones, warp
// passes, warp passes that ran WENO-IS)
// 3D: per stage two launches (x and y faces of every z plane, then z faces of
// every y plane with the RK stage); Lp holds the x + y part of the divergence
int fused3d_smem_bytes();
cudaError_t fused3d_prepare();
void launch_stage3d(const GridDev& g, int stage, double* U, float* U32, const float* Kin, float* Kout, float* Lp,
                    double dt_fixed, double cfl, unsigned long long* lmax, double* dt_out, uint8_t* mask_x,
                    uint8_t* mask_y, uint8_t* mask_z, float eps_rel, int mood, int weights, unsigned long long* nbad,
                    unsigned long long* census, int tile, bool pdl, bool img_in, float* img_out,
                    unsigned long long* clear0, unsigned long long* clear1, const CUtensorMap* tmk,
                    const CUtensorMap* tmv, const CUtensorMap* tmk2, const CUtensorMap* tmv2, cudaStream_t s);
// tmk2, tmv2 (nullable, with tmk and tmv): descriptors of the second pass's
// boxes (fused2d_encode_map codes 6 and 7); interior z rows of the second
// pass then load by TMA
void launch_gate_decide(const float* lstat, unsigned long long* nbad, unsigned long long* lmax, int flags, int* redo,
                        double* stats, int* drift_dev, cudaGraphConditionalHandle cond, cudaStream_t s);
void launch_restore(const int* redo, const double* src, double* dst, int64_t n, cudaStream_t s);

// ---- batched tubes, mixed precision, persistent (ws_tubes_mixed.cu) ----
extern const int kNumTubeConfigs;
int tube_chunk_size(int config);
void launch_tubes_stage_mixed(const TubesDev& t, int config, int stage, double* U, float* U32, const float* Kin,
                              float* Kout, double dt_fixed, double cfl, unsigned long long* lmax, double* dt_out,
                              const int64_t* chunk_tube, const int* chunk_start, int64_t nitems, unsigned* counter,
                              uint8_t* mask, float eps_rel, int mood, int weights, unsigned long long* nbad,
                              cudaStream_t s);

// ---- learned gate (ws_learned.cu) ----
void launch_face_samples(const GridDev& g, int d, const float* Q, int64_t stride, int64_t out0, int64_t max_out,
                         float* feats, uint8_t* labels, float eps_rel, int weights, cudaStream_t s);

// ---- batched tubes (ws_tubes.cu) ----
void launch_tubes_ghost(const TubesDev& t, double* U, cudaStream_t s);
void launch_tubes_prim(const TubesDev& t, const double* U, double* Q, cudaStream_t s);
void launch_tubes_cfl(const TubesDev& t, const double* Q, unsigned long long* lmax, cudaStream_t s);
void launch_tubes_face_fp64(const TubesDev& t, const double* Q, double* Fh, double* us, uint8_t* mask, double eps,
                            int mood, int weights, cudaStream_t s);
void launch_tubes_update(const TubesDev& t, int stage, const double* Un, const double* Us, double* Uout,
                         const double* Fh, const double* us, const double* dt_dev, unsigned long long* nbad,
                         cudaStream_t s);

}  // namespace ws
