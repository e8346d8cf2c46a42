/*
 * ws.h -- C ABI of the GB300 WENO-IS two-phase solver library (libws_gb300.so).
 *
 * The library advances the quasi-conservative two-phase model of Wang, Xiang,
 * Zhang & Hu (arXiv 1707.00592): the Euler equations with the stiffened-gas
 * EOS rho e = Gamma p + Pi (Sec. 2, Eqs. governing-equation and eos) and the
 * non-conservative advection of phi = (Gamma, Pi) = (1/(gamma-1),
 * gamma P_inf/(gamma-1)) (Eqs. material-equation, material-properties).
 * Space: cell-averaged finite volumes (Sec. 3.1), characteristic
 * primitive-variable WENO-IS reconstruction (Secs. 3.2, 3.3), MOOD positivity
 * cascade (Sec. 3.4) and HLLC fluxes (Sec. 3.2.1); time: SSP-RK3 (Sec. 3.1).
 *
 * Conventions for every entry point
 *  - All state pointers are DEVICE pointers (cudaMalloc'd or torch tensors on
 *    the context's device) unless the name ends in _host.  The caller owns
 *    them; the library never frees them and never keeps them past the call.
 *  - A state buffer holds nv = ndim + 4 fields of FP64 in structure-of-arrays
 *    order (rho, rho u_1 .. rho u_ndim, E, Gamma, Pi), each field a padded
 *    [z][y][x] block (x fastest) with 3 ghost cells on both sides of every
 *    active direction: padded extent n[d] + 6 for d < ndim, 1 otherwise.
 *    ws_state_size() returns the number of doubles.  In batched-tube mode
 *    (ws_grid.ntubes > 0) each field is the concatenation of the tubes' padded
 *    segments, tube t on [tube_offsets[t], tube_offsets[t+1]).
 *  - Ghost cells of a state passed to ws_step / ws_flux_divergence /
 *    ws_cfl_dt are scratch: the FP64 path overwrites them from the boundary
 *    conditions, the fused mixed-precision paths apply the boundary
 *    conditions while loading and leave them as they were.  Their contents
 *    are not inputs and should not be relied on.  Interior cells are only
 *    written by ws_step (and ws_run_host, ws_census_step).
 *  - Work is enqueued on the CUDA stream given to ws_init, in order.  Calls
 *    return once the work is enqueued, except where a host-side result is
 *    requested (noted per call), which synchronises that stream.
 *  - Every call returns a WS_* status; ws_last_error() gives a message.  No
 *    call aborts the process or lets a C++ exception cross the ABI.  A context
 *    is not thread-safe: one host thread at a time.
 */
#ifndef WS_GB300_H
#define WS_GB300_H

#include <stdint.h>

#if defined(__GNUC__)
#define WS_API __attribute__((visibility("default")))
#else
#define WS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define WS_OK 0
#define WS_EINVAL 1    /* bad argument: grid, options, size or pointer */
#define WS_ECUDA 2     /* a CUDA runtime call failed */
#define WS_ENONPHYS 3  /* a cell ended the step with rho <= 0, Gamma <= 0 or (Gamma+1)p + Pi <= 0 */
#define WS_ETIMEOUT 4  /* a bounded device-side wait gave up */
#define WS_ENOTSUP 5   /* combination of options not built */

/* boundary kinds (per direction and side) */
#define WS_BC_TRANSMISSIVE 0 /* zero-gradient ("constant extrapolation", non-reflecting), Sec. 6 */
#define WS_BC_PERIODIC 1     /* Sec. 4 */
#define WS_BC_REFLECTIVE 2   /* slip wall: mirror, normal momentum negated */

/* arithmetic of the sweep */
#define WS_PREC_FP64 0  /* everything in FP64; same operation order as the FP64 oracle */
#define WS_PREC_MIXED 1 /* FP32 projection, WENO-IS and HLLC; FP64 pressure recovery,
                           MOOD test, flux divergence and RK accumulation */

/* nonlinear weights */
#define WS_W_MODIFIED 0 /* Sec. 3.3.2, Eq. (weighting-modification): the scheme */
#define WS_W_BASIC 1    /* Sec. 3.3.1, Eq. (weight-new) with q = 1 */
#define WS_W_JS 2       /* the comparison scheme of Secs. 5 and 6: classical WENO-JS (Jiang & Shu 1996),
                           3-point candidates, d = (1,6,3)/10, alpha_k = d_k/(eps + beta_k)^2; under MOOD
                           its 3rd-order level is the scheme's own (the 2-point candidates, modified weights) */

typedef struct ws_grid {
  int ndim;                    /* 1, 2 or 3 */
  int n[3];                    /* interior cells per direction (n[d] >= 1; unused dims ignored) */
  double dx[3];                /* uniform cell size per direction (> 0) */
  int bc[3][2];                /* WS_BC_* per direction, [d][0] low side, [d][1] high side */
  int64_t ntubes;              /* > 0: batched independent 1D tubes (ndim must be 1); in mixed precision
                                  one persistent launch per RK stage works through (tube, chunk) items */
  const int64_t *tube_offsets; /* HOST array of ntubes+1 padded offsets; each tube has
                                  len = off[t+1]-off[t]-6 >= 6 interior cells, dx = 1/len,
                                  transmissive ends; copied at ws_init */
} ws_grid;

typedef struct ws_opts {
  int precision; /* WS_PREC_* */
  int weights;   /* WS_W_* */
  int mood;      /* 1: MOOD positivity cascade 5th -> 3rd -> 1st (Sec. 3.4); 0: off */
  int learned;   /* 1: smooth-face gate by the face-classifier MLP (mixed precision only) */
  double eps;    /* WENO epsilon (the paper leaves it open).  FP64: absolute, <= 0 selects 1e-40.
                    Mixed: relative to beta1 + beta2 + tau5 of the stencil (floor 1e-30), <= 0
                    selects 1e-10 -- keeps tau5/(beta+eps) within FP32 range for p ~ 1e9.
                    WS_W_JS: the absolute epsilon of WENO-JS in both precisions, <= 0 selects
                    Jiang & Shu's 1e-6 (its MOOD 3rd-order level then uses the defaults above) */
  double cfl;    /* CFL number; <= 0 selects 0.5 (Secs. 5, 6) */
  int check;     /* 1: ws_step synchronises and returns WS_ENONPHYS when a cell is inadmissible */
} ws_opts;

typedef struct ws_ctx ws_ctx;

/* Create a context on the current CUDA device.  Validates the grid (ndim,
 * n, dx, bc, tube offsets) and options, allocates the context's scratch
 * (primitive cache, face fluxes, RK stage state, MOOD masks) and returns it in
 * *out.  stream: a cudaStream_t (NULL = legacy default stream).
 * The problem is the initial-value problem of Sec. 2: the Euler equations
 * (Eq. governing-equation) closed by the stiffened-gas EOS rho e = Gamma p +
 * Pi (Eq. eos), with the material functions Gamma = 1/(gamma-1) and Pi =
 * gamma P_inf/(gamma-1) (Eq. material-properties) advected by Eq.
 * (material-equation).  The EOS parameters are therefore not arguments of
 * ws_init: every cell of the state carries its own Gamma and Pi (two of its
 * fields), which is also what describes a mixture cell of a smeared
 * interface, where no single (gamma, P_inf) exists.  A fluid with (gamma,
 * P_inf) enters through ws_prim_to_cons with those two fields set.
 * Errors: WS_EINVAL (bad grid/options; *out untouched), WS_ECUDA. */
WS_API int ws_init(const ws_grid *grid, const ws_opts *opts, void *stream, ws_ctx **out);

/* Number of doubles in one state buffer (nv fields x padded cells). */
WS_API int64_t ws_state_size(const ws_ctx *ctx);

/* Number of MOOD mask bytes written per RHS evaluation (all directions).  The
 * mask of direction d covers faces i+1/2, i = -1..n_d-1, at every interior
 * transverse position, laid out [z][y][x] with extent n_d+1 along d;
 * directions follow one another.  Byte = code(left) | code(right) << 2 with
 * code 0/1/2 for 5th/3rd/1st order. */
WS_API int64_t ws_mask_size(const ws_ctx *ctx);

/* Primitive (rho, u_1..u_ndim, p, Gamma, Pi) -> conservative state, every
 * padded cell (Eq. eos: E = Gamma p + Pi + rho |u|^2 / 2).  Q, U: device
 * buffers of ws_state_size() doubles; Q may not alias U. */
WS_API int ws_prim_to_cons(ws_ctx *ctx, const double *Q, double *U);

/* Conservative -> primitive, every padded cell; p = (E - rho|u|^2/2 - Pi)/Gamma in FP64. */
WS_API int ws_cons_to_prim(ws_ctx *ctx, const double *U, double *Q);

/* The semi-discrete operator of Sec. 3.1, Eqs. (semi-discrezization-euler)
 * and (semi-discrezization-material): L(U) = -sum_d (F_{i+1/2} - F_{i-1/2})/dx_d,
 * plus phi_i sum_d (u_{i+1/2} - u_{i-1/2})/dx_d for Gamma and Pi, on interior
 * cells (ghost entries of L are not written).  U's ghosts are filled first.
 * The MOOD mask of this evaluation is kept (see ws_get_mood, stage 0).
 * Not available in batched-tube mode (WS_ENOTSUP). */
WS_API int ws_flux_divergence(ws_ctx *ctx, double *U, double *L);

/* CFL step of U: dt = cfl / max_cells sum_d (|u_d| + c)/dx_d.  Synchronises;
 * *dt is a host double (batched-tube mode: the minimum over tubes). */
WS_API int ws_cfl_dt(ws_ctx *ctx, double *U, double *dt);

/* One SSP-RK3 step (Shu & Osher; Sec. 3.1) of U in place:
 *   U1 = U + dt L(U);  U2 = 3/4 U + 1/4 (U1 + dt L(U1));  U <- 1/3 U + 2/3 (U2 + dt L(U2)).
 * dt <= 0 takes the CFL step computed on the device from U (per tube in
 * batched-tube mode); dt > 0 is used as given (every tube).  dt_used
 * (nullable, HOST) receives the step (ntubes values in batched-tube mode) and
 * then the call synchronises.  With opts.check = 1 the call synchronises and
 * returns WS_ENONPHYS if any interior cell ends inadmissible (U is left as
 * computed).  The MOOD masks of the three stages are kept for ws_get_mood. */
WS_API int ws_step(ws_ctx *ctx, double *U, double dt, double *dt_used);

/* End-to-end form for host-resident data: copies the state from HOST memory
 * U_host (ws_state_size() doubles; pinned memory gives full copy speed) to
 * the context's device buffer, runs nsteps ws_step's (dt as in ws_step), and
 * copies the state back to U_host.  Synchronises.  dt_used (nullable, HOST)
 * receives the last step's dt (ntubes values in batched-tube mode).  On the
 * fused 2D mixed-precision path (learned gate off) the copies go by bands of
 * tile rows on two internal copy streams: stage 0 of the first step starts on
 * each band as it arrives and each band of the last step's stage 2 is copied
 * back while the next computes; the results are those of ws_step.  The
 * opts.check test of ws_step is not made here. */
WS_API int ws_run_host(ws_ctx *ctx, double *U_host, int nsteps, double dt, double *dt_used);

/* MOOD record of the last ws_step (3 stages) or ws_flux_divergence (stage 0
 * only).  mask (nullable, DEVICE): receives 3 x ws_mask_size() bytes, stage
 * major.  counts (nullable, HOST int64[9]): faces-sides per direction d and
 * level k (5th, 3rd, 1st) at counts[3*d + k], summed over the stages of that
 * call and both sides.  Synchronises when counts is given. */
WS_API int ws_get_mood(ws_ctx *ctx, uint8_t *mask, int64_t counts[9]);

/* Number of inadmissible interior cells found at the end of the last
 * ws_step (HOST out).  Synchronises. */
WS_API int ws_nonphysical(ws_ctx *ctx, int64_t *count);

/* Census step (a measurement aid; the paper has no counterpart): one ws_step
 * of U in place, with the same kernels' arithmetic and results, that also
 * counts how the reconstruction of Sec. 3.3 was evaluated.  A characteristic
 * variable whose six stencil values are flat to 1e-6 of their magnitude takes
 * the linear weights; every other one takes WENO-IS.  counts (HOST int64[4]),
 * summed over the three RK stages and every face evaluation (the fused stage
 * evaluates all faces of each 32 x 15 tile, so a face on the edge between two
 * tiles is evaluated twice):
 *   [0] face-variables (one per characteristic variable per face evaluation),
 *   [1] those whose stencil was flat,
 *   [2] warp passes (32 consecutive faces evaluating one variable together),
 *   [3] warp passes in which at least one face took WENO-IS.
 * Only on the fused mixed-precision 2D and 3D paths (WS_EINVAL elsewhere); the
 * learned gate, if set, is not applied.  dt, dt_used and opts.check as in
 * ws_step.  Synchronises. */
WS_API int ws_census_step(ws_ctx *ctx, double *U, double dt, double *dt_used, int64_t counts[4]);

/* ---- learned smooth-face gate (not in the paper) ----
 * A 24 -> 32 -> 32 -> 1 MLP (ReLU, ReLU, sigmoid) marks faces whose WENO-IS
 * value would equal the 5th-order linear-weight value (d = (4,2,3,1)/10 of
 * Sec. 3.3.1) to 1e-6 of the stencil's range; those faces skip the
 * smoothness indicators and nonlinear weights.  Inputs of face i+1/2: the
 * characteristic variables w1, w2, w6 and w_Gamma (Sec. 3.2, Eq.
 * eigen-vectors) of cells i-2..i+3, each normalised over the stencil as
 * (w - mean)/(max - min + 1e-30), ordered [variable][cell].
 * Parameters: WS_MLP_NPARAM FP32 values W1[32][24], b1[32], W2[32][32],
 * b2[32], W3[32], b3 (DEVICE arrays in the calls below). */
#define WS_MLP_NPARAM 1889
#define WS_MLP_NIN 24

/* Training samples from state U (mixed-precision context, grid mode): every
 * stride-th face of each direction (directions one after another), at most
 * max_out.  feats (DEVICE, max_out x 24 FP32) and labels (DEVICE, max_out
 * bytes: 1 = the face needs WENO-IS -- MOOD lowers a side, or WENO-IS and the
 * linear weights differ by more than 1e-6 of the range for some variable and
 * side; 0 = smooth).  *count (HOST) receives the number written.  U's ghosts
 * are filled first.  Synchronises. */
WS_API int ws_face_samples(ws_ctx *ctx, double *U, int64_t stride, int64_t max_out, float *feats,
                           uint8_t *labels, int64_t *count);

/* logits[i] (DEVICE, n FP32) of samples X (DEVICE, n x 24 FP32) under params
 * (FP32 forward pass).  Enqueued on `stream`. */
WS_API int ws_mlp_forward(const float *params, const float *X, int64_t n, float *logits, void *stream);

/* Gradient (DEVICE, WS_MLP_NPARAM FP32, overwritten) and *loss (DEVICE FP32,
 * overwritten) of the mean binary cross-entropy over n samples, positives
 * weighted by pos_weight.  Enqueued on `stream`.  The sums are formed in 64-bit
 * fixed point (units of 2^-48, each contribution rounded once), so the result
 * does not depend on the order of the threads: the same inputs give the same
 * bits on every run.  They use one accumulator per device inside the library:
 * calls on different streams must not run at the same time. */
WS_API int ws_mlp_grad(const float *params, const float *X, const uint8_t *y, int64_t n, float pos_weight,
                       float *grad, float *loss, void *stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) of params with moment
 * buffers m, v (DEVICE, WS_MLP_NPARAM FP32 each, zero before step 1); step
 * counts from 1.  Enqueued on `stream`. */
WS_API int ws_mlp_adam(float *params, float *m, float *v, const float *grad, int64_t step, float lr, void *stream);

/* Switch the learned gate on for the fused 2D mixed-precision path
 * (WS_ENOTSUP elsewhere).  params: DEVICE, WS_MLP_NPARAM FP32 values (copied
 * and converted to BF16 tensor-core fragments); NULL switches the gate off.
 * A face whose logit is below `threshold` takes the linear weights; every
 * face still goes through the MOOD cascade (a gated side that fails falls
 * back to 3rd-order WENO-IS, then 1st order).  Each gated ws_step keeps a
 * copy of U and, on the device (no host round trip), redoes the step
 * without the gate if (flags & WS_GATE_REDO_NONPHYS) a cell ends
 * inadmissible, if (flags & WS_GATE_REDO_DRIFT) on the 1/64 of the tiles
 * checked that step (rotating) the linear-weight face values differ from
 * WENO-IS by more than 1e-6 in relative L1, or if (flags &
 * WS_GATE_REDO_MOOD) any gated face needed the MOOD cascade.  With (flags &
 * WS_GATE_PER_STEP) the MLP runs once per step, on U^n in RK stage 0, and
 * stages 1 and 2 apply the same decisions to their intermediate states (which
 * lie within a CFL fraction of a cell of U^n); the drift check still runs in
 * every stage.  Without it the MLP runs in every stage.  On a context created
 * with a stream, a gated step is one CUDA graph launch whose redo branch is a
 * conditional node set by the device.  Resets the statistics of
 * ws_gate_stats. */
#define WS_GATE_REDO_MOOD 1
#define WS_GATE_REDO_DRIFT 2
#define WS_GATE_REDO_NONPHYS 4
#define WS_GATE_PER_STEP 8
WS_API int ws_set_mlp(ws_ctx *ctx, const float *params, float threshold, int flags);

/* The gate's decisions on state U (DEVICE): smooth (DEVICE, ws_mask_size()
 * bytes, laid out like one stage of the MOOD mask) receives 1 for faces that
 * would take the linear weights, 0 otherwise.  Enqueued on the context's
 * stream. */
WS_API int ws_gate_eval(ws_ctx *ctx, double *U, uint8_t *smooth);

/* Gate statistics since ws_set_mlp (HOST out[6]): gated steps, steps redone
 * without the gate, faces the MLP sent to the linear weights, faces examined,
 * largest drift ratio seen, faces with a constant stencil (these need no
 * reconstruction and bypass the MLP); face counts are summed over RK stages.
 * Synchronises. */
WS_API int ws_gate_stats(ws_ctx *ctx, double out[6]);

/* Chooses the kernel configuration of the context by timing each candidate
 * for `steps` CFL steps (after one warm-up step) on a scratch copy of U
 * (DEVICE; U itself is not modified), in two rounds over the candidates; a
 * candidate's time is its faster round.  Every candidate gives bit-identical
 * results; only the time differs.
 *  - Fused 2D/3D mixed-precision stages (learned gate off): the tile of cells
 *    a CTA owns and its thread count -- 32 x 15 cells on 512 threads (two CTAs
 *    per SM), 32 x 31 on 1024 (one CTA per SM; 2D only: with 7 fields its
 *    shared memory exceeds a CTA's limit) or 32 x 7 on 256 (four CTAs per SM)
 *    -- or, 2D only, rows of 32 x 15 tiles closed by rows of 32 x 7 tiles,
 *    both on 512 threads in one launch (the smaller closing CTAs even out the
 *    end of the launch's last wave; the split is chosen for the GPU's SM
 *    count by a list schedule of the launch's CTAs, 0.6 the cost of a full
 *    one for a 32 x 7 CTA, and reported as tail_rows)
 *    -- the loads: 0 every CTA loads its tile and 3-cell halo cell by cell,
 *    applying the boundary conditions; 1 a CTA whose halo lies inside the
 *    grid loads the stage's FP32 image and increments as two TMA boxes (the
 *    others as with 0; in the second 3D pass, of z faces, a CTA whose z halo
 *    lies inside the grid) -- and the
 *    launch schedule: 0 one launch per
 *    stage (per pass in 3D), consecutive launches with programmatic
 *    dependent launch (the next launch's CTAs wait on the device for the
 *    previous grid instead of being launched after it); 1 the same launches
 *    without it.  Candidate index = 4 x tile + 2 x loads + schedule; tiles
 *    0, 1, 2, 3 = 32 x 15, 32 x 31, 32 x 7, 32 x 15 closed by 32 x 7 in 2D
 *    (16 candidates), 0, 1 = 32 x 15, 32 x 7 in 3D (8 candidates).
 *    ws_get_stage_config reports the choice.
 *  - Batched tubes in mixed precision: the chunk of cells a CTA of the
 *    persistent stage kernel processes and its thread count, from (255, 128),
 *    (255, 256), (511, 256), (511, 512), (1023, 512) (a chunk of 2^k - 1
 *    cells has 2^k faces, a whole number per thread).
 * *choice (HOST, nullable) receives the index chosen, or -1 when the context
 * has nothing to tune.  Allocates a scratch state for the duration of the
 * call.  Synchronises.  The choice stays with the context (a CUDA graph of
 * ws_set_graph is captured again). */
WS_API int ws_autotune(ws_ctx *ctx, const double *U, int steps, int *choice);

/* Sets the fused stages' configuration to candidate `index` of ws_autotune
 * (the default is 14 in 2D: 32 x 15 tile rows closed by 32 x 7 rows, TMA
 * loads, stage launches with programmatic dependent launch -- 12 if the
 * driver cannot describe the buffers for TMA; 3 in 3D: 32 x 15 tiles, TMA
 * loads, plain launches -- 1 without TMA).  A TMA candidate
 * falls back to cell-by-cell loads when the driver refuses a descriptor
 * (ws_get_stage_config then reports loads 0).  WS_EINVAL on a context without
 * fused stages or an index that is not a candidate. */
WS_API int ws_set_stage_config(ws_ctx *ctx, int index);

/* The fused stages' configuration (HOST outs, each nullable): candidate
 * index, tile width and height in cells (of the first tile shape for 2D tile
 * 3), threads per CTA, schedule and loads (0 or 1 each, as in ws_autotune),
 * and tail_rows: for 2D tile 3 the number of 32 x 15 tile rows before the
 * 32 x 7 rows (all the grid's tile rows when no split pays), otherwise -1.
 * WS_EINVAL without fused stages. */
WS_API int ws_get_stage_config(ws_ctx *ctx, int *index, int *tile_x, int *tile_y, int *threads, int *schedule,
                               int *tma, int *tail_rows);

/* enable = 1 declares that U, the state of consecutive ws_step calls of this
 * context, changes between them only through those calls.  The fused 2D and
 * 3D mixed-precision stages then carry the FP32 image of the state (every field
 * rounded to FP32, E - Pi formed in FP64 first) from one step's last stage to
 * the next step's first: stage 2 writes the image of the new state, and the
 * next step's stage 0 reads it instead of loading and converting the FP64
 * state of its tiles and halos.  The results are the same, bit for bit.  The
 * next step starts over from the FP64 state after a ws_step on another state
 * or any other call that reads or writes the state (ws_prim_to_cons,
 * ws_flux_divergence, ws_census_step, ws_run_host, ws_face_samples,
 * ws_gate_eval, ws_autotune, ws_set_stage_config, ws_set_mlp) -- but not
 * after a change the caller makes to U itself, which this promise rules out.
 * Resident steps are not replayed from a CUDA graph (ws_set_graph).  Allocates
 * two image buffers (nv FP32 fields each) on first use.  enable = 0: off (the
 * default).  WS_ENOTSUP on a context without the fused stages (FP64, 1D,
 * batched tubes). */
WS_API int ws_set_resident(ws_ctx *ctx, int enable);

/* enable != 0: ws_step calls that take the CFL step (dt <= 0) replay one CUDA
 * graph holding the whole step (CFL reduction and the three RK stages)
 * instead of launching its kernels one by one; the graph is captured on the
 * first such call for a given state pointer U (and again when U changes).
 * Needs a stream other than the legacy default stream; ignored while
 * ws_profile recording is on.  Results are identical either way.
 * 0: launch kernels directly (the default). */
WS_API int ws_set_graph(ws_ctx *ctx, int enable);

/* ---- measurement helpers (not part of the method) ---- */

/* kernel classes for ws_profile_read */
#define WS_K_GHOST 0   /* ghost layers */
#define WS_K_PRIM 1    /* conservative -> primitive cache */
#define WS_K_CFL 2     /* CFL max-reduction and dt */
#define WS_K_FACE 3    /* face sweep: projection, WENO-IS, MOOD, HLLC */
#define WS_K_UPDATE 4  /* flux divergence + RK stage */
#define WS_K_OTHER 5
#define WS_NKERNEL 8

/* enable == 1: from now on record a CUDA event pair around every kernel the
 * context launches (on its stream) and reset the totals; 2: resume recording
 * without resetting; 0: stop recording.  The three stages of a plain fused 2D
 * step follow one another with programmatic dependent launch, which events
 * between them would undo: one event pair spans the three and counts as three
 * launches of WS_K_FACE (the span includes the two short gaps). */
WS_API int ws_profile(ws_ctx *ctx, int enable);

/* Device time (ms, summed over launches, from the recorded events) and launch
 * count per kernel class, over the launches made while recording was on since
 * the last ws_profile(ctx, 1).  ms and launches are HOST arrays of WS_NKERNEL
 * entries (either may be NULL).  Synchronises. */
WS_API int ws_profile_read(ws_ctx *ctx, double ms[WS_NKERNEL], int64_t launches[WS_NKERNEL]);

/* Throughput of dependent fused multiply-add chains on the current device:
 * kind 0 = FP64 (DFMA), 1 = FP32 (FFMA); *tflops receives 2 x FMAs / s / 1e12
 * over a launch of blocks x 256 threads (blocks <= 0: 8 per SM).  Synchronises. */
WS_API int ws_peak_probe(int kind, int blocks, double *tflops);

/* ---- allocation-free flux divergence ----
 * The paper has no counterpart to this entry point: it serves callers that
 * cannot call cudaMalloc, such as a host application whose device memory is
 * owned by another allocator or a fixed budget (a framework's caching pool, a
 * plugin host), or a latency-critical loop that must not allocate after
 * start-up.  They cannot create a ws_ctx (ws_init allocates scratch), so this
 * call takes the grid and options directly and uses as scratch one file-scope
 * device array of WS_NOALLOC_SCRATCH_BYTES that every GPU loading the library
 * holds until the process exits.  It allocates nothing: no cudaMalloc, no
 * cudaFree, no allocating library routine.
 *
 * Computes the same L(U) as ws_flux_divergence (FP64, same kernels, same bits;
 * no MOOD mask is kept).  U (DEVICE, ghosts overwritten from the boundary
 * conditions) and L (DEVICE, interior written) are caller buffers in the state
 * layout above.  Grids whose primitive cache plus face fluxes exceed the
 * scratch (beyond 313 x 313 cells in 2D, 38^3 in 3D or 174756 cells in 1D) are
 * rejected with WS_EINVAL; batched tubes and mixed precision with WS_ENOTSUP;
 * the options are checked as ws_init checks them (WS_EINVAL).  U, L and the
 * stream must belong to the current CUDA device: the scratch used is that
 * device's copy of the array.
 * err (nullable, HOST, err_len bytes) receives a message on failure.
 * Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default).
 * The first call on each device looks up the scratch's device address with
 * cudaGetSymbolAddress, with that device current; make that first call
 * before any stream capture.  All calls share the one array and it keeps the
 * last call's contents (each call writes what it reads first, so nothing needs
 * clearing); calls whose work overlaps on the GPU, from any thread or stream,
 * race on it and must be serialised by the caller. */
#define WS_NOALLOC_SCRATCH_BYTES (16LL * 1024 * 1024)
WS_API int ws_flux_divergence_noalloc(const ws_grid *grid, const ws_opts *opts, void *stream, double *U,
                                      double *L, char *err, int err_len);

/* Applies the mixed-precision kernels' integer-pipe conversions to n DEVICE
 * doubles: out32[i] = in[i] rounded to FP32 (nearest even; +-0 below the FP32
 * normal range, +-inf above it, NaN kept), out64[i] = out32[i] widened back
 * (exact; +-0 for subnormals).  A test hook: the paper has no counterpart.
 * Runs on the legacy default stream and synchronises the device. */
WS_API int ws_convert_probe(int64_t n, const double *in, float *out32, double *out64);

/* Message of the last failing call on ctx (never NULL; "" when none). */
WS_API const char *ws_last_error(const ws_ctx *ctx);

/* Message of the last ws_init failure (for calls that got no context). */
WS_API const char *ws_init_error(void);

/* Free the context and its scratch.  NULL is a no-op. */
WS_API void ws_destroy(ws_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* WS_GB300_H */
