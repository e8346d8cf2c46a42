// Host side of the C ABI declared in include/ws.h: validation, scratch
// ownership and the stream-ordered launch sequence of an SSP-RK3 step.
#include <algorithm>
#include <optional>
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "ws_internal.h"

using namespace ws;

namespace {

char g_init_err[512] = "";

int fail(ws_ctx* c, int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(c ? c->err : g_init_err, 512, fmt, ap);
  va_end(ap);
  return code;
}

#define CK(ctx, call)                                                                              \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail(ctx, WS_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

int check_launch(ws_ctx* c, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, WS_ECUDA, "%s launch failed: %s", what, cudaGetErrorString(e));
  return WS_OK;
}

// fused 2D, tile 3: the split of the grid's tile rows for this GPU (two
// resident CTAs per SM)
static void set_tail_rows(ws_ctx* c) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  c->tail_rows = fused2d_tail_rows(c->gd, 2 * nsm);
}

// fused 2D and 3D: TMA descriptors of the FP32 buffers for the current tile
// shape (3D: of the first pass, and [5..9] of the second)
void encode_maps(ws_ctx* c) {
  c->tmap_ok = 0;
  if (!c->fused) return;
  // second descriptors: the closing rows of 2D tile 3, the second 3D pass
  const int code2 = c->gd.ndim == 3 ? (c->stage_tile == 2 ? 7 : 6) : (c->stage_tile == 3 ? 4 : -1);
  const float* bufs[5] = {c->Ka, c->Kb, c->Q32, c->img[0], c->img[1]};
  for (int k = 0; k < 5; ++k)
    if (bufs[k] && fused2d_encode_map(c->gd, c->stage_tile, bufs[k], &c->tmap[k]) &&
        (code2 < 0 || fused2d_encode_map(c->gd, code2, bufs[k], &c->tmap[5 + k])))
      c->tmap_ok |= 1u << k;
}

// the descriptors of a launch's K and image buffers, or null (then every tile
// loads cell by cell)
const CUtensorMap* map_of(const ws_ctx* c, const float* buf) {
  if (!c->stage_tma) return nullptr;
  const float* bufs[5] = {c->Ka, c->Kb, c->Q32, c->img[0], c->img[1]};
  for (int k = 0; k < 5; ++k)
    if (buf && bufs[k] == buf) return (c->tmap_ok >> k & 1u) ? &c->tmap[k] : nullptr;
  return nullptr;
}

// the descriptor of the closing rows' boxes (tile 3) beside map_of's
const CUtensorMap* map2_of(const ws_ctx* c, const CUtensorMap* m) {
  return m ? m + 5 : nullptr;
}

template <typename T>
int dalloc(ws_ctx* c, T** p, int64_t count) {
  *p = nullptr;
  if (count <= 0) return WS_OK;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (size_t)count);
  if (e != cudaSuccess) return fail(c, WS_ECUDA, "cudaMalloc(%lld bytes): %s", (long long)(sizeof(T) * count),
                                    cudaGetErrorString(e));
  return WS_OK;
}

// Records an event pair around the launches of its scope and counts the kernel
// launches of its class, while profiling is on.
struct KScope {
  ws_ctx* c;
  int cls;
  int n;
  size_t slot = (size_t)-1;
  KScope(ws_ctx* c_, int cls_, int nkernels = 1) : c(c_), cls(cls_), n(nkernels) {
    if (!c->prof_on) return;
    if (c->ev_used + 2 > c->ev.size()) {
      for (int k = 0; k < 64; ++k) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        c->ev.push_back(e);
      }
      c->ev_cls.resize(c->ev.size() / 2);
    }
    slot = c->ev_used;
    c->ev_used += 2;
    c->ev_cls[slot / 2] = cls;
    cudaEventRecord(c->ev[slot], c->stream);
  }
  ~KScope() {
    if (c->prof_on) c->nlaunch[cls] += n;
    if (slot != (size_t)-1) cudaEventRecord(c->ev[slot + 1], c->stream);
  }
};

void free_all(ws_ctx* c) {
  cudaFree(c->S1);
  cudaFree(c->Q);
  cudaFree(c->Q32);
  cudaFree(c->chain);
  cudaFree(c->img[0]);
  cudaFree(c->img[1]);
  cudaFree(c->Ka);
  cudaFree(c->Kb);
  cudaFree(c->Lp);
  for (int d = 0; d < 3; ++d) {
    cudaFree(c->Fh[d]);
    cudaFree(c->us[d]);
    cudaFree(c->Fh32[d]);
    cudaFree(c->us32[d]);
  }
  cudaFree(c->mask);
  cudaFree(c->dt_dev);
  cudaFree(c->lmax);
  cudaFree(c->nbad);
  cudaFree(c->census);
  cudaFree(c->Uhost_dev);
  cudaFree(c->off_dev);
  cudaFree(c->cell_tube);
  cudaFree(c->chunk_tube);
  cudaFree(c->chunk_start);
  cudaFree(c->counters);
  cudaFree(c->mood_counts);
  cudaFree(c->mask_off_dev);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  c->ev.clear();
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  c->graph_exec = nullptr;
  if (c->ggraph_exec) cudaGraphExecDestroy(c->ggraph_exec);
  c->ggraph_exec = nullptr;
  for (cudaEvent_t e : c->band_ev) cudaEventDestroy(e);
  c->band_ev.clear();
  if (c->cp_in) cudaStreamDestroy(c->cp_in);
  if (c->cp_out) cudaStreamDestroy(c->cp_out);
  c->cp_in = c->cp_out = nullptr;
  cudaFree(c->gate_drift);
  cudaFree(c->gate_tile_flags);
  cudaFree(c->mlp_frag);
  cudaFree(c->mlp_bias);
  cudaFree(c->lstat);
  cudaFree(c->gate_redo);
  cudaFree(c->gate_stats);
}

bool tubes(const ws_ctx* c) { return c->grid.ntubes > 0; }

// work items of the persistent mixed-precision tube kernel: chunks of CH cells
int build_chunks(ws_ctx* c, int config) {
  int CH = tube_chunk_size(config);
  std::vector<int64_t> ct;
  std::vector<int> cs;
  for (int64_t t = 0; t < c->td.ntubes; ++t) {
    int64_t len = c->off_host[t + 1] - c->off_host[t] - 2 * NG;
    for (int64_t s0 = 0; s0 < len; s0 += CH) {
      ct.push_back(t);
      cs.push_back((int)s0);
    }
  }
  cudaFree(c->chunk_tube);
  cudaFree(c->chunk_start);
  c->chunk_tube = nullptr;
  c->chunk_start = nullptr;
  int rc;
  if ((rc = dalloc(c, &c->chunk_tube, (int64_t)ct.size())) || (rc = dalloc(c, &c->chunk_start, (int64_t)cs.size())))
    return rc;
  CK(c, cudaMemcpy(c->chunk_tube, ct.data(), ct.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  CK(c, cudaMemcpy(c->chunk_start, cs.data(), cs.size() * sizeof(int), cudaMemcpyHostToDevice));
  c->nchunks = (int64_t)ct.size();
  c->tube_config = config;
  return WS_OK;
}
bool mixed(const ws_ctx* c) { return c->opts.precision == WS_PREC_MIXED; }

// one RHS evaluation of the stage state Us into the face arrays
int rhs_faces(ws_ctx* c, double* Us) {
  const GridDev& g = c->gd;
  {
    KScope k(c, WS_K_GHOST, g.ndim);
    for (int d = 0; d < g.ndim; ++d) launch_ghost(g, Us, d, c->stream);
  }
  {
    KScope k(c, WS_K_PRIM);
    if (mixed(c))
      launch_prim32(g, Us, c->Q32, c->stream);
    else
      launch_prim(g, Us, c->Q, c->stream);
  }
  return check_launch(c, "ghost/prim");
}

int faces(ws_ctx* c, int stage_slot) {
  const GridDev& g = c->gd;
  uint8_t* mbase = c->mask + (int64_t)stage_slot * c->nmask;
  for (int d = 0; d < g.ndim; ++d) {
    KScope k(c, WS_K_FACE);
    if (mixed(c))
      launch_face_mixed(g, d, c->Q32, c->Fh32[d], c->us32[d], mbase + c->mask_off[d], (float)c->opts.eps,
                        c->opts.mood, c->opts.weights, c->stream);
    else
      launch_face_fp64(g, d, c->Q, c->Fh[d], c->us[d], mbase + c->mask_off[d], c->opts.eps, c->opts.mood,
                       c->opts.weights, c->stream);
  }
  return check_launch(c, "face sweep");
}

int update(ws_ctx* c, int stage, const double* Un, const double* Us, double* Uout) {
  KScope k(c, WS_K_UPDATE);
  if (mixed(c))
    launch_update_mixed(c->gd, stage, Un, Us, Uout, c->Fh32, c->us32, c->Q32, c->dt_dev, c->nbad, c->stream);
  else
    launch_update(c->gd, stage, Un, Us, Uout, c->Fh, c->us, c->dt_dev, c->nbad, c->stream);
  return check_launch(c, "update");
}

// ---- batched tubes ----
int tube_rhs(ws_ctx* c, double* Us, int stage_slot, bool cfl) {
  {
    KScope k(c, WS_K_GHOST);
    launch_tubes_ghost(c->td, Us, c->stream);
  }
  {
    KScope k(c, WS_K_PRIM);
    launch_tubes_prim(c->td, Us, c->Q, c->stream);
  }
  if (cfl) {
    CK(c, cudaMemsetAsync(c->lmax, 0, sizeof(unsigned long long) * c->td.ntubes, c->stream));
    KScope k(c, WS_K_CFL);
    launch_tubes_cfl(c->td, c->Q, c->lmax, c->stream);
  }
  uint8_t* mbase = c->mask + (int64_t)stage_slot * c->nmask;
  KScope k(c, WS_K_FACE);
  launch_tubes_face_fp64(c->td, c->Q, c->Fh[0], c->us[0], mbase, c->opts.eps, c->opts.mood, c->opts.weights,
                         c->stream);
  return check_launch(c, "tube sweep");
}

// The three fused RK stages (the CFL reduction happens inside stage 0, dt is
// derived in stage 1).  run_if: the stages run only if *run_if != 0.
int fused_run3(ws_ctx* c, double* U, double dt, const GateArgs* gate, const int* run_if,
               unsigned long long* census = nullptr) {
  const GridDev& g = c->gd;
  // The plain stages may follow one another with programmatic dependent
  // launch, so one pair of profiling events spans all of a step's stage
  // launches (events between them would serialise the launches); the gated
  // and census steps time each stage on its own.
  const int per_stage = g.ndim == 3 ? 2 : 1;
  const bool one_scope = !gate && !run_if && !census;
  // plain steps take the chained slots (no memset before the step); the
  // others, and a step captured into a graph, use the context's own counters
  unsigned long long *lmax = c->lmax, *nbad = c->nbad, *clr0 = nullptr, *clr1 = nullptr;
  if (one_scope && !c->capturing && c->chain) {
    const int64_t n = c->chain_n++;
    lmax = c->chain + (n & 1);
    nbad = c->chain + 2 + (n & 1);
    clr0 = c->chain + ((n + 1) & 1);
    clr1 = c->chain + 2 + ((n + 1) & 1);
  } else {
    if (!run_if) CK(c, cudaMemsetAsync(c->lmax, 0, sizeof(unsigned long long), c->stream));
    if (one_scope) CK(c, cudaMemsetAsync(c->nbad, 0, sizeof(unsigned long long), c->stream));
  }
  c->nbad_last = nbad;
  std::optional<KScope> all;
  if (one_scope) all.emplace(c, WS_K_FACE, 3 * per_stage);
  // ws_set_resident: a plain 2D step on the state the previous step left
  // starts from that step's FP32 image (stage 0 then skips the FP64 loads)
  // and leaves the image of its own result in the other buffer
  float* u32 = c->Q32;
  bool img_in = false;
  float* img_out = nullptr;
  if (c->resident && one_scope) {
    if (c->img_cur >= 0 && c->img_U == U) {
      u32 = c->img[c->img_cur];
      img_in = true;
    }
    const int out = u32 == c->img[0] ? 1 : 0;
    img_out = c->img[out];
    c->img_cur = out;
    c->img_U = U;
  } else {
    c->img_cur = -1;
  }
  for (int s = 0; s < 3; ++s) {
    uint8_t* mb = c->mask + (int64_t)s * c->nmask;
    std::optional<KScope> k;
    if (!one_scope) k.emplace(c, WS_K_FACE, per_stage);
    const float* Kin = s == 1 ? c->Ka : c->Kb;
    float* Kout = s == 0 ? c->Ka : c->Kb;
    if (g.ndim == 3) {
      const CUtensorMap *tmk = map_of(c, Kin), *tmv = map_of(c, u32);
      if (!tmk || !tmv) tmk = tmv = nullptr;
      launch_stage3d(g, s, U, u32, Kin, Kout, c->Lp, dt, c->opts.cfl, lmax, c->dt_dev, mb + c->mask_off[0],
                     mb + c->mask_off[1], mb + c->mask_off[2], (float)c->opts.eps, c->opts.mood, c->opts.weights, nbad,
                     census, c->stage_tile, c->stage_sched == 0, s == 0 && img_in, s == 2 ? img_out : nullptr,
                     s == 2 ? clr0 : nullptr, s == 2 ? clr1 : nullptr, tmk, tmv, map2_of(c, tmk), map2_of(c, tmv),
                     c->stream);
    } else {
      const CUtensorMap *tmk = map_of(c, Kin), *tmv = map_of(c, u32);
      if (!tmk || !tmv) tmk = tmv = nullptr;
      launch_stage2d(g, s, U, u32, Kin, Kout, dt, c->opts.cfl, lmax, c->dt_dev, mb + c->mask_off[0],
                     mb + c->mask_off[1], (float)c->opts.eps, c->opts.mood, c->opts.weights, nbad, gate, run_if,
                     census, c->stage_tile, c->stage_sched == 0, s == 0 && img_in, s == 2 ? img_out : nullptr, tmk,
                     tmv, s == 2 ? clr0 : nullptr, s == 2 ? clr1 : nullptr, c->tail_rows, map2_of(c, tmk),
                     map2_of(c, tmv), c->stream);
    }
  }
  return check_launch(c, "fused stage");
}

GateArgs gate_args(ws_ctx* c) {
  return GateArgs{c->mlp_frag, c->mlp_bias, c->mlp_thr, -1, c->S1, c->lstat,
                  (c->gate_flags & WS_GATE_PER_STEP) ? c->gate_tile_flags : nullptr, c->gate_drift};
}

int step_device(ws_ctx* c, double* U, double dt) {
  const GridDev& g = c->gd;
  int rc;
  c->nbad_last = c->nbad;
  // a plain fused step clears (or rotates) its own counter
  if (!(c->fused && !c->learned_on)) CK(c, cudaMemsetAsync(c->nbad, 0, sizeof(unsigned long long), c->stream));
  if (tubes(c) && mixed(c)) {
    const int64_t nt = c->td.ntubes;
    CK(c, cudaMemsetAsync(c->lmax, 0, sizeof(unsigned long long) * nt, c->stream));
    CK(c, cudaMemsetAsync(c->counters, 0, 3 * sizeof(unsigned), c->stream));
    for (int s = 0; s < 3; ++s) {
      KScope k(c, WS_K_FACE);
      const float* Kin = s == 1 ? c->Ka : c->Kb;
      float* Kout = s == 0 ? c->Ka : c->Kb;
      launch_tubes_stage_mixed(c->td, c->tube_config, s, U, c->Q32, Kin, Kout, dt, c->opts.cfl, c->lmax, c->dt_dev,
                               c->chunk_tube, c->chunk_start, c->nchunks, c->counters + s,
                               c->mask + (int64_t)s * c->nmask, (float)c->opts.eps, c->opts.mood, c->opts.weights,
                               c->nbad, c->stream);
    }
    c->last_stages = 3;
    return check_launch(c, "mixed tube stage");
  }
  if (tubes(c)) {
    const int64_t nt = c->td.ntubes;
    for (int s = 0; s < 3; ++s) {
      double* Us = s == 0 ? U : c->S1;
      if ((rc = tube_rhs(c, Us, s, s == 0 && dt <= 0.0))) return rc;
      if (s == 0) {
        KScope k(c, WS_K_CFL);
        launch_set_dt(nullptr, dt, c->opts.cfl, c->lmax, c->dt_dev, nt, c->stream);
      }
      double* Uout = s == 2 ? U : c->S1;
      KScope k(c, WS_K_UPDATE);
      launch_tubes_update(c->td, s, U, Us, Uout, c->Fh[0], c->us[0], c->dt_dev, c->nbad, c->stream);
      if ((rc = check_launch(c, "tube update"))) return rc;
    }
    c->last_stages = 3;
    return WS_OK;
  }
  if (c->fused) {
    if (!c->learned_on) {
      if ((rc = fused_run3(c, U, dt, nullptr, nullptr))) return rc;
    } else {
      // gated step, then on the device: keep or redo it without the gate
      // (restored from the backup taken in stage 0), with no host round trip
      CK(c, cudaMemsetAsync(c->nbad, 0, sizeof(unsigned long long), c->stream));
      GateArgs ga = gate_args(c);
      CK(c, cudaMemsetAsync(c->lstat, 0, 8 * sizeof(float), c->stream));
      if ((rc = fused_run3(c, U, dt, &ga, nullptr))) return rc;
      {
        KScope k(c, WS_K_OTHER, 2);
        launch_gate_decide(c->lstat, c->nbad, c->lmax, c->gate_flags, c->gate_redo, c->gate_stats, c->gate_drift, 0,
                           c->stream);
        launch_restore(c->gate_redo, c->S1, U, c->nstate, c->stream);
      }
      if ((rc = fused_run3(c, U, dt, nullptr, c->gate_redo))) return rc;
    }
    c->last_stages = 3;
    return WS_OK;
  }
  for (int s = 0; s < 3; ++s) {
    double* Us = s == 0 ? U : c->S1;
    if ((rc = rhs_faces(c, Us))) return rc;
    if (s == 0) {
      if (dt <= 0.0) {
        CK(c, cudaMemsetAsync(c->lmax, 0, sizeof(unsigned long long), c->stream));
        KScope k(c, WS_K_CFL);
        if (mixed(c))
          launch_cfl32(g, c->Q32, c->lmax, c->stream);
        else
          launch_cfl(g, c->Q, c->lmax, c->stream);
      }
      KScope k(c, WS_K_CFL);
      launch_set_dt(nullptr, dt, c->opts.cfl, c->lmax, c->dt_dev, 1, c->stream);
    }
    if ((rc = faces(c, s))) return rc;
    double* Uout = s == 2 ? U : c->S1;
    if ((rc = update(c, s, U, Us, Uout))) return rc;
  }
  c->last_stages = 3;
  return WS_OK;
}

}  // namespace

extern "C" {

const char* ws_init_error(void) { return g_init_err; }

const char* ws_last_error(const ws_ctx* ctx) { return ctx ? ctx->err : g_init_err; }

int ws_init(const ws_grid* grid, const ws_opts* opts, void* stream, ws_ctx** out) {
  g_init_err[0] = 0;
  if (!grid || !opts || !out) return fail(nullptr, WS_EINVAL, "null argument");
  ws_grid gr = *grid;
  ws_opts op = *opts;
  bool tb = gr.ntubes > 0;
  if (gr.ndim < 1 || gr.ndim > 3) return fail(nullptr, WS_EINVAL, "ndim must be 1, 2 or 3 (got %d)", gr.ndim);
  if (tb && gr.ndim != 1) return fail(nullptr, WS_EINVAL, "batched tubes need ndim = 1");
  if (tb && !gr.tube_offsets) return fail(nullptr, WS_EINVAL, "tube_offsets is NULL");
  if (!tb) {
    for (int d = 0; d < gr.ndim; ++d) {
      if (gr.n[d] < 1) return fail(nullptr, WS_EINVAL, "n[%d] = %d < 1", d, gr.n[d]);
      if (!(gr.dx[d] > 0.0)) return fail(nullptr, WS_EINVAL, "dx[%d] must be > 0", d);
      for (int s = 0; s < 2; ++s)
        if (gr.bc[d][s] < 0 || gr.bc[d][s] > 2) return fail(nullptr, WS_EINVAL, "bad bc[%d][%d]", d, s);
      if ((gr.bc[d][0] == WS_BC_PERIODIC) != (gr.bc[d][1] == WS_BC_PERIODIC))
        return fail(nullptr, WS_EINVAL, "periodic bc must be set on both sides of direction %d", d);
      if (gr.n[d] < NG && (gr.bc[d][0] != WS_BC_TRANSMISSIVE || gr.bc[d][1] != WS_BC_TRANSMISSIVE))
        return fail(nullptr, WS_EINVAL, "n[%d] = %d < 3 needs transmissive ends", d, gr.n[d]);
    }
  }
  if (op.precision != WS_PREC_FP64 && op.precision != WS_PREC_MIXED)
    return fail(nullptr, WS_EINVAL, "bad precision %d", op.precision);
  if (op.weights != WS_W_MODIFIED && op.weights != WS_W_BASIC && op.weights != WS_W_JS)
    return fail(nullptr, WS_EINVAL, "bad weights %d", op.weights);
  if (op.mood != 0 && op.mood != 1) return fail(nullptr, WS_EINVAL, "mood must be 0 or 1");
  if (op.learned && op.precision != WS_PREC_MIXED)
    return fail(nullptr, WS_EINVAL, "the learned gate runs in mixed precision only");
  if (op.eps <= 0.0) op.eps = op.weights == WS_W_JS ? 1e-6 : (op.precision == WS_PREC_FP64 ? 1e-40 : 1e-10);
  if (op.cfl <= 0.0) op.cfl = 0.5;
  if (op.learned) return fail(nullptr, WS_ENOTSUP, "the learned face gate is not built in this library");

  ws_ctx* c = new (std::nothrow) ws_ctx();
  if (!c) return fail(nullptr, WS_ECUDA, "out of host memory");
  c->grid = gr;
  c->opts = op;
  c->stream = (cudaStream_t)stream;
  c->grid.tube_offsets = nullptr;
  cudaGetDevice(&c->dev);
  GridDev& g = c->gd;
  g.ndim = gr.ndim;
  g.nv = gr.ndim + 4;
  int rc = WS_OK;
  if (!tb) {
    for (int d = 0; d < 3; ++d) {
      bool act = d < gr.ndim;
      g.n[d] = act ? gr.n[d] : 1;
      g.G[d] = act ? NG : 0;
      g.P[d] = act ? (int64_t)gr.n[d] + 2 * NG : 1;
      g.dx[d] = act ? gr.dx[d] : 1.0;
      g.bc[d][0] = act ? gr.bc[d][0] : 0;
      g.bc[d][1] = act ? gr.bc[d][1] : 0;
    }
    g.st[0] = 1;
    g.st[1] = g.P[0];
    g.st[2] = g.P[0] * g.P[1];
    g.N = g.P[0] * g.P[1] * g.P[2];
    for (int d = 0; d < 3; ++d) g.st32[d] = g.st[d];
    g.N32 = g.N;
    g.ncell = (int64_t)g.n[0] * g.n[1] * g.n[2];
    int64_t off = 0;
    for (int d = 0; d < 3; ++d) {
      for (int e = 0; e < 3; ++e) g.fe[d][e] = g.n[e] + (e == d ? 1 : 0);
      g.nfaces[d] = d < gr.ndim ? g.fe[d][0] * g.fe[d][1] * g.fe[d][2] : 0;
      c->mask_off[d] = off;
      off += g.nfaces[d];
    }
    c->nmask = off;
    c->nstate = (int64_t)g.nv * g.N;
    if ((rc = dalloc(c, &c->S1, c->nstate)) || (rc = dalloc(c, &c->mask, 3 * c->nmask)) ||
        (rc = dalloc(c, &c->dt_dev, 1)) || (rc = dalloc(c, &c->lmax, 1)) || (rc = dalloc(c, &c->nbad, 1)))
      goto bad;
    if (op.precision == WS_PREC_MIXED) {
      const bool fused2d = gr.ndim == 2 && !getenv("WS_NO_FUSED");
      const bool fused3d = gr.ndim == 3 && !getenv("WS_NO_FUSED");
      if (fused2d || fused3d) {  // FP32 rows padded to a multiple of four floats (TMA boxes)
        g.st32[1] = (g.P[0] + 3) / 4 * 4;
        g.st32[2] = g.st32[1] * g.P[1];
        g.N32 = g.st32[2] * g.P[2];
      }
      if ((rc = dalloc(c, &c->Q32, std::max((int64_t)(g.nv + 1) * g.N, (int64_t)g.nv * g.N32)))) goto bad;
      if (fused2d) {
        if ((rc = dalloc(c, &c->Ka, (int64_t)g.nv * g.N32)) || (rc = dalloc(c, &c->Kb, (int64_t)g.nv * g.N32)) ||
            (rc = dalloc(c, &c->census, 4)))
          goto bad;
        if (fused2d_prepare() != cudaSuccess) {
          rc = fail(c, WS_ECUDA, "cannot enable %d bytes of shared memory for the fused stage", fused2d_smem_bytes());
          goto bad;
        }
        c->fused = true;
        c->stage_tile = 3;  // 32 x 15 tile rows closed by 32 x 7 rows
        set_tail_rows(c);
        encode_maps(c);
        c->stage_tma = c->tmap_ok == 0x7u ? 1 : 0;
      }
      if (fused3d) {
        if ((rc = dalloc(c, &c->Ka, (int64_t)g.nv * g.N32)) || (rc = dalloc(c, &c->Kb, (int64_t)g.nv * g.N32)) ||
            (rc = dalloc(c, &c->Lp, (int64_t)g.nv * g.N32)) || (rc = dalloc(c, &c->census, 4)))
          goto bad;
        if (fused3d_prepare() != cudaSuccess) {
          rc = fail(c, WS_ECUDA, "cannot enable %d bytes of shared memory for the fused stage", fused3d_smem_bytes());
          goto bad;
        }
        c->fused = true;
        c->stage_sched = 1;  // the 3D passes measured faster with plain launches
        encode_maps(c);
        c->stage_tma = c->tmap_ok == 0x7u ? 1 : 0;
      }
      if (c->fused) {  // slots of consecutive plain steps, cleared once here
        if ((rc = dalloc(c, &c->chain, 4))) goto bad;
        if (cudaMemset(c->chain, 0, 4 * sizeof(unsigned long long)) != cudaSuccess) {
          rc = fail(c, WS_ECUDA, "cannot clear the step counters");
          goto bad;
        }
      }
      for (int d = 0; d < gr.ndim; ++d)
        if ((rc = dalloc(c, &c->Fh32[d], (int64_t)g.nv * g.nfaces[d])) ||
            (rc = dalloc(c, &c->us32[d], g.nfaces[d])))
          goto bad;
    } else {
      if ((rc = dalloc(c, &c->Q, (int64_t)(g.nv + 1) * g.N))) goto bad;
      for (int d = 0; d < gr.ndim; ++d)
        if ((rc = dalloc(c, &c->Fh[d], (int64_t)g.nv * g.nfaces[d])) || (rc = dalloc(c, &c->us[d], g.nfaces[d])))
          goto bad;
    }
  } else {
    int64_t nt = gr.ntubes;
    std::vector<int64_t> off(grid->tube_offsets, grid->tube_offsets + nt + 1);
    if (off[0] != 0) {
      rc = fail(c, WS_EINVAL, "tube_offsets[0] must be 0");
      goto bad;
    }
    int64_t nface = 0;
    for (int64_t t = 0; t < nt; ++t) {
      int64_t len = off[t + 1] - off[t] - 2 * NG;
      if (len < 2 * NG) {
        rc = fail(c, WS_EINVAL, "tube %lld has %lld interior cells (< 6)", (long long)t, (long long)len);
        goto bad;
      }
      nface += len + 1;
    }
    int64_t total = off[nt];
    std::vector<int> ct(total);
    for (int64_t t = 0; t < nt; ++t)
      for (int64_t i = off[t]; i < off[t + 1]; ++i) ct[i] = (int)t;
    g.n[0] = 1;  // unused in tube mode
    g.n[1] = g.n[2] = 1;
    g.N = total;
    g.N32 = total;
    g.st32[0] = 1;
    g.st32[1] = g.st32[2] = total;
    g.nv = 5;
    c->nstate = 5 * total;
    c->nmask = total;  // one byte per padded cell: face i+1/2 stored at cell i (faces -1/2 .. len-1/2)
    c->mask_off[0] = 0;
    c->td.ntubes = nt;
    c->td.total = total;
    (void)nface;
    if ((rc = dalloc(c, &c->S1, c->nstate)) || (rc = dalloc(c, &c->Q, 6 * total)) ||
        (rc = dalloc(c, &c->mask, 3 * c->nmask)) || (rc = dalloc(c, &c->dt_dev, nt)) ||
        (rc = dalloc(c, &c->lmax, nt)) || (rc = dalloc(c, &c->nbad, 1)) || (rc = dalloc(c, &c->Fh[0], 5 * total)) ||
        (rc = dalloc(c, &c->us[0], total)) || (rc = dalloc(c, &c->off_dev, nt + 1)) ||
        (rc = dalloc(c, &c->cell_tube, total)))
      goto bad;
    if (cudaMemcpy(c->off_dev, off.data(), sizeof(int64_t) * (nt + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->cell_tube, ct.data(), sizeof(int) * total, cudaMemcpyHostToDevice) != cudaSuccess) {
      rc = fail(c, WS_ECUDA, "copying tube offsets failed");
      goto bad;
    }
    c->td.off = c->off_dev;
    c->td.cell_tube = c->cell_tube;
    c->off_host = off;
    if (op.precision == WS_PREC_MIXED) {
      if ((rc = dalloc(c, &c->Q32, 5 * total)) || (rc = dalloc(c, &c->Ka, 5 * total)) ||
          (rc = dalloc(c, &c->Kb, 5 * total)) || (rc = dalloc(c, &c->counters, 3)) || (rc = build_chunks(c, 2)))
        goto bad;
    }
  }
  if ((rc = dalloc(c, &c->mood_counts, 9)) || (rc = dalloc(c, &c->mask_off_dev, 3))) goto bad;
  if (cudaMemcpy(c->mask_off_dev, c->mask_off, 3 * sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess) {
    rc = fail(c, WS_ECUDA, "copying mask offsets failed");
    goto bad;
  }
  // tube masks hold one byte per padded cell; the bytes that carry no face stay 0xff
  if (cudaMemset(c->mask, tb ? 0xff : 0, 3 * c->nmask) != cudaSuccess) {
    rc = fail(c, WS_ECUDA, "cudaMemset failed");
    goto bad;
  }
  *out = c;
  return WS_OK;
bad:
  snprintf(g_init_err, sizeof g_init_err, "%s", c->err);
  free_all(c);
  delete c;
  return rc;
}

int64_t ws_state_size(const ws_ctx* ctx) { return ctx ? ctx->nstate : -1; }

int64_t ws_mask_size(const ws_ctx* ctx) { return ctx ? ctx->nmask : -1; }

int ws_prim_to_cons(ws_ctx* c, const double* Q, double* U) {
  if (!c || !Q || !U || Q == U) return fail(c, WS_EINVAL, "bad pointers");
  c->img_cur = -1;  // the carried FP32 image no longer follows U
  GridDev g = c->gd;
  if (tubes(c)) {
    g.ndim = 1;
    g.n[0] = (int)1;
  }
  launch_prim_to_cons(g, Q, U, c->stream);
  return check_launch(c, "prim_to_cons");
}

int ws_cons_to_prim(ws_ctx* c, const double* U, double* Q) {
  if (!c || !Q || !U || Q == U) return fail(c, WS_EINVAL, "bad pointers");
  launch_cons_to_prim_all(c->gd, U, Q, c->stream);
  return check_launch(c, "cons_to_prim");
}

int ws_flux_divergence(ws_ctx* c, double* U, double* L) {
  if (!c || !U || !L || U == L) return fail(c, WS_EINVAL, "bad pointers");
  c->img_cur = -1;  // the carried FP32 image no longer follows U
  if (tubes(c)) return fail(c, WS_ENOTSUP, "ws_flux_divergence is not available for batched tubes");
  int rc;
  if ((rc = rhs_faces(c, U)) || (rc = faces(c, 0)) || (rc = update(c, -1, U, U, L))) return rc;
  c->last_stages = 1;
  return WS_OK;
}

int ws_cfl_dt(ws_ctx* c, double* U, double* dt) {
  if (!c || !U || !dt) return fail(c, WS_EINVAL, "bad pointers");
  int64_t n = tubes(c) ? c->td.ntubes : 1;
  if (tubes(c)) {
    launch_tubes_ghost(c->td, U, c->stream);
    launch_tubes_prim(c->td, U, c->Q, c->stream);
    CK(c, cudaMemsetAsync(c->lmax, 0, sizeof(unsigned long long) * n, c->stream));
    launch_tubes_cfl(c->td, c->Q, c->lmax, c->stream);
  } else {
    int rc = rhs_faces(c, U);
    if (rc) return rc;
    CK(c, cudaMemsetAsync(c->lmax, 0, sizeof(unsigned long long), c->stream));
    if (mixed(c))
      launch_cfl32(c->gd, c->Q32, c->lmax, c->stream);
    else
      launch_cfl(c->gd, c->Q, c->lmax, c->stream);
  }
  launch_set_dt(nullptr, 0.0, c->opts.cfl, c->lmax, c->dt_dev, n, c->stream);
  int rc = check_launch(c, "cfl");
  if (rc) return rc;
  std::vector<double> h(n);
  CK(c, cudaMemcpyAsync(h.data(), c->dt_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  double m = h[0];
  for (int64_t i = 1; i < n; ++i) m = h[i] < m ? h[i] : m;
  *dt = m;
  return WS_OK;
}

// one CFL step replayed from a CUDA graph (captured on first use per U)
int step_graph(ws_ctx* c, double* U) {
  if (!c->graph_exec || c->graph_U != U) {
    if (c->graph_exec) {
      CK(c, cudaGraphExecDestroy(c->graph_exec));
      c->graph_exec = nullptr;
    }
    CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    c->capturing = true;
    int rc = step_device(c, U, 0.0);
    c->capturing = false;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return fail(c, WS_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      c->graph_exec = nullptr;
      return fail(c, WS_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
    c->graph_U = U;
  }
  CK(c, cudaGraphLaunch(c->graph_exec, c->stream));
  c->last_stages = 3;
  return WS_OK;
}

// The gated step as one graph: the gated stages and the decision kernel, then
// an IF node whose body (restore U from the stage-0 backup, the three plain
// stages) runs only when the decision kernel sets its condition.  Rebuilt when
// U, dt or the gate change.
int gated_step_graph(ws_ctx* c, double* U, double dt) {
  if (!c->ggraph_exec || c->ggraph_U != U || c->ggraph_dt != dt) {
    if (c->ggraph_exec) {
      CK(c, cudaGraphExecDestroy(c->ggraph_exec));
      c->ggraph_exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    CK(c, cudaGraphCreate(&g, 0));
    struct GraphGuard {
      cudaGraph_t g;
      ~GraphGuard() {
        if (g) cudaGraphDestroy(g);
      }
    } guard{g};
    cudaGraphConditionalHandle cond;
    CK(c, cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault));
    // main part: the gated stages and the decision
    CK(c, cudaStreamBeginCaptureToGraph(c->stream, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    int rc = WS_OK;
    {
      cudaError_t e1 = cudaMemsetAsync(c->nbad, 0, sizeof(unsigned long long), c->stream);
      cudaError_t e2 = cudaMemsetAsync(c->lstat, 0, 8 * sizeof(float), c->stream);
      GateArgs ga = gate_args(c);
      if (e1 != cudaSuccess || e2 != cudaSuccess) rc = fail(c, WS_ECUDA, "memset in capture failed");
      if (!rc) rc = fused_run3(c, U, dt, &ga, nullptr);
      if (!rc) {
        launch_gate_decide(c->lstat, c->nbad, c->lmax, c->gate_flags, c->gate_redo, c->gate_stats, c->gate_drift,
                           cond, c->stream);
        rc = check_launch(c, "gate decision");
      }
    }
    cudaGraph_t cap = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->stream, &cap);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(c, WS_ECUDA, "capture of the gated step failed: %s", cudaGetErrorString(e));
    // the decision kernel is the one node without dependents
    size_t nn = 0;
    CK(c, cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    CK(c, cudaGraphGetNodes(g, nodes.data(), &nn));
    cudaGraphNode_t leaf = nullptr;
    int nleaf = 0;
    for (size_t i = 0; i < nn; ++i) {
      size_t nd = 0;
      CK(c, cudaGraphNodeGetDependentNodes(nodes[i], nullptr, nullptr, &nd));
      if (nd == 0) {
        leaf = nodes[i];
        ++nleaf;
      }
    }
    if (nleaf != 1) return fail(c, WS_ECUDA, "gated step graph: %d leaf nodes", nleaf);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    CK(c, cudaGraphAddNode(&cnode, g, &leaf, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    // redo branch
    CK(c, cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    launch_restore(c->gate_redo, c->S1, U, c->nstate, c->stream);
    rc = check_launch(c, "restore");
    if (!rc) rc = fused_run3(c, U, dt, nullptr, nullptr);
    e = cudaStreamEndCapture(c->stream, &cap);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(c, WS_ECUDA, "capture of the redo branch failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->ggraph_exec, g, 0);
    if (e != cudaSuccess) {
      c->ggraph_exec = nullptr;
      return fail(c, WS_ECUDA, "gated step graph instantiation failed: %s", cudaGetErrorString(e));
    }
    c->ggraph_U = U;
    c->ggraph_dt = dt;
  }
  CK(c, cudaGraphLaunch(c->ggraph_exec, c->stream));
  c->last_stages = 3;
  return WS_OK;
}

int ws_step(ws_ctx* c, double* U, double dt, double* dt_used) {
  if (!c || !U) return fail(c, WS_EINVAL, "bad pointers");
  c->nbad_last = c->nbad;
  // a captured step would replay one fixed pair of image buffers, so resident
  // steps are launched directly
  bool graph = c->graph_on && dt <= 0.0 && c->stream != nullptr && !c->prof_on && !c->learned_on && !c->resident;
  bool ggraph = c->learned_on && c->fused && c->stream != nullptr && !c->prof_on;
  int rc = ggraph ? gated_step_graph(c, U, dt) : graph ? step_graph(c, U) : step_device(c, U, dt);
  if (rc) return rc;
  if (dt_used) {
    int64_t n = tubes(c) ? c->td.ntubes : 1;
    CK(c, cudaMemcpyAsync(dt_used, c->dt_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
  }
  if (c->opts.check) {
    unsigned long long nb = 0;
    CK(c, cudaMemcpyAsync(&nb, c->nbad_last ? c->nbad_last : c->nbad, sizeof nb, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (nb) return fail(c, WS_ENONPHYS, "%llu inadmissible cells after the step", nb);
  }
  return WS_OK;
}

int ws_census_step(ws_ctx* c, double* U, double dt, double* dt_used, int64_t counts[4]) {
  if (!c || !U || !counts) return fail(c, WS_EINVAL, "bad pointers");
  c->img_cur = -1;  // the carried FP32 image no longer follows U
  if (!c->fused) return fail(c, WS_EINVAL, "the census needs a fused mixed-precision 2D or 3D context");
  CK(c, cudaMemsetAsync(c->census, 0, 4 * sizeof(unsigned long long), c->stream));
  CK(c, cudaMemsetAsync(c->nbad, 0, sizeof(unsigned long long), c->stream));
  int rc = fused_run3(c, U, dt, nullptr, nullptr, c->census);
  if (rc) return rc;
  c->last_stages = 3;
  unsigned long long h[4];
  CK(c, cudaMemcpyAsync(h, c->census, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  if (dt_used) CK(c, cudaMemcpyAsync(dt_used, c->dt_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  for (int k = 0; k < 4; ++k) counts[k] = (int64_t)h[k];
  if (c->opts.check) {
    unsigned long long nb = 0;
    CK(c, cudaMemcpyAsync(&nb, c->nbad, sizeof nb, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (nb) return fail(c, WS_ENONPHYS, "%llu inadmissible cells after the step", nb);
  }
  return WS_OK;
}

// ws_run_host on the fused 2D path: the state comes in by bands of tile rows
// and stage 0 of the first step starts on each band as soon as it and the
// 3-row halo below it have arrived; stage 1 needs the CFL step of the whole
// grid and runs once all of stage 0 is done; stage 2 of the last step runs by
// bands again and each finished band goes back to the host while the next one
// computes.  The kernels and their arithmetic are those of ws_step.
int run_host_banded(ws_ctx* c, double* U_host, int nsteps, double dt, double* dt_used) {
  const GridDev& g = c->gd;
  const int TYv = fused2d_tile_height(c->stage_tile);
  const int nrt = (g.n[1] + TYv - 1) / TYv;
  const int B = nrt < 8 ? nrt : 8;
  if (!c->cp_in) {
    CK(c, cudaStreamCreateWithFlags(&c->cp_in, cudaStreamNonBlocking));
    CK(c, cudaStreamCreateWithFlags(&c->cp_out, cudaStreamNonBlocking));
  }
  while ((int)c->band_ev.size() < 2 * B + 2) {
    cudaEvent_t e;
    CK(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    c->band_ev.push_back(e);
  }
  cudaEvent_t* ev_in = c->band_ev.data();
  cudaEvent_t* ev_s2 = ev_in + B;
  cudaEvent_t ev_start = ev_in[2 * B], ev_out = ev_in[2 * B + 1];
  const int64_t P0 = g.P[0], P1 = g.P[1];
  const size_t pitch = sizeof(double) * (size_t)g.N;  // between fields
  // band k: tile rows [r0, r1) and the padded rows it carries (the first and
  // last bands also carry the ghost rows)
  auto tiles = [&](int k, int& r0, int& r1) {
    r0 = (int)((int64_t)k * nrt / B);
    r1 = (int)((int64_t)(k + 1) * nrt / B);
  };
  auto rows = [&](int k, int64_t& p0, int64_t& p1) {
    int r0, r1;
    tiles(k, r0, r1);
    p0 = k == 0 ? 0 : NG + (int64_t)r0 * TYv;
    p1 = k == B - 1 ? P1 : NG + (int64_t)r1 * TYv;
  };
  auto copy_band = [&](int k, bool in, cudaStream_t st) -> cudaError_t {
    int64_t p0, p1;
    rows(k, p0, p1);
    size_t width = sizeof(double) * (size_t)((p1 - p0) * P0);
    double* d = c->Uhost_dev + p0 * P0;
    double* h = U_host + p0 * P0;
    return in ? cudaMemcpy2DAsync(d, pitch, h, pitch, width, g.nv, cudaMemcpyHostToDevice, st)
              : cudaMemcpy2DAsync(h, pitch, d, pitch, width, g.nv, cudaMemcpyDeviceToHost, st);
  };
  auto stage = [&](int st, int r0, int nr) {
    uint8_t* mb = c->mask + (int64_t)st * c->nmask;
    const float* Kin = st == 1 ? c->Ka : c->Kb;
    float* Kout = st == 0 ? c->Ka : c->Kb;
    const CUtensorMap *tmk = map_of(c, Kin), *tmv = map_of(c, c->Q32);
    if (!tmk || !tmv) tmk = tmv = nullptr;
    launch_stage2d_band(g, st, c->Uhost_dev, c->Q32, Kin, Kout, dt, c->opts.cfl, c->lmax, c->dt_dev,
                        mb + c->mask_off[0], mb + c->mask_off[1], (float)c->opts.eps, c->opts.mood, c->opts.weights,
                        c->nbad, r0, nr, c->stage_tile, tmk, tmv, c->stream);
  };
  // the copy streams start after the work already queued on the context's stream
  CK(c, cudaEventRecord(ev_start, c->stream));
  CK(c, cudaStreamWaitEvent(c->cp_in, ev_start, 0));
  for (int k = 0; k < B; ++k) {
    CK(c, copy_band(k, true, c->cp_in));
    CK(c, cudaEventRecord(ev_in[k], c->cp_in));
  }
  for (int n = 0; n < nsteps; ++n) {
    CK(c, cudaMemsetAsync(c->nbad, 0, sizeof(unsigned long long), c->stream));
    CK(c, cudaMemsetAsync(c->lmax, 0, sizeof(unsigned long long), c->stream));
    // stage 0: band k needs its rows and the halo rows of band k + 1 (all
    // bands when y is periodic: the first band's halo wraps to the last rows)
    const bool wrap = g.bc[1][0] == WS_BC_PERIODIC || g.bc[1][1] == WS_BC_PERIODIC;
    for (int k = 0; k < B; ++k) {
      int r0, r1;
      tiles(k, r0, r1);
      if (n == 0) CK(c, cudaStreamWaitEvent(c->stream, ev_in[wrap || k + 1 >= B ? B - 1 : k + 1], 0));
      if (n > 0 && k > 0) continue;
      stage(0, n == 0 ? r0 : 0, n == 0 ? r1 - r0 : nrt);
    }
    stage(1, 0, nrt);
    if (n + 1 < nsteps) {
      stage(2, 0, nrt);
      continue;
    }
    CK(c, cudaStreamWaitEvent(c->cp_out, ev_start, 0));
    for (int k = 0; k < B; ++k) {  // stage 2 of the last step, each band copied out when done
      int r0, r1;
      tiles(k, r0, r1);
      stage(2, r0, r1 - r0);
      CK(c, cudaEventRecord(ev_s2[k], c->stream));
      CK(c, cudaStreamWaitEvent(c->cp_out, ev_s2[k], 0));
      CK(c, copy_band(k, false, c->cp_out));
    }
  }
  if (nsteps == 0) {  // nothing computed: the state goes straight back
    CK(c, cudaStreamWaitEvent(c->cp_out, ev_in[B - 1], 0));
    for (int k = 0; k < B; ++k) CK(c, copy_band(k, false, c->cp_out));
  }
  int rc = check_launch(c, "banded stage");
  if (rc) return rc;
  CK(c, cudaEventRecord(ev_out, c->cp_out));
  CK(c, cudaStreamWaitEvent(c->stream, ev_out, 0));
  if (dt_used) CK(c, cudaMemcpyAsync(dt_used, c->dt_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->last_stages = 3;
  return WS_OK;
}

int ws_run_host(ws_ctx* c, double* U_host, int nsteps, double dt, double* dt_used) {
  if (!c || !U_host || nsteps < 0) return fail(c, WS_EINVAL, "bad arguments");
  c->img_cur = -1;  // the carried FP32 image no longer follows U
  c->nbad_last = c->nbad;
  if (!c->Uhost_dev) {
    int rc = dalloc(c, &c->Uhost_dev, c->nstate);
    if (rc) return rc;
  }
  if (c->fused && c->gd.ndim == 2 && !c->learned_on && !c->prof_on)
    return run_host_banded(c, U_host, nsteps, dt, dt_used);
  size_t bytes = sizeof(double) * (size_t)c->nstate;
  CK(c, cudaMemcpyAsync(c->Uhost_dev, U_host, bytes, cudaMemcpyHostToDevice, c->stream));
  for (int k = 0; k < nsteps; ++k) {
    int rc = step_device(c, c->Uhost_dev, dt);
    if (rc) return rc;
  }
  CK(c, cudaMemcpyAsync(U_host, c->Uhost_dev, bytes, cudaMemcpyDeviceToHost, c->stream));
  if (dt_used) {
    int64_t n = tubes(c) ? c->td.ntubes : 1;
    CK(c, cudaMemcpyAsync(dt_used, c->dt_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  }
  CK(c, cudaStreamSynchronize(c->stream));
  return WS_OK;
}

int ws_get_mood(ws_ctx* c, uint8_t* mask, int64_t counts[9]) {
  if (!c) return fail(c, WS_EINVAL, "null context");
  if (mask) CK(c, cudaMemcpyAsync(mask, c->mask, 3 * c->nmask, cudaMemcpyDeviceToDevice, c->stream));
  if (counts) {
    int ndim = tubes(c) ? 1 : c->gd.ndim;
    CK(c, cudaMemsetAsync(c->mood_counts, 0, 9 * sizeof(unsigned long long), c->stream));
    if (c->last_stages > 0)
      launch_mood_count(c->mask, c->nmask, c->last_stages, c->mask_off_dev, ndim, c->mood_counts, c->stream);
    unsigned long long h[9];
    CK(c, cudaMemcpyAsync(h, c->mood_counts, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    for (int i = 0; i < 9; ++i) counts[i] = (int64_t)h[i];
  }
  return check_launch(c, "mood count");
}

int ws_nonphysical(ws_ctx* c, int64_t* count) {
  if (!c || !count) return fail(c, WS_EINVAL, "bad pointers");
  unsigned long long nb = 0;
  CK(c, cudaMemcpyAsync(&nb, c->nbad_last ? c->nbad_last : c->nbad, sizeof nb, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  *count = (int64_t)nb;
  return WS_OK;
}

int ws_face_samples(ws_ctx* c, double* U, int64_t stride, int64_t max_out, float* feats, uint8_t* labels,
                    int64_t* count) {
  if (!c || !U || !count || stride < 1 || max_out < 0 || (max_out > 0 && (!feats || !labels)))
    return fail(c, WS_EINVAL, "bad arguments");
  c->img_cur = -1;  // the carried FP32 image no longer follows U
  if (tubes(c) || !mixed(c)) return fail(c, WS_ENOTSUP, "face samples need a mixed-precision grid context");
  const GridDev& g = c->gd;
  for (int d = 0; d < g.ndim; ++d) launch_ghost(g, U, d, c->stream);
  launch_prim32(g, U, c->Q32, c->stream);
  int64_t out = 0;
  for (int d = 0; d < g.ndim && out < max_out; ++d) {
    launch_face_samples(g, d, c->Q32, stride, out, max_out, feats, labels, (float)c->opts.eps, c->opts.weights,
                        c->stream);
    out += (g.nfaces[d] + stride - 1) / stride;
  }
  *count = out < max_out ? out : max_out;
  int rc = check_launch(c, "face samples");
  if (rc) return rc;
  CK(c, cudaStreamSynchronize(c->stream));
  return WS_OK;
}

// BF16 m16n8k16 B fragments of the gate MLP: for k-step ks and n-tile nt, lane
// (g = lane/4, t = lane%4) holds B[16ks+2t .. +1][8nt+g] and B[16ks+2t+8 .. +9][8nt+g]
// with B[k][n] = W[n][k]; entries outside W are zero
static uint32_t bf16_bits(float v) {
  uint32_t u;
  memcpy(&u, &v, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0u;
  u += 0x7fffu + ((u >> 16) & 1u);  // round to nearest even
  return u >> 16;
}

static void build_frags(const float* W, int nout, int nin, int ksteps, int ntiles, uint32_t* out /* [ks][nt][32][2] */) {
  for (int ks = 0; ks < ksteps; ++ks)
    for (int nt = 0; nt < ntiles; ++nt)
      for (int lane = 0; lane < 32; ++lane) {
        int g = lane >> 2, t = lane & 3, n = nt * 8 + g;
        auto B = [&](int k) -> float { return (n < nout && k < nin) ? W[n * nin + k] : 0.0f; };
        int k0 = ks * 16 + 2 * t;
        uint32_t lo = bf16_bits(B(k0)) | (bf16_bits(B(k0 + 1)) << 16);
        uint32_t hi = bf16_bits(B(k0 + 8)) | (bf16_bits(B(k0 + 9)) << 16);
        uint32_t* o = out + (((size_t)(ks * ntiles + nt) * 32 + lane) * 2);
        o[0] = lo;
        o[1] = hi;
      }
}

int ws_set_mlp(ws_ctx* c, const float* params, float threshold, int flags) {
  if (!c) return fail(c, WS_EINVAL, "null context");
  c->img_cur = -1;  // the carried FP32 image no longer follows U
  if (!params) {
    c->learned_on = false;
    if (c->ggraph_exec) {
      cudaGraphExecDestroy(c->ggraph_exec);
      c->ggraph_exec = nullptr;
    }
    return WS_OK;
  }
  if (!c->fused || c->gd.ndim != 2)
    return fail(c, WS_ENOTSUP, "the learned gate runs in the fused 2D mixed-precision path only");
  std::vector<float> P(WS_MLP_NPARAM);
  CK(c, cudaMemcpy(P.data(), params, sizeof(float) * WS_MLP_NPARAM, cudaMemcpyDeviceToHost));
  const float* W1 = P.data();
  const float* b1 = W1 + 32 * 24;
  const float* W2 = b1 + 32;
  const float* b2 = W2 + 32 * 32;
  const float* W3 = b2 + 32;
  const float* b3 = W3 + 32;
  std::vector<uint32_t> F(18 * 32 * 2);
  build_frags(W1, 32, 24, 2, 4, F.data());
  build_frags(W2, 32, 32, 2, 4, F.data() + 8 * 64);
  build_frags(W3, 1, 32, 2, 1, F.data() + 16 * 64);
  std::vector<float> B(65);
  for (int i = 0; i < 32; ++i) {
    B[i] = b1[i];
    B[32 + i] = b2[i];
  }
  B[64] = b3[0];
  int rc;
  if (!c->mlp_frag) {
    if ((rc = dalloc(c, &c->mlp_frag, 18 * 32)) || (rc = dalloc(c, &c->mlp_bias, 65)) ||
        (rc = dalloc(c, &c->lstat, 8)) || (rc = dalloc(c, &c->gate_redo, 1)) || (rc = dalloc(c, &c->gate_stats, 6)))
      return rc;
  }
  if ((flags & WS_GATE_PER_STEP) && !c->gate_tile_flags &&
      (rc = dalloc(c, &c->gate_tile_flags, fused2d_gate_flag_bytes(c->gd))))
    return rc;
  CK(c, cudaMemset(c->gate_stats, 0, 6 * sizeof(double)));
  CK(c, cudaMemcpy(c->mlp_frag, F.data(), F.size() * 4, cudaMemcpyHostToDevice));
  CK(c, cudaMemcpy(c->mlp_bias, B.data(), 65 * sizeof(float), cudaMemcpyHostToDevice));
  c->mlp_thr = threshold;
  c->gate_flags = flags;
  c->learned_on = true;
  if (!c->gate_drift && (rc = dalloc(c, &c->gate_drift, 1))) return rc;
  CK(c, cudaMemset(c->gate_drift, 0, sizeof(int)));
  if (c->ggraph_exec) {  // parameters baked into the gated step graph changed
    CK(c, cudaGraphExecDestroy(c->ggraph_exec));
    c->ggraph_exec = nullptr;
  }
  return WS_OK;
}

int ws_gate_eval(ws_ctx* c, double* U, uint8_t* smooth) {
  if (!c || !U || !smooth) return fail(c, WS_EINVAL, "bad pointers");
  if (!c->learned_on) return fail(c, WS_EINVAL, "no gate set (ws_set_mlp)");
  GateArgs ga{c->mlp_frag, c->mlp_bias, c->mlp_thr, -1, c->S1, c->lstat, nullptr, nullptr};
  CK(c, cudaMemsetAsync(smooth, 0, (size_t)c->nmask, c->stream));
  c->img_cur = -1;
  launch_stage2d(c->gd, 3, U, c->Q32, c->Ka, c->Kb, 0.0, c->opts.cfl, c->lmax, c->dt_dev, smooth,
                 smooth + c->mask_off[1], (float)c->opts.eps, c->opts.mood, c->opts.weights, c->nbad, &ga, nullptr,
                 nullptr, 0, false, false, nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr,
                 c->stream);
  return check_launch(c, "gate eval");
}

int ws_gate_stats(ws_ctx* c, double out[6]) {
  if (!c || !out) return fail(c, WS_EINVAL, "bad pointers");
  for (int i = 0; i < 6; ++i) out[i] = 0.0;
  if (!c->gate_stats) return WS_OK;
  CK(c, cudaMemcpyAsync(out, c->gate_stats, 6 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return WS_OK;
}

// Fused stage configurations: index = 2 x tile slot + schedule (0 stage
// launches with programmatic dependent launch, 1 plain stage launches).
// Stage configurations: index = (2 x tile + loads) x 2 + schedule (loads: 0
// cell by cell, 1 TMA boxes for interior tiles -- in 3D, of both passes).
static int stage_load_modes(const ws_ctx*) { return 2; }

static bool stage_config_valid(const ws_ctx* c, int index) {
  return index >= 0 && index < 2 * stage_load_modes(c) * fused_num_tiles(c->gd.ndim);
}

static void set_stage_config(ws_ctx* c, int index) {
  c->img_cur = -1;
  const int nl = stage_load_modes(c);
  c->stage_tile = fused_tile_index(c->gd.ndim, index / (2 * nl));
  c->stage_tma = nl == 2 ? (index / 2) % 2 : 0;
  c->stage_sched = index % 2;
  if (c->gd.ndim == 2 && c->stage_tile == 3) set_tail_rows(c);
  encode_maps(c);
  if (c->stage_tma && (c->tmap_ok & 0x7u) != 0x7u) c->stage_tma = 0;  // the driver refused a descriptor
  if (c->graph_exec) {
    cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
  }
}

static int stage_config_index(const ws_ctx* c) {
  int k = 0;
  for (int j = 0; j < fused_num_tiles(c->gd.ndim); ++j)
    if (fused_tile_index(c->gd.ndim, j) == c->stage_tile) k = j;
  const int nl = stage_load_modes(c);
  return (nl * k + (nl == 2 ? c->stage_tma : 0)) * 2 + c->stage_sched;
}

// The fused 2D/3D stages: every configuration steps a scratch copy of U for
// `steps` CFL steps after one warm-up step, in two rounds over all the
// configurations (a configuration's time is its faster round, which keeps a
// passing disturbance from deciding); the fastest is kept.
static int autotune_fused(ws_ctx* c, const double* U, int steps, int* choice) {
  double* Ut = nullptr;
  int rc = dalloc(c, &Ut, c->nstate);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int bestk = -1;
  const int keep = stage_config_index(c);
  const bool prof = c->prof_on;
  c->prof_on = false;
  int ncand = 0;
  while (stage_config_valid(c, ncand)) ++ncand;
  std::vector<float> tk((size_t)ncand, 1e30f);
  for (int round = 0; round < 2 && rc == WS_OK; ++round) {
    for (int k = 0; k < ncand && rc == WS_OK; ++k) {
      set_stage_config(c, k);
      cudaMemcpyAsync(Ut, U, sizeof(double) * c->nstate, cudaMemcpyDeviceToDevice, c->stream);
      if ((rc = step_device(c, Ut, 0.0))) break;  // warm-up
      cudaEventRecord(e0, c->stream);
      for (int s = 0; s < steps && rc == WS_OK; ++s) rc = step_device(c, Ut, 0.0);
      cudaEventRecord(e1, c->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = fail(c, WS_ECUDA, "autotune step failed");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rc == WS_OK) tk[(size_t)k] = std::min(tk[(size_t)k], ms);
    }
  }
  for (int k = 0; k < ncand && rc == WS_OK; ++k)
    if (tk[(size_t)k] < best) {
      best = tk[(size_t)k];
      bestk = k;
    }
  c->prof_on = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(Ut);
  if (rc || bestk < 0) {
    set_stage_config(c, keep);
    return rc ? rc : fail(c, WS_ECUDA, "autotune found no configuration");
  }
  set_stage_config(c, bestk);
  if (choice) *choice = bestk;
  return WS_OK;
}

int ws_autotune(ws_ctx* c, const double* U, int steps, int* choice) {
  if (!c || !U || steps < 1) return fail(c, WS_EINVAL, "bad arguments");
  c->img_cur = -1;  // the carried FP32 image no longer follows U
  if (c->fused && !c->learned_on) return autotune_fused(c, U, steps, choice);
  if (!(tubes(c) && mixed(c))) {
    if (choice) *choice = -1;
    return WS_OK;  // nothing to tune
  }
  // time each configuration on a scratch copy of U
  double* Ut = nullptr;
  int rc = dalloc(c, &Ut, c->nstate);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int bestc = c->tube_config;
  bool prof = c->prof_on;
  c->prof_on = false;
  for (int cfg = 0; cfg < kNumTubeConfigs && rc == WS_OK; ++cfg) {
    if ((rc = build_chunks(c, cfg))) break;
    cudaMemcpyAsync(Ut, U, sizeof(double) * c->nstate, cudaMemcpyDeviceToDevice, c->stream);
    if ((rc = step_device(c, Ut, 0.0))) break;  // warm-up
    cudaEventRecord(e0, c->stream);
    for (int k = 0; k < steps && rc == WS_OK; ++k) rc = step_device(c, Ut, 0.0);
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      bestc = cfg;
    }
  }
  c->prof_on = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(Ut);
  if (rc) return rc;
  if ((rc = build_chunks(c, bestc))) return rc;
  if (c->graph_exec) {
    cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
  }
  if (choice) *choice = bestc;
  return WS_OK;
}

int ws_set_resident(ws_ctx* c, int enable) {
  if (!c) return fail(c, WS_EINVAL, "null context");
  c->img_cur = -1;
  if (!enable) {
    c->resident = false;
    return WS_OK;
  }
  if (!c->fused) return fail(c, WS_ENOTSUP, "resident state needs the fused 2D/3D stages");
  for (int k = 0; k < 2; ++k) {
    int rc;
    if (!c->img[k] && (rc = dalloc(c, &c->img[k], (int64_t)c->gd.nv * c->gd.N32))) return rc;
  }
  encode_maps(c);
  c->resident = true;
  return WS_OK;
}

int ws_set_stage_config(ws_ctx* c, int index) {
  if (!c) return fail(c, WS_EINVAL, "null context");
  if (!c->fused) return fail(c, WS_EINVAL, "the context has no fused stage (2D/3D mixed precision)");
  if (!stage_config_valid(c, index)) return fail(c, WS_EINVAL, "bad configuration %d", index);
  set_stage_config(c, index);
  return WS_OK;
}

int ws_get_stage_config(ws_ctx* c, int* index, int* tile_x, int* tile_y, int* threads, int* schedule, int* tma,
                        int* tail_rows) {
  if (!c) return fail(c, WS_EINVAL, "null context");
  if (!c->fused) return fail(c, WS_EINVAL, "the context has no fused stage (2D/3D mixed precision)");
  if (index) *index = stage_config_index(c);
  if (tile_x) *tile_x = 32;
  if (tile_y) *tile_y = fused2d_tile_height(c->stage_tile);
  if (threads) *threads = fused_tile_threads(c->stage_tile);
  if (schedule) *schedule = c->stage_sched;
  if (tma) *tma = c->stage_tma;
  if (tail_rows) *tail_rows = c->gd.ndim == 2 && c->stage_tile == 3 ? c->tail_rows : -1;
  return WS_OK;
}

int ws_set_graph(ws_ctx* c, int enable) {
  if (!c) return fail(c, WS_EINVAL, "null context");
  c->graph_on = enable != 0;
  return WS_OK;
}

int ws_profile(ws_ctx* c, int enable) {
  if (!c) return fail(c, WS_EINVAL, "null context");
  if (enable == 1) {
    CK(c, cudaStreamSynchronize(c->stream));
    c->ev_used = 0;
    for (int k = 0; k < WS_NKERNEL; ++k) c->nlaunch[k] = 0;
  }
  c->prof_on = enable != 0;
  return WS_OK;
}

int ws_profile_read(ws_ctx* c, double ms[WS_NKERNEL], int64_t launches[WS_NKERNEL]) {
  if (!c) return fail(c, WS_EINVAL, "null context");
  CK(c, cudaStreamSynchronize(c->stream));
  double acc[WS_NKERNEL] = {0};
  for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
    float t = 0.f;
    CK(c, cudaEventElapsedTime(&t, c->ev[i], c->ev[i + 1]));
    acc[c->ev_cls[i / 2]] += t;
  }
  for (int k = 0; k < WS_NKERNEL; ++k) {
    if (ms) ms[k] = acc[k];
    if (launches) launches[k] = c->nlaunch[k];
  }
  return WS_OK;
}

void ws_destroy(ws_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
}

}  // extern "C"
