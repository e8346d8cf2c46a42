// Allocation-free form of the flux divergence, for callers that cannot call
// cudaMalloc.  Examples: a host application whose device memory is owned by
// another allocator or a fixed budget (a framework's caching pool, a plugin
// host), or a latency-critical loop that must not allocate after start-up.
// Such callers cannot create a ws_ctx, since ws_init allocates the context's
// scratch.  This entry point instead uses one file-scope device array as its
// scratch; the caller passes only the state U and the output L.
//
// The array lives in every GPU that loads the library until the process
// exits.  Its size is fixed (WS_NOALLOC_SCRATCH_BYTES in ws.h); grids whose
// scratch would not fit are rejected with WS_EINVAL.
#include <cuda_runtime.h>
#include <stdio.h>

#include <mutex>

#include "ws_internal.h"

using namespace ws;

namespace {

constexpr int64_t kScratchDoubles = WS_NOALLOC_SCRATCH_BYTES / 8;
constexpr int kMaxDevices = 64;

// The scratch: primitive cache and face fluxes of one flux-divergence call.
// Every call overwrites what it reads before reading it, so nothing needs to
// start at zero; the array keeps the last call's contents.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// Device address of the array per device.  In host code the array's name is
// only a host-side stand-in, so the address is looked up once per device
// with cudaGetSymbolAddress while that device is current.
std::mutex g_mu;
double* g_addr[kMaxDevices] = {nullptr};

// writes the message into the caller's buffer (if any) and returns code
struct Err {
  char* buf;
  int len;
  int operator()(int code, const char* msg) const {
    if (buf && len > 0) snprintf(buf, (size_t)len, "ws_flux_divergence_noalloc: %s", msg);
    return code;
  }
};

int scratch_address(double** out, const Err& fail) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(WS_ECUDA, "no CUDA device");
  if (dev < 0 || dev >= kMaxDevices) return fail(WS_ENOTSUP, "device index >= 64");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return fail(WS_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
    g_addr[dev] = (double*)p;
  }
  *out = g_addr[dev];
  return WS_OK;
}

int64_t round256(int64_t doubles) { return (doubles + 31) / 32 * 32; }

}  // namespace

extern "C" WS_API int ws_flux_divergence_noalloc(const ws_grid* grid, const ws_opts* opts, void* stream, double* U,
                                                 double* L, char* err, int err_len) {
  const Err fail{err, err_len};
  if (err && err_len > 0) err[0] = 0;
  if (!grid || !opts || !U || !L || U == L) return fail(WS_EINVAL, "bad pointers");
  const ws_grid& gr = *grid;
  if (gr.ntubes > 0) return fail(WS_ENOTSUP, "batched tubes are not supported");
  // the option checks of ws_init
  if (opts->precision != WS_PREC_FP64 && opts->precision != WS_PREC_MIXED) return fail(WS_EINVAL, "bad precision");
  if (opts->weights != WS_W_MODIFIED && opts->weights != WS_W_BASIC && opts->weights != WS_W_JS)
    return fail(WS_EINVAL, "bad weights");
  if (opts->mood != 0 && opts->mood != 1) return fail(WS_EINVAL, "mood must be 0 or 1");
  if (opts->learned && opts->precision != WS_PREC_MIXED)
    return fail(WS_EINVAL, "the learned gate runs in mixed precision only");
  if (opts->precision != WS_PREC_FP64) return fail(WS_ENOTSUP, "FP64 only");
  if (gr.ndim < 1 || gr.ndim > 3) return fail(WS_EINVAL, "ndim must be 1, 2 or 3");
  GridDev g{};
  g.ndim = gr.ndim;
  g.nv = gr.ndim + 4;
  for (int d = 0; d < 3; ++d) {
    bool act = d < gr.ndim;
    if (act) {
      if (gr.n[d] < 1 || !(gr.dx[d] > 0.0)) return fail(WS_EINVAL, "bad n or dx");
      for (int s = 0; s < 2; ++s)
        if (gr.bc[d][s] < 0 || gr.bc[d][s] > 2) return fail(WS_EINVAL, "bad bc");
      if ((gr.bc[d][0] == WS_BC_PERIODIC) != (gr.bc[d][1] == WS_BC_PERIODIC))
        return fail(WS_EINVAL, "periodic bc needs both sides");
      if (gr.n[d] < NG && (gr.bc[d][0] != WS_BC_TRANSMISSIVE || gr.bc[d][1] != WS_BC_TRANSMISSIVE))
        return fail(WS_EINVAL, "n < 3 needs transmissive ends");
    }
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
  g.ncell = (int64_t)g.n[0] * g.n[1] * g.n[2];
  for (int d = 0; d < 3; ++d) {
    for (int e = 0; e < 3; ++e) g.fe[d][e] = g.n[e] + (e == d ? 1 : 0);
    g.nfaces[d] = d < gr.ndim ? g.fe[d][0] * g.fe[d][1] * g.fe[d][2] : 0;
  }
  // scratch layout: primitive cache (nv+1 fields), then per direction the
  // face fluxes (nv fields) and face velocities, each block 256-byte aligned
  int64_t need = round256((int64_t)(g.nv + 1) * g.N);
  for (int d = 0; d < gr.ndim; ++d) need += round256((int64_t)g.nv * g.nfaces[d]) + round256(g.nfaces[d]);
  if (need > kScratchDoubles) {
    char msg[160];
    snprintf(msg, sizeof msg, "grid needs %lld bytes of scratch, more than the %lld-byte static scratch",
             (long long)(need * 8), (long long)WS_NOALLOC_SCRATCH_BYTES);
    return fail(WS_EINVAL, msg);
  }
  double* base = nullptr;
  int rc = scratch_address(&base, fail);
  if (rc) return rc;
  double* Q = base;
  int64_t off = round256((int64_t)(g.nv + 1) * g.N);
  double* Fh[3] = {nullptr, nullptr, nullptr};
  double* us[3] = {nullptr, nullptr, nullptr};
  for (int d = 0; d < gr.ndim; ++d) {
    Fh[d] = base + off;
    off += round256((int64_t)g.nv * g.nfaces[d]);
    us[d] = base + off;
    off += round256(g.nfaces[d]);
  }
  cudaStream_t s = (cudaStream_t)stream;
  double eps = opts->eps > 0.0 ? opts->eps : (opts->weights == WS_W_JS ? 1e-6 : 1e-40);
  for (int d = 0; d < g.ndim; ++d) launch_ghost(g, U, d, s);
  launch_prim(g, U, Q, s);
  for (int d = 0; d < g.ndim; ++d) launch_face_fp64(g, d, Q, Fh[d], us[d], nullptr, eps, opts->mood, opts->weights, s);
  launch_update(g, -1, U, U, L, Fh, us, nullptr, nullptr, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(WS_ECUDA, cudaGetErrorString(e));
  return WS_OK;
}
