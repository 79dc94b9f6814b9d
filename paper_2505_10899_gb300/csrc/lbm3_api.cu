// Host runtime behind include/lbm3_api.h: parameter checks, workspace
// carving, tiling, CUDA-graph replay of the step loop, state import/export,
// phase volumes and error reporting for the three-dimensional step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include <cuda_runtime.h>

#include "../../include/lbm3_api.h"
#include "launch3.h"
#include "lbm3_layout.h"
#include "lbm_trace.h"

namespace lbmk {
int set_last_error(int code, const char* msg);  // lbm_api.cu: lbm_last_error()
}

using lbmk3::Bufs;
using lbmk3::Host3;

struct lbm3_handle {
  lbm3_params prm{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;  // private stream for graph capture
  char* ws = nullptr;
  size_t ws_bytes = 0;
  Bufs b{};
  Host3 hp{};
  int32_t* flags = nullptr;
  int8_t* labels = nullptr;
  int nregions = 1;
  double* part = nullptr;
  int64_t part_cap = 0;  // doubles
  double* vol = nullptr;
  double* staging = nullptr;
  double* track = nullptr;
  int bx = 32, by = 8, zc = 32;
  int variant = lbmk3::kVarRegs;  // step-kernel variant in use
  int variant_req = 0;            // requested: 0 automatic
  int64_t t = 0;
  int parity = 0;
  cudaGraphExec_t gexec = nullptr;
  int graph_parity = -1;
};

namespace {

int fail(int code, const std::string& m) { return lbmk::set_last_error(code, m.c_str()); }

#define L3_CUDA(call)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(LBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
  } while (0)

constexpr size_t kAlign = 256;
constexpr int kGraphSteps = 64;     // steps per captured graph (even)
constexpr int kVolParts = 152 * 8;  // CTAs of the labelled volume reduction
constexpr int64_t kMaxNodes = 2147483647;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

int64_t nodes(const lbm3_params& p) { return (int64_t)p.nx * p.ny * p.nz; }

size_t elem(int prec) { return prec == LBM3_F64 ? 8 : 4; }        // T
size_t selem(int prec) { return prec == LBM3_F64 ? 8 : (prec == LBM3_F32 ? 4 : 2); }  // S

int check(const lbm3_params* p) {
  if (!p) return fail(LBM_ERR_ARG, "null params");
  if (p->abi_version != LBM_ABI_VERSION) return fail(LBM_ERR_ARG, "abi_version mismatch");
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail(LBM_ERR_ARG, "nx, ny, nz must be >= 1");
  if (nodes(*p) > kMaxNodes) return fail(LBM_ERR_ARG, "box too large (at most 2^31 - 1 nodes)");
  if (p->precision != LBM3_F64 && p->precision != LBM3_F32 && p->precision != LBM3_F16)
    return fail(LBM_ERR_ARG, "precision");
  if (p->reserved != 0) return fail(LBM_ERR_ARG, "reserved must be 0");
  if (!(p->W > 0) || !std::isfinite(p->W)) return fail(LBM_ERR_ARG, "W must be > 0");
  if (!std::isfinite(p->sigma) || !std::isfinite(p->lambda)) return fail(LBM_ERR_ARG, "sigma, lambda");
  if (!(p->xi >= 0) || !std::isfinite(p->xi)) return fail(LBM_ERR_ARG, "xi must be >= 0");
  if (!(p->tau_g > 0.5) || !std::isfinite(p->tau_g)) return fail(LBM_ERR_ARG, "tau_g must be > 1/2");
  if (!(p->rho_l > 0) || !(p->rho_g > 0) || !std::isfinite(p->rho_l) || !std::isfinite(p->rho_g))
    return fail(LBM_ERR_ARG, "densities must be > 0");
  if (!(p->tau_f_l > 0.5) || !(p->tau_f_g > 0.5) || !std::isfinite(p->tau_f_l) ||
      !std::isfinite(p->tau_f_g))
    return fail(LBM_ERR_ARG, "tau_f must be > 1/2");
  return LBM_OK;
}

int zc_min(const lbm3_params& p) { return std::min(8, p.nz); }

struct Carve {
  size_t f, g, g0, g0lo, J, lab, part, vol, staging, total;
  int64_t plane, part_cap;
};

Carve carve(const lbm3_params& p) {
  Carve c{};
  const int64_t n = nodes(p);
  c.plane = (n + 63) / 64 * 64;
  const size_t es = elem(p.precision), ss = selem(p.precision);
  size_t o = kAlign;  // header: error flags
  c.f = o;
  o = align_up(o + 2 * 19 * (size_t)c.plane * ss);
  c.g = o;
  o = align_up(o + 2 * 6 * (size_t)c.plane * ss);
  c.g0 = o;
  o = align_up(o + 2 * (size_t)c.plane * es);
  c.g0lo = o;  // FP32 arithmetic only: low part of g_0
  if (p.precision != LBM3_F64) o = align_up(o + 2 * (size_t)c.plane * es);
  c.J = o;
  o = align_up(o + 2 * 3 * (size_t)c.plane * es);
  c.lab = o;
  o = align_up(o + (size_t)n);
  // partial sums: the fused per-CTA volumes of the finest allowed tiling, or
  // the labelled reduction's kVolParts x 8
  c.part_cap = std::max<int64_t>(lbmk3::n_ctas(p.nx, p.ny, p.nz, 32, 4, zc_min(p)),
                                 (int64_t)kVolParts * lbmk3::kMaxRegions);
  c.part = o;
  o = align_up(o + (size_t)c.part_cap * 8);
  c.vol = o;
  o = align_up(o + lbmk3::kMaxRegions * 8);
  c.staging = o;
  o = align_up(o + (size_t)n * 8);
  c.total = o;
  return c;
}

Host3 host_params(const lbm3_params& p, int64_t plane) {
  Host3 h{};
  h.nx = p.nx, h.ny = p.ny, h.nz = p.nz;
  h.plane = plane;
  const double beta = 12.0 * p.sigma / p.W, kappa = 1.5 * p.sigma * p.W;  // Sec. 2
  h.beta4 = 4.0 * beta;
  h.kappa = kappa;
  h.lambda = p.lambda;
  h.lamW = p.lambda / p.W;
  h.xi = p.xi;
  h.tfac = 4.0 / ((1.0 + 2.0 * p.xi) * (1.0 + 2.0 * p.xi));
  h.W = p.W;
  h.wg = 1.0 / p.tau_g;
  h.hg = 1.0 - 0.5 / p.tau_g;
  const double cs2 = 1.0 / 3.0;
  const double mu_l = p.rho_l * cs2 * (p.tau_f_l - 0.5), mu_g = p.rho_g * cs2 * (p.tau_f_g - 0.5);
  h.rho_g = p.rho_g;
  h.drho = p.rho_l - p.rho_g;
  h.mu_g = mu_g;
  h.dmu = mu_l - mu_g;
  // tau_f is uniform when both fluids share the kinematic viscosity and the
  // density does not vary, or the viscosities and densities scale together
  h.var_tau = !(p.tau_f_l == p.tau_f_g) ? 1 : 0;
  h.wf = 1.0 / p.tau_f_l;
  h.hf = 1.0 - 0.5 / p.tau_f_l;
  return h;
}

template <typename F>
cudaError_t dispatch(int prec, F&& fn) {
  if (prec == LBM3_F64) return fn(lbmk3::K3<double, double>());
  if (prec == LBM3_F32) return fn(lbmk3::K3<float, float>());
  return fn(lbmk3::K3<float, __half>());
}

cudaError_t launch_step(lbm3_handle* h, cudaStream_t s, int parity, int mode, double* out,
                        int which, bool track) {
  const int64_t nc = lbmk3::n_ctas(h->prm.nx, h->prm.ny, h->prm.nz, h->bx, h->by, h->zc);
  double* vp = (mode == lbmk3::kModeStep && track) ? h->part : nullptr;
  cudaError_t e = dispatch(h->prm.precision, [&](auto k) {
    return decltype(k)::step(h->b, h->hp, parity, h->variant, h->bx, h->by, h->zc, mode,
                             h->flags, vp, out, which, s);
  });
  if (e == cudaSuccess && vp) e = lbmk3::volume3_final_launch(h->part, (int)nc, 1, 1, h->track, s);
  return e;
}

int enqueue_steps(lbm3_handle* h, cudaStream_t s, int parity, int count) {
  for (int k = 0; k < count; ++k) {
    cudaError_t e = launch_step(h, s, parity, lbmk3::kModeStep, nullptr, 0, h->track != nullptr);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("step launch: ") + cudaGetErrorString(e));
    parity ^= 1;
  }
  return LBM_OK;
}

void drop_graph(lbm3_handle* h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  h->gexec = nullptr;
  h->graph_parity = -1;
}

int build_graph(lbm3_handle* h) {
  drop_graph(h);
  cudaGraph_t g = nullptr;
  L3_CUDA(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  const int rc = enqueue_steps(h, h->cap, h->parity, kGraphSteps);
  cudaError_t e = cudaStreamEndCapture(h->cap, &g);
  if (rc != LBM_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&h->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->gexec = nullptr;
    return fail(LBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  h->graph_parity = h->parity;
  return LBM_OK;
}

int read_flags(lbm3_handle* h) {
  int32_t fl = 0;
  L3_CUDA(cudaMemcpyAsync(&fl, h->flags, sizeof fl, cudaMemcpyDeviceToHost, h->stream));
  L3_CUDA(cudaStreamSynchronize(h->stream));
  if (fl & lbmk3::kFlagTimeout3) return fail(LBM_ERR_TIMEOUT, "a bounded device wait timed out");
  if (fl & lbmk3::kFlagNonFinite) return fail(LBM_ERR_NONFINITE, "non-finite value in the fields");
  return LBM_OK;
}

int plane_io(lbm3_handle* h, int kind, int i, double* host, bool to_device) {
  const int64_t n = nodes(h->prm);
  if (to_device)
    L3_CUDA(cudaMemcpyAsync(h->staging, host, n * 8, cudaMemcpyHostToDevice, h->stream));
  L3_CUDA(dispatch(h->prm.precision, [&](auto k) {
    return decltype(k)::plane(h->b, h->hp, h->parity, kind, i, h->staging, to_device ? 1 : 0,
                              h->stream);
  }));
  if (!to_device)
    L3_CUDA(cudaMemcpyAsync(host, h->staging, n * 8, cudaMemcpyDeviceToHost, h->stream));
  L3_CUDA(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

}  // namespace

extern "C" {

size_t lbm3_workspace_bytes(const lbm3_params* p) {
  if (check(p) != LBM_OK) return 0;
  return carve(*p).total;
}

int lbm3_init(const lbm3_params* p, void* d_ws, size_t ws_bytes, const double* h_phi0,
              const double* h_u0, void* stream, lbm3_handle** out) {
  lbmk::TraceRange trace("lbm3_init");
  if (!out) return fail(LBM_ERR_ARG, "null output handle");
  *out = nullptr;
  int rc = check(p);
  if (rc != LBM_OK) return rc;
  if (!h_phi0) return fail(LBM_ERR_ARG, "null phi0");
  const Carve c = carve(*p);
  if (!d_ws || ws_bytes < c.total || (reinterpret_cast<uintptr_t>(d_ws) % kAlign) != 0)
    return fail(LBM_ERR_WORKSPACE, "workspace missing, too small or not 256-byte aligned");
  lbm3_handle* h = new lbm3_handle;
  h->prm = *p;
  h->stream = static_cast<cudaStream_t>(stream);
  h->ws = static_cast<char*>(d_ws);
  h->ws_bytes = ws_bytes;
  const size_t ss = selem(p->precision), es = elem(p->precision);
  for (int k = 0; k < 2; ++k) {
    h->b.f[k] = h->ws + c.f + (size_t)k * 19 * c.plane * ss;
    h->b.g[k] = h->ws + c.g + (size_t)k * 6 * c.plane * ss;
    h->b.g0[k] = h->ws + c.g0 + (size_t)k * c.plane * es;
    h->b.g0lo[k] = p->precision == LBM3_F64 ? nullptr : h->ws + c.g0lo + (size_t)k * c.plane * es;
    h->b.J[k] = h->ws + c.J + (size_t)k * 3 * c.plane * es;
  }
  h->flags = reinterpret_cast<int32_t*>(h->ws);
  h->labels = reinterpret_cast<int8_t*>(h->ws + c.lab);
  h->part = reinterpret_cast<double*>(h->ws + c.part);
  h->part_cap = c.part_cap;
  h->vol = reinterpret_cast<double*>(h->ws + c.vol);
  h->staging = reinterpret_cast<double*>(h->ws + c.staging);
  h->hp = host_params(*p, c.plane);
  // default tiling: 32 x 8 columns, zc planes such that a step has about
  // 8 CTAs per SM
  const int64_t cols = lbmk3::n_ctas(p->nx, p->ny, 1, 32, 8, 1);
  int zc = (int)std::max<int64_t>(1, cols * p->nz / (152 * 8));
  zc = std::max(zc_min(*p), std::min(zc, 64));
  h->bx = 32, h->by = 8, h->zc = std::min(zc, p->nz);
  auto bail = [&](int code) {
    if (h->cap) cudaStreamDestroy(h->cap);
    delete h;
    return code;
  };
  const int64_t n = nodes(*p);
  cudaError_t e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->ws, 0, kAlign, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->labels, 0, (size_t)n, h->stream);
  // phi0 and u0 pass through the staging area and the f/J buffers of parity 1
  // (free until the first step): phi0 in staging, u0 in buffer-1 f planes.
  double* d_phi0 = h->staging;
  double* d_u0 = nullptr;
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_phi0, h_phi0, n * 8, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && h_u0) {
    // 3 n doubles fit in the 19 parity-1 f planes for every storage type
    d_u0 = static_cast<double*>(h->b.f[1]);
    e = cudaMemcpyAsync(d_u0, h_u0, 3 * n * 8, cudaMemcpyHostToDevice, h->stream);
  }
  if (e == cudaSuccess) {
    e = dispatch(p->precision, [&](auto k) {
      return decltype(k)::init(h->b, h->hp, 0, d_phi0, d_u0, h->stream);
    });
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return bail(fail(LBM_ERR_CUDA, std::string("init: ") + cudaGetErrorString(e)));
  *out = h;
  return LBM_OK;
}

int lbm3_step(lbm3_handle* h, int64_t nsteps) {
  lbmk::TraceRange trace("lbm3_step");
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  if (nsteps < 0) return fail(LBM_ERR_ARG, "nsteps must be >= 0");
  while (nsteps >= kGraphSteps) {
    if (!h->gexec || h->graph_parity != h->parity) {
      const int rc = build_graph(h);
      if (rc != LBM_OK) return rc;
    }
    // the graph was captured on the private stream; order it after prior
    // work of the handle's stream by launching it there
    L3_CUDA(cudaGraphLaunch(h->gexec, h->stream));
    nsteps -= kGraphSteps;
    h->t += kGraphSteps;  // kGraphSteps is even: parity unchanged
  }
  if (nsteps > 0) {
    const int rc = enqueue_steps(h, h->stream, h->parity, (int)nsteps);
    if (rc != LBM_OK) return rc;
    h->t += nsteps;
    h->parity ^= (int)(nsteps & 1);
  }
  return LBM_OK;
}

int lbm3_set_regions(lbm3_handle* h, const int8_t* h_labels, int32_t nregions) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  if (nregions < 1 || nregions > lbmk3::kMaxRegions) return fail(LBM_ERR_ARG, "nregions in [1, 8]");
  if (!h_labels && nregions != 1) return fail(LBM_ERR_ARG, "no labels: one region");
  const int64_t n = nodes(h->prm);
  if (h_labels) {
    for (int64_t k = 0; k < n; ++k)
      if (h_labels[k] < -1 || h_labels[k] >= nregions) return fail(LBM_ERR_ARG, "label out of range");
    L3_CUDA(cudaMemcpyAsync(h->labels, h_labels, (size_t)n, cudaMemcpyHostToDevice, h->stream));
  } else {
    L3_CUDA(cudaMemsetAsync(h->labels, 0, (size_t)n, h->stream));
  }
  L3_CUDA(cudaStreamSynchronize(h->stream));
  h->nregions = nregions;
  return LBM_OK;
}

int lbm3_volume(lbm3_handle* h, double* h_out) {
  lbmk::TraceRange trace("lbm3_volume");
  if (!h || !h_out) return fail(LBM_ERR_ARG, "null argument");
  L3_CUDA(dispatch(h->prm.precision, [&](auto k) {
    return decltype(k)::volume(h->b, h->hp, h->parity, h->labels, h->nregions, h->part,
                               kVolParts, h->vol, h->stream);
  }));
  L3_CUDA(cudaMemcpyAsync(h_out, h->vol, h->nregions * 8, cudaMemcpyDeviceToHost, h->stream));
  return read_flags(h);
}

int lbm3_track_volume(lbm3_handle* h, double* d_out) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  h->track = d_out;
  drop_graph(h);
  return LBM_OK;
}

int lbm3_fields(lbm3_handle* h, double* phi, double* u, double* pr) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  const int64_t n = nodes(h->prm);
  double* outs[5] = {phi, u, u ? u + n : nullptr, u ? u + 2 * n : nullptr, pr};
  for (int w = 0; w < 5; ++w) {
    if (!outs[w]) continue;
    L3_CUDA(launch_step(h, h->stream, h->parity, lbmk3::kModeFields, h->staging, w, false));
    L3_CUDA(cudaMemcpyAsync(outs[w], h->staging, n * 8, cudaMemcpyDeviceToHost, h->stream));
    L3_CUDA(cudaStreamSynchronize(h->stream));
  }
  return read_flags(h);
}

int lbm3_get_state(lbm3_handle* h, double* f, double* g, double* j, int64_t* t) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  const int64_t n = nodes(h->prm);
  int rc = LBM_OK;
  for (int i = 0; f && i < 19 && rc == LBM_OK; ++i) rc = plane_io(h, 0, i, f + i * n, false);
  for (int i = 0; g && i < 7 && rc == LBM_OK; ++i) rc = plane_io(h, 1, i, g + i * n, false);
  for (int i = 0; j && i < 3 && rc == LBM_OK; ++i) rc = plane_io(h, 2, i, j + i * n, false);
  if (t) *t = h->t;
  return rc;
}

int lbm3_set_state(lbm3_handle* h, const double* f, const double* g, const double* j, int64_t t) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  const int64_t n = nodes(h->prm);
  int rc = LBM_OK;
  // plane_io copies in through the staging area; the host data is not modified
  for (int i = 0; f && i < 19 && rc == LBM_OK; ++i) rc = plane_io(h, 0, i, const_cast<double*>(f + i * n), true);
  for (int i = 0; g && i < 7 && rc == LBM_OK; ++i) rc = plane_io(h, 1, i, const_cast<double*>(g + i * n), true);
  for (int i = 0; j && i < 3 && rc == LBM_OK; ++i) rc = plane_io(h, 2, i, const_cast<double*>(j + i * n), true);
  h->t = t;
  return rc;
}

int64_t lbm3_time(const lbm3_handle* h) { return h ? h->t : -1; }

int lbm3_get_tiling(const lbm3_handle* h, int32_t* bx, int32_t* by, int32_t* zc, int32_t* n_ctas) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  if (bx) *bx = h->bx;
  if (by) *by = h->by;
  if (zc) *zc = h->zc;
  if (n_ctas) *n_ctas = (int32_t)lbmk3::n_ctas(h->prm.nx, h->prm.ny, h->prm.nz, h->bx, h->by, h->zc);
  return LBM_OK;
}

int lbm3_set_tiling(lbm3_handle* h, int32_t bx, int32_t by, int32_t zc) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  if (!lbmk3::tile_ok(bx, by)) return fail(LBM_ERR_ARG, "unsupported (bx, by)");
  if (zc < zc_min(h->prm) || zc > h->prm.nz) return fail(LBM_ERR_ARG, "zc out of range");
  const int sb = (int)selem(h->prm.precision), nx = h->prm.nx;
  if (h->variant_req && !lbmk3::variant_ok(h->variant_req, sb, bx, by, nx))
    return fail(LBM_ERR_ARG, "tiling not available for the requested kernel variant");
  // keep the variant in use if it runs this tile, else the one made for it
  int v = h->variant;
  if (!lbmk3::variant_ok(v, sb, bx, by, nx))
    v = lbmk3::tile_bulk_ok(bx, by)    ? lbmk3::kVarBulk
        : lbmk3::tile_regs_ok(bx, by)  ? lbmk3::kVarRegs
        : lbmk3::tile_strip_ok(bx, by) ? lbmk3::kVarStrip
                                       : lbmk3::kVarStripOcc;
  if (!lbmk3::variant_ok(v, sb, bx, by, nx))
    return fail(LBM_ERR_ARG, "tiling not available for this box or precision");
  h->bx = bx, h->by = by, h->zc = zc;
  h->variant = v;
  drop_graph(h);
  return LBM_OK;
}

int lbm3_set_kernel(lbm3_handle* h, int32_t variant) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  if (variant < 0 || variant > lbmk3::kVarStripOcc) return fail(LBM_ERR_ARG, "variant in [0, 6]");
  const int sb = (int)selem(h->prm.precision), nx = h->prm.nx;
  int bx = h->bx, by = h->by;
  const int v = variant ? variant : lbmk3::kVarRegs;
  if (v == lbmk3::kVarRegs && !lbmk3::tile_regs_ok(bx, by)) {
    // automatic or register kernel on a tile it does not run: the default tile
    bx = 32;
    by = 8;
  }
  if (v == lbmk3::kVarBulk && !lbmk3::tile_bulk_ok(bx, by)) {
    // the bulk-copy kernel runs its own tiles only: take the one for nx
    bx = nx <= 128 ? 128 : 256;
    by = nx <= 128 ? 4 : 2;
  }
  if (v == lbmk3::kVarStrip && !(lbmk3::tile_strip_ok(bx, by) && nx % bx == 0 && nx >= 2 * bx)) {
    // the strip kernel runs its own tiles only: 64 x 4 where nx allows, else 32 x 8
    const bool wide = nx % 64 == 0 && nx >= 128;
    bx = wide ? 64 : 32;
    by = wide ? 4 : 8;
  }
  if (v == lbmk3::kVarStripOcc && !lbmk3::tile_strip_occ_ok(bx, by)) {
    bx = 64;  // the occupancy form runs 64-column tiles only
    by = 4;
  }
  if (!lbmk3::variant_ok(v, sb, bx, by, nx))
    return fail(LBM_ERR_ARG, "variant not available for this precision or box");
  h->variant_req = variant;
  h->variant = v;
  h->bx = bx, h->by = by;
  drop_graph(h);
  return LBM_OK;
}

int32_t lbm3_get_kernel(const lbm3_handle* h) { return h ? h->variant : -1; }

int lbm3_set_wait_limit(lbm3_handle* h, int64_t cycles) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  h->hp.wait_cycles = cycles < 0 ? lbmk::kWaitCycles : (long long)cycles;
  drop_graph(h);  // captured launches hold the old bound
  return LBM_OK;
}

int lbm3_autotune(lbm3_handle* h, int32_t trials, int32_t* ovar, int32_t* obx, int32_t* oby,
                  int32_t* ozc, double* best_ms) {
  lbmk::TraceRange trace("lbm3_autotune");
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  if (trials < 1 || trials > 100) return fail(LBM_ERR_ARG, "trials must lie in [1, 100]");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  L3_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(LBM_ERR_CUDA, "event create failed");
  }
  const int sb = (int)selem(h->prm.precision), nx = h->prm.nx;
  const int kv = h->variant, kb = h->bx, kby = h->by, kz = h->zc;
  double best = 1e300;
  int bv = kv, bb = kb, bby = kby, bz = kz;
  int rc = LBM_OK;
  const int tiles[7][2] = {{32, 4}, {32, 8}, {32, 16}, {64, 4}, {128, 4}, {256, 2}, {64, 2}};
  for (int v = lbmk3::kVarRegs; v <= lbmk3::kVarStripOcc && rc == LBM_OK; ++v) {
    if (h->variant_req && v != h->variant_req) continue;
    for (const auto& tl : tiles) {
      if (!lbmk3::variant_ok(v, sb, tl[0], tl[1], nx)) continue;
      for (int zc : {8, 16, 32, 64}) {
        const int z = std::min(std::max(zc, zc_min(h->prm)), h->prm.nz);
        if (zc > 8 && z != zc) continue;  // nz too small for this zc
        h->variant = v, h->bx = tl[0], h->by = tl[1], h->zc = z;
        // trial steps read the current source buffers and write the other
        // set, which the next real step overwrites: the state does not change
        cudaError_t e = launch_step(h, h->stream, h->parity, lbmk3::kModeStep, nullptr, 0, false);
        if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
        for (int k = 0; k < trials && e == cudaSuccess; ++k)
          e = launch_step(h, h->stream, h->parity, lbmk3::kModeStep, nullptr, 0, false);
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
          rc = fail(LBM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
          break;
        }
        if (ms / trials < best) best = ms / trials, bv = v, bb = tl[0], bby = tl[1], bz = z;
      }
      if (rc != LBM_OK) break;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->variant = rc == LBM_OK ? bv : kv;
  h->bx = rc == LBM_OK ? bb : kb;
  h->by = rc == LBM_OK ? bby : kby;
  h->zc = rc == LBM_OK ? bz : kz;
  drop_graph(h);
  if (rc != LBM_OK) return rc;
  if (ovar) *ovar = bv;
  if (obx) *obx = bb;
  if (oby) *oby = bby;
  if (ozc) *ozc = bz;
  if (best_ms) *best_ms = best;
  return read_flags(h);
}

int lbm3_status(lbm3_handle* h) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  const cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
  int32_t fl = 0;
  L3_CUDA(cudaMemcpy(&fl, h->flags, sizeof fl, cudaMemcpyDeviceToHost));
  L3_CUDA(cudaMemset(h->flags, 0, sizeof fl));
  if (fl & lbmk3::kFlagTimeout3) return fail(LBM_ERR_TIMEOUT, "a bounded device wait timed out");
  if (fl & lbmk3::kFlagNonFinite) return fail(LBM_ERR_NONFINITE, "non-finite value in the fields");
  return LBM_OK;
}

void lbm3_destroy(lbm3_handle* h) {
  if (!h) return;
  drop_graph(h);
  if (h->cap) cudaStreamDestroy(h->cap);
  delete h;
}

}  // extern "C"
