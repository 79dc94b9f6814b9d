// Host runtime behind the C ABI of include/lbm_api.h: parameter checks,
// workspace carving, work-item tiling, CUDA-graph replay of the step loop,
// state import/export, checkpointing and error reporting.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lbm_api.h"
#include "launch.h"
#include "lbm_handle.h"
#include "lbm_check.h"
#include "lbm_layout.h"
#include "lbm_trace.h"

using lbmk::CaseDev;
using lbmk::Item;
using lbmk::Layout;
using lbmk::Phys;
using lbmk::StepArgs;
using lbmk::Tiling;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define LBM_CUDA(call)                                                        \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess)                                                    \
      return fail(LBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

constexpr size_t kAlign = 256;
constexpr int kGraphSteps = 64;  // steps per captured graph (even)
constexpr int kDirectSteps = 4;  // shorter runs are launched without a graph

size_t align_up(size_t v, size_t a = kAlign) { return (v + a - 1) / a * a; }

// Inverse squared norms of the rows of M (Eq. 24): M^-1 = M^T diag(D).
const double kD[9] = {1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 6, 1.0 / 12,
                      1.0 / 6, 1.0 / 12, 1.0 / 4,  1.0 / 4};


}  // namespace


namespace {

bool same(double a, double b) { return a == b || (std::isnan(a) && std::isnan(b)); }

int check_params(const lbm_params* c, int n) {
  if (!c || n < 1) return fail(LBM_ERR_ARG, "no cases");
  for (int k = 0; k < n; ++k) {
    const lbm_params& p = c[k];
    char buf[160];
    auto bad = [&](const char* what) {
      snprintf(buf, sizeof buf, "case %d: %s", k, what);
      return fail(LBM_ERR_ARG, buf);
    };
    if (p.abi_version != LBM_ABI_VERSION) return bad("abi_version mismatch");
    if (p.nx < 1 || p.ny < 1 || p.nx > (1 << 20) || p.ny > (1 << 20))
      return bad("nx, ny must lie in [1, 2^20]");
    // kernels address a 9-plane buffer with 32-bit element offsets
    if ((int64_t)p.nx * p.ny > 230000000) return bad("grid too large (at most 2.3e8 nodes)");
    if (p.precision != LBM_F64 && p.precision != LBM_F32) return bad("precision");
    if (p.flow != LBM_FLOW_COUPLED && p.flow != LBM_FLOW_VORTEX) return bad("flow");
    if (!(p.W > 0) || !std::isfinite(p.W)) return bad("W must be > 0");
    if (!std::isfinite(p.sigma) || !std::isfinite(p.lambda)) return bad("sigma, lambda");
    if (!(p.xi >= 0) || !std::isfinite(p.xi)) return bad("xi must be >= 0");
    if (!(p.tau_g > 0.5) || !std::isfinite(p.tau_g)) return bad("tau_g must be > 1/2");
    if (p.flow == LBM_FLOW_COUPLED) {
      if (!(p.rho_l > 0) || !(p.rho_g > 0) || !std::isfinite(p.rho_l) || !std::isfinite(p.rho_g))
        return bad("densities must be > 0");
      if (!(p.tau_f_l > 0.5) || !(p.tau_f_g > 0.5) || !std::isfinite(p.tau_f_l) ||
          !std::isfinite(p.tau_f_g))
        return bad("tau_f must be > 1/2");
    } else {
      if (!(p.vortex_T != 0) || !std::isfinite(p.vortex_T) || !std::isfinite(p.vortex_U))
        return bad("vortex_T must be nonzero");
    }
    if (p.walls != 0 && p.walls != 1) return bad("walls must be 0 or 1");
    if (p.walls && p.flow != LBM_FLOW_COUPLED) return bad("walls need the coupled flow");
    if (!std::isfinite(p.u_wall_top) || !std::isfinite(p.u_wall_bottom))
      return bad("wall velocities must be finite");
    for (int i = 0; i < 9; ++i) {
      const bool tied_f = (i == 7 || i == 8), tied_g = (i == 3 || i == 5);
      if (!tied_f && !(p.s_f[i] > 0 && p.s_f[i] < 2)) return bad("s_f rates must lie in (0,2)");
      if (!tied_g && !(p.s_g[i] > 0 && p.s_g[i] < 2)) return bad("s_g rates must lie in (0,2)");
    }
    if (k > 0) {
      const lbm_params& q = c[0];
      bool ok = p.precision == q.precision && p.flow == q.flow && same(p.W, q.W) &&
                same(p.sigma, q.sigma) && same(p.lambda, q.lambda) && same(p.xi, q.xi) &&
                same(p.tau_g, q.tau_g) && same(p.vortex_U, q.vortex_U) &&
                same(p.vortex_T, q.vortex_T);
      for (int i = 0; i < 9; ++i) ok = ok && same(p.s_f[i], q.s_f[i]) && same(p.s_g[i], q.s_g[i]);
      if (!ok) return bad("launch-uniform fields differ from case 0");
    }
  }
  return LBM_OK;
}

size_t elem_size(int precision) { return precision == LBM_F64 ? 8 : 4; }

// Chains: contiguous ranges of the given cases of nearly equal node counts.
std::vector<int> split_chains(const lbm_params* c, const std::vector<int>& ids, int nchains) {
  const int n = (int)ids.size();
  nchains = std::max(1, std::min(nchains, n));
  int64_t total = 0;
  for (int k : ids) total += (int64_t)c[k].nx * c[k].ny;
  std::vector<int> b(nchains + 1, 0);
  b[nchains] = n;
  int64_t acc = 0;
  int k = 0;
  for (int ch = 1; ch < nchains; ++ch) {
    const int64_t want = total * ch / nchains;
    while (k < n - (nchains - ch) &&
           (k < b[ch - 1] + 1 || acc + (int64_t)c[ids[k]].nx * c[ids[k]].ny / 2 < want))
      acc += (int64_t)c[ids[k]].nx * c[ids[k]].ny, ++k;
    b[ch] = k;
  }
  return b;
}

// Whole-row strip width of a case when the tiling's strips are 128 wide: a
// case whose row fits one of the widths 64, 96, 192 or 256 (the smallest that
// holds it, 128 included) runs its rows as single strips of that width in a
// chain of its own, which copies each row once per plane and needs no
// periodic-wrap pieces; 0: the case runs the tiling's strips.
int row_width(int nx) {
  for (int w : {64, 96, 128, 192, 256})
    if (nx <= w) return w == 128 ? 0 : w;
  return 0;
}

// The chains and work items of a tiling.  Work items are strips of the
// chain's width, runs of `rows` rows.  Items are grouped by chain; within a
// chain the cases go largest first (their items are the slowest), so the
// small ones fill the end of the step.  The items of one case stay
// contiguous: [beg[k], end[k]).  Without whole rows (rowmode false, or a
// tiling other than 128-wide strips) the chains are nreq contiguous case
// ranges of nearly equal node counts; with them, the cases of the tiling's
// strips form up to nreq such chains and each whole-row width one more.
struct Plan {
  std::vector<int> chain_case, chain_cases, chain_bx, chain_item, beg, end, case_chain;
  std::vector<Item> items;
};

Plan make_plan(const lbm_params* c, int n, const Tiling& t, int nreq, bool rowmode) {
  Plan pl;
  std::vector<int> generic;
  std::vector<int> byw[4];
  const int widths[4] = {64, 96, 192, 256};
  rowmode = rowmode && t.bx == 128;
  for (int k = 0; k < n; ++k) {
    const int w = rowmode ? row_width(c[k].nx) : 0;
    int q = -1;
    for (int j = 0; j < 4; ++j)
      if (widths[j] == w) q = j;
    if (q < 0) generic.push_back(k);
    else byw[q].push_back(k);
  }
  auto add_chain = [&](const std::vector<int>& ids, int beg_i, int end_i, int bx) {
    pl.chain_case.push_back((int)pl.chain_cases.size());
    for (int r = beg_i; r < end_i; ++r) pl.chain_cases.push_back(ids[r]);
    pl.chain_bx.push_back(bx);
  };
  if (!generic.empty()) {
    const std::vector<int> b = split_chains(c, generic, nreq);
    for (size_t ch = 0; ch + 1 < b.size(); ++ch) add_chain(generic, b[ch], b[ch + 1], t.bx);
  }
  for (int j = 0; j < 4; ++j)
    if (!byw[j].empty()) add_chain(byw[j], 0, (int)byw[j].size(), widths[j]);
  pl.chain_case.push_back((int)pl.chain_cases.size());
  const int nch = (int)pl.chain_bx.size();
  pl.beg.assign(n, 0);
  pl.end.assign(n, 0);
  pl.case_chain.assign(n, 0);
  pl.chain_item.assign(nch + 1, 0);
  for (int ch = 0; ch < nch; ++ch) {
    pl.chain_item[ch] = (int)pl.items.size();
    std::vector<int> order(pl.chain_cases.begin() + pl.chain_case[ch],
                           pl.chain_cases.begin() + pl.chain_case[ch + 1]);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      return (int64_t)c[a].nx * c[a].ny > (int64_t)c[b].nx * c[b].ny;
    });
    const int bx = pl.chain_bx[ch];
    for (int k : order) {
      pl.case_chain[k] = ch;
      pl.beg[k] = (int)pl.items.size();
      for (int y0 = 0; y0 < c[k].ny; y0 += t.rows)
        for (int x0 = 0; x0 < c[k].nx; x0 += bx)
          pl.items.push_back(Item{k, x0, y0, std::min(t.rows, c[k].ny - y0)});
      pl.end[k] = (int)pl.items.size();
    }
  }
  pl.chain_item[nch] = (int)pl.items.size();
  return pl;
}

// Default tiling: the widest strip that leaves at most 15% of the threads idle
// on ragged strips, and runs of 16 rows (short runs balance the load across
// SMs; the halo rows they re-read come from L2) unless the batch is too small
// to give every SM several CTAs.
Tiling choose_tiling(const lbm_params* c, int n) {
  int64_t nodes = 0;
  for (int k = 0; k < n; ++k) nodes += (int64_t)c[k].nx * c[k].ny;
  Tiling t;
  t.bx = 32;
  for (int bx : {128, 64}) {
    int64_t padded = 0;
    for (int k = 0; k < n; ++k) padded += (int64_t)((c[k].nx + bx - 1) / bx) * bx * c[k].ny;
    if (padded * 100 <= nodes * 115) {
      t.bx = bx;
      break;
    }
  }
  const int64_t want = 152 * 12;  // CTAs for a full machine
  int64_t rows = nodes / (t.bx * want);
  while (rows < 4 && t.bx > 32) {
    t.bx /= 2;
    rows = nodes / (t.bx * want);
  }
  t.rows = (int)std::max<int64_t>(2, std::min<int64_t>(16, rows));
  return t;
}

// Work items of the finest tiling (bx = 32, rows = 2): the workspace holds
// item and partial-sum tables of this size so that any tiling fits.
int max_items(const lbm_params* c, int n) {
  int64_t m = 0;
  for (int k = 0; k < n; ++k) m += (int64_t)((c[k].nx + 31) / 32) * ((c[k].ny + 1) / 2);
  return (int)std::min<int64_t>(m, INT32_MAX);
}

Layout make_layout(const lbm_params* c, int n, int n_items, int total_regions) {
  Layout L;
  const size_t es = elem_size(c[0].precision);
  const bool coupled = c[0].flow == LBM_FLOW_COUPLED;
  size_t off = 0;
  L.hdr = off;
  off = align_up(off + 64);
  L.cases = off;
  off = align_up(off + (size_t)n * std::max(sizeof(CaseDev<float>), sizeof(CaseDev<double>)));
  L.items = off;
  off = align_up(off + (size_t)n_items * sizeof(Item));
  L.part = off;
  off = align_up(off + (size_t)n_items * lbmk::kMaxRegions * sizeof(double));
  L.vol = off;
  off = align_up(off + (size_t)std::max(total_regions, n * lbmk::kMaxRegions) * sizeof(double));
  L.init = off;
  off = align_up(off + (size_t)n * sizeof(lbmk::InitSrc));
  L.chainc = off;  // case indices, chain by chain
  off = align_up(off + (size_t)n * sizeof(int));
  int64_t maxp = 0;
  for (int k = 0; k < n; ++k) maxp = std::max<int64_t>(maxp, (int64_t)c[k].nx * c[k].ny);
  L.staging = off;
  off = align_up(off + (size_t)maxp * 4 * sizeof(double));
  L.f.resize(n);
  L.g.resize(n);
  L.glo.resize(n);
  L.J.resize(n);
  L.lab.resize(n);
  L.plane.resize(n);
  for (int k = 0; k < n; ++k) {
    const int64_t nn = (int64_t)c[k].nx * c[k].ny;
    const int64_t plane = (nn + 63) / 64 * 64;
    L.plane[k] = plane;
    const size_t pb = (size_t)plane * es;
    L.g[k] = off;
    off = align_up(off + 2 * 9 * pb);
    if (coupled) {
      L.f[k] = off;
      off = align_up(off + 2 * 9 * pb);
    } else {
      L.f[k] = 0;
    }
    L.J[k] = off;  // two buffers of 2 planes
    off = align_up(off + 4 * pb);
    L.glo[k] = off;  // FP32: low part of g_0, one plane per buffer
    if (es == 4) off = align_up(off + 2 * pb);
    L.lab[k] = off;
    off = align_up(off + (size_t)plane);
  }
  L.total = off;
  return L;
}

template <typename T>
Phys<T> make_phys(const lbm_params& p) {
  Phys<T> ph{};
  const double beta = 12.0 * p.sigma / p.W, kappa = 1.5 * p.sigma * p.W;  // Sec. 2
  ph.beta4 = (T)(4.0 * beta);
  ph.kappa = (T)kappa;
  ph.lambda = (T)p.lambda;
  ph.lamW = (T)(p.lambda / p.W);
  ph.xi = (T)p.xi;
  ph.tfac = (T)(4.0 / ((1.0 + 2.0 * p.xi) * (1.0 + 2.0 * p.xi)));
  // the kernels' psi_k is ln(a/b) in FP64 and log2(a/b) in FP32, psi = (W/4) ln(a/b),
  // and they form q = 12 grad(psi_k): |grad(psi)| = (W s / 48) |q|, s = 1 or ln 2
  const double qs = 48.0 * lbmk::kNormalMin / (p.W * (sizeof(T) == 4 ? 0.69314718055994531 : 1.0));
  ph.qmin2 = (T)(qs * qs);
  double sg[9];
  for (int i = 0; i < 9; ++i) sg[i] = p.s_g[i];
  sg[3] = sg[5] = 1.0 / p.tau_g;  // Eq. 34
  for (int i = 0; i < 9; ++i) {
    ph.fsD[i] = (T)(-p.s_f[i] * kD[i]);
    ph.fhD[i] = (T)((1.0 - 0.5 * p.s_f[i]) * kD[i]);
    ph.gsD[i] = (T)(-sg[i] * kD[i]);
    ph.ghD3[i] = (T)((1.0 - 0.5 * sg[i]) * kD[i] / 3.0);
  }
  ph.vU = p.vortex_U;
  ph.vT = p.vortex_T;
  return ph;
}

template <typename T>
CaseDev<T> make_case(const lbm_handle* h, int k) {
  const lbm_params& p = h->params[k];
  const Layout& L = h->L;
  CaseDev<T> c{};
  const size_t pb = (size_t)L.plane[k] * sizeof(T);
  c.g[0] = (T*)(h->ws + L.g[k]);
  c.g[1] = (T*)(h->ws + L.g[k] + 9 * pb);
  if (h->flow == LBM_FLOW_COUPLED) {
    c.f[0] = (T*)(h->ws + L.f[k]);
    c.f[1] = (T*)(h->ws + L.f[k] + 9 * pb);
  }
  c.J[0] = (T*)(h->ws + L.J[k]);
  c.J[1] = (T*)(h->ws + L.J[k] + 2 * pb);
  c.g0lo[0] = sizeof(T) == 4 ? (T*)(h->ws + L.glo[k]) : nullptr;
  c.g0lo[1] = sizeof(T) == 4 ? (T*)(h->ws + L.glo[k] + pb) : nullptr;
  c.labels = nullptr;
  c.plane = L.plane[k];
  c.nx = p.nx;
  c.ny = p.ny;
  const double cs2 = 1.0 / 3.0;
  const double rho_l = h->flow == LBM_FLOW_COUPLED ? p.rho_l : 1.0;
  const double rho_g = h->flow == LBM_FLOW_COUPLED ? p.rho_g : 1.0;
  c.rho_g = (T)rho_g;
  c.drho = (T)(rho_l - rho_g);
  const double mu_l = rho_l * cs2 * (p.tau_f_l - 0.5), mu_g = rho_g * cs2 * (p.tau_f_g - 0.5);
  c.mu_g = (T)mu_g;
  c.dmu = (T)(mu_l - mu_g);
  c.var_tau = (p.tau_f_l != p.tau_f_g) ? 1 : 0;
  const double s7 = 1.0 / p.tau_f_l;  // Eq. 27, uniform tau_f
  c.sD7 = (T)(-0.25 * s7);
  c.hD7 = (T)(0.25 * (1.0 - 0.5 * s7));
  c.nregions = h->nregions[k];
  c.walls = p.walls;
  c.u_top = (T)(p.walls ? p.u_wall_top : 0.0);
  c.u_bot = (T)(p.walls ? p.u_wall_bottom : 0.0);
  c.vol_base = h->vol_base[k];
  c.item_begin = h->item_begin[k];
  c.item_end = h->item_end[k];
  return c;
}

template <typename T>
CaseDev<T>& case_of(lbm_handle* h, int c) {
  if constexpr (sizeof(T) == 4) return h->cf[c]; else return h->cd[c];
}

int upload_cases(lbm_handle* h) {
  if (h->precision == LBM_F32) {
    h->cf.resize(h->ncases);
    for (int k = 0; k < h->ncases; ++k) {
      CaseDev<float> c = make_case<float>(h, k);
      c.labels = h->cf[k].labels;
      h->cf[k] = c;
    }
    LBM_CUDA(cudaMemcpyAsync(h->cases_dev, h->cf.data(), h->cf.size() * sizeof(CaseDev<float>),
                             cudaMemcpyHostToDevice, h->stream));
  } else {
    h->cd.resize(h->ncases);
    for (int k = 0; k < h->ncases; ++k) {
      CaseDev<double> c = make_case<double>(h, k);
      c.labels = h->cd[k].labels;
      h->cd[k] = c;
    }
    LBM_CUDA(cudaMemcpyAsync(h->cases_dev, h->cd.data(), h->cd.size() * sizeof(CaseDev<double>),
                             cudaMemcpyHostToDevice, h->stream));
  }
  // the host vectors must stay alive until the copy ran: synchronise
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

bool use_tma(const lbm_handle* h) {
  return h->kernel == 2 || (h->kernel == 0 && h->tma_ok);
}

// Batches small enough for one persistent cooperative launch to pay off.
constexpr int64_t kPersistMaxNodes = 4 << 20;

int64_t total_nodes(const lbm_handle* h) {
  int64_t n = 0;
  for (const lbm_params& p : h->params) n += (int64_t)p.nx * p.ny;
  return n;
}

unsigned int* bar_count(lbm_handle* h) { return (unsigned int*)(h->ws + h->L.hdr + 32); }
unsigned int* bar_gen(lbm_handle* h) { return (unsigned int*)(h->ws + h->L.hdr + 36); }


template <typename T>
StepArgs<T> step_args(const lbm_handle* h, int parity, int64_t t_off) {
  StepArgs<T> a{};
  if constexpr (sizeof(T) == 4) a.ph = h->pf; else a.ph = h->pd;
  a.cases = (const CaseDev<T>*)h->cases_dev;
  a.items = h->items_dev;
  a.t_base = h->t_dev;
  a.t_off = t_off;
  a.parity = parity;
  a.flags = h->flags;
  a.wait_cycles = h->wait_cycles;
  return a;
}

int launch_persist(lbm_handle* h, cudaStream_t s, int parity, int nsteps, int flip) {
  const bool coupled = h->flow == LBM_FLOW_COUPLED;
  const int n = (int)h->items.size();
  // a launch whose barrier wait gave up leaves arrivals counted: start at 0
  LBM_CUDA(cudaMemsetAsync(bar_count(h), 0, sizeof(unsigned int), s));
  cudaError_t e;
  if (h->precision == LBM_F32)
    e = lbmk::launch_persistent<float>(step_args<float>(h, parity, 0), h->tile.bx, coupled, n,
                                       nsteps, flip, bar_count(h), bar_gen(h), s);
  else
    e = lbmk::launch_persistent<double>(step_args<double>(h, parity, 0), h->tile.bx, coupled, n,
                                        nsteps, flip, bar_count(h), bar_gen(h), s);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("persistent launch: ") + cudaGetErrorString(e));
  return LBM_OK;
}

// Enqueue `count` consecutive steps starting from source buffer `parity`.
// Each chain runs on its own stream (chain 0 on s, the others on the
// handle's auxiliary streams, forked from and joined back into s), so that
// under stream capture the chains become parallel branches of one graph.
// flip = false: every step reads the same source buffers (autotuning
// trials; the state is not changed).  vol: fused per-case volumes into
// h->track.  clock: advance the device step clock by `count` at the end.
int enqueue_steps(lbm_handle* h, cudaStream_t s, int parity, int count, bool flip, bool vol,
                  bool clock) {
  const bool coupled = h->flow == LBM_FLOW_COUPLED;
  const int nch = h->nchains;
  if (nch > 1) {
    LBM_CUDA(cudaEventRecord(h->fork_ev, s));
    for (int c = 1; c < nch; ++c) LBM_CUDA(cudaStreamWaitEvent(h->aux[c - 1], h->fork_ev, 0));
  }
  for (int c = 0; c < nch; ++c) {
    cudaStream_t sc = c == 0 ? s : h->aux[c - 1];
    const int i0 = h->chain_item[c], ni = h->chain_item[c + 1] - i0;
    const int q0 = h->chain_case[c], nc = h->chain_case[c + 1] - q0;
    const int bx = h->chain_bx[c];
    for (int j = 0; j < count; ++j) {
      const int par = flip ? (parity + j) & 1 : parity;
      const int64_t toff = flip ? j : 0;
      cudaError_t e;
      if (h->precision == LBM_F32) {
        StepArgs<float> a = step_args<float>(h, par, toff);
        a.items = h->items_dev + i0;
        a.vol_part = (vol && h->track) ? h->part + (int64_t)i0 * lbmk::kMaxRegions : nullptr;
        e = lbmk::launch_step<float>(a, bx, coupled, lbmk::kModeStep, use_tma(h), ni, sc);
        if (e == cudaSuccess && vol && h->track)
          e = lbmk::launch_volume_final<float>((const CaseDev<float>*)h->cases_dev,
                                               h->chain_cases_dev + q0, nc, h->part, h->track,
                                               h->t_dev, toff, h->track_slots,
                                               h->total_regions, sc);
      } else {
        StepArgs<double> a = step_args<double>(h, par, toff);
        a.items = h->items_dev + i0;
        a.vol_part = (vol && h->track) ? h->part + (int64_t)i0 * lbmk::kMaxRegions : nullptr;
        e = lbmk::launch_step<double>(a, bx, coupled, lbmk::kModeStep, use_tma(h), ni, sc);
        if (e == cudaSuccess && vol && h->track)
          e = lbmk::launch_volume_final<double>((const CaseDev<double>*)h->cases_dev,
                                               h->chain_cases_dev + q0, nc, h->part, h->track,
                                               h->t_dev, toff, h->track_slots,
                                               h->total_regions, sc);
      }
      if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("step launch: ") + cudaGetErrorString(e));
    }
  }
  for (int c = 1; c < nch; ++c) {
    LBM_CUDA(cudaEventRecord(h->join_ev[c - 1], h->aux[c - 1]));
    LBM_CUDA(cudaStreamWaitEvent(s, h->join_ev[c - 1], 0));
  }
  if (clock) LBM_CUDA(lbmk::launch_clock(h->t_dev, count, s));
  return LBM_OK;
}

void drop_graph(lbm_handle* h) {
  // launches of these graphs that are still queued must run first
  if (!h->graphs.empty()) cudaStreamSynchronize(h->stream);
  for (auto& g : h->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
  h->seen.clear();
}

// Capture `count` steps from source buffer `parity` (with or without flipping
// buffers) on the private capture stream and instantiate them.
int capture_steps(lbm_handle* h, int parity, int count, bool flip, bool vol, bool clock,
                  cudaGraphExec_t* out) {
  *out = nullptr;
  LBM_CUDA(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  int rc = enqueue_steps(h, h->cap, parity, count, flip, vol, clock);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->cap, &g);
  if (rc != LBM_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    *out = nullptr;
    return fail(LBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  return LBM_OK;
}

constexpr size_t kGraphCache = 8;

bool graph_cached(const lbm_handle* h, int count, int parity) {
  for (const auto& g : h->graphs)
    if (g.count == count && g.parity == parity) return true;
  return false;
}

// Whether a run of (count, parity) was met before; records it if not (the
// last 16 kinds of run are remembered).
bool seen_before(lbm_handle* h, int count, int parity) {
  const int key = 2 * count + parity;
  for (int k : h->seen)
    if (k == key) return true;
  if (h->seen.size() >= 16) h->seen.erase(h->seen.begin());
  h->seen.push_back(key);
  return false;
}

// The graph of `count` steps from source buffer `parity`, built on first use.
int step_graph(lbm_handle* h, int count, int parity, cudaGraphExec_t* out) {
  for (const auto& g : h->graphs)
    if (g.count == count && g.parity == parity) {
      *out = g.exec;
      return LBM_OK;
    }
  lbmk::StepGraph g;
  g.count = count;
  g.parity = parity;
  int rc = capture_steps(h, parity, count, true, true, true, &g.exec);
  if (rc) return rc;
  if (h->graphs.size() >= kGraphCache) {
    // the oldest entry goes, once its queued launches have run
    LBM_CUDA(cudaStreamSynchronize(h->stream));
    cudaGraphExecDestroy(h->graphs.front().exec);
    h->graphs.erase(h->graphs.begin());
  }
  h->graphs.push_back(g);
  *out = g.exec;
  return LBM_OK;
}

int check_case(const lbm_handle* h, int c) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  if (c < 0 || c >= h->ncases) return fail(LBM_ERR_ARG, "case index out of range");
  return LBM_OK;
}

int read_flags(lbm_handle* h) {
  int32_t fl = 0;
  LBM_CUDA(cudaMemcpyAsync(&fl, h->flags, sizeof fl, cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  if (fl & lbmk::kFlagBounds)
    return fail(LBM_ERR_BOUNDS, "index out of range (build with index checks)");
  if (fl & lbmk::kFlagTimeout) return fail(LBM_ERR_TIMEOUT, "a bounded device wait timed out");
  if (fl & lbmk::kFlagNonFinite) return fail(LBM_ERR_NONFINITE, "non-finite macroscopic field");
  return LBM_OK;
}

template <typename T>
int do_fields(lbm_handle* h, int c, double* phi, double* ux, double* uy, double* p) {
  const int64_t n = (int64_t)h->params[c].nx * h->params[c].ny;
  double* st = h->staging;
  StepArgs<T> a = step_args<T>(h, h->parity, 0);
  a.items = h->items_dev + h->item_begin[c];
  a.out_phi = st;
  a.out_ux = st + n;
  a.out_uy = st + 2 * n;
  a.out_p = st + 3 * n;
  cudaError_t e = lbmk::launch_step<T>(a, h->chain_bx[h->case_chain[c]], h->flow == LBM_FLOW_COUPLED,
                                       lbmk::kModeFields, use_tma(h),
                                       h->item_end[c] - h->item_begin[c], h->stream);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("fields: ") + cudaGetErrorString(e));
  double* outs[4] = {phi, ux, uy, p};
  for (int q = 0; q < 4; ++q)
    if (outs[q])
      LBM_CUDA(cudaMemcpyAsync(outs[q], st + q * n, n * sizeof(double), cudaMemcpyDeviceToHost,
                               h->stream));
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

template <typename T>
int do_get_state(lbm_handle* h, int c, double* f, double* g, double* j) {
  const lbm_params& p = h->params[c];
  const int64_t n = (int64_t)p.nx * p.ny;
  const CaseDev<T>& cd = case_of<T>(h, c);
  double* st = h->staging;
  for (int which = 0; which < 2; ++which) {
    double* out = which == 0 ? g : f;
    const T* buf = which == 0 ? cd.g[h->parity] : cd.f[h->parity];
    if (!out || !buf) continue;
    for (int i = 0; i < 9; ++i) {
      cudaError_t e =
          lbmk::launch_plane_export<T>(st, buf, cd.plane, i, p.nx, p.ny, cd.walls, h->stream);
      if (e == cudaSuccess && which == 1 && cd.walls)  // f arriving from a wall
        e = lbmk::launch_wall_f_fix<T>(st, cd, h->parity, i, 1.0, h->stream);
      if (e == cudaSuccess && which == 0 && i == 0 && cd.g0lo[h->parity])
        e = lbmk::launch_add_lo_f64<T>(st, cd.g0lo[h->parity], n, h->stream);  // g_0 = hi + lo
      if (e != cudaSuccess) return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
      LBM_CUDA(cudaMemcpyAsync(out + i * n, st, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      LBM_CUDA(cudaStreamSynchronize(h->stream));
    }
  }
  if (j) {
    for (int q = 0; q < 2; ++q) {
      cudaError_t e = lbmk::launch_copy_to_f64<T>(st, cd.J[h->parity] + q * cd.plane, n, h->stream);
      if (e != cudaSuccess) return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
      LBM_CUDA(cudaMemcpyAsync(j + q * n, st, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      LBM_CUDA(cudaStreamSynchronize(h->stream));
    }
  }
  return LBM_OK;
}

template <typename T>
int do_set_state(lbm_handle* h, int c, const double* f, const double* g, const double* j) {
  const lbm_params& p = h->params[c];
  const int64_t n = (int64_t)p.nx * p.ny;
  const CaseDev<T>& cd = case_of<T>(h, c);
  double* st = h->staging;
  for (int which = 0; which < 2; ++which) {
    const double* in = which == 0 ? g : f;
    T* buf = which == 0 ? cd.g[h->parity] : cd.f[h->parity];
    if (!in || !buf) continue;
    for (int i = 0; i < 9; ++i) {
      LBM_CUDA(cudaMemcpyAsync(st, in + i * n, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
      cudaError_t e = cudaSuccess;
      if (which == 1 && cd.walls)  // g is already in place: rho(phi) is known
        e = lbmk::launch_wall_f_fix<T>(st, cd, h->parity, i, -1.0, h->stream);
      if (e == cudaSuccess)
        e = lbmk::launch_plane_import<T>(buf, cd.plane, st, i, p.nx, p.ny, cd.walls, h->stream);
      if (e == cudaSuccess && which == 0 && i == 0 && cd.g0lo[h->parity])
        e = lbmk::launch_lo_from_f64<T>(cd.g0lo[h->parity], buf, st, n, h->stream);
      if (e != cudaSuccess) return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
      LBM_CUDA(cudaStreamSynchronize(h->stream));
    }
  }
  if (j) {
    for (int q = 0; q < 2; ++q) {
      LBM_CUDA(cudaMemcpyAsync(st, j + q * n, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
      cudaError_t e = lbmk::launch_copy_to_T<T>(cd.J[h->parity] + q * cd.plane, st, n, h->stream);
      if (e != cudaSuccess) return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
      LBM_CUDA(cudaStreamSynchronize(h->stream));
    }
  }
  return LBM_OK;
}

int set_clock(lbm_handle* h) {
  LBM_CUDA(cudaMemcpyAsync(h->t_dev, &h->t, sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

struct CkptHeader {
  char magic[8];
  int32_t abi, precision, flow, ncases;
  int64_t t;
  uint64_t payload;
  char pad[24];
};

size_t state_bytes_case(const lbm_handle* h, int k) {
  const size_t es = elem_size(h->precision);
  const int64_t n = (int64_t)h->params[k].nx * h->params[k].ny;
  const int planes = (h->flow == LBM_FLOW_COUPLED ? 18 : 9) + 2 + (es == 4 ? 1 : 0);
  return (size_t)planes * n * es;
}

// New tiling or chain count: rebuild the item table and the case table.
// Whole-row chains need the bulk-copy kernel (FP32; the FP64 kernels are
// bound by the FP64 pipe, where the strip layout hardly matters).
bool rowmode(const lbm_handle* h) {
  return h->row_chains && use_tma(h) && h->precision == LBM_F32;
}

void apply_plan(lbm_handle* h, Plan& pl) {
  h->nchains = (int)pl.chain_bx.size();
  h->chain_case.swap(pl.chain_case);
  h->chain_cases.swap(pl.chain_cases);
  h->chain_bx.swap(pl.chain_bx);
  h->chain_item.swap(pl.chain_item);
  h->case_chain.swap(pl.case_chain);
  h->items.swap(pl.items);
  h->item_begin.swap(pl.beg);
  h->item_end.swap(pl.end);
}

int upload_plan(lbm_handle* h) {
  LBM_CUDA(cudaMemcpyAsync(h->items_dev, h->items.data(), h->items.size() * sizeof(Item),
                           cudaMemcpyHostToDevice, h->stream));
  LBM_CUDA(cudaMemcpyAsync(h->chain_cases_dev, h->chain_cases.data(),
                           h->chain_cases.size() * sizeof(int), cudaMemcpyHostToDevice,
                           h->stream));
  return upload_cases(h);
}

int retile(lbm_handle* h, const Tiling& t, int nchains) {
  Plan pl = make_plan(h->params.data(), h->ncases, t, nchains, rowmode(h));
  if ((int64_t)pl.items.size() > max_items(h->params.data(), h->ncases))
    return fail(LBM_ERR_ARG, "tiling needs more work items than the workspace holds");
  drop_graph(h);
  // the previous step's kernels may still read the item table
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  h->tile = t;
  h->chains_req = nchains;
  apply_plan(h, pl);
  return upload_plan(h);
}

}  // namespace

namespace lbmk {
int set_last_error(int code, const char* msg) { return fail(code, msg); }
}  // namespace lbmk

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

int32_t lbm_abi_version(void) { return LBM_ABI_VERSION; }

const char* lbm_last_error(void) { return g_err.c_str(); }

const char* lbm_status_string(int s) {
  switch (s) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument";
    case LBM_ERR_CUDA: return "CUDA error";
    case LBM_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case LBM_ERR_NONFINITE: return "non-finite value in the fields";
    case LBM_ERR_TIMEOUT: return "device wait timed out";
    case LBM_ERR_UNIMPLEMENTED: return "not implemented";
    case LBM_ERR_BOUNDS: return "index out of range (build with index checks)";
    default: return "unknown status";
  }
}

size_t lbm_workspace_bytes(const lbm_params* cases, int32_t ncases) {
  if (check_params(cases, ncases) != LBM_OK) return 0;
  return make_layout(cases, ncases, max_items(cases, ncases), ncases * lbmk::kMaxRegions).total;
}

int lbm_init(const lbm_params* cases, int32_t ncases, void* d_workspace, size_t ws_bytes,
             const double* const* h_phi0, const double* const* h_u0, void* stream,
             lbm_handle** out) {
  lbmk::TraceRange trace("lbm_init");
  if (!out) return fail(LBM_ERR_ARG, "out is null");
  *out = nullptr;
  int rc = check_params(cases, ncases);
  if (rc) return rc;
  if (!h_phi0) return fail(LBM_ERR_ARG, "h_phi0 is null");
  for (int k = 0; k < ncases; ++k)
    if (!h_phi0[k]) return fail(LBM_ERR_ARG, "h_phi0[c] is null");
  if (!d_workspace) return fail(LBM_ERR_WORKSPACE, "workspace is null");
  if ((uintptr_t)d_workspace % kAlign) return fail(LBM_ERR_WORKSPACE, "workspace not 256-byte aligned");

  lbm_handle* h = new lbm_handle();
  h->ncases = ncases;
  h->params.assign(cases, cases + ncases);
  h->precision = cases[0].precision;
  h->flow = cases[0].flow;
  h->stream = (cudaStream_t)stream;
  h->tile = choose_tiling(cases, ncases);
  h->chains_req = std::min(2, ncases);
  h->nregions.assign(ncases, 1);
  h->vol_base.resize(ncases);
  for (int k = 0; k < ncases; ++k) h->vol_base[k] = k;
  h->total_regions = ncases;
  h->L = make_layout(cases, ncases, max_items(cases, ncases), ncases * lbmk::kMaxRegions);
  if (ws_bytes < h->L.total) {
    const size_t need = h->L.total;
    delete h;
    return fail(LBM_ERR_WORKSPACE, "workspace too small: need " + std::to_string(need));
  }
  h->ws = (char*)d_workspace;
  h->ws_bytes = ws_bytes;
  h->flags = (int32_t*)(h->ws + h->L.hdr);
  h->t_dev = (int64_t*)(h->ws + h->L.hdr + 16);
  h->cases_dev = h->ws + h->L.cases;
  h->items_dev = (Item*)(h->ws + h->L.items);
  h->part = (double*)(h->ws + h->L.part);
  h->vol = (double*)(h->ws + h->L.vol);
  h->staging = (double*)(h->ws + h->L.staging);
  h->pf = make_phys<float>(cases[0]);
  h->pd = make_phys<double>(cases[0]);
  {
    const int vec = h->precision == LBM_F32 ? 4 : 2;  // elements per 16 bytes
    h->tma_ok = true;
    for (int k = 0; k < ncases; ++k)
      if (cases[k].nx % vec != 0 || cases[k].nx < 4) h->tma_ok = false;
    // the bulk-copy kernel stages periodic source rows only: walls run the
    // register-pipelined kernel
    for (int k = 0; k < ncases; ++k)
      if (cases[k].walls) h->tma_ok = false;
  }
  h->chain_cases_dev = (int*)(h->ws + h->L.chainc);
  {
    Plan pl = make_plan(cases, ncases, h->tile, h->chains_req, rowmode(h));
    apply_plan(h, pl);
  }

  auto cleanup = [&](int code) {
    lbm_destroy(h);
    return code;
  };
  if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess)
    return cleanup(fail(LBM_ERR_CUDA, "cannot create capture stream"));
  if (ncases > 1) {  // chains need a stream and an event each (one case: one chain)
    for (int c = 0; c < lbmk::kMaxChains - 1; ++c)
      if (cudaStreamCreateWithFlags(&h->aux[c], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->join_ev[c], cudaEventDisableTiming) != cudaSuccess)
        return cleanup(fail(LBM_ERR_CUDA, "cannot create chain streams"));
    if (cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming) != cudaSuccess)
      return cleanup(fail(LBM_ERR_CUDA, "cannot create chain events"));
  }
  {
    cudaError_t e = h->precision == LBM_F32 ? lbmk::prepare_tma<float>() : lbmk::prepare_tma<double>();
    if (e != cudaSuccess)
      return cleanup(fail(LBM_ERR_CUDA, std::string("kernel attributes: ") + cudaGetErrorString(e)));
  }
  if (cudaMemsetAsync(h->ws + h->L.hdr, 0, 64, h->stream) != cudaSuccess)
    return cleanup(fail(LBM_ERR_CUDA, "header upload failed"));
  // items, chains and cases; labels planes: zero (region 0 everywhere)
  // until lbm_set_regions
  rc = upload_plan(h);
  if (rc) return cleanup(rc);

  // Initial fields.  Where the device can read the caller's arrays itself
  // (page-locked host memory, over the CPU-GPU link, or device memory), the
  // init kernel reads them in place; other (pageable) arrays are first
  // copied into the case's buffer of parity 1 (f planes, or g planes
  // without hydrodynamics), which the init kernel does not write and the
  // first step overwrites.  Then one launch initialises every case.  One
  // synchronisation at the end: on return the host arrays are no longer read.
  const bool vortex = h->flow == LBM_FLOW_VORTEX;
  const size_t es = elem_size(h->precision);
  std::vector<lbmk::InitSrc> src(ncases);
  auto readable = [](const void* p) -> const double* {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
      cudaGetLastError();  // clear the error of an unknown pointer
      return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged ||
        a.type == cudaMemoryTypeHost)
      return (const double*)a.devicePointer;
    return nullptr;
  };
  for (int k = 0; k < ncases; ++k) {
    const lbm_params& p = cases[k];
    const int64_t n = (int64_t)p.nx * p.ny;
    const size_t pb = (size_t)h->L.plane[k] * es;
    double* st = (double*)(h->ws + (vortex ? h->L.g[k] : h->L.f[k]) + 9 * pb);
    lbmk::InitSrc& q = src[k];
    q.rho_g = vortex ? 1.0 : p.rho_g;
    q.drho = vortex ? 0.0 : p.rho_l - p.rho_g;
    q.phi = readable(h_phi0[k]);
    if (!q.phi) {
      if (cudaMemcpyAsync(st, h_phi0[k], n * sizeof(double), cudaMemcpyHostToDevice,
                          h->stream) != cudaSuccess)
        return cleanup(fail(LBM_ERR_CUDA, "initial-field upload failed"));
      q.phi = st;
    }
    q.u = nullptr;
    if (!vortex && h_u0 && h_u0[k]) {
      q.u = readable(h_u0[k]);
      if (!q.u) {
        if (cudaMemcpyAsync(st + n, h_u0[k], 2 * n * sizeof(double), cudaMemcpyHostToDevice,
                            h->stream) != cudaSuccess)
          return cleanup(fail(LBM_ERR_CUDA, "initial-field upload failed"));
        q.u = st + n;
      }
    }
  }
  const lbmk::InitSrc* src_dev = (const lbmk::InitSrc*)(h->ws + h->L.init);
  if (cudaMemcpyAsync((void*)src_dev, src.data(), src.size() * sizeof(lbmk::InitSrc),
                      cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return cleanup(fail(LBM_ERR_CUDA, "init table upload failed"));
  {
    const lbm_params& p = cases[0];  // launch-uniform physics
    const double beta4 = 4.0 * (12.0 * p.sigma / p.W), kappa = 1.5 * p.sigma * p.W;
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < h->nchains && e == cudaSuccess; ++c) {  // one launch per strip width
      const int i0 = h->chain_item[c], ni = h->chain_item[c + 1] - i0;
      if (h->precision == LBM_F32)
        e = lbmk::launch_init_items<float>((const CaseDev<float>*)h->cases_dev, h->items_dev + i0,
                                           ni, h->chain_bx[c], src_dev, beta4, kappa, p.lambda,
                                           vortex, p.vortex_U, 0, h->stream);
      else
        e = lbmk::launch_init_items<double>((const CaseDev<double>*)h->cases_dev,
                                            h->items_dev + i0, ni, h->chain_bx[c], src_dev, beta4,
                                            kappa, p.lambda, vortex, p.vortex_U, 0, h->stream);
    }
    if (e != cudaSuccess) return cleanup(fail(LBM_ERR_CUDA, std::string("init: ") + cudaGetErrorString(e)));
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess)
    return cleanup(fail(LBM_ERR_CUDA, "init sync failed"));
  *out = h;
  return LBM_OK;
}

int lbm_step(lbm_handle* h, int64_t nsteps) {
  lbmk::TraceRange trace("lbm_step");
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  if (nsteps < 0) return fail(LBM_ERR_ARG, "nsteps < 0");
  if (h->kernel == 3 && !h->track) {
    // persistent kernel: chunks of at most 65536 steps per cooperative launch
    while (nsteps > 0) {
      const int cnt = (int)std::min<int64_t>(nsteps, 65536);
      int rc = launch_persist(h, h->stream, h->parity, cnt, 1);
      if (rc) return rc;
      LBM_CUDA(lbmk::launch_clock(h->t_dev, cnt, h->stream));
      h->parity ^= (cnt & 1);
      h->t += cnt;
      nsteps -= cnt;
    }
    return LBM_OK;
  }
  // short runs are launched directly: a graph pays off only over several
  // steps, and a caller that steps many handles one step at a time would
  // otherwise cycle through as many graphs
  if (nsteps < kDirectSteps) {
    int rc = enqueue_steps(h, h->stream, h->parity, (int)nsteps, true, true, true);
    if (rc) return rc;
    h->parity ^= (int)(nsteps & 1);
    h->t += nsteps;
    return LBM_OK;
  }
  // chunks of kGraphSteps steps, then the remainder, each a cached graph.
  // A (count, parity) met for the first time is launched directly: its
  // graph is built when it comes again (or ahead of time by
  // lbm_prepare_steps), so a one-off run does not pay for capturing and
  // instantiating a graph that is never replayed.
  while (nsteps > 0) {
    const int cnt = (int)std::min<int64_t>(nsteps, kGraphSteps);
    cudaGraphExec_t gx = nullptr;
    if (!graph_cached(h, cnt, h->parity) && !seen_before(h, cnt, h->parity)) {
      int rc = enqueue_steps(h, h->stream, h->parity, cnt, true, true, true);
      if (rc) return rc;
    } else {
      int rc = step_graph(h, cnt, h->parity, &gx);
      if (rc) return rc;
      LBM_CUDA(cudaGraphLaunch(gx, h->stream));
    }
    h->parity ^= (cnt & 1);
    h->t += cnt;
    nsteps -= cnt;
  }
  return LBM_OK;
}

int lbm_prepare_steps(lbm_handle* h, int64_t nsteps) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  if (nsteps < 0) return fail(LBM_ERR_ARG, "nsteps < 0");
  if (h->kernel == 3 && !h->track) return LBM_OK;  // one cooperative launch, nothing to capture
  if (nsteps < kDirectSteps) return LBM_OK;         // launched directly
  int parity = h->parity;
  while (nsteps > 0) {
    const int cnt = (int)std::min<int64_t>(nsteps, kGraphSteps);
    cudaGraphExec_t gx = nullptr;
    int rc = step_graph(h, cnt, parity, &gx);
    if (rc) return rc;
    parity ^= (cnt & 1);
    nsteps -= cnt;
    if (cnt == kGraphSteps && nsteps >= kGraphSteps) nsteps = nsteps % kGraphSteps;  // same graph
  }
  return LBM_OK;
}

int lbm_set_regions(lbm_handle* h, int32_t c, const int8_t* h_labels, int32_t nregions) {
  int rc = check_case(h, c);
  if (rc) return rc;
  if (nregions < 1 || nregions > lbmk::kMaxRegions)
    return fail(LBM_ERR_ARG, "nregions must lie in [1, 8]");
  if (h->track && (h_labels || nregions != 1))
    return fail(LBM_ERR_ARG, "switch volume tracking off before declaring labelled regions");
  const int64_t n = (int64_t)h->params[c].nx * h->params[c].ny;
  const int8_t* dlab = nullptr;
  if (h_labels) {
    for (int64_t k = 0; k < n; ++k)
      if (h_labels[k] >= nregions) return fail(LBM_ERR_ARG, "label >= nregions");
    int8_t* d = (int8_t*)(h->ws + h->L.lab[c]);
    LBM_CUDA(cudaMemcpyAsync(d, h_labels, n, cudaMemcpyHostToDevice, h->stream));
    dlab = d;
  }
  h->nregions[c] = nregions;
  int base = 0;
  for (int k = 0; k < h->ncases; ++k) {
    h->vol_base[k] = base;
    base += h->nregions[k];
  }
  h->total_regions = base;
  if (h->precision == LBM_F32) h->cf[c].labels = dlab;
  else h->cd[c].labels = dlab;
  return upload_cases(h);
}

int32_t lbm_num_regions(const lbm_handle* h) { return h ? h->total_regions : 0; }

int lbm_set_kernel(lbm_handle* h, int32_t variant) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  if (variant < 0 || variant > 3) return fail(LBM_ERR_ARG, "kernel variant must be 0, 1, 2 or 3");
  if (variant == 2 && !h->tma_ok)
    return fail(LBM_ERR_ARG, "bulk-copy kernel needs nx a multiple of 16 bytes and nx >= 4");
  if (variant == 3 && total_nodes(h) > kPersistMaxNodes)
    return fail(LBM_ERR_ARG, "persistent kernel is for batches of at most 4 Mi nodes");
  if (variant == h->kernel) return LBM_OK;
  const int keep = h->kernel;
  h->kernel = variant;
  const int rc = retile(h, h->tile, h->chains_req);  // whole-row chains follow the kernel
  if (rc != LBM_OK) h->kernel = keep;
  return rc;
}

int32_t lbm_get_kernel(const lbm_handle* h) {
  if (!h) return -1;
  if (h->kernel == 3) return 3;
  return use_tma(h) ? 2 : 1;
}

int lbm_autotune(lbm_handle* h, int32_t trials, int32_t* best_kernel, int32_t* best_bx,
                 int32_t* best_rows, double* best_ms) {
  lbmk::TraceRange trace("lbm_autotune");
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  if (trials < 1 || trials > 100) return fail(LBM_ERR_ARG, "trials must lie in [1, 100]");
  const bool coupled = h->flow == LBM_FLOW_COUPLED;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  LBM_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(LBM_ERR_CUDA, "event create failed");
  }
  // Trial launches read the current source buffers and write the other
  // buffer set (populations and phi*u), which the next real step overwrites
  // completely: the state is not changed and the clock does not advance.
  // lbm_step replays the step kernels of variants 1 and 2 as CUDA graphs
  // (one branch per chain): time their trials the same way, as one captured
  // graph of n steps (replayed once untimed, then timed).  At least 8 trial
  // steps, so that a small grid is timed in steady state rather than by its
  // launch overhead.
  const int n_trial = trials < 8 ? 8 : trials;
  const Tiling keep_tile = h->tile;
  const int keep_kernel = h->kernel;
  const bool keep_rows = h->row_chains;
  double best = 1e300;
  Tiling best_t = keep_tile;
  int best_k = use_tma(h) ? 2 : 1;
  bool best_rc = keep_rows;
  int rc = LBM_OK;
  for (int kv : {2, 1, 3}) {
    if (kv == 2 && !h->tma_ok) continue;
    if (kv == 3 && total_nodes(h) > kPersistMaxNodes) continue;
    for (int bx : {128, 64, 32}) {
      for (int rows : {2, 4, 8, 16, 32, 64, 128}) {
        // whole-row chains exist for the FP32 bulk-copy kernel on 128-wide
        // strips only: try them on and off there
        const int nrc = (kv == 2 && bx == 128 && h->precision == LBM_F32) ? 2 : 1;
        for (int rcv = 0; rcv < nrc; ++rcv) {
          h->kernel = kv;
          h->row_chains = rcv == 1;
          rc = lbm_set_tiling(h, bx, rows);
          if (rc != LBM_OK) break;
          cudaError_t e = cudaSuccess;
          if (kv == 3) {  // one launch of n_trial steps without flipping buffers
            rc = launch_persist(h, h->stream, h->parity, 1, 0);
            if (rc == LBM_OK) e = cudaEventRecord(e0, h->stream);
            if (rc == LBM_OK && e == cudaSuccess) rc = launch_persist(h, h->stream, h->parity, n_trial, 0);
            if (rc != LBM_OK) break;
          } else {
            cudaGraphExec_t gx = nullptr;
            rc = capture_steps(h, h->parity, n_trial, false, false, false, &gx);
            if (rc != LBM_OK) break;
            e = cudaGraphLaunch(gx, h->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
            if (e == cudaSuccess) e = cudaGraphLaunch(gx, h->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (gx) cudaGraphExecDestroy(gx);
          }
          if (kv == 3 && e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
          if (kv == 3 && e == cudaSuccess) e = cudaEventSynchronize(e1);
          float ms = 0.f;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
          if (e != cudaSuccess) {
            rc = fail(LBM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
            break;
          }
          if (ms / n_trial < best) {
            best = ms / n_trial;
            best_t.bx = bx;
            best_t.rows = rows;
            best_k = kv;
            best_rc = rcv == 1;
          }
        }
        if (rc != LBM_OK) break;
      }
      if (rc != LBM_OK) break;
    }
    if (rc != LBM_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != LBM_OK) {
    h->kernel = keep_kernel;
    h->row_chains = keep_rows;
    lbm_set_tiling(h, keep_tile.bx, keep_tile.rows);
    return rc;
  }
  h->kernel = best_k;
  h->row_chains = best_rc;
  rc = lbm_set_tiling(h, best_t.bx, best_t.rows);
  if (rc != LBM_OK) return rc;
  if (best_kernel) *best_kernel = best_k;
  if (best_bx) *best_bx = best_t.bx;
  if (best_rows) *best_rows = best_t.rows;
  if (best_ms) *best_ms = best;
  return read_flags(h);
}

int lbm_get_tiling(const lbm_handle* h, int32_t* bx, int32_t* rows, int32_t* n_items) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  if (bx) *bx = h->tile.bx;
  if (rows) *rows = h->tile.rows;
  if (n_items) *n_items = (int32_t)h->items.size();
  return LBM_OK;
}

int lbm_set_tiling(lbm_handle* h, int32_t bx, int32_t rows) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  if (!lbmk::valid_bx(bx) || rows < 2 || rows > 1024)
    return fail(LBM_ERR_ARG, "bx must be 32, 64 or 128 and rows in [2, 1024]");
  Tiling t;
  t.bx = bx;
  t.rows = rows;
  return retile(h, t, h->chains_req);
}

int lbm_set_wait_limit(lbm_handle* h, int64_t cycles) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  if (cycles < 0) cycles = lbmk::kWaitCycles;
  if (cycles != h->wait_cycles) drop_graph(h);
  h->wait_cycles = cycles;
  return LBM_OK;
}

int lbm_set_chains(lbm_handle* h, int32_t nchains) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  if (nchains < 1 || nchains > 4) return fail(LBM_ERR_ARG, "nchains must lie in [1, 4]");
  return retile(h, h->tile, std::min<int>(nchains, h->ncases));
}

int32_t lbm_get_chains(const lbm_handle* h) { return h ? h->nchains : 0; }

int lbm_set_row_chains(lbm_handle* h, int32_t on) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  if (on != 0 && on != 1) return fail(LBM_ERR_ARG, "on must be 0 or 1");
  if ((on != 0) == h->row_chains) return LBM_OK;
  h->row_chains = on != 0;
  const int rc = retile(h, h->tile, h->chains_req);
  if (rc != LBM_OK) h->row_chains = !h->row_chains;
  return rc;
}

int32_t lbm_get_row_chains(const lbm_handle* h) { return h && rowmode(h) ? 1 : 0; }

int lbm_track_volume_history(lbm_handle* h, double* out, int64_t nslots) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  if (out) {
    if (nslots < 1) return fail(LBM_ERR_ARG, "nslots < 1");
    for (int k = 0; k < h->ncases; ++k)
      if (h->nregions[k] != 1 ||
          (h->precision == LBM_F32 ? h->cf[k].labels != nullptr : h->cd[k].labels != nullptr))
        return fail(LBM_ERR_ARG, "volume tracking needs one unlabelled region per case");
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, out) != cudaSuccess) cudaGetLastError();
    const bool ok = (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged ||
                     at.type == cudaMemoryTypeHost) && at.devicePointer != nullptr;
    if (!ok) return fail(LBM_ERR_ARG, "volume output must be device or page-locked host memory");
    out = static_cast<double*>(at.devicePointer);
  } else {
    nslots = 1;
  }
  if (out != h->track || nslots != h->track_slots) drop_graph(h);
  h->track = out;
  h->track_slots = nslots;
  return LBM_OK;
}

int lbm_track_volume(lbm_handle* h, double* d_out) {
  return lbm_track_volume_history(h, d_out, 1);
}

int lbm_volume_async(lbm_handle* h, double* d_out) {
  lbmk::TraceRange trace("lbm_volume");
  if (!h || !d_out) return fail(LBM_ERR_ARG, "null argument");
  cudaError_t e = cudaSuccess;
  // item partials chain by chain (each chain's strip width), then the cases
  for (int c = 0; c < h->nchains && e == cudaSuccess; ++c) {
    const int i0 = h->chain_item[c], ni = h->chain_item[c + 1] - i0;
    double* part = h->part + (int64_t)i0 * lbmk::kMaxRegions;
    if (h->precision == LBM_F32)
      e = lbmk::launch_volume_partial<float>((const CaseDev<float>*)h->cases_dev, h->items_dev + i0,
                                             ni, h->chain_bx[c], h->parity, part, h->stream);
    else
      e = lbmk::launch_volume_partial<double>((const CaseDev<double>*)h->cases_dev,
                                              h->items_dev + i0, ni, h->chain_bx[c], h->parity,
                                              part, h->stream);
  }
  if (e == cudaSuccess) {
    if (h->precision == LBM_F32)
      e = lbmk::launch_volume_final<float>((const CaseDev<float>*)h->cases_dev, nullptr, h->ncases,
                                           h->part, d_out, nullptr, 0, 0, 0, h->stream);
    else
      e = lbmk::launch_volume_final<double>((const CaseDev<double>*)h->cases_dev, nullptr,
                                            h->ncases, h->part, d_out, nullptr, 0, 0, 0, h->stream);
  }
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("volume: ") + cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_volume(lbm_handle* h, double* h_out) {
  if (!h || !h_out) return fail(LBM_ERR_ARG, "null argument");
  int rc = lbm_volume_async(h, h->vol);
  if (rc) return rc;
  LBM_CUDA(cudaMemcpyAsync(h_out, h->vol, h->total_regions * sizeof(double), cudaMemcpyDeviceToHost,
                           h->stream));
  return read_flags(h);
}

int lbm_fields(lbm_handle* h, int32_t c, double* phi, double* ux, double* uy, double* p) {
  int rc = check_case(h, c);
  if (rc) return rc;
  if (h->precision == LBM_F32) return do_fields<float>(h, c, phi, ux, uy, p);
  return do_fields<double>(h, c, phi, ux, uy, p);
}

int lbm_get_state(lbm_handle* h, int32_t c, double* f, double* g, double* j, int64_t* t) {
  int rc = check_case(h, c);
  if (rc) return rc;
  if (t) *t = h->t;
  if (h->flow != LBM_FLOW_COUPLED) f = nullptr;
  if (h->precision == LBM_F32) return do_get_state<float>(h, c, f, g, j);
  return do_get_state<double>(h, c, f, g, j);
}

int lbm_set_state(lbm_handle* h, int32_t c, const double* f, const double* g, const double* j,
                  int64_t t) {
  int rc = check_case(h, c);
  if (rc) return rc;
  if (t < 0) return fail(LBM_ERR_ARG, "t < 0");
  if (h->flow != LBM_FLOW_COUPLED) f = nullptr;
  rc = (h->precision == LBM_F32) ? do_set_state<float>(h, c, f, g, j)
                                 : do_set_state<double>(h, c, f, g, j);
  if (rc) return rc;
  h->t = t;
  return set_clock(h);
}

int64_t lbm_time(const lbm_handle* h) { return h ? h->t : -1; }

size_t lbm_checkpoint_bytes(const lbm_handle* h) {
  if (!h) return 0;
  size_t b = sizeof(CkptHeader);
  for (int k = 0; k < h->ncases; ++k) b += state_bytes_case(h, k);
  return b;
}

int lbm_save(lbm_handle* h, void* h_buf, size_t bytes) {
  if (!h || !h_buf) return fail(LBM_ERR_ARG, "null argument");
  if (bytes < lbm_checkpoint_bytes(h)) return fail(LBM_ERR_ARG, "buffer too small");
  CkptHeader hd{};
  memcpy(hd.magic, "LBMCKPT2", 8);
  hd.abi = LBM_ABI_VERSION;
  hd.precision = h->precision;
  hd.flow = h->flow;
  hd.ncases = h->ncases;
  hd.t = h->t;
  hd.payload = lbm_checkpoint_bytes(h) - sizeof(CkptHeader);
  memcpy(h_buf, &hd, sizeof hd);
  char* p = (char*)h_buf + sizeof hd;
  const size_t es = elem_size(h->precision);
  for (int k = 0; k < h->ncases; ++k) {
    const int64_t n = (int64_t)h->params[k].nx * h->params[k].ny;
    const size_t pb = (size_t)h->L.plane[k] * es;
    const char* gb = h->ws + h->L.g[k] + h->parity * 9 * pb;
    LBM_CUDA(cudaMemcpy2DAsync(p, n * es, gb, pb, n * es, 9, cudaMemcpyDeviceToHost, h->stream));
    p += 9 * n * es;
    if (h->flow == LBM_FLOW_COUPLED) {
      const char* fb = h->ws + h->L.f[k] + h->parity * 9 * pb;
      LBM_CUDA(cudaMemcpy2DAsync(p, n * es, fb, pb, n * es, 9, cudaMemcpyDeviceToHost, h->stream));
      p += 9 * n * es;
    }
    LBM_CUDA(cudaMemcpy2DAsync(p, n * es, h->ws + h->L.J[k] + h->parity * 2 * pb, pb, n * es, 2,
                               cudaMemcpyDeviceToHost,
                               h->stream));
    p += 2 * n * es;
    if (es == 4) {  // low part of g_0
      LBM_CUDA(cudaMemcpyAsync(p, h->ws + h->L.glo[k] + h->parity * pb, n * es,
                               cudaMemcpyDeviceToHost, h->stream));
      p += n * es;
    }
  }
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_load(lbm_handle* h, const void* h_buf, size_t bytes) {
  if (!h || !h_buf) return fail(LBM_ERR_ARG, "null argument");
  if (bytes < lbm_checkpoint_bytes(h)) return fail(LBM_ERR_ARG, "buffer too small");
  CkptHeader hd;
  memcpy(&hd, h_buf, sizeof hd);
  if (memcmp(hd.magic, "LBMCKPT2", 8) != 0 || hd.abi != LBM_ABI_VERSION ||
      hd.precision != h->precision || hd.flow != h->flow || hd.ncases != h->ncases ||
      hd.payload != lbm_checkpoint_bytes(h) - sizeof(CkptHeader))
    return fail(LBM_ERR_ARG, "checkpoint does not match this handle");
  const char* p = (const char*)h_buf + sizeof hd;
  const size_t es = elem_size(h->precision);
  for (int k = 0; k < h->ncases; ++k) {
    const int64_t n = (int64_t)h->params[k].nx * h->params[k].ny;
    const size_t pb = (size_t)h->L.plane[k] * es;
    char* gb = h->ws + h->L.g[k] + h->parity * 9 * pb;
    LBM_CUDA(cudaMemcpy2DAsync(gb, pb, p, n * es, n * es, 9, cudaMemcpyHostToDevice, h->stream));
    p += 9 * n * es;
    if (h->flow == LBM_FLOW_COUPLED) {
      char* fb = h->ws + h->L.f[k] + h->parity * 9 * pb;
      LBM_CUDA(cudaMemcpy2DAsync(fb, pb, p, n * es, n * es, 9, cudaMemcpyHostToDevice, h->stream));
      p += 9 * n * es;
    }
    LBM_CUDA(cudaMemcpy2DAsync(h->ws + h->L.J[k] + h->parity * 2 * pb, pb, p, n * es, n * es, 2,
                               cudaMemcpyHostToDevice,
                               h->stream));
    p += 2 * n * es;
    if (es == 4) {
      LBM_CUDA(cudaMemcpyAsync(h->ws + h->L.glo[k] + h->parity * pb, p, n * es,
                               cudaMemcpyHostToDevice, h->stream));
      p += n * es;
    }
  }
  h->t = hd.t;
  return set_clock(h);
}

size_t lbm_snapshot_bytes(const lbm_handle* h, int32_t c) {
  if (!h || c < 0 || c >= h->ncases) return 0;
  const int planes = h->precision == LBM_F32 ? 21 : 20;  // FP32: + low part of g_0
  return (size_t)planes * h->params[c].nx * h->params[c].ny * elem_size(h->precision);
}

// Device copy of the state of case c: [f*: 9][g*: 9][phi*u: 2] planes of
// nx*ny elements each, pull layout (f planes zero in vortex mode).
int lbm_snapshot(lbm_handle* h, int32_t c, void* d_buf) {
  int rc = check_case(h, c);
  if (rc) return rc;
  if (!d_buf) return fail(LBM_ERR_ARG, "d_buf is null");
  const int64_t n = (int64_t)h->params[c].nx * h->params[c].ny;
  const bool coupled = h->flow == LBM_FLOW_COUPLED;
  cudaError_t e;
  if (h->precision == LBM_F32) {
    const CaseDev<float>& cd = h->cf[c];
    e = lbmk::launch_snapshot<float>(coupled ? cd.f[h->parity] : nullptr, cd.g[h->parity],
                                     cd.J[h->parity], cd.g0lo[h->parity], cd.plane, n,
                                     (float*)d_buf, h->stream);
  } else {
    const CaseDev<double>& cd = h->cd[c];
    e = lbmk::launch_snapshot<double>(coupled ? cd.f[h->parity] : nullptr, cd.g[h->parity],
                                      cd.J[h->parity], nullptr, cd.plane, n, (double*)d_buf,
                                      h->stream);
  }
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("snapshot: ") + cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_restore(lbm_handle* h, int32_t c, const void* d_buf) {
  int rc = check_case(h, c);
  if (rc) return rc;
  if (!d_buf) return fail(LBM_ERR_ARG, "d_buf is null");
  const int64_t n = (int64_t)h->params[c].nx * h->params[c].ny;
  const size_t es = elem_size(h->precision), pb = (size_t)h->L.plane[c] * es, nb = n * es;
  const char* in = (const char*)d_buf;
  if (h->flow == LBM_FLOW_COUPLED)
    LBM_CUDA(cudaMemcpy2DAsync(h->ws + h->L.f[c] + h->parity * 9 * pb, pb, in, nb, nb, 9,
                               cudaMemcpyDeviceToDevice, h->stream));
  LBM_CUDA(cudaMemcpy2DAsync(h->ws + h->L.g[c] + h->parity * 9 * pb, pb, in + 9 * nb, nb, nb, 9,
                             cudaMemcpyDeviceToDevice, h->stream));
  LBM_CUDA(cudaMemcpy2DAsync(h->ws + h->L.J[c] + h->parity * 2 * pb, pb, in + 18 * nb, nb, nb, 2,
                             cudaMemcpyDeviceToDevice, h->stream));
  if (es == 4)  // FP32: the low part of the g_0 float pair
    LBM_CUDA(cudaMemcpyAsync(h->ws + h->L.glo[c] + h->parity * pb, in + 20 * nb, nb,
                             cudaMemcpyDeviceToDevice, h->stream));
  return LBM_OK;
}

int lbm_record_steps(lbm_handle* h, int64_t count, void* d_states, int64_t stride_bytes) {
  lbmk::TraceRange trace("lbm_record_steps");
  if (!h || !d_states) return fail(LBM_ERR_ARG, "null argument");
  if (h->ncases != 1) return fail(LBM_ERR_ARG, "recording needs a single-case handle");
  if (count < 0) return fail(LBM_ERR_ARG, "count < 0");
  if (count > 1 && stride_bytes < (int64_t)lbm_snapshot_bytes(h, 0))
    return fail(LBM_ERR_ARG, "stride_bytes smaller than a snapshot");
  for (int64_t j = 0; j < count; ++j) {
    int rc = lbm_snapshot(h, 0, (char*)d_states + j * stride_bytes);
    if (rc) return rc;
    rc = lbm_step(h, 1);
    if (rc) return rc;
  }
  return LBM_OK;
}

int lbm_set_time(lbm_handle* h, int64_t t) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  if (t < 0) return fail(LBM_ERR_ARG, "t < 0");
  h->t = t;
  LBM_CUDA(lbmk::launch_set_clock(h->t_dev, t, h->stream));  // asynchronous
  return LBM_OK;
}

int lbm_status(lbm_handle* h) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
  int rc = read_flags(h);
  LBM_CUDA(cudaMemsetAsync(h->flags, 0, sizeof(int32_t), h->stream));
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  return rc;
}


void lbm_destroy(lbm_handle* h) {
  if (!h) return;
  drop_graph(h);
  if (h->cap) cudaStreamDestroy(h->cap);
  for (int c = 0; c < lbmk::kMaxChains - 1; ++c) {
    if (h->aux[c]) cudaStreamDestroy(h->aux[c]);
    if (h->join_ev[c]) cudaEventDestroy(h->join_ev[c]);
  }
  if (h->fork_ev) cudaEventDestroy(h->fork_ev);
  delete h;
}

}  // extern "C"
