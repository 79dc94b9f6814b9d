// Internal definition of the opaque lbm_handle, shared by the host runtime
// (lbm_api.cu) and the reverse-mode code (lbm_adjoint.cu).  Not part of the
// public ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lbm_api.h"
#include "lbm_layout.h"

namespace lbmk {

struct Layout {
  size_t hdr = 0, cases = 0, items = 0, part = 0, vol = 0, init = 0, chainc = 0, staging = 0;
  std::vector<size_t> f, g, J, lab;  // per-case offsets (f: 2 buffers back to back)
  std::vector<size_t> glo;           // FP32: low part of g_0, 2 planes per case
  std::vector<int64_t> plane;
  size_t total = 0;
};

struct Tiling {
  int bx = 128;
  int rows = 32;
};

// Independent case groups ("chains") whose steps are captured as parallel
// branches of one CUDA graph, so that the last CTAs of one group's step run
// beside the next group's work instead of leaving SMs idle.
constexpr int kMaxChains = 8;  // 4 of the tiling's strips + 4 whole-row widths

// A captured and instantiated sequence of `count` steps starting from source
// buffer `parity`.
struct StepGraph {
  int count = 0, parity = 0;
  cudaGraphExec_t exec = nullptr;
};

}  // namespace lbmk

struct lbm_handle {
  int ncases = 0;
  int precision = LBM_F32;
  int flow = LBM_FLOW_COUPLED;
  std::vector<lbm_params> params;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;  // private stream for graph capture
  lbmk::Layout L;
  lbmk::Tiling tile;
  std::vector<lbmk::Item> items;
  std::vector<int> item_begin, item_end, vol_base, nregions;
  int total_regions = 0;
  int64_t t = 0;   // step index
  int parity = 0;  // source buffer
  lbmk::Phys<float> pf{};
  lbmk::Phys<double> pd{};
  std::vector<lbmk::CaseDev<float>> cf;
  std::vector<lbmk::CaseDev<double>> cd;
  int nchains = 1;              // chains of the current plan
  int chains_req = 2;           // chains requested for the tiling's strips
  bool row_chains = false;      // whole-row chains requested (lbm_set_row_chains)
  std::vector<int> chain_case;  // chain c: its cases chain_cases[chain_case[c] .. chain_case[c+1])
  std::vector<int> chain_cases; //   (case indices, chain by chain)
  std::vector<int> chain_item;  //          items [chain_item[c], chain_item[c+1])
  std::vector<int> chain_bx;    //          strip width of its CTAs
  std::vector<int> case_chain;  // chain of each case
  int* chain_cases_dev = nullptr;  // chain_cases on the device (per-chain volume sums)
  cudaStream_t aux[lbmk::kMaxChains - 1] = {};  // capture streams of chains 1..
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[lbmk::kMaxChains - 1] = {};
  std::vector<lbmk::StepGraph> graphs;  // cache, oldest first
  std::vector<int> seen;                // kinds of run met so far (2 count + parity)
  double* track = nullptr;  // fused volume output (device address), or null
  int64_t track_slots = 1;  // steps of volume history in `track`
  bool tma_ok = false;      // every case allows the bulk-copy kernel
  int kernel = 0;           // 0 auto, 1 register-pipelined, 2 bulk-copy staged
  long long wait_cycles = lbmk::kWaitCycles;  // bound of the device waits
  // device pointers
  int32_t* flags = nullptr;
  int64_t* t_dev = nullptr;
  lbmk::Item* items_dev = nullptr;
  void* cases_dev = nullptr;
  double* part = nullptr;
  double* vol = nullptr;
  double* staging = nullptr;
  int64_t max_plane = 0;
  // reverse mode (lbm_adjoint_attach): caller-provided FP64 scratch
  char* adj_ws = nullptr;
  size_t adj_ws_bytes = 0;
};
