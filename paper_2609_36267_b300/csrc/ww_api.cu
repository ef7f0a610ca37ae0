// C-ABI entry points (include/ww.h): argument checks, the cost-table cache,
// workspaces and the whole-path orchestration.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "ww_internal.cuh"

namespace {

struct LutData {
  double nlooks = 0.0;
  int16_t table[ww::kNGamma * ww::kNAlpha];
  double cost100[ww::kNGamma * ww::kNAlpha];
  float ratio100[ww::kNGamma * ww::kNAlpha];  // 100 ln(P0/P+) for the interpolated lookup
  bool has_cost100 = false;
  bool has_ratio = false;
  std::mutex mu;
  int16_t* dev[64] = {nullptr};
  float* dev_ratio[64] = {nullptr};
  // page-locked copy of `table`, made once when the table is built (null where no
  // device is available); uploads from it are asynchronous and can be captured
  int16_t* pinned = nullptr;
  void make_pinned() {
    void* p = nullptr;
    if (cudaHostAlloc(&p, sizeof(table), cudaHostAllocDefault) == cudaSuccess) {
      std::memcpy(p, table, sizeof(table));
      pinned = static_cast<int16_t*>(p);
    } else {
      cudaGetLastError();
    }
  }
  ~LutData() {
    for (auto* p : dev)
      if (p) cudaFree(p);
    for (auto* p : dev_ratio)
      if (p) cudaFree(p);
    if (pinned) cudaFreeHost(pinned);
  }
};

std::mutex g_cache_mu;
std::map<uint64_t, std::shared_ptr<LutData>> g_cache;

uint64_t key_of(double L) {
  uint64_t k;
  std::memcpy(&k, &L, 8);
  return k;
}

std::shared_ptr<LutData>& data_of(const ww_lut* lut) {
  return *reinterpret_cast<std::shared_ptr<LutData>*>(lut->shared);
}

bool grid_ok(int64_t m, int64_t n) {
  return m >= 2 && n >= 2 && m <= (1ll << 30) && n <= (1ll << 30) && (m - 1) * (n - 1) < (1ll << 31) &&
         m * n < (1ll << 40);
}

bool params_ok(const ww_params* p) { return ww::params_valid(p); }

}  // namespace

bool ww::params_valid(const ww_params* p) {
  return p && (p->slope_estimator == 0 || p->slope_estimator == 1) && (p->cost_lookup == 0 || p->cost_lookup == 1) &&
         p->box_half_width >= 0 && p->box_half_width <= 3 && p->steep_cap_ppm >= 0 &&
         p->steep_cap_ppm <= 1000000 && p->max_passes > 0 && p->wait_polls > 0 && std::isfinite(p->steep_rad) &&
         (p->graph_loop == 0 || p->graph_loop == 1) && p->search_ctas_per_sm >= 0 && p->search_ctas_per_sm <= 64 &&
         p->band_min >= 1 && p->band_mult >= 0 && p->band_mult <= 1024 && p->band_growth >= 2 &&
         p->band_growth <= 64 && p->band_start_ppm >= 0 && p->band_start_ppm <= 1000000 && p->full_passes >= 0 &&
         p->ground_sink_below >= 0 && p->zero_stop_below >= 0 && p->zero_band_hops >= 1 && p->zero_band_hops_min >= 1;
}

namespace ww {

const int16_t* lut_device_table(const ww_lut* lut, cudaStream_t, ww_status* st) {
  auto& d = data_of(lut);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    *st = WW_ERR_CUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> g(d->mu);
  if (!d->dev[dev]) {
    int16_t* p = nullptr;
    if (cudaMalloc(&p, sizeof(d->table)) != cudaSuccess) {
      *st = WW_ERR_OOM;
      return nullptr;
    }
    if (cudaMemcpy(p, d->table, sizeof(d->table), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(p);
      *st = WW_ERR_CUDA;
      return nullptr;
    }
    d->dev[dev] = p;
  }
  *st = WW_OK;
  return d->dev[dev];
}

const float* lut_device_ratio(const ww_lut* lut, ww_status* st) {
  auto& d = data_of(lut);
  if (!d->has_ratio) {
    *st = WW_ERR_INVALID_ARG;
    return nullptr;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    *st = WW_ERR_CUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> g(d->mu);
  if (!d->dev_ratio[dev]) {
    float* p = nullptr;
    if (cudaMalloc(&p, sizeof(d->ratio100)) != cudaSuccess) {
      *st = WW_ERR_OOM;
      return nullptr;
    }
    if (cudaMemcpy(p, d->ratio100, sizeof(d->ratio100), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(p);
      *st = WW_ERR_CUDA;
      return nullptr;
    }
    d->dev_ratio[dev] = p;
  }
  *st = WW_OK;
  return d->dev_ratio[dev];
}

const int16_t* lut_host_table(const ww_lut* lut) { return data_of(lut)->table; }

const int16_t* lut_pinned_table(const ww_lut* lut) { return data_of(lut)->pinned; }

}  // namespace ww

extern "C" {

const char* ww_status_string(ww_status s) {
  switch (s) {
    case WW_OK: return "ok";
    case WW_ERR_INVALID_ARG: return "invalid argument";
    case WW_ERR_CUDA: return "CUDA error";
    case WW_ERR_OOM: return "out of memory";
    case WW_ERR_INFEASIBLE: return "infeasible: supplies cannot be routed within unit capacities";
    case WW_ERR_TIMEOUT: return "iteration limit reached";
    case WW_ERR_OVERFLOW: return "32-bit distance overflow";
    case WW_ERR_NOT_IMPLEMENTED: return "not implemented";
    case WW_ERR_INTERNAL: return "internal invariant violated";
    default: return "unknown status";
  }
}

void ww_params_default(ww_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->box_half_width = 2;
  p->steep_rad = 1.0f;
  p->steep_cap_ppm = 30000;
  p->max_passes = 100000;
  p->wait_polls = 1 << 25;
  p->graph_loop = 1;
  p->search_ctas_per_sm = 0;
  p->band_min = 1024;
  p->band_mult = 4;
  p->band_growth = 8;
  p->band_start_ppm = 1000000;
  p->full_passes = 0;
  p->ground_sink_below = 0;
  p->zero_stop_below = 64;
  p->zero_band_hops = 512;
  p->zero_band_hops_min = 512;
}

ww_status ww_build_lut(double nlooks, ww_lut** out) {
  if (!out || !(nlooks > 1.0) || !std::isfinite(nlooks)) return WW_ERR_INVALID_ARG;
  std::shared_ptr<LutData> d;
  {
    std::lock_guard<std::mutex> g(g_cache_mu);
    auto it = g_cache.find(key_of(nlooks));
    if (it != g_cache.end()) d = it->second;
  }
  if (!d) {
    auto nd = std::make_shared<LutData>();
    nd->nlooks = nlooks;
    int st = ww::lut_build_host(nlooks, nd->table, nd->cost100, nd->ratio100);
    if (st != WW_OK) return st;
    nd->has_cost100 = true;
    nd->has_ratio = true;
    nd->make_pinned();
    std::lock_guard<std::mutex> g(g_cache_mu);
    auto it = g_cache.find(key_of(nlooks));
    if (it != g_cache.end())
      d = it->second;
    else
      d = g_cache[key_of(nlooks)] = nd;
  }
  ww_lut* l = new (std::nothrow) ww_lut;
  if (!l) return WW_ERR_OOM;
  l->nlooks = nlooks;
  l->shared = new std::shared_ptr<LutData>(d);
  *out = l;
  return WW_OK;
}

ww_status ww_lut_from_table(double nlooks, const int16_t* host_table, ww_lut** out) {
  if (!out || !host_table || !(nlooks > 0.0)) return WW_ERR_INVALID_ARG;
  auto d = std::make_shared<LutData>();
  d->nlooks = nlooks;
  std::memcpy(d->table, host_table, sizeof(d->table));
  d->make_pinned();
  ww_lut* l = new (std::nothrow) ww_lut;
  if (!l) return WW_ERR_OOM;
  l->nlooks = nlooks;
  l->shared = new std::shared_ptr<LutData>(d);
  *out = l;
  return WW_OK;
}

ww_status ww_lut_from_tables(double nlooks, const int16_t* host_table, const float* ratio100, ww_lut** out) {
  if (!ratio100) return WW_ERR_INVALID_ARG;
  ww_status st = ww_lut_from_table(nlooks, host_table, out);
  if (st != WW_OK) return st;
  auto& d = data_of(*out);
  std::memcpy(d->ratio100, ratio100, sizeof(d->ratio100));
  d->has_ratio = true;
  return WW_OK;
}

ww_status ww_lut_ratio_table(const ww_lut* lut, float* ratio100) {
  if (!lut || !ratio100) return WW_ERR_INVALID_ARG;
  auto& d = data_of(lut);
  if (!d->has_ratio) return WW_ERR_INVALID_ARG;
  std::memcpy(ratio100, d->ratio100, sizeof(d->ratio100));
  return WW_OK;
}

ww_status ww_lut_table(const ww_lut* lut, int16_t* host_table, double* cost100) {
  if (!lut) return WW_ERR_INVALID_ARG;
  auto& d = data_of(lut);
  if (host_table) std::memcpy(host_table, d->table, sizeof(d->table));
  if (cost100) {
    if (!d->has_cost100) return WW_ERR_INVALID_ARG;
    std::memcpy(cost100, d->cost100, sizeof(d->cost100));
  }
  return WW_OK;
}

void ww_lut_free(ww_lut* lut) {
  if (!lut) return;
  delete reinterpret_cast<std::shared_ptr<LutData>*>(lut->shared);
  delete lut;
}

int64_t ww_workspace_bytes(int64_t m, int64_t n) {
  if (!grid_ok(m, n)) return -1;
  int64_t P = m * n, N = (m - 1) * (n - 1);
  // the potentials are the solver's own array (counted in solver_bytes)
  int64_t grid = N /*residues*/ + 4 * P * 2 /*costs*/ + 2 * P /*flows*/ + 64;
  int64_t steep = 65536 * 4 + 64 + ((2 * P + 1023) / 1024) * 4 + ww::steep_list_capacity(P, 30000) * 4;
  return grid + steep + 4 * P /*phase*/ + ww::solver_bytes(N, ww::tiles_for(m, n), 1);
}

ww_status ww_workspace_create(int64_t max_rows, int64_t max_cols, ww_workspace** out) {
  if (!out || !grid_ok(max_rows, max_cols)) return WW_ERR_INVALID_ARG;
  ww_workspace* ws = new (std::nothrow) ww_workspace;
  if (!ws) return WW_ERR_OOM;
  std::memset(ws, 0, sizeof(*ws));
  cudaGetDevice(&ws->device);
  ws->max_rows = max_rows;
  ws->max_cols = max_cols;
  const int64_t m = max_rows, n = max_cols, P = m * n, N = (m - 1) * (n - 1);
  ws->blocksum_len = (2 * P + 1023) / 1024;
  ws->steep_list_cap = ww::steep_list_capacity(P, 30000);  // the default 3% cap
  bool ok = cudaMalloc(&ws->residues, N) == cudaSuccess && cudaMalloc(&ws->ground, 64) == cudaSuccess &&
            cudaMalloc(&ws->costs, 4 * P * 2) == cudaSuccess && cudaMalloc(&ws->flows, 2 * P) == cudaSuccess &&
            cudaMalloc(&ws->total_cost, 64) == cudaSuccess && cudaMalloc(&ws->dev_status, 64) == cudaSuccess &&
            cudaMalloc(&ws->hist, 65536 * 4) == cudaSuccess && cudaMalloc(&ws->steep_ctr, 64) == cudaSuccess &&
            cudaMalloc(&ws->blocksum, ws->blocksum_len * 4) == cudaSuccess &&
            cudaMalloc(&ws->steep_list, ws->steep_list_cap * 4) == cudaSuccess &&
            cudaMalloc(&ws->psi, P * 4) == cudaSuccess;
  if (ok) ok = cudaMemset(ws->hist, 0, 65536 * 4) == cudaSuccess;
  ww_status st = ok ? ww::solver_alloc(&ws->sv, N, ww::tiles_for(m, n), 1) : WW_ERR_OOM;
  if (st != WW_OK) {
    cudaGetLastError();
    ww_workspace_free(ws);
    return st;
  }
  // the unwrap's potentials (N + 1, ground last) live in the solver's array
  ws->potentials = ws->sv.pot;
  *out = ws;
  return WW_OK;
}

void ww_workspace_free(ww_workspace* ws) {
  if (!ws) return;
  cudaFree(ws->residues);
  cudaFree(ws->ground);
  cudaFree(ws->costs);
  cudaFree(ws->flows);
  cudaFree(ws->total_cost);
  cudaFree(ws->dev_status);
  cudaFree(ws->hist);
  cudaFree(ws->steep_ctr);
  cudaFree(ws->blocksum);
  cudaFree(ws->steep_list);
  cudaFree(ws->psi);
  ww::solver_free(&ws->sv);
  delete ws;
}

static bool fits(const ww_workspace* ws, int64_t m, int64_t n) {
  return ws && m <= ws->max_rows && n <= ws->max_cols;
}

ww_status ww_residues(const void* ifg, int32_t is_complex, const float* coh, const uint8_t* mask, int64_t m,
                      int64_t n, int8_t* residues, int32_t* ground, ww_stream stream) {
  if (!ifg || !residues || !ground || !grid_ok(m, n)) return WW_ERR_INVALID_ARG;
  return ww::launch_residues(ifg, is_complex ? 1 : 0, coh, mask, m, n, residues, ground, (cudaStream_t)stream);
}

ww_status ww_costs(const void* ifg, int32_t is_complex, const float* coh, const uint8_t* mask, int64_t m, int64_t n,
                   const ww_lut* lut, const ww_params* params, ww_workspace* ws, int16_t* costs, ww_stream stream) {
  ww_params def;
  ww_params_default(&def);
  const ww_params* p = params ? params : &def;
  if (!ifg || !coh || !lut || !costs || !grid_ok(m, n) || !params_ok(p) || !fits(ws, m, n))
    return WW_ERR_INVALID_ARG;
  ww_status st;
  const int16_t* dt = ww::lut_device_table(lut, (cudaStream_t)stream, &st);
  if (!dt) return st;
  const float* dr = nullptr;
  if (p->cost_lookup == 1 && !(dr = ww::lut_device_ratio(lut, &st))) return st;
  return ww::launch_costs(ifg, is_complex ? 1 : 0, coh, mask, m, n, dt, dr, p, ws, costs, (cudaStream_t)stream);
}

ww_status ww_solve_mcf(const int8_t* residues, const int32_t* ground, const int16_t* costs, int64_t m, int64_t n,
                       const ww_params* params, ww_workspace* ws, int8_t* flows, int64_t* potentials,
                       int64_t* total_cost, int32_t* dev_status, ww_stream stream) {
  ww_params def;
  ww_params_default(&def);
  const ww_params* p = params ? params : &def;
  if (!residues || !ground || !costs || !flows || !potentials || !total_cost || !dev_status || !grid_ok(m, n) ||
      !params_ok(p) || !fits(ws, m, n))
    return WW_ERR_INVALID_ARG;
  ww::ProbHost ph{m, n, residues, ground, costs, flows, nullptr, total_cost, dev_status};
  return ww::solve_problems(&ph, 1, &ws->sv, p, potentials, &ws->stats, (cudaStream_t)stream);
}

ww_status ww_solve_mcf_resume(const int8_t* residues, const int32_t* ground, const int16_t* costs, int64_t m,
                              int64_t n, const ww_params* params, ww_workspace* ws, int8_t* flows,
                              int64_t* potentials, int64_t* total_cost, int32_t* dev_status, ww_stream stream) {
  ww_params def;
  ww_params_default(&def);
  const ww_params* p = params ? params : &def;
  if (!residues || !ground || !costs || !flows || !potentials || !total_cost || !dev_status || !grid_ok(m, n) ||
      !params_ok(p) || !fits(ws, m, n))
    return WW_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // the given pair must be a valid starting point: capacities, and no residual
  // arc of negative reduced cost (conservation is what the solve restores)
  int64_t* counts = ws->total_cost;  // 8 int64 of workspace scratch
  ww_status st = ww::launch_certificate(residues, ground, costs, flows, potentials, m, n, counts, s);
  if (st != WW_OK) return st;
  int64_t h[4] = {0, 0, 0, 0};
  WW_CUDA_TRY(cudaMemcpyAsync(h, counts, sizeof(h), cudaMemcpyDeviceToHost, s));
  WW_CUDA_TRY(cudaStreamSynchronize(s));
  if (h[0] != 0 || h[2] != 0) return WW_ERR_INVALID_ARG;
  ww::ProbHost ph{m, n, residues, ground, costs, flows, nullptr, total_cost, dev_status};
  ph.resume = true;
  return ww::solve_problems(&ph, 1, &ws->sv, p, potentials, &ws->stats, s);
}

ww_status ww_get_solve_stats(const ww_workspace* ws, ww_solve_stats* out) {
  if (!ws || !out) return WW_ERR_INVALID_ARG;
  *out = ws->stats;
  return WW_OK;
}

ww_status ww_integrate(const void* ifg, int32_t is_complex, const float* coh, const uint8_t* mask,
                       const int8_t* flows, int64_t m, int64_t n, float* unwrapped, int32_t* cycles,
                       ww_stream stream) {
  if (!ifg || !flows || !unwrapped || !cycles || !grid_ok(m, n)) return WW_ERR_INVALID_ARG;
  return ww::launch_integrate(ifg, is_complex ? 1 : 0, coh, mask, flows, m, n, unwrapped, cycles,
                              (cudaStream_t)stream);
}

ww_status ww_components(const int16_t* costs, const int8_t* flows, const float* unwrapped, int64_t m, int64_t n,
                        int32_t threshold, int32_t* labels, ww_stream stream) {
  if (!costs || !flows || !unwrapped || !labels || m < 1 || n < 1 || m > (1ll << 30) || n > (1ll << 30) ||
      m * n >= (1ll << 31) || threshold < 0)
    return WW_ERR_INVALID_ARG;
  return ww::launch_components(costs, flows, unwrapped, m, n, threshold, labels, (cudaStream_t)stream);
}

ww_status ww_unwrap(const void* ifg, int32_t is_complex, const float* coh, double nlooks, const uint8_t* mask,
                    int64_t m, int64_t n, const ww_params* params, ww_workspace* ws, float* unwrapped,
                    int32_t* cycles, int64_t* total_cost, ww_stream stream) {
  ww_params def;
  ww_params_default(&def);
  const ww_params* p = params ? params : &def;
  if (!ifg || !coh || !unwrapped || !cycles || !grid_ok(m, n) || !params_ok(p) || !fits(ws, m, n))
    return WW_ERR_INVALID_ARG;
  ww_lut* lut = nullptr;
  ww_status st = ww_build_lut(nlooks, &lut);
  if (st != WW_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int16_t* dt = ww::lut_device_table(lut, s, &st);
  const float* dr = nullptr;
  if (dt && p->cost_lookup == 1) dr = ww::lut_device_ratio(lut, &st);
  if (!dt || (p->cost_lookup == 1 && !dr)) {
    ww_lut_free(lut);
    return st;
  }
  int c = is_complex ? 1 : 0;
  const void* src = ifg;
  // validity inputs of the later steps: for a complex input the phase pass folds
  // the mask and the coherence test into the phase (NaN = invalid), so residues
  // and integration read the phase alone and the costs the phase and coherence
  const uint8_t* vmask = mask;
  const float* vcoh = coh;
  if (c) {
    st = ww::launch_phase(ifg, coh, mask, m, n, ws->psi, s);
    src = ws->psi;
    c = 0;
    vmask = nullptr;
    vcoh = nullptr;
  }
  // residues are computed inside the cost tiles (same pixels, one pass)
  if (st == WW_OK) WW_CUDA_TRY(cudaMemsetAsync(ws->ground, 0, sizeof(int32_t), s));
  if (st == WW_OK)
    st = ww::launch_costs(src, c, coh, vmask, m, n, dt, dr, p, ws, ws->costs, s, ws->residues, ws->ground);
  if (st == WW_OK) {
    ww::ProbHost ph{m, n, ws->residues, ws->ground, ws->costs, ws->flows, nullptr, ws->total_cost, ws->dev_status};
    st = ww::solve_problems(&ph, 1, &ws->sv, p, ws->potentials, &ws->stats, s);
  }
  ww_status st2 = ww::launch_integrate(src, c, vcoh, vmask, ws->flows, m, n, unwrapped, cycles, s);
  if (st == WW_OK) st = st2;
  if (total_cost && cudaMemcpyAsync(total_cost, ws->total_cost, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    st = WW_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) st = WW_ERR_CUDA;
  ww_lut_free(lut);
  return st;
}

ww_status ww_workspace_last_unwrap(const ww_workspace* ws, const int8_t** residues, const int32_t** ground,
                                   const int16_t** costs, const int8_t** flows, const int64_t** potentials) {
  if (!ws) return WW_ERR_INVALID_ARG;
  if (residues) *residues = ws->residues;
  if (ground) *ground = ws->ground;
  if (costs) *costs = ws->costs;
  if (flows) *flows = ws->flows;
  if (potentials) *potentials = ws->potentials;
  return WW_OK;
}

ww_status ww_certificate(const int8_t* residues, const int32_t* ground, const int16_t* costs, const int8_t* flows,
                         const int64_t* potentials, int64_t m, int64_t n, int64_t* counts, ww_stream stream) {
  if (!residues || !ground || !costs || !flows || !potentials || !counts || !grid_ok(m, n))
    return WW_ERR_INVALID_ARG;
  return ww::launch_certificate(residues, ground, costs, flows, potentials, m, n, counts, (cudaStream_t)stream);
}

}  // extern "C"

// ---------------- batched form ----------------
struct ww_batch {
  int device;
  int64_t max_items, max_pixels, max_item_pixels;
  ww::SolverWs sv;
  int8_t* residues;     // concatenated per item
  int32_t* ground;      // [max_items]
  int16_t* costs;       // [4 * max_pixels]
  int8_t* flows;        // [2 * max_pixels]
  int64_t* total_cost;  // [max_items]
  int32_t* status;      // [max_items]
  // item table of the batched grid launches
  ww::GridBatch grid;
  float* psi;  // phase of the complex items [max_pixels]
  // pinned copies of the per-item results (filled by the whole-batch graph)
  int64_t* h_total_cost;
  int32_t* h_status;
  ww_solve_stats stats;
};

namespace {

// The whole batch as ONE CUDA graph launch:
//   A (child graph): item table upload, residues, costs and steep rule of every
//     item, solver join (layout upload, per-problem initialisation);
//   B (conditional while node): forward + reverse passes until the device
//     finds nothing left to balance;
//   C (child graph): per-item totals and statuses, integration of every item,
//     copies of the results and solver counters into pinned host memory.
// Host-built tables sit in pinned staging that the host leaves untouched until
// the launch completes.  A and C both upload the grid item table; it is built
// once, before capture, so both copies carry the same content.
ww_status batch_graph(ww_batch* b, int64_t count, const ww_params* p, const std::vector<ww::ProbHost>& probs,
                      cudaStream_t s) {
  ww::Session S(&b->sv, b->sv.pot, b->sv.n_cap, p, s);
  if (S.err != WW_OK) return S.err;
  std::vector<int> all;
  int64_t node_off = 0, tile_off = 0;
  for (int64_t k = 0; k < count; ++k) {
    const int slot = S.add(probs[k], node_off, tile_off);
    if (slot != (int)k) return WW_ERR_INTERNAL;
    all.push_back(slot);
    node_off += (probs[k].m - 1) * (probs[k].n - 1);
    tile_off += ww::tiles_for(probs[k].m, probs[k].n);
  }
  S.set_ncand_unknown(true);
  cudaStream_t cs = nullptr;
  cudaGraph_t g = nullptr, ga = nullptr, gc = nullptr;
  cudaGraphExec_t ex = nullptr;
  cudaGraphNode_t na, nb, nc;
  ww_status e = WW_ERR_CUDA;
  auto capture = [&](cudaGraph_t* out, auto&& body) -> ww_status {
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return WW_ERR_CUDA;
    ww_status e1 = body();
    cudaGraph_t gr = nullptr;
    const bool ok = cudaStreamEndCapture(cs, &gr) == cudaSuccess;
    if (e1 != WW_OK || !ok) {
      if (gr) cudaGraphDestroy(gr);
      return e1 != WW_OK ? e1 : WW_ERR_CUDA;
    }
    *out = gr;
    return WW_OK;
  };
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return WW_ERR_CUDA;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) goto done;
  S.set_stream(cs);
  e = capture(&ga, [&] {
    ww_status e1 = ww::launch_pre_batch(&b->grid, (int)count, p, cs);
    return e1 == WW_OK ? S.commit() : e1;
  });
  if (e != WW_OK) goto done;
  e = WW_ERR_CUDA;
  if (cudaGraphAddChildGraphNode(&na, g, nullptr, 0, ga) != cudaSuccess) goto done;
  e = S.add_loop_node(g, &na, &nb);
  if (e != WW_OK) goto done;
  e = capture(&gc, [&] {
    ww_status e1 = S.finalize_enqueue(all);
    if (e1 == WW_OK) e1 = ww::launch_integrate_batch(&b->grid, (int)count, cs);
    if (e1 == WW_OK &&
        (cudaMemcpyAsync(b->h_total_cost, b->total_cost, count * 8, cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
         cudaMemcpyAsync(b->h_status, b->status, count * 4, cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
         cudaMemcpyAsync(b->sv.host_ctr, b->sv.ctr, S.ctr_bytes(), cudaMemcpyDeviceToHost, cs) != cudaSuccess))
      e1 = WW_ERR_CUDA;
    return e1;
  });
  if (e != WW_OK) goto done;
  e = WW_ERR_CUDA;
  if (cudaGraphAddChildGraphNode(&nc, g, &nb, 1, gc) != cudaSuccess) goto done;
  if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) goto done;
  if (cudaGraphLaunch(ex, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) goto done;
  b->stats = ww_solve_stats{};
  S.fill_stats(&b->stats);
  b->stats.residues = 0;
  e = WW_OK;
done:
  S.set_stream(s);
  if (ex) cudaGraphExecDestroy(ex);
  if (ga) cudaGraphDestroy(ga);
  if (gc) cudaGraphDestroy(gc);
  if (g) cudaGraphDestroy(g);
  if (cs) cudaStreamDestroy(cs);
  if (e != WW_OK) cudaGetLastError();
  return e;
}

}  // namespace

// Tiles of an m x n item: ceil((m-1)/32) ceil((n-1)/32) <= P/1024 + (m+n)/32 + 1, and
// m + n <= P/2 + 2 for m, n >= 2, so a batch needs at most P/1024 + P/64 + 2 per item.
static int64_t batch_tiles(int64_t items, int64_t pixels) { return pixels / 1024 + pixels / 64 + 4 * items + 64; }

extern "C" {

int64_t ww_batch_bytes(int64_t max_items, int64_t max_pixels, int64_t max_item_pixels) {
  if (max_items < 1 || max_pixels < 4 || max_item_pixels < 4) return -1;
  int64_t tiles = batch_tiles(max_items, max_pixels);
  return max_pixels * (1 + 8 + 2 + 4) + max_items * 16 + ww::grid_batch_bytes((int)max_items, max_pixels) +
         ww::solver_bytes(max_pixels, tiles, max_items);
}

ww_status ww_batch_create(int64_t max_items, int64_t max_pixels, int64_t max_item_pixels, ww_batch** out) {
  if (!out || max_items < 1 || max_pixels < 4 || max_item_pixels < 4 || max_item_pixels > max_pixels)
    return WW_ERR_INVALID_ARG;
  ww_batch* b = new (std::nothrow) ww_batch;
  if (!b) return WW_ERR_OOM;
  std::memset(b, 0, sizeof(*b));
  cudaGetDevice(&b->device);
  b->max_items = max_items;
  b->max_pixels = max_pixels;
  b->max_item_pixels = max_item_pixels;
  const int64_t tiles = batch_tiles(max_items, max_pixels);
  bool ok = cudaMalloc(&b->residues, max_pixels) == cudaSuccess &&
            cudaMalloc(&b->ground, max_items * 4) == cudaSuccess &&
            cudaMalloc(&b->costs, 4 * max_pixels * 2) == cudaSuccess &&
            cudaMalloc(&b->flows, 2 * max_pixels) == cudaSuccess &&
            cudaMalloc(&b->total_cost, max_items * 8) == cudaSuccess &&
            cudaMalloc(&b->status, max_items * 4) == cudaSuccess && cudaMalloc(&b->psi, max_pixels * 4) == cudaSuccess;
  if (ok) ok = ww::grid_batch_alloc(&b->grid, (int)max_items, max_pixels) == WW_OK;
  if (ok)
    ok = cudaMallocHost(&b->h_total_cost, max_items * 8) == cudaSuccess &&
         cudaMallocHost(&b->h_status, max_items * 4) == cudaSuccess;
  ww_status st = ok ? ww::solver_alloc(&b->sv, max_pixels, tiles, max_items) : WW_ERR_OOM;
  if (st != WW_OK) {
    cudaGetLastError();
    ww_batch_free(b);
    return st;
  }
  *out = b;
  return WW_OK;
}

void ww_batch_free(ww_batch* b) {
  if (!b) return;
  cudaFree(b->residues);
  cudaFree(b->ground);
  cudaFree(b->costs);
  cudaFree(b->flows);
  cudaFree(b->total_cost);
  cudaFree(b->status);
  cudaFree(b->psi);
  ww::grid_batch_free(&b->grid);
  cudaFreeHost(b->h_total_cost);
  cudaFreeHost(b->h_status);
  ww::solver_free(&b->sv);
  delete b;
}

ww_status ww_batch_stats(const ww_batch* b, ww_solve_stats* out) {
  if (!b || !out) return WW_ERR_INVALID_ARG;
  *out = b->stats;
  return WW_OK;
}

ww_status ww_unwrap_batch(ww_batch_item* items, int64_t count, const ww_params* params, ww_batch* b,
                          ww_stream stream) {
  ww_params def;
  ww_params_default(&def);
  const ww_params* p = params ? params : &def;
  if (!items || !b || count < 1 || count > b->max_items || !params_ok(p)) return WW_ERR_INVALID_ARG;
  int64_t tot = 0;
  for (int64_t k = 0; k < count; ++k) {
    const ww_batch_item& it = items[k];
    if (!it.ifg || !it.coh || !it.unwrapped || !it.cycles || !grid_ok(it.m, it.n) ||
        it.m * it.n > b->max_item_pixels)
      return WW_ERR_INVALID_ARG;
    tot += it.m * it.n;
  }
  if (tot > b->max_pixels) return WW_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // tables per number of looks (cached by the library)
  std::vector<ww_lut*> luts(count, nullptr);
  std::map<uint64_t, ww_lut*> by_l;
  ww_status st = WW_OK;
  for (int64_t k = 0; k < count && st == WW_OK; ++k) {
    uint64_t key = key_of(items[k].nlooks);
    auto it = by_l.find(key);
    if (it != by_l.end()) {
      luts[k] = it->second;
      continue;
    }
    ww_lut* l = nullptr;
    st = ww_build_lut(items[k].nlooks, &l);
    if (st == WW_OK) luts[k] = by_l[key] = l;
  }
  std::vector<ww::ProbHost> probs(count);
  int64_t off = 0;
  // phase timing under WW_TRACE: pre-solve kernels, solve, integration
  cudaEvent_t tev[4] = {nullptr, nullptr, nullptr, nullptr};
  const bool tr = ww::trace_enabled();
  if (tr)
    for (auto& e : tev) cudaEventCreate(&e);
  if (tr) cudaEventRecord(tev[0], s);
  int64_t filled = 0;
  for (int64_t k = 0; k < count && st == WW_OK; ++k) {
    const ww_batch_item& it = items[k];
    const int16_t* dt = ww::lut_device_table(luts[k], s, &st);
    if (!dt) break;
    const float* dr = nullptr;
    if (p->cost_lookup == 1 && !(dr = ww::lut_device_ratio(luts[k], &st))) break;
    ++filled;
    ww::ProbHost& ph = probs[k];
    ph.m = it.m;
    ph.n = it.n;
    ph.res = b->residues + off;
    ph.ground = b->ground + k;
    ph.costs = b->costs + 4 * off;
    ph.flows = b->flows + 2 * off;
    ph.pot_out = nullptr;
    ph.total_cost = b->total_cost + k;
    ph.status = b->status + k;
    ww::GridItem& g = b->grid.h_items[k];
    g = ww::GridItem{};
    g.ifg = it.ifg;
    g.coh = it.coh;
    g.mask = it.mask;
    g.m = it.m;
    g.n = it.n;
    g.is_complex = it.is_complex ? 1 : 0;
    if (g.is_complex) {
      // the phase once, into the batch's phase buffer; every step then reads it
      g.phase_src = it.ifg;
      g.ifg = b->psi + off;
      g.is_complex = 0;
    }
    g.res = const_cast<int8_t*>(ph.res);
    g.ground = const_cast<int32_t*>(ph.ground);
    g.costs = const_cast<int16_t*>(ph.costs);
    g.table = dt;
    g.ratio = dr;
    g.flows = ph.flows;
    g.unw = it.unwrapped;
    g.cyc = it.cycles;
    off += it.m * it.n;
  }
  if (st == WW_OK && p->graph_loop && !tr) {
    // one graph launch for the whole batch
    st = batch_graph(b, count, p, probs, s);
    for (int64_t k = 0; k < count; ++k) {
      items[k].total_cost = st == WW_OK ? b->h_total_cost[k] : 0;
      items[k].status = st == WW_OK ? b->h_status[k] : st;
    }
    for (auto& kv : by_l) ww_lut_free(kv.second);
    if (st != WW_OK) return st;
    for (int64_t k = 0; k < count; ++k)
      if (items[k].status != WW_OK) return items[k].status;
    return WW_OK;
  }
  if (st == WW_OK) st = ww::launch_pre_batch(&b->grid, (int)count, p, s);
  if (tr) cudaEventRecord(tev[1], s);
  if (st == WW_OK) st = ww::solve_problems(probs.data(), (int)count, &b->sv, p, nullptr, &b->stats, s);
  if (tr) cudaEventRecord(tev[2], s);
  if (filled == count) {
    // integration runs even after a solver failure (the caller's outputs are always written)
    ww_status s2 = ww::launch_integrate_batch(&b->grid, (int)count, s);
    if (st == WW_OK) st = s2;
  }
  std::vector<int64_t> tc(count);
  std::vector<int32_t> sts(count);
  if (tr) cudaEventRecord(tev[3], s);
  if (cudaMemcpyAsync(tc.data(), b->total_cost, count * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(sts.data(), b->status, count * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    st = st == WW_OK ? WW_ERR_CUDA : st;
  if (tr) {
    float a = 0, b2 = 0, c = 0;
    cudaEventElapsedTime(&a, tev[0], tev[1]);
    cudaEventElapsedTime(&b2, tev[1], tev[2]);
    cudaEventElapsedTime(&c, tev[2], tev[3]);
    std::fprintf(stderr, "[ww] batch %lld items: residues+costs %.3f ms, solve %.3f ms, integrate %.3f ms\n",
                 (long long)count, a, b2, c);
    for (auto& e : tev) cudaEventDestroy(e);
  }
  for (int64_t k = 0; k < count; ++k) {
    items[k].total_cost = tc[k];
    items[k].status = st == WW_OK ? sts[k] : st;
  }
  for (auto& kv : by_l) ww_lut_free(kv.second);
  return st;
}

}  // extern "C"
