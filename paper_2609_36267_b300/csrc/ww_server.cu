// Continuous-batching server (the served form): requests join a running
// multi-problem solve between passes and leave when balanced.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "ww_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

// FIFO ring allocator over [0, cap): ranges are handed out in order; a freed
// range is reclaimed once every range allocated before it is free too.
struct Ring {
  struct Range {
    int64_t off, len;
    bool freed;
  };
  int64_t cap = 0, head = 0;
  std::deque<Range> live;

  bool alloc(int64_t len, int64_t* off) {
    while (!live.empty() && live.front().freed) live.pop_front();
    if (len > cap) return false;
    if (live.empty()) {
      head = 0;
      *off = 0;
      head = len;
      live.push_back({0, len, false});
      return true;
    }
    int64_t tail = live.front().off;
    int64_t o = -1;
    if (head >= tail) {
      if (head + len <= cap) o = head;
      else if (len <= tail) o = 0;
    } else if (head + len <= tail) {
      o = head;
    }
    if (o < 0) return false;
    head = o + len;
    live.push_back({o, len, false});
    *off = o;
    return true;
  }
  void release(int64_t off) {
    for (auto& r : live)
      if (r.off == off && !r.freed) {
        r.freed = true;
        break;
      }
    while (!live.empty() && live.front().freed) live.pop_front();
  }
};

struct Request {
  int64_t ticket;
  ww_batch_item item;
  Clock::time_point t_submit, t_done;
  bool done = false;
  int slot = -1;
  int64_t pix_off = 0, node_off = 0, tile_off = 0;
  ww_lut* lut = nullptr;
};

// Device bytes a server with room for `pixels` pixels of requests in flight
// allocates: per pixel residues 1, costs 8, flows 2, phase 4; per request slot
// ground, total cost and status; the grid-batch tables (item table, steep
// counters, selection histograms, tie counts, candidate lists); the solver
// state (nodes, tiles, problems).  Every cudaMalloc of ww_server_create is counted.
int64_t server_tiles(int64_t pixels, int32_t max_active) { return pixels / 1024 + pixels / 64 + 4 * max_active + 64; }
int64_t server_bytes(int64_t pixels, int32_t max_active) {
  return pixels * (1 + 8 + 2 + 4) + (int64_t)max_active * (4 + 8 + 4) + ww::grid_batch_bytes(max_active, pixels) +
         ww::solver_bytes(pixels, server_tiles(pixels, max_active), max_active);
}

}  // namespace

struct ww_server {
  ww_server_config cfg;
  ww_params prm;
  int device = 0;
  cudaStream_t stream = nullptr;
  ww::SolverWs sv;
  int8_t* residues = nullptr;
  int16_t* costs = nullptr;
  int8_t* flows = nullptr;
  float* psi = nullptr;  // phase of complex requests, by pixel range
  int32_t* ground = nullptr;
  int64_t* total_cost = nullptr;
  int32_t* status = nullptr;
  ww::GridBatch grid;  // item tables of the batched grid launches (admission, retirement)
  Ring pix, node, tile;
  ww::Session* session = nullptr;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv, done_cv;
  std::deque<Request*> waiting;
  const Request* head_blocked = nullptr;  // the queue's head while it does not fit
  int head_rounds = 0;                    // worker rounds it has waited for room
  std::map<int64_t, Request*> tickets;
  std::vector<Request*> by_slot;
  int64_t next_ticket = 1;
  bool stop = false;
  ww_server_stats stats{};
  ww_status fatal = WW_OK;
  int64_t resident_bytes = 0;  // device bytes allocated at creation (all of it counted against the budget)
};

namespace {

bool admit_one(ww_server* S, Request* r) {
  const ww_batch_item& it = r->item;
  const int64_t P = it.m * it.n, N = (it.m - 1) * (it.n - 1), T = ww::tiles_for(it.m, it.n);
  int64_t po, no, to;
  if (!S->pix.alloc(P, &po)) return false;
  if (!S->node.alloc(N, &no)) {
    S->pix.release(po);
    return false;
  }
  if (!S->tile.alloc(T, &to)) {
    S->pix.release(po);
    S->node.release(no);
    return false;
  }
  r->pix_off = po;
  r->node_off = no;
  r->tile_off = to;
  return true;
}

void release_ranges(ww_server* S, Request* r) {
  S->pix.release(r->pix_off);
  S->node.release(r->node_off);
  S->tile.release(r->tile_off);
}

void fail_request(ww_server* S, Request* r, ww_status st) {
  std::lock_guard<std::mutex> g(S->mu);
  r->item.status = st;
  r->item.total_cost = 0;
  r->done = true;
  r->t_done = Clock::now();
  S->stats.completed++;
  S->done_cv.notify_all();
}

void worker_loop(ww_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t s = S->stream;
  const int max_slots = (int)S->sv.p_cap;
  S->by_slot.assign(max_slots, nullptr);
  int active = 0;
  for (;;) {
    std::vector<Request*> admitted;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] { return S->stop || !S->waiting.empty() || active > 0; });
      if (S->stop && S->waiting.empty() && active == 0) break;
      // Admission in arrival order against the rings and the slot limit.  A
      // request that does not fit yet lets up to kAdmitLookahead later ones that
      // do fit pass it; once the head has waited kHeadPatience rounds nothing
      // passes it until the requests in flight free its room.
      constexpr int kAdmitLookahead = 64, kHeadPatience = 16;
      const int limit = std::min<int>(max_slots, S->cfg.max_active);
      size_t k = 0;
      int skipped = 0;
      while (k < S->waiting.size() && active + (int)admitted.size() < limit) {
        Request* r = S->waiting[k];
        if (admit_one(S, r)) {
          S->waiting.erase(S->waiting.begin() + (std::ptrdiff_t)k);
          admitted.push_back(r);
          if (k == 0) {
            S->head_blocked = nullptr;
            S->head_rounds = 0;
          }
          continue;
        }
        if (k == 0) {
          if (S->head_blocked != r) {
            S->head_blocked = r;
            S->head_rounds = 0;
          }
          if (++S->head_rounds > kHeadPatience) break;
        }
        if (++skipped > kAdmitLookahead) break;
        ++k;
      }
    }
    auto t_busy = Clock::now();
    // residues and costs of every admitted request in one set of launches
    int nq = 0;
    std::vector<Request*> joined;
    for (Request* r : admitted) {
      const ww_batch_item& it = r->item;
      ww_status st = ww_build_lut(it.nlooks, &r->lut);
      const int16_t* dt = st == WW_OK ? ww::lut_device_table(r->lut, s, &st) : nullptr;
      const float* dr = (dt && S->prm.cost_lookup == 1) ? ww::lut_device_ratio(r->lut, &st) : nullptr;
      const int slot0 = S->session->next_slot();
      if (!dt || (S->prm.cost_lookup == 1 && !dr) || slot0 < 0) {
        release_ranges(S, r);
        fail_request(S, r, st != WW_OK ? st : WW_ERR_INTERNAL);
        continue;
      }
      int8_t* res = S->residues + r->pix_off;
      int16_t* cst = S->costs + 4 * r->pix_off;
      int8_t* fl = S->flows + 2 * r->pix_off;
      // per-slot ground charge, total cost and status words
      ww::ProbHost ph{it.m, it.n, res, S->ground + slot0, cst, fl, nullptr, S->total_cost + slot0, S->status + slot0};
      const int slot = S->session->add(ph, r->node_off, r->tile_off);
      if (slot != slot0) {
        if (slot >= 0) S->session->remove(slot);
        release_ranges(S, r);
        fail_request(S, r, WW_ERR_INTERNAL);
        continue;
      }
      ww::GridItem& g = S->grid.h_items[nq++];
      g = ww::GridItem{};
      g.ifg = it.ifg;
      g.coh = it.coh;
      g.mask = it.mask;
      g.m = it.m;
      g.n = it.n;
      g.is_complex = it.is_complex ? 1 : 0;
      if (g.is_complex) {
        g.phase_src = it.ifg;
        g.ifg = S->psi + r->pix_off;
        g.is_complex = 0;
      }
      g.res = res;
      g.ground = S->ground + slot;
      g.costs = cst;
      g.table = dt;
      g.ratio = dr;
      r->slot = slot;
      joined.push_back(r);
    }
    ww_status pre = nq > 0 ? ww::launch_pre_batch(&S->grid, nq, &S->prm, s) : WW_OK;
    for (Request* r : joined) {
      if (pre != WW_OK) {
        S->session->remove(r->slot);
        release_ranges(S, r);
        fail_request(S, r, pre);
        continue;
      }
      S->by_slot[r->slot] = r;
      ++active;
      std::lock_guard<std::mutex> g(S->mu);
      S->stats.admitted++;
      S->stats.peak_active = std::max<int64_t>(S->stats.peak_active, active);
    }
    ww_status st = S->session->commit();
    std::vector<int32_t> left;
    if (st == WW_OK) st = S->session->left(&left);
    bool work = false;
    for (int k = 0; k < max_slots && st == WW_OK; ++k)
      if (S->by_slot[k] && left[k] > 0) work = true;
    if (st == WW_OK && work) {
      ww_solve_stats ps{};
      st = S->session->pass(&ps);
      if (st == WW_OK && S->session->status() != WW_OK) st = S->session->status();
      if (st == WW_OK) st = S->session->left(&left);
      std::lock_guard<std::mutex> g(S->mu);
      S->stats.passes++;
    }
    // retire balanced requests (or everything on a solver failure)
    std::vector<int> fin;
    for (int k = 0; k < max_slots; ++k)
      if (S->by_slot[k] && (st != WW_OK || left[k] == 0)) fin.push_back(k);
    if (!fin.empty()) {
      std::vector<int32_t> sts;
      ww_status fs = S->session->finalize(fin, &sts);
      // integration of every finished request in one set of launches
      for (size_t q = 0; q < fin.size(); ++q) {
        Request* r = S->by_slot[fin[q]];
        const ww_batch_item& it = r->item;
        ww::GridItem& g = S->grid.h_items[q];
        g = ww::GridItem{};
        g.ifg = it.ifg;
        g.coh = it.coh;
        g.mask = it.mask;
        g.m = it.m;
        g.n = it.n;
        g.is_complex = it.is_complex ? 1 : 0;
        if (g.is_complex) {  // the phase computed on admission
          g.ifg = S->psi + r->pix_off;
          g.is_complex = 0;
        }
        g.flows = S->flows + 2 * r->pix_off;
        g.unw = it.unwrapped;
        g.cyc = it.cycles;
      }
      ww_status is = ww::launch_integrate_batch(&S->grid, (int)fin.size(), s);
      std::vector<int64_t> tcs(max_slots, 0);
      if (cudaMemcpyAsync(tcs.data(), S->total_cost, 8 * (size_t)max_slots, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        is = is == WW_OK ? WW_ERR_CUDA : is;
      for (size_t q = 0; q < fin.size(); ++q) {
        Request* r = S->by_slot[fin[q]];
        ww_status rs = st != WW_OK ? st : (fs != WW_OK ? fs : (is != WW_OK ? is : sts[q]));
        S->session->remove(fin[q]);
        S->by_slot[fin[q]] = nullptr;
        --active;
        release_ranges(S, r);
        ww_lut_free(r->lut);
        r->lut = nullptr;
        std::lock_guard<std::mutex> g(S->mu);
        r->item.status = rs;
        r->item.total_cost = tcs[fin[q]];
        r->done = true;
        r->t_done = Clock::now();
        S->stats.completed++;
      }
      S->done_cv.notify_all();
      if (st != WW_OK) {
        // a failed solve ends this session; start a clean one for later requests
        delete S->session;
        S->session = new ww::Session(&S->sv, S->sv.pot, S->sv.n_cap, &S->prm, s);
      }
    }
    std::lock_guard<std::mutex> g(S->mu);
    S->stats.busy_ms += std::chrono::duration<double, std::milli>(Clock::now() - t_busy).count();
  }
}

}  // namespace

extern "C" {

ww_status ww_server_create(const ww_server_config* cfg, const ww_params* params, ww_server** out) {
  if (!cfg || !out || cfg->hbm_budget_bytes < (1 << 20) || cfg->max_request_pixels < 4 || cfg->max_active < 1 ||
      (params && !ww::params_valid(params)))
    return WW_ERR_INVALID_ARG;
  ww_server* S = new (std::nothrow) ww_server;
  if (!S) return WW_ERR_OOM;
  S->cfg = *cfg;
  ww_params_default(&S->prm);
  if (params) S->prm = *params;
  S->prm.max_passes = 1 << 30;
  cudaGetDevice(&S->device);
  // the largest pixel pool whose whole allocation fits the budget; a budget that
  // cannot hold one request of the largest accepted size is refused
  const int64_t cap_px = (1ll << 31) - (1ll << 22);
  if (cfg->max_request_pixels > cap_px || server_bytes(cfg->max_request_pixels, cfg->max_active) > cfg->hbm_budget_bytes) {
    delete S;
    return WW_ERR_INVALID_ARG;
  }
  int64_t lo = cfg->max_request_pixels, hi = std::min<int64_t>(cap_px, cfg->hbm_budget_bytes / 15);
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo + 1) / 2;
    if (server_bytes(mid, cfg->max_active) <= cfg->hbm_budget_bytes)
      lo = mid;
    else
      hi = mid - 1;
  }
  const int64_t pixels = lo;
  const int64_t tiles = server_tiles(pixels, cfg->max_active);
  S->resident_bytes = server_bytes(pixels, cfg->max_active);
  S->pix.cap = pixels;
  S->node.cap = pixels;
  S->tile.cap = tiles;
  bool ok = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMalloc(&S->residues, pixels) == cudaSuccess && cudaMalloc(&S->costs, 8 * pixels) == cudaSuccess &&
            cudaMalloc(&S->flows, 2 * pixels) == cudaSuccess && cudaMalloc(&S->psi, 4 * pixels) == cudaSuccess &&
            cudaMalloc(&S->ground, 4 * (int64_t)cfg->max_active) == cudaSuccess &&
            cudaMalloc(&S->total_cost, 8 * (int64_t)cfg->max_active) == cudaSuccess &&
            cudaMalloc(&S->status, 4 * (int64_t)cfg->max_active) == cudaSuccess &&
            ww::grid_batch_alloc(&S->grid, (int)cfg->max_active, pixels) == WW_OK;
  ww_status st = ok ? ww::solver_alloc(&S->sv, pixels, tiles, cfg->max_active) : WW_ERR_OOM;
  if (st != WW_OK) {
    cudaGetLastError();
    S->stop = true;
    ww_server_destroy(S);
    return st;
  }
  S->session = new ww::Session(&S->sv, S->sv.pot, S->sv.n_cap, &S->prm, S->stream);
  S->worker = std::thread(worker_loop, S);
  *out = S;
  return WW_OK;
}

ww_status ww_server_submit(ww_server* S, const ww_batch_item* req, int64_t* ticket) {
  if (!S || !req || !ticket) return WW_ERR_INVALID_ARG;
  const ww_batch_item& it = *req;
  std::lock_guard<std::mutex> g(S->mu);
  S->stats.submitted++;
  const int64_t P = it.m * it.n;
  if (!it.ifg || !it.coh || !it.unwrapped || !it.cycles || it.m < 2 || it.n < 2 || !(it.nlooks > 1.0) ||
      P > S->cfg.max_request_pixels || P > S->pix.cap || ww::tiles_for(it.m, it.n) > S->tile.cap) {
    S->stats.rejected++;
    return WW_ERR_INVALID_ARG;
  }
  Request* r = new Request;
  r->ticket = S->next_ticket++;
  r->item = it;
  r->t_submit = Clock::now();
  S->tickets[r->ticket] = r;
  S->waiting.push_back(r);
  *ticket = r->ticket;
  S->cv.notify_all();
  return WW_OK;
}

static void fill_result(const Request* r, ww_batch_item* result, double* latency_ms) {
  if (result) {
    result->total_cost = r->item.total_cost;
    result->status = r->item.status;
  }
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
}

ww_status ww_server_poll(ww_server* S, int64_t ticket, int32_t* done, ww_batch_item* result, double* latency_ms) {
  if (!S || !done) return WW_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) return WW_ERR_INVALID_ARG;
  *done = it->second->done ? 1 : 0;
  if (it->second->done) fill_result(it->second, result, latency_ms);
  return WW_OK;
}

ww_status ww_server_wait(ww_server* S, int64_t ticket, double timeout_ms, ww_batch_item* result, double* latency_ms) {
  if (!S) return WW_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) return WW_ERR_INVALID_ARG;
  Request* r = it->second;
  bool ok = S->done_cv.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), [&] { return r->done; });
  if (!ok) return WW_ERR_TIMEOUT;
  fill_result(r, result, latency_ms);
  return WW_OK;
}

ww_status ww_server_release(ww_server* S, int64_t ticket) {
  if (!S) return WW_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end() || !it->second->done) return WW_ERR_INVALID_ARG;
  delete it->second;
  S->tickets.erase(it);
  return WW_OK;
}

ww_status ww_server_get_stats(ww_server* S, ww_server_stats* out) {
  if (!S || !out) return WW_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(S->mu);
  *out = S->stats;
  out->peak_resident_bytes = S->resident_bytes;
  return WW_OK;
}

void ww_server_destroy(ww_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stop = true;
    S->cv.notify_all();
  }
  if (S->worker.joinable()) S->worker.join();
  delete S->session;
  for (auto& kv : S->tickets) delete kv.second;
  cudaFree(S->residues);
  cudaFree(S->costs);
  cudaFree(S->flows);
  cudaFree(S->psi);
  cudaFree(S->ground);
  cudaFree(S->total_cost);
  cudaFree(S->status);
  ww::grid_batch_free(&S->grid);
  if (S->sv.n_cap) ww::solver_free(&S->sv);
  if (S->stream) cudaStreamDestroy(S->stream);
  delete S;
}

}  // extern "C"
