// MCF solve (Sec. II-A Eq. 2) by successive shortest paths with node
// potentials and parallel augmentation (Sec. II-C).
//
// State: per pixel edge the cycle difference dk in {-1,0,1} (two unit arcs per
// edge; dk = x(a) - x(a-bar)), per node its imbalance and an int64 potential p.
// The residual arcs across an edge are: in the "+" direction (the arc that
// raises dk) cost c+ if dk = 0, -c- if dk = -1 (cancelling), none if dk = +1;
// in the "-" direction cost c- if dk = 0, -c+ if dk = +1, none if dk = -1.
// Reduced cost c - p(tail) + p(head) stays >= 0 on every residual arc.
//
// One pass:
//   search   multi-root shortest-path forest over reduced costs.  Forward
//            passes grow from every excess node and from the ground node G;
//            reverse passes grow backwards from every deficit node and from G.
//            Labels pack (distance:32 | hops:29 | direction:3); the minimum
//            label is unique, so the forest is deterministic, and the hop
//            count breaks zero-cost ties in breadth-first order (the paper's
//            FIFO tie-break).  The search is label-correcting over 32x32 node
//            tiles held in shared memory; a worklist of tiles whose halo
//            changed drives it to the fixed point (exact distances).
//   select   every candidate (deficit in forward passes, excess node in
//            reverse passes) walks to its tree root; each tree keeps its
//            nearest candidate (atomicMin on distance, then node id).
//   augment  one unit along each tree path (trees are node-disjoint, so
//            paths share no arc); G may end or start any number of them,
//            since the ring it stands for is uncapacitated and free.
//   update   p += D - d (forward) or p -= D - d (reverse) for nodes with
//            d < D, D the largest augmented distance: every tree arc used
//            becomes tight, every residual arc stays non-negative.
// G's own balance is implied by the others (the supplies sum to zero), so
// treating it as a free source/sink keeps the optimum of Eq. 2.
#include <cuda_runtime.h>

#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "ww_internal.cuh"

namespace ww {

constexpr int TS = 32;         // tile side in nodes
constexpr int TSH = TS + 2;    // with halo
constexpr int SEARCH_THREADS = 256;
constexpr int kMaxLocalSweeps = 8192;
constexpr int kMaxSearchGrid = 148 * 64;  // ring slack: at most one outstanding ticket per CTA

enum : int32_t { kErrOverflow = 1, kErrInternal = 2, kErrWalk = 4, kErrSpin = 8 };

struct McfCtr {
  int32_t list_count[2];
  uint32_t D;
  int32_t naug;
  int32_t ncand;
  int32_t ncand_next;
  int32_t err;
  int32_t pad;
  long long g_net;
  unsigned long long tile_visits;
  long long total_cost;
  unsigned long long local_rounds;
  unsigned long long visit_cycles;
  int32_t found;       // candidates reached by the current search
  int32_t capped_any;  // a tile discarded a candidate at or beyond the cap
};

namespace {

struct Grid {
  int64_t m, n, R, C, N, P;  // pixel rows/cols, node rows/cols, nodes, pixels
  int tiles_x, tiles_y;
};

// Raw residual cost of the arc entering node (i,j) from direction dir (forward
// search: arc u->v) or leaving it toward dir (reverse search: arc v->u).
// Returns false if the arc does not exist.
template <bool FWD>
__device__ __forceinline__ bool arc_cost(const int16_t* __restrict__ costs, const int8_t* __restrict__ flows,
                                         const Grid& g, int64_t i, int64_t j, int dir, int32_t* cost) {
  const int64_t P = g.P;
  int64_t e;
  int plane;        // 0: h edge, 1: v edge
  bool plus;        // move raises dk
  switch (dir) {
    case kDirUp: e = i * g.n + j; plane = 0; plus = FWD; break;
    case kDirDown: e = (i + 1) * g.n + j; plane = 0; plus = !FWD; break;
    case kDirLeft: e = i * g.n + j; plane = 1; plus = !FWD; break;
    default: e = i * g.n + j + 1; plane = 1; plus = FWD; break;
  }
  int dk = flows[plane * P + e];
  int32_t cp = costs[(2 * plane) * P + e], cm = costs[(2 * plane + 1) * P + e];
  if (plus) {
    if (dk > 0) return false;
    *cost = dk == 0 ? cp : -cm;
  } else {
    if (dk < 0) return false;
    *cost = dk == 0 ? cm : -cp;
  }
  return true;
}

__device__ __forceinline__ int64_t nb_node(const Grid& g, int64_t i, int64_t j, int dir) {
  switch (dir) {
    case kDirUp: return i > 0 ? (i - 1) * g.C + j : -1;
    case kDirDown: return i + 1 < g.R ? (i + 1) * g.C + j : -1;
    case kDirLeft: return j > 0 ? i * g.C + j - 1 : -1;
    default: return j + 1 < g.C ? i * g.C + j + 1 : -1;
  }
}

// ---- tile worklist shared by all CTAs of one persistent search launch ----
// Producers reserve ring positions with atomicAdd(tail) and then publish the
// tile in that slot; consumers take tickets with atomicAdd(head) and wait for
// their slot to be published.  A tile is queued at most once at a time (flag
// `inq`), and at most one ticket per CTA is outstanding, so a ring of
// tiles + CTAs slots never wraps onto an unconsumed entry.  `pending` counts
// tiles queued or in process; it is decremented only after a tile's
// neighbours have been queued, so it reaches zero exactly at convergence, and
// a consumer whose slot is still empty then leaves.
struct SearchQ {
  int32_t head, tail, pending, pad;
};

constexpr int kSpinLimit = 1 << 25;  // idle polls (~100 ns each) before giving up

__device__ __forceinline__ int ld_volatile(const int32_t* p) { return *((volatile const int32_t*)p); }

// Returns false if the slot stayed occupied past the wait limit (reported as an error).
__device__ __forceinline__ bool q_push(int tile, int ring, SearchQ* q, int32_t* slots, int32_t* inq) {
  if (atomicExch(&inq[tile], 1) != 0) return true;
  atomicAdd(&q->pending, 1);
  int pos = atomicAdd(&q->tail, 1);
  __threadfence();
  int* slot = &slots[pos % ring];
  for (int spin = 0; spin < kSpinLimit; ++spin) {
    if (atomicCAS(slot, 0, tile + 1) == 0) return true;
    __nanosleep(100);
  }
  return false;
}

// Returns a tile, -1 when the search has converged, -2 on a bounded-wait timeout.
__device__ int q_pop(int ring, SearchQ* q, int32_t* slots, int32_t* inq) {
  const int h = atomicAdd(&q->head, 1);
  int* slot = &slots[h % ring];
  for (int spin = 0; spin < kSpinLimit; ++spin) {
    int v = ld_volatile(slot);
    if (v != 0) {
      atomicExch(slot, 0);
      atomicExch(&inq[v - 1], 0);
      __threadfence();
      return v - 1;
    }
    if (ld_volatile(&q->pending) == 0) return -1;
    __nanosleep(spin < 64 ? 20 : 200);
  }
  return -2;
}

constexpr uint64_t KINF = kInf >> 3;                  // (distance, hops) part of an unreached label
constexpr uint64_t KDIST_INF = 0xFFFFFFFFull << 29;   // distance field all ones

__device__ __forceinline__ uint64_t sat_add(uint64_t a, uint64_t b) {
  uint64_t s = a + b;  // a, b <= KINF < 2^61: no wrap
  return s < KINF ? s : KINF;
}

__device__ __forceinline__ uint64_t arc_weight(uint32_t w) {
  return w == kNoArc ? KINF : (((uint64_t)w << 29) + 1ull);  // +w distance, +1 hop
}

// Segmented directional min-plus scan over four 32-cell lines per warp.
// Lane = 8*line + seg; seg owns cells 4*seg .. 4*seg+3 of its line (in scan
// order when forward, mirrored when backward).  For one line with cells k in
// scan order, labels K_k (distance,hops) and entering-arc weights b_k:
//   c_k = min(K_k, c_{k-1} + b_k),  c_{-1} = halo,
// computed as a sequential pass inside each segment, an exclusive scan of the
// segment aggregates (A, B) across the 8 segments (operator
// (A1,B1).(A2,B2) = (min(A2, A1+B2), B1+B2)), and a sequential fix-up that
// offers every cell the candidate from its predecessor (direction code dir).
// `cell(k)` / `wt(k)` address the lane's k-th cell in scan order.
template <bool FORWARD, class CellF, class WtF>
__device__ __forceinline__ unsigned scan_segments(CellF cell, WtF wt, uint64_t halo_key, int dir, int seg,
                                                  uint64_t capK, bool* capped, int* err) {
  uint64_t K[4], b[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    K[k] = *cell(k) >> 3;
    b[k] = arc_weight(wt(k));
  }
  uint64_t A = K[0], B = b[0];
#pragma unroll
  for (int k = 1; k < 4; ++k) {
    A = min(K[k], sat_add(A, b[k]));
    B = sat_add(B, b[k]);
  }
  const uint64_t h = halo_key >> 3;
  const bool first = FORWARD ? seg == 0 : seg == 7;
  if (first) A = min(A, sat_add(h, B));
#pragma unroll
  for (int off = 1; off < 8; off <<= 1) {
    uint64_t Ap = FORWARD ? __shfl_up_sync(0xffffffffu, A, off, 8) : __shfl_down_sync(0xffffffffu, A, off, 8);
    uint64_t Bp = FORWARD ? __shfl_up_sync(0xffffffffu, B, off, 8) : __shfl_down_sync(0xffffffffu, B, off, 8);
    bool has = FORWARD ? seg >= off : seg + off < 8;
    if (has) {
      A = min(A, sat_add(Ap, B));
      B = sat_add(Bp, B);
    }
  }
  uint64_t cin = FORWARD ? __shfl_up_sync(0xffffffffu, A, 1, 8) : __shfl_down_sync(0xffffffffu, A, 1, 8);
  if (first) cin = h;
  unsigned changed = 0;
  uint64_t prev = cin;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    uint64_t cand = sat_add(prev, b[k]);
    uint64_t cur = K[k];
    if (cand < KINF) {
      if (cand >= KDIST_INF) {
        *err |= kErrOverflow;
      } else if (cand >= capK) {
        // beyond this search's distance band: dropped, the tile is re-seeded
        // if the band is widened
        if (cand < cur) *capped = true;
      } else {
        uint64_t* c = cell(k);
        uint64_t key = (cand << 3) | (uint64_t)dir;
        if (key < *c) {
          *c = key;
          changed |= 1u << k;
        }
        cur = min(cur, cand);
      }
    }
    prev = cur;
  }
  return changed;  // bit k: the lane's k-th cell (scan order) improved
}

constexpr int LROW = TS + 3;  // padded row stride of the label tile (halo 1 each side + 1 pad)
constexpr int RCOL = TS + 1;  // padded row stride of the arc-weight planes

template <bool FWD>
__global__ void __launch_bounds__(SEARCH_THREADS) k_search(Grid g, const int16_t* __restrict__ costs,
                                                           const int8_t* __restrict__ flows,
                                                           const int64_t* __restrict__ pot, uint64_t* labels,
                                                           SearchQ* q, int32_t* slots, int32_t* inq, McfCtr* ctr,
                                                           uint64_t capK, int32_t* capped_flag) {
  __shared__ uint64_t lab[TSH][LROW];
  __shared__ uint32_t rc[4][TS][RCOL];
  __shared__ int side[4];
  __shared__ int s_tile;
  __shared__ unsigned rowdirty, coldirty, rowdirty_next, coldirty_next;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;  // 8 warps
  const int ring = g.tiles_x * g.tiles_y + (int)gridDim.x + 64;
  const int64_t pG = pot[g.N];
  int err = 0;
  if (tid == 0) {
    rowdirty_next = 0;
    coldirty_next = 0;
  }
  for (;;) {
    if (tid == 0) s_tile = q_pop(ring, q, slots, inq);
    __syncthreads();
    const int tile = s_tile;
    if (tile < 0) {
      if (tid == 0 && tile == -2) atomicOr(&ctr->err, kErrSpin);
      break;
    }
    const int64_t ti = tile / g.tiles_x, tj = tile % g.tiles_x;
    const int64_t i0 = ti * TS, j0 = tj * TS;
    if (tid < 4) side[tid] = 0;
    const long long t_start = clock64();
    // labels with halo; directly outside the grid stands G, a root (label 0)
    for (int qd = tid; qd < TSH * TSH; qd += SEARCH_THREADS) {
      int r = qd / TSH, c = qd % TSH;
      int64_t i = i0 + r - 1, j = j0 + c - 1;
      uint64_t v;
      if (i < 0 || j < 0 || i >= g.R || j >= g.C) {
        bool ring = (i >= -1 && i <= g.R && j >= -1 && j <= g.C);
        v = ring ? 0ull : kInf;
      } else {
        v = *((volatile const uint64_t*)&labels[i * g.C + j]);
      }
      lab[r][c] = v;
    }
    // reduced costs of the four arcs of every node (row = warp + 8k, col = lane)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int ly = warp + 8 * k;
      int64_t i = i0 + ly, j = j0 + lane;
      bool ex = i < g.R && j < g.C;
      int64_t pv = ex ? pot[i * g.C + j] : 0;
#pragma unroll
      for (int d = 1; d <= 4; ++d) {
        uint32_t r = kNoArc;
        int32_t c;
        if (ex && arc_cost<FWD>(costs, flows, g, i, j, d, &c)) {
          int64_t u = nb_node(g, i, j, d);
          int64_t pu = u >= 0 ? pot[u] : pG;
          int64_t red = FWD ? (int64_t)c - pu + pv : (int64_t)c - pv + pu;
          if (red < 0) {
            err |= kErrInternal;
            red = 0;
          }
          if (red >= (int64_t)kNoArc)
            err |= kErrOverflow;
          else
            r = (uint32_t)red;
        }
        rc[d - 1][ly][lane] = r;
      }
    }
    __syncthreads();
    uint64_t orig[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) orig[k] = lab[warp + 8 * k + 1][lane + 1];
    // local fixed point by directional scans: rows left->right and right->left,
    // then columns top->bottom and bottom->top; a line is rescanned only if a
    // scan in the other orientation changed one of its cells (all start dirty)
    if (tid == 0) {
      rowdirty = 0xFFFFFFFFu;
      coldirty = 0xFFFFFFFFu;
    }
    __syncthreads();
    const int grp = lane >> 3, seg = lane & 7;
    bool capped = false;
    int round = 0;
    for (; round < kMaxLocalSweeps; ++round) {
      // rows 4*warp + grp; this lane holds columns 4*seg..4*seg+3
      const unsigned rd = rowdirty;
      const int r = 4 * warp + grp;
      unsigned chr = 0;
      if ((rd >> (4 * warp)) & 0xFu) {
        uint64_t* rowp = &lab[r + 1][0];
        const uint32_t* wl = &rc[kDirLeft - 1][r][0];
        const uint32_t* wr = &rc[kDirRight - 1][r][0];
        unsigned f = scan_segments<true>([&](int k) { return rowp + 1 + 4 * seg + k; },
                                         [&](int k) { return wl[4 * seg + k]; }, rowp[0], kDirLeft, seg, capK,
                                         &capped, &err);
        unsigned bk = scan_segments<false>([&](int k) { return rowp + 1 + 4 * seg + 3 - k; },
                                           [&](int k) { return wr[4 * seg + 3 - k]; }, rowp[TS + 1], kDirRight, seg,
                                           capK, &capped, &err);
        // columns touched: bit k of f is column 4seg+k, bit k of bk is column 4seg+3-k
        unsigned cols = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if ((f >> k) & 1u) cols |= 1u << (4 * seg + k);
          if ((bk >> k) & 1u) cols |= 1u << (4 * seg + 3 - k);
        }
        chr = cols;
      }
      __syncthreads();
      if (tid == 0) rowdirty = 0;
      // reduce the changed-column masks of the block
      unsigned cm = __reduce_or_sync(0xffffffffu, chr);
      if (lane == 0 && cm) atomicOr(&coldirty_next, cm);
      __syncthreads();
      if (tid == 0) {
        coldirty |= coldirty_next;
        coldirty_next = 0;
      }
      __syncthreads();
      const unsigned cd = coldirty;
      const int c = 4 * warp + grp;
      unsigned chc = 0;
      if ((cd >> (4 * warp)) & 0xFu) {
        const uint32_t* wu = &rc[kDirUp - 1][0][c];
        const uint32_t* wd = &rc[kDirDown - 1][0][c];
        unsigned f = scan_segments<true>([&](int k) { return &lab[4 * seg + k + 1][c + 1]; },
                                         [&](int k) { return wu[(4 * seg + k) * RCOL]; }, lab[0][c + 1], kDirUp,
                                         seg, capK, &capped, &err);
        unsigned bk = scan_segments<false>([&](int k) { return &lab[4 * seg + 3 - k + 1][c + 1]; },
                                           [&](int k) { return wd[(4 * seg + 3 - k) * RCOL]; }, lab[TS + 1][c + 1],
                                           kDirDown, seg, capK, &capped, &err);
        unsigned rows = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if ((f >> k) & 1u) rows |= 1u << (4 * seg + k);
          if ((bk >> k) & 1u) rows |= 1u << (4 * seg + 3 - k);
        }
        chc = rows;
      }
      __syncthreads();
      if (tid == 0) coldirty = 0;
      unsigned rm = __reduce_or_sync(0xffffffffu, chc);
      if (lane == 0 && rm) atomicOr(&rowdirty_next, rm);
      __syncthreads();
      if (tid == 0) {
        rowdirty = rowdirty_next;
        rowdirty_next = 0;
      }
      __syncthreads();
      if (rowdirty == 0) break;
    }
    // write back and note which tile sides changed
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int ly = warp + 8 * k;
      int64_t i = i0 + ly, j = j0 + lane;
      uint64_t v = lab[ly + 1][lane + 1];
      if (i < g.R && j < g.C && v != orig[k]) {
        // the same tile may be in process in two CTAs (it can be re-queued
        // while in flight); atomicMin keeps every label monotone
        atomicMin((unsigned long long*)&labels[i * g.C + j], (unsigned long long)v);
        if (ly == 0) side[0] = 1;
        if (ly == TS - 1) side[1] = 1;
        if (lane == 0) side[2] = 1;
        if (lane == TS - 1) side[3] = 1;
      }
    }
    if (__syncthreads_or(capped) && tid == 0) {
      capped_flag[tile] = 1;
      ctr->capped_any = 1;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      bool ok = true;
      if (side[0] && ti > 0) ok &= q_push(tile - g.tiles_x, ring, q, slots, inq);
      if (side[1] && ti + 1 < g.tiles_y) ok &= q_push(tile + g.tiles_x, ring, q, slots, inq);
      if (side[2] && tj > 0) ok &= q_push(tile - 1, ring, q, slots, inq);
      if (side[3] && tj + 1 < g.tiles_x) ok &= q_push(tile + 1, ring, q, slots, inq);
      if (!ok) err |= kErrSpin;
      atomicAdd(&ctr->tile_visits, 1ull);
      atomicAdd(&ctr->local_rounds, (unsigned long long)(round + 1));
      atomicAdd(&ctr->visit_cycles, (unsigned long long)(clock64() - t_start));
      __threadfence();
      atomicSub(&q->pending, 1);
    }
    __syncthreads();
  }
  if (err) atomicOr(&ctr->err, err);
}

__global__ void k_init_state(Grid g, const int8_t* res, int32_t* excess, int32_t* cand, McfCtr* ctr) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.N; v += (int64_t)gridDim.x * blockDim.x) {
    int32_t r = res[v];
    excess[v] = r;
    if (r != 0) cand[atomicAdd(&ctr->ncand, 1)] = (int32_t)v;
  }
}

template <bool FWD>
__global__ void k_init_labels(Grid g, const int32_t* excess, uint64_t* labels) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.N; v += (int64_t)gridDim.x * blockDim.x) {
    int32_t e = excess[v];
    bool root = FWD ? e > 0 : e < 0;
    labels[v] = root ? 0ull : kInf;
  }
}

__device__ __forceinline__ int32_t& ctr_err(const McfCtr* c) { return const_cast<McfCtr*>(c)->err; }

// Seed the worklist: tiles holding a root, and every border tile (G is a root).
template <bool FWD>
__global__ void k_seed_tiles(Grid g, const int32_t* excess, const int32_t* cand, const McfCtr* ctr, SearchQ* q,
                             int32_t* slots, int32_t* inq, int search_grid) {
  const int nc = ctr->ncand;
  const int nborder = 2 * g.tiles_x + 2 * g.tiles_y;
  const int ring = g.tiles_x * g.tiles_y + search_grid + 64;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nc + nborder;
       k += (int64_t)gridDim.x * blockDim.x) {
    int tile;
    if (k < nc) {
      int32_t v = cand[k];
      int32_t e = excess[v];
      if (!(FWD ? e > 0 : e < 0)) continue;
      int64_t i = v / g.C, j = v % g.C;
      tile = (int)((i / TS) * g.tiles_x + j / TS);
    } else {
      int b = (int)(k - nc);
      if (b < g.tiles_x) tile = b;
      else if (b < 2 * g.tiles_x) tile = (g.tiles_y - 1) * g.tiles_x + (b - g.tiles_x);
      else if (b < 2 * g.tiles_x + g.tiles_y) tile = (b - 2 * g.tiles_x) * g.tiles_x;
      else tile = (b - 2 * g.tiles_x - g.tiles_y) * g.tiles_x + g.tiles_x - 1;
    }
    if (!q_push(tile, ring, q, slots, inq)) atomicOr(&ctr_err(ctr), kErrSpin);
  }
}

// Widen the distance band: queue every tile that dropped a candidate.
__global__ void k_reseed(Grid g, int32_t* capped_flag, SearchQ* q, int32_t* slots, int32_t* inq, int search_grid,
                         McfCtr* ctr) {
  const int T = g.tiles_x * g.tiles_y;
  const int ring = T + search_grid + 64;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
    if (capped_flag[t]) {
      capped_flag[t] = 0;
      if (!q_push(t, ring, q, slots, inq)) atomicOr(&ctr->err, kErrSpin);
    }
  }
}

// Candidates (deficits forward, excess nodes reverse) the search has reached.
template <bool FWD>
__global__ void k_count_found(const int32_t* excess, const uint64_t* labels, const int32_t* cand, McfCtr* ctr) {
  const int nc = ctr->ncand;
  int c = 0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += gridDim.x * blockDim.x) {
    int32_t t = cand[q];
    int32_t e = excess[t];
    if ((FWD ? e < 0 : e > 0) && labels[t] != kInf) ++c;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(&ctr->found, c);
}

// Walk from v along the forest to its root.  Returns the root, or -1 on a walk
// longer than the node count (reported as an internal error).
__device__ __forceinline__ int64_t walk_root(const Grid& g, const uint64_t* labels, int64_t v) {
  for (int64_t steps = 0; steps <= g.N; ++steps) {
    int d = label_dir(labels[v]);
    if (d == kDirRoot) return v;
    int64_t u = nb_node(g, v / g.C, v % g.C, d);
    if (u < 0) return v;  // parent is G: v roots a subtree of G
    v = u;
  }
  return -1;
}

template <bool FWD>
__global__ void k_select(Grid g, const int32_t* excess, const uint64_t* labels, const int32_t* cand,
                         int32_t* cand_root, uint64_t* best, McfCtr* ctr) {
  const int nc = ctr->ncand;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += gridDim.x * blockDim.x) {
    int32_t t = cand[q];
    int32_t e = excess[t];
    cand_root[q] = -1;
    if (!(FWD ? e < 0 : e > 0)) continue;
    uint64_t l = labels[t];
    if (l == kInf) continue;
    int64_t r = walk_root(g, labels, t);
    if (r < 0) {
      atomicOr(&ctr->err, kErrWalk);
      continue;
    }
    cand_root[q] = (int32_t)r;
    atomicMin((unsigned long long*)&best[r], ((l >> 32) << 32) | (uint64_t)(uint32_t)t);
  }
}

template <bool FWD>
__global__ void k_augment(Grid g, int32_t* excess, const uint64_t* labels, const int32_t* cand,
                          const int32_t* cand_root, const uint64_t* best, int8_t* flows, McfCtr* ctr) {
  const int nc = ctr->ncand;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += gridDim.x * blockDim.x) {
    int32_t r = cand_root[q];
    if (r < 0) continue;
    int32_t t = cand[q];
    uint64_t l = labels[t];
    if (best[r] != (((l >> 32) << 32) | (uint64_t)(uint32_t)t)) continue;
    atomicMax(&ctr->D, (uint32_t)(l >> 32));
    atomicAdd(&ctr->naug, 1);
    // flip dk along the path t -> ... -> r (-> G)
    int64_t v = t;
    for (int64_t steps = 0; steps <= g.N; ++steps) {
      int d = label_dir(labels[v]);
      if (d == kDirRoot) break;
      int64_t i = v / g.C, j = v % g.C;
      int64_t e;
      int plane;
      int s;  // +1 if the forward-direction move raises dk
      switch (d) {
        case kDirUp: e = i * g.n + j; plane = 0; s = 1; break;
        case kDirDown: e = (i + 1) * g.n + j; plane = 0; s = -1; break;
        case kDirLeft: e = i * g.n + j; plane = 1; s = -1; break;
        default: e = i * g.n + j + 1; plane = 1; s = 1; break;
      }
      flows[plane * g.P + e] += (int8_t)(FWD ? s : -s);
      int64_t u = nb_node(g, i, j, d);
      if (u < 0) break;
      v = u;
    }
    bool real_root = label_dir(labels[r]) == kDirRoot;
    if (FWD) {
      excess[t] += 1;
      if (real_root) excess[r] -= 1;
      else atomicAdd((unsigned long long*)&ctr->g_net, 1ull);  // G emitted one unit
    } else {
      excess[t] -= 1;
      if (real_root) excess[r] += 1;
      else atomicAdd((unsigned long long*)&ctr->g_net, ~0ull);  // G absorbed one unit
    }
  }
}

__global__ void k_reset_best(const int32_t* cand_root, uint64_t* best, const McfCtr* ctr) {
  const int nc = ctr->ncand;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += gridDim.x * blockDim.x) {
    int32_t r = cand_root[q];
    if (r >= 0) best[r] = kInf;
  }
}

template <bool FWD>
__global__ void k_potentials(Grid g, const uint64_t* labels, int64_t* pot, const McfCtr* ctr) {
  const uint32_t D = ctr->D;
  if (ctr->naug == 0) return;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.N; v += (int64_t)gridDim.x * blockDim.x) {
    uint64_t l = labels[v];
    if (l == kInf) continue;
    uint32_t d = (uint32_t)(l >> 32);
    if (d < D) pot[v] += FWD ? (int64_t)(D - d) : -(int64_t)(D - d);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) pot[g.N] += FWD ? (int64_t)D : -(int64_t)D;
}

__global__ void k_compact(const int32_t* excess, const int32_t* cand, int32_t* cand2, McfCtr* ctr) {
  const int nc = ctr->ncand;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += gridDim.x * blockDim.x) {
    int32_t v = cand[q];
    if (excess[v] != 0) cand2[atomicAdd(&ctr->ncand_next, 1)] = v;
  }
}

__global__ void k_finish_pass(McfCtr* ctr) {
  ctr->ncand = ctr->ncand_next;
  ctr->ncand_next = 0;
}

// total cost sum c_a x_a (block partial sums, int64 atomics)
__global__ void k_total_cost(const int16_t* costs, const int8_t* flows, int64_t P, long long* out) {
  long long s = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P; e += (int64_t)gridDim.x * blockDim.x) {
    int a = flows[e], b = flows[P + e];
    if (a == 1) s += costs[e];
    if (a == -1) s += costs[P + e];
    if (b == 1) s += costs[2 * P + e];
    if (b == -1) s += costs[3 * P + e];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd((unsigned long long*)out, (unsigned long long)s);
}

__global__ void k_write_result(const McfCtr* ctr, const int32_t* ground, int32_t status_host, int32_t* dev_status,
                               int64_t* total_cost) {
  int32_t st = status_host;
  if (st == WW_OK) {
    if (ctr->err & kErrOverflow) st = WW_ERR_OVERFLOW;
    else if (ctr->err) st = WW_ERR_INTERNAL;
    else if (ctr->g_net != (long long)*ground) st = WW_ERR_INTERNAL;
  }
  *dev_status = st;
  *total_cost = ctr->total_cost;
}

bool trace_enabled() {
  static int on = -1;
  if (on < 0) {
    const char* e = std::getenv("WW_TRACE");
    on = (e && e[0] == '1') ? 1 : 0;
  }
  return on == 1;
}

int grid_blocks(int64_t work, int threads, int cap) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

}  // namespace

int64_t solver_bytes(int64_t m, int64_t n) {
  int64_t N = (m - 1) * (n - 1);
  int64_t tiles = ((m - 1 + TS - 1) / TS) * ((n - 1 + TS - 1) / TS);
  return N * (4 + 8 + 8 + 4 + 4 + 4) + tiles * 4 * 3 + (int64_t)sizeof(McfCtr) + 4096;
}

ww_status solver_alloc(ww_workspace* ws, int64_t m, int64_t n) {
  int64_t N = (m - 1) * (n - 1);
  int64_t tiles = ((m - 1 + TS - 1) / TS) * ((n - 1 + TS - 1) / TS);
  if (cudaMalloc(&ws->excess, N * 4) != cudaSuccess) return WW_ERR_OOM;
  if (cudaMalloc(&ws->labels, N * 8) != cudaSuccess) return WW_ERR_OOM;
  if (cudaMalloc(&ws->best, N * 8) != cudaSuccess) return WW_ERR_OOM;
  if (cudaMalloc(&ws->cand, N * 4) != cudaSuccess) return WW_ERR_OOM;
  if (cudaMalloc(&ws->cand2, N * 4) != cudaSuccess) return WW_ERR_OOM;
  if (cudaMalloc(&ws->cand_root, N * 4) != cudaSuccess) return WW_ERR_OOM;
  if (cudaMalloc(&ws->tile_stamp, tiles * 4) != cudaSuccess) return WW_ERR_OOM;
  if (cudaMalloc(&ws->tile_list[0], (tiles + kMaxSearchGrid + 64) * 4) != cudaSuccess) return WW_ERR_OOM;
  if (cudaMalloc(&ws->tile_list[1], tiles * 4) != cudaSuccess) return WW_ERR_OOM;
  if (cudaMalloc(&ws->counters, sizeof(McfCtr)) != cudaSuccess) return WW_ERR_OOM;
  if (cudaMalloc(&ws->search_q, sizeof(SearchQ)) != cudaSuccess) return WW_ERR_OOM;
  if (cudaMallocHost(&ws->host_counters, sizeof(McfCtr)) != cudaSuccess) return WW_ERR_OOM;
  cudaEvent_t* ev = reinterpret_cast<cudaEvent_t*>(ws->events);
  if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) return WW_ERR_CUDA;
  if (cudaMemset(ws->best, 0xFF, N * 8) != cudaSuccess) return WW_ERR_CUDA;
  // queue flags and ring slots start (and end every search) all zero
  if (cudaMemset(ws->tile_stamp, 0, tiles * 4) != cudaSuccess) return WW_ERR_CUDA;
  if (cudaMemset(ws->tile_list[0], 0, (tiles + kMaxSearchGrid + 64) * 4) != cudaSuccess) return WW_ERR_CUDA;
  if (cudaMemset(ws->tile_list[1], 0, tiles * 4) != cudaSuccess) return WW_ERR_CUDA;
  ws->epoch = 0;
  return WW_OK;
}

void solver_free(ww_workspace* ws) {
  cudaFree(ws->excess);
  cudaFree(ws->labels);
  cudaFree(ws->best);
  cudaFree(ws->cand);
  cudaFree(ws->cand2);
  cudaFree(ws->cand_root);
  cudaFree(ws->tile_stamp);
  cudaFree(ws->tile_list[0]);
  cudaFree(ws->tile_list[1]);
  cudaFree(ws->counters);
  cudaFree(ws->search_q);
  cudaFreeHost(ws->host_counters);
  cudaEvent_t* ev = reinterpret_cast<cudaEvent_t*>(ws->events);
  if (ev[0]) cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
}

// One multi-root search: labels reset, worklist seeded with root and border
// tiles, then persistent launches drain the worklist to the fixed point below a
// distance cap.  Nodes whose true distance is below the cap end with exact
// labels.  If no candidate was reached and some tile dropped candidates at the
// cap, the cap grows (x8) and the search resumes from those tiles.
template <bool FWD>
static ww_status run_search(const Grid& g, const int16_t* costs, const int8_t* flows, const int64_t* pot,
                            ww_workspace* ws, McfCtr* dctr, McfCtr* hctr, uint64_t cap, int sm_count,
                            cudaStream_t s) {
  const int nb_nodes = grid_blocks(g.N, 256, sm_count * 16);
  k_init_labels<FWD><<<nb_nodes, 256, 0, s>>>(g, ws->excess, ws->labels);
  SearchQ* q = reinterpret_cast<SearchQ*>(ws->search_q);
  WW_CUDA_TRY(cudaMemsetAsync(q, 0, sizeof(SearchQ), s));
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_search<FWD>, SEARCH_THREADS, 0);
  per_sm = per_sm < 1 ? 1 : per_sm;
  const int search_grid = std::min(sm_count * per_sm, kMaxSearchGrid);
  k_seed_tiles<FWD><<<grid_blocks(g.N / 64 + 1024, 256, sm_count * 4), 256, 0, s>>>(
      g, ws->excess, ws->cand, dctr, q, ws->tile_list[0], ws->tile_stamp, search_grid);
  cudaEvent_t* ev = reinterpret_cast<cudaEvent_t*>(ws->events);
  const int T = g.tiles_x * g.tiles_y;
  float ms_total = 0.0f;
  for (int band = 0; band < 64; ++band) {
    const uint64_t capK = cap >= 0xFFFFFFFFull ? KINF : (cap << 29);
    WW_CUDA_TRY(cudaMemsetAsync(&dctr->found, 0, 2 * sizeof(int32_t), s));  // found, capped_any
    WW_CUDA_TRY(cudaEventRecord(ev[0], s));
    k_search<FWD><<<search_grid, SEARCH_THREADS, 0, s>>>(g, costs, flows, pot, ws->labels, q, ws->tile_list[0],
                                                         ws->tile_stamp, dctr, capK, ws->tile_list[1]);
    WW_CUDA_TRY(cudaEventRecord(ev[1], s));
    WW_CUDA_TRY(cudaGetLastError());
    ++ws->stats.search_iterations;
    if (capK == KINF) break;
    k_count_found<FWD><<<grid_blocks(hctr->ncand > 0 ? hctr->ncand : 1, 256, sm_count * 8), 256, 0, s>>>(
        ws->excess, ws->labels, ws->cand, dctr);
    WW_CUDA_TRY(cudaMemcpyAsync(&hctr->found, &dctr->found, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    WW_CUDA_TRY(cudaStreamSynchronize(s));
    if (hctr->found > 0 || !hctr->capped_any) break;  // the pass adds this last launch's time
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess) ms_total += ms;
    cap = cap >= (0xFFFFFFFFull >> 3) ? 0xFFFFFFFFull : cap * 8;
    WW_CUDA_TRY(cudaMemsetAsync(q, 0, sizeof(SearchQ), s));
    k_reseed<<<grid_blocks(T, 256, sm_count * 8), 256, 0, s>>>(g, ws->tile_list[1], q, ws->tile_list[0],
                                                                 ws->tile_stamp, search_grid, dctr);
  }
  ws->stats.ms_search_gpu += ms_total;  // earlier bands; the pass adds the last launch
  return WW_OK;
}

template <bool FWD>
static ww_status run_pass(const Grid& g, const int16_t* costs, int8_t* flows, int64_t* pot, ww_workspace* ws,
                          McfCtr* dctr, McfCtr* hctr, const ww_params* p, int sm_count, cudaStream_t s) {
  auto t0 = std::chrono::steady_clock::now();
  // full search while many roots remain; distance bands once only a few are left
  uint64_t cap = 0xFFFFFFFFull;
  if (ws->stats.passes >= 2 && hctr->ncand * 1000ll < g.N) cap = std::max<uint64_t>(4096, 4ull * ws->last_D);
  ww_status st = run_search<FWD>(g, costs, flows, pot, ws, dctr, hctr, cap, sm_count, s);
  if (st != WW_OK) return st;
  const int nb = grid_blocks(hctr->ncand > 0 ? hctr->ncand : g.N, 256, sm_count * 16);
  WW_CUDA_TRY(cudaMemsetAsync(&dctr->D, 0, 2 * sizeof(int32_t), s));  // D, naug
  k_select<FWD><<<nb, 256, 0, s>>>(g, ws->excess, ws->labels, ws->cand, ws->cand_root, ws->best, dctr);
  k_augment<FWD><<<nb, 256, 0, s>>>(g, ws->excess, ws->labels, ws->cand, ws->cand_root, ws->best, flows, dctr);
  k_reset_best<<<nb, 256, 0, s>>>(ws->cand_root, ws->best, dctr);
  k_potentials<FWD><<<grid_blocks(g.N, 256, sm_count * 16), 256, 0, s>>>(g, ws->labels, pot, dctr);
  k_compact<<<nb, 256, 0, s>>>(ws->excess, ws->cand, ws->cand2, dctr);
  k_finish_pass<<<1, 1, 0, s>>>(dctr);
  WW_CUDA_TRY(cudaGetLastError());
  std::swap(ws->cand, ws->cand2);
  WW_CUDA_TRY(cudaMemcpyAsync(hctr, dctr, sizeof(McfCtr), cudaMemcpyDeviceToHost, s));
  WW_CUDA_TRY(cudaStreamSynchronize(s));
  cudaEvent_t* ev = reinterpret_cast<cudaEvent_t*>(ws->events);
  float ms = 0.0f;
  if (cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess) ws->stats.ms_search_gpu += ms;
  if (hctr->naug > 0) ws->last_D = hctr->D;
  if (trace_enabled())
    std::fprintf(stderr, "[ww] pass %lld %s: cap %llu, last search %.3f ms, augment %d (D %u), left %d, "
                 "tile visits %llu, rounds %llu\n",
                 (long long)ws->stats.passes, FWD ? "fwd" : "rev", (unsigned long long)cap, ms, hctr->naug, hctr->D,
                 hctr->ncand,
                 (unsigned long long)hctr->tile_visits, (unsigned long long)hctr->local_rounds);
  ws->stats.ms_other += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return WW_OK;
}

ww_status solve_mcf(const int8_t* res, const int32_t* ground, const int16_t* costs, int64_t m, int64_t n,
                    const ww_params* p, ww_workspace* ws, int8_t* flows, int64_t* pot, int64_t* total_cost,
                    int32_t* dev_status, cudaStream_t s) {
  Grid g;
  g.m = m;
  g.n = n;
  g.R = m - 1;
  g.C = n - 1;
  g.N = g.R * g.C;
  g.P = m * n;
  g.tiles_x = (int)((g.C + TS - 1) / TS);
  g.tiles_y = (int)((g.R + TS - 1) / TS);
  int dev = 0, sm_count = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
  McfCtr* dctr = reinterpret_cast<McfCtr*>(ws->counters);
  McfCtr* hctr = reinterpret_cast<McfCtr*>(ws->host_counters);
  ws->stats = ww_solve_stats{};
  ws->last_D = 0;
  WW_CUDA_TRY(cudaMemsetAsync(dctr, 0, sizeof(McfCtr), s));
  WW_CUDA_TRY(cudaMemsetAsync(flows, 0, 2 * g.P, s));
  WW_CUDA_TRY(cudaMemsetAsync(pot, 0, (g.N + 1) * sizeof(int64_t), s));
  k_init_state<<<grid_blocks(g.N, 256, sm_count * 16), 256, 0, s>>>(g, res, ws->excess, ws->cand, dctr);
  WW_CUDA_TRY(cudaGetLastError());
  WW_CUDA_TRY(cudaMemcpyAsync(hctr, dctr, sizeof(McfCtr), cudaMemcpyDeviceToHost, s));
  WW_CUDA_TRY(cudaStreamSynchronize(s));
  ws->stats.residues = hctr->ncand;
  ww_status st = WW_OK;
  int idle = 0;
  int64_t pass = 0;
  while (hctr->ncand > 0) {
    if (pass >= p->max_passes) {
      st = WW_ERR_TIMEOUT;
      break;
    }
    bool fwd = (pass % 2) == 0;
    st = fwd ? run_pass<true>(g, costs, flows, pot, ws, dctr, hctr, p, sm_count, s)
             : run_pass<false>(g, costs, flows, pot, ws, dctr, hctr, p, sm_count, s);
    ++pass;
    ws->stats.passes = pass;
    if (st != WW_OK) break;
    ws->stats.augmentations += hctr->naug;
    if (hctr->err) break;
    idle = hctr->naug == 0 ? idle + 1 : 0;
    if (idle >= 2) {
      st = WW_ERR_INFEASIBLE;
      break;
    }
  }
  ws->stats.passes = pass;
  ws->stats.ground_net = hctr->g_net;
  WW_CUDA_TRY(cudaMemsetAsync(&dctr->total_cost, 0, sizeof(long long), s));
  k_total_cost<<<grid_blocks(g.P, 256, sm_count * 16), 256, 0, s>>>(costs, flows, g.P, &dctr->total_cost);
  k_write_result<<<1, 1, 0, s>>>(dctr, ground, st, dev_status, total_cost);
  WW_CUDA_TRY(cudaGetLastError());
  int32_t hst = 0;
  WW_CUDA_TRY(cudaMemcpyAsync(&hst, dev_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  WW_CUDA_TRY(cudaStreamSynchronize(s));
  ws->stats.tile_visits = (int64_t)hctr->tile_visits;
  ws->stats.local_rounds = (int64_t)hctr->local_rounds;
  ws->stats.visit_cycles = (int64_t)hctr->visit_cycles;
  return hst;
}

// ---------------- certificate (harness) ----------------
__global__ void k_certificate(const int8_t* res, const int32_t* ground, const int16_t* costs, const int8_t* flows,
                              const int64_t* pot, int64_t m, int64_t n, unsigned long long* counts) {
  const int64_t P = m * n, R = m - 1, C = n - 1, N = R * C;
  unsigned long long cap = 0, cons = 0, neg = 0;
  long long cost = 0;
  auto node = [&](int64_t i, int64_t j) -> int64_t { return (i < 0 || j < 0 || i >= R || j >= C) ? N : i * C + j; };
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = k / n, j = k % n;
    for (int plane = 0; plane < 2; ++plane) {
      int dk = flows[plane * P + k];
      bool exists = plane == 0 ? (j + 1 < n) : (i + 1 < m);
      if (dk > 1 || dk < -1 || (!exists && dk != 0)) ++cap;
      if (!exists) continue;
      int64_t a, b;  // "+" arc runs a -> b
      if (plane == 0) {
        a = node(i - 1, j);
        b = node(i, j);
      } else {
        a = node(i, j);
        b = node(i, j - 1);
      }
      int32_t cp = costs[(2 * plane) * P + k], cm = costs[(2 * plane + 1) * P + k];
      if (dk == 1) cost += cp;
      if (dk == -1) cost += cm;
      int64_t pa = pot[a], pb = pot[b];
      // residual arcs of x(+) = [dk==1], x(-) = [dk==-1]
      if (dk != 1 && cp - pa + pb < 0) ++neg;       // + arc unsaturated: a->b cost cp
      if (dk == 1 && -cp - pb + pa < 0) ++neg;      // + arc saturated: b->a cost -cp
      if (dk != -1 && cm - pb + pa < 0) ++neg;      // - arc unsaturated: b->a cost cm
      if (dk == -1 && -cm - pa + pb < 0) ++neg;     // - arc saturated: a->b cost -cm
    }
  }
  // conservation at interior nodes: out - in = residue
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = v / C, j = v % C;
    int net = flows[(i + 1) * n + j] - flows[i * n + j] + flows[P + i * n + j] - flows[P + i * n + j + 1];
    if (net != res[v]) ++cons;
  }
  atomicAdd(&counts[0], cap);
  atomicAdd(&counts[1], cons);
  atomicAdd(&counts[2], neg);
  atomicAdd(&counts[3], (unsigned long long)cost);
}

// G: out - in over the border edges must equal r_G
__global__ void k_certificate_ground(const int32_t* ground, const int8_t* flows, int64_t m, int64_t n,
                                     unsigned long long* counts) {
  const int64_t P = m * n;
  long long net = 0;
  for (int64_t j = threadIdx.x; j < n - 1; j += blockDim.x) {
    net += flows[j];                  // h(0,j): G above, + arc leaves G
    net -= flows[(m - 1) * n + j];    // h(m-1,j): G below, + arc enters G
  }
  for (int64_t i = threadIdx.x; i < m - 1; i += blockDim.x) {
    net -= flows[P + i * n];          // v(i,0): G left, + arc (right->left) enters G
    net += flows[P + i * n + n - 1];  // v(i,n-1): G right, + arc leaves G
  }
  for (int o = 16; o > 0; o >>= 1) net += __shfl_xor_sync(0xffffffffu, net, o);
  __shared__ long long s[32];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = net;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s[k];
    if (t != (long long)*ground) atomicAdd(&counts[1], 1ull);
  }
}

ww_status launch_certificate(const int8_t* res, const int32_t* ground, const int16_t* costs, const int8_t* flows,
                             const int64_t* pot, int64_t m, int64_t n, int64_t* counts, cudaStream_t s) {
  WW_CUDA_TRY(cudaMemsetAsync(counts, 0, 4 * sizeof(int64_t), s));
  k_certificate<<<grid_blocks(m * n, 256, 148 * 16), 256, 0, s>>>(res, ground, costs, flows, pot, m, n,
                                                               (unsigned long long*)counts);
  k_certificate_ground<<<1, 1024, 0, s>>>(ground, flows, m, n, (unsigned long long*)counts);
  WW_CUDA_TRY(cudaGetLastError());
  return WW_OK;
}

}  // namespace ww
