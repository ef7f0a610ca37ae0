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

#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "ww_internal.cuh"

namespace ww {

constexpr int TS = 32;         // tile side in nodes
constexpr int TSH = TS + 2;    // with halo
constexpr int SEARCH_THREADS = 256;
constexpr int kMaxLocalSweeps = 8192;
constexpr int kMaxSearchGrid = 148 * 64;  // ring slack: at most one outstanding ticket per CTA

enum : int32_t { kErrOverflow = 1, kErrInternal = 2, kErrWalk = 4, kErrSpin = 8 };

// One problem of a (possibly one-element) batch.  Node arrays of all problems
// are concatenated (node_off); tiles are numbered consecutively (tile_off).
// All problems share one free ground node, whose potential sits after the
// last node: the supplies of every problem sum to zero, so no flow can cross
// between problems through it and the joint optimum is the sum of the optima.
struct ProbDev {
  int64_t m, n, R, C, N;
  int64_t node_off, tile_off;
  int64_t garc_off;      // first index of this problem's ground arcs (2C + 2R of them)
  int32_t tiles_x, tiles_y;
  const int8_t* res;
  const int32_t* ground;
  const int16_t* costs;
  int8_t* flows;
  int64_t* pot_out;      // caller's potentials (N + 1) or nullptr when pot is the caller's array
  int64_t* total_cost;   // device int64
  int32_t* status;       // device int32
  int32_t resume;        // start from the flows in `flows` (and the caller's potentials), not from zero
  int32_t resume_pad;
};

struct McfCtr {
  int32_t list_count[2];
  uint32_t D;
  int32_t naug;
  int32_t ncand;
  int32_t ncand_next;
  int32_t err;
  int32_t cand_sel;    // which half of the candidate buffer is current
  long long g_net;
  unsigned long long tile_visits;
  long long total_cost;
  unsigned long long local_rounds;
  unsigned long long visit_cycles;
  int32_t found;       // candidates reached by the current search
  int32_t capped_any;  // a tile dropped a candidate at or beyond the cap
  uint32_t cap;        // distance cap of the current search (0xFFFFFFFF = none)
  uint32_t last_D;     // largest augmented distance of the last pass that augmented
  int32_t passes;
  int32_t idle;        // consecutive passes without augmentation
  int32_t band_again;  // the band loop continues
  int32_t go_on;       // the pass loop continues
  int32_t status;      // solver status (WW_OK while running)
  int32_t max_passes;
  int64_t n_total;     // nodes of the active problems
  int64_t n_cap_nodes; // node capacity (the candidate list halves are this far apart)
  long long aug_total; // augmentations over all passes
  uint32_t band_min, band_mult, band_growth, band_start_ppm, full_passes;  // search schedule
  unsigned long long load_cycles, relax_cycles;              // phases of the tile visits
  unsigned long long settled_visits;  // nodes holding a finite label at the end of a tile visit, summed
  // ground as a sink (late passes): the ground is no root; it is reached through
  // border arcs at distance dG, and augmentation is limited to distance <= dG
  int32_t gsink;
  uint32_t dG;
  uint32_t ground_sink_below;  // use it while at most this many nodes are imbalanced
  int32_t gsink_pad;
  // zero-distance first band (late passes): the band keeps only labels of distance
  // 0 and fewer than zero_hops hops; augmenting inside it changes no potential (D = 0)
  int32_t zstop;       // this pass starts with such a band
  uint32_t zero_hops;  // largest hop radius of the zero band
  uint32_t zhop[3];    // hop radius of each stage of the zero band (widened while nothing is reached)
  int32_t zstage;      // current stage
  uint32_t zero_stop_below;  // use it while at most this many nodes are imbalanced
  uint32_t cap0;       // the pass's ordinary first cap (after the zero band)
  // first negative reduced cost seen (diagnostics): flag, node, direction, value, pass
  int32_t dbg_set, dbg_dir;
  long long dbg_node, dbg_red;
  int32_t dbg_pass, dbg_pad;
  int32_t ntouched;    // tiles listed as visited in this pass
  uint32_t wait_polls; // polls of a worklist wait before it gives up (WW_ERR_TIMEOUT)
  unsigned long long visits32;  // tile visits relaxed in 32-bit keys
  unsigned long long redo64;    // of which redone in 64-bit keys (a candidate left the 32-bit range)
  unsigned long long pop_cycles;  // SM cycles spent taking tiles from the worklist (waits included)
  unsigned long long touched_total;  // distinct tiles visited, summed over passes
  int32_t nseg;        // tile segments of this pass's augmenting paths (k_augment -> k_flip_segments)
  int32_t nseg_pad;
};

// Problems live in slots (stable ids); `order` lists the active slots sorted by
// node offset.  The shared ground potential sits at pot[g_index].
struct Batch {
  const ProbDev* probs;      // by slot
  const int32_t* order;      // active slots by ascending node_off
  int nact;                  // active slots
  const int32_t* tile_prob;  // global tile -> slot
  int64_t g_index;           // index of the ground potential
  int64_t n_total;           // nodes of the active problems (pass policy)
  int64_t t_total;           // upper bound of the tile ids in use
};

__device__ __forceinline__ int prob_of_node(const Batch& b, int64_t v) {
  int lo = 0, hi = b.nact - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (b.probs[b.order[mid]].node_off <= v) lo = mid;
    else hi = mid - 1;
  }
  return b.order[lo];
}

namespace {

// Raw residual cost of the arc entering node (i,j) from direction dir (forward
// search: arc u->v) or leaving it toward dir (reverse search: arc v->u).
// Returns false if the arc does not exist.
template <bool FWD>
__device__ __forceinline__ bool arc_cost(const ProbDev& p, int64_t i, int64_t j, int dir, int32_t* cost) {
  const int64_t P = p.m * p.n;
  int64_t e;
  int plane;  // 0: h edge, 1: v edge
  bool plus;  // move raises dk
  switch (dir) {
    case kDirUp: e = i * p.n + j; plane = 0; plus = FWD; break;
    case kDirDown: e = (i + 1) * p.n + j; plane = 0; plus = !FWD; break;
    case kDirLeft: e = i * p.n + j; plane = 1; plus = !FWD; break;
    default: e = i * p.n + j + 1; plane = 1; plus = FWD; break;
  }
  int dk = p.flows[plane * P + e];
  int32_t cp = p.costs[(2 * plane) * P + e], cm = p.costs[(2 * plane + 1) * P + e];
  if (plus) {
    if (dk > 0) return false;
    *cost = dk == 0 ? cp : -cm;
  } else {
    if (dk < 0) return false;
    *cost = dk == 0 ? cm : -cp;
  }
  return true;
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

// Every wait polls at most `limit` times (ww_params.wait_polls, default 2^25
// polls of ~100-200 ns, seconds in all); running out is reported as an error.
__device__ __forceinline__ int ld_volatile(const int32_t* p) { return *((volatile const int32_t*)p); }

// Returns false if the slot stayed occupied past the wait limit (reported as an error).
__device__ __forceinline__ bool q_push(int tile, int ring, SearchQ* q, int32_t* slots, int32_t* inq, uint32_t limit) {
  if (atomicExch(&inq[tile], 1) != 0) return true;
  atomicAdd(&q->pending, 1);
  int pos = atomicAdd(&q->tail, 1);
  __threadfence();
  int* slot = &slots[pos % ring];
  for (uint32_t spin = 0; spin < limit; ++spin) {
    if (atomicCAS(slot, 0, tile + 1) == 0) return true;
    __nanosleep(100);
  }
  return false;
}

// Returns a tile, -1 when the search has converged, -2 on a bounded-wait timeout.
__device__ int q_pop(int ring, SearchQ* q, int32_t* slots, int32_t* inq, uint32_t limit) {
  const int h = atomicAdd(&q->head, 1);
  int* slot = &slots[h % ring];
  for (uint32_t spin = 0; spin < limit; ++spin) {
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

// Takes the tile at the worklist's head only if one is already published there
// (never waits): -1 if none is, or another CTA took it first.
__device__ int q_try_pop(int ring, SearchQ* q, int32_t* slots, int32_t* inq) {
  const int h = ld_volatile(&q->head);
  int* slot = &slots[h % ring];
  const int v = ld_volatile(slot);
  if (v == 0 || atomicCAS(&q->head, h, h + 1) != h) return -1;
  atomicExch(slot, 0);
  atomicExch(&inq[v - 1], 0);
  __threadfence();
  return v - 1;
}

constexpr uint64_t KINF = kInf >> 3;                  // (distance, hops) part of an unreached label
constexpr uint64_t KDIST_INF = 0xFFFFFFFFull << 29;   // distance field all ones

// Label keys of the local relaxation in two widths.
//  64-bit cells: (distance:32 | hops:29 | dir:3); a kept distance that overflows
//    32 bits is reported.
//  32-bit cells: (distance - d0:13 | hops - h0:15 | dir:3), relative to the
//    smallest distance d0 and hop count h0 among the finite labels of the tile
//    and its halo.  Subtracting the same d0 and h0 from every label keeps the
//    (distance, hops, dir) order and commutes with adding an arc, so a visit gives
//    the same labels in either width as long as every key it keeps fits: the
//    visit's finite labels span fewer than kDistSpan32 distance units and at most
//    kHopSpan32 hops, and the visit converges within kRounds32 rounds (a value
//    carried in a round is a label read in that round plus at most one arc per
//    sweep step of the round, 4 x 32, so no hop field carries); else the visit is
//    redone in 64 bits.  The arc weights are clamped to kDistSpan32 units; a
//    finite key plus a clamped weight stays below 2^29 - 1 (the unreached key), so
//    every candidate is either unreached, at or beyond capK, or kept, as in 64
//    bits.  capK is the band's cap relative to d0 when that is at most kDistSpan32
//    units, else the local limit kDistSpan32 << 15: a candidate dropped there may
//    lie inside the band, and the visit is then redone in 64 bits.
constexpr uint32_t kDistSpan32 = 8191;         // distance span of a 32-bit visit (exclusive)
constexpr uint32_t kHopSpan32 = 16383;         // hop span of the labels entering a 32-bit visit
constexpr int kRounds32 = 64;                  // rounds of a 32-bit visit (16383 + 64 * 129 < 2^15)
constexpr uint32_t KINF32 = 0x1FFFFFFFu;      // key of an unreached 32-bit cell (0xFFFFFFFF >> 3)
constexpr uint32_t kLocalCap32 = kDistSpan32 << 15;

// 32-bit weight of an arc of reduced cost w (kNoArc: no arc): +w distance (clamped), +1 hop
__device__ __forceinline__ uint32_t weight32(uint32_t w) {
  return w == kNoArc ? KINF32 : ((min(w, kDistSpan32) << 15) + 1u);
}

template <class KT>
struct Keys;
template <>
struct Keys<uint64_t> {
  static constexpr int kRounds = kMaxLocalSweeps;
  __device__ static __forceinline__ uint64_t inf() { return KINF; }
  // the arc-weight planes hold reduced costs
  __device__ static __forceinline__ uint64_t weight(uint32_t w) {
    return w == kNoArc ? KINF : (((uint64_t)w << 29) + 1ull);  // +w distance, +1 hop
  }
  __device__ static __forceinline__ bool overflow(uint64_t cand) { return cand >= KDIST_INF; }
};
template <>
struct Keys<uint32_t> {
  static constexpr int kRounds = kRounds32;
  __device__ static __forceinline__ uint32_t inf() { return KINF32; }
  // the arc-weight planes hold weight32() values
  __device__ static __forceinline__ uint32_t weight(uint32_t w) { return w; }
  __device__ static __forceinline__ bool overflow(uint32_t) { return false; }
};

constexpr int LROW = TS + 3;  // padded row stride of the label tile (halo 1 each side + 1 pad)
constexpr int RCOL = TS + 1;  // padded row stride of the arc-weight planes

// One directional sweep of one line of the tile by one lane: the cells k in
// sweep order with labels K_k and entering-arc weights b_k become
//   c_k = min(K_k, c_{k-1} + b_k),  c_{-1} = the halo label,
// a candidate keeping direction code dir, kept only below the cap.  The carried
// value is min(K_k, c_{k-1} + b_k) whether or not it is kept: a value at or
// beyond the cap only leads to more such values, none of which is written.
// ROW: the line is row `line`, else column `line`; FORWARD: increasing index.
// Cells are read a few at a time; the sweeps of the other directions run at the
// same time, and a lower value one of them wrote may be overwritten (the
// writer's line is then swept again).  Returns the mask of cells written (bit =
// index along the line).
template <class KT, bool ROW, bool FORWARD>
__device__ __forceinline__ unsigned sweep_line(KT (*L)[LROW], const uint32_t (*W)[RCOL], int line, KT capK8, int dir,
                                               int* err) {
  using KK = Keys<KT>;
  const int h = FORWARD ? 0 : TS + 1;
  KT prev = (ROW ? L[line + 1][h] : L[h][line + 1]) >> 3;
  unsigned ch = 0;
  bool ov = false;
  constexpr int CH = sizeof(KT) == 4 ? 8 : 4;  // cells read ahead (registers)
  for (int c0 = 0; c0 < TS; c0 += CH) {
    KT cell[CH];
    uint32_t w[CH];
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      const int k = FORWARD ? c0 + s : TS - 1 - c0 - s;
      cell[s] = ROW ? L[line + 1][k + 1] : L[k + 1][line + 1];
      w[s] = ROW ? W[line][k] : W[k][line];
    }
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      const int k = FORWARD ? c0 + s : TS - 1 - c0 - s;
      // prev <= inf and weight <= inf: no wrap in either width
      const KT cand = prev + KK::weight(w[s]);
      prev = min(cell[s] >> 3, cand);
      // key < capK << 3 exactly when cand < capK (the low three bits hold dir)
      const KT key = (min(cand, KK::inf()) << 3) | (KT)dir;
      bool imp = key < min(cell[s], capK8);
      if (KK::overflow(cand) && imp) {
        ov = true;  // only without a cap: a capped band keeps distances below 2^31
        imp = false;
      }
      if (imp) {
        (ROW ? L[line + 1][k + 1] : L[k + 1][line + 1]) = key;
        ch |= 1u << k;
      }
    }
  }
  if (ov) *err |= kErrOverflow;
  return ch;
}

// Local fixed point of one tile: warps 0..3 sweep rows left to right, rows
// right to left, columns top to bottom and columns bottom to top at the same
// time (lane = line).  Every value a sweep carries is a label it read plus arcs,
// so any interleaving leaves valid labels, and a round in which no sweep writes
// leaves the fixed point.  A line is swept again only if another sweep wrote one
// of its cells.  L is the label tile with its halo, rc the four arc-weight
// planes, s_mask two rounds of change masks.  Run by warps 0..3 only (their own
// barrier), so the other warps of the block are free meanwhile.  Returns the
// rounds run; *guard is set when the fixed point was not reached within
// Keys<KT>::kRounds rounds.
template <class KT>
__device__ __forceinline__ int relax_tile(KT (*L)[LROW], const uint32_t (*rc)[TS][RCOL], KT capK,
                                          unsigned (*s_mask)[8], bool* guard, int* err) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const KT capK8 = capK << 3;  // capK < 2^61
  unsigned mine = 0xFFFFFFFFu;  // lines this warp sweeps in the next round
  int par = 0, round = 0;
  for (;; ++round) {
    if (round == Keys<KT>::kRounds) {
      *guard = true;
      break;
    }
    unsigned ch = 0;
    if ((mine >> lane) & 1u) {
      if (warp == 0) ch = sweep_line<KT, true, true>(L, rc[kDirLeft - 1], lane, capK8, kDirLeft, err);
      else if (warp == 1) ch = sweep_line<KT, true, false>(L, rc[kDirRight - 1], lane, capK8, kDirRight, err);
      else if (warp == 2) ch = sweep_line<KT, false, true>(L, rc[kDirUp - 1], lane, capK8, kDirUp, err);
      else ch = sweep_line<KT, false, false>(L, rc[kDirDown - 1], lane, capK8, kDirDown, err);
    }
    // lines this warp wrote, and the lines of the other orientation it crossed
    const unsigned lines = __ballot_sync(0xffffffffu, ch != 0);
    const unsigned cross = __reduce_or_sync(0xffffffffu, ch);
    if (lane == 0) {
      s_mask[par][warp] = lines;
      s_mask[par][4 + warp] = cross;
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");  // warps 0..3
    const unsigned* m = s_mask[par];
    if ((m[0] | m[1] | m[2] | m[3]) == 0) break;
    // rows: written by the other row sweep or crossed by a column sweep; columns alike
    if (warp == 0) mine = m[1] | m[6] | m[7];
    else if (warp == 1) mine = m[0] | m[6] | m[7];
    else if (warp == 2) mine = m[3] | m[4] | m[5];
    else if (warp == 3) mine = m[2] | m[4] | m[5];
    par ^= 1;
  }
  return round + 1;
}

// After the fixed point: does an arc into one of this thread's cells (rows
// warp + 8k, column lane) carry a finite candidate at or beyond the cap that
// would improve the cell?  Then the band dropped it, and the tile is re-seeded
// if the band is widened.
template <class KT>
__device__ __forceinline__ bool tile_capped(const KT (*L)[LROW], const uint32_t (*rc)[TS][RCOL], KT capK) {
  using KK = Keys<KT>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  bool capped = false;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int r = warp + 8 * k, c = lane;
    const KT cur = L[r + 1][c + 1] >> 3;
    // the neighbour each arc-weight plane enters from
    KT from[4];
    from[kDirUp - 1] = L[r][c + 1];
    from[kDirDown - 1] = L[r + 2][c + 1];
    from[kDirLeft - 1] = L[r + 1][c];
    from[kDirRight - 1] = L[r + 1][c + 2];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const KT cand = (from[d] >> 3) + KK::weight(rc[d][r][c]);
      capped |= cand >= capK && cand < KK::inf() && cand < cur;
    }
  }
  return capped;
}

// Per-pass cache of a tile's arc costs (potentials, flows and costs are fixed
// while a pass searches, and a tile is visited several times per pass): 4 planes
// of 32 x 32 reduced costs, stamped with the pass that wrote them.
constexpr int64_t kRcTileBytes = 4 * TS * TS * 4;

__device__ __forceinline__ int ld_acquire(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int32_t* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// smem arc-cost planes <-> the tile's cache entry, 16 bytes per access (L2 only:
// other CTAs write entries during the launch)
__device__ __forceinline__ void rc_from_cache(const uint32_t* __restrict__ src, uint32_t (*rc)[TS][RCOL]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int q = threadIdx.x + SEARCH_THREADS * u;  // 16-byte chunk: plane, row, 4 columns
    const int d = q >> 8, r = (q >> 3) & 31, c = (q & 7) * 4;
    const uint4 v = __ldcg(reinterpret_cast<const uint4*>(src) + q);
    rc[d][r][c] = v.x;
    rc[d][r][c + 1] = v.y;
    rc[d][r][c + 2] = v.z;
    rc[d][r][c + 3] = v.w;
  }
}
__device__ __forceinline__ void rc_to_cache(const uint32_t (*rc)[TS][RCOL], uint32_t* __restrict__ dst) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int q = threadIdx.x + SEARCH_THREADS * u;
    const int d = q >> 8, r = (q >> 3) & 31, c = (q & 7) * 4;
    __stcg(reinterpret_cast<uint4*>(dst) + q, make_uint4(rc[d][r][c], rc[d][r][c + 1], rc[d][r][c + 2], rc[d][r][c + 3]));
  }
}
// the planes as weight32() values (this thread's chunks, as above)
__device__ __forceinline__ void rc_narrow(uint32_t (*rc)[TS][RCOL]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int q = threadIdx.x + SEARCH_THREADS * u;
    const int d = q >> 8, r = (q >> 3) & 31, c = (q & 7) * 4;
#pragma unroll
    for (int k = 0; k < 4; ++k) rc[d][r][c + k] = weight32(rc[d][r][c + k]);
  }
}

// Reduced costs of the four arcs of every node of a tile, edge by edge: each
// edge's flow and two costs are read once and give the arcs of both of its
// nodes.  rc[dir-1][node] is the arc entering the node from dir (forward search)
// or leaving it toward dir (reverse search); kNoArc where there is none.
// NARROW: stored as weight32() values, else as reduced costs.
template <bool FWD, bool NARROW>
__device__ __forceinline__ void build_rc(const ProbDev& p, int64_t i0, int64_t j0, const int64_t (*spot)[TSH],
                                         uint32_t (*rc)[TS][RCOL], int* err) {
  const int tid = threadIdx.x;
  const int64_t P = p.m * p.n;
  auto put = [](uint32_t w) { return NARROW ? weight32(w) : w; };
  // h edges h(i, j), i = i0 + er (er = 0..TS), j = j0 + lx: node A = (i-1, j) above, B = (i, j) below
  for (int q = tid; q < (TS + 1) * TS; q += SEARCH_THREADS) {
    const int er = q / TS, lx = q % TS;
    const int64_t i = i0 + er, j = j0 + lx;
    const bool a_in = i - 1 >= 0 && i - 1 < p.R && j < p.C;
    const bool b_in = i < p.R && j < p.C;
    uint32_t up_b = kNoArc, down_a = kNoArc;  // rc[Up][B], rc[Down][A]
    if (a_in || b_in) {
      const int64_t e = i * p.n + j;
      const int dk = p.flows[e];
      const int32_t cp = p.costs[e], cm = p.costs[P + e];
      const int64_t pa = spot[er][lx + 1], pb = spot[er + 1][lx + 1];
      // A->B raises dk (available unless dk = +1); B->A lowers it (unless dk = -1)
      const bool ab_ok = dk <= 0, ba_ok = dk >= 0;
      const int64_t ab = ab_ok ? (int64_t)(dk == 0 ? cp : -cm) - pa + pb : 0;
      const int64_t ba = ba_ok ? (int64_t)(dk == 0 ? cm : -cp) - pb + pa : 0;
      // forward: entering B from above = A->B, entering A from below = B->A; reverse: the opposite arcs
      const bool ok_ub = FWD ? ab_ok : ba_ok, ok_da = FWD ? ba_ok : ab_ok;
      const int64_t r_ub = FWD ? ab : ba, r_da = FWD ? ba : ab;
      if (b_in && ok_ub) {
        if (r_ub < 0) *err |= kErrInternal;
        if (r_ub >= (int64_t)kNoArc) *err |= kErrOverflow;
        else up_b = (uint32_t)max(r_ub, (int64_t)0);
      }
      if (a_in && ok_da) {
        if (r_da < 0) *err |= kErrInternal;
        if (r_da >= (int64_t)kNoArc) *err |= kErrOverflow;
        else down_a = (uint32_t)max(r_da, (int64_t)0);
      }
    }
    if (er < TS) rc[kDirUp - 1][er][lx] = put(up_b);
    if (er > 0) rc[kDirDown - 1][er - 1][lx] = put(down_a);
  }
  // v edges v(i, j), i = i0 + ly, j = j0 + ec (ec = 0..TS): node L = (i, j-1) left, Rn = (i, j) right
  for (int q = tid; q < TS * (TS + 1); q += SEARCH_THREADS) {
    const int ly = q / (TS + 1), ec = q % (TS + 1);
    const int64_t i = i0 + ly, j = j0 + ec;
    const bool l_in = i < p.R && j - 1 >= 0 && j - 1 < p.C;
    const bool r_in = i < p.R && j < p.C;
    uint32_t left_r = kNoArc, right_l = kNoArc;  // rc[Left][Rn], rc[Right][L]
    if (l_in || r_in) {
      const int64_t e = i * p.n + j;
      const int dk = p.flows[P + e];
      const int32_t cp = p.costs[2 * P + e], cm = p.costs[3 * P + e];
      const int64_t pl = spot[ly + 1][ec], pr = spot[ly + 1][ec + 1];
      // Rn->L raises dk (available unless dk = +1); L->Rn lowers it (unless dk = -1)
      const bool rl_ok = dk <= 0, lr_ok = dk >= 0;
      const int64_t rl = rl_ok ? (int64_t)(dk == 0 ? cp : -cm) - pr + pl : 0;
      const int64_t lr = lr_ok ? (int64_t)(dk == 0 ? cm : -cp) - pl + pr : 0;
      // forward: entering Rn from the left = L->Rn, entering L from the right = Rn->L
      const bool ok_lr = FWD ? lr_ok : rl_ok, ok_rl = FWD ? rl_ok : lr_ok;
      const int64_t r_lr = FWD ? lr : rl, r_rl = FWD ? rl : lr;
      if (r_in && ok_lr) {
        if (r_lr < 0) *err |= kErrInternal;
        if (r_lr >= (int64_t)kNoArc) *err |= kErrOverflow;
        else left_r = (uint32_t)max(r_lr, (int64_t)0);
      }
      if (l_in && ok_rl) {
        if (r_rl < 0) *err |= kErrInternal;
        if (r_rl >= (int64_t)kNoArc) *err |= kErrOverflow;
        else right_l = (uint32_t)max(r_rl, (int64_t)0);
      }
    }
    if (ec < TS) rc[kDirLeft - 1][ly][ec] = put(left_r);
    if (ec > 0) rc[kDirRight - 1][ly][ec - 1] = put(right_l);
  }
}

template <bool FWD>
__global__ void __launch_bounds__(SEARCH_THREADS, 5) k_search(Batch b, const int64_t* __restrict__ pot,
                                                           uint64_t* labels, SearchQ* q, int32_t* slots,
                                                           int32_t* inq, McfCtr* ctr, int32_t* capped_flag,
                                                           int32_t* touched, int32_t* tlist, uint32_t* rc_cache,
                                                           int32_t* rc_pass, int32_t rc_entries) {
  __shared__ uint64_t lab[TSH][LROW];
  __shared__ uint32_t lab32[TSH][LROW];  // the same labels as 32-bit cells (a 32-bit visit)
  __shared__ uint32_t rc[4][TS][RCOL];
  __shared__ int64_t spot[TSH][TSH];  // potentials with halo (the ground outside the grid)
  __shared__ int side[4];
  __shared__ int s_tile, s_hit;
  __shared__ int s_next;  // a tile taken from the worklist during the previous visit (-1: none)
  // smallest / largest distance and hop count of the finite labels of the tile and its halo
  __shared__ uint32_t s_dmin, s_dmax, s_hmin, s_hmax;
  __shared__ unsigned s_mask[2][8];  // change masks of the relaxation rounds
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;  // 8 warps
  const int ring = (int)b.t_total + (int)gridDim.x + 64;
  const int64_t pG = pot[b.g_index];
  const uint32_t cap = ctr->cap;
  // the zero band keeps keys (0, hops < radius): distance 0 within the stage's hop radius
  const uint64_t capK = (ctr->zstop != 0 && cap == 1u) ? (uint64_t)ctr->zhop[ctr->zstage]
                        : (cap == 0xFFFFFFFFu ? KINF : ((uint64_t)cap << 29));
  const bool gsink = ctr->gsink != 0;
  const uint32_t wait_polls = ctr->wait_polls;
  const int stamp = ctr->passes + 1;  // this pass in the arc-cost cache
  int err = 0;
  if (tid == 0) s_next = -1;
  for (;;) {
    if (tid == 0) {
      const long long t_pop = clock64();
      int t = s_next;
      s_next = -1;
      if (t < 0) t = q_pop(ring, q, slots, inq, wait_polls);
      s_tile = t;
      // a cache entry of this pass holds every arc cost of the tile (acquire:
      // the entry's stores are seen before its stamp)
      s_hit = t >= 0 && t < rc_entries && ld_acquire(&rc_pass[t]) == stamp;
      atomicAdd(&ctr->pop_cycles, (unsigned long long)(clock64() - t_pop));
    }
    __syncthreads();
    const int tile = s_tile;
    if (tile < 0) {
      if (tid == 0 && tile == -2) atomicOr(&ctr->err, kErrSpin);
      break;
    }
    const ProbDev& p = b.probs[b.tile_prob[tile]];
    const int64_t lt = tile - p.tile_off;
    const int64_t ti = lt / p.tiles_x, tj = lt % p.tiles_x;
    const int64_t i0 = ti * TS, j0 = tj * TS;
    uint64_t* plab = labels + p.node_off;
    const int64_t* ppot = pot + p.node_off;
    if (tid < 4) side[tid] = 0;
    if (tid == 0) {
      s_dmin = 0xFFFFFFFFu;
      s_hmin = 0xFFFFFFFFu;
      s_dmax = 0;
      s_hmax = 0;
    }
    // first visit of the tile in this pass: list it, so that its labels are
    // reset after the pass without a sweep over every node
    if (tid == 0 && atomicExch(&touched[tile], 1) == 0) {
      const int k = atomicAdd(&ctr->ntouched, 1);
      if (k < (int)b.t_total) tlist[k] = tile;
      else err |= kErrInternal;
    }
    const long long t_start = clock64();
    const bool hit = s_hit != 0, cached = tile < rc_entries;
    uint32_t* rc_entry = rc_cache + (int64_t)tile * (kRcTileBytes / 4);
    uint32_t dmin = 0xFFFFFFFFu, dmax = 0, hmin = 0xFFFFFFFFu, hmax = 0;
    // labels with halo; directly outside the grid stands G, a root (label 0)
    for (int qd = tid; qd < TSH * TSH; qd += SEARCH_THREADS) {
      int r = qd / TSH, c = qd % TSH;
      int64_t i = i0 + r - 1, j = j0 + c - 1;
      uint64_t v;
      int64_t pv;
      if (i < 0 || j < 0 || i >= p.R || j >= p.C) {
        bool ring = (i >= -1 && i <= p.R && j >= -1 && j <= p.C);
        v = (ring && !gsink) ? 0ull : kInf;
        pv = pG;
      } else {
        v = *((volatile const uint64_t*)&plab[i * p.C + j]);
        pv = hit ? 0 : ppot[i * p.C + j];  // potentials only to build the arc costs
      }
      lab[r][c] = v;
      spot[r][c] = pv;
      if (v != kInf) {
        const uint32_t d = (uint32_t)(v >> 32), h = (uint32_t)(v >> 3) & 0x1FFFFFFFu;
        dmin = min(dmin, d);
        dmax = max(dmax, d);
        hmin = min(hmin, h);
        hmax = max(hmax, h);
      }
    }
    __syncthreads();
    dmin = __reduce_min_sync(0xffffffffu, dmin);
    dmax = __reduce_max_sync(0xffffffffu, dmax);
    hmin = __reduce_min_sync(0xffffffffu, hmin);
    hmax = __reduce_max_sync(0xffffffffu, hmax);
    if (lane == 0) {
      atomicMin(&s_dmin, dmin);
      atomicMax(&s_dmax, dmax);
      atomicMin(&s_hmin, hmin);
      atomicMax(&s_hmax, hmax);
    }
    __syncthreads();
    // key width of this visit (see Keys): 32 bits when the finite labels' spans
    // fit, with the band's cap exact when it lies within the 32-bit range
    const uint32_t d0 = s_dmin, h0 = s_hmin;
    bool narrow = d0 != 0xFFFFFFFFu && s_dmax - d0 < kDistSpan32 && s_hmax - h0 <= kHopSpan32;
    bool local = false;  // the 32-bit range, not the band, limits this visit
    uint32_t capK32 = kLocalCap32;
    if (narrow) {
      if (ctr->zstop != 0 && cap == 1u) {
        // zero band: keys (0, hops < radius); every kept label has distance 0
        const uint32_t zh = ctr->zhop[ctr->zstage];
        if (d0 != 0 || zh <= h0) narrow = false;
        else if (zh - h0 <= 32767u) capK32 = zh - h0;
        else capK32 = 32767u, local = true;
      } else if (cap != 0xFFFFFFFFu && cap - d0 <= kDistSpan32) {
        capK32 = (cap - d0) << 15;  // cap > d0: every kept label lies below the cap
      } else {
        // distances d0 + kDistSpan32 and beyond are left to a 64-bit visit
        local = true;
        if (d0 > 0xFFFFFFFEu - kDistSpan32) narrow = false;
      }
    }
    uint64_t orig[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) orig[k] = lab[warp + 8 * k + 1][lane + 1];
    // arc costs: from this pass's cache entry, or built and stored there
    if (hit) {
      rc_from_cache(rc_entry, rc);
    } else {
      build_rc<FWD, false>(p, i0, j0, spot, rc, &err);
      __syncthreads();
      if (cached) {
        rc_to_cache(rc, rc_entry);
        __threadfence();
      }
    }
    if (narrow) rc_narrow(rc);  // the same chunks this thread moved (cache and conversion): no barrier needed
    if (!hit && cached) {
      __syncthreads();
      if (tid == 0 && err == 0) st_release(&rc_pass[tile], stamp);
    }
    if (narrow) {
      for (int qd = tid; qd < TSH * TSH; qd += SEARCH_THREADS) {
        const int r = qd / TSH, c = qd % TSH;
        const uint64_t v = lab[r][c];
        uint32_t x = 0xFFFFFFFFu;
        if (v != kInf) {
          const uint32_t d = (uint32_t)(v >> 32) - d0, h = ((uint32_t)(v >> 3) & 0x1FFFFFFFu) - h0;
          x = (((d << 15) | h) << 3) | (uint32_t)(v & 7u);
        }
        lab32[r][c] = x;
      }
    }
    __syncthreads();
    const long long t_loaded = clock64();
    bool capped = false, guard = false;
    int rounds = 0;
    if (narrow) {
      if (warp < 4) rounds = relax_tile<uint32_t>(lab32, rc, capK32, s_mask, &guard, &err);
      else if (tid == 4 * 32) s_next = q_try_pop(ring, q, slots, inq);  // the next tile, if one is waiting
      __syncthreads();
      capped = tile_capped<uint32_t>(lab32, rc, capK32);
      if (__syncthreads_or((local && capped) || guard)) {
        // a candidate left the 32-bit range: the 64-bit visit from the loaded labels
        narrow = false;
        guard = false;
        if (tid == 0) atomicAdd(&ctr->redo64, 1ull);
        // the reduced costs again: from the cache entry (written above on a miss),
        // else built anew (potentials are loaded on every uncached visit)
        if (cached) rc_from_cache(rc_entry, rc);
        else build_rc<FWD, false>(p, i0, j0, spot, rc, &err);
        __syncthreads();
      }
    }
    if (!narrow) {
      if (warp < 4) rounds += relax_tile<uint64_t>(lab, rc, capK, s_mask, &guard, &err);
      else if (tid == 4 * 32 && s_next < 0) s_next = q_try_pop(ring, q, slots, inq);
      __syncthreads();
      capped = tile_capped<uint64_t>(lab, rc, capK);
      if (guard) err |= kErrInternal;  // no fixed point within the round limit
    }
    __syncthreads();
    const long long t_relaxed = clock64();
    // write back and note which tile sides changed; count the reached nodes
    unsigned reached = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int ly = warp + 8 * k;
      int64_t i = i0 + ly, j = j0 + lane;
      uint64_t v = lab[ly + 1][lane + 1];
      if (narrow) {
        const uint32_t x = lab32[ly + 1][lane + 1];
        v = x == 0xFFFFFFFFu ? kInf
                             : (((uint64_t)((x >> 18) + d0) << 32) | ((uint64_t)(((x >> 3) & 0x7FFFu) + h0) << 3) |
                                (uint64_t)(x & 7u));
      }
      reached += __popc(__ballot_sync(0xffffffffu, i < p.R && j < p.C && v != kInf));
      if (i < p.R && j < p.C && v != orig[k]) {
        // the same tile may be in process in two CTAs (it can be re-queued
        // while in flight); atomicMin keeps every label monotone
        atomicMin((unsigned long long*)&plab[i * p.C + j], (unsigned long long)v);
        if (ly == 0) side[0] = 1;
        if (ly == TS - 1) side[1] = 1;
        if (lane == 0) side[2] = 1;
        if (lane == TS - 1) side[3] = 1;
      }
    }
    if (narrow && tid == 0) atomicAdd(&ctr->visits32, 1ull);
    if (lane == 0 && reached) atomicAdd(&ctr->settled_visits, (unsigned long long)reached);
    if (__syncthreads_or(capped) && tid == 0) {
      capped_flag[tile] = 1;
      ctr->capped_any = 1;
    }
    __threadfence();
    __syncthreads();
    // the neighbours across the changed sides, one thread each (0 above, 1 below,
    // 2 left, 3 right); each push is made visible before the visit counts as done
    if (tid < 4 && side[tid]) {
      const bool exists = tid == 0 ? ti > 0 : tid == 1 ? ti + 1 < p.tiles_y : tid == 2 ? tj > 0 : tj + 1 < p.tiles_x;
      const int nb = tid == 0 ? tile - (int)p.tiles_x : tid == 1 ? tile + (int)p.tiles_x : tid == 2 ? tile - 1 : tile + 1;
      if (exists && !q_push(nb, ring, q, slots, inq, wait_polls)) err |= kErrSpin;
      __threadfence();
    }
    if (tid == 32) {
      atomicAdd(&ctr->tile_visits, 1ull);
      atomicAdd(&ctr->local_rounds, (unsigned long long)rounds);
      atomicAdd(&ctr->visit_cycles, (unsigned long long)(clock64() - t_start));
      atomicAdd(&ctr->load_cycles, (unsigned long long)(t_loaded - t_start));
      atomicAdd(&ctr->relax_cycles, (unsigned long long)(t_relaxed - t_loaded));
    }
    __syncthreads();
    if (tid == 0) atomicSub(&q->pending, 1);
  }
  if (err) atomicOr(&ctr->err, err);
}

__device__ __forceinline__ int32_t* cand_cur(int32_t* base, const McfCtr* c, int64_t) {
  return base + (c->cand_sel ? c->n_cap_nodes : 0);
}
__device__ __forceinline__ int32_t* cand_nxt(int32_t* base, const McfCtr* c, int64_t) {
  return base + (c->cand_sel ? 0 : c->n_cap_nodes);
}

// A problem joins: imbalances from its residues, its imbalanced nodes appended
// to the current list, every node potential set to the current ground
// potential (all its reduced costs then equal its raw costs, >= 0) and every
// label unreached.
// Grid: x over the problem's nodes, y over the listed slots.
__global__ void k_init_state(Batch b, const int32_t* slots, int32_t* excess, int32_t* cand_base, int64_t* pot,
                             uint64_t* labels, int32_t* prob_left, McfCtr* ctr) {
  const int slot = slots[blockIdx.y];
  const ProbDev& p = b.probs[slot];
  const int64_t pg = pot[b.g_index];
  int32_t* cand = cand_cur(cand_base, ctr, ctr->n_cap_nodes);
  const int64_t P = p.m * p.n;
  int cnt = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < p.N; v += (int64_t)gridDim.x * blockDim.x) {
    int32_t r = p.res[v];
    if (p.resume) {
      // imbalance left by the given flows: supply minus net outflow of node (i, j),
      // whose four edges are h(i,j) [above], h(i+1,j) [below], v(i,j) [left], v(i,j+1)
      const int64_t i = v / p.C, j = v - (v / p.C) * p.C;
      const int net = (int)p.flows[(i + 1) * p.n + j] - (int)p.flows[i * p.n + j] + (int)p.flows[P + i * p.n + j] -
                      (int)p.flows[P + i * p.n + j + 1];
      r -= net;
    } else {
      pot[p.node_off + v] = pg;
    }
    excess[p.node_off + v] = r;
    labels[p.node_off + v] = kInf;
    // one list append per warp: the warp's imbalanced nodes take consecutive
    // slots in lane order (the list order does not matter to the solver)
    const unsigned act = __activemask(), bal = __ballot_sync(act, r != 0);
    const int lead = __ffs((int)act) - 1, lane = (int)(threadIdx.x & 31);
    int base = 0;
    if (lane == lead && bal) base = atomicAdd(&ctr->ncand, __popc(bal));
    base = __shfl_sync(act, base, lead);
    if (r != 0) {
      cand[base + __popc(bal & ((1u << lane) - 1u))] = (int32_t)(p.node_off + v);
      ++cnt;
    }
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&prob_left[slot], cnt);
}

// Per-pass setup: distance cap (full search while many imbalanced nodes
// remain, a band of band_mult x the last augmented distance once few are left),
// counters and the worklist.
__global__ void k_pass_setup(McfCtr* ctr, SearchQ* q) {
  if (!ctr->go_on) return;
  ctr->nseg = 0;
  ctr->D = 0;
  ctr->naug = 0;
  ctr->found = 0;
  ctr->capped_any = 0;
  ctr->band_again = 1;
  uint32_t cap = 0xFFFFFFFFu;
  if ((uint32_t)ctr->passes >= ctr->full_passes &&
      (long long)ctr->ncand * 1000000ll < (long long)ctr->band_start_ppm * ctr->n_total) {
    const unsigned long long c = (unsigned long long)ctr->band_mult * ctr->last_D;
    const unsigned long long lo = ctr->band_min;
    cap = (uint32_t)(c < lo ? lo : (c > 0x7FFFFFFFull ? 0x7FFFFFFFull : c));
    if (cap == 0) cap = 1;
  }
  ctr->cap0 = cap;
  ctr->zstop = (cap != 0xFFFFFFFFu && (uint32_t)ctr->ncand <= ctr->zero_stop_below) ? 1 : 0;
  ctr->zstage = 0;
  if (ctr->zstop) cap = 1;  // distance 0 only: the zero band first
  ctr->cap = cap;
  ctr->gsink = (uint32_t)ctr->ncand <= ctr->ground_sink_below ? 1 : 0;
  ctr->dG = 0xFFFFFFFFu;
  q->head = q->tail = q->pending = 0;
}

// Labels at the start of a pass: every label is unreached already (set when a
// problem joins, and reset after each pass on the tiles the search visited and
// at the listed nodes), so only the roots are set, to distance 0: the excess
// nodes forward, the deficit nodes reverse.
template <bool FWD>
__global__ void k_set_roots(const int32_t* excess, int32_t* cand_base, int64_t n_total, uint64_t* labels,
                            const McfCtr* ctr) {
  if (!ctr->go_on) return;
  const int nc = ctr->ncand;
  const int32_t* cand = cand_cur(cand_base, ctr, n_total);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += gridDim.x * blockDim.x) {
    const int32_t v = cand[q];
    const int32_t e = excess[v];
    if (FWD ? e > 0 : e < 0) labels[v] = 0ull;
  }
}

__device__ __forceinline__ int32_t& ctr_err(const McfCtr* c) { return const_cast<McfCtr*>(c)->err; }

// Seed the worklist: tiles holding a root, and the border tiles (the ground
// node is a root) of every problem that is not yet balanced.
template <bool FWD>
__global__ void k_seed_tiles(Batch b, const int32_t* excess, int32_t* cand_base, const McfCtr* ctr,
                             const int32_t* prob_left, const int32_t* border, int32_t n_border, SearchQ* q,
                             int32_t* slots, int32_t* inq, int search_grid) {
  if (!ctr->go_on) return;
  const int nc = ctr->ncand;
  const int32_t* cand = cand_cur(cand_base, ctr, b.n_total);
  const int ring = (int)b.t_total + search_grid + 64;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nc + n_border;
       k += (int64_t)gridDim.x * blockDim.x) {
    int tile;
    if (k < nc) {
      int32_t v = cand[k];
      int32_t e = excess[v];
      if (!(FWD ? e > 0 : e < 0)) continue;
      const ProbDev& p = b.probs[prob_of_node(b, v)];
      int64_t loc = v - p.node_off, i = loc / p.C, j = loc % p.C;
      const int64_t ti = i / TS, tj = j / TS;
      tile = (int)(p.tile_off + ti * p.tiles_x + tj);
      // a root's label is set before the search, not by a tile visit, so no visit
      // reports it as changed: a root on a tile edge also seeds the tile across
      // that edge, which reads it as halo
      bool ok = true;
      const uint32_t lim = ctr->wait_polls;
      if (i % TS == 0 && ti > 0) ok &= q_push(tile - p.tiles_x, ring, q, slots, inq, lim);
      if (i % TS == TS - 1 && ti + 1 < p.tiles_y) ok &= q_push(tile + p.tiles_x, ring, q, slots, inq, lim);
      if (j % TS == 0 && tj > 0) ok &= q_push(tile - 1, ring, q, slots, inq, lim);
      if (j % TS == TS - 1 && tj + 1 < p.tiles_x) ok &= q_push(tile + 1, ring, q, slots, inq, lim);
      if (!ok) atomicOr(&ctr_err(ctr), kErrSpin);
    } else {
      if (ctr->gsink) continue;  // the ground is no root in this pass
      tile = border[k - nc];
      if (prob_left[b.tile_prob[tile]] == 0) continue;
    }
    if (!q_push(tile, ring, q, slots, inq, ctr->wait_polls)) atomicOr(&ctr_err(ctr), kErrSpin);
  }
}

// Candidates (deficits forward, excess nodes reverse) reached by the search.
template <bool FWD>
__global__ void k_count_found(const int32_t* excess, const uint64_t* labels, int32_t* cand_base, int64_t n_total,
                              McfCtr* ctr) {
  if (!ctr->band_again) return;
  const int nc = ctr->ncand;
  const int32_t* cand = cand_cur(cand_base, ctr, n_total);
  int c = 0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += gridDim.x * blockDim.x) {
    int32_t t = cand[q];
    int32_t e = excess[t];
    if ((FWD ? e < 0 : e > 0) && labels[t] != kInf) ++c;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && ctr->gsink && ctr->dG != 0xFFFFFFFFu) ++c;  // the ground
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(&ctr->found, c);
}

// After a band: widen (x band_growth, or unbounded on the last band) if no candidate was
// reached and some tile dropped candidates at the cap; otherwise the band loop
// is over.  Runs on one thread.
__global__ void k_band_decide(McfCtr* ctr, SearchQ* q, int last_band) {
  if (!ctr->band_again) return;
  bool again = ctr->cap != 0xFFFFFFFFu && ctr->found == 0 && ctr->capped_any && ctr->err == 0;
  if (again) {
    const unsigned long long w = (unsigned long long)ctr->cap * ctr->band_growth;
    if (ctr->zstop && ctr->cap == 1u && ctr->zstage < 2 && ctr->zhop[ctr->zstage + 1] > ctr->zhop[ctr->zstage]) {
      ctr->zstage += 1;  // the zero band with the next hop radius
    } else if (ctr->zstop && ctr->cap == 1u) {
      ctr->cap = ctr->cap0;  // after the zero band: the pass's ordinary first band
      ctr->zstop = 0;
    } else {
      ctr->cap = (last_band || w >= 0x7FFFFFFFull) ? 0xFFFFFFFFu : (uint32_t)w;
    }
    q->head = q->tail = q->pending = 0;
    ctr->capped_any = 0;
  }
  ctr->band_again = again ? 1 : 0;
}

// Widen the band: queue every tile that dropped a candidate.
__global__ void k_reseed(Batch b, int32_t* capped_flag, SearchQ* q, int32_t* slots, int32_t* inq, int search_grid,
                         McfCtr* ctr) {
  if (!ctr->band_again) return;
  const int ring = (int)b.t_total + search_grid + 64;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < b.t_total;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (capped_flag[t]) {
      capped_flag[t] = 0;
      if (!q_push((int)t, ring, q, slots, inq, ctr->wait_polls)) atomicOr(&ctr->err, kErrSpin);
    }
  }
}

// After the last band: drop the leftover "dropped at cap" flags.
__global__ void k_clear_capped(Batch b, int32_t* capped_flag, const McfCtr* ctr) {
  if (!ctr->go_on) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < b.t_total;
       t += (int64_t)gridDim.x * blockDim.x)
    capped_flag[t] = 0;
}

// One step from node (i, j) toward its parent in direction d; false when the
// parent is the ground node (d points out of the grid).
__device__ __forceinline__ bool step_parent(const ProbDev& p, int d, int64_t* i, int64_t* j) {
  switch (d) {
    case kDirUp: if (*i == 0) return false; --*i; return true;
    case kDirDown: if (*i + 1 >= p.R) return false; ++*i; return true;
    case kDirLeft: if (*j == 0) return false; --*j; return true;
    default: if (*j + 1 >= p.C) return false; ++*j; return true;
  }
}

// The root of local node v's search tree: the end of its parent chain, a root
// (direction kDirRoot) or the node whose parent is the ground.  The walk crosses
// a tile per step: from a node to the last node of its parent chain inside its
// tile (k_tile_exits), then one step to that node's parent.  Every node on the
// chain holds a label of this pass, so its tile was visited and its exit is
// current.  -1 if the chain is longer than the grid (corrupt labels).
__device__ __forceinline__ int64_t walk_root_tiles(const ProbDev& p, const uint64_t* plab, const uint16_t* pexit,
                                                   int64_t v) {
  int64_t i = v / p.C, j = v - (v / p.C) * p.C;
  for (int64_t steps = 0; steps <= p.N; ++steps) {
    const int ex = pexit[i * p.C + j];
    i = (i / TS) * TS + ex / TS;
    j = (j / TS) * TS + ex % TS;
    const int d = label_dir(plab[i * p.C + j]);
    if (d == kDirRoot) return i * p.C + j;
    if (!step_parent(p, d, &i, &j)) return i * p.C + j;  // parent is the ground
  }
  return -1;
}

// After a pass's search: for every node of a tile the pass visited, the
// tile-local index of the node where its parent chain leaves the tile (the node
// itself when its parent lies outside the tile or is the ground, or when it is
// a root or unreached), by pointer jumping in shared memory: a chain inside a
// tile has at most 1024 nodes, so 10 rounds.  Labels are final here (the
// search has converged), and parent chains have no cycles.
__global__ void __launch_bounds__(256) k_tile_exits(Batch b, const uint64_t* labels, const int32_t* tlist,
                                                    uint16_t* exits, const McfCtr* ctr) {
  if (!ctr->go_on || ctr->err) return;
  __shared__ uint16_t e[2][TS * TS];
  const int nt = ctr->ntouched;
  for (int k = blockIdx.x; k < nt; k += gridDim.x) {
    const int tile = tlist[k];
    const ProbDev& p = b.probs[b.tile_prob[tile]];
    const int64_t lt = tile - p.tile_off;
    const int64_t i0 = (lt / p.tiles_x) * TS, j0 = (lt % p.tiles_x) * TS;
    const uint64_t* plab = labels + p.node_off;
    for (int q = threadIdx.x; q < TS * TS; q += blockDim.x) {
      const int r = q / TS, c = q % TS;
      int nx = q;
      if (i0 + r < p.R && j0 + c < p.C) {
        const uint64_t lab = plab[(i0 + r) * p.C + j0 + c];
        if (lab != kInf) {
          int rr = r, cc = c;
          switch (label_dir(lab)) {
            case kDirUp: --rr; break;
            case kDirDown: ++rr; break;
            case kDirLeft: --cc; break;
            case kDirRight: ++cc; break;
            default: rr = -1; break;  // a root
          }
          if (rr >= 0 && rr < TS && cc >= 0 && cc < TS && i0 + rr < p.R && j0 + cc < p.C) nx = rr * TS + cc;
        }
      }
      e[0][q] = (uint16_t)nx;
    }
    __syncthreads();
    int cur = 0;
    for (int round = 0; round < 10; ++round) {
      for (int q = threadIdx.x; q < TS * TS; q += blockDim.x) e[cur ^ 1][q] = e[cur][e[cur][q]];
      cur ^= 1;
      __syncthreads();
    }
    for (int q = threadIdx.x; q < TS * TS; q += blockDim.x) {
      const int r = q / TS, c = q % TS;
      if (i0 + r < p.R && j0 + c < p.C) exits[p.node_off + (i0 + r) * p.C + j0 + c] = e[cur][q];
    }
    __syncthreads();
  }
}

// Ground arc k of a problem (k < 2C + 2R): its border node (local) and the side
// of the node the ground lies on.
__device__ __forceinline__ void ground_arc(const ProbDev& p, int64_t k, int64_t* v, int* side) {
  if (k < p.C) {
    *v = k;
    *side = kDirUp;
  } else if (k < 2 * p.C) {
    *v = (p.R - 1) * p.C + (k - p.C);
    *side = kDirDown;
  } else if (k < 2 * p.C + p.R) {
    *v = (k - 2 * p.C) * p.C;
    *side = kDirLeft;
  } else {
    *v = (k - 2 * p.C - p.R) * p.C + p.C - 1;
    *side = kDirRight;
  }
}

// Distance through ground arc k (forward search: v -> G; reverse: G -> v), or
// 0xFFFFFFFF when v is unreached or the arc is not residual.
template <bool FWD>
__device__ __forceinline__ uint32_t ground_arc_dist(const ProbDev& p, const uint64_t* plab, const int64_t* ppot,
                                                    int64_t pG, int64_t k, int64_t* vout, int* sout) {
  int64_t v;
  int side;
  ground_arc(p, k, &v, &side);
  *vout = v;
  *sout = side;
  const uint64_t l = plab[v];
  if (l == kInf) return 0xFFFFFFFFu;
  int32_t c;
  // forward search: the arc leaving v toward the ground; reverse: entering v from it
  if (!arc_cost<!FWD>(p, v / p.C, v % p.C, side, &c)) return 0xFFFFFFFFu;
  const int64_t red = FWD ? (int64_t)c - ppot[v] + pG : (int64_t)c - pG + ppot[v];
  const int64_t d = (int64_t)(l >> 32) + (red < 0 ? 0 : red);
  return d >= 0xFFFFFFFFll ? 0xFFFFFFFEu : (uint32_t)d;
}

// Ground-sink passes: dG = the ground's distance (below the band cap).
// Grid: x over a problem's ground arcs, y over the active problems.
template <bool FWD>
__global__ void k_ground_dist(Batch b, const uint64_t* labels, const int64_t* pot, McfCtr* ctr) {
  if (!ctr->go_on || !ctr->gsink || !ctr->band_again) return;
  const ProbDev& p = b.probs[b.order[blockIdx.y]];
  const int64_t na = 2 * (p.C + p.R), pG = pot[b.g_index];
  const uint32_t cap = ctr->cap;
  uint32_t best_d = 0xFFFFFFFFu;
  bool beyond = false;  // the ground is reachable, but only at or past the cap
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < na; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t v;
    int side;
    const uint32_t d = ground_arc_dist<FWD>(p, labels + p.node_off, pot + p.node_off, pG, k, &v, &side);
    if (d < cap && d < best_d) best_d = d;
    if (d != 0xFFFFFFFFu && d >= cap) beyond = true;
  }
  for (int o = 16; o > 0; o >>= 1) best_d = min(best_d, __shfl_xor_sync(0xffffffffu, best_d, o));
  if ((threadIdx.x & 31) == 0 && best_d != 0xFFFFFFFFu) atomicMin(&ctr->dG, best_d);
  // like a label dropped at the cap: a wider band may reach the ground
  if (__any_sync(0xffffffffu, beyond) && (threadIdx.x & 31) == 0) ctr->capped_any = 1;
}

__device__ __forceinline__ uint32_t ground_vid(const ProbDev& p, int64_t k) {
  return 0x80000000u | (uint32_t)(p.garc_off + k);
}

// Trees that reach the ground at exactly dG propose it (ground candidates farther
// away could not augment: the pass radius is at most dG).
template <bool FWD>
__global__ void k_select_ground(Batch b, const uint64_t* labels, const uint16_t* exits, const int64_t* pot,
                                uint64_t* best, McfCtr* ctr) {
  if (!ctr->go_on || ctr->err || !ctr->gsink || ctr->dG == 0xFFFFFFFFu) return;
  const ProbDev& p = b.probs[b.order[blockIdx.y]];
  const int64_t na = 2 * (p.C + p.R), pG = pot[b.g_index];
  const uint64_t* plab = labels + p.node_off;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < na; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t v;
    int side;
    const uint32_t d = ground_arc_dist<FWD>(p, plab, pot + p.node_off, pG, k, &v, &side);
    if (d != ctr->dG) continue;
    const int64_t r = walk_root_tiles(p, plab, exits + p.node_off, v);
    if (r < 0) {
      atomicOr(&ctr->err, kErrWalk);
      continue;
    }
    atomicMin((unsigned long long*)&best[p.node_off + r], ((uint64_t)d << 32) | ground_vid(p, k));
  }
}

template <bool FWD>
__global__ void k_select(Batch b, const int32_t* excess, const uint64_t* labels, const uint16_t* exits,
                         int32_t* cand_base, int32_t* cand_root, uint64_t* best, McfCtr* ctr) {
  if (!ctr->go_on) return;
  // a search that stopped on an error left labels that are not shortest
  // distances: the pass then augments nothing, so flows and potentials stay
  // the consistent pair of the last complete pass (a resumable state)
  const bool aborted = ctr->err != 0;
  const int nc = ctr->ncand;
  const int32_t* cand = cand_cur(cand_base, ctr, b.n_total);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += gridDim.x * blockDim.x) {
    int32_t t = cand[q];
    int32_t e = excess[t];
    cand_root[q] = -1;
    if (aborted) continue;
    if (!(FWD ? e < 0 : e > 0)) continue;
    uint64_t l = labels[t];
    if (l == kInf) continue;
    const ProbDev& p = b.probs[prob_of_node(b, t)];
    int64_t r = walk_root_tiles(p, labels + p.node_off, exits + p.node_off, t - p.node_off);
    if (r < 0) {
      atomicOr(&ctr->err, kErrWalk);
      continue;
    }
    r += p.node_off;
    cand_root[q] = (int32_t)r;
    atomicMin((unsigned long long*)&best[r], ((l >> 32) << 32) | (uint64_t)(uint32_t)t);
  }
}

// s = +1 if a move u -> v along the parent direction d of v (u is v's parent) raises dk
__device__ __forceinline__ void dir_edge(const ProbDev& p, int64_t i, int64_t j, int d, int64_t* e, int* plane,
                                         int* s) {
  switch (d) {
    case kDirUp: *e = i * p.n + j; *plane = 0; *s = 1; break;
    case kDirDown: *e = (i + 1) * p.n + j; *plane = 0; *s = -1; break;
    case kDirLeft: *e = i * p.n + j; *plane = 1; *s = -1; break;
    default: *e = i * p.n + j + 1; *plane = 1; *s = 1; break;
  }
}

// Flip dk along the path from local node v to its tree root (forward: the flow
// runs root -> v; reverse: v -> root), stopping at the root or the ground.
// The parent's label is loaded before the flow of the current edge is
// updated, so that the two memory round trips of a step overlap.
template <bool FWD>
__device__ __forceinline__ void flip_path(const ProbDev& p, const uint64_t* plab, int64_t v) {
  const int64_t P = p.m * p.n;
  int64_t i = v / p.C, j = v - (v / p.C) * p.C;
  uint64_t lab = plab[v];
  for (int64_t steps = 0; steps <= p.N; ++steps) {
    const int d = label_dir(lab);
    if (d == kDirRoot) break;
    int64_t e;
    int plane, s;
    dir_edge(p, i, j, d, &e, &plane, &s);
    const bool inside = step_parent(p, d, &i, &j);
    if (inside) lab = plab[i * p.C + j];
    p.flows[plane * P + e] += (int8_t)(FWD ? s : -s);
    if (!inside) break;
  }
}

// The winner of every tree: its unit of flow runs along its path (forward: root
// -> t; reverse: t -> root).  The paths of one pass lie in different trees, so
// they share no node; each is cut into its tile segments (from a node to the
// end of its chain inside the tile, k_tile_exits), whose first nodes are listed
// for k_flip_segments, which flips every segment at once.
template <bool FWD>
__global__ void k_augment(Batch b, int32_t* excess, const uint64_t* labels, const uint16_t* exits, int32_t* cand_base,
                          const int32_t* cand_root, const uint64_t* best, long long* g_net, int32_t* segs,
                          McfCtr* ctr) {
  if (!ctr->go_on) return;
  const int nc = ctr->ncand;
  const int32_t* cand = cand_cur(cand_base, ctr, b.n_total);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += gridDim.x * blockDim.x) {
    int32_t r = cand_root[q];
    if (r < 0) continue;
    int32_t t = cand[q];
    uint64_t l = labels[t];
    if (best[r] != (((l >> 32) << 32) | (uint64_t)(uint32_t)t)) continue;
    if (ctr->gsink && (uint32_t)(l >> 32) > ctr->dG) continue;  // beyond the ground: not this pass
    atomicMax(&ctr->D, (uint32_t)(l >> 32));
    atomicAdd(&ctr->naug, 1);
    const int pi = prob_of_node(b, t);
    const ProbDev& p = b.probs[pi];
    const uint64_t* plab = labels + p.node_off;
    const uint16_t* pexit = exits + p.node_off;
    int64_t v = t - p.node_off;
    int64_t i = v / p.C, j = v - (v / p.C) * p.C;
    for (int64_t steps = 0; steps <= p.N; ++steps) {
      segs[atomicAdd(&ctr->nseg, 1)] = (int32_t)(p.node_off + i * p.C + j);
      const int ex = pexit[i * p.C + j];
      i = (i / TS) * TS + ex / TS;
      j = (j / TS) * TS + ex % TS;
      const int d = label_dir(plab[i * p.C + j]);
      if (d == kDirRoot || !step_parent(p, d, &i, &j)) break;  // the root, or the ground past the exit
    }
    bool real_root = label_dir(labels[r]) == kDirRoot;
    if (FWD) {
      excess[t] += 1;
      if (real_root) excess[r] -= 1;
      else atomicAdd((unsigned long long*)&g_net[pi], 1ull);  // the ground node emitted a unit
    } else {
      excess[t] -= 1;
      if (real_root) excess[r] += 1;
      else atomicAdd((unsigned long long*)&g_net[pi], ~0ull);  // the ground node absorbed a unit
    }
  }
}

// Flip dk along every listed tile segment: from its first node along the parent
// directions to the end of its chain inside the tile, including the edge from
// that node to its parent (the next segment's first node, or the ground), but
// not past a root.  The parent's label is loaded before the flow of the
// current edge is updated, so that the two memory round trips of a step overlap.
template <bool FWD>
__global__ void k_flip_segments(Batch b, const uint64_t* labels, const uint16_t* exits, const int32_t* segs,
                                const McfCtr* ctr) {
  if (!ctr->go_on) return;
  const int ns = ctr->nseg;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < ns; q += gridDim.x * blockDim.x) {
    const int32_t g = segs[q];
    const ProbDev& p = b.probs[prob_of_node(b, g)];
    const uint64_t* plab = labels + p.node_off;
    const uint16_t* pexit = exits + p.node_off;
    const int64_t P = p.m * p.n, v = g - p.node_off;
    int64_t i = v / p.C, j = v - (v / p.C) * p.C;
    uint64_t lab = plab[v];
    for (int64_t steps = 0; steps <= TS * TS; ++steps) {
      const int d = label_dir(lab);
      if (d == kDirRoot) break;
      // the end of the chain inside the tile: its own exit
      const bool last = pexit[i * p.C + j] == (uint16_t)((i % TS) * TS + (j % TS));
      int64_t e;
      int plane, s;
      dir_edge(p, i, j, d, &e, &plane, &s);
      const bool inside = step_parent(p, d, &i, &j);
      if (inside && !last) lab = plab[i * p.C + j];
      p.flows[plane * P + e] += (int8_t)(FWD ? s : -s);
      if (!inside || last) break;
    }
  }
}

__global__ void k_reset_best(Batch b, const int32_t* cand_root, uint64_t* best, int32_t* prob_left, int nslots,
                             const McfCtr* ctr) {
  if (!ctr->go_on) return;
  const int nc = ctr->ncand;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += gridDim.x * blockDim.x) {
    int32_t r = cand_root[q];
    if (r >= 0) best[r] = kInf;
  }
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nslots; q += gridDim.x * blockDim.x) prob_left[q] = 0;
}

// Trees whose best candidate is the ground: one unit through the ground arc
// (forward: root -> ... -> v -> G, the ground absorbs; reverse: G -> v -> ... -> root).
template <bool FWD>
__global__ void k_augment_ground(Batch b, int32_t* excess, const uint64_t* labels, const uint16_t* exits,
                                 const int64_t* pot, uint64_t* best, long long* g_net, McfCtr* ctr) {
  if (!ctr->go_on || ctr->err || !ctr->gsink || ctr->dG == 0xFFFFFFFFu) return;
  const int slot = b.order[blockIdx.y];
  const ProbDev& p = b.probs[slot];
  const int64_t na = 2 * (p.C + p.R), pG = pot[b.g_index], P = p.m * p.n;
  const uint64_t* plab = labels + p.node_off;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < na; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t v;
    int side;
    const uint32_t d = ground_arc_dist<FWD>(p, plab, pot + p.node_off, pG, k, &v, &side);
    if (d != ctr->dG) continue;
    const int64_t r = walk_root_tiles(p, plab, exits + p.node_off, v);
    if (r < 0 || best[p.node_off + r] != (((uint64_t)d << 32) | ground_vid(p, k))) continue;
    // clear the tree's word here: once the ground arc is flipped it is no longer
    // residual, so no later pass over the arcs could tell which trees proposed it
    best[p.node_off + r] = kInf;
    atomicMax(&ctr->D, d);
    atomicAdd(&ctr->naug, 1);
    // the ground arc: on the move v -> G, v is the parent of G, which lies on `side` of v
    const int64_t i = v / p.C, j = v % p.C;
    int64_t e;
    int plane, sgn;
    dir_edge(p, i, j, side, &e, &plane, &sgn);
    p.flows[plane * P + e] += (int8_t)(FWD ? -sgn : sgn);
    flip_path<FWD>(p, plab, v);
    if (FWD) {
      excess[p.node_off + r] -= 1;
      atomicAdd((unsigned long long*)&g_net[slot], ~0ull);  // the ground absorbed a unit
    } else {
      excess[p.node_off + r] += 1;
      atomicAdd((unsigned long long*)&g_net[slot], 1ull);  // the ground emitted a unit
    }
  }
}

// After a pass, on the tiles the search visited (one block per tile, grid-
// stride over the list): potentials p += D - d forward (p -= D - d reverse)
// for the nodes labelled below the largest augmented distance D, then every
// label back to unreached and the tile unlisted.  Nodes outside these tiles
// hold no label (roots lie on seeded tiles, which the search visits).
template <bool FWD>
__global__ void k_potentials(Batch b, uint64_t* labels, int64_t* pot, int32_t* touched, const int32_t* tlist,
                             const McfCtr* ctr) {
  const bool apply = ctr->go_on && ctr->err == 0 && ctr->naug != 0 && ctr->D != 0;  // D = 0: none below it
  const uint32_t D = ctr->D;
  const int nt = ctr->ntouched;
  for (int k = blockIdx.x; k < nt; k += gridDim.x) {
    const int tile = tlist[k];
    const ProbDev& p = b.probs[b.tile_prob[tile]];
    const int64_t lt = tile - p.tile_off;
    const int64_t i0 = (lt / p.tiles_x) * TS, j0 = (lt % p.tiles_x) * TS;
    for (int q = threadIdx.x; q < TS * TS; q += blockDim.x) {
      const int64_t i = i0 + q / TS, j = j0 + q % TS;
      if (i >= p.R || j >= p.C) continue;
      const int64_t v = p.node_off + i * p.C + j;
      const uint64_t l = labels[v];
      if (l == kInf) continue;
      const uint32_t d = (uint32_t)(l >> 32);
      if (apply && d < D) pot[v] += FWD ? (int64_t)(D - d) : -(int64_t)(D - d);
      labels[v] = kInf;
    }
    if (threadIdx.x == 0) touched[tile] = 0;
  }
}

// The ground node is a root of every search (distance 0).
template <bool FWD>
__global__ void k_potential_ground(Batch b, int64_t* pot, const McfCtr* ctr) {
  if (!ctr->go_on || ctr->err || ctr->naug == 0 || ctr->gsink) return;  // a sink ground lies at distance >= D
  pot[b.g_index] += FWD ? (int64_t)ctr->D : -(int64_t)ctr->D;
}

__global__ void k_compact(Batch b, const int32_t* excess, int32_t* cand_base, uint64_t* labels, int32_t* prob_left,
                          McfCtr* ctr) {
  if (!ctr->go_on) return;
  const int nc = ctr->ncand;
  const int32_t* cand = cand_cur(cand_base, ctr, b.n_total);
  int32_t* next = cand_nxt(cand_base, ctr, b.n_total);
  const int lane = (int)(threadIdx.x & 31);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += gridDim.x * blockDim.x) {
    int32_t v = cand[q];
    labels[v] = kInf;  // a root on a tile the search did not reach (an aborted search)
    const bool keep = excess[v] != 0;
    // one list append per warp (slots in lane order), one count per problem in the warp
    const unsigned act = __activemask(), bal = __ballot_sync(act, keep);
    const int lead = __ffs((int)act) - 1;
    int base = 0;
    if (lane == lead && bal) base = atomicAdd(&ctr->ncand_next, __popc(bal));
    base = __shfl_sync(act, base, lead);
    const int slot = keep ? prob_of_node(b, v) : -1;
    const unsigned same = __match_any_sync(act, slot);
    if (keep) {
      next[base + __popc(bal & ((1u << lane) - 1u))] = v;
      if (lane == __ffs((int)same) - 1) atomicAdd(&prob_left[slot], __popc(same));
    }
  }
}

// End of a pass: swap the candidate lists and decide whether to go on.
__global__ void k_finish_pass(McfCtr* ctr) {
  ctr->touched_total += (unsigned long long)ctr->ntouched;
  ctr->ntouched = 0;  // the list was reset with the labels
  if (!ctr->go_on) return;
  ctr->ncand = ctr->ncand_next;
  ctr->ncand_next = 0;
  ctr->cand_sel ^= 1;
  ctr->passes += 1;
  ctr->aug_total += ctr->naug;
  if (ctr->naug > 0) {
    ctr->last_D = ctr->D;
    ctr->idle = 0;
  } else {
    ctr->idle += 1;
  }
  int st = WW_OK;
  if (ctr->err & kErrOverflow) st = WW_ERR_OVERFLOW;
  else if (ctr->err & kErrSpin) st = WW_ERR_TIMEOUT;
  else if (ctr->err) st = WW_ERR_INTERNAL;
  else if (ctr->ncand > 0 && ctr->idle >= 2) st = WW_ERR_INFEASIBLE;
  else if (ctr->ncand > 0 && ctr->passes >= ctr->max_passes) st = WW_ERR_TIMEOUT;
  ctr->status = st;
  ctr->go_on = (st == WW_OK && ctr->ncand > 0) ? 1 : 0;
}

// Total cost of the listed slots; grid: x over a problem's pixels, y over the list.
// Flows are mostly zero: with both planes 16-byte aligned the flows are read
// 16 edges at a time and the costs only where an edge carries flow.
__device__ __forceinline__ long long edge_cost(const ProbDev& p, int64_t P, int64_t e, int a, int c) {
  long long s = 0;
  if (a == 1) s += p.costs[e];
  if (a == -1) s += p.costs[P + e];
  if (c == 1) s += p.costs[2 * P + e];
  if (c == -1) s += p.costs[3 * P + e];
  return s;
}

__global__ void k_total_cost(Batch b, const int32_t* slots, long long* tc) {
  const int slot = slots[blockIdx.y];
  const ProbDev& p = b.probs[slot];
  const int64_t P = p.m * p.n;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
  long long s = 0;
  if ((reinterpret_cast<uintptr_t>(p.flows) & 15) == 0 && (P & 15) == 0) {
    const uint4* fa = reinterpret_cast<const uint4*>(p.flows);
    const uint4* fc = reinterpret_cast<const uint4*>(p.flows + P);
    for (int64_t k = t0; k < P / 16; k += stride) {
      const uint4 a = fa[k], c = fc[k];
      if ((a.x | a.y | a.z | a.w | c.x | c.y | c.z | c.w) == 0) continue;
      const int8_t* ab = reinterpret_cast<const int8_t*>(&a);
      const int8_t* cb = reinterpret_cast<const int8_t*>(&c);
#pragma unroll
      for (int t = 0; t < 16; ++t)
        if (ab[t] | cb[t]) s += edge_cost(p, P, 16 * k + t, ab[t], cb[t]);
    }
  } else {
    for (int64_t e = t0; e < P; e += stride) s += edge_cost(p, P, e, p.flows[e], p.flows[P + e]);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd((unsigned long long*)&tc[slot], (unsigned long long)s);
}

// Potentials out for the listed slots (when the solve used library storage).
__global__ void k_copy_pot(Batch b, const int32_t* slots, const int64_t* pot) {
  const ProbDev& p = b.probs[slots[blockIdx.y]];
  if (!p.pot_out) return;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= p.N; v += (int64_t)gridDim.x * blockDim.x)
    p.pot_out[v] = v < p.N ? pot[p.node_off + v] : pot[b.g_index];
}

// Status and total cost of the listed slots; ground balance check (G's net
// outflow must equal r_G once every other node is balanced).
__global__ void k_write_results(Batch b, const int32_t* slots, int nlist, const McfCtr* ctr, const long long* g_net,
                                const long long* tc, int32_t* status_all) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nlist; q += gridDim.x * blockDim.x) {
    const int slot = slots[q];
    const ProbDev& p = b.probs[slot];
    int32_t st = ctr->status;
    if (st == WW_OK && g_net[slot] != (long long)*p.ground) st = WW_ERR_INTERNAL;
    *p.status = st;
    status_all[q] = st;
    *p.total_cost = tc[slot];
  }
}

int grid_blocks(int64_t work, int threads, int cap) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

}  // namespace

bool trace_enabled() {
  static int on = -1;
  if (on < 0) {
    const char* e = std::getenv("WW_TRACE");
    on = (e && e[0] == '1') ? 1 : 0;
  }
  return on == 1;
}
// ---------------- host side ----------------

// Arc-cost cache entries: the tiles that problems with n_nodes nodes in all
// cover, by area plus their ragged edges for aspect ratios up to 16:1 (an R x C
// problem has at most RC/1024 + (R + C)/32 + 1 tiles, R + C <= 4.25 sqrt(RC),
// and the sum of sqrt(RC) over the problems is at most sqrt(n_probs n_nodes)).
// Tile ids are handed out from 0, so these entries cover the tiles in use; the
// tile capacity itself is a looser bound, and tiles past the entries go uncached.
int64_t rc_cache_entries(int64_t n_nodes, int64_t n_tiles, int64_t n_probs) {
  const int64_t edges = (int64_t)std::ceil(4.25 / TS * std::sqrt((double)n_probs * (double)n_nodes));
  return std::min<int64_t>(n_tiles, n_nodes / (TS * TS) + edges + 4 * n_probs + 64);
}

int64_t solver_bytes(int64_t n_nodes, int64_t n_tiles, int64_t n_probs) {
  return n_nodes * (4 + 8 + 8 + 8 + 4 + 2 + 4) + (n_nodes + 1) * 8 + n_tiles * 4 * 8 +
         rc_cache_entries(n_nodes, n_tiles, n_probs) * (kRcTileBytes + 4) + (kMaxSearchGrid + 64) * 4 +
         n_probs * (sizeof(ProbDev) + 4 + 8 + 8 + 16 + 12) + (int64_t)sizeof(McfCtr) + 4096;
}

ww_status solver_alloc(SolverWs* sv, int64_t n_nodes, int64_t n_tiles, int64_t n_probs) {
  std::memset(sv, 0, sizeof(*sv));
  sv->n_cap = n_nodes;
  sv->t_cap = n_tiles;
  sv->p_cap = n_probs;
  const int64_t nb = 2 * n_tiles + 4 * n_probs;
  bool ok = cudaMalloc(&sv->excess, n_nodes * 4) == cudaSuccess && cudaMalloc(&sv->labels, n_nodes * 8) == cudaSuccess &&
            cudaMalloc(&sv->best, n_nodes * 8) == cudaSuccess && cudaMalloc(&sv->cand, 2 * n_nodes * 4) == cudaSuccess &&
            cudaMalloc(&sv->cand_root, n_nodes * 4) == cudaSuccess &&
            cudaMalloc(&sv->pot, (n_nodes + 1) * 8) == cudaSuccess && cudaMalloc(&sv->inq, n_tiles * 4) == cudaSuccess &&
            cudaMalloc(&sv->slots, (n_tiles + kMaxSearchGrid + 64) * 4) == cudaSuccess &&
            cudaMalloc(&sv->capped, n_tiles * 4) == cudaSuccess && cudaMalloc(&sv->tile_prob, n_tiles * 4) == cudaSuccess &&
            cudaMalloc(&sv->touched, n_tiles * 4) == cudaSuccess && cudaMalloc(&sv->tlist, n_tiles * 4) == cudaSuccess &&
            cudaMalloc(&sv->rc_cache, rc_cache_entries(n_nodes, n_tiles, n_probs) * kRcTileBytes) == cudaSuccess &&
            cudaMalloc(&sv->rc_pass, rc_cache_entries(n_nodes, n_tiles, n_probs) * 4) == cudaSuccess &&
            cudaMalloc(&sv->exits, n_nodes * 2) == cudaSuccess && cudaMalloc(&sv->segs, n_nodes * 4) == cudaSuccess &&
            cudaMalloc(&sv->border, nb * 4) == cudaSuccess && cudaMalloc(&sv->probs, n_probs * sizeof(ProbDev)) == cudaSuccess &&
            cudaMalloc(&sv->prob_left, n_probs * 4) == cudaSuccess && cudaMalloc(&sv->g_net, n_probs * 8) == cudaSuccess &&
            cudaMalloc(&sv->tc, n_probs * 8) == cudaSuccess && cudaMalloc(&sv->ctr, sizeof(McfCtr)) == cudaSuccess &&
            cudaMalloc(&sv->order, n_probs * 4) == cudaSuccess && cudaMalloc(&sv->slot_list, n_probs * 4) == cudaSuccess &&
            cudaMalloc(&sv->status_all, n_probs * 4) == cudaSuccess &&
            cudaMalloc(&sv->q, sizeof(SearchQ)) == cudaSuccess &&
            cudaMallocHost(&sv->host_ctr, sizeof(McfCtr)) == cudaSuccess &&
            cudaMallocHost(&sv->host_probs, n_probs * sizeof(ProbDev)) == cudaSuccess &&
            cudaMallocHost(&sv->h_lists, (4 * n_probs + nb) * 4) == cudaSuccess;
  sv->nb_cap = nb;
  sv->rc_entries = rc_cache_entries(n_nodes, n_tiles, n_probs);
  if (!ok) return WW_ERR_OOM;
  // best labels start unreached; worklist flags, ring slots, cap flags and visit
  // flags start (and end every search or pass) zero
  if (cudaMemset(sv->best, 0xFF, n_nodes * 8) != cudaSuccess || cudaMemset(sv->inq, 0, n_tiles * 4) != cudaSuccess ||
      cudaMemset(sv->slots, 0, (n_tiles + kMaxSearchGrid + 64) * 4) != cudaSuccess ||
      cudaMemset(sv->capped, 0, n_tiles * 4) != cudaSuccess || cudaMemset(sv->touched, 0, n_tiles * 4) != cudaSuccess)
    return WW_ERR_CUDA;
  cudaEvent_t* ev = reinterpret_cast<cudaEvent_t*>(sv->events);
  if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) return WW_ERR_CUDA;
  return WW_OK;
}

void solver_free(SolverWs* sv) {
  cudaFree(sv->excess);
  cudaFree(sv->labels);
  cudaFree(sv->best);
  cudaFree(sv->cand);
  cudaFree(sv->cand_root);
  cudaFree(sv->pot);
  cudaFree(sv->inq);
  cudaFree(sv->slots);
  cudaFree(sv->capped);
  cudaFree(sv->touched);
  cudaFree(sv->tlist);
  cudaFree(sv->rc_cache);
  cudaFree(sv->rc_pass);
  cudaFree(sv->exits);
  cudaFree(sv->segs);
  cudaFree(sv->tile_prob);
  cudaFree(sv->border);
  cudaFree(sv->probs);
  cudaFree(sv->prob_left);
  cudaFree(sv->g_net);
  cudaFree(sv->tc);
  cudaFree(sv->ctr);
  cudaFree(sv->order);
  cudaFree(sv->slot_list);
  cudaFree(sv->status_all);
  cudaFree(sv->q);
  cudaFreeHost(sv->host_ctr);
  cudaFreeHost(sv->host_probs);
  cudaFreeHost(sv->h_lists);
  cudaEvent_t* ev = reinterpret_cast<cudaEvent_t*>(sv->events);
  if (ev[0]) cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
}

namespace {

int search_grid_size(int sm_count, int want_per_sm) {
  static int per_sm = 0;
  if (per_sm == 0) {
    int a = 1, b = 1;
    // five tiles per SM: ask for the largest shared-memory share of the unified L1
    cudaFuncSetAttribute(k_search<true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    cudaFuncSetAttribute(k_search<false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_search<true>, SEARCH_THREADS, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_search<false>, SEARCH_THREADS, 0);
    per_sm = std::max(1, std::min(a, b));
  }
  const int k = want_per_sm > 0 ? std::min(want_per_sm, per_sm) : per_sm;
  return std::min(sm_count * k, kMaxSearchGrid);
}

// band launches per pass: the zero band (one stage, or up to three when its hop
// radius is staged), then caps c, 8c, ... until the second-to-last launch opens
// the cap completely
constexpr int kBands = 4, kBandsStaged = 6;

// Joining problems (grid: x strides, y over the joiners): tile -> problem map,
// zero flows and per-problem counters.
__global__ void k_join(const ProbDev* probs, const int32_t* slots, int32_t* tile_prob, int32_t* prob_left,
                       long long* g_net, long long* tc) {
  const int slot = slots[blockIdx.y];
  const ProbDev& p = probs[slot];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t0 == 0) {
    prob_left[slot] = 0;
    tc[slot] = 0;
  }
  const int64_t nt = (int64_t)p.tiles_x * p.tiles_y;
  for (int64_t t = t0; t < nt; t += stride) tile_prob[p.tile_off + t] = slot;
  if (p.resume) {
    // keep the given flows; the ground's net outflow so far is read off its arcs
    // (first and last pixel row of h, first and last column of v)
    long long gn = 0;
    for (int64_t j = t0; j < p.C; j += stride)
      gn += (long long)p.flows[j] - (long long)p.flows[(p.m - 1) * p.n + j];
    for (int64_t i = t0; i < p.R; i += stride)
      gn += (long long)p.flows[p.m * p.n + i * p.n + p.n - 1] - (long long)p.flows[p.m * p.n + i * p.n];
    for (int o = 16; o > 0; o >>= 1) gn += __shfl_xor_sync(0xffffffffu, gn, o);
    if ((threadIdx.x & 31) == 0 && gn) atomicAdd((unsigned long long*)&g_net[slot], (unsigned long long)gn);
    return;
  }
  // flows, 2 m n bytes: unaligned head, 16-byte words, tail
  uint8_t* f = reinterpret_cast<uint8_t*>(p.flows);
  const int64_t nb = 2 * p.m * p.n;
  const int64_t head = min(nb, (int64_t)((16 - (reinterpret_cast<uintptr_t>(f) & 15)) & 15));
  const int64_t nw = (nb - head) / 16;
  for (int64_t k = t0; k < head; k += stride) f[k] = 0;
  uint4* w = reinterpret_cast<uint4*>(f + head);
  for (int64_t k = t0; k < nw; k += stride) w[k] = make_uint4(0u, 0u, 0u, 0u);
  for (int64_t k = head + 16 * nw + t0; k < nb; k += stride) f[k] = 0;
}

// Per-slot counters a join starts from (before k_join, which adds to g_net on a resume).
__global__ void k_join_clear(const int32_t* slots, int count, long long* g_net) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x) g_net[slots[q]] = 0;
}

// After membership changes: go on if anything is imbalanced.
__global__ void k_resume(McfCtr* ctr, int64_t n_total) {
  ctr->n_total = n_total;
  ctr->idle = 0;
  if (ctr->status == WW_OK) ctr->go_on = ctr->ncand > 0 ? 1 : 0;
}

}  // namespace

Session::Session(SolverWs* sv_, int64_t* pot_, int64_t g_index_, const ww_params* prm, cudaStream_t s,
                 bool keep_ground_pot)
    : sv(sv_), pot(pot_), g_index(g_index_), stream(s) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
  search_grid = search_grid_size(sm_count, prm->search_ctas_per_sm);
  used.assign(sv->p_cap, 0);
  McfCtr* hc = reinterpret_cast<McfCtr*>(sv->host_ctr);
  std::memset(hc, 0, sizeof(McfCtr));
  hc->status = WW_OK;
  hc->cap = 0xFFFFFFFFu;
  hc->max_passes = prm->max_passes;
  hc->n_cap_nodes = sv->n_cap;
  hc->band_min = (uint32_t)std::max(1, prm->band_min);
  hc->band_mult = (uint32_t)std::max(0, prm->band_mult);
  hc->band_growth = (uint32_t)std::max(2, prm->band_growth);
  hc->band_start_ppm = (uint32_t)std::max(0, prm->band_start_ppm);
  hc->full_passes = (uint32_t)std::max(0, prm->full_passes);
  hc->ground_sink_below = (uint32_t)std::max(0, prm->ground_sink_below);
  hc->zero_stop_below = (uint32_t)std::max(0, prm->zero_stop_below);
  hc->zero_hops = (uint32_t)std::max(1, std::min(prm->zero_band_hops, (1 << 29) - 1));
  // zero-band stages: from zero_band_hops_min to zero_band_hops, geometric
  {
    const double lo = std::max(1, std::min(prm->zero_band_hops_min, (int32_t)hc->zero_hops));
    const double hi = hc->zero_hops;
    hc->zhop[0] = (uint32_t)lo;
    hc->zhop[1] = (uint32_t)std::max(lo, std::min(hi, std::round(std::sqrt(lo * hi))));
    hc->zhop[2] = (uint32_t)hi;
    staged_zero = hc->zhop[0] < hc->zhop[2];
  }
  hc->wait_polls = (uint32_t)std::max(1, prm->wait_polls);
  // the worklist flags and ring start empty (a search that stopped on an error
  // may have left entries behind); the ground potential starts at 0 unless a
  // resumed solve brings its own
  const int64_t ring = sv->t_cap + kMaxSearchGrid + 64;
  err = cudaMemcpyAsync(sv->ctr, hc, sizeof(McfCtr), cudaMemcpyHostToDevice, s) == cudaSuccess &&
                cudaMemsetAsync(sv->inq, 0, sv->t_cap * 4, s) == cudaSuccess &&
                cudaMemsetAsync(sv->slots, 0, ring * 4, s) == cudaSuccess &&
                cudaMemsetAsync(sv->capped, 0, sv->t_cap * 4, s) == cudaSuccess &&
                cudaMemsetAsync(sv->touched, 0, sv->t_cap * 4, s) == cudaSuccess &&
                cudaMemsetAsync(sv->rc_pass, 0, sv->rc_entries * 4, s) == cudaSuccess &&  // pass numbers restart
                (keep_ground_pot || cudaMemsetAsync(pot + g_index, 0, 8, s) == cudaSuccess)
            ? WW_OK
            : WW_ERR_CUDA;
}

int Session::add(const ProbHost& ph, int64_t node_off, int64_t tile_off) {
  int slot = -1;
  for (int k = 0; k < (int)used.size(); ++k)
    if (!used[k]) {
      slot = k;
      break;
    }
  if (slot < 0) return -1;
  ProbDev& d = reinterpret_cast<ProbDev*>(sv->host_probs)[slot];
  d.m = ph.m;
  d.n = ph.n;
  d.R = d.m - 1;
  d.C = d.n - 1;
  d.N = d.R * d.C;
  d.tiles_x = (int32_t)((d.C + TS - 1) / TS);
  d.tiles_y = (int32_t)((d.R + TS - 1) / TS);
  d.node_off = node_off;
  d.tile_off = tile_off;
  d.res = ph.res;
  d.ground = ph.ground;
  d.costs = ph.costs;
  d.flows = ph.flows;
  d.pot_out = ph.pot_out;
  d.total_cost = ph.total_cost;
  d.status = ph.status;
  d.resume = ph.resume ? 1 : 0;
  used[slot] = 1;
  pending.push_back(slot);
  return slot;
}

void Session::remove(int slot) {
  if (slot >= 0 && slot < (int)used.size()) used[slot] = 0;
  pending.erase(std::remove(pending.begin(), pending.end(), slot), pending.end());
}

int64_t Session::tiles_of(int slot) const {
  const ProbDev& d = reinterpret_cast<const ProbDev*>(sv->host_probs)[slot];
  return (int64_t)d.tiles_x * d.tiles_y;
}

ww_status Session::commit() {
  const ProbDev* hp = reinterpret_cast<const ProbDev*>(sv->host_probs);
  order.clear();
  for (int k = 0; k < (int)used.size(); ++k)
    if (used[k]) order.push_back(k);
  std::sort(order.begin(), order.end(), [&](int a, int b) { return hp[a].node_off < hp[b].node_off; });
  n_total = 0;
  t_high = 0;
  max_nodes = 1;
  int32_t* h_order = sv->h_lists;
  int32_t* h_border = h_order + sv->p_cap;
  int32_t* h_join = h_border + sv->nb_cap;
  std::vector<int32_t> border;
  int64_t garcs = 0;
  max_garcs = 1;
  for (int k : order) {
    ProbDev& dm = reinterpret_cast<ProbDev*>(sv->host_probs)[k];
    dm.garc_off = garcs;
    garcs += 2 * (dm.R + dm.C);
    max_garcs = std::max(max_garcs, 2 * (dm.R + dm.C));
  }
  if (garcs >= (1ll << 31)) return WW_ERR_INVALID_ARG;
  for (int k : order) {
    const ProbDev& d = hp[k];
    n_total += d.N;
    t_high = std::max(t_high, d.tile_off + (int64_t)d.tiles_x * d.tiles_y);
    max_nodes = std::max(max_nodes, d.N + 1);
    // border tiles: first and last tile row, first and last tile of the rows between
    const int64_t tx = d.tiles_x, ty = d.tiles_y;
    for (int64_t ti = 0; ti < ty; ++ti) {
      if (ti == 0 || ti == ty - 1) {
        for (int64_t tj = 0; tj < tx; ++tj) border.push_back((int32_t)(d.tile_off + ti * tx + tj));
      } else {
        border.push_back((int32_t)(d.tile_off + ti * tx));
        if (tx > 1) border.push_back((int32_t)(d.tile_off + ti * tx + tx - 1));
      }
    }
  }
  n_border = (int64_t)border.size();
  if (n_border > sv->nb_cap) return WW_ERR_INTERNAL;
  std::copy(order.begin(), order.end(), h_order);
  std::copy(border.begin(), border.end(), h_border);
  cudaStream_t s = stream;
  // uploads from pinned staging: the caller syncs the stream before the next commit
  WW_CUDA_TRY(cudaMemcpyAsync(sv->probs, hp, used.size() * sizeof(ProbDev), cudaMemcpyHostToDevice, s));
  if (!order.empty()) {
    WW_CUDA_TRY(cudaMemcpyAsync(sv->order, h_order, order.size() * 4, cudaMemcpyHostToDevice, s));
    WW_CUDA_TRY(cudaMemcpyAsync(sv->border, h_border, border.size() * 4, cudaMemcpyHostToDevice, s));
  }
  if (!pending.empty()) {
    if (pending.size() > 65535) return WW_ERR_INVALID_ARG;
    int64_t biggest = 1;
    for (int k : pending) biggest = std::max(biggest, hp[k].N);
    std::copy(pending.begin(), pending.end(), h_join);
    WW_CUDA_TRY(cudaMemcpyAsync(sv->slot_list, h_join, pending.size() * 4, cudaMemcpyHostToDevice, s));
    dim3 gi(grid_blocks(biggest, 256, std::max(1, sm_count * 16 / (int)pending.size() + 1)), (unsigned)pending.size());
    k_join_clear<<<1, 256, 0, s>>>(sv->slot_list, (int)pending.size(), sv->g_net);
    k_join<<<gi, 256, 0, s>>>(reinterpret_cast<const ProbDev*>(sv->probs), sv->slot_list, sv->tile_prob,
                              sv->prob_left, sv->g_net, sv->tc);
    k_init_state<<<gi, 256, 0, s>>>(batch(), sv->slot_list, sv->excess, sv->cand, pot, sv->labels, sv->prob_left,
                                    reinterpret_cast<McfCtr*>(sv->ctr));
    pending.clear();
  }
  k_resume<<<1, 1, 0, s>>>(reinterpret_cast<McfCtr*>(sv->ctr), n_total);
  WW_CUDA_TRY(cudaGetLastError());
  return WW_OK;
}

Batch Session::batch() const {
  Batch b;
  b.probs = reinterpret_cast<const ProbDev*>(sv->probs);
  b.order = sv->order;
  b.nact = (int)order.size();
  b.tile_prob = sv->tile_prob;
  b.g_index = g_index;
  b.n_total = n_total;
  b.t_total = t_high;
  return b;
}

template <bool FWD>
ww_status Session::enqueue_pass() {
  cudaStream_t s = stream;
  McfCtr* ctr = reinterpret_cast<McfCtr*>(sv->ctr);
  SearchQ* q = reinterpret_cast<SearchQ*>(sv->q);
  cudaEvent_t* ev = reinterpret_cast<cudaEvent_t*>(sv->events);
  const Batch b = batch();
  const McfCtr* hc = reinterpret_cast<const McfCtr*>(sv->host_ctr);
  const int64_t nc_bound = ncand_unknown ? n_total : std::max<int64_t>(1, hc->ncand);
  const int grid_cand = grid_blocks(nc_bound + n_border, 256, sm_count * 16);
  const int grid_tiles = grid_blocks(t_high, 256, sm_count * 8);
  k_pass_setup<<<1, 1, 0, s>>>(ctr, q);
  k_set_roots<FWD><<<grid_cand, 256, 0, s>>>(sv->excess, sv->cand, 0, sv->labels, ctr);
  k_seed_tiles<FWD><<<grid_cand, 256, 0, s>>>(b, sv->excess, sv->cand, ctr, sv->prob_left, sv->border,
                                              (int32_t)n_border, q, sv->slots, sv->inq, search_grid);
  if (!capturing) WW_CUDA_TRY(cudaEventRecord(ev[0], s));
  const dim3 ga(grid_blocks(max_garcs, 256, std::max(1, sm_count * 4 / std::max(1, b.nact) + 1)),
                (unsigned)std::max(1, b.nact));
  const int bands = staged_zero ? kBandsStaged : kBands;
  for (int band = 0; band < bands; ++band) {
    k_search<FWD><<<search_grid, SEARCH_THREADS, 0, s>>>(b, pot, sv->labels, q, sv->slots, sv->inq, ctr, sv->capped,
                                                         sv->touched, sv->tlist, sv->rc_cache, sv->rc_pass,
                                                         (int32_t)sv->rc_entries);
    k_ground_dist<FWD><<<ga, 256, 0, s>>>(b, sv->labels, pot, ctr);
    k_count_found<FWD><<<grid_cand, 256, 0, s>>>(sv->excess, sv->labels, sv->cand, 0, ctr);
    k_band_decide<<<1, 1, 0, s>>>(ctr, q, band == bands - 2 ? 1 : 0);
    if (band + 1 < bands)
      k_reseed<<<grid_tiles, 256, 0, s>>>(b, sv->capped, q, sv->slots, sv->inq, search_grid, ctr);
  }
  if (!capturing) WW_CUDA_TRY(cudaEventRecord(ev[1], s));
  k_clear_capped<<<grid_tiles, 256, 0, s>>>(b, sv->capped, ctr);
  k_tile_exits<<<sm_count * 8, 256, 0, s>>>(b, sv->labels, sv->tlist, sv->exits, ctr);
  k_select<FWD><<<grid_cand, 256, 0, s>>>(b, sv->excess, sv->labels, sv->exits, sv->cand, sv->cand_root, sv->best,
                                          ctr);
  k_select_ground<FWD><<<ga, 256, 0, s>>>(b, sv->labels, sv->exits, pot, sv->best, ctr);
  k_augment<FWD><<<grid_cand, 256, 0, s>>>(b, sv->excess, sv->labels, sv->exits, sv->cand, sv->cand_root, sv->best,
                                           sv->g_net, sv->segs, ctr);
  k_flip_segments<FWD><<<sm_count * 16, 256, 0, s>>>(b, sv->labels, sv->exits, sv->segs, ctr);
  k_augment_ground<FWD><<<ga, 256, 0, s>>>(b, sv->excess, sv->labels, sv->exits, pot, sv->best, sv->g_net, ctr);
  k_reset_best<<<grid_cand, 256, 0, s>>>(b, sv->cand_root, sv->best, sv->prob_left, (int)sv->p_cap, ctr);
  k_potentials<FWD><<<sm_count * 8, 256, 0, s>>>(b, sv->labels, pot, sv->touched, sv->tlist, ctr);
  k_potential_ground<FWD><<<1, 1, 0, s>>>(b, pot, ctr);
  k_compact<<<grid_cand, 256, 0, s>>>(b, sv->excess, sv->cand, sv->labels, sv->prob_left, ctr);
  k_finish_pass<<<1, 1, 0, s>>>(ctr);
  WW_CUDA_TRY(cudaGetLastError());
  return WW_OK;
}

ww_status Session::pass(ww_solve_stats* st) {
  McfCtr* hc = reinterpret_cast<McfCtr*>(sv->host_ctr);
  ww_status e = (parity++ % 2 == 0) ? enqueue_pass<true>() : enqueue_pass<false>();
  if (e != WW_OK) return e;
  WW_CUDA_TRY(cudaMemcpyAsync(hc, sv->ctr, sizeof(McfCtr), cudaMemcpyDeviceToHost, stream));
  WW_CUDA_TRY(cudaStreamSynchronize(stream));
  cudaEvent_t* ev = reinterpret_cast<cudaEvent_t*>(sv->events);
  float ms = 0.0f;
  if (cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess && st) st->ms_search_gpu += ms;
  fill_stats(st);
  if (trace_enabled()) {
    std::fprintf(stderr,
                 "[ww] pass %d: cap %u, search %.3f ms, augment %d (D %u), left %d, visits %llu (32-bit %llu, redone "
                 "%llu), tiles %lld, cycles visit %llu pop %llu, status %d, go_on %d, ground sink %d (dG %u)\n",
                 hc->passes, hc->cap, ms, hc->naug, hc->D, hc->ncand, (unsigned long long)hc->tile_visits,
                 (unsigned long long)hc->visits32, (unsigned long long)hc->redo64, (long long)hc->touched_total,
                 (unsigned long long)hc->visit_cycles, (unsigned long long)hc->pop_cycles, hc->status, hc->go_on,
                 hc->gsink, hc->dG);
    if (hc->err)
      std::fprintf(stderr, "[ww]   error flags %d; first negative reduced cost: node %lld dir %d value %lld (pass %d)\n",
                   hc->err, hc->dbg_node, hc->dbg_dir, hc->dbg_red, hc->dbg_pass);
  }
  return WW_OK;
}

namespace {
// Loop condition of the graph-resident pass loop: go on while the solver does.
__global__ void k_loop_cond(cudaGraphConditionalHandle h, const McfCtr* ctr) {
  cudaGraphSetConditional(h, ctr->go_on ? 1u : 0u);
}
}  // namespace

// The remaining passes as one conditional while node of graph g: its body is
// a forward and a reverse pass (a pass after the last one is a no-op: its
// kernels return when go_on is 0) followed by the loop condition, which is
// set on the device.  The body is captured from enqueue_pass on a side stream.
ww_status Session::add_loop_node(cudaGraph_t g, const cudaGraphNode_t* dep, cudaGraphNode_t* out) {
  if (parity % 2 != 0) return WW_ERR_INTERNAL;
  cudaGraphConditionalHandle h;
  if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) return WW_ERR_CUDA;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  if (cudaGraphAddNode(out, g, dep, nullptr, dep ? 1 : 0, &np) != cudaSuccess) return WW_ERR_CUDA;
  cudaGraph_t body = np.conditional.phGraph_out[0];
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return WW_ERR_CUDA;
  ww_status e = WW_ERR_CUDA;
  if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    cudaStream_t saved = stream;
    stream = cs;
    capturing = true;
    ww_status e1 = enqueue_pass<true>();
    ww_status e2 = e1 == WW_OK ? enqueue_pass<false>() : e1;
    k_loop_cond<<<1, 1, 0, cs>>>(h, reinterpret_cast<const McfCtr*>(sv->ctr));
    capturing = false;
    stream = saved;
    cudaGraph_t captured = nullptr;
    const bool cap_ok = cudaStreamEndCapture(cs, &captured) == cudaSuccess;
    e = e2 != WW_OK ? e2 : (cap_ok ? WW_OK : WW_ERR_CUDA);
  }
  cudaStreamDestroy(cs);
  if (e != WW_OK) cudaGetLastError();
  return e;
}

// All remaining passes in one graph launch.
ww_status Session::run_graph(ww_solve_stats* st) {
  const McfCtr* hc = reinterpret_cast<const McfCtr*>(sv->host_ctr);
  const int64_t passes0 = hc->passes;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  cudaGraphNode_t node;
  ww_status e = WW_ERR_CUDA;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return WW_ERR_CUDA;
  e = add_loop_node(g, nullptr, &node);
  if (e == WW_OK) {
    e = WW_ERR_CUDA;
    if (cudaGraphInstantiate(&ex, g, 0) == cudaSuccess && cudaGraphLaunch(ex, stream) == cudaSuccess &&
        cudaMemcpyAsync(sv->host_ctr, sv->ctr, sizeof(McfCtr), cudaMemcpyDeviceToHost, stream) == cudaSuccess &&
        cudaStreamSynchronize(stream) == cudaSuccess)
      e = WW_OK;
  }
  if (e == WW_OK) {
    parity += 2 * (int)((hc->passes - passes0 + 1) / 2);
    fill_stats(st);
  }
  if (ex) cudaGraphExecDestroy(ex);
  if (g) cudaGraphDestroy(g);
  if (e != WW_OK) cudaGetLastError();
  return e;
}

void Session::fill_stats(ww_solve_stats* st) const {
  const McfCtr* hc = reinterpret_cast<const McfCtr*>(sv->host_ctr);
  if (!st) return;
  st->augmentations = hc->aug_total;
  st->passes = hc->passes;
  st->search_iterations = hc->passes;
  st->tile_visits = (int64_t)hc->tile_visits;
  st->local_rounds = (int64_t)hc->local_rounds;
  st->visit_cycles = (int64_t)hc->visit_cycles;
  st->load_cycles = (int64_t)hc->load_cycles;
  st->relax_cycles = (int64_t)hc->relax_cycles;
  st->settled_visits = (int64_t)hc->settled_visits;
  st->narrow_visits = (int64_t)hc->visits32;
  st->narrow_redone = (int64_t)hc->redo64;
}

int64_t Session::ctr_bytes() const { return (int64_t)sizeof(McfCtr); }

const McfCtr& Session::ctr() const { return *reinterpret_cast<const McfCtr*>(sv->host_ctr); }
int32_t Session::status() const { return ctr().status; }
int32_t Session::ncand() const { return ctr().ncand; }
bool Session::go_on() const { return ctr().go_on != 0; }
int Session::next_slot() const {
  for (int k = 0; k < (int)used.size(); ++k)
    if (!used[k]) return k;
  return -1;
}

ww_status Session::left(std::vector<int32_t>* out) {
  out->assign(used.size(), 0);
  WW_CUDA_TRY(cudaMemcpyAsync(out->data(), sv->prob_left, used.size() * 4, cudaMemcpyDeviceToHost, stream));
  WW_CUDA_TRY(cudaStreamSynchronize(stream));
  return WW_OK;
}

namespace {
__global__ void k_zero_slots(const int32_t* slots, int count, long long* tc) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x) tc[slots[q]] = 0;
}
}  // namespace

const int32_t* Session::finalized_status() const { return sv->h_lists + 3 * sv->p_cap + sv->nb_cap; }

ww_status Session::finalize_enqueue(const std::vector<int>& list) {
  if (list.empty()) return WW_OK;
  if (list.size() > 65535 || (int64_t)list.size() > sv->p_cap) return WW_ERR_INVALID_ARG;
  cudaStream_t s = stream;
  const ProbDev* hp = reinterpret_cast<const ProbDev*>(sv->host_probs);
  int32_t* h_fin = sv->h_lists + 2 * sv->p_cap + sv->nb_cap;
  int32_t* h_st = h_fin + sv->p_cap;
  int64_t biggest = 1;
  for (int k : list) biggest = std::max(biggest, hp[k].m * hp[k].n);
  std::copy(list.begin(), list.end(), h_fin);
  WW_CUDA_TRY(cudaMemcpyAsync(sv->slot_list, h_fin, list.size() * 4, cudaMemcpyHostToDevice, s));
  const Batch b = batch();
  const int nl = (int)list.size();
  k_zero_slots<<<grid_blocks(nl, 256, 64), 256, 0, s>>>(sv->slot_list, nl, sv->tc);
  dim3 gt(grid_blocks(biggest, 256, std::max(1, sm_count * 16 / nl + 1)), (unsigned)nl);
  k_total_cost<<<gt, 256, 0, s>>>(b, sv->slot_list, sv->tc);
  k_copy_pot<<<gt, 256, 0, s>>>(b, sv->slot_list, pot);
  k_write_results<<<grid_blocks((int64_t)nl, 256, 64), 256, 0, s>>>(
      b, sv->slot_list, nl, reinterpret_cast<McfCtr*>(sv->ctr), sv->g_net, sv->tc, sv->status_all);
  WW_CUDA_TRY(cudaGetLastError());
  WW_CUDA_TRY(cudaMemcpyAsync(h_st, sv->status_all, list.size() * 4, cudaMemcpyDeviceToHost, s));
  return WW_OK;
}

ww_status Session::finalize(const std::vector<int>& list, std::vector<int32_t>* statuses) {
  if (list.empty()) return WW_OK;
  ww_status e = finalize_enqueue(list);
  if (e != WW_OK) return e;
  WW_CUDA_TRY(cudaStreamSynchronize(stream));
  const int32_t* h_st = finalized_status();
  statuses->assign(h_st, h_st + list.size());
  if (trace_enabled()) {
    std::vector<long long> gn(sv->p_cap);
    cudaMemcpy(gn.data(), sv->g_net, sv->p_cap * 8, cudaMemcpyDeviceToHost);
    const McfCtr* hc = reinterpret_cast<const McfCtr*>(sv->host_ctr);
    for (size_t q = 0; q < list.size(); ++q)
      std::fprintf(stderr, "[ww] finalize slot %d: status %d, ground net %lld (solver status %d)\n", list[q], h_st[q],
                   gn[list[q]], hc->status);
  }
  return WW_OK;
}

ww_status solve_problems(const ProbHost* ph, int nprob, SolverWs* sv, const ww_params* prm, int64_t* pot_global,
                         ww_solve_stats* stats, cudaStream_t s) {
  if (nprob <= 0 || nprob > sv->p_cap) return WW_ERR_INVALID_ARG;
  if (pot_global && nprob != 1) return WW_ERR_INVALID_ARG;
  int64_t n_total = 0, t_total = 0;
  for (int k = 0; k < nprob; ++k) {
    n_total += (ph[k].m - 1) * (ph[k].n - 1);
    t_total += tiles_for(ph[k].m, ph[k].n);
  }
  if (n_total > sv->n_cap || t_total > sv->t_cap || n_total >= (1ll << 31)) return WW_ERR_INVALID_ARG;
  // a single problem may keep its potentials in the caller's array (ground last)
  int64_t* pot = pot_global ? pot_global : sv->pot;
  const auto t_setup = std::chrono::steady_clock::now();
  const int64_t g_index = pot_global ? (ph[0].m - 1) * (ph[0].n - 1) : sv->n_cap;
  // a resumed single problem keeps its potentials, the ground's included
  if (!pot_global)
    for (int k = 0; k < nprob; ++k)
      if (ph[k].resume) return WW_ERR_INVALID_ARG;
  Session S(sv, pot, g_index, prm, s, pot_global && ph[0].resume);
  if (S.err != WW_OK) return S.err;
  int64_t node_off = 0, tile_off = 0;
  std::vector<int> all;
  for (int k = 0; k < nprob; ++k) {
    ProbHost h = ph[k];
    if (pot_global) h.pot_out = nullptr;
    all.push_back(S.add(h, node_off, tile_off));
    node_off += (h.m - 1) * (h.n - 1);
    tile_off += tiles_for(h.m, h.n);
  }
  ww_status e = S.commit();
  if (e != WW_OK) return e;
  ww_solve_stats st{};
  WW_CUDA_TRY(cudaMemcpyAsync(sv->host_ctr, sv->ctr, sizeof(McfCtr), cudaMemcpyDeviceToHost, s));
  WW_CUDA_TRY(cudaStreamSynchronize(s));
  st.residues = S.ncand();
  auto t0 = std::chrono::steady_clock::now();
  if (trace_enabled())
    std::fprintf(stderr, "[ww] session setup %.3f ms for %d problems, %lld nodes\n",
                 std::chrono::duration<double, std::milli>(t0 - t_setup).count(), nprob, (long long)n_total);
  if (prm->graph_loop && !trace_enabled() && S.go_on()) {
    e = S.run_graph(&st);
    if (e != WW_OK) return e;
  }
  while (S.go_on()) {
    e = S.pass(&st);
    if (e != WW_OK) return e;
  }
  const auto t1 = std::chrono::steady_clock::now();
  st.ms_search = std::chrono::duration<double, std::milli>(t1 - t0).count();
  std::vector<int32_t> sts;
  e = S.finalize(all, &sts);
  if (e != WW_OK) return e;
  long long g0 = 0;
  WW_CUDA_TRY(cudaMemcpyAsync(&g0, sv->g_net + all[0], 8, cudaMemcpyDeviceToHost, s));
  WW_CUDA_TRY(cudaStreamSynchronize(s));
  st.ground_net = g0;
  st.ms_other = std::chrono::duration<double, std::milli>(t0 - t_setup + (std::chrono::steady_clock::now() - t1)).count();
  if (stats) *stats = st;
  for (int32_t x : sts)
    if (x != WW_OK) return x;
  return WW_OK;
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
