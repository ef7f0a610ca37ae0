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
#include <vector>

#include "ww_internal.cuh"

namespace ww {

constexpr int TS = 32;         // tile side in nodes
constexpr int TSH = TS + 2;    // with halo
constexpr int SEARCH_THREADS = 256;
constexpr int kMaxLocalSweeps = 8192;

enum : int32_t { kErrOverflow = 1, kErrInternal = 2, kErrWalk = 4 };

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
};

namespace {

struct Grid {
  int64_t m, n, R, C, N, P;  // pixel rows/cols, node rows/cols, nodes, pixels
  int tiles_x, tiles_y;
};

__device__ __forceinline__ void activate(int tile, int epoch, int32_t* stamp, int32_t* list, int32_t* count) {
  if (atomicExch(&stamp[tile], epoch) != epoch) {
    int pos = atomicAdd(count, 1);
    list[pos] = tile;
  }
}

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

template <bool FWD>
__global__ void __launch_bounds__(SEARCH_THREADS) k_search(Grid g, const int16_t* __restrict__ costs,
                                                           const int8_t* __restrict__ flows,
                                                           const int64_t* __restrict__ pot,
                                                           uint64_t* labels, const int32_t* list_in,
                                                           const int32_t* count_in, int32_t* list_out,
                                                           int32_t* count_out, int32_t* stamp, int epoch,
                                                           McfCtr* ctr) {
  __shared__ uint64_t lab[TSH][TSH];
  __shared__ uint32_t rc[4][TS][TS];
  __shared__ int side[4];
  const int tid = threadIdx.x;
  const int lx = tid & 31, ly0 = tid >> 5;  // column lx, rows ly0 + 8k
  const int count = *count_in;
  const int64_t pG = pot[g.N];
  for (int t = blockIdx.x; t < count; t += gridDim.x) {
    const int tile = list_in[t];
    const int64_t ti = tile / g.tiles_x, tj = tile % g.tiles_x;
    const int64_t i0 = ti * TS, j0 = tj * TS;
    if (tid < 4) side[tid] = 0;
    // labels with halo; outside the grid stands G, a root (label 0)
    for (int q = tid; q < TSH * TSH; q += SEARCH_THREADS) {
      int r = q / TSH, c = q % TSH;
      int64_t i = i0 + r - 1, j = j0 + c - 1;
      uint64_t v;
      if (i < 0 || j < 0 || i >= g.R || j >= g.C) {
        bool ring = (i >= -1 && i <= g.R && j >= -1 && j <= g.C);  // direct neighbour of the grid
        v = ring ? 0ull : kInf;
      } else {
        v = *((volatile const uint64_t*)&labels[i * g.C + j]);
      }
      lab[r][c] = v;
    }
    // reduced costs of the four arcs of every node in the tile
    uint64_t orig[4];
    int err = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int ly = ly0 + 8 * k;
      int64_t i = i0 + ly, j = j0 + lx;
      bool ex = i < g.R && j < g.C;
      int64_t v = i * g.C + j;
      int64_t pv = ex ? pot[v] : 0;
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
          if (red >= (int64_t)kNoArc) {
            err |= kErrOverflow;
          } else {
            r = (uint32_t)red;
          }
        }
        rc[d - 1][ly][lx] = r;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) orig[k] = lab[ly0 + 8 * k + 1][lx + 1];
    // local relaxation to the tile's fixed point
    for (int sweep = 0; sweep < kMaxLocalSweeps; ++sweep) {
      bool ch = false;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        int ly = ly0 + 8 * k;
        int r = ly + 1, c = lx + 1;
        uint64_t cur = lab[r][c];
        uint64_t best = cur;
#pragma unroll
        for (int d = 1; d <= 4; ++d) {
          uint32_t w = rc[d - 1][ly][lx];
          if (w == kNoArc) continue;
          int rr = d == kDirUp ? r - 1 : d == kDirDown ? r + 1 : r;
          int cc = d == kDirLeft ? c - 1 : d == kDirRight ? c + 1 : c;
          uint64_t lu = *((volatile uint64_t*)&lab[rr][cc]);
          if (lu == kInf) continue;
          uint64_t du = lu >> 32;
          if (du + w >= 0xFFFFFFFFull) {
            err |= kErrOverflow;
            continue;
          }
          uint64_t cand = (((lu & ~7ull) + ((uint64_t)w << 32) + 8ull) & ~7ull) | (uint64_t)d;
          if (cand < best) best = cand;
        }
        if (best < cur) {
          lab[r][c] = best;
          ch = true;
        }
      }
      if (!__syncthreads_or(ch)) break;
    }
    // write back and note which tile sides changed
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int ly = ly0 + 8 * k;
      int64_t i = i0 + ly, j = j0 + lx;
      uint64_t v = lab[ly + 1][lx + 1];
      if (i < g.R && j < g.C && v != orig[k]) {
        labels[i * g.C + j] = v;
        if (ly == 0) side[0] = 1;
        if (ly == TS - 1) side[1] = 1;
        if (lx == 0) side[2] = 1;
        if (lx == TS - 1) side[3] = 1;
      }
    }
    if (err) atomicOr(&ctr->err, err);
    __syncthreads();
    if (tid == 0) {
      if (side[0] && ti > 0) activate(tile - g.tiles_x, epoch, stamp, list_out, count_out);
      if (side[1] && ti + 1 < g.tiles_y) activate(tile + g.tiles_x, epoch, stamp, list_out, count_out);
      if (side[2] && tj > 0) activate(tile - 1, epoch, stamp, list_out, count_out);
      if (side[3] && tj + 1 < g.tiles_x) activate(tile + 1, epoch, stamp, list_out, count_out);
      atomicAdd(&ctr->tile_visits, 1ull);
    }
    __syncthreads();
  }
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

template <bool FWD>
__global__ void k_seed_tiles(Grid g, const int32_t* excess, const int32_t* cand, const McfCtr* ctr,
                             int32_t* stamp, int32_t* list, int32_t* count, int epoch) {
  const int nc = ctr->ncand;
  const int nborder = 2 * g.tiles_x + 2 * g.tiles_y;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nc + nborder;
       q += (int64_t)gridDim.x * blockDim.x) {
    int tile;
    if (q < nc) {
      int32_t v = cand[q];
      int32_t e = excess[v];
      if (!(FWD ? e > 0 : e < 0)) continue;
      int64_t i = v / g.C, j = v % g.C;
      tile = (int)((i / TS) * g.tiles_x + j / TS);
    } else {
      int b = (int)(q - nc);
      if (b < g.tiles_x) tile = b;                                             // top row
      else if (b < 2 * g.tiles_x) tile = (g.tiles_y - 1) * g.tiles_x + (b - g.tiles_x);  // bottom row
      else if (b < 2 * g.tiles_x + g.tiles_y) tile = (b - 2 * g.tiles_x) * g.tiles_x;     // left col
      else tile = (b - 2 * g.tiles_x - g.tiles_y) * g.tiles_x + g.tiles_x - 1;           // right col
    }
    activate(tile, epoch, stamp, list, count);
  }
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
  if (cudaMalloc(&ws->tile_list[0], tiles * 4) != cudaSuccess) return WW_ERR_OOM;
  if (cudaMalloc(&ws->tile_list[1], tiles * 4) != cudaSuccess) return WW_ERR_OOM;
  if (cudaMalloc(&ws->counters, sizeof(McfCtr)) != cudaSuccess) return WW_ERR_OOM;
  if (cudaMallocHost(&ws->host_counters, sizeof(McfCtr)) != cudaSuccess) return WW_ERR_OOM;
  cudaEvent_t* ev = reinterpret_cast<cudaEvent_t*>(ws->events);
  if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) return WW_ERR_CUDA;
  if (cudaMemset(ws->best, 0xFF, N * 8) != cudaSuccess) return WW_ERR_CUDA;
  if (cudaMemset(ws->tile_stamp, 0, tiles * 4) != cudaSuccess) return WW_ERR_CUDA;
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
  cudaFreeHost(ws->host_counters);
  cudaEvent_t* ev = reinterpret_cast<cudaEvent_t*>(ws->events);
  if (ev[0]) cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
}

template <bool FWD>
static ww_status run_search(const Grid& g, const int16_t* costs, const int8_t* flows, const int64_t* pot,
                            ww_workspace* ws, McfCtr* dctr, McfCtr* hctr, int max_sweeps, int sm_count,
                            int64_t* iters, cudaStream_t s) {
  const int nb_nodes = grid_blocks(g.N, 256, sm_count * 16);
  k_init_labels<FWD><<<nb_nodes, 256, 0, s>>>(g, ws->excess, ws->labels);
  int cur = 0;
  WW_CUDA_TRY(cudaMemsetAsync(&dctr->list_count[0], 0, 2 * sizeof(int32_t), s));
  int epoch = ++ws->epoch;
  k_seed_tiles<FWD><<<grid_blocks(g.N / 64 + 1024, 256, sm_count * 4), 256, 0, s>>>(
      g, ws->excess, ws->cand, dctr, ws->tile_stamp, ws->tile_list[cur], &dctr->list_count[cur], epoch);
  int32_t count = 1;  // unknown on the host: launch the first sweep unconditionally
  cudaEvent_t* ev = reinterpret_cast<cudaEvent_t*>(ws->events);
  const int max_blocks = sm_count * 6;
  for (int it = 0; it < max_sweeps; ++it) {
    int nxt = cur ^ 1;
    epoch = ++ws->epoch;
    WW_CUDA_TRY(cudaMemsetAsync(&dctr->list_count[nxt], 0, sizeof(int32_t), s));
    int blocks = it == 0 ? max_blocks : std::min(max_blocks, std::max(1, count));
    WW_CUDA_TRY(cudaEventRecord(ev[0], s));
    k_search<FWD><<<blocks, SEARCH_THREADS, 0, s>>>(g, costs, flows, pot, ws->labels, ws->tile_list[cur],
                                                   &dctr->list_count[cur], ws->tile_list[nxt],
                                                   &dctr->list_count[nxt], ws->tile_stamp, epoch, dctr);
    WW_CUDA_TRY(cudaGetLastError());
    WW_CUDA_TRY(cudaEventRecord(ev[1], s));
    WW_CUDA_TRY(cudaMemcpyAsync(&hctr->list_count[nxt], &dctr->list_count[nxt], sizeof(int32_t),
                                cudaMemcpyDeviceToHost, s));
    WW_CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess) ws->stats.ms_search_gpu += ms;
    ++*iters;
    count = hctr->list_count[nxt];
    cur = nxt;
    if (count == 0) return WW_OK;
  }
  return WW_ERR_TIMEOUT;
}

template <bool FWD>
static ww_status run_pass(const Grid& g, const int16_t* costs, int8_t* flows, int64_t* pot, ww_workspace* ws,
                          McfCtr* dctr, McfCtr* hctr, const ww_params* p, int sm_count, cudaStream_t s) {
  auto t0 = std::chrono::steady_clock::now();
  ww_status st = run_search<FWD>(g, costs, flows, pot, ws, dctr, hctr, p->max_sweeps, sm_count,
                                 &ws->stats.search_iterations, s);
  auto t1 = std::chrono::steady_clock::now();
  ws->stats.ms_search += std::chrono::duration<double, std::milli>(t1 - t0).count();
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
  ws->stats.ms_other += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
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
