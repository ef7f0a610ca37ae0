// Bridging of mask-separated regions (Sec. II-D): the valid pixels of an
// unwrapped field fall into 4-connected regions whose relative 2pi levels the
// wrapped phase does not fix.  Regions are taken in order of decreasing size
// (ties: smaller first pixel first); every region after the first attaches to
// the nearest region already taken through the closest pair of pixels (squared
// Euclidean distance; ties: smaller parent rank, then smaller parent pixel
// index, then smaller child pixel index).  Across each such edge the offset is
// round((median_parent - median_child) / 2pi) whole cycles, each median taken
// over the unwrapped phase of the endpoint's region inside a window x window
// box centred on the endpoint, with the parent already shifted, so offsets
// propagate from parent to child.
//
// GPU design:
//   * regions: the component-label union-find with every edge between valid
//     pixels reliable; sizes by warp-aggregated atomics; the size order of the
//     (usually few) regions is sorted on the host;
//   * closest pairs: a closest pair of two regions always joins two pixels that
//     each have an invalid 4-neighbour (from any other pixel one step toward the
//     partner is strictly closer, and a valid neighbour belongs to the same
//     region), so only those "boundary" pixels take part.  They are grouped by
//     region rank; the pixels of every region taken before region k form a
//     prefix of that list, so all regions are answered at once by one
//     brute-force pass over (child boundary pixel, prefix) pairs, tiled through
//     shared memory; two cheap passes settle the ties;
//   * window medians: one block per edge endpoint sorts the window's values of
//     its region (bitonic sort in shared memory) and keeps the two middle ones;
//   * offsets: one thread walks the edges in rank order (each offset needs its
//     parent's), forming each median in FP64 as the middle value (odd count) or
//     the mean of the two middle values (even count) of phase + 2pi shift;
//   * the shift is applied to every valid pixel: phase in FP64 with one
//     rounding to fp32, cycle counts in int32.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "ww_internal.cuh"

namespace ww {
namespace {

constexpr double kTwoPiBridge = 6.283185307179586;  // fp64 nearest 2pi
constexpr int kMaxWindow = 127;
constexpr int kSortCap = 16384;  // >= kMaxWindow^2, a power of two

// size of each region, indexed by its root (label - 1); warp-aggregated
__global__ void k_region_sizes(const int32_t* __restrict__ labels, int64_t P, int32_t* __restrict__ size) {
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < P; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = base + threadIdx.x;
    const int32_t r = k < P ? labels[k] - 1 : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, r);
    if (r >= 0 && (threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1)) atomicAdd(&size[r], __popc(peers));
  }
}

// roots (pixels whose label points at themselves) with their sizes, compacted
__global__ void k_list_roots(const int32_t* __restrict__ labels, int64_t P, const int32_t* __restrict__ size,
                             int32_t* __restrict__ roots, int32_t* __restrict__ nroots) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x)
    if (labels[k] == (int32_t)k + 1) roots[atomicAdd(nroots, 1)] = (int32_t)k;
}

__global__ void k_scatter_rank(const int32_t* __restrict__ roots_sorted, int32_t R, int32_t* __restrict__ rank_at) {
  for (int32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < R; q += gridDim.x * blockDim.x)
    rank_at[roots_sorted[q]] = q;
}

__device__ __forceinline__ bool invalid_px(const float* unw, int64_t k) { return isnan(unw[k]); }

// rank map; boundary pixels (valid, with an invalid 4-neighbour inside the image) counted per rank
__global__ void k_rank_map(const float* __restrict__ unw, const int32_t* __restrict__ labels,
                           const int32_t* __restrict__ rank_at, int64_t m, int64_t n, int32_t* __restrict__ rank,
                           int32_t* __restrict__ bcount) {
  const int64_t P = m * n;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < P; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = base + threadIdx.x;
    int32_t rk = -1;
    bool bnd = false;
    if (k < P) {
      const int32_t lab = labels[k];
      rk = lab > 0 ? rank_at[lab - 1] : -1;
      rank[k] = rk;
      if (rk >= 0) {
        const int64_t i = k / n, j = k - (k / n) * n;
        bnd = (i > 0 && invalid_px(unw, k - n)) || (i + 1 < m && invalid_px(unw, k + n)) ||
              (j > 0 && invalid_px(unw, k - 1)) || (j + 1 < n && invalid_px(unw, k + 1));
      }
    }
    const int32_t key = bnd ? rk : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (key >= 0 && (threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1)) atomicAdd(&bcount[key], __popc(peers));
  }
}

// boundary pixels into their rank's slice of the list (order inside a slice free)
__global__ void k_scatter_boundary(const float* __restrict__ unw, const int32_t* __restrict__ rank, int64_t m,
                                   int64_t n, int32_t* __restrict__ cursor, int32_t* __restrict__ blist) {
  const int64_t P = m * n;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t rk = rank[k];
    if (rk < 0) continue;
    const int64_t i = k / n, j = k - (k / n) * n;
    const bool bnd = (i > 0 && invalid_px(unw, k - n)) || (i + 1 < m && invalid_px(unw, k + n)) ||
                     (j > 0 && invalid_px(unw, k - 1)) || (j + 1 < n && invalid_px(unw, k + 1));
    if (bnd) blist[atomicAdd(&cursor[rk], 1)] = (int32_t)k;
  }
}

constexpr int kPairThreads = 256;

// Pass A: for every region k >= 1, the smallest (d^2, parent rank) over pairs of
// a boundary pixel b of region k and a boundary pixel a of a region taken
// before it (the list prefix [0, bstart[k])).  Candidates are staged in shared
// memory 256 at a time; packed key = d^2 << 32 | rank(a).
__global__ void __launch_bounds__(kPairThreads) k_pairs_nearest(const int32_t* __restrict__ blist,
                                                                const int32_t* __restrict__ rank,
                                                                const int32_t* __restrict__ bstart, int32_t R,
                                                                int64_t n, unsigned long long* __restrict__ key1) {
  __shared__ int32_t ci[kPairThreads], cj[kPairThreads], cr[kPairThreads];
  const int32_t B = bstart[R];
  const int32_t first = bstart[1];
  for (int64_t base = first + (int64_t)blockIdx.x * kPairThreads; base < B;
       base += (int64_t)gridDim.x * kPairThreads) {
    const int64_t q = base + threadIdx.x;
    const bool have = q < B;
    int32_t bi = 0, bj = 0, kb = 0, lim = 0;
    if (have) {
      const int32_t p = blist[q];
      bi = (int32_t)(p / n);
      bj = (int32_t)(p - (int64_t)bi * n);
      kb = rank[p];
      lim = bstart[kb];
    }
    // the block's largest prefix: its last pixel has the largest rank (slices are in rank order)
    const int64_t qlast = min(base + kPairThreads, (int64_t)B) - 1;
    const int32_t lim_blk = bstart[rank[blist[qlast]]];
    unsigned long long best = ~0ull;
    for (int32_t t0 = 0; t0 < lim_blk; t0 += kPairThreads) {
      __syncthreads();
      const int32_t c = t0 + threadIdx.x;
      if (c < lim_blk) {
        const int32_t p = blist[c];
        ci[threadIdx.x] = (int32_t)(p / n);
        cj[threadIdx.x] = (int32_t)(p - (int64_t)(p / n) * n);
        cr[threadIdx.x] = rank[p];
      }
      __syncthreads();
      const int32_t cnt = min(kPairThreads, lim - t0);
      for (int32_t u = 0; u < cnt; ++u) {
        const int64_t di = bi - ci[u], dj = bj - cj[u];
        const unsigned long long d2 = (unsigned long long)(di * di + dj * dj);
        const unsigned long long key = (d2 << 32) | (uint32_t)cr[u];
        best = key < best ? key : best;
      }
    }
    if (have && best != ~0ull) atomicMin(&key1[kb], best);
  }
}

// Pass B: the smallest parent pixel index among the parent region's boundary
// pixels at the minimal distance from some boundary pixel of region k.
__global__ void k_pairs_parent_pixel(const int32_t* __restrict__ blist, const int32_t* __restrict__ rank,
                                     const int32_t* __restrict__ bstart, int32_t R, int64_t n,
                                     const unsigned long long* __restrict__ key1, int32_t* __restrict__ pa) {
  const int32_t B = bstart[R];
  for (int64_t q = bstart[1] + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < B;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = blist[q];
    const int32_t kb = rank[p];
    const unsigned long long k1 = key1[kb];
    const int64_t D = (int64_t)(k1 >> 32);
    const int32_t par = (int32_t)(k1 & 0xFFFFFFFFu);
    const int64_t bi = p / n, bj = p - (p / n) * n;
    int32_t bestp = 0x7FFFFFFF;
    for (int32_t c = bstart[par]; c < bstart[par + 1]; ++c) {
      const int32_t a = blist[c];
      const int64_t di = bi - a / n, dj = bj - (a - (int64_t)(a / n) * n);
      if (di * di + dj * dj == D && a < bestp) bestp = a;
    }
    if (bestp != 0x7FFFFFFF) atomicMin(&pa[kb], bestp);
  }
}

// Pass C: the smallest child pixel index at the minimal distance from the chosen parent pixel.
__global__ void k_pairs_child_pixel(const int32_t* __restrict__ blist, const int32_t* __restrict__ rank,
                                    const int32_t* __restrict__ bstart, int32_t R, int64_t n,
                                    const unsigned long long* __restrict__ key1, const int32_t* __restrict__ pa,
                                    int32_t* __restrict__ pb) {
  const int32_t B = bstart[R];
  for (int64_t q = bstart[1] + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < B;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = blist[q];
    const int32_t kb = rank[p];
    const int32_t a = pa[kb];
    const int64_t di = p / n - a / n, dj = (p - (int64_t)(p / n) * n) - (a - (int64_t)(a / n) * n);
    if (di * di + dj * dj == (int64_t)(key1[kb] >> 32)) atomicMin(&pb[kb], p);
  }
}

// One block per edge endpoint (2 (R-1) blocks; endpoint e: edge k = 1 + e / 2,
// parent side when e is even): the two middle values of the unwrapped phase of
// the endpoint's region inside the window, and their count.
__global__ void __launch_bounds__(1024) k_window_median(const float* __restrict__ unw, const int32_t* __restrict__ rank,
                                                        int64_t m, int64_t n, int32_t half,
                                                        const unsigned long long* __restrict__ key1,
                                                        const int32_t* __restrict__ pa, const int32_t* __restrict__ pb,
                                                        double* __restrict__ mid, int32_t* __restrict__ count) {
  extern __shared__ float v[];
  __shared__ int32_t s_cnt;
  const int e = blockIdx.x;
  const int k = 1 + e / 2;
  const bool parent = (e & 1) == 0;
  const int64_t p = parent ? pa[k] : pb[k];
  const int32_t region = parent ? (int32_t)(key1[k] & 0xFFFFFFFFu) : k;
  const int64_t ci = p / n, cj = p - (p / n) * n;
  const int64_t i0 = max((int64_t)0, ci - half), i1 = min(m - 1, ci + half);
  const int64_t j0 = max((int64_t)0, cj - half), j1 = min(n - 1, cj + half);
  const int64_t w = j1 - j0 + 1, cells = (i1 - i0 + 1) * w;
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  for (int64_t c = threadIdx.x; c < cells; c += blockDim.x) {
    const int64_t i = i0 + c / w, j = j0 + c % w, kk = i * n + j;
    if (rank[kk] == region) v[atomicAdd(&s_cnt, 1)] = unw[kk];
  }
  __syncthreads();
  const int cnt = s_cnt;
  int size = 1;
  while (size < cnt) size <<= 1;
  for (int c = cnt + threadIdx.x; c < size; c += blockDim.x) v[c] = INFINITY;
  __syncthreads();
  // bitonic sort of v[0, size) ascending
  for (int kk = 2; kk <= size; kk <<= 1) {
    for (int jj = kk >> 1; jj > 0; jj >>= 1) {
      for (int t = threadIdx.x; t < size; t += blockDim.x) {
        const int x = t ^ jj;
        if (x > t) {
          const bool up = (t & kk) == 0;
          const float a = v[t], b = v[x];
          if ((a > b) == up) {
            v[t] = b;
            v[x] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    mid[2 * e] = (double)v[(cnt - 1) / 2];
    mid[2 * e + 1] = (double)v[cnt / 2];
    count[e] = cnt;
  }
}

// Offsets in rank order, one thread: each edge needs its parent's final shift.
// median = lo + c (odd count) or ((lo + c) + (hi + c)) / 2 (even), c = 2pi shift.
__global__ void k_bridge_offsets(int32_t R, const unsigned long long* __restrict__ key1, const double* __restrict__ mid,
                                 const int32_t* __restrict__ count, int32_t* __restrict__ shift) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  shift[0] = 0;
  for (int32_t k = 1; k < R; ++k) {
    const int32_t par = (int32_t)(key1[k] & 0xFFFFFFFFu);
    const int ep = 2 * (k - 1), ec = ep + 1;
    const double cp = __dmul_rn(kTwoPiBridge, (double)shift[par]);
    const double mp = (count[ep] & 1) ? __dadd_rn(mid[2 * ep], cp)
                                      : __ddiv_rn(__dadd_rn(__dadd_rn(mid[2 * ep], cp), __dadd_rn(mid[2 * ep + 1], cp)), 2.0);
    const double mc = (count[ec] & 1) ? mid[2 * ec] : __ddiv_rn(__dadd_rn(mid[2 * ec], mid[2 * ec + 1]), 2.0);
    shift[k] = (int32_t)rint(__ddiv_rn(__dsub_rn(mp, mc), kTwoPiBridge));
  }
}

__global__ void k_bridge_apply(float* __restrict__ unw, int32_t* __restrict__ cycles, const int32_t* __restrict__ rank,
                               const int32_t* __restrict__ shift_of, int64_t P, int32_t* __restrict__ region_out,
                               int32_t* __restrict__ shift_out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t rk = rank[k];
    const int32_t s = rk >= 0 ? shift_of[rk] : 0;
    if (rk >= 0 && s != 0) {
      unw[k] = __double2float_rn(__dadd_rn((double)unw[k], __dmul_rn(kTwoPiBridge, (double)s)));
      if (cycles) cycles[k] += s;
    }
    if (region_out) region_out[k] = rk;
    if (shift_out) shift_out[k] = s;
  }
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

}  // namespace
}  // namespace ww

extern "C" ww_status ww_bridge(float* unwrapped, int32_t* cycles, int64_t m, int64_t n, int32_t window,
                               int32_t* region, int32_t* shift, int32_t* n_regions, ww_stream stream) {
  using namespace ww;
  if (!unwrapped || m < 1 || n < 1 || m > (1ll << 30) || n > (1ll << 30) || m * n >= (1ll << 31) || window < 1 ||
      window > kMaxWindow || (window & 1) == 0)
    return WW_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t P = m * n;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = (int)std::min<int64_t>((P + 255) / 256, (int64_t)sms * 16);
  DevBuf labels, work, rank;
  // labels: the regions (union-find over every edge between valid pixels)
  if (cudaMalloc(&labels.p, P * 4) != cudaSuccess || cudaMalloc(&work.p, P * 4 + 64) != cudaSuccess ||
      cudaMalloc(&rank.p, P * 4) != cudaSuccess)
    return WW_ERR_OOM;
  ww_status st = launch_components(nullptr, nullptr, unwrapped, m, n, 0, labels.as<int32_t>(), s);
  if (st != WW_OK) return st;
  // region sizes by root, then the roots compacted into the tail of the same buffer
  int32_t* size = work.as<int32_t>();
  WW_CUDA_TRY(cudaMemsetAsync(size, 0, P * 4 + 64, s));
  k_region_sizes<<<blocks, 256, 0, s>>>(labels.as<int32_t>(), P, size);
  DevBuf roots;
  int32_t* nroots = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(work.p) + P * 4);
  if (cudaMalloc(&roots.p, P * 4) != cudaSuccess) return WW_ERR_OOM;
  k_list_roots<<<blocks, 256, 0, s>>>(labels.as<int32_t>(), P, size, roots.as<int32_t>(), nroots);
  int32_t R = 0;
  WW_CUDA_TRY(cudaMemcpyAsync(&R, nroots, 4, cudaMemcpyDeviceToHost, s));
  WW_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<int32_t> hroots(R), hsize(R);
  if (R > 0) {
    WW_CUDA_TRY(cudaMemcpy(hroots.data(), roots.p, (size_t)R * 4, cudaMemcpyDeviceToHost));
    std::sort(hroots.begin(), hroots.end());
    // sizes of the roots (gathered on the host from the device array, one copy per root
    // would be slow for many regions: copy the whole size array only when there are many)
    std::vector<int32_t> all;
    if ((int64_t)R * 8 > P) {
      all.resize(P);
      WW_CUDA_TRY(cudaMemcpy(all.data(), size, P * 4, cudaMemcpyDeviceToHost));
      for (int32_t q = 0; q < R; ++q) hsize[q] = all[hroots[q]];
    } else {
      for (int32_t q = 0; q < R; ++q) WW_CUDA_TRY(cudaMemcpy(&hsize[q], size + hroots[q], 4, cudaMemcpyDeviceToHost));
    }
    std::vector<int32_t> order(R);
    for (int32_t q = 0; q < R; ++q) order[q] = q;
    // decreasing size, ties: smaller first pixel (the root is the region's smallest index)
    std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
      return hsize[a] != hsize[b] ? hsize[a] > hsize[b] : hroots[a] < hroots[b];
    });
    for (int32_t q = 0; q < R; ++q) hsize[q] = hroots[order[q]];  // roots in rank order
    WW_CUDA_TRY(cudaMemcpy(roots.p, hsize.data(), (size_t)R * 4, cudaMemcpyHostToDevice));
  }
  if (n_regions) *n_regions = R;
  int32_t* rank_at = size;  // reused: root -> rank
  if (R > 0) k_scatter_rank<<<std::max(1, std::min(sms * 16, (R + 255) / 256)), 256, 0, s>>>(roots.as<int32_t>(), R, rank_at);
  // boundary pixels per rank, their slices (exclusive scan on the host) and the list
  DevBuf bbuf;
  if (cudaMalloc(&bbuf.p, (size_t)(R + 1) * 4 * 2) != cudaSuccess) return WW_ERR_OOM;
  int32_t* bcount = bbuf.as<int32_t>();
  int32_t* bstart = bcount + (R + 1);
  WW_CUDA_TRY(cudaMemsetAsync(bcount, 0, (size_t)(R + 1) * 4, s));
  k_rank_map<<<blocks, 256, 0, s>>>(unwrapped, labels.as<int32_t>(), rank_at, m, n, rank.as<int32_t>(), bcount);
  std::vector<int32_t> hb(R + 1, 0);
  if (R > 0) WW_CUDA_TRY(cudaMemcpyAsync(hb.data(), bcount, (size_t)R * 4, cudaMemcpyDeviceToHost, s));
  WW_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<int32_t> hs(R + 1, 0);
  for (int32_t q = 0; q < R; ++q) hs[q + 1] = hs[q] + hb[q];
  std::vector<int32_t> shift_of(std::max(R, 1), 0);
  DevBuf sbuf;
  if (cudaMalloc(&sbuf.p, (size_t)std::max(R, 1) * 4) != cudaSuccess) return WW_ERR_OOM;
  WW_CUDA_TRY(cudaMemsetAsync(sbuf.p, 0, (size_t)std::max(R, 1) * 4, s));
  if (R > 1) {
    WW_CUDA_TRY(cudaMemcpyAsync(bstart, hs.data(), (size_t)(R + 1) * 4, cudaMemcpyHostToDevice, s));
    WW_CUDA_TRY(cudaMemcpyAsync(bcount, hs.data(), (size_t)R * 4, cudaMemcpyHostToDevice, s));  // cursors
    int32_t* blist = labels.as<int32_t>();  // labels are no longer needed: the list takes their place
    k_scatter_boundary<<<blocks, 256, 0, s>>>(unwrapped, rank.as<int32_t>(), m, n, bcount, blist);
    // per region k: key1 (d^2, parent rank), parent pixel, child pixel
    DevBuf kbuf, pbuf, mbuf;
    if (cudaMalloc(&kbuf.p, (size_t)R * 8) != cudaSuccess || cudaMalloc(&pbuf.p, (size_t)R * 8) != cudaSuccess ||
        cudaMalloc(&mbuf.p, (size_t)(R - 1) * 2 * (2 * 8 + 4)) != cudaSuccess)
      return WW_ERR_OOM;
    unsigned long long* key1 = kbuf.as<unsigned long long>();
    int32_t* pa = pbuf.as<int32_t>();
    int32_t* pb = pa + R;
    WW_CUDA_TRY(cudaMemsetAsync(key1, 0xFF, (size_t)R * 8, s));
    WW_CUDA_TRY(cudaMemsetAsync(pa, 0x7F, (size_t)R * 8, s));  // 0x7F7F7F7F: above any pixel index
    const int64_t nchild = hs[R] - hs[1];
    const int pblocks = (int)std::max<int64_t>(1, std::min<int64_t>((nchild + kPairThreads - 1) / kPairThreads,
                                                                      (int64_t)sms * 8));
    k_pairs_nearest<<<pblocks, kPairThreads, 0, s>>>(blist, rank.as<int32_t>(), bstart, R, n, key1);
    k_pairs_parent_pixel<<<pblocks, kPairThreads, 0, s>>>(blist, rank.as<int32_t>(), bstart, R, n, key1, pa);
    k_pairs_child_pixel<<<pblocks, kPairThreads, 0, s>>>(blist, rank.as<int32_t>(), bstart, R, n, key1, pa, pb);
    double* mid = mbuf.as<double>();
    int32_t* count = reinterpret_cast<int32_t*>(mid + (size_t)(R - 1) * 2 * 2);
    const size_t smem = kSortCap * sizeof(float);
    WW_CUDA_TRY(cudaFuncSetAttribute(k_window_median, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_window_median<<<(unsigned)(2 * (R - 1)), 1024, smem, s>>>(unwrapped, rank.as<int32_t>(), m, n, window / 2, key1,
                                                               pa, pb, mid, count);
    k_bridge_offsets<<<1, 1, 0, s>>>(R, key1, mid, count, sbuf.as<int32_t>());
  }
  k_bridge_apply<<<blocks, 256, 0, s>>>(unwrapped, cycles, rank.as<int32_t>(), sbuf.as<int32_t>(), P, region, shift);
  WW_CUDA_TRY(cudaGetLastError());
  WW_CUDA_TRY(cudaStreamSynchronize(s));
  return WW_OK;
}
