// Connected-component labels of an unwrapped field (Sec. II-D): a pixel edge is
// reliable when both of its pixels are valid and moving its ambiguity
// difference by +1 or -1 would raise the MCF objective by more than a
// threshold; components grow over reliable edges.
//
// Union-find on the label array itself, which holds parent + 1 (0 = invalid
// pixel), so a root holds its own label and the compressed array is the result:
//   1. rows: one warp per row links each valid pixel to the start of its run
//      of reliable horizontal edges (ballot per 32 pixels, the run carried
//      across segments); a run start is its own root;
//   2. one thread per pixel unites it with its lower neighbour over a reliable
//      vertical edge: the larger of the two roots is hooked under the smaller
//      by compare-and-swap (a root's pointer changes only from itself), and
//      finds halve their paths with plain stores of an ancestor;
//   3. every pixel's pointer is set to its root by read-only finds, which
//      leaves root + 1 (the label) in every valid pixel.
// Pointers only ever point to smaller indices, so every chain ends at a root
// within as many steps as its start index and each component's root is its
// smallest row-major index: the labels are unique, whatever the schedule.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "ww_internal.cuh"

namespace ww {
namespace {

// parent index of x (the array stores parent + 1; -1 for an invalid pixel)
__device__ __forceinline__ int32_t ld_parent(const int32_t* parent, int32_t x) {
  return *((volatile const int32_t*)(parent + x)) - 1;
}

// Root of x with path halving (each visited node skips to its grandparent).
__device__ __forceinline__ int32_t find_halving(int32_t* parent, int32_t x) {
  for (int32_t s = 0, lim = x; s <= lim; ++s) {
    const int32_t p = ld_parent(parent, x);
    if (p == x) return x;
    const int32_t gp = ld_parent(parent, p);
    if (gp != p) parent[x] = gp + 1;
    x = gp;
  }
  return x;  // not reached: the chain from x has at most x steps
}

__device__ __forceinline__ int32_t find_readonly(const int32_t* parent, int32_t x) {
  for (int32_t s = 0, lim = x; s <= lim; ++s) {
    const int32_t p = ld_parent(parent, x);
    if (p == x) return x;
    x = p;
  }
  return x;
}

__device__ __forceinline__ void unite(int32_t* parent, int32_t a, int32_t b) {
  // every failed swap means b's root was hooked under a smaller index, so the
  // loop runs at most b + 1 times
  for (int32_t s = 0, lim = b; s <= lim; ++s) {
    a = find_halving(parent, a);
    b = find_halving(parent, b);
    if (a == b) return;
    if (a > b) {
      const int32_t t = a;
      a = b;
      b = t;
    }
    if (atomicCAS(parent + b, b + 1, a + 1) == b + 1) return;
  }
}

// Reliable: both pixels valid, no flow on the edge, min(c+, c-) > threshold.
__device__ __forceinline__ bool reliable(int8_t dk, int16_t cp, int16_t cm, int32_t threshold) {
  return dk == 0 && min((int32_t)cp, (int32_t)cm) > threshold;
}

// Without cost planes (costs == nullptr, the regions of the bridging step) every
// edge between two valid pixels counts as reliable.
__device__ __forceinline__ bool reliable_at(const int16_t* costs, const int8_t* flows, int64_t P, int64_t e,
                                            int plane, int32_t threshold) {
  if (!costs) return true;
  return reliable(__ldg(flows + plane * P + e), __ldg(costs + 2 * plane * P + e), __ldg(costs + (2 * plane + 1) * P + e),
                  threshold);
}

// Phase 1: one warp per row, 32 pixels per step.
__global__ void k_cc_rows(const int16_t* __restrict__ costs, const int8_t* __restrict__ flows,
                          const float* __restrict__ unw, int64_t m, int64_t n, int32_t threshold,
                          int32_t* __restrict__ parent) {
  const int64_t P = m * n;
  const unsigned lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < m; i += warps) {
    int32_t carry = -1;  // root of the previous segment's last pixel
    for (int64_t j0 = 0; j0 < n; j0 += 32) {
      const int64_t j = j0 + lane, k = i * n + j;
      const bool valid = j < n && !isnan(__ldg(unw + k));
      // h edge (i,j-1)-(i,j): dk = flows[0], c+ = costs[0], c- = costs[1] at (i,j-1)
      const bool link = valid && j > 0 && !isnan(__ldg(unw + k - 1)) && reliable_at(costs, flows, P, k - 1, 0, threshold);
      const unsigned starts = __ballot_sync(0xffffffffu, valid && !link);
      const unsigned upto = starts & (0xffffffffu >> (31 - lane));
      // a linked pixel with no start at or below its lane continues the previous segment's run
      const int32_t root = upto ? (int32_t)(i * n + j0 + (31 - __clz(upto))) : carry;
      if (j < n) parent[k] = valid ? root + 1 : 0;
      carry = __shfl_sync(0xffffffffu, root, 31);
    }
  }
}

// Phase 2: vertical edges, one thread per pixel.
__global__ void k_cc_cols(const int16_t* __restrict__ costs, const int8_t* __restrict__ flows,
                          const float* __restrict__ unw, int64_t m, int64_t n, int32_t threshold,
                          int32_t* parent) {
  const int64_t P = m * n;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P - n; k += (int64_t)gridDim.x * blockDim.x) {
    // v edge (i,j)-(i+1,j): dk = flows[1], c+ = costs[2], c- = costs[3]
    if (!isnan(__ldg(unw + k)) && !isnan(__ldg(unw + k + n)) && reliable_at(costs, flows, P, k, 1, threshold))
      unite(parent, (int32_t)k, (int32_t)(k + n));
  }
}

// Every pointer to its root: reads follow chains, each thread writes only its
// own pixel (an ancestor either way for the other threads' chains).
__global__ void k_cc_compress(int64_t P, int32_t* parent) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = ld_parent(parent, (int32_t)k);
    if (p < 0 || p == (int32_t)k) continue;
    parent[k] = find_readonly(parent, p) + 1;
  }
}

}  // namespace

ww_status launch_components(const int16_t* costs, const int8_t* flows, const float* unwrapped, int64_t m, int64_t n,
                            int32_t threshold, int32_t* labels, cudaStream_t s) {
  const int64_t P = m * n;
  if (P == 0) return WW_OK;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = (int)std::min<int64_t>((P + 255) / 256, (int64_t)sms * 16);
  const int row_blocks = (int)std::min<int64_t>((m + 7) / 8, (int64_t)sms * 16);
  k_cc_rows<<<row_blocks, 256, 0, s>>>(costs, flows, unwrapped, m, n, threshold, labels);
  if (m > 1) k_cc_cols<<<blocks, 256, 0, s>>>(costs, flows, unwrapped, m, n, threshold, labels);
  k_cc_compress<<<blocks, 256, 0, s>>>(P, labels);
  WW_CUDA_TRY(cudaGetLastError());
  return WW_OK;
}

}  // namespace ww
