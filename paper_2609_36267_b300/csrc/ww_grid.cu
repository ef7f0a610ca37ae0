// Stencil and scan kernels of the hot path:
//   k_residues       Eq. 1 residues + ground charge (Sec. II-A)
//   k_costs          slope estimate, LUT gather, mask rule (Sec. II-B)
//   k_steep_*        steep-edge bound with its 3% cap (Sec. II-B)
//   k_integrate_*    integration in integer cycles (Sec. II-A, II-C)
// All are HBM-bound streaming stencils; inputs are staged through shared memory
// tiles so each pixel is read from HBM once per kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "ww_internal.cuh"

namespace ww {
namespace {

// ---------------- residues ----------------
constexpr int RTX = 32, RTY = 32, RTT = 8;  // node tile RTY x RTX, thread block RTX x RTT

// One RTY x RTX tile of nodes, tile (by, bx); each thread takes RTY / RTT rows.
// The pixel tile (+1 row and column) is loaded with every load of a thread
// issued before the first store, and the block adds its charge sum to r_G once.
__device__ __forceinline__ void residues_tile(const void* __restrict__ ifg, int is_complex,
                                              const float* __restrict__ coh, const uint8_t* __restrict__ mask,
                                              int64_t m, int64_t n, int8_t* __restrict__ res,
                                              int32_t* __restrict__ ground, int64_t bx, int64_t by) {
  __shared__ float sp[RTY + 1][RTX + 1];
  const int64_t i0 = by * RTY, j0 = bx * RTX;
  const int tid = threadIdx.y * RTX + threadIdx.x;
  {
    constexpr int kQ = (RTY + 1) * (RTX + 1), kU = (kQ + RTX * RTT - 1) / (RTX * RTT);
    float v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int q = tid + u * RTX * RTT;
      const int64_t i = i0 + q / (RTX + 1), j = j0 + q % (RTX + 1);
      v[u] = (q < kQ && i < m && j < n) ? load_pixel(ifg, is_complex, coh, mask, i * n + j).psi : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int q = tid + u * RTX * RTT;
      if (q < kQ) sp[q / (RTX + 1)][q % (RTX + 1)] = v[u];
    }
  }
  __syncthreads();
  const int tx = threadIdx.x;
  int s = 0;
#pragma unroll
  for (int k = 0; k < RTY / RTT; ++k) {
    const int ty = threadIdx.y + k * RTT;
    const int64_t i = i0 + ty, j = j0 + tx;
    if (i < m - 1 && j < n - 1) {
      int n_top = wrap_count(__fsub_rn(sp[ty][tx + 1], sp[ty][tx]));
      int n_right = wrap_count(__fsub_rn(sp[ty + 1][tx + 1], sp[ty][tx + 1]));
      int n_bottom = wrap_count(__fsub_rn(sp[ty + 1][tx + 1], sp[ty + 1][tx]));
      int n_left = wrap_count(__fsub_rn(sp[ty + 1][tx], sp[ty][tx]));
      const int r = -(n_top + n_right - n_bottom - n_left);
      res[i * (n - 1) + j] = (int8_t)r;
      s += r;
    }
  }
  // block sum of charges -> ground gets minus the total
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ int ws[RTT];
  if (tx == 0) ws[threadIdx.y] = s;
  __syncthreads();
  if (tid == 0) {
    int t = 0;
    for (int k = 0; k < RTT; ++k) t += ws[k];
    if (t) atomicAdd(ground, -t);
  }
}

__global__ void __launch_bounds__(RTX* RTT) k_residues(const void* __restrict__ ifg, int is_complex,
                                                        const float* __restrict__ coh,
                                                        const uint8_t* __restrict__ mask, int64_t m,
                                                        int64_t n, int8_t* __restrict__ res,
                                                        int32_t* __restrict__ ground) {
  const int64_t gx = (n - 1 + RTX - 1) / RTX, b = blockIdx.x;  // one-dimensional grid of tiles
  residues_tile(ifg, is_complex, coh, mask, m, n, res, ground, b % gx, b / gx);
}

// ---------------- costs ----------------
constexpr int CTX = 32, CTY = 32, CW = 3;  // tile, max box half-width

struct SteepCtr {
  unsigned long long valid_edges;   // [0]
  unsigned long long candidates;    // [1]
  unsigned long long above;         // [2] candidates strictly above the high-bits bin
  unsigned long long hi_bin;        // [3]
  unsigned long long threshold;     // [4] exact |d| bits of the cut
  unsigned long long take_at_thr;   // [5] candidates equal to threshold to zero
  unsigned long long mode;          // [6] 0 none/all, 1 select
  unsigned long long pad;
};

__device__ __forceinline__ float edge_d(float a, float b) {
  float dp = __fsub_rn(b, a);
  return __fsub_rn(dp, __fmul_rn(kTwoPiF, (float)wrap_count(dp)));
}

// Slope estimate from the window sum S of the fixed-point (2^22) gradients of
// its cnt valid edges: fp32(S) / (cnt 2^22) with the divisor exact and the
// quotient correctly rounded (fp32(S) itself rounds once |S| exceeds 2^24).
__device__ __forceinline__ float slope_of_sum(int32_t S, int cnt) {
  return __fdiv_rn(__int2float_rn(S), __fmul_rn((float)cnt, kQScale));
}

// Phasor slope estimate: integer sums of the window's edge phasors (length 2^30
// each, at most 49 of them: below 2^36), each sum rounded once to fp32, then the
// CORDIC atan2; 0 for an empty window.
template <int EXP>
__device__ __forceinline__ float window_phasor(const int32_t (*xs)[EXP], const int32_t (*ys)[EXP],
                                               const uint8_t (*es)[EXP], int R, int C, int w) {
  long long SX = 0, SY = 0;
  for (int d = -w; d <= w; ++d)
    for (int e = -w; e <= w; ++e)
      if (es[R + d][C + e]) {
        SX += xs[R + d][C + e];
        SY += ys[R + d][C + e];
      }
  return cordic_phase(__ll2float_rn(SX), __ll2float_rn(SY));
}

// One CTY x CTX tile of pixels (both edges of each pixel), tile (by, bx).
// Steep candidates are counted, and their edge keys appended to `list` while
// it has room (`list` may be null).
// SLOPE 0: slope estimate = fixed-point mean of the window's wrapped gradients
// (separable sums); SLOPE 1: argument of the sum of their unit phasors (CORDIC
// rotation per edge, integer window sums, CORDIC atan2).  LOOKUP 0: nearest bin
// of the int16 table; LOOKUP 1: bilinear interpolation of `ratio`.
template <int SLOPE, int LOOKUP, int W>
__device__ __forceinline__ void costs_tile(const void* __restrict__ ifg, int is_complex,
                                           const float* __restrict__ coh, const uint8_t* __restrict__ mask,
                                           int64_t m, int64_t n, const int16_t* __restrict__ table,
                                           const float* __restrict__ ratio, int w, float steep_rad,
                                           int16_t* __restrict__ costs, SteepCtr* ctr, uint32_t* __restrict__ list,
                                           unsigned long long list_cap, int64_t bx, int64_t by,
                                           int8_t* __restrict__ res = nullptr, int32_t* __restrict__ ground = nullptr) {
  // W >= 0: the window half width w is the compile-time W and the tile's halo
  // is W wide; W < 0: any w up to CW at run time, halo CW
  constexpr int HW = W < 0 ? CW : W;
  constexpr int PX = CTX + 2 * HW + 1, PY = CTY + 2 * HW + 1;  // pixel tile
  constexpr int EX = CTX + 2 * HW, EY = CTY + 2 * HW;          // edge tile
  if constexpr (W >= 0) w = W;
  __shared__ float sp[PY][PX];
  __shared__ float sc[PY][PX];
  __shared__ uint8_t sv[PY][PX];
  // SLOPE 0: fixed-point gradients; SLOPE 1: cos part of the edge phasors
  __shared__ int32_t qh[EY][EX + 1], qv[EY][EX + 1];
  __shared__ int32_t yh[SLOPE ? EY : 1][EX + 1], yv[SLOPE ? EY : 1][EX + 1];  // sin part (SLOPE 1)
  __shared__ uint8_t eh[EY][EX + 1], ev[EY][EX + 1];
  // per edge: its wrap count + 1 (bits 0-1, for the residues) and the steep test (bit 2)
  __shared__ uint8_t fh[EY][EX + 1], fv[EY][EX + 1];
  __shared__ int32_t rh[SLOPE ? 1 : EY][CTX], rv[SLOPE ? 1 : EY][CTX];  // row (horizontal) partial sums
  __shared__ uint8_t nh[SLOPE ? 1 : EY][CTX], nv[SLOPE ? 1 : EY][CTX];  // row partial counts
  const int64_t i0 = by * CTY, j0 = bx * CTX;
  const int tid = threadIdx.x;
  // 1. prepared pixels, tile origin (i0 - HW, j0 - HW); every load of a thread
  // is issued before its first store
  {
    constexpr int kU = (PY * PX + 255) / 256;
    Pix px[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int q = tid + 256 * u;
      const int64_t i = i0 - HW + q / PX, j = j0 - HW + q % PX;
      px[u] = Pix{0.0f, 0.0f, false};
      if (q < PY * PX && i >= 0 && i < m && j >= 0 && j < n) px[u] = load_pixel(ifg, is_complex, coh, mask, i * n + j);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int q = tid + 256 * u;
      if (q >= PY * PX) continue;
      const int r = q / PX, c = q % PX;
      sp[r][c] = px[u].psi;
      sc[r][c] = px[u].coh;
      sv[r][c] = px[u].valid ? 1 : 0;
    }
  }
  __syncthreads();
  // 2. fixed-point wrapped gradients of every edge in the extended tile
  for (int q = tid; q < EY * EX; q += 256) {
    int r = q / EX, c = q % EX;
    int64_t i = i0 - HW + r, j = j0 - HW + c;
    int32_t a = 0, b = 0, ya = 0, yb = 0;
    uint8_t ea = 0, eb = 0, fa = 0, fb = 0;
    if (i >= 0 && i < m && j >= 0) {
      // the wrapped difference of edge_d, kept apart: its wrap count serves the
      // residues whether or not the pixels are valid (invalid phases are 0)
      if (j + 1 < n) {
        const float dp = __fsub_rn(sp[r][c + 1], sp[r][c]);
        const int wc = wrap_count(dp);
        fa = (uint8_t)(wc + 1);
        if (sv[r][c] && sv[r][c + 1]) {
          const float d = __fsub_rn(dp, __fmul_rn(kTwoPiF, (float)wc));
          if constexpr (SLOPE == 0)
            a = __float2int_rn(__fmul_rn(d, kQScale));
          else
            cordic_cos_sin(__float2int_rn(__fmul_rn(d, 536870912.0f)), &a, &ya);
          ea = 1;
          if (fabsf(d) > steep_rad) fa |= 4;
        }
      }
      if (i + 1 < m && j < n) {
        const float dp = __fsub_rn(sp[r + 1][c], sp[r][c]);
        const int wc = wrap_count(dp);
        fb = (uint8_t)(wc + 1);
        if (sv[r][c] && sv[r + 1][c]) {
          const float d = __fsub_rn(dp, __fmul_rn(kTwoPiF, (float)wc));
          if constexpr (SLOPE == 0)
            b = __float2int_rn(__fmul_rn(d, kQScale));
          else
            cordic_cos_sin(__float2int_rn(__fmul_rn(d, 536870912.0f)), &b, &yb);
          eb = 1;
          if (fabsf(d) > steep_rad) fb |= 4;
        }
      }
    }
    qh[r][c] = a;
    eh[r][c] = ea;
    qv[r][c] = b;
    ev[r][c] = eb;
    fh[r][c] = fa;
    fv[r][c] = fb;
    if constexpr (SLOPE == 1) {
      yh[r][c] = ya;
      yv[r][c] = yb;
    }
  }
  __syncthreads();
  // 3. horizontal window sums for the output columns, every extended row
  for (int q = tid; q < (SLOPE ? 0 : EY * CTX); q += 256) {
    int r = q / CTX, c = q % CTX;
    int32_t sa = 0, sb = 0;
    int ca = 0, cb = 0;
    if constexpr (W >= 0) {
#pragma unroll
      for (int d = -W; d <= W; ++d) {
        const int cc = c + HW + d;
        sa += qh[r][cc];
        ca += eh[r][cc];
        sb += qv[r][cc];
        cb += ev[r][cc];
      }
    } else {
      for (int d = -w; d <= w; ++d) {
        const int cc = c + HW + d;
        sa += qh[r][cc];
        ca += eh[r][cc];
        sb += qv[r][cc];
        cb += ev[r][cc];
      }
    }
    rh[r][c] = sa;
    nh[r][c] = (uint8_t)ca;
    rv[r][c] = sb;
    nv[r][c] = (uint8_t)cb;
  }
  __syncthreads();
  // 4. vertical sums, slope estimate, LUT gather, mask rule; steep candidates.
  // A thread takes column c of the tile and a strip of kStrip consecutive rows,
  // so the vertical window sums of the mean slope slide down the strip (the
  // same integer sums as summing each window anew).
  const int64_t P = m * n;
  unsigned cnt_valid = 0;
  int charge = 0;  // sum of this thread's residues (Eq. 1), when res is given
  const unsigned lane = tid & 31, warp = tid >> 5;
  constexpr int kStrip = CTY / 8;  // 8 warps of 32 columns cover the tile's rows
  const int c = (int)lane, r0 = (int)warp * kStrip, C = c + HW;
  unsigned hcand = 0, vcand = 0;  // steep candidates of the strip: bit t for row r0 + t
  int32_t wsh = 0, wsv = 0;       // SLOPE 0: window sums of the h and v gradients
  int wch = 0, wcv = 0;           // and of their valid counts
  if constexpr (SLOPE == 0) {
    for (int d = -w; d <= w; ++d) {
      const int RR = r0 + HW + d;
      wsh += rh[RR][c];
      wch += nh[RR][c];
      wsv += rv[RR][c];
      wcv += nv[RR][c];
    }
  }
#pragma unroll
  for (int t = 0; t < kStrip; ++t) {
    const int r = r0 + t, R = r + HW;
    if constexpr (SLOPE == 0) {
      if (t > 0) {  // the window moves down one row
        const int in = R + w, out = R - w - 1;
        wsh += rh[in][c] - rh[out][c];
        wch += (int)nh[in][c] - (int)nh[out][c];
        wsv += rv[in][c] - rv[out][c];
        wcv += (int)nv[in][c] - (int)nv[out][c];
      }
    }
    const int64_t i = i0 + r, j = j0 + c;
    if (i >= m || j >= n) continue;
    const int64_t k = i * n + j;
    // h edge (i,j)
    int16_t hp = 0, hm = 0;
    if (eh[R][C]) {
      float ah;
      if constexpr (SLOPE == 0)
        ah = slope_of_sum(wsh, wch);
      else
        ah = window_phasor(qh, yh, eh, R, C, w);
      const float ge = fminf(sc[R][C], sc[R][C + 1]);
      if (LOOKUP == 0) {
        const int ig = gamma_index(ge);
        hp = __ldg(table + ig * kNAlpha + alpha_index(ah));
        hm = __ldg(table + ig * kNAlpha + alpha_index(-ah));
      } else {
        hp = bilinear_cost(ratio, ah, ge);
        hm = bilinear_cost(ratio, -ah, ge);
      }
      ++cnt_valid;
      if (fh[R][C] & 4) hcand |= 1u << t;
    }
    costs[k] = hp;
    costs[P + k] = hm;
    int16_t vp = 0, vm = 0;
    if (ev[R][C]) {
      float av;
      if constexpr (SLOPE == 0)
        av = slope_of_sum(wsv, wcv);
      else
        av = window_phasor(qv, yv, ev, R, C, w);
      const float ge = fminf(sc[R][C], sc[R + 1][C]);
      if (LOOKUP == 0) {
        const int ig = gamma_index(ge);
        vp = __ldg(table + ig * kNAlpha + alpha_index(av));
        vm = __ldg(table + ig * kNAlpha + alpha_index(-av));
      } else {
        vp = bilinear_cost(ratio, av, ge);
        vm = bilinear_cost(ratio, -av, ge);
      }
      ++cnt_valid;
      if (fv[R][C] & 4) vcand |= 1u << t;
    }
    costs[2 * P + k] = vp;
    costs[3 * P + k] = vm;
    // residue of the node whose top-left pixel is (i,j), from the same prepared phases
    if (res && i < m - 1 && j < n - 1) {
      // -(top + right - bottom - left) of the four wrap counts around the node
      // (the +1 of the stored counts cancels)
      const int rr = -((fh[R][C] & 3) + (fv[R][C + 1] & 3) - (fh[R + 1][C] & 3) - (fv[R][C] & 3));
      res[i * (n - 1) + j] = (int8_t)rr;
      charge += rr;
    }
  }
  // count the candidates of the block (one global atomic) and place each thread's
  // keys after the earlier threads' (an exclusive scan of the per-thread counts)
  const unsigned mine = __popc(hcand) + __popc(vcand);
  unsigned incl = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
    if ((int)lane >= o) incl += y;
  }
  __shared__ unsigned s_wsum[8];
  __shared__ unsigned long long s_base;
  __shared__ unsigned s_valid[8];
  __shared__ int s_charge[8];
  if (lane == 31) s_wsum[warp] = incl;
  for (int o = 16; o > 0; o >>= 1) cnt_valid += __shfl_xor_sync(0xffffffffu, cnt_valid, o);
  if (lane == 0) s_valid[warp] = cnt_valid;
  if (res) {
    for (int o = 16; o > 0; o >>= 1) charge += __shfl_xor_sync(0xffffffffu, charge, o);
    if (lane == 0) s_charge[warp] = charge;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned tot = 0;
    unsigned long long v = 0;
    for (int w2 = 0; w2 < 8; ++w2) {
      tot += s_wsum[w2];
      v += s_valid[w2];
    }
    s_base = tot ? atomicAdd(&ctr->candidates, (unsigned long long)tot) : 0ull;
    if (v) atomicAdd(&ctr->valid_edges, v);
    if (res) {
      int t = 0;
      for (int w2 = 0; w2 < 8; ++w2) t += s_charge[w2];
      if (t) atomicAdd(ground, -t);  // the ground takes minus the total charge
    }
  }
  __syncthreads();
  if (list && mine) {
    unsigned long long at = s_base + (incl - mine);
    for (unsigned w2 = 0; w2 < warp; ++w2) at += s_wsum[w2];
#pragma unroll
    for (int t = 0; t < kStrip; ++t) {
      const int64_t k = (i0 + r0 + t) * n + (j0 + c);
      if ((hcand >> t) & 1u) {
        if (at < list_cap) list[at] = (uint32_t)k;
        ++at;
      }
      if ((vcand >> t) & 1u) {
        if (at < list_cap) list[at] = (uint32_t)(P + k);
        ++at;
      }
    }
  }
}

template <int SLOPE, int LOOKUP, int W>
__global__ void __launch_bounds__(256) k_costs(const void* __restrict__ ifg, int is_complex,
                                               const float* __restrict__ coh,
                                               const uint8_t* __restrict__ mask, int64_t m, int64_t n,
                                               const int16_t* __restrict__ table, const float* __restrict__ ratio,
                                               int w, float steep_rad, int16_t* __restrict__ costs, SteepCtr* ctr,
                                               uint32_t* list, unsigned long long list_cap, int8_t* res,
                                               int32_t* ground) {
  // one-dimensional grid of tiles (gridDim.y would cap the rows at 65535 tiles)
  const int64_t gx = (n + CTX - 1) / CTX, b = blockIdx.x;
  costs_tile<SLOPE, LOOKUP, W>(ifg, is_complex, coh, mask, m, n, table, ratio, w, steep_rad, costs, ctr, list, list_cap,
                               b % gx, b / gx, res, ground);
}

// the k_costs variant for a parameter set
using CostsKernel = void (*)(const void*, int, const float*, const uint8_t*, int64_t, int64_t, const int16_t*,
                             const float*, int, float, int16_t*, SteepCtr*, uint32_t*, unsigned long long, int8_t*,
                             int32_t*);
// (the default 5 x 5 window has its own instances)
CostsKernel costs_kernel(const ww_params* p) {
  if (p->box_half_width == 2) {
    if (p->slope_estimator == 0) return p->cost_lookup == 0 ? k_costs<0, 0, 2> : k_costs<0, 1, 2>;
    return p->cost_lookup == 0 ? k_costs<1, 0, 2> : k_costs<1, 1, 2>;
  }
  if (p->slope_estimator == 0) return p->cost_lookup == 0 ? k_costs<0, 0, -1> : k_costs<0, 1, -1>;
  return p->cost_lookup == 0 ? k_costs<1, 0, -1> : k_costs<1, 1, -1>;
}

// number of k_costs tiles (one block each) of an m x n image
unsigned cost_tiles(int64_t m, int64_t n) { return (unsigned)(((n + CTX - 1) / CTX) * ((m + CTY - 1) / CTY)); }

// Within the cap (mode 0) with every candidate in the list: zero the listed edges.
__global__ void k_steep_zero_list(const SteepCtr* ctr, const uint32_t* list, unsigned long long list_cap,
                                  int64_t P, int16_t* costs) {
  if (ctr->mode != 0 || ctr->candidates > list_cap) return;
  const unsigned long long nc = ctr->candidates;
  for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < nc;
       q += (unsigned long long)gridDim.x * blockDim.x) {
    const int64_t key = list[q];
    const int plane = key >= P;
    const int64_t k = plane ? key - P : key;
    costs[(2 * plane) * P + k] = 0;
    costs[(2 * plane + 1) * P + k] = 0;
  }
}

// ---- steep-edge bound (Sec. II-B): global selection over candidate edges ----
// Edge key order: h plane (i*n+j) then v plane (m*n + i*n+j).  |d| as fp32 bits
// (monotone for non-negative floats).

__device__ __forceinline__ bool steep_edge(const void* ifg, int is_complex, const float* coh,
                                           const uint8_t* mask, int64_t m, int64_t n, int64_t key,
                                           float steep_rad, uint32_t* bits) {
  const int64_t P = m * n;
  int plane = key >= P;
  int64_t k = plane ? key - P : key;
  int64_t i = k / n, j = k % n;
  if (plane == 0 && j + 1 >= n) return false;
  if (plane == 1 && i + 1 >= m) return false;
  Pix a = load_pixel(ifg, is_complex, coh, mask, k);
  if (!a.valid) return false;
  Pix b = load_pixel(ifg, is_complex, coh, mask, plane ? k + n : k + 1);
  if (!b.valid) return false;
  float d = fabsf(edge_d(a.psi, b.psi));
  if (!(d > steep_rad)) return false;
  *bits = __float_as_uint(d);
  return true;
}

__global__ void k_steep_plan(SteepCtr* ctr, int32_t cap_ppm) {
  // mode 0: zero every candidate (count within the cap); mode 1: select
  unsigned long long cap = (ctr->valid_edges * (unsigned long long)cap_ppm) / 1000000ull;
  ctr->mode = ctr->candidates > cap ? 1ull : 0ull;
  ctr->pad = cap;
}

__global__ void k_steep_hist(const void* ifg, int is_complex, const float* coh, const uint8_t* mask,
                             int64_t m, int64_t n, float steep_rad, const SteepCtr* ctr,
                             uint32_t* hist, int level) {
  if (ctr->mode != 1) return;
  const int64_t E = 2 * m * n;
  for (int64_t key = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; key < E;
       key += (int64_t)gridDim.x * blockDim.x) {
    uint32_t b;
    if (!steep_edge(ifg, is_complex, coh, mask, m, n, key, steep_rad, &b)) continue;
    if (level == 0)
      atomicAdd(&hist[b >> 16], 1u);
    else if ((b >> 16) == (uint32_t)ctr->hi_bin)
      atomicAdd(&hist[b & 0xFFFFu], 1u);
  }
}

// One block of 1024 threads (32 warps) over the 65,536 bins, walked from the top
// bin down.  Warp w owns the contiguous range of 2048 bins
// [65535 - 2048 w - 2047, 65535 - 2048 w]; its lanes read 32 consecutive bins
// per step (coalesced).  The warp totals are scanned from the top to find the
// warp whose range reaches the cap; that warp then walks its range 32 bins at
// a time with a warp scan to find the bin.  Every bin is cleared afterwards
// (coalesced) for the next level or call.
constexpr int kFindThreads = 1024;
constexpr int kFindWarps = kFindThreads / 32, kFindSpan = 65536 / kFindWarps;  // 2048 bins per warp

__global__ void __launch_bounds__(kFindThreads) k_steep_find(SteepCtr* ctr, uint32_t* hist, int level) {
  if (ctr->mode != 1) return;
  __shared__ unsigned long long wsum[kFindWarps];
  __shared__ int s_warp;
  __shared__ unsigned long long s_before;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int top = 65535 - kFindSpan * w;  // highest bin of this warp's range
  unsigned long long s = 0;
  for (int c = 0; c < kFindSpan; c += 32) s += hist[top - c - lane];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) wsum[w] = s;
  __syncthreads();
  const unsigned long long cap = ctr->pad;
  const unsigned long long base = level == 0 ? 0ull : ctr->above;
  if (t == 0) {
    // the first warp range (from the top) where the running count reaches the cap;
    // cap == 0 takes nothing: the cut lies above every bin (walk of warp 0 finds bin 65535)
    unsigned long long acc = base;
    int hit = -1;
    for (int k = 0; k < kFindWarps; ++k) {
      if (acc + wsum[k] >= cap) {
        hit = k;
        break;
      }
      acc += wsum[k];
    }
    s_warp = hit;
    s_before = acc;
  }
  __syncthreads();
  if (w == s_warp) {
    unsigned long long acc = s_before;
    for (int c = 0; c < kFindSpan; c += 32) {
      const int b = top - c - lane;
      const unsigned long long h = hist[b];
      unsigned long long inc = h;  // inclusive scan over the lanes (descending bins)
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
      }
      const unsigned reach = __ballot_sync(0xffffffffu, acc + inc >= cap);
      if (reach) {
        const int first = __ffs(reach) - 1;
        if (lane == first) {
          const unsigned long long before_bin = acc + inc - h;
          if (level == 0) {
            ctr->hi_bin = (unsigned long long)b;
            ctr->above = before_bin;
          } else {
            ctr->threshold = ((unsigned long long)ctr->hi_bin << 16) | (unsigned long long)b;
            ctr->take_at_thr = cap - before_bin;
          }
        }
        break;
      }
      acc += __shfl_sync(0xffffffffu, inc, 31);
    }
  }
  __syncthreads();
  for (int b = t; b < 65536; b += kFindThreads) hist[b] = 0;  // ready for the next level / call
}

// mode 0: zero all candidates; mode 1: zero |d| > threshold, and the first
// take_at_thr ties in key order (ranked with per-block tie counts).
constexpr int kSteepChunk = 1024;  // keys per block in the tie-ranking passes

__global__ void k_steep_ties(const void* ifg, int is_complex, const float* coh, const uint8_t* mask,
                             int64_t m, int64_t n, float steep_rad, const SteepCtr* ctr,
                             uint32_t* blocksum) {
  if (ctr->mode != 1) return;
  const int64_t E = 2 * m * n, chunks = (E + kSteepChunk - 1) / kSteepChunk;
  __shared__ unsigned s[32];
  // a fixed grid walks the chunks (the usual case, within the cap, returns at once)
  for (int64_t chunk = blockIdx.x; chunk < chunks; chunk += gridDim.x) {
    const int64_t base = chunk * kSteepChunk;
    unsigned c = 0;
    for (int64_t key = base + threadIdx.x; key < min(E, base + kSteepChunk); key += blockDim.x) {
      uint32_t b;
      if (steep_edge(ifg, is_complex, coh, mask, m, n, key, steep_rad, &b) && b == (uint32_t)ctr->threshold)
        ++c;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned t = 0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s[k];
      blocksum[chunk] = t;
    }
    __syncthreads();
  }
}

// Exclusive scan of the per-chunk tie counts, one block: each thread scans a
// contiguous slice, then the slice totals are scanned in shared memory.
__global__ void __launch_bounds__(kFindThreads) k_steep_scan(const SteepCtr* ctr, uint32_t* blocksum,
                                                             int64_t nblocks) {
  if (ctr->mode != 1) return;
  __shared__ uint32_t part[kFindThreads];
  const int t = threadIdx.x;
  const int64_t per = (nblocks + kFindThreads - 1) / kFindThreads;
  const int64_t b0 = t * per, b1 = min(nblocks, b0 + per);
  uint32_t s = 0;
  for (int64_t b = b0; b < b1; ++b) s += blocksum[b];
  part[t] = s;
  __syncthreads();
  for (int off = 1; off < kFindThreads; off <<= 1) {
    uint32_t v = t >= off ? part[t - off] : 0u;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  uint32_t acc = t ? part[t - 1] : 0u;
  for (int64_t b = b0; b < b1; ++b) {
    uint32_t v = blocksum[b];
    blocksum[b] = acc;
    acc += v;
  }
}

__global__ void k_steep_zero(const void* ifg, int is_complex, const float* coh, const uint8_t* mask,
                             int64_t m, int64_t n, float steep_rad, const SteepCtr* ctr,
                             const uint32_t* blocksum, int16_t* costs, unsigned long long list_cap) {
  const int64_t E = 2 * m * n, P = m * n;
  const int mode = (int)ctr->mode;
  if (mode == 0 && ctr->candidates <= list_cap) return;  // the candidate list covered it
  const uint32_t thr = (uint32_t)ctr->threshold;
  const unsigned long long take = ctr->take_at_thr;
  __shared__ unsigned warp_ties[32];
  const int64_t chunks = (E + kSteepChunk - 1) / kSteepChunk;
  for (int64_t chunk = blockIdx.x; chunk < chunks; chunk += gridDim.x) {
  const int64_t base = chunk * kSteepChunk;
  unsigned running = mode == 1 ? blocksum[chunk] : 0;
  for (int64_t off = 0; off < kSteepChunk; off += blockDim.x) {
    int64_t key = base + off + threadIdx.x;
    uint32_t b = 0;
    bool cand = key < E && steep_edge(ifg, is_complex, coh, mask, m, n, key, steep_rad, &b);
    bool zero = false, tie = false;
    if (cand) {
      if (mode == 0) zero = true;
      else if (b > thr) zero = true;
      else if (b == thr) tie = true;
    }
    // rank ties in key order inside this block slice
    unsigned bal = __ballot_sync(0xffffffffu, tie);
    unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_ties[wid] = __popc(bal);
    __syncthreads();
    unsigned before = 0, total = 0;
    for (unsigned k = 0; k < (blockDim.x >> 5); ++k) {
      if (k < wid) before += warp_ties[k];
      total += warp_ties[k];
    }
    unsigned rank = running + before + __popc(bal & ((1u << lane) - 1u));
    if (tie && rank < take) zero = true;
    running += total;
    __syncthreads();
    if (zero) {
      int plane = key >= P;
      int64_t k = plane ? key - P : key;
      costs[(2 * plane) * P + k] = 0;
      costs[(2 * plane + 1) * P + k] = 0;
    }
  }
  }
}

// ---------------- integration ----------------
// Column 0 (single block): K(i+1,0) = K(i,0) + dk_v(i,0) - n_v(i,0).
__device__ __forceinline__ void integrate_col0(const void* ifg, int is_complex, const float* coh,
                                               const uint8_t* mask, const int8_t* flows, int64_t m, int64_t n,
                                               int32_t* cycles) {
  __shared__ int32_t carry_s;
  __shared__ int32_t ws[32];
  const int64_t P = m * n;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int64_t base = 0; base < m; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    int32_t inc = 0;  // increment from row i-1 to row i
    if (i >= 1 && i < m) {
      int64_t k = (i - 1) * n;
      float a = load_pixel(ifg, is_complex, coh, mask, k).psi;
      float b = load_pixel(ifg, is_complex, coh, mask, k + n).psi;
      inc = (int32_t)flows[P + k] - wrap_count(__fsub_rn(b, a));
    }
    // inclusive block scan
    int32_t v = inc;
    unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      int32_t t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= (unsigned)o) v += t;
    }
    if (lane == 31) ws[wid] = v;
    __syncthreads();
    int32_t add = 0;
    for (unsigned k = 0; k < wid; ++k) add += ws[k];
    int32_t total = 0;
    for (unsigned k = 0; k < (blockDim.x >> 5); ++k) total += ws[k];
    v += add + carry_s;
    if (i < m) cycles[i * n] = v;
    __syncthreads();
    if (threadIdx.x == 0) carry_s += total;
    __syncthreads();
  }
}

__global__ void k_integrate_col0(const void* ifg, int is_complex, const float* coh, const uint8_t* mask,
                                 const int8_t* flows, int64_t m, int64_t n, int32_t* cycles) {
  integrate_col0(ifg, is_complex, coh, mask, flows, m, n, cycles);
}

// Rows: one block per row; K(i,j+1) = K(i,j) + dk_h(i,j) - n_h(i,j); then
// phi = (float)((double)psi + (double)K * 2pi), NaN where invalid.
constexpr int kRowThreads = 256, kRowItems = 8;

// The output phi = fp32(fp64(psi) + fp64(K) * 2pi_fp64) with its three
// roundings (product, sum, narrowing) reproduced exactly, with one fp64
// addition per pixel: the product and both conversions are integer steps (the
// fp64 pipe of this GPU runs at a small fraction of the integer rate).

// 2pi as an fp64 number: kTwoPiSig * 2^-50 with a 53-bit significand
constexpr uint64_t kTwoPiSig = 0x1921FB54442D18ull;

// Bits of the fp64 product K * 2pi (K != 0), rounded to nearest, ties to even:
// the exact product of |K| < 2^31 and the significand has 53..84 bits and is
// rounded to its top 53.
__device__ __forceinline__ uint64_t k_two_pi_bits(int32_t K) {
  const uint32_t a = K < 0 ? 0u - (uint32_t)K : (uint32_t)K;
  const unsigned __int128 p = (unsigned __int128)a * kTwoPiSig;
  const uint64_t ph = (uint64_t)(p >> 64), pl = (uint64_t)p;
  const int len = ph ? 128 - __clzll((long long)ph) : 64 - __clzll((long long)pl);  // 53..84
  const int sh = len - 53;                                                          // 0..31
  uint64_t sig = (uint64_t)(p >> sh);
  if (sh > 0) {
    const uint64_t rem = pl & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (sig & 1))) ++sig;
  }
  int e = sh;
  if (sig >> 53) {  // rounded up to 2^53
    sig >>= 1;
    ++e;
  }
  // sig 2^(e - 50) with sig in [2^52, 2^53): biased exponent e - 50 + 52 + 1023
  return ((uint64_t)(K < 0) << 63) | ((uint64_t)(e + 1025) << 52) | (sig & ((1ull << 52) - 1));
}

// Bits of the fp64 number equal to a finite fp32 value (subnormals normalised).
__device__ __forceinline__ uint64_t f32_to_f64_bits(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint64_t sign = (uint64_t)(b >> 31) << 63;
  const uint32_t e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
  if (e != 0) return sign | ((uint64_t)(e + 896) << 52) | ((uint64_t)m << 29);
  if (m == 0) return sign;
  const int top = 31 - __clz((int)m);  // m 2^-149 = 1.f 2^(top - 149)
  return sign | ((uint64_t)(top + 874) << 52) | ((uint64_t)((m << (23 - top)) & 0x7FFFFFu) << 29);
}

// The fp32 number nearest (ties to even) an fp64 value that is zero or whose
// fp32 rounding is a normal number (every sum psi + K 2pi with K != 0: it is 0,
// at least 2^-50 in magnitude, or within half an fp32 ulp of a finite psi).
__device__ __forceinline__ float f64_bits_to_f32(uint64_t d) {
  const uint32_t sign = (uint32_t)(d >> 63) << 31;
  const uint32_t e = (uint32_t)(d >> 52) & 0x7FFu;
  if (e == 0) return __uint_as_float(sign);
  const uint64_t m = d & ((1ull << 52) - 1);
  uint32_t r = ((e - 896u) << 23) | (uint32_t)(m >> 29);
  const uint32_t rem = (uint32_t)m & 0x1FFFFFFFu;
  if (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ++r;  // a carry moves into the exponent
  return __uint_as_float(sign | r);
}

// fp32(fp64(psi) + t) for a finite psi, t = the bits of fp64(K) * 2pi (K != 0).
__device__ __forceinline__ float unwrap_value(float psi, uint64_t t) {
  const double s = __dadd_rn(__longlong_as_double((long long)f32_to_f64_bits(psi)), __longlong_as_double((long long)t));
  return f64_bits_to_f32((uint64_t)__double_as_longlong(s));
}

__device__ __forceinline__ void integrate_row(const void* ifg, int is_complex, const float* coh,
                                              const uint8_t* mask, const int8_t* flows, int64_t m, int64_t n,
                                              float* unw, int32_t* cycles, int64_t i) {
  __shared__ int32_t ws[kRowThreads / 32];
  __shared__ float first_psi[kRowThreads];
  __shared__ int32_t carry_s;
  const int64_t row = i * n;
  if (threadIdx.x == 0) carry_s = cycles[row];  // K(i,0) from the column pass
  __syncthreads();
  const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // validity from the phase alone (NaN = invalid) with 8-byte aligned rows: each
  // thread's 8 pixels come as two 128-bit phase loads and one 64-bit flow load
  const bool vec = !is_complex && !coh && !mask && (n & 7) == 0 &&
                   ((reinterpret_cast<uintptr_t>(ifg) | reinterpret_cast<uintptr_t>(flows) |
                     reinterpret_cast<uintptr_t>(unw) | reinterpret_cast<uintptr_t>(cycles)) & 15) == 0;
  for (int64_t seg = 0; seg < n; seg += kRowThreads * kRowItems) {
    int64_t j0 = seg + (int64_t)threadIdx.x * kRowItems;
    float psi[kRowItems];
    bool val[kRowItems];
    int8_t fl[kRowItems];
    if (vec && j0 + kRowItems <= n) {
      const float4* src = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(ifg) + row + j0);
      const float4 a = __ldg(src), b = __ldg(src + 1);
      const float raw[kRowItems] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
      const uint2 f = __ldg(reinterpret_cast<const uint2*>(flows + row + j0));
#pragma unroll
      for (int t = 0; t < kRowItems; ++t) {
        val[t] = isfinite(raw[t]);
        psi[t] = val[t] ? raw[t] : 0.0f;
        fl[t] = (int8_t)(((t < 4 ? f.x : f.y) >> (8 * (t & 3))) & 0xFFu);
      }
    } else {
#pragma unroll
      for (int t = 0; t < kRowItems; ++t) {
        int64_t j = j0 + t;
        Pix p{0.0f, 0.0f, false};
        if (j < n) p = load_pixel(ifg, is_complex, coh, mask, row + j);
        psi[t] = p.psi;
        val[t] = p.valid;
        fl[t] = j < n ? flows[row + j] : (int8_t)0;
      }
    }
    first_psi[threadIdx.x] = psi[0];
    __syncthreads();
    float next_psi;  // pixel j0 + kRowItems
    if (threadIdx.x + 1 < kRowThreads)
      next_psi = first_psi[threadIdx.x + 1];
    else {
      int64_t j = j0 + kRowItems;
      next_psi = j < n ? load_pixel(ifg, is_complex, coh, mask, row + j).psi : 0.0f;
    }
    // increments inc[t] = K(j0+t+1) - K(j0+t)
    int32_t local[kRowItems];
    int32_t s = 0;
#pragma unroll
    for (int t = 0; t < kRowItems; ++t) {
      int64_t j = j0 + t;
      int32_t inc = 0;
      if (j + 1 < n) {
        float b = t + 1 < kRowItems ? psi[t + 1] : next_psi;
        inc = (int32_t)fl[t] - wrap_count(__fsub_rn(b, psi[t]));
      }
      local[t] = s;  // exclusive prefix within this thread
      s += inc;
    }
    // block exclusive scan of per-thread sums
    int32_t v = s;
    for (int o = 1; o < 32; o <<= 1) {
      int32_t t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= (unsigned)o) v += t;
    }
    if (lane == 31) ws[wid] = v;
    __syncthreads();
    int32_t add = 0, total = 0;
    for (unsigned k = 0; k < kRowThreads / 32; ++k) {
      if (k < wid) add += ws[k];
      total += ws[k];
    }
    int32_t base = carry_s + add + (v - s);
    int32_t Ks[kRowItems];
    float outs[kRowItems];
    // the product K 2pi once per run of equal K (neighbours mostly share it)
    int32_t lastK = 0;
    uint64_t tK = 0;
#pragma unroll
    for (int t = 0; t < kRowItems; ++t) {
      const int32_t K = base + local[t];
      Ks[t] = K;
      if (!val[t]) {
        outs[t] = __int_as_float(0x7fc00000);
      } else if (K == 0) {
        outs[t] = psi[t] == 0.0f ? 0.0f : psi[t];  // psi + (+0): -0 becomes +0, the rest is exact
      } else {
        if (K != lastK) {
          lastK = K;
          tK = k_two_pi_bits(K);
        }
        outs[t] = unwrap_value(psi[t], tK);
      }
    }
    if (vec && j0 + kRowItems <= n) {
      int4* kc = reinterpret_cast<int4*>(cycles + row + j0);
      float4* uo = reinterpret_cast<float4*>(unw + row + j0);
      kc[0] = make_int4(Ks[0], Ks[1], Ks[2], Ks[3]);
      kc[1] = make_int4(Ks[4], Ks[5], Ks[6], Ks[7]);
      uo[0] = make_float4(outs[0], outs[1], outs[2], outs[3]);
      uo[1] = make_float4(outs[4], outs[5], outs[6], outs[7]);
    } else {
#pragma unroll
      for (int t = 0; t < kRowItems; ++t) {
        const int64_t j = j0 + t;
        if (j >= n) break;
        cycles[row + j] = Ks[t];
        unw[row + j] = outs[t];
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) carry_s += total;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kRowThreads) k_integrate_rows(const void* ifg, int is_complex,
                                                                const float* coh, const uint8_t* mask,
                                                                const int8_t* flows, int64_t m, int64_t n,
                                                                float* unw, int32_t* cycles) {
  if ((int64_t)blockIdx.x >= m) return;
  integrate_row(ifg, is_complex, coh, mask, flows, m, n, unw, cycles, blockIdx.x);
}

// ---------------- batched launches ----------------
// One launch covers every item of a batch: the items' blocks are numbered
// consecutively (GridItem::blk[kind]) and each block finds its item by a
// binary search over those offsets, then runs the same per-tile code as the
// single-image kernels.

template <int KIND>
__device__ __forceinline__ int item_of_block(const GridItem* it, int count, int64_t b) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (it[mid].blk[KIND] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

constexpr int kPhasePerBlock = 256 * 8;

__global__ void k_phase_b(const GridItem* __restrict__ items, int count) {
  const int64_t b = blockIdx.x;
  const GridItem& it = items[item_of_block<kBlkPhase>(items, count, b)];
  const int64_t P = it.m * it.n;
  const int64_t base = (b - it.blk[kBlkPhase]) * kPhasePerBlock;
  const float2* z = reinterpret_cast<const float2*>(it.phase_src);
  float* psi = const_cast<float*>(reinterpret_cast<const float*>(it.ifg));
  for (int64_t k = base + threadIdx.x; k < min(P, base + kPhasePerBlock); k += blockDim.x) {
    const float2 v = __ldg(z + k);
    psi[k] = (isfinite(v.x) && isfinite(v.y)) ? cordic_phase(v.x, v.y) : __int_as_float(0x7fc00000);
  }
}

__global__ void __launch_bounds__(RTX* RTT) k_residues_b(const GridItem* __restrict__ items, int count) {
  const int64_t b = blockIdx.x;
  const GridItem& it = items[item_of_block<kBlkRes>(items, count, b)];
  const int64_t local = b - it.blk[kBlkRes];
  const int64_t gx = (it.n - 1 + RTX - 1) / RTX;
  residues_tile(it.ifg, it.is_complex, it.coh, it.mask, it.m, it.n, it.res, it.ground, local % gx, local / gx);
}

template <int SLOPE, int LOOKUP>
__global__ void __launch_bounds__(256) k_costs_b(const GridItem* __restrict__ items, int count, int w,
                                                 float steep_rad) {
  const int64_t b = blockIdx.x;
  const GridItem& it = items[item_of_block<kBlkCost>(items, count, b)];
  const int64_t local = b - it.blk[kBlkCost];
  const int64_t gx = (it.n + CTX - 1) / CTX;
  costs_tile<SLOPE, LOOKUP, -1>(it.ifg, it.is_complex, it.coh, it.mask, it.m, it.n, it.table, it.ratio, w, steep_rad,
             it.costs,
             reinterpret_cast<SteepCtr*>(it.steep), it.cand_list, (unsigned long long)it.cand_cap, local % gx,
             local / gx);
}

// Cap test of every item (one thread per item); mode 1 marks the items that
// need the selection.
__global__ void k_steep_plan_b(GridItem* items, int count, int32_t cap_ppm) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
    SteepCtr* ctr = reinterpret_cast<SteepCtr*>(items[k].steep);
    unsigned long long cap = (ctr->valid_edges * (unsigned long long)cap_ppm) / 1000000ull;
    // 0: zero every candidate; 1: select the cap largest; 3: cap 0, zero nothing
    ctr->mode = ctr->candidates <= cap ? 0ull : (cap == 0 ? 3ull : 1ull);
    ctr->pad = cap;
    ctr->above = 0;
    ctr->hi_bin = 0;
  }
}

// ---- batched exact selection for items over their cap ----
// Radix select of the cap-th largest |d| among an item's steep candidates.
// Keys are key = bits(|d|) - bits(steep_rad) (fp32 bits are monotone for
// values >= 0, and every candidate has |d| > steep_rad), so they span only
// the range up to bits(PI_F) - bits(steep_rad): three digits of at most 11
// bits each (shifts and widths from the host, SelDigits) cover it.  Each level
// histograms the candidates whose higher digits equal the prefix found so far
// (warp-aggregated shared-memory histogram per block, flushed with one atomic
// per non-empty bin into the item's 2048 global bins); then one block per item
// walks its bins from the top.
constexpr int kSelBins = 2048;
constexpr int kSelChunk = 16384;  // keys per block of the histogram passes

struct SelDigits {
  uint32_t base;     // bits(steep_rad), 0 when steep_rad <= 0
  int shift[3], width[3];
};

__global__ void __launch_bounds__(256) k_sel_hist_b(const GridItem* __restrict__ items, int count, float steep_rad,
                                                    uint32_t* hist_all, SelDigits dg, int level) {
  __shared__ uint32_t h[kSelBins];
  const int64_t b = blockIdx.x;
  const int k = item_of_block<kBlkSel>(items, count, b);
  const GridItem& it = items[k];
  const SteepCtr* ctr = reinterpret_cast<const SteepCtr*>(it.steep);
  if (ctr->mode != 1) return;
  for (int q = threadIdx.x; q < kSelBins; q += blockDim.x) h[q] = 0;
  __syncthreads();
  const int sh = dg.shift[level];
  const uint32_t dmask = (1u << dg.width[level]) - 1u;
  const int psh = level > 0 ? dg.shift[level - 1] : 0;
  const uint32_t prefix = (uint32_t)ctr->hi_bin;
  const int64_t E = 2 * it.m * it.n;
  const int64_t base = (b - it.blk[kBlkSel]) * kSelChunk;
  const int64_t end = min(E, base + kSelChunk);
  const unsigned lane = threadIdx.x & 31;
  for (int64_t k0 = base; k0 < end; k0 += blockDim.x) {  // same trip count for every thread
    const int64_t key = k0 + threadIdx.x;
    int bin = -1;
    uint32_t bits;
    if (key < end && steep_edge(it.ifg, it.is_complex, it.coh, it.mask, it.m, it.n, key, steep_rad, &bits)) {
      const uint32_t kk = bits - dg.base;
      if (level == 0 || (kk >> psh) == prefix) bin = (int)((kk >> sh) & dmask);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, bin);
    if (bin >= 0 && lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(&h[bin], (uint32_t)__popc(peers));
  }
  __syncthreads();
  uint32_t* g = hist_all + (int64_t)k * kSelBins;
  for (int q = threadIdx.x; q < kSelBins; q += blockDim.x)
    if (h[q]) atomicAdd(&g[q], h[q]);
}

// One block (256 threads, 8 bins each) per item: the bin holding the
// (cap - above)-th largest candidate of this level; bins are cleared after.
__global__ void __launch_bounds__(256) k_sel_find_b(const GridItem* __restrict__ items, uint32_t* hist_all,
                                                    SelDigits dg, int level) {
  const GridItem& it = items[blockIdx.x];
  SteepCtr* ctr = reinterpret_cast<SteepCtr*>(it.steep);
  if (ctr->mode != 1) return;
  __shared__ unsigned long long part[256];
  uint32_t* g = hist_all + (int64_t)blockIdx.x * kSelBins;
  const int t = threadIdx.x;
  // read before the barriers below: one thread rewrites the counters afterwards
  const unsigned long long need = ctr->pad - ctr->above;  // >= 1 while selecting
  const uint64_t prefix_in = ctr->hi_bin;
  const int hi = kSelBins - 1 - 8 * t;  // this thread's bins hi, hi-1, ..., hi-7 (from the top)
  unsigned long long sum = 0;
  for (int q = 0; q < 8; ++q) sum += g[hi - q];
  part[t] = sum;
  __syncthreads();
  for (int off = 1; off < 256; off <<= 1) {
    unsigned long long v = t >= off ? part[t - off] : 0ull;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  const unsigned long long before = t ? part[t - 1] : 0ull;
  if (before < need && part[t] >= need) {
    unsigned long long acc = before;
    for (int q = 0; q < 8; ++q) {
      const int bin = hi - q;
      const unsigned long long c = g[bin];
      if (acc + c >= need) {
        const uint64_t prefix = level == 0 ? (uint64_t)bin : ((prefix_in << dg.width[level]) | (uint64_t)bin);
        ctr->hi_bin = prefix;
        ctr->above = (ctr->pad - need) + acc;
        if (level == 2) {
          ctr->threshold = prefix + dg.base;  // exact |d| bits of the cut
          ctr->take_at_thr = need - acc;      // candidates equal to it to zero, in key order
        }
        break;
      }
      acc += c;
    }
  }
  __syncthreads();
  for (int q = 0; q < 8; ++q) g[hi - q] = 0;
}

// Ties at the cut: count per 1024-key chunk (blocksum indexed by the global
// steep block number).
__global__ void k_sel_ties_b(const GridItem* __restrict__ items, int count, float steep_rad, uint32_t* blocksum) {
  const int64_t b = blockIdx.x;
  const GridItem& it = items[item_of_block<kBlkSteep>(items, count, b)];
  const SteepCtr* ctr = reinterpret_cast<const SteepCtr*>(it.steep);
  if (ctr->mode != 1) return;
  const int64_t E = 2 * it.m * it.n;
  const int64_t base = (b - it.blk[kBlkSteep]) * kSteepChunk;
  const uint32_t thr = (uint32_t)ctr->threshold;
  unsigned c = 0;
  for (int64_t key = base + threadIdx.x; key < min(E, base + kSteepChunk); key += blockDim.x) {
    uint32_t bits;
    if (steep_edge(it.ifg, it.is_complex, it.coh, it.mask, it.m, it.n, key, steep_rad, &bits) && bits == thr) ++c;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  __shared__ unsigned sm[32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned tot = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += sm[q];
    blocksum[b] = tot;
  }
}

// Exclusive scan of one item's chunk tie counts (one block per item).
__global__ void __launch_bounds__(kFindThreads) k_sel_scan_b(const GridItem* __restrict__ items, uint32_t* blocksum) {
  const GridItem& it = items[blockIdx.x];
  const SteepCtr* ctr = reinterpret_cast<const SteepCtr*>(it.steep);
  if (ctr->mode != 1) return;
  const int64_t nblocks = (2 * it.m * it.n + kSteepChunk - 1) / kSteepChunk;
  uint32_t* bs = blocksum + it.blk[kBlkSteep];
  __shared__ uint32_t part[kFindThreads];
  const int t = threadIdx.x;
  const int64_t per = (nblocks + kFindThreads - 1) / kFindThreads;
  const int64_t b0 = t * per, b1 = min(nblocks, b0 + per);
  uint32_t sum = 0;
  for (int64_t q = b0; q < b1; ++q) sum += bs[q];
  part[t] = sum;
  __syncthreads();
  for (int off = 1; off < kFindThreads; off <<= 1) {
    uint32_t v = t >= off ? part[t - off] : 0u;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  uint32_t acc = t ? part[t - 1] : 0u;
  for (int64_t q = b0; q < b1; ++q) {
    uint32_t v = bs[q];
    bs[q] = acc;
    acc += v;
  }
}

// Zero the selected edges: |d| above the cut, and the first take_at_thr ties
// in key order (rank = ties in earlier chunks + ties earlier in this chunk).
__global__ void k_sel_zero_b(const GridItem* __restrict__ items, int count, float steep_rad,
                             const uint32_t* blocksum) {
  const int64_t b = blockIdx.x;
  const GridItem& it = items[item_of_block<kBlkSteep>(items, count, b)];
  const SteepCtr* ctr = reinterpret_cast<const SteepCtr*>(it.steep);
  if (ctr->mode != 1) return;
  const int64_t P = it.m * it.n, E = 2 * P;
  const int64_t base = (b - it.blk[kBlkSteep]) * kSteepChunk;
  const uint32_t thr = (uint32_t)ctr->threshold;
  const unsigned long long take = ctr->take_at_thr;
  __shared__ unsigned warp_ties[32];
  unsigned running = blocksum[b];
  for (int64_t off = 0; off < kSteepChunk; off += blockDim.x) {
    const int64_t key = base + off + threadIdx.x;
    uint32_t bits = 0;
    const bool cand = key < E && steep_edge(it.ifg, it.is_complex, it.coh, it.mask, it.m, it.n, key, steep_rad, &bits);
    bool zero = cand && bits > thr;
    const bool tie = cand && bits == thr;
    const unsigned bal = __ballot_sync(0xffffffffu, tie);
    const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_ties[wid] = __popc(bal);
    __syncthreads();
    unsigned before = 0, total = 0;
    for (unsigned q = 0; q < (blockDim.x >> 5); ++q) {
      if (q < wid) before += warp_ties[q];
      total += warp_ties[q];
    }
    const unsigned rank = running + before + __popc(bal & ((1u << lane) - 1u));
    if (tie && rank < take) zero = true;
    running += total;
    __syncthreads();
    if (zero) {
      const int plane = key >= P;
      const int64_t k = plane ? key - P : key;
      it.costs[(2 * plane) * P + k] = 0;
      it.costs[(2 * plane + 1) * P + k] = 0;
    }
  }
}

// Items within their cap: every steep candidate costs 0 in both directions.
// Grid: x strides over an item's candidate list, y over the items.
__global__ void k_steep_zero_list_b(const GridItem* __restrict__ items) {
  const GridItem& it = items[blockIdx.y];
  const SteepCtr* ctr = reinterpret_cast<const SteepCtr*>(it.steep);
  if (ctr->mode != 0 || !it.cand_list || ctr->candidates > (unsigned long long)it.cand_cap) return;
  const unsigned long long nc = ctr->candidates;
  const int64_t P = it.m * it.n;
  for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < nc;
       q += (unsigned long long)gridDim.x * blockDim.x) {
    const int64_t key = it.cand_list[q];
    const int plane = key >= P;
    const int64_t k = plane ? key - P : key;
    it.costs[(2 * plane) * P + k] = 0;
    it.costs[(2 * plane + 1) * P + k] = 0;
  }
}

// The same for items without a complete list: a pass over every edge.
// Items with no candidate, or over the cap (selected separately), are skipped.
__global__ void k_steep_zero_all_b(const GridItem* __restrict__ items, int count, float steep_rad) {
  const int64_t b = blockIdx.x;
  const GridItem& it = items[item_of_block<kBlkSteep>(items, count, b)];
  const SteepCtr* ctr = reinterpret_cast<const SteepCtr*>(it.steep);
  if (ctr->mode != 0 || ctr->candidates == 0) return;
  if (it.cand_list && ctr->candidates <= (unsigned long long)it.cand_cap) return;  // listed
  const int64_t P = it.m * it.n, E = 2 * P;
  const int64_t base = (b - it.blk[kBlkSteep]) * kSteepChunk;
  for (int64_t key = base + threadIdx.x; key < min(E, base + kSteepChunk); key += blockDim.x) {
    uint32_t bits;
    if (!steep_edge(it.ifg, it.is_complex, it.coh, it.mask, it.m, it.n, key, steep_rad, &bits)) continue;
    const int plane = key >= P;
    const int64_t k = plane ? key - P : key;
    it.costs[(2 * plane) * P + k] = 0;
    it.costs[(2 * plane + 1) * P + k] = 0;
  }
}

__global__ void __launch_bounds__(1024) k_integrate_col0_b(const GridItem* __restrict__ items) {
  const GridItem& it = items[blockIdx.x];
  integrate_col0(it.ifg, it.is_complex, it.coh, it.mask, it.flows, it.m, it.n, it.cyc);
}

__global__ void __launch_bounds__(kRowThreads) k_integrate_rows_b(const GridItem* __restrict__ items, int count) {
  const int64_t b = blockIdx.x;
  const GridItem& it = items[item_of_block<kBlkRow>(items, count, b)];
  integrate_row(it.ifg, it.is_complex, it.coh, it.mask, it.flows, it.m, it.n, it.unw, it.cyc,
                b - it.blk[kBlkRow]);
}

}  // namespace

ww_status launch_residues(const void* ifg, int is_complex, const float* coh, const uint8_t* mask,
                          int64_t m, int64_t n, int8_t* res, int32_t* ground, cudaStream_t s) {
  WW_CUDA_TRY(cudaMemsetAsync(ground, 0, sizeof(int32_t), s));
  const int64_t tiles = ((n - 1 + RTX - 1) / RTX) * ((m - 1 + RTY - 1) / RTY);
  k_residues<<<(unsigned)tiles, dim3(RTX, RTT), 0, s>>>(ifg, is_complex, coh, mask, m, n, res, ground);
  WW_CUDA_TRY(cudaGetLastError());
  return WW_OK;
}

namespace {
// Wrapped phase of a complex interferogram, once per pixel (fixed-point CORDIC); a
// non-finite sample gives NaN, which the float-input kernels treat as invalid
// exactly as the complex-input kernels treat the non-finite sample.
// With coh/mask given, every validity test of a pixel (mask, finite coherence,
// finite sample) is folded into the phase as NaN, so the later steps can read
// the phase alone for validity.
__global__ void k_phase(const float2* __restrict__ z, const float* __restrict__ coh, const uint8_t* __restrict__ mask,
                        int64_t P, float* __restrict__ psi) {
  // grid-stride loop with the next pixel's loads issued before this pixel's CORDIC
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  float2 v = make_float2(0.0f, 0.0f);
  float cv = 0.0f;
  uint8_t mv = 1;
  if (k < P) {
    v = __ldg(z + k);
    if (coh) cv = __ldg(coh + k);
    if (mask) mv = __ldg(mask + k);
  }
  for (; k < P; k += stride) {
    const int64_t kn = k + stride;
    float2 vn = make_float2(0.0f, 0.0f);
    float cn = 0.0f;
    uint8_t mn = 1;
    if (kn < P) {
      vn = __ldg(z + kn);
      if (coh) cn = __ldg(coh + kn);
      if (mask) mn = __ldg(mask + kn);
    }
    const bool ok = isfinite(v.x) && isfinite(v.y) && isfinite(cv) && mv != 0;
    psi[k] = ok ? cordic_phase(v.x, v.y) : __int_as_float(0x7fc00000);
    v = vn;
    cv = cn;
    mv = mn;
  }
}
}  // namespace

ww_status launch_phase(const void* ifg, const float* coh, const uint8_t* mask, int64_t m, int64_t n, float* psi,
                       cudaStream_t s) {
  const int64_t P = m * n;
  int blocks = (int)std::min<int64_t>((P + 255) / 256, 148 * 16);
  k_phase<<<blocks, 256, 0, s>>>(reinterpret_cast<const float2*>(ifg), coh, mask, P, psi);
  WW_CUDA_TRY(cudaGetLastError());
  return WW_OK;
}

int64_t steep_list_capacity(int64_t pixels, int32_t cap_ppm) {
  return (2 * pixels) / 1000000 * cap_ppm + ((2 * pixels) % 1000000) * cap_ppm / 1000000 + 2;
}

ww_status launch_costs(const void* ifg, int is_complex, const float* coh, const uint8_t* mask,
                       int64_t m, int64_t n, const int16_t* dtable, const float* dratio, const ww_params* p,
                       ww_workspace* ws, int16_t* costs, cudaStream_t s, int8_t* res, int32_t* ground) {
  if (p->cost_lookup == 1 && !dratio) return WW_ERR_INVALID_ARG;
  SteepCtr* ctr = reinterpret_cast<SteepCtr*>(ws->steep_ctr);
  WW_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(SteepCtr), s));
  // candidate list: within the cap every candidate fits (cap + 1 <= capacity), so the
  // common case zeroes the listed edges instead of scanning every edge again
  const int64_t need = steep_list_capacity(m * n, p->steep_cap_ppm);
  const bool use_list = ws->steep_list && need <= ws->steep_list_cap && 2 * m * n < (1ll << 32);
  uint32_t* list = use_list ? ws->steep_list : nullptr;
  const unsigned long long list_cap = use_list ? (unsigned long long)ws->steep_list_cap : 0ull;
  costs_kernel(p)<<<cost_tiles(m, n), 256, 0, s>>>(ifg, is_complex, coh, mask, m, n, dtable, dratio,
                                                   p->box_half_width, p->steep_rad, costs, ctr, list, list_cap, res,
                                                   ground);
  WW_CUDA_TRY(cudaGetLastError());
  k_steep_plan<<<1, 1, 0, s>>>(ctr, p->steep_cap_ppm);
  if (use_list) k_steep_zero_list<<<148 * 4, 256, 0, s>>>(ctr, list, list_cap, m * n, costs);
  const int64_t E = 2 * m * n;
  int hist_blocks = 148 * 8;
  k_steep_hist<<<hist_blocks, 256, 0, s>>>(ifg, is_complex, coh, mask, m, n, p->steep_rad, ctr, ws->hist, 0);
  k_steep_find<<<1, kFindThreads, 0, s>>>(ctr, ws->hist, 0);
  k_steep_hist<<<hist_blocks, 256, 0, s>>>(ifg, is_complex, coh, mask, m, n, p->steep_rad, ctr, ws->hist, 1);
  k_steep_find<<<1, kFindThreads, 0, s>>>(ctr, ws->hist, 1);
  int64_t nb = (E + kSteepChunk - 1) / kSteepChunk;
  const unsigned nb_grid = (unsigned)std::min<int64_t>(nb, 148 * 16);
  k_steep_ties<<<nb_grid, 256, 0, s>>>(ifg, is_complex, coh, mask, m, n, p->steep_rad, ctr, ws->blocksum);
  k_steep_scan<<<1, kFindThreads, 0, s>>>(ctr, ws->blocksum, nb);
  k_steep_zero<<<nb_grid, 256, 0, s>>>(ifg, is_complex, coh, mask, m, n, p->steep_rad, ctr, ws->blocksum,
                                            costs, list_cap);
  WW_CUDA_TRY(cudaGetLastError());
  return WW_OK;
}

int64_t grid_batch_bytes(int cap, int64_t max_pixels) {
  return (int64_t)cap * ((int64_t)sizeof(GridItem) + (int64_t)sizeof(SteepCtr) + kSelBins * 4) +
         (2 * max_pixels / kSteepChunk + cap + 1) * 4 + (steep_list_capacity(max_pixels, 30000) + 2 * cap) * 4;
}

ww_status grid_batch_alloc(GridBatch* gb, int cap, int64_t max_pixels) {
  *gb = GridBatch{};
  gb->cap = cap;
  gb->blocksum_len = 2 * max_pixels / kSteepChunk + cap + 1;  // >= sum of ceil(2 m n / chunk)
  if (cudaMalloc(&gb->d_items, cap * sizeof(GridItem)) != cudaSuccess ||
      cudaMallocHost(&gb->h_items, cap * sizeof(GridItem)) != cudaSuccess ||
      cudaMalloc(&gb->d_steep, cap * sizeof(SteepCtr)) != cudaSuccess ||
      cudaMalloc(&gb->hist, (int64_t)cap * kSelBins * 4) != cudaSuccess ||
      cudaMalloc(&gb->blocksum, gb->blocksum_len * 4) != cudaSuccess)
    return WW_ERR_OOM;
  // candidate lists for the default 3% cap: sum over items of (cap_k + 2) <= this
  gb->list_pool_cap = steep_list_capacity(max_pixels, 30000) + 2 * (int64_t)cap;
  if (cudaMalloc(&gb->list_pool, gb->list_pool_cap * 4) != cudaSuccess) return WW_ERR_OOM;
  // the find pass clears the bins it used, so they stay zero between calls
  if (cudaMemset(gb->hist, 0, (int64_t)cap * kSelBins * 4) != cudaSuccess) return WW_ERR_CUDA;
  return WW_OK;
}

void grid_batch_free(GridBatch* gb) {
  cudaFree(gb->d_items);
  cudaFreeHost(gb->h_items);
  cudaFree(gb->d_steep);
  cudaFree(gb->hist);
  cudaFree(gb->blocksum);
  cudaFree(gb->list_pool);
  *gb = GridBatch{};
}

namespace {
__global__ void k_prep_b(GridItem* items, int count) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
    *items[k].ground = 0;
    *reinterpret_cast<SteepCtr*>(items[k].steep) = SteepCtr{};
  }
}
}  // namespace

namespace {
uint32_t float_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}
}  // namespace

ww_status launch_pre_batch(GridBatch* gb, int count, const ww_params* p, cudaStream_t s) {
  if (count < 1 || count > gb->cap || count > 65535) return WW_ERR_INVALID_ARG;
  GridItem* h = gb->h_items;
  int64_t off[kBlkKinds] = {};
  int64_t list_off = 0;
  for (int k = 0; k < count; ++k) {
    GridItem& it = h[k];
    it.steep = reinterpret_cast<SteepCtr*>(gb->d_steep) + k;
    const int64_t need = steep_list_capacity(it.m * it.n, p->steep_cap_ppm);
    if (list_off + need <= gb->list_pool_cap && 2 * it.m * it.n < (1ll << 32)) {
      it.cand_list = gb->list_pool + list_off;
      it.cand_cap = need;
      list_off += need;
    } else {
      it.cand_list = nullptr;
      it.cand_cap = 0;
    }
    for (int q = 0; q < kBlkKinds; ++q) it.blk[q] = off[q];
    const int64_t E = 2 * it.m * it.n;
    off[kBlkRes] += ((it.n - 1 + RTX - 1) / RTX) * ((it.m - 1 + RTY - 1) / RTY);
    off[kBlkCost] += ((it.n + CTX - 1) / CTX) * ((it.m + CTY - 1) / CTY);
    off[kBlkSteep] += (E + kSteepChunk - 1) / kSteepChunk;
    off[kBlkRow] += it.m;
    off[kBlkSel] += (E + kSelChunk - 1) / kSelChunk;
    it.blk[kBlkPhase] = off[kBlkPhase];
    if (it.phase_src) {
      if (it.is_complex) return WW_ERR_INVALID_ARG;  // ifg must be the float phase buffer
      off[kBlkPhase] += (it.m * it.n + kPhasePerBlock - 1) / kPhasePerBlock;
    }
  }
  for (int64_t o : off)
    if (o >= (1ll << 31)) return WW_ERR_INVALID_ARG;
  if (off[kBlkSteep] > gb->blocksum_len) return WW_ERR_INVALID_ARG;
  WW_CUDA_TRY(cudaMemcpyAsync(gb->d_items, h, count * sizeof(GridItem), cudaMemcpyHostToDevice, s));
  const int pb = (count + 255) / 256;
  // phase of the complex items once (their ifg is the float buffer it lands in)
  if (off[kBlkPhase] > 0) k_phase_b<<<(unsigned)off[kBlkPhase], 256, 0, s>>>(gb->d_items, count);
  k_prep_b<<<pb, 256, 0, s>>>(gb->d_items, count);
  k_residues_b<<<(unsigned)off[kBlkRes], dim3(RTX, RTT), 0, s>>>(gb->d_items, count);
  auto kb = p->slope_estimator == 0 ? (p->cost_lookup == 0 ? k_costs_b<0, 0> : k_costs_b<0, 1>)
                                     : (p->cost_lookup == 0 ? k_costs_b<1, 0> : k_costs_b<1, 1>);
  kb<<<(unsigned)off[kBlkCost], 256, 0, s>>>(gb->d_items, count, p->box_half_width, p->steep_rad);
  k_steep_plan_b<<<pb, 256, 0, s>>>(gb->d_items, count, p->steep_cap_ppm);
  // items within their cap
  k_steep_zero_list_b<<<dim3(4, (unsigned)count), 256, 0, s>>>(gb->d_items);
  k_steep_zero_all_b<<<(unsigned)off[kBlkSteep], 256, 0, s>>>(gb->d_items, count, p->steep_rad);
  // items over their cap: exact selection, all items at once
  SelDigits dg;
  dg.base = p->steep_rad > 0.0f ? float_bits(p->steep_rad) : 0u;
  {
    const uint32_t span = 0x40490FDBu - std::min(dg.base, 0x40490FDBu);  // largest key: |d| = PI_F
    int nb = 1;
    while (nb < 32 && (span >> nb) != 0) ++nb;
    dg.shift[0] = std::max(0, nb - 11);
    dg.shift[1] = std::max(0, dg.shift[0] - 11);
    dg.shift[2] = 0;
    dg.width[0] = nb - dg.shift[0];
    dg.width[1] = dg.shift[0] - dg.shift[1];
    dg.width[2] = dg.shift[1];
  }
  for (int level = 0; level < 3; ++level) {
    k_sel_hist_b<<<(unsigned)off[kBlkSel], 256, 0, s>>>(gb->d_items, count, p->steep_rad, gb->hist, dg, level);
    k_sel_find_b<<<count, 256, 0, s>>>(gb->d_items, gb->hist, dg, level);
  }
  k_sel_ties_b<<<(unsigned)off[kBlkSteep], 256, 0, s>>>(gb->d_items, count, p->steep_rad, gb->blocksum);
  k_sel_scan_b<<<count, kFindThreads, 0, s>>>(gb->d_items, gb->blocksum);
  k_sel_zero_b<<<(unsigned)off[kBlkSteep], 256, 0, s>>>(gb->d_items, count, p->steep_rad, gb->blocksum);
  WW_CUDA_TRY(cudaGetLastError());
  return WW_OK;
}

ww_status launch_integrate_batch(GridBatch* gb, int count, cudaStream_t s) {
  if (count < 1 || count > gb->cap) return WW_ERR_INVALID_ARG;
  GridItem* h = gb->h_items;
  int64_t rows = 0;
  for (int k = 0; k < count; ++k) {
    h[k].blk[kBlkRow] = rows;
    rows += h[k].m;
  }
  if (rows >= (1ll << 31)) return WW_ERR_INVALID_ARG;
  WW_CUDA_TRY(cudaMemcpyAsync(gb->d_items, h, count * sizeof(GridItem), cudaMemcpyHostToDevice, s));
  k_integrate_col0_b<<<count, 1024, 0, s>>>(gb->d_items);
  k_integrate_rows_b<<<(unsigned)rows, kRowThreads, 0, s>>>(gb->d_items, count);
  WW_CUDA_TRY(cudaGetLastError());
  return WW_OK;
}

ww_status launch_integrate(const void* ifg, int is_complex, const float* coh, const uint8_t* mask,
                           const int8_t* flows, int64_t m, int64_t n, float* unw, int32_t* cyc,
                           cudaStream_t s) {
  k_integrate_col0<<<1, 1024, 0, s>>>(ifg, is_complex, coh, mask, flows, m, n, cyc);
  k_integrate_rows<<<(unsigned)m, kRowThreads, 0, s>>>(ifg, is_complex, coh, mask, flows, m, n, unw, cyc);
  WW_CUDA_TRY(cudaGetLastError());
  return WW_OK;
}

}  // namespace ww

// ---------------- cost step without any device allocation ----------------
// For callers that cannot call cudaMalloc: for example code whose device memory
// is owned by another allocator (a framework's caching pool) or a real-time
// loop that must not pay cudaMalloc's implicit device synchronisation.  The
// steep-edge selection scratch and the cost table live in one file-scope
// device array instead of a workspace; every GPU that loads this library holds
// it (about 1.4 MB) until the process exits.
namespace ww {
namespace {

constexpr int64_t kNoAllocMaxPixels = 1ll << 27;  // m*n limit of ww_costs_noalloc
constexpr int64_t kNoAllocChunks = (2 * kNoAllocMaxPixels + kSteepChunk - 1) / kSteepChunk;
constexpr size_t kNoAllocTableBytes = sizeof(int16_t) * kNGamma * kNAlpha;  // 64 KiB
constexpr size_t kNoAllocHistOff = kNoAllocTableBytes;
constexpr size_t kNoAllocCtrOff = kNoAllocHistOff + 65536 * sizeof(uint32_t);
constexpr size_t kNoAllocBlocksumOff = kNoAllocCtrOff + 256;
constexpr size_t kNoAllocBytes = kNoAllocBlocksumOff + kNoAllocChunks * sizeof(uint32_t);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch, looked up once per device (the host-side
// name is only a stand-in and must never be passed to a kernel).
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[64] = {nullptr};

ww_status noalloc_scratch(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return WW_ERR_CUDA;
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return WW_ERR_CUDA;
    g_noalloc_ptr[dev] = static_cast<unsigned char*>(ptr);
  }
  *out = g_noalloc_ptr[dev];
  return WW_OK;
}

}  // namespace
}  // namespace ww

extern "C" ww_status ww_costs_noalloc(const void* ifg, int32_t is_complex, const float* coh, const uint8_t* mask,
                                      int64_t m, int64_t n, const ww_lut* lut, const ww_params* params,
                                      int16_t* costs, ww_stream stream) {
  using namespace ww;
  ww_params def;
  ww_params_default(&def);
  const ww_params* p = params ? params : &def;
  if (!ifg || !coh || !lut || !costs || m < 2 || n < 2) return WW_ERR_INVALID_ARG;
  if (m > kNoAllocMaxPixels || n > kNoAllocMaxPixels || m * n > kNoAllocMaxPixels) return WW_ERR_INVALID_ARG;
  if (!params_valid(p) || p->slope_estimator != 0 || p->cost_lookup != 0) return WW_ERR_INVALID_ARG;
  unsigned char* base = nullptr;
  ww_status st = noalloc_scratch(&base);
  if (st != WW_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  int16_t* dtable = reinterpret_cast<int16_t*>(base);
  uint32_t* hist = reinterpret_cast<uint32_t*>(base + kNoAllocHistOff);
  SteepCtr* ctr = reinterpret_cast<SteepCtr*>(base + kNoAllocCtrOff);
  uint32_t* blocksum = reinterpret_cast<uint32_t*>(base + kNoAllocBlocksumOff);
  const int c = is_complex ? 1 : 0;
  // every call shares the array: copy this call's table, clear what starts at zero.
  // The table comes from its page-locked copy, so the upload does not wait for the
  // stream; only if that copy could not be made is the pageable one used.
  const int16_t* src = lut_pinned_table(lut);
  WW_CUDA_TRY(cudaMemcpyAsync(dtable, src ? src : lut_host_table(lut), kNoAllocTableBytes, cudaMemcpyHostToDevice, s));
  WW_CUDA_TRY(cudaMemsetAsync(hist, 0, 65536 * sizeof(uint32_t), s));
  WW_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(SteepCtr), s));
  costs_kernel(p)<<<cost_tiles(m, n), 256, 0, s>>>(ifg, c, coh, mask, m, n, dtable, nullptr, p->box_half_width,
                                                 p->steep_rad, costs, ctr, nullptr, 0ull, nullptr, nullptr);
  k_steep_plan<<<1, 1, 0, s>>>(ctr, p->steep_cap_ppm);
  const int hist_blocks = 148 * 8;
  k_steep_hist<<<hist_blocks, 256, 0, s>>>(ifg, c, coh, mask, m, n, p->steep_rad, ctr, hist, 0);
  k_steep_find<<<1, kFindThreads, 0, s>>>(ctr, hist, 0);
  k_steep_hist<<<hist_blocks, 256, 0, s>>>(ifg, c, coh, mask, m, n, p->steep_rad, ctr, hist, 1);
  k_steep_find<<<1, kFindThreads, 0, s>>>(ctr, hist, 1);
  const int64_t nb = (2 * m * n + kSteepChunk - 1) / kSteepChunk;
  const unsigned nb_grid = (unsigned)std::min<int64_t>(nb, 148 * 16);
  k_steep_ties<<<nb_grid, 256, 0, s>>>(ifg, c, coh, mask, m, n, p->steep_rad, ctr, blocksum);
  k_steep_scan<<<1, kFindThreads, 0, s>>>(ctr, blocksum, nb);
  k_steep_zero<<<nb_grid, 256, 0, s>>>(ifg, c, coh, mask, m, n, p->steep_rad, ctr, blocksum, costs, 0ull);
  WW_CUDA_TRY(cudaGetLastError());
  return WW_OK;
}
