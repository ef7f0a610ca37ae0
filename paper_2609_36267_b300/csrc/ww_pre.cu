// Steps before and after the unwrap proper (Sec. II-B Eq. 3, Sec. II-D):
//   ww_multilook        multilooked interferogram and Eq. (3) sample coherence
//                       from two SLC images (fp32, fixed summation order);
//   ww_goldstein        adaptive power-spectrum filter in overlapping patches;
//   ww_transfer_cycles  the integer solution of a filtered phase moved to the
//                       original wrapped phase.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "ww_internal.cuh"

namespace ww {
namespace {

// ---- multilook + Eq. (3) ----
// One thread per output pixel; the looks are visited row-major and every
// product and sum is rounded once in that order, so the result does not depend
// on the launch shape.  A warp's 32 outputs read 32 adjacent look windows of
// each SLC row, which the L1 cache turns into whole-line reads.
__global__ void k_multilook(const float2* __restrict__ z1, const float2* __restrict__ z2, int64_t M, int64_t N,
                            int ly, int lx, int64_t m, int64_t n, float2* __restrict__ ifg, float* __restrict__ coh) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < m * n; o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = o / n, j = o - (o / n) * n;
    float re = 0.0f, im = 0.0f, p1 = 0.0f, p2 = 0.0f;
    for (int a = 0; a < ly; ++a) {
      const int64_t row = (i * ly + a) * N + j * lx;
      for (int b = 0; b < lx; ++b) {
        const float2 u = __ldg(z1 + row + b), v = __ldg(z2 + row + b);
        const float t_re = __fadd_rn(__fmul_rn(u.x, v.x), __fmul_rn(u.y, v.y));  // z1 conj(z2)
        const float t_im = __fsub_rn(__fmul_rn(u.y, v.x), __fmul_rn(u.x, v.y));
        re = __fadd_rn(re, t_re);
        im = __fadd_rn(im, t_im);
        p1 = __fadd_rn(p1, __fadd_rn(__fmul_rn(u.x, u.x), __fmul_rn(u.y, u.y)));
        p2 = __fadd_rn(p2, __fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y)));
      }
    }
    ifg[o] = make_float2(re, im);
    const float den = __fsqrt_rn(__fmul_rn(p1, p2));
    const float g = den > 0.0f ? __fdiv_rn(__fsqrt_rn(__fadd_rn(__fmul_rn(re, re), __fmul_rn(im, im))), den) : 0.0f;
    coh[o] = fminf(g, 1.0f);
  }
}

// ---- Goldstein filter ----
constexpr int GP = 32;  // patch size (the DFT length)

struct GoldArgs {
  const float2* ifg;
  int64_t m, n, npy, npx;
  int step, smooth;
  float alpha;
  float2* patches;  // [npy * npx][GP][GP], weighted filtered patches
};

// In-place 32-point DFTs of the 32 rows (rows = true) or columns of a
// shared-memory patch; sign -1 forward, +1 inverse (unscaled).
__device__ void dft32(float2 (*a)[GP + 1], float2 (*tmp)[GP + 1], const float2* tw, bool rows, float sign) {
  for (int e = threadIdx.x; e < GP * GP; e += blockDim.x) {
    const int line = e / GP, k = e % GP;
    float sr = 0.0f, si = 0.0f;
    for (int t = 0; t < GP; ++t) {
      const float2 x = rows ? a[line][t] : a[t][line];
      const float2 w = tw[(k * t) & (GP - 1)];
      const float wi = sign * w.y;
      sr += x.x * w.x - x.y * wi;
      si += x.x * wi + x.y * w.x;
    }
    if (rows)
      tmp[line][k] = make_float2(sr, si);
    else
      tmp[k][line] = make_float2(sr, si);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < GP * GP; e += blockDim.x) a[e / GP][e % GP] = tmp[e / GP][e % GP];
  __syncthreads();
}

__device__ __forceinline__ float tri_weight(int t) { return 1.0f - fabsf((2.0f * t + 1.0f) / GP - 1.0f); }

// One block per patch: FFT, spectrum weighting by the smoothed, max-normalised
// amplitude to the power alpha, inverse FFT, the separable triangular weight.
__global__ void __launch_bounds__(256) k_goldstein_patch(GoldArgs g, const float2* __restrict__ twiddle) {
  __shared__ float2 a[GP][GP + 1], tmp[GP][GP + 1];
  __shared__ float amp[GP][GP + 1];
  __shared__ float2 tw[GP];
  __shared__ float red[256];
  const int64_t p = blockIdx.x;
  const int64_t y0 = (p / g.npx) * g.step, x0 = (p % g.npx) * g.step;
  if (threadIdx.x < GP) tw[threadIdx.x] = twiddle[threadIdx.x];
  for (int e = threadIdx.x; e < GP * GP; e += blockDim.x) {
    const int r = e / GP, c = e % GP;
    const int64_t i = y0 + r, j = x0 + c;
    a[r][c] = (i < g.m && j < g.n) ? g.ifg[i * g.n + j] : make_float2(0.0f, 0.0f);
  }
  __syncthreads();
  dft32(a, tmp, tw, true, -1.0f);
  dft32(a, tmp, tw, false, -1.0f);
  for (int e = threadIdx.x; e < GP * GP; e += blockDim.x) {
    const float2 z = a[e / GP][e % GP];
    amp[e / GP][e % GP] = sqrtf(z.x * z.x + z.y * z.y);
  }
  __syncthreads();
  // circular box mean of the amplitude into tmp.x, and its maximum
  const int h = g.smooth / 2;
  float mx = 0.0f;
  for (int e = threadIdx.x; e < GP * GP; e += blockDim.x) {
    const int r = e / GP, c = e % GP;
    float s = 0.0f;
    for (int dy = -h; dy <= h; ++dy)
      for (int dx = -h; dx <= h; ++dx) s += amp[(r + dy + GP) & (GP - 1)][(c + dx + GP) & (GP - 1)];
    s /= (float)(g.smooth * g.smooth);
    tmp[r][c].x = s;
    mx = fmaxf(mx, s);
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  const float smax = red[0];
  for (int e = threadIdx.x; e < GP * GP; e += blockDim.x) {
    const int r = e / GP, c = e % GP;
    const float hgain = smax > 0.0f ? (g.alpha == 0.0f ? 1.0f : powf(tmp[r][c].x / smax, g.alpha)) : 0.0f;
    a[r][c] = make_float2(a[r][c].x * hgain, a[r][c].y * hgain);
  }
  __syncthreads();
  dft32(a, tmp, tw, true, 1.0f);
  dft32(a, tmp, tw, false, 1.0f);
  float2* out = g.patches + p * GP * GP;
  for (int e = threadIdx.x; e < GP * GP; e += blockDim.x) {
    const int r = e / GP, c = e % GP;
    const float w = tri_weight(r) * tri_weight(c) * (1.0f / (GP * GP));
    out[e] = make_float2(a[r][c].x * w, a[r][c].y * w);
  }
}

// Every output pixel: the weighted patch values covering it, in patch order,
// divided by the summed weights.
__global__ void k_goldstein_gather(GoldArgs g, float2* __restrict__ out) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < g.m * g.n; o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = o / g.n, j = o - (o / g.n) * g.n;
    const int64_t py1 = i / g.step, px1 = j / g.step;
    const int64_t py0 = i >= GP ? (i - GP) / g.step + 1 : 0, px0 = j >= GP ? (j - GP) / g.step + 1 : 0;
    float sr = 0.0f, si = 0.0f, sw = 0.0f;
    for (int64_t py = py0; py <= py1 && py < g.npy; ++py)
      for (int64_t px = px0; px <= px1 && px < g.npx; ++px) {
        const int r = (int)(i - py * g.step), c = (int)(j - px * g.step);
        const float2 v = g.patches[(py * g.npx + px) * GP * GP + r * GP + c];
        sr += v.x;
        si += v.y;
        sw += tri_weight(r) * tri_weight(c);
      }
    out[o] = make_float2(sr / sw, si / sw);
  }
}

// ---- cycle transfer ----
__global__ void k_transfer(const float* __restrict__ filt, const void* __restrict__ ifg, int is_complex,
                           const float* __restrict__ coh, const uint8_t* __restrict__ mask, int64_t P,
                           float* __restrict__ unw, int32_t* __restrict__ cyc) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    const Pix px = load_pixel(ifg, is_complex, coh, mask, k);
    const float pf = filt[k];
    if (!px.valid || isnan(pf)) {
      unw[k] = __int_as_float(0x7fc00000);
      cyc[k] = 0;
      continue;
    }
    const double K = rint(__ddiv_rn(__dsub_rn((double)pf, (double)px.psi), kTwoPiD));
    cyc[k] = (int32_t)K;
    unw[k] = __double2float_rn(__dadd_rn((double)px.psi, __dmul_rn(K, kTwoPiD)));
  }
}

int grid_for(int64_t work) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, (int64_t)sms * 16));
}

}  // namespace
}  // namespace ww

extern "C" {

ww_status ww_multilook(const void* slc1, const void* slc2, int64_t M, int64_t N, int32_t looks_y, int32_t looks_x,
                       void* ifg, float* coh, ww_stream stream) {
  using namespace ww;
  if (!slc1 || !slc2 || !ifg || !coh || looks_y < 1 || looks_x < 1 || M < looks_y || N < looks_x ||
      M > (1ll << 31) || N > (1ll << 31))
    return WW_ERR_INVALID_ARG;
  const int64_t m = M / looks_y, n = N / looks_x;
  cudaStream_t s = (cudaStream_t)stream;
  k_multilook<<<grid_for(m * n), 256, 0, s>>>(reinterpret_cast<const float2*>(slc1), reinterpret_cast<const float2*>(slc2),
                                               M, N, looks_y, looks_x, m, n, reinterpret_cast<float2*>(ifg), coh);
  WW_CUDA_TRY(cudaGetLastError());
  return WW_OK;
}

ww_status ww_goldstein(const void* ifg, int64_t m, int64_t n, float alpha, int32_t step, int32_t smooth, void* out,
                       ww_stream stream) {
  using namespace ww;
  if (!ifg || !out || m < 1 || n < 1 || !(alpha >= 0.0f) || !std::isfinite(alpha) || step < 1 || step > GP ||
      smooth < 1 || smooth > GP || (smooth & 1) == 0 || m * n >= (1ll << 40))
    return WW_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  GoldArgs g;
  g.ifg = reinterpret_cast<const float2*>(ifg);
  g.m = m;
  g.n = n;
  g.npy = (m + step - 1) / step;
  g.npx = (n + step - 1) / step;
  g.step = step;
  g.smooth = smooth;
  g.alpha = alpha;
  if (g.npy * g.npx >= (1ll << 31)) return WW_ERR_INVALID_ARG;
  // twiddles exp(-2 pi i t / 32), computed in double on the host and rounded once
  float2 htw[GP];
  for (int t = 0; t < GP; ++t)
    htw[t] = make_float2((float)std::cos(2.0 * M_PI * t / GP), (float)-std::sin(2.0 * M_PI * t / GP));
  float2* dtw = nullptr;
  if (cudaMalloc(&dtw, sizeof(htw)) != cudaSuccess) return WW_ERR_OOM;
  if (cudaMalloc(&g.patches, (size_t)g.npy * g.npx * GP * GP * sizeof(float2)) != cudaSuccess) {
    cudaFree(dtw);
    return WW_ERR_OOM;
  }
  ww_status st = WW_OK;
  if (cudaMemcpyAsync(dtw, htw, sizeof(htw), cudaMemcpyHostToDevice, s) != cudaSuccess) st = WW_ERR_CUDA;
  if (st == WW_OK) {
    k_goldstein_patch<<<(unsigned)(g.npy * g.npx), 256, 0, s>>>(g, dtw);
    k_goldstein_gather<<<grid_for(m * n), 256, 0, s>>>(g, reinterpret_cast<float2*>(out));
    if (cudaGetLastError() != cudaSuccess) st = WW_ERR_CUDA;
  }
  // the scratch is freed once the stream has passed the kernels
  if (cudaStreamSynchronize(s) != cudaSuccess && st == WW_OK) st = WW_ERR_CUDA;
  cudaFree(g.patches);
  cudaFree(dtw);
  return st;
}

ww_status ww_transfer_cycles(const float* unwrapped_filtered, const void* ifg, int32_t is_complex, const float* coh,
                             const uint8_t* mask, int64_t m, int64_t n, float* unwrapped, int32_t* cycles,
                             ww_stream stream) {
  using namespace ww;
  if (!unwrapped_filtered || !ifg || !unwrapped || !cycles || m < 1 || n < 1 || m * n >= (1ll << 40))
    return WW_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  k_transfer<<<grid_for(m * n), 256, 0, s>>>(unwrapped_filtered, ifg, is_complex ? 1 : 0, coh, mask, m * n, unwrapped,
                                              cycles);
  WW_CUDA_TRY(cudaGetLastError());
  return WW_OK;
}

}  // extern "C"
