// CPU oracle, grid steps: input preparation, residues (Eq. 1), slope estimate,
// LUT indices and costs (Sec. II-B), steep-edge bound, integer integration.
// TEST INFRASTRUCTURE ONLY (see wwo.h).  Built with -ffp-contract=off so every
// fp32 operation rounds once, in the order written.
#include "wwo.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace {

const float kPiF = 3.14159274101257324f;      // fp32 nearest to pi, 0x40490FDB
const float kTwoPiF = 6.28318548202514648f;   // 0x40C90FDB
const float kAlphaScale = 40.7436637878417969f; // fp32(256 / (2 pi)), 0x4222F983
const double kTwoPiD = 6.283185307179586;       // double nearest to 2 pi

// ---- CORDIC atan2 in fixed point (angle unit 2^-29 rad) ----
// Table: round(atan(2^-i) * 2^29), i = 0..29.
const int64_t kAtanQ[30] = {421657428, 248918915, 131521918, 66762579, 33510843, 16771758,
                            8387925,   4194219,   2097141,   1048575,  524288,   262144,
                            131072,    65536,     32768,     16384,    8192,     4096,
                            2048,      1024,      512,       256,      128,      64,
                            32,        16,        8,         4,        2,        1};
const int64_t kHalfPiQ = 843314857;  // round(pi/2 * 2^29)

// Decompose a finite float into integer mantissa M and exponent E (v = M * 2^E).
void decompose(float v, int64_t* M, int* E, int* neg) {
  uint32_t b;
  std::memcpy(&b, &v, 4);
  *neg = (int)(b >> 31);
  int be = (int)((b >> 23) & 0xFF);
  uint32_t fr = b & 0x7FFFFF;
  if (be == 0) {
    *M = fr;
    *E = -149;
  } else {
    *M = (int64_t)(fr | 0x800000u);
    *E = be - 150;
  }
}

int bitlen(int64_t x) {
  int k = 0;
  while (x > 0) {
    ++k;
    x >>= 1;
  }
  return k;
}

int64_t scale_to(int64_t M, int E, int top, int neg) {
  // M * 2^(E + 30 - top), truncated toward zero, then signed
  int sh = E + 30 - top;
  int64_t r;
  if (M == 0) return 0;
  if (sh >= 0)
    r = M << sh;
  else if (-sh >= 63)
    r = 0;
  else
    r = M >> (-sh);
  return neg ? -r : r;
}

float cordic_atan2(float im, float re) {
  int64_t Mx, My;
  int Ex, Ey, nx, ny;
  decompose(re, &Mx, &Ex, &nx);
  decompose(im, &My, &Ey, &ny);
  if (Mx == 0 && My == 0) return 0.0f;
  int tx = Mx ? Ex + bitlen(Mx) : -100000;
  int ty = My ? Ey + bitlen(My) : -100000;
  int top = std::max(tx, ty);
  int64_t X = scale_to(Mx, Ex, top, nx);
  int64_t Y = scale_to(My, Ey, top, ny);
  int64_t Z = 0;
  if (X < 0) {
    if (Y >= 0) {
      int64_t t = X;
      X = Y;
      Y = -t;
      Z = kHalfPiQ;
    } else {
      int64_t t = X;
      X = -Y;
      Y = t;
      Z = -kHalfPiQ;
    }
  }
  for (int i = 0; i < 30; ++i) {
    int64_t xs = X >> i, ys = Y >> i;
    if (Y >= 0) {
      X = X + ys;
      Y = Y - xs;
      Z += kAtanQ[i];
    } else {
      X = X - ys;
      Y = Y + xs;
      Z -= kAtanQ[i];
    }
  }
  float psi = (float)Z * (1.0f / 536870912.0f);
  if (psi > kPiF) psi = kPiF;
  if (psi < -kPiF) psi = -kPiF;
  return psi;
}

// ---- CORDIC rotation: (cos t, sin t) 2^30 for t = Z 2^-29 rad ----
// Start vector (K^-1 2^30, 0), K^-1 = prod_i (1 + 2^-2i)^(-1/2) over the 30
// iterations, so the result has length 2^30; angles beyond +-pi/2 are first
// turned by a quarter turn.  Each iteration turns by -+atan(2^-i) toward Z = 0.
const int64_t kInvGainQ30 = 652032874;  // round(2^30 prod (1 + 2^-2i)^(-1/2))

void cordic_cos_sin(int64_t Z, int64_t* c, int64_t* s) {
  int64_t X = kInvGainQ30, Y = 0;
  if (Z > kHalfPiQ) {
    X = 0;
    Y = kInvGainQ30;
    Z -= kHalfPiQ;
  } else if (Z < -kHalfPiQ) {
    X = 0;
    Y = -kInvGainQ30;
    Z += kHalfPiQ;
  }
  for (int i = 0; i < 30; ++i) {
    int64_t xs = X >> i, ys = Y >> i;
    if (Z >= 0) {
      X = X - ys;
      Y = Y + xs;
      Z -= kAtanQ[i];
    } else {
      X = X + ys;
      Y = Y - xs;
      Z += kAtanQ[i];
    }
  }
  *c = X;
  *s = Y;
}

// Wrap count of a phase difference: +1 above pi, -1 at or below -pi (the
// wrapped gradient then lies in (-pi, pi]).
inline int wrap_count(float dpsi) { return (dpsi > kPiF ? 1 : 0) - (dpsi <= -kPiF ? 1 : 0); }

inline float wrapped(float dpsi, int ncount) { return dpsi - kTwoPiF * (float)ncount; }

inline int alpha_index(float x) {
  float t = x + kPiF;
  t = t * kAlphaScale;
  int k = (int)std::floor(t);
  return std::min(255, std::max(0, k));
}

inline int gamma_index(float g) {
  int k = (int)std::floor(g * 128.0f);
  return std::min(127, std::max(0, k));
}

}  // namespace

extern "C" {

void wwo_phase_from_complex(const float* ifg, int64_t count, float* psi) {
  for (int64_t k = 0; k < count; ++k) psi[k] = cordic_atan2(ifg[2 * k + 1], ifg[2 * k]);
}

void wwo_prepare(const float* phase, const float* ifg, const float* coh, const uint8_t* mask,
                 int64_t m, int64_t n, float* psi, float* coh_out, uint8_t* valid) {
  for (int64_t k = 0; k < m * n; ++k) {
    bool ok = mask[k] != 0 && std::isfinite(coh[k]);
    float p = 0.0f;
    if (ifg) {
      ok = ok && std::isfinite(ifg[2 * k]) && std::isfinite(ifg[2 * k + 1]);
      if (ok) p = cordic_atan2(ifg[2 * k + 1], ifg[2 * k]);
    } else {
      ok = ok && std::isfinite(phase[k]);
      if (ok) p = phase[k];
    }
    valid[k] = ok ? 1 : 0;
    psi[k] = ok ? p : 0.0f;
    coh_out[k] = ok ? coh[k] : 0.0f;
  }
}

// Eq. (1): r_p = (1/2pi) sum s_pe d_e around the loop (i,j),(i,j+1),(i+1,j+1),(i+1,j).
// With d_e = dpsi_e - 2pi n_e and the telescoping sum of dpsi, r_p is minus the
// oriented sum of wrap counts; the ground node takes minus the total (Sec. II-A).
void wwo_residues(const float* psi, int64_t m, int64_t n, int8_t* res, int32_t* ground) {
  int64_t total = 0;
  for (int64_t i = 0; i + 1 < m; ++i) {
    for (int64_t j = 0; j + 1 < n; ++j) {
      const float* r0 = psi + i * n;
      const float* r1 = psi + (i + 1) * n;
      int n_top = wrap_count(r0[j + 1] - r0[j]);          // h(i,j), forward
      int n_right = wrap_count(r1[j + 1] - r0[j + 1]);    // v(i,j+1), forward
      int n_bottom = wrap_count(r1[j + 1] - r1[j]);       // h(i+1,j), traversed backward
      int n_left = wrap_count(r1[j] - r0[j]);             // v(i,j), traversed backward
      int r = -(n_top + n_right - n_bottom - n_left);
      res[i * (n - 1) + j] = (int8_t)r;
      total += r;
    }
  }
  *ground = (int32_t)(-total);
}

// Box-filtered slope estimate (Sec. II-B).  mode 0: arithmetic mean of the
// wrapped gradients of valid same-orientation edges in a (2w+1)^2 window,
// summed in fixed point (2^22 units) so the sum is exact and order-free.
// mode 1: the argument of the sum of their unit phasors exp(i d), each from a
// fixed-point CORDIC rotation of round(d 2^29), summed as integers, the
// argument by the CORDIC atan2 of the two sums (each rounded once to fp32).
void wwo_alpha_hat2(const float* psi, const uint8_t* valid, int64_t m, int64_t n, int32_t w, int32_t mode,
                    float* alpha);

void wwo_alpha_hat(const float* psi, const uint8_t* valid, int64_t m, int64_t n, int32_t w,
                   float* alpha) {
  wwo_alpha_hat2(psi, valid, m, n, w, 0, alpha);
}

void wwo_alpha_hat2(const float* psi, const uint8_t* valid, int64_t m, int64_t n, int32_t w, int32_t mode,
                    float* alpha) {
  std::vector<int32_t> q(2 * m * n, 0);
  std::vector<int64_t> pc(2 * m * n, 0), ps(2 * m * n, 0);  // unit phasors of the edges (mode 1)
  std::vector<uint8_t> ev(2 * m * n, 0);
  auto edge = [&](int64_t k, int64_t k2, int64_t slot) {
    float dp = psi[k2] - psi[k];
    float d = wrapped(dp, wrap_count(dp));
    q[slot] = (int32_t)std::nearbyint(d * 4194304.0f);
    cordic_cos_sin((int64_t)std::nearbyint(d * 536870912.0f), &pc[slot], &ps[slot]);
    ev[slot] = 1;
  };
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) {
      int64_t k = i * n + j;
      if (j + 1 < n && valid[k] && valid[k + 1]) edge(k, k + 1, k);
      if (i + 1 < m && valid[k] && valid[k + n]) edge(k, k + n, m * n + k);
    }
  for (int plane = 0; plane < 2; ++plane) {
    int64_t rows = plane == 0 ? m : m - 1;
    int64_t cols = plane == 0 ? n - 1 : n;
    for (int64_t i = 0; i < m; ++i)
      for (int64_t j = 0; j < n; ++j) {
        int64_t k = plane * m * n + i * n + j;
        alpha[k] = 0.0f;
        if (i >= rows || j >= cols || !ev[k]) continue;
        int64_t S = 0, cnt = 0, SX = 0, SY = 0;
        for (int64_t a = std::max<int64_t>(0, i - w); a <= std::min<int64_t>(rows - 1, i + w); ++a)
          for (int64_t b = std::max<int64_t>(0, j - w); b <= std::min<int64_t>(cols - 1, j + w); ++b) {
            int64_t kk = plane * m * n + a * n + b;
            if (ev[kk]) {
              S += q[kk];
              SX += pc[kk];
              SY += ps[kk];
              ++cnt;
            }
          }
        if (mode == 0)
          alpha[k] = cnt ? (float)S / ((float)cnt * 4194304.0f) : 0.0f;
        else
          alpha[k] = cordic_atan2((float)SY, (float)SX);
      }
  }
}

// Bilinear lookup of the cost between bin centres: x = (a + PI_F) 256/2pi - 1/2
// and y = g 128 - 1/2 locate the slope and coherence between the centres
// (clamped to the outermost pair, weights clamped to [0, 1]); the table holds
// 100 ln(P0/P+) (Eq. 4 before the max and the floor) at the centres; the result
// is floor of the interpolated value, saturated to [0, 32767].  fp32 throughout,
// every operation rounded once in the order written.
static int16_t bilinear_cost(const float* ratio, float a, float g) {
  float x = (a + kPiF) * kAlphaScale - 0.5f;
  float y = g * 128.0f - 0.5f;
  int j0 = std::min(254, std::max(0, (int)std::floor(x)));
  int k0 = std::min(126, std::max(0, (int)std::floor(y)));
  float fx = std::min(1.0f, std::max(0.0f, x - (float)j0));
  float fy = std::min(1.0f, std::max(0.0f, y - (float)k0));
  const float* r0 = ratio + k0 * 256 + j0;
  const float* r1 = r0 + 256;
  float v0 = r0[0] + fx * (r0[1] - r0[0]);
  float v1 = r1[0] + fx * (r1[1] - r1[0]);
  float v = v0 + fy * (v1 - v0);
  if (!(v > 0.0f)) return 0;
  if (v >= 32767.0f) return 32767;
  return (int16_t)std::floor(v);
}

int64_t wwo_costs2(const float* psi, const float* coh, const uint8_t* valid, int64_t m, int64_t n,
                   const int16_t* table, const float* ratio, int32_t w, int32_t slope_mode, int32_t lookup,
                   float steep_rad, int32_t steep_cap_ppm, int16_t* costs);

int64_t wwo_costs(const float* psi, const float* coh, const uint8_t* valid, int64_t m, int64_t n,
                  const int16_t* table, int32_t w, float steep_rad, int32_t steep_cap_ppm,
                  int16_t* costs) {
  return wwo_costs2(psi, coh, valid, m, n, table, nullptr, w, 0, 0, steep_rad, steep_cap_ppm, costs);
}

int64_t wwo_costs2(const float* psi, const float* coh, const uint8_t* valid, int64_t m, int64_t n,
                   const int16_t* table, const float* ratio, int32_t w, int32_t slope_mode, int32_t lookup,
                   float steep_rad, int32_t steep_cap_ppm, int16_t* costs) {
  std::vector<float> alpha(2 * m * n);
  wwo_alpha_hat2(psi, valid, m, n, w, slope_mode, alpha.data());
  std::memset(costs, 0, sizeof(int16_t) * 4 * m * n);
  struct Cand {
    float mag;
    int64_t key;
  };
  std::vector<Cand> cands;
  int64_t n_valid_edges = 0;
  for (int plane = 0; plane < 2; ++plane)
    for (int64_t i = 0; i < m; ++i)
      for (int64_t j = 0; j < n; ++j) {
        int64_t k = i * n + j;
        int64_t k2 = plane == 0 ? k + 1 : k + n;
        bool exists = plane == 0 ? (j + 1 < n) : (i + 1 < m);
        if (!exists || !valid[k] || !valid[k2]) continue;
        ++n_valid_edges;
        float ge = std::min(coh[k], coh[k2]);  // edge coherence: min of endpoints
        int ig = gamma_index(ge);
        float a = alpha[plane * m * n + k];
        int ip = alpha_index(a);
        int im = alpha_index(-a);
        // the arc giving dk=+1 costs c(alpha-hat); the opposite arc c(-alpha-hat)
        if (lookup == 0) {
          costs[(2 * plane) * m * n + k] = table[ig * 256 + ip];
          costs[(2 * plane + 1) * m * n + k] = table[ig * 256 + im];
        } else {
          costs[(2 * plane) * m * n + k] = bilinear_cost(ratio, a, ge);
          costs[(2 * plane + 1) * m * n + k] = bilinear_cost(ratio, -a, ge);
        }
        float dp = psi[k2] - psi[k];
        float d = wrapped(dp, wrap_count(dp));
        float mag = std::fabs(d);
        if (mag > steep_rad) cands.push_back({mag, plane * m * n + k});
      }
  // Steep-edge bound: zero cost for edges whose unsmoothed |d| exceeds the
  // threshold, at most cap = floor(ppm * valid_edges / 1e6) of them, chosen by
  // |d| descending then edge key ascending (h plane before v plane).
  int64_t cap = (n_valid_edges * (int64_t)steep_cap_ppm) / 1000000;
  if ((int64_t)cands.size() > cap) {
    std::stable_sort(cands.begin(), cands.end(), [](const Cand& x, const Cand& y) {
      if (x.mag != y.mag) return x.mag > y.mag;
      return x.key < y.key;
    });
    cands.resize(cap);
  }
  for (const Cand& c : cands) {
    int plane = (int)(c.key / (m * n));
    int64_t k = c.key % (m * n);
    costs[(2 * plane) * m * n + k] = 0;
    costs[(2 * plane + 1) * m * n + k] = 0;
  }
  return (int64_t)cands.size();
}

// Integration in integer cycles: K(0,0)=0; K_v = K_u + dk_e - n_e down column 0
// and then along each row.  phi = psi + 2 pi K with the fixed FP64 sequence
// (double)K * 2pi, + (double)psi, rounded once to fp32.  Masked pixels -> NaN.
void wwo_integrate(const float* psi, const uint8_t* valid, const int8_t* flows, int64_t m, int64_t n,
                   float* unwrapped, int32_t* cycles) {
  const int8_t* dkh = flows;
  const int8_t* dkv = flows + m * n;
  std::vector<int64_t> K(m * n, 0);
  for (int64_t i = 0; i + 1 < m; ++i) {
    int64_t k = i * n;
    K[k + n] = K[k] + dkv[k] - wrap_count(psi[k + n] - psi[k]);
  }
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j + 1 < n; ++j) {
      int64_t k = i * n + j;
      K[k + 1] = K[k] + dkh[k] - wrap_count(psi[k + 1] - psi[k]);
    }
  for (int64_t k = 0; k < m * n; ++k) {
    cycles[k] = (int32_t)K[k];
    if (!valid[k]) {
      unwrapped[k] = std::nanf("");
      continue;
    }
    double t = (double)K[k] * kTwoPiD;
    double s = (double)psi[k] + t;
    unwrapped[k] = (float)s;
  }
}

}  // extern "C"

// ---- Multilooking and Eq. (3) sample coherence from two SLC images ----
// For output pixel (i, j) over the ly x lx looks (rows i ly .. i ly + ly - 1,
// columns j lx .. j lx + lx - 1 of the SLCs, row-major order): the cross
// product sum S12 = sum z1 conj(z2) and the powers S11 = sum |z1|^2,
// S22 = sum |z2|^2, every product and sum in fp32 rounded once in the order
// written; the multilooked interferogram is S12 and the sample coherence
// gamma = sqrt(re^2 + im^2) / sqrt(S11 S22), clamped to 1, 0 when a power is 0.
extern "C" void wwo_multilook(const float* slc1, const float* slc2, int64_t M, int64_t N, int32_t ly, int32_t lx,
                              float* ifg, float* coh) {
  const int64_t m = M / ly, n = N / lx;
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) {
      float re = 0.0f, im = 0.0f, p1 = 0.0f, p2 = 0.0f;
      for (int32_t a = 0; a < ly; ++a)
        for (int32_t b = 0; b < lx; ++b) {
          const int64_t k = (i * ly + a) * N + (j * lx + b);
          const float ar = slc1[2 * k], ai = slc1[2 * k + 1], br = slc2[2 * k], bi = slc2[2 * k + 1];
          const float t_re = ar * br + ai * bi;  // z1 conj(z2)
          const float t_im = ai * br - ar * bi;
          re = re + t_re;
          im = im + t_im;
          p1 = p1 + (ar * ar + ai * ai);
          p2 = p2 + (br * br + bi * bi);
        }
      const int64_t o = i * n + j;
      ifg[2 * o] = re;
      ifg[2 * o + 1] = im;
      const float den = std::sqrt(p1 * p2);
      float g = den > 0.0f ? std::sqrt(re * re + im * im) / den : 0.0f;
      coh[o] = g > 1.0f ? 1.0f : g;
    }
}
