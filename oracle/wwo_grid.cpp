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

// Box-filtered slope estimate (Sec. II-B): arithmetic mean of the wrapped
// gradients of valid same-orientation edges in a (2w+1)^2 window, summed in
// fixed point (2^22 units) so the sum is exact and order-free.
void wwo_alpha_hat(const float* psi, const uint8_t* valid, int64_t m, int64_t n, int32_t w,
                   float* alpha) {
  std::vector<int32_t> q(2 * m * n, 0);
  std::vector<uint8_t> ev(2 * m * n, 0);
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) {
      int64_t k = i * n + j;
      if (j + 1 < n && valid[k] && valid[k + 1]) {
        float dp = psi[k + 1] - psi[k];
        float d = wrapped(dp, wrap_count(dp));
        q[k] = (int32_t)std::nearbyint(d * 4194304.0f);
        ev[k] = 1;
      }
      if (i + 1 < m && valid[k] && valid[k + n]) {
        float dp = psi[k + n] - psi[k];
        float d = wrapped(dp, wrap_count(dp));
        q[m * n + k] = (int32_t)std::nearbyint(d * 4194304.0f);
        ev[m * n + k] = 1;
      }
    }
  for (int plane = 0; plane < 2; ++plane) {
    int64_t rows = plane == 0 ? m : m - 1;
    int64_t cols = plane == 0 ? n - 1 : n;
    for (int64_t i = 0; i < m; ++i)
      for (int64_t j = 0; j < n; ++j) {
        int64_t k = plane * m * n + i * n + j;
        alpha[k] = 0.0f;
        if (i >= rows || j >= cols || !ev[k]) continue;
        int64_t S = 0, cnt = 0;
        for (int64_t a = std::max<int64_t>(0, i - w); a <= std::min<int64_t>(rows - 1, i + w); ++a)
          for (int64_t b = std::max<int64_t>(0, j - w); b <= std::min<int64_t>(cols - 1, j + w); ++b) {
            int64_t kk = plane * m * n + a * n + b;
            if (ev[kk]) {
              S += q[kk];
              ++cnt;
            }
          }
        alpha[k] = cnt ? (float)S / ((float)cnt * 4194304.0f) : 0.0f;
      }
  }
}

int64_t wwo_costs(const float* psi, const float* coh, const uint8_t* valid, int64_t m, int64_t n,
                  const int16_t* table, int32_t w, float steep_rad, int32_t steep_cap_ppm,
                  int16_t* costs) {
  std::vector<float> alpha(2 * m * n);
  wwo_alpha_hat(psi, valid, m, n, w, alpha.data());
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
        costs[(2 * plane) * m * n + k] = table[ig * 256 + ip];
        costs[(2 * plane + 1) * m * n + k] = table[ig * 256 + im];
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
