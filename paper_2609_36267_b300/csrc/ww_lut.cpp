// Host FP64 construction of the int16 arc-cost table (Sec. II-B, Eqs. 4-7).
//
// For each coherence bin centre gh and number of looks L:
//   * the L-look phase-noise pdf f(eta | g, L) of Lee et al. (cited in Sec. II-B),
//     evaluated as f = L (1-g^2)^L / (pi 2^L) * I(b), b = g cos(eta),
//     I(b) = Int_0^inf cosh((L-1)t)(cosh t - b)^-(L+1) dt, and after the change of
//     variable t = 2 asinh(a tan th), a^2 = (1-b)/2,
//     I(b) = 2a (2a^2)^-(L+1) Int_0^{pi/2} cosh(2(L-1) asinh(a tan th))
//                              cos^(2L+1)(th) / sqrt(cos^2 th + a^2 sin^2 th) dth,
//     a smooth integrand on a finite interval (fixed Gauss-Legendre panels);
//   * Eq. 5: the pdf marginalised over a uniform prior on the true coherence g
//     with the sample-coherence pdf of Touzi et al. (cited in Sec. II-B),
//     f(gh | g, L) = 2(L-1)(1-g^2)^L gh (1-gh^2)^(L-2) (1-z)^(1-2L) 2F1(1-L,1-L;1;z),
//     z = g^2 gh^2 (Euler's transformation of 2F1(L,L;1;z); positive series),
//     integrated in the variable s = atanh(g);
//   * the edge noise Delta eta = eta_v - eta_u of two independent pixels (pdf
//     f~*f~ on [-2pi, 2pi]); its tail probability Sg(s) = P(Delta eta > s);
//   * Eq. 6: q+(alpha) = Sg(pi - alpha), q-(alpha) = Sg(pi + alpha),
//     q0 = 1 - q+ - q-;
//   * Eq. 7: P_j = Int q_j(alpha) N(alpha; alpha-hat, sigma) dalpha over
//     alpha-hat +- 8 sigma, weights normalised on that interval, with
//     sigma^2 = E[wrap(Delta eta)^2] (which equals pi^2/3 for uniform noise,
//     the limit stated in Sec. II-B);
//   * Eq. 4: c = max(0, -ln(P+/P0)), stored as floor(100 c) saturating at 32767.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>
#include <vector>

#include "ww_internal.cuh"

namespace {

const double kPi = 3.14159265358979323846;
const double kSPanelsPerUnit = 16.0;

void legendre_rule(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double d = 1.0;
    for (int it = 0; it < 64; ++it) {
      double a = 1.0, b = 0.0;
      for (int k = 1; k <= n; ++k) {
        double c = b;
        b = a;
        a = ((2.0 * k - 1.0) * z * b - (k - 1.0) * c) / k;
      }
      d = n * (z * a - b) / (z * z - 1.0);
      double dz = a / d;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * d * d);
  }
}

struct Rule {
  std::vector<double> x, w;
};

// log of the phase pdf for true coherence g (omg = 1 - g), phase eta.
double log_phase_pdf(double eta, double g, double omg, double L, const Rule& r) {
  double sh = std::sin(0.5 * eta);
  double a2 = 0.5 * (omg + 2.0 * g * sh * sh);  // (1 - g cos eta)/2 without cancellation
  double a = std::sqrt(a2);
  const int panels = 4;
  const double hw = 0.5 * kPi / panels;
  double vals[4 * 32];
  int nn = (int)r.x.size();
  double vmax = -INFINITY;
  for (int p = 0; p < panels; ++p)
    for (int k = 0; k < nn; ++k) {
      double th = hw * (p + 0.5) + 0.5 * hw * r.x[k];
      double c = std::cos(th), s = std::sin(th);
      double y = 2.0 * (L - 1.0) * std::asinh(a * s / c);
      y = std::fabs(y);
      double lch = y + std::log1p(std::exp(-2.0 * y)) - 0.6931471805599453;
      double v = lch + (2.0 * L + 1.0) * std::log(c) - 0.5 * std::log(c * c + a2 * s * s);
      vals[p * nn + k] = v;
      vmax = std::max(vmax, v);
    }
  double acc = 0.0;
  for (int p = 0; p < panels; ++p)
    for (int k = 0; k < nn; ++k) acc += 0.5 * hw * r.w[k] * std::exp(vals[p * nn + k] - vmax);
  double logI = std::log(2.0 * a) - (L + 1.0) * std::log(2.0 * a2) + vmax + std::log(acc);
  return std::log(L) + L * (std::log(omg) + std::log1p(g)) - std::log(kPi) - L * 0.6931471805599453 + logI;
}

// log of the sample-coherence pdf, via the Euler-transformed series.
double log_coh_pdf(double gh, double g, double omg, double L) {
  double z = g * g * gh * gh;
  double term = 1.0, sum = 1.0, scale = 0.0;
  for (long k = 1; k < 50000000; ++k) {
    double q = (k - L) / k;
    term *= q * q * z;
    sum += term;
    if (sum > 1e250) {
      sum *= 1e-250;
      term *= 1e-250;
      scale += 250.0 * 2.302585092994046;
    }
    if (term == 0.0 || (k > 2.0 * L + 2.0 && term < 1e-19 * sum)) break;
  }
  return std::log(2.0 * (L - 1.0)) + L * (std::log(omg) + std::log1p(g)) + std::log(gh) +
         (L - 2.0) * std::log1p(-gh * gh) + (1.0 - 2.0 * L) * std::log1p(-z) + std::log(sum) + scale;
}

// Composite Simpson over count samples (count-1 intervals); a 3/8 rule closes an odd count.
double simpson(const double* y, long count, double h) {
  if (count < 2) return 0.0;
  if (count == 2) return 0.5 * h * (y[0] + y[1]);
  long intervals = count - 1;
  double s = 0.0;
  long end = intervals;
  if (intervals % 2 == 1) {
    if (intervals == 1) return 0.5 * h * (y[0] + y[1]);
    end = intervals - 3;
    long b = end;
    s += 3.0 * h / 8.0 * (y[b] + 3.0 * y[b + 1] + 3.0 * y[b + 2] + y[b + 3]);
  }
  for (long i = 0; i + 2 <= end; i += 2) s += h / 3.0 * (y[i] + 4.0 * y[i + 1] + y[i + 2]);
  return s;
}

struct RowTables {
  long nh = 0;              // intervals on [0, pi]
  std::vector<double> f;    // pdf on -pi + i h, i = 0..2N
  std::vector<double> surv; // P(eta > x_i)
  std::vector<double> lsg;  // log P(Delta eta > s_k), s_k = k h, k = 0..2N
  double sigma = 0.0;
};

void row_tables(const std::vector<double>& f_in, long nh, RowTables& R) {
  R.nh = nh;
  const long N2 = 2L * nh + 1;
  const double h = kPi / nh;
  R.f = f_in;
  double z = simpson(R.f.data(), N2, h);
  for (double& v : R.f) v /= z;
  // survival P(eta > x_i): Simpson from the +pi end over an even number of
  // intervals, with one 3/8 block where the count is odd
  R.surv.assign(N2, 0.0);
  for (long i = N2 - 1; i >= 0; --i) R.surv[i] = simpson(&R.f[i], N2 - i, h);
  (void)0;
  // tail of the edge noise and sigma
  R.lsg.assign(N2, -INFINITY);
  std::vector<double> prod(N2), w2(N2, 0.0);
  for (long k = 0; k < N2; ++k) {
    long cnt = N2 - k;
    for (long i = 0; i < cnt; ++i) prod[i] = R.f[i] * R.surv[i + k];
    double sg = simpson(prod.data(), cnt, h);
    if (k == 0) sg = 0.5;
    R.lsg[k] = sg > 0 ? std::log(sg) : -INFINITY;
    for (long i = 0; i < cnt; ++i) prod[i] = R.f[i] * R.f[i + k];
    double gk = simpson(prod.data(), cnt, h);
    double s = k * h;
    double wv = s <= kPi ? s : s - 2.0 * kPi;
    w2[k] = wv * wv * gk;
  }
  double half1 = simpson(w2.data(), nh + 1, h);
  double half2 = simpson(w2.data() + nh, nh + 1, h);
  R.sigma = std::sqrt(2.0 * (half1 + half2));
}

// P(Delta eta > s) by 4-point Lagrange interpolation of the log tail.
double tail(const RowTables& R, double s) {
  const double h = kPi / R.nh;
  const long K = 2L * R.nh;
  if (s >= 2.0 * kPi) return 0.0;
  if (s <= -2.0 * kPi) return 1.0;
  if (s < 0.0) return 1.0 - tail(R, -s);
  double u = s / h;
  long i0 = std::min(std::max((long)std::floor(u) - 1, 0L), K - 3);
  bool fin = std::isfinite(R.lsg[i0]) && std::isfinite(R.lsg[i0 + 1]) && std::isfinite(R.lsg[i0 + 2]) &&
             std::isfinite(R.lsg[i0 + 3]);
  double acc = 0.0;
  for (int j = 0; j < 4; ++j) {
    double l = 1.0;
    for (int q = 0; q < 4; ++q)
      if (q != j) l *= (u - (i0 + q)) / (double)(j - q);
    acc += l * (fin ? R.lsg[i0 + j] : (std::isfinite(R.lsg[i0 + j]) ? std::exp(R.lsg[i0 + j]) : 0.0));
  }
  return fin ? std::exp(acc) : std::max(acc, 0.0);
}

void row_costs(const RowTables& R, const Rule& r12, double* c100_row, int16_t* tab_row, float* ratio_row) {
  const double sg = R.sigma;
  const int panels = 64;
  for (int j = 0; j < ww::kNAlpha; ++j) {
    double ah = -kPi + (j + 0.5) * (2.0 * kPi / ww::kNAlpha);
    const double lo = ah - 8.0 * sg, hi = ah + 8.0 * sg;
    // q+ vanishes for alpha <= -pi and q- for alpha >= pi (|Delta eta| <= 2 pi):
    // the integrand's second derivative jumps at +-pi, so the Gauss panels end there
    double brk[4] = {lo, hi, hi, hi};
    int nb = 1;
    for (double c : {-kPi, kPi})
      if (c > lo && c < hi) brk[nb++] = c;
    brk[nb] = hi;
    double W = 0.0, S0 = 0.0, Sp = 0.0;
    for (int seg = 0; seg < nb; ++seg) {
      const double a = brk[seg], b = brk[seg + 1];
      const int np = std::max(4, (int)std::ceil(panels * (b - a) / (hi - lo)));
      const double hw = (b - a) / np;
      for (int p = 0; p < np; ++p)
        for (size_t k = 0; k < r12.x.size(); ++k) {
          double al = a + hw * (p + 0.5) + 0.5 * hw * r12.x[k];
          double wt = 0.5 * hw * r12.w[k] * std::exp(-0.5 * (al - ah) * (al - ah) / (sg * sg));
          double qp = tail(R, kPi - al);
          double qm = tail(R, kPi + al);
          double q0 = std::max(0.0, 1.0 - qp - qm);
          W += wt;
          S0 += wt * q0;
          Sp += wt * qp;
        }
    }
    double p0 = S0 / W, pp = Sp / W, c100;
    if (!(pp > 0.0))
      c100 = INFINITY;
    else if (!(p0 > 0.0))
      c100 = 0.0;
    else
      c100 = std::max(0.0, -100.0 * std::log(pp / p0));
    c100_row[j] = c100;
    double fl = std::floor(c100);
    tab_row[j] = (int16_t)(fl >= 32767.0 ? 32767 : (int)fl);
    // 100 ln(P0/P+) before the max and the floor, for the interpolated lookup
    // (saturated like the table: P+ = 0 -> 32767, P0 = 0 -> the lower bound)
    const double r = !(pp > 0.0) ? 32767.0 : (!(p0 > 0.0) ? -10000.0 : -100.0 * std::log(pp / p0));
    ratio_row[j] = (float)std::min(32767.0, std::max(-10000.0, r));
  }
}

template <class F>
void parallel_for(long count, F fn) {
  unsigned nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
  std::atomic<long> next(0);
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; ++t)
    th.emplace_back([&]() {
      for (long i; (i = next.fetch_add(1)) < count;) fn(i);
    });
  for (auto& x : th) x.join();
}

}  // namespace

namespace ww {

int lut_build_host(double L, int16_t* table, double* cost100, float* ratio100) {
  if (!(L > 1.0) || !std::isfinite(L)) return WW_ERR_INVALID_ARG;
  // intervals on [0, pi]; the high-coherence rows are sharper for many looks
  const long NH = L > 16.0 ? 8192 : 4096;
  Rule r24, r12, r8;
  legendre_rule(24, r24.x, r24.w);
  legendre_rule(12, r12.x, r12.w);
  legendre_rule(8, r8.x, r8.w);
  // coherence nodes in s = atanh(g): 8-point panels of width 1/16 (the
  // posterior over g is only ~0.3 wide in s at low sample coherence and many looks)
  const double gh_max = (kNGamma - 0.5) / kNGamma;
  double smax = std::atanh(gh_max) + 30.0 / (L - 1.0) + 3.0;
  smax = std::min(smax, 40.0);
  int panels = (int)std::ceil(smax * kSPanelsPerUnit);
  double pw = smax / panels;
  std::vector<double> gs, omgs, lw;  // g, 1-g, log(weight * dg/ds)
  for (int p = 0; p < panels; ++p)
    for (int k = 0; k < 8; ++k) {
      double s = pw * (p + 0.5) + 0.5 * pw * r8.x[k];
      double g = std::tanh(s);
      double omg = 2.0 / (std::exp(2.0 * s) + 1.0);
      double ch = std::cosh(s);
      gs.push_back(g);
      omgs.push_back(omg);
      lw.push_back(std::log(0.5 * pw * r8.w[k]) - 2.0 * std::log(ch));  // dg = sech^2 s ds
    }
  const int Q = (int)gs.size();
  // phase pdf table on eta_i = i pi / NH, i = 0..NH (even in eta)
  std::vector<double> F((size_t)(NH + 1) * Q);
  parallel_for(NH + 1, [&](long i) {
    double eta = i * kPi / NH;
    for (int q = 0; q < Q; ++q) F[(size_t)i * Q + q] = std::exp(log_phase_pdf(eta, gs[q], omgs[q], L, r24));
  });
  parallel_for(kNGamma, [&](long kg) {
    double gh = (kg + 0.5) / kNGamma;
    std::vector<double> lt(Q), wq(Q);
    double mx = -INFINITY;
    for (int q = 0; q < Q; ++q) {
      lt[q] = log_coh_pdf(gh, gs[q], omgs[q], L) + lw[q];
      mx = std::max(mx, lt[q]);
    }
    double Z = 0.0;
    for (int q = 0; q < Q; ++q) {
      wq[q] = std::exp(lt[q] - mx);
      Z += wq[q];
    }
    std::vector<double> f(2 * NH + 1);
    for (int i = 0; i <= NH; ++i) {
      double acc = 0.0;
      const double* row = &F[(size_t)i * Q];
      for (int q = 0; q < Q; ++q) acc += wq[q] * row[q];
      f[NH + i] = f[NH - i] = acc / Z;
    }
    RowTables R;
    row_tables(f, NH, R);
    std::vector<double> c(kNAlpha);
    row_costs(R, r12, c.data(), table + kg * kNAlpha, ratio100 + kg * kNAlpha);
    if (cost100)
      for (int j = 0; j < kNAlpha; ++j) cost100[kg * kNAlpha + j] = c[j];
  });
  return WW_OK;
}

}  // namespace ww
