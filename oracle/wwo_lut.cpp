// CPU oracle, Sec. II-B cost model in FP64: Eqs. (4)-(7).
// TEST INFRASTRUCTURE ONLY (see wwo.h).
//
// Densities
//   L-look phase pdf (Lee et al. 1994, cited in Sec. II-B).  Written here as the
//   equivalent one-dimensional integral
//     f(eta | g, L) = L (1-g^2)^L / (pi 2^L) * Int_0^inf cosh((L-1)t) / (cosh t - b)^(L+1) dt,
//   b = g cos(eta), obtained from the complex-Wishart joint density of the
//   sample covariance by integrating out the two powers (a K-Bessel kernel)
//   and using K_nu(u) = Int cosh(nu t) exp(-u cosh t) dt.  The tests pin it
//   against the hypergeometric closed form, the single-look closed form,
//   normalisation and Monte Carlo looks.
//   Sample-coherence pdf (Touzi et al. 1999, cited in Sec. II-B)
//     f(gh | g, L) = 2(L-1)(1-g^2)^L gh (1-gh^2)^(L-2) 2F1(L, L; 1; g^2 gh^2),
//   the 2F1 summed directly (all terms positive) in log space.
// Pipeline per (L, gh): Eq. (5) marginal pdf on a uniform eta grid, the edge
// noise Delta eta = eta_v - eta_u with pdf f~*f~ on [-2pi, 2pi], Eq. (6)
// q0/q+ as tail probabilities of Delta eta shifted by alpha, Eq. (7) Gaussian
// slope marginalisation over alpha-hat +- 8 sigma with weights normalised on
// that interval, Eq. (4) c = max(0, -ln(P+/P0)), stored as floor(100 c) in int16.
#include "wwo.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace {

const double kPi = 3.14159265358979323846;

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= n; ++j) {
        double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      double z1 = z;
      z = z1 - p1 / pp;
      if (std::fabs(z - z1) < 1e-16) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
}

struct GL {
  std::vector<double> x8, w8, x16, w16;
  GL() {
    gauss_legendre(8, x8, w8);
    gauss_legendre(16, x16, w16);
  }
};
const GL& gl() {
  static GL g;
  return g;
}

double log_cosh(double y) {
  y = std::fabs(y);
  return y + std::log1p(std::exp(-2.0 * y)) - std::log(2.0);
}

// Lee integral on a finite interval: with t = 2 asinh(a tan th), a^2 = (1-b)/2,
//   Int_0^inf cosh((L-1)t) (cosh t - b)^-(L+1) dt
//     = 2a (2a^2)^-(L+1) Int_0^{pi/2} cosh(2(L-1) asinh(a tan th)) cos^(2L+1) th
//                                     / sqrt(cos^2 th + a^2 sin^2 th) dth.
double lee_log_theta(double th, double a, double L) {
  double c = std::cos(th), s = std::sin(th);
  if (c <= 0.0) return -INFINITY;
  return log_cosh(2.0 * (L - 1.0) * std::asinh(a * s / c)) + (2.0 * L + 1.0) * std::log(c) -
         0.5 * std::log(c * c + a * a * s * s);
}

// Adaptive quadrature on [a, b]: 8- vs 16-point Gauss-Legendre, bisect on disagreement.
template <class F>
double adapt(F f, double a, double b, double tol, int depth) {
  const GL& g = gl();
  double c = 0.5 * (a + b), r = 0.5 * (b - a);
  double i8 = 0.0, i16 = 0.0;
  for (int k = 0; k < 8; ++k) i8 += g.w8[k] * f(c + r * g.x8[k]);
  for (int k = 0; k < 16; ++k) i16 += g.w16[k] * f(c + r * g.x16[k]);
  i8 *= r;
  i16 *= r;
  // accept at the requested tolerance, or once the two rules agree to rounding level
  double err = std::fabs(i16 - i8);
  if (depth <= 0 || err <= tol || err <= 1e-14 * std::fabs(i16)) return i16;
  return adapt(f, a, c, 0.5 * tol, depth - 1) + adapt(f, c, b, 0.5 * tol, depth - 1);
}

// omg = 1 - g carried separately so that 1 - b and 1 - g^2 keep full relative
// precision as g -> 1: 1 - b = omg + 2 g sin^2(eta/2), 1 - g^2 = omg (1 + g).
double lee_log_pdf(double eta, double g, double omg, double L) {
  double sh = std::sin(0.5 * eta);
  double a = std::sqrt(0.5 * (omg + 2.0 * g * sh * sh));
  const double half_pi = 0.5 * kPi;
  double hmax = -INFINITY;
  for (int k = 0; k < 64; ++k) hmax = std::max(hmax, lee_log_theta(half_pi * k / 64.0, a, L));
  auto f = [&](double th) { return std::exp(lee_log_theta(th, a, L) - hmax); };
  double total = 0.0;
  for (int p = 0; p < 4; ++p) total += adapt(f, half_pi * p / 4.0, half_pi * (p + 1) / 4.0, 1e-15, 24);
  double log_int = std::log(2.0 * a) - (L + 1.0) * std::log(2.0 * a * a) + hmax + std::log(total);
  double logc = std::log(L) + L * (std::log(omg) + std::log1p(g)) - std::log(kPi) - L * std::log(2.0);
  return logc + log_int;
}

// log 2F1(L, L; 1; z), all terms positive: t_k = t_{k-1} ((L+k-1)/k)^2 z, t_0 = 1.
// Summed in linear space with a running power-of-two rescale against overflow.
double log_hyp_LL1(double L, double z) {
  if (z <= 0.0) return 0.0;
  double t = 1.0, sum = 1.0, log_scale = 0.0;
  for (long k = 1; k < 100000000; ++k) {
    double r = (L + k - 1.0) / k;
    t *= r * r * z;
    sum += t;
    if (sum > 1e280) {
      t *= 1e-280;
      sum *= 1e-280;
      log_scale += 280.0 * std::log(10.0);
    }
    if (k > L && t < 1e-18 * sum) break;
  }
  return std::log(sum) + log_scale;
}

double touzi_log_pdf(double gh, double g, double omg, double L) {
  return std::log(2.0 * (L - 1.0)) + L * (std::log(omg) + std::log1p(g)) + std::log(gh) +
         (L - 2.0) * std::log1p(-gh * gh) + log_hyp_LL1(L, g * g * gh * gh);
}

// 4th-order integral over [x_i, x_{i+1}] of tabulated y (uniform spacing h)
// from the cubic through 4 neighbours; one-sided at the ends; trapezoid if < 4 points.
double interval_int(const double* y, long count, long i, double h) {
  if (count < 4) return 0.5 * h * (y[i] + y[i + 1]);
  double v;
  if (i == 0)
    v = h / 24.0 * (9.0 * y[0] + 19.0 * y[1] - 5.0 * y[2] + y[3]);
  else if (i == count - 2)
    v = h / 24.0 * (9.0 * y[i + 1] + 19.0 * y[i] - 5.0 * y[i - 1] + y[i - 2]);
  else
    v = h / 24.0 * (-y[i - 1] + 13.0 * y[i] + 13.0 * y[i + 1] - y[i + 2]);
  double lo = 0.0;
  return std::max(v, lo);
}

double integrate_tab(const double* y, long count, double h) {
  double s = 0.0;
  for (long i = 0; i + 1 < count; ++i) s += interval_int(y, count, i, h);
  return s;
}

struct Tables {
  int nh;
  double h;
  std::vector<double> f;   // pdf on x_i = -pi + i h, i = 0..2nh
  std::vector<double> St;  // P(eta > x_i)
  std::vector<double> Sg;  // P(Delta eta > s_k), s_k = k h, k = 0..2nh
  std::vector<double> lSg; // log Sg (or -inf)
  double sigma;
};

void build_tables(const double* f_in, int nh, Tables& T) {
  T.nh = nh;
  T.h = kPi / nh;
  const long N = 2L * nh + 1;
  T.f.assign(f_in, f_in + N);
  // normalise the tabulated pdf
  double z = integrate_tab(T.f.data(), N, T.h);
  for (double& v : T.f) v /= z;
  // survival of the single-pixel noise, summed from the +pi end
  T.St.assign(N, 0.0);
  for (long i = N - 2; i >= 0; --i) T.St[i] = T.St[i + 1] + interval_int(T.f.data(), N, i, T.h);
  // Delta eta = eta_v - eta_u: P(Delta eta > s) = Int f(x) P(eta > x + s) dx
  const long K = 2L * nh;
  T.Sg.assign(K + 1, 0.0);
  std::vector<double> prod(N);
  for (long k = 0; k <= K; ++k) {
    if (k >= N - 1) {
      T.Sg[k] = 0.0;
      continue;
    }
    long cnt = N - k;  // x_i with x_i + s_k <= pi
    for (long i = 0; i < cnt; ++i) prod[i] = T.f[i] * T.St[i + k];
    T.Sg[k] = integrate_tab(prod.data(), cnt, T.h);
  }
  T.Sg[0] = 0.5;  // exact by symmetry of Delta eta
  T.lSg.assign(K + 1, -INFINITY);
  for (long k = 0; k <= K; ++k)
    if (T.Sg[k] > 0) T.lSg[k] = std::log(T.Sg[k]);
  // sigma_alpha^2 = E[wrap(Delta eta)^2] with g = f*f (pdf of Delta eta)
  std::vector<double> w2g(K + 1, 0.0);
  for (long k = 0; k <= K && k < N; ++k) {
    long cnt = N - k;
    for (long i = 0; i < cnt; ++i) prod[i] = T.f[i] * T.f[i + k];
    double gk = integrate_tab(prod.data(), cnt, T.h);
    double s = k * T.h;
    double wv = s <= kPi ? s : s - 2.0 * kPi;
    w2g[k] = wv * wv * gk;
  }
  // wrap(s)^2 has a kink at s = pi: integrate [0, pi] and [pi, 2pi] separately
  T.sigma = std::sqrt(2.0 * (integrate_tab(w2g.data(), nh + 1, T.h) +
                             integrate_tab(w2g.data() + nh, nh + 1, T.h)));
}

// P(Delta eta > s) at any s, by 6-point Lagrange interpolation of log Sg.
double Sg_at(const Tables& T, double s) {
  const double twopi = 2.0 * kPi;
  if (s >= twopi) return 0.0;
  if (s <= -twopi) return 1.0;
  if (s < 0.0) return 1.0 - Sg_at(T, -s);
  const long K = 2L * T.nh;
  double u = s / T.h;
  long i0 = (long)std::floor(u) - 2;
  i0 = std::max(0L, std::min(i0, K - 5));
  bool logok = true;
  for (long j = 0; j < 6; ++j)
    if (!(T.Sg[i0 + j] > 0)) logok = false;
  double acc = 0.0;
  for (long j = 0; j < 6; ++j) {
    double lj = 1.0;
    for (long q = 0; q < 6; ++q)
      if (q != j) lj *= (u - (i0 + q)) / (double)(j - q);
    acc += lj * (logok ? T.lSg[i0 + j] : T.Sg[i0 + j]);
  }
  if (logok) return std::exp(acc);
  return std::max(acc, 0.0);
}

void probabilities(const Tables& T, double ah, double* p0, double* pp, double* pm) {
  const GL& g = gl();
  const double sg = T.sigma;
  const int panels = 96;
  double a = ah - 8.0 * sg, b = ah + 8.0 * sg;
  // q+(alpha) = P(Delta eta > pi - alpha) is zero for alpha <= -pi (|Delta eta| <= 2pi)
  // and q-(alpha) for alpha >= pi; their second derivatives jump there, so the
  // interval is split at -pi and pi and each piece gets its own panels.
  double cuts[4] = {a, 0.0, 0.0, b};
  int nc = 1;
  if (-kPi > a && -kPi < b) cuts[nc++] = -kPi;
  if (kPi > a && kPi < b) cuts[nc++] = kPi;
  cuts[nc] = b;
  double W = 0.0, S0 = 0.0, Sp = 0.0, Sm = 0.0;
  for (int piece = 0; piece < nc; ++piece) {
    const double lo = cuts[piece], hi = cuts[piece + 1];
    const int np = std::max(8, (int)std::ceil(panels * (hi - lo) / (b - a)));
    const double hw = (hi - lo) / np;
    for (int p = 0; p < np; ++p) {
      double c = lo + (p + 0.5) * hw;
      for (int k = 0; k < 16; ++k) {
        double al = c + 0.5 * hw * g.x16[k];
        double wt = 0.5 * hw * g.w16[k] * std::exp(-0.5 * (al - ah) * (al - ah) / (sg * sg));
        double qp = Sg_at(T, kPi - al);  // G = alpha + Delta eta > pi
        double qm = Sg_at(T, kPi + al);  // G <= -pi
        double q0 = 1.0 - qp - qm;
        if (q0 < 0) q0 = 0;
        W += wt;
        S0 += wt * q0;
        Sp += wt * qp;
        Sm += wt * qm;
      }
    }
  }
  *p0 = S0 / W;
  *pp = Sp / W;
  *pm = Sm / W;
}

int lambda_nodes(double L, int panels_per_unit, std::vector<double>& lam, std::vector<double>& wl) {
  const GL& g = gl();
  double gh_max = 127.5 / 128.0;
  double Lmax = std::max(8.0, -std::log(1.0 - gh_max) + 45.0 / (L - 1.0 + 1e-9) + 4.0);
  Lmax = std::min(Lmax, 60.0);
  int panels = (int)std::ceil(Lmax * panels_per_unit);
  double hw = Lmax / panels;
  lam.clear();
  wl.clear();
  for (int p = 0; p < panels; ++p)
    for (int k = 0; k < 8; ++k) {
      lam.push_back((p + 0.5) * hw + 0.5 * hw * g.x8[k]);
      wl.push_back(0.5 * hw * g.w8[k]);
    }
  return (int)lam.size();
}

// Eq. (5) on the symmetric grid, given a precomputed table F[i][q] = f(eta_i | gamma_q)
// for eta_i = i pi / nh, i = 0..nh.
void marginal_from_table(const std::vector<double>& F, int nh, const std::vector<double>& lam,
                         const std::vector<double>& wl, double L, double gh, double* out) {
  const int Q = (int)lam.size();
  std::vector<double> W(Q);
  std::vector<double> lt(Q);
  double lmax = -INFINITY;
  for (int q = 0; q < Q; ++q) {
    double g = -std::expm1(-lam[q]);
    lt[q] = touzi_log_pdf(gh, g, std::exp(-lam[q]), L) - lam[q] + std::log(wl[q]);  // dgamma = e^-lambda dlambda
    lmax = std::max(lmax, lt[q]);
  }
  double Z = 0.0;
  for (int q = 0; q < Q; ++q) {
    W[q] = std::exp(lt[q] - lmax);
    Z += W[q];
  }
  for (int i = 0; i <= nh; ++i) {
    double s = 0.0;
    for (int q = 0; q < Q; ++q) s += W[q] * F[(size_t)i * Q + q];
    s /= Z;
    out[nh + i] = s;
    out[nh - i] = s;
  }
}

void lee_table(double L, int nh, const std::vector<double>& lam, std::vector<double>& F) {
  const int Q = (int)lam.size();
  F.assign((size_t)(nh + 1) * Q, 0.0);
  for (int i = 0; i <= nh; ++i) {
    double eta = i * kPi / nh;
    for (int q = 0; q < Q; ++q) {
      double g = -std::expm1(-lam[q]);
      F[(size_t)i * Q + q] = std::exp(lee_log_pdf(eta, g, std::exp(-lam[q]), L));
    }
  }
}

}  // namespace

extern "C" {

double wwo_lee_pdf(double eta, double gamma, double L) {
  if (gamma >= 1.0) return 0.0;
  return std::exp(lee_log_pdf(eta, gamma, 1.0 - gamma, L));
}

double wwo_touzi_pdf(double gh, double gamma, double L) {
  if (gh <= 0.0 || gh >= 1.0 || gamma >= 1.0) return 0.0;
  return std::exp(touzi_log_pdf(gh, gamma, 1.0 - gamma, L));
}

int wwo_marginal_pdf(double L, double gh, int32_t nh, int32_t lambda_panels, double* f) {
  if (!(L > 1.0) || nh < 4) return -1;
  std::vector<double> lam, wl, F;
  lambda_nodes(L, lambda_panels, lam, wl);
  lee_table(L, nh, lam, F);
  marginal_from_table(F, nh, lam, wl, L, gh, f);
  return 0;
}

double wwo_sigma_from_pdf(const double* f, int32_t nh) {
  Tables T;
  build_tables(f, nh, T);
  return T.sigma;
}

void wwo_probabilities(const double* f, int32_t nh, double alpha_hat, double* p0, double* pplus,
                       double* pminus, double* sigma) {
  Tables T;
  build_tables(f, nh, T);
  probabilities(T, alpha_hat, p0, pplus, pminus);
  *sigma = T.sigma;
}

int wwo_lut_build(double L, int32_t nh, int32_t lambda_panels, double* cost100, int16_t* table, float* ratio100) {
  if (!(L > 1.0) || nh < 16) return -1;
  std::vector<double> lam, wl, F;
  lambda_nodes(L, lambda_panels, lam, wl);
  lee_table(L, nh, lam, F);
  std::vector<double> f(2 * nh + 1);
  for (int k = 0; k < 128; ++k) {
    double gh = (k + 0.5) / 128.0;  // bin centres
    marginal_from_table(F, nh, lam, wl, L, gh, f.data());
    Tables T;
    build_tables(f.data(), nh, T);
    for (int j = 0; j < 256; ++j) {
      double ah = -kPi + (j + 0.5) * (2.0 * kPi / 256.0);
      double p0, pp, pm;
      probabilities(T, ah, &p0, &pp, &pm);
      double c100;
      if (!(pp > 0.0))
        c100 = INFINITY;
      else if (!(p0 > 0.0))
        c100 = 0.0;
      else
        c100 = std::max(0.0, -100.0 * std::log(pp / p0));
      cost100[k * 256 + j] = c100;
      double fl = std::floor(c100);
      table[k * 256 + j] = (int16_t)(fl >= 32767.0 ? 32767 : (int)fl);
      if (ratio100) {
        // 100 ln(P0/P+) before the max and the floor, for interpolated lookup;
        // P+ = 0 saturates, P0 = 0 gives the lower bound
        double r = !(pp > 0.0) ? 32767.0 : (!(p0 > 0.0) ? -10000.0 : -100.0 * std::log(pp / p0));
        ratio100[k * 256 + j] = (float)std::min(32767.0, std::max(-10000.0, r));
      }
    }
  }
  return 0;
}

}  // extern "C"
