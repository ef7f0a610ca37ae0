"""Independent FP64 evaluation of the cost model's probabilities (Sec. II-B,
Eqs. 5-7), used only to pin the oracle's cost tables.

It shares no numerical design with the oracle (oracle/wwo_lut.cpp) or with the
library: no uniform phase grid, no tabulated tail, no interpolation and no
change of variable in the coherence integral.

* Lee's L-look phase density f(eta | g, L) (cited in Sec. II-B).  For
  b = g cos(eta) >= 0 its hypergeometric closed form is a sum of two positive
  terms and is evaluated directly (scipy's 2F1).  For b < 0 the two terms
  cancel, so the density is taken from the complex-Wishart law of the sample
  covariance instead: integrating the joint density of the two powers and the
  cross product over the powers leaves
      f(eta) = (1-g^2)^L / (pi Gamma(L) 2^L) Int_0^inf r^L K_{L-1}(r) e^{b r} dr,
  a positive integrand (composite Gauss-Legendre in r).
* Touzi's sample-coherence density by its hypergeometric closed form.
* Eq. 5: the coherence marginal (uniform prior on g) by composite
  Gauss-Legendre in g itself, on panels that narrow geometrically toward g = 1.
* The edge noise Delta eta = eta_v - eta_u of two independent pixels (density
  f~*f~, support [-2pi, 2pi]) is never formed: Eqs. 6-7 are evaluated as one
  double integral over the two pixels' phase errors (x, y) on a product
  Gauss-Legendre grid, with the Gaussian slope of Eq. 7 (truncated to
  alpha-hat +- 8 sigma and renormalised there) integrated in closed form:
      P+ = E_{x,y}[ P(alpha > pi - (y - x)) ],
      P0 = E_{x,y}[ P(-pi - (y - x) < alpha <= pi - (y - x)) ],
  which by Fubini equals Int q_j(alpha) N(alpha) dalpha with q+ and q0 the
  tail and centred integrals of Eq. 6.
* sigma_alpha^2 = E[wrap(Delta eta)^2] (the reading whose limit is the pi^2/3
  the paper states) from the Fourier series of the periodic function wrap(d)^2,
      wrap(d)^2 = pi^2/3 + 4 sum_k (-1)^k cos(k d) / k^2,
  so sigma^2 = pi^2/3 + 4 sum_k (-1)^k a_k^2 / k^2 with a_k = E[cos(k eta)].
"""
from __future__ import annotations

import numpy as np
from scipy import special as sp

# coherence panels: uniform on [0, 1/2], then edges 1 - 2^-(1 + j/8)
_G_UNIFORM_PANELS = 25
_G_GEOMETRIC_PANELS = 150


def gl_panels(a: float, b: float, panels: int, order: int):
    """Nodes and weights of composite Gauss-Legendre on [a, b]."""
    x, w = np.polynomial.legendre.leggauss(order)
    e = np.linspace(a, b, panels + 1)
    c = 0.5 * (e[:-1] + e[1:])
    h = 0.5 * (e[1:] - e[:-1])
    return (c[:, None] + h[:, None] * x[None]).ravel(), (h[:, None] * w[None]).ravel()


def lee_log_pdf(eta: np.ndarray, g: np.ndarray, L: float) -> np.ndarray:
    """log f(eta_i | g_j, L) for 1-D arrays eta, g (0 <= g < 1) -> [i, j]."""
    eta = np.atleast_1d(np.asarray(eta, np.float64))
    g = np.atleast_1d(np.asarray(g, np.float64))
    beta = g[None, :] * np.cos(eta)[:, None]
    out = np.empty(beta.shape)
    pos = beta >= 0
    b = beta[pos]
    with np.errstate(divide="ignore"):
        lt1 = (sp.gammaln(L + 0.5) - sp.gammaln(L) - np.log(2 * np.sqrt(np.pi)) + np.log(b)
               - (L + 0.5) * np.log1p(-b * b))
    t1 = np.where(b > 0, np.exp(lt1), 0.0)
    t2 = sp.hyp2f1(L, 1.0, 0.5, b * b) / (2 * np.pi)
    out[pos] = np.log(t1 + t2)
    neg = ~pos
    b = beta[neg]
    R = L + 30 * np.sqrt(L) + 80
    r, wr = gl_panels(0.0, R, 25, 16)
    lk = L * np.log(r) + np.log(sp.kve(L - 1, r)) - r + np.log(wr)  # K = kve e^-r
    vals = np.empty(b.size)
    for s in range(0, b.size, 20000):
        z = lk[None, :] + b[s:s + 20000, None] * r[None, :]
        zm = z.max(axis=1)
        vals[s:s + 20000] = zm + np.log(np.exp(z - zm[:, None]).sum(axis=1))
    out[neg] = vals - sp.gammaln(L) - L * np.log(2) - np.log(np.pi)
    return out + L * np.log1p(-g[None, :] ** 2)


def touzi_log_pdf(gh: float, g: np.ndarray, L: float) -> np.ndarray:
    """log f(gh | g, L): 2(L-1)(1-g^2)^L gh (1-gh^2)^(L-2) 2F1(L, L; 1; g^2 gh^2)."""
    g = np.asarray(g, np.float64)
    return (np.log(2 * (L - 1)) + L * np.log1p(-g ** 2) + np.log(gh) + (L - 2) * np.log1p(-gh * gh)
            + np.log(sp.hyp2f1(L, L, 1.0, g ** 2 * gh ** 2)))


def coherence_nodes(order: int = 8):
    edges = np.concatenate([np.linspace(0.0, 0.5, _G_UNIFORM_PANELS + 1),
                            1.0 - 0.5 * 2.0 ** (-np.arange(1, _G_GEOMETRIC_PANELS + 1) / 8.0)])
    x, w = np.polynomial.legendre.leggauss(order)
    c = 0.5 * (edges[:-1] + edges[1:])
    h = 0.5 * (edges[1:] - edges[:-1])
    return (c[:, None] + h[:, None] * x[None]).ravel(), (h[:, None] * w[None]).ravel()


class Marginals:
    """Eq. 5 marginal densities f~(x | gh, L) at Gauss-Legendre nodes x of [-pi, pi]."""

    def __init__(self, L: float, eta_panels: int = 400, eta_order: int = 8):
        self.L = float(L)
        self.x, self.wx = gl_panels(-np.pi, np.pi, eta_panels, eta_order)
        self.half = self.x >= 0  # panels are symmetric: the x < 0 half mirrors x >= 0
        self.g, self.wg = coherence_nodes()
        self.F = lee_log_pdf(self.x[self.half], self.g, self.L)  # [x >= 0, g]
        self.Fmax = self.F.max(axis=1)

    def pdf(self, gh: float) -> np.ndarray:
        lw = touzi_log_pdf(gh, self.g, self.L) + np.log(self.wg)
        W = np.exp(lw - lw.max())
        fh = (np.exp(self.F - self.Fmax[:, None]) * W[None, :]).sum(axis=1) / W.sum()
        lf = np.log(fh) + self.Fmax
        f = np.empty(self.x.size)
        f[self.half] = np.exp(lf)
        f[~self.half] = np.exp(lf)[::-1]
        return f


def sigma_alpha(x: np.ndarray, wx: np.ndarray, f: np.ndarray) -> float:
    """sqrt(E[wrap(eta_v - eta_u)^2]) from the Fourier coefficients of f."""
    p = wx * f / np.sum(wx * f)
    ks = np.arange(1, x.size // 4 + 1)  # well inside what the nodes resolve
    a = np.cos(np.outer(ks, x)) @ p
    small = np.nonzero(np.abs(a) < 1e-11)[0]
    if not small.size:
        raise ValueError("phase grid too coarse for this density's Fourier coefficients")
    K = small[0]  # beyond here a_k^2 / k^2 < 1e-22
    return float(np.sqrt(np.pi ** 2 / 3 + 4 * np.sum(((-1.0) ** ks * a * a / ks ** 2)[:K])))


def probabilities(x: np.ndarray, wx: np.ndarray, f: np.ndarray, alpha_hat: float):
    """-> (P0, P+, sigma_alpha) of Eqs. 6-7 for the marginal density f at nodes x."""
    sig = sigma_alpha(x, wx, f)
    p = wx * f / np.sum(wx * f)
    z = sp.ndtr(8.0) - sp.ndtr(-8.0)

    def below(t):  # P(alpha <= t), alpha ~ N(alpha_hat, sig) on alpha_hat +- 8 sig
        u = np.clip((t - alpha_hat) / sig, -8.0, 8.0)
        return (sp.ndtr(u) - sp.ndtr(-8.0)) / z

    def above(t):  # P(alpha > t), as an upper-tail difference
        u = np.clip((t - alpha_hat) / sig, -8.0, 8.0)
        return (sp.ndtr(-u) - sp.ndtr(-8.0)) / z

    P0 = Pp = 0.0
    for s in range(0, x.size, 1024):
        d = x[None, :] - x[s:s + 1024, None]  # y - x, rows x_i, columns y_j
        w = p[s:s + 1024, None] * p[None, :]
        Pp += float(np.sum(w * above(np.pi - d)))
        P0 += float(np.sum(w * (below(np.pi - d) - below(-np.pi - d))))
    return P0, Pp, sig


def cost100(P0: float, Pp: float) -> float:
    """100 c of Eq. 4 (before flooring): max(0, -100 ln(P+/P0))."""
    return max(0.0, -100.0 * np.log(Pp / P0))


def bin_centres(k: int, j: int):
    """(gamma-hat, alpha-hat) at the centre of coherence bin k and slope bin j."""
    return (k + 0.5) / 128.0, -np.pi + (j + 0.5) * 2.0 * np.pi / 256.0
