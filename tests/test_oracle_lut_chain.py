"""Pins of the oracle's Eqs. 5-7 chain against an independent quadrature.

The oracle builds P0 and P+ by tabulating the coherence marginal (Eq. 5) on a
uniform phase grid, convolving it with itself, interpolating the tail of the
edge noise (Eq. 6) and integrating it against the Gaussian slope (Eq. 7).
tests/lut_reference.py evaluates the same probabilities with none of those
steps (closed forms and a Wishart integral for the densities, Gauss-Legendre in
the coherence itself, one product-quadrature double integral for Eqs. 6-7, a
Fourier series for sigma_alpha).  A dropped convolution, the wrong tail, a
mis-shifted slope or a wrong sigma would separate the two by far more than the
tolerances here.  The reference's own densities are first pinned to the
hypergeometric closed forms the paper cites (Sec. II-B)."""
import os

import numpy as np
import pytest

import lut_reference as R
import oracle
from test_oracle_lut import lee_closed_form, touzi_closed_form

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("eta,g,L", [(2.0, 0.8, 9), (3.1, 0.999, 50), (2.7, 0.9, 6), (1.7, 0.99, 50),
                                     (0.3, 0.5, 4), (0.0, 0.95, 50), (1.5, 0.3, 16), (2.2, 0.6, 4.5)])
def test_reference_lee_density_matches_closed_form(eta, g, L):
    """Both branches of the reference's Lee density (closed form for cos(eta) >= 0,
    Wishart integral where the closed form cancels) against the
    hypergeometric form evaluated with enough digits."""
    v = float(np.exp(R.lee_log_pdf(np.array([eta]), np.array([g]), L))[0, 0])
    assert v == pytest.approx(lee_closed_form(eta, g, L), rel=1e-11)


@pytest.mark.parametrize("gh,g,L", [(0.3, 0.5, 4), (0.9, 0.8, 9), (0.99, 0.99, 50), (0.05, 0.3, 16)])
def test_reference_touzi_density_matches_closed_form(gh, g, L):
    v = float(np.exp(R.touzi_log_pdf(gh, np.array([g]), L))[0])
    assert v == pytest.approx(touzi_closed_form(gh, g, L), rel=1e-11)


def test_reference_sigma_uniform_limit():
    """Sec. II-B: sigma_alpha -> pi/sqrt(3) as the phase noise becomes uniform
    (every Fourier coefficient vanishes)."""
    x, wx = R.gl_panels(-np.pi, np.pi, 50, 8)
    assert R.sigma_alpha(x, wx, np.full(x.size, 1 / (2 * np.pi))) == pytest.approx(np.pi / np.sqrt(3), rel=1e-14)


@pytest.fixture(scope="module")
def marg9():
    return R.Marginals(9.0)


@pytest.mark.parametrize("k", [6, 64])
def test_oracle_probabilities_match_independent_quadrature(marg9, k):
    """P0 and P+ (each separately, P0 as the centred integral) and sigma_alpha
    of the oracle at L = 9 against the reference, 1e-7 relative."""
    gh = (k + 0.5) / 128
    f = marg9.pdf(gh)
    fo = oracle.marginal_pdf(9.0, gh, nh=512, lambda_panels=8)
    for j in (0, 60, 128, 250):
        ah = R.bin_centres(k, j)[1]
        P0, Pp, sig = R.probabilities(marg9.x, marg9.wx, f, ah)
        o = oracle.probabilities(fo, ah)
        assert o["pplus"] == pytest.approx(Pp, rel=1e-7), (k, j)
        assert o["p0"] == pytest.approx(P0, rel=1e-7), (k, j)
        assert o["sigma"] == pytest.approx(sig, rel=1e-9)


# (L, [(coherence bin k, slope bin j)]): gamma-hat near 0.05, 0.5 and 0.95,
# alpha-hat near -pi, 0 and +pi
POINTS = {
    4.0: [(6, 1), (64, 128), (121, 254)],
    9.0: [(121, 0), (64, 200)],
    50.0: [(6, 0), (6, 128), (6, 254), (64, 1), (64, 128), (64, 255), (121, 40), (121, 128), (121, 254)],
}


@pytest.mark.parametrize("L", sorted(POINTS))
def test_golden_tables_match_independent_quadrature(L, marg9):
    """The stored oracle tables (tests/golden) against the reference at bin
    centres: 100 c within 2e-5, i.e. P+/P0 within 2e-7 relative."""
    M = marg9 if L == 9.0 else R.Marginals(L)
    z = np.load(os.path.join(GOLDEN, f"lut_oracle_L{L:g}.npz"))
    for k, j in POINTS[L]:
        gh, ah = R.bin_centres(k, j)
        P0, Pp, _ = R.probabilities(M.x, M.wx, M.pdf(gh), ah)
        want = R.cost100(P0, Pp)
        assert z["cost100"][k, j] == pytest.approx(want, abs=2e-5), (L, k, j)
        assert z["table"][k, j] == min(32767, int(np.floor(want))), (L, k, j)
