"""Pins for the oracle's preprocessing steps: multilooking with the Eq. (3)
sample coherence, the adaptive power-spectrum (Goldstein) filter, and the
transfer of integer cycles from a filtered phase to the original one
(Sec. II-B Eq. 3, Sec. II-D)."""
import numpy as np
import pytest

import oracle
from paper_2609_36267_b300 import synth


def slc_pair(seed, M, N, gamma, phi):
    rng = np.random.default_rng(seed)
    x = (rng.normal(size=(M, N)) + 1j * rng.normal(size=(M, N))) / np.sqrt(2)
    y = (rng.normal(size=(M, N)) + 1j * rng.normal(size=(M, N))) / np.sqrt(2)
    z1 = x
    z2 = (gamma * x + np.sqrt(1 - gamma ** 2) * y) * np.exp(-1j * phi)
    return z1.astype(np.complex64), z2.astype(np.complex64)


def test_multilook_matches_float64_sums():
    z1, z2 = slc_pair(1, 40, 66, 0.7, 0.4)
    ifg, coh = oracle.multilook(z1, z2, 4, 6)
    a, b = z1.astype(np.complex128), z2.astype(np.complex128)
    S12 = (a * np.conj(b)).reshape(10, 4, 11, 6).sum(axis=(1, 3))
    S11 = (np.abs(a) ** 2).reshape(10, 4, 11, 6).sum(axis=(1, 3))
    S22 = (np.abs(b) ** 2).reshape(10, 4, 11, 6).sum(axis=(1, 3))
    assert np.allclose(ifg, S12, rtol=2e-6, atol=2e-6 * np.abs(S12).max())
    assert np.allclose(coh, np.abs(S12) / np.sqrt(S11 * S22), atol=2e-6)


def test_multilook_coherence_special_cases():
    rng = np.random.default_rng(2)
    z1 = (rng.normal(size=(30, 30)) + 1j * rng.normal(size=(30, 30))).astype(np.complex64)
    # proportional images: gamma = 1 (to rounding), phase = -arg(c)
    c = np.complex64(0.3 - 1.7j)
    ifg, coh = oracle.multilook(z1, (z1 * c).astype(np.complex64), 3, 5)
    assert np.all(np.abs(coh - 1) < 1e-5) and np.all(coh <= 1)
    assert np.allclose(np.angle(ifg), -np.angle(c), atol=1e-5)
    # a zero image: coherence 0
    _, coh0 = oracle.multilook(z1, np.zeros_like(z1), 3, 5)
    assert not coh0.any()
    # trailing rows and columns that do not fill a look window are dropped
    ifg2, _ = oracle.multilook(z1[:29, :28], z1[:29, :28], 3, 5)
    assert ifg2.shape == (9, 5)


def test_multilook_sample_coherence_distribution():
    """Eq. (3) over L looks estimates gamma: for L = 20 the mean of the sample
    coherence at gamma = 0.6 lies close to the Touzi density's mean."""
    z1, z2 = slc_pair(3, 400, 400, 0.6, 1.0)
    _, coh = oracle.multilook(z1, z2, 4, 5)
    from scipy import integrate
    mean = integrate.quad(lambda x: x * oracle.touzi_pdf(x, 0.6, 20.0), 0, 1)[0]
    assert abs(coh.mean() - mean) < 0.01


def test_goldstein_keeps_a_pure_fringe_and_reduces_noise():
    """A fringe on a DFT frequency of the 32-pixel patches occupies one bin of
    every whole patch, which the filter passes unchanged; pixels reached only by
    the zero-padded patches at the far edges are excluded."""
    m, n = 96, 112
    ii, jj = np.mgrid[0:m, 0:n]
    phase = 2 * np.pi * (3 * jj + 2 * ii) / 32
    clean = np.exp(1j * phase)
    out = oracle.goldstein(clean, alpha=0.8)
    inner = (slice(0, m - 32), slice(0, n - 32))
    assert np.max(np.abs(np.angle(out * np.conj(clean)))[inner]) < 1e-9
    rng = np.random.default_rng(4)
    clean = np.exp(1j * (0.35 * jj + 0.2 * ii))
    noisy = clean * np.exp(1j * rng.normal(0, 0.8, (m, n)))
    filt = oracle.goldstein(noisy, alpha=0.8)
    err_in = np.abs(np.angle(noisy * np.conj(clean))).mean()
    err_out = np.abs(np.angle(filt * np.conj(clean))).mean()
    assert err_out < 0.6 * err_in


def test_goldstein_alpha_zero_is_the_identity():
    """alpha = 0: every patch passes unchanged (H = 1), and the weighted overlap
    sum divided by the weights gives back the input."""
    rng = np.random.default_rng(5)
    z = rng.normal(size=(50, 70)) + 1j * rng.normal(size=(50, 70))
    out = oracle.goldstein(z, alpha=0.0)
    assert np.allclose(out, z, atol=1e-12)


def test_transfer_cycles():
    x = synth.small_random(8, 40, 50, lo=0.3, hi=0.95)
    psi, _, valid = oracle.prepare(x.coh, x.mask, phase=x.phase)
    rng = np.random.default_rng(1)
    K = rng.integers(-5, 6, size=psi.shape)
    filt = (psi.astype(np.float64) + 2 * np.pi * K + rng.uniform(-0.5, 0.5, psi.shape)).astype(np.float32)
    out, Kt = oracle.transfer_cycles(filt, psi, valid)
    v = valid.astype(bool)
    assert np.array_equal(Kt[v], K[v])
    want = (psi.astype(np.float64) + 6.283185307179586 * K).astype(np.float32)
    assert np.array_equal(out[v], want[v])
    assert np.isnan(out[~v]).all()
