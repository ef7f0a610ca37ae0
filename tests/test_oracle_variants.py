"""Pins for the oracle's cost-model variants (Sec. II-B leaves the slope
estimator's form and the runtime lookup open): the complex-phasor slope
estimate against numpy's angle of the phasor sum and against the plain mean
for a constant gradient; the bilinear lookup against exact linear tables, the
table values at the bin centres, and its clamping at the grid's edges."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
PI_F = np.float32(np.pi)
A_SCALE = np.float32(256 / (2 * np.pi))


def wrapped_gradients(psi, valid):
    """fp32 wrapped gradients of the valid h and v edges (as the oracle forms them)."""
    m, n = psi.shape
    out = np.zeros((2, m, n), np.float32)
    ok = np.zeros((2, m, n), bool)
    for plane, (a, b) in enumerate(((psi[:, :-1], psi[:, 1:]), (psi[:-1, :], psi[1:, :]))):
        dp = (b - a).astype(np.float32)
        nc = (dp > PI_F).astype(np.float32) - (dp <= -PI_F).astype(np.float32)
        d = (dp - np.float32(2 * np.pi) * nc).astype(np.float32)
        if plane == 0:
            out[0, :, :-1], ok[0, :, :-1] = d, valid[:, :-1] & valid[:, 1:]
        else:
            out[1, :-1, :], ok[1, :-1, :] = d, valid[:-1, :] & valid[1:, :]
    return out, ok


@pytest.mark.parametrize("seed", range(4))
def test_phasor_slope_is_the_angle_of_the_phasor_sum(seed):
    rng = np.random.default_rng(seed)
    m, n, w = 23, 31, 2
    psi = rng.uniform(-np.pi, np.pi, (m, n)).astype(np.float32)
    if seed % 2:
        psi = np.cumsum(rng.normal(0, 0.7, (m, n)), axis=1).astype(np.float32)
        psi = (np.angle(np.exp(1j * psi))).astype(np.float32)
    valid = rng.uniform(size=(m, n)) > 0.1
    a = oracle.alpha_hat(psi, valid.astype(np.uint8), w, mode=1)
    d, ok = wrapped_gradients(psi, valid)
    for plane in range(2):
        for i in range(m):
            for j in range(n):
                if not ok[plane, i, j]:
                    assert a[plane, i, j] == 0.0
                    continue
                win = (slice(max(0, i - w), i + w + 1), slice(max(0, j - w), j + w + 1))
                z = np.sum(np.exp(1j * d[plane][win][ok[plane][win]].astype(np.float64)))
                want = np.angle(z)
                got = float(a[plane, i, j])
                err = abs(np.angle(np.exp(1j * (got - want))))
                # CORDIC quantisation (2^-29 rad steps, 2^30-length phasors) and one
                # fp32 rounding of each sum; near-cancelling sums are ill-conditioned
                assert err <= 2e-6 / max(abs(z) / 25, 1e-3), (plane, i, j, got, want, abs(z))


def test_phasor_slope_equals_the_mean_for_a_constant_gradient():
    m, n = 12, 15
    ii, jj = np.mgrid[0:m, 0:n]
    for gx, gy in ((0.3, -0.2), (-2.9, 1.1), (1.5, 3.0)):
        psi = np.angle(np.exp(1j * (gx * jj + gy * ii))).astype(np.float32)
        valid = np.ones((m, n), np.uint8)
        a1 = oracle.alpha_hat(psi, valid, 2, mode=1)
        a0 = oracle.alpha_hat(psi, valid, 2, mode=0)
        d, ok = wrapped_gradients(psi, valid.astype(bool))
        assert np.allclose(a1[ok], d[ok], atol=2e-6)
        assert np.allclose(a0[ok], d[ok], atol=2e-6)


def _costs_with_ratio(ratio, psi, coh, valid):
    return oracle.costs(psi, coh, valid, np.zeros((128, 256), np.int16), steep_rad=10.0, lookup=1, ratio=ratio)[0]


def test_bilinear_lookup_is_exact_on_a_linear_table():
    """Table 0.25 j + 3 k (exact in fp32): the interpolated value at slope position
    x and coherence position y is 0.25 x + 3 y, floored."""
    k = np.arange(128)[:, None]
    j = np.arange(256)[None, :]
    ratio = (0.25 * j + 3.0 * k).astype(np.float32)
    rng = np.random.default_rng(5)
    m, n = 20, 25
    psi = rng.uniform(-np.pi, np.pi, (m, n)).astype(np.float32)
    coh = rng.uniform(0.01, 0.99, (m, n)).astype(np.float32)
    valid = np.ones((m, n), np.uint8)
    c = _costs_with_ratio(ratio, psi, coh, valid)
    al = oracle.alpha_hat(psi, valid)
    for plane in range(2):
        g = np.minimum(coh[:, :-1], coh[:, 1:]) if plane == 0 else np.minimum(coh[:-1, :], coh[1:, :])
        a = al[0, :, :-1] if plane == 0 else al[1, :-1, :]
        got = c[2 * plane, :, :-1] if plane == 0 else c[2, :-1, :]
        x = np.clip((((a + PI_F) * A_SCALE).astype(np.float32) - np.float32(0.5)).astype(np.float64), 0, 255)
        y = np.clip(((g * np.float32(128)).astype(np.float32) - np.float32(0.5)).astype(np.float64), 0, 127)
        want = 0.25 * x + 3.0 * y
        near = np.abs(want - np.round(want)) < 1e-3
        assert np.array_equal(got[~near], np.floor(want[~near]).astype(np.int16))


def test_bilinear_lookup_at_bin_centres_and_edges():
    z = np.load(os.path.join(GOLDEN, "lut_oracle_L9.npz"))
    ratio, table = z["ratio100"], z["table"]
    # the table's own floors at the centres (where 100 c is not within 1e-3 of an integer)
    for kk, jj in ((3, 7), (64, 128), (100, 200), (127, 255), (0, 0)):
        g = np.float32((kk + 0.5) / 128)
        a = np.float32(-np.pi + (jj + 0.5) * 2 * np.pi / 256)
        psi = np.zeros((2, 2), np.float32)
        psi[:, 1] = a  # every h edge carries gradient a, so the 5x5 mean is a
        coh = np.full((2, 2), g, np.float32)
        c = _costs_with_ratio(ratio, psi, coh, np.ones((2, 2), np.uint8))
        r = float(ratio[kk, jj])
        if abs(r - round(r)) > 1e-3 and r < 32767:
            assert c[0, 0, 0] == max(0, int(np.floor(r))) == table[kk, jj], (kk, jj, c[0, 0, 0], r)
    # beyond the outermost centres the lookup holds the edge values (no extrapolation)
    psi = np.zeros((2, 2), np.float32)
    psi[:, 1] = PI_F
    coh = np.full((2, 2), np.float32(0.999), np.float32)
    c = _costs_with_ratio(ratio, psi, coh, np.ones((2, 2), np.uint8))
    assert c[0, 0, 0] == max(0, min(32767, int(np.floor(ratio[127, 255]))))
