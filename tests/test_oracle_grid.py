"""Pins for the oracle's grid steps: phase from complex, residues (Eq. 1),
slope estimate / LUT indices / costs (Sec. II-B), steep rule, integration."""
import numpy as np
import pytest

import oracle
from paper_2609_36267_b300 import synth

PI_F = np.float32(np.pi)
TWO_PI_F = np.float32(2 * np.pi)


def wrap64(x):
    return (x + np.pi) % (2 * np.pi) - np.pi


def f32_ulp(x):
    x = np.abs(np.asarray(x, np.float32))
    return np.spacing(np.maximum(x, np.float32(1e-30)))


# ---------------- complex -> phase (CORDIC) ----------------

def test_cordic_against_arctan2():
    rng = np.random.default_rng(7)
    z = (rng.standard_normal(200000) + 1j * rng.standard_normal(200000)).astype(np.complex64)
    z[:1000] *= np.float32(1e-30)
    z[1000:2000] *= np.float32(1e30)
    z[2000:3000] = (rng.standard_normal(1000) * 1e-6 + 1j * rng.standard_normal(1000)).astype(np.complex64)
    psi = oracle.phase_from_complex(z)
    ref = np.arctan2(z.imag.astype(np.float64), z.real.astype(np.float64))
    err = np.abs(psi.astype(np.float64) - ref)
    # fixed-point CORDIC: absolute error within 2e-8 rad, or 1 fp32 ulp at large angles
    err = np.minimum(err, np.abs(np.abs(err) - 2 * np.pi))
    assert np.all(err <= np.maximum(2e-8, f32_ulp(ref)))
    assert err.max() < 2.5e-7
    assert np.all(np.abs(psi) <= PI_F)


def test_cordic_axes_and_zero():
    z = np.array([1, 1j, -1, -1j, 0, 1 + 1j, -1 - 1j, -1 + 0j, 3e-39 + 0j], np.complex64)
    psi = oracle.phase_from_complex(z)
    expect = np.array([0, np.pi / 2, np.pi, -np.pi / 2, 0, np.pi / 4, -3 * np.pi / 4, np.pi, 0])
    assert np.allclose(psi, expect, atol=3e-7)
    assert psi[4] == 0.0


# ---------------- residues ----------------

def test_residue_vortex_positive_and_negative():
    m, n = 9, 11
    i0, j0 = 3.5, 6.5  # centre of loop (3, 6)
    i = np.arange(m)[:, None]
    j = np.arange(n)[None, :]
    for sign in (1, -1):
        psi = np.arctan2(sign * (i - i0), (j - j0)).astype(np.float32)
        r, g = oracle.residues(psi)
        nz = np.argwhere(r != 0)
        assert nz.tolist() == [[3, 6]]
        # going (i,j)->(i,j+1)->(i+1,j+1)->(i+1,j) the angle advances by +2pi
        assert r[3, 6] == sign
        assert g == -sign


def test_residues_zero_for_sub_nyquist_field():
    m, n = 64, 80
    i = np.arange(m)[:, None]
    j = np.arange(n)[None, :]
    truth = 0.9 * j + 0.4 * i + 3.0 * np.sin(i / 7.0) * np.cos(j / 9.0)
    psi = wrap64(truth).astype(np.float32)
    r, g = oracle.residues(psi)
    assert not r.any() and g == 0


def test_residues_match_real_valued_eq1_and_balance():
    x = synth.small_random(11, 40, 57, lo=0.05, hi=0.6)
    psi = x.phase
    r, g = oracle.residues(psi)
    assert int(r.sum()) + g == 0
    assert set(np.unique(r)).issubset({-2, -1, 0, 1, 2})
    # Eq. (1) evaluated literally in float64 from the fp32 phases
    p = psi.astype(np.float64)
    dh = wrap64(p[:, 1:] - p[:, :-1])
    dv = wrap64(p[1:, :] - p[:-1, :])
    loop = (dh[:-1, :] + dv[:, 1:] - dh[1:, :] - dv[:, :-1]) / (2 * np.pi)
    assert np.allclose(loop, np.round(loop), atol=1e-5)
    assert np.array_equal(np.round(loop).astype(np.int8), r)
    assert np.count_nonzero(r) > 20


# ---------------- slope estimate, indices, costs ----------------

def probe_table():
    k = np.arange(128)[:, None]
    j = np.arange(256)[None, :]
    return (k * 256 + j).astype(np.int16)


def decode(c):
    return c.astype(np.int64) // 256, c.astype(np.int64) % 256


def test_alpha_hat_constant_gradient():
    m, n = 20, 30
    j = np.arange(n)[None, :]
    for a in (0.3, -1.7, 2.9):
        psi = np.broadcast_to(wrap64(a * j), (m, n)).astype(np.float32).copy()
        valid = np.ones((m, n), np.uint8)
        al = oracle.alpha_hat(psi, valid)
        assert np.allclose(al[0][:, : n - 1], a, atol=2e-6)
        assert np.allclose(al[1][: m - 1, :], 0.0, atol=2e-6)


def test_alpha_and_gamma_bins_contain_values():
    rng = np.random.default_rng(3)
    m, n = 24, 31
    psi = rng.uniform(-np.pi, np.pi, (m, n)).astype(np.float32)
    coh = rng.uniform(0, 1, (m, n)).astype(np.float32)
    valid = np.ones((m, n), np.uint8)
    c, _ = oracle.costs(psi, coh, valid, probe_table(), steep_rad=10.0)
    al = oracle.alpha_hat(psi, valid)
    ig, ia = decode(c[0][:, : n - 1])
    a = al[0][:, : n - 1].astype(np.float64)
    centre = -np.pi + (ia + 0.5) * 2 * np.pi / 256
    assert np.all(np.abs(a - centre) <= np.pi / 256 + 1e-6)
    ge = np.minimum(coh[:, :-1], coh[:, 1:]).astype(np.float64)
    assert np.all(np.abs(ge - (ig + 0.5) / 128) <= 0.5 / 128 + 1e-7)
    # reverse arc uses -alpha-hat
    _, ia2 = decode(c[1][:, : n - 1])
    centre2 = -np.pi + (ia2 + 0.5) * 2 * np.pi / 256
    assert np.all(np.abs(-a - centre2) <= np.pi / 256 + 1e-6)


def test_index_formula_fixed_points():
    # a field whose box mean is exactly 0 lands in bin 128 (centre +pi/256), the
    # fp32 formula floor((0 + PI_F) * fp32(256/2pi)) = floor(128.0000028) = 128
    m, n = 8, 8
    psi = np.zeros((m, n), np.float32)
    coh = np.full((m, n), 0.999, np.float32)
    valid = np.ones((m, n), np.uint8)
    c, _ = oracle.costs(psi, coh, valid, probe_table())
    ig, ia = decode(c[0][:, :-1])
    assert np.all(ia == 128) and np.all(ig == 127)
    ig, ia = decode(c[1][:, :-1])
    assert np.all(ia == 128)


def test_costs_flip_symmetry():
    x = synth.small_random(5, 33, 41)
    psi, coh, valid = oracle.prepare(x.coh, x.mask, phase=x.phase)
    tab = probe_table()
    c, _ = oracle.costs(psi, coh, valid, tab, steep_rad=10.0)
    cf, _ = oracle.costs(psi[:, ::-1].copy(), coh[:, ::-1].copy(), valid[:, ::-1].copy(), tab, steep_rad=10.0)
    n = psi.shape[1]
    # h edge (i,j) maps to (i, n-2-j) with the gradient negated: +/- arcs swap
    assert np.array_equal(c[0][:, : n - 1], cf[1][:, : n - 1][:, ::-1])
    assert np.array_equal(c[1][:, : n - 1], cf[0][:, : n - 1][:, ::-1])


def test_mask_zero_costs_and_min_coherence():
    rng = np.random.default_rng(9)
    m, n = 16, 18
    psi = rng.uniform(-1, 1, (m, n)).astype(np.float32)
    coh = rng.uniform(0, 1, (m, n)).astype(np.float32)
    mask = np.ones((m, n), np.uint8)
    mask[5, 7] = 0
    mask[10:12, 2:5] = 0
    ps, co, valid = oracle.prepare(coh, mask, phase=psi)
    c, _ = oracle.costs(ps, co, valid, np.full((128, 256), 77, np.int16), steep_rad=10.0)
    vh = (valid[:, :-1] & valid[:, 1:]).astype(bool)
    vv = (valid[:-1, :] & valid[1:, :]).astype(bool)
    assert np.all(c[0][:, :-1][~vh] == 0) and np.all(c[1][:, :-1][~vh] == 0)
    assert np.all(c[2][:-1, :][~vv] == 0) and np.all(c[3][:-1, :][~vv] == 0)
    assert np.all(c[0][:, :-1][vh] == 77) and np.all(c[2][:-1, :][vv] == 77)
    # NaN inputs count as masked
    psi2 = psi.copy()
    psi2[3, 3] = np.nan
    _, _, v2 = oracle.prepare(coh, np.ones((m, n), np.uint8), phase=psi2)
    assert v2[3, 3] == 0 and v2.sum() == m * n - 1


def test_steep_rule_cap_and_order():
    rng = np.random.default_rng(1)
    m, n = 30, 30
    psi = np.zeros((m, n), np.float32)
    # plant steep horizontal gradients of distinct sizes in a few rows
    vals = rng.uniform(1.05, 3.0, 60)
    for t, v in enumerate(vals):
        i, j = t // 15 * 2 + 1, (t % 15) * 2
        psi[i, j + 1] = psi[i, j] + np.float32(v)
    coh = np.full((m, n), 0.9, np.float32)
    valid = np.ones((m, n), np.uint8)
    tab = np.full((128, 256), 100, np.int16)
    al_steep = None
    c_all, k_all = oracle.costs(psi, coh, valid, tab, steep_cap_ppm=1000000)
    n_valid_edges = m * (n - 1) + (m - 1) * n
    cap = n_valid_edges * 30000 // 1000000
    c_cap, k_cap = oracle.costs(psi, coh, valid, tab, steep_cap_ppm=30000)
    d = np.abs(wrap64(psi[:, 1:].astype(np.float64) - psi[:, :-1]))
    dv = np.abs(wrap64(psi[1:, :].astype(np.float64) - psi[:-1, :]))
    n_cand = int((d > 1).sum() + (dv > 1).sum())
    assert k_all == n_cand > cap
    assert k_cap == cap
    zeroed = (c_cap[0][:, :-1] == 0)
    # the zeroed h edges are exactly the cap largest |d| (all candidates here are distinct)
    order = np.sort(np.concatenate([d[d > 1], dv[dv > 1]]))[::-1]
    thr = order[cap - 1]
    assert zeroed.sum() + (c_cap[2][:-1, :] == 0).sum() == cap
    assert np.all(d[zeroed] >= thr - 1e-6)
    assert np.all((c_cap[0][:, :-1] == 0) == (c_cap[1][:, :-1] == 0))


# ---------------- integration ----------------

def test_integration_rewrap_and_itoh():
    m, n = 40, 50
    i = np.arange(m)[:, None]
    j = np.arange(n)[None, :]
    truth = 0.8 * j + 0.5 * i + 2.0 * np.sin(i / 5.0)
    psi = wrap64(truth).astype(np.float32)
    valid = np.ones((m, n), np.uint8)
    flows = np.zeros((2, m, n), np.int8)
    unw, K = oracle.integrate(psi, valid, flows)
    # Itoh: noise-free sub-Nyquist phase integrates to truth up to one 2pi multiple
    off = unw.astype(np.float64) - truth
    assert np.allclose(off, off[0, 0], atol=1e-4)
    assert abs(off[0, 0] / (2 * np.pi) - round(off[0, 0] / (2 * np.pi))) < 1e-5
    # rewrap: phi is psi + 2 pi K rounded once to fp32
    exact = psi.astype(np.float64) + 2 * np.pi * K
    assert np.all(np.abs(unw - exact) <= 0.5 * f32_ulp(exact) + 1e-12)
    assert K[0, 0] == 0


def test_integration_masked_nodata():
    m, n = 6, 7
    psi = np.zeros((m, n), np.float32)
    valid = np.ones((m, n), np.uint8)
    valid[2, 3] = 0
    unw, K = oracle.integrate(psi, valid, np.zeros((2, m, n), np.int8))
    assert np.isnan(unw[2, 3]) and np.isfinite(np.delete(unw.ravel(), 2 * n + 3)).all()
