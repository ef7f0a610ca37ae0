"""Pins for the oracle's MCF solve (Eq. 2, Sec. II-C) and its integration."""
import numpy as np
import pytest

import oracle
from paper_2609_36267_b300 import synth


def random_case(seed, m, n, lo=0.02, hi=0.6, mask_frac=0.0):
    x = synth.small_random(seed, m, n, lo=lo, hi=hi, mask_frac=mask_frac, corr_px=3.0)
    psi, coh, valid = oracle.prepare(x.coh, x.mask, phase=x.phase)
    rng = np.random.default_rng(seed)
    table = rng.integers(0, 400, (128, 256)).astype(np.int16)
    costs, _ = oracle.costs(psi, coh, valid, table)
    res, g = oracle.residues(psi)
    return psi, valid, costs, res, g


@pytest.mark.parametrize("seed", range(40))
def test_ssp_matches_exhaustive_enumeration(seed):
    rng = np.random.default_rng(1000 + seed)
    m = int(rng.integers(2, 6))
    n = int(rng.integers(2, 6))
    psi, valid, costs, res, g = random_case(seed, m, n, mask_frac=0.2 if seed % 3 == 0 else 0.0)
    st, flows, pot, tc = oracle.solve_mcf(res, g, costs)
    assert st == 0
    assert oracle.brute_force(psi, costs) == tc
    code, tc2, _ = oracle.check_certificate(res, g, costs, flows, pot)
    assert code == 0 and tc2 == tc


def lp_optimum(res, g, costs):
    """Eq. (2) as a plain LP (unit capacities, balance at every node incl. G),
    solved by HiGHS; the node-arc incidence matrix is totally unimodular."""
    from scipy.optimize import linprog
    from scipy.sparse import coo_matrix
    _, m, n = costs.shape
    G = (m - 1) * (n - 1)
    node = lambda i, j: i * (n - 1) + j if (0 <= i < m - 1 and 0 <= j < n - 1) else G
    tails, heads, cst = [], [], []
    for i in range(m):
        for j in range(n - 1):
            a, b = node(i - 1, j), node(i, j)
            tails += [a, b]; heads += [b, a]; cst += [costs[0, i, j], costs[1, i, j]]
    for i in range(m - 1):
        for j in range(n):
            l, r = node(i, j - 1), node(i, j)
            tails += [r, l]; heads += [l, r]; cst += [costs[2, i, j], costs[3, i, j]]
    A = len(cst)
    rows = np.concatenate([tails, heads])
    cols = np.concatenate([np.arange(A), np.arange(A)])
    vals = np.concatenate([np.ones(A), -np.ones(A)])
    M = coo_matrix((vals, (rows, cols)), shape=(G + 1, A)).tocsr()
    b = np.concatenate([res.ravel().astype(float), [float(g)]])
    out = linprog(np.asarray(cst, float), A_eq=M, b_eq=b, bounds=(0, 1), method="highs")
    return out.status, (round(out.fun) if out.status == 0 else None)


@pytest.mark.parametrize("seed", range(8))
def test_ssp_matches_lp_with_charge_two(seed):
    rng = np.random.default_rng(seed)
    m, n = int(rng.integers(6, 14)), int(rng.integers(6, 14))
    res = rng.choice([-2, -1, 0, 0, 0, 0, 1, 2], size=(m - 1, n - 1)).astype(np.int8)
    g = -int(res.sum())
    costs = rng.integers(0, 300, (4, m, n)).astype(np.int16)
    costs[rng.random((4, m, n)) < 0.1] = 0
    st, flows, pot, tc = oracle.solve_mcf(res, g, costs)
    lst, lopt = lp_optimum(res, g, costs)
    if st == 0:
        assert lst == 0 and lopt == tc
        assert oracle.check_certificate(res, g, costs, flows, pot)[0] == 0
    else:
        assert st == -4 and lst == 2 and not oracle.feasible(res, g)


@pytest.mark.parametrize("seed", range(4))
def test_ssp_matches_lp_on_phase_cases(seed):
    psi, valid, costs, res, g = random_case(300 + seed, 17, 23, mask_frac=0.15)
    st, flows, pot, tc = oracle.solve_mcf(res, g, costs)
    assert st == 0
    assert lp_optimum(res, g, costs) == (0, tc)


@pytest.mark.parametrize("seed", range(6))
def test_ssp_certificate_and_curl_free_medium(seed):
    psi, valid, costs, res, g = random_case(50 + seed, 37, 45, mask_frac=0.1)
    st, flows, pot, tc = oracle.solve_mcf(res, g, costs)
    assert st == 0 and np.count_nonzero(res) > 10
    code, tc2, _ = oracle.check_certificate(res, g, costs, flows, pot)
    assert code == 0 and tc2 == tc == oracle.flow_cost(costs, flows)
    # corrected gradients are curl-free: integrating rows-first and columns-first agree
    unw, K = oracle.integrate(psi, valid, flows)
    m, n = psi.shape
    wc = lambda d: (d > np.float32(np.pi)).astype(np.int64) - (d <= -np.float32(np.pi)).astype(np.int64)
    nh = wc(psi[:, 1:] - psi[:, :-1])
    nv = wc(psi[1:, :] - psi[:-1, :])
    K2 = np.zeros((m, n), np.int64)
    K2[0, 1:] = np.cumsum(flows[0, 0, : n - 1] - nh[0])
    K2[1:, :] = K2[0][None, :] + np.cumsum(flows[1, : m - 1, :] - nv, axis=0)
    assert np.array_equal(K2, K)


def test_certificate_rejects_suboptimal_and_broken_flows():
    psi, valid, costs, res, g = random_case(77, 12, 14)
    st, flows, pot, tc = oracle.solve_mcf(res, g, costs)
    assert oracle.check_certificate(res, g, costs, flows, pot)[0] == 0
    bad = flows.copy()
    k = np.argwhere(bad[0, :, :-1] == 0)[0]
    bad[0, k[0], k[1]] = 1
    assert oracle.check_certificate(res, g, costs, bad, pot)[0] == 2  # conservation
    bad = flows.copy()
    bad[1, 0, 0] = 2
    assert oracle.check_certificate(res, g, costs, bad, pot)[0] == 1  # capacity
    # a feasible but non-optimal flow: raise K by one at one pixel, i.e. a unit
    # circulation around that pixel's four incident edges
    worse = 0
    for (i, j) in [(3, 4), (5, 6), (7, 2), (2, 9)]:
        cyc = flows.copy()
        for plane, a, b, d in ((0, i, j - 1, 1), (0, i, j, -1), (1, i - 1, j, 1), (1, i, j, -1)):
            cyc[plane, a, b] += d
        if np.abs(cyc).max() > 1:
            continue
        code, tcc, _ = oracle.check_certificate(res, g, costs, cyc, pot)
        assert code in (0, 3) and tcc >= tc
        if tcc > tc:
            assert code == 3
            worse += 1
    assert worse > 0


def test_infeasible_block_of_charges():
    m, n = 14, 14
    res = np.zeros((m - 1, n - 1), np.int8)
    res[3:9, 3:9] = 1  # net +36 inside a boundary of 24 unit arcs
    res[0, 0] = -1
    g = -int(res.sum())
    costs = np.ones((4, m, n), np.int16)
    assert not oracle.feasible(res, g)
    st, *_ = oracle.solve_mcf(res, g, costs)
    assert st == -4
    res2 = np.zeros_like(res)
    res2[3:5, 3:5] = 1
    assert oracle.feasible(res2, -4)
    assert oracle.solve_mcf(res2, -4, costs)[0] == 0


def test_zero_residues_zero_flow():
    m, n = 10, 12
    i = np.arange(m)[:, None]
    j = np.arange(n)[None, :]
    psi = ((0.7 * j + 0.2 * i + np.pi) % (2 * np.pi) - np.pi).astype(np.float32)
    res, g = oracle.residues(psi)
    costs = np.full((4, m, n), 5, np.int16)
    st, flows, pot, tc = oracle.solve_mcf(res, g, costs)
    assert st == 0 and tc == 0 and not flows.any()
