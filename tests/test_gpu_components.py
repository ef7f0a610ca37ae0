"""Connected-component labels on the GPU (ww_components, Sec. II-D) against the
oracle's breadth-first search, bit for bit: the labels (1 + the smallest
row-major index of each component, 0 where invalid) are unique, so any
schedule of the union-find must give the oracle's grid.  Inputs are seeded
synthetic planes, and the oracle's own unwrap of a small scene."""
import numpy as np
import pytest

import oracle
import paper_2609_36267_b300 as ww
from paper_2609_36267_b300 import synth

from gpu_helpers import golden_table, oracle_pipeline, to_dev

pytestmark = pytest.mark.gpu


def random_planes(seed, m, n, invalid=0.08, flow=0.04, hi=400):
    rng = np.random.default_rng(seed)
    costs = rng.integers(0, hi, size=(4, m, n)).astype(np.int16)
    flows = np.where(rng.random((2, m, n)) < flow, rng.choice([-1, 1], size=(2, m, n)), 0).astype(np.int8)
    valid = rng.random((m, n)) >= invalid
    unw = np.where(valid, rng.normal(size=(m, n)), np.nan).astype(np.float32)
    return costs, flows, unw, valid


@pytest.mark.parametrize("shape,thr", [((1, 1), 0), ((1, 37), 50), ((41, 1), 50), ((2, 2), 0), ((33, 32), 100),
                                       ((257, 301), 100), ((300, 333), 250), ((512, 600), 30), ((96, 4096), 200)])
def test_components_match_oracle(shape, thr):
    m, n = shape
    costs, flows, unw, valid = random_planes(m * 7919 + n, m, n)
    got = ww.components(to_dev(costs), to_dev(flows), to_dev(unw), thr).cpu().numpy()
    want = oracle.components(costs, flows, valid, thr)
    assert np.array_equal(got, want)


def test_components_all_reliable_and_none_reliable():
    m, n = 200, 310
    costs, flows, unw, valid = random_planes(5, m, n, invalid=0.0, flow=0.0)
    costs[:] = 1000
    got = ww.components(to_dev(costs), to_dev(flows), to_dev(unw), 0).cpu().numpy()
    assert (got == 1).all()  # one component rooted at pixel 0
    got = ww.components(to_dev(costs), to_dev(flows), to_dev(unw), 1000).cpu().numpy()
    assert np.array_equal(got, np.arange(1, m * n + 1).reshape(m, n))  # every pixel alone


def test_components_on_oracle_unwrap():
    """Planes from the oracle's own pipeline (costs, optimal flows, validity) of
    a masked complex scene."""
    x = synth.small_random(22, 300, 333, mask_frac=0.1, want_complex=True, lo=0.05, hi=0.9)
    ref = oracle_pipeline(x, golden_table(x.nlooks))
    st, flows, _, _ = oracle.solve_mcf(ref["res"], ref["g"], ref["costs"])
    assert st == 0
    valid = ref["valid"].astype(bool)
    unw = np.where(valid, 0.0, np.nan).astype(np.float32)
    for thr in (0, 50, 200):
        got = ww.components(to_dev(ref["costs"]), to_dev(flows), to_dev(unw), thr).cpu().numpy()
        assert np.array_equal(got, oracle.components(ref["costs"], flows, valid, thr))


def test_components_large_against_csgraph():
    """4096 x 4096: the same labels as scipy's connected components of the
    reliable-edge graph, made canonical by the smallest index."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components

    m, n, thr = 4096, 4096, 120
    costs, flows, unw, valid = random_planes(11, m, n, hi=300)
    got = ww.components(to_dev(costs), to_dev(flows), to_dev(unw), thr).cpu().numpy().ravel()
    idx = np.arange(m * n).reshape(m, n)
    eh = valid[:, :-1] & valid[:, 1:] & (flows[0, :, :-1] == 0) & (np.minimum(costs[0, :, :-1], costs[1, :, :-1]) > thr)
    ev = valid[:-1, :] & valid[1:, :] & (flows[1, :-1, :] == 0) & (np.minimum(costs[2, :-1, :], costs[3, :-1, :]) > thr)
    a = np.concatenate([idx[:, :-1][eh], idx[:-1, :][ev]])
    b = np.concatenate([idx[:, 1:][eh], idx[1:, :][ev]])
    g = coo_matrix((np.ones(a.size, np.int8), (a, b)), shape=(m * n, m * n))
    _, comp = connected_components(g, directed=False)
    root = np.full(comp.max() + 1, m * n, np.int64)
    np.minimum.at(root, comp, np.arange(m * n))
    want = np.where(valid.ravel(), root[comp] + 1, 0)
    assert np.array_equal(got, want)


def test_components_rejects_bad_arguments():
    import ctypes
    import torch

    t = torch.zeros(8, dtype=torch.int32, device="cuda")
    L = ww.lib()
    p = ctypes.c_void_p(t.data_ptr())
    assert L.ww_components(p, p, p, 2, 2, -1, p, None) == -1           # negative threshold
    assert L.ww_components(p, p, p, 1 << 16, 1 << 15, 0, p, None) == -1  # 2^31 pixels
    assert L.ww_components(None, p, p, 2, 2, 0, p, None) == -1
    assert L.ww_components(p, p, p, 0, 2, 0, p, None) == -1
