"""Pins for the oracle's connected-component labels (Sec. II-D): reliable edges
are those whose +-1 ambiguity change raises the objective by more than the
threshold; labels grow over them.  Pinned against scipy.ndimage.label (every
edge reliable), networkx connected components, and hand-built special cases
for each part of the reliability rule (flow, threshold, both directions, the
planes of h and v edges, invalid pixels)."""
import networkx as nx
import numpy as np
import pytest
from scipy import ndimage

import oracle

BIG = 10000


def canonical(lab):
    """Relabel components by 1 + their smallest row-major index (0 stays 0)."""
    lab = np.asarray(lab)
    out = np.zeros(lab.shape, np.int64)
    flat = lab.ravel()
    for v in np.unique(flat[flat != 0]):
        idx = np.flatnonzero(flat == v)
        out.ravel()[idx] = idx.min() + 1
    return out


def test_all_reliable_equals_ndimage_label():
    rng = np.random.default_rng(1)
    m, n = 40, 57
    valid = rng.random((m, n)) > 0.45  # many components
    costs = np.full((4, m, n), BIG, np.int16)
    flows = np.zeros((2, m, n), np.int8)
    want, _ = ndimage.label(valid)  # 4-connectivity
    got = oracle.components(costs, flows, valid, 0)
    assert np.array_equal(got, canonical(want))


@pytest.mark.parametrize("seed", range(6))
def test_matches_networkx_components(seed):
    rng = np.random.default_rng(100 + seed)
    m, n = rng.integers(1, 12), rng.integers(1, 12)
    valid = rng.random((m, n)) > 0.2
    costs = rng.integers(0, 60, size=(4, m, n)).astype(np.int16)
    flows = rng.choice([-1, 0, 0, 0, 1], size=(2, m, n)).astype(np.int8)
    T = 20
    g = nx.Graph()
    g.add_nodes_from(i * n + j for i in range(m) for j in range(n) if valid[i, j])
    for i in range(m):
        for j in range(n):
            if j + 1 < n and valid[i, j] and valid[i, j + 1] and flows[0, i, j] == 0 \
                    and costs[0, i, j] > T and costs[1, i, j] > T:
                g.add_edge(i * n + j, i * n + j + 1)
            if i + 1 < m and valid[i, j] and valid[i + 1, j] and flows[1, i, j] == 0 \
                    and costs[2, i, j] > T and costs[3, i, j] > T:
                g.add_edge(i * n + j, (i + 1) * n + j)
    want = np.zeros(m * n, np.int64)
    for comp in nx.connected_components(g):
        want[list(comp)] = min(comp) + 1
    assert np.array_equal(oracle.components(costs, flows, valid, T).ravel(), want)


def two_pixels(horizontal, cp, cm, dk, other=BIG, valid=(True, True)):
    """A 1x2 (h edge) or 2x1 (v edge) image; the other orientation's planes get `other`."""
    shape = (1, 2) if horizontal else (2, 1)
    costs = np.full((4,) + shape, other, np.int16)
    flows = np.zeros((2,) + shape, np.int8)
    a = 0 if horizontal else 2
    costs[a][0, 0], costs[a + 1][0, 0] = cp, cm
    flows[0 if horizontal else 1][0, 0] = dk
    return costs, flows, np.array(valid).reshape(shape)


@pytest.mark.parametrize("horizontal", [True, False])
def test_reliability_rule_cases(horizontal):
    joined, cut = [1, 1], [1, 2]
    lab = lambda *a, T=50, **k: list(oracle.components(*two_pixels(horizontal, *a, **k), T).ravel())
    assert lab(100, 100, 0) == joined
    assert lab(100, 100, 1) == cut          # an edge carrying flow can drop it at a negative change
    assert lab(100, 100, -1) == cut
    assert lab(51, 51, 0) == joined         # strictly above the threshold
    assert lab(50, 100, 0) == cut
    assert lab(100, 50, 0) == cut           # both directions count
    assert lab(100, 100, 0, T=99) == joined
    assert lab(100, 100, 0, T=100) == cut
    assert lab(100, 100, 0, other=0) == joined   # the other orientation's planes do not matter
    assert lab(0, 0, 0, other=BIG) == cut
    assert lab(100, 100, 0, valid=(True, False)) == [1, 0]
    assert lab(100, 100, 0, valid=(False, True)) == [0, 2]


def test_label_is_smallest_index_of_a_u_shape():
    # a U: the component's top-right arm starts at a smaller index than its bottom
    valid = np.array([[1, 0, 1],
                      [1, 0, 1],
                      [1, 1, 1]], bool)
    costs = np.full((4, 3, 3), BIG, np.int16)
    flows = np.zeros((2, 3, 3), np.int8)
    got = oracle.components(costs, flows, valid, 0)
    assert np.array_equal(got, np.where(valid, 1, 0))
    flows[0, 2, 0] = 1  # cut the bottom-left h edge: the left arm alone, the rest labelled from pixel 2
    got = oracle.components(costs, flows, valid, 0)
    assert np.array_equal(got, np.array([[1, 0, 3], [1, 0, 3], [1, 3, 3]]))
