"""Cost-model variants on the GPU (ww_params.slope_estimator, cost_lookup):
cost planes bit-exact against the oracle's variants, and the whole path with
each variant at the oracle's optimum on the same cost planes."""
import numpy as np
import pytest

import oracle
import paper_2609_36267_b300 as ww
from paper_2609_36267_b300 import synth

from gpu_helpers import GOLDEN, device_inputs, oracle_prepare, to_dev

pytestmark = pytest.mark.gpu

VARIANTS = [(1, 0), (0, 1), (1, 1)]


def golden(L):
    import os

    z = np.load(os.path.join(GOLDEN, f"lut_oracle_L{float(L):g}.npz"))
    return z["table"], z["ratio100"]


def cases():
    return {
        "cfg1_256": lambda: synth.config1(),
        "ragged_257x301_mask": lambda: synth.small_random(21, 257, 301, mask_frac=0.08, lo=0.05, hi=0.8),
        "complex_300x333_mask": lambda: synth.small_random(22, 300, 333, mask_frac=0.1, want_complex=True,
                                                           lo=0.05, hi=0.9),
        "tall_130x33": lambda: synth.small_random(23, 130, 33, lo=0.02, hi=0.5),
    }


@pytest.fixture(scope="module")
def ws():
    return ww.Workspace(512, 512)


@pytest.mark.parametrize("slope,lookup", VARIANTS)
@pytest.mark.parametrize("name", list(cases()))
def test_variant_costs_bit_exact(name, slope, lookup, ws):
    x = cases()[name]()
    tab, ratio = golden(x.nlooks)
    ifg, coh, mask = device_inputs(x)
    prm = ww.default_params(slope_estimator=slope, cost_lookup=lookup)
    c = ww.costs(ifg, coh, ww.Lut.from_tables(x.nlooks, tab, ratio), ws, mask, params=prm).cpu().numpy()
    psi, co, valid = oracle_prepare(x)
    c_o, _ = oracle.costs(psi, co, valid, tab, slope_mode=slope, lookup=lookup, ratio=ratio)
    assert np.array_equal(c, c_o)


@pytest.mark.parametrize("slope,lookup", VARIANTS)
def test_variant_steep_selection_over_cap(slope, lookup, ws):
    rng = np.random.default_rng(4)
    m, n = 150, 170
    ph = rng.uniform(-np.pi, np.pi, (m, n)).astype(np.float32)
    coh = rng.uniform(0, 1, (m, n)).astype(np.float32)
    mask = (rng.uniform(size=(m, n)) > 0.05).astype(np.uint8)
    tab, ratio = golden(4.0)
    prm = ww.default_params(slope_estimator=slope, cost_lookup=lookup)
    c = ww.costs(to_dev(ph), to_dev(coh), ww.Lut.from_tables(4.0, tab, ratio), ws, to_dev(mask),
                 params=prm).cpu().numpy()
    psi, co, valid = oracle.prepare(coh, mask, phase=ph)
    c_o, nsteep = oracle.costs(psi, co, valid, tab, slope_mode=slope, lookup=lookup, ratio=ratio)
    assert nsteep > 0 and np.array_equal(c, c_o)


@pytest.mark.parametrize("slope,lookup", VARIANTS)
def test_variant_unwrap_reaches_the_oracle_optimum(slope, lookup, ws):
    """Whole path with the library's own tables: the optimum equals the oracle's on
    the same table values (the library's 100 ln(P0/P+) table is read back)."""
    x = synth.small_random(31, 200, 230, mask_frac=0.06, want_complex=True, lo=0.05, hi=0.9)
    ifg, coh, mask = device_inputs(x)
    prm = ww.default_params(slope_estimator=slope, cost_lookup=lookup)
    unw, K, tc = ww.unwrap(ifg, coh, x.nlooks, mask, ws=ws, params=prm)
    lut = ww.Lut.build(x.nlooks)
    psi, co, valid = oracle_prepare(x)
    res, g = oracle.residues(psi)
    c_o, _ = oracle.costs(psi, co, valid, lut.table(), slope_mode=slope, lookup=lookup, ratio=lut.ratio100())
    st_o, _, _, tc_o = oracle.solve_mcf(res, g, c_o)
    assert st_o == 0 and tc == tc_o


def test_variants_in_the_batched_form():
    xs = [synth.small_random(40 + k, 60 + 13 * k, 70 + 7 * k, nlooks=9.0, lo=0.05, hi=0.9) for k in range(4)]
    prm = ww.default_params(slope_estimator=1, cost_lookup=1)
    res = ww.unwrap_batch([(to_dev(x.phase), to_dev(x.coh), x.nlooks, to_dev(x.mask)) for x in xs], params=prm)
    lut = ww.Lut.build(9.0)
    for x, (unw, K, tc, st) in zip(xs, res):
        psi, co, valid = oracle.prepare(x.coh, x.mask, phase=x.phase)
        r, g = oracle.residues(psi)
        c_o, _ = oracle.costs(psi, co, valid, lut.table(), slope_mode=1, lookup=1, ratio=lut.ratio100())
        assert st == 0 and tc == oracle.solve_mcf(r, g, c_o)[3]
