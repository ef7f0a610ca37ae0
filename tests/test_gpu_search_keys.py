"""Key widths of the search's tile visits (GPU).

A visit relaxes in 32-bit keys relative to the tile's smallest label when the
labels' spans fit (every visit of the banded default schedule on these scenes)
and in 64-bit keys otherwise; a 32-bit visit whose candidates leave its range
is redone in 64 bits.  Unbanded passes (no distance cap) make the spans wide,
so both other forms run; the result must still be the oracle's optimum with a
valid certificate, like the default schedule's."""
import numpy as np
import pytest

import oracle
import paper_2609_36267_b300 as ww
from paper_2609_36267_b300 import synth

from gpu_helpers import golden_table, numpy_certificate, oracle_pipeline, to_dev

pytestmark = pytest.mark.gpu


def solve(ref, ws, prm):
    flows, pot, tc, status = ww.solve_mcf(to_dev(ref["res"]), to_dev(np.array([ref["g"]], np.int32)),
                                          to_dev(ref["costs"]), ws, params=prm, check=False)
    return status, flows.cpu().numpy(), pot.cpu().numpy(), int(tc.cpu()[0])


@pytest.mark.parametrize("name,make", [("cfg2_512", lambda: synth.config2(m=512, n=512)),
                                       ("cfg1_256", lambda: synth.config1())])
def test_wide_keys_reach_the_optimum(name, make):
    x = make()
    ref = oracle_pipeline(x, golden_table(x.nlooks))
    st_o, _, _, tc_o = oracle.solve_mcf(ref["res"], ref["g"], ref["costs"])
    assert st_o == 0
    ws = ww.Workspace(*x.shape)
    prm = ww.default_params()
    prm.full_passes = 1 << 20  # every pass searches without a distance cap
    prm.zero_stop_below = 0
    status, flows, pot, tc = solve(ref, ws, prm)
    st = ws.stats()
    assert status == ww.WW_OK, ww.status_string(status)
    assert tc == tc_o
    ok, tc2, why = numpy_certificate(ref["res"], ref["g"], ref["costs"], flows, pot)
    assert ok and tc2 == tc, why
    wide = st["tile_visits"] - st["narrow_visits"] + st["narrow_redone"]
    print(f"{name}: cost {tc}, visits {st['tile_visits']}, 32-bit {st['narrow_visits']}, "
          f"redone {st['narrow_redone']}")
    assert wide > 0  # the 64-bit form ran (directly or as a redo)
    # the default banded schedule on the same instance: the same optimum
    status_d, _, _, tc_d = solve(ref, ww.Workspace(*x.shape), ww.default_params())
    assert status_d == ww.WW_OK and tc_d == tc_o
