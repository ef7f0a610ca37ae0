"""Served form: continuous batching.  Requests are admitted between solver
passes while others are in flight; every result must equal the oracle's
optimum and the same request unwrapped alone."""
import numpy as np
import pytest

import oracle
import paper_2609_36267_b300 as ww
from paper_2609_36267_b300 import synth

from gpu_helpers import golden_table, oracle_pipeline, to_dev

pytestmark = pytest.mark.gpu


def requests(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        m, n = int(rng.integers(16, 240)), int(rng.integers(16, 260))
        L = float(rng.choice([4.0, 9.0, 16.0]))
        out.append(synth.small_random(900 + seed * 100 + k, m, n, nlooks=L,
                                      mask_frac=0.1 if k % 4 == 0 else 0.0, want_complex=(k % 3 == 0),
                                      lo=0.05, hi=0.9))
    return out


def dev(x):
    ifg = to_dev(x.ifg) if x.is_complex else to_dev(x.phase)
    return ifg, to_dev(x.coh), x.nlooks, to_dev(x.mask)


def test_server_results_equal_oracle_and_alone():
    xs = requests(24, 1)
    srv = ww.Server(hbm_budget_bytes=256 << 20, max_request_pixels=256 * 256, max_active=5)
    tickets = []
    for k, x in enumerate(xs):
        tickets.append(srv.submit(*dev(x)))
        if k == 10:  # some arrive while the first ones are on the GPU
            srv.wait(tickets[0])
            tickets[0] = None
    ws = ww.Workspace(256, 260)
    for x, t in zip(xs, tickets):
        if t is None:
            continue
        unw, K, tc, st, lat = srv.wait(t)
        assert st == ww.WW_OK and lat > 0
        ref = oracle_pipeline(x, golden_table(x.nlooks))
        st_o, _, _, tc_o = oracle.solve_mcf(ref["res"], ref["g"], ref["costs"])
        assert tc == tc_o
        _, K1, tc1 = ww.unwrap(*dev(x), ws=ws)
        assert tc1 == tc
        # ties between optimal flows (Sec. II-C): the matching fraction is reported
        agree = float(np.mean(K1.cpu().numpy() == K.cpu().numpy()))
        print(f"served request {x.shape}: cost {tc}, K agreement alone vs in the mix {agree:.4f}")
        u = unw.cpu().numpy()
        v = ~np.isnan(u)
        assert np.array_equal(v, ref["valid"].astype(bool))
        exact = ref["psi"].astype(np.float64) + 2 * np.pi * K.cpu().numpy()
        assert np.max(np.abs(u[v] - exact[v]), initial=0.0) <= 1e-5
    s = srv.stats()
    assert s["completed"] == 24 and s["rejected"] == 0 and s["peak_active"] <= 5
    srv.close()


def test_server_rejects_oversize_and_bad_requests():
    srv = ww.Server(hbm_budget_bytes=64 << 20, max_request_pixels=64 * 64, max_active=2)
    big = synth.small_random(3, 100, 100)
    with pytest.raises(ww.WWError):
        srv.submit(*dev(big))
    small = synth.small_random(4, 40, 50)
    t = srv.submit(*dev(small))
    unw, K, tc, st, lat = srv.wait(t)
    assert st == ww.WW_OK
    s = srv.stats()
    assert s["rejected"] == 1 and s["completed"] == 1
    srv.close()
