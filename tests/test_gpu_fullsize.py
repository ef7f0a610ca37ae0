"""The 74-Mpixel earthquake scene (8192 x 9000, complex64, L = 50) through the
C-ABI at full size, in the launch configuration the benchmark times.

Residues and cost planes are compared with the oracle over the whole image
(bit-exact).  The optimal flow of this size is out of the oracle's reach, so
the solve is proven optimal by LP duality instead: capacity, conservation at
every node and at the ground, and a non-negative reduced cost on every residual
arc, checked both by the library's GPU certificate and in numpy over every row;
the reported total cost must equal the cost of the flow.
Integration is checked on sampled rows against the flows and the rewrap rule."""
import numpy as np
import pytest

import oracle
import paper_2609_36267_b300 as ww
from paper_2609_36267_b300 import synth

from gpu_helpers import band_certificate, device_inputs, golden_table, oracle_prepare

pytestmark = pytest.mark.gpu


@pytest.mark.timeout(1800)
def test_earthquake_full_size():
    import torch

    x = synth.cached("config3")
    m, n = x.shape
    assert (m, n) == (8192, 9000) and x.is_complex
    tab = golden_table(50.0)
    ifg, coh, mask = device_inputs(x)
    psi, cohp, valid = oracle_prepare(x)

    r, g = ww.residues(ifg, coh, mask)
    res_o, g_o = oracle.residues(psi)
    res_d = r.cpu().numpy()
    assert np.array_equal(res_d, res_o.reshape(m - 1, n - 1)) and int(g.cpu()[0]) == g_o
    assert np.count_nonzero(res_d) > 100000

    ws = ww.Workspace(m, n)
    c = ww.costs(ifg, coh, ww.Lut.from_table(50.0, tab), ws, mask)
    costs_o, _ = oracle.costs(psi, cohp, valid, tab)
    costs_d = c.cpu().numpy()
    assert np.array_equal(costs_d, costs_o)
    del costs_o

    prm = ww.default_params()
    prm.graph_loop = 0  # the benchmark's configuration (host-driven pass loop)
    flows, pot, tc, st = ww.solve_mcf(r, g, c, ws, params=prm)
    assert st == ww.WW_OK
    fl = flows.cpu().numpy()
    po = pot.cpu().numpy()
    total = int(tc.cpu()[0])
    # capacity and conservation over the whole image (int16 arithmetic)
    assert np.abs(fl.astype(np.int16)).max() <= 1
    assert not fl[0, :, n - 1].any() and not fl[1, m - 1, :].any()
    h = fl[0].astype(np.int16)
    v = fl[1].astype(np.int16)
    net = h[1:, : n - 1] - h[:-1, : n - 1] + v[: m - 1, : n - 1] - v[: m - 1, 1:]
    assert np.array_equal(net, res_d.astype(np.int16))
    gnet = int(h[0, : n - 1].sum()) - int(h[m - 1, : n - 1].sum()) - int(v[: m - 1, 0].sum()) + int(
        v[: m - 1, n - 1].sum())
    assert gnet == int(g.cpu()[0])
    del net, h, v
    # reported total cost = cost of the flow
    cost_of_flow = 0
    for plane, (cp, cm) in enumerate(((0, 1), (2, 3))):
        f = fl[plane]
        cost_of_flow += int(costs_d[cp][f == 1].astype(np.int64).sum() + costs_d[cm][f == -1].astype(np.int64).sum())
    assert cost_of_flow == total
    # the certificate over every residual arc: on the GPU (ww_certificate), and
    # independently in numpy over all rows in bands of 256 rows
    counts = ww.certificate(r, g, c, flows, pot)
    assert counts[:3] == (0, 0, 0) and counts[3] == total
    for a in range(0, m, 256):
        assert band_certificate(res_d, costs_d, fl, po, a, min(m, a + 256)) == 0, a

    # integration: cycles follow the flows and the wrap counts; phi rewraps to psi
    unw, K = ww.integrate(ifg, flows, coh, mask)
    Kd = K.cpu().numpy()
    ud = unw.cpu().numpy()
    assert Kd[0, 0] == 0
    wc = lambda d: (d > np.float32(np.pi)).astype(np.int64) - (d <= -np.float32(np.pi)).astype(np.int64)
    rows = np.linspace(0, m - 2, 16).astype(int)
    for i in rows:
        dpsi = (psi[i, 1:] - psi[i, :-1]).astype(np.float32)
        assert np.array_equal(Kd[i, 1:] - Kd[i, :-1], fl[0, i, : n - 1].astype(np.int64) - wc(dpsi))
        dcol = (psi[i + 1, :] - psi[i, :]).astype(np.float32)
        assert np.array_equal(Kd[i + 1, :] - Kd[i, :], fl[1, i, :].astype(np.int64) - wc(dcol))
        ok = valid[i].astype(bool)
        exact = (psi[i].astype(np.float64) + np.float64(2 * np.pi) * Kd[i]).astype(np.float32)
        assert np.array_equal(ud[i][ok], exact[ok])
        assert np.isnan(ud[i][~ok]).all()
    torch.cuda.synchronize()
