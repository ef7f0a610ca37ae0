"""GPU path vs the CPU oracle, through the C-ABI (ctypes binding over libww.so).

Bar: residues, ground charge, LUT indices, cost planes, steep selection and
integer cycle maps bit-exact; the MCF total cost equal to the oracle's optimum
with a valid potential certificate; unwrapped phase equal to the oracle's
bit for bit (same FP64 rounding sequence)."""
import numpy as np
import pytest

import oracle
import paper_2609_36267_b300 as ww
from paper_2609_36267_b300 import synth

from gpu_helpers import (device_array, device_inputs, golden_table, numpy_certificate, oracle_pipeline, probe_table,
                         to_dev)

pytestmark = pytest.mark.gpu


def cases():
    out = {
        "cfg1_256": lambda: synth.config1(),
        "ragged_257x301_mask": lambda: synth.small_random(21, 257, 301, mask_frac=0.08, lo=0.05, hi=0.8),
        "complex_300x333_mask": lambda: synth.small_random(22, 300, 333, mask_frac=0.1, want_complex=True,
                                                           lo=0.05, hi=0.9),
        "cfg2_512": lambda: synth.config2(m=512, n=512),
        "tall_130x33": lambda: synth.small_random(23, 130, 33, lo=0.02, hi=0.5),
        "wide_33x130": lambda: synth.small_random(24, 33, 130, lo=0.02, hi=0.5),
    }
    return out


def with_nan(x):
    x.phase[3, 5] = np.nan
    x.coh[7, 1] = np.inf
    if x.ifg is not None:
        x.ifg[9, 9] = np.complex64(complex(np.nan, 1.0))
    return x


@pytest.fixture(scope="module")
def ws():
    return ww.Workspace(2048, 2048)


@pytest.mark.parametrize("name", list(cases()))
def test_residues_bit_exact(name):
    x = with_nan(cases()[name]())
    ifg, coh, mask = device_inputs(x)
    r, g = ww.residues(ifg, coh, mask)
    ref = oracle_pipeline(x, probe_table())
    assert np.array_equal(r.cpu().numpy(), ref["res"])
    assert int(g.cpu()[0]) == ref["g"]


@pytest.mark.parametrize("name", list(cases()))
def test_cost_indices_bit_exact(name, ws):
    """Probe table (entry = 256*i_gamma + i_alpha) makes the cost planes the LUT indices."""
    x = with_nan(cases()[name]())
    ifg, coh, mask = device_inputs(x)
    lut = ww.Lut.from_table(x.nlooks, probe_table())
    c = ww.costs(ifg, coh, lut, ws, mask).cpu().numpy()
    ref = oracle_pipeline(x, probe_table())
    assert np.array_equal(c, ref["costs"])


@pytest.mark.parametrize("name", ["cfg1_256", "complex_300x333_mask", "cfg2_512"])
def test_costs_with_oracle_table_bit_exact(name, ws):
    x = cases()[name]()
    tab = golden_table(x.nlooks)
    ifg, coh, mask = device_inputs(x)
    c = ww.costs(ifg, coh, ww.Lut.from_table(x.nlooks, tab), ws, mask).cpu().numpy()
    assert np.array_equal(c, oracle_pipeline(x, tab)["costs"])


def noise_case(seed, m, n, levels=None):
    """Pure phase noise: about 2/3 of edges are steep, far over the 3% cap; with
    `levels` the phases take few distinct values, so |d| ties at the cut."""
    rng = np.random.default_rng(seed)
    ph = rng.uniform(-np.pi, np.pi, (m, n))
    if levels:
        ph = np.round(ph / (2 * np.pi) * levels) / levels * 2 * np.pi
        ph = np.clip(ph, -np.pi, np.pi)
    ph = ph.astype(np.float32)
    coh = rng.uniform(0, 1, (m, n)).astype(np.float32)
    mask = (rng.uniform(size=(m, n)) > 0.05).astype(np.uint8)
    return synth.Interferogram(phase=ph, coh=coh, mask=mask, nlooks=4.0, truth=np.zeros((m, n)))


@pytest.mark.parametrize("levels,ppm", [(None, 30000), (7, 30000), (12, 5000), (None, 0), (5, 999999)])
def test_steep_selection_over_cap_bit_exact(levels, ppm, ws):
    x = noise_case(5 + (levels or 0), 211, 173, levels)
    ifg, coh, mask = device_inputs(x)
    prm = ww.default_params(steep_cap_ppm=ppm)
    lut = ww.Lut.from_table(4.0, probe_table())
    c = ww.costs(ifg, coh, lut, ws, mask, params=prm).cpu().numpy()
    ref = oracle_pipeline(x, probe_table(), steep_cap_ppm=ppm)
    assert np.array_equal(c, ref["costs"])
    assert ref["nsteep"] > 0 or ppm == 0


@pytest.mark.parametrize("name", list(cases()))
def test_integrate_bit_exact_with_oracle_flows(name):
    x = with_nan(cases()[name]())
    ref = oracle_pipeline(x, golden_table(x.nlooks))
    st, flows, pot, tc = oracle.solve_mcf(ref["res"], ref["g"], ref["costs"])
    assert st == 0
    unw_o, K_o = oracle.integrate(ref["psi"], ref["valid"], flows)
    ifg, coh, mask = device_inputs(x)
    unw, K = ww.integrate(ifg, to_dev(flows), coh, mask)
    assert np.array_equal(K.cpu().numpy(), K_o)
    u = unw.cpu().numpy()
    assert np.array_equal(np.isnan(u), np.isnan(unw_o))
    assert np.array_equal(u[~np.isnan(u)].view(np.uint32), unw_o[~np.isnan(unw_o)].view(np.uint32))


def solve_and_check(ref, ws, params=None):
    res, g, costs = ref["res"], ref["g"], ref["costs"]
    flows, pot, tc, status = ww.solve_mcf(to_dev(res), to_dev(np.array([g], np.int32)), to_dev(costs), ws,
                                          params=params, check=False)
    return status, flows.cpu().numpy(), pot.cpu().numpy(), int(tc.cpu()[0])


@pytest.mark.parametrize("name", list(cases()))
def test_solve_equals_oracle_optimum_with_certificate(name, ws):
    x = cases()[name]()
    ref = oracle_pipeline(x, golden_table(x.nlooks))
    st_o, flows_o, pot_o, tc_o = oracle.solve_mcf(ref["res"], ref["g"], ref["costs"])
    assert st_o == 0
    status, flows, pot, tc = solve_and_check(ref, ws)
    assert status == ww.WW_OK, ww.status_string(status)
    assert tc == tc_o
    code, tc2, bad = oracle.check_certificate(ref["res"], ref["g"], ref["costs"], flows, pot)
    assert code == 0 and tc2 == tc
    ok, tc3, why = numpy_certificate(ref["res"], ref["g"], ref["costs"], flows, pot)
    assert ok, why
    import torch
    counts = ww.certificate(to_dev(ref["res"]), to_dev(np.array([ref["g"]], np.int32)), to_dev(ref["costs"]),
                            to_dev(flows), to_dev(pot))
    assert counts[:3] == (0, 0, 0) and counts[3] == tc
    # report how much of the cycle map matches the oracle's (ties allow several optima)
    _, K_g = oracle.integrate(ref["psi"], ref["valid"], flows)
    _, K_o = oracle.integrate(ref["psi"], ref["valid"], flows_o)
    agree = float(np.mean(K_g == K_o))
    print(f"{name}: cost {tc}, residues {np.count_nonzero(ref['res'])}, K agreement {agree:.4f}, "
          f"stats {ws.stats()}")


def test_solve_is_deterministic(ws):
    x = synth.config2(m=512, n=512)
    ref = oracle_pipeline(x, golden_table(x.nlooks))
    a = solve_and_check(ref, ws)
    b = solve_and_check(ref, ws)
    assert a[0] == b[0] == 0
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


@pytest.mark.parametrize("seed", range(6))
def test_solve_charge_two_random_supplies(seed, ws):
    rng = np.random.default_rng(seed)
    m, n = int(rng.integers(20, 90)), int(rng.integers(20, 90))
    res = rng.choice([-2, -1, 0, 0, 0, 0, 0, 0, 1, 2], size=(m - 1, n - 1)).astype(np.int8)
    g = -int(res.sum())
    costs = rng.integers(0, 500, (4, m, n)).astype(np.int16)
    costs[rng.random((4, m, n)) < 0.15] = 0
    ref = dict(res=res, g=g, costs=costs)
    st_o, _, _, tc_o = oracle.solve_mcf(res, g, costs)
    status, flows, pot, tc = solve_and_check(ref, ws)
    if st_o == 0:
        assert status == 0 and tc == tc_o
        assert numpy_certificate(res, g, costs, flows, pot)[0]
    else:
        assert status == ww.WW_ERR_INFEASIBLE


def test_solve_infeasible_block(ws):
    m = n = 14
    res = np.zeros((m - 1, n - 1), np.int8)
    res[3:9, 3:9] = 1
    res[0, 0] = -1
    g = -int(res.sum())
    costs = np.ones((4, m, n), np.int16)
    assert not oracle.feasible(res, g)
    status, *_ = solve_and_check(dict(res=res, g=g, costs=costs), ws)
    assert status == ww.WW_ERR_INFEASIBLE


def _resume_to_optimum(ref, ws, flows, pot, tc_o):
    """Continue from (flows, pot) with the default parameters: the optimum with a certificate."""
    fl, po = to_dev(flows), to_dev(pot)
    tc, status = ww.solve_mcf_resume(to_dev(ref["res"]), to_dev(np.array([ref["g"]], np.int32)),
                                     to_dev(ref["costs"]), ws, fl, po, check=False)
    assert status == ww.WW_OK, ww.status_string(status)
    assert int(tc.cpu()[0]) == tc_o
    ok, tc2, why = numpy_certificate(ref["res"], ref["g"], ref["costs"], fl.cpu().numpy(), po.cpu().numpy())
    assert ok and tc2 == tc_o, why


def test_solve_pass_limit_times_out_and_resumes(ws):
    """A pass limit stops the solve with WW_ERR_TIMEOUT; the flows and potentials
    it returns are a valid (unbalanced) state that resumes to the optimum."""
    x = synth.config2(m=256, n=256)
    ref = oracle_pipeline(x, golden_table(x.nlooks))
    st_o, _, _, tc_o = oracle.solve_mcf(ref["res"], ref["g"], ref["costs"])
    status, flows, pot, _ = solve_and_check(ref, ws, params=ww.default_params(max_passes=1))
    assert status == ww.WW_ERR_TIMEOUT
    ok, _, why = numpy_certificate(ref["res"], ref["g"], ref["costs"], flows, pot)
    assert not ok and why == "conservation"  # capacities and reduced costs hold, supplies not yet routed
    _resume_to_optimum(ref, ws, flows, pot, tc_o)


def test_worklist_wait_limit_times_out_and_resumes(ws):
    """A device worklist wait that runs out (wait_polls = 1: a search CTA whose
    worklist slot is still empty gives up at its first poll) ends the search
    with an error flag; the kernel returns, the pass augments nothing, the solve
    reports WW_ERR_TIMEOUT, and its state resumes to the optimum.  Nothing traps."""
    x = synth.config2(m=512, n=512)
    ref = oracle_pipeline(x, golden_table(x.nlooks))
    st_o, _, _, tc_o = oracle.solve_mcf(ref["res"], ref["g"], ref["costs"])
    for graph_loop in (0, 1):
        status, flows, pot, _ = solve_and_check(ref, ws, params=ww.default_params(wait_polls=1, graph_loop=graph_loop))
        assert status == ww.WW_ERR_TIMEOUT, ww.status_string(status)
        _resume_to_optimum(ref, ws, flows, pot, tc_o)
    # the workspace is reusable after the aborted searches
    status, flows, pot, tc = solve_and_check(ref, ws)
    assert status == ww.WW_OK and tc == tc_o


def test_resume_rejects_an_invalid_starting_pair(ws):
    """A potential that leaves a residual arc with negative reduced cost is refused
    before any pass (the flows and potentials are left as given)."""
    x = synth.config1()
    ref = oracle_pipeline(x, golden_table(x.nlooks))
    flows = np.zeros((2,) + ref["costs"].shape[1:], np.int8)
    pot = np.zeros(ref["res"].size + 1, np.int64)
    pot[1000] = 10 ** 6
    fl, po = to_dev(flows), to_dev(pot)
    tc, status = ww.solve_mcf_resume(to_dev(ref["res"]), to_dev(np.array([ref["g"]], np.int32)),
                                     to_dev(ref["costs"]), ws, fl, po, check=False)
    assert status == ww.WW_ERR_INVALID_ARG
    assert np.array_equal(po.cpu().numpy(), pot) and not fl.cpu().numpy().any()


@pytest.mark.parametrize("m,n", [(2, 2), (2, 9), (9, 2), (3, 3), (33, 33), (65, 2)])
def test_tiny_grids(m, n, ws):
    x = synth.small_random(m * 100 + n, m, n, lo=0.0, hi=0.3)
    ref = oracle_pipeline(x, golden_table(9.0))
    ifg, coh, mask = device_inputs(x)
    r, g = ww.residues(ifg, coh, mask)
    assert np.array_equal(r.cpu().numpy(), ref["res"]) and int(g.cpu()[0]) == ref["g"]
    c = ww.costs(ifg, coh, ww.Lut.from_table(9.0, golden_table(9.0)), ws, mask).cpu().numpy()
    assert np.array_equal(c, ref["costs"])
    st_o, _, _, tc_o = oracle.solve_mcf(ref["res"], ref["g"], ref["costs"])
    status, flows, pot, tc = solve_and_check(ref, ws)
    assert status == 0 and tc == tc_o
    assert numpy_certificate(ref["res"], ref["g"], ref["costs"], flows, pot)[0]


def test_tall_image_beyond_65535_tile_rows():
    """An image taller than 65535 tiles of the residue and cost kernels (both use a
    one-dimensional grid of tiles): residues and cost planes bit-exact."""
    m, n = 2_100_000, 3
    x = synth.small_random(91, m, n, lo=0.05, hi=0.9)
    ifg, coh, mask = device_inputs(x)
    ref = oracle_pipeline(x, probe_table())
    r, g = ww.residues(ifg, coh, mask)
    assert np.array_equal(r.cpu().numpy(), ref["res"]) and int(g.cpu()[0]) == ref["g"]
    c = ww.costs(ifg, coh, ww.Lut.from_table(x.nlooks, probe_table()), ww.Workspace(m, n), mask)
    assert np.array_equal(c.cpu().numpy(), ref["costs"])


def test_all_masked_and_single_valid_pixel(ws):
    for keep in (0, 1):
        x = synth.small_random(77, 40, 50)
        x.mask[:] = 0
        if keep:
            x.mask[20, 25] = 1
        ref = oracle_pipeline(x, golden_table(9.0))
        assert not ref["res"].any()
        unw, K, tc = ww.unwrap(to_dev(x.phase), to_dev(x.coh), 9.0, to_dev(x.mask), ws=ws)
        u = unw.cpu().numpy()
        assert tc == 0 and not K.cpu().numpy().any()
        assert np.isnan(u).sum() == x.mask.size - keep


@pytest.mark.parametrize("name", ["cfg1_256", "complex_300x333_mask", "cfg2_512", "ragged_257x301_mask"])
def test_unwrap_end_to_end(name, ws):
    """Whole path with the library's own table; optimal cost equal to the
    oracle's optimum on the same table values, rewrap within 1e-5 rad."""
    x = cases()[name]()
    ifg, coh, mask = device_inputs(x)
    unw, K, tc = ww.unwrap(ifg, coh, x.nlooks, mask, ws=ws)
    u, Kn = unw.cpu().numpy(), K.cpu().numpy()
    # the oracle on the library's own table (equal to the oracle's tables, see
    # test_lib_cpu.py, but the solve is compared on exactly what the path used)
    lib_tab = ww.Lut.build(x.nlooks).table()
    ref = oracle_pipeline(x, lib_tab)
    st_o, flows_o, _, tc_o = oracle.solve_mcf(ref["res"], ref["g"], ref["costs"])
    assert st_o == 0 and tc == tc_o
    # the residues and cost planes this call computed (in one fused pass for a
    # complex input), read back from the workspace: bit-exact
    m, n = x.shape
    p_res, p_g, p_costs, _, _ = ws.last_unwrap_pointers()
    assert np.array_equal(device_array(p_res, (m - 1, n - 1), np.int8), ref["res"])
    assert int(device_array(p_g, (1,), np.int32)[0]) == ref["g"]
    assert np.array_equal(device_array(p_costs, (4, m, n), np.int16), ref["costs"])
    v = ~np.isnan(u)
    assert np.array_equal(v, ref["valid"].astype(bool))
    exact = ref["psi"].astype(np.float64) + 2 * np.pi * Kn
    assert np.max(np.abs(u[v] - exact[v]), initial=0.0) <= 1e-5
    assert Kn[0, 0] == 0


def test_complex_phase_bit_exact_extremes(ws):
    """Phase of complex samples over the whole fp32 range (random bit patterns,
    subnormals, signed zeros, axes, equal parts, parts 2^100 apart): the
    unwrapped output equals fp32(psi + 2 pi K) in fp64 with the oracle's psi
    and the returned K, bit for bit, at every valid pixel."""
    rng = np.random.default_rng(31)
    m, n = 96, 80
    bits = rng.integers(0, 2**32, size=(m, n, 2), dtype=np.uint64).astype(np.uint32)
    bits[(bits & 0x7F800000) == 0x7F800000] &= 0xBF7FFFFF  # keep every part finite
    z = bits.view(np.float32).copy()
    special = np.array([0.0, -0.0, 1.0, -1.0, 1e-45, -1e-45, 1.1754942e-38, 3.4028235e38, -3.4028235e38,
                        1e-30, 1e30, 0.5, -3.0], np.float32)
    k = 0
    for a in special:
        for b in special:
            z[k // n, k % n] = (a, b)
            k += 1
    t = rng.uniform(-1, 1, size=(m // 4, n, 2)).astype(np.float32)
    z[m // 2: m // 2 + m // 4] = t * np.float32(2.0) ** rng.integers(-120, 120, size=(m // 4, n, 1)).astype(np.float32)
    ifg = np.ascontiguousarray(z).view(np.complex64).reshape(m, n)
    coh = rng.uniform(0.05, 0.9, size=(m, n)).astype(np.float32)
    mask = np.ones((m, n), np.uint8)
    unw, K, tc = ww.unwrap(to_dev(ifg), to_dev(coh), 4.0, to_dev(mask), ws=ws)
    u, Kn = unw.cpu().numpy(), K.cpu().numpy()
    psi, _, valid = oracle.prepare(coh, mask, ifg=ifg)
    v = valid.astype(bool)
    assert v.all()
    want = (psi.astype(np.float64) + Kn.astype(np.float64) * 6.283185307179586).astype(np.float32)
    assert np.array_equal(u.view(np.uint32)[v], want.view(np.uint32)[v])


def _tie_phase(K):
    """A phase that puts fp64(psi + fp64(K 2pi)) exactly on a rounding boundary:
    halfway between two fp32 values when such a psi is an fp32 number, else
    halfway between two fp64 values (an odd multiple of half an fp64 ulp of K 2pi)."""
    t = np.float64(K) * np.float64(2 * np.pi)
    g = np.float32(t)
    for q in range(-2, 3):
        lo = g
        for _ in range(abs(q)):
            lo = np.nextafter(lo, np.float32(np.inf) if q > 0 else np.float32(-np.inf))
        mid = (np.float64(lo) + np.float64(np.nextafter(lo, np.float32(np.inf)))) / 2
        d = mid - t
        if np.float64(np.float32(d)) == d and abs(d) < 1e-3:
            return np.float32(d)
    e = np.frexp(t)[1]
    return np.float32((2 * (abs(K) % 7) + 1) * np.ldexp(1.0, int(e) - 54))


def test_integrate_rounding_bit_exact():
    """Integration output fp32(fp64(psi) + fp64(K) 2pi) bit for bit on inputs
    built to stress its two roundings: exact ties of both roundings with |K| up
    to ~10^4 (either side of the integer path's |K| < 2^11 bound), wrapped
    phases, phases beyond +-4 and arbitrary fp32 values; K follows the row
    recurrence K(j+1) - K(j) = dk_h(j) - wrap(psi(j+1) - psi(j))."""
    rng = np.random.default_rng(77)
    m, n = 64, 4096
    flows = np.zeros((2, m, n), np.int8)
    psi = np.zeros((m, n), np.float32)
    for i in range(0, 16):  # ties: tiny phases, so every wrap count is 0 and K is the flow sum
        f = rng.integers(-127, 128, size=n).astype(np.int8)
        f[-1] = 0
        flows[0, i] = f
        K = np.concatenate([[0], np.cumsum(f[:-1].astype(np.int64))])
        psi[i, 1:] = [_tie_phase(int(k)) for k in K[1:]]
    psi[16:32, 1:] = rng.uniform(-np.pi, np.pi, size=(16, n - 1)).astype(np.float32)
    flows[0, 16:32] = rng.integers(-1, 2, size=(16, n))
    big = rng.uniform(4.0, 1e4, size=(16, n - 1)) * rng.choice([-1.0, 1.0], size=(16, n - 1))
    psi[32:48, 1:] = big.astype(np.float32)
    flows[0, 32:48] = rng.integers(-100, 101, size=(16, n))
    bits = rng.integers(0, 2**32, size=(16, n - 1), dtype=np.uint64).astype(np.uint32)
    bits[(bits & 0x7F800000) == 0x7F800000] &= 0xBF7FFFFF
    psi[48:64, 1:] = bits.view(np.float32)
    flows[0, 48:64] = rng.integers(-3, 4, size=(16, n))
    unw, cyc = ww.integrate(to_dev(psi), to_dev(flows))
    u, K = unw.cpu().numpy(), cyc.cpu().numpy().astype(np.int64)
    assert (K[:, 0] == 0).all()
    with np.errstate(over="ignore"):
        d = psi[:, 1:] - psi[:, :-1]  # fp32 differences (+-inf where they overflow, as on the device)
    pi32 = np.float32(np.pi)
    wrap = (d > pi32).astype(np.int64) - (d <= -pi32).astype(np.int64)
    assert np.array_equal(K[:, 1:] - K[:, :-1], flows[0, :, :-1].astype(np.int64) - wrap)
    assert np.abs(K[:16]).max() >= 2048  # both sides of the integer path's bound
    want = (psi.astype(np.float64) + K.astype(np.float64) * 6.283185307179586).astype(np.float32)
    assert np.array_equal(u.view(np.uint32), want.view(np.uint32))
