"""Preprocessing on the GPU against the oracle: multilook with the Eq. (3)
sample coherence (bit-exact: the summation order is specified), the
Goldstein filter (fp32 against the oracle's FP64 FFTs, within 1e-5 of the
local amplitude), and the cycle transfer to the original phase (bit-exact),
including a whole filtered-unwrap-transfer chain."""
import numpy as np
import pytest

import oracle
import paper_2609_36267_b300 as ww
from paper_2609_36267_b300 import synth

from gpu_helpers import golden_table, to_dev

pytestmark = pytest.mark.gpu


def slc_pair(seed, M, N, gamma=0.6, fringes=3.0):
    rng = np.random.default_rng(seed)
    jj = np.arange(N)[None, :]
    phi = 2 * np.pi * fringes * jj / N + np.zeros((M, 1))
    x = (rng.normal(size=(M, N)) + 1j * rng.normal(size=(M, N))) / np.sqrt(2)
    y = (rng.normal(size=(M, N)) + 1j * rng.normal(size=(M, N))) / np.sqrt(2)
    z2 = (gamma * x + np.sqrt(1 - gamma ** 2) * y) * np.exp(-1j * phi)
    return (x * 3.7).astype(np.complex64), (z2 * 0.8).astype(np.complex64)


@pytest.mark.parametrize("M,N,ly,lx", [(64, 90, 4, 6), (257, 301, 5, 10), (33, 40, 1, 1), (100, 7, 3, 7)])
def test_multilook_bit_exact(M, N, ly, lx):
    z1, z2 = slc_pair(M + N, M, N)
    ifg_o, coh_o = oracle.multilook(z1, z2, ly, lx)
    ifg, coh = ww.multilook(to_dev(z1), to_dev(z2), ly, lx)
    assert np.array_equal(ifg.cpu().numpy().view(np.uint32), ifg_o.view(np.uint32))
    assert np.array_equal(coh.cpu().numpy().view(np.uint32), coh_o.view(np.uint32))


@pytest.mark.parametrize("alpha,step,smooth", [(0.5, 16, 3), (0.8, 8, 5), (0.0, 16, 3), (1.0, 32, 1)])
def test_goldstein_matches_fp64_filter(alpha, step, smooth):
    x = synth.small_random(12, 150, 173, want_complex=True, lo=0.2, hi=0.9)
    z = x.ifg.astype(np.complex64)
    want = oracle.goldstein(z.astype(np.complex128), alpha=alpha, step=step, smooth=smooth)
    got = ww.goldstein(to_dev(z), alpha=alpha, step=step, smooth=smooth).cpu().numpy().astype(np.complex128)
    scale = np.abs(want)
    assert np.all(np.abs(got - want) <= 1e-5 * np.maximum(scale, np.median(scale)))


def test_filtered_unwrap_transfers_to_the_original_phase():
    """Sec. II-D: the filtered phase is unwrapped, and its integer cycles are
    moved to the unfiltered phase; cycles and output bit-exact with the oracle."""
    x = synth.small_random(13, 200, 220, want_complex=True, mask_frac=0.06, lo=0.1, hi=0.9)
    ifg, coh, mask = to_dev(x.ifg), to_dev(x.coh), to_dev(x.mask)
    filt = ww.goldstein(ifg, alpha=0.6)
    unw_f, K_f, tc = ww.unwrap(filt, coh, x.nlooks, mask)
    unw, K = ww.transfer_cycles(unw_f, ifg, coh, mask)
    psi, _, valid = oracle.prepare(x.coh, x.mask, ifg=x.ifg)
    out_o, K_o = oracle.transfer_cycles(unw_f.cpu().numpy(), psi, valid)
    assert np.array_equal(K.cpu().numpy(), K_o)
    u = unw.cpu().numpy()
    assert np.array_equal(np.isnan(u), np.isnan(out_o))
    v = ~np.isnan(u)
    assert np.array_equal(u[v].view(np.uint32), out_o[v].view(np.uint32))
    # the result rewraps to the original phase
    assert np.max(np.abs(u[v] - (psi[v].astype(np.float64) + 2 * np.pi * K_o[v])), initial=0) <= 1e-5 * 64


def test_multilook_feeds_the_unwrap():
    """SLC pair -> multilook + Eq. (3) -> whole path; the optimum equals the
    oracle's on its own multilooked inputs."""
    z1, z2 = slc_pair(21, 300, 500, gamma=0.8, fringes=12.0)
    ifg, coh = ww.multilook(to_dev(z1), to_dev(z2), 2, 4)
    unw, K, tc = ww.unwrap(ifg, coh, 8.0, None)
    ifg_o, coh_o = oracle.multilook(z1, z2, 2, 4)
    psi, co, valid = oracle.prepare(coh_o, np.ones(coh_o.shape, np.uint8), ifg=ifg_o)
    lut = ww.Lut.build(8.0)
    r, g = oracle.residues(psi)
    c, _ = oracle.costs(psi, co, valid, lut.table())
    assert tc == oracle.solve_mcf(r, g, c)[3]
