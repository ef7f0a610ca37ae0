"""Bridging of mask-separated regions (ww_bridge, Sec. II-D) against the
oracle: region ranks, per-pixel cycle offsets and the bridged phase bit for
bit, on the oracle's pin scenes and on masked unwrapped scenes."""
import numpy as np
import pytest

import oracle
import paper_2609_36267_b300 as ww
from paper_2609_36267_b300 import synth

from gpu_helpers import to_dev

pytestmark = pytest.mark.gpu

TWO_PI = 2 * np.pi


def check_against_oracle(u, window=65, cycles=None):
    """u: float32 [m,n] unwrapped phase, NaN where invalid."""
    u = np.ascontiguousarray(u, np.float32)
    valid = ~np.isnan(u)
    out_o, shift_o, region_o = oracle.bridge(u.astype(np.float64), valid, window=window)
    ud = to_dev(u)
    cd = to_dev(cycles) if cycles is not None else None
    region, shift, nr = ww.bridge(ud, cd, window=window)
    assert nr == (region_o.max() + 1 if valid.any() else 0)
    assert np.array_equal(region.cpu().numpy(), region_o)
    assert np.array_equal(shift.cpu().numpy(), shift_o.astype(np.int32))
    got = ud.cpu().numpy()
    want = out_o.astype(np.float32)
    assert np.array_equal(np.isnan(got), ~valid)
    assert np.array_equal(got[valid].view(np.uint32), want[valid].view(np.uint32))
    if cycles is not None:
        assert np.array_equal(cd.cpu().numpy()[valid], (cycles + shift_o)[valid])
    return shift_o, region_o


def four_regions(m=40, n=50):
    ii, jj = np.mgrid[0:m, 0:n]
    truth = 0.02 * jj + 0.015 * ii
    valid = np.ones((m, n), bool)
    valid[:, 20] = False
    valid[25, :] = False
    return truth, valid


@pytest.mark.parametrize("seed", range(3))
def test_bridge_four_regions_with_offsets(seed):
    rng = np.random.default_rng(seed)
    truth, valid = four_regions()
    _, _, region = oracle.bridge(truth, valid)
    offsets = rng.integers(-6, 7, size=4)
    u = np.where(valid, truth + TWO_PI * offsets[np.maximum(region, 0)], np.nan)
    cyc = rng.integers(-5, 5, size=u.shape).astype(np.int32)
    shift, _ = check_against_oracle(u, cycles=cyc)
    assert (shift[region == 0] == 0).all()


def test_bridge_nearest_region_and_window_region_only():
    m, n = 30, 60
    u = np.zeros((m, n))
    valid = np.zeros((m, n), bool)
    valid[:, 0:25] = True
    valid[0:14, 35:60] = True
    valid[15:22, 45:60] = True
    u[:, 35:60] = 2.0
    u[15:22, 45:60] = 5.0
    check_against_oracle(np.where(valid, u, np.nan))
    m, n = 20, 40
    u = np.zeros((m, n))
    valid = np.zeros((m, n), bool)
    valid[:, 0:15] = True
    valid[0:9, 17:40] = True
    valid[10:20, 17:40] = True
    u[0:9, 17:40] = 3 * TWO_PI + 0.3
    u[10:20, 17:40] = 0.1 + 40 * TWO_PI
    check_against_oracle(np.where(valid, u, np.nan))


def test_bridge_single_region_and_all_invalid():
    rng = np.random.default_rng(3)
    u = (rng.normal(size=(20, 30)) * 10).astype(np.float32)
    u[5, 7] = np.nan
    shift, region = check_against_oracle(u)
    assert (shift == 0).all()
    check_against_oracle(np.full((7, 9), np.nan, np.float32))


@pytest.mark.parametrize("window", [1, 5, 65, 127])
def test_bridge_masked_unwrapped_scene(window):
    """A generated scene unwrapped by the library, then split by a river and
    islands of mask with random whole-cycle offsets per region (ties in the
    distances are common on the pixel grid)."""
    x = synth.small_random(77, 96, 120, nlooks=9.0, mask_frac=0.12, lo=0.3, hi=0.95)
    unw, K, tc = ww.unwrap(to_dev(x.phase), to_dev(x.coh), x.nlooks, to_dev(x.mask))
    u = unw.cpu().numpy()
    u[:, 55:60] = np.nan  # a river
    u[40:43, :] = np.nan
    valid = ~np.isnan(u)
    _, _, region = oracle.bridge(u.astype(np.float64), valid)
    rng = np.random.default_rng(window)
    off = rng.integers(-9, 10, size=region.max() + 1)
    u = np.where(valid, u + (TWO_PI * off[np.maximum(region, 0)]).astype(np.float32), np.nan).astype(np.float32)
    shift, region2 = check_against_oracle(u, window=window, cycles=K.cpu().numpy())
    assert region2.max() >= 3


def test_bridge_many_small_islands():
    rng = np.random.default_rng(11)
    m, n = 70, 90
    valid = rng.uniform(size=(m, n)) > 0.45  # percolation-like: many regions
    u = np.where(valid, rng.normal(size=(m, n)) + TWO_PI * rng.integers(-3, 4, size=(m, n)), np.nan)
    shift, region = check_against_oracle(u.astype(np.float32), window=9)
    assert region.max() > 50
