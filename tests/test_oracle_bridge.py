"""Pins for the oracle's bridging of mask-separated regions (Sec. II-D): a
smooth field cut into regions with arbitrary whole-cycle offsets is restored
up to one global cycle count (that of the largest region); offsets added to
any other region before bridging do not change the result; a single region
is untouched; a region is attached to its nearest already-bridged region,
and the window median uses only the endpoint region's pixels."""
import numpy as np
import pytest

import oracle

TWO_PI = 2 * np.pi


def four_regions(m=40, n=50):
    ii, jj = np.mgrid[0:m, 0:n]
    truth = 0.02 * jj + 0.015 * ii
    valid = np.ones((m, n), bool)
    valid[:, 20] = False
    valid[25, :] = False
    return truth, valid


@pytest.mark.parametrize("seed", range(5))
def test_restores_smooth_field_up_to_the_largest_regions_cycles(seed):
    rng = np.random.default_rng(seed)
    truth, valid = four_regions()
    _, _, region = oracle.bridge(truth, valid)
    offsets = rng.integers(-6, 7, size=4)
    u = truth + TWO_PI * offsets[np.maximum(region, 0)]
    out, shift, region2 = oracle.bridge(u, valid)
    assert np.array_equal(region, region2)
    d = (out - truth)[valid]
    assert np.allclose(d, TWO_PI * offsets[0], atol=1e-9)  # region 0 is the largest and keeps its level
    assert (shift[region == 0] == 0).all()


def test_largest_region_first():
    truth, valid = four_regions()
    _, _, region = oracle.bridge(truth, valid)
    sizes = [int((region == k).sum()) for k in range(4)]
    assert sizes == sorted(sizes, reverse=True) == [25 * 29, 25 * 20, 14 * 29, 14 * 20]


def test_single_region_untouched():
    rng = np.random.default_rng(3)
    u = rng.normal(size=(20, 30)) * 10
    valid = np.ones((20, 30), bool)
    valid[5, 7] = False  # a hole does not split it
    out, shift, region = oracle.bridge(u, valid)
    assert (shift == 0).all() and (region[valid] == 0).all() and (region[~valid] == -1).all()
    assert np.array_equal(out[valid], u[valid]) and np.isnan(out[~valid]).all()


def test_attaches_to_the_nearest_bridged_region():
    # A (largest, level 0) | gap | B (level 2.0, close to C) ; C (level 5.0) touches B only across one
    # masked row and lies far from A.  Through B: round((2 - 5) / 2pi) = 0 -> C stays 5.0; through A it
    # would be round((0 - 5) / 2pi) = -1.
    m, n = 30, 60
    u = np.zeros((m, n))
    valid = np.zeros((m, n), bool)
    valid[:, 0:25] = True                  # A: 750 pixels
    valid[0:14, 35:60] = True              # B: 350 pixels
    valid[15:22, 45:60] = True             # C: 105 pixels, one masked row below B
    u[:, 35:60] = 2.0
    u[15:22, 45:60] = 5.0
    out, shift, region = oracle.bridge(u, valid)
    assert region[0, 0] == 0 and region[0, 40] == 1 and region[16, 50] == 2
    assert np.allclose(out[15:22, 45:60], 5.0)
    assert np.allclose(out[0:14, 35:60], 2.0)


def test_window_median_uses_only_the_endpoint_region():
    # B's window around the bridge endpoint also covers a third region D at a far level;
    # the median must ignore D's pixels.
    m, n = 20, 40
    u = np.zeros((m, n))
    valid = np.zeros((m, n), bool)
    valid[:, 0:15] = True       # A: 300, level 0
    valid[0:9, 17:40] = True    # B: 207, level 3*2pi + 0.3 (bridged to 0.3)
    valid[10:20, 17:40] = True  # D: 230 > B, level 0.1 + 40*2pi, nearer to A than B? both 2 away: D ranks first
    u[0:9, 17:40] = 3 * TWO_PI + 0.3
    u[10:20, 17:40] = 0.1 + 40 * TWO_PI
    out, shift, region = oracle.bridge(u, valid, window=65)
    assert np.allclose(out[0:9, 17:40], 0.3)
    assert np.allclose(out[10:20, 17:40], 0.1)
