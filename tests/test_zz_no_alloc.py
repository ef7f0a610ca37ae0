"""ww_costs_noalloc: the cost step for callers that cannot allocate device
memory (their device memory belongs to another allocator, or they must not pay
cudaMalloc's implicit device synchronisation).  It must give the same cost
planes as ww_costs, which uses a library-allocated workspace, call after call,
although every call reuses one static scratch array inside the library.

This file is collected last on purpose (pytest orders files by name)."""
import ctypes

import numpy as np
import pytest

import paper_2609_36267_b300 as ww
from paper_2609_36267_b300 import synth


def test_noalloc_rejects_grids_over_its_limit():
    """Argument check only (no device work): more than 2^27 pixels is refused."""
    dummy = ctypes.c_void_p(256)
    lut = ww.Lut.from_table(9.0, np.zeros((128, 256), np.int16))
    st = ww.lib().ww_costs_noalloc(dummy, 0, dummy, None, 1 << 14, 1 << 14, lut.handle, None, dummy, None)
    assert st == ww.WW_ERR_INVALID_ARG
    st = ww.lib().ww_costs_noalloc(dummy, 0, dummy, None, 1, 100, lut.handle, None, dummy, None)
    assert st == ww.WW_ERR_INVALID_ARG
    # the same parameter checks as ww_costs: a NaN steep threshold would silently
    # disable the steep-edge cap (Sec. II-B)
    bad = ww.default_params(steep_rad=float("nan"))
    st = ww.lib().ww_costs_noalloc(dummy, 0, dummy, None, 100, 100, lut.handle, ctypes.byref(bad), dummy, None)
    assert st == ww.WW_ERR_INVALID_ARG


def _noise(seed, m, n):
    rng = np.random.default_rng(seed)
    ph = rng.uniform(-np.pi, np.pi, (m, n)).astype(np.float32)
    coh = rng.uniform(0, 1, (m, n)).astype(np.float32)
    mask = (rng.uniform(size=(m, n)) > 0.05).astype(np.uint8)
    return synth.Interferogram(phase=ph, coh=coh, mask=mask, nlooks=4.0, truth=np.zeros((m, n)))


@pytest.mark.gpu
def test_noalloc_matches_workspace_costs_on_consecutive_calls():
    import torch

    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    # first call: pure noise, far over the 3% steep cap (selection path uses the
    # scratch); second call: a smooth scene with a different table and size
    cases = [(_noise(3, 211, 173), np.arange(128 * 256, dtype=np.int64).reshape(128, 256) % 20011),
             (synth.small_random(8, 300, 333, mask_frac=0.1, want_complex=True, lo=0.05, hi=0.9),
              (np.arange(128 * 256, dtype=np.int64).reshape(128, 256) * 7) % 30011)]
    ws = ww.Workspace(300, 333)
    for x, tab in cases:
        lut = ww.Lut.from_table(x.nlooks, tab.astype(np.int16))
        ifg = dev(x.ifg) if x.is_complex else dev(x.phase)
        coh, mask = dev(x.coh), dev(x.mask)
        ref = ww.costs(ifg, coh, lut, ws, mask).cpu().numpy()
        got = ww.costs_noalloc(ifg, coh, lut, mask).cpu().numpy()
        assert np.array_equal(got, ref)
        assert np.count_nonzero(ref) > 0


@pytest.mark.gpu
def test_noalloc_call_after_the_first_is_captured_into_a_graph():
    """After its first call on a device (which looks up the scratch array's
    address), the entry point enqueues only an upload from the table's
    page-locked copy, two memsets and kernel launches, so a later call can be
    captured into a CUDA graph; each replay gives ww_costs's planes."""
    import torch

    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    x = _noise(5, 190, 207)
    tab = ((np.arange(128 * 256, dtype=np.int64).reshape(128, 256) * 13) % 25013).astype(np.int16)
    lut = ww.Lut.from_table(x.nlooks, tab)
    ifg, coh, mask = dev(x.phase), dev(x.coh), dev(x.mask)
    ref = ww.costs(ifg, coh, lut, ww.Workspace(190, 207), mask).cpu().numpy()
    out = torch.empty((4, 190, 207), dtype=torch.int16, device="cuda")
    ww.costs_noalloc(ifg, coh, lut, mask, out=out)  # first call on this device: outside the capture
    torch.cuda.synchronize()
    out.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=s):
        ww.costs_noalloc(ifg, coh, lut, mask, out=out)
    for _ in range(2):
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref)
