"""Shared helpers for the GPU parity tests (inputs, oracle references, checks)."""
import os

import numpy as np

import oracle
import paper_2609_36267_b300 as ww
from paper_2609_36267_b300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


def golden_table(L):
    return np.load(os.path.join(GOLDEN, f"lut_oracle_L{float(L):g}.npz"))["table"]


def probe_table():
    k = np.arange(128)[:, None]
    j = np.arange(256)[None, :]
    return (k * 256 + j).astype(np.int16)


def to_dev(x):
    import torch

    if x is None:
        return None
    t = torch.from_numpy(np.ascontiguousarray(x))
    return t.cuda()


def device_inputs(x: synth.Interferogram, use_complex=None):
    """-> (ifg tensor, coh tensor, mask tensor) for an Interferogram."""
    cplx = x.is_complex if use_complex is None else use_complex
    ifg = to_dev(x.ifg) if cplx else to_dev(x.phase)
    return ifg, to_dev(x.coh), to_dev(x.mask)


def oracle_prepare(x: synth.Interferogram, use_complex=None):
    cplx = x.is_complex if use_complex is None else use_complex
    if cplx:
        return oracle.prepare(x.coh, x.mask, ifg=x.ifg)
    return oracle.prepare(x.coh, x.mask, phase=x.phase)


def oracle_pipeline(x, table, steep_cap_ppm=30000, use_complex=None):
    psi, coh, valid = oracle_prepare(x, use_complex)
    res, g = oracle.residues(psi)
    costs, nsteep = oracle.costs(psi, coh, valid, table, steep_cap_ppm=steep_cap_ppm)
    return dict(psi=psi, coh=coh, valid=valid, res=res, g=g, costs=costs, nsteep=nsteep)


def numpy_certificate(res, g, costs, flows, pot):
    """Independent vectorised check (harness code): capacity, conservation at
    every node and at G, non-negative reduced cost on every residual arc.
    Returns (ok, total_cost, detail)."""
    res = np.asarray(res, np.int64)
    _, m, n = costs.shape
    R, C = m - 1, n - 1
    G = R * C
    dkh = flows[0].astype(np.int64)
    dkv = flows[1].astype(np.int64)
    if np.abs(dkh).max(initial=0) > 1 or np.abs(dkv).max(initial=0) > 1:
        return False, None, "capacity"
    if dkh[:, n - 1].any() or dkv[m - 1, :].any():
        return False, None, "flow on missing edge"
    node = np.full((m + 1, n + 1), G, np.int64)  # node index of loop (i-1, j-1) at [i, j]
    node[1:m, 1:n] = np.arange(G).reshape(R, C)
    pot = np.asarray(pot, np.int64)
    c = costs.astype(np.int64)
    total = 0
    bad = 0
    # h(i,j): above node (i-1,j), below node (i,j); + arc above->below
    ab = node[0:m, 1:n]  # above, indexed [i, j] for j < n-1
    be = node[1:m + 1, 1:n]
    dk = dkh[:, : n - 1]
    cp, cm = c[0][:, : n - 1], c[1][:, : n - 1]
    pa, pb = pot[ab], pot[be]
    bad += np.count_nonzero((dk != 1) & (cp - pa + pb < 0))
    bad += np.count_nonzero((dk == 1) & (-cp - pb + pa < 0))
    bad += np.count_nonzero((dk != -1) & (cm - pb + pa < 0))
    bad += np.count_nonzero((dk == -1) & (-cm - pa + pb < 0))
    total += int(cp[dk == 1].sum() + cm[dk == -1].sum())
    # v(i,j): left node (i,j-1), right node (i,j); + arc right->left
    le = node[1:m, 0:n]
    ri = node[1:m, 1:n + 1]
    dk = dkv[: m - 1, :]
    cp, cm = c[2][: m - 1, :], c[3][: m - 1, :]
    pa, pb = pot[ri], pot[le]
    bad += np.count_nonzero((dk != 1) & (cp - pa + pb < 0))
    bad += np.count_nonzero((dk == 1) & (-cp - pb + pa < 0))
    bad += np.count_nonzero((dk != -1) & (cm - pb + pa < 0))
    bad += np.count_nonzero((dk == -1) & (-cm - pa + pb < 0))
    total += int(cp[dk == 1].sum() + cm[dk == -1].sum())
    if bad:
        return False, total, f"{bad} negative reduced costs"
    net = dkh[1:, : n - 1] - dkh[:-1, : n - 1] + dkv[: m - 1, : n - 1] - dkv[: m - 1, 1:]
    if not np.array_equal(net, res.reshape(R, C)):
        return False, total, "conservation"
    gnet = dkh[0, : n - 1].sum() - dkh[m - 1, : n - 1].sum() - dkv[: m - 1, 0].sum() + dkv[: m - 1, n - 1].sum()
    if gnet != g:
        return False, total, "ground conservation"
    return True, total, "ok"


def band_certificate(res, costs, flows, pot, a, b):
    """numpy_certificate restricted to pixel rows [a, b): capacity, the reduced
    cost of every residual arc of the h edges of rows a..b-1 and the v edges of
    rows a..min(b, m-1)-1, conservation at the nodes of rows a..min(b, m-1)-1.
    res is the (m-1) x (n-1) residue plane.  Returns the number of violations."""
    _, m, n = costs.shape
    R, C = m - 1, n - 1
    G = R * C
    pot = np.asarray(pot)

    def node(i, j):  # node index array for row i (scalar) and column array j; G outside
        i = np.full_like(j, i)
        inside = (i >= 0) & (i < R) & (j >= 0) & (j < C)
        return np.where(inside, i * C + j, G)

    bad = 0
    jh = np.arange(n - 1)
    jv = np.arange(n)
    for i in range(a, b):
        dk = flows[0, i, : n - 1].astype(np.int64)
        bad += np.count_nonzero(np.abs(dk) > 1)
        cp, cm = costs[0, i, : n - 1].astype(np.int64), costs[1, i, : n - 1].astype(np.int64)
        pa, pb = pot[node(i - 1, jh)], pot[node(i, jh)]
        bad += np.count_nonzero((dk != 1) & (cp - pa + pb < 0))
        bad += np.count_nonzero((dk == 1) & (-cp - pb + pa < 0))
        bad += np.count_nonzero((dk != -1) & (cm - pb + pa < 0))
        bad += np.count_nonzero((dk == -1) & (-cm - pa + pb < 0))
        if i < m - 1:
            dk = flows[1, i, :].astype(np.int64)
            bad += np.count_nonzero(np.abs(dk) > 1)
            cp, cm = costs[2, i, :].astype(np.int64), costs[3, i, :].astype(np.int64)
            pa, pb = pot[node(i, jv)], pot[node(i, jv - 1)]
            bad += np.count_nonzero((dk != 1) & (cp - pa + pb < 0))
            bad += np.count_nonzero((dk == 1) & (-cp - pb + pa < 0))
            bad += np.count_nonzero((dk != -1) & (cm - pb + pa < 0))
            bad += np.count_nonzero((dk == -1) & (-cm - pa + pb < 0))
            net = (flows[0, i + 1, : n - 1].astype(np.int64) - flows[0, i, : n - 1]
                   + flows[1, i, : n - 1].astype(np.int64) - flows[1, i, 1:])
            bad += np.count_nonzero(net != res[i])
    return bad


def device_array(ptr, shape, dtype):
    """A host copy of a device array given by its raw address (library workspace memory)."""
    import ctypes

    import torch

    count = int(np.prod(shape)) * np.dtype(dtype).itemsize
    out = np.empty(shape, dtype)
    torch.cuda.synchronize()
    lib = "/usr/local/cuda/lib64/libcudart.so"
    cudart = ctypes.CDLL(lib if os.path.exists(lib) else "libcudart.so")
    cudart.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
    assert cudart.cudaMemcpy(out.ctypes.data, ctypes.c_void_p(ptr), count, 2) == 0  # device to host
    return out
