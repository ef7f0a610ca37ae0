"""CPU oracle for the Whirlwind MCF unwrapper hot path.

TEST INFRASTRUCTURE ONLY.  A plain, slow, single-threaded C++ restatement of
the paper's definitions (Sec. II: Eq. 1 residues, Eqs. 4-7 costs, Eq. 2 MCF by
successive shortest paths, integer integration).  Only the tests, the smoke
check and the benchmark's CPU-baseline leg use it; the product path never does.
It shares no code with the CUDA library.

Pinned functions and their pins (see tests/test_oracle_*.py):
  residues        vortex, noise-free Itoh field, charge balance, brute recount
  phase (CORDIC)  numpy arctan2 within 2 ulp, exact axis cases
  costs/indices   hand-evaluated index formula, probe tables, masks, steep rule
  MCF             exhaustive enumeration (<= 5x5), certificate, max-flow
  integration     rewrap identity, Itoh integration on sub-Nyquist fields
  components      scipy.ndimage.label (every edge reliable), networkx
                  components, the reliability rule case by case
  bridge          a smooth field cut into regions with whole-cycle offsets is
                  restored up to the largest region's cycles; offset
                  invariance; nearest-region attachment; region-only medians
  Lee pdf         mpmath hypergeometric closed form, single-look closed form,
                  normalisation, Monte Carlo looks
  Touzi pdf       mpmath hypergeometric, gamma=0 closed form, normalisation,
                  Monte Carlo looks
  sigma_alpha     pi/sqrt(3) for a uniform pdf (the limit stated in Sec. II-B)
  P0/P+/costs     P0+P+ +P- = 1, costs >= 0, the orderings stated in Sec. II-B
  cost variants   phasor slope vs numpy's angle of the phasor sum, constant
                  gradients; bilinear lookup exact on linear tables, centres, edges
  multilook/Eq. 3 numpy fp64 sums within fp32 rounding, gamma = 1 for
                  proportional images, scale and phase invariance
  Goldstein       alpha = 0 keeps a single patch-interior field, a pure fringe
                  pattern is kept, noise is reduced (numpy FFT restatement)
  cycle transfer  rewrap identity, K = 0 when the filtered field equals psi
Parity unpinned: the absolute LUT values (the paper prints no table), and
sigma_alpha's formula away from gamma -> 0 (the paper gives only the limit).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SOURCES = ["wwo_grid.cpp", "wwo_mcf.cpp", "wwo_lut.cpp"]


def build(force: bool = False) -> str:
    """Compile liboracle.so with plain g++ (-O2, no FP contraction)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "wwo.h")])
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp] + srcs
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        i32 = ctypes.c_int32
        d = ctypes.c_double
        f = ctypes.c_float
        L.wwo_phase_from_complex.argtypes = [P, i64, P]
        L.wwo_prepare.argtypes = [P, P, P, P, i64, i64, P, P, P]
        L.wwo_residues.argtypes = [P, i64, i64, P, P]
        L.wwo_alpha_hat.argtypes = [P, P, i64, i64, i32, P]
        L.wwo_costs.argtypes = [P, P, P, i64, i64, P, i32, f, i32, P]
        L.wwo_costs.restype = i64
        L.wwo_integrate.argtypes = [P, P, P, i64, i64, P, P]
        L.wwo_solve_mcf.argtypes = [P, i32, P, i64, i64, P, P, P]
        L.wwo_solve_mcf.restype = ctypes.c_int
        L.wwo_check_certificate.argtypes = [P, i32, P, i64, i64, P, P, P, P]
        L.wwo_check_certificate.restype = ctypes.c_int
        L.wwo_flow_cost.argtypes = [P, i64, i64, P]
        L.wwo_flow_cost.restype = i64
        L.wwo_brute_force.argtypes = [P, P, i64, i64]
        L.wwo_brute_force.restype = i64
        L.wwo_feasible.argtypes = [P, i32, i64, i64]
        L.wwo_feasible.restype = ctypes.c_int
        L.wwo_lee_pdf.argtypes = [d, d, d]
        L.wwo_lee_pdf.restype = d
        L.wwo_touzi_pdf.argtypes = [d, d, d]
        L.wwo_touzi_pdf.restype = d
        L.wwo_marginal_pdf.argtypes = [d, d, i32, i32, P]
        L.wwo_marginal_pdf.restype = ctypes.c_int
        L.wwo_sigma_from_pdf.argtypes = [P, i32]
        L.wwo_sigma_from_pdf.restype = d
        L.wwo_probabilities.argtypes = [P, i32, d, P, P, P, P]
        L.wwo_lut_build.argtypes = [d, i32, i32, P, P, P]
        L.wwo_multilook.argtypes = [P, P, i64, i64, i32, i32, P, P]
        L.wwo_alpha_hat2.argtypes = [P, P, i64, i64, i32, i32, P]
        L.wwo_costs2.argtypes = [P, P, P, i64, i64, P, P, i32, i32, i32, f, i32, P]
        L.wwo_costs2.restype = i64
        L.wwo_lut_build.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def phase_from_complex(ifg: np.ndarray) -> np.ndarray:
    z = np.ascontiguousarray(ifg, dtype=np.complex64)
    out = np.empty(z.shape, np.float32)
    lib().wwo_phase_from_complex(_p(z), z.size, _p(out))
    return out


def prepare(coh, mask, phase=None, ifg=None):
    """-> (psi, coh, valid) with masked/non-finite pixels zeroed (psi=0, coh=0)."""
    coh = np.ascontiguousarray(coh, np.float32)
    mask = np.ascontiguousarray(mask, np.uint8)
    m, n = coh.shape
    psi = np.empty((m, n), np.float32)
    co = np.empty((m, n), np.float32)
    valid = np.empty((m, n), np.uint8)
    if ifg is not None:
        z = np.ascontiguousarray(ifg, np.complex64)
        lib().wwo_prepare(None, _p(z), _p(coh), _p(mask), m, n, _p(psi), _p(co), _p(valid))
    else:
        ph = np.ascontiguousarray(phase, np.float32)
        lib().wwo_prepare(_p(ph), None, _p(coh), _p(mask), m, n, _p(psi), _p(co), _p(valid))
    return psi, co, valid


def residues(psi: np.ndarray):
    psi = np.ascontiguousarray(psi, np.float32)
    m, n = psi.shape
    r = np.empty((m - 1, n - 1), np.int8)
    g = np.zeros(1, np.int32)
    lib().wwo_residues(_p(psi), m, n, _p(r), _p(g))
    return r, int(g[0])


def alpha_hat(psi, valid, half_width=2, mode=0):
    """Slope estimate planes [2][m][n]; mode 0 = fixed-point mean of the wrapped
    gradients, mode 1 = argument of the sum of their unit phasors (CORDIC)."""
    psi = np.ascontiguousarray(psi, np.float32)
    valid = np.ascontiguousarray(valid, np.uint8)
    m, n = psi.shape
    out = np.empty((2, m, n), np.float32)
    lib().wwo_alpha_hat2(_p(psi), _p(valid), m, n, half_width, int(mode), _p(out))
    return out


def costs(psi, coh, valid, table, half_width=2, steep_rad=1.0, steep_cap_ppm=30000, slope_mode=0, lookup=0,
          ratio=None):
    """Cost planes [4][m][n] and the number of steep edges zeroed.  slope_mode:
    0 fixed-point mean, 1 phasor sum; lookup: 0 nearest bin of `table`, 1
    bilinear interpolation of `ratio` (float32 [128,256], 100 ln(P0/P+))."""
    psi = np.ascontiguousarray(psi, np.float32)
    coh = np.ascontiguousarray(coh, np.float32)
    valid = np.ascontiguousarray(valid, np.uint8)
    table = np.ascontiguousarray(table, np.int16)
    assert table.size == 128 * 256
    rt = np.ascontiguousarray(ratio if ratio is not None else np.zeros((128, 256)), np.float32)
    assert rt.size == 128 * 256 and (lookup == 0 or ratio is not None)
    m, n = psi.shape
    out = np.empty((4, m, n), np.int16)
    nsteep = lib().wwo_costs2(_p(psi), _p(coh), _p(valid), m, n, _p(table), _p(rt), half_width, int(slope_mode),
                              int(lookup), float(steep_rad), int(steep_cap_ppm), _p(out))
    return out, int(nsteep)


def integrate(psi, valid, flows):
    psi = np.ascontiguousarray(psi, np.float32)
    valid = np.ascontiguousarray(valid, np.uint8)
    flows = np.ascontiguousarray(flows, np.int8)
    m, n = psi.shape
    unw = np.empty((m, n), np.float32)
    cyc = np.empty((m, n), np.int32)
    lib().wwo_integrate(_p(psi), _p(valid), _p(flows), m, n, _p(unw), _p(cyc))
    return unw, cyc


def solve_mcf(res, ground, costs_planes):
    res = np.ascontiguousarray(res, np.int8)
    c = np.ascontiguousarray(costs_planes, np.int16)
    _, m, n = c.shape
    flows = np.zeros((2, m, n), np.int8)
    pot = np.zeros((m - 1) * (n - 1) + 1, np.int64)
    tc = np.zeros(1, np.int64)
    st = lib().wwo_solve_mcf(_p(res), int(ground), _p(c), m, n, _p(flows), _p(pot), _p(tc))
    return st, flows, pot, int(tc[0])


def check_certificate(res, ground, costs_planes, flows, potentials):
    """-> (code, total_cost, bad_index); code 0 = optimal flow with valid potentials."""
    res = np.ascontiguousarray(res, np.int8)
    c = np.ascontiguousarray(costs_planes, np.int16)
    fl = np.ascontiguousarray(flows, np.int8)
    pot = np.ascontiguousarray(potentials, np.int64)
    _, m, n = c.shape
    tc = np.zeros(1, np.int64)
    bad = np.zeros(1, np.int64)
    code = lib().wwo_check_certificate(_p(res), int(ground), _p(c), m, n, _p(fl), _p(pot), _p(tc), _p(bad))
    return code, int(tc[0]), int(bad[0])


def flow_cost(costs_planes, flows):
    c = np.ascontiguousarray(costs_planes, np.int16)
    fl = np.ascontiguousarray(flows, np.int8)
    _, m, n = c.shape
    return int(lib().wwo_flow_cost(_p(c), m, n, _p(fl)))


def brute_force(psi, costs_planes):
    psi = np.ascontiguousarray(psi, np.float32)
    c = np.ascontiguousarray(costs_planes, np.int16)
    m, n = psi.shape
    assert m * n <= 30
    return int(lib().wwo_brute_force(_p(psi), _p(c), m, n))


def feasible(res, ground):
    res = np.ascontiguousarray(res, np.int8)
    m, n = res.shape[0] + 1, res.shape[1] + 1
    return bool(lib().wwo_feasible(_p(res), int(ground), m, n))


def lee_pdf(eta, gamma, L):
    return float(lib().wwo_lee_pdf(float(eta), float(gamma), float(L)))


def touzi_pdf(gh, gamma, L):
    return float(lib().wwo_touzi_pdf(float(gh), float(gamma), float(L)))


def marginal_pdf(L, gh, nh=512, lambda_panels=8):
    f = np.empty(2 * nh + 1, np.float64)
    st = lib().wwo_marginal_pdf(float(L), float(gh), nh, lambda_panels, _p(f))
    assert st == 0
    return f


def sigma_from_pdf(f):
    f = np.ascontiguousarray(f, np.float64)
    nh = (f.size - 1) // 2
    return float(lib().wwo_sigma_from_pdf(_p(f), nh))


def probabilities(f, alpha_hat_value):
    f = np.ascontiguousarray(f, np.float64)
    nh = (f.size - 1) // 2
    out = np.zeros(4, np.float64)
    o = [out[i:i + 1] for i in range(4)]
    lib().wwo_probabilities(_p(f), nh, float(alpha_hat_value), _p(o[0]), _p(o[1]), _p(o[2]), _p(o[3]))
    return dict(p0=out[0], pplus=out[1], pminus=out[2], sigma=out[3])


def lut_build(L, nh=8192, lambda_panels=8):
    """-> (cost100 float64 [128,256], table int16 [128,256], ratio100 float32 [128,256]);
    slow (minutes at the default)."""
    c = np.empty((128, 256), np.float64)
    t = np.empty((128, 256), np.int16)
    r = np.empty((128, 256), np.float32)
    st = lib().wwo_lut_build(float(L), nh, lambda_panels, _p(c), _p(t), _p(r))
    assert st == 0
    return c, t, r


def components(costs_planes, flows, valid, threshold: int):
    """Connected-component labels (Sec. II-D), plain breadth-first search.

    A pixel edge is reliable when both of its pixels are valid and moving its
    ambiguity difference dk by +1 or by -1 would raise the MCF objective by more
    than `threshold` (>= 0).  With the unit-capacity costs of Sec. II-B that
    change is +c+ / +c- for an edge without flow, and -c+ or -c- (removing the
    flow) for an edge that carries flow, so: reliable <=> dk = 0 and
    min(c+, c-) > threshold.  Planes: h edge (i,j)-(i,j+1) has dk = flows[0],
    c+ = costs[0], c- = costs[1]; v edge (i,j)-(i+1,j) has dk = flows[1],
    c+ = costs[2], c- = costs[3].  Labels grow over reliable edges; a pixel's
    label is 1 + the smallest row-major index in its component, 0 where invalid.
    """
    from collections import deque

    c = np.asarray(costs_planes, np.int64)
    fl = np.asarray(flows, np.int64)
    ok = np.asarray(valid, bool)
    m, n = ok.shape
    rel_h = np.zeros((m, n), bool)
    rel_v = np.zeros((m, n), bool)
    rel_h[:, :-1] = ok[:, :-1] & ok[:, 1:] & (fl[0, :, :-1] == 0) & (np.minimum(c[0, :, :-1], c[1, :, :-1]) > threshold)
    rel_v[:-1, :] = ok[:-1, :] & ok[1:, :] & (fl[1, :-1, :] == 0) & (np.minimum(c[2, :-1, :], c[3, :-1, :]) > threshold)
    labels = np.zeros((m, n), np.int64)
    for s in range(m * n):  # row-major: the first pixel reached is its component's smallest index
        i0, j0 = divmod(s, n)
        if not ok[i0, j0] or labels[i0, j0]:
            continue
        labels[i0, j0] = s + 1
        q = deque([(i0, j0)])
        while q:
            i, j = q.popleft()
            for a, b, edge in ((i, j + 1, j + 1 < n and rel_h[i, j]), (i, j - 1, j > 0 and rel_h[i, j - 1]),
                               (i + 1, j, i + 1 < m and rel_v[i, j]), (i - 1, j, i > 0 and rel_v[i - 1, j])):
                if edge and not labels[a, b]:
                    labels[a, b] = s + 1
                    q.append((a, b))
    return labels.astype(np.int32)


def bridge(unwrapped, valid, window: int = 65):
    """Bridging of mask-separated regions (Sec. II-D), plainly.

    Regions are the 4-connected components of the valid pixels.  Taken in order
    of decreasing size (ties: smaller first pixel first), every region after the
    first is attached to the nearest region already taken, through the closest
    pair of pixels (squared Euclidean distance; ties: smaller parent-region
    rank, then smaller pixel indices).  Across each such edge the offset is
    round((median_parent - median_child) / 2pi) cycles, each median taken over
    the unwrapped phase of the endpoint's region inside a window x window box
    centred on the endpoint (numpy median, round half to even); the child's
    phase is shifted by 2pi times that offset before its own children are
    attached, so offsets propagate from parent to child.  Returns (bridged
    phase float64, cycle offset per pixel int64, region index per pixel, -1
    where invalid), regions numbered in their processing order."""
    u = np.array(unwrapped, np.float64)
    ok = np.asarray(valid, bool)
    m, n = ok.shape
    costs = np.ones((4, m, n), np.int16)
    flows = np.zeros((2, m, n), np.int8)
    lab = components(costs, flows, ok, 0).astype(np.int64)  # every edge between valid pixels
    roots = np.unique(lab[lab > 0])
    sizes = {r: int((lab == r).sum()) for r in roots}
    order = sorted(roots, key=lambda r: (-sizes[r], r))
    region = np.full((m, n), -1, np.int64)
    for rank, r in enumerate(order):
        region[lab == r] = rank
    shift = np.zeros((m, n), np.int64)
    h = window // 2
    pix = [np.argwhere(region == k) for k in range(len(order))]

    def median_at(i, j, k):
        box = region[max(0, i - h):i + h + 1, max(0, j - h):j + h + 1] == k
        vals = (u + 2 * np.pi * shift)[max(0, i - h):i + h + 1, max(0, j - h):j + h + 1][box]
        return float(np.median(vals))

    for k in range(1, len(order)):
        best = None
        for q in range(k):
            a, b = pix[q], pix[k]
            d = ((a[:, None, :] - b[None, :, :]) ** 2).sum(axis=2)
            flat = int(np.argmin(d))  # row-major over (parent pixel, child pixel): smallest indices on ties
            ia, ib = divmod(flat, d.shape[1])
            key = (int(d.flat[flat]), q)
            if best is None or key < best[0]:
                best = (key, tuple(a[ia]), tuple(b[ib]))
        _, pa, pb = best
        off = int(np.rint((median_at(*pa, region[pa]) - median_at(*pb, k)) / (2 * np.pi)))
        shift[region == k] = off  # the parent's median already includes its own shift
    out = np.where(ok, u + 2 * np.pi * shift, np.nan)
    return out, shift, region


def multilook(slc1, slc2, looks_y: int, looks_x: int):
    """Multilooked interferogram and Eq. (3) sample coherence from two SLC images
    (complex64 [M, N]) over ly x lx looks: S12 = sum z1 conj(z2), gamma =
    |S12| / sqrt(S11 S22) (clamped to 1; 0 when a power is 0), fp32 in a fixed
    order (row-major over the looks, every product and sum rounded once).
    -> (ifg complex64 [M//ly, N//lx], coh float32)."""
    z1 = np.ascontiguousarray(slc1, np.complex64)
    z2 = np.ascontiguousarray(slc2, np.complex64)
    M, N = z1.shape
    m, n = M // looks_y, N // looks_x
    ifg = np.empty((m, n), np.complex64)
    coh = np.empty((m, n), np.float32)
    lib().wwo_multilook(_p(z1), _p(z2), M, N, int(looks_y), int(looks_x), _p(ifg), _p(coh))
    return ifg, coh


def goldstein(ifg, alpha=0.5, patch=32, step=16, smooth=3):
    """Adaptive power-spectrum (Goldstein) filter of a wrapped interferogram in
    overlapping Fourier-domain patches (Sec. II-D), plainly, in float64.

    Patches of patch x patch pixels start at every multiple of `step` in both
    directions that lies inside the image (pixels beyond the image count as 0).
    Per patch: Z = FFT2(patch); S = the smooth x smooth circular box mean of |Z|,
    divided by its maximum; Z' = Z S^alpha; z' = IFFT2(Z').  The patches are
    added with the separable triangular weight w(t) = 1 - |(2t + 1)/patch - 1|
    (t = 0 .. patch-1 along each axis) and the sum is divided by the summed
    weights.  -> complex128 [m, n]."""
    z = np.asarray(ifg, np.complex128)
    m, n = z.shape
    t = np.arange(patch)
    w1 = 1.0 - np.abs((2 * t + 1) / patch - 1.0)
    w = np.outer(w1, w1)
    acc = np.zeros((m, n), np.complex128)
    wsum = np.zeros((m, n), np.float64)
    h = smooth // 2
    for y0 in range(0, m, step):
        for x0 in range(0, n, step):
            blk = np.zeros((patch, patch), np.complex128)
            ys, xs = min(patch, m - y0), min(patch, n - x0)
            blk[:ys, :xs] = z[y0:y0 + ys, x0:x0 + xs]
            Z = np.fft.fft2(blk)
            a = np.abs(Z)
            S = np.zeros_like(a)
            for dy in range(-h, h + 1):
                for dx in range(-h, h + 1):
                    S += np.roll(np.roll(a, dy, axis=0), dx, axis=1)
            S /= smooth * smooth
            mx = S.max()
            H = (S / mx) ** alpha if mx > 0 else np.zeros_like(S)
            out = np.fft.ifft2(Z * H)
            acc[y0:y0 + ys, x0:x0 + xs] += (w * out)[:ys, :xs]
            wsum[y0:y0 + ys, x0:x0 + xs] += w[:ys, :xs]
    return acc / wsum


def transfer_cycles(unwrapped_filtered, psi, valid):
    """The integer solution of a preprocessed (filtered) phase moved to the
    original wrapped phase psi (Sec. II-D): K = rint((phi_f - psi) / 2pi) in
    float64 (half to even), phi = fp32(psi + 2pi K) with the integration's
    single rounding; NaN where invalid or where phi_f is NaN.
    -> (unwrapped float32, cycles int32)."""
    pf = np.asarray(unwrapped_filtered, np.float32).astype(np.float64)
    ps = np.asarray(psi, np.float32)
    ok = np.asarray(valid, bool) & ~np.isnan(pf)
    two_pi = 6.283185307179586
    K = np.where(ok, np.rint((pf - ps.astype(np.float64)) / two_pi), 0.0).astype(np.int64)
    out = (ps.astype(np.float64) + K.astype(np.float64) * two_pi).astype(np.float32)
    out[~ok] = np.nan
    return out, K.astype(np.int32)
