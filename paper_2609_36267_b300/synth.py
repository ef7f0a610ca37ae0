"""Seeded synthetic interferograms shaped like the paper's workloads.

This module only makes inputs: wrapped phase (or the complex interferogram),
sample coherence, a validity mask and the number of looks.  It holds none of the
unwrapper's arithmetic (no residues, costs, flows or integration), so both the
CUDA path and the CPU oracle can consume its output.

Multilook noise is drawn exactly, without simulating each look.  For L looks of
two unit-variance circular complex Gaussians with correlation gamma, write
z2 = gamma*z1 + sqrt(1-gamma^2)*w with w independent of z1.  Then
  A = sum|z1|^2 ~ Gamma(L, 1),
  sum z1 w^* = sqrt(A) * nu with nu ~ CN(0, 1),
  sum|w|^2 = |nu|^2 + Q with Q ~ Gamma(L - 1, 1) independent,
so the Hermitian product C = sum z1 z2^* and the powers A, B = sum|z2|^2 follow
from four draws per pixel.  The sample coherence is the estimator of Sec. II-B
Eq. (3), |C| / sqrt(A B); the interferogram is C * exp(i * truth).  Non-integer
L (equivalent looks) is supported because Gamma(L) is.

Every generator takes an integer seed and uses numpy's PCG64.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * np.pi


@dataclass
class Interferogram:
    """One synthetic unwrap request.

    phase:  float32 (m, n) wrapped phase in [-pi, pi] (always present)
    ifg:    complex64 (m, n) interferogram, or None for phase-only inputs
    coh:    float32 (m, n) sample coherence
    mask:   uint8 (m, n), 1 = valid, 0 = masked
    nlooks: effective number of looks L (> 1)
    truth:  float64 (m, n) noise-free unwrapped phase (radians)
    """

    phase: np.ndarray
    coh: np.ndarray
    mask: np.ndarray
    nlooks: float
    truth: np.ndarray
    ifg: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.phase.shape

    @property
    def is_complex(self) -> bool:
        return self.ifg is not None


def smooth_field(rng: np.random.Generator, m: int, n: int, lo: float, hi: float,
                 corr_px: float = 32.0) -> np.ndarray:
    """Smooth random field rescaled to [lo, hi].

    White noise on a grid coarsened by corr_px/2, a separable 1-2-1 blur applied
    three times there, then bilinear upsampling to (m, n).  Cheap at 74 Mpixel.
    """
    step = max(corr_px / 2.0, 1.0)
    cm = int(np.ceil(m / step)) + 3
    cn = int(np.ceil(n / step)) + 3
    c = rng.standard_normal((cm, cn))
    for _ in range(3):
        c = 0.25 * np.roll(c, 1, 0) + 0.5 * c + 0.25 * np.roll(c, -1, 0)
        c = 0.25 * np.roll(c, 1, 1) + 0.5 * c + 0.25 * np.roll(c, -1, 1)
    yi = np.arange(m) / step + 1.0
    xi = np.arange(n) / step + 1.0
    y0 = np.floor(yi).astype(np.int64)
    x0 = np.floor(xi).astype(np.int64)
    fy = (yi - y0)[:, None]
    fx = (xi - x0)[None, :]
    out = np.empty((m, n), dtype=np.float64)
    # row-chunked bilinear interpolation keeps peak memory near one output copy
    ch = 1024
    for r in range(0, m, ch):
        sl = slice(r, min(m, r + ch))
        a = c[y0[sl]][:, x0]
        b = c[y0[sl]][:, x0 + 1]
        cc = c[y0[sl] + 1][:, x0]
        d = c[y0[sl] + 1][:, x0 + 1]
        fys = fy[sl]
        out[sl] = (a * (1 - fx) + b * fx) * (1 - fys) + (cc * (1 - fx) + d * fx) * fys
    mn, mx = out.min(), out.max()
    out -= mn
    out *= (hi - lo) / max(mx - mn, 1e-300)
    out += lo
    return out


def multilook_noise(rng: np.random.Generator, gamma: np.ndarray, nlooks: float):
    """Exact L-look Hermitian product C and sample coherence for coherence gamma.

    Returns (C complex128, coh float64).  See the module docstring.
    """
    shape = gamma.shape
    g = np.clip(gamma, 0.0, 1.0)
    s = np.sqrt(1.0 - g * g)
    a = rng.gamma(nlooks, 1.0, size=shape)
    nu = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * np.sqrt(0.5)
    if nlooks > 1.0:
        q = rng.gamma(nlooks - 1.0, 1.0, size=shape)
    else:
        q = np.zeros(shape)
    sa = np.sqrt(a)
    c = g * a + s * sa * nu
    b = g * g * a + s * s * (np.abs(nu) ** 2 + q) + 2.0 * g * s * sa * nu.real
    coh = np.abs(c) / np.sqrt(a * b)
    return c, np.clip(coh, 0.0, 1.0)


def brute_force_looks(rng: np.random.Generator, gamma: float, nlooks: int, count: int):
    """Reference construction with every look simulated (for statistical checks).

    Returns (phase of sum z1 z2^*, sample coherence) for `count` independent
    multilooked samples at true coherence gamma.
    """
    z1 = (rng.standard_normal((count, nlooks)) + 1j * rng.standard_normal((count, nlooks))) * np.sqrt(0.5)
    w = (rng.standard_normal((count, nlooks)) + 1j * rng.standard_normal((count, nlooks))) * np.sqrt(0.5)
    z2 = gamma * z1 + np.sqrt(1 - gamma * gamma) * w
    c = np.sum(z1 * np.conj(z2), axis=1)
    a = np.sum(np.abs(z1) ** 2, axis=1)
    b = np.sum(np.abs(z2) ** 2, axis=1)
    return np.angle(c), np.abs(c) / np.sqrt(a * b)


def _finish(rng, truth, gamma, nlooks, mask, want_complex, meta):
    c, coh = multilook_noise(rng, gamma, nlooks)
    ifg = c * np.exp(1j * truth)
    phase = np.angle(ifg).astype(np.float32)
    out = Interferogram(phase=phase, coh=coh.astype(np.float32), mask=mask.astype(np.uint8),
                        nlooks=float(nlooks), truth=truth, meta=meta)
    if want_complex:
        out.ifg = (ifg / max(nlooks, 1.0)).astype(np.complex64)
    return out


def _gaussian_bump(m, n, ci, cj, sigma, amp):
    i = np.arange(m)[:, None]
    j = np.arange(n)[None, :]
    return amp * np.exp(-((i - ci) ** 2 + (j - cj) ** 2) / (2.0 * sigma * sigma))


def _polygon_mask(rng, m, n, frac, nvert=12):
    """Random star-shaped polygon covering about `frac` of the image (1 inside)."""
    area = frac * m * n
    r0 = np.sqrt(area / np.pi)
    ci = rng.uniform(0.25 * m, 0.75 * m)
    cj = rng.uniform(0.25 * n, 0.75 * n)
    ang = np.sort(rng.uniform(0, 2 * np.pi, nvert))
    rad = r0 * rng.uniform(0.75, 1.25, nvert)
    i = np.arange(m)[:, None] - ci
    j = np.arange(n)[None, :] - cj
    theta = np.mod(np.arctan2(i, j), 2 * np.pi)
    rr = np.hypot(i, j)
    # radius of the polygon boundary along theta, by linear interpolation of the vertices
    a_ext = np.concatenate([ang - 2 * np.pi, ang, ang + 2 * np.pi])
    r_ext = np.concatenate([rad, rad, rad])
    rb = np.interp(theta, a_ext, r_ext)
    inside = rr <= rb
    # rescale the covered fraction to the target by one radial scaling
    got = inside.mean()
    if got > 0:
        inside = rr <= rb * np.sqrt(frac / got)
    return inside


def _blob_mask(rng, m, n, frac, blob_px=40.0):
    """Random blobs covering about `frac` of the image (1 inside a blob)."""
    f = smooth_field(rng, m, n, 0.0, 1.0, corr_px=blob_px)
    thr = np.quantile(f[:: max(1, m // 512), :: max(1, n // 512)], 1.0 - frac)
    return f > thr


def config1(seed: int = 1001) -> Interferogram:
    """256x256: 2-cycle ramp plus 3 Gaussian bumps; coherence in [0.2, 0.95]; L=9; float32 phase."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = n = 256
    j = np.arange(n)[None, :]
    truth = np.broadcast_to(TWO_PI * 2.0 * j / n, (m, n)).astype(np.float64).copy()
    for _ in range(3):
        amp = rng.uniform(2, 6) * rng.choice([-1.0, 1.0]) * TWO_PI
        sig = rng.uniform(20, 40)
        truth += _gaussian_bump(m, n, rng.uniform(0, m), rng.uniform(0, n), sig, amp)
    gamma = smooth_field(rng, m, n, 0.2, 0.95)
    mask = np.ones((m, n), np.uint8)
    return _finish(rng, truth, gamma, 9.0, mask, False, {"name": "single 256x256 ramp+bumps", "seed": seed})


def config2(seed: int = 2001, m: int = 2048, n: int = 2048, nlooks: float = 6.0) -> Interferogram:
    """2048x2048: two lobes (+15, -12 cycles) + 1-cycle ramp; decorrelated disk; 10% water; L=6; complex64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sc = min(m, n) / 2048.0
    j = np.arange(n)[None, :]
    truth = np.broadcast_to(TWO_PI * 1.0 * j / n, (m, n)).astype(np.float64).copy()
    c1 = (rng.uniform(0.35, 0.5) * m, rng.uniform(0.35, 0.5) * n)
    c2 = (c1[0] + rng.uniform(0.1, 0.2) * m, c1[1] + rng.uniform(0.1, 0.2) * n)
    truth += _gaussian_bump(m, n, c1[0], c1[1], rng.uniform(250, 400) * sc, 15.0 * TWO_PI)
    truth += _gaussian_bump(m, n, c2[0], c2[1], rng.uniform(250, 400) * sc, -12.0 * TWO_PI)
    gamma = smooth_field(rng, m, n, 0.3, 0.95)
    di, dj = rng.uniform(0.15, 0.85) * m, rng.uniform(0.15, 0.85) * n
    ii = np.arange(m)[:, None]
    jj = np.arange(n)[None, :]
    gamma[(ii - di) ** 2 + (jj - dj) ** 2 <= (150.0 * sc) ** 2] = 0.05
    water = _polygon_mask(rng, m, n, 0.10)
    mask = (~water).astype(np.uint8)
    return _finish(rng, truth, gamma, nlooks, mask, True, {"name": f"single {m}x{n} lobes+disk+water", "seed": seed})


def _strike_slip(m, n, p0, theta, fringes, depth):
    """Screw-dislocation surface phase: fringes * (2/pi) * atan(s/D) * 2pi, tapered along strike."""
    i = np.arange(m, dtype=np.float64)[:, None]
    j = np.arange(n, dtype=np.float64)[None, :]
    ux, uy = np.cos(theta), np.sin(theta)
    dx = j - p0[1]
    dy = i - p0[0]
    s = -dx * uy + dy * ux  # signed distance from the trace
    t = dx * ux + dy * uy  # distance along strike
    half = 0.45 * np.hypot(m, n)
    taper = np.clip(1.5 - np.abs(t) / half, 0.0, 1.0)
    return fringes * (2.0 / np.pi) * np.arctan(s / depth) * TWO_PI * taper, np.abs(s)


def config3(seed: int = 3001, m: int = 8192, n: int = 9000, nlooks: float = 50.0) -> Interferogram:
    """Large earthquake scene: two intersecting strike-slip ruptures (~40 fringes each),
    50-px decorrelated band along each trace, coherence [0.2, 0.9], 5% masked blobs, L=50, complex64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sc = min(m, n) / 8192.0
    th1 = rng.uniform(0.2, 0.5)
    th2 = th1 + np.pi / 2 + rng.uniform(-0.15, 0.15)
    p1 = (rng.uniform(0.4, 0.6) * m, rng.uniform(0.4, 0.6) * n)
    p2 = (p1[0] + rng.uniform(-0.1, 0.1) * m, p1[1] + rng.uniform(-0.1, 0.1) * n)
    ph1, s1 = _strike_slip(m, n, p1, th1, rng.uniform(18, 22), rng.uniform(300, 400) * sc)
    ph2, s2 = _strike_slip(m, n, p2, th2, rng.uniform(18, 22), rng.uniform(300, 400) * sc)
    truth = ph1 + ph2
    del ph1, ph2
    gamma = smooth_field(rng, m, n, 0.2, 0.9)
    band = (s1 <= 25.0 * max(sc, 0.25)) | (s2 <= 25.0 * max(sc, 0.25))
    del s1, s2
    gamma[band] = rng.uniform(0.02, 0.09, size=int(band.sum()))
    del band
    mask = (~_blob_mask(rng, m, n, 0.05)).astype(np.uint8)
    return _finish(rng, truth, gamma, nlooks, mask, True, {"name": f"earthquake {m}x{n}", "seed": seed})


def small_random(seed: int, m: int, n: int, nlooks: float = 9.0, mask_frac: float = 0.0,
                 lo: float = 0.15, hi: float = 0.95, fringes: float = 3.0, want_complex: bool = False,
                 corr_px: float = 8.0) -> Interferogram:
    """Small random case for tests: ramp + bump, coherence field, optional blob mask."""
    rng = np.random.Generator(np.random.PCG64(seed))
    j = np.arange(n)[None, :]
    truth = np.broadcast_to(TWO_PI * fringes * j / max(n, 1), (m, n)).astype(np.float64).copy()
    truth += _gaussian_bump(m, n, rng.uniform(0, m), rng.uniform(0, n), max(m, n) / 4.0,
                            rng.uniform(-2, 2) * TWO_PI)
    gamma = smooth_field(rng, m, n, lo, hi, corr_px=corr_px)
    if mask_frac > 0:
        mask = (~_blob_mask(rng, m, n, mask_frac, blob_px=max(4.0, min(m, n) / 6.0))).astype(np.uint8)
    else:
        mask = np.ones((m, n), np.uint8)
    return _finish(rng, truth, gamma, nlooks, mask, want_complex, {"name": f"random {m}x{n}", "seed": seed})


def batch_item(index: int, base_seed: int = 4000, min_px: int = 256 * 256, max_px: int = 2048 * 2048,
               scale: float = 1.0) -> Interferogram:
    """One item of the uneven batched workload: size uniform in [min_px, max_px] (times `scale`),
    aspect 1:1 to 1:4 in a random orientation, built like the 256x256 case with random lobes,
    decorrelated patches and masks, L in {4, 9, 16}."""
    rng = np.random.Generator(np.random.PCG64(base_seed + index))
    npx = rng.uniform(min_px, max_px) * scale
    a = rng.uniform(1.0, 4.0)
    rows = max(8, int(round(np.sqrt(npx / a))))
    cols = max(8, int(round(npx / rows)))
    if rng.uniform() < 0.5:
        rows, cols = cols, rows
    nlooks = float(rng.choice([4.0, 9.0, 16.0]))
    j = np.arange(cols)[None, :]
    truth = np.broadcast_to(TWO_PI * rng.uniform(0.5, 3.0) * j / cols, (rows, cols)).astype(np.float64).copy()
    for _ in range(int(rng.integers(1, 4))):
        truth += _gaussian_bump(rows, cols, rng.uniform(0, rows), rng.uniform(0, cols),
                                rng.uniform(0.05, 0.2) * max(rows, cols), rng.uniform(-6, 6) * TWO_PI)
    gamma = smooth_field(rng, rows, cols, 0.2, 0.95)
    if rng.uniform() < 0.5:
        ii = np.arange(rows)[:, None]
        jj = np.arange(cols)[None, :]
        r = rng.uniform(0.03, 0.1) * min(rows, cols)
        gamma[(ii - rng.uniform(0, rows)) ** 2 + (jj - rng.uniform(0, cols)) ** 2 <= r * r] = 0.05
    if rng.uniform() < 0.5:
        mask = (~_blob_mask(rng, rows, cols, rng.uniform(0.02, 0.1), blob_px=max(8.0, min(rows, cols) / 8.0))).astype(np.uint8)
    else:
        mask = np.ones((rows, cols), np.uint8)
    return _finish(rng, truth, gamma, nlooks, mask, False, {"name": f"batch item {index}", "seed": base_seed + index})


def cached(name: str, **kwargs) -> Interferogram:
    """generator `name` (config1/config2/config3/...) with kwargs, memoised as an
    .npz under $WW_SYNTH_CACHE when that variable names a directory (the big
    scenes take minutes of single-threaded numpy to generate)."""
    import hashlib
    import os

    fn = globals()[name]
    d = os.environ.get("WW_SYNTH_CACHE")
    if not d:
        return fn(**kwargs)
    key = hashlib.sha1(repr((name, sorted(kwargs.items()))).encode()).hexdigest()[:16]
    path = os.path.join(d, f"{name}_{key}.npz")
    if os.path.exists(path):
        z = np.load(path, allow_pickle=False)
        ifg = z["ifg"] if z["ifg"].size else None
        return Interferogram(phase=z["phase"], coh=z["coh"], mask=z["mask"], nlooks=float(z["nlooks"]),
                             truth=z["truth"], ifg=ifg, meta={"name": str(z["name"])})
    x = fn(**kwargs)
    os.makedirs(d, exist_ok=True)
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, phase=x.phase, coh=x.coh, mask=x.mask, nlooks=np.float64(x.nlooks), truth=x.truth,
             ifg=x.ifg if x.ifg is not None else np.zeros(0, np.complex64), name=str(x.meta.get("name", name)))
    os.replace(tmp, path)
    return x
