"""B300-native hot path of the Whirlwind MCF phase unwrapper (arxiv 2609.36267).

Thin ctypes binding over libww.so (include/ww.h).  Every step of the path runs
in the library's CUDA kernels; this module only passes device pointers, sizes
and the current torch stream.  There is no CPU fallback: if libww.so is missing
or fails to load, every call raises.

    import torch, paper_2609_36267_b300 as ww
    ws = ww.Workspace(m, n)
    unw, K, cost = ww.unwrap(ifg, coh, nlooks, mask, ws=ws)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libww.so")

WW_OK = 0
WW_ERR_INVALID_ARG = -1
WW_ERR_CUDA = -2
WW_ERR_OOM = -3
WW_ERR_INFEASIBLE = -4
WW_ERR_TIMEOUT = -5
WW_ERR_OVERFLOW = -6
WW_ERR_NOT_IMPLEMENTED = -7
WW_ERR_INTERNAL = -8

N_GAMMA, N_ALPHA = 128, 256


class WWError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


class Params(ctypes.Structure):
    _fields_ = [("box_half_width", ctypes.c_int32), ("steep_rad", ctypes.c_float),
                ("steep_cap_ppm", ctypes.c_int32), ("max_passes", ctypes.c_int32),
                ("wait_polls", ctypes.c_int32), ("graph_loop", ctypes.c_int32),
                ("search_ctas_per_sm", ctypes.c_int32), ("band_min", ctypes.c_int32),
                ("band_mult", ctypes.c_int32), ("band_growth", ctypes.c_int32),
                ("band_start_ppm", ctypes.c_int32), ("full_passes", ctypes.c_int32),
                ("ground_sink_below", ctypes.c_int32), ("zero_stop_below", ctypes.c_int32),
                ("zero_band_hops", ctypes.c_int32), ("zero_band_hops_min", ctypes.c_int32),
                ("slope_estimator", ctypes.c_int32), ("cost_lookup", ctypes.c_int32)]


class SolveStats(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int64), ("augmentations", ctypes.c_int64),
                ("search_iterations", ctypes.c_int64), ("tile_visits", ctypes.c_int64),
                ("residues", ctypes.c_int64), ("ground_net", ctypes.c_int64),
                ("ms_search", ctypes.c_double), ("ms_other", ctypes.c_double),
                ("ms_search_gpu", ctypes.c_double), ("local_rounds", ctypes.c_int64),
                ("visit_cycles", ctypes.c_int64), ("load_cycles", ctypes.c_int64),
                ("relax_cycles", ctypes.c_int64), ("settled_visits", ctypes.c_int64),
                ("narrow_visits", ctypes.c_int64), ("narrow_redone", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchItem(ctypes.Structure):
    _fields_ = [("ifg", ctypes.c_void_p), ("is_complex", ctypes.c_int32), ("coh", ctypes.c_void_p),
                ("mask", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("nlooks", ctypes.c_double),
                ("unwrapped", ctypes.c_void_p), ("cycles", ctypes.c_void_p), ("total_cost", ctypes.c_int64),
                ("status", ctypes.c_int32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_request_pixels", ctypes.c_int64),
                ("max_active", ctypes.c_int32), ("reserved", ctypes.c_int32 * 7)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("passes", ctypes.c_int64), ("peak_active", ctypes.c_int64),
                ("peak_resident_bytes", ctypes.c_int64), ("busy_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Load libww.so (raises if it is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libww.so not built at {LIB_PATH}; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        i64, i32, d = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        L.ww_status_string.argtypes = [i32]
        L.ww_status_string.restype = ctypes.c_char_p
        L.ww_params_default.argtypes = [ctypes.POINTER(Params)]
        L.ww_build_lut.argtypes = [d, ctypes.POINTER(P)]
        L.ww_lut_from_table.argtypes = [d, P, ctypes.POINTER(P)]
        L.ww_lut_table.argtypes = [P, P, P]
        L.ww_lut_free.argtypes = [P]
        L.ww_workspace_create.argtypes = [i64, i64, ctypes.POINTER(P)]
        L.ww_workspace_free.argtypes = [P]
        L.ww_workspace_bytes.argtypes = [i64, i64]
        L.ww_workspace_bytes.restype = i64
        L.ww_residues.argtypes = [P, i32, P, P, i64, i64, P, P, P]
        L.ww_costs.argtypes = [P, i32, P, P, i64, i64, P, ctypes.POINTER(Params), P, P, P]
        L.ww_costs_noalloc.argtypes = [P, i32, P, P, i64, i64, P, ctypes.POINTER(Params), P, P]
        L.ww_solve_mcf.argtypes = [P, P, P, i64, i64, ctypes.POINTER(Params), P, P, P, P, P, P]
        L.ww_solve_mcf_resume.argtypes = [P, P, P, i64, i64, ctypes.POINTER(Params), P, P, P, P, P, P]
        L.ww_get_solve_stats.argtypes = [P, ctypes.POINTER(SolveStats)]
        L.ww_workspace_last_unwrap.argtypes = [P] + [ctypes.POINTER(P)] * 5
        L.ww_integrate.argtypes = [P, i32, P, P, P, i64, i64, P, P, P]
        L.ww_unwrap.argtypes = [P, i32, P, d, P, i64, i64, ctypes.POINTER(Params), P, P, P,
                                ctypes.POINTER(i64), P]
        L.ww_certificate.argtypes = [P, P, P, P, P, i64, i64, P, P]
        L.ww_components.argtypes = [P, P, P, i64, i64, i32, P, P]
        L.ww_lut_from_tables.argtypes = [d, P, P, ctypes.POINTER(P)]
        L.ww_multilook.argtypes = [P, P, i64, i64, i32, i32, P, P, P]
        L.ww_goldstein.argtypes = [P, i64, i64, ctypes.c_float, i32, i32, P, P]
        L.ww_transfer_cycles.argtypes = [P, P, i32, P, P, i64, i64, P, P, P]
        L.ww_lut_ratio_table.argtypes = [P, P]
        L.ww_bridge.argtypes = [P, P, i64, i64, i32, P, P, ctypes.POINTER(i32), P]
        L.ww_batch_create.argtypes = [i64, i64, i64, ctypes.POINTER(P)]
        L.ww_batch_free.argtypes = [P]
        L.ww_batch_bytes.argtypes = [i64, i64, i64]
        L.ww_batch_bytes.restype = i64
        L.ww_unwrap_batch.argtypes = [ctypes.POINTER(BatchItem), i64, ctypes.POINTER(Params), P, P]
        L.ww_batch_stats.argtypes = [P, ctypes.POINTER(SolveStats)]
        L.ww_autotune_batch.argtypes = [ctypes.POINTER(BatchItem), i64, ctypes.POINTER(Params), P, i32,
                                        ctypes.POINTER(Params), ctypes.POINTER(TuneReport), P]
        L.ww_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(Params), ctypes.POINTER(P)]
        L.ww_server_submit.argtypes = [P, ctypes.POINTER(BatchItem), ctypes.POINTER(i64)]
        L.ww_server_poll.argtypes = [P, i64, ctypes.POINTER(i32), ctypes.POINTER(BatchItem),
                                     ctypes.POINTER(ctypes.c_double)]
        L.ww_server_wait.argtypes = [P, i64, ctypes.c_double, ctypes.POINTER(BatchItem),
                                     ctypes.POINTER(ctypes.c_double)]
        L.ww_server_release.argtypes = [P, i64]
        L.ww_server_get_stats.argtypes = [P, ctypes.POINTER(ServerStats)]
        L.ww_server_destroy.argtypes = [P]
        for f in ("ww_build_lut", "ww_lut_from_table", "ww_lut_table", "ww_workspace_create", "ww_residues",
                  "ww_costs", "ww_costs_noalloc", "ww_solve_mcf", "ww_solve_mcf_resume", "ww_get_solve_stats",
                  "ww_workspace_last_unwrap", "ww_integrate", "ww_unwrap",
                  "ww_certificate", "ww_components", "ww_bridge", "ww_lut_from_tables", "ww_lut_ratio_table", "ww_multilook", "ww_goldstein",
                  "ww_transfer_cycles", "ww_batch_create", "ww_unwrap_batch", "ww_batch_stats", "ww_autotune_batch",
                  "ww_server_create",
                  "ww_server_submit", "ww_server_poll", "ww_server_wait", "ww_server_release", "ww_server_get_stats"):
            getattr(L, f).restype = i32
        _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().ww_status_string(int(status)).decode()


def _check(status: int, what: str):
    if status != WW_OK:
        raise WWError(status, what)


def default_params(**kw) -> Params:
    p = Params()
    lib().ww_params_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Lut:
    """A cost table for one number of looks (library-owned, cached per nlooks)."""

    def __init__(self, handle, nlooks):
        self._h = ctypes.c_void_p(handle)
        self.nlooks = nlooks

    @classmethod
    def build(cls, nlooks: float) -> "Lut":
        h = ctypes.c_void_p()
        _check(lib().ww_build_lut(float(nlooks), ctypes.byref(h)), "ww_build_lut")
        return cls(h.value, nlooks)

    @classmethod
    def from_table(cls, nlooks: float, table: np.ndarray) -> "Lut":
        t = np.ascontiguousarray(table, np.int16)
        assert t.size == N_GAMMA * N_ALPHA
        h = ctypes.c_void_p()
        _check(lib().ww_lut_from_table(float(nlooks), t.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)),
               "ww_lut_from_table")
        return cls(h.value, nlooks)

    @classmethod
    def from_tables(cls, nlooks: float, table: np.ndarray, ratio100: np.ndarray) -> "Lut":
        """An int16 table plus the fp32 100 ln(P0/P+) table of the interpolated lookup."""
        t = np.ascontiguousarray(table, np.int16)
        r = np.ascontiguousarray(ratio100, np.float32)
        assert t.size == N_GAMMA * N_ALPHA and r.size == N_GAMMA * N_ALPHA
        h = ctypes.c_void_p()
        _check(lib().ww_lut_from_tables(float(nlooks), t.ctypes.data_as(ctypes.c_void_p),
                                        r.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)), "ww_lut_from_tables")
        return cls(h.value, nlooks)

    def ratio100(self) -> np.ndarray:
        r = np.empty((N_GAMMA, N_ALPHA), np.float32)
        _check(lib().ww_lut_ratio_table(self._h, r.ctypes.data_as(ctypes.c_void_p)), "ww_lut_ratio_table")
        return r

    def table(self) -> np.ndarray:
        t = np.empty((N_GAMMA, N_ALPHA), np.int16)
        _check(lib().ww_lut_table(self._h, t.ctypes.data_as(ctypes.c_void_p), None), "ww_lut_table")
        return t

    def cost100(self) -> np.ndarray:
        c = np.empty((N_GAMMA, N_ALPHA), np.float64)
        _check(lib().ww_lut_table(self._h, None, c.ctypes.data_as(ctypes.c_void_p)), "ww_lut_table")
        return c

    @property
    def handle(self):
        return self._h

    def __del__(self):
        try:
            if self._h and _lib is not None:
                _lib.ww_lut_free(self._h)
                self._h = None
        except Exception:
            pass


class Workspace:
    """Device scratch for one request of up to rows x cols (not shared by overlapping calls)."""

    def __init__(self, rows: int, cols: int):
        h = ctypes.c_void_p()
        _check(lib().ww_workspace_create(int(rows), int(cols), ctypes.byref(h)), "ww_workspace_create")
        self._h = h
        self.rows, self.cols = rows, cols

    @staticmethod
    def bytes(rows, cols) -> int:
        return int(lib().ww_workspace_bytes(int(rows), int(cols)))

    @property
    def handle(self):
        return self._h

    def stats(self) -> dict:
        s = SolveStats()
        _check(lib().ww_get_solve_stats(self._h, ctypes.byref(s)), "ww_get_solve_stats")
        return s.as_dict()

    def last_unwrap_pointers(self):
        """Device addresses (residues, ground, costs, flows, potentials) of the last ww_unwrap."""
        ptrs = [ctypes.c_void_p() for _ in range(5)]
        _check(lib().ww_workspace_last_unwrap(self._h, *[ctypes.byref(p) for p in ptrs]), "ww_workspace_last_unwrap")
        return tuple(p.value for p in ptrs)

    def certify_last_unwrap(self, m: int, n: int):
        """GPU certificate counts of the last ww_unwrap on this workspace (an m x n
        image): (capacity violations, conservation violations, negative reduced
        costs, total cost), on exactly the arrays that call solved with."""
        torch = _torch()
        ptrs = [ctypes.c_void_p() for _ in range(5)]
        _check(lib().ww_workspace_last_unwrap(self._h, *[ctypes.byref(p) for p in ptrs]), "ww_workspace_last_unwrap")
        counts = torch.zeros(4, dtype=torch.int64, device="cuda")
        res, g, costs, flows, pot = ptrs
        _check(lib().ww_certificate(res, g, costs, flows, pot, int(m), int(n), _ptr(counts), _stream()),
               "ww_certificate")
        return tuple(int(x) for x in counts.cpu())

    def close(self):
        if self._h:
            lib().ww_workspace_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------- tensor marshalling ----------------

def _torch():
    import torch

    return torch


def _stream():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return ctypes.c_void_p(t.data_ptr())


def _ifg(ifg):
    torch = _torch()
    if ifg.dtype == torch.complex64:
        return _ptr(ifg), 1
    assert ifg.dtype == torch.float32, "phase must be float32 or complex64"
    return _ptr(ifg), 0


def residues(ifg, coh=None, mask=None):
    """-> (residues int8 [(m-1),(n-1)], ground int32 [1]) on the device."""
    torch = _torch()
    m, n = ifg.shape
    r = torch.empty((m - 1, n - 1), dtype=torch.int8, device=ifg.device)
    g = torch.empty(1, dtype=torch.int32, device=ifg.device)
    p, c = _ifg(ifg)
    _check(lib().ww_residues(p, c, _ptr(coh), _ptr(mask), m, n, _ptr(r), _ptr(g), _stream()), "ww_residues")
    return r, g


def costs(ifg, coh, lut: Lut, ws: Workspace, mask=None, params: Params | None = None):
    """-> costs int16 [4, m, n] on the device."""
    torch = _torch()
    m, n = ifg.shape
    out = torch.empty((4, m, n), dtype=torch.int16, device=ifg.device)
    p, c = _ifg(ifg)
    prm = params or default_params()
    _check(lib().ww_costs(p, c, _ptr(coh), _ptr(mask), m, n, lut.handle, ctypes.byref(prm), ws.handle,
                          _ptr(out), _stream()), "ww_costs")
    return out


def costs_noalloc(ifg, coh, lut: Lut, mask=None, params: Params | None = None, out=None):
    """ww_costs without a workspace or any device allocation by the library
    (scratch in a static device array; calls that overlap on the GPU race)."""
    torch = _torch()
    m, n = ifg.shape
    if out is None:
        out = torch.empty((4, m, n), dtype=torch.int16, device=ifg.device)
    p, c = _ifg(ifg)
    prm = params or default_params()
    _check(lib().ww_costs_noalloc(p, c, _ptr(coh), _ptr(mask), m, n, lut.handle, ctypes.byref(prm), _ptr(out),
                                  _stream()), "ww_costs_noalloc")
    return out


def solve_mcf(res, ground, cost_planes, ws: Workspace, params: Params | None = None, check=True):
    """-> (flows int8 [2,m,n], potentials int64 [(m-1)(n-1)+1], total_cost int64 [1], status int)."""
    torch = _torch()
    _, m, n = cost_planes.shape
    dev = cost_planes.device
    flows = torch.empty((2, m, n), dtype=torch.int8, device=dev)
    pot = torch.empty((m - 1) * (n - 1) + 1, dtype=torch.int64, device=dev)
    tc = torch.empty(1, dtype=torch.int64, device=dev)
    st = torch.empty(1, dtype=torch.int32, device=dev)
    prm = params or default_params()
    status = lib().ww_solve_mcf(_ptr(res), _ptr(ground), _ptr(cost_planes), m, n, ctypes.byref(prm), ws.handle,
                                _ptr(flows), _ptr(pot), _ptr(tc), _ptr(st), _stream())
    if check:
        _check(status, "ww_solve_mcf")
    return flows, pot, tc, status


def solve_mcf_resume(res, ground, cost_planes, ws: Workspace, flows, pot, params: Params | None = None,
                     check=True):
    """Continue a solve from (flows, potentials), updated in place -> (total_cost int64 [1], status int)."""
    torch = _torch()
    _, m, n = cost_planes.shape
    tc = torch.empty(1, dtype=torch.int64, device=cost_planes.device)
    st = torch.empty(1, dtype=torch.int32, device=cost_planes.device)
    prm = params or default_params()
    status = lib().ww_solve_mcf_resume(_ptr(res), _ptr(ground), _ptr(cost_planes), m, n, ctypes.byref(prm),
                                       ws.handle, _ptr(flows), _ptr(pot), _ptr(tc), _ptr(st), _stream())
    if check:
        _check(status, "ww_solve_mcf_resume")
    return tc, status


def integrate(ifg, flows, coh=None, mask=None):
    """-> (unwrapped float32 [m,n], cycles int32 [m,n])."""
    torch = _torch()
    m, n = ifg.shape
    unw = torch.empty((m, n), dtype=torch.float32, device=ifg.device)
    cyc = torch.empty((m, n), dtype=torch.int32, device=ifg.device)
    p, c = _ifg(ifg)
    _check(lib().ww_integrate(p, c, _ptr(coh), _ptr(mask), _ptr(flows), m, n, _ptr(unw), _ptr(cyc), _stream()),
           "ww_integrate")
    return unw, cyc


def components(cost_planes, flows, unwrapped, threshold: int = 0, out=None):
    """Connected-component labels (ww_components) -> int32 [m, n] on the device:
    1 + the smallest row-major index of each pixel's component, 0 where invalid."""
    torch = _torch()
    _, m, n = cost_planes.shape
    labels = out if out is not None else torch.empty((m, n), dtype=torch.int32, device=cost_planes.device)
    _check(lib().ww_components(_ptr(cost_planes), _ptr(flows), _ptr(unwrapped), m, n, int(threshold), _ptr(labels),
                               _stream()), "ww_components")
    return labels


def multilook(slc1, slc2, looks_y: int, looks_x: int):
    """Multilooked interferogram and Eq. (3) coherence -> (ifg complex64, coh float32)."""
    torch = _torch()
    M, N = slc1.shape
    m, n = M // looks_y, N // looks_x
    ifg = torch.empty((m, n), dtype=torch.complex64, device=slc1.device)
    coh = torch.empty((m, n), dtype=torch.float32, device=slc1.device)
    _check(lib().ww_multilook(_ptr(slc1), _ptr(slc2), M, N, int(looks_y), int(looks_x), _ptr(ifg), _ptr(coh),
                              _stream()), "ww_multilook")
    return ifg, coh


def goldstein(ifg, alpha: float = 0.5, step: int = 16, smooth: int = 3):
    """Adaptive power-spectrum filter of a complex64 interferogram -> complex64."""
    torch = _torch()
    m, n = ifg.shape
    out = torch.empty_like(ifg)
    _check(lib().ww_goldstein(_ptr(ifg), m, n, float(alpha), int(step), int(smooth), _ptr(out), _stream()),
           "ww_goldstein")
    return out


def transfer_cycles(unwrapped_filtered, ifg, coh=None, mask=None):
    """Cycles of a filtered unwrap moved to the original phase -> (unwrapped, cycles)."""
    torch = _torch()
    m, n = ifg.shape
    unw = torch.empty((m, n), dtype=torch.float32, device=ifg.device)
    cyc = torch.empty((m, n), dtype=torch.int32, device=ifg.device)
    p, c = _ifg(ifg)
    _check(lib().ww_transfer_cycles(_ptr(unwrapped_filtered), p, c, _ptr(coh), _ptr(mask), m, n, _ptr(unw),
                                    _ptr(cyc), _stream()), "ww_transfer_cycles")
    return unw, cyc


def bridge(unwrapped, cycles=None, window: int = 65):
    """Bridging of mask-separated regions (ww_bridge), in place on `unwrapped`
    (and `cycles` if given) -> (region int32 [m,n], shift int32 [m,n], regions)."""
    torch = _torch()
    m, n = unwrapped.shape
    region = torch.empty((m, n), dtype=torch.int32, device=unwrapped.device)
    shift = torch.empty((m, n), dtype=torch.int32, device=unwrapped.device)
    nr = ctypes.c_int32()
    _check(lib().ww_bridge(_ptr(unwrapped), _ptr(cycles), m, n, int(window), _ptr(region), _ptr(shift),
                           ctypes.byref(nr), _stream()), "ww_bridge")
    return region, shift, nr.value


def unwrap(ifg, coh, nlooks: float, mask=None, ws: Workspace | None = None, params: Params | None = None,
           out=None):
    """Whole path.  -> (unwrapped float32 [m,n], cycles int32 [m,n], total_cost int)."""
    torch = _torch()
    m, n = ifg.shape
    if ws is None:
        ws = Workspace(m, n)
    if out is None:
        unw = torch.empty((m, n), dtype=torch.float32, device=ifg.device)
        cyc = torch.empty((m, n), dtype=torch.int32, device=ifg.device)
    else:
        unw, cyc = out
    p, c = _ifg(ifg)
    tc = ctypes.c_int64(0)
    prm = params or default_params()
    _check(lib().ww_unwrap(p, c, _ptr(coh), float(nlooks), _ptr(mask), m, n, ctypes.byref(prm), ws.handle,
                           _ptr(unw), _ptr(cyc), ctypes.byref(tc), _stream()), "ww_unwrap")
    return unw, cyc, tc.value


def certificate(res, ground, cost_planes, flows, potentials):
    """GPU certificate counts: (capacity violations, conservation violations,
    negative reduced costs, total cost)."""
    torch = _torch()
    _, m, n = cost_planes.shape
    counts = torch.zeros(4, dtype=torch.int64, device=cost_planes.device)
    _check(lib().ww_certificate(_ptr(res), _ptr(ground), _ptr(cost_planes), _ptr(flows), _ptr(potentials), m, n,
                                _ptr(counts), _stream()), "ww_certificate")
    return tuple(int(x) for x in counts.cpu())


class Batch:
    """Device scratch for batched unwraps (up to max_items items, max_pixels in total)."""

    def __init__(self, max_items: int, max_pixels: int, max_item_pixels: int | None = None):
        h = ctypes.c_void_p()
        mip = max_item_pixels or max_pixels
        _check(lib().ww_batch_create(int(max_items), int(max_pixels), int(mip), ctypes.byref(h)), "ww_batch_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def stats(self) -> dict:
        st = SolveStats()
        _check(lib().ww_batch_stats(self._h, ctypes.byref(st)), "ww_batch_stats")
        return st.as_dict()

    def close(self):
        if self._h:
            lib().ww_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _batch_items(requests):
    torch = _torch()
    outs = []
    arr = (BatchItem * len(requests))()
    total = 0
    biggest = 0
    for k, (ifg, coh, nlooks, mask) in enumerate(requests):
        m, n = ifg.shape
        unw = torch.empty((m, n), dtype=torch.float32, device=ifg.device)
        cyc = torch.empty((m, n), dtype=torch.int32, device=ifg.device)
        p, c = _ifg(ifg)
        arr[k] = BatchItem(p.value, c, _ptr(coh).value, _ptr(mask).value if mask is not None else None, m, n,
                           float(nlooks), unw.data_ptr(), cyc.data_ptr(), 0, 0)
        outs.append((unw, cyc))
        total += m * n
        biggest = max(biggest, m * n)
    return arr, outs, total, biggest


class TuneReport(ctypes.Structure):
    _fields_ = [("trials", ctypes.c_int32), ("default_ms", ctypes.c_float), ("best_ms", ctypes.c_float),
                ("reserved", ctypes.c_int32 * 5)]


def autotune_batch(requests, batch: Batch | None = None, start: Params | None = None, repeats: int = 2):
    """Pick the search schedule for a batched workload from a sample of it
    (requests as for unwrap_batch).  -> (Params, {"trials", "default_ms", "best_ms"})."""
    arr, outs, total, biggest = _batch_items(requests)
    if batch is None:
        batch = Batch(len(requests), total, biggest)
    best = Params()
    rep = TuneReport()
    _check(lib().ww_autotune_batch(arr, len(requests), ctypes.byref(start or default_params()), batch.handle,
                                   int(repeats), ctypes.byref(best), ctypes.byref(rep), _stream()),
           "ww_autotune_batch")
    del outs
    return best, {"trials": rep.trials, "default_ms": rep.default_ms, "best_ms": rep.best_ms}


def unwrap_batch(requests, batch: Batch | None = None, params: Params | None = None, check=True):
    """requests: list of (ifg, coh, nlooks, mask) device tensors.  Returns a list
    of (unwrapped, cycles, total_cost, status) in the same order."""
    arr, outs, total, biggest = _batch_items(requests)
    if batch is None:
        batch = Batch(len(requests), total, biggest)
    prm = params or default_params()
    st = lib().ww_unwrap_batch(arr, len(requests), ctypes.byref(prm), batch.handle, _stream())
    if check:
        _check(st, "ww_unwrap_batch")
    return [(u, k, arr[i].total_cost, arr[i].status) for i, (u, k) in enumerate(outs)]


class Server:
    """Continuous-batching unwrap server (library worker thread + CUDA stream).

    submit() synchronises the caller's current stream so the request's inputs are
    ready, then queues it; wait() returns (unwrapped, cycles, total_cost, status,
    latency_ms).  Tensors are kept alive until the request completes."""

    def __init__(self, hbm_budget_bytes: int, max_request_pixels: int, max_active: int = 64,
                 params: Params | None = None):
        cfg = ServerConfig(int(hbm_budget_bytes), int(max_request_pixels), int(max_active))
        h = ctypes.c_void_p()
        prm = params or default_params()
        _check(lib().ww_server_create(ctypes.byref(cfg), ctypes.byref(prm), ctypes.byref(h)), "ww_server_create")
        self._h = h
        self._keep = {}

    def submit(self, ifg, coh, nlooks, mask=None, out=None) -> int:
        torch = _torch()
        m, n = ifg.shape
        if out is None:
            unw = torch.empty((m, n), dtype=torch.float32, device=ifg.device)
            cyc = torch.empty((m, n), dtype=torch.int32, device=ifg.device)
        else:
            unw, cyc = out
        torch.cuda.current_stream().synchronize()
        p, c = _ifg(ifg)
        item = BatchItem(p.value, c, _ptr(coh).value, _ptr(mask).value if mask is not None else None, m, n,
                         float(nlooks), unw.data_ptr(), cyc.data_ptr(), 0, 0)
        t = ctypes.c_int64()
        _check(lib().ww_server_submit(self._h, ctypes.byref(item), ctypes.byref(t)), "ww_server_submit")
        self._keep[t.value] = (ifg, coh, mask, unw, cyc)
        return t.value

    def poll(self, ticket: int) -> bool:
        d = ctypes.c_int32()
        _check(lib().ww_server_poll(self._h, int(ticket), ctypes.byref(d), None, None), "ww_server_poll")
        return bool(d.value)

    def wait(self, ticket: int, timeout_ms: float = 600000.0):
        res = BatchItem()
        lat = ctypes.c_double()
        _check(lib().ww_server_wait(self._h, int(ticket), float(timeout_ms), ctypes.byref(res), ctypes.byref(lat)),
               "ww_server_wait")
        _, _, _, unw, cyc = self._keep.pop(ticket)
        lib().ww_server_release(self._h, int(ticket))
        return unw, cyc, res.total_cost, res.status, lat.value

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().ww_server_get_stats(self._h, ctypes.byref(st)), "ww_server_get_stats")
        return st.as_dict()

    def close(self):
        if self._h:
            lib().ww_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
