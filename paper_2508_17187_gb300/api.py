"""Python binding of the awgrid C ABI with the same names (cf_set_create, plan_create,
grid_visibilities, degrid_visibilities, grid_normalize).  It checks and marshals torch tensors
and passes their device pointers; all arithmetic happens in libawgrid.so."""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import AWG_CF_BF16, AWG_CF_FP32, AWG_DEGRID_SUBTRACT, AWG_GRID_FP64, AWG_GRID_KAHAN, CfParams, check

__all__ = ["CFSet", "Plan", "CleanWorkspace", "cf_set_create", "cf_set_create_from_table", "plan_create",
           "clean_hogbom", "gcal_solve", "grid_visibilities",
           "degrid_visibilities", "grid_normalize", "AWG_CF_FP32", "AWG_CF_BF16", "AWG_GRID_KAHAN", "AWG_GRID_FP64",
           "AWG_DEGRID_SUBTRACT"]


def _stream_ptr(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t: Optional[torch.Tensor]) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr() if t is not None else None)


def _need(t: torch.Tensor, name: str, dtype, shape=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (the library has no CPU path)")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


class CFSet:
    """Owns an awg_cf_set (device-resident CF tables)."""

    def __init__(self, handle: ctypes.c_void_p, grid_n: int, oversampling: int, n_pa_bins: int, n_subbands: int):
        self._h = handle
        self.grid_n = grid_n
        self.oversampling = oversampling
        self.n_pa_bins = n_pa_bins
        self.n_subbands = n_subbands
        n_cf = ctypes.c_int32()
        n_val = ctypes.c_int64()
        sep = ctypes.c_int32()
        check(_lib.load().cf_set_info(self._h, ctypes.byref(n_cf), ctypes.byref(n_val), ctypes.byref(sep)),
              "cf_set_info")
        self.n_cf = int(n_cf.value)
        self.n_values = int(n_val.value)
        self.rank = int(sep.value)            # outer-product terms per CF; 0 for full tables
        self.separable = self.rank > 0
        fused = ctypes.c_int32()
        check(_lib.load().cf_set_fused_terms(self._h, ctypes.byref(fused)), "cf_set_fused_terms")
        self.fused_terms = int(fused.value)   # terms combined per tap by the kernels; 0 if not fused

    def params(self) -> dict:
        """The parameters the set was made with (cf_set_get_params), A-term bins as arrays."""
        p = CfParams()
        pa = np.zeros(max(self.n_pa_bins, 1), dtype=np.float64)
        sb = np.zeros(max(self.n_subbands, 1), dtype=np.float64)
        check(_lib.load().cf_set_get_params(self.handle, ctypes.byref(p), pa.ctypes.data_as(ctypes.c_void_p),
                                            sb.ctypes.data_as(ctypes.c_void_p)), "cf_set_get_params")
        out = {name: getattr(p, name) for name, _ in CfParams._fields_
               if name not in ("pa_bin_centers_rad", "subband_freq_hz")}
        if p.use_a:
            out["pa_bin_centers_rad"], out["subband_freq_hz"] = pa[:p.n_pa_bins], sb[:p.n_subbands]
        return out

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("CF set already destroyed")
        return self._h

    def autotune(self, uvw_m: torch.Tensor, freq_hz: torch.Tensor, pa_bin: Optional[torch.Tensor] = None,
                 chan_subband: Optional[torch.Tensor] = None, n_pol: int = 4, stream=None):
        """Pick the faster compiled kernel configuration per support by timing both on a plan of
        this geometry (see cf_set_autotune in awgrid.h); plans made earlier become invalid.
        Returns ({support: choice}, {support: (ms of configurations 0, 1, 2 and 3)})."""
        _need(uvw_m, "uvw_m", torch.float64)
        _need(freq_hz, "freq_hz", torch.float64)
        if pa_bin is not None:
            _need(pa_bin, "pa_bin", torch.int32, (uvw_m.shape[0],))
        if chan_subband is not None:
            _need(chan_subband, "chan_subband", torch.int32, (freq_hz.shape[0],))
        choice = np.zeros(65, dtype=np.int32)
        ms = np.zeros((4, 65), dtype=np.float32)
        check(_lib.load().cf_set_autotune(self.handle, _ptr(uvw_m), uvw_m.shape[0], _ptr(freq_hz), freq_hz.shape[0],
                                          _ptr(pa_bin), _ptr(chan_subband), int(n_pol), _stream_ptr(stream),
                                          choice.ctypes.data_as(ctypes.c_void_p), ms.ctypes.data_as(ctypes.c_void_p)),
              "cf_set_autotune")
        picked = {S: int(choice[S]) for S in range(65) if choice[S] >= 0}
        return picked, {S: tuple(float(ms[c, S]) for c in range(4)) for S in picked}

    def mueller(self):
        """[(p, q), ...] Mueller elements of a full-polarisation set (empty otherwise)."""
        n = ctypes.c_int32()
        ep = np.zeros(16, dtype=np.int32)
        eq = np.zeros(16, dtype=np.int32)
        check(_lib.load().cf_set_mueller(self.handle, ctypes.byref(n), ep.ctypes.data_as(ctypes.c_void_p),
                                         eq.ctypes.data_as(ctypes.c_void_p)), "cf_set_mueller")
        return [(int(ep[i]), int(eq[i])) for i in range(n.value)]

    def choose(self, support: int, config: int):
        """Select kernel configuration 0, 1, 2 or 3 for one support by hand (see cf_set_choose)."""
        check(_lib.load().cf_set_choose(self.handle, int(support), int(config)), "cf_set_choose")

    def supports(self) -> np.ndarray:
        out = np.zeros(self.n_cf, dtype=np.int32)
        check(_lib.load().cf_set_get_supports(self.handle, out.ctypes.data_as(ctypes.c_void_p)), "cf_set_get_supports")
        return out

    def copy_table(self, cf_index: int) -> np.ndarray:
        S = int(self.supports()[cf_index])
        OS = self.oversampling
        out = np.zeros((OS + 1, OS + 1, S, S, 2), dtype=np.float32)
        check(_lib.load().cf_set_copy_table(self.handle, int(cf_index), out.ctypes.data_as(ctypes.c_void_p)),
              "cf_set_copy_table")
        return out[..., 0] + 1j * out[..., 1]

    def copy_factors(self, cf_index: int):
        """Stored factors of a separable CF (cf_set_copy_factors): (fx, fy, scale) with fx, fy
        complex64 [rank, OS+1, S] and the element scalar; CF = scale * sum_k fy[k] (x) fx[k]."""
        S = int(self.supports()[cf_index])
        OS = self.oversampling
        fx = np.zeros((self.rank, OS + 1, S, 2), dtype=np.float32)
        fy = np.zeros_like(fx)
        sc = np.zeros(2, dtype=np.float32)
        for k in range(self.rank):
            check(_lib.load().cf_set_copy_factors(self.handle, int(cf_index), k, fx[k].ctypes.data_as(ctypes.c_void_p),
                                                  fy[k].ctypes.data_as(ctypes.c_void_p),
                                                  sc.ctypes.data_as(ctypes.c_void_p)), "cf_set_copy_factors")
        return fx[..., 0] + 1j * fx[..., 1], fy[..., 0] + 1j * fy[..., 1], complex(sc[0], sc[1])

    def close(self):
        if self._h is not None:
            check(_lib.load().cf_set_destroy(self._h), "cf_set_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _params(grid_n, cell_rad, oversampling=20, ps_support=7, use_ps=True, use_w=False, n_wplanes=1,
            w_max_lambda=0.0, use_a=False, n_pa_bins=1, pa_bin_centers_rad=None, n_subbands=1,
            subband_freq_hz=None, max_support=7, dish_diameter_m=25.0, ellipticity=0.05, cf_dtype=AWG_CF_FP32,
            separable=True, use_pol=False, squint_rad=0.0, leakage=0.0, mueller_threshold=0.01):
    p = CfParams()
    p.grid_n = int(grid_n)
    p.cell_rad = float(cell_rad)
    p.oversampling = int(oversampling)
    p.ps_support = int(ps_support)
    p.use_ps = int(bool(use_ps))
    p.use_w = int(bool(use_w))
    p.n_wplanes = int(n_wplanes)
    p.w_max_lambda = float(w_max_lambda)
    p.use_a = int(bool(use_a))
    p.n_pa_bins = int(n_pa_bins)
    p.n_subbands = int(n_subbands)
    p.max_support = int(max_support)
    p.dish_diameter_m = float(dish_diameter_m)
    p.ellipticity = float(ellipticity)
    p.cf_dtype = int(cf_dtype)
    p.separable = int(bool(separable))
    p.use_pol = int(bool(use_pol))
    p.squint_rad = float(squint_rad)
    p.leakage_re = float(complex(leakage).real)
    p.leakage_im = float(complex(leakage).imag)
    p.mueller_threshold = float(mueller_threshold)
    keep = []
    if pa_bin_centers_rad is not None:
        a = np.ascontiguousarray(pa_bin_centers_rad, dtype=np.float64)
        keep.append(a)
        p.pa_bin_centers_rad = a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    if subband_freq_hz is not None:
        a = np.ascontiguousarray(subband_freq_hz, dtype=np.float64)
        keep.append(a)
        p.subband_freq_hz = a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return p, keep


def cf_set_create(stream=None, **params) -> CFSet:
    """Build the CF set of Tab. AWP-CFSETUP on the host in FP64 and upload it (see awgrid.h)."""
    p, keep = _params(**params)
    h = ctypes.c_void_p()
    check(_lib.load().cf_set_create(ctypes.byref(p), _stream_ptr(stream), ctypes.byref(h)), "cf_set_create")
    del keep
    return CFSet(h, p.grid_n, p.oversampling, p.n_pa_bins, p.n_subbands)


def cf_set_create_from_table(supports: Sequence[int], table: np.ndarray, stream=None, **params) -> CFSet:
    """CF set from caller tables: table complex, all CFs concatenated, each [OS+1][OS+1][S][S]."""
    p, keep = _params(**params)
    sup = np.ascontiguousarray(supports, dtype=np.int32)
    tab = np.ascontiguousarray(np.stack([np.real(table), np.imag(table)], -1).astype(np.float32).reshape(-1))
    h = ctypes.c_void_p()
    check(_lib.load().cf_set_create_from_table(ctypes.byref(p), sup.ctypes.data_as(ctypes.c_void_p),
                                               tab.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream),
                                               ctypes.byref(h)), "cf_set_create_from_table")
    del keep
    return CFSet(h, p.grid_n, p.oversampling, p.n_pa_bins, p.n_subbands)


def cf_set_save(cf: CFSet, path) -> None:
    """Write the CF set to a CF cache file (see cf_set_save in awgrid.h); blocking."""
    check(_lib.load().cf_set_save(cf.handle, str(path).encode()), "cf_set_save")


def cf_set_load(path, stream=None) -> CFSet:
    """Load a CF set from a CF cache file written by cf_set_save, without rebuilding it."""
    h = ctypes.c_void_p()
    check(_lib.load().cf_set_load(str(path).encode(), _stream_ptr(stream), ctypes.byref(h)), "cf_set_load")
    p = CfParams()
    check(_lib.load().cf_set_get_params(h, ctypes.byref(p), None, None), "cf_set_get_params")
    return CFSet(h, p.grid_n, p.oversampling, p.n_pa_bins, p.n_subbands)


class Plan:
    """Owns an awg_plan: the per-sample index and tiled ordering of R x C samples."""

    def __init__(self, cf: CFSet, uvw_m: torch.Tensor, freq_hz: torch.Tensor, pa_bin: Optional[torch.Tensor] = None,
                 chan_subband: Optional[torch.Tensor] = None, phase_shift=None, stream=None):
        _need(uvw_m, "uvw_m", torch.float64)
        _need(freq_hz, "freq_hz", torch.float64)
        if uvw_m.dim() != 2 or uvw_m.shape[1] != 3:
            raise ValueError("uvw_m must be [R, 3]")
        if pa_bin is not None:
            _need(pa_bin, "pa_bin", torch.int32, (uvw_m.shape[0],))
        if chan_subband is not None:
            _need(chan_subband, "chan_subband", torch.int32, (freq_hz.shape[0],))
        self.cf = cf
        self.n_rows = int(uvw_m.shape[0])
        self.n_chan = int(freq_hz.shape[0])
        ph = None
        if phase_shift is not None:
            ph = np.ascontiguousarray(phase_shift, dtype=np.float64)
        h = ctypes.c_void_p()
        check(_lib.load().plan_create(cf.handle, _ptr(uvw_m), self.n_rows, _ptr(freq_hz), self.n_chan, _ptr(pa_bin),
                                      _ptr(chan_subband),
                                      ph.ctypes.data_as(ctypes.c_void_p) if ph is not None else None,
                                      _stream_ptr(stream), ctypes.byref(h)), "plan_create")
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("plan already destroyed")
        return self._h

    def set_row_phase(self, row_dlm: Optional[torch.Tensor], uvw_m: torch.Tensor, freq_hz: torch.Tensor, stream=None):
        """Per-row phase centres (mosaic pointings / pointing offsets): row_dlm f64 [R, 2] on the
        device, or None to return to the plan-wide shift (see plan_set_row_phase)."""
        _need(uvw_m, "uvw_m", torch.float64, (self.n_rows, 3))
        _need(freq_hz, "freq_hz", torch.float64, (self.n_chan,))
        if row_dlm is not None:
            _need(row_dlm, "row_dlm", torch.float64, (self.n_rows, 2))
        check(_lib.load().plan_set_row_phase(self.handle, _ptr(row_dlm), _ptr(uvw_m), _ptr(freq_hz),
                                             _stream_ptr(stream)), "plan_set_row_phase")

    def update(self, uvw_m, freq_hz, pa_bin=None, chan_subband=None, stream=None):
        _need(uvw_m, "uvw_m", torch.float64, (self.n_rows, 3))
        _need(freq_hz, "freq_hz", torch.float64, (self.n_chan,))
        check(_lib.load().plan_update(self.handle, _ptr(uvw_m), _ptr(freq_hz), _ptr(pa_bin), _ptr(chan_subband),
                                      _stream_ptr(stream)), "plan_update")

    def stats(self):
        """(kept samples, dropped samples, sum over kept samples of S^2); synchronises."""
        k, d, t = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        check(_lib.load().plan_stats(self.handle, ctypes.byref(k), ctypes.byref(d), ctypes.byref(t)), "plan_stats")
        return int(k.value), int(d.value), int(t.value)

    def check(self):
        """Raise AwgError (AWG_ERR_TIMEOUT) if a launch of this plan ended on a bounded wait that
        gave up (plan_check); synchronises."""
        check(_lib.load().plan_check(self.handle), "plan_check")

    def index(self) -> dict:
        """Host copy of the per-sample index in sample order (plan_copy_index): int32 arrays
        [R * C] 'kept' (records of the sample), 'cf', 'p0x', 'p0y', 'ox', 'oy' (-1 when dropped);
        synchronises."""
        n = self.n_rows * self.n_chan
        out = {k: np.empty(max(n, 1), dtype=np.int32) for k in ("kept", "cf", "p0x", "p0y", "ox", "oy")}
        ptrs = [out[k].ctypes.data_as(ctypes.c_void_p) for k in ("kept", "cf", "p0x", "p0y", "ox", "oy")]
        check(_lib.load().plan_copy_index(self.handle, *ptrs), "plan_copy_index")
        return {k: v[:n] for k, v in out.items()}

    def close(self):
        if self._h is not None:
            check(_lib.load().plan_destroy(self._h), "plan_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_create(cf: CFSet, uvw_m, freq_hz, pa_bin=None, chan_subband=None, phase_shift=None, stream=None) -> Plan:
    return Plan(cf, uvw_m, freq_hz, pa_bin, chan_subband, phase_shift, stream)


def _pols(vis: torch.Tensor) -> int:
    return int(vis.shape[-1])


def grid_visibilities(cf: CFSet, plan: Plan, vis: torch.Tensor, weight: torch.Tensor, grid: torch.Tensor,
                      sumwt: torch.Tensor, grid_lo: Optional[torch.Tensor] = None, flags: int = 0, stream=None):
    """G (Eq. IMAGE-MOD): grid += sum conj(CF) * weight * vis; sumwt += sum weight (see awgrid.h)."""
    R, C = plan.n_rows, plan.n_chan
    P = _pols(vis)
    N = cf.grid_n
    _need(vis, "vis", torch.complex64, (R, C, P))
    _need(weight, "weight", torch.float32, (R, C, P))
    _need(grid, "grid", torch.complex128 if flags & AWG_GRID_FP64 else torch.complex64, (N, N, P))
    _need(sumwt, "sumwt", torch.float64, (P,))
    if grid_lo is not None:
        _need(grid_lo, "grid_lo", torch.complex64, (N, N, P))
    check(_lib.load().grid_visibilities(cf.handle, plan.handle, _ptr(vis), _ptr(weight), P, _ptr(grid), _ptr(grid_lo),
                                        _ptr(sumwt), int(flags), _stream_ptr(stream)), "grid_visibilities")


def degrid_visibilities(cf: CFSet, plan: Plan, grid: torch.Tensor, vis_out: torch.Tensor, stream=None,
                        subtract: bool = False):
    """D (Eq. ME-MOD-GRIDDED): vis_out = sum CF * grid (overwritten; dropped samples get 0).  With
    subtract, vis_out holds the observed visibilities and receives the residual V - D(grid) of Eq.
    ResIm in place (dropped samples keep their input)."""
    R, C = plan.n_rows, plan.n_chan
    P = _pols(grid)
    N = cf.grid_n
    _need(grid, "grid", torch.complex64, (N, N, P))
    _need(vis_out, "vis_out", torch.complex64, (R, C, P))
    flags = AWG_DEGRID_SUBTRACT if subtract else 0
    check(_lib.load().degrid_visibilities(cf.handle, plan.handle, _ptr(grid), _ptr(vis_out), P, flags,
                                          _stream_ptr(stream)), "degrid_visibilities")


def grid_normalize(cf: CFSet, image: torch.Tensor, sumwt: Optional[torch.Tensor] = None, direction: int = 0,
                   stream=None):
    """Divide by the PS taper T(x) T(y) (and by sumwt for direction 0), in place."""
    N = cf.grid_n
    P = _pols(image)
    _need(image, "image", torch.complex64, (N, N, P))
    if sumwt is not None:
        _need(sumwt, "sumwt", torch.float64, (P,))
    check(_lib.load().grid_normalize(cf.handle, _ptr(image), P, _ptr(sumwt), int(direction), _stream_ptr(stream)),
          "grid_normalize")


class CleanWorkspace:
    """Device workspace of clean_hogbom (holds the iteration state and the component count)."""

    def __init__(self, device="cuda"):
        nbytes = int(_lib.load().clean_hogbom_workspace_bytes())
        self.buf = torch.zeros((nbytes + 15) // 16 * 4, dtype=torch.float32, device=device)

    def components(self) -> int:
        n = ctypes.c_int32()
        check(_lib.load().clean_hogbom_components(_ptr(self.buf), ctypes.byref(n)), "clean_hogbom_components")
        return int(n.value)


def clean_hogbom(residual: torch.Tensor, model: torch.Tensor, psf: torch.Tensor, n_iter: int, gain: float = 0.1,
                 threshold: float = 0.0, window=None, workspace: Optional[CleanWorkspace] = None,
                 stream=None) -> CleanWorkspace:
    """Hogbom minor cycle in place on residual / model (f32 [N, N]) with psf (f32 [Np, Np], peak at
    Np/2); window = (x0, x1, y0, y1) or None.  Asynchronous; returns the workspace (component count)."""
    N = residual.shape[0]
    _need(residual, "residual", torch.float32, (N, N))
    _need(model, "model", torch.float32, (N, N))
    if psf.dim() != 2 or psf.shape[0] != psf.shape[1]:
        raise ValueError("psf must be square")
    _need(psf, "psf", torch.float32)
    ws = workspace or CleanWorkspace(residual.device)
    win = None
    if window is not None:
        win = np.ascontiguousarray(window, dtype=np.int32)
        if win.shape != (4,):
            raise ValueError("window must be (x0, x1, y0, y1)")
    check(_lib.load().clean_hogbom(_ptr(residual), _ptr(model), N, _ptr(psf), psf.shape[0], int(n_iter), float(gain),
                                   float(threshold), None if win is None else win.ctypes.data_as(ctypes.c_void_p),
                                   _ptr(ws.buf), _stream_ptr(stream)), "clean_hogbom")
    return ws


def gcal_solve(vis: torch.Tensor, model: torch.Tensor, weight: torch.Tensor, ant1: torch.Tensor, ant2: torch.Tensor,
               n_ant: int, sol_int: int, sol_chan: int, alpha: float = 0.5, delta: float = 1e-10,
               max_iter: int = 200, ref_ant: int = 0, stream=None):
    """G-Jones solve (see gcal_solve in awgrid.h).  vis / model c64 [R, C, P], weight f32 [R, C, P]
    on the device, rows time-major over the len(ant1) baselines.  Returns (gains c128
    [n_ts, n_fs, n_hands, n_ant], iterations int32 [n_ts, n_fs, n_hands]); asynchronous."""
    R, C, P = vis.shape
    _need(vis, "vis", torch.complex64, (R, C, P))
    _need(model, "model", torch.complex64, (R, C, P))
    _need(weight, "weight", torch.float32, (R, C, P))
    n_bl = ant1.shape[0]
    _need(ant1, "ant1", torch.int32, (n_bl,))
    _need(ant2, "ant2", torch.int32, (n_bl,))
    if R % n_bl:
        raise ValueError("the number of rows must be a multiple of the number of baselines")
    n_int = R // n_bl
    n_ts, n_fs, n_h = -(-n_int // sol_int), -(-C // sol_chan), (1 if P == 1 else 2)
    gains = torch.empty((n_ts, n_fs, n_h, n_ant), dtype=torch.complex128, device=vis.device)
    iters = torch.empty((n_ts, n_fs, n_h), dtype=torch.int32, device=vis.device)
    nbytes = int(_lib.load().gcal_workspace_bytes(R, C, P, n_bl, sol_int, sol_chan))
    ws = torch.empty(max(nbytes, 16) // 8 + 2, dtype=torch.float64, device=vis.device)
    check(_lib.load().gcal_solve(_ptr(vis), _ptr(model), _ptr(weight), R, C, P, n_bl, _ptr(ant1), _ptr(ant2),
                                 int(n_ant), int(sol_int), int(sol_chan), float(alpha), float(delta), int(max_iter),
                                 int(ref_ant), _ptr(gains), _ptr(iters), _ptr(ws), _stream_ptr(stream)), "gcal_solve")
    return gains, iters
