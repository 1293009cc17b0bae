"""Gridding G and degridding D as plain FP64 sums (oracle).

G follows Eq. IMAGE-MOD (Sec. 2): every kept sample adds conj(c) * w * V over the S x S
taps of its CF slice; the grid is complex128 [N, N, P] (pixel-major, pols innermost).
D follows Eq. ME-MOD-GRIDDED: V = sum over the same taps of c * grid.  The loops are in
``oracle_c.c`` (compiled here with gcc, -ffp-contract=off, OpenMP); ``grid_numpy`` and
``degrid_numpy`` restate the same sums with numpy for small inputs.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import sysconfig
import threading

import numpy as np

from .index import SampleIndex

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle_c.c")
_SO = os.path.join(_HERE, "_oracle_c.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle_c.c into _oracle_c.so (gcc, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
               _SRC, "-o", _SO + ".tmp"]
        subprocess.check_call(cmd)
        os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            p = ctypes.c_void_p
            i64, i32 = ctypes.c_int64, ctypes.c_int
            lib.oracle_grid.argtypes = [i64, p, p, p, p, p, p, p, p, i32, p, p, p, i32, p, i32, p, p, i32]
            lib.oracle_grid.restype = None
            lib.oracle_degrid.argtypes = [i64, p, p, p, p, p, p, p, p, i32, p, i32, p, i32, p, p, i32]
            lib.oracle_degrid.restype = None
            lib.oracle_grid_rows.argtypes = [i64, p, p, p, p, p, p, p, p, i32, p, p, p, i32, p, i32, i64, i64, p, i32]
            lib.oracle_grid_rows.restype = None
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def default_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def _prep(idx: SampleIndex):
    valid = np.ascontiguousarray(idx.valid.astype(np.uint8))
    cf = np.ascontiguousarray(idx.cf.astype(np.int32))
    p0x = np.ascontiguousarray(idx.p0x.astype(np.int64))
    p0y = np.ascontiguousarray(idx.p0y.astype(np.int64))
    ox = np.ascontiguousarray(idx.ox.astype(np.int32))
    oy = np.ascontiguousarray(idx.oy.astype(np.int32))
    sup = np.ascontiguousarray(idx.support.astype(np.int32))
    ph = None
    if idx.phasor is not None:
        ph = np.ascontiguousarray(np.stack([idx.phasor.real, idx.phasor.imag], -1).astype(np.float64))
    return valid, cf, p0x, p0y, ox, oy, sup, ph


def grid(idx: SampleIndex, cf_buf, cf_off, OS: int, N: int, vis, weight, nthreads=None):
    """G: returns (grid complex128 [N, N, P], sumwt float64 [P]).  vis [n, P], weight [n, P]."""
    lib = _load()
    n = idx.valid.shape[0]
    vis = np.asarray(vis).reshape(n, -1)
    P = vis.shape[1]
    vis_ri = np.ascontiguousarray(np.stack([vis.real, vis.imag], -1).astype(np.float64))
    wt = np.ascontiguousarray(np.asarray(weight, dtype=np.float64).reshape(n, P))
    cfd = np.ascontiguousarray(np.stack([cf_buf.real, cf_buf.imag], -1).astype(np.float64))
    off = np.ascontiguousarray(np.asarray(cf_off, dtype=np.int64))
    g = np.zeros((N, N, P, 2), dtype=np.float64)
    sw = np.zeros(P, dtype=np.float64)
    valid, cf, p0x, p0y, ox, oy, sup, ph = _prep(idx)
    lib.oracle_grid(n, _ptr(valid), _ptr(cf), _ptr(p0x), _ptr(p0y), _ptr(ox), _ptr(oy), _ptr(sup),
                    _ptr(ph), P, _ptr(vis_ri), _ptr(wt), _ptr(off), OS, _ptr(cfd), N, _ptr(g), _ptr(sw),
                    nthreads or default_threads())
    return g[..., 0] + 1j * g[..., 1], sw


def grid_rows(idx: SampleIndex, cf_buf, cf_off, OS: int, N: int, vis, weight, row_lo: int, row_hi: int,
              nthreads=None):
    """G restricted to grid rows [row_lo, row_hi): complex128 [row_hi - row_lo, N, P]."""
    lib = _load()
    n = idx.valid.shape[0]
    vis = np.asarray(vis).reshape(n, -1)
    P = vis.shape[1]
    vis_ri = np.ascontiguousarray(np.stack([vis.real, vis.imag], -1).astype(np.float64))
    wt = np.ascontiguousarray(np.asarray(weight, dtype=np.float64).reshape(n, P))
    cfd = np.ascontiguousarray(np.stack([cf_buf.real, cf_buf.imag], -1).astype(np.float64))
    off = np.ascontiguousarray(np.asarray(cf_off, dtype=np.int64))
    band = np.zeros((row_hi - row_lo, N, P, 2), dtype=np.float64)
    valid, cf, p0x, p0y, ox, oy, sup, ph = _prep(idx)
    lib.oracle_grid_rows(n, _ptr(valid), _ptr(cf), _ptr(p0x), _ptr(p0y), _ptr(ox), _ptr(oy), _ptr(sup), _ptr(ph),
                         P, _ptr(vis_ri), _ptr(wt), _ptr(off), OS, _ptr(cfd), N, row_lo, row_hi, _ptr(band),
                         nthreads or default_threads())
    return band[..., 0] + 1j * band[..., 1]


def degrid(idx: SampleIndex, cf_buf, cf_off, OS: int, grid_c, nthreads=None):
    """D: returns complex128 [n, P] (zero for dropped samples)."""
    lib = _load()
    n = idx.valid.shape[0]
    N, _, P = grid_c.shape
    gri = np.ascontiguousarray(np.stack([grid_c.real, grid_c.imag], -1).astype(np.float64))
    cfd = np.ascontiguousarray(np.stack([cf_buf.real, cf_buf.imag], -1).astype(np.float64))
    off = np.ascontiguousarray(np.asarray(cf_off, dtype=np.int64))
    out = np.zeros((n, P, 2), dtype=np.float64)
    valid, cf, p0x, p0y, ox, oy, sup, ph = _prep(idx)
    lib.oracle_degrid(n, _ptr(valid), _ptr(cf), _ptr(p0x), _ptr(p0y), _ptr(ox), _ptr(oy), _ptr(sup),
                      _ptr(ph), P, _ptr(off), OS, _ptr(cfd), N, _ptr(gri), _ptr(out),
                      nthreads or default_threads())
    return out[..., 0] + 1j * out[..., 1]


def _slice(cf_buf, cf_off, OS, cf, oy, ox, S):
    base = int(cf_off[cf]) + (int(oy) * (OS + 1) + int(ox)) * S * S
    return cf_buf[base:base + S * S].reshape(S, S)


def grid_numpy(idx: SampleIndex, cf_buf, cf_off, OS: int, N: int, vis, weight):
    """Same sum as ``grid`` with numpy (one sample at a time; small inputs only)."""
    n = idx.valid.shape[0]
    vis = np.asarray(vis).reshape(n, -1).astype(np.complex128)
    P = vis.shape[1]
    wt = np.asarray(weight, dtype=np.float64).reshape(n, P)
    g = np.zeros((N, N, P), dtype=np.complex128)
    sw = np.zeros(P)
    for s in np.nonzero(idx.valid)[0]:
        S = int(idx.support[s])
        c = _slice(cf_buf, cf_off, OS, idx.cf[s], idx.oy[s], idx.ox[s], S)
        a = wt[s] * vis[s]
        if idx.phasor is not None:
            a = a * idx.phasor[s]
        y0, x0 = int(idx.p0y[s]), int(idx.p0x[s])
        g[y0:y0 + S, x0:x0 + S, :] += np.conj(c)[:, :, None] * a[None, None, :]
        sw += wt[s]
    return g, sw


def degrid_numpy(idx: SampleIndex, cf_buf, cf_off, OS: int, grid_c):
    n = idx.valid.shape[0]
    P = grid_c.shape[2]
    out = np.zeros((n, P), dtype=np.complex128)
    for s in np.nonzero(idx.valid)[0]:
        S = int(idx.support[s])
        c = _slice(cf_buf, cf_off, OS, idx.cf[s], idx.oy[s], idx.ox[s], S)
        y0, x0 = int(idx.p0y[s]), int(idx.p0x[s])
        v = (c[:, :, None] * grid_c[y0:y0 + S, x0:x0 + S, :]).sum(axis=(0, 1))
        if idx.phasor is not None:
            v = v * np.conj(idx.phasor[s])
        out[s] = v
    return out


def grid_mueller(p, idx: SampleIndex, cf_buf, cf_off, OS: int, N: int, vis, weight, nthreads=None):
    """Full-polarisation G with the sparse Mueller matrix of CFs (Sec. 2, Sec. 6): grid pol q
    receives conj(CF_pq) w_p V_p for every kept element (p, q); sum of weights per pol from the
    diagonal elements.  vis, weight [n, 4]; returns (grid complex128 [N, N, 4], sumwt [4])."""
    from .cf import mueller_elements
    vis = np.asarray(vis).reshape(-1, 4)
    weight = np.asarray(weight, dtype=np.float64).reshape(-1, 4)
    g = np.zeros((N, N, 4), dtype=np.complex128)
    sw = np.zeros(4)
    for e, (pp, qq) in enumerate(mueller_elements(p)):
        idx_e = dataclasses.replace(idx, cf=idx.cf + e * p.n_base)
        ge, swe = grid(idx_e, cf_buf, cf_off, OS, N, vis[:, pp:pp + 1], weight[:, pp:pp + 1], nthreads)
        g[..., qq] += ge[..., 0]
        if pp == qq:
            sw[qq] += swe[0]
    return g, sw


def degrid_mueller(p, idx: SampleIndex, cf_buf, cf_off, OS: int, grid_c, nthreads=None):
    """Full-polarisation D: vis pol p = sum over kept elements (p, q) of CF_pq applied to grid pol q."""
    from .cf import mueller_elements
    out = np.zeros((idx.valid.shape[0], 4), dtype=np.complex128)
    for e, (pp, qq) in enumerate(mueller_elements(p)):
        idx_e = dataclasses.replace(idx, cf=idx.cf + e * p.n_base)
        out[:, pp] += degrid(idx_e, cf_buf, cf_off, OS, grid_c[..., qq:qq + 1], nthreads)[:, 0]
    return out
