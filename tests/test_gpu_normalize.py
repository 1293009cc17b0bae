"""grid_normalize (the taper and sum-of-weights division of Eq. IMAGE-MOD with the PS term of
Tab. AWP-CFSETUP) against the oracle.

The library divides by T(x - N/2) T(y - N/2) with T from its own spheroidal solver (Sturm bisection
and inverse iteration in cf_build.cpp), rounded to FP32; the oracle's T comes from LAPACK's
tridiagonal eigen-solver (oracle/pswf.py).  Both are FP64 evaluations of psi_0, so per pixel the
two corrections agree to the FP32 rounding of the library's 1/T values and of the product, a few
units of 2^-24 relative; the element-wise gates below allow 1e-6 relative.  The whole dirty-image
chain (gridding, the caller's inverse FFT, grid_normalize) is gated like every dirty image: 1e-5
relative RMS over the inner half of the field (readings R12 and R13).
"""
import numpy as np
import pytest

import synth
from oracle import image as oimage
from oracle import index as oindex
from oracle import cf as ocf
from oracle import ops as oops
from tests.helpers import inner_half, library_params, oracle_params, rel_rms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def awg():
    import paper_2508_17187_gb300 as m
    from paper_2508_17187_gb300 import _lib
    _lib.load()          # fails loudly when the library is missing: there is no fallback
    assert torch.cuda.is_available()
    return m


def _cf(awg, N=512, ps_support=7, use_ps=True):
    wl = synth.make_workload("standard", n_int=4, with_vis=False)
    op = oracle_params(wl, grid_n=N, ps_support=ps_support, use_ps=use_ps, max_support=8, oversampling=4)
    return op, awg.cf_set_create(**library_params(op))


def _oracle_tt(op):
    t = oimage.taper_image(op.grid_n, op.ps_support) if op.use_ps else np.ones(op.grid_n)
    return t[:, None] * t[None, :]


@pytest.mark.parametrize("P", [1, 2, 4])
def test_direction1_divides_by_the_oracle_taper(awg, P):
    """Model image before F: image / (T T), compared pixel by pixel over the whole image."""
    op, cf = _cf(awg)
    N = op.grid_n
    rng = np.random.default_rng(11)
    img = (rng.standard_normal((N, N, P)) + 1j * rng.standard_normal((N, N, P))).astype(np.complex64)
    t = torch.as_tensor(img).cuda()
    awg.grid_normalize(cf, t, None, direction=1)
    got = t.cpu().numpy().astype(np.complex128)
    want = img.astype(np.complex128) / _oracle_tt(op)[:, :, None]
    rel = np.abs(got - want) / np.abs(want)
    assert rel.max() < 1e-6, rel.max()


@pytest.mark.parametrize("P", [1, 2, 4])
def test_direction0_divides_by_sumwt_and_the_oracle_taper(awg, P):
    """After F-dagger: image / (sumwt[p] T T) per pol, pixel by pixel; sumwt = NULL means 1."""
    op, cf = _cf(awg, N=256)
    N = op.grid_n
    rng = np.random.default_rng(12)
    img = (rng.standard_normal((N, N, P)) + 1j * rng.standard_normal((N, N, P))).astype(np.complex64)
    sumwt = rng.uniform(1e3, 1e7, P)
    t = torch.as_tensor(img).cuda()
    awg.grid_normalize(cf, t, torch.as_tensor(sumwt).cuda(), direction=0)
    got = t.cpu().numpy().astype(np.complex128)
    want = img.astype(np.complex128) / (sumwt[None, None, :] * _oracle_tt(op)[:, :, None])
    rel = np.abs(got - want) / np.abs(want)
    assert rel.max() < 1e-6, rel.max()
    t = torch.as_tensor(img).cuda()
    awg.grid_normalize(cf, t, None, direction=0)
    got = t.cpu().numpy().astype(np.complex128)
    want = img.astype(np.complex128) / _oracle_tt(op)[:, :, None]
    assert (np.abs(got - want) / np.abs(want)).max() < 1e-6


def test_unaligned_image_and_no_taper(awg):
    """An image that starts 8 bytes past a 16-byte boundary (the float2 path of the kernel), and a
    set without the PS term (T = 1: only the sum of weights divides)."""
    op, cf = _cf(awg, N=128)
    N, P = op.grid_n, 4
    rng = np.random.default_rng(13)
    img = (rng.standard_normal((N, N, P)) + 1j * rng.standard_normal((N, N, P))).astype(np.complex64)
    buf = torch.zeros(N * N * P + 1, dtype=torch.complex64, device="cuda")
    view = buf[1:].view(N, N, P)
    assert view.data_ptr() % 16 == 8
    view.copy_(torch.as_tensor(img).cuda())
    awg.grid_normalize(cf, view, None, direction=1)
    got = view.cpu().numpy().astype(np.complex128)
    want = img.astype(np.complex128) / _oracle_tt(op)[:, :, None]
    assert (np.abs(got - want) / np.abs(want)).max() < 1e-6
    assert buf[0].item() == 0
    op0, cf0 = _cf(awg, N=128, use_ps=False)
    t = torch.as_tensor(img).cuda()
    sw = np.array([2.0, 4.0, 8.0, 16.0])
    awg.grid_normalize(cf0, t, torch.as_tensor(sw).cuda(), direction=0)
    assert np.allclose(t.cpu().numpy(), img / sw[None, None, :], rtol=1e-7, atol=0)


def test_dirty_image_chain_matches_oracle(awg):
    """Gridding, the inverse FFT (torch.fft, same origin convention as the oracle) and
    grid_normalize(direction 0) with the library's own sum of weights, against
    oracle.image.dirty_image of the oracle's FP64 grid and sum of weights."""
    wl = synth.make_workload("wproj", n_int=20, n_chan=8, grid_n=512, n_wplanes=6, max_support=32)
    op = oracle_params(wl)
    N, P = wl.grid_n, wl.n_pol
    cf = awg.cf_set_create(**library_params(op))
    plan = awg.plan_create(cf, torch.as_tensor(wl.uvw_m).cuda(), torch.as_tensor(wl.freq_hz).cuda())
    g = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda")
    sw = torch.zeros(P, dtype=torch.float64, device="cuda")
    awg.grid_visibilities(cf, plan, torch.as_tensor(wl.vis).cuda(), torch.as_tensor(wl.weight).cuda(), g, sw)
    x = torch.fft.ifftshift(g, dim=(0, 1))
    img = torch.fft.fftshift(torch.fft.ifft2(x, dim=(0, 1), norm="forward"), dim=(0, 1)).contiguous()
    awg.grid_normalize(cf, img, sw, direction=0)
    got = img.real.cpu().numpy().astype(np.float64)

    idx = oindex.sample_index(op, wl.uvw_m, wl.freq_hz)
    tabs = ocf.cf_set(op, which=set(np.unique(idx.cf[idx.valid]).tolist()))
    buf, off, _ = ocf.flatten_cf_set(op, tabs)
    n = wl.n_rows * wl.n_chan
    g_o, sw_o = oops.grid(idx, buf, off, op.oversampling, N, wl.vis.reshape(n, P), wl.weight.reshape(n, P))
    want = oimage.dirty_image(g_o, sw_o, op.ps_support)
    assert np.allclose(sw.cpu().numpy(), sw_o, rtol=1e-12)
    err = rel_rms(inner_half(got), inner_half(want))
    assert err < 1e-5, err
