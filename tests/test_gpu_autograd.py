"""Differentiable forward model (the autograd workload): 1024^2 sky -> F -> D to 5.01M visibilities
(351 baselines x 223 integrations x 64 channels, 1 pol, W-projection supports 8-32).

* DegridFn's hand-written backward (gridding) is the adjoint of its forward (degridding).
* The chi^2 gradient (Eq. ImChisq) from autograd matches central finite differences along random
  directions inside the inner half of the field.  chi^2 is a quadratic in the image, so a
  central difference has no truncation error and a large step only leaves FP32 rounding.
* The same gradient matches the oracle's FP64 -2 Re[T^-1 F^H D^H W (V - D F T^-1 I)] (Eq. ResIm).
* Ten steepest-descent major cycles (Eq. ModelUpdate, step 1 / lambda_max of the normal operator)
  lower chi^2 at every step.
"""
import time

import numpy as np
import pytest

import synth
from oracle import cf as ocf
from oracle import image as oimage
from oracle import index as oindex
from oracle import ops as oops
from tests.helpers import inner_half, library_params, oracle_params, rel_rms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import paper_2508_17187_gb300 as awg
    from paper_2508_17187_gb300 import autograd as ag
    from paper_2508_17187_gb300 import _lib
    _lib.load()
    wl = synth.make_workload("autograd", vis_device="cuda")
    op = oracle_params(wl)
    cf = awg.cf_set_create(**library_params(op))
    plan = awg.plan_create(cf, torch.as_tensor(wl.uvw_m).cuda(), torch.as_tensor(wl.freq_hz).cuda())
    fm = ag.ForwardModel(cf, plan, n_pol=1)
    sky = synth.gaussian_blob_sky(wl.grid_n, wl.cell_rad, wl.sky_l, wl.sky_m, wl.sky_flux)
    image = torch.as_tensor(sky).cuda()[..., None] * 0.5
    return awg, ag, wl, op, cf, plan, fm, image


def test_degrid_backward_is_adjoint(setup):
    awg, ag, wl, op, cf, plan, fm, image = setup
    N = wl.grid_n
    g = torch.Generator(device="cuda").manual_seed(synth.SEED_FD)
    X = torch.randn((N, N, 1), dtype=torch.complex64, device="cuda", generator=g)
    Y = torch.randn((wl.n_rows, wl.n_chan, 1), dtype=torch.complex64, device="cuda", generator=g)
    X.requires_grad_(True)
    out = ag.DegridFn.apply(X, cf, plan, fm.ones_w)
    (gx,) = torch.autograd.grad(out, X, grad_outputs=Y)
    lhs = torch.vdot(out.detach().reshape(-1).to(torch.complex128), Y.reshape(-1).to(torch.complex128))
    rhs = torch.vdot(X.detach().reshape(-1).to(torch.complex128), gx.reshape(-1).to(torch.complex128))
    assert abs(complex(lhs - rhs)) <= 1e-5 * abs(complex(lhs))


def test_chi2_gradient_finite_differences(setup):
    awg, ag, wl, op, cf, plan, fm, image = setup
    vis, wt = wl.vis, wl.weight
    I = image.clone().requires_grad_(True)
    loss = ag.chi2(fm(I), vis, wt)
    (grad,) = torch.autograd.grad(loss, I)
    g = torch.Generator(device="cuda").manual_seed(synth.SEED_FD)
    N = wl.grid_n
    inner = torch.zeros(I.shape, device="cuda")
    inner[N // 4:3 * N // 4, N // 4:3 * N // 4] = 1.0
    for _ in range(3):
        # directions inside the inner half of the field: outside it the model divides by a taper
        # product down to ~1e-7, and FP32 rounding of those amplified pixels would swamp the
        # difference being measured
        d = torch.randn(I.shape, device="cuda", generator=g) * inner
        eps = 1e-2 * float(image.norm()) / float(d.norm())
        with torch.no_grad():
            lp = ag.chi2(fm(image + eps * d), vis, wt)
            lm = ag.chi2(fm(image - eps * d), vis, wt)
        fd = float((lp - lm) / (2 * eps))
        an = float((grad.double() * d.double()).sum())
        assert abs(fd - an) <= 1e-3 * abs(an), (fd, an)


def test_chi2_gradient_matches_oracle_adjoint(setup):
    awg, ag, wl, op, cf, plan, fm, image = setup
    N = wl.grid_n
    I = image.clone().requires_grad_(True)
    loss = ag.chi2(fm(I), wl.vis, wl.weight)
    (grad,) = torch.autograd.grad(loss, I)
    # oracle: -2 Re[T^-1 F^H D^H W (V - D F T^-1 I)] in FP64
    idx = oindex.sample_index(op, wl.uvw_m, wl.freq_hz)
    tabs = ocf.cf_set(op, which=set(np.unique(idx.cf[idx.valid]).tolist()))
    buf, off, _ = ocf.flatten_cf_set(op, tabs)
    img = image.cpu().numpy().astype(np.float64)
    mgrid = oimage.model_to_grid(img, wl.ps_support)
    m = oops.degrid(idx, buf, off, op.oversampling, mgrid)
    vis = wl.vis.cpu().numpy().reshape(-1, 1).astype(np.complex128)
    w = wl.weight.cpu().numpy().reshape(-1, 1).astype(np.float64)
    r = w * (vis - m)
    g, _ = oops.grid(idx, buf, off, op.oversampling, N, r, np.ones_like(w))
    t = oimage.taper_image(N, wl.ps_support)
    ref = -2.0 * (oimage.grid_to_image(g) / (t[:, None] * t[None, :])[:, :, None]).real
    got = grad.cpu().numpy().astype(np.float64)
    assert rel_rms(inner_half(got), inner_half(ref)) < 1e-5


def test_major_cycle_lowers_chi2(setup):
    awg, ag, wl, op, cf, plan, fm, image = setup
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    img, hist = ag.major_cycle(fm, wl.vis, wl.weight, n_iter=10)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert all(b < a for a, b in zip(hist, hist[1:])), hist
    print(f"10 major cycles: {dt:.3f} s, chi2 {hist[0]:.4e} -> {hist[-1]:.4e}")
