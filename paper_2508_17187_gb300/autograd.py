"""Differentiable imaging forward model on top of the C ABI.

Eq. ImChisq (Sec. 5.2) writes the imaging chi^2 as [V - D F I]^H W [V - D F I]; its gradient with
respect to the image is the residual image of Eq. ResIm, F^H G W (V - D F I), because G is the
adjoint of D.  `DegridFn` makes that explicit for PyTorch: its forward is degridding
(degrid_visibilities) and its hand-written backward is gridding (grid_visibilities with unit
weights), which is exactly D^H for the complex-linear operators of this library.  PyTorch's
complex convention passes dL/d(conj y) to backward and expects A^H of it for y = A x.

`ForwardModel` maps a real image [N, N] (or [N, N, P]) to model visibilities: divide by the PS
taper T(x)T(y), F (torch.fft, the library has no FFT), then D.  `residual_image` and
`major_cycle` run Eq. ResIm / Eq. ModelUpdate (steepest descent, step from the largest eigenvalue
of the normal operator).
"""
from __future__ import annotations

from typing import Optional

import torch

from . import api


class DegridFn(torch.autograd.Function):
    """vis = D(grid); backward: grad_grid = G(grad_vis) with unit weights."""

    @staticmethod
    def forward(ctx, grid: torch.Tensor, cf: "api.CFSet", plan: "api.Plan", ones: torch.Tensor):
        grid = grid.contiguous()
        P = grid.shape[-1]
        out = torch.empty((plan.n_rows, plan.n_chan, P), dtype=torch.complex64, device=grid.device)
        api.degrid_visibilities(cf, plan, grid, out)
        ctx.cf, ctx.plan = cf, plan
        ctx.save_for_backward(ones)
        ctx.grid_shape = tuple(grid.shape)
        return out

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (ones,) = ctx.saved_tensors
        g = torch.zeros(ctx.grid_shape, dtype=torch.complex64, device=grad_out.device)
        sw = torch.zeros(ctx.grid_shape[-1], dtype=torch.float64, device=grad_out.device)
        api.grid_visibilities(ctx.cf, ctx.plan, grad_out.contiguous().to(torch.complex64), ones, g, sw)
        return g, None, None, None


def image_to_grid(image: torch.Tensor, inv_taper2d: torch.Tensor) -> torch.Tensor:
    """F of image / (T T): [N, N, P] complex grid with the uv origin at N/2 (differentiable)."""
    x = image.to(torch.complex64) * inv_taper2d[..., None]
    x = torch.fft.ifftshift(x, dim=(0, 1))
    g = torch.fft.fft2(x, dim=(0, 1))
    return torch.fft.fftshift(g, dim=(0, 1))


class ForwardModel:
    """image [N, N, P] (real) -> model visibilities [R, C, P], differentiable through DegridFn."""

    def __init__(self, cf: "api.CFSet", plan: "api.Plan", n_pol: int, device="cuda"):
        self.cf, self.plan, self.P = cf, plan, n_pol
        N = cf.grid_n
        # 1 / (T(x) T(y)) from the library's own taper: grid_normalize(direction=1) on ones
        ones = torch.ones((N, N, 1), dtype=torch.complex64, device=device)
        api.grid_normalize(cf, ones, None, direction=1)
        self.inv_taper2d = ones[..., 0].real.contiguous()
        self.ones_w = torch.ones((plan.n_rows, plan.n_chan, n_pol), dtype=torch.float32, device=device)

    def __call__(self, image: torch.Tensor) -> torch.Tensor:
        grid = image_to_grid(image, self.inv_taper2d)
        return DegridFn.apply(grid, self.cf, self.plan, self.ones_w)


def chi2(model_vis: torch.Tensor, vis: torch.Tensor, weight: torch.Tensor) -> torch.Tensor:
    """Eq. Chisq: sum w |V - V_model|^2 (FP64 accumulation)."""
    r = (vis - model_vis)
    return (weight.double() * (r.real.double() ** 2 + r.imag.double() ** 2)).sum()


def residual_vis(fm: ForwardModel, image: torch.Tensor, vis: torch.Tensor) -> torch.Tensor:
    """The data residual V - D F I of Eq. ResIm, formed by the degridding itself
    (AWG_DEGRID_SUBTRACT) in one pass over the visibilities."""
    res = vis.contiguous().clone()
    api.degrid_visibilities(fm.cf, fm.plan, image_to_grid(image, fm.inv_taper2d).contiguous(), res, subtract=True)
    return res


def chi2_of_residual(res: torch.Tensor, weight: torch.Tensor) -> torch.Tensor:
    """Eq. Chisq from a data residual: sum w |res|^2 (FP64 accumulation, as chi2)."""
    return (weight.double() * (res.real.double() ** 2 + res.imag.double() ** 2)).sum()


def image_of_residual(fm: ForwardModel, res: torch.Tensor, weight: torch.Tensor) -> torch.Tensor:
    """F^H G W res, normalised by the weights and the taper: the residual image of a data residual."""
    cf, plan = fm.cf, fm.plan
    N, P = cf.grid_n, fm.P
    g = torch.zeros((N, N, P), dtype=torch.complex64, device=res.device)
    sw = torch.zeros(P, dtype=torch.float64, device=res.device)
    api.grid_visibilities(cf, plan, res.contiguous(), weight, g, sw)
    im = torch.fft.fftshift(torch.fft.ifft2(torch.fft.ifftshift(g, dim=(0, 1)), dim=(0, 1)), dim=(0, 1)) * (N * N)
    im = im.contiguous()
    api.grid_normalize(cf, im, sw, direction=0)
    return im.real


def residual_image(fm: ForwardModel, image: torch.Tensor, vis: torch.Tensor, weight: torch.Tensor) -> torch.Tensor:
    """Eq. ResIm for one partition: F^H G W (V - D F I), normalised by the weights and the taper."""
    return image_of_residual(fm, residual_vis(fm, image, vis), weight)


def inner_mask(N: int, device="cuda") -> torch.Tensor:
    """1 on the inner half of the field (|x|, |y| < N/4), where the PS taper is above 0.25."""
    m = torch.zeros((N, N, 1), dtype=torch.float32, device=device)
    m[N // 4:3 * N // 4, N // 4:3 * N // 4] = 1.0
    return m


def largest_eigenvalue(fm: ForwardModel, weight: torch.Tensor, mask: torch.Tensor, n_power: int = 8) -> float:
    """Power iteration on the masked normal operator x -> mask F^H G W D F (mask x) (the residual image
    of zero data is minus this): its largest eigenvalue bounds the stable steepest-descent step."""
    N, P = fm.cf.grid_n, fm.P
    zero = torch.zeros((fm.plan.n_rows, fm.plan.n_chan, P), dtype=torch.complex64, device=weight.device)
    g = torch.Generator(device=weight.device).manual_seed(3)
    x = torch.randn((N, N, P), device=weight.device, generator=g) * mask
    lam = 1.0
    with torch.no_grad():
        for _ in range(n_power):
            x = x / x.norm()
            hx = -residual_image(fm, x, zero, weight) * mask
            lam = float((hx * x).sum())
            x = hx
    return lam


def major_cycle(fm: ForwardModel, vis: torch.Tensor, weight: torch.Tensor, n_iter: int = 10,
                gain: Optional[float] = None, image: Optional[torch.Tensor] = None,
                mask: Optional[torch.Tensor] = None):
    """Eq. ModelUpdate, I <- I + gain * mask * residual image, with the StepSize component's step
    gain = 1 / lambda_max of the masked normal operator unless given; returns (image, chi2 after each
    iteration).  Each iteration degrids once (the residual V - D F I, in place) and grids once.  The default mask keeps the model inside the inner half of the field: near the edge
    the taper correction divides by T(x)T(y) -> 0 on the way in and again on the way out."""
    N, P = fm.cf.grid_n, fm.P
    if image is None:
        image = torch.zeros((N, N, P), dtype=torch.float32, device=vis.device)
    if mask is None:
        mask = inner_mask(N, vis.device)
    if gain is None:
        gain = 1.0 / largest_eigenvalue(fm, weight, mask)
    # one degridding per cycle: the data residual of the updated image gives its chi^2 and the next
    # cycle's residual image
    hist = []
    with torch.no_grad():
        res = residual_vis(fm, image, vis)
        for _ in range(n_iter):
            image = image + gain * mask * image_of_residual(fm, res, weight)
            res = residual_vis(fm, image, vis)
            hist.append(float(chi2_of_residual(res, weight)))
    return image, hist
