"""Imaging major cycle with a Hogbom minor cycle (Sec. 5.2): residual image (Eq. ResIm) from the
library's gridding and degridding, point components found on the GPU (clean_hogbom), model update
(Eq. ModelUpdate).  Every step is stream-ordered device work, so one whole major cycle can be
captured in a CUDA graph.

Images are single-plane FP32 [N, N] (the first polarisation product); the FFT is torch.fft, as
everywhere in this package.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import api
from .autograd import ForwardModel, chi2, inner_mask, residual_image


def dirty_beam(fm: ForwardModel, weight: torch.Tensor) -> torch.Tensor:
    """Point-spread function of the weighted sampling: the residual image of unit visibilities
    against an empty model, i.e. F^H G W 1 / (sum w T T); FP32 [N, N] with its peak at (N/2, N/2)."""
    N = fm.cf.grid_n
    ones = torch.ones((fm.plan.n_rows, fm.plan.n_chan, fm.P), dtype=torch.complex64, device=weight.device)
    zero = torch.zeros((N, N, fm.P), dtype=torch.float32, device=weight.device)
    return residual_image(fm, zero, ones, weight)[..., 0].contiguous()


class CleanCycle:
    """Major cycles of residual imaging plus a Hogbom minor cycle; holds the PSF, the model and
    the minor-cycle workspace so that `step` allocates nothing of its own."""

    def __init__(self, fm: ForwardModel, vis: torch.Tensor, weight: torch.Tensor, n_minor: int = 100,
                 gain: float = 0.1, threshold: float = 0.0, window=None):
        N = fm.cf.grid_n
        self.fm, self.vis, self.weight = fm, vis, weight
        self.n_minor, self.gain, self.threshold = n_minor, gain, threshold
        self.window = window if window is not None else (N // 4, 3 * N // 4, N // 4, 3 * N // 4)
        self.psf = dirty_beam(fm, weight)
        self.model = torch.zeros((N, N), dtype=torch.float32, device=vis.device)
        self.residual = torch.zeros((N, N), dtype=torch.float32, device=vis.device)
        self.ws = api.CleanWorkspace(vis.device)

    def step(self):
        """One major cycle: residual image of the current model, then n_minor Hogbom iterations
        that add components to the model (in place)."""
        r = residual_image(self.fm, self.model[..., None].expand(-1, -1, self.fm.P), self.vis, self.weight)
        self.residual.copy_(r[..., 0])
        api.clean_hogbom(self.residual, self.model, self.psf, self.n_minor, self.gain, self.threshold, self.window,
                         self.ws)

    def chi2(self) -> float:
        return float(chi2(self.fm(self.model[..., None].expand(-1, -1, self.fm.P)), self.vis, self.weight))


def clean_major_cycles(fm: ForwardModel, vis: torch.Tensor, weight: torch.Tensor, n_major: int = 3,
                       n_minor: int = 100, gain: float = 0.1, threshold: float = 0.0, window=None):
    """Run n_major cycles; returns (model image, chi^2 before and after each cycle)."""
    cc = CleanCycle(fm, vis, weight, n_minor, gain, threshold, window)
    hist = [cc.chi2()]
    for _ in range(n_major):
        cc.step()
        hist.append(cc.chi2())
    return cc.model, hist
