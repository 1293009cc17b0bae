"""FP64 CPU oracle for AW-projection gridding and degridding.

TEST INFRASTRUCTURE ONLY.  Nothing in the library path imports, calls, links or runs
anything in this package; only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may.  It shares no code
with the CUDA library (no kernels, headers, helpers, tables or constant generators);
the only code both sides see is the seeded input generator in ``synth``.

What it computes, and the passages it follows:

* ``pswf``   - the zeroth prolate spheroidal wave function psi_0(c, x), the
  "anti-aliasing Prolate Spheroidal" term of Tab. AWP-CFSETUP (Sec. 6), from the
  Legendre-basis form of the spheroidal differential equation.
* ``cf``     - convolution functions PS, PS*W, PS*A, PS*A*W of Tab. AWP-CFSETUP
  as the Fourier transform of the image-plane product of the terms, written out as
  a direct DFT (two matrix products), oversampled and cropped.
* ``index``  - per-sample uv scaling, w-plane and CF selection (CF_ij(nu, w, t) of
  Eq. CIJ), grid pixel and oversampling offset.
* ``ops``    - the gridding operator G (Eq. IMAGE-MOD, conjugated kernel) and the
  degridding operator D (Eq. ME-MOD-GRIDDED) as the plain sums they are, in FP64.
* ``image``  - F-dagger of the grid, the taper correction, the brute-force DFT
  image and analytic point-source visibilities (Eq. ME with a point-source sky).
* ``clean``  - the Hogbom minor cycle (Sec. 5.2, Eq. ModelUpdate with point components), in
  FP32 because its peak search decides integer positions.
* ``gcal``   - the direction-independent G-Jones solver (Sec. 5.1: Eq. VAvg, Eq. CalUpdateDir,
  Eq. CalUpdateModel) in FP64.

Every function states the passage it follows.  Where the paper is silent, the
reading taken is stated beside the function that takes it.  Parity of the
synthetic A-term model is unpinned (the paper gives no A-term formula).
"""
from . import pswf, cf, index, ops, image, clean, gcal  # noqa: F401
