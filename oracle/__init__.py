"""FP64 CPU oracle for the 4D-rotor Gaussian splatting render and its gradient.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(``paper_2402_03307_gb300``) never does, and the two share no code.

The oracle is the plain definition of what the renderer computes, written in
plain PyTorch CPU operations in float64, one step per passage of the paper:

  rotor.py       rotor normalisation F_norm (appendix A.1) and the rotor ->
                 4x4 rotation map F_map (appendix A.2)
  slicing.py     Sigma4 = R S S^T R^T (Sec. 3.2.1) and the temporal slice
                 (Eq. 6/7 of Sec. 3.2.2, appendix A.3, numerically stable form)
  sh.py          real spherical harmonics up to degree 3 (view colour, Sec. 3.1)
  projection.py  world -> camera -> EWA 2D covariance (Sec. 3.1)
  render.py      per-pixel brute-force front-to-back compositing over every
                 Gaussian in global depth order (Eq. 3), no tiles and no sort
                 kernel; gradients by torch.autograd of the same function

Every threshold decision (3-sigma cutoff, alpha >= 1/255, T < 1e-4, depth
order) is also reported with its margin so that tests can tell pixels whose
result depends on rounding from pixels whose result is unique.
"""
from .rotor import rotor_epsilon, rotor_normalize, rotor_to_matrix  # noqa: F401
from .slicing import covariance4, slice_at  # noqa: F401
from .sh import sh_basis, sh_color  # noqa: F401
from .projection import camera_tensors, project  # noqa: F401
from .render import (  # noqa: F401
    ALPHA_MAX, ALPHA_MIN, NEAR, POWER_CUT, T_MIN, TEMPORAL_CUT, DILATION,
    preprocess, render, render_pixels, render_grad, render_grad_pixels, pixel_alternatives, to_f64,
)
