"""GB300 (sm_103a) renderer for 4D-rotor Gaussian splatting (arXiv 2402.03307).

The compute path is libr4g.so (hand-written CUDA kernels behind a C ABI,
declared in include/r4g.h); this package is its PyTorch-facing binding.
Importing it loads the library and fails if it has not been built
(``paper_2402_03307_gb300.build.build()``).
"""
from . import abi  # noqa: F401
from .render import (  # noqa: F401
    PARAM_NAMES, BatchGraph, BatchResult, Render4DBatchFunction, Render4DFunction, Renderer, RenderResult,
    camera_struct, densify, densify_config, density_stats, gaussians_struct, image_loss, knn4d, opacity_reset,
    regularizers, render, render_batch, render_flow, sort32, sort_pairs, view_struct, views_tensor,
)

abi.lib()  # fail loudly here if libr4g.so is missing
