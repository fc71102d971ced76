"""Plain, slow CPU oracle of the Bezier Splatting rasterizer.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything in this package.  The
product path (the CUDA library and its Python binding) never imports, links or
calls it, and this package imports nothing from the product package.

Floating point work is fp64 (torch CPU ops, so that autograd gives the exact
derivative of the same definition).  The two places where floating point
decides an integer -- the per-curve depth key and the tile rectangle of a
Gaussian -- are computed in float32 with a fixed sequence of correctly rounded
IEEE operations (numpy float32), the precision the CUDA kernels decide them in.

Modules
  curves   Section 3.2-3.3: Bezier curves, Gaussian sampling, draw order
  raster   Section 3.4: alpha blending (Eq. 9-10), per-pixel brute force
  binning  Section 3.4: tile rectangles and (tile, depth) keys
  loss     Section 3.5: the L2 term of Eq. 13
  prune_densify  Section 3.5, Algorithm 1, Appendix B: pruning, splitting,
           error regions and circular initialisation of new curves
  adam     Section 4.1: the Adam update (Kingma and Ba), box-projected
  cull     Section 3.4's blend and its hand-derived backward in C (OpenMP,
           exact box culling): the multi-core CPU baseline
  bounds   the sums of absolute per-pixel terms that scale the float32
           rounding of the gradients (Section 3.4's reverse walk, carried
           through the sampling of Section 3.3)

Parity pins: every function is pinned by a test in tests/test_oracle_*.py
against closed forms, invariants, brute force or finite differences; none is
"parity unpinned".
"""

from .curves import (  # noqa: F401
    bernstein, bezier, chain_sample_params, closed_boundaries, closed_tau,
    sample_open, sample_closed, covariance, area_keys_f32, draw_order,
    gaussian_table, table_to_f32, SampleCfg,
)
from .raster import render_pixels, render_image, render_grads  # noqa: F401
from .binning import tile_rects_f32, tile_keys, key_bits  # noqa: F401
from .loss import l2_loss  # noqa: F401
from .prune_densify import PDCfg, prune_densify  # noqa: F401
from .adam import adam_step  # noqa: F401
