"""GB300 (sm_103a) render-and-compare step of appearance-driven mesh simplification.

The CUDA library (csrc/, C ABI in include/adms.h) renders a latent textured
mesh under batches of cameras and lights, antialiases silhouettes, takes the
tone-mapped L1 loss against reference renders, backpropagates to vertex
positions and texels, and applies Adam. `binding` mirrors the C ABI;
`engine.Context` is a thin convenience layer over it.
"""

from . import binding  # noqa: F401

__all__ = ["binding"]
