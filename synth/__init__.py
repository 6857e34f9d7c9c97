"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package generates *inputs only*: procedural meshes, textures, cameras and
lights shaped like the workloads of appearance-driven simplification (the
paper's Sec. 3 setup: a low-poly latent mesh with textures, optimized against
renders of a high-poly reference from random cameras and lights). It contains
none of the method's arithmetic (no rasterization, shading, loss, gradients or
optimizer); both the oracle and the CUDA path consume the arrays it returns.
"""

from .scenes import (  # noqa: F401
    icosphere,
    equirect_uv_corners,
    radial_sinusoids,
    radial_fbm,
    noise_textures,
    procedural_textures,
    constant_texture,
    Mesh,
)
from .views import (  # noqa: F401
    VIEW_DTYPE,
    look_at,
    perspective,
    make_view,
    sample_views,
    fixed_view,
)
from .workloads import (  # noqa: F401
    Scene,
    config_small,
    config_plain,
    config_tess,
    job_mix,
    job_scenes,
)
from .aggregate import (  # noqa: F401
    quad_cloud,
    config_aggregate,
)
from .rig import (  # noqa: F401
    bone_weights,
    bone_pose,
)
