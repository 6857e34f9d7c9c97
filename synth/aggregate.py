"""Aggregate-geometry workload (the foliage application of Sec. 6).

The paper replaces the leaves of a procedural plant (1.2M and 1.7M triangles)
by 11k and 6.5k textured quads whose shape, materials and opacity are
optimized under an L2 loss, rendered with depth peeling. Its Moana assets are
not available; these seeded quad clouds stand in for them: a reference canopy
of many small opaque leaf quads and a candidate of a few larger, half-opaque
billboard quads, both filling the same ellipsoid.
"""

from __future__ import annotations

import numpy as np

from . import scenes
from .scenes import Mesh


def quad_cloud(n_quads, seed, size=(0.05, 0.1), radii=(0.9, 0.7, 0.9)):
    """n_quads planar quads with centres uniform in an ellipsoid of the given
    radii, uniformly random orientation and half-sides uniform in `size`.

    Every quad has its own 4 vertices and 2 triangles ((0, 1, 2), (0, 2, 3))
    and maps to its own cell of a square texture atlas (cells row-major, a
    tenth of a cell left free on every side), so quads share no texels."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n_quads, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    c = d * rng.uniform(0.0, 1.0, size=(n_quads, 1)) ** (1.0 / 3.0) * np.asarray(radii)
    n = rng.normal(size=(n_quads, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    a = np.where(np.abs(n[:, :1]) < 0.9, np.array([[1.0, 0.0, 0.0]]), np.array([[0.0, 1.0, 0.0]]))
    t = np.cross(n, a)
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    b = np.cross(n, t)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=(n_quads, 1))
    t, b = np.cos(phi) * t + np.sin(phi) * b, -np.sin(phi) * t + np.cos(phi) * b
    h = rng.uniform(size[0], size[1], size=(n_quads, 1))
    corners = np.stack([c - h * t - h * b, c + h * t - h * b, c + h * t + h * b, c - h * t + h * b], axis=1)
    cells = int(np.ceil(np.sqrt(n_quads)))
    k = np.arange(n_quads)
    u0, v0 = (k % cells) / cells, (k // cells) / cells
    m, w = 0.1 / cells, 0.8 / cells
    uv = np.stack([np.stack([u0 + m, v0 + m], 1), np.stack([u0 + m + w, v0 + m], 1),
                   np.stack([u0 + m + w, v0 + m + w], 1), np.stack([u0 + m, v0 + m + w], 1)], axis=1)
    base = 4 * k[:, None]
    tri = np.concatenate([base + np.array([[0, 1, 2]]), base + np.array([[0, 2, 3]])], axis=1).reshape(-1, 3)
    return Mesh(np.ascontiguousarray(corners.reshape(-1, 3), dtype=np.float32),
                np.ascontiguousarray(uv.reshape(-1, 2), dtype=np.float32),
                np.ascontiguousarray(tri, dtype=np.int32), np.ascontiguousarray(tri, dtype=np.int32))


def config_aggregate(ref_tris=1_200_000, cand_tris=11_000, ref_tex_res=2048, tex_res=2048, aux_res=1024,
                     n_views=8, res=512, layers=8, seed=0):
    """Foliage workload: 11k candidate quad triangles against a 1.2M-triangle canopy.

    Reference: ref_tris / 2 opaque leaf quads (half-sides 0.015-0.03) with
    2048^2 procedural maps (seed 3) spread over the atlas. Candidate:
    cand_tris / 2 billboard quads (half-sides 0.08-0.16), a 2048^2 noise base
    colour whose opacity channel starts at 0.5, 1024^2 noise (gamma, r, m) and
    normal maps; positions, base colour with opacity, (gamma, r, m) and normals
    optimized. Eight random views at 512^2, squared-L2 loss, 8 peeling layers."""
    from .workloads import Scene

    rkd, rorm, rnrm = scenes.procedural_textures(ref_tex_res, seed=3)
    ref = Scene(mesh=quad_cloud(ref_tris // 2, seed + 11, size=(0.015, 0.03)), kd=rkd, orm=rorm, nrm=rnrm)
    kd, _ = scenes.noise_textures(tex_res, seed=seed)
    kd[..., 3] = 0.5
    _, nrm = scenes.noise_textures(aux_res, seed=seed + 1)
    cand = Scene(mesh=quad_cloud(cand_tris // 2, seed + 12, size=(0.08, 0.16)), kd=kd,
                 orm=scenes.uniform_orm(aux_res, seed=seed), nrm=nrm,
                 optimize={"pos": True, "kd": True, "orm": True, "nrm": True})
    return dict(ref=ref, cand=cand, loss="l2", n_views=n_views, res=res, layers=layers, fixed_view=False)
