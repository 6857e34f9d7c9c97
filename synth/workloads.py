"""Workload recipes: candidate/reference scenes sized like the paper's runs.

The paper optimizes sphere or decimated starts of 0.5k-18k triangles against
references of 81k-1.7M triangles, with 2048^2 textures and batches of 1-8
views (Sec. 5.3, Sec. 4.1, supplemental triangle sweeps). Its scanned assets
are not available, so these seeded procedural scenes stand in for them.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import scenes
from .scenes import Mesh


@dataclass
class Scene:
    mesh: Mesh
    kd: np.ndarray                 # (H, W, 4) float32 base colour (+alpha)
    orm: np.ndarray                # (H, W, 4) float32 (gamma, r, m, pad)
    nrm: np.ndarray                # (H, W, 4) float32 tangent-space normal (x, y, z, pad)
    disp: np.ndarray | None = None  # (H, W) float32 scalar displacement (tessellated scenes)
    tess_levels: int = 0
    mips: bool = True
    optimize: dict = field(default_factory=dict)  # which parameters are latent


def _mesh(freq, displace=None):
    p, tri = scenes.icosphere(freq)
    uv, tri_uv = scenes.equirect_uv_corners(p, tri)
    if displace is not None:
        p = displace(p)
    return Mesh(np.ascontiguousarray(p, dtype=np.float32), uv, tri, tri_uv)


def config_small():
    """One-step workload: 320-tri candidate vs a 20,480-tri reference, 256^2 view.

    Reference: frequency-32 icosphere displaced radially by 8 seeded sinusoids
    (amplitude 0.05, seed 1), constant albedo 0.7, roughness 0.5. Candidate:
    frequency-4 icosphere, 256^2 noise base-colour and normal maps (seed 0),
    fixed (gamma, r, m) = (0, 0.5, 0). Plain L1 loss, one directional light.
    """
    ref = Scene(
        mesh=_mesh(32, lambda p: scenes.radial_sinusoids(p, seed=1)),
        kd=scenes.constant_texture((0.7, 0.7, 0.7, 1.0)),
        orm=scenes.constant_texture((0.0, 0.5, 0.0)),
        nrm=scenes.constant_texture((0.0, 0.0, 1.0)),
    )
    kd, nrm = scenes.noise_textures(256, seed=0)
    cand = Scene(
        mesh=_mesh(4),
        kd=kd,
        orm=scenes.constant_texture((0.0, 0.5, 0.0)),
        nrm=nrm,
        optimize={"pos": True, "kd": True, "orm": False, "nrm": True},
    )
    return dict(ref=ref, cand=cand, loss="l1", n_views=1, res=256, fixed_view=True)


def config_plain(tex_res=1024, ref_tex_res=2048, ref_freq=100, cand_freq=16, n_views=8, res=512):
    """Batched-view workload: 5,120-tri candidate vs a 200k-tri reference.

    Reference: frequency-100 icosphere with 4-octave fBm radial displacement
    (seed 2) and 2048^2 procedural maps (seed 3). Candidate: frequency-16
    icosphere with 1024^2 noise maps and full mip chains (seed 0). Eight random
    views at 512^2 with one point and one directional light; tone-mapped
    log-L1 loss.
    """
    rkd, rorm, rnrm = scenes.procedural_textures(ref_tex_res, seed=3)
    ref = Scene(mesh=_mesh(ref_freq, lambda p: scenes.radial_fbm(p, seed=2)), kd=rkd, orm=rorm, nrm=rnrm)
    kd, nrm = scenes.noise_textures(tex_res, seed=0)
    cand = Scene(
        mesh=_mesh(cand_freq),
        kd=kd,
        orm=scenes.uniform_orm(tex_res, seed=0),
        nrm=nrm,
        optimize={"pos": True, "kd": True, "orm": True, "nrm": True},
    )
    return dict(ref=ref, cand=cand, loss="logl1", n_views=n_views, res=res, fixed_view=False)


def config_tess(ref_freq=224, base_freq=7, levels=3, disp_res=1024, nrm_res=2048, n_views=16, res=1024):
    """Displacement workload: 980-tri base mesh tessellated 3 times (62,720 tris).

    Latents: base positions, a 1024^2 scalar displacement map (zero start) and a
    2048^2 normal map (noise start); base colour and (gamma, r, m) are constant
    and diffuse-dominated. Reference: frequency-224 icosphere (1,003,520 tris)
    with fBm displacement.
    """
    ref = Scene(
        mesh=_mesh(ref_freq, lambda p: scenes.radial_fbm(p, seed=4, amplitude=0.06)),
        kd=scenes.constant_texture((0.7, 0.7, 0.7, 1.0)),
        orm=scenes.constant_texture((0.5, 0.7, 0.0)),
        nrm=scenes.constant_texture((0.0, 0.0, 1.0)),
    )
    _, nrm = scenes.noise_textures(nrm_res, seed=0)
    cand = Scene(
        mesh=_mesh(base_freq),
        kd=scenes.constant_texture((0.7, 0.7, 0.7, 1.0)),
        orm=scenes.constant_texture((0.5, 0.7, 0.0)),
        nrm=nrm,
        disp=np.zeros((disp_res, disp_res), dtype=np.float32),
        tess_levels=levels,
        optimize={"pos": True, "kd": False, "orm": False, "nrm": True, "disp": True},
    )
    return dict(ref=ref, cand=cand, loss="logl1", n_views=n_views, res=res, fixed_view=False)


def job_mix(n_jobs=64, seed=0, tri_range=(500, 20000), tex_choices=(256, 512, 1024, 2048),
            res_choices=(256, 512, 1024), view_range=(4, 16)):
    """Uneven job descriptors: candidate frequency, texture size, views, resolution.

    Candidate triangle counts are log-uniform on `tri_range` (rounded to the
    nearest geodesic frequency n = round(sqrt(T / 20))); references carry 10x
    their candidate's triangles. Returns a list of dicts (recipes, not arrays).
    """
    rng = np.random.default_rng(seed)
    jobs = []
    for j in range(n_jobs):
        t = float(np.exp(rng.uniform(np.log(tri_range[0]), np.log(tri_range[1]))))
        n = max(1, int(round((t / 20.0) ** 0.5)))
        nr = max(1, int(round((10 * 20 * n * n / 20.0) ** 0.5)))
        jobs.append(
            dict(
                job=j,
                cand_freq=n,
                ref_freq=nr,
                tex_res=int(rng.choice(tex_choices)),
                n_views=int(rng.integers(view_range[0], view_range[1] + 1)),
                res=int(rng.choice(res_choices)),
                seed=j,
            )
        )
    return jobs


_REF_MAPS = {}


def job_scenes(recipe, ref_tex_cap=1024):
    """(candidate, reference) scenes of one job_mix recipe.

    Candidate: frequency-`cand_freq` icosphere with `tex_res`^2 noise maps and
    full mip chains, every latent optimized. Reference: frequency-`ref_freq`
    icosphere with 4-octave fBm radial displacement seeded by the job, and
    procedural maps at min(tex_res, ref_tex_cap)^2 (seed 3) shared by all
    jobs of that size: the maps only feed frozen reference renders, and the
    host-side generator costs seconds per 2048^2 set.
    """
    r = recipe
    rt = min(r["tex_res"], ref_tex_cap)
    if rt not in _REF_MAPS:
        _REF_MAPS[rt] = scenes.procedural_textures(rt, seed=3)
    rkd, rorm, rnrm = _REF_MAPS[rt]
    ref = Scene(mesh=_mesh(r["ref_freq"], lambda p: scenes.radial_fbm(p, seed=1000 + r["seed"])),
                kd=rkd, orm=rorm, nrm=rnrm)
    kd, nrm = scenes.noise_textures(r["tex_res"], seed=r["seed"])
    cand = Scene(mesh=_mesh(r["cand_freq"]), kd=kd, orm=scenes.uniform_orm(r["tex_res"], seed=r["seed"]), nrm=nrm,
                 optimize={"pos": True, "kd": True, "orm": True, "nrm": True})
    return cand, ref
