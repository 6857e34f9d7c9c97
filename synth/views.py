"""Random cameras and lights (the paper's "virtual photo-goniometer", Sec. 3).

Each view is a packed record matching the C struct `adms_view`: a row-major
fp32 MVP matrix (clip = MVP [x y z 1]^T, OpenGL conventions), the eye
position, one point light (position, intensity) and one directional light
(unit vector towards the light, irradiance). The matrix is built in float64
and rounded once to float32; both the oracle and the CUDA path consume that
float32 matrix as data.
"""

from __future__ import annotations

import numpy as np

VIEW_DTYPE = np.dtype(
    [
        ("mvp", np.float32, (16,)),
        ("eye", np.float32, (3,)),
        ("pad0", np.float32),
        ("light_pos", np.float32, (3,)),
        ("light_I", np.float32),
        ("light_dir", np.float32, (3,)),
        ("light_E", np.float32),
    ]
)
assert VIEW_DTYPE.itemsize == 112

FOVY_DEG = 45.0
NEAR = 0.1
FAR = 100.0


def look_at(eye, target=(0.0, 0.0, 0.0)):
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    up = np.array([0.0, 1.0, 0.0])
    if abs(f @ up) > 0.999:
        up = np.array([0.0, 0.0, 1.0])
    s = np.cross(f, up)
    s /= np.linalg.norm(s)
    u = np.cross(s, f)
    m = np.eye(4)
    m[0, :3], m[1, :3], m[2, :3] = s, u, -f
    m[:3, 3] = -m[:3, :3] @ eye
    return m


def perspective(fovy_deg=FOVY_DEG, aspect=1.0, near=NEAR, far=FAR):
    f = 1.0 / np.tan(np.radians(fovy_deg) / 2.0)
    m = np.zeros((4, 4))
    m[0, 0] = f / aspect
    m[1, 1] = f
    m[2, 2] = (far + near) / (near - far)
    m[2, 3] = 2.0 * far * near / (near - far)
    m[3, 2] = -1.0
    return m


def make_view(eye, width, height, light_pos=(0, 0, 0), light_I=0.0, light_dir=(0, 0, 1), light_E=0.0):
    rec = np.zeros((), dtype=VIEW_DTYPE)
    mvp = perspective(aspect=width / height) @ look_at(eye)
    rec["mvp"] = mvp.reshape(-1).astype(np.float32)
    rec["eye"] = np.asarray(eye, dtype=np.float32)
    rec["light_pos"] = np.asarray(light_pos, dtype=np.float32)
    rec["light_I"] = np.float32(light_I)
    d = np.asarray(light_dir, dtype=np.float64)
    rec["light_dir"] = (d / np.linalg.norm(d)).astype(np.float32)
    rec["light_E"] = np.float32(light_E)
    return rec


def fixed_view(width, height, eye=(0.0, 0.0, 3.0), light_dir=(1.0, 1.0, 1.0), light_E=3.0):
    """One camera on +z looking at the origin, one directional light."""
    out = np.zeros(1, dtype=VIEW_DTYPE)
    out[0] = make_view(eye, width, height, light_dir=light_dir, light_E=light_E)
    return out


def _unit(rng):
    d = rng.normal(size=3)
    return d / np.linalg.norm(d)


def sample_views(seed, iteration, n_views, width, height, r_min=2.5, r_max=4.0,
                 point_radius=4.0, point_I=20.0, dir_E=1.0):
    """Random views keyed by (seed, iteration, view index).

    Eye uniform on the sphere of radius U[r_min, r_max], looking at the origin;
    one point light uniform on the sphere of radius `point_radius` with
    intensity `point_I`; one directional light with a uniform direction and
    irradiance `dir_E`. The key makes each job's cameras independent of which
    other jobs share its batch.
    """
    out = np.zeros(n_views, dtype=VIEW_DTYPE)
    for k in range(n_views):
        rng = np.random.default_rng([int(seed), int(iteration), int(k)])
        eye = _unit(rng) * rng.uniform(r_min, r_max)
        lp = _unit(rng) * point_radius
        ld = _unit(rng)
        out[k] = make_view(eye, width, height, light_pos=lp, light_I=point_I, light_dir=ld, light_E=dir_E)
    return out
