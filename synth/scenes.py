"""Procedural meshes and textures (seeded, deterministic, numpy only).

Meshes are frequency-n geodesic icospheres (20 n^2 triangles, 10 n^2 + 2
vertices) with per-triangle equirectangular UV corners. They stand in for the
paper's scanned assets (sphere starts and high-poly references, Sec. 3 and
Sec. 4.1), which are not available here.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_PHI = (1.0 + 5.0 ** 0.5) / 2.0


@dataclass
class Mesh:
    """Indexed triangle mesh with a separate UV index buffer.

    pos:    (V, 3) float32 unique positions
    uv:     (T, 2) float32 UV corners (u wraps, v in [0, 1])
    tri_pos:(F, 3) int32 position indices, consistently wound outwards
    tri_uv: (F, 3) int32 UV-corner indices
    """

    pos: np.ndarray
    uv: np.ndarray
    tri_pos: np.ndarray
    tri_uv: np.ndarray

    @property
    def n_verts(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_tris(self) -> int:
        return int(self.tri_pos.shape[0])


def _icosahedron():
    v = np.array(
        [
            [-1, _PHI, 0], [1, _PHI, 0], [-1, -_PHI, 0], [1, -_PHI, 0],
            [0, -1, _PHI], [0, 1, _PHI], [0, -1, -_PHI], [0, 1, -_PHI],
            [_PHI, 0, -1], [_PHI, 0, 1], [-_PHI, 0, -1], [-_PHI, 0, 1],
        ],
        dtype=np.float64,
    )
    f = np.array(
        [
            [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
            [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
            [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
            [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
        ],
        dtype=np.int64,
    )
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    # A fixed tilt keeps every lattice point away from the UV poles (|y| = 1).
    ax, az = 0.31, 0.17
    rx = np.array([[1, 0, 0], [0, np.cos(ax), -np.sin(ax)], [0, np.sin(ax), np.cos(ax)]])
    rz = np.array([[np.cos(az), -np.sin(az), 0], [np.sin(az), np.cos(az), 0], [0, 0, 1]])
    v = v @ (rz @ rx).T
    return v, f


def icosphere(freq: int):
    """Frequency-`freq` geodesic icosphere on the unit sphere.

    Returns (pos float64 (V,3), tri int32 (F,3)) with F = 20 freq^2 and
    V = 10 freq^2 + 2, every triangle wound so that its normal points outwards.
    Lattice points shared between icosahedron faces are merged exactly through
    an integer key (base-vertex ids and integer barycentric weights).
    """
    n = int(freq)
    if n < 1:
        raise ValueError("freq must be >= 1")
    bv, bf = _icosahedron()
    ii, jj = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    keep = ii + jj <= n
    ii, jj = ii[keep], jj[keep]
    n_loc = ii.size
    loc_index = -np.ones((n + 1, n + 1), dtype=np.int64)
    loc_index[ii, jj] = np.arange(n_loc)

    ids = np.repeat(bf, n_loc, axis=0).reshape(20, n_loc, 3)
    w = np.stack([n - ii - jj, ii, jj], axis=1)[None].repeat(20, axis=0)
    # canonical key: (id, weight) pairs with weight > 0, sorted by id
    ids = np.where(w > 0, ids, 15)
    order = np.argsort(ids, axis=2, kind="stable")
    ids_s = np.take_along_axis(ids, order, axis=2)
    w_s = np.take_along_axis(np.where(w > 0, w, 0), order, axis=2)
    key = (
        ids_s[..., 0] | (ids_s[..., 1] << 4) | (ids_s[..., 2] << 8)
        | (w_s[..., 0] << 12) | (w_s[..., 1] << 21) | (w_s[..., 2] << 30)
    ).reshape(-1)
    ukey, first, inverse = np.unique(key, return_index=True, return_inverse=True)
    ids_u = ids_s.reshape(-1, 3)[first]
    w_u = w_s.reshape(-1, 3)[first].astype(np.float64)
    bv_pad = np.concatenate([bv, np.zeros((4, 3))], axis=0)  # id 15 -> zero row
    p = (w_u[:, :, None] * bv_pad[ids_u]).sum(axis=1) / n
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    gidx = inverse.reshape(20, n_loc)

    # two triangles per lattice cell
    tris = []
    for a in range(n):
        for b in range(n - a):
            tris.append((loc_index[a, b], loc_index[a + 1, b], loc_index[a, b + 1]))
            if a + b + 1 < n:
                tris.append((loc_index[a + 1, b], loc_index[a + 1, b + 1], loc_index[a, b + 1]))
    lt = np.asarray(tris, dtype=np.int64)
    tri = gidx[:, lt].reshape(-1, 3)
    # outward winding
    a, b, c = p[tri[:, 0]], p[tri[:, 1]], p[tri[:, 2]]
    flip = np.einsum("ij,ij->i", np.cross(b - a, c - a), a + b + c) < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]
    assert p.shape[0] == 10 * n * n + 2 and tri.shape[0] == 20 * n * n
    return p, tri.astype(np.int32)


def equirect_uv_corners(pos: np.ndarray, tri: np.ndarray):
    """Per-triangle-corner equirectangular UVs.

    u = atan2(z, x) / 2pi + 0.5 and v = acos(y) / pi. A triangle that straddles
    the u seam gets 1 added to its small u values (textures wrap in u). Returns
    (uv float32 (3F, 2), tri_uv int32 (F, 3)).
    """
    d = pos / np.linalg.norm(pos, axis=1, keepdims=True)
    u = np.arctan2(d[:, 2], d[:, 0]) / (2 * np.pi) + 0.5
    v = np.arccos(np.clip(d[:, 1], -1.0, 1.0)) / np.pi
    cu = u[tri]
    cv = v[tri]
    seam = cu.max(axis=1) - cu.min(axis=1) > 0.5
    cu = np.where(seam[:, None] & (cu < 0.5), cu + 1.0, cu)
    uv = np.stack([cu, cv], axis=2).reshape(-1, 2).astype(np.float32)
    tri_uv = np.arange(3 * tri.shape[0], dtype=np.int32).reshape(-1, 3)
    return uv, tri_uv


def _unit_vectors(rng, k):
    d = rng.normal(size=(k, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def radial_sinusoids(pos: np.ndarray, seed: int, n_terms: int = 8, amplitude: float = 0.05):
    """r = 1 + sum_k (amplitude / n_terms) sin(f_k (d_k . p) + phi_k), f in [2, 8]."""
    rng = np.random.default_rng(seed)
    d = _unit_vectors(rng, n_terms)
    f = rng.uniform(2.0, 8.0, size=n_terms)
    phi = rng.uniform(0.0, 2 * np.pi, size=n_terms)
    p = pos / np.linalg.norm(pos, axis=1, keepdims=True)
    r = 1.0 + (amplitude / n_terms) * np.sin(f[None] * (p @ d.T) + phi[None]).sum(axis=1)
    return p * r[:, None]


def _splitmix64(x):
    with np.errstate(over="ignore"):
        x = (x + np.uint64(0x9E3779B97F4A7C15)) & np.uint64(0xFFFFFFFFFFFFFFFF)
        z = x
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & np.uint64(0xFFFFFFFFFFFFFFFF)
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & np.uint64(0xFFFFFFFFFFFFFFFF)
        return z ^ (z >> np.uint64(31))


def _lattice_value(ix, iy, iz, salt):
    with np.errstate(over="ignore"):
        h = (
            ix.astype(np.int64).astype(np.uint64) * np.uint64(0x8DA6B343)
            ^ iy.astype(np.int64).astype(np.uint64) * np.uint64(0xD8163841)
            ^ iz.astype(np.int64).astype(np.uint64) * np.uint64(0xCB1AB31F)
            ^ np.uint64(salt)
        )
        h = _splitmix64(h)
    return (h >> np.uint64(11)).astype(np.float64) / float(1 << 53) * 2.0 - 1.0


def _value_noise3(x, salt):
    i = np.floor(x).astype(np.int64)
    f = x - i
    s = f * f * (3.0 - 2.0 * f)
    out = 0.0
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                w = (
                    (s[:, 0] if dx else 1 - s[:, 0])
                    * (s[:, 1] if dy else 1 - s[:, 1])
                    * (s[:, 2] if dz else 1 - s[:, 2])
                )
                out = out + w * _lattice_value(i[:, 0] + dx, i[:, 1] + dy, i[:, 2] + dz, salt)
    return out


def fbm3(p, seed, octaves=4, base_freq=2.0, lacunarity=2.0, gain=0.5):
    """Value-noise fBm in [-1, 1] (lattice values hashed with splitmix64)."""
    total, amp, norm = 0.0, 1.0, 0.0
    for o in range(octaves):
        salt = int(_splitmix64(np.uint64(seed * 1000 + o)))
        total = total + amp * _value_noise3(p * (base_freq * lacunarity ** o), salt)
        norm += amp
        amp *= gain
    return total / norm


def radial_fbm(pos: np.ndarray, seed: int, amplitude: float = 0.05, octaves: int = 4):
    p = pos / np.linalg.norm(pos, axis=1, keepdims=True)
    r = 1.0 + amplitude * fbm3(p, seed, octaves=octaves)
    return p * r[:, None]


def _value_noise2_periodic(u, v, cells_u, cells_v, salt):
    x = u * cells_u
    y = v * cells_v
    ix = np.floor(x).astype(np.int64)
    iy = np.floor(y).astype(np.int64)
    fx, fy = x - ix, y - iy
    sx, sy = fx * fx * (3 - 2 * fx), fy * fy * (3 - 2 * fy)
    z = np.zeros_like(ix)
    out = 0.0
    for dx in (0, 1):
        for dy in (0, 1):
            w = (sx if dx else 1 - sx) * (sy if dy else 1 - sy)
            out = out + w * _lattice_value((ix + dx) % cells_u, iy + dy, z, salt)
    return out


def _fbm2(u, v, seed, octaves=4, cells=8):
    total, amp, norm = 0.0, 1.0, 0.0
    for o in range(octaves):
        c = cells * (2 ** o)
        salt = int(_splitmix64(np.uint64(seed * 1000 + 17 + o)))
        total = total + amp * _value_noise2_periodic(u, v, c, c // 2, salt)
        norm += amp
        amp *= 0.5
    return total / norm


def noise_textures(res: int, seed: int = 0):
    """Uniform-noise initial guesses (the paper starts from random maps, Sec. 3).

    Returns (kd (res,res,4) ~ U[0,1], normal (res,res,4) with xy ~ U[-1,1],
    z ~ U[0,1], w = 0), float32, rows = v, columns = u.
    """
    rng = np.random.default_rng(seed)
    kd = rng.uniform(0.0, 1.0, size=(res, res, 4)).astype(np.float32)
    nrm = np.zeros((res, res, 4), dtype=np.float32)
    nrm[..., 0:2] = rng.uniform(-1.0, 1.0, size=(res, res, 2))
    nrm[..., 2] = rng.uniform(0.0, 1.0, size=(res, res))
    return kd, nrm


def uniform_orm(res: int, seed: int):
    """Uniform-noise (gamma, r, m) map: gamma, m in [0, 1], r in [0.08, 1]."""
    rng = np.random.default_rng(seed + 7919)
    orm = np.zeros((res, res, 4), dtype=np.float32)
    orm[..., 0] = rng.uniform(0.0, 1.0, size=(res, res))
    orm[..., 1] = rng.uniform(0.08, 1.0, size=(res, res))
    orm[..., 2] = rng.uniform(0.0, 1.0, size=(res, res))
    return orm


def procedural_textures(res: int, seed: int):
    """Seeded fBm base-colour, (gamma, r, m) and tangent-space normal maps.

    All maps are (res, res, 4) float32, periodic in u so they wrap seamlessly.
    """
    u = (np.arange(res) + 0.5) / res
    v = (np.arange(res) + 0.5) / res
    uu, vv = np.meshgrid(u, v)
    uu, vv = uu.reshape(-1), vv.reshape(-1)
    a = _fbm2(uu, vv, seed)
    b = _fbm2(uu, vv, seed + 1)
    h = _fbm2(uu, vv, seed + 2, octaves=4, cells=16)
    c0 = np.array([0.75, 0.45, 0.25])
    c1 = np.array([0.15, 0.35, 0.60])
    t = np.clip(0.5 + 0.8 * a, 0.0, 1.0)[:, None]
    kd = np.concatenate([c0 * (1 - t) + c1 * t, np.ones((uu.size, 1))], axis=1)
    orm = np.stack(
        [np.zeros_like(a), np.clip(0.45 + 0.4 * b, 0.08, 1.0), np.clip(2.0 * b, 0.0, 1.0), np.zeros_like(a)],
        axis=1,
    )
    hh = h.reshape(res, res)
    gx = (np.roll(hh, -1, axis=1) - np.roll(hh, 1, axis=1)) * (res / 64.0)
    gy = np.zeros_like(hh)
    gy[1:-1] = (hh[2:] - hh[:-2]) * (res / 64.0)
    nz = np.ones_like(hh)
    nrm = np.stack([-gx, -gy, nz], axis=2)
    nrm /= np.linalg.norm(nrm, axis=2, keepdims=True)
    nrm = np.concatenate([nrm, np.zeros((res, res, 1))], axis=2)
    f32 = lambda x: np.ascontiguousarray(x.reshape(res, res, 4), dtype=np.float32)  # noqa: E731
    return f32(kd), f32(orm), f32(nrm)


def constant_texture(value, res: int = 1):
    v = np.zeros(4, dtype=np.float32)
    v[: len(value)] = value
    return np.ascontiguousarray(np.broadcast_to(v, (res, res, 4)), dtype=np.float32)
