"""Pins of the oracle's visibility (raster.c) against closed forms and brute force.

The brute-force reference below tests every pixel against every triangle with
a per-pixel edge test written independently of the oracle's per-row interval
solver (scanline)."""

import numpy as np
import pytest

import synth
from oracle import visibility as V

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


def raster_xy(XY, z, tri, W, H):
    """Call the oracle rasterizer on given snapped sub-pixel coordinates."""
    lib = V._load()
    XY = np.ascontiguousarray(XY, dtype=np.int32)
    z = np.ascontiguousarray(z, dtype=np.float32)
    ok = np.ones(len(z), np.int8)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    keys = np.full((H, W), EMPTY, dtype=np.uint64)
    asign = np.zeros(len(tri), np.int8)
    lib.oracle_raster(V._ptr(XY), V._ptr(z), V._ptr(ok), V._ptr(tri), len(tri), W, H, V._ptr(keys), V._ptr(asign))
    return keys, asign


def brute_force(XY, z, tri, W, H):
    """Every pixel x every triangle; per-pixel inside test with the top-left rule."""
    keys = np.full((H, W), EMPTY, dtype=np.uint64)
    jj, ii = np.meshgrid(np.arange(H, dtype=np.int64), np.arange(W, dtype=np.int64), indexing="ij")
    Sx, Sy = 256 * ii + 128, 256 * jj + 128
    for f, (a, b, c) in enumerate(tri):
        P = [XY[a].astype(np.int64), XY[b].astype(np.int64), XY[c].astype(np.int64)]
        area = (P[1][0] - P[0][0]) * (P[2][1] - P[0][1]) - (P[1][1] - P[0][1]) * (P[2][0] - P[0][0])
        if area == 0:
            continue
        Q = P if area > 0 else [P[0], P[2], P[1]]
        inside = np.ones((H, W), bool)
        for k in range(3):
            A, B = Q[(k + 1) % 3], Q[(k + 2) % 3]
            dx, dy = B[0] - A[0], B[1] - A[1]
            E = dx * (Sy - A[1]) - dy * (Sx - A[0])
            tl = dy < 0 or (dy == 0 and dx > 0)
            inside &= (E > 0) | ((E == 0) & tl)
        e20 = (P[0][0] - P[2][0]) * (Sy - P[2][1]) - (P[0][1] - P[2][1]) * (Sx - P[2][0])
        e01 = (P[1][0] - P[0][0]) * (Sy - P[0][1]) - (P[1][1] - P[0][1]) * (Sx - P[0][0])
        fa = np.float32(area)
        b1 = e20.astype(np.float32) / fa
        b2 = e01.astype(np.float32) / fa
        z0, z1, z2 = np.float32(z[a]), np.float32(z[b]), np.float32(z[c])
        d = (z0 + b1 * (z1 - z0)) + b2 * (z2 - z0)
        d = d.astype(np.float32)
        inside &= (d >= 0) & (d <= 1)
        d = np.where(d == 0, np.float32(0), d).astype(np.float32)
        key = (d.view(np.uint32).astype(np.uint64) << np.uint64(32)) | np.uint64(f)
        keys = np.where(inside & (key < keys), key, keys)
    return keys


def quad_tris(x0, y0, x1, y1, base=0):
    XY = np.array([[x0, y0], [x1, y0], [x1, y1], [x0, y1]], dtype=np.int32)
    tri = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32) + base
    return XY, tri


@pytest.mark.parametrize("k", [1, 2, 3, 7, 16])
@pytest.mark.parametrize("wind", [1, -1])
def test_axis_aligned_quad_covers_k_squared(k, wind):
    # corners on pixel-centre lines: x = 256 i + 128
    W = H = 32
    i0, j0 = 5, 3
    XY, tri = quad_tris(256 * i0 + 128, 256 * j0 + 128, 256 * (i0 + k) + 128, 256 * (j0 + k) + 128)
    if wind < 0:
        tri = tri[:, [0, 2, 1]]
    keys, _ = raster_xy(XY, np.full(4, 0.5), tri, W, H)
    cov = keys != EMPTY
    assert cov.sum() == k * k
    assert cov[j0:j0 + k, i0:i0 + k].all()


def test_shared_edges_partition_exactly():
    """Two quads sharing an edge and the two triangles of each quad (sharing a
    diagonal) cover every pixel of the union exactly once."""
    W = H = 24
    rng = np.random.default_rng(0)
    for _ in range(50):
        xs = np.sort(rng.integers(0, 256 * W, size=3))
        ys = np.sort(rng.integers(0, 256 * H, size=2))
        XYa, ta = quad_tris(xs[0], ys[0], xs[1], ys[1])
        XYb, tb = quad_tris(xs[1], ys[0], xs[2], ys[1], base=4)
        XY = np.concatenate([XYa, XYb])
        tris = np.concatenate([ta, tb])
        count = np.zeros((H, W), int)
        for f in range(4):
            keys, _ = raster_xy(XY, np.full(8, 0.5), tris[f:f + 1], W, H)
            count += keys != EMPTY
        assert count.max() <= 1
        # union = samples with x in [xs0, xs2) and y in [ys0, ys1) (left/top inclusive)
        S = 256 * np.arange(W) + 128
        T = 256 * np.arange(H) + 128
        want = ((T >= ys[0]) & (T < ys[1]))[:, None] & ((S >= xs[0]) & (S < xs[2]))[None, :]
        np.testing.assert_array_equal(count == 1, want)


def test_fan_around_vertex_covers_once():
    """Triangles fanned around a shared vertex tile the disc without overlap."""
    W = H = 40
    c = np.array([256 * 20 + 128, 256 * 20 + 128])
    rng = np.random.default_rng(1)
    n = 9
    ang = np.sort(rng.uniform(0, 2 * np.pi, n))
    rim = np.stack([c[0] + 4000 * np.cos(ang), c[1] + 4000 * np.sin(ang)], axis=1).round().astype(np.int32)
    XY = np.concatenate([c[None].astype(np.int32), rim])
    tris = np.array([[0, 1 + i, 1 + (i + 1) % n] for i in range(n)], dtype=np.int32)
    count = np.zeros((H, W), int)
    for f in range(n):
        keys, _ = raster_xy(XY, np.full(n + 1, 0.5), tris[f:f + 1], W, H)
        count += keys != EMPTY
    assert count.max() == 1
    assert count[20, 20] == 1


@pytest.mark.parametrize("seed", range(6))
def test_random_scenes_match_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    W, H = 37, 29
    F = int(rng.integers(1, 51))
    XY = np.stack([rng.integers(-2000, 256 * W + 2000, 3 * F), rng.integers(-2000, 256 * H + 2000, 3 * F)],
                  axis=1).astype(np.int32)
    if seed % 2 == 0:  # snap some vertices onto sample lines to exercise ties
        XY[::3] = (XY[::3] // 256) * 256 + 128
    z = rng.uniform(-0.2, 1.2, 3 * F).astype(np.float32)
    if seed == 4:
        z[:] = 0.25  # equal depths: lower id must win
    tri = np.arange(3 * F, dtype=np.int32).reshape(F, 3)
    got, _ = raster_xy(XY, z, tri, W, H)
    want = brute_force(XY, z, tri, W, H)
    np.testing.assert_array_equal(got, want)


def test_coplanar_tie_lower_id_wins():
    W = H = 16
    XY, tri = quad_tris(0, 0, 256 * 16, 256 * 16)
    XY = np.concatenate([XY, XY])
    tri = np.concatenate([tri[:1], tri[:1] + 4])  # the same triangle twice
    keys, _ = raster_xy(XY, np.full(8, 0.3), tri, W, H)
    ids = (keys[keys != EMPTY] & np.uint64(0xFFFFFFFF))
    assert ids.size > 0 and (ids == 0).all()


def test_transform_projects_origin_to_centre_and_snaps():
    view = synth.fixed_view(64, 48)[0]
    pos = np.array([[0, 0, 0], [0, 0, 1.0], [0.25, -0.125, 0.0]], dtype=np.float32)
    t = V.transform(view["mvp"], pos, 64, 48)
    assert t["ok"].all()
    assert tuple(t["XY"][0]) == (32 * 256, 24 * 256)
    assert tuple(t["XY"][1]) == (32 * 256, 24 * 256)
    # float64 projection of the third point agrees with the snap to 1/256 px
    M = view["mvp"].astype(np.float64).reshape(4, 4)
    c = M @ np.array([0.25, -0.125, 0.0, 1.0])
    sx = (c[0] / c[3]) * 32 + 32
    sy = 24 - (c[1] / c[3]) * 24
    assert abs(t["XY"][2][0] - sx * 256) <= 0.5 + 1e-3
    assert abs(t["XY"][2][1] - sy * 256) <= 0.5 + 1e-3
    # depth maps near -> 0, far -> 1 monotonically
    assert 0 < t["z01"][0] < t["z01"][1] < 1 or 0 < t["z01"][1] < t["z01"][0] < 1


def test_behind_camera_is_culled():
    view = synth.fixed_view(32, 32)[0]
    pos = np.array([[0, 0, 4.0], [1, 0, 4.0], [0, 1, 4.0]], dtype=np.float32)  # behind the eye at z=3
    keys, asign, t = V.raster(view["mvp"], pos, np.array([[0, 1, 2]]), 32, 32)
    assert not t["ok"].any()
    assert (keys == EMPTY).all() and asign[0] == 0


def test_sphere_silhouette_coverage_matches_disc_area():
    """A unit sphere at distance 3 covers about the area of its projected disc."""
    p, tri = synth.icosphere(16)
    W = H = 256
    view = synth.fixed_view(W, H)[0]
    keys, _, _ = V.raster(view["mvp"], p.astype(np.float32), tri, W, H)
    cov = (keys != EMPTY).sum()
    # projected radius in pixels: tan(asin(1/3)) / tan(22.5 deg) * H/2
    r_px = np.tan(np.arcsin(1 / 3)) / np.tan(np.radians(22.5)) * (H / 2)
    disc = np.pi * r_px ** 2
    assert abs(cov - disc) / disc < 0.03
