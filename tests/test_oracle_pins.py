"""Pins of the float64 oracle against closed forms, invariants and finite differences.

Each test fixes a property that the paper or the mathematics determines
independently of the oracle's code, so that a dropped term, a wrong sign or a
swapped operand in the oracle fails at least one of them."""

import math

import numpy as np
import pytest
import torch

import synth
from oracle import render as R
from oracle import skinning as SK
from oracle import step as S
from oracle import visibility as V
from oracle import tessellate as TS

F64 = torch.float64


# ----------------------------------------------------------------------------- barycentrics

def _random_tri_view(seed):
    rng = np.random.default_rng(seed)
    view = synth.sample_views(seed, 0, 1, 64, 64)[0]
    P = torch.as_tensor(rng.uniform(-0.7, 0.7, size=(3, 3)))
    M = torch.as_tensor(view["mvp"].astype(np.float64).reshape(4, 4))
    clip = torch.cat([P, torch.ones(3, 1, dtype=F64)], 1) @ M.T
    scr = R.screen_coords(clip, 64, 64)
    return P, M, clip, scr


@pytest.mark.parametrize("seed", range(5))
def test_barycentrics_sum_to_one_and_reproject(seed):
    P, M, clip, scr = _random_tri_view(seed)
    rng = np.random.default_rng(seed + 10)
    # points inside the screen triangle
    a = rng.dirichlet([1, 1, 1], size=200)
    q = torch.as_tensor(a) @ scr
    s = [scr[k].expand(200, 2) for k in range(3)]
    w = [clip[k, 3].expand(200) for k in range(3)]
    beta, _ = R.perspective_barycentrics(s, w, q)
    b = torch.stack(beta, 1)
    assert torch.allclose(b.sum(1), torch.ones(200, dtype=F64), atol=1e-12)
    # the interpolated 3D point projects back onto the pixel (perspective correctness)
    p = b @ P
    c = torch.cat([p, torch.ones(200, 1, dtype=F64)], 1) @ M.T
    back = R.screen_coords(c, 64, 64)
    assert torch.allclose(back, q, atol=1e-9)


def test_barycentrics_at_vertices_are_unit_vectors():
    P, M, clip, scr = _random_tri_view(3)
    s = [scr[k].expand(3, 2) for k in range(3)]
    w = [clip[k, 3].expand(3) for k in range(3)]
    beta, _ = R.perspective_barycentrics(s, w, scr)
    assert torch.allclose(torch.stack(beta, 1), torch.eye(3, dtype=F64), atol=1e-12)


def test_barycentric_derivatives_match_differences():
    P, M, clip, scr = _random_tri_view(7)
    q = scr.mean(0, keepdim=True)
    s = [scr[k][None] for k in range(3)]
    w = [clip[k, 3][None] for k in range(3)]
    _, db = R.perspective_barycentrics(s, w, q)
    h = 1e-5
    for axis in (0, 1):
        e = torch.zeros(1, 2, dtype=F64)
        e[0, axis] = h
        bp, _ = R.perspective_barycentrics(s, w, q + e)
        bm, _ = R.perspective_barycentrics(s, w, q - e)
        for k in range(3):
            fd = (bp[k] - bm[k]) / (2 * h)
            assert abs(float(fd - db[axis][k])) < 1e-7


# ----------------------------------------------------------------------------- textures

def test_constant_texture_is_exact():
    tex = torch.full((8, 8, 4), 0.3125, dtype=F64)
    lv = R.mip_chain(tex)
    assert len(lv) == 4
    rng = np.random.default_rng(0)
    u = torch.as_tensor(rng.uniform(-2, 3, 500))
    v = torch.as_tensor(rng.uniform(-0.5, 1.5, 500))
    lod = torch.as_tensor(rng.uniform(0, 3, 500))
    out = R.trilinear(lv, u, v, lod)
    assert torch.allclose(out, torch.full_like(out, 0.3125), rtol=0, atol=4e-16)


def test_bilinear_at_texel_centres_returns_texels():
    rng = np.random.default_rng(1)
    tex = torch.as_tensor(rng.uniform(size=(16, 8, 4)))
    ys, xs = np.meshgrid(np.arange(16), np.arange(8), indexing="ij")
    u = torch.as_tensor((xs.reshape(-1) + 0.5) / 8)
    v = torch.as_tensor((ys.reshape(-1) + 0.5) / 16)
    out = R.bilinear(tex, u, v)
    assert torch.allclose(out, tex.reshape(-1, 4), atol=1e-14)
    # u wraps: u + 1 samples the same texel
    assert torch.allclose(R.bilinear(tex, u + 1.0, v), out, atol=1e-12)


def test_mip_of_linear_ramp_is_exact():
    n = 32
    ys, xs = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5, indexing="ij")
    ramp = 0.25 * xs - 0.125 * ys + 1.0
    tex = torch.as_tensor(np.repeat(ramp[:, :, None], 4, axis=2))
    for k, lv in enumerate(R.mip_chain(tex)):
        m = n >> k
        yk, xk = np.meshgrid((np.arange(m) + 0.5) * (n / m), (np.arange(m) + 0.5) * (n / m), indexing="ij")
        want = 0.25 * xk - 0.125 * yk + 1.0
        assert np.allclose(lv[..., 0].numpy(), want, atol=1e-12)


def test_trilinear_blends_adjacent_levels():
    rng = np.random.default_rng(2)
    lv = R.mip_chain(torch.as_tensor(rng.uniform(size=(16, 16, 4))))
    u = torch.as_tensor([0.3]), torch.as_tensor([0.6])
    for lod in (0.0, 1.0, 1.25, 2.5, 4.0):
        k = int(math.floor(lod))
        f = lod - k
        want = (1 - f) * R.bilinear(lv[k], *u) + (f * R.bilinear(lv[min(k + 1, 4)], *u) if f > 0 else 0)
        got = R.trilinear(lv, u[0], u[1], torch.as_tensor([lod]))
        assert torch.allclose(got, want, atol=1e-14)


def test_lod_of_uniform_minification():
    # du/dx = s / W texels per pixel along x, nothing along y -> lod = log2 s
    for s_ in (0.5, 1.0, 3.0, 8.0):
        dx = torch.as_tensor([[s_ / 64, 0.0]], dtype=F64)
        dy = torch.as_tensor([[0.0, 0.5 / 64]], dtype=F64)
        lod = R.texture_lod(dx, dy, 64, 64, 7)
        assert abs(float(lod) - max(0.0, math.log2(s_))) < 1e-12


# ----------------------------------------------------------------------------- shading

def _view(**kw):
    v = synth.fixed_view(8, 8)[0].copy()
    for k, x in kw.items():
        v[k] = x
    return v


def _flat_inputs(n, kd, orm, normal=(0.0, 0.0, 1.0)):
    p = torch.zeros(n, 3, dtype=F64)
    nn = torch.as_tensor(np.tile([0.0, 0.0, 1.0], (n, 1)))
    tt = torch.as_tensor(np.tile([1.0, 0.0, 0.0], (n, 1)))
    kd_ = torch.as_tensor(np.tile(kd, (n, 1)))
    orm_ = torch.as_tensor(np.tile(orm, (n, 1)))
    nm = torch.as_tensor(np.tile(normal, (n, 1)))
    return p, nn, tt, kd_, orm_, nm


@pytest.mark.parametrize("theta_deg", [0.0, 30.0, 60.0, 89.0])
def test_lambertian_plane_radiance(theta_deg):
    """gamma = 1 removes the specular lobe and m = 0 leaves L = kd / pi E cos(theta)."""
    th = math.radians(theta_deg)
    l = np.array([math.sin(th), 0.0, math.cos(th)])
    view = _view(light_dir=l.astype(np.float32), light_E=np.float32(2.5), light_I=np.float32(0.0))
    kd = [0.2, 0.5, 0.8, 1.0]
    inp = _flat_inputs(4, kd, [1.0, 0.5, 0.0, 0.0])
    col = R.shade(*inp, view)
    ldir = view["light_dir"].astype(np.float64)
    want = np.array(kd[:3]) / math.pi * 2.5 * ldir[2]
    assert np.allclose(col.numpy(), want[None], atol=1e-12)


def test_point_light_inverse_square():
    view = _view(light_pos=np.array([0, 0, 2.0], np.float32), light_I=np.float32(8.0), light_E=np.float32(0.0))
    inp = _flat_inputs(1, [0.6, 0.6, 0.6, 1], [1.0, 0.5, 0.0, 0.0])
    col = R.shade(*inp, view)
    assert np.allclose(col.numpy(), 0.6 / math.pi * 8.0 / 4.0, atol=1e-12)


def test_light_below_horizon_contributes_nothing():
    view = _view(light_dir=np.array([0, 0, -1], np.float32), light_E=np.float32(3.0))
    col = R.shade(*_flat_inputs(2, [0.5, 0.5, 0.5, 1], [0.0, 0.3, 0.5, 0.0]), view)
    assert torch.all(col == 0)


@pytest.mark.parametrize("r", [0.3, 0.5, 1.0])
def test_ggx_distribution_is_normalised(r):
    """int_hemisphere D(h) (n.h) dw = 1 (numerical quadrature in cos theta)."""
    a2 = torch.as_tensor((max(r, R.ROUGH_MIN) ** 2) ** 2, dtype=F64)
    x = torch.linspace(0, 1, 200001, dtype=F64)  # x = cos(theta_h)
    f = R.ggx_d(x, a2) * x
    integral = 2 * math.pi * torch.trapezoid(f, x)
    assert abs(float(integral) - 1.0) < 1e-4


def test_fresnel_and_masking_limits():
    a2 = torch.as_tensor(0.1, dtype=F64)
    assert float(R.schlick_f(torch.as_tensor(0.04, dtype=F64), torch.as_tensor(1.0, dtype=F64))) == pytest.approx(0.04)
    assert float(R.schlick_f(torch.as_tensor(0.04, dtype=F64), torch.as_tensor(0.0, dtype=F64))) == pytest.approx(1.0)
    assert float(R.smith_g1(torch.as_tensor(1.0, dtype=F64), a2)) == pytest.approx(1.0)
    assert float(R.smith_g1(torch.as_tensor(1.0, dtype=F64), torch.as_tensor(1.0, dtype=F64))) == pytest.approx(1.0)


def test_metal_has_no_diffuse_and_specular_colour_is_kd():
    """m = 1: diffuse term vanishes and ks = kd (Sec. 5.2); at normal incidence with
    light = view direction, F = ks exactly and spec = D F G / (4 n.l n.v) n.l E."""
    view = _view(light_dir=np.array([0, 0, 1], np.float32), light_E=np.float32(1.0))
    kd = np.array([0.9, 0.5, 0.1, 1.0])
    col = R.shade(*_flat_inputs(1, kd, [0.0, 0.5, 1.0, 0.0]), view)
    # eye at (0, 0, 3) above the plane point at the origin: v = l = h = n
    a2 = (0.5 ** 2) ** 2
    D = a2 / (math.pi * (a2) ** 2)
    G = 1.0
    want = D * kd[:3] * G / 4.0
    assert np.allclose(col.numpy()[0], want, rtol=1e-12)


def test_gamma_scales_specular_colour():
    view = _view(light_dir=np.array([0, 0, 1], np.float32), light_E=np.float32(1.0))
    base = R.shade(*_flat_inputs(1, [0.0, 0.0, 0.0, 1], [0.0, 0.5, 0.0, 0.0]), view)
    half = R.shade(*_flat_inputs(1, [0.0, 0.0, 0.0, 1], [0.5, 0.5, 0.0, 0.0]), view)
    # at v.h = 1, F = ks' = (1 - gamma) 0.04
    assert np.allclose(half.numpy(), 0.5 * base.numpy(), rtol=1e-12)


def test_normal_map_tilts_shading_normal():
    """A tangent-space normal (sin a, 0, cos a) with T = +x tilts n toward +x."""
    a = 0.4
    l = np.array([math.sin(a), 0.0, math.cos(a)])
    view = _view(light_dir=l.astype(np.float32), light_E=np.float32(1.0))
    inp = _flat_inputs(1, [0.5, 0.5, 0.5, 1], [1.0, 0.5, 0.0, 0.0], normal=(math.sin(a), 0.0, math.cos(a)))
    col = R.shade(*inp, view)
    ld = view["light_dir"].astype(np.float64)
    assert np.allclose(col.numpy(), 0.5 / math.pi * float(np.dot(ld, l)), atol=1e-7)


# ----------------------------------------------------------------------------- mesh frame

def test_vertex_normals_of_the_icosahedron_point_outwards():
    """By symmetry each icosahedron vertex normal is its radial direction
    exactly; on finer geodesic spheres it stays within a fraction of a
    degree of it. An inward (flipped) cross product gives -p instead."""
    p, tri = synth.icosphere(1)
    n = R.vertex_normals(torch.as_tensor(p), torch.as_tensor(tri.astype(np.int64))).numpy()
    assert np.abs(n - p).max() < 1e-12
    p, tri = synth.icosphere(8)
    n = R.vertex_normals(torch.as_tensor(p), torch.as_tensor(tri.astype(np.int64))).numpy()
    assert (n * p).sum(1).min() > 0.999


def test_vertex_normal_weights_faces_by_area():
    """A vertex shared by a face of area a in the plane z = 0 (normal +z) and a
    face of area b in the plane x = 0 (normal +x) has the normal
    normalize(b, 0, a): each unnormalised face normal is 2 x area x unit normal."""
    a, b = 0.5 * 2.0 * 1.0, 0.5 * 1.0 * 3.0
    pos = torch.as_tensor([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [0.0, 1.0, 0.0],
                           [0.0, 0.0, -3.0]], dtype=F64)
    # face 0: (0, 1, 2) counter-clockwise seen from +z; face 1: (0, 3, 2) from +x
    tri = torch.as_tensor([[0, 1, 2], [0, 3, 2]])
    n = R.vertex_normals(pos, tri).numpy()
    want = np.array([b, 0.0, a]) / math.hypot(a, b)
    assert np.abs(n[0] - want).max() < 1e-15
    assert np.abs(n[1] - [0, 0, 1]).max() < 1e-15 and np.abs(n[3] - [1, 0, 0]).max() < 1e-15


def _planar_quad(flip_u=False, flip_v=False):
    pos = torch.as_tensor([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [1.0, 1.0, 0.0], [0.0, 1.0, 0.0]], dtype=F64)
    uv = pos[:, :2].clone()
    if flip_u:
        uv[:, 0] = 1.0 - uv[:, 0]
    if flip_v:
        uv[:, 1] = 1.0 - uv[:, 1]
    tri = torch.as_tensor([[0, 1, 2], [0, 2, 3]])
    return pos, uv, tri


@pytest.mark.parametrize("flip_u,flip_v,want", [(False, False, 1.0), (True, False, -1.0),
                                                (False, True, 1.0), (True, True, -1.0)])
def test_vertex_tangent_of_a_planar_quad_follows_increasing_u(flip_u, flip_v, want):
    """u along +x gives the tangent +x exactly and u along -x gives -x; the
    direction of v does not change it (the tangent is dp/du, not dp/dv)."""
    pos, uv, tri = _planar_quad(flip_u, flip_v)
    t = R.vertex_tangents(pos, uv, tri, tri).numpy()
    assert np.abs(t - np.array([want, 0.0, 0.0])).max() < 1e-15


def test_face_tangent_is_the_direction_of_dp_du():
    """For an affine map of a triangle from uv to positions, the tangent is
    the normalised dp/du, found here by solving [e1 e2] = [dp/du dp/dv] [d1 d2]
    with a library solve, for random triangles of either uv orientation."""
    rng = np.random.default_rng(11)
    for _ in range(50):
        P = rng.normal(size=(3, 3))
        T = rng.uniform(0, 1, size=(3, 2))
        e = np.stack([P[1] - P[0], P[2] - P[0]], 1)       # 3 x 2
        d = np.stack([T[1] - T[0], T[2] - T[0]], 1)       # 2 x 2
        J = np.linalg.solve(d.T, e.T).T                   # e = J d, J = [dp/du dp/dv]
        want = J[:, 0] / np.linalg.norm(J[:, 0])
        tri = torch.as_tensor([[0, 1, 2]])
        got = R.vertex_tangents(torch.as_tensor(P), torch.as_tensor(T), tri, tri).numpy()
        for k in range(3):
            assert np.abs(got[k] - want).max() < 1e-9


def test_vertex_tangents_of_the_equirectangular_sphere_follow_longitude():
    """u = atan2(z, x) / 2 pi + 1/2 increases with longitude, so dp/du is along
    (-z, 0, x): the vertex tangents of a fine geodesic sphere lie within a few
    degrees of it away from the poles, and nearly perpendicular to the normals."""
    p, tri = synth.icosphere(16)
    uv, tri_uv = synth.equirect_uv_corners(p, tri)
    pos = torch.as_tensor(p)
    t = R.vertex_tangents(pos, torch.as_tensor(uv.astype(np.float64)), torch.as_tensor(tri.astype(np.int64)),
                          torch.as_tensor(tri_uv.astype(np.int64))).numpy()
    n = R.vertex_normals(pos, torch.as_tensor(tri.astype(np.int64))).numpy()
    away = np.abs(p[:, 1]) < 0.9
    lon = np.stack([-p[:, 2], np.zeros(len(p)), p[:, 0]], 1)
    lon /= np.linalg.norm(lon, axis=1, keepdims=True)
    cosang = (t * lon).sum(1)[away]
    assert cosang.min() > math.cos(math.radians(3.0))
    assert np.abs((t * n).sum(1)[away]).max() < 0.05


# ----------------------------------------------------------------------------- antialiasing

def _aa_setup(tau, W=8, H=4, colour=(0.2, 0.4, 0.8)):
    """A quad covering x in [0, xe] with xe = i0 + 0.5 + tau, over an empty background."""
    i0 = 3
    xe = i0 + 0.5 + tau
    scr = torch.as_tensor([[-1.0, -1.0], [xe, -1.0], [xe, H + 1.0], [-1.0, H + 1.0]], dtype=F64)
    XY = np.round(scr.numpy() * 256).astype(np.int32)
    tri = np.array([[0, 1, 2], [0, 2, 3]])
    lib = V._load()
    keys = np.full((H, W), V.EMPTY_KEY, dtype=np.uint64)
    asign = np.zeros(2, np.int8)
    z = np.full(4, 0.5, np.float32)
    ok = np.ones(4, np.int8)
    tri32 = tri.astype(np.int32)
    lib.oracle_raster(V._ptr(XY), V._ptr(z), V._ptr(ok), V._ptr(tri32), 2, W, H, V._ptr(keys), V._ptr(asign))
    cov = keys != V.EMPTY_KEY
    pre = torch.zeros(H, W, 3, dtype=F64)
    pre[torch.as_tensor(cov)] = torch.as_tensor(colour, dtype=F64)
    adj = R.edge_adjacency(tri)
    sil = R.silhouette_flags(asign, adj)
    out = R.antialias(pre, keys, scr, torch.as_tensor(tri), sil, W, H)
    return pre, out, i0


@pytest.mark.parametrize("tau", [0.1, 0.3, 0.49, 0.51, 0.7, 0.95])
def test_aa_vertical_edge_is_linear_in_tau(tau):
    c = np.array([0.2, 0.4, 0.8])
    pre, out, i0 = _aa_setup(tau)
    o = out[:, i0].numpy()
    s = out[:, i0 + 1].numpy()
    if tau > 0.5:
        assert np.allclose(s, (tau - 0.5) * c[None], atol=1e-12)
        assert np.allclose(o, c[None], atol=1e-12)
    else:
        assert np.allclose(o, (0.5 + tau) * c[None], atol=1e-12)
        assert np.allclose(s, 0.0, atol=1e-12)
    # total "coverage" across the pair is (1/2 + tau) c on both sides of 1/2
    assert np.allclose(o + s, (0.5 + tau) * c[None], atol=1e-12)
    # pixels away from the edge are untouched
    assert torch.equal(out[:, : i0], pre[:, : i0])


def test_aa_is_continuous_at_half():
    _, a, i0 = _aa_setup(0.5 - 1e-9)
    _, b, _ = _aa_setup(0.5 + 1e-9)
    assert torch.allclose(a, b, atol=1e-8)


def test_aa_interior_edge_has_no_blend():
    """The shared diagonal of a quad is not a silhouette edge: no blending even
    where the two triangles have different colours."""
    W = H = 8
    scr = torch.as_tensor([[-1.0, -1.0], [W + 1.0, -1.0], [W + 1.0, H + 1.0], [-1.0, H + 1.0]], dtype=F64)
    XY = np.round(scr.numpy() * 256).astype(np.int32)
    tri = np.array([[0, 1, 2], [0, 2, 3]])
    keys, asign = V.np.full((H, W), V.EMPTY_KEY, dtype=np.uint64), np.zeros(2, np.int8)
    lib = V._load()
    lib.oracle_raster(V._ptr(XY), V._ptr(np.full(4, 0.5, np.float32)), V._ptr(np.ones(4, np.int8)),
                      V._ptr(tri.astype(np.int32)), 2, W, H, V._ptr(keys), V._ptr(asign))
    tid = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
    pre = torch.where(torch.as_tensor(tid == 0)[..., None], torch.tensor([1.0, 0, 0], dtype=F64),
                      torch.tensor([0, 0, 1.0], dtype=F64))
    sil = R.silhouette_flags(asign, R.edge_adjacency(tri))
    assert not sil[0, 2] and not sil[1, 0]   # the diagonal 0-2
    out = R.antialias(pre, keys, scr, torch.as_tensor(tri), sil, W, H)
    assert torch.equal(out, pre)


# ----------------------------------------------------------------------------- loss

def test_srgb_is_continuous_at_threshold():
    t = R.SRGB_T
    lo = 12.92 * t
    hi = (1 + R.SRGB_A) * t ** (1 / 2.4) - R.SRGB_A
    assert abs(lo - hi) < 1e-6
    x = torch.as_tensor([t - 1e-12, t + 1e-12], dtype=F64)
    y = R.srgb(x)
    assert abs(float(y[1] - y[0])) < 1e-6


def test_tonemap_values():
    x = torch.as_tensor([0.0, math.e - 1.0], dtype=F64)   # log(x + 1) = 0, 1
    y = R.tonemap(x)
    assert float(y[0]) == 0.0
    assert float(y[1]) == pytest.approx(1.0)   # Gamma(1) = 1.055 - 0.055


def test_tonemap_counts_negative_radiance_as_black():
    # below zero (and below -1, where log(x + 1) has no value) the tone map is
    # flat at Gamma(log 1) = 0 with zero slope; NaN is kept so a broken job shows
    x = torch.tensor([-3.0, -1.0, -0.25, 0.0, 0.5], dtype=F64, requires_grad=True)
    y = R.tonemap(x)
    assert torch.all(y[:4] == 0.0) and float(y[4].detach()) > 0.0
    (g,) = torch.autograd.grad(y.sum(), x)
    assert torch.all(g[:3] == 0.0) and float(g[4]) > 0.0
    assert math.isnan(float(R.tonemap(torch.as_tensor([float("nan")], dtype=F64))[0]))
    a = torch.as_tensor([[[[-2.0, 0.3, 0.1]]]], dtype=F64)
    b = torch.as_tensor([[[[0.0, 0.3, 0.1]]]], dtype=F64)
    ref = torch.full_like(a, 0.2)
    assert float(R.image_loss(a, ref, "logl1")) == float(R.image_loss(b, ref, "logl1"))


@pytest.mark.parametrize("kind", ["l1", "logl1", "l2"])
def test_loss_zero_at_equality_with_zero_gradient(kind):
    rng = np.random.default_rng(0)
    x = torch.as_tensor(rng.uniform(0, 3, (2, 4, 4, 3)), dtype=F64).requires_grad_(True)
    L = R.image_loss(x, x.detach().clone(), kind)
    (g,) = torch.autograd.grad(L, x)
    assert float(L.detach()) == 0.0 and torch.all(g == 0)


def test_l1_loss_is_mean_abs():
    x = torch.as_tensor([[1.0, 2.0, 3.0]], dtype=F64)
    y = torch.as_tensor([[0.5, 2.5, 3.0]], dtype=F64)
    assert float(R.image_loss(x, y, "l1")) == pytest.approx(1.0 / 3.0)


# ----------------------------------------------------------------------------- Laplacian, schedules, Adam

def test_laplacian_planar_grid_interior_is_zero():
    n = 6
    ys, xs = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    pos = torch.as_tensor(np.stack([xs, ys, np.zeros_like(xs)], -1).reshape(-1, 3).astype(np.float64))
    idx = lambda x, y: y * n + x  # noqa: E731
    tri = []
    for y in range(n - 1):
        for x in range(n - 1):
            tri += [[idx(x, y), idx(x + 1, y), idx(x + 1, y + 1)], [idx(x, y), idx(x + 1, y + 1), idx(x, y + 1)]]
    d = R.laplacian_delta(pos, R.one_ring(np.array(tri), n * n)).numpy().reshape(n, n, 3)
    assert np.abs(d[1:-1, 1:-1]).max() < 1e-14
    assert np.abs(d[0, 0]).max() > 0.1


def test_laplacian_icosahedron_closed_form():
    """Each icosahedron vertex has 5 neighbours at cos(angle) = 1/sqrt(5):
    delta_i = (1 - 1/sqrt(5)) v_i and L_delta = (1 - 1/sqrt(5))^2."""
    p, tri = synth.icosphere(1)
    pos = torch.as_tensor(p)
    ring = R.one_ring(tri, 12)
    assert all(len(r) == 5 for r in ring)
    d = R.laplacian_delta(pos, ring)
    c = 1 - 1 / math.sqrt(5)
    assert torch.allclose(d, c * pos, atol=1e-12)
    assert float(R.laplacian_loss(pos, ring)) == pytest.approx(c * c, rel=1e-12)
    # relative mode against itself is zero
    assert float(R.laplacian_loss(pos, ring, d)) == 0.0


def test_lambda_schedule_closed_form_of_the_recursive_reading():
    """The recursive reading of the schedule after Eq. 5 multiplies the excess
    over lambda_min by 10^(-k s) at every step s = 1..t, so the product
    telescopes: lambda_t - lambda_min = (lambda_0 - lambda_min) 10^(-k t (t + 1) / 2)."""
    lam0 = 2.0
    lmin = 0.02 * lam0
    lam = lam0
    got = {}
    for t in range(1, 3001):
        lam = R.lambda_schedule(lam, lam0, t)
        got[t] = lam
    for t in (1, 2, 1000, 2000, 3000):
        want = lmin + (lam0 - lmin) * 10.0 ** (-1e-6 * t * (t + 1) / 2)
        assert got[t] == pytest.approx(want, rel=1e-12)
    # about 2-3k steps to decay to lambda_min: a tenth of the excess left at t = 1000,
    # under 1e-4 of it at t = 3000
    assert (got[1000] - lmin) / (lam0 - lmin) == pytest.approx(10 ** -0.5005, rel=1e-9)
    assert (got[3000] - lmin) / (lam0 - lmin) < 1e-4


def test_learning_rate_schedule_closed_form():
    """lr_t = lr_0 10^(-0.0002 t) (Sec. 5.3): a tenth every 5000 steps."""
    assert R.learning_rate(0.01, 5000) == pytest.approx(0.001, rel=1e-12)
    assert R.learning_rate(0.01, 10000) == pytest.approx(0.0001, rel=1e-12)
    assert R.learning_rate(0.01, 0) == 0.01


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(3)
    p = torch.as_tensor(rng.uniform(-1, 1, (50, 4)))
    g = torch.as_tensor(rng.normal(size=(50, 4)) * 10.0 ** rng.uniform(-9, 1, (50, 4)))
    z = torch.zeros_like(p)
    lr = 0.01
    p1, m1, v1 = R.adam_update(p, g, z, z, 0, lr, "pos")
    want = p - lr * g / (g.abs() + 1e-8)
    assert torch.allclose(p1, want, rtol=0, atol=1e-15)
    assert torch.allclose(m1, 0.1 * g) and torch.allclose(v1, 0.001 * g * g)


def test_adam_clamps_ranges():
    p = torch.as_tensor([[0.99, 0.09, 0.5, 0.0]], dtype=F64)
    g = torch.as_tensor([[-1.0, 1.0, 0.0, 0.0]], dtype=F64)
    z = torch.zeros_like(p)
    p1, _, _ = R.adam_update(p, g, z, z, 0, 0.1, "orm")
    assert float(p1[0, 0]) == 1.0 and float(p1[0, 1]) == pytest.approx(R.ROUGH_MIN)
    n = torch.as_tensor([[0.0, 0.0, 0.05, 0.0]], dtype=F64)
    p2, _, _ = R.adam_update(n, torch.as_tensor([[0, 0, 1.0, 0]], dtype=F64), z, z, 0, 0.1, "nrm")
    assert float(p2[0, 2]) == 0.0


# ----------------------------------------------------------------------------- tessellation

def test_tessellation_counts_and_flat_positions():
    p, tri = synth.icosphere(2)
    mesh_uv, tri_uv = synth.equirect_uv_corners(p, tri)
    ts = TS.Tessellation(tri.astype(np.int64), tri_uv.astype(np.int64), mesh_uv.astype(np.float64), 3)
    n = 2 * 8
    assert ts.tri.shape[0] == 20 * n * n and ts.n_verts == 10 * n * n + 2
    pos = torch.as_tensor(p)
    nrm = R.vertex_normals(pos, torch.as_tensor(tri.astype(np.int64)))
    flat = ts.displaced_positions(pos, nrm, torch.zeros(4, 4, dtype=F64))
    # zero displacement: each vertex lies in the plane of its owning base triangle
    a, b, c = (pos[ts.base_idx[:, k]] for k in range(3))
    nrm_f = torch.linalg.cross(b - a, c - a)
    assert float(((flat - a) * nrm_f).sum(1).abs().max()) < 1e-12
    # constant displacement d moves every vertex by exactly d
    moved = ts.displaced_positions(pos, nrm, torch.full((4, 4), 0.05, dtype=F64))
    assert torch.allclose((moved - flat).norm(dim=1), torch.full((ts.n_verts,), 0.05, dtype=F64), atol=1e-12)
    # the tessellated mesh is closed and consistently wound (every directed edge once)
    e = np.concatenate([ts.tri[:, [0, 1]], ts.tri[:, [1, 2]], ts.tri[:, [2, 0]]])
    s = set(map(tuple, e))
    assert len(s) == len(e) and all((y, x) in s for x, y in s)


def test_tessellation_float32_contract_matches_float64():
    """The float32 positions visibility uses equal the float64 displaced positions
    to float32 rounding, for a random displacement map."""
    p, tri = synth.icosphere(3)
    uv, tri_uv = synth.equirect_uv_corners(p, tri)
    ts = TS.Tessellation(tri.astype(np.int64), tri_uv.astype(np.int64), uv.astype(np.float64), 2)
    rng = np.random.default_rng(4)
    disp = rng.uniform(-0.05, 0.05, (16, 16)).astype(np.float32)
    pos32 = p.astype(np.float32)
    f32 = ts.positions_f32(pos32, tri, disp)
    bp = torch.as_tensor(pos32.astype(np.float64))
    nrm = R.vertex_normals(bp, torch.as_tensor(tri.astype(np.int64)))
    f64 = ts.displaced_positions(bp, nrm, torch.as_tensor(disp.astype(np.float64))).numpy()
    assert np.abs(f32 - f64).max() < 2e-6


# ----------------------------------------------------------------------------- gradients vs central differences

def _tiny_job(loss="logl1", tess=0, skin=0):
    p, tri = synth.icosphere(3)
    uv, tri_uv = synth.equirect_uv_corners(p, tri)
    mesh = synth.Mesh(p.astype(np.float32), uv, tri, tri_uv)
    rng = np.random.default_rng(5)
    kd = rng.uniform(0.1, 0.9, (16, 16, 4)).astype(np.float32)
    orm = np.stack([rng.uniform(0, 1, (16, 16)), rng.uniform(0.1, 1, (16, 16)), rng.uniform(0, 1, (16, 16)),
                    np.zeros((16, 16))], -1).astype(np.float32)
    nrm = np.stack([rng.uniform(-0.5, 0.5, (16, 16)), rng.uniform(-0.5, 0.5, (16, 16)),
                    rng.uniform(0.5, 1, (16, 16)), np.zeros((16, 16))], -1).astype(np.float32)
    disp = rng.uniform(-0.02, 0.02, (8, 8)).astype(np.float32) if tess else None
    sc = synth.Scene(mesh=mesh, kd=kd, orm=orm, nrm=nrm, disp=disp, tess_levels=tess,
                     optimize={"pos": True, "kd": True, "orm": True, "nrm": True, "disp": bool(tess)})
    if not skin:
        return S.OracleJob(sc, loss=loss)
    job = S.OracleJob(sc, loss=loss, skin_weights=synth.bone_weights(p, skin, seed=2))
    job.bones = torch.as_tensor(synth.bone_pose(skin, 2, 0).astype(np.float64))
    return job


@pytest.mark.parametrize("loss,tess,skin", [("logl1", 0, 0), ("l1", 0, 0), ("logl1", 1, 0), ("logl1", 0, 4)])
def test_gradients_match_central_differences(loss, tess, skin):
    """Central differences on 64 random latents with visibility, LOD and the AA
    edge choice held fixed: h = 1e-3 for texels; h = 1e-5 for positions and
    displacement, whose moves of 1e-3 cross kinks of the piecewise-bilinear
    filter and of |.| in the loss."""
    job = _tiny_job(loss, tess, skin)
    H = W = 40
    views = synth.sample_views(11, 0, 2, W, H, r_min=2.2, r_max=2.6)
    rng = np.random.default_rng(9)
    refs = torch.as_tensor(rng.uniform(0, 1.5, (2, H, W, 3)))
    params = {k: v.clone().requires_grad_(job.optimize[k]) for k, v in job.params.items()}
    lods = {}
    base = S.objective(job, params, views, refs, H, W, lam=0.3, lods=lods)
    vis = (base["out"]["keys"], base["out"]["asign"])
    live = [k for k in params if job.optimize[k]]
    grads = dict(zip(live, torch.autograd.grad(base["total"], [params[k] for k in live])))
    # 64 random latents among those the image actually touches
    picks = []
    for k in live:
        nz = torch.nonzero(grads[k].reshape(-1)).squeeze(1).numpy()
        if nz.size:
            picks += [(k, int(i)) for i in rng.choice(nz, size=min(nz.size, 16), replace=False)]
    picks = picks[:64]
    assert len(picks) >= 40
    errs = []
    for k, i in picks:
        h = 1e-5 if k in ("pos", "disp", "w") else 1e-3
        vals = []
        for sgn in (1, -1):
            pp = {kk: vv.detach().clone() for kk, vv in params.items()}
            pp[k].view(-1)[i] += sgn * h
            vals.append(float(S.objective(job, pp, views, refs, H, W, vis=vis, lam=0.3, lods=lods)["total"]))
        fd = (vals[0] - vals[1]) / (2 * h)
        an = float(grads[k].reshape(-1)[i])
        errs.append(abs(fd - an) / max(abs(an), 1e-4 * max(float(g.abs().max()) for g in grads.values())))
    errs = np.array(errs)
    # only |.| and the clamps are kinks; a pick straddling one within +-h may disagree
    assert np.median(errs) < 1e-5
    assert (errs < 1e-3).mean() >= 0.95


# ---------------------------------------------------------------- per-level latent textures (Sec. 6)
def _per_level_case():
    c = synth.config_small()
    c["cand"].optimize = {"pos": True, "kd": True, "orm": False, "nrm": True}
    views = synth.fixed_view(64, 64)
    ref = S.render_reference(c["ref"], views, 64, 64)[0].numpy()
    return c, views, ref


def _grads(job, views, ref):
    params = {k: v.clone().requires_grad_(job.optimize[k]) for k, v in job.params.items()}
    obj = S.objective(job, params, views, torch.as_tensor(ref.astype(np.float64)), 64, 64, lam=0.0)
    live = [k for k in params if job.optimize[k]]
    gs = torch.autograd.grad(obj["total"], [params[k] for k in live], allow_unused=True)
    return obj, {k: (g if g is not None else torch.zeros_like(params[k])) for k, g in zip(live, gs)}


def test_per_level_textures_start_as_the_box_filter_chain():
    c, views, ref = _per_level_case()
    std, lev = S.OracleJob(c["cand"], loss="l1"), S.OracleJob(c["cand"], loss="l1", per_level=True)
    assert sum(k.startswith("kd@") for k in lev.params) == 8   # 256^2: levels 1..8
    a = S.render(std, std.params, views, 64, 64)["img"]
    b = S.render(lev, lev.params, views, 64, 64)["img"]
    assert torch.equal(a, b)


def test_per_level_gradients_fold_to_the_standard_gradient():
    # the standard job's level-0 gradient is the adjoint of the box-filter chain applied
    # to the per-level gradients: sum over k of 4^-k times level k's gradient, spread
    # over each level-k texel's 2^k x 2^k block of level-0 texels
    c, views, ref = _per_level_case()
    std, lev = S.OracleJob(c["cand"], loss="l1"), S.OracleJob(c["cand"], loss="l1", per_level=True)
    _, gs = _grads(std, views, ref)
    _, gl = _grads(lev, views, ref)
    for name in ("kd", "nrm"):
        fold = gl[name].clone()
        k = 1
        while f"{name}@{k}" in gl:
            g = gl[f"{name}@{k}"]
            fold += g.repeat_interleave(2 ** k, 0).repeat_interleave(2 ** k, 1) / 4.0 ** k
            k += 1
        assert float(fold.abs().max()) > 0
        assert torch.allclose(fold, gs[name], rtol=1e-10, atol=1e-14 * float(gs[name].abs().max()))
        assert float(gl[f"{name}@2"].abs().max()) > 0   # a sampled coarse level gets its own gradient


def test_per_level_step_updates_levels_independently():
    c, views, ref = _per_level_case()
    lev = S.OracleJob(c["cand"], loss="l1", per_level=True, lam0=1.0)
    before = {k: v.clone() for k, v in lev.params.items()}
    S.step(lev, views, ref, 64, 64)
    # the 1x1 level is not sampled at this view's LOD: zero gradient, unchanged by Adam
    assert torch.equal(lev.params["kd@8"], before["kd@8"])
    # a sampled level moved on its own: it is no longer the box filter of the new level 0
    assert not torch.equal(lev.params["kd@2"], before["kd@2"])
    chain = R.mip_chain(lev.params["kd"])
    assert not torch.allclose(chain[2], lev.params["kd@2"])
    # clamps act per level as on level 0
    assert float(lev.params["kd@2"].min()) >= 0.0 and float(lev.params["kd@2"].max()) <= 1.0


# ---------------------------------------------------------------- skinning (Eq. 2)
def _rig(n_bones=5, seed=3):
    p, tri = synth.icosphere(4)
    return p.astype(np.float32), synth.bone_weights(p, n_bones, seed), synth.bone_pose(n_bones, seed, 1)


def test_skinning_with_identity_bones_and_convex_weights_is_the_rest_pose():
    pos, w, _ = _rig()
    eye = np.tile(np.eye(4, dtype=np.float32), (w.shape[1], 1, 1))
    f64 = SK.skin(torch.as_tensor(pos.astype(np.float64)), torch.as_tensor(w.astype(np.float64)),
                  torch.as_tensor(eye.astype(np.float64))).numpy()
    assert np.abs(f64 - pos).max() < 1e-6          # the float32 weights sum to 1 within 1e-7
    one_hot = np.eye(w.shape[1], dtype=np.float32)[np.argmax(w, 1)]
    assert np.array_equal(V.skin_positions_f32(pos, one_hot, eye), pos)


def test_skinning_one_bone_is_its_affine_map():
    pos, _, pose = _rig(n_bones=1)
    M = pose[0]
    want = (pos.astype(np.float64) @ M[:3, :3].T.astype(np.float64)) + M[:3, 3]
    got = SK.skin(torch.as_tensor(pos.astype(np.float64)), torch.ones((len(pos), 1), dtype=F64),
                  torch.as_tensor(pose.astype(np.float64))).numpy()
    assert np.abs(got - want).max() < 1e-12
    # the float32 contract, restated step by step in numpy float32 (no fused operations)
    f = np.float32
    t = [((M[r, 0] * pos[:, 0] + M[r, 1] * pos[:, 1]) + M[r, 2] * pos[:, 2]) + M[r, 3] for r in range(3)]
    ref32 = np.stack([f(0) + f(1) * t[r] for r in range(3)], 1).astype(np.float32)
    assert np.array_equal(V.skin_positions_f32(pos, np.ones((len(pos), 1), np.float32), pose), ref32)


def test_skinning_is_linear_in_the_weights():
    pos, w, pose = _rig()
    rng = np.random.default_rng(4)
    w2 = rng.uniform(-0.5, 0.5, w.shape)
    P, Bn = torch.as_tensor(pos.astype(np.float64)), torch.as_tensor(pose.astype(np.float64))
    a = SK.skin(P, torch.as_tensor(w.astype(np.float64)), Bn)
    b = SK.skin(P, torch.as_tensor(w2), Bn)
    c = SK.skin(P, torch.as_tensor(w.astype(np.float64) + w2), Bn)
    assert torch.allclose(a + b, c, atol=1e-13)
    assert torch.allclose(SK.skin(P, 2.5 * torch.as_tensor(w2), Bn), 2.5 * b, atol=1e-13)


def test_skinning_float32_contract_is_near_float64():
    pos, w, pose = _rig()
    f32 = V.skin_positions_f32(pos, w, pose)
    f64 = SK.skin(torch.as_tensor(pos.astype(np.float64)), torch.as_tensor(w.astype(np.float64)),
                  torch.as_tensor(pose.astype(np.float64))).numpy()
    assert np.abs(f32 - f64).max() < 2e-6
    assert np.abs(f32 - pos).max() > 1e-2            # the pose moved the mesh


# ---------------------------------------------------------------- MSAA training render (Sec. 5.2, antialiasing)
def test_msaa_interior_pixels_equal_the_one_sample_render():
    # a pixel whose s x s samples all see the triangle under its centre is that
    # triangle shaded once at the centre with the pixel's LOD: the 1-spp value
    c = synth.config_plain(tex_res=64, ref_tex_res=64, ref_freq=8, cand_freq=6, n_views=1, res=48)
    views = synth.sample_views(3, 0, 2, 48, 48)
    one = S.OracleJob(c["cand"], loss="l1")
    ms = S.OracleJob(c["cand"], loss="l1", msaa=2)
    with torch.no_grad():
        a = S.render(one, one.params, views, 48, 48, aa=False)
        b = S.render(ms, ms.params, views, 48, 48, aa=False)
    tid = lambda k: np.where(k == np.uint64(R.EMPTY), -1, (k & np.uint64(0xFFFFFFFF)).astype(np.int64))
    t1, t2 = tid(a["keys"]), tid(b["keys"]).reshape(2, 48, 2, 48, 2)
    same = (t2 == t1[:, :, None, :, None]).all(axis=(2, 4)) & (t1 >= 0)
    assert same.mean() > 0.2
    x, y = a["img"].numpy()[same], b["img"].numpy()[same]
    assert np.abs(x - y).max() <= 1e-12 * np.abs(x).max()
    assert not np.allclose(a["img"].numpy(), b["img"].numpy())   # edges do differ: coverage is integrated


def _lambert_quad(half):
    pos = np.array([[-half, -half, 0], [half, -half, 0], [half, half, 0], [-half, half, 0]], np.float32)
    uv = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float32)
    tri = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    mesh = synth.Mesh(pos, uv, tri, tri.copy())
    return synth.Scene(mesh=mesh, kd=synth.constant_texture((0.6, 0.3, 0.9, 1.0)),
                       orm=synth.constant_texture((1.0, 1.0, 0.0)), nrm=synth.constant_texture((0.0, 0.0, 1.0)),
                       optimize={})


@pytest.mark.parametrize("mode", ["msaa", "ssaa"])
def test_supersampled_coverage_of_a_lambertian_quad(mode):
    # gamma = 1 removes the specular lobe and a directional light on a plane gives one
    # radiance c everywhere, so with antialiasing off each pixel is c times the share of
    # its 2 x 2 samples inside the quad, decided here from the float64 projection
    W = H = 40
    sc = _lambert_quad(0.537)
    view = synth.make_view((0.0, 0.0, 3.0), W, H, light_dir=(0.3, 0.2, 1.0), light_E=2.0)
    views = np.zeros(1, dtype=synth.VIEW_DTYPE)
    views[0] = view
    job = S.OracleJob(sc, loss="l1", msaa=2 if mode == "msaa" else 1)
    with torch.no_grad():
        img = S.render(job, job.params, views, H, W, aa=False, ssaa=2 if mode == "ssaa" else 1)["img"][0].numpy()
    M = view["mvp"].astype(np.float64).reshape(4, 4)
    corner = M @ np.array([0.537, 0.537, 0.0, 1.0])
    ex = (corner[0] / corner[3] * 0.5 + 0.5) * W          # right edge, pixels
    ey = (0.5 - corner[1] / corner[3] * 0.5) * H          # top edge (y down)
    lo_x, lo_y = W - ex, H - ey                           # left / bottom edges by symmetry
    c = img[H // 2, W // 2]
    lam = np.array([0.6, 0.3, 0.9]) / math.pi * 2.0 * (np.array([0.3, 0.2, 1.0]) / np.linalg.norm([0.3, 0.2, 1.0]))[2]
    assert np.allclose(c, lam, rtol=1e-6)
    checked = 0
    for j in range(H):
        for i in range(W):
            xs = [i + 0.25, i + 0.75]
            ys = [j + 0.25, j + 0.75]
            if min(abs(x - e) for x in xs for e in (lo_x, ex)) < 1e-3 or min(abs(y - e) for y in ys for e in (ey, lo_y)) < 1e-3:
                continue
            cov = sum((lo_x < x < ex) and (ey < y < lo_y) for x in xs for y in ys) / 4.0
            assert np.allclose(img[j, i], cov * lam, rtol=1e-6, atol=1e-12), (i, j, cov)
            checked += cov not in (0.0, 1.0)
    assert checked > 20      # partly covered edge pixels were checked
