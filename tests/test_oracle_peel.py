"""Pins of the oracle's depth peeling (order-independent transparency, Sec. 5.2)
against brute force, closed forms, exact reductions to the opaque render and
central differences."""

import math

import numpy as np
import pytest
import torch

import synth
from oracle import render as R
from oracle import step as S
from oracle import visibility as V


def _soup(seed, n):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-0.8, 0.8, (3 * n, 3)).astype(np.float32)
    tri = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    # a repeated triangle: two fragments of equal depth at every covered pixel
    pos = np.concatenate([pos, pos[:3]])
    tri = np.concatenate([tri, np.array([[3 * n, 3 * n + 1, 3 * n + 2]], np.int32)])
    return pos, tri


@pytest.mark.parametrize("seed", range(4))
def test_peeled_layers_are_the_sorted_fragment_keys(seed):
    # brute force: every triangle rasterized alone gives its fragment key at each
    # pixel; layer l must be the (l+1)-th smallest of them, EMPTY beyond
    W = H = 24
    pos, tri = _soup(seed, 12)
    mvp = synth.sample_views(seed, 0, 1, W, H, r_min=2.2, r_max=2.6)[0]["mvp"]
    frags = [[] for _ in range(H * W)]
    for f in range(tri.shape[0]):
        k, _, _ = V.raster(mvp, pos, tri[f:f + 1], W, H)
        k = k.reshape(-1)
        for p in np.nonzero(k != V.EMPTY_KEY)[0]:
            frags[p].append((int(k[p]) >> 32 << 32) | f)
    depth = max(len(x) for x in frags)
    assert depth >= 3
    keys, _ = V.raster_peeled(mvp, pos, tri, W, H, depth + 1)
    for p in range(H * W):
        want = sorted(frags[p]) + [int(V.EMPTY_KEY)] * (depth + 1 - len(frags[p]))
        got = [int(keys[l].reshape(-1)[p]) for l in range(depth + 1)]
        assert got == want, p
    # the repeated triangle's two copies sit in consecutive layers
    assert any(len(set(x >> 32 for x in fr)) < len(fr) for fr in frags)


def _cloud_scene(opaque, n_quads=30, seed=4):
    mesh = synth.quad_cloud(n_quads, seed, size=(0.15, 0.3), radii=(0.6, 0.5, 0.6))
    kd, nrm = synth.noise_textures(32, seed=seed)
    kd[..., 3] = 1.0 if opaque else np.random.default_rng(seed).uniform(0.2, 0.9, (32, 32))
    return synth.Scene(mesh=mesh, kd=kd, orm=synth.scenes.uniform_orm(32, seed), nrm=nrm,
                       optimize={"pos": True, "kd": True, "orm": True, "nrm": True})


@pytest.mark.parametrize("layers,aa", [(3, False), (1, True)])
def test_opaque_peel_reduces_to_the_opaque_render(layers, aa):
    # opacity 1 makes every blend return the nearer layer's colour: without
    # antialiasing any number of layers, and with it one layer, give the opaque image
    # (up to the rounding of the filtered opacity, 1 within a few ulps)
    sc = _cloud_scene(opaque=True)
    views = synth.sample_views(7, 0, 2, 40, 40, r_min=2.2, r_max=2.6)
    a = S.OracleJob(sc, loss="l2")
    b = S.OracleJob(sc, loss="l2", layers=layers)
    with torch.no_grad():
        x = S.render(a, a.params, views, 40, 40, aa=aa)["img"]
        y = S.render(b, b.params, views, 40, 40, aa=aa)["img"]
    assert float(x.abs().max()) > 0
    assert float((x - y).abs().max()) <= 1e-13 * float(x.abs().max())


def test_layers_beyond_the_depth_complexity_change_nothing():
    sc = _cloud_scene(opaque=False)
    views = synth.sample_views(8, 0, 2, 40, 40, r_min=2.2, r_max=2.6)
    j = S.OracleJob(sc, loss="l2", layers=12)
    with torch.no_grad():
        out = S.render(j, j.params, views, 40, 40)
    k = out["keys"]
    used = max(l for l in range(12) if (k[:, l] != V.EMPTY_KEY).any()) + 1
    assert 2 <= used < 12
    j2 = S.OracleJob(sc, loss="l2", layers=used)
    with torch.no_grad():
        img2 = S.render(j2, j2.params, views, 40, 40)["img"]
    assert torch.equal(out["img"], img2)
    # and fewer layers than that does change it
    j3 = S.OracleJob(sc, loss="l2", layers=1)
    with torch.no_grad():
        img3 = S.render(j3, j3.params, views, 40, 40)["img"]
    assert not torch.equal(out["img"], img3)


def _two_quads(alpha_f, alpha_b, front_first):
    # front quad (half 0.3, z = 0.2) over a back quad (half 0.45, z = -0.2), both facing
    # +z; texture columns 0-1 hold the front colour, 2-3 the back one, and each quad's
    # uv sits between its two columns, so bilinear filtering returns its colour exactly
    front = np.array([[-0.3, -0.3, 0.2], [0.3, -0.3, 0.2], [0.3, 0.3, 0.2], [-0.3, 0.3, 0.2]])
    back = np.array([[-0.45, -0.45, -0.2], [0.45, -0.45, -0.2], [0.45, 0.45, -0.2], [-0.45, 0.45, -0.2]])
    quads = [front, back] if front_first else [back, front]
    us = [0.25, 0.75] if front_first else [0.75, 0.25]
    pos = np.concatenate(quads).astype(np.float32)
    uv = np.array([[u, 0.5] for u in us for _ in range(4)], np.float32)
    tri = np.array([[0, 1, 2], [0, 2, 3], [4, 5, 6], [4, 6, 7]], np.int32)
    kd = np.zeros((4, 4, 4), np.float32)
    kd[:, 0:2] = (0.6, 0.3, 0.9, alpha_f)
    kd[:, 2:4] = (0.2, 0.8, 0.4, alpha_b)
    sc = synth.Scene(mesh=synth.Mesh(pos, uv, tri, tri.copy()), kd=kd,
                     orm=synth.constant_texture((1.0, 1.0, 0.0), 4), nrm=synth.constant_texture((0.0, 0.0, 1.0), 4),
                     optimize={})
    return sc


@pytest.mark.parametrize("alpha_f,alpha_b", [(0.3, 0.8), (1.0, 0.5), (0.0, 1.0), (0.55, 0.55)])
def test_two_translucent_quads_composite_in_closed_form(alpha_f, alpha_b):
    # gamma = 1 and m = 0 leave L = kd / pi E n.l on each quad; with antialiasing off
    # back-to-front blending over black gives alpha_f L_f + (1 - alpha_f) alpha_b L_b
    # where both cover a pixel, alpha L where one does, 0 elsewhere; the order of the
    # triangles in the mesh does not matter
    W = H = 40
    view = synth.make_view((0.0, 0.0, 3.0), W, H, light_dir=(0.3, 0.2, 1.0), light_E=2.0)
    views = np.zeros(1, dtype=synth.VIEW_DTYPE)
    views[0] = view
    # the texture holds float32 values
    f32 = lambda x: np.asarray(x, np.float32).astype(np.float64)  # noqa: E731
    nl = float(view["light_dir"][2])   # the view record holds the unit light direction in float32
    Lf = f32([0.6, 0.3, 0.9]) / math.pi * 2.0 * nl
    Lb = f32([0.2, 0.8, 0.4]) / math.pi * 2.0 * nl
    alpha_f, alpha_b = float(f32(alpha_f)), float(f32(alpha_b))
    M = view["mvp"].astype(np.float64).reshape(4, 4)

    def extent(h, z):   # pixel-space half-open interval covered along x (and y by symmetry)
        c = M @ np.array([h, h, z, 1.0])
        e = (c[0] / c[3] * 0.5 + 0.5) * W
        return W - e, e

    fx0, fx1 = extent(0.3, 0.2)
    bx0, bx1 = extent(0.45, -0.2)
    imgs = []
    for order in (True, False):
        job = S.OracleJob(_two_quads(alpha_f, alpha_b, order), loss="l2", layers=2)
        with torch.no_grad():
            imgs.append(S.render(job, job.params, views, H, W, aa=False)["img"][0].numpy())
    assert np.array_equal(imgs[0], imgs[1])
    img = imgs[0]
    seen = set()
    for j in range(H):
        for i in range(W):
            x, y = i + 0.5, j + 0.5
            if min(abs(x - e) for e in (fx0, fx1, bx0, bx1)) < 1e-3 or min(abs(y - e) for e in (fx0, fx1, bx0, bx1)) < 1e-3:
                continue
            inf = fx0 < x < fx1 and fx0 < y < fx1
            inb = bx0 < x < bx1 and bx0 < y < bx1
            want = (alpha_f * Lf + (1 - alpha_f) * alpha_b * Lb) if inf else (alpha_b * Lb if inb else np.zeros(3))
            assert np.allclose(img[j, i], want, rtol=1e-9, atol=1e-12), (i, j)
            seen.add((inf, inb))
    assert seen == {(True, True), (False, True), (False, False)}


def test_peel_gradients_match_central_differences():
    """Central differences of the L2 objective on 64 latents (opacity texels among
    them) with visibility, LOD and the AA edge choices held fixed."""
    sc = _cloud_scene(opaque=False, n_quads=24, seed=6)
    job = S.OracleJob(sc, loss="l2", layers=4)
    H = W = 36
    views = synth.sample_views(12, 0, 2, W, H, r_min=2.0, r_max=2.4)
    rng = np.random.default_rng(10)
    refs = torch.as_tensor(rng.uniform(0, 0.6, (2, H, W, 3)))
    params = {k: v.clone().requires_grad_(job.optimize[k]) for k, v in job.params.items()}
    lods = {}
    base = S.objective(job, params, views, refs, H, W, lam=0.3, lods=lods)
    vis = (base["out"]["keys"], base["out"]["asign"])
    assert (vis[0][:, 1] != V.EMPTY_KEY).any()     # a second layer exists
    live = [k for k in params if job.optimize[k]]
    grads = dict(zip(live, torch.autograd.grad(base["total"], [params[k] for k in live])))
    ga = grads["kd"][..., 3].reshape(-1)
    picks = [("kd", int(4 * i + 3)) for i in rng.choice(torch.nonzero(ga).squeeze(1).numpy(), 16, replace=False)]
    for k in live:
        nz = torch.nonzero(grads[k].reshape(-1)).squeeze(1).numpy()
        picks += [(k, int(i)) for i in rng.choice(nz, size=min(nz.size, 12), replace=False)]
    picks = picks[:64]
    assert len(picks) >= 50
    scale = max(float(g.abs().max()) for g in grads.values())
    errs = []
    for k, i in picks:
        h = 1e-5 if k == "pos" else 1e-3
        vals = []
        for sgn in (1, -1):
            pp = {kk: vv.detach().clone() for kk, vv in params.items()}
            pp[k].view(-1)[i] += sgn * h
            vals.append(float(S.objective(job, pp, views, refs, H, W, vis=vis, lam=0.3, lods=lods)["total"]))
        fd = (vals[0] - vals[1]) / (2 * h)
        an = float(grads[k].reshape(-1)[i])
        errs.append(abs(fd - an) / max(abs(an), 1e-4 * scale))
    errs = np.array(errs)
    assert np.median(errs) < 1e-5
    assert (errs < 1e-3).mean() >= 0.95
