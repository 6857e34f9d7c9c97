"""Shared parity-test cases: seeded scenes, views and reference images.

Reference images fed to both sides come from the oracle (float64, rounded to
float32 once), never from the CUDA path."""

from __future__ import annotations

import numpy as np
import torch

import synth
from oracle import step as S


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def sphere_scene(freq, tex, seed, tess=0):
    """A frequency-`freq` icosphere with tex^2 noise maps, every latent
    optimized; with tess > 0 also a 32^2 random displacement map and that many
    levels of edge-midpoint splitting."""
    from synth.workloads import Scene
    p, tri = synth.icosphere(freq)
    uv, tri_uv = synth.equirect_uv_corners(p, tri)
    mesh = synth.Mesh(p.astype(np.float32), uv, tri, tri_uv)
    kd, nrm = synth.noise_textures(tex, seed=seed)
    orm = synth.scenes.uniform_orm(tex, seed)
    disp = np.random.default_rng(seed).uniform(-0.02, 0.02, (32, 32)).astype(np.float32) if tess else None
    return Scene(mesh=mesh, kd=kd, orm=orm, nrm=nrm, disp=disp, tess_levels=tess,
                 optimize={"pos": True, "kd": True, "orm": True, "nrm": True, "disp": bool(tess)})


def small_case():
    """One 256^2 view, 320-tri candidate with 256^2 maps vs the 20,480-tri reference, plain L1."""
    c = synth.config_small()
    views = synth.fixed_view(256, 256)
    return c, views, 256, 256


def plain_case(res=128, n_views=8, tex=256, ref_tex=256, ref_freq=32, seed=5):
    """The batched-view workload shrunk for the oracle: 5,120-tri candidate, 8 random views."""
    c = synth.config_plain(tex_res=tex, ref_tex_res=ref_tex, ref_freq=ref_freq, n_views=n_views, res=res)
    views = synth.sample_views(seed, 0, n_views, res, res)
    return c, views, res, res


def tess_case(res=128, n_views=2, base_freq=4, levels=2, seed=8):
    """The displacement workload shrunk for the oracle: a frequency-4 base
    icosphere (320 tris) split twice (5,120 tris), a 32^2 displacement map, a
    64^2 normal map, against a frequency-24 fBm reference."""
    c = synth.config_tess(ref_freq=24, base_freq=base_freq, levels=levels, disp_res=32, nrm_res=64, n_views=n_views,
                          res=res)
    rng = np.random.default_rng(seed)
    c["cand"].disp = rng.uniform(-0.03, 0.03, c["cand"].disp.shape).astype(np.float32)
    views = synth.sample_views(seed, 0, n_views, res, res, r_min=2.4, r_max=3.0)
    return c, views, res, res


def oracle_reference(scene, views, H, W):
    img, keys = S.render_reference(scene, views, H, W)
    return img.numpy().astype(np.float32), keys


def unambiguous_inputs(scene, views, refs, H, W, loss, texel_margin=2e-6, tries=16):
    """The candidate scene with its UV corners shifted by (k, k) 1e-3 for the first
    k at which no texture lookup of the oracle's render lies within `texel_margin`
    texel of a bilinear cell boundary (u wraps; v clamps at the poles on both
    sides alike), and the references with the L1 kinks of that render removed
    (unkinked_reference).

    A lookup that close to a cell boundary has no unique uv-derivative at float32
    resolution (the float32 texture coordinate carries up to ~1e-6 texel of
    rounding on these cases): the GPU and the float64 oracle may take different
    one-sided derivatives there, both valid. On the returned inputs every such
    decision is the same at either precision, so gradients can be compared as
    whole vectors."""
    import dataclasses

    for k in range(tries):
        mesh = scene.mesh
        uv = mesh.uv.copy()
        uv += np.float32(k * 1e-3)
        sc = dataclasses.replace(scene, mesh=dataclasses.replace(mesh, uv=uv))
        job = S.OracleJob(sc, loss=loss)
        diags = []
        with torch.no_grad():
            S.render(job, job.params, views, H, W, diags=diags)
        if min(float(dg["texel_margin"].min()) for dg in diags if len(dg["texel_margin"])) > texel_margin:
            return sc, unkinked_reference(sc, views, refs, H, W, loss)
    raise AssertionError("no u shift keeps every lookup away from the cell boundaries")


def unkinked_reference(scene, views, refs, H, W, loss, step=1e-3):
    """The reference images with every channel whose loss residual against the
    oracle's candidate image x lies within LOSS_MARGIN of the L1 kink set to
    x - step (x + step where that would be negative): `step` away from x in
    radiance, so that the residual's sign is the same at float32 and float64.

    At such a channel |f(x) - f(y)| has no unique derivative at float32
    resolution: the GPU's float32 image and the oracle's float64 one can fall on
    opposite sides, and a whole-vector gradient comparison would mix two valid
    subgradients. Both sides are then run on these references. L2 has no kink:
    refs are returned as is."""
    from oracle import render as R

    refs = np.array(refs, dtype=np.float32, copy=True)
    if loss == "l2":
        return refs
    job = S.OracleJob(scene, loss=loss)
    with torch.no_grad():
        img = S.render(job, job.params, views, H, W)["img"].numpy()
    x, y = torch.as_tensor(img), torch.as_tensor(refs.astype(np.float64))
    if loss == "logl1":
        x, y = R.tonemap(x), R.tonemap(y)
    r = (x - y).numpy()
    close = (np.abs(r) < LOSS_MARGIN) & (r != 0)
    below = img - step
    refs[close] = np.where(below[close] >= 0, below[close], img[close] + step).astype(np.float32)
    return refs


def chain_levels(chain, h, w, levels):
    """Split a texture's mip chain (total_texels, 4), level after level, into
    per-level (h_k, w_k, 4) arrays."""
    out, off = [], 0
    for k in range(levels):
        hk, wk = max(h >> k, 1), max(w >> k, 1)
        out.append(chain[off: off + hk * wk].reshape(hk, wk, 4))
        off += hk * wk
    return out


def fold_mips(g, h, w, levels):
    """Level-0 gradient of a texture from the gradients of its whole mip chain.

    g: (total_texels, 4) laid out level after level; each level-k texel is the
    mean of its 2^k x 2^k level-0 texels (square power-of-two textures)."""
    out = g[: h * w].reshape(h, w, 4).double().clone()
    off = h * w
    for k in range(1, levels):
        hk, wk = max(h >> k, 1), max(w >> k, 1)
        lv = g[off: off + hk * wk].reshape(hk, wk, 4).double()
        out += lv.repeat_interleave(h // hk, 0).repeat_interleave(w // wk, 1) / float((h // hk) * (w // wk))
        off += hk * wk
    return out


def oracle_grads(scene, views, refs, H, W, loss, per_level=False, skin_weights=None, bones=None, msaa=1, layers=0):
    """Oracle image-loss gradients (lambda = 0), images, keys, loss, and the
    vertices whose gradient is not unique at float32 resolution. msaa = s > 1:
    keys on the s x s sample grid, images per pixel. layers = L: depth-peeled,
    keys (B, L, H, W)."""
    job = S.OracleJob(scene, loss=loss, per_level=per_level, skin_weights=skin_weights, msaa=msaa, layers=layers)
    if bones is not None:
        job.bones = torch.as_tensor(np.asarray(bones, dtype=np.float64))
        job.shade_f32_skin = True   # the GPU shades the float32 skinned positions it renders
    params = {k: v.clone().requires_grad_(job.optimize[k]) for k, v in job.params.items()}
    diags = []
    obj = S.objective(job, params, views, torch.as_tensor(refs.astype(np.float64)), H, W, lam=0.0, diags=diags)
    live = [k for k in params if job.optimize[k]]
    grads = dict(zip(live, [g.detach().numpy() for g in torch.autograd.grad(obj["total"], [params[k] for k in live])]))
    img = obj["out"]["img"].detach().numpy()
    if layers:
        amb = _peeled_ambiguous(job, diags, obj["out"]["keys"], img, refs, H, W)
    elif job.tess is None:
        amb = ambiguous_vertices(diags, obj["out"]["keys"], img, refs, job.tri_np, loss, sub=max(msaa, 1))
    else:
        # render vertices -> the base vertices they are interpolated from
        amb_r = ambiguous_vertices(diags, obj["out"]["keys"], img, refs, job.tess.tri, loss)
        base = set()
        for v in amb_r:
            base |= set(job.tess.base_idx[v].tolist())
        amb = base
    return dict(grads=grads, img=img, pre=obj["out"]["pre"].detach().numpy(), keys=obj["out"]["keys"],
                loss=float(obj["image"].detach()), ambiguous=amb)


def _peeled_ambiguous(job, diags, keys, img, refs, H, W):
    # every layer of every view is checked like a view of its own
    L = job.layers
    flat = [dg["layers"][l] for dg in diags for l in range(L)]
    return ambiguous_vertices(flat, keys.reshape(-1, H, W), np.repeat(np.asarray(img), L, axis=0),
                              np.repeat(np.asarray(refs), L, axis=0), job.tri_np, job.loss)


def oracle_ambiguous(job, views, refs, H, W):
    """The vertices whose gradient is one-sided (ambiguous_vertices) at an
    oracle job's current parameters, for a plain (untessellated) mesh."""
    params = {k: v.detach() for k, v in job.params.items()}
    diags = []
    with torch.no_grad():
        obj = S.objective(job, params, views, torch.as_tensor(np.asarray(refs, dtype=np.float64)), H, W, lam=0.0,
                          diags=diags)
    if job.layers:
        return _peeled_ambiguous(job, diags, obj["out"]["keys"], obj["out"]["img"].numpy(), refs, H, W)
    return ambiguous_vertices(diags, obj["out"]["keys"], obj["out"]["img"].numpy(), refs, job.tri_np, job.loss,
                              sub=max(job.msaa, 1))


# Margins to the discrete decisions inside the differentiable path. The CUDA
# path evaluates texel coordinates to ~1e-6 texels and screen positions to
# ~1e-6 pixels, so a lookup or crossing farther than these margins from its
# boundary takes the same side on both sides of the comparison.
TEXEL_MARGIN = 5e-5   # texels: bilinear cell boundary (uv-derivative is one-sided there)
NL_MARGIN = 1e-5      # n.l = 0: a light switches on or off
AA_MARGIN = 1e-4      # pixels: silhouette crossing tests and tau = 1/2
LOSS_MARGIN = 1e-5    # |f(x) - f(y)|: sign of the L1 residual


def ambiguous_vertices(diags, keys, img, refs, tri, loss, sub=1):
    """Vertices touched by pixels within a margin of a kink of the forward.

    At such a pixel the forward is continuous but its derivative is one-sided,
    and the float32 kernel may legitimately take the other side: the gradient
    is not unique there, so parity tests compare the other vertices exactly
    and these only for validity. sub = s > 1: keys and margins on the s x s sample
    grid, images per pixel (a pixel near an L1 kink marks all its samples)."""
    from oracle import render as R

    tri = np.asarray(tri)
    verts = set()
    for b, dg in enumerate(diags):
        if not dg:
            continue
        kb = keys[b]
        tid = np.where(kb == np.uint64(R.EMPTY), -1, (kb & np.uint64(0xFFFFFFFF)).astype(np.int64)).reshape(-1)
        bad = set(dg["tri"][(dg["texel_margin"] < TEXEL_MARGIN) | (dg["nl_margin"] < NL_MARGIN)].tolist())
        for o, s, m in dg.get("aa_pairs", []):
            sel = m < AA_MARGIN
            bad |= set(tid[o[sel]].tolist()) | set(tid[s[sel]].tolist())
        x = torch.as_tensor(img[b].astype(np.float64))
        y = torch.as_tensor(np.asarray(refs[b], dtype=np.float64))
        if loss == "logl1":
            x, y = R.tonemap(x), R.tonemap(y)
        close = ((x - y).abs() < LOSS_MARGIN).any(dim=2).numpy() & ((x - y).abs().sum(dim=2) > 0).numpy()
        if loss == "l2":   # a smooth loss: no sign kink
            close[:] = False
        if sub > 1:
            close = np.repeat(np.repeat(close, sub, axis=0), sub, axis=1)
        H, W = close.shape
        for j, i in zip(*np.nonzero(close)):
            for dj, di in ((0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)):
                jj, ii = j + dj, i + di
                if 0 <= jj < H and 0 <= ii < W:
                    bad.add(int(tid[jj * W + ii]))
        bad.discard(-1)
        for f in bad:
            verts |= set(tri[f].tolist())
    return verts


def assert_grads_match(got, orc, label, tol=1e-3):
    """Per latent within `tol` relative L2 of the oracle. Vertex gradients touched
    by a pixel sitting on a kink of the forward (texel-cell boundary, n.l = 0, AA
    crossing thresholds, L1 sign) are one-sided and not unique: those vertices
    are additionally held to a validity bar (each within 50% of the oracle's
    one-sided value). The whole vector, those vertices included, is held to
    `tol`, and so is the vector of all other vertices."""
    for name, want in orc["grads"].items():
        g = got[name]
        assert np.linalg.norm(want) > 0, name
        if name in ("pos", "w"):   # rows per vertex (skinning weights: one row per vertex too)
            amb = np.zeros(len(want), bool)
            amb[sorted(orc["ambiguous"])] = True
            assert amb.mean() < 0.3, f"{label}: {amb.sum()} ambiguous vertices"
            err = rel_l2(g[~amb], want[~amb])
            print(f"{label} {name}: {amb.sum()} of {len(amb)} vertices one-sided; rel L2 of the rest {err:.3e}, "
                  f"of all {rel_l2(g, want):.3e}")
            for v in np.nonzero(amb)[0]:
                assert np.linalg.norm(g[v] - want[v]) <= 0.5 * np.linalg.norm(want[v]) + 1e-3 * np.abs(want).max()
            assert rel_l2(g, want) < tol, f"{label} {name}: rel L2 of all vertices {rel_l2(g, want):.3e}"
        else:
            err = rel_l2(g, want)
        assert err < tol, f"{label} {name}: rel L2 {err:.3e}"
