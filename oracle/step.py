"""Oracle of one full optimization step (TEST INFRASTRUCTURE ONLY).

Eq. 1 (empirical risk over random views) sampled with one batch of views:
render the latent mesh (Sec. 5.1-5.2), compare with the reference images
(Sec. 5.3 loss), add the Laplacian term with the lambda schedule (Eq. 4, 5),
differentiate, and apply Adam with the learning-rate schedule (Sec. 5.3).
"""

from __future__ import annotations

import numpy as np
import torch

from . import render as R
from . import visibility
from . import skinning as SK
from . import tessellate as TS

F64 = torch.float64
LATENTS = ("pos", "kd", "orm", "nrm", "disp")


class OracleJob:
    """Latent state of one simplification job in float64.

    scene: synth.Scene. Textures are (h, w, 4); `disp` (h, w) when present."""

    def __init__(self, scene, loss="logl1", lr0=0.01, lam0=None, relative_laplacian=False, per_level=False,
                 skin_weights=None, skin_lr_scale=1.0, msaa=1, layers=0):
        m = scene.mesh
        self.tri = torch.as_tensor(m.tri_pos.astype(np.int64))
        self.tri_uv = torch.as_tensor(m.tri_uv.astype(np.int64))
        self.uv = torch.as_tensor(m.uv.astype(np.float64))
        self.tri_np = m.tri_pos.astype(np.int64)
        self.params = {
            "pos": torch.as_tensor(m.pos.astype(np.float64)),
            "kd": torch.as_tensor(scene.kd.astype(np.float64)),
            "orm": torch.as_tensor(scene.orm.astype(np.float64)),
            "nrm": torch.as_tensor(scene.nrm.astype(np.float64)),
        }
        if scene.disp is not None:
            self.params["disp"] = torch.as_tensor(scene.disp.astype(np.float64))
        self.tess_levels = int(scene.tess_levels)
        self.msaa = int(msaa)   # s x s visibility samples per pixel, shaded once per pixel (Sec. 5.2)
        # layers = L >= 1: transparency by L depth-peeling passes, opacity from the
        # base colour's fourth channel (Sec. 5.2, 6); 0: opaque, alpha unused
        self.layers = int(layers)
        if self.layers and self.msaa > 1:
            raise ValueError("depth peeling with multisampling is not supported")
        self.mips = bool(scene.mips)
        self.optimize = {k: bool(scene.optimize.get(k, False)) for k in self.params}
        # Per-level latent textures (the prefiltering variant of Sec. 6): every mip
        # level of an optimized texture is its own latent "name@k" (k >= 1), starting
        # from the box-filter chain of the given level 0 (reading: the paper does not
        # say how the levels start)
        # Skinning (Eq. 2): dense weights (V, B) are a latent "w"; the bone matrices of
        # the frame being rendered are set per step in self.bones (B, 4, 4)
        self.bones = None
        # True: shade the float32 skinned positions that visibility (and the GPU) use,
        # differentiated through the float64 operator; False: shade the float64 ones
        self.shade_f32_skin = False
        if skin_weights is not None:
            w = torch.as_tensor(np.asarray(skin_weights, dtype=np.float64))
            self.params["w"] = w
            self.optimize["w"] = skin_lr_scale > 0
            self.bones = torch.eye(4, dtype=torch.float64).repeat(w.shape[1], 1, 1)
        # learning-rate factor per latent (the weights' own; the rest take lr_t)
        self.lr_scale = {"w": float(skin_lr_scale)}
        self.per_level = bool(per_level) and self.mips
        if self.per_level:
            for name in ("kd", "orm", "nrm"):
                if not self.optimize[name]:
                    continue
                chain = R.mip_chain(self.params[name])
                for k in range(1, len(chain)):
                    self.params[f"{name}@{k}"] = chain[k].detach().clone()
                    self.optimize[f"{name}@{k}"] = True
        self.loss = loss
        self.lr0 = float(lr0)
        self.lam0_user = lam0
        self.lam0 = None
        self.lam = None
        self.t = 0
        self.m = {k: torch.zeros_like(v) for k, v in self.params.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.params.items()}
        self.ring = R.one_ring(self.tri_np, m.pos.shape[0])
        self.delta_ref = R.laplacian_delta(self.params["pos"], self.ring) if relative_laplacian else None
        if self.tess_levels > 0:
            self.tess = TS.Tessellation(self.tri_np, m.tri_uv.astype(np.int64), m.uv.astype(np.float64),
                                        self.tess_levels)
            self.adj = R.edge_adjacency(self.tess.tri)
        else:
            self.tess = None
            self.adj = R.edge_adjacency(self.tri_np)


def geometry(job, params):
    """Render mesh: positions (tessellated + displaced if the job has levels),
    smooth normals and tangents (Sec. 5.1)."""
    if job.tess is None:
        pos, tri, uv, tri_uv = params["pos"], job.tri, job.uv, job.tri_uv
        if job.bones is not None:
            pos = SK.skin(pos, params["w"], job.bones)
            if job.shade_f32_skin:
                p32 = visibility.skin_positions_f32(params["pos"].detach().numpy(), params["w"].detach().numpy(),
                                                    job.bones.numpy())
                pos = pos + (torch.as_tensor(p32.astype(np.float64)) - pos).detach()
    else:
        base_n = R.vertex_normals(params["pos"], job.tri)
        pos = job.tess.displaced_positions(params["pos"], base_n, params["disp"])
        tri = torch.as_tensor(job.tess.tri)
        uv = torch.as_tensor(job.tess.corner_uv)
        tri_uv = torch.as_tensor(job.tess.tri_uv)
    return dict(pos=pos, tri=tri, uv=uv, tri_uv=tri_uv,
                nrm=R.vertex_normals(pos, tri), tan=R.vertex_tangents(pos, uv, tri, tri_uv))


def texture_levels(job, params):
    out = {}
    for name in ("kd", "orm", "nrm"):
        if job.per_level and f"{name}@1" in params:
            n = 1 + sum(1 for k in params if k.startswith(name + "@"))
            out[name] = [params[name]] + [params[f"{name}@{k}"] for k in range(1, n)]
        else:
            out[name] = R.mip_chain(params[name]) if job.mips else [params[name]]
    return out


def render(job, params, views, height, width, aa=True, vis=None, lods=None, diags=None, ssaa=1):
    """Images of a batch of views. vis = (keys, asign) holds visibility fixed;
    lods = a dict filled on first use and reused after it holds the LOD fixed;
    diags = a list that receives each view's decision margins (render_view).
    With job.msaa = s > 1 visibility, pre-AA colours and antialiasing are on the
    s x s sample grid (keys, pre and img_samples at (s height, s width)) and img
    is their per-pixel mean; ssaa = s > 1 does the same but shades every sample
    at its own position (a supersampled render, for references)."""
    s = job.msaa if job.msaa > 1 else ssaa
    if s > 1:
        height, width = height * s, width * s
    geo = geometry(job, params)
    tex = texture_levels(job, params)
    if job.layers:
        if s > 1:
            raise ValueError("depth peeling with supersampling is not supported")
        return _render_peeled(job, geo, tex, views, height, width, aa, vis, lods, diags)
    if vis is None:
        if job.bones is not None:   # float32 contract of the skinned positions (raster.c)
            pos32 = visibility.skin_positions_f32(params["pos"].detach().numpy(), params["w"].detach().numpy(),
                                                  job.bones.numpy())
        elif job.tess is None:
            pos32 = geo["pos"].detach().numpy().astype(np.float32)
        else:   # float32 contract of the displaced positions (raster.c)
            pos32 = job.tess.positions_f32(params["pos"].detach().numpy(), job.tri_np,
                                           params["disp"].detach().numpy())
        vis = visibility.raster_views(views, pos32, geo["tri"].numpy(), width, height)
    keys, asign = vis
    pres, imgs = [], []
    for b in range(len(views)):
        store = None if lods is None else lods.setdefault(b, {})
        dg = None if diags is None else {}
        pre, img = R.render_view(geo, tex, views[b], keys[b], asign[b], job.adj, width, height, aa=aa,
                                 lod_store=store, diag=dg, msaa=job.msaa)
        if diags is not None:
            diags.append(dg)
        pres.append(pre)
        imgs.append(img)
    samples = torch.stack(imgs)
    img = torch.stack([R.resolve(x, s) for x in imgs]) if s > 1 else samples
    return dict(pre=torch.stack(pres), img=img, img_samples=samples, keys=keys, asign=asign, geo=geo)


def _render_peeled(job, geo, tex, views, height, width, aa, vis, lods, diags):
    """render() of a depth-peeled job: keys (B, L, H, W), layer 0's colours as pre."""
    if vis is None:
        pos32 = geo["pos"].detach().numpy().astype(np.float32)
        if job.tess is not None or job.bones is not None:
            raise ValueError("depth peeling runs on plain meshes")
        vis = visibility.raster_views_peeled(views, pos32, geo["tri"].numpy(), width, height, job.layers)
    keys, asign = vis
    pres, imgs = [], []
    for b in range(len(views)):
        store = None if lods is None else lods.setdefault(b, {})
        dg = None if diags is None else {}
        pre, img = R.peel_view(geo, tex, views[b], keys[b], asign[b], job.adj, width, height, aa=aa,
                               lod_store=store, diag=dg)
        if diags is not None:
            diags.append(dg)
        pres.append(pre)
        imgs.append(img)
    img = torch.stack(imgs)
    return dict(pre=torch.stack(pres), img=img, img_samples=img, keys=keys, asign=asign, geo=geo)


def render_reference(scene, views, height, width, ssaa=1):
    """Reference images (forward only; the reference is a black box, Sec. 3);
    ssaa = s > 1 renders s x s shaded samples per pixel and averages them."""
    job = OracleJob(scene, loss="l1")
    with torch.no_grad():
        out = render(job, job.params, views, height, width, ssaa=ssaa)
    return out["img"], out["keys"]


def objective(job, params, views, refs, height, width, vis=None, lam=None, lods=None, diags=None):
    """L_opt = L_image + lambda_t L_delta (Eq. 5) for one batch; returns parts."""
    out = render(job, params, views, height, width, vis=vis, lods=lods, diags=diags)
    l_img = R.image_loss(out["img"], refs, job.loss)
    total = l_img
    l_lap = torch.zeros((), dtype=F64)
    if job.optimize.get("pos", False):
        l_lap = R.laplacian_loss(params["pos"], job.ring, job.delta_ref)
        if lam is None:
            lam = current_lambda(job, float(l_img.detach()), float(l_lap.detach()))
        total = l_img + lam * l_lap
    return dict(total=total, image=l_img, laplacian=l_lap, lam=lam, out=out)


def current_lambda(job, l_img, l_lap):
    """lambda_0 = 0.25 L_image / L_delta at t = 0 unless user-given; then Eq. 5."""
    if job.t == 0:
        if job.lam0_user is not None:
            return float(job.lam0_user)
        if l_lap == 0.0:
            raise ValueError("lambda_0 heuristic needs L_delta > 0; give lambda_0")
        return 0.25 * l_img / l_lap
    return R.lambda_schedule(job.lam, job.lam0, job.t)


def step(job, views, refs, height, width):
    """One forward + backward + Adam step. Returns a dict with the visibility,
    images, losses, gradients (before the update) and the updated latents."""
    params = {k: v.clone().requires_grad_(job.optimize[k]) for k, v in job.params.items()}
    refs = torch.as_tensor(np.asarray(refs, dtype=np.float64))
    obj = objective(job, params, views, refs, height, width)
    live = [k for k in params if job.optimize[k]]
    grads = dict(zip(live, torch.autograd.grad(obj["total"], [params[k] for k in live], allow_unused=True)))
    grads = {k: (g if g is not None else torch.zeros_like(params[k])) for k, g in grads.items()}
    if job.t == 0:
        job.lam0 = obj["lam"]
    job.lam = obj["lam"]
    lr = R.learning_rate(job.lr0, job.t)
    for k in live:
        job.params[k], job.m[k], job.v[k] = R.adam_update(job.params[k], grads[k], job.m[k], job.v[k], job.t,
                                                          lr * job.lr_scale.get(k, 1.0), k)
    job.t += 1
    return dict(keys=obj["out"]["keys"], asign=obj["out"]["asign"], pre=obj["out"]["pre"].detach(),
                img=obj["out"]["img"].detach(), loss=float(obj["total"].detach()), image_loss=float(obj["image"].detach()),
                laplacian=float(obj["laplacian"].detach() if torch.is_tensor(obj["laplacian"]) else obj["laplacian"]), lam=obj["lam"], grads=grads, lr=lr)
