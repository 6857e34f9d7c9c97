"""Per-stage torch.autograd.Functions over the library's per-stage C calls.

The render-and-compare step as a chain of differentiable primitives (Sec. 5.2
builds the renderer from a rasterizer, attribute interpolation, filtered
texture lookups and an antialiasing pass; Sec. 3 differentiates the image loss
through all of them), each Function's backward one hand-written adjoint call of
libadms.so:

    Tess     base positions, displacement map -> render positions    adms_tess_fwd / _bwd (+ base frame)
    Frame    positions -> (positions, unit normals, unit tangents)   adms_frame_fwd / _bwd
    Setup    positions -> clip coordinates                           adms_setup_fwd / _bwd
    Raster   clip -> barycentrics (keys, LOD derivatives alongside)  adms_raster_fwd / _bwd
    Shade    barycentrics, vertex attributes, mip chains -> colour   adms_shade_fwd / _bwd
    AALoss   colour, clip, reference -> image loss                   adms_aa_loss_fwd / _bwd
    MipChain level 0 -> whole mip chain                              adms_mip_fwd / _bwd

A Pipeline holds what the calls of one (mesh, views, image size) share: the
mesh topology, the device views, the workspace, and the non-differentiable
buffers (keys, LOD derivatives). With recompute=True the raster buffers are
not kept after the forward: the backward of AALoss (the first to run) rebuilds
keys, barycentrics, colours and dL/d(colour) from the saved positions,
attributes and textures. This module only allocates tensors and marshals
arguments; every step runs in the CUDA library.
"""

from __future__ import annotations

import numpy as np
import torch

from . import binding as B

LOSS = B.LOSS


def mip_levels(h, w):
    n = 1
    while max(h, w) >> (n - 1) > 1:
        n += 1
    return n


def chain_texels(h, w, levels):
    return sum(max(h >> k, 1) * max(w >> k, 1) for k in range(levels))


class Pipeline:
    """Shared state of the per-stage calls for one mesh under one batch of views."""

    def __init__(self, tri, uv, tri_uv, n_verts, views, H, W, device="cuda", list_entries=None, recompute=False):
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        adj, vf_off, vf_face = B.adms_mesh_topology(tri, n_verts)
        dev = torch.device(device)
        self.V, self.F = int(n_verts), int(tri.shape[0])
        self.tri = torch.as_tensor(tri, device=dev)
        self.tri_uv = torch.as_tensor(np.ascontiguousarray(tri_uv, dtype=np.int32), device=dev)
        self.uv = torch.as_tensor(np.ascontiguousarray(uv, dtype=np.float32), device=dev)
        self.adj = torch.as_tensor(adj, device=dev)
        self.vf_off = torch.as_tensor(vf_off, device=dev)
        self.vf_face = torch.as_tensor(vf_face, device=dev)
        self.set_views(views)
        self.H, self.W = int(H), int(W)
        entries = list_entries or max(8 * self.B * self.F, 1 << 16)
        nbytes = B.adms_stage_workspace_bytes(self.V, self.F, self.B, self.H, self.W, entries)
        if nbytes == 0:
            raise ValueError("invalid sizes for the per-stage workspace")
        self.work = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        assert self.work.data_ptr() % 256 == 0
        self.recompute = recompute
        self.keys = self.rast = self.rast_db = self.pre = self.gprime = None
        self.saved = None  # what the recompute needs: positions, attributes, mip chains, reference

    def set_views(self, views):
        """views: numpy records of synth views (adms_view layout) or a device uint8 tensor."""
        if isinstance(views, np.ndarray):
            self.B = len(views)
            self.views = torch.from_numpy(views.view(np.uint8).copy()).cuda()
        else:
            self.views = views
            self.B = views.numel() // 112

    def mesh(self, pos):
        return B.stage_mesh(pos.detach().contiguous(), self.uv, self.tri, self.tri_uv, self.adj, self.vf_off,
                            self.vf_face)

    def empty(self, *shape, dtype=torch.float32):
        return torch.empty(shape, dtype=dtype, device=self.work.device)

    def zeros(self, *shape, dtype=torch.float32):
        return torch.zeros(shape, dtype=dtype, device=self.work.device)

    # the raster buffers, rebuilt from the saved inputs (recompute mode)
    def rebuild(self):
        pos, vpos4, vnrm4, vtan4, maps, ref, kind, scale = self.saved
        m = self.mesh(pos)
        clip = self.empty(self.B, self.V, 4)
        B.adms_setup_fwd(m, self.views, self.B, self.H, self.W, clip, self.work)
        self.keys = self.empty(self.B, self.H, self.W, dtype=torch.int64)
        self.rast = self.empty(self.B, self.H, self.W, 2)
        self.rast_db = self.empty(self.B, self.H, self.W, 4)
        B.adms_raster_fwd(m, self.views, self.B, self.H, self.W, clip, self.keys, self.rast, self.rast_db, self.work)
        self.pre = self.empty(self.B, self.H, self.W, 4)
        B.adms_shade_fwd(m, self.views, self.B, self.H, self.W, self.keys, self.rast, self.rast_db, vpos4, vnrm4, vtan4,
                         B.stage_textures(maps), self.pre)
        self.gprime = self.empty(self.B, self.H, self.W, 4)
        loss = self.zeros(1, dtype=torch.float64)
        B.adms_aa_loss_fwd(m, self.views, self.B, self.H, self.W, clip, self.keys, self.pre, ref, kind, scale, None,
                           loss, self.gprime, self.work)
        return clip


def _tex_tuple(chain, h, w, levels, grad=None):
    return (chain.detach().contiguous(), grad, h, w, levels)


class Frame(torch.autograd.Function):
    """Sec. 5.1: (vpos4, vnrm4, vtan4) [V][4] of the positions."""

    @staticmethod
    def forward(fctx, pipe, pos):
        m = pipe.mesh(pos)
        out = [pipe.empty(pipe.V, 4) for _ in range(3)]
        B.adms_frame_fwd(m, *out)
        fctx.pipe, fctx.pos = pipe, pos.detach()
        return tuple(out)

    @staticmethod
    def backward(fctx, g_vpos4, g_vnrm4, g_vtan4):
        pipe = fctx.pipe
        g = [(t[:, :3] if t is not None else pipe.zeros(pipe.V, 3)).double().contiguous()
             for t in (g_vpos4, g_vnrm4, g_vtan4)]
        g_pos = pipe.zeros(pipe.V, 3)
        B.adms_frame_bwd(pipe.mesh(fctx.pos), g[0], g[1], g[2], g_pos, pipe.empty(2 * pipe.V, 4))
        return None, g_pos


class Setup(torch.autograd.Function):
    """Sec. 5.2 vertex transform: clip [B][V][4]; the triangle setup goes to the workspace."""

    @staticmethod
    def forward(fctx, pipe, pos):
        clip = pipe.empty(pipe.B, pipe.V, 4)
        B.adms_setup_fwd(pipe.mesh(pos), pipe.views, pipe.B, pipe.H, pipe.W, clip, pipe.work)
        fctx.pipe = pipe
        return clip

    @staticmethod
    def backward(fctx, g_clip):
        pipe = fctx.pipe
        g_pos = pipe.zeros(pipe.V, 3)
        B.adms_setup_bwd(pipe.views, pipe.B, pipe.V, g_clip.double().contiguous(), g_pos)
        return None, g_pos


class Raster(torch.autograd.Function):
    """Sec. 5.2 rasterization: barycentrics rast [B][H][W][2] (keys and LOD
    derivatives kept in the pipeline; keep_keys holds them fixed)."""

    @staticmethod
    def forward(fctx, pipe, pos, clip, keep_keys=False):
        if not keep_keys:
            pipe.keys = pipe.empty(pipe.B, pipe.H, pipe.W, dtype=torch.int64)
            pipe.rast_db = pipe.empty(pipe.B, pipe.H, pipe.W, 4)
        rast = pipe.empty(pipe.B, pipe.H, pipe.W, 2)
        B.adms_raster_fwd(pipe.mesh(pos), pipe.views, pipe.B, pipe.H, pipe.W, clip.detach().contiguous(), pipe.keys,
                          rast, pipe.rast_db, pipe.work, keep_keys=keep_keys)
        pipe.rast = rast.detach()
        fctx.pipe, fctx.pos, fctx.clip = pipe, pos.detach(), clip.detach()
        return rast

    @staticmethod
    def backward(fctx, g_rast):
        pipe = fctx.pipe
        g_clip = pipe.zeros(pipe.B, pipe.V, 4, dtype=torch.float64)
        B.adms_raster_bwd(pipe.mesh(fctx.pos), pipe.views, pipe.B, pipe.H, pipe.W, fctx.clip, pipe.keys,
                          g_rast.contiguous(), g_clip, pipe.work)
        return None, None, g_clip.float(), None


class Shade(torch.autograd.Function):
    """Sec. 5.2 shading: pre-AA colour [B][H][W][4] from the barycentrics, the
    vertex attributes and the three mip chains (base colour, (gamma, r, m), normal)."""

    @staticmethod
    def forward(fctx, pipe, pos, rast, vpos4, vnrm4, vtan4, dims, kd, orm, nrm):
        maps = [_tex_tuple(c, *d) for c, d in zip((kd, orm, nrm), dims)]
        pre = pipe.empty(pipe.B, pipe.H, pipe.W, 4)
        B.adms_shade_fwd(pipe.mesh(pos), pipe.views, pipe.B, pipe.H, pipe.W, pipe.keys, rast.detach().contiguous(),
                         pipe.rast_db, vpos4.detach(), vnrm4.detach(), vtan4.detach(), B.stage_textures(maps), pre)
        pipe.pre = pre.detach()
        fctx.pipe, fctx.pos, fctx.dims = pipe, pos.detach(), dims
        fctx.attrs = (vpos4.detach(), vnrm4.detach(), vtan4.detach())
        fctx.chains = (kd, orm, nrm)
        fctx.rast = None if pipe.recompute else rast.detach()
        return pre

    @staticmethod
    def backward(fctx, g_pre):
        pipe = fctx.pipe
        rast = fctx.rast if fctx.rast is not None else pipe.rast
        grads = [torch.zeros_like(c) if c.requires_grad else None for c in fctx.chains]
        maps = [_tex_tuple(c, *d, grad=g) for c, d, g in zip(fctx.chains, fctx.dims, grads)]
        gv = [pipe.zeros(pipe.V, 3, dtype=torch.float64) for _ in range(3)]
        g_rast = pipe.empty(pipe.B, pipe.H, pipe.W, 2)
        B.adms_shade_bwd(pipe.mesh(fctx.pos), pipe.views, pipe.B, pipe.H, pipe.W, pipe.keys, rast, pipe.rast_db,
                         *fctx.attrs, B.stage_textures(maps), g_pre.contiguous(), gv[0], gv[1], gv[2], g_rast)
        pad = [torch.nn.functional.pad(g.float(), (0, 1)) for g in gv]
        return (None, None, g_rast, pad[0], pad[1], pad[2], None, *grads)


class AALoss(torch.autograd.Function):
    """Sec. 5.2 silhouette antialiasing + Sec. 5.3 image loss (float64 scalar)."""

    @staticmethod
    def forward(fctx, pipe, pos, pre, clip, ref, kind, scale):
        loss = pipe.zeros(1, dtype=torch.float64)
        gprime = pipe.empty(pipe.B, pipe.H, pipe.W, 4)
        B.adms_aa_loss_fwd(pipe.mesh(pos), pipe.views, pipe.B, pipe.H, pipe.W, clip.detach().contiguous(), pipe.keys,
                           pre.detach().contiguous(), ref, LOSS[kind], scale, None, loss, gprime, pipe.work)
        fctx.pipe, fctx.pos, fctx.clip = pipe, pos.detach(), clip.detach()
        if pipe.recompute:
            # drop the raster buffers; AALoss.backward rebuilds them
            pipe.keys = pipe.rast = pipe.rast_db = pipe.pre = pipe.gprime = None
            fctx.pre = fctx.gprime = None
        else:
            fctx.pre, fctx.gprime = pre.detach(), gprime
        return loss[0]   # float64: the per-pixel terms are summed in float64

    @staticmethod
    def backward(fctx, g_loss):
        pipe = fctx.pipe
        if pipe.recompute:
            clip = pipe.rebuild()
            pre, gprime = pipe.pre, pipe.gprime
        else:
            clip, pre, gprime = fctx.clip, fctx.pre, fctx.gprime
        g_pre = pipe.empty(pipe.B, pipe.H, pipe.W, 4)
        g_clip = pipe.zeros(pipe.B, pipe.V, 4, dtype=torch.float64)
        B.adms_aa_loss_bwd(pipe.mesh(fctx.pos), pipe.views, pipe.B, pipe.H, pipe.W, clip, pipe.keys, pre, gprime,
                           g_loss.reshape(1).float().contiguous(), g_pre, g_clip, pipe.work)
        return None, None, g_pre, g_clip.float(), None, None, None


class TessMesh:
    """A base mesh split `levels` times (Sec. 5.1): the render mesh's topology and
    UVs, and the tables the displacement stage reads."""

    def __init__(self, tri, tri_uv, uv, n_verts, levels, device="cuda"):
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        tab = B.adms_tessellation(tri, tri_uv, uv, n_verts, levels)
        _, bvf_off, bvf_face = B.adms_mesh_topology(tri, n_verts)
        dev = torch.device(device)
        t = lambda a: torch.as_tensor(a, device=dev)   # noqa: E731
        self.Vb, self.Fb, self.Vt, self.n_seg = int(n_verts), int(tri.shape[0]), int(tab["owner"].shape[0]), 1 << levels
        self.rtri, self.rtri_uv, self.ruv = tab["rtri"], tab["rtri_uv"], tab["ruv"]
        self.dev = dict(base_tri=t(tri), bvf_off=t(bvf_off), bvf_face=t(bvf_face), owner=t(tab["owner"]),
                        wts=t(tab["wts"]), vert_uv=t(tab["vert_uv"]))
        self.desc = B.tess_desc(self.Vb, self.Fb, self.Vt, self.n_seg, **self.dev)
        # the base mesh as a stage mesh: its frame adjoint takes the base normals' gradient
        self.base_uv = t(np.ascontiguousarray(uv, dtype=np.float32))
        self.base_tri_uv = t(np.ascontiguousarray(tri_uv, dtype=np.int32))
        self.base_adj = t(np.full((self.Fb, 3), -1, np.int32))

    def base_mesh(self, base_pos):
        return B.stage_mesh(base_pos, self.base_uv, self.dev["base_tri"], self.base_tri_uv, self.base_adj,
                            self.dev["bvf_off"], self.dev["bvf_face"])


class Tess(torch.autograd.Function):
    """Sec. 5.1, Eq. 3: render positions [Vt][3] from base positions and the
    displacement map [dh][dw]; backward through the displacement lookup, the
    lattice interpolation and the smooth base normals."""

    @staticmethod
    def forward(fctx, tm, base_pos, disp):
        bp, d = base_pos.detach().contiguous(), disp.detach().contiguous()
        base_nrm = torch.empty(tm.Vb, 3, dtype=torch.float32, device=bp.device)
        pos = torch.empty(tm.Vt, 3, dtype=torch.float32, device=bp.device)
        B.adms_tess_fwd(tm.desc, bp, d, base_nrm, pos)
        fctx.tm, fctx.bp, fctx.d, fctx.nrm = tm, bp, d, base_nrm
        return pos

    @staticmethod
    def backward(fctx, g_pos):
        tm, bp = fctx.tm, fctx.bp
        g_bpos = torch.zeros(tm.Vb, 3, dtype=torch.float64, device=bp.device)
        g_bnrm = torch.zeros(tm.Vb, 3, dtype=torch.float64, device=bp.device)
        g_disp = torch.zeros_like(fctx.d)
        B.adms_tess_bwd(tm.desc, bp, fctx.nrm, fctx.d, g_pos.contiguous(), g_bpos, g_bnrm, g_disp)
        g_base = torch.zeros(tm.Vb, 3, dtype=torch.float32, device=bp.device)
        B.adms_frame_bwd(tm.base_mesh(bp), g_bpos, g_bnrm, torch.zeros_like(g_bnrm), g_base,
                         torch.empty(2 * tm.Vb, 4, device=bp.device))
        return None, g_base, g_disp


class MipChain(torch.autograd.Function):
    """Sec. 5.2 filtered lookups: level 0 [h][w][4] -> the whole mip chain (texels x 4)."""

    @staticmethod
    def forward(fctx, tex0):
        h, w = tex0.shape[0], tex0.shape[1]
        levels = mip_levels(h, w)
        chain = torch.empty(chain_texels(h, w, levels), 4, dtype=torch.float32, device=tex0.device)
        chain[: h * w] = tex0.reshape(h * w, 4)
        B.adms_mip_fwd(chain, h, w, levels)
        fctx.dims = (h, w, levels)
        return chain

    @staticmethod
    def backward(fctx, g_chain):
        h, w, levels = fctx.dims
        g0 = torch.empty(h, w, 4, dtype=torch.float32, device=g_chain.device)
        B.adms_mip_bwd(g_chain.contiguous(), h, w, levels, g0)
        return g0


def render_loss(pipe, pos, kd, orm, nrm, ref, kind="logl1", mips=True, keep_keys=False):
    """L_image of one batch (Sec. 5.3) through the chained stage Functions.

    pos [V][3]; kd, orm, nrm level-0 textures [h][w][4] (mip chains built here
    when mips, else level 0 only); ref [B][H][W][3]. keep_keys reuses the
    pipeline's keys and LOD derivatives (visibility and LOD held fixed)."""
    chains, dims = [], []
    for t in (kd, orm, nrm):
        h, w = t.shape[0], t.shape[1]
        if mips:
            chains.append(MipChain.apply(t))
            dims.append((h, w, mip_levels(h, w)))
        else:
            chains.append(t.reshape(h * w, 4))
            dims.append((h, w, 1))
    vpos4, vnrm4, vtan4 = Frame.apply(pipe, pos)
    clip = Setup.apply(pipe, pos)
    rast = Raster.apply(pipe, pos, clip, keep_keys)
    pre = Shade.apply(pipe, pos, rast, vpos4, vnrm4, vtan4, tuple(dims), *chains)
    scale = 1.0 / (3.0 * pipe.B * pipe.H * pipe.W)
    ref = ref.contiguous()
    pipe.saved = (pos.detach(), vpos4.detach(), vnrm4.detach(), vtan4.detach(),
                  [_tex_tuple(c, *d) for c, d in zip(chains, dims)], ref, LOSS[kind], scale)
    return AALoss.apply(pipe, pos, pre, clip, ref, kind, scale)
