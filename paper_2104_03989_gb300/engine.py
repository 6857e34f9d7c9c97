"""Python front of the C ABI: jobs built from arrays, torch views of job state.

Argument marshalling only; every step runs in libadms.so. Device buffers the
caller passes (reference images, outputs) are torch CUDA tensors.
"""

from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class _DevArray:
    """Exposes a raw device pointer through __cuda_array_interface__ so torch can wrap it."""

    def __init__(self, ptr, shape, typestr="<f4"):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def device_view(ptr, shape, dtype=torch.float32):
    """A torch tensor aliasing library-owned device memory (valid while the job lives)."""
    if not ptr:
        return None
    typestr = {torch.float32: "<f4", torch.int64: "<i8"}[dtype]
    return torch.as_tensor(_DevArray(ptr, shape, typestr), device="cuda")


def _c32(a, dtype):
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


class Context:
    """One adms context on the current CUDA device and a CUDA stream."""

    def __init__(self, hbm_budget_bytes=0, stream=None):
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = B.adms_ctx_create(hbm_budget_bytes, self.stream)
        self._keep = {}

    def close(self):
        if self.ctx:
            B.adms_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ jobs
    def create_job(self, scene, optimize=None, loss="logl1", lr0=0.01, lambda0=0.0, batch_views=0, aa=True,
                   relative_laplacian=False, frozen=False, seed=0, per_level_textures=False, samples=1,
                   shade_samples=False, layers=0, raster_direct_px=0, raster_depth_filter=False):
        """scene: object with .mesh (pos, uv, tri_pos, tri_uv), .kd, .orm, .nrm, .mips (numpy).
        per_level_textures: every mip level of each optimized texture is its own latent.
        samples: s x s samples per pixel (MSAA; shade_samples=True: supersampling).
        layers: depth-peeling passes of a transparent render (0: opaque).
        raster_direct_px: raster tuning, bbox samples up to which a triangle skips binning (0: 16).
        raster_depth_filter: raster tuning for dense clouds of small triangles (read before atomicMin)."""
        mesh, mat, opt, keep = self._descs(scene, optimize, loss, lr0, lambda0, batch_views, aa, relative_laplacian,
                                           frozen, per_level_textures, samples, shade_samples, layers,
                                           raster_direct_px, raster_depth_filter)
        return B.adms_job_create(self.ctx, mesh, mat, opt, seed)

    def export_job(self, job):
        """The job's resumable state as a uint8 numpy array (a checkpoint)."""
        return B.adms_job_export(self.ctx, job)

    def import_job(self, blob, scene, optimize=None, loss="logl1", lr0=0.01, lambda0=0.0, batch_views=0, aa=True,
                   relative_laplacian=False, frozen=False, per_level_textures=False, samples=1, shade_samples=False,
                   layers=0, raster_direct_px=0, raster_depth_filter=False):
        """A new job resumed from export_job's output; scene and options as given
        when the exported job was created."""
        mesh, mat, opt, keep = self._descs(scene, optimize, loss, lr0, lambda0, batch_views, aa, relative_laplacian,
                                           frozen, per_level_textures, samples, shade_samples, layers,
                                           raster_direct_px, raster_depth_filter)
        return B.adms_job_import(self.ctx, mesh, mat, opt, np.ascontiguousarray(blob, dtype=np.uint8))

    @staticmethod
    def _descs(scene, optimize, loss, lr0, lambda0, batch_views, aa, relative_laplacian, frozen, per_level_textures,
               samples=1, shade_samples=False, layers=0, raster_direct_px=0, raster_depth_filter=False):
        m = scene.mesh
        arrays = dict(pos=_c32(m.pos, np.float32), uv=_c32(m.uv, np.float32), tri=_c32(m.tri_pos, np.int32),
                      tri_uv=_c32(m.tri_uv, np.int32), kd=_c32(scene.kd, np.float32),
                      orm=_c32(scene.orm, np.float32), nrm=_c32(scene.nrm, np.float32))
        disp = getattr(scene, "disp", None)
        arrays["disp"] = None if disp is None else _c32(disp, np.float32)
        levels = int(getattr(scene, "tess_levels", 0))
        mesh = B.mesh_desc(arrays["pos"], arrays["uv"], arrays["tri"], arrays["tri_uv"])
        mat = B.material_desc(arrays["kd"], arrays["orm"], arrays["nrm"], arrays["disp"], getattr(scene, "mips", True))
        opt = None
        if not frozen or levels or samples > 1 or layers or raster_direct_px or raster_depth_filter:
            opt = B.opt_params(optimize if optimize is not None else getattr(scene, "optimize", {}), loss=loss,
                               tess_levels=levels, batch_views=batch_views, relative_laplacian=relative_laplacian,
                               aa=aa, lr0=lr0, lambda0=lambda0, per_level_textures=per_level_textures,
                               samples=samples, shade_samples=shade_samples, layers=layers,
                               raster_direct_px=raster_direct_px, raster_depth_filter=raster_depth_filter)
            if frozen:
                for k in ("optimize_pos", "optimize_kd", "optimize_orm", "optimize_nrm", "optimize_disp"):
                    setattr(opt, k, 0)
        return mesh, mat, opt, arrays

    def destroy_job(self, job):
        B.adms_job_destroy(self.ctx, job)

    def reserve(self, job, n_views, H, W):
        B.adms_job_reserve(self.ctx, job, n_views, H, W)

    def bytes_in_use(self):
        return B.adms_bytes_in_use(self.ctx)

    def params(self, job):
        """torch views of a job's latents and gradients (level 0 of textures)."""
        pv = B.adms_job_params(self.ctx, job)
        V = pv.n_verts
        out = {"t": pv.t}
        out["pos"] = device_view(pv.pos, (V, 3))
        out["g_pos"] = device_view(pv.g_pos, (V, 3))
        for name in ("kd", "orm", "nrm"):
            h, w, L = getattr(pv, name + "_h"), getattr(pv, name + "_w"), getattr(pv, name + "_levels")
            total = sum(max(h >> k, 1) * max(w >> k, 1) for k in range(L))
            out[name] = device_view(getattr(pv, name), (h, w, 4))
            out[name + "_chain"] = device_view(getattr(pv, name), (total, 4))
            out["g_" + name] = device_view(getattr(pv, "g_" + name), (h, w, 4))
            out["g_" + name + "_chain"] = device_view(getattr(pv, "g_" + name), (total, 4))
            out[name + "_levels"] = L
        if pv.disp:
            out["disp"] = device_view(pv.disp, (pv.disp_h, pv.disp_w))
            out["g_disp"] = device_view(pv.g_disp, (pv.disp_h, pv.disp_w))
        if pv.n_bones:
            out["w"] = device_view(pv.skin_w, (V, pv.n_bones))
            out["g_w"] = device_view(pv.g_skin_w, (V, pv.n_bones))
        return out

    def skinning(self, job, weights, lr_scale=1.0):
        """Dense skinning (Eq. 2) of the job's rest positions; weights (V, B),
        optimized with learning rate lr_t * lr_scale (0: fixed)."""
        w = _c32(weights, np.float32)
        B.adms_job_skinning(self.ctx, job, w, w.shape[1], lr_scale)

    def set_bones(self, job, bones):
        """The frame's bone matrices (B, 4, 4): numpy (copied) or a CUDA tensor."""
        b = bones if isinstance(bones, torch.Tensor) else _c32(bones, np.float32)
        B.adms_job_set_bones(self.ctx, job, b)

    def jobs_status(self, jobs):
        """Device int32 tensor of each job's latched status (0 or an adms status), stream-ordered."""
        out = torch.empty(len(jobs), dtype=torch.int32, device="cuda")
        B.adms_jobs_status(self.ctx, list(jobs), out)
        return out

    def stats(self, job):
        s = B.adms_job_stats(self.ctx, job)
        return dict(image_loss=s.image_loss, laplacian=s.laplacian, lam=s.lambda_, lr=s.lr, t=s.t,
                    status=s.status, tile_overflows=s.tile_overflows, call_loss=s.call_loss)

    # ------------------------------------------------------------------ the step
    @staticmethod
    def _views(views):
        if isinstance(views, torch.Tensor):
            return views
        return np.ascontiguousarray(views)

    def render_reference(self, job, views, H, W, out=None):
        views = self._views(views)
        n = len(views)
        if out is None:
            out = torch.empty((n, H, W, 3), dtype=torch.float32, device="cuda")
        B.adms_render_reference(self.ctx, job, views, H, W, out)
        return out

    def forward_loss(self, jobs, views_list, refs, out_img=None, out_loss=None):
        """jobs: list of handles; views_list: list of view arrays; refs: list of (B, H, W, 3) CUDA tensors."""
        views = np.ascontiguousarray(np.concatenate([np.asarray(v) for v in views_list])) \
            if not isinstance(views_list[0], torch.Tensor) else torch.cat(list(views_list))
        vpj = [len(v) for v in views_list]
        hw = [(int(r.shape[1]), int(r.shape[2])) for r in refs]
        if out_loss is None:
            out_loss = torch.zeros(len(jobs), dtype=torch.float32, device="cuda")
        B.adms_forward_loss(self.ctx, list(jobs), views, vpj, hw, refs, out_loss, out_img)
        self._keep["fwd"] = (views, refs)
        return out_loss

    def backward(self, jobs, recompute_raster=False):
        B.adms_backward(self.ctx, list(jobs), int(recompute_raster))

    def step(self, jobs):
        B.adms_optimizer_step(self.ctx, list(jobs))

    def keys(self, job, shape):
        out = torch.empty(shape, dtype=torch.int64, device="cuda")
        B.adms_job_keys(self.ctx, job, out)
        return out

    def set_stream(self, stream):
        """Stream of the calls that follow (a torch.cuda.Stream)."""
        self.stream = stream
        B.adms_ctx_set_stream(self.ctx, stream)

    def set_ref_event(self, event):
        """forward_loss waits on this torch.cuda.Event (reference images ready) right
        before reading the references; None: no wait."""
        self._keep["ref_event"] = event
        B.adms_ctx_set_ref_event(self.ctx, event)

    def set_pipelining(self, enable=True):
        """Defer each optimizer step's texture update to the job's next forward_loss,
        where it runs beside the raster; results unchanged (adms_ctx_set_pipelining)."""
        B.adms_ctx_set_pipelining(self.ctx, enable)

    def sync(self):
        B.adms_sync(self.ctx)
