"""ctypes binding of libadms.so (argument marshalling only).

Every function named adms_* here calls the C entry point of the same name and
raises AdmsError on a non-zero status. All computation runs in the CUDA
library; this module only converts numpy arrays / torch tensors into the
pointers and structs of include/adms.h. There is no CPU fallback: if the
library cannot be loaded, lib() raises.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libadms.so")

ADMS_OK, ADMS_ERR_ARG, ADMS_ERR_BUDGET, ADMS_ERR_CUDA, ADMS_ERR_TIMEOUT, ADMS_ERR_NONFINITE, ADMS_ERR_STATE = (
    0, -1, -2, -3, -4, -5, -6)
LOSS = {"l1": 0, "logl1": 1, "l2": 2}


class AdmsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"adms status {status}: {msg}")
        self.status = status


class adms_view(C.Structure):
    _fields_ = [("mvp", C.c_float * 16), ("eye", C.c_float * 3), ("pad0", C.c_float),
                ("light_pos", C.c_float * 3), ("light_I", C.c_float), ("light_dir", C.c_float * 3),
                ("light_E", C.c_float)]


class adms_mesh_desc(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_uv", C.c_int32), ("n_tris", C.c_int32), ("pos", C.c_void_p),
                ("uv", C.c_void_p), ("tri_pos", C.c_void_p), ("tri_uv", C.c_void_p)]


class adms_material_desc(C.Structure):
    _fields_ = [("kd", C.c_void_p), ("orm", C.c_void_p), ("nrm", C.c_void_p), ("disp", C.c_void_p),
                ("kd_h", C.c_int32), ("kd_w", C.c_int32), ("orm_h", C.c_int32), ("orm_w", C.c_int32),
                ("nrm_h", C.c_int32), ("nrm_w", C.c_int32), ("disp_h", C.c_int32), ("disp_w", C.c_int32),
                ("mips", C.c_int32)]


class adms_opt_params(C.Structure):
    _fields_ = [("optimize_pos", C.c_int32), ("optimize_kd", C.c_int32), ("optimize_orm", C.c_int32),
                ("optimize_nrm", C.c_int32), ("optimize_disp", C.c_int32), ("loss", C.c_int32),
                ("tess_levels", C.c_int32), ("batch_views", C.c_int32), ("relative_laplacian", C.c_int32),
                ("aa", C.c_int32), ("lr0", C.c_float), ("lambda0", C.c_float), ("per_level_textures", C.c_int32),
                ("samples", C.c_int32), ("shade_samples", C.c_int32), ("layers", C.c_int32),
                ("raster_direct_px", C.c_int32), ("raster_depth_filter", C.c_int32)]


class adms_param_view(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("kd", C.c_void_p), ("orm", C.c_void_p), ("nrm", C.c_void_p),
                ("disp", C.c_void_p), ("g_pos", C.c_void_p), ("g_kd", C.c_void_p), ("g_orm", C.c_void_p),
                ("g_nrm", C.c_void_p), ("g_disp", C.c_void_p), ("n_verts", C.c_int32),
                ("n_tris_render", C.c_int32), ("kd_h", C.c_int32), ("kd_w", C.c_int32), ("orm_h", C.c_int32),
                ("orm_w", C.c_int32), ("nrm_h", C.c_int32), ("nrm_w", C.c_int32), ("disp_h", C.c_int32),
                ("disp_w", C.c_int32), ("kd_levels", C.c_int32), ("orm_levels", C.c_int32),
                ("nrm_levels", C.c_int32), ("t", C.c_int32), ("skin_w", C.c_void_p), ("g_skin_w", C.c_void_p), ("n_bones", C.c_int32)]


class adms_stats(C.Structure):
    _fields_ = [("image_loss", C.c_float), ("laplacian", C.c_float), ("lambda_", C.c_float), ("lr", C.c_float),
                ("t", C.c_int32), ("status", C.c_int32), ("tile_overflows", C.c_int64), ("call_loss", C.c_double)]


class adms_stage_mesh(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_uv", C.c_int32), ("n_tris", C.c_int32), ("pos", C.c_void_p),
                ("uv", C.c_void_p), ("tri", C.c_void_p), ("tri_uv", C.c_void_p), ("adj", C.c_void_p),
                ("vf_off", C.c_void_p), ("vf_face", C.c_void_p)]


class adms_stage_texture(C.Structure):
    _fields_ = [("tex", C.c_void_p), ("grad", C.c_void_p), ("h", C.c_int32), ("w", C.c_int32),
                ("levels", C.c_int32)]


class adms_tess_desc(C.Structure):
    _fields_ = [("n_base_verts", C.c_int32), ("n_base_tris", C.c_int32), ("n_verts", C.c_int32),
                ("n_segments", C.c_int32), ("base_tri", C.c_void_p), ("bvf_off", C.c_void_p), ("bvf_face", C.c_void_p),
                ("owner", C.c_void_p), ("wts", C.c_void_p), ("vert_uv", C.c_void_p)]


assert C.sizeof(adms_view) == 112

# name -> (argtypes, restype)
P = C.c_void_p
SIGNATURES = {
    "adms_ctx_create": ([C.POINTER(P), C.c_size_t, P], C.c_int),
    "adms_ctx_destroy": ([P], C.c_int),
    "adms_ctx_set_stream": ([P, P], C.c_int),
    "adms_ctx_set_ref_event": ([P, P], C.c_int),
    "adms_sync": ([P], C.c_int),
    "adms_last_error": ([P], C.c_char_p),
    "adms_bytes_in_use": ([P], C.c_size_t),
    "adms_job_create": ([P, C.POINTER(adms_mesh_desc), C.POINTER(adms_material_desc), C.POINTER(adms_opt_params),
                         C.c_uint64, C.POINTER(C.c_int32)], C.c_int),
    "adms_job_destroy": ([P, C.c_int32], C.c_int),
    "adms_job_reserve": ([P, C.c_int32, C.c_int32, C.c_int32, C.c_int32], C.c_int),
    "adms_ctx_release_batches": ([P], C.c_int),
    "adms_job_skinning": ([P, C.c_int32, P, C.c_int32, C.c_float], C.c_int),
    "adms_job_set_bones": ([P, C.c_int32, P], C.c_int),
    "adms_job_params": ([P, C.c_int32, C.POINTER(adms_param_view)], C.c_int),
    "adms_job_stats": ([P, C.c_int32, C.POINTER(adms_stats)], C.c_int),
    "adms_jobs_status": ([P, P, C.c_int32, P], C.c_int),
    "adms_render_reference": ([P, C.c_int32, P, C.c_int32, C.c_int32, C.c_int32, P], C.c_int),
    "adms_forward_loss": ([P, P, C.c_int32, P, P, P, P, P, P], C.c_int),
    "adms_backward": ([P, P, C.c_int32, C.c_int32], C.c_int),
    "adms_optimizer_step": ([P, P, C.c_int32], C.c_int),
    "adms_job_keys": ([P, C.c_int32, P, C.c_size_t], C.c_int),
    "adms_job_fold_gradients": ([P, C.c_int32, P, P, P], C.c_int),
    "adms_job_zero_gradients": ([P, C.c_int32], C.c_int),
    "adms_job_invalidate": ([P, C.c_int32], C.c_int),
    "adms_laplacian": ([P, C.c_int32, P, P], C.c_int),
    "adms_job_export": ([P, C.c_int32, P, C.POINTER(C.c_size_t)], C.c_int),
    "adms_job_import": ([P, C.POINTER(adms_mesh_desc), C.POINTER(adms_material_desc), C.POINTER(adms_opt_params),
                         P, C.c_size_t, C.POINTER(C.c_int32)], C.c_int),
    "adms_mesh_topology": ([P, C.c_int32, C.c_int32, P, P, P], C.c_int),
    "adms_stage_workspace_bytes": ([C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int64], C.c_size_t),
    "adms_frame_fwd": ([C.POINTER(adms_stage_mesh), P, P, P, P], C.c_int),
    "adms_frame_bwd": ([C.POINTER(adms_stage_mesh), P, P, P, P, P, P], C.c_int),
    "adms_setup_fwd": ([C.POINTER(adms_stage_mesh), P, C.c_int32, C.c_int32, C.c_int32, P, P, C.c_size_t, P], C.c_int),
    "adms_setup_bwd": ([P, C.c_int32, C.c_int32, P, P, P], C.c_int),
    "adms_raster_fwd": ([C.POINTER(adms_stage_mesh), P, C.c_int32, C.c_int32, C.c_int32, P, P, C.c_int32, P, P, P,
                         C.c_size_t, P], C.c_int),
    "adms_raster_bwd": ([C.POINTER(adms_stage_mesh), P, C.c_int32, C.c_int32, C.c_int32, P, P, P, P, P, C.c_size_t,
                         P], C.c_int),
    "adms_shade_fwd": ([C.POINTER(adms_stage_mesh), P, C.c_int32, C.c_int32, C.c_int32, P, P, P, P, P, P,
                        C.POINTER(adms_stage_texture), P, P], C.c_int),
    "adms_shade_bwd": ([C.POINTER(adms_stage_mesh), P, C.c_int32, C.c_int32, C.c_int32, P, P, P, P, P, P,
                        C.POINTER(adms_stage_texture), P, P, P, P, P, P], C.c_int),
    "adms_aa_loss_fwd": ([C.POINTER(adms_stage_mesh), P, C.c_int32, C.c_int32, C.c_int32, P, P, P, P, C.c_int32,
                          C.c_float, P, P, P, P, C.c_size_t, P], C.c_int),
    "adms_aa_loss_bwd": ([C.POINTER(adms_stage_mesh), P, C.c_int32, C.c_int32, C.c_int32, P, P, P, P, P, P, P, P,
                          C.c_size_t, P], C.c_int),
    "adms_tessellation": ([P, P, P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P, P, P, P, P, P, P], C.c_int),
    "adms_tess_fwd": ([C.POINTER(adms_tess_desc), P, P, C.c_int32, C.c_int32, P, P, P], C.c_int),
    "adms_tess_bwd": ([C.POINTER(adms_tess_desc), P, P, P, C.c_int32, C.c_int32, P, P, P, P, P], C.c_int),
    "adms_mip_fwd": ([P, C.c_int32, C.c_int32, C.c_int32, P], C.c_int),
    "adms_mip_bwd": ([P, C.c_int32, C.c_int32, C.c_int32, P, P], C.c_int),
    "adms_visibility_noalloc": ([P, C.c_int32, P, C.c_int32, P, C.c_int32, C.c_int32, C.c_int32, P, P], C.c_int),
    "adms_autotune": ([P, P, C.c_int32, P, P, P, P], C.c_int),
    "adms_ctx_tuning": ([P, P], C.c_int),
    "adms_ctx_set_tuning": ([P, C.POINTER(C.c_int32)], C.c_int),
    "adms_graph_begin": ([P], C.c_int),
    "adms_graph_end": ([P, C.POINTER(P)], C.c_int),
    "adms_graph_launch": ([P, P], C.c_int),
    "adms_graph_destroy": ([P], C.c_int),
    "adms_ctx_profile": ([P, C.c_int32], C.c_int),
    "adms_ctx_test_wait_timeout": ([P, C.c_int32], C.c_int),
    "adms_ctx_set_pipelining": ([P, C.c_int32], C.c_int),
    "adms_ctx_stage_times": ([P, P, P, C.c_int32], C.c_int),
    "adms_stage_count": ([], C.c_int32),
    "adms_stage_name": ([C.c_int32], C.c_char_p),
    "adms_launch_count": ([], C.c_int64),
}

_lib = None


def lib():
    """Load libadms.so (built by paper_2104_03989_gb300.build). Raises if missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(ctx, status):
    if status != ADMS_OK:
        msg = lib().adms_last_error(ctx).decode() if ctx else ""
        raise AdmsError(status, msg)


def ptr(x):
    """Pointer of a numpy array (host) or torch tensor (host or device)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr()
    return int(x)


# ----------------------------------------------------------------------------- thin wrappers

def adms_ctx_create(hbm_budget_bytes=0, stream=None):
    out = P()
    st = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    _check(None, lib().adms_ctx_create(C.byref(out), hbm_budget_bytes, st))
    return out


def adms_ctx_destroy(ctx):
    _check(None, lib().adms_ctx_destroy(ctx))


def adms_ctx_set_stream(ctx, stream):
    st = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    _check(ctx, lib().adms_ctx_set_stream(ctx, st))


def adms_ctx_set_ref_event(ctx, event):
    """event: a torch.cuda.Event (or a raw cudaEvent_t handle), or None."""
    ev = None if event is None else (event.cuda_event if hasattr(event, "cuda_event") else event)
    _check(ctx, lib().adms_ctx_set_ref_event(ctx, ev))


def adms_sync(ctx):
    _check(ctx, lib().adms_sync(ctx))


def adms_bytes_in_use(ctx):
    return int(lib().adms_bytes_in_use(ctx))


def mesh_desc(pos, uv, tri_pos, tri_uv):
    d = adms_mesh_desc(int(pos.shape[0]), int(uv.shape[0]), int(tri_pos.shape[0]), ptr(pos), ptr(uv), ptr(tri_pos),
                       ptr(tri_uv))
    d._keep = (pos, uv, tri_pos, tri_uv)
    return d


def material_desc(kd, orm, nrm, disp=None, mips=True):
    d = adms_material_desc(ptr(kd), ptr(orm), ptr(nrm), ptr(disp), kd.shape[0], kd.shape[1], orm.shape[0],
                           orm.shape[1], nrm.shape[0], nrm.shape[1], 0 if disp is None else disp.shape[0],
                           0 if disp is None else disp.shape[1], 1 if mips else 0)
    d._keep = (kd, orm, nrm, disp)
    return d


def opt_params(optimize=None, loss="logl1", tess_levels=0, batch_views=0, relative_laplacian=False, aa=True,
               lr0=0.01, lambda0=0.0, per_level_textures=False, samples=1, shade_samples=False, layers=0,
               raster_direct_px=0, raster_depth_filter=False):
    o = optimize or {}
    return adms_opt_params(int(o.get("pos", 0)), int(o.get("kd", 0)), int(o.get("orm", 0)), int(o.get("nrm", 0)),
                           int(o.get("disp", 0)), LOSS[loss], tess_levels, batch_views, int(relative_laplacian),
                           int(aa), lr0, lambda0, int(per_level_textures), int(samples), int(shade_samples),
                           int(layers), int(raster_direct_px), int(raster_depth_filter))


def adms_job_create(ctx, mesh, mat, opt=None, seed=0):
    out = C.c_int32()
    _check(ctx, lib().adms_job_create(ctx, C.byref(mesh), C.byref(mat), C.byref(opt) if opt is not None else None,
                                      seed, C.byref(out)))
    return out.value


def adms_job_destroy(ctx, job):
    _check(ctx, lib().adms_job_destroy(ctx, job))


def adms_job_skinning(ctx, job, weights, n_bones, lr_scale=1.0):
    _check(ctx, lib().adms_job_skinning(ctx, job, ptr(weights), int(n_bones), float(lr_scale)))


def adms_job_set_bones(ctx, job, bones):
    _check(ctx, lib().adms_job_set_bones(ctx, job, ptr(bones)))


def adms_ctx_release_batches(ctx):
    _check(ctx, lib().adms_ctx_release_batches(ctx))


def adms_job_reserve(ctx, job, n_views, H, W):
    _check(ctx, lib().adms_job_reserve(ctx, job, int(n_views), int(H), int(W)))


def adms_job_params(ctx, job):
    out = adms_param_view()
    _check(ctx, lib().adms_job_params(ctx, job, C.byref(out)))
    return out


def adms_job_stats(ctx, job):
    out = adms_stats()
    _check(ctx, lib().adms_job_stats(ctx, job, C.byref(out)))
    return out


def adms_jobs_status(ctx, jobs, out):
    """Each job's latched status into the device int32 tensor out (stream-ordered)."""
    arr = (C.c_int32 * len(jobs))(*jobs)
    _check(ctx, lib().adms_jobs_status(ctx, arr, len(jobs), ptr(out)))


def adms_render_reference(ctx, job, views, H, W, out_rgb):
    _check(ctx, lib().adms_render_reference(ctx, job, ptr(views), len(views), H, W, ptr(out_rgb)))


def adms_forward_loss(ctx, jobs, views, views_per_job, hw, ref_rgb, out_loss, out_img=None):
    n = len(jobs)
    jobs_a = (C.c_int32 * n)(*jobs)
    vpj = (C.c_int32 * n)(*views_per_job)
    hw_a = (C.c_int32 * (2 * n))(*[int(x) for p in hw for x in p])
    refs = (C.c_void_p * n)(*[ptr(r) for r in ref_rgb])
    imgs = (C.c_void_p * n)(*[ptr(i) for i in out_img]) if out_img is not None else None
    _check(ctx, lib().adms_forward_loss(ctx, jobs_a, n, ptr(views), vpj, hw_a, refs, ptr(out_loss), imgs))


def adms_backward(ctx, jobs, recompute_raster=0):
    n = len(jobs)
    _check(ctx, lib().adms_backward(ctx, (C.c_int32 * n)(*jobs), n, int(recompute_raster)))


def adms_optimizer_step(ctx, jobs):
    n = len(jobs)
    _check(ctx, lib().adms_optimizer_step(ctx, (C.c_int32 * n)(*jobs), n))


def adms_job_keys(ctx, job, out_keys):
    _check(ctx, lib().adms_job_keys(ctx, job, ptr(out_keys), out_keys.numel()))


def adms_job_fold_gradients(ctx, job, g_kd=None, g_orm=None, g_nrm=None):
    _check(ctx, lib().adms_job_fold_gradients(ctx, job, ptr(g_kd), ptr(g_orm), ptr(g_nrm)))


def adms_job_zero_gradients(ctx, job):
    _check(ctx, lib().adms_job_zero_gradients(ctx, job))


def adms_job_invalidate(ctx, job):
    _check(ctx, lib().adms_job_invalidate(ctx, job))


def adms_laplacian(ctx, job, out_loss, g_pos=None):
    _check(ctx, lib().adms_laplacian(ctx, job, ptr(out_loss), ptr(g_pos)))


def adms_job_export(ctx, job):
    n = C.c_size_t(0)
    _check(ctx, lib().adms_job_export(ctx, job, None, C.byref(n)))
    buf = np.zeros(n.value, dtype=np.uint8)
    _check(ctx, lib().adms_job_export(ctx, job, ptr(buf), C.byref(n)))
    return buf


def adms_job_import(ctx, mesh, mat, opt, buf):
    out = C.c_int32()
    _check(ctx, lib().adms_job_import(ctx, C.byref(mesh), C.byref(mat), C.byref(opt) if opt is not None else None,
                                      ptr(buf), buf.nbytes, C.byref(out)))
    return out.value


def adms_autotune(ctx, jobs, views, views_per_job, hw, ref_rgb):
    n = len(jobs)
    jobs_a = (C.c_int32 * n)(*jobs)
    vpj = (C.c_int32 * n)(*views_per_job)
    hw_a = (C.c_int32 * (2 * n))(*[int(x) for p in hw for x in p])
    refs = (C.c_void_p * n)(*[ptr(r) for r in ref_rgb])
    _check(ctx, lib().adms_autotune(ctx, jobs_a, n, ptr(views), vpj, hw_a, refs))


def adms_ctx_set_tuning(ctx, tile_w, shade, aa_loss, backward, raster):
    _check(ctx, lib().adms_ctx_set_tuning(ctx, (C.c_int32 * 5)(tile_w, shade, aa_loss, backward, raster)))


def adms_ctx_tuning(ctx):
    out = (C.c_int32 * 5)()
    _check(ctx, lib().adms_ctx_tuning(ctx, out))
    return {"tile_w": out[0], "blocks_per_sm": {"shade": out[1], "aa_loss": out[2], "backward": out[3],
                                                "raster": out[4]}}


def adms_visibility_noalloc(pos, tri, views, n_views, H, W, keys, stream=None):
    """Keys [n_views][H][W] into `keys` without any allocation (see include/adms.h)."""
    st = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    status = lib().adms_visibility_noalloc(ptr(pos), int(pos.shape[0]), ptr(tri), int(tri.shape[0]), ptr(views),
                                           int(n_views), int(H), int(W), ptr(keys), st)
    if status != ADMS_OK:
        raise AdmsError(status, "adms_visibility_noalloc")


# ----------------------------------------------------------------------------- per-stage calls

def _stream(stream):
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


def _stage(status, name):
    if status != ADMS_OK:
        raise AdmsError(status, name)


def stage_mesh(pos, uv, tri, tri_uv, adj, vf_off, vf_face):
    """adms_stage_mesh of device tensors (kept alive by the returned struct)."""
    m = adms_stage_mesh(int(pos.shape[0]), int(uv.shape[0]), int(tri.shape[0]), ptr(pos), ptr(uv), ptr(tri),
                        ptr(tri_uv), ptr(adj), ptr(vf_off), ptr(vf_face))
    m._keep = (pos, uv, tri, tri_uv, adj, vf_off, vf_face)
    return m


def stage_textures(maps):
    """adms_stage_texture[3] of (chain, grad or None, h, w, levels) tuples."""
    arr = (adms_stage_texture * 3)()
    for i, (chain, grad, h, w, levels) in enumerate(maps):
        arr[i] = adms_stage_texture(ptr(chain), ptr(grad), int(h), int(w), int(levels))
    arr._keep = maps
    return arr


def adms_mesh_topology(tri, n_verts):
    """Host numpy int32 tri (F, 3) -> (adj (F, 3), vf_off (V+1,), vf_face (3F,)) int32."""
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    F = tri.shape[0]
    adj = np.empty((F, 3), np.int32)
    vf_off = np.empty(n_verts + 1, np.int32)
    vf_face = np.empty(3 * F, np.int32)
    _stage(lib().adms_mesh_topology(ptr(tri), int(n_verts), F, ptr(adj), ptr(vf_off), ptr(vf_face)),
           "adms_mesh_topology")
    return adj, vf_off, vf_face


def adms_stage_workspace_bytes(n_verts, n_tris, n_views, H, W, list_entries):
    return int(lib().adms_stage_workspace_bytes(n_verts, n_tris, n_views, H, W, list_entries))


def adms_frame_fwd(mesh, vpos4, vnrm4, vtan4, stream=None):
    _stage(lib().adms_frame_fwd(C.byref(mesh), ptr(vpos4), ptr(vnrm4), ptr(vtan4), _stream(stream)), "adms_frame_fwd")


def adms_frame_bwd(mesh, g_vpos, g_vnrm, g_vtan, g_pos, tmp, stream=None):
    _stage(lib().adms_frame_bwd(C.byref(mesh), ptr(g_vpos), ptr(g_vnrm), ptr(g_vtan), ptr(g_pos), ptr(tmp),
                                _stream(stream)), "adms_frame_bwd")


def adms_setup_fwd(mesh, views, n_views, H, W, clip, work, stream=None):
    _stage(lib().adms_setup_fwd(C.byref(mesh), ptr(views), n_views, H, W, ptr(clip), ptr(work), work.numel(),
                                _stream(stream)), "adms_setup_fwd")


def adms_setup_bwd(views, n_views, n_verts, g_clip, g_pos, stream=None):
    _stage(lib().adms_setup_bwd(ptr(views), n_views, n_verts, ptr(g_clip), ptr(g_pos), _stream(stream)),
           "adms_setup_bwd")


def adms_raster_fwd(mesh, views, n_views, H, W, clip, keys, rast, rast_db, work, stream=None, keep_keys=False):
    _stage(lib().adms_raster_fwd(C.byref(mesh), ptr(views), n_views, H, W, ptr(clip), ptr(keys), int(bool(keep_keys)),
                                 ptr(rast), ptr(rast_db), ptr(work), work.numel(), _stream(stream)), "adms_raster_fwd")


def adms_raster_bwd(mesh, views, n_views, H, W, clip, keys, g_rast, g_clip, work, stream=None):
    _stage(lib().adms_raster_bwd(C.byref(mesh), ptr(views), n_views, H, W, ptr(clip), ptr(keys), ptr(g_rast),
                                 ptr(g_clip), ptr(work), work.numel(), _stream(stream)), "adms_raster_bwd")


def adms_shade_fwd(mesh, views, n_views, H, W, keys, rast, rast_db, vpos4, vnrm4, vtan4, maps, pre, stream=None):
    _stage(lib().adms_shade_fwd(C.byref(mesh), ptr(views), n_views, H, W, ptr(keys), ptr(rast), ptr(rast_db),
                                ptr(vpos4), ptr(vnrm4), ptr(vtan4), maps, ptr(pre), _stream(stream)), "adms_shade_fwd")


def adms_shade_bwd(mesh, views, n_views, H, W, keys, rast, rast_db, vpos4, vnrm4, vtan4, maps, g_pre, g_vpos,
                   g_vnrm, g_vtan, g_rast, stream=None):
    _stage(lib().adms_shade_bwd(C.byref(mesh), ptr(views), n_views, H, W, ptr(keys), ptr(rast), ptr(rast_db),
                                ptr(vpos4), ptr(vnrm4), ptr(vtan4), maps, ptr(g_pre), ptr(g_vpos), ptr(g_vnrm),
                                ptr(g_vtan), ptr(g_rast), _stream(stream)), "adms_shade_bwd")


def adms_aa_loss_fwd(mesh, views, n_views, H, W, clip, keys, pre, ref, loss_kind, loss_scale, img, loss, gprime,
                     work, stream=None):
    _stage(lib().adms_aa_loss_fwd(C.byref(mesh), ptr(views), n_views, H, W, ptr(clip), ptr(keys), ptr(pre), ptr(ref),
                                  int(loss_kind), float(loss_scale), ptr(img), ptr(loss), ptr(gprime), ptr(work),
                                  work.numel(), _stream(stream)), "adms_aa_loss_fwd")


def adms_aa_loss_bwd(mesh, views, n_views, H, W, clip, keys, pre, gprime, g_loss, g_pre, g_clip, work, stream=None):
    _stage(lib().adms_aa_loss_bwd(C.byref(mesh), ptr(views), n_views, H, W, ptr(clip), ptr(keys), ptr(pre),
                                  ptr(gprime), ptr(g_loss), ptr(g_pre), ptr(g_clip), ptr(work), work.numel(),
                                  _stream(stream)), "adms_aa_loss_bwd")


def adms_tessellation(tri, tri_uv, uv, n_verts, levels):
    """Host tessellation tables of a base mesh: dict of numpy arrays (rtri, rtri_uv,
    ruv, owner, wts, vert_uv) and the counts (see include/adms.h)."""
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    tri_uv = np.ascontiguousarray(tri_uv, dtype=np.int32)
    uv = np.ascontiguousarray(uv, dtype=np.float32)
    counts = np.zeros(3, np.int32)
    args = (ptr(tri), ptr(tri_uv), ptr(uv), int(n_verts), int(uv.shape[0]), int(tri.shape[0]), int(levels))
    _stage(lib().adms_tessellation(*args, ptr(counts), None, None, None, None, None, None), "adms_tessellation")
    Vt, Ft, Tt = (int(x) for x in counts)
    out = dict(rtri=np.empty((Ft, 3), np.int32), rtri_uv=np.empty((Ft, 3), np.int32), ruv=np.empty((Tt, 2), np.float32),
               owner=np.empty((Vt, 3), np.int32), wts=np.empty((Vt, 3), np.int32), vert_uv=np.empty((Vt, 2), np.float32))
    _stage(lib().adms_tessellation(*args, ptr(counts), ptr(out["rtri"]), ptr(out["rtri_uv"]), ptr(out["ruv"]),
                                   ptr(out["owner"]), ptr(out["wts"]), ptr(out["vert_uv"])), "adms_tessellation")
    return out


def tess_desc(n_base_verts, n_base_tris, n_verts, n_segments, base_tri, bvf_off, bvf_face, owner, wts, vert_uv):
    d = adms_tess_desc(int(n_base_verts), int(n_base_tris), int(n_verts), int(n_segments), ptr(base_tri), ptr(bvf_off),
                       ptr(bvf_face), ptr(owner), ptr(wts), ptr(vert_uv))
    d._keep = (base_tri, bvf_off, bvf_face, owner, wts, vert_uv)
    return d


def adms_tess_fwd(tess, base_pos, disp, base_nrm, pos, stream=None):
    _stage(lib().adms_tess_fwd(C.byref(tess), ptr(base_pos), ptr(disp), int(disp.shape[0]), int(disp.shape[1]),
                               ptr(base_nrm), ptr(pos), _stream(stream)), "adms_tess_fwd")


def adms_tess_bwd(tess, base_pos, base_nrm, disp, g_pos, g_base_pos, g_base_nrm, g_disp, stream=None):
    _stage(lib().adms_tess_bwd(C.byref(tess), ptr(base_pos), ptr(base_nrm), ptr(disp), int(disp.shape[0]),
                               int(disp.shape[1]), ptr(g_pos), ptr(g_base_pos), ptr(g_base_nrm), ptr(g_disp),
                               _stream(stream)), "adms_tess_bwd")


def adms_mip_fwd(chain, h, w, levels, stream=None):
    _stage(lib().adms_mip_fwd(ptr(chain), h, w, levels, _stream(stream)), "adms_mip_fwd")


def adms_mip_bwd(g_chain, h, w, levels, g_level0, stream=None):
    _stage(lib().adms_mip_bwd(ptr(g_chain), h, w, levels, ptr(g_level0), _stream(stream)), "adms_mip_bwd")


def adms_graph_begin(ctx):
    _check(ctx, lib().adms_graph_begin(ctx))


def adms_graph_end(ctx):
    g = P()
    _check(ctx, lib().adms_graph_end(ctx, C.byref(g)))
    return g


def adms_graph_launch(ctx, graph):
    _check(ctx, lib().adms_graph_launch(ctx, graph))


def adms_graph_destroy(graph):
    _check(None, lib().adms_graph_destroy(graph))


def adms_ctx_profile(ctx, enable=True):
    _check(ctx, lib().adms_ctx_profile(ctx, int(enable)))


def adms_ctx_test_wait_timeout(ctx, enable=True):
    _check(ctx, lib().adms_ctx_test_wait_timeout(ctx, int(enable)))


def adms_ctx_set_pipelining(ctx, enable=True):
    _check(ctx, lib().adms_ctx_set_pipelining(ctx, int(enable)))


def adms_ctx_stage_times(ctx):
    """{stage name: (gpu ms, launches)} accumulated since the previous call."""
    n = int(lib().adms_stage_count())
    ms = np.zeros(n, dtype=np.float64)
    cnt = np.zeros(n, dtype=np.int64)
    _check(ctx, lib().adms_ctx_stage_times(ctx, ptr(ms), ptr(cnt), n))
    return {lib().adms_stage_name(i).decode(): (float(ms[i]), int(cnt[i])) for i in range(n)}


def adms_launch_count():
    return int(lib().adms_launch_count())
