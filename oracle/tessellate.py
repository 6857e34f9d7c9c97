"""Edge-midpoint tessellation and displacement (Sec. 5.1, Eq. 3). TEST INFRASTRUCTURE ONLY.

Splitting every triangle into four at its edge midpoints, `levels` times,
gives the regular lattice of n = 2^levels segments per base edge. Every
tessellated vertex is therefore a point with integer barycentric coordinates
(i, j, k) / n on one base triangle; points on shared base edges and corners
are merged. The topology is fixed up front (constant tessellation factor, as
in the paper); positions are recomputed from the base latents every step:

    v   = sum_k w_k p_k                      (base positions)
    n   = normalize(sum_k w_k nhat_k)        (interpolated smooth base normal)
    t   = sum_k w_k uv_k                     (base UV corners of the owning face)
    v^d = v + tex2d(disp, t) * n             (Eq. 3; bilinear level-0 lookup)

reading: the owning face of a shared vertex is the lowest-numbered base face
that contains it.
"""

from __future__ import annotations

import numpy as np
import torch

from . import render as R


class Tessellation:
    def __init__(self, tri, tri_uv, uv, levels):
        n = 1 << int(levels)
        F = tri.shape[0]
        ii, jj = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
        keep = ii + jj <= n
        bi, bj = ii[keep], jj[keep]            # weights of corners 1 and 2; corner 0 gets n - i - j
        L = bi.size
        loc = -np.ones((n + 1, n + 1), dtype=np.int64)
        loc[bi, bj] = np.arange(L)
        w = np.stack([n - bi - bj, bi, bj], axis=1)                     # (L, 3)
        ids = tri[:, None, :].repeat(L, axis=1)                          # (F, L, 3)
        ww = np.broadcast_to(w[None], (F, L, 3))
        idk = np.where(ww > 0, ids, np.iinfo(np.int64).max)
        order = np.argsort(idk, axis=2, kind="stable")
        ids_s = np.take_along_axis(idk, order, axis=2)
        w_s = np.take_along_axis(np.where(ww > 0, ww, 0), order, axis=2)
        big = np.int64(tri.max() + 2)
        ids_c = np.where(ids_s == np.iinfo(np.int64).max, big - 1, ids_s)
        key = (((ids_c[..., 0] * big + ids_c[..., 1]) * big + ids_c[..., 2]) * (n + 1) + w_s[..., 0]) * (n + 1) \
            + w_s[..., 1]
        flat_key = key.reshape(-1)
        _, first, inverse = np.unique(flat_key, return_index=True, return_inverse=True)
        # first occurrence in face-major order = lowest-numbered owning face
        owner_face = first // L
        owner_loc = first % L
        self.n_verts = first.size
        self.n_seg = n
        self.face = owner_face
        self.wi = w[owner_loc].astype(np.int32)                          # (Vt, 3) integer weights
        self.w = w[owner_loc].astype(np.float64) / n                     # (Vt, 3)
        self.base_idx = tri[owner_face]                                   # (Vt, 3)
        self.vert_uv = (self.w[:, :, None] * uv[tri_uv[owner_face]]).sum(axis=1)  # (Vt, 2) displacement lookup
        gidx = inverse.reshape(F, L)
        lt = []
        for a in range(n):
            for b in range(n - a):
                lt.append((loc[a, b], loc[a + 1, b], loc[a, b + 1]))
                if a + b + 1 < n:
                    lt.append((loc[a + 1, b], loc[a + 1, b + 1], loc[a, b + 1]))
        lt = np.asarray(lt, dtype=np.int64)
        self.tri = gidx[:, lt].reshape(-1, 3)                             # (F n^2, 3)
        # sub-triangles inherit the base winding; their UV corners come from their own
        # base face, so triangles along a u seam keep the seam-shifted u values
        corner_uv = (w[None, :, :, None].astype(np.float64) / n * uv[tri_uv][:, None, :, :]).sum(axis=2)
        self.corner_uv = corner_uv.reshape(-1, 2)                         # (F L, 2)
        self.tri_uv = (np.arange(F)[:, None, None] * L + lt[None]).reshape(-1, 3)

    def positions_f32(self, base_pos, base_tri, disp):
        """The float32 displaced positions visibility uses (contract in raster.c)."""
        from . import visibility

        base_pos = np.ascontiguousarray(base_pos, dtype=np.float32)
        base_tri = np.ascontiguousarray(base_tri, dtype=np.int32)
        nb = base_pos.shape[0]
        counts = np.bincount(base_tri.reshape(-1), minlength=nb)
        vf_off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
        faces = np.repeat(np.arange(base_tri.shape[0], dtype=np.int32), 3)
        order = np.argsort(base_tri.reshape(-1), kind="stable")      # faces ascending within each vertex
        vf_face = np.ascontiguousarray(faces[order], dtype=np.int32)
        disp = np.ascontiguousarray(disp, dtype=np.float32)
        out = np.zeros((self.n_verts, 3), np.float32)
        nrm = np.zeros((nb, 3), np.float32)
        lib = visibility._load()
        P = visibility._ptr
        lib.oracle_tess_positions(P(base_pos), P(base_tri), P(vf_off), P(vf_face), nb, self.n_verts,
                                  P(np.ascontiguousarray(self.base_idx, dtype=np.int32)),
                                  P(np.ascontiguousarray(self.wi)), self.n_seg,
                                  P(np.ascontiguousarray(self.vert_uv, dtype=np.float32)), P(disp),
                                  disp.shape[0], disp.shape[1], P(nrm), P(out))
        return out

    def displaced_positions(self, base_pos, base_nrm, disp):
        w = torch.as_tensor(self.w)
        idx = torch.as_tensor(self.base_idx)
        v = sum(w[:, k:k + 1] * base_pos[idx[:, k]] for k in range(3))
        n = R.normalize(sum(w[:, k:k + 1] * base_nrm[idx[:, k]] for k in range(3)))
        uv = torch.as_tensor(self.vert_uv)
        d = R.bilinear(disp[:, :, None], uv[:, 0], uv[:, 1])               # (Vt, 1)
        return v + d * n
