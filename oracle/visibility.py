"""ctypes front of the oracle's C visibility code (TEST INFRASTRUCTURE ONLY).

See raster.c for the exact float32 / int64 contract (transform, 8-bit
sub-pixel snapping, top-left fill rule, packed depth|id keys).
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import _build

EMPTY_KEY = np.uint64(0xFFFFFFFFFFFFFFFF)

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build())
        P = ctypes.c_void_p
        lib.oracle_transform.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P, P]
        lib.oracle_transform.restype = None
        lib.oracle_raster.argtypes = [P, P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P]
        lib.oracle_raster.restype = None
        lib.oracle_raster_layer.argtypes = [P, P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P]
        lib.oracle_raster_layer.restype = None
        lib.oracle_tess_positions.argtypes = [P, P, P, P, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, P, P,
                                              ctypes.c_int, ctypes.c_int, P, P]
        lib.oracle_tess_positions.restype = None
        lib.oracle_skin_positions.argtypes = [P, ctypes.c_int, P, ctypes.c_int, P, P]
        lib.oracle_skin_positions.restype = None
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def transform(mvp, pos, width, height):
    """float32 transform + snap of (V, 3) positions by one 4x4 row-major MVP.

    Returns dict(clip (V,4) f32, XY (V,2) i32, z01 (V,) f32, ok (V,) i8)."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    mvp = np.ascontiguousarray(np.asarray(mvp, dtype=np.float32).reshape(16))
    V = pos.shape[0]
    clip = np.zeros((V, 4), np.float32)
    XY = np.zeros((V, 2), np.int32)
    z01 = np.zeros(V, np.float32)
    ok = np.zeros(V, np.int8)
    lib.oracle_transform(_ptr(mvp), _ptr(pos), V, int(width), int(height), _ptr(clip), _ptr(XY), _ptr(z01), _ptr(ok))
    return dict(clip=clip, XY=XY, z01=z01, ok=ok)


def raster(mvp, pos, tri, width, height):
    """Visibility of one view: (keys (H, W) uint64, area_sign (F,) int8, transform dict)."""
    lib = _load()
    t = transform(mvp, pos, width, height)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    F = tri.shape[0]
    keys = np.full((height, width), EMPTY_KEY, dtype=np.uint64)
    asign = np.zeros(F, np.int8)
    lib.oracle_raster(_ptr(t["XY"]), _ptr(t["z01"]), _ptr(t["ok"]), _ptr(tri), F, int(width), int(height),
                      _ptr(keys), _ptr(asign))
    return keys, asign, t


def raster_views(views, pos, tri, width, height):
    """Visibility for a batch of views: keys (B, H, W) uint64, area_sign (B, F) int8."""
    keys, signs = [], []
    for v in views:
        k, s, _ = raster(v["mvp"], pos, tri, width, height)
        keys.append(k)
        signs.append(s)
    return np.stack(keys), np.stack(signs)


def raster_peeled(mvp, pos, tri, width, height, layers):
    """Depth peeling of one view (Sec. 5.2): layer 0 is the ordinary nearest-key
    visibility; layer l keeps, per pixel, the nearest fragment whose key is
    strictly greater than layer l-1's (EMPTY once a pixel runs out of
    fragments). Keys order by depth first and triangle id second, so coplanar
    fragments peel one at a time. Returns keys (layers, H, W), area_sign (F,)."""
    lib = _load()
    t = transform(mvp, pos, width, height)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    F = tri.shape[0]
    keys = np.full((layers, height, width), EMPTY_KEY, dtype=np.uint64)
    asign = np.zeros(F, np.int8)
    for l in range(layers):
        out = np.full((height, width), EMPTY_KEY, dtype=np.uint64)
        if l == 0:
            lib.oracle_raster(_ptr(t["XY"]), _ptr(t["z01"]), _ptr(t["ok"]), _ptr(tri), F, int(width), int(height),
                              _ptr(out), _ptr(asign))
        else:
            fl = np.ascontiguousarray(keys[l - 1])
            lib.oracle_raster_layer(_ptr(t["XY"]), _ptr(t["z01"]), _ptr(t["ok"]), _ptr(tri), F, int(width),
                                    int(height), _ptr(fl), _ptr(out), _ptr(asign))
        keys[l] = out
    return keys, asign


def raster_views_peeled(views, pos, tri, width, height, layers):
    """Depth-peeled visibility for a batch of views: keys (B, L, H, W), area_sign (B, F)."""
    keys, signs = [], []
    for v in views:
        k, s = raster_peeled(v["mvp"], pos, tri, width, height, layers)
        keys.append(k)
        signs.append(s)
    return np.stack(keys), np.stack(signs)


def skin_positions_f32(pos, weights, bones):
    """Skinned positions (Eq. 2) under the float32 contract of raster.c
    (oracle_skin_positions): pos (V, 3), weights (V, B), bones (B, 4, 4)."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    weights = np.ascontiguousarray(weights, dtype=np.float32)
    bones = np.ascontiguousarray(np.asarray(bones, dtype=np.float32).reshape(-1, 16))
    out = np.zeros_like(pos)
    lib.oracle_skin_positions(_ptr(pos), pos.shape[0], _ptr(weights), bones.shape[0], _ptr(bones), _ptr(out))
    return out
