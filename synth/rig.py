"""Seeded skinning inputs: dense bone weights and per-frame bone poses.

Inputs only (no arithmetic of the method): weights fall off with the distance
from each vertex to a bone centre on the unit sphere and sum to 1 per vertex;
a pose gives every bone a rotation about a random axis through its centre and
a small translation, keyed by (seed, frame).
"""

from __future__ import annotations

import numpy as np


def bone_centres(n_bones, seed):
    rng = np.random.default_rng([int(seed), 7])
    c = rng.normal(size=(n_bones, 3))
    return c / np.linalg.norm(c, axis=1, keepdims=True)


def bone_weights(pos, n_bones, seed, sharpness=6.0):
    """(V, B) float32 weights, rows summing to 1."""
    c = bone_centres(n_bones, seed)
    d2 = ((np.asarray(pos, dtype=np.float64)[:, None, :] - c[None, :, :]) ** 2).sum(-1)
    w = np.exp(-sharpness * d2)
    return (w / w.sum(1, keepdims=True)).astype(np.float32)


def bone_pose(n_bones, seed, frame, max_angle=0.3, max_shift=0.05):
    """(B, 4, 4) float32 row-major affine bone matrices of one animation frame."""
    c = bone_centres(n_bones, seed)
    rng = np.random.default_rng([int(seed), int(frame), 11])
    out = np.zeros((n_bones, 4, 4))
    for b in range(n_bones):
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        ang = rng.uniform(-max_angle, max_angle)
        K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
        Rm = np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * (K @ K)
        t = c[b] - Rm @ c[b] + rng.uniform(-max_shift, max_shift, 3)   # rotate about the bone centre, then shift
        out[b, :3, :3] = Rm
        out[b, :3, 3] = t
        out[b, 3, 3] = 1.0
    return out.astype(np.float32)
