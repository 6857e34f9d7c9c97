"""Dense linear-blend skinning (Eq. 2), float64. Test infrastructure: part of
the oracle; only tests, the smoke check and the bench's CPU legs use it.

v^s_i = sum_b w_ib M_b v_i with v_i in homogeneous coordinates [x, y, z, 1];
the bones are affine (last row 0 0 0 1), so the skinned position is the first
three components. Reading: the weights are used as given (Eq. 2 has no
normalisation), every vertex-bone pair is a latent (the dense operator the
paper describes), and no range is imposed on them.
"""

from __future__ import annotations

import torch


def skin(pos, weights, bones):
    """pos (V, 3), weights (V, B), bones (B, 4, 4) -> (V, 3), all float64 torch."""
    ph = torch.cat([pos, torch.ones_like(pos[:, :1])], dim=1)           # (V, 4)
    per_bone = torch.einsum("brc,vc->vbr", bones[:, :3, :], ph)         # (V, B, 3): M_b v_i
    return (weights[:, :, None] * per_bone).sum(dim=1)
