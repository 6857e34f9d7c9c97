"""Shape checks of the seeded input generators the oracle and the CUDA path share
(no method arithmetic lives there)."""

import numpy as np

import synth


def test_quad_cloud_quads_are_planar_disjoint_and_own_their_atlas_cells():
    n = 37
    m = synth.quad_cloud(n, seed=3, size=(0.05, 0.1), radii=(0.9, 0.7, 0.9))
    assert m.pos.shape == (4 * n, 3) and m.tri_pos.shape == (2 * n, 3)
    assert np.array_equal(m.tri_pos, m.tri_uv)
    q = m.pos.reshape(n, 4, 3).astype(np.float64)
    # planar rectangles: opposite sides equal, adjacent sides orthogonal, half-sides in range
    e0, e1 = q[:, 1] - q[:, 0], q[:, 3] - q[:, 0]
    assert np.allclose(q[:, 2] - q[:, 3], e0, atol=1e-6) and np.allclose(q[:, 2] - q[:, 1], e1, atol=1e-6)
    assert np.abs(np.sum(e0 * e1, axis=1)).max() < 1e-6
    half = np.linalg.norm(e0, axis=1) / 2
    assert (half > 0.05 - 1e-6).all() and (half < 0.1 + 1e-6).all()
    # centres inside the ellipsoid
    c = q.mean(axis=1) / np.array([0.9, 0.7, 0.9])
    assert (np.sum(c * c, axis=1) <= 1 + 1e-6).all()
    # both triangles of a quad share its diagonal and face the same way
    n0 = np.cross(q[:, 1] - q[:, 0], q[:, 2] - q[:, 0])
    n1 = np.cross(q[:, 2] - q[:, 0], q[:, 3] - q[:, 0])
    assert (np.sum(n0 * n1, axis=1) > 0).all()
    # atlas cells: inside [0, 1], and no two quads' uv boxes overlap
    uv = m.uv.reshape(n, 4, 2)
    lo, hi = uv.min(axis=1), uv.max(axis=1)
    assert (lo > 0).all() and (hi < 1).all()
    for i in range(n):
        sep = (hi[i] <= lo) | (lo[i] >= hi)
        sep[i] = True
        assert sep.any(axis=1).all()


def test_aggregate_config_sizes():
    c = synth.config_aggregate(ref_tris=2000, cand_tris=200, ref_tex_res=32, tex_res=32, aux_res=16)
    assert c["ref"].mesh.n_tris == 2000 and c["cand"].mesh.n_tris == 200
    assert c["loss"] == "l2" and c["layers"] == 8
    assert np.all(c["cand"].kd[..., 3] == np.float32(0.5))
    assert all(c["cand"].optimize[k] for k in ("pos", "kd", "orm", "nrm"))
