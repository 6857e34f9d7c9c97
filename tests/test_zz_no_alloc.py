"""adms_visibility_noalloc: visibility for callers that cannot allocate device memory.

Some callers run inside another framework's memory pool or a fixed arena, or
in a frame loop where a cudaMalloc (and the synchronisation it implies) is not
allowed. This entry point keeps its scratch in a file-scope device array; the
test checks, through the C ABI, that two calls in a row give the oracle's keys
bit for bit and the same keys as the context-based raster, that a problem whose
tile lists do not fit the array still gives the oracle's keys (tiles fall back
to scanning every triangle), and that an oversized request is refused before
any GPU work. This file is collected last on purpose."""

import numpy as np
import pytest
import torch

import synth
from oracle import visibility as OV

pytestmark = pytest.mark.gpu


def _noalloc_keys(B, pos, tri, views, H, W):
    n = len(views)
    dv = torch.from_numpy(views.view(np.uint8).copy()).cuda()
    got = torch.full((n, H, W), 7, dtype=torch.int64, device="cuda")
    st = B.adms_visibility_noalloc(pos, tri, dv, n, H, W, got, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return st, got


def test_noalloc_keys_match_oracle_and_context_path_on_two_calls(gpu_lib):
    from paper_2104_03989_gb300 import binding as B
    from paper_2104_03989_gb300.engine import Context

    c = synth.config_plain(tex_res=64, ref_tex_res=64, ref_freq=16)
    mesh = c["cand"].mesh                       # 5,120 triangles
    H, W, n = 200, 232, 3                       # ragged tiles
    ctx = Context()
    job = ctx.create_job(c["cand"], frozen=True)
    pos = torch.as_tensor(np.ascontiguousarray(mesh.pos, dtype=np.float32)).cuda()
    tri = torch.as_tensor(np.ascontiguousarray(mesh.tri_pos, dtype=np.int32)).cuda()
    for call in range(2):
        views = synth.sample_views(40 + call, 0, n, W, H)
        want, _ = OV.raster_views(views, mesh.pos, mesh.tri_pos, W, H)
        ctx.render_reference(job, views, H, W)
        ctx_keys = ctx.keys(job, (n, H, W))
        st, got = _noalloc_keys(B, pos, tri, views, H, W)
        assert st is None or st == 0
        np.testing.assert_array_equal(got.cpu().numpy().view(np.uint64), want, err_msg=f"call {call}")
        assert torch.equal(got, ctx_keys), f"call {call}"
        assert (got != -1).any()
    ctx.close()


def _binned_pairs(pos, tri, views, H, W):
    """(tile, triangle) pairs the raster bins: triangles with a nonzero snapped area
    whose pixel-centre bounding box holds more than 16 pixels, one pair per 16x16
    tile the box touches (from the oracle's float32 transform and snapping)."""
    total = 0
    a, b, c = tri[:, 0], tri[:, 1], tri[:, 2]
    for v in views:
        t = OV.transform(v["mvp"], pos, W, H)
        X, Y, ok = t["XY"][:, 0].astype(np.int64), t["XY"][:, 1].astype(np.int64), t["ok"].astype(bool)
        area = (X[b] - X[a]) * (Y[c] - Y[a]) - (Y[b] - Y[a]) * (X[c] - X[a])
        lo = lambda m: np.maximum(-((128 - m) // 256), 0)   # ceil((m - 128) / 256), at least 0
        mx, Mx = np.minimum(X[a], np.minimum(X[b], X[c])), np.maximum(X[a], np.maximum(X[b], X[c]))
        my, My = np.minimum(Y[a], np.minimum(Y[b], Y[c])), np.maximum(Y[a], np.maximum(Y[b], Y[c]))
        i0, i1 = lo(mx), np.minimum((Mx - 128) // 256, W - 1)
        j0, j1 = lo(my), np.minimum((My - 128) // 256, H - 1)
        binned = ok[a] & ok[b] & ok[c] & (area != 0) & (i0 <= i1) & (j0 <= j1) & ((i1 - i0 + 1) * (j1 - j0 + 1) > 16)
        tiles = (i1 // 16 - i0 // 16 + 1) * (j1 // 16 - j0 // 16 + 1)
        total += int(tiles[binned].sum())
    return total


def test_noalloc_tile_list_overflow_matches_oracle(gpu_lib):
    """4,000 large random triangles over 100 shared vertices under 64 views at
    128^2: the per-view setup records take most of the 32 MiB array, and the
    (tile, triangle) pairs exceed the list space left by more than twice, so most
    tiles fall back to scanning every triangle of their view, with the oracle's
    keys all the same."""
    from paper_2104_03989_gb300 import binding as B

    rng = np.random.default_rng(3)
    pos = rng.uniform(-1.2, 1.2, (100, 3)).astype(np.float32)
    tri = np.stack([rng.choice(100, 3, replace=False) for _ in range(4000)]).astype(np.int32)
    H = W = 128
    views = synth.sample_views(3, 0, 64, W, H, r_min=3.0, r_max=3.5)
    # list space left after the fixed parts (each rounded up to 256 bytes)
    al = lambda x: (x + 255) // 256 * 256                   # noqa: E731
    nb, nv, nf, nt = 64, 100, 4000, 64 * 8 * 8
    fixed = 3 * al(nb * nv * 16) + al(nb * nf * 96) + al(nb * nf * 8) + 2 * al(nb * nf) + al(nf * 12) \
        + 3 * al(nt * 4) + 2 * 256
    capacity = ((32 << 20) - fixed) // 4
    assert _binned_pairs(pos, tri, views, H, W) > 2 * capacity
    want, _ = OV.raster_views(views, pos, tri, W, H)
    st, got = _noalloc_keys(B, torch.as_tensor(pos).cuda(), torch.as_tensor(tri).cuda(), views, H, W)
    np.testing.assert_array_equal(got.cpu().numpy().view(np.uint64), want)
    assert (want != OV.EMPTY_KEY).mean() > 0.5


def test_noalloc_refuses_oversized_problem(gpu_lib):
    from paper_2104_03989_gb300 import binding as B

    pos = torch.zeros((3, 3), device="cuda")
    tri = torch.zeros((1, 3), dtype=torch.int32, device="cuda")
    views = torch.zeros(112, dtype=torch.uint8, device="cuda")
    keys = torch.zeros(1, dtype=torch.int64, device="cuda")
    # claims 100 views x 1M triangles: far beyond the 32 MiB scratch; refused on the host
    status = B.lib().adms_visibility_noalloc(pos.data_ptr(), 3, tri.data_ptr(), 1 << 20, views.data_ptr(), 100,
                                             16, 16, keys.data_ptr(), None)
    assert status == B.ADMS_ERR_ARG
