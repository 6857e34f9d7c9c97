"""adms_visibility_noalloc: visibility for callers that cannot allocate device memory.

Some callers run inside another framework's memory pool or a fixed arena, or
in a frame loop where a cudaMalloc (and the synchronisation it implies) is not
allowed. This entry point keeps its scratch in a file-scope device array; the
test checks, through the C ABI, that two calls in a row give the same keys bit
for bit as the context-based raster, and that an oversized request is refused
before any GPU work. This file is collected last on purpose."""

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_keys_match_context_path_on_two_calls(gpu_lib):
    from paper_2104_03989_gb300 import binding as B
    from paper_2104_03989_gb300.engine import Context

    c = synth.config_plain(tex_res=64, ref_tex_res=64, ref_freq=16)
    mesh = c["cand"].mesh                       # 5,120 triangles
    H, W, n = 200, 232, 3                       # ragged tiles
    ctx = Context()
    job = ctx.create_job(c["cand"], frozen=True)
    pos = torch.as_tensor(np.ascontiguousarray(mesh.pos, dtype=np.float32)).cuda()
    tri = torch.as_tensor(np.ascontiguousarray(mesh.tri_pos, dtype=np.int32)).cuda()
    stream = torch.cuda.current_stream()
    for call in range(2):
        views = synth.sample_views(40 + call, 0, n, W, H)
        ctx.render_reference(job, views, H, W)
        want = ctx.keys(job, (n, H, W))
        dv = torch.from_numpy(views.view(np.uint8).copy()).cuda()
        got = torch.full((n, H, W), 7, dtype=torch.int64, device="cuda")
        B.adms_visibility_noalloc(pos, tri, dv, n, H, W, got, stream)
        torch.cuda.synchronize()
        assert torch.equal(got, want), f"call {call}"
        assert (got != -1).any()
    ctx.close()


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
