"""A step recorded as a CUDA graph through the C ABI replays like direct calls."""

import numpy as np
import pytest
import torch

import synth

from cases import oracle_reference, rel_l2

pytestmark = pytest.mark.gpu


def test_graph_replay_matches_direct_calls(gpu_lib):
    from paper_2104_03989_gb300 import binding as B
    from paper_2104_03989_gb300.engine import Context

    c = synth.config_small()
    H = W = 128
    views = synth.sample_views(4, 0, 2, W, H, r_min=2.6, r_max=3.2)
    ref_np, _ = oracle_reference(c["ref"], views, H, W)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = Context(stream=stream)
        refs = torch.as_tensor(ref_np).cuda()
        dv = torch.from_numpy(views.view(np.uint8).copy()).cuda()
        direct = ctx.create_job(c["cand"], loss="l1")
        graphed = ctx.create_job(c["cand"], loss="l1")
        loss = torch.zeros(2, device="cuda")
        vpj = [len(views)]
        for job in (direct, graphed):  # sizes the scratch of both jobs
            B.adms_forward_loss(ctx.ctx, [job], dv, vpj, [(H, W)], [refs], loss)
            B.adms_backward(ctx.ctx, [job])
            B.adms_optimizer_step(ctx.ctx, [job])
        B.adms_graph_begin(ctx.ctx)
        B.adms_forward_loss(ctx.ctx, [graphed], dv, vpj, [(H, W)], [refs], loss[1:])
        B.adms_backward(ctx.ctx, [graphed])
        B.adms_optimizer_step(ctx.ctx, [graphed])
        g = B.adms_graph_end(ctx.ctx)
        for _ in range(3):
            B.adms_forward_loss(ctx.ctx, [direct], dv, vpj, [(H, W)], [refs], loss[:1])
            B.adms_backward(ctx.ctx, [direct])
            B.adms_optimizer_step(ctx.ctx, [direct])
            B.adms_graph_launch(ctx.ctx, g)
        torch.cuda.synchronize()
        pa, pb = ctx.params(direct), ctx.params(graphed)
        assert pa["t"] == pb["t"] == 4
        for name in ("pos", "kd", "nrm"):
            a = pa[name].double().cpu().numpy()
            b = pb[name].double().cpu().numpy()
            assert rel_l2(b, a) < 1e-6, name
        assert abs(float(loss[0]) - float(loss[1])) <= 1e-6 * abs(float(loss[0]))
        B.adms_graph_destroy(g)
        ctx.close()


def test_capture_refuses_new_scratch(gpu_lib):
    from paper_2104_03989_gb300 import binding as B
    from paper_2104_03989_gb300.engine import Context

    c = synth.config_small()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = Context(stream=stream)
        job = ctx.create_job(c["cand"], loss="l1")
        views = synth.fixed_view(64, 64)
        refs = torch.zeros((1, 64, 64, 3), device="cuda")
        dv = torch.from_numpy(views.view(np.uint8).copy()).cuda()
        loss = torch.zeros(1, device="cuda")
        torch.cuda.synchronize()
        B.adms_graph_begin(ctx.ctx)
        with pytest.raises(B.AdmsError) as err:
            B.adms_forward_loss(ctx.ctx, [job], dv, [1], [(64, 64)], [refs], loss)
        assert err.value.status == B.ADMS_ERR_STATE
        B.adms_graph_destroy(B.adms_graph_end(ctx.ctx))
        # after a warm-up call the same forward records fine
        B.adms_forward_loss(ctx.ctx, [job], dv, [1], [(64, 64)], [refs], loss)
        torch.cuda.synchronize()
        ctx.close()
