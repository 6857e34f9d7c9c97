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


def test_reference_render_on_a_second_stream_matches_one_stream(gpu_lib):
    """The reference rendered on its own stream, the loss waiting on its event
    (adms_ctx_set_ref_event), directly and captured into one graph across both
    streams, gives the step of the one-stream sequence."""
    from paper_2104_03989_gb300 import binding as B
    from paper_2104_03989_gb300.engine import Context

    c = synth.config_small()
    H = W = 128
    views = synth.sample_views(6, 0, 2, W, H, r_min=2.6, r_max=3.2)
    main, side = torch.cuda.Stream(), torch.cuda.Stream()
    fork, ready = torch.cuda.Event(), torch.cuda.Event()
    with torch.cuda.stream(main):
        ctx = Context(stream=main)
        dv = torch.from_numpy(views.view(np.uint8).copy()).cuda()
        ref_job = ctx.create_job(c["ref"], frozen=True)
        jobs = {k: ctx.create_job(c["cand"], loss="l1") for k in ("one", "two", "graph")}
        refs = {k: torch.zeros((2, H, W, 3), device="cuda") for k in jobs}
        loss = torch.zeros(3, device="cuda")

        def step(k, li, overlap):
            if overlap:
                fork.record(main)
                side.wait_event(fork)
                B.adms_ctx_set_stream(ctx.ctx, side)
            B.adms_render_reference(ctx.ctx, ref_job, dv.view(2, -1), H, W, refs[k])
            if overlap:
                ready.record(side)
                B.adms_ctx_set_stream(ctx.ctx, main)
                B.adms_ctx_set_ref_event(ctx.ctx, ready)
            B.adms_forward_loss(ctx.ctx, [jobs[k]], dv, [2], [(H, W)], [refs[k]], loss[li:li + 1])
            B.adms_ctx_set_ref_event(ctx.ctx, None)
            B.adms_backward(ctx.ctx, [jobs[k]])
            B.adms_optimizer_step(ctx.ctx, [jobs[k]])

        step("one", 0, False)
        step("two", 1, True)
        step("graph", 2, True)     # sizes the scratch before capture
        B.adms_graph_begin(ctx.ctx)
        step("graph", 2, True)
        g = B.adms_graph_end(ctx.ctx)
        for _ in range(2):
            step("one", 0, False)
            step("two", 1, True)
            B.adms_graph_launch(ctx.ctx, g)
        torch.cuda.synchronize()
        for k in ("two", "graph"):
            assert torch.equal(refs[k], refs["one"])
        p = {k: ctx.params(j) for k, j in jobs.items()}
        assert p["one"]["t"] == p["two"]["t"] == p["graph"]["t"] == 3
        for k in ("two", "graph"):
            for name in ("pos", "kd", "nrm"):
                a = p["one"][name].double().cpu().numpy()
                b = p[k][name].double().cpu().numpy()
                assert rel_l2(b, a) < 1e-6, (k, name)
        l = loss.cpu().numpy()
        assert abs(l[1] - l[0]) <= 1e-6 * abs(l[0]) and abs(l[2] - l[0]) <= 1e-6 * abs(l[0])
        B.adms_graph_destroy(g)
        ctx.close()


def test_pipelined_graphs_match_sequential_steps(gpu_lib):
    """The bench's pipelined step: two graphs alternate two view slots and two
    reference buffers; each renders the next batch's references on a second
    stream while the candidate steps on the current batch with the references the
    previous launch rendered. Four steps equal four sequential steps."""
    from paper_2104_03989_gb300 import binding as B
    from paper_2104_03989_gb300.engine import Context

    c = synth.config_small()
    H = W = 96
    n = 5
    views = [torch.from_numpy(synth.sample_views(8, i, 2, W, H, r_min=2.6, r_max=3.2).view(np.uint8).copy()).cuda()
             for i in range(n + 1)]
    main, side = torch.cuda.Stream(), torch.cuda.Stream()
    fork, join = torch.cuda.Event(), torch.cuda.Event()
    with torch.cuda.stream(main):
        ctx = Context(stream=main)
        ref_job = ctx.create_job(c["ref"], frozen=True)
        seq, pipe = ctx.create_job(c["cand"], loss="l1"), ctx.create_job(c["cand"], loss="l1")
        ref = torch.zeros((2, H, W, 3), device="cuda")
        bufs = [torch.zeros((2, H, W, 3), device="cuda") for _ in range(2)]
        slots = torch.zeros((2, views[0].numel()), dtype=torch.uint8, device="cuda")
        loss = torch.zeros(2, device="cuda")

        def seq_step(i, job):
            B.adms_render_reference(ctx.ctx, ref_job, views[i].view(2, -1), H, W, ref)
            B.adms_forward_loss(ctx.ctx, [job], views[i], [2], [(H, W)], [ref], loss[:1])
            B.adms_backward(ctx.ctx, [job])
            B.adms_optimizer_step(ctx.ctx, [job])

        def pipelined(cur):
            fork.record(main)
            side.wait_event(fork)
            B.adms_ctx_set_stream(ctx.ctx, side)
            B.adms_render_reference(ctx.ctx, ref_job, slots[1 - cur].view(2, -1), H, W, bufs[1 - cur])
            join.record(side)
            B.adms_ctx_set_stream(ctx.ctx, main)
            B.adms_forward_loss(ctx.ctx, [pipe], slots[cur], [2], [(H, W)], [bufs[cur]], loss[1:])
            B.adms_backward(ctx.ctx, [pipe])
            B.adms_optimizer_step(ctx.ctx, [pipe])
            main.wait_event(join)

        seq_step(0, seq)          # step 0 directly for both (sizes all scratch)
        seq_step(0, pipe)
        graphs = []
        for cur in (0, 1):
            B.adms_graph_begin(ctx.ctx)
            pipelined(cur)
            graphs.append(B.adms_graph_end(ctx.ctx))
        slots[0].copy_(views[1])
        B.adms_render_reference(ctx.ctx, ref_job, slots[0].view(2, -1), H, W, bufs[0])
        losses = []
        for s in range(4):
            seq_step(1 + s, seq)
            slots[1 - s % 2].copy_(views[2 + s])
            B.adms_graph_launch(ctx.ctx, graphs[s % 2])
            losses.append(loss.clone())
        torch.cuda.synchronize()
        for l in losses:
            assert abs(float(l[1]) - float(l[0])) <= 1e-6 * abs(float(l[0]))
        pa, pb = ctx.params(seq), ctx.params(pipe)
        assert pa["t"] == pb["t"] == 5
        for name in ("pos", "kd", "nrm"):
            assert rel_l2(pb[name].double().cpu().numpy(), pa[name].double().cpu().numpy()) < 1e-6, name
        for g in graphs:
            B.adms_graph_destroy(g)
        ctx.close()
