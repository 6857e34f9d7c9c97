"""Uneven jobs in one persistent launch per stage: each job's visibility,
image, loss and gradients are the same alone and in the mix (only the order
of floating-point atomics differs: within 1e-6 relative), before and after
the autotuner, and a batched step replays from a CUDA graph."""

import numpy as np
import pytest
import torch

import synth
from cases import rel_l2, sphere_scene as _scene

pytestmark = pytest.mark.gpu


SPECS = [  # (freq, texture, views, H, W, tessellation levels)
    (4, 64, 2, 96, 96, 0),
    (8, 128, 3, 80, 128, 0),
    (3, 32, 1, 64, 64, 1),
]


def _jobs(ctx):
    jobs, views, refs = [], [], []
    for k, (freq, tex, nv, H, W, tess) in enumerate(SPECS):
        jobs.append(ctx.create_job(_scene(freq, tex, 10 + k, tess), loss="logl1", seed=k))
        views.append(synth.sample_views(100 + k, 0, nv, W, H, r_min=2.4, r_max=3.2))
        rng = np.random.default_rng(200 + k)
        refs.append(torch.as_tensor(rng.uniform(0, 1, (nv, H, W, 3)).astype(np.float32)).cuda())
    return jobs, views, refs


def _state(ctx, job, shape):
    p = ctx.params(job)
    out = {"g_pos": p["g_pos"].double().cpu().numpy(), "keys": ctx.keys(job, shape).cpu().numpy()}
    for n in ("kd", "orm", "nrm"):
        out["g_" + n] = p["g_" + n + "_chain"].double().cpu().numpy()
    if "g_disp" in p:
        out["g_disp"] = p["g_disp"].double().cpu().numpy()
    return out


def _compare(a, b):
    np.testing.assert_array_equal(a["keys"], b["keys"])
    for k in a:
        if k != "keys":
            assert rel_l2(b[k], a[k]) < 1e-6, k


def test_jobs_alone_equal_jobs_in_the_mix(gpu_lib):
    from paper_2104_03989_gb300 import binding as B
    from paper_2104_03989_gb300.engine import Context

    ctx = Context()
    alone, views, refs = _jobs(ctx)
    mixed, _, _ = _jobs(ctx)
    shapes = [(s[2], s[3], s[4]) for s in SPECS]
    imgs_alone, losses_alone = [], []
    for j, v, r in zip(alone, views, refs):
        img = torch.zeros_like(r)
        losses_alone.append(float(ctx.forward_loss([j], [v], [r], out_img=[img])[0]))
        imgs_alone.append(img)
        ctx.backward([j])
    imgs_mix = [torch.zeros_like(r) for r in refs]
    losses_mix = ctx.forward_loss(mixed, views, refs, out_img=imgs_mix).cpu().numpy()
    ctx.backward(mixed)
    torch.cuda.synchronize()
    for k in range(len(SPECS)):
        _compare(_state(ctx, alone[k], shapes[k]), _state(ctx, mixed[k], shapes[k]))
        assert rel_l2(imgs_mix[k].cpu().numpy(), imgs_alone[k].cpu().numpy()) < 1e-6
        assert abs(losses_mix[k] - losses_alone[k]) <= 1e-6 * losses_alone[k]

    # the autotuner keeps the results and leaves the jobs untouched
    B.adms_autotune(ctx.ctx, mixed, np.ascontiguousarray(np.concatenate(views)), [len(v) for v in views],
                    [(r.shape[1], r.shape[2]) for r in refs], refs)
    tune = B.adms_ctx_tuning(ctx.ctx)
    assert tune["tile_w"] in (8, 16, 32)
    for j in alone:
        B.adms_job_zero_gradients(ctx.ctx, j)
    for j, v, r in zip(alone, views, refs):
        ctx.forward_loss([j], [v], [r])
        ctx.backward([j])
    ctx.forward_loss(mixed, views, refs)
    ctx.backward(mixed)
    torch.cuda.synchronize()
    for k in range(len(SPECS)):
        _compare(_state(ctx, alone[k], shapes[k]), _state(ctx, mixed[k], shapes[k]))
    ctx.close()


def test_batched_step_replays_from_a_graph(gpu_lib):
    from paper_2104_03989_gb300 import binding as B
    from paper_2104_03989_gb300.engine import Context

    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = Context(stream=stream)
        direct, views, refs = _jobs(ctx)
        graphed, _, _ = _jobs(ctx)
        dv = torch.from_numpy(np.concatenate([v.view(np.uint8) for v in views]).copy()).cuda()
        vpj = [len(v) for v in views]
        hw = [(r.shape[1], r.shape[2]) for r in refs]
        loss = torch.zeros(2 * len(SPECS), device="cuda")

        def step(jobs, out):
            B.adms_forward_loss(ctx.ctx, jobs, dv, vpj, hw, refs, out)
            B.adms_backward(ctx.ctx, jobs)
            B.adms_optimizer_step(ctx.ctx, jobs)

        step(direct, loss[:3])
        step(graphed, loss[3:])
        B.adms_graph_begin(ctx.ctx)
        step(graphed, loss[3:])
        g = B.adms_graph_end(ctx.ctx)
        for _ in range(2):
            step(direct, loss[:3])
            B.adms_graph_launch(ctx.ctx, g)
        torch.cuda.synchronize()
        for a, b in zip(direct, graphed):
            pa, pb = ctx.params(a), ctx.params(b)
            assert pa["t"] == pb["t"] == 3
            for n in ("pos", "kd", "nrm"):
                assert rel_l2(pb[n].double().cpu().numpy(), pa[n].double().cpu().numpy()) < 1e-6, n
        B.adms_graph_destroy(g)
        ctx.close()
