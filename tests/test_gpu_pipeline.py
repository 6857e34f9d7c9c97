"""Pipelined optimizer steps (adms_ctx_set_pipelining): each step's texture update
is deferred to the job's next forward_loss, where it runs beside the frame and
raster; every result equals that of sequential steps (only the order of
floating-point atomics differs: within 1e-6 relative), directly and from a CUDA
graph, and the texture memory itself shows the deferral."""

import numpy as np
import pytest
import torch

import synth
from cases import rel_l2, sphere_scene

pytestmark = pytest.mark.gpu

CASES = [  # (freq, texture, views, H, W, tessellation levels)
    (4, 64, 2, 96, 96, 0),
    (3, 32, 2, 64, 80, 1),
]


def _setup(ctx, case, k):
    freq, tex, nv, H, W, tess = case
    job = ctx.create_job(sphere_scene(freq, tex, 30 + k, tess), loss="logl1", seed=k)
    rng = np.random.default_rng(300 + k)
    refs = torch.as_tensor(rng.uniform(0, 1, (nv, H, W, 3)).astype(np.float32)).cuda()
    return job, refs


def _views(case, step):
    _, _, nv, H, W, _ = case
    return synth.sample_views(400 + step, 0, nv, W, H, r_min=2.4, r_max=3.2)


def _latents(ctx, job):
    p = ctx.params(job)
    out = {n: p[n].double().cpu().numpy() for n in ("pos", "kd_chain", "orm_chain", "nrm_chain")}
    if "disp" in p:
        out["disp"] = p["disp"].double().cpu().numpy()
    return p["t"], out


@pytest.mark.parametrize("case", CASES, ids=["plain", "tessellated"])
def test_pipelined_steps_equal_sequential_steps(gpu_lib, case):
    from paper_2104_03989_gb300.engine import Context

    seq, pipe = Context(), Context()
    pipe.set_pipelining(True)
    js, refs = _setup(seq, case, 0)
    jp, _ = _setup(pipe, case, 0)
    kd0 = pipe.params(jp)["kd"].clone()
    kd_view = pipe.params(jp)["kd"]  # read below without any call naming the job
    losses = []
    for step in range(4):
        v = _views(case, step)
        ls = float(seq.forward_loss([js], [v], [refs])[0])
        lp = float(pipe.forward_loss([jp], [v], [refs])[0])
        losses.append((ls, lp))
        seq.backward([js])
        pipe.backward([jp])
        seq.step([js])
        pipe.step([jp])
        if step == 0:
            # the first texture step is still deferred: level 0 of kd as it was
            torch.cuda.synchronize()
            assert torch.equal(kd_view, kd0)
    for ls, lp in losses:
        assert abs(lp - ls) <= 1e-6 * abs(ls), (ls, lp)
    ts, a = _latents(seq, js)
    tp, b = _latents(pipe, jp)  # adms_job_params issues the deferred step first
    assert ts == tp == 4
    for n in a:
        assert rel_l2(b[n], a[n]) < 1e-6, n
    h, w = kd0.shape[:2]
    assert not np.array_equal(b["kd_chain"][: h * w].reshape(h, w, 4), kd0.double().cpu().numpy())
    seq.close()
    pipe.close()


def test_pipelined_graph_replays_and_refuses_a_different_pending_set(gpu_lib):
    from paper_2104_03989_gb300 import binding as B
    from paper_2104_03989_gb300.engine import Context

    case = CASES[0]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        seq, pipe = Context(stream=stream), Context(stream=stream)
        pipe.set_pipelining(True)
        js, refs = _setup(seq, case, 1)
        jp, _ = _setup(pipe, case, 1)
        v = _views(case, 0)
        dv = torch.from_numpy(np.ascontiguousarray(v).view(np.uint8).reshape(-1).copy()).cuda()
        nv, H, W = case[2], case[3], case[4]
        loss = torch.zeros(2, device="cuda")

        def step(ctx, job, out):
            B.adms_forward_loss(ctx.ctx, [job], dv, [nv], [(H, W)], [refs], out)
            B.adms_backward(ctx.ctx, [job])
            B.adms_optimizer_step(ctx.ctx, [job])

        step(seq, js, loss[:1])
        step(pipe, jp, loss[1:])  # leaves the texture step deferred
        B.adms_graph_begin(pipe.ctx)
        step(pipe, jp, loss[1:])  # records the deferred step beside the raster
        g = B.adms_graph_end(pipe.ctx)
        for _ in range(3):
            step(seq, js, loss[:1])
            B.adms_graph_launch(pipe.ctx, g)
        torch.cuda.synchronize()
        assert abs(float(loss[1]) - float(loss[0])) <= 1e-6 * abs(float(loss[0]))
        ts, a = _latents(seq, js)
        tp, b = _latents(pipe, jp)  # issues the last replay's deferred step
        assert ts == tp == 4
        for n in a:
            assert rel_l2(b[n], a[n]) < 1e-6, n
        # nothing is deferred now: the graph, recorded with a deferred step, is refused
        with pytest.raises(B.AdmsError) as e:
            B.adms_graph_launch(pipe.ctx, g)
        assert e.value.status == B.ADMS_ERR_STATE
        B.adms_graph_destroy(g)
        seq.close()
        pipe.close()
