"""Checkpoint/resume: a job exported between optimizer steps and imported into
a new job continues exactly as the original (up to the order of float atomics:
within 1e-5 relative after two more steps), with the same step count and
schedules; blobs that do not match the job layout are refused."""

import numpy as np
import pytest
import torch

import synth

from cases import rel_l2, sphere_scene

pytestmark = pytest.mark.gpu


def _step(ctx, job, t, nv=2, res=64):
    views = synth.sample_views(5, t, nv, res, res, r_min=2.4, r_max=3.2)
    ref = torch.as_tensor(np.random.default_rng(100 + t).uniform(0, 1, (nv, res, res, 3)).astype(np.float32)).cuda()
    loss = ctx.forward_loss([job], [views], [ref])
    ctx.backward([job])
    ctx.step([job])
    return float(loss[0])


def _latents(ctx, job):
    p = ctx.params(job)
    out = {k: p[k].double().cpu().numpy() for k in ("pos", "kd", "orm", "nrm", "disp") if k in p and p[k] is not None}
    out["t"] = p["t"]
    return out


@pytest.mark.parametrize("tess,relative", [(0, False), (1, True)])
def test_export_import_resumes_the_run(gpu_lib, tess, relative):
    from paper_2104_03989_gb300.engine import Context

    ctx = Context()
    scene = sphere_scene(4, 64, 1, tess)
    opts = dict(loss="logl1", lr0=0.01, relative_laplacian=relative)
    a = ctx.create_job(scene, seed=7, **opts)
    for t in range(3):
        _step(ctx, a, t)
    blob = ctx.export_job(a)
    b = ctx.import_job(blob, scene, **opts)
    assert _latents(ctx, b)["t"] == 3
    sa, sb = ctx.stats(a), ctx.stats(b)
    assert sa["lam"] == sb["lam"] and sa["lr"] == sb["lr"] and sa["t"] == sb["t"]
    for t in (3, 4):
        la, lb = _step(ctx, a, t), _step(ctx, b, t)
        assert abs(la - lb) <= 1e-6 * abs(la)
    A, Bl = _latents(ctx, a), _latents(ctx, b)
    assert A["t"] == Bl["t"] == 5
    for k in A:
        if k != "t":
            assert rel_l2(Bl[k], A[k]) < 1e-5, k
    # a blob is only accepted by a job of the same layout
    from paper_2104_03989_gb300 import binding as B
    with pytest.raises(B.AdmsError) as e:
        ctx.import_job(blob, sphere_scene(4, 128, 1, tess), **opts)
    assert e.value.status == B.ADMS_ERR_ARG
    with pytest.raises(B.AdmsError):
        ctx.import_job(blob[:-4], scene, **opts)
    ctx.close()
