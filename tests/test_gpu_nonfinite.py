"""Failure detection on the device: a NaN in one job's texture, or in one job's
reference image, latches ADMS_ERR_NONFINITE in that job's status (read back in
stream order with adms_jobs_status); its optimizer steps are skipped, so its
latents never take a NaN from an update, and the other jobs of the same batched
calls get the results they get alone. Nothing here faults or hangs the GPU: the
NaNs are ordinary float inputs written from the host."""

import math

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

NONFINITE = -5
H = W = 96


def _scene():
    c = synth.config_small()
    views = synth.fixed_view(W, H)
    return c, views


def _poison_texture(ctx, job):
    """NaN over a 24 x 24 block of the base colour at the centre of the visible
    hemisphere (u ~ 3/4, v ~ 1/2 seen from +z), mip chain rebuilt from it."""
    from paper_2104_03989_gb300 import binding as B

    kd = ctx.params(job)["kd"]
    h, w = kd.shape[0], kd.shape[1]
    kd[h // 2 - 12: h // 2 + 12, 3 * w // 4 - 12: 3 * w // 4 + 12, :3] = float("nan")
    B.adms_job_invalidate(ctx.ctx, job)


def _latents(ctx, job):
    p = ctx.params(job)
    return {n: p[n].detach().clone() for n in ("pos", "kd", "nrm")}


def test_nonfinite_jobs_are_latched_skipped_and_leave_the_others_unchanged(gpu_lib):
    from paper_2104_03989_gb300.engine import Context

    c, views = _scene()
    ctx = Context()
    ref_job = ctx.create_job(c["ref"], frozen=True)
    ref = ctx.render_reference(ref_job, views, H, W)
    A, Bj, Cj = (ctx.create_job(c["cand"], loss="l1") for _ in range(3))
    _poison_texture(ctx, A)
    ref_b = ref.clone()
    ref_b[0, H // 2, W // 2, 1] = float("nan")
    before = {j: _latents(ctx, j) for j in (A, Bj)}
    for _ in range(2):
        ctx.forward_loss([A, Bj, Cj], [views] * 3, [ref, ref_b, ref])
        ctx.backward([A, Bj, Cj])
        ctx.step([A, Bj, Cj])
    status = ctx.jobs_status([A, Bj, Cj]).cpu().numpy()
    assert list(status) == [NONFINITE, NONFINITE, 0]
    assert ctx.stats(A)["status"] == NONFINITE and ctx.stats(Cj)["status"] == 0
    # the latched jobs were not updated: their latents are as they were (the injected
    # NaN block aside) and finite
    for j in (A, Bj):
        now = _latents(ctx, j)
        for n, t in now.items():
            same = (t == before[j][n]) | (torch.isnan(t) & torch.isnan(before[j][n]))
            assert bool(same.all()), (j, n)
    assert bool(torch.isfinite(_latents(ctx, Bj)["kd"]).all())
    # the healthy job equals the same job run alone
    D = ctx.create_job(c["cand"], loss="l1")
    for _ in range(2):
        ctx.forward_loss([D], [views], [ref])
        ctx.backward([D])
        ctx.step([D])
    got, want = _latents(ctx, Cj), _latents(ctx, D)
    for n in got:
        assert bool(torch.isfinite(got[n]).all())
        err = float((got[n] - want[n]).double().norm() / want[n].double().norm())
        assert err < 1e-5, (n, err)
    assert list(ctx.jobs_status([D]).cpu().numpy()) == [0]
    ctx.close()


def test_single_job_with_a_nan_texture_is_latched_and_not_updated(gpu_lib):
    from paper_2104_03989_gb300.engine import Context

    c, views = _scene()
    ctx = Context()
    ref = ctx.render_reference(ctx.create_job(c["ref"], frozen=True), views, H, W)
    job = ctx.create_job(c["cand"], loss="l1")
    _poison_texture(ctx, job)
    before = _latents(ctx, job)
    loss = ctx.forward_loss([job], [views], [ref])
    ctx.backward([job])
    ctx.step([job])
    assert not math.isfinite(float(loss[0]))
    assert ctx.stats(job)["status"] == NONFINITE
    after = _latents(ctx, job)
    assert bool((after["pos"] == before["pos"]).all()) and bool(torch.isfinite(after["pos"]).all())
    ctx.close()


def test_adam_wait_that_runs_out_latches_a_timeout_and_the_context_stays_usable(gpu_lib):
    """The streamed texture Adam waits on the device for each tile's TMA copies,
    bounded by 2 s of the GPU's global timer. The test hook makes every such wait
    expect 16 bytes more than its copies deliver (a phase that never completes):
    the waits run out, the job latches ADMS_ERR_TIMEOUT and its textures are not
    updated; with the hook off, the same context steps another job normally.
    Nothing faults: every copy lands, only the barrier's byte count stays short."""
    from paper_2104_03989_gb300 import binding as B
    from paper_2104_03989_gb300.engine import Context

    TIMEOUT = -4
    c, views = _scene()
    ctx = Context()
    ref_job = ctx.create_job(c["ref"], frozen=True)
    ref = ctx.render_reference(ref_job, views, H, W)
    job = ctx.create_job(c["cand"], loss="l1")
    before = _latents(ctx, job)
    ctx.forward_loss([job], [views], [ref])
    ctx.backward([job])
    B.adms_ctx_test_wait_timeout(ctx.ctx, True)
    ctx.step([job])
    B.adms_ctx_test_wait_timeout(ctx.ctx, False)
    torch.cuda.synchronize()
    assert int(ctx.jobs_status([job]).cpu()[0]) == TIMEOUT
    assert ctx.stats(job)["status"] == TIMEOUT
    now = _latents(ctx, job)
    for n in ("kd", "nrm"):
        assert torch.equal(now[n], before[n]), n
    # the context still runs a normal step
    other = ctx.create_job(c["cand"], loss="l1")
    start = _latents(ctx, other)
    ctx.forward_loss([other], [views], [ref])
    ctx.backward([other])
    ctx.step([other])
    torch.cuda.synchronize()
    assert int(ctx.jobs_status([other]).cpu()[0]) == 0
    moved = _latents(ctx, other)
    assert not torch.equal(moved["kd"], start["kd"])
    assert bool(torch.isfinite(moved["kd"]).all())
    ctx.close()
