"""Dense skinning (Eq. 2) through the C ABI against the float64 oracle on the
same seeded inputs: visibility of the skinned mesh bit-exact (both sides follow
one float32 evaluation of the skinned positions, which both then shade; the
oracle differentiates them through its float64 operator), images within 1e-5,
gradients of rest positions, weights and textures within 1e-3, two Adam steps
under two animation frames within 1e-4, and a checkpoint that brings the
skinning back."""

import numpy as np
import pytest
import torch

import synth
from oracle import step as S

from cases import assert_grads_match, fold_mips, oracle_grads, oracle_reference, rel_l2, sphere_scene

pytestmark = pytest.mark.gpu

N_BONES, H, W = 6, 96, 96


@pytest.fixture(scope="module")
def rig(gpu_lib):
    from paper_2104_03989_gb300.engine import Context

    cand = sphere_scene(6, 64, 1)
    ref = sphere_scene(16, 64, 51)
    weights = synth.bone_weights(cand.mesh.pos, N_BONES, seed=4)
    poses = [synth.bone_pose(N_BONES, 4, f) for f in range(2)]
    views = [synth.sample_views(21, f, 3, W, H, r_min=2.4, r_max=3.0) for f in range(2)]
    refs = [oracle_reference(ref, views[f], H, W)[0] for f in range(2)]
    ctx = Context()
    yield cand, weights, poses, views, refs, ctx
    ctx.close()


def test_skinned_visibility_images_and_gradients(rig):
    cand, weights, poses, views, refs, ctx = rig
    job = ctx.create_job(cand, loss="logl1")
    ctx.skinning(job, weights)
    ctx.set_bones(job, poses[0])
    img = torch.zeros((3, H, W, 3), device="cuda")
    loss = float(ctx.forward_loss([job], [views[0]], [torch.as_tensor(refs[0]).cuda()], out_img=[img])[0])
    keys = ctx.keys(job, (3, H, W)).cpu().numpy().view(np.uint64)
    ctx.backward([job])
    torch.cuda.synchronize()
    orc = oracle_grads(cand, views[0], refs[0], H, W, "logl1", skin_weights=weights, bones=poses[0])
    np.testing.assert_array_equal(keys, orc["keys"])
    assert rel_l2(img.cpu().numpy(), orc["img"]) < 1e-5
    assert abs(loss - orc["loss"]) / orc["loss"] < 1e-5
    p = ctx.params(job)
    got = {"pos": p["g_pos"].double().cpu().numpy(), "w": p["g_w"].double().cpu().numpy()}
    for name in ("kd", "orm", "nrm"):
        got[name] = fold_mips(p["g_" + name + "_chain"].cpu(), *p[name].shape[:2], p[name + "_levels"]).numpy()
    assert_grads_match(got, orc, "skinned")
    ctx.destroy_job(job)


def test_skinned_adam_steps_over_two_frames_and_checkpoint(rig):
    cand, weights, poses, views, refs, ctx = rig
    job = ctx.create_job(cand, loss="logl1")
    ctx.skinning(job, weights)
    ojob = S.OracleJob(cand, loss="logl1", skin_weights=weights)
    ojob.shade_f32_skin = True
    for f in range(2):
        ctx.set_bones(job, poses[f])
        ctx.forward_loss([job], [views[f]], [torch.as_tensor(refs[f]).cuda()])
        ctx.backward([job])
        ctx.step([job])
        ojob.bones = torch.as_tensor(poses[f].astype(np.float64))
        S.step(ojob, views[f], refs[f].astype(np.float64), H, W)
    torch.cuda.synchronize()
    p = ctx.params(job)
    assert p["t"] == 2
    for name in ("pos", "w", "kd", "nrm"):
        got = p[name].double().cpu().numpy()
        want = ojob.params[name].numpy()
        assert rel_l2(got, want) < 1e-4, (name, rel_l2(got, want))
    assert not np.allclose(p["w"].cpu().numpy(), weights)   # the weights are latents and moved

    # a checkpoint brings the skinning back: weights, moments and the last bones
    blob = ctx.export_job(job)
    job2 = ctx.import_job(blob, cand, loss="logl1")
    p2 = ctx.params(job2)
    assert torch.equal(p2["w"], p["w"]) and p2["t"] == 2
    k1, k2 = [], []
    for j, keys in ((job, k1), (job2, k2)):
        ctx.forward_loss([j], [views[1]], [torch.as_tensor(refs[1]).cuda()])
        keys.append(ctx.keys(j, (3, H, W)).cpu().numpy())
        ctx.backward([j])
    np.testing.assert_array_equal(k1[0], k2[0])
    ctx.destroy_job(job)
    ctx.destroy_job(job2)
