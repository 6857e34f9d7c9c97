"""Per-mip-level latent textures (Sec. 6, prefiltering): through the C ABI
against the float64 oracle on the same seeded inputs. The levels start as the
box-filter chain, so the first render equals the standard job's; every level's
own gradient within 1e-3 relative L2 of the oracle's; every level of every
texture after two Adam steps within 1e-4 (the tolerance of the standard
step test)."""

import numpy as np
import pytest
import torch

from oracle import step as S

from cases import chain_levels, oracle_grads, oracle_reference, plain_case, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case(gpu_lib):
    from paper_2104_03989_gb300.engine import Context

    c, views, H, W = plain_case(res=96, n_views=4, tex=128, ref_tex=128, ref_freq=24, seed=13)
    ref_np, _ = oracle_reference(c["ref"], views, H, W)
    ctx = Context()
    yield c, views, H, W, ref_np, ctx
    ctx.close()


def test_per_level_first_render_and_level_gradients(case):
    c, views, H, W, ref_np, ctx = case
    refs = torch.as_tensor(ref_np).cuda()
    std = ctx.create_job(c["cand"], loss="logl1")
    lev = ctx.create_job(c["cand"], loss="logl1", per_level_textures=True)
    imgs = [torch.zeros((len(views), H, W, 3), device="cuda") for _ in range(2)]
    ctx.forward_loss([std], [views], [refs], out_img=[imgs[0]])
    ctx.forward_loss([lev], [views], [refs], out_img=[imgs[1]])
    ctx.backward([lev])
    ctx.backward([std])
    torch.cuda.synchronize()
    assert torch.equal(imgs[0], imgs[1])
    orc = oracle_grads(c["cand"], views, ref_np, H, W, "logl1", per_level=True)
    assert rel_l2(imgs[1].cpu().numpy(), orc["img"]) < 1e-5
    p = ctx.params(lev)
    for name in ("kd", "orm", "nrm"):
        L = p[name + "_levels"]
        h, w = p[name].shape[:2]
        got = chain_levels(p["g_" + name + "_chain"].double().cpu().numpy(), h, w, L)
        sampled = 0
        for k in range(L):
            want = orc["grads"][name if k == 0 else f"{name}@{k}"]
            if np.linalg.norm(want) == 0:
                assert np.abs(got[k]).max() == 0, (name, k)   # unsampled level: no gradient on either side
                continue
            sampled += 1
            assert rel_l2(got[k], want) < 1e-3, (name, k, rel_l2(got[k], want))
        assert sampled >= 2, name
    ctx.destroy_job(std)
    ctx.destroy_job(lev)


def test_per_level_adam_steps_match_oracle(case):
    c, views, H, W, ref_np, ctx = case
    refs = torch.as_tensor(ref_np).cuda()
    job = ctx.create_job(c["cand"], loss="logl1", per_level_textures=True)
    ojob = S.OracleJob(c["cand"], loss="logl1", per_level=True)
    for _ in range(2):
        ctx.forward_loss([job], [views], [refs])
        ctx.backward([job])
        ctx.step([job])
        S.step(ojob, views, ref_np.astype(np.float64), H, W)
    torch.cuda.synchronize()
    p = ctx.params(job)
    assert p["t"] == 2
    for name in ("kd", "orm", "nrm"):
        L = p[name + "_levels"]
        h, w = p[name].shape[:2]
        got = chain_levels(p[name + "_chain"].double().cpu().numpy(), h, w, L)
        for k in range(L):
            want = ojob.params[name if k == 0 else f"{name}@{k}"].numpy()
            assert rel_l2(got[k], want) < 1e-4, (name, k, rel_l2(got[k], want))
    # the coarse levels were not rebuilt from level 0 (they are latents of their own)
    kd = chain_levels(p["kd_chain"].double().cpu().numpy(), *p["kd"].shape[:2], p["kd_levels"])
    box = kd[0].reshape(kd[0].shape[0] // 2, 2, kd[0].shape[1] // 2, 2, 4).mean(axis=(1, 3))
    assert not np.allclose(box, kd[1], atol=1e-6)
    pos = p["pos"].double().cpu().numpy()
    assert rel_l2(pos, ojob.params["pos"].numpy()) < 1e-4
    ctx.destroy_job(job)
