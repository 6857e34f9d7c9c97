"""GPU path (through the C ABI) against the float64 oracle on identical seeded inputs.

Bars: visibility keys bit-exact; images within 1e-5 relative L2; gradients
within 1e-3 relative L2 (per latent); latents after Adam steps within 1e-4
relative L2 (Adam divides each coordinate by its own |g|, so coordinates whose
gradient is near eps amplify float32 rounding)."""

import numpy as np
import pytest
import torch

import synth
from oracle import step as S
from oracle import visibility as OV

from cases import (fold_mips, oracle_grads, oracle_reference, plain_case, rel_l2, small_case, tess_case,
                   unambiguous_inputs)

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-5
GRAD_TOL = 1e-3
STEP_TOL = 1e-4


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    from paper_2104_03989_gb300.engine import Context

    c = Context()
    yield c
    c.close()


def _keys_np(ctx, job, B, H, W):
    k = ctx.keys(job, (B, H, W)).cpu().numpy().view(np.uint64)
    return k


def _run_case(ctx, case, loss, unambiguous=False):
    """unambiguous: run on inputs where every kink of the forward is decided alike at
    float32 and float64 (cases.unambiguous_inputs); returns the candidate scene used."""
    c, views, H, W = case
    ref_np, _ = oracle_reference(c["ref"], views, H, W)
    cand = c["cand"]
    if unambiguous:
        cand, ref_np = unambiguous_inputs(cand, views, ref_np, H, W, loss)
    refs = torch.as_tensor(ref_np).cuda()
    job = ctx.create_job(cand, loss=loss, lr0=0.01)
    img = torch.zeros((len(views), H, W, 3), device="cuda")
    loss_t = ctx.forward_loss([job], [views], [refs], out_img=[img])
    keys = _keys_np(ctx, job, len(views), H, W)
    ctx.backward([job])
    torch.cuda.synchronize()
    p = ctx.params(job)
    grads = {"pos": p["g_pos"].double().cpu().numpy()}
    for name in ("kd", "orm", "nrm"):
        if p["g_" + name] is not None:
            grads[name] = fold_mips(p["g_" + name + "_chain"].cpu(), *p[name].shape[:2], p[name + "_levels"]).numpy()
    return dict(job=job, refs=refs, ref_np=ref_np, img=img.cpu().numpy(), loss=float(loss_t[0]), keys=keys,
                grads=grads, cand=cand)


@pytest.fixture(scope="module")
def small(ctx):
    case = small_case()
    gpu = _run_case(ctx, case, "l1", unambiguous=True)
    orc = oracle_grads(gpu["cand"], case[1], gpu["ref_np"], case[2], case[3], "l1")
    return case, gpu, orc


@pytest.fixture(scope="module")
def plain(ctx):
    case = plain_case()
    gpu = _run_case(ctx, case, "logl1", unambiguous=True)
    orc = oracle_grads(gpu["cand"], case[1], gpu["ref_np"], case[2], case[3], "logl1")
    return case, gpu, orc


@pytest.mark.parametrize("which", ["small", "plain"])
def test_keys_bit_exact(which, request):
    case, gpu, orc = request.getfixturevalue(which)
    assert gpu["keys"].dtype == np.uint64
    np.testing.assert_array_equal(gpu["keys"], orc["keys"])
    assert (gpu["keys"] != OV.EMPTY_KEY).any()


@pytest.mark.parametrize("which", ["small", "plain"])
def test_images_and_loss(which, request):
    case, gpu, orc = request.getfixturevalue(which)
    assert rel_l2(gpu["img"], orc["img"]) < IMG_TOL
    assert abs(gpu["loss"] - orc["loss"]) / orc["loss"] < IMG_TOL


@pytest.mark.parametrize("which", ["small", "plain"])
def test_gradients(which, request):
    """Per latent within 1e-3 relative L2. Vertex gradients touched by a pixel
    sitting on a kink of the forward (texel-cell boundary, n.l = 0, AA
    crossing thresholds, L1 sign) are one-sided and not unique: those
    vertices are additionally checked for validity (each within 50% of the
    oracle's one-sided value); the whole vector, those vertices included, is
    held to 1e-3 as well."""
    case, gpu, orc = request.getfixturevalue(which)
    for name, want in orc["grads"].items():
        got = gpu["grads"][name]
        assert np.linalg.norm(want) > 0, name
        if name == "pos":
            amb = np.zeros(len(want), bool)
            amb[sorted(orc["ambiguous"])] = True
            assert amb.mean() < 0.3, f"{amb.sum()} ambiguous vertices"
            err = rel_l2(got[~amb], want[~amb])
            print(f"{which} pos: {amb.sum()} of {len(amb)} vertices one-sided; rel L2 of the rest {err:.3e}, "
                  f"of all {rel_l2(got, want):.3e}")
            # one-sided vertices: same direction and magnitude to within the texel jump
            for v in np.nonzero(amb)[0]:
                assert np.linalg.norm(got[v] - want[v]) <= 0.5 * np.linalg.norm(want[v]) + 1e-3 * np.abs(want).max()
            assert rel_l2(got, want) < GRAD_TOL, f"pos: rel L2 of all vertices {rel_l2(got, want):.3e}"
        else:
            err = rel_l2(got, want)
        assert err < GRAD_TOL, f"{name}: rel L2 {err:.3e}"


@pytest.fixture(scope="module")
def tess(ctx):
    case = tess_case()
    c, views, H, W = case
    gpu = _run_case(ctx, case, "logl1")
    orc = oracle_grads(c["cand"], views, gpu["ref_np"], H, W, "logl1")
    p = ctx.params(gpu["job"])
    gpu["grads"]["disp"] = p["g_disp"].double().cpu().numpy()
    return case, gpu, orc


def test_tessellated_keys_images_and_gradients(tess):
    """Tessellated + displaced render mesh (Sec. 5.1, Eq. 3): keys bit-exact
    (float32 contract of the displaced positions), images within 1e-5,
    gradients w.r.t. base positions, displacement and normal map within 1e-3."""
    case, gpu, orc = tess
    np.testing.assert_array_equal(gpu["keys"], orc["keys"])
    assert (gpu["keys"] != OV.EMPTY_KEY).any()
    assert rel_l2(gpu["img"], orc["img"]) < IMG_TOL
    for name in ("disp", "nrm"):
        err = rel_l2(gpu["grads"][name], orc["grads"][name])
        print(f"tess {name}: rel L2 {err:.3e}")
        assert err < GRAD_TOL, name
    want, got = orc["grads"]["pos"], gpu["grads"]["pos"]
    amb = np.zeros(len(want), bool)
    amb[sorted(orc["ambiguous"])] = True
    err = rel_l2(got[~amb], want[~amb])
    print(f"tess pos: {amb.sum()} of {len(amb)} base vertices one-sided; rel L2 of the rest {err:.3e}")
    assert err < GRAD_TOL
    assert rel_l2(got, want) < GRAD_TOL, f"tess pos: rel L2 of all base vertices {rel_l2(got, want):.3e}"


def test_reference_render_parity(ctx):
    c, views, H, W = plain_case()
    ref_np, okeys = oracle_reference(c["ref"], views, H, W)
    rjob = ctx.create_job(c["ref"], frozen=True)
    out = ctx.render_reference(rjob, views, H, W)
    keys = _keys_np(ctx, rjob, len(views), H, W)
    np.testing.assert_array_equal(keys, okeys)
    assert rel_l2(out.cpu().numpy(), ref_np) < IMG_TOL
    ctx.destroy_job(rjob)


def test_adam_step_matches_oracle(ctx):
    case = small_case()
    c, views, H, W = case
    ref_np, _ = oracle_reference(c["ref"], views, H, W)
    refs = torch.as_tensor(ref_np).cuda()
    job = ctx.create_job(c["cand"], loss="l1", lr0=0.01)
    ojob = S.OracleJob(c["cand"], loss="l1", lr0=0.01)
    for it in range(2):
        ctx.forward_loss([job], [views], [refs])
        ctx.backward([job])
        ctx.step([job])
        S.step(ojob, views, ref_np.astype(np.float64), H, W)
    torch.cuda.synchronize()
    p = ctx.params(job)
    st = ctx.stats(job)
    assert st["t"] == 2
    assert abs(st["lam"] - ojob.lam) / ojob.lam < 1e-4
    for name in ("pos", "kd", "nrm"):
        got = p[name].double().cpu().numpy()
        want = ojob.params[name].numpy()
        err = rel_l2(got, want)
        worst = float(np.abs(got - want).max())
        assert err < STEP_TOL, f"{name}: rel L2 {err:.3e}, max abs {worst:.3e}"
    ctx.destroy_job(job)


def test_ragged_size_and_empty_view(ctx):
    """Image sizes that are not tile multiples, and a view that sees nothing."""
    c = synth.config_small()
    H, W = 75, 100
    views = synth.sample_views(3, 0, 2, W, H, r_min=2.5, r_max=3.0)
    # second view looks away from the mesh: everything is behind the camera
    from synth.views import look_at, perspective
    mvp = perspective(aspect=W / H) @ look_at((0.0, 0.0, 3.0), (0.0, 0.0, 6.0))
    views[1]["mvp"] = mvp.reshape(-1).astype(np.float32)
    ref_np, okeys = oracle_reference(c["ref"], views, H, W)
    assert (okeys[1] == OV.EMPTY_KEY).all()
    refs = torch.as_tensor(ref_np).cuda()
    job = ctx.create_job(c["cand"], loss="l1")
    img = torch.zeros((2, H, W, 3), device="cuda")
    ctx.forward_loss([job], [views], [refs], out_img=[img])
    keys = _keys_np(ctx, job, 2, H, W)
    ctx.backward([job])
    torch.cuda.synchronize()
    orc = oracle_grads(c["cand"], views, ref_np, H, W, "l1")
    np.testing.assert_array_equal(keys, orc["keys"])
    assert (keys[1] == OV.EMPTY_KEY).all()
    assert rel_l2(img.cpu().numpy(), orc["img"]) < IMG_TOL
    p = ctx.params(job)
    assert rel_l2(p["g_pos"].double().cpu().numpy(), orc["grads"]["pos"]) < GRAD_TOL
    ctx.destroy_job(job)


def test_negative_reference_radiance(ctx):
    """The tone map counts negative radiance as black on both sides (a pixel
    below -1 has no log(x + 1)): a reference with patches at -2.5 and -0.5
    gives a finite loss and the oracle's loss and gradients."""
    c, views, H, W = plain_case(res=64, n_views=2, tex=64, ref_tex=64, ref_freq=16, seed=9)
    ref_np, _ = oracle_reference(c["ref"], views, H, W)
    ref_np = ref_np.copy()
    ref_np[0, 20:36, 20:36, :] = -2.5
    ref_np[1, 10:30, 30:50, 1] = -0.5
    refs = torch.as_tensor(ref_np).cuda()
    job = ctx.create_job(c["cand"], loss="logl1", lr0=0.01)
    loss = float(ctx.forward_loss([job], [views], [refs])[0])
    ctx.backward([job])
    torch.cuda.synchronize()
    orc = oracle_grads(c["cand"], views, ref_np, H, W, "logl1")
    assert np.isfinite(loss) and abs(loss - orc["loss"]) / orc["loss"] < IMG_TOL
    p = ctx.params(job)
    got = fold_mips(p["g_kd_chain"].cpu(), *p["kd"].shape[:2], p["kd_levels"]).numpy()
    assert rel_l2(got, orc["grads"]["kd"]) < GRAD_TOL
    ctx.destroy_job(job)
