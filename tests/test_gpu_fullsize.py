"""Parity at the full sizes of the throughput workloads, with the batch sizes
and resolutions the bench times.

Plain method (200,000-tri reference with 2048² maps, 5,120-tri candidate with
1024² maps, 8 views at 512²): every view's visibility bit-exact against the
oracle for both meshes; one full-size view's reference image, candidate image,
loss and gradients against the float64 oracle.

Aggregate-geometry workload (1.2M-tri leaf canopy rasterized with the warp-wide
direct path, 11k-tri billboards with 8 depth-peeling layers, 8 views at 512²):
every view's reference visibility and every layer of every view's candidate
visibility bit-exact; one full-size view's image, loss and gradients against the
float64 oracle (a seeded reference image).

Displacement workload (1,003,520-tri reference, 980-tri base mesh tessellated
to 62,720 tris, 16 views at 1024²): every view's visibility bit-exact for both
meshes (the oracle's float32 contract of the displaced positions), and central
differences (h = 1e-3) of the autograd Function, raster buffers recomputed in
its backward, on 64 random normal-map texels against its analytic gradient."""

import numpy as np
import pytest
import torch

import synth
from oracle import step as S
from oracle import visibility as OV

from cases import assert_grads_match, fold_mips, oracle_grads, oracle_reference, rel_l2

pytestmark = pytest.mark.gpu


def _keys(ctx, job, shape):
    return ctx.keys(job, shape).cpu().numpy().view(np.uint64)


@pytest.fixture(scope="module")
def plain_full(gpu_lib):
    from paper_2104_03989_gb300.engine import Context

    c = synth.config_plain()
    views = synth.sample_views(7, 0, 8, 512, 512)
    ctx = Context()
    ref = ctx.create_job(c["ref"], frozen=True)
    cand = ctx.create_job(c["cand"], loss="logl1")
    yield c, views, ctx, ref, cand
    ctx.close()


def test_plain_full_size_visibility(plain_full):
    c, views, ctx, ref, cand = plain_full
    ctx.render_reference(ref, views, 512, 512)
    want, _ = OV.raster_views(views, c["ref"].mesh.pos, c["ref"].mesh.tri_pos, 512, 512)
    np.testing.assert_array_equal(_keys(ctx, ref, (8, 512, 512)), want)
    zeros = torch.zeros((8, 512, 512, 3), device="cuda")
    ctx.forward_loss([cand], [views], [zeros])
    ctx.backward([cand])   # leaves the job without a pending forward
    want, _ = OV.raster_views(views, c["cand"].mesh.pos, c["cand"].mesh.tri_pos, 512, 512)
    got = _keys(ctx, cand, (8, 512, 512))
    np.testing.assert_array_equal(got, want)
    assert (got != OV.EMPTY_KEY).mean() > 0.3


def test_plain_full_size_images_and_gradients(plain_full):
    c, views, ctx, ref, cand = plain_full
    from paper_2104_03989_gb300 import binding as B

    v0 = views[:1]
    ref_np, _ = oracle_reference(c["ref"], v0, 512, 512)
    gpu_ref = ctx.render_reference(ref, v0, 512, 512).cpu().numpy()
    assert rel_l2(gpu_ref, ref_np) < 1e-5
    B.adms_job_zero_gradients(ctx.ctx, cand)
    img = torch.zeros((1, 512, 512, 3), device="cuda")
    loss = float(ctx.forward_loss([cand], [v0], [torch.as_tensor(ref_np).cuda()], out_img=[img])[0])
    ctx.backward([cand])
    torch.cuda.synchronize()
    orc = oracle_grads(c["cand"], v0, ref_np, 512, 512, "logl1")
    assert rel_l2(img.cpu().numpy(), orc["img"]) < 1e-5
    assert abs(loss - orc["loss"]) / orc["loss"] < 1e-5
    p = ctx.params(cand)
    got = {"pos": p["g_pos"].double().cpu().numpy()}
    for name in ("kd", "orm", "nrm"):
        got[name] = fold_mips(p["g_" + name + "_chain"].cpu(), *p[name].shape[:2], p[name + "_levels"]).numpy()
    assert_grads_match(got, orc, "plain full size")


@pytest.fixture(scope="module")
def tess_full(gpu_lib):
    from paper_2104_03989_gb300.engine import Context

    c = synth.config_tess()
    c["cand"].disp = np.random.default_rng(3).uniform(-0.02, 0.02, c["cand"].disp.shape).astype(np.float32)
    views = synth.sample_views(11, 0, 16, 1024, 1024, r_min=2.5, r_max=3.5)
    ctx = Context()
    ref = ctx.create_job(c["ref"], frozen=True)
    cand = ctx.create_job(c["cand"], loss="logl1")
    yield c, views, ctx, ref, cand
    ctx.close()


def test_tess_full_size_visibility(tess_full):
    c, views, ctx, ref, cand = tess_full
    ctx.render_reference(ref, views, 1024, 1024)
    want, _ = OV.raster_views(views, c["ref"].mesh.pos, c["ref"].mesh.tri_pos, 1024, 1024)
    np.testing.assert_array_equal(_keys(ctx, ref, (16, 1024, 1024)), want)
    zeros = torch.zeros((16, 1024, 1024, 3), device="cuda")
    ctx.forward_loss([cand], [views], [zeros])
    ctx.backward([cand])
    job = S.OracleJob(c["cand"])
    pos32 = job.tess.positions_f32(job.params["pos"].numpy(), job.tri_np, job.params["disp"].numpy())
    want, _ = OV.raster_views(views, pos32, job.tess.tri, 1024, 1024)
    got = _keys(ctx, cand, (16, 1024, 1024))
    np.testing.assert_array_equal(got, want)
    assert (got != OV.EMPTY_KEY).mean() > 0.3


def test_tess_full_size_autograd_finite_differences(tess_full):
    from paper_2104_03989_gb300 import autograd as AG

    c, views, ctx, ref, cand = tess_full
    rng = np.random.default_rng(5)
    refs = torch.as_tensor(rng.uniform(0, 1, (16, 1024, 1024, 3)).astype(np.float32)).cuda()
    lat = AG.latents(ctx, cand)
    assert set(lat) == {"pos", "nrm", "disp"}
    L = AG.render_loss(ctx, cand, views, refs, lat)
    L.backward()
    g = lat["nrm"].grad.reshape(-1)
    nz = torch.nonzero(g.abs() > 1e-3 * g.abs().max()).squeeze(1).cpu().numpy()
    picks = rng.choice(nz, size=64, replace=False)
    errs = []
    with torch.no_grad():
        flat = lat["nrm"].view(-1)
        for i in picks:
            x0 = float(flat[i])
            vals = []
            for s in (1, -1):
                flat[i] = x0 + s * 1e-3
                AG.invalidate(ctx, cand)
                ctx.forward_loss([cand], [views], [refs])
                vals.append(ctx.stats(cand)["call_loss"])
            flat[i] = x0
            AG.invalidate(ctx, cand)
            fd = (vals[0] - vals[1]) / 2e-3
            an = float(g[i])
            errs.append(abs(fd - an) / abs(an))
    errs = np.array(errs)
    print(f"tess full size: FD rel error median {np.median(errs):.2e}, 90th pct {np.percentile(errs, 90):.2e}")
    assert np.median(errs) < 1e-3
    assert (errs < 1e-2).mean() >= 0.9


@pytest.fixture(scope="module")
def agg_full(gpu_lib):
    from paper_2104_03989_gb300.engine import Context

    c = synth.config_aggregate()
    views = synth.sample_views(9, 0, 8, 512, 512)
    ctx = Context()
    ref = ctx.create_job(c["ref"], frozen=True, raster_direct_px=256, raster_depth_filter=True)
    cand = ctx.create_job(c["cand"], loss="l2", layers=8)
    yield c, views, ctx, ref, cand
    ctx.close()


def test_aggregate_full_size_visibility(agg_full):
    c, views, ctx, ref, cand = agg_full
    refs = ctx.render_reference(ref, views, 512, 512)
    want, _ = OV.raster_views(views, c["ref"].mesh.pos, c["ref"].mesh.tri_pos, 512, 512)
    np.testing.assert_array_equal(_keys(ctx, ref, (8, 512, 512)), want)
    ctx.forward_loss([cand], [views], [refs])
    ctx.backward([cand])
    want, _ = OV.raster_views_peeled(views, c["cand"].mesh.pos, c["cand"].mesh.tri_pos, 512, 512, 8)
    got = _keys(ctx, cand, (8, 8, 512, 512))
    np.testing.assert_array_equal(got, want.transpose(1, 0, 2, 3))
    assert (got[7] != OV.EMPTY_KEY).mean() > 0.2     # the eighth layer is in use


def test_aggregate_full_size_image_and_gradients(agg_full):
    c, views, ctx, ref, cand = agg_full
    v1 = views[:1]
    ref_np = np.random.default_rng(17).uniform(0.0, 0.3, (1, 512, 512, 3)).astype(np.float32)
    job = ctx.create_job(c["cand"], loss="l2", layers=8)
    img = torch.zeros((1, 512, 512, 3), device="cuda")
    loss = float(ctx.forward_loss([job], [v1], [torch.as_tensor(ref_np).cuda()], out_img=[img])[0])
    ctx.backward([job])
    torch.cuda.synchronize()
    orc = oracle_grads(c["cand"], v1, ref_np, 512, 512, "l2", layers=8)
    assert rel_l2(img.cpu().numpy(), orc["img"]) < 1e-5
    assert abs(loss - orc["loss"]) / orc["loss"] < 1e-5
    p = ctx.params(job)
    got = {"pos": p["g_pos"].double().cpu().numpy()}
    for name in ("kd", "orm", "nrm"):
        got[name] = fold_mips(p["g_" + name + "_chain"].cpu(), *p[name].shape[:2], p[name + "_levels"]).numpy()
    assert_grads_match(got, orc, "aggregate full size")
    ctx.destroy_job(job)
