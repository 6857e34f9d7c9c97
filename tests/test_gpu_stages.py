"""The per-stage C calls (adms_{frame,setup,raster,shade,aa_loss,mip}_{fwd,bwd})
behind their torch.autograd.Functions.

Chained, they give the oracle's keys bit for bit, its loss within 1e-5 and its
gradients within 1e-3 (whole vectors), and the whole-step call's gradients; in
recompute mode (raster buffers rebuilt in the backward) the same gradients. Each
stage's backward is checked by central differences of its own forward on at
least 64 parameters, positions included, with visibility and texture LOD held
fixed (keep_keys), as the adjoints assume. Steps: 1e-3 for positions where no
texture is read (frame, setup + raster), 1e-4 for positions moving texture
coordinates (a step of 1e-3 moves them by ~0.04 texel and crosses the kinks of
the piecewise-bilinear filter) and for colours entering |.| of the loss, 1e-2 for
texels (shading is linear in the base colour, smooth in the normal map)."""

import numpy as np
import pytest
import torch

from cases import oracle_grads, oracle_reference, plain_case, rel_l2, small_case, unambiguous_inputs

pytestmark = pytest.mark.gpu



def _inputs(which):
    from paper_2104_03989_gb300 import stages as ST

    case, loss = (small_case(), "l1") if which == "small" else (plain_case(), "logl1")
    c, views, H, W = case
    ref_np, _ = oracle_reference(c["ref"], views, H, W)
    cand, ref_np = unambiguous_inputs(c["cand"], views, ref_np, H, W, loss)
    m = cand.mesh
    pipe = ST.Pipeline(m.tri_pos, m.uv, m.tri_uv, m.n_verts, views, H, W)
    lat = {"pos": torch.tensor(m.pos, device="cuda")}
    for n in ("kd", "orm", "nrm"):
        lat[n] = torch.tensor(getattr(cand, n), device="cuda")
    for n, t in lat.items():
        t.requires_grad_(bool(cand.optimize.get(n, False)))
    return ST, cand, views, H, W, ref_np, loss, pipe, lat


def _render(ST, pipe, lat, ref, loss, mips, keep_keys=False):
    return ST.render_loss(pipe, lat["pos"], lat["kd"], lat["orm"], lat["nrm"], ref, loss, mips=mips,
                          keep_keys=keep_keys)


@pytest.mark.parametrize("which", ["small", "plain"])
def test_stage_chain_matches_oracle_and_step_call(which, gpu_lib):
    from paper_2104_03989_gb300.engine import Context

    ST, cand, views, H, W, ref_np, loss, pipe, lat = _inputs(which)
    ref = torch.as_tensor(ref_np).cuda()
    L = _render(ST, pipe, lat, ref, loss, cand.mips)
    keys = pipe.keys.cpu().numpy().view(np.uint64)
    loss_val = float(L.detach())
    pre = pipe.pre[..., :3].cpu().numpy()
    L.backward()
    orc = oracle_grads(cand, views, ref_np, H, W, loss)
    np.testing.assert_array_equal(keys, orc["keys"])
    assert rel_l2(pre, orc["pre"]) < 1e-5
    assert abs(loss_val - orc["loss"]) / orc["loss"] < 1e-5
    # the whole-step call on the same inputs
    ctx = Context()
    job = ctx.create_job(cand, loss=loss)
    ctx.forward_loss([job], [views], [ref])
    ctx.backward([job])
    p = ctx.params(job)
    for name, want in orc["grads"].items():
        got = lat[name].grad.double().cpu().numpy().reshape(want.shape)
        err = rel_l2(got, want)
        if name == "pos":
            step = p["g_pos"].double().cpu().numpy()
        else:
            step = torch.empty(p[name].shape, dtype=torch.float32, device="cuda")
            from paper_2104_03989_gb300 import binding as B
            B.adms_job_fold_gradients(ctx.ctx, job, **{"g_" + name: step})
            step = step.double().cpu().numpy()
        print(f"{which} {name}: stages vs oracle {err:.3e}, vs step call {rel_l2(got, step):.3e}")
        assert err < 1e-3, name
        assert rel_l2(got, step) < 1e-3, name
    ctx.close()


def test_recompute_mode_gives_the_same_gradients(gpu_lib):
    from paper_2104_03989_gb300 import stages as ST

    ST, cand, views, H, W, ref_np, loss, pipe, lat = _inputs("plain")
    ref = torch.as_tensor(ref_np).cuda()
    L = _render(ST, pipe, lat, ref, loss, cand.mips)
    L.backward()
    kept = {n: t.grad.clone() for n, t in lat.items() if t.requires_grad}
    m = cand.mesh
    pipe2 = ST.Pipeline(m.tri_pos, m.uv, m.tri_uv, m.n_verts, views, H, W, recompute=True)
    lat2 = {n: t.detach().clone().requires_grad_(t.requires_grad) for n, t in lat.items()}
    L2 = _render(ST, pipe2, lat2, ref, loss, cand.mips)
    assert pipe2.keys is None and pipe2.pre is None   # nothing of the raster kept after the forward
    L2.backward()
    assert abs(float(L2) - float(L)) <= 1e-12 * abs(float(L))   # float64 sums in another atomic order
    for n, g in kept.items():
        assert rel_l2(lat2[n].grad.cpu(), g.cpu()) < 1e-6, n


def _fd_check(label, f, params, rng, min_total=64):
    """Central differences of the scalar f() in the picked entries of each
    parameter (entries whose analytic gradient is above a fraction of the
    largest, 1e-3 unless the parameter tuple gives a fifth element) against the
    analytic gradient already in .grad; median relative error < 1e-3, 90% under
    1e-2. f() sums float32 stage outputs, so its rounding noise is about constant
    in absolute terms: on an entry with a tiny gradient it is a large relative
    error that says nothing about the backward."""
    errs, groups = [], []
    with torch.no_grad():
        for p in params:
            name, t, k, h = p[:4]
            floor = p[4] if len(p) > 4 else 1e-3
            g = t.grad.reshape(-1)
            nz = torch.nonzero(g.abs() > floor * g.abs().max()).squeeze(1).cpu().numpy()
            for i in rng.choice(nz, size=min(len(nz), k), replace=False):
                flat = t.data.view(-1)
                x0 = float(flat[i])
                vals = []
                for s in (1, -1):
                    flat[i] = x0 + s * h
                    vals.append(float(f()))
                flat[i] = x0
                fd = (vals[0] - vals[1]) / (2 * h)
                an = float(g[i])
                errs.append(abs(fd - an) / abs(an))
                groups.append(name)
    errs, groups = np.array(errs), np.array(groups)
    per = ", ".join(f"{n} {np.median(errs[groups == n]):.1e}" for n in dict.fromkeys(groups))
    print(f"{label}: central differences on {len(errs)} parameters, rel error median {np.median(errs):.2e} "
          f"({per}), 90th pct {np.percentile(errs, 90):.2e}")
    assert len(errs) >= min_total
    assert np.median(errs) < 1e-3
    assert (errs < 1e-2).mean() >= 0.9


def _smooth_maps(n):
    """Low-frequency base colour and normal maps (n x n): the derivative jumps of the
    bilinear filter at cell boundaries are second order in the texel size, so a
    position step that moves texture coordinates across cells changes the
    difference quotient by a negligible amount (on noise maps each crossing is
    as large as the cancelling sum it perturbs)."""
    v, u = np.meshgrid((np.arange(n) + 0.5) / n, (np.arange(n) + 0.5) / n, indexing="ij")
    s, c = np.sin(2 * np.pi * (2 * u + v)), np.cos(2 * np.pi * (u - 3 * v))
    kd = np.stack([0.5 + 0.3 * s, 0.5 + 0.3 * c, 0.5 + 0.2 * s * c, np.ones_like(u)], -1)
    nx, ny = 0.3 * s, 0.3 * c
    nrm = np.stack([nx, ny, np.sqrt(1 - nx * nx - ny * ny), np.zeros_like(u)], -1)
    return (torch.tensor(kd.astype(np.float32), device="cuda"), torch.tensor(nrm.astype(np.float32), device="cuda"))


def test_each_stage_backward_against_central_differences(gpu_lib):
    ST, cand, views, H, W, ref_np, loss, pipe, lat = _inputs("small")
    ref = torch.as_tensor(ref_np).cuda()
    rng = np.random.default_rng(1)
    gen = torch.Generator().manual_seed(1)   # the random projections, drawn on the host
    randn = lambda *shape: torch.randn(*shape, generator=gen).cuda()   # noqa: E731
    lat["kd"], lat["nrm"] = _smooth_maps(lat["kd"].shape[0])
    pos = lat["pos"].detach().clone().requires_grad_(True)
    dbl = lambda x: x.double()   # noqa: E731

    # frame: a random projection of (normals, tangents) w.r.t. positions
    R = randn(2, pipe.V, 4)
    def frame():
        _, n4, t4 = ST.Frame.apply(pipe, pos)
        return (dbl(n4) * R[0]).sum() + (dbl(t4) * R[1]).sum()
    frame().backward()
    _fd_check("frame", frame, [("pos", pos, 64, 1e-3)], rng)

    # setup + raster (visibility and LOD fixed): a random projection of the barycentrics
    pos.grad = None
    clip0 = ST.Setup.apply(pipe, pos.detach())
    ST.Raster.apply(pipe, pos.detach(), clip0)            # keys and LOD derivatives of the unperturbed mesh
    covered = (pipe.keys != -1).unsqueeze(-1).float()
    Rr = randn(pipe.B, pipe.H, pipe.W, 2) * covered
    def raster():
        clip = ST.Setup.apply(pipe, pos)
        return (dbl(ST.Raster.apply(pipe, pos, clip, True)) * Rr).sum()
    raster().backward()
    _fd_check("setup + raster", raster, [("pos", pos, 64, 1e-3)], rng)

    # shade: a random projection of the colours w.r.t. texels and positions (through
    # the attributes and the barycentrics), visibility and LOD fixed
    pos.grad = None
    kd = lat["kd"].detach().clone().requires_grad_(True)
    nrm = lat["nrm"].detach().clone().requires_grad_(True)
    Rs = randn(pipe.B, pipe.H, pipe.W, 4) * covered
    Rs[..., 3] = 0
    def shade():
        chains = [ST.MipChain.apply(t) for t in (kd, lat["orm"].detach(), nrm)]
        d = tuple((t.shape[0], t.shape[1], ST.mip_levels(t.shape[0], t.shape[1])) for t in (kd, lat["orm"], nrm))
        v4, n4, t4 = ST.Frame.apply(pipe, pos)
        clip = ST.Setup.apply(pipe, pos)
        rast = ST.Raster.apply(pipe, pos, clip, True)
        return (dbl(ST.Shade.apply(pipe, pos, rast, v4, n4, t4, d, *chains)) * Rs).sum()
    shade().backward()
    # positions: entries above 1e-2 of the largest (the noise floor of a 1e-4 step
    # through the float32 shading is about 1e-3 of a typical entry)
    _fd_check("shade", shade, [("kd", kd, 32, 1e-2), ("nrm", nrm, 32, 1e-2), ("pos", pos, 64, 1e-4, 1e-2)], rng,
              min_total=128)

    # aa_loss: the loss w.r.t. the pre-AA colours and (through the silhouette
    # crossings) the positions, visibility fixed
    pos.grad = None
    v4, n4, t4 = ST.Frame.apply(pipe, pos.detach())
    chains = [ST.MipChain.apply(lat[n].detach()) for n in ("kd", "orm", "nrm")]
    d = tuple((lat[n].shape[0], lat[n].shape[1], ST.mip_levels(lat[n].shape[0], lat[n].shape[1]))
              for n in ("kd", "orm", "nrm"))
    pre0 = ST.Shade.apply(pipe, pos.detach(), ST.Raster.apply(pipe, pos.detach(), clip0, True), v4, n4, t4, d, *chains)
    pre = pre0.detach().clone().requires_grad_(True)
    scale = 1.0 / (3.0 * pipe.B * pipe.H * pipe.W)
    def aa():
        clip = ST.Setup.apply(pipe, pos)
        return dbl(ST.AALoss.apply(pipe, pos, pre, clip, ref, loss, scale)) * 1e3
    aa().backward()
    _fd_check("aa_loss", aa, [("pre", pre, 64, 1e-4), ("pos", pos, 64, 1e-5)], rng, min_total=96)

    # mip chain: a random projection of the chain w.r.t. level-0 texels
    t0 = lat["kd"].detach().clone().requires_grad_(True)
    Rm = None
    def mip():
        nonlocal Rm
        ch = ST.MipChain.apply(t0)
        if Rm is None:
            Rm = randn(*ch.shape)
        return (dbl(ch) * Rm).sum()
    mip().backward()
    _fd_check("mip", mip, [("kd", t0, 64, 1e-2)], rng)


def test_stage_calls_refuse_bad_arguments(gpu_lib):
    from paper_2104_03989_gb300 import binding as B
    from paper_2104_03989_gb300 import stages as ST

    _, cand, views, H, W, ref_np, loss, pipe, lat = _inputs("small")
    m = pipe.mesh(lat["pos"])
    clip = torch.empty(pipe.B, pipe.V, 4, device="cuda")
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.AdmsError):
        B.adms_setup_fwd(m, pipe.views, pipe.B, H, W, clip, small)          # workspace too small
    with pytest.raises(B.AdmsError):
        B.adms_setup_fwd(m, pipe.views, pipe.B, H, 0, clip, pipe.work)      # empty image
    bad = B.stage_textures([(lat["kd"].detach(), None, 255, 256, 1)] * 3)  # not a power of two
    with pytest.raises(B.AdmsError):
        B.adms_shade_fwd(m, pipe.views, pipe.B, H, W, torch.empty(1, device="cuda"), clip, clip, clip, clip, clip,
                         bad, clip)
    assert ST.mip_levels(256, 256) == 9


def _tess_inputs():
    from paper_2104_03989_gb300 import stages as ST
    from cases import tess_case

    c, views, H, W = tess_case()
    cand = c["cand"]
    ref_np, _ = oracle_reference(c["ref"], views, H, W)
    m = cand.mesh
    tm = ST.TessMesh(m.tri_pos, m.tri_uv, m.uv, m.n_verts, cand.tess_levels)
    pipe = ST.Pipeline(tm.rtri, tm.ruv, tm.rtri_uv, tm.Vt, views, H, W)
    lat = {"pos": torch.tensor(m.pos, device="cuda"), "disp": torch.tensor(cand.disp, device="cuda")}
    for n in ("kd", "orm", "nrm"):
        lat[n] = torch.tensor(getattr(cand, n), device="cuda")
    for n, t in lat.items():
        t.requires_grad_(bool(cand.optimize.get(n, False)))
    return ST, cand, views, H, W, ref_np, tm, pipe, lat


def test_tessellation_stage_chain_matches_oracle(gpu_lib):
    """Tess (Eq. 3) -> frame -> setup -> raster -> shade -> aa_loss on the
    displacement workload shrunk for the oracle: keys bit-exact (the float32
    contract of the displaced positions), loss within 1e-5, gradients of base
    positions, displacement texels and normal map within 1e-3."""
    ST, cand, views, H, W, ref_np, tm, pipe, lat = _tess_inputs()
    ref = torch.as_tensor(ref_np).cuda()
    pos = ST.Tess.apply(tm, lat["pos"], lat["disp"])
    L = ST.render_loss(pipe, pos, lat["kd"], lat["orm"], lat["nrm"], ref, "logl1", mips=cand.mips)
    keys = pipe.keys.cpu().numpy().view(np.uint64)
    loss_val = float(L.detach())
    L.backward()
    orc = oracle_grads(cand, views, ref_np, H, W, "logl1")
    np.testing.assert_array_equal(keys, orc["keys"])
    assert abs(loss_val - orc["loss"]) / orc["loss"] < 1e-5
    for name, want in orc["grads"].items():
        got = lat[name].grad.double().cpu().numpy().reshape(want.shape)
        err = rel_l2(got, want)
        print(f"tess stages {name}: rel L2 {err:.3e}")
        assert err < 1e-3, name


def test_tessellation_stage_against_central_differences(gpu_lib):
    """Central differences (h = 1e-3) of a random projection of the displaced
    render positions in 64 base-position coordinates and 64 displacement texels."""
    ST, cand, views, H, W, ref_np, tm, pipe, lat = _tess_inputs()
    rng = np.random.default_rng(4)
    bp = lat["pos"].detach().clone().requires_grad_(True)
    dm = lat["disp"].detach().clone().requires_grad_(True)
    R = torch.randn(tm.Vt, 3, generator=torch.Generator().manual_seed(4), dtype=torch.float64).cuda()
    f = lambda: (ST.Tess.apply(tm, bp, dm).double() * R).sum()   # noqa: E731
    f().backward()
    _fd_check("tess", f, [("pos", bp, 64, 1e-3), ("disp", dm, 64, 1e-3)], rng, min_total=128)
