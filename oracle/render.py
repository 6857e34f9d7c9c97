"""Float64 oracle of one render-and-compare step (TEST INFRASTRUCTURE ONLY).

Written step by step in the order of the paper's pipeline (Sec. 3 overview;
Sec. 5.1 mesh operations; Sec. 5.2 renderer; Sec. 5.3 optimization) with
plain PyTorch CPU tensor ops in float64. Gradients come from reverse-mode
differentiation of this float64 forward with the visibility keys and the
texture LOD held fixed, i.e. the exact adjoint of the forward as written.

Where the paper is silent, this module fixes one reading (camera model, fill
rule, LOD rule, texture wrap, diffuse term, GGX variant, antialiasing rule,
loss normalisation, clamps); each such place says "reading:".

The float32 visibility (snapping, fill rule, depth keys) lives in raster.c.
"""

from __future__ import annotations

import math

import numpy as np
import torch

from . import visibility

F64 = torch.float64
EMPTY = 0xFFFFFFFFFFFFFFFF
EPS_NORM = 1e-20        # normalize(x) = x / sqrt(max(x.x, EPS_NORM))
NV_MIN = 1e-4           # reading: n.v clamped from below
ROUGH_MIN = 0.08        # reading: alpha = max(r, 0.08)^2
SRGB_T = 0.0031308      # sRGB transfer threshold (Sec. 5.3)
SRGB_A = 0.055          # sRGB transfer constant a (Sec. 5.3)
ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8   # Adam defaults (Sec. 5.3)
LR_K = 0.0002           # lr_t = lr0 * 10^(-k t) (Sec. 5.3)
LAMBDA_K = 1e-6         # lambda schedule constant k (Eq. 5 text)
LAMBDA_MIN_FRAC = 0.02  # lambda_min = 2% of lambda_0 (Eq. 5 text)


# ----------------------------------------------------------------------------- helpers

def t64(x):
    return torch.as_tensor(np.asarray(x), dtype=F64)


def normalize(x):
    return x / torch.sqrt(torch.clamp((x * x).sum(-1, keepdim=True), min=EPS_NORM))


def dot(a, b):
    return (a * b).sum(-1, keepdim=True)


def cross2(a, b):
    return a[..., 0] * b[..., 1] - a[..., 1] * b[..., 0]


# ----------------------------------------------------------------------------- topology

def edge_adjacency(tri):
    """adj[f, k] = the other face across edge (tri[f,k], tri[f,(k+1)%3]), or -1.

    Edges shared by more than two faces count as open (-1)."""
    tri = np.asarray(tri)
    owners = {}
    for f in range(tri.shape[0]):
        for k in range(3):
            a, b = int(tri[f, k]), int(tri[f, (k + 1) % 3])
            owners.setdefault((min(a, b), max(a, b)), []).append((f, k))
    adj = -np.ones((tri.shape[0], 3), dtype=np.int64)
    for lst in owners.values():
        if len(lst) == 2:
            (f0, k0), (f1, k1) = lst
            adj[f0, k0] = f1
            adj[f1, k1] = f0
    return adj


def one_ring(tri, n_verts):
    """Sorted one-ring neighbour lists N_i (vertices sharing an edge with i)."""
    nb = [set() for _ in range(n_verts)]
    for a, b, c in np.asarray(tri):
        for x, y in ((a, b), (b, c), (c, a)):
            nb[x].add(int(y))
            nb[y].add(int(x))
    return [sorted(s) for s in nb]


# ----------------------------------------------------------------------------- mesh frame (Sec. 5.1)

def vertex_normals(pos, tri):
    """Smooth vertex normals: normalised sum of the unnormalised face normals."""
    p0, p1, p2 = pos[tri[:, 0]], pos[tri[:, 1]], pos[tri[:, 2]]
    fn = torch.linalg.cross(p1 - p0, p2 - p0, dim=1)
    acc = torch.zeros_like(pos)
    for k in range(3):
        acc = acc.index_add(0, tri[:, k], fn)
    return normalize(acc)


def vertex_tangents(pos, uv, tri, tri_uv):
    """Vertex tangents from positions and UVs.

    reading: per face T = (e1 dv2 - e2 dv1) / det(duv) (the direction of
    increasing u), normalised; faces with det = 0 contribute nothing; the
    vertex tangent is the normalised sum over its faces."""
    p0, p1, p2 = pos[tri[:, 0]], pos[tri[:, 1]], pos[tri[:, 2]]
    t0, t1, t2 = uv[tri_uv[:, 0]], uv[tri_uv[:, 1]], uv[tri_uv[:, 2]]
    e1, e2 = p1 - p0, p2 - p0
    d1, d2 = t1 - t0, t2 - t0
    det = d1[:, 0] * d2[:, 1] - d2[:, 0] * d1[:, 1]
    tv = e1 * d2[:, 1:2] - e2 * d1[:, 1:2]
    ft = normalize(tv) * torch.sign(det)[:, None]
    acc = torch.zeros_like(pos)
    for k in range(3):
        acc = acc.index_add(0, tri[:, k], ft)
    return normalize(acc)


# ----------------------------------------------------------------------------- textures

def mip_chain(tex):
    """Full mip chain: level k = 2x2 box average of level k-1 down to 1x1."""
    levels = [tex]
    while levels[-1].shape[0] > 1 or levels[-1].shape[1] > 1:
        t = levels[-1]
        h, w, c = t.shape
        sh, sw = (2 if h > 1 else 1), (2 if w > 1 else 1)
        levels.append(t.reshape(h // sh, sh, w // sw, sw, c).mean(dim=(1, 3)))
    return levels


def bilinear(tex, u, v):
    """Bilinear lookup; texel centres at (x + 0.5) / w; u wraps, v clamps."""
    h, w, _ = tex.shape
    x = u * w - 0.5
    y = v * h - 0.5
    x0 = torch.floor(x).detach()
    y0 = torch.floor(y).detach()
    fx = (x - x0)[:, None]
    fy = (y - y0)[:, None]
    ix0 = torch.remainder(x0.long(), w)
    ix1 = torch.remainder(x0.long() + 1, w)
    iy0 = torch.clamp(y0.long(), 0, h - 1)
    iy1 = torch.clamp(y0.long() + 1, 0, h - 1)
    t00, t10 = tex[iy0, ix0], tex[iy0, ix1]
    t01, t11 = tex[iy1, ix0], tex[iy1, ix1]
    return (1 - fx) * (1 - fy) * t00 + fx * (1 - fy) * t10 + (1 - fx) * fy * t01 + fx * fy * t11


def trilinear(levels, u, v, lod):
    """Trilinear filtering between levels floor(lod) and floor(lod)+1 (lod fixed)."""
    L = len(levels) - 1
    lod = lod.detach()
    l0 = torch.floor(lod).long()
    fr = (lod - l0.to(F64))[:, None]
    l1 = torch.clamp(l0 + 1, max=L)
    out = torch.zeros((u.shape[0], levels[0].shape[2]), dtype=F64)
    for k in range(L + 1):
        w = torch.where((l0 == k)[:, None], 1 - fr, torch.zeros_like(fr)) + torch.where(
            (l1 == k)[:, None], fr, torch.zeros_like(fr))
        sel = torch.nonzero((w[:, 0] > 0)).squeeze(1)
        if sel.numel() == 0:
            continue
        val = bilinear(levels[k], u[sel], v[sel]) * w[sel]
        out = out.index_add(0, sel, val)
    return out


def texture_lod(duv_dx, duv_dy, tex_h, tex_w, n_levels):
    """reading: rho = max(|(du/dx W, dv/dx H)|, |(du/dy W, dv/dy H)|),
    lod = clamp(log2 rho, 0, n_levels - 1)."""
    ax = torch.sqrt((duv_dx[:, 0] * tex_w) ** 2 + (duv_dx[:, 1] * tex_h) ** 2)
    ay = torch.sqrt((duv_dy[:, 0] * tex_w) ** 2 + (duv_dy[:, 1] * tex_h) ** 2)
    rho = torch.maximum(ax, ay)
    lod = torch.log2(rho)
    lod = torch.nan_to_num(lod, nan=0.0, neginf=0.0)
    return torch.clamp(lod, 0.0, float(n_levels - 1))


# ----------------------------------------------------------------------------- shading (Sec. 5.2)

def ggx_d(nh, a2):
    """GGX normal distribution D(h) = a2 / (pi ((n.h)^2 (a2 - 1) + 1)^2) (Walter et al. 2007)."""
    return a2 / (math.pi * (nh * nh * (a2 - 1) + 1) ** 2)


def smith_g1(x, a2):
    """Separable Smith-GGX masking G1(x) = 2x / (x + sqrt(a2 + (1 - a2) x^2))."""
    return 2 * x / (x + torch.sqrt(a2 + (1 - a2) * x * x))


def schlick_f(f0, vh):
    """Schlick Fresnel F = f0 + (1 - f0)(1 - v.h)^5."""
    return f0 + (1 - f0) * (1 - vh) ** 5


def shading_frame(n_i, t_i, nmap):
    """Shading normal from the interpolated frame and the tangent-space normal map:
    N = normalize(n), T = normalize(t - (t.N) N), B = N x T,
    n = normalize(nx T + ny B + nz N)."""
    N = normalize(n_i)
    tt = t_i - dot(t_i, N) * N
    T = normalize(tt)
    Bt = torch.linalg.cross(N, T, dim=1)
    return normalize(nmap[:, 0:1] * T + nmap[:, 1:2] * Bt + nmap[:, 2:3] * N)


def view_lights(view, p):
    """(l, E) pairs: point light l = normalize(L - p), E = I / |L - p|^2;
    directional light l = given unit vector, E = irradiance. Zero-strength lights are off."""
    lights = []
    if float(view["light_I"]) != 0.0:
        d = t64(view["light_pos"])[None] - p
        lights.append((normalize(d), float(view["light_I"]) / dot(d, d)))
    if float(view["light_E"]) != 0.0:
        lights.append((t64(view["light_dir"])[None].expand_as(p), float(view["light_E"])))
    return lights


def shade(p, n_i, t_i, kd, orm, nmap, view):
    """Diffuse + isotropic GGX with the (gamma, r, m) parameterisation of Sec. 5.2.

    ks = (1 - m) 0.04 + m kd follows the paper, and gamma scales the whole
    specular lobe by (1 - gamma), so its normal-incidence colour is the
    paper's ks' = (1 - gamma) ks and gamma = 1 removes the lobe (reading).
    The rest is a reading (Karis-style): diffuse kd (1 - m) / pi, GGX D,
    Schlick F(ks) on v.h, separable Smith G with alpha = max(r, 0.08)^2, n.v
    clamped to >= 1e-4, lights with n.l <= 0 contribute nothing, point light
    falloff 1 / d^2, no ambient term:
        color = sum_lights (diffuse + (1 - gamma) D F G / (4 n.l n.v)) E n.l"""
    ns = shading_frame(n_i, t_i, nmap)
    eye = t64(view["eye"])[None]
    vdir = normalize(eye - p)
    nv = torch.clamp(dot(ns, vdir), min=NV_MIN)
    gam, r, m = orm[:, 0:1], orm[:, 1:2], orm[:, 2:3]
    kd3 = kd[:, 0:3]
    alpha = torch.clamp(r, min=ROUGH_MIN) ** 2
    a2 = alpha * alpha
    ks = (1 - m) * 0.04 + m * kd3
    diff = kd3 * (1 - m) / math.pi
    color = torch.zeros_like(kd3)
    for l, E in view_lights(view, p):
        nl = dot(ns, l)
        lit = nl > 0
        nls = torch.where(lit, nl, torch.ones_like(nl))
        h = normalize(l + vdir)
        nh = torch.clamp(dot(ns, h), min=0.0)
        vh = torch.clamp(dot(vdir, h), min=0.0)
        D = ggx_d(nh, a2)
        F = schlick_f(ks, vh)
        G = smith_g1(nls, a2) * smith_g1(nv, a2)
        spec = (1 - gam) * D * F * G / (4 * nls * nv)
        color = color + torch.where(lit, (diff + spec) * E * nls, torch.zeros_like(color))
    return color


# ----------------------------------------------------------------------------- one view

def screen_coords(clip, width, height):
    hw, hh = width / 2.0, height / 2.0
    sx = clip[:, 0] / clip[:, 3] * hw + hw
    sy = hh - clip[:, 1] / clip[:, 3] * hh
    return torch.stack([sx, sy], dim=1)


def perspective_barycentrics(s, w, q):
    """Perspective-correct barycentrics at screen points q.

    s: three (N, 2) screen-space vertex positions (float, unsnapped), w: three
    (N,) clip w, q: (N, 2) pixel centres. Screen barycentrics are ratios of
    2D cross products; beta_k = (lambda_k / w_k) / sum_j (lambda_j / w_j).
    Also returns the analytic screen derivatives (d beta / dx, d beta / dy),
    computed without gradient tracking (they only feed the texture LOD)."""
    area = cross2(s[1] - s[0], s[2] - s[0])
    lam = [cross2(s[1] - q, s[2] - q) / area, cross2(s[2] - q, s[0] - q) / area,
           cross2(s[0] - q, s[1] - q) / area]
    r = [lam[k] / w[k] for k in range(3)]
    R = r[0] + r[1] + r[2]
    beta = [r[k] / R for k in range(3)]
    with torch.no_grad():
        dl_dx = [(s[1][:, 1] - s[2][:, 1]) / area, (s[2][:, 1] - s[0][:, 1]) / area,
                 (s[0][:, 1] - s[1][:, 1]) / area]
        dl_dy = [(s[2][:, 0] - s[1][:, 0]) / area, (s[0][:, 0] - s[2][:, 0]) / area,
                 (s[1][:, 0] - s[0][:, 0]) / area]
        dbeta = []
        for dl in (dl_dx, dl_dy):
            dr = [dl[k] / w[k] for k in range(3)]
            dR = dr[0] + dr[1] + dr[2]
            dbeta.append([(dr[k] * R - r[k] * dR) / (R * R) for k in range(3)])
    return beta, dbeta


def texel_margin(levels, uv, lod):
    """Distance (in texels) of each lookup's texel coordinates to the nearest
    cell boundary, over the mip levels the trilinear filter actually uses.

    At a cell boundary piecewise-bilinear filtering has a kink: its value is
    continuous but its uv-derivative is one-sided, so a float32 evaluation may
    legitimately take the other side. Tests use this to tell such lookups apart."""
    L = len(levels) - 1
    lod = lod.detach()
    l0 = torch.floor(lod).long()
    fr = lod - l0.to(F64)
    l1 = torch.clamp(l0 + 1, max=L)
    out = torch.full_like(lod, float("inf"))
    for k in range(L + 1):
        used = (l0 == k) | ((l1 == k) & (fr > 0))
        h, w = levels[k].shape[0], levels[k].shape[1]
        for c, n in ((uv[:, 0], w), (uv[:, 1], h)):
            if n == 1:   # one texel across: both taps read it, no kink
                continue
            x = c * n - 0.5
            f = x - torch.floor(x)
            m = torch.minimum(f, 1 - f)
            out = torch.where(used, torch.minimum(out, m), out)
    return out


def render_view(geo, tex_levels, view, keys, asign, adj, width, height, aa=True, lod_store=None, diag=None,
                msaa=1):
    """Pre-AA and AA images (H, W, 3) of one view with fixed visibility keys.

    geo: dict pos (V,3), nrm (V,3), tan (V,3), uv (T,2), tri (F,3), tri_uv (F,3)
    tex_levels: dict kd/orm/nrm -> list of mip levels (h, w, 4)
    keys: (H, W) uint64 visibility from raster.c; asign: (F,) int8 area signs.
    lod_store: optional dict; texture LODs and the antialiasing edge choices
    are read from it when present and stored into it otherwise (finite
    differences hold them fixed, like the visibility keys).
    diag: optional dict filled with per-pixel margins to the discrete
    decisions inside the differentiable path (texel cells, n.l = 0, AA tau
    and crossing tests), for tests that must tell kinks apart.
    msaa = s > 1 (the antialiasing paragraph of Sec. 5.2, reading): keys and
    width, height are those of the s x s sample grid of each pixel; every sample
    takes its triangle shaded once per pixel, at the pixel's centre, with the
    LOD of the pixel's footprint; antialiasing acts on the sample grid."""
    pre, _, scr = shade_pixels(geo, tex_levels, view, keys, width, height, lod_store=lod_store, diag=diag,
                               msaa=msaa)
    if not aa:
        return pre, pre
    sil = silhouette_flags(asign, adj)
    aa_store = None if lod_store is None else lod_store.setdefault("aa", {})
    return pre, antialias(pre, keys, scr, geo["tri"], sil, width, height, aa_store=aa_store, diag=diag)


def shade_pixels(geo, tex_levels, view, keys, width, height, lod_store=None, diag=None, msaa=1):
    """Shaded colour (H, W, 3) and base-colour alpha (H, W) of the covered
    pixels of one view (zero elsewhere), and the view's screen positions.
    Arguments as for render_view."""
    pos, tri, tri_uv = geo["pos"], geo["tri"], geo["tri_uv"]
    M = t64(np.asarray(view["mvp"], dtype=np.float32).astype(np.float64).reshape(4, 4))
    clip = torch.cat([pos, torch.ones_like(pos[:, :1])], dim=1) @ M.T
    scr = screen_coords(clip, width, height)

    flat = keys.reshape(-1)
    covered = flat != np.uint64(EMPTY)
    pix = np.nonzero(covered)[0]
    fid = torch.as_tensor((flat[pix] & np.uint64(0xFFFFFFFF)).astype(np.int64))
    pixt = torch.as_tensor(pix.astype(np.int64))
    if msaa > 1:   # the centre of the pixel that holds the sample, in sample-grid units
        qx = ((pixt % width) // msaa).to(F64) * msaa + 0.5 * msaa
        qy = ((pixt // width) // msaa).to(F64) * msaa + 0.5 * msaa
    else:
        qx = (pixt % width).to(F64) + 0.5
        qy = (pixt // width).to(F64) + 0.5
    q = torch.stack([qx, qy], dim=1)

    vi = tri[fid]                       # (N, 3) position indices
    ui = tri_uv[fid]                    # (N, 3) uv indices
    s = [scr[vi[:, k]] for k in range(3)]
    w = [clip[vi[:, k], 3] for k in range(3)]
    beta, dbeta = perspective_barycentrics(s, w, q)

    def interp(attr, idx):
        return sum(beta[k][:, None] * attr[idx[:, k]] for k in range(3))

    p = interp(pos, vi)
    n_i = interp(geo["nrm"], vi)
    t_i = interp(geo["tan"], vi)
    uv = interp(geo["uv"], ui)
    # screen derivatives per pixel (s sample-grid steps per pixel under MSAA)
    duv = [msaa * sum(db[k][:, None] * geo["uv"][ui[:, k]] for k in range(3)) for db in dbeta]

    margins = []

    def fetch(name):
        lv = tex_levels[name]
        if lod_store is not None and name in lod_store:
            lod = lod_store[name]
        else:
            lod = texture_lod(duv[0], duv[1], lv[0].shape[0], lv[0].shape[1], len(lv))
            if lod_store is not None:
                lod_store[name] = lod
        if diag is not None:
            margins.append(texel_margin(lv, uv.detach(), lod))
        return trilinear(lv, uv[:, 0], uv[:, 1], lod)

    kd_s, orm_s, nrm_s = fetch("kd"), fetch("orm"), fetch("nrm")
    col = shade(p, n_i, t_i, kd_s, orm_s, nrm_s, view)
    if diag is not None:
        with torch.no_grad():
            ns = shading_frame(n_i, t_i, nrm_s)
            nl = torch.stack([dot(ns, l)[:, 0].abs() for l, _ in view_lights(view, p)], 1).min(1).values
        diag.update(pix=pix, tri=fid.numpy(), texel_margin=torch.stack(margins, 1).min(1).values.numpy(),
                    nl_margin=nl.numpy())
    img = torch.zeros((height * width, 3), dtype=F64).index_copy(0, pixt, col)
    alpha = torch.zeros(height * width, dtype=F64).index_copy(0, pixt, kd_s[:, 3])
    return img.reshape(height, width, 3), alpha.reshape(height, width), scr


def peel_view(geo, tex_levels, view, layer_keys, asign, adj, width, height, aa=True, lod_store=None, diag=None):
    """Order-independent transparency by depth peeling (Sec. 5.2, reading).

    layer_keys: (L, H, W) keys of the peeled layers, front to back
    (visibility.raster_peeled). Each layer is shaded like an opaque render and
    takes its opacity from the base-colour texture's fourth channel (zero where
    the layer is empty). Blending runs back to front from a black background:
    with A_L = 0, for l = L-1 .. 0
        B_l = alpha_l c_l + (1 - alpha_l) A_{l+1},
        A_l = antialias(B_l) with layer l's visibility (the identity when aa is off),
    and the image is A_0. lod_store / diag as for render_view, kept per layer
    (diag["layers"][l] holds layer l's margins). Returns (layer 0's shaded
    colours, the image)."""
    L = layer_keys.shape[0]
    sil = silhouette_flags(asign, adj) if aa else None
    acc = torch.zeros((height, width, 3), dtype=F64)
    diags = [None] * L
    pre0 = None
    for l in reversed(range(L)):
        st = None if lod_store is None else lod_store.setdefault(("layer", l), {})
        dg = None if diag is None else {}
        col, alpha, scr = shade_pixels(geo, tex_levels, view, layer_keys[l], width, height, lod_store=st, diag=dg)
        a = alpha[..., None]
        blended = a * col + (1 - a) * acc
        if aa:
            aa_store = None if st is None else st.setdefault("aa", {})
            acc = antialias(blended, layer_keys[l], scr, geo["tri"], sil, width, height, aa_store=aa_store, diag=dg)
        else:
            acc = blended
        diags[l] = dg
        if l == 0:
            pre0 = col
    if diag is not None:
        diag["layers"] = diags
    return pre0, acc


# ----------------------------------------------------------------------------- antialiasing

def resolve(img, s):
    """Pixel = mean of its s x s samples: (sH, sW, 3) -> (H, W, 3)."""
    if s == 1:
        return img
    h, w = img.shape[0] // s, img.shape[1] // s
    return img.reshape(h, s, w, s, img.shape[2]).mean(dim=(1, 3))


def silhouette_flags(asign, adj):
    """reading: edge k of face f is a silhouette edge in a view when it has no
    neighbour or the neighbour's snapped screen area has a different sign
    (0 for a culled or degenerate neighbour)."""
    asign = np.asarray(asign, dtype=np.int64)
    nb = np.where(adj >= 0, asign[np.maximum(adj, 0)], 99)
    return (adj < 0) | (nb != asign[:, None])


def antialias(pre, keys, scr, tri, sil, width, height, aa_store=None, diag=None):
    """Silhouette antialiasing (reading of Laine et al. 2020's analytic AA).

    For each horizontally or vertically adjacent pixel pair with different
    triangle ids, the pixel with the smaller key owns the pair (an empty pixel
    never does). Among its triangle's silhouette edges, the one crossing the
    open segment between the two pixel centres closest to the owner's centre
    gives the crossing parameter tau in (0, 1) from the owner. If tau > 1/2 the
    other pixel moves toward the owner's colour by (tau - 1/2); if tau < 1/2
    the owner moves toward the other colour by (1/2 - tau). All moves are
    computed from the pre-AA image and summed.

    aa_store: optional dict; the chosen edge of every pair is read from it when
    present and stored into it otherwise (finite differences hold it fixed)."""
    H, W = height, width
    k = keys.astype(np.uint64)
    tid = np.where(k == np.uint64(EMPTY), -1, (k & np.uint64(0xFFFFFFFF)).astype(np.int64))
    flat = pre.reshape(-1, 3)
    delta = torch.zeros_like(flat)
    for axis in (0, 1):   # 0: horizontal pairs (i, i+1); 1: vertical pairs (j, j+1)
        if axis == 0:
            jj, ii = np.meshgrid(np.arange(H), np.arange(W - 1), indexing="ij")
            pj, pi, qj, qi = jj, ii, jj, ii + 1
        else:
            jj, ii = np.meshgrid(np.arange(H - 1), np.arange(W), indexing="ij")
            pj, pi, qj, qi = jj, ii, jj + 1, ii
        pj, pi, qj, qi = (a.reshape(-1) for a in (pj, pi, qj, qi))
        cand = tid[pj, pi] != tid[qj, qi]
        pj, pi, qj, qi = pj[cand], pi[cand], qj[cand], qi[cand]
        if pj.size == 0:
            continue
        p_own = k[pj, pi] < k[qj, qi]
        oj = np.where(p_own, pj, qj)
        oi = np.where(p_own, pi, qi)
        sj = np.where(p_own, qj, pj)
        si = np.where(p_own, qi, pi)
        sigma = torch.as_tensor(np.where(p_own, 1.0, -1.0))
        fo = torch.as_tensor(tid[oj, oi])
        o_c = torch.as_tensor(np.stack([oi + 0.5, oj + 0.5], axis=1).astype(np.float64))
        u_ax, x_ax = (1, 0) if axis == 0 else (0, 1)   # coordinate fixed along the pair / measured one

        def crossing(e):
            a = scr[tri[fo, e]]
            b = scr[tri[fo, (e + 1) % 3]]
            den = b[:, u_ax] - a[:, u_ax]
            dens = torch.where(den != 0, den, torch.ones_like(den))
            sp = (o_c[:, u_ax] - a[:, u_ax]) / dens
            xc = a[:, x_ax] + sp * (b[:, x_ax] - a[:, x_ax])
            return sigma * (xc - o_c[:, x_ax]), sp, den

        if diag is not None:
            with torch.no_grad():
                sil_o = torch.as_tensor(sil[tid[oj, oi]])
                margin = torch.full((pj.size,), float("inf"), dtype=F64)
                for e in range(3):
                    tau_e, sp, den = crossing(e)
                    m = torch.minimum(torch.minimum(sp.abs(), (1 - sp).abs()),
                                      torch.minimum(tau_e.abs(), (1 - tau_e).abs()))
                    m = torch.minimum(m, (tau_e - 0.5).abs())
                    margin = torch.where(sil_o[:, e] & (den != 0), torch.minimum(margin, m), margin)
            prev = diag.get("aa_pairs", [])
            prev.append((oj * W + oi, sj * W + si, margin.numpy()))
            diag["aa_pairs"] = prev
        if aa_store is not None and axis in aa_store:
            choice = aa_store[axis]
        else:
            with torch.no_grad():
                sil_o = sil[tid[oj, oi]]                    # (n, 3)
                best = torch.full((pj.size,), float("inf"), dtype=F64)
                choice = torch.full((pj.size,), -1, dtype=torch.long)
                for e in range(3):
                    tau_e, sp, den = crossing(e)
                    ok = torch.as_tensor(sil_o[:, e]) & (den != 0) & (sp >= 0) & (sp <= 1)
                    ok = ok & (tau_e > 0) & (tau_e < 1)
                    take = ok & (tau_e < best)
                    best = torch.where(take, tau_e, best)
                    choice = torch.where(take, torch.full_like(choice, e), choice)
            if aa_store is not None:
                aa_store[axis] = choice
        tau = torch.full((pj.size,), 0.5, dtype=F64)
        for e in range(3):
            tau = torch.where(choice == e, crossing(e)[0], tau)
        oidx = torch.as_tensor(oj * W + oi)
        sidx = torch.as_tensor(sj * W + si)
        c_o, c_s = flat[oidx], flat[sidx]
        to_s = (tau > 0.5)[:, None]
        to_o = (tau < 0.5)[:, None]
        d_s = torch.where(to_s, (tau[:, None] - 0.5) * (c_o - c_s), torch.zeros_like(c_o))
        d_o = torch.where(to_o, (0.5 - tau[:, None]) * (c_s - c_o), torch.zeros_like(c_o))
        delta = delta.index_add(0, sidx, d_s).index_add(0, oidx, d_o)
    return (flat + delta).reshape(H, W, 3)


# ----------------------------------------------------------------------------- objective (Sec. 5.3)

def srgb(x):
    """sRGB transfer function Gamma with a = 0.055 (Sec. 5.3)."""
    hi = (1 + SRGB_A) * torch.clamp(x, min=SRGB_T) ** (1.0 / 2.4) - SRGB_A
    return torch.where(x <= SRGB_T, 12.92 * x, hi)


def tonemap(x):
    """x' = Gamma(log(x + 1)), natural log (reading of Sec. 5.3), of the
    radiance clamped at 0: the antialiasing blends can leave a pixel below
    zero and even below -1, where the log has no value (reading: a negative
    colour counts as black). torch.clamp keeps NaN."""
    return srgb(torch.log(torch.clamp(x, min=0.0) + 1))


def image_loss(img, ref, kind):
    """reading: mean over every pixel (background included) and channel."""
    if kind == "l1":
        return (img - ref).abs().mean()
    if kind == "logl1":
        return (tonemap(img) - tonemap(ref)).abs().mean()
    if kind == "l2":
        return ((img - ref) ** 2).mean()
    raise ValueError(kind)


def laplacian_delta(pos, ring):
    """Uniform differential delta_i = v_i - mean_{j in N_i} v_j (Sec. 5.3)."""
    idx = torch.as_tensor(np.concatenate([np.asarray(r, dtype=np.int64) for r in ring]))
    owner = torch.as_tensor(np.repeat(np.arange(len(ring)), [len(r) for r in ring]))
    cnt = torch.as_tensor(np.array([len(r) for r in ring], dtype=np.float64))
    s = torch.zeros_like(pos).index_add(0, owner, pos[idx])
    return pos - s / cnt[:, None]


def laplacian_loss(pos, ring, delta_ref=None):
    """Eq. 4: L_delta = 1/n sum_i |delta_i - delta'_i|^2 (delta' = 0: absolute)."""
    d = laplacian_delta(pos, ring)
    if delta_ref is not None:
        d = d - delta_ref
    return (d * d).sum(dim=1).mean()


def lambda_schedule(lam_prev, lam0, t):
    """Eq. 5 text, read recursively: lambda_t = (lambda_{t-1} - lambda_min) 10^(-k t) + lambda_min."""
    lmin = LAMBDA_MIN_FRAC * lam0
    return (lam_prev - lmin) * 10.0 ** (-LAMBDA_K * t) + lmin


def learning_rate(lr0, t):
    """lr_t = lr0 * 10^(-0.0002 t) (Sec. 5.3)."""
    return lr0 * 10.0 ** (-LR_K * t)


CLAMPS = {
    "kd": [(0.0, 1.0)] * 4,
    "orm": [(0.0, 1.0), (ROUGH_MIN, 1.0), (0.0, 1.0), (None, None)],
    "nrm": [(-1.0, 1.0), (-1.0, 1.0), (0.0, 1.0), (None, None)],
    "pos": None,
    "disp": None,
}


def adam_update(p, g, m, v, t, lr, name):
    """Adam (Kingma & Ba, default parameters, Sec. 5.3), then the reading's clamps."""
    m = ADAM_B1 * m + (1 - ADAM_B1) * g
    v = ADAM_B2 * v + (1 - ADAM_B2) * g * g
    mh = m / (1 - ADAM_B1 ** (t + 1))
    vh = v / (1 - ADAM_B2 ** (t + 1))
    p = p - lr * mh / (torch.sqrt(vh) + ADAM_EPS)
    cl = CLAMPS.get(name.split("@")[0])  # a per-level texture "kd@3" clamps like kd
    if cl is not None:
        chans = []
        for c, (lo, hi) in enumerate(cl):
            x = p[..., c]
            if lo is not None:
                x = torch.clamp(x, lo, hi)
            chans.append(x)
        p = torch.stack(chans, dim=-1)
    return p, m, v
