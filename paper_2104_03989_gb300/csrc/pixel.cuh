// Per-pixel device code shared by the fused per-pixel kernels (shade.cu) and the
// per-stage kernels (stages.cu): perspective-correct barycentrics and attribute
// interpolation, mip-mapped texture lookups, tangent-space normal mapping and
// GGX shading with their adjoints, the silhouette antialiasing pairs, the tone
// map and image loss (Sec. 5.2 renderer, Sec. 5.3 objective).
//
// Precision: screen positions arrive as float-float pairs computed in
// double-float arithmetic per vertex, so offsets from the pixel centre keep
// float32 relative precision; attributes are interpolated as corner-0 value +
// weighted corner differences, which keeps texel coordinates of large textures
// accurate and lets the barycentric adjoint use (a_j - a) without cancellation.
#pragma once

#include "kernels.cuh"

namespace adms {

// ------------------------------------------------------------------ pixel geometry
struct PixGeo {
    int vi[3], ui[3];
    float4 c[3];      // clip coordinates (w, and the adjoint of the projection)
    float2 d[3];      // screen position minus pixel centre
    float e[3], area, lam[3], r[3], R, beta[3];
    float3 p, n, t;   // interpolated position, normal, tangent
    float3 dp, dn, dt;  // interpolated minus corner 0
    float2 duv;       // interpolated uv minus corner 0
    TexCoord tc;
    float2 duv_dx, duv_dy;
};

// a / b: IEEE division, or with FAST the approximate division (2 ulp). FAST is taken
// only where the result feeds a gradient (the backward's recomputation and
// adjoints, held to 1e-3); images and visibility keep IEEE arithmetic.
template <bool FAST>
__device__ __forceinline__ float fdiv(float a, float b) {
    return FAST ? __fdividef(a, b) : a / b;
}
// sqrt(x) for x > 0: IEEE, or with FAST x rsqrt(x) (approximate, as fdiv)
template <bool FAST>
__device__ __forceinline__ float fsqrt(float x) {
    return FAST ? x * rsqrtf(x) : sqrtf(x);
}

__device__ __forceinline__ float2 rel_screen(float4 S, float ox, float oy) {
    return make_float2((S.x - ox) + S.y, (S.z - oy) + S.w);
}

// the point a sample is shaded at: its own centre, or under MSAA the centre of
// its pixel (s x s samples per pixel); screen units of the sample grid
__device__ __forceinline__ void shade_point(const ShadeArgs& A, int px, int py, float& qx, float& qy) {
    if (A.msaa > 1) {
        qx = (float)((px / A.msaa) * A.msaa) + 0.5f * (float)A.msaa;
        qy = (float)((py / A.msaa) * A.msaa) + 0.5f * (float)A.msaa;
    } else {
        qx = (float)px + 0.5f;
        qy = (float)py + 0.5f;
    }
}

// Perspective-correct barycentrics of sample (px, py) in triangle f: corner ids,
// clip coordinates, screen offsets d_k from the shading point, e_k = cross(d_k+1,
// d_k+2), lam_k = e_k / area, r_k = lam_k / w_k, beta_k = r_k / R.
template <bool FAST = false>
__device__ __forceinline__ void pix_bary(const ShadeArgs& A, int b, int px, int py, int f, PixGeo& g) {
    float qx, qy;
    shade_point(A, px, py, qx, qy);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        g.vi[k] = __ldg(A.tri + (3 * f + k));
        g.ui[k] = __ldg(A.tri_uv + (3 * f + k));
        size_t o = (size_t)b * A.V + g.vi[k];
        g.c[k] = __ldg(A.clip + (o));
        g.d[k] = rel_screen(__ldg(A.scr + (o)), qx, qy);
    }
    g.e[0] = cross2(g.d[1], g.d[2]);
    g.e[1] = cross2(g.d[2], g.d[0]);
    g.e[2] = cross2(g.d[0], g.d[1]);
    g.area = cross2(make_float2(g.d[1].x - g.d[0].x, g.d[1].y - g.d[0].y),
                    make_float2(g.d[2].x - g.d[0].x, g.d[2].y - g.d[0].y));
    float ia = fdiv<FAST>(1.f, g.area);
    g.R = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        g.lam[k] = g.e[k] * ia;
        g.r[k] = fdiv<FAST>(g.lam[k], g.c[k].w);
        g.R += g.r[k];
    }
    float iR = fdiv<FAST>(1.f, g.R);
#pragma unroll
    for (int k = 0; k < 3; ++k) g.beta[k] = g.r[k] * iR;
}

// screen derivatives of beta_1 and beta_2 per sample-grid step (texture LOD only):
// (d beta_1 / dx, d beta_2 / dx, d beta_1 / dy, d beta_2 / dy)
template <bool FAST = false>
__device__ __forceinline__ float4 bary_derivs(const PixGeo& g) {
    float ia = fdiv<FAST>(1.f, g.area), iR = fdiv<FAST>(1.f, g.R);
    float dlx[3] = {(g.d[1].y - g.d[2].y) * ia, (g.d[2].y - g.d[0].y) * ia, (g.d[0].y - g.d[1].y) * ia};
    float dly[3] = {(g.d[2].x - g.d[1].x) * ia, (g.d[0].x - g.d[2].x) * ia, (g.d[1].x - g.d[0].x) * ia};
    float drx[3], dry[3], dRx = 0.f, dRy = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        drx[k] = fdiv<FAST>(dlx[k], g.c[k].w);
        dry[k] = fdiv<FAST>(dly[k], g.c[k].w);
        dRx += drx[k];
        dRy += dry[k];
    }
    return make_float4((drx[1] * g.R - g.r[1] * dRx) * iR * iR, (drx[2] * g.R - g.r[2] * dRx) * iR * iR,
                       (dry[1] * g.R - g.r[1] * dRy) * iR * iR, (dry[2] * g.R - g.r[2] * dRy) * iR * iR);
}

// Attributes at barycentrics (1 - b1 - b2, b1, b2) of the triangle with corners
// g.vi, g.ui, as corner 0 plus weighted corner differences; with LOD, the uv
// screen derivatives from db (bary_derivs), times s under MSAA (per pixel).
template <bool LOD>
__device__ __forceinline__ void pix_attr(const ShadeArgs& A, PixGeo& g, float b1, float b2, float4 db) {
    float3 p0 = f3(A.vpos[g.vi[0]]), n0 = f3(A.vnrm[g.vi[0]]), t0 = f3(A.vtan[g.vi[0]]);
    float2 u0 = A.uv[g.ui[0]];
    float2 u1 = A.uv[g.ui[1]], u2 = A.uv[g.ui[2]];
    float2 du1 = make_float2(u1.x - u0.x, u1.y - u0.y), du2 = make_float2(u2.x - u0.x, u2.y - u0.y);
    g.dp = b1 * (f3(A.vpos[g.vi[1]]) - p0) + b2 * (f3(A.vpos[g.vi[2]]) - p0);
    g.dn = b1 * (f3(A.vnrm[g.vi[1]]) - n0) + b2 * (f3(A.vnrm[g.vi[2]]) - n0);
    g.dt = b1 * (f3(A.vtan[g.vi[1]]) - t0) + b2 * (f3(A.vtan[g.vi[2]]) - t0);
    g.p = p0 + g.dp;
    g.n = n0 + g.dn;
    g.t = t0 + g.dt;
    g.duv = make_float2(b1 * du1.x + b2 * du2.x, b1 * du1.y + b2 * du2.y);
    g.tc.u0 = u0.x;
    g.tc.v0 = u0.y;
    g.tc.du = g.duv.x;
    g.tc.dv = g.duv.y;
    g.tc.du_lo = 0.f;
    g.tc.dv_lo = 0.f;
    if (!LOD) return;
    g.duv_dx = make_float2(db.x * du1.x + db.y * du2.x, db.x * du1.y + db.y * du2.y);
    g.duv_dy = make_float2(db.z * du1.x + db.w * du2.x, db.z * du1.y + db.w * du2.y);
    if (A.msaa > 1) {  // derivatives per pixel: s sample-grid steps
        float sc = (float)A.msaa;
        g.duv_dx = make_float2(g.duv_dx.x * sc, g.duv_dx.y * sc);
        g.duv_dy = make_float2(g.duv_dy.x * sc, g.duv_dy.y * sc);
    }
}

// Perspective-correct barycentrics and interpolated attributes (corner 0 plus
// weighted differences) of sample (px, py) inside triangle f. LOD = false skips
// the screen derivatives of uv (the adjoint's second pass).
template <bool LOD = true, bool FAST = false>
__device__ __forceinline__ void pix_geo(const ShadeArgs& A, int b, int px, int py, int f, PixGeo& g) {
    pix_bary<FAST>(A, b, px, py, f, g);
    pix_attr<LOD>(A, g, g.beta[1], g.beta[2], LOD ? bary_derivs<FAST>(g) : make_float4(0.f, 0.f, 0.f, 0.f));
}

// ------------------------------------------------------------------ shading
struct ShadeIn {
    float3 p, n_i, t_i;
    float4 kd, orm, nm;
};

struct ShadeGrad {
    float3 p, n_i, t_i;
    float4 kd, orm, nm;
};

// color = sum_lights E (n.l) kd (1 - m) / pi + (1 - gamma) D F(ks) G E / (4 n.v)
template <bool BWD>
__device__ __forceinline__ float3 shade_eval(const adms_view& vw, const ShadeIn& in, float3 gc, ShadeGrad* G) {
    // shading frame
    Nrm3 Nn = nrm3(in.n_i);
    float3 N = Nn.y;
    float s_tn = dot3(in.t_i, N);
    float3 tt = in.t_i - s_tn * N;
    Nrm3 Tn = nrm3(tt);
    float3 T = Tn.y;
    float3 Bt = cross3(N, T);
    float3 mm = in.nm.x * T + in.nm.y * Bt + in.nm.z * N;
    Nrm3 NSn = nrm3(mm);
    float3 ns = NSn.y;
    Nrm3 Vn = nrm3(f3(vw.eye[0], vw.eye[1], vw.eye[2]) - in.p);
    float3 V = Vn.y;
    float nv_raw = dot3(ns, V);
    float nv = fmaxf(nv_raw, ADMS_NV_MIN);
    float gam = in.orm.x, r = in.orm.y, m = in.orm.z;
    float rr = fmaxf(r, ADMS_ROUGH_MIN);
    float alpha = rr * rr, a2 = alpha * alpha;
    float3 kd = f3(in.kd.x, in.kd.y, in.kd.z);
    float3 ks = f3(0.04f, 0.04f, 0.04f) * (1.f - m) + m * kd;
    float3 diff = kd * ((1.f - m) * (1.f / ADMS_PI));
    float sqv = fsqrt<BWD>(a2 + (1.f - a2) * nv * nv);  // > 0: a2 >= 0.08^4
    float G1v = fdiv<BWD>(2.f * nv, nv + sqv);

    float3 color = zero3();
    // backward accumulators
    float3 g_ns = zero3(), g_V = zero3(), g_p = zero3(), g_ks = zero3(), g_diff = zero3();
    float g_a2 = 0.f, g_nv = 0.f, g_gam = 0.f;

#pragma unroll
    for (int li = 0; li < 2; ++li) {
        bool point = li == 0;
        float strength = point ? vw.light_I : vw.light_E;
        if (strength == 0.f) continue;
        float3 l, d = zero3();
        float E, dd = 0.f;
        Nrm3 Ln;
        if (point) {
            d = f3(vw.light_pos[0], vw.light_pos[1], vw.light_pos[2]) - in.p;
            Ln = nrm3(d);
            l = Ln.y;
            dd = dot3(d, d);
            E = fdiv<BWD>(vw.light_I, dd);
        } else {
            l = f3(vw.light_dir[0], vw.light_dir[1], vw.light_dir[2]);
            E = vw.light_E;
        }
        float nl = dot3(ns, l);
        if (!(nl > 0.f)) continue;
        Nrm3 Hn = nrm3(l + V);
        float3 h = Hn.y;
        float nh_raw = dot3(ns, h), vh_raw = dot3(V, h);
        float nh = fmaxf(nh_raw, 0.f), vh = fmaxf(vh_raw, 0.f);
        // nh^2 (a2 - 1) + 1 = (1 - nh^2) + a2 nh^2, with 1 - nh^2 = |ns x h|^2 for unit
        // vectors: the cross-product form keeps float32 precision at sharp highlights
        float3 nxh = cross3(ns, h);
        float den = nh_raw > 0.f ? dot3(nxh, nxh) + a2 * nh * nh : 1.f;
        float D = fdiv<BWD>(a2, ADMS_PI * den * den);
        float om = 1.f - vh;
        float om2 = om * om;
        float om5 = om2 * om2 * om;
        float3 F = ks + (f3(1.f, 1.f, 1.f) - ks) * om5;
        float sql = fsqrt<BWD>(a2 + (1.f - a2) * nl * nl);
        float G1l = fdiv<BWD>(2.f * nl, nl + sql);
        float q4 = fdiv<BWD>(E, 4.f * nv);
        float S0 = D * G1l * G1v * q4;
        float S = (1.f - gam) * S0;
        color += (E * nl) * diff + S * F;
        if (BWD) {
            g_diff += (E * nl) * gc;
            float gdotdiff = dot3(gc, diff);
            float g_nl = E * gdotdiff;
            float g_E = nl * gdotdiff;
            float3 g_F = S * gc;
            float g_S = dot3(gc, F);
            g_gam += -g_S * S0;
            float g_S0 = g_S * (1.f - gam);
            float g_D = g_S0 * G1l * G1v * q4;
            float g_G1l = g_S0 * D * G1v * q4;
            float g_G1v = g_S0 * D * G1l * q4;
            g_E += fdiv<BWD>(g_S0 * D * G1l * G1v, 4.f * nv);
            g_nv += fdiv<BWD>(-g_S0 * S0, nv);
            g_ks += g_F * (1.f - om5);
            float g_om5 = dot3(g_F, f3(1.f, 1.f, 1.f) - ks);
            float g_vh = -5.f * om2 * om2 * g_om5;
            float dl = sql * (nl + sql) * (nl + sql);
            g_nl += fdiv<BWD>(g_G1l * 2.f * a2, dl);
            g_a2 += g_G1l * fdiv<BWD>(-nl * (1.f - nl * nl), dl);
            float dv = sqv * (nv + sqv) * (nv + sqv);
            g_nv += fdiv<BWD>(g_G1v * 2.f * a2, dv);
            g_a2 += g_G1v * fdiv<BWD>(-nv * (1.f - nv * nv), dv);
            float pd3 = ADMS_PI * den * den * den;
            g_a2 += g_D * (fdiv<BWD>(1.f, ADMS_PI * den * den) - fdiv<BWD>(2.f * a2 * nh * nh, pd3));
            float g_nh = g_D * fdiv<BWD>(-4.f * a2 * nh * (a2 - 1.f), pd3);
            float g_nhr = nh_raw >= 0.f ? g_nh : 0.f;
            float g_vhr = vh_raw >= 0.f ? g_vh : 0.f;
            float3 g_h = g_nhr * ns + g_vhr * V;
            g_ns += g_nhr * h;
            g_V += g_vhr * h;
            float3 g_hu = nrm3_bwd(Hn, g_h);
            float3 g_l = g_hu;
            g_V += g_hu;
            g_ns += g_nl * l;
            g_l += g_nl * ns;
            if (point) {
                float3 g_d = nrm3_bwd(Ln, g_l) + (fdiv<BWD>(-2.f * E, dd) * g_E) * d;
                g_p -= g_d;
            }
        }
    }
    if (BWD) {
        float g_alpha = 2.f * alpha * g_a2;
        float g_rr = 2.f * rr * g_alpha;
        float g_r = r >= ADMS_ROUGH_MIN ? g_rr : 0.f;
        float3 g_kd = m * g_ks + ((1.f - m) * (1.f / ADMS_PI)) * g_diff;
        float g_m = dot3(g_ks, kd - f3(0.04f, 0.04f, 0.04f)) - dot3(g_diff, kd) * (1.f / ADMS_PI);
        float g_nvr = nv_raw >= ADMS_NV_MIN ? g_nv : 0.f;
        g_ns += g_nvr * V;
        g_V += g_nvr * ns;
        g_p -= nrm3_bwd(Vn, g_V);
        // the frame's adjoint evaluates the frame again from (n_i, t_i, nm) rather than
        // holding its ~25 values across the lights; the empty asm keeps the compiler
        // from merging the two evaluations back into one
        float3 n_i = in.n_i, t_i = in.t_i;
        float4 nm4 = in.nm;
        asm volatile("" : "+f"(n_i.x), "+f"(n_i.y), "+f"(n_i.z), "+f"(t_i.x), "+f"(t_i.y), "+f"(t_i.z),
                     "+f"(nm4.x), "+f"(nm4.y), "+f"(nm4.z));
        Nn = nrm3(n_i);
        N = Nn.y;
        s_tn = dot3(t_i, N);
        Tn = nrm3(t_i - s_tn * N);
        T = Tn.y;
        Bt = cross3(N, T);
        NSn = nrm3(nm4.x * T + nm4.y * Bt + nm4.z * N);
        float3 g_mm = nrm3_bwd(NSn, g_ns);
        float3 g_T = nm4.x * g_mm, g_Bt = nm4.y * g_mm, g_N = nm4.z * g_mm;
        g_N += cross3(T, g_Bt);
        g_T += cross3(g_Bt, N);
        float3 g_tt = nrm3_bwd(Tn, g_T);
        float3 g_ti = g_tt;
        float g_s = -dot3(N, g_tt);
        g_N += -s_tn * g_tt;
        g_ti += g_s * N;
        g_N += g_s * t_i;
        G->p = g_p;
        G->n_i = nrm3_bwd(Nn, g_N);
        G->t_i = g_ti;
        G->kd = make_float4(g_kd.x, g_kd.y, g_kd.z, 0.f);
        G->orm = make_float4(g_gam, g_r, g_m, 0.f);
        G->nm = make_float4(dot3(g_mm, T), dot3(g_mm, Bt), dot3(g_mm, N), 0.f);
    }
    return color;
}

__device__ __forceinline__ int key_tri(unsigned long long k) { return k == ADMS_EMPTY_KEY ? -1 : (int)(k & 0xffffffffu); }

__device__ __forceinline__ ShadeIn shade_inputs(const ShadeArgs& A, const PixGeo& g, float lod[3]) {
    lod[0] = tex_lod(A.kd, g.duv_dx, g.duv_dy);
    lod[1] = tex_lod(A.orm, g.duv_dx, g.duv_dy);
    lod[2] = tex_lod(A.nrm, g.duv_dx, g.duv_dy);
    ShadeIn in;
    in.p = g.p;
    in.n_i = g.n;
    in.t_i = g.t;
    in.kd = tex_sample(A.kd, g.tc, lod[0]);
    in.orm = tex_sample(A.orm, g.tc, lod[1]);
    in.nm = tex_sample(A.nrm, g.tc, lod[2]);
    return in;
}

// The texture coordinate's offset from corner 0 recomputed in double-float:
// (r1 (u1 - u0) + r2 (u2 - u0)) / (r0 + r1 + r2), r_k = e_k / w_k, from the
// double-float screen positions. The float32 offset carries ~1e-7 of its
// length in rounding; over a triangle spanning tens of texels that is ~2e-6
// texel, which moves pixels under sharp highlights on noise textures by ~1e-5.
__device__ __forceinline__ void refine_tc(const ShadeArgs& A, int b, int px, int py, PixGeo& g) {
    float qx, qy;
    shade_point(A, px, py, qx, qy);
    DF dx[3], dy[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float4 S = A.scr[(size_t)b * A.V + g.vi[k]];
        dx[k] = df_add_f(df_two_sum(S.x, -qx), S.y);
        dy[k] = df_add_f(df_two_sum(S.z, -qy), S.w);
    }
    DF rk[3];
    rk[0] = df_div_f(df_sub(df_mul(dx[1], dy[2]), df_mul(dy[1], dx[2])), g.c[0].w);
    rk[1] = df_div_f(df_sub(df_mul(dx[2], dy[0]), df_mul(dy[2], dx[0])), g.c[1].w);
    rk[2] = df_div_f(df_sub(df_mul(dx[0], dy[1]), df_mul(dy[0], dx[1])), g.c[2].w);
    DF Rd = df_add(df_add(rk[0], rk[1]), rk[2]);
    float2 u0 = A.uv[g.ui[0]], u1 = A.uv[g.ui[1]], u2 = A.uv[g.ui[2]];
    DF nu = df_add(df_mul(rk[1], df_two_sum(u1.x, -u0.x)), df_mul(rk[2], df_two_sum(u2.x, -u0.x)));
    DF nv = df_add(df_mul(rk[1], df_two_sum(u1.y, -u0.y)), df_mul(rk[2], df_two_sum(u2.y, -u0.y)));
    DF qu = df_div_df(nu, Rd), qv = df_div_df(nv, Rd);
    g.tc.du = qu.hi;
    g.tc.dv = qv.hi;
    g.tc.du_lo = qu.lo;
    g.tc.dv_lo = qv.lo;
    // the uv screen derivatives (texture LOD) with compensated two-term products:
    // their differences cancel, and the LOD's rounding moves trilinear weights
    float ia = 1.f / g.area, iR = 1.f / g.R, iR2 = iR * iR;
    float dlx[3] = {(g.d[1].y - g.d[2].y) * ia, (g.d[2].y - g.d[0].y) * ia, (g.d[0].y - g.d[1].y) * ia};
    float dly[3] = {(g.d[2].x - g.d[1].x) * ia, (g.d[0].x - g.d[2].x) * ia, (g.d[1].x - g.d[0].x) * ia};
    float drx[3], dry[3], dRx = 0.f, dRy = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        drx[k] = dlx[k] / g.c[k].w;
        dry[k] = dly[k] / g.c[k].w;
        dRx += drx[k];
        dRy += dry[k];
    }
    float2 du1 = make_float2(u1.x - u0.x, u1.y - u0.y), du2 = make_float2(u2.x - u0.x, u2.y - u0.y);
    float db1x = dot2_acc(drx[1], g.R, -g.r[1], dRx) * iR2, db2x = dot2_acc(drx[2], g.R, -g.r[2], dRx) * iR2;
    float db1y = dot2_acc(dry[1], g.R, -g.r[1], dRy) * iR2, db2y = dot2_acc(dry[2], g.R, -g.r[2], dRy) * iR2;
    g.duv_dx = make_float2(dot2_acc(db1x, du1.x, db2x, du2.x), dot2_acc(db1x, du1.y, db2x, du2.y));
    g.duv_dy = make_float2(dot2_acc(db1y, du1.x, db2y, du2.x), dot2_acc(db1y, du1.y, db2y, du2.y));
    if (A.msaa > 1) {
        float sc = (float)A.msaa;
        g.duv_dx = make_float2(g.duv_dx.x * sc, g.duv_dx.y * sc);
        g.duv_dy = make_float2(g.duv_dy.x * sc, g.duv_dy.y * sc);
    }
}

// texels of the largest texture that the triangle's uv offsets span at the finest
// level sampled: the lever arm of the barycentrics' rounding on texel coordinates
__device__ __forceinline__ float tc_lever(const ShadeArgs& A, const PixGeo& g, const float lod[3]) {
    float2 u0 = A.uv[g.ui[0]], u1 = A.uv[g.ui[1]], u2 = A.uv[g.ui[2]];
    float su = fmaxf(fabsf(u1.x - u0.x), fabsf(u2.x - u0.x)), sv = fmaxf(fabsf(u1.y - u0.y), fabsf(u2.y - u0.y));
    float lever = 0.f;
    const TexDev* ts[3] = {&A.kd, &A.orm, &A.nrm};
#pragma unroll
    for (int k = 0; k < 3; ++k)
        lever = fmaxf(lever, fmaxf(su * (float)ts[k]->w0, sv * (float)ts[k]->h0) * exp2f(-floorf(lod[k])));
    return lever;
}

// shading of one listed pixel again, with the refined texture coordinate and LOD
__device__ __forceinline__ void shade_refine_px(const ShadeArgs& A, int pix) {
    int hw = A.H * A.W;
    int b = pix / hw, rem = pix - b * hw;
    int py = rem / A.W, px = rem - py * A.W;
    int f = key_tri(__ldg(A.keys + (pix)));
    PixGeo g;
    pix_geo(A, b, px, py, f, g);
    refine_tc(A, b, px, py, g);
    float lod[3];
    ShadeIn in = shade_inputs(A, g, lod);
    float3 c = shade_eval<false>(A.views[b], in, zero3(), nullptr);
    float4 v = make_float4(c.x, c.y, c.z, A.peel ? in.kd.w : 1.f);
    if (A.msaa > 1) {
        // every sample of the pixel that shows this triangle takes this shading
        int sm = A.msaa, ox = (px / sm) * sm, oy = (py / sm) * sm;
        for (int y = oy; y < min(oy + sm, A.H); ++y)
            for (int x = ox; x < min(ox + sm, A.W); ++x) {
                size_t q = ((size_t)b * A.H + y) * A.W + x;
                if (key_tri(__ldg(A.keys + (q))) == f) A.pre[q] = v;
            }
    } else {
        A.pre[pix] = v;
    }
}

// ------------------------------------------------------------------ shading forward
// shading of triangle f at sample (px, py), refining it (INLINE) or listing it for
// the refinement pass when bright on a triangle that spans many texels
template <bool INLINE = false>
__device__ __forceinline__ float4 shade_covered(const ShadeArgs& A, int b, int px, int py, int f, size_t pix) {
    PixGeo g;
    pix_geo(A, b, px, py, f, g);
    float lod[3];
    ShadeIn in = shade_inputs(A, g, lod);
    float3 c = shade_eval<false>(A.views[b], in, zero3(), nullptr);
    // Bright pixels (sharp highlights) carry almost all of the error a float32
    // texture coordinate causes: on the noise-textured workloads the 0.35% of
    // pixels above 0.5 carry 98% of it. Those on triangles spanning more than two
    // texels at the sampled level are shaded again with the refined coordinate and
    // LOD: here (INLINE, for small grids, where a second launch costs more than
    // the branch) or by k_shade_refine from a list (a separate pass keeps the
    // shading kernel's registers to the common path). The backward, held to 1e-3,
    // keeps the float32 ones.
    if (A.refine && fmaxf(c.x, fmaxf(c.y, c.z)) > 0.5f && tc_lever(A, g, lod) > 2.f) {
        if (INLINE) {
            refine_tc(A, b, px, py, g);
            in = shade_inputs(A, g, lod);
            c = shade_eval<false>(A.views[b], in, zero3(), nullptr);
        } else {
            A.refine[1 + atomicAdd(A.refine, 1)] = (int)pix;  // for k_shade_refine
        }
    }
    return make_float4(c.x, c.y, c.z, A.peel ? in.kd.w : 1.f);  // a peeled layer keeps its opacity
}

template <bool INLINE = false>
__device__ __forceinline__ void shade_fwd_px(const ShadeArgs& A, int b, int px, int py) {
    if (px >= A.W || py >= A.H) return;
    size_t pix = ((size_t)b * A.H + py) * A.W + px;
    int f = key_tri(__ldg(A.keys + (pix)));
    A.pre[pix] = f >= 0 ? shade_covered<INLINE>(A, b, px, py, f, pix) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// Under MSAA every sample of a pixel that shows one triangle has the same shading
// (at the pixel's centre, with the pixel's LOD), so the (pixel, triangle) groups of
// an R x R-sample region at (rx0, ry0) are shaded once each. A group's leader is its
// first sample in the region (row-major); tri: the region's triangle ids (-1: empty
// or outside); returns the leader's index in the region, -1 for f < 0.
__device__ __forceinline__ int group_leader(int sm, int rx0, int ry0, int R, int px, int py, int f,
                                            const int* tri) {
    if (f < 0) return -1;
    int ox = (px / sm) * sm, oy = (py / sm) * sm;
    for (int y = max(oy, ry0); y < min(oy + sm, ry0 + R); ++y)
        for (int x = max(ox, rx0); x < min(ox + sm, rx0 + R); ++x) {
            int t = (y - ry0) * R + (x - rx0);
            if (tri[t] == f) return t;
        }
    return -1;
}

// ------------------------------------------------------------------ antialiasing
struct PairTau {
    int edge;       // -1: no blend
    float tau, sp;
    float2 a, b;    // edge endpoints relative to the owner's pixel centre
    int va, vb;     // edge endpoints (position indices)
};

// The owner's silhouette edge crossing the open segment between the centres of
// the owner (oi, oj) and the other pixel at +sigma along `axis`, nearest to the
// owner; tau is the crossing's distance from the owner's centre in pixels.
__device__ __forceinline__ PairTau pair_tau(const ShadeArgs& A, int b, int axis, int oi, int oj, int fo, float sigma) {
    PairTau pt;
    pt.edge = -1;
    pt.tau = 0.5f;
    float best = 1e30f;
    float ox = (float)oi + 0.5f, oy = (float)oj + 0.5f;
    unsigned mask = __ldg(A.silmask + ((size_t)b * A.F + fo));
    if (!mask) return pt;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        if (!((mask >> e) & 1u)) continue;
        int va = __ldg(A.tri + (3 * fo + e)), vb = __ldg(A.tri + (3 * fo + (e + 1) % 3));
        float2 sa = rel_screen(__ldg(A.scr + ((size_t)b * A.V + va)), ox, oy);
        float2 sb = rel_screen(__ldg(A.scr + ((size_t)b * A.V + vb)), ox, oy);
        float au = axis == 0 ? sa.y : sa.x, bu = axis == 0 ? sb.y : sb.x;
        float ax = axis == 0 ? sa.x : sa.y, bx = axis == 0 ? sb.x : sb.y;
        float den = bu - au;
        if (den == 0.f) continue;
        float sp = -au / den;
        if (!(sp >= 0.f && sp <= 1.f)) continue;
        float tau = sigma * (ax + sp * (bx - ax));
        if (tau > 0.f && tau < 1.f && tau < best) {
            best = tau;
            pt.edge = e;
            pt.tau = tau;
            pt.sp = sp;
            pt.a = sa;
            pt.b = sb;
            pt.va = va;
            pt.vb = vb;
        }
    }
    return pt;
}

struct PairInfo {
    bool p_owner;
    float sigma;
    PairTau t;
};

// pair of pixel p = (px, py) with its neighbour q; false when both show the same
// triangle (or both are empty) or when no silhouette edge crosses between them
__device__ __forceinline__ bool pair_eval(const ShadeArgs& A, int b, int px, int py, unsigned long long kp, int qx,
                                          int qy, unsigned long long kq, int axis, PairInfo& pi) {
    int tp = key_tri(kp), tq = key_tri(kq);
    if (tp == tq) return false;
    pi.p_owner = kp < kq;
    int oi = pi.p_owner ? px : qx, oj = pi.p_owner ? py : qy;
    int si = pi.p_owner ? qx : px, sj = pi.p_owner ? qy : py;
    pi.sigma = axis == 0 ? (float)(si - oi) : (float)(sj - oj);
    pi.t = pair_tau(A, b, axis, oi, oj, pi.p_owner ? tp : tq, pi.sigma);
    return pi.t.edge >= 0;
}

__device__ __forceinline__ float3 f3of(float4 a) { return f3(a.x, a.y, a.z); }

// the colour antialiasing acts on: the shaded colour, or for a depth-peeled layer
// its blend over the composite behind it, alpha c + (1 - alpha) under (black
// background behind the last layer; alpha 0 where the layer is empty)
template <bool PEEL>
__device__ __forceinline__ float3 layer_colour(const ShadeArgs& A, size_t pix) {
    float4 p = A.pre[pix];
    if (!PEEL) return f3of(p);
    float3 u = A.under ? f3of(A.under[pix]) : zero3();
    return p.w * f3of(p) + (1.f - p.w) * u;
}

// Gamma(log(max(x, 0) + 1)) with the sRGB Gamma of Sec. 5.3, and its
// derivative. Radiance is non-negative; the antialiasing blends can undershoot
// below zero beside a bright pixel (a pixel blended toward several darker
// neighbours), and log(x + 1) has no value below -1, so negative colours count
// as black (derivative 0). NaN stays NaN.
__device__ __forceinline__ float tonemap(float x, float* dfdx) {
    bool neg = x < 0.f;
    if (neg) x = 0.f;
    float y = log1pf(x);
    float dy = neg ? 0.f : 1.f / (1.f + x);
    if (y <= 0.0031308f) {
        *dfdx = 12.92f * dy;
        return 12.92f * y;
    }
    // y^(1/2.4) as 2^(log2(y) / 2.4): a few ulp (the loss is held to 1e-5, its
    // gradient to 1e-3), far cheaper than the correctly rounded power; y > 0.0031308 here
    float pw = exp2f(log2f(y) * (1.f / 2.4f));
    *dfdx = (1.055f / 2.4f) * pw / y * dy;
    return 1.055f * pw - 0.055f;
}

__device__ __forceinline__ float loss_term(int kind, float x, float y, float* g) {
    if (kind == ADMS_LOSS_L1) {
        float d = x - y;
        *g = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        return fabsf(d);
    }
    if (kind == ADMS_LOSS_L2) {
        float d = x - y;
        *g = 2.f * d;
        return d * d;
    }
    float dfx, dfy;
    float fx = tonemap(x, &dfx), fy = tonemap(y, &dfy);
    float d = fx - fy;
    *g = d > 0.f ? dfx : (d < 0.f ? -dfx : 0.f);
    return fabsf(d);
}

__device__ __forceinline__ void neighbour(int nbi, int px, int py, int& qx, int& qy) {
    qx = px + (nbi == 0 ? -1 : nbi == 1 ? 1 : 0);
    qy = py + (nbi == 2 ? -1 : nbi == 3 ? 1 : 0);
}

// one block of pixels: AA, loss terms and dL/d(AA colour); the block's loss sum
// goes to A.loss_acc (block-collective: every thread of the block calls it)
// PEEL: A is a layer of a depth-peeled composite (A.peel set); a separate
// instantiation keeps the opaque path's registers to its own needs
template <bool PEEL = false>
__device__ __forceinline__ void aa_loss_block(const ShadeArgs& A, int b, int px, int py, double* red) {
    bool inside = px < A.W && py < A.H;
    double lsum = 0.0;
    if (inside) {
        size_t pix = ((size_t)b * A.H + py) * A.W + px;
        unsigned long long kp = __ldg(A.keys + (pix));
        float3 cp = layer_colour<PEEL>(A, pix);
        float3 out = cp;
        unsigned amask = 0;  // neighbours whose pair blends (tau != 1/2): the backward visits only these
        if (A.aa) {
#pragma unroll
            for (int nbi = 0; nbi < 4; ++nbi) {
                int qx, qy;
                neighbour(nbi, px, py, qx, qy);
                if (qx < 0 || qx >= A.W || qy < 0 || qy >= A.H) continue;
                size_t qpix = ((size_t)b * A.H + qy) * A.W + qx;
                PairInfo pi;
                if (!pair_eval(A, b, px, py, kp, qx, qy, __ldg(A.keys + (qpix)), nbi < 2 ? 0 : 1, pi)) continue;
                float om = pi.t.tau - 0.5f;
                if (om != 0.f) amask |= 1u << nbi;
                // the other pixel blends toward the owner when tau > 1/2, the owner toward it when tau < 1/2
                bool p_target = om > 0.f ? !pi.p_owner : (om < 0.f ? pi.p_owner : false);
                if (p_target) out += fabsf(om) * (layer_colour<PEEL>(A, qpix) - cp);
            }
        }
        if (A.ref) {
            const float* y = A.ref + pix * 3;
            float g0, g1, g2;
            lsum = (double)loss_term(A.loss_kind, out.x, y[0], &g0) + (double)loss_term(A.loss_kind, out.y, y[1], &g1) +
                   (double)loss_term(A.loss_kind, out.z, y[2], &g2);
            A.gprime[pix] = make_float4(g0 * A.loss_scale, g1 * A.loss_scale, g2 * A.loss_scale, __uint_as_float(amask));
        }
        if (A.out_img) {
            A.out_img[pix * 3] = out.x;
            A.out_img[pix * 3 + 1] = out.y;
            A.out_img[pix * 3 + 2] = out.z;
        }
        if (A.acol) A.acol[pix] = make_float4(out.x, out.y, out.z, __uint_as_float(amask));
    }
    lsum = warp_sum_d(lsum);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lsum;
    __syncthreads();
    if (threadIdx.x == 0 && A.loss_acc) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(A.loss_acc, s * (double)A.loss_scale);
    }
}

// ------------------------------------------------------------------ backward
// Vertex gradients of the fused backward: every lane of a warp writes the 27 values
// of its pixel (position, unit normal and unit tangent gradients of the three
// corners) and its triangle's three vertex ids (columns 27-29, as int bits) into its
// row of a per-warp 32 x 31 shared-memory array; lanes that share a triangle are
// summed column by column (lane j sums value j over the group, rows in ascending
// lane order) and one lane per value issues a float64 atomic at the vertex the
// group's first row names. The row stride 31 is odd, so the 32 lanes writing one
// value and the 27 lanes reading one row each touch distinct banks.
#define ADMS_VROW 31
#define ADMS_VROW_IDS 27
__device__ __forceinline__ void scatter_vertex_rows(const ShadeArgs& A, int f, const float* rows) {
    int lane = threadIdx.x & 31;
    __syncwarp();
    unsigned todo = __ballot_sync(0xffffffffu, f >= 0);
    while (todo) {
        int lead = __ffs(todo) - 1;
        int ft = __shfl_sync(0xffffffffu, f, lead);
        unsigned grp = __ballot_sync(0xffffffffu, f == ft);
        if (lane < ADMS_VROW_IDS) {
            float sum = 0.f;
            for (unsigned m = grp; m; m &= m - 1) sum += rows[(__ffs(m) - 1) * ADMS_VROW + lane];
            if (sum != 0.f) {
                int corner = lane / 9, comp = lane - 9 * corner;
                int vtx = __float_as_int(rows[lead * ADMS_VROW + ADMS_VROW_IDS + corner]);
                double* dst = comp < 3 ? A.g_pos : (comp < 6 ? A.g_nrm : A.g_tan);
                atomicAdd(dst + 3 * vtx + comp % 3, (double)sum);
                if (!isfinite(sum) && A.status) atomicExch(A.status, (int)ADMS_ERR_NONFINITE);
            }
        }
        todo &= ~grp;
    }
    __syncwarp();  // the rows are rewritten by the warp's next pixels
}

__device__ __forceinline__ void atomic_add3(double* p, float3 v) {
    atomicAdd(p, (double)v.x);
    atomicAdd(p + 1, (double)v.y);
    atomicAdd(p + 2, (double)v.z);
}
__device__ __forceinline__ void atomic_add4(double* p, float4 v) {
    atomicAdd(p, (double)v.x);
    atomicAdd(p + 1, (double)v.y);
    atomicAdd(p + 2, (double)v.z);
    atomicAdd(p + 3, (double)v.w);
}

// one pixel of the fused backward; warp-collective (vertex scatter)
// AA adjoint at one sample: dL/d(the colour AA acts on) there, gathered from the
// sample's own dL/d(AA colour) and its blending neighbours'; the crossing edges'
// vertex gradients are scattered here (warp-divergent, plain atomics): into the
// positions (A.g_pos), or with CLIP into the clip coordinates of the view
// (A.g_clip [B][V][4]) with dL/d(AA colour) taken as scale x A.gprime
template <bool PEEL, bool CLIP = false>
__device__ __forceinline__ float3 aa_adjoint(const ShadeArgs& A, int b, int px, int py, size_t pix,
                                             unsigned long long kp, float scale = 1.f) {
    const adms_view& vw = A.views[b];
    float hW = 0.5f * (float)A.W, hH = 0.5f * (float)A.H;
    float4 gp4 = __ldg(A.gprime + (pix));
    float3 gp = f3of(gp4);
    float3 gc = gp;
    unsigned amask = __float_as_uint(gp4.w);  // pairs that blended in the forward (bit per neighbour)
    if (amask) {
        float3 cp = layer_colour<PEEL>(A, pix);
#pragma unroll
        for (int nbi = 0; nbi < 4; ++nbi) {
            if (!((amask >> nbi) & 1u)) continue;
            int qx, qy;
            neighbour(nbi, px, py, qx, qy);
            if (qx < 0 || qx >= A.W || qy < 0 || qy >= A.H) continue;
            size_t qpix = ((size_t)b * A.H + qy) * A.W + qx;
            int axis = nbi < 2 ? 0 : 1;
            PairInfo pi;
            if (!pair_eval(A, b, px, py, kp, qx, qy, __ldg(A.keys + (qpix)), axis, pi)) continue;
            float om = pi.t.tau - 0.5f;
            if (om == 0.f) continue;
            bool p_target = om > 0.f ? !pi.p_owner : pi.p_owner;
            float3 gq = f3of(__ldg(A.gprime + (qpix)));
            float w = fabsf(om);
            if (p_target) gc -= w * gp;
            else gc += w * gq;
            // d tau: once per pair, by its left / top pixel
            if (nbi == 1 || nbi == 3) {
                float3 cq = layer_colour<PEEL>(A, qpix);
                float3 gT = p_target ? gp : gq;
                float3 cT = p_target ? cp : cq, cS = p_target ? cq : cp;
                float g_tau = (om > 0.f ? 1.f : -1.f) * dot3(gT, cS - cT);
                float au = axis == 0 ? pi.t.a.y : pi.t.a.x, bu = axis == 0 ? pi.t.b.y : pi.t.b.x;
                float ax = axis == 0 ? pi.t.a.x : pi.t.a.y, bx = axis == 0 ? pi.t.b.x : pi.t.b.y;
                float du = bu - au, dx = bx - ax, sp = pi.t.sp;
                float k = pi.sigma * g_tau * (CLIP ? scale : 1.f);
                float ga_x = k * (1.f - sp), ga_u = k * dx * (sp - 1.f) / du;
                float gb_x = k * sp, gb_u = -k * dx * sp / du;
                float2 gsa = axis == 0 ? make_float2(ga_x, ga_u) : make_float2(ga_u, ga_x);
                float2 gsb = axis == 0 ? make_float2(gb_x, gb_u) : make_float2(gb_u, gb_x);
                float4 ca = __ldg(A.clip + ((size_t)b * A.V + pi.t.va)), cb = __ldg(A.clip + ((size_t)b * A.V + pi.t.vb));
                if (CLIP) {
                    atomic_add4(A.g_clip + 4 * ((size_t)b * A.V + pi.t.va), screen_bwd(ca, hW, hH, gsa));
                    atomic_add4(A.g_clip + 4 * ((size_t)b * A.V + pi.t.vb), screen_bwd(cb, hW, hH, gsb));
                } else {
                    atomic_add3(A.g_pos + 3 * pi.t.va, clip_to_pos_grad(vw.mvp, screen_bwd(ca, hW, hH, gsa)));
                    atomic_add3(A.g_pos + 3 * pi.t.vb, clip_to_pos_grad(vw.mvp, screen_bwd(cb, hW, hH, gsb)));
                }
            }
        }
    }
    return gc;
}

// The three maps share their texel taps when they have the same size (one LOD and
// one bilinear footprint per level serve all three): the usual case of equally
// sized latent maps.
__device__ __forceinline__ bool shared_taps(const ShadeArgs& A) {
    return A.kd.w0 == A.orm.w0 && A.kd.w0 == A.nrm.w0 && A.kd.h0 == A.orm.h0 && A.kd.h0 == A.nrm.h0 &&
           A.kd.levels == A.orm.levels && A.kd.levels == A.nrm.levels;
}

// tex_sample of the three maps with shared taps (the same arithmetic, map by map)
__device__ __forceinline__ void tex_sample3(const ShadeArgs& A, const TexCoord& tc, float lod, float4 out[3]) {
    const float4* ts[3] = {A.kd.tex, A.orm.tex, A.nrm.tex};
    int l0 = (int)floorf(lod);
    float fr = lod - (float)l0;
    int l1 = min(l0 + 1, A.kd.levels - 1);
#pragma unroll
    for (int m = 0; m < 3; ++m) out[m] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        int k = s == 0 ? l0 : l1;
        float wl = s == 0 ? 1.f - fr : fr;
        if (wl == 0.f) continue;
        BilinTap b = bilin_tap(A.kd, k, tc);
        float w00 = wl * (1.f - b.fx) * (1.f - b.fy), w10 = wl * b.fx * (1.f - b.fy);
        float w01 = wl * (1.f - b.fx) * b.fy, w11 = wl * b.fx * b.fy;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            out[m] = f4madd(out[m], w00, __ldg(ts[m] + b.idx[0]));
            out[m] = f4madd(out[m], w10, __ldg(ts[m] + b.idx[1]));
            out[m] = f4madd(out[m], w01, __ldg(ts[m] + b.idx[2]));
            out[m] = f4madd(out[m], w11, __ldg(ts[m] + b.idx[3]));
        }
    }
}

// adjoint of tex_sample3: the texel gradients of the optimized maps are scattered,
// d/d(u, v) of g[0] . kd + g[1] . orm + g[2] . nm returned
__device__ __forceinline__ float2 tex_sample3_bwd(const ShadeArgs& A, const TexCoord& tc, float lod, const float4 g[3]) {
    const float4* ts[3] = {A.kd.tex, A.orm.tex, A.nrm.tex};
    float4* gs[3] = {A.kd.grad, A.orm.grad, A.nrm.grad};
    int l0 = (int)floorf(lod);
    float fr = lod - (float)l0;
    int l1 = min(l0 + 1, A.kd.levels - 1);
    float2 guv = make_float2(0.f, 0.f);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        int k = s == 0 ? l0 : l1;
        float wl = s == 0 ? 1.f - fr : fr;
        if (wl == 0.f) continue;
        BilinTap b = bilin_tap(A.kd, k, tc);
        float w00 = wl * (1.f - b.fx) * (1.f - b.fy), w10 = wl * b.fx * (1.f - b.fy);
        float w01 = wl * (1.f - b.fx) * b.fy, w11 = wl * b.fx * b.fy;
        float gfx = 0.f, gfy = 0.f;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            float4 t00 = __ldg(ts[m] + b.idx[0]), t10 = __ldg(ts[m] + b.idx[1]);
            float4 t01 = __ldg(ts[m] + b.idx[2]), t11 = __ldg(ts[m] + b.idx[3]);
            gfx += dot4(g[m], f4madd(f4scale(f4sub(t10, t00), 1.f - b.fy), b.fy, f4sub(t11, t01)));
            gfy += dot4(g[m], f4madd(f4scale(f4sub(t01, t00), 1.f - b.fx), b.fx, f4sub(t11, t10)));
            if (gs[m]) {
                atomicAdd(gs[m] + b.idx[0], f4scale(g[m], w00));
                atomicAdd(gs[m] + b.idx[1], f4scale(g[m], w10));
                atomicAdd(gs[m] + b.idx[2], f4scale(g[m], w01));
                atomicAdd(gs[m] + b.idx[3], f4scale(g[m], w11));
            }
        }
        guv.x += wl * gfx * b.sw;
        guv.y += wl * gfy * b.sh;
    }
    return guv;
}

// tex_sample3 that also leaves, for each map m, dS_m/du and dS_m/dv (the derivatives
// of its trilinear sample w.r.t. the texture coordinate, float4 each) in
// stash[8 m .. 8 m + 7] (a lane's private shared-memory row): the adjoint then needs
// no second read of the texels
__device__ __forceinline__ void tex_sample3_stash(const ShadeArgs& A, const TexCoord& tc, float lod, float4 out[3],
                                                  float* stash) {
    const float4* ts[3] = {A.kd.tex, A.orm.tex, A.nrm.tex};
    int l0 = (int)floorf(lod);
    float fr = lod - (float)l0;
    int l1 = min(l0 + 1, A.kd.levels - 1);
    float4 du[3], dv[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        out[m] = du[m] = dv[m] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        int k = s == 0 ? l0 : l1;
        float wl = s == 0 ? 1.f - fr : fr;
        if (wl == 0.f) continue;
        BilinTap b = bilin_tap(A.kd, k, tc);
        float w00 = wl * (1.f - b.fx) * (1.f - b.fy), w10 = wl * b.fx * (1.f - b.fy);
        float w01 = wl * (1.f - b.fx) * b.fy, w11 = wl * b.fx * b.fy;
        float su = wl * b.sw, sv = wl * b.sh;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            float4 t00 = __ldg(ts[m] + b.idx[0]), t10 = __ldg(ts[m] + b.idx[1]);
            float4 t01 = __ldg(ts[m] + b.idx[2]), t11 = __ldg(ts[m] + b.idx[3]);
            out[m] = f4madd(out[m], w00, t00);
            out[m] = f4madd(out[m], w10, t10);
            out[m] = f4madd(out[m], w01, t01);
            out[m] = f4madd(out[m], w11, t11);
            du[m] = f4madd(du[m], su, f4madd(f4scale(f4sub(t10, t00), 1.f - b.fy), b.fy, f4sub(t11, t01)));
            dv[m] = f4madd(dv[m], sv, f4madd(f4scale(f4sub(t01, t00), 1.f - b.fx), b.fx, f4sub(t11, t10)));
        }
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        float* q = stash + 8 * m;
        q[0] = du[m].x;
        q[1] = du[m].y;
        q[2] = du[m].z;
        q[3] = du[m].w;
        q[4] = dv[m].x;
        q[5] = dv[m].y;
        q[6] = dv[m].z;
        q[7] = dv[m].w;
    }
}

// adjoint of tex_sample3_stash: the texel gradients of the optimized maps scattered,
// d/d(u, v) of g[0] . kd + g[1] . orm + g[2] . nm from the stashed derivatives
__device__ __forceinline__ float2 tex_sample3_bwd_stash(const ShadeArgs& A, const TexCoord& tc, float lod,
                                                        const float4 g[3], const float* stash) {
    float4* gs[3] = {A.kd.grad, A.orm.grad, A.nrm.grad};
    float2 guv = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const float* q = stash + 8 * m;
        guv.x += g[m].x * q[0] + g[m].y * q[1] + g[m].z * q[2] + g[m].w * q[3];
        guv.y += g[m].x * q[4] + g[m].y * q[5] + g[m].z * q[6] + g[m].w * q[7];
    }
    if (!gs[0] && !gs[1] && !gs[2]) return guv;
    int l0 = (int)floorf(lod);
    float fr = lod - (float)l0;
    int l1 = min(l0 + 1, A.kd.levels - 1);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        int k = s == 0 ? l0 : l1;
        float wl = s == 0 ? 1.f - fr : fr;
        if (wl == 0.f) continue;
        BilinTap b = bilin_tap(A.kd, k, tc);
        float w00 = wl * (1.f - b.fx) * (1.f - b.fy), w10 = wl * b.fx * (1.f - b.fy);
        float w01 = wl * (1.f - b.fx) * b.fy, w11 = wl * b.fx * b.fy;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            if (!gs[m]) continue;
            atomicAdd(gs[m] + b.idx[0], f4scale(g[m], w00));
            atomicAdd(gs[m] + b.idx[1], f4scale(g[m], w10));
            atomicAdd(gs[m] + b.idx[2], f4scale(g[m], w01));
            atomicAdd(gs[m] + b.idx[3], f4scale(g[m], w11));
        }
    }
    return guv;
}

// shading adjoint of triangle f at sample (px, py) for dL/d(colour) gc (and, for a
// peeled layer, dL/d(opacity) g_alpha): texel gradients scattered here, the three
// corners' position / normal / tangent gradients written to vrow[27] (corner k at
// 9k: position xyz, normal xyz, tangent xyz). The geometry is evaluated twice, once
// for the shading inputs and once after the BRDF and texture adjoints for the
// barycentric adjoint, so that nothing of it stays live across them.
template <bool PEEL>
__device__ __forceinline__ void shading_adjoint(const ShadeArgs& A, int b, int px, int py, int f, float3 gc,
                                                float g_alpha, float* vrow) {
    const adms_view& vw = A.views[b];
    float hW = 0.5f * (float)A.W, hH = 0.5f * (float)A.H;
    bool shared = shared_taps(A);
    TexCoord tc;
    float lod[3];
    ShadeGrad G;
    {
        PixGeo g;
        pix_geo<true, true>(A, b, px, py, f, g);
        ShadeIn in;
        in.p = g.p;
        in.n_i = g.n;
        in.t_i = g.t;
        if (shared) {
            lod[0] = lod[1] = lod[2] = tex_lod<true>(A.kd, g.duv_dx, g.duv_dy);
            float4 smp[3];
            tex_sample3_stash(A, g.tc, lod[0], smp, vrow);  // the row holds the uv derivatives until phase 4
            in.kd = smp[0];
            in.orm = smp[1];
            in.nm = smp[2];
        } else {
            lod[0] = tex_lod<true>(A.kd, g.duv_dx, g.duv_dy);
            lod[1] = tex_lod<true>(A.orm, g.duv_dx, g.duv_dy);
            lod[2] = tex_lod<true>(A.nrm, g.duv_dx, g.duv_dy);
            in.kd = tex_sample(A.kd, g.tc, lod[0]);
            in.orm = tex_sample(A.orm, g.tc, lod[1]);
            in.nm = tex_sample(A.nrm, g.tc, lod[2]);
        }
        tc = g.tc;
        shade_eval<true>(vw, in, gc, &G);
    }
    if (PEEL) G.kd.w = g_alpha;  // the opacity is the base colour's fourth channel
    float2 guv;
    if (shared) {
        float4 gt[3] = {G.kd, G.orm, G.nm};
        guv = tex_sample3_bwd_stash(A, tc, lod[0], gt, vrow);
    } else {
        guv = tex_sample_bwd(A.kd, tc, lod[0], G.kd);
        float2 g2 = tex_sample_bwd(A.orm, tc, lod[1], G.orm);
        float2 g3 = tex_sample_bwd(A.nrm, tc, lod[2], G.nm);
        guv.x += g2.x + g3.x;
        guv.y += g2.y + g3.y;
    }
    PixGeo g;
    pix_geo<false, true>(A, b, px, py, f, g);
    // interpolation: attr = sum_k beta_k attr_k, beta_k = r_k / R  =>  d attr / d r_j = (attr_j - attr) / R
    float gr[3];
    {
        float2 u0 = A.uv[g.ui[0]];
        float3 p0 = f3(A.vpos[g.vi[0]]), n0 = f3(A.vnrm[g.vi[0]]), t0 = f3(A.vtan[g.vi[0]]);
        float iR = fdiv<true>(1.f, g.R);
        gr[0] = -(dot3(G.p, g.dp) + dot3(G.n_i, g.dn) + dot3(G.t_i, g.dt) + guv.x * g.duv.x + guv.y * g.duv.y) * iR;
#pragma unroll
        for (int k = 1; k < 3; ++k) {
            float2 uk = A.uv[g.ui[k]];
            float3 ep = f3(A.vpos[g.vi[k]]) - p0 - g.dp;
            float3 en = f3(A.vnrm[g.vi[k]]) - n0 - g.dn;
            float3 et = f3(A.vtan[g.vi[k]]) - t0 - g.dt;
            float eu = (uk.x - u0.x) - g.duv.x, ev = (uk.y - u0.y) - g.duv.y;
            gr[k] = (dot3(G.p, ep) + dot3(G.n_i, en) + dot3(G.t_i, et) + guv.x * eu + guv.y * ev) * iR;
        }
    }
    float glam[3], gw[3], sgl = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float iw = fdiv<true>(1.f, g.c[k].w);
        glam[k] = gr[k] * iw;
        gw[k] = -gr[k] * g.r[k] * iw;
        sgl += glam[k] * g.lam[k];
    }
    float ia = fdiv<true>(1.f, g.area);
    float ge[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) ge[k] = (glam[k] - sgl) * ia;
    const float2* d = g.d;
    float2 gs[3];
    // e0 = cross(d1, d2), e1 = cross(d2, d0), e2 = cross(d0, d1)
    gs[0] = make_float2(-ge[1] * d[2].y + ge[2] * d[1].y, ge[1] * d[2].x - ge[2] * d[1].x);
    gs[1] = make_float2(ge[0] * d[2].y - ge[2] * d[0].y, -ge[0] * d[2].x + ge[2] * d[0].x);
    gs[2] = make_float2(-ge[0] * d[1].y + ge[1] * d[0].y, ge[0] * d[1].x - ge[1] * d[0].x);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float4 gcl = screen_bwd(g.c[k], hW, hH, gs[k]);
        gcl.w += gw[k];
        float3 gpk = g.beta[k] * G.p + clip_to_pos_grad(vw.mvp, gcl);
        float3 gnk = g.beta[k] * G.n_i, gtk = g.beta[k] * G.t_i;
        float* r = vrow + 9 * k;
        r[0] = gpk.x;
        r[1] = gpk.y;
        r[2] = gpk.z;
        r[3] = gnk.x;
        r[4] = gnk.y;
        r[5] = gnk.z;
        r[6] = gtk.x;
        r[7] = gtk.y;
        r[8] = gtk.z;
        vrow[ADMS_VROW_IDS + k] = __int_as_float(g.vi[k]);
    }
}

// one pixel of the fused backward; warp-collective (vertex scatter). rows: the
// warp's 32 x ADMS_VROW floats of shared memory
template <bool PEEL = false>
__device__ __forceinline__ void shade_bwd_px(const ShadeArgs& A, int b, int px, int py, float* rows) {
    bool inside = px < A.W && py < A.H;
    int f = -1;
    if (inside) {
        size_t pix = ((size_t)b * A.H + py) * A.W + px;
        unsigned long long kp = __ldg(A.keys + (pix));
        f = key_tri(kp);
        float3 gc = aa_adjoint<PEEL>(A, b, px, py, pix, kp);
        // a peeled layer: gc is dL/d(blend); split it into the layer's colour, its
        // opacity and the composite behind it (the next layer's dL/d(AA colour))
        float g_alpha = 0.f;
        if (PEEL) {
            float4 pr = A.pre[pix];
            float4 un = A.under ? A.under[pix] : make_float4(0.f, 0.f, 0.f, 0.f);
            if (A.g_under) {
                float3 gu = (1.f - pr.w) * gc;
                A.g_under[pix] = make_float4(gu.x, gu.y, gu.z, un.w);
            }
            g_alpha = dot3(gc, f3of(pr) - f3of(un));
            gc = pr.w * gc;
        }
        if (f >= 0 && (gc.x != 0.f || gc.y != 0.f || gc.z != 0.f || g_alpha != 0.f))
            shading_adjoint<PEEL>(A, b, px, py, f, gc, g_alpha, rows + (threadIdx.x & 31) * ADMS_VROW);
        else
            f = -1;
    }
    scatter_vertex_rows(A, f, rows);
}

}  // namespace adms
