// Shared device helpers for the render-and-compare kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "adms.h"

#define ADMS_EMPTY_KEY 0xFFFFFFFFFFFFFFFFull
#define ADMS_PI 3.14159265358979323846f
#define ADMS_EPS_NORM 1e-20f   // normalize(x) = x / sqrt(max(x.x, 1e-20))
#define ADMS_NV_MIN 1e-4f      // n.v clamped from below
#define ADMS_ROUGH_MIN 0.08f   // alpha = max(r, 0.08)^2
#define ADMS_MAX_LEVELS 16
#define ADMS_TILE 16           // raster / shading tile edge in pixels

// ------------------------------------------------------------------ float3 helpers
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 f3(const float4& a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator-(float3 a) { return f3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float3 operator*(float3 a, float3 b) { return f3(a.x * b.x, a.y * b.y, a.z * b.z); }
__device__ __forceinline__ float3& operator+=(float3& a, float3 b) { a.x += b.x; a.y += b.y; a.z += b.z; return a; }
__device__ __forceinline__ float3& operator-=(float3& a, float3 b) { a.x -= b.x; a.y -= b.y; a.z -= b.z; return a; }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 zero3() { return f3(0.f, 0.f, 0.f); }
__device__ __forceinline__ float cross2(float2 a, float2 b) { return a.x * b.y - a.y * b.x; }

// normalize with the guard x / sqrt(max(x.x, eps)) and its adjoint
struct Nrm3 {
    float3 y;
    float inv;
    bool big;
};
__device__ __forceinline__ Nrm3 nrm3(float3 x) {
    float d = dot3(x, x);
    Nrm3 r;
    r.big = d > ADMS_EPS_NORM;
    r.inv = rsqrtf(fmaxf(d, ADMS_EPS_NORM));
    r.y = x * r.inv;
    return r;
}
__device__ __forceinline__ float3 nrm3_bwd(const Nrm3& n, float3 gy) {
    if (n.big) return n.inv * (gy - n.y * dot3(n.y, gy));
    return n.inv * gy;
}

// ------------------------------------------------------------------ warp helpers
__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}
__device__ __forceinline__ double warp_sum_d(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// ------------------------------------------------------------------ double-float
// hi + lo with |lo| <= ulp(hi) / 2: about 48 significant bits from float32
// operations. Error-free sum (Knuth's TwoSum) and product (Dekker's, with an
// FMA for the product's rounding error); each operation is explicitly rounded
// so that no FMA contraction changes the error terms.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {  // |a| >= |b|
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
// a + b, a * b, a / b on double-float values (about 2^-44 relative)
__device__ __forceinline__ DF df_add(DF a, DF b) {
    DF s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, DF{-b.hi, -b.lo}); }
__device__ __forceinline__ DF df_add_f(DF a, float b) {
    DF s = df_two_sum(a.hi, b);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    DF p = df_two_prod(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return df_fast_two_sum(p.hi, e);
}
__device__ __forceinline__ DF df_div_f(DF a, float b) {
    float q1 = __fdiv_rn(a.hi, b);
    DF p = df_two_prod(q1, b);
    float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p.hi), p.lo), a.lo);
    return df_fast_two_sum(q1, __fdiv_rn(r, b));
}
__device__ __forceinline__ DF df_div_df(DF a, DF b) {
    float q1 = __fdiv_rn(a.hi, b.hi);
    DF p = df_mul(DF{q1, 0.f}, b);  // q1 * b
    DF r = df_sub(a, p);
    return df_fast_two_sum(q1, __fdiv_rn(r.hi, b.hi));
}
// a * b + c * d in float with one product's rounding error recovered (Kahan)
__device__ __forceinline__ float dot2_acc(float a, float b, float c, float d) {
    float w = __fmul_rn(c, d);
    float e = __fmaf_rn(c, d, -w);
    float f = __fmaf_rn(a, b, w);
    return __fadd_rn(f, e);
}

// ------------------------------------------------------------------ textures
// One texture with its full mip chain in one buffer, float4 texels.
struct TexDev {
    const float4* tex;  // all levels, level k at off[k]
    float4* grad;       // same layout; nullptr when not optimized
    int w0, h0, levels;
    int off[ADMS_MAX_LEVELS];
};

__device__ __forceinline__ int lvl_w(const TexDev& t, int k) { return max(t.w0 >> k, 1); }
__device__ __forceinline__ int lvl_h(const TexDev& t, int k) { return max(t.h0 >> k, 1); }

// LOD: rho = max(|(du/dx w, dv/dx h)|, |(du/dy w, dv/dy h)|); lod = clamp(log2 rho, 0, levels-1).
// FAST (the backward's recomputation, whose results only feed gradients): log2 rho
// as log2(rho^2) / 2 with the approximate log2, no square roots.
template <bool FAST = false>
__device__ __forceinline__ float tex_lod(const TexDev& t, float2 dx, float2 dy) {
    if (t.levels <= 1) return 0.f;
    float ax = (dx.x * t.w0) * (dx.x * t.w0) + (dx.y * t.h0) * (dx.y * t.h0);
    float ay = (dy.x * t.w0) * (dy.x * t.w0) + (dy.y * t.h0) * (dy.y * t.h0);
    float lod = FAST ? 0.5f * __log2f(fmaxf(ax, ay)) : log2f(fmaxf(sqrtf(ax), sqrtf(ay)));
    if (!(lod > 0.f)) lod = 0.f;  // also catches NaN and -inf
    return fminf(lod, (float)(t.levels - 1));
}

// Texture coordinate kept as (u0 + du, v0 + dv): u0 is the UV of the triangle's
// first corner and du the interpolated offset from it as a double-float
// (du + du_lo). The offset spans up to the triangle's texel extent (tens of
// texels on 1024² maps), and with noise textures under sharp highlights a
// texel-coordinate error of 1e-6 texel already moves a pixel by ~1e-5.
struct TexCoord {
    float u0, v0, du, dv, du_lo, dv_lo;
};

// integer part and fraction of (a0 * n - 1/2) + (d + dlo) * n, n a power of two;
// the fraction keeps float32 precision whatever the offset's size
__device__ __forceinline__ void texel_coord(float a0, float d, float dlo, int n, int& i, float& f) {
    float X0 = a0 * (float)n - 0.5f;  // exact: power-of-two scale, then a half-ulp-safe shift
    float i0 = floorf(X0);
    if (dlo == 0.f) {  // float32 offset
        float r = (X0 - i0) + d * (float)n;
        float ri = floorf(r);
        i = (int)i0 + (int)ri;
        f = r - ri;
        return;
    }
    DF s = df_two_sum(X0 - i0, d * (float)n);  // X0 - i0 and d n exact
    float lo = __fadd_rn(s.lo, dlo * (float)n);
    float ri = floorf(s.hi);
    float fr = __fadd_rn(s.hi - ri, lo);      // s.hi - ri exact
    if (fr < 0.f) {
        fr = __fadd_rn(fr, 1.f);
        ri -= 1.f;
    } else if (fr >= 1.f) {
        fr = __fsub_rn(fr, 1.f);
        ri += 1.f;
    }
    i = (int)i0 + (int)ri;
    f = fr;
}

struct BilinTap {
    int idx[4];   // absolute texel indices (00, 10, 01, 11)
    float fx, fy;
    float sw, sh;  // level size, for du/dv chain
};

__device__ __forceinline__ BilinTap bilin_tap(const TexDev& t, int k, const TexCoord& tc) {
    BilinTap b;
    int w = lvl_w(t, k), h = lvl_h(t, k);
    int ix0, iy0;
    texel_coord(tc.u0, tc.du, tc.du_lo, w, ix0, b.fx);
    texel_coord(tc.v0, tc.dv, tc.dv_lo, h, iy0, b.fy);
    int ixa = ix0 & (w - 1);  // u wraps: w is a power of two (two's complement: negative ix0 wraps too)
    int ixb = (ixa + 1) & (w - 1);
    int iya = min(max(iy0, 0), h - 1), iyb = min(max(iy0 + 1, 0), h - 1);
    int base = t.off[k];
    b.idx[0] = base + iya * w + ixa;
    b.idx[1] = base + iya * w + ixb;
    b.idx[2] = base + iyb * w + ixa;
    b.idx[3] = base + iyb * w + ixb;
    b.sw = (float)w;
    b.sh = (float)h;
    return b;
}

__device__ __forceinline__ float4 f4madd(float4 a, float s, float4 b) {
    return make_float4(a.x + s * b.x, a.y + s * b.y, a.z + s * b.z, a.w + s * b.w);
}

// trilinear sample (lod held fixed)
__device__ __forceinline__ float4 tex_sample(const TexDev& t, const TexCoord& tc, float lod) {
    int l0 = (int)floorf(lod);
    float fr = lod - (float)l0;
    int l1 = min(l0 + 1, t.levels - 1);
    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        int k = s == 0 ? l0 : l1;
        float wl = s == 0 ? 1.f - fr : fr;
        if (wl == 0.f) continue;
        BilinTap b = bilin_tap(t, k, tc);
        float4 t00 = __ldg(t.tex + b.idx[0]), t10 = __ldg(t.tex + b.idx[1]);
        float4 t01 = __ldg(t.tex + b.idx[2]), t11 = __ldg(t.tex + b.idx[3]);
        out = f4madd(out, wl * (1.f - b.fx) * (1.f - b.fy), t00);
        out = f4madd(out, wl * b.fx * (1.f - b.fy), t10);
        out = f4madd(out, wl * (1.f - b.fx) * b.fy, t01);
        out = f4madd(out, wl * b.fx * b.fy, t11);
    }
    return out;
}

__device__ __forceinline__ float dot4(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }
__device__ __forceinline__ float4 f4scale(float4 a, float s) { return make_float4(a.x * s, a.y * s, a.z * s, a.w * s); }
__device__ __forceinline__ float4 f4sub(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }

// adjoint of tex_sample: scatters texel gradients (if t.grad) and returns d/d(u, v)
__device__ __forceinline__ float2 tex_sample_bwd(const TexDev& t, const TexCoord& tc, float lod, float4 g) {
    int l0 = (int)floorf(lod);
    float fr = lod - (float)l0;
    int l1 = min(l0 + 1, t.levels - 1);
    float2 guv = make_float2(0.f, 0.f);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        int k = s == 0 ? l0 : l1;
        float wl = s == 0 ? 1.f - fr : fr;
        if (wl == 0.f) continue;
        BilinTap b = bilin_tap(t, k, tc);
        float4 t00 = __ldg(t.tex + b.idx[0]), t10 = __ldg(t.tex + b.idx[1]);
        float4 t01 = __ldg(t.tex + b.idx[2]), t11 = __ldg(t.tex + b.idx[3]);
        float gfx = wl * dot4(g, f4madd(f4scale(f4sub(t10, t00), 1.f - b.fy), b.fy, f4sub(t11, t01)));
        float gfy = wl * dot4(g, f4madd(f4scale(f4sub(t01, t00), 1.f - b.fx), b.fx, f4sub(t11, t10)));
        guv.x += gfx * b.sw;
        guv.y += gfy * b.sh;
        if (t.grad) {
            atomicAdd(t.grad + b.idx[0], f4scale(g, wl * (1.f - b.fx) * (1.f - b.fy)));
            atomicAdd(t.grad + b.idx[1], f4scale(g, wl * b.fx * (1.f - b.fy)));
            atomicAdd(t.grad + b.idx[2], f4scale(g, wl * (1.f - b.fx) * b.fy));
            atomicAdd(t.grad + b.idx[3], f4scale(g, wl * b.fx * b.fy));
        }
    }
    return guv;
}

// ------------------------------------------------------------------ views
__device__ __forceinline__ float2 screen_of(float4 c, float hW, float hH) {
    return make_float2(c.x / c.w * hW + hW, hH - c.y / c.w * hH);
}

// adjoint of screen_of: d/d(clip)
__device__ __forceinline__ float4 screen_bwd(float4 c, float hW, float hH, float2 g) {
    float iw = 1.f / c.w;
    float4 gc;
    gc.x = g.x * hW * iw;
    gc.y = -g.y * hH * iw;
    gc.z = 0.f;
    gc.w = (-g.x * hW * c.x + g.y * hH * c.y) * iw * iw;
    return gc;
}

// d/d(position) of clip = M [p 1]: M[:, :3]^T gc
__device__ __forceinline__ float3 clip_to_pos_grad(const float* M, float4 gc) {
    return f3(M[0] * gc.x + M[4] * gc.y + M[8] * gc.z + M[12] * gc.w,
              M[1] * gc.x + M[5] * gc.y + M[9] * gc.z + M[13] * gc.w,
              M[2] * gc.x + M[6] * gc.y + M[10] * gc.z + M[14] * gc.w);
}

// ------------------------------------------------------------------ errors
#define ADMS_LAUNCH_CHECK() cudaGetLastError()
