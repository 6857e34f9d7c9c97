// Per-stage calls: the renderer as separate differentiable primitives, each with
// its adjoint, for an autograd system that chains them (Sec. 5.2 builds the
// renderer from a rasterizer, attribute interpolation, filtered texture lookups
// and an antialiasing pass; Sec. 3 differentiates the image loss through all of
// them to every latent).
//
//   frame    (Sec. 5.1)  positions -> unit smooth normals and tangents
//   setup    (Sec. 5.2)  positions -> clip coordinates; triangle setup and tile bins
//   raster   (Sec. 5.2)  -> visibility keys and perspective-correct barycentrics
//   shade    (Sec. 5.2)  barycentrics -> interpolated attributes, mip-mapped
//                        lookups, normal mapping, GGX -> pre-antialiasing colour
//   aa_loss  (Sec. 5.2, 5.3) silhouette antialiasing + image loss
//
// Unlike the fused step, the per-pixel barycentrics travel between raster and
// shade as a buffer (b1, b2 per pixel, with their screen derivatives for the
// LOD), so that raster's adjoint (dL/d(b1, b2) -> clip coordinates) and shade's
// (dL/d(colour) -> texels, vertex attributes, dL/d(b1, b2)) are separate calls.
// The arithmetic is the fused kernels' own (pixel.cuh). Every buffer is the
// caller's; nothing is allocated here.
#include "pixel.cuh"

using namespace adms;

namespace {

// ------------------------------------------------------------------ workspace
struct StageWork {
    RasterScratch s;
    size_t bytes;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// carve the setup / raster scratch out of `base` (null: only count the bytes)
StageWork carve_work(unsigned char* base, size_t V, size_t F, size_t B, int H, int W, size_t list_entries) {
    StageWork w{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return base ? base + o : nullptr;
    };
    size_t ntiles = B * (size_t)((W + ADMS_TILE - 1) / ADMS_TILE) * (size_t)((H + ADMS_TILE - 1) / ADMS_TILE);
    w.s.scr = reinterpret_cast<float4*>(take(B * V * sizeof(float4)));
    w.s.vs = reinterpret_cast<VtxS*>(take(B * V * sizeof(VtxS)));
    w.s.rec = reinterpret_cast<TriRec*>(take(B * F * sizeof(TriRec)));
    w.s.bin = reinterpret_cast<TriBin*>(take(B * F * sizeof(TriBin)));
    w.s.asign = reinterpret_cast<int8_t*>(take(B * F));
    w.s.silmask = reinterpret_cast<uint8_t*>(take(B * F));
    w.s.tile_count = reinterpret_cast<int*>(take(ntiles * sizeof(int)));
    w.s.tile_off = reinterpret_cast<int*>(take(ntiles * sizeof(int)));
    w.s.tile_cursor = reinterpret_cast<int*>(take(ntiles * sizeof(int)));
    w.s.total_pairs = reinterpret_cast<long long*>(take(sizeof(long long)));
    w.s.overflow_ctr = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long)));
    w.s.list = reinterpret_cast<int*>(take(list_entries * sizeof(int)));
    w.s.list_capacity = (long long)list_entries;
    w.bytes = off;
    return w;
}

// list entries a workspace of `bytes` holds for this problem (0 if it does not fit)
bool work_of(void* work, size_t work_bytes, size_t V, size_t F, size_t B, int H, int W, StageWork& w) {
    StageWork probe = carve_work(nullptr, V, F, B, H, W, 0);
    if (!work || work_bytes < probe.bytes + 4 * sizeof(int) || (reinterpret_cast<uintptr_t>(work) & 255)) return false;
    size_t entries = (work_bytes - probe.bytes) / sizeof(int);
    w = carve_work(static_cast<unsigned char*>(work), V, F, B, H, W, entries);
    return w.bytes <= work_bytes;
}

bool sizes_ok(const adms_stage_mesh* m, int B, int H, int W) {
    return m && m->pos && m->tri && m->n_verts > 0 && m->n_tris > 0 && B > 0 && H > 0 && W > 0 && H <= 16384 &&
           W <= 16384;
}

TexDev tex_dev(const adms_stage_texture& t) {
    TexDev d{};
    d.tex = reinterpret_cast<const float4*>(t.tex);
    d.grad = reinterpret_cast<float4*>(t.grad);
    d.w0 = t.w;
    d.h0 = t.h;
    d.levels = t.levels;
    int off = 0;
    for (int k = 0; k < ADMS_MAX_LEVELS; ++k) {
        d.off[k] = off;
        if (k < t.levels) off += std::max(t.w >> k, 1) * std::max(t.h >> k, 1);
    }
    return d;
}

bool tex_ok(const adms_stage_texture& t) {
    auto pow2 = [](int x) { return x > 0 && (x & (x - 1)) == 0; };
    int full = 1;
    while ((std::max(t.w, t.h) >> (full - 1)) > 1) ++full;
    return t.tex && pow2(t.w) && pow2(t.h) && t.levels >= 1 && t.levels <= std::min(full, ADMS_MAX_LEVELS);
}

ShadeArgs stage_args(const adms_stage_mesh* m, const adms_view* views, int B, int H, int W) {
    ShadeArgs a;
    memset(&a, 0, sizeof(a));
    a.B = B;
    a.H = H;
    a.W = W;
    a.V = m->n_verts;
    a.F = m->n_tris;
    a.views = views;
    a.uv = reinterpret_cast<const float2*>(m->uv);
    a.tri = m->tri;
    a.tri_uv = m->tri_uv;
    a.aa = 1;
    return a;
}

dim3 pix_grid(int B, int H, int W) {
    return dim3(((W + ADMS_TILE - 1) / ADMS_TILE) * ((H + ADMS_TILE - 1) / ADMS_TILE), B);
}

__device__ __forceinline__ void tile_pixel(int W, int& px, int& py) {
    int tiles_x = (W + ADMS_TILE - 1) / ADMS_TILE;
    px = (blockIdx.x % tiles_x) * ADMS_TILE + (threadIdx.x & 15);
    py = (blockIdx.x / tiles_x) * ADMS_TILE + (threadIdx.x >> 4);
}

// ------------------------------------------------------------------ kernels
// barycentrics (b1, b2) of each covered pixel and their screen derivatives (not
// written when rast_db is null)
__global__ void __launch_bounds__(256) k_stage_bary(ShadeArgs A, float2* __restrict__ rast,
                                                    float4* __restrict__ rast_db) {
    int px, py;
    tile_pixel(A.W, px, py);
    if (px >= A.W || py >= A.H) return;
    int b = blockIdx.y;
    size_t pix = ((size_t)b * A.H + py) * A.W + px;
    int f = key_tri(A.keys[pix]);
    if (f < 0) {
        rast[pix] = make_float2(0.f, 0.f);
        if (rast_db) rast_db[pix] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    PixGeo g;
    pix_bary(A, b, px, py, f, g);
    rast[pix] = make_float2(g.beta[1], g.beta[2]);
    if (rast_db) rast_db[pix] = bary_derivs(g);
}

__device__ __forceinline__ void corner_ids(const ShadeArgs& A, int f, PixGeo& g) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        g.vi[k] = A.tri[3 * f + k];
        g.ui[k] = A.tri_uv[3 * f + k];
    }
}

// the three maps' trilinear samples at g's texture coordinate (LODs into lod)
__device__ __forceinline__ void stage_samples(const ShadeArgs& A, const PixGeo& g, float lod[3], ShadeIn& in) {
    in.p = g.p;
    in.n_i = g.n;
    in.t_i = g.t;
    if (shared_taps(A)) {
        lod[0] = lod[1] = lod[2] = tex_lod(A.kd, g.duv_dx, g.duv_dy);
        float4 smp[3];
        tex_sample3(A, g.tc, lod[0], smp);
        in.kd = smp[0];
        in.orm = smp[1];
        in.nm = smp[2];
    } else {
        lod[0] = tex_lod(A.kd, g.duv_dx, g.duv_dy);
        lod[1] = tex_lod(A.orm, g.duv_dx, g.duv_dy);
        lod[2] = tex_lod(A.nrm, g.duv_dx, g.duv_dy);
        in.kd = tex_sample(A.kd, g.tc, lod[0]);
        in.orm = tex_sample(A.orm, g.tc, lod[1]);
        in.nm = tex_sample(A.nrm, g.tc, lod[2]);
    }
}

// pre-antialiasing colour from the barycentrics buffer
__global__ void __launch_bounds__(256) k_stage_shade_fwd(ShadeArgs A, const float2* __restrict__ rast,
                                                         const float4* __restrict__ rast_db) {
    int px, py;
    tile_pixel(A.W, px, py);
    if (px >= A.W || py >= A.H) return;
    int b = blockIdx.y;
    size_t pix = ((size_t)b * A.H + py) * A.W + px;
    int f = key_tri(A.keys[pix]);
    if (f < 0) {
        A.pre[pix] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    PixGeo g;
    corner_ids(A, f, g);
    float2 bb = rast[pix];
    pix_attr<true>(A, g, bb.x, bb.y, rast_db[pix]);
    float lod[3];
    ShadeIn in;
    stage_samples(A, g, lod, in);
    float3 c = shade_eval<false>(A.views[b], in, zero3(), nullptr);
    A.pre[pix] = make_float4(c.x, c.y, c.z, 1.f);
}

// Adjoint of k_stage_shade_fwd for dL/d(pre) = g_pre: texel gradients scattered
// into the maps' gradient chains, dL/d(b1, b2) per pixel into g_rast, and the
// corners' position / unit normal / unit tangent gradients summed per warp and
// triangle into A.g_pos, A.g_nrm, A.g_tan. The attributes are corner 0 plus
// b1, b2 times the corner differences, so corner 0 takes weight 1 - b1 - b2.
__global__ void __launch_bounds__(256, 3) k_stage_shade_bwd(ShadeArgs A, const float2* __restrict__ rast,
                                                            const float4* __restrict__ rast_db,
                                                            const float4* __restrict__ g_pre, float2* __restrict__ g_rast) {
    __shared__ float rows_all[8 * 32 * ADMS_VROW];
    float* rows = rows_all + (threadIdx.x >> 5) * 32 * ADMS_VROW;
    int px, py;
    tile_pixel(A.W, px, py);
    int b = blockIdx.y;
    int f = -1;
    if (px < A.W && py < A.H) {
        size_t pix = ((size_t)b * A.H + py) * A.W + px;
        f = key_tri(A.keys[pix]);
        float3 gc = f3of(g_pre[pix]);
        float2 gb = make_float2(0.f, 0.f);
        if (f >= 0 && (gc.x != 0.f || gc.y != 0.f || gc.z != 0.f)) {
            float2 bb = rast[pix];
            TexCoord tc;
            float lod[3];
            ShadeGrad G;
            {
                PixGeo g;
                corner_ids(A, f, g);
                pix_attr<true>(A, g, bb.x, bb.y, rast_db[pix]);
                ShadeIn in;
                stage_samples(A, g, lod, in);
                tc = g.tc;
                shade_eval<true>(A.views[b], in, gc, &G);
            }
            float2 guv;
            if (shared_taps(A)) {
                float4 gt[3] = {G.kd, G.orm, G.nm};
                guv = tex_sample3_bwd(A, tc, lod[0], gt);
            } else {
                guv = tex_sample_bwd(A.kd, tc, lod[0], G.kd);
                float2 g2 = tex_sample_bwd(A.orm, tc, lod[1], G.orm);
                float2 g3 = tex_sample_bwd(A.nrm, tc, lod[2], G.nm);
                guv.x += g2.x + g3.x;
                guv.y += g2.y + g3.y;
            }
            int vi[3], ui[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                vi[k] = A.tri[3 * f + k];
                ui[k] = A.tri_uv[3 * f + k];
            }
            float3 p0 = f3(A.vpos[vi[0]]), n0 = f3(A.vnrm[vi[0]]), t0 = f3(A.vtan[vi[0]]);
            float2 u0 = A.uv[ui[0]];
            float gbk[3];
#pragma unroll
            for (int k = 1; k < 3; ++k) {
                float2 uk = A.uv[ui[k]];
                gbk[k] = dot3(G.p, f3(A.vpos[vi[k]]) - p0) + dot3(G.n_i, f3(A.vnrm[vi[k]]) - n0) +
                         dot3(G.t_i, f3(A.vtan[vi[k]]) - t0) + guv.x * (uk.x - u0.x) + guv.y * (uk.y - u0.y);
            }
            gb = make_float2(gbk[1], gbk[2]);
            float w[3] = {1.f - bb.x - bb.y, bb.x, bb.y};
            float* r = rows + (threadIdx.x & 31) * ADMS_VROW;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                float3 gp = w[k] * G.p, gn = w[k] * G.n_i, gt = w[k] * G.t_i;
                r[9 * k + 0] = gp.x;
                r[9 * k + 1] = gp.y;
                r[9 * k + 2] = gp.z;
                r[9 * k + 3] = gn.x;
                r[9 * k + 4] = gn.y;
                r[9 * k + 5] = gn.z;
                r[9 * k + 6] = gt.x;
                r[9 * k + 7] = gt.y;
                r[9 * k + 8] = gt.z;
                r[ADMS_VROW_IDS + k] = __int_as_float(vi[k]);
            }
        } else {
            f = -1;
        }
        g_rast[pix] = gb;
    }
    scatter_vertex_rows(A, f, rows);
}

// Adjoint of the barycentrics: dL/d(b1, b2) per pixel -> dL/d(clip coordinates)
// of the triangle's corners in that view. With b_k = r_k / R, dL/dr_j =
// (dL/db_j [j >= 1] - (dL/db1 b1 + dL/db2 b2)) / R; then the chain of pix_bary
// (r_k = lam_k / w_k, lam_k = e_k / area, e_k from the screen offsets, the screen
// position from clip). The 12 values per pixel (4 per corner) are summed per warp
// and triangle through shared memory (odd stride 13) before float64 atomics.
#define ADMS_CROW 13
__global__ void __launch_bounds__(256) k_stage_raster_bwd(ShadeArgs A, const float2* __restrict__ g_rast) {
    __shared__ float rows_all[8 * 32 * ADMS_CROW];
    float* rows = rows_all + (threadIdx.x >> 5) * 32 * ADMS_CROW;
    int lane = threadIdx.x & 31;
    int px, py;
    tile_pixel(A.W, px, py);
    int b = blockIdx.y;
    int f = -1;
    if (px < A.W && py < A.H) {
        size_t pix = ((size_t)b * A.H + py) * A.W + px;
        f = key_tri(A.keys[pix]);
        float2 gb = g_rast[pix];
        if (f >= 0 && (gb.x != 0.f || gb.y != 0.f)) {
            float hW = 0.5f * (float)A.W, hH = 0.5f * (float)A.H;
            PixGeo g;
            pix_bary(A, b, px, py, f, g);
            float iR = 1.f / g.R;
            float s = gb.x * g.beta[1] + gb.y * g.beta[2];
            float gr[3] = {-s * iR, (gb.x - s) * iR, (gb.y - s) * iR};
            float glam[3], gw[3], sgl = 0.f;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                glam[k] = gr[k] / g.c[k].w;
                gw[k] = -gr[k] * g.r[k] / g.c[k].w;
                sgl += glam[k] * g.lam[k];
            }
            float ia = 1.f / g.area;
            float ge[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) ge[k] = (glam[k] - sgl) * ia;
            const float2* d = g.d;
            float2 gs[3];
            gs[0] = make_float2(-ge[1] * d[2].y + ge[2] * d[1].y, ge[1] * d[2].x - ge[2] * d[1].x);
            gs[1] = make_float2(ge[0] * d[2].y - ge[2] * d[0].y, -ge[0] * d[2].x + ge[2] * d[0].x);
            gs[2] = make_float2(-ge[0] * d[1].y + ge[1] * d[0].y, ge[0] * d[1].x - ge[1] * d[0].x);
            float* r = rows + lane * ADMS_CROW;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                float4 gcl = screen_bwd(g.c[k], hW, hH, gs[k]);
                gcl.w += gw[k];
                r[4 * k + 0] = gcl.x;
                r[4 * k + 1] = gcl.y;
                r[4 * k + 2] = gcl.z;
                r[4 * k + 3] = gcl.w;
            }
        } else {
            f = -1;
        }
    }
    __syncwarp();
    unsigned todo = __ballot_sync(0xffffffffu, f >= 0);
    while (todo) {
        int lead = __ffs(todo) - 1;
        int ft = __shfl_sync(0xffffffffu, f, lead);
        unsigned grp = __ballot_sync(0xffffffffu, f == ft);
        if (lane < 12) {
            float sum = 0.f;
            for (unsigned m = grp; m; m &= m - 1) sum += rows[(__ffs(m) - 1) * ADMS_CROW + lane];
            if (sum != 0.f) {
                int vtx = A.tri[3 * ft + lane / 4];
                atomicAdd(A.g_clip + 4 * ((size_t)b * A.V + vtx) + (lane & 3), (double)sum);
            }
        }
        todo &= ~grp;
    }
}

// adjoint of the vertex transform clip = M [p 1]: g_pos += sum over views of
// M[:, :3]^T g_clip, one thread per vertex (no atomics)
__global__ void k_stage_setup_bwd(const adms_view* __restrict__ views, int B, int V, const double* __restrict__ g_clip,
                                  float* __restrict__ g_pos) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    double g[3] = {0.0, 0.0, 0.0};
    for (int b = 0; b < B; ++b) {
        const float* M = views[b].mvp;
        const double* gc = g_clip + 4 * ((size_t)b * V + v);
#pragma unroll
        for (int i = 0; i < 3; ++i)
            g[i] += (double)M[i] * gc[0] + (double)M[4 + i] * gc[1] + (double)M[8 + i] * gc[2] + (double)M[12 + i] * gc[3];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) g_pos[3 * v + i] += (float)g[i];
}

// adjoint of antialiasing + loss: dL/d(pre) = the AA adjoint of g_loss x gprime;
// silhouette-edge gradients into A.g_clip
__global__ void __launch_bounds__(256) k_stage_aa_bwd(ShadeArgs A, const float* __restrict__ g_loss,
                                                      float4* __restrict__ g_pre) {
    int px, py;
    tile_pixel(A.W, px, py);
    if (px >= A.W || py >= A.H) return;
    int b = blockIdx.y;
    size_t pix = ((size_t)b * A.H + py) * A.W + px;
    float scale = g_loss ? *g_loss : 1.f;
    float3 gc = scale * aa_adjoint<false, true>(A, b, px, py, pix, A.keys[pix], scale);
    g_pre[pix] = make_float4(gc.x, gc.y, gc.z, 0.f);
}

#define ADMS_STAGE_CHECK(expr)                            \
    do {                                                  \
        if ((expr) != cudaSuccess) return ADMS_ERR_CUDA; \
    } while (0)

}  // namespace

extern "C" {

size_t adms_stage_workspace_bytes(int32_t n_verts, int32_t n_tris, int32_t n_views, int32_t H, int32_t W,
                                  int64_t list_entries) {
    if (n_verts <= 0 || n_tris <= 0 || n_views <= 0 || H <= 0 || W <= 0 || list_entries < 4) return 0;
    return carve_work(nullptr, n_verts, n_tris, n_views, H, W, (size_t)list_entries).bytes;
}

adms_status adms_frame_fwd(const adms_stage_mesh* m, float* vpos4, float* vnrm4, float* vtan4, void* cuda_stream) {
    if (!m || !m->pos || !m->uv || !m->tri || !m->tri_uv || !m->vf_off || !m->vf_face || !vpos4 || !vnrm4 || !vtan4 ||
        m->n_verts <= 0 || m->n_tris <= 0)
        return ADMS_ERR_ARG;
    FrameArgs a{};
    a.V = m->n_verts;
    a.F = m->n_tris;
    a.pos = m->pos;
    a.uv = reinterpret_cast<const float2*>(m->uv);
    a.tri = m->tri;
    a.tri_uv = m->tri_uv;
    a.vf_off = m->vf_off;
    a.vf_face = m->vf_face;
    a.vpos = reinterpret_cast<float4*>(vpos4);
    a.vnrm = reinterpret_cast<float4*>(vnrm4);
    a.vtan = reinterpret_cast<float4*>(vtan4);
    ADMS_STAGE_CHECK(frame_forward(a, (cudaStream_t)cuda_stream));
    return ADMS_OK;
}

adms_status adms_frame_bwd(const adms_stage_mesh* m, double* g_vpos, const double* g_vnrm, const double* g_vtan,
                           float* g_pos, float* tmp, void* cuda_stream) {
    if (!m || !m->pos || !m->uv || !m->tri || !m->tri_uv || !m->vf_off || !m->vf_face || !g_vpos || !g_vnrm ||
        !g_vtan || !g_pos || !tmp || m->n_verts <= 0 || m->n_tris <= 0)
        return ADMS_ERR_ARG;
    FrameArgs a{};
    a.V = m->n_verts;
    a.F = m->n_tris;
    a.pos = m->pos;
    a.uv = reinterpret_cast<const float2*>(m->uv);
    a.tri = m->tri;
    a.tri_uv = m->tri_uv;
    a.vf_off = m->vf_off;
    a.vf_face = m->vf_face;
    a.g_nrm = g_vnrm;
    a.g_tan = g_vtan;
    a.tmp_n = reinterpret_cast<float4*>(tmp);
    a.tmp_t = reinterpret_cast<float4*>(tmp) + m->n_verts;
    a.g_pos_acc = g_vpos;
    a.g_pos = g_pos;
    ADMS_STAGE_CHECK(frame_backward(a, (cudaStream_t)cuda_stream));
    return ADMS_OK;
}

adms_status adms_setup_fwd(const adms_stage_mesh* m, const adms_view* views, int32_t n_views, int32_t H, int32_t W,
                           float* clip, void* work, size_t work_bytes, void* cuda_stream) {
    if (!sizes_ok(m, n_views, H, W) || !m->adj || !views || !clip) return ADMS_ERR_ARG;
    StageWork w;
    if (!work_of(work, work_bytes, m->n_verts, m->n_tris, n_views, H, W, w)) return ADMS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    w.s.clip = reinterpret_cast<float4*>(clip);
    RasterIn in;
    in.pos = m->pos;
    in.tri = m->tri;
    in.adj = m->adj;
    in.views = views;
    in.B = n_views;
    in.V = m->n_verts;
    in.F = m->n_tris;
    in.W = W;
    in.H = H;
    in.keys = nullptr;
    in.small_px = 0;  // every triangle binned: the keys are raster_fwd's alone
    ADMS_STAGE_CHECK(cudaMemsetAsync(w.s.overflow_ctr, 0, sizeof(unsigned long long), st));
    ADMS_STAGE_CHECK(raster_prepare(in, w.s, st));
    return ADMS_OK;
}

adms_status adms_setup_bwd(const adms_view* views, int32_t n_views, int32_t n_verts, const double* g_clip, float* g_pos,
                           void* cuda_stream) {
    if (!views || !g_clip || !g_pos || n_views <= 0 || n_verts <= 0) return ADMS_ERR_ARG;
    k_stage_setup_bwd<<<(n_verts + 127) / 128, 128, 0, (cudaStream_t)cuda_stream>>>(views, n_views, n_verts, g_clip,
                                                                                    g_pos);
    count_launches(1);
    ADMS_STAGE_CHECK(cudaGetLastError());
    return ADMS_OK;
}

adms_status adms_raster_fwd(const adms_stage_mesh* m, const adms_view* views, int32_t n_views, int32_t H, int32_t W,
                            const float* clip, uint64_t* keys, int32_t keep_keys, float* rast, float* rast_db,
                            void* work, size_t work_bytes, void* cuda_stream) {
    if (!sizes_ok(m, n_views, H, W) || !m->tri_uv || !views || !clip || !keys || !rast || !rast_db) return ADMS_ERR_ARG;
    StageWork w;
    if (!work_of(work, work_bytes, m->n_verts, m->n_tris, n_views, H, W, w)) return ADMS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    w.s.clip = reinterpret_cast<float4*>(const_cast<float*>(clip));
    RasterIn in;
    in.pos = m->pos;
    in.tri = m->tri;
    in.adj = m->adj;
    in.views = views;
    in.B = n_views;
    in.V = m->n_verts;
    in.F = m->n_tris;
    in.W = W;
    in.H = H;
    in.keys = reinterpret_cast<unsigned long long*>(keys);
    in.small_px = 0;
    if (!keep_keys) {
        ADMS_STAGE_CHECK(cudaMemsetAsync(keys, 0xFF, sizeof(uint64_t) * (size_t)n_views * H * W, st));
        ADMS_STAGE_CHECK(raster_tiles(in, w.s, st));
    }
    ShadeArgs a = stage_args(m, views, n_views, H, W);
    a.clip = reinterpret_cast<const float4*>(clip);
    a.scr = w.s.scr;
    a.keys = in.keys;
    k_stage_bary<<<pix_grid(n_views, H, W), 256, 0, st>>>(a, reinterpret_cast<float2*>(rast),
                                                          keep_keys ? nullptr : reinterpret_cast<float4*>(rast_db));
    count_launches(1);
    ADMS_STAGE_CHECK(cudaGetLastError());
    return ADMS_OK;
}

adms_status adms_raster_bwd(const adms_stage_mesh* m, const adms_view* views, int32_t n_views, int32_t H, int32_t W,
                            const float* clip, const uint64_t* keys, const float* g_rast, double* g_clip, void* work,
                            size_t work_bytes, void* cuda_stream) {
    if (!sizes_ok(m, n_views, H, W) || !views || !clip || !keys || !g_rast || !g_clip) return ADMS_ERR_ARG;
    StageWork w;
    if (!work_of(work, work_bytes, m->n_verts, m->n_tris, n_views, H, W, w)) return ADMS_ERR_ARG;
    ShadeArgs a = stage_args(m, views, n_views, H, W);
    a.clip = reinterpret_cast<const float4*>(clip);
    a.scr = w.s.scr;
    a.keys = reinterpret_cast<const unsigned long long*>(keys);
    a.g_clip = g_clip;
    k_stage_raster_bwd<<<pix_grid(n_views, H, W), 256, 0, (cudaStream_t)cuda_stream>>>(
        a, reinterpret_cast<const float2*>(g_rast));
    count_launches(1);
    ADMS_STAGE_CHECK(cudaGetLastError());
    return ADMS_OK;
}

static adms_status shade_stage_args(const adms_stage_mesh* m, const adms_view* views, int32_t n_views, int32_t H,
                                    int32_t W, const uint64_t* keys, const float* rast, const float* rast_db,
                                    const float* vpos4, const float* vnrm4, const float* vtan4,
                                    const adms_stage_texture* maps, ShadeArgs& a) {
    if (!sizes_ok(m, n_views, H, W) || !m->uv || !m->tri_uv || !views || !keys || !rast || !rast_db || !vpos4 ||
        !vnrm4 || !vtan4 || !maps || !tex_ok(maps[0]) || !tex_ok(maps[1]) || !tex_ok(maps[2]))
        return ADMS_ERR_ARG;
    a = stage_args(m, views, n_views, H, W);
    a.keys = reinterpret_cast<const unsigned long long*>(keys);
    a.vpos = reinterpret_cast<const float4*>(vpos4);
    a.vnrm = reinterpret_cast<const float4*>(vnrm4);
    a.vtan = reinterpret_cast<const float4*>(vtan4);
    a.kd = tex_dev(maps[0]);
    a.orm = tex_dev(maps[1]);
    a.nrm = tex_dev(maps[2]);
    return ADMS_OK;
}

adms_status adms_shade_fwd(const adms_stage_mesh* m, const adms_view* views, int32_t n_views, int32_t H, int32_t W,
                           const uint64_t* keys, const float* rast, const float* rast_db, const float* vpos4,
                           const float* vnrm4, const float* vtan4, const adms_stage_texture* maps, float* pre,
                           void* cuda_stream) {
    ShadeArgs a;
    adms_status s = shade_stage_args(m, views, n_views, H, W, keys, rast, rast_db, vpos4, vnrm4, vtan4, maps, a);
    if (s) return s;
    if (!pre) return ADMS_ERR_ARG;
    a.pre = reinterpret_cast<float4*>(pre);
    k_stage_shade_fwd<<<pix_grid(n_views, H, W), 256, 0, (cudaStream_t)cuda_stream>>>(
        a, reinterpret_cast<const float2*>(rast), reinterpret_cast<const float4*>(rast_db));
    count_launches(1);
    ADMS_STAGE_CHECK(cudaGetLastError());
    return ADMS_OK;
}

adms_status adms_shade_bwd(const adms_stage_mesh* m, const adms_view* views, int32_t n_views, int32_t H, int32_t W,
                           const uint64_t* keys, const float* rast, const float* rast_db, const float* vpos4,
                           const float* vnrm4, const float* vtan4, const adms_stage_texture* maps, const float* g_pre,
                           double* g_vpos, double* g_vnrm, double* g_vtan, float* g_rast, void* cuda_stream) {
    ShadeArgs a;
    adms_status s = shade_stage_args(m, views, n_views, H, W, keys, rast, rast_db, vpos4, vnrm4, vtan4, maps, a);
    if (s) return s;
    if (!g_pre || !g_vpos || !g_vnrm || !g_vtan || !g_rast) return ADMS_ERR_ARG;
    a.g_pos = g_vpos;
    a.g_nrm = g_vnrm;
    a.g_tan = g_vtan;
    k_stage_shade_bwd<<<pix_grid(n_views, H, W), 256, 0, (cudaStream_t)cuda_stream>>>(
        a, reinterpret_cast<const float2*>(rast), reinterpret_cast<const float4*>(rast_db),
        reinterpret_cast<const float4*>(g_pre), reinterpret_cast<float2*>(g_rast));
    count_launches(1);
    ADMS_STAGE_CHECK(cudaGetLastError());
    return ADMS_OK;
}

adms_status adms_aa_loss_fwd(const adms_stage_mesh* m, const adms_view* views, int32_t n_views, int32_t H, int32_t W,
                             const float* clip, const uint64_t* keys, const float* pre, const float* ref,
                             int32_t loss_kind, float loss_scale, float* img, double* loss, float* gprime, void* work,
                             size_t work_bytes, void* cuda_stream) {
    if (!sizes_ok(m, n_views, H, W) || !views || !clip || !keys || !pre || loss_kind < ADMS_LOSS_L1 ||
        loss_kind > ADMS_LOSS_L2 || (ref && (!loss || !gprime)) || (!ref && !img))
        return ADMS_ERR_ARG;
    StageWork w;
    if (!work_of(work, work_bytes, m->n_verts, m->n_tris, n_views, H, W, w)) return ADMS_ERR_ARG;
    ShadeArgs a = stage_args(m, views, n_views, H, W);
    a.clip = reinterpret_cast<const float4*>(clip);
    a.scr = w.s.scr;
    a.silmask = w.s.silmask;
    a.keys = reinterpret_cast<const unsigned long long*>(keys);
    a.pre = reinterpret_cast<float4*>(const_cast<float*>(pre));
    a.ref = ref;
    a.loss_kind = loss_kind;
    a.loss_scale = loss_scale;
    a.loss_acc = ref ? loss : nullptr;
    a.gprime = reinterpret_cast<float4*>(gprime);
    a.out_img = img;
    ADMS_STAGE_CHECK(aa_loss_forward(a, (cudaStream_t)cuda_stream));
    return ADMS_OK;
}

adms_status adms_aa_loss_bwd(const adms_stage_mesh* m, const adms_view* views, int32_t n_views, int32_t H, int32_t W,
                             const float* clip, const uint64_t* keys, const float* pre, const float* gprime,
                             const float* g_loss, float* g_pre, double* g_clip, void* work, size_t work_bytes,
                             void* cuda_stream) {
    if (!sizes_ok(m, n_views, H, W) || !views || !clip || !keys || !pre || !gprime || !g_pre || !g_clip)
        return ADMS_ERR_ARG;
    StageWork w;
    if (!work_of(work, work_bytes, m->n_verts, m->n_tris, n_views, H, W, w)) return ADMS_ERR_ARG;
    ShadeArgs a = stage_args(m, views, n_views, H, W);
    a.clip = reinterpret_cast<const float4*>(clip);
    a.scr = w.s.scr;
    a.silmask = w.s.silmask;
    a.keys = reinterpret_cast<const unsigned long long*>(keys);
    a.pre = reinterpret_cast<float4*>(const_cast<float*>(pre));
    a.gprime = reinterpret_cast<float4*>(const_cast<float*>(gprime));
    a.g_clip = g_clip;
    k_stage_aa_bwd<<<pix_grid(n_views, H, W), 256, 0, (cudaStream_t)cuda_stream>>>(a, g_loss,
                                                                                   reinterpret_cast<float4*>(g_pre));
    count_launches(1);
    ADMS_STAGE_CHECK(cudaGetLastError());
    return ADMS_OK;
}

static bool tess_ok(const adms_tess_desc* t, const float* base_pos, const float* disp, int32_t dh, int32_t dw) {
    auto pow2 = [](int x) { return x > 0 && (x & (x - 1)) == 0; };
    return t && t->base_tri && t->bvf_off && t->bvf_face && t->owner && t->wts && t->vert_uv && base_pos && disp &&
           t->n_base_verts > 0 && t->n_base_tris > 0 && t->n_verts > 0 && t->n_segments >= 2 && pow2(dh) && pow2(dw);
}

static TessArgs tess_stage_args(const adms_tess_desc* t, const float* base_pos, const float* disp, int32_t dh,
                                int32_t dw) {
    TessArgs a{};
    a.Vb = t->n_base_verts;
    a.Fb = t->n_base_tris;
    a.Vt = t->n_verts;
    a.n_seg = t->n_segments;
    a.base_pos = base_pos;
    a.base_tri = t->base_tri;
    a.bvf_off = t->bvf_off;
    a.bvf_face = t->bvf_face;
    a.owner = t->owner;
    a.wts = t->wts;
    a.vert_uv = reinterpret_cast<const float2*>(t->vert_uv);
    a.disp = disp;
    a.dh = dh;
    a.dw = dw;
    return a;
}

adms_status adms_tess_fwd(const adms_tess_desc* t, const float* base_pos, const float* disp, int32_t dh, int32_t dw,
                          float* base_nrm, float* pos, void* cuda_stream) {
    if (!tess_ok(t, base_pos, disp, dh, dw) || !base_nrm || !pos) return ADMS_ERR_ARG;
    TessArgs a = tess_stage_args(t, base_pos, disp, dh, dw);
    a.base_nrm = base_nrm;
    a.pos_out = pos;
    ADMS_STAGE_CHECK(tess_forward(a, (cudaStream_t)cuda_stream));
    return ADMS_OK;
}

adms_status adms_tess_bwd(const adms_tess_desc* t, const float* base_pos, const float* base_nrm, const float* disp,
                          int32_t dh, int32_t dw, const float* g_pos, double* g_base_pos, double* g_base_nrm,
                          float* g_disp, void* cuda_stream) {
    if (!tess_ok(t, base_pos, disp, dh, dw) || !base_nrm || !g_pos || !g_base_pos || !g_base_nrm) return ADMS_ERR_ARG;
    TessArgs a = tess_stage_args(t, base_pos, disp, dh, dw);
    a.base_nrm = const_cast<float*>(base_nrm);
    a.g_pos_t = g_pos;
    a.g_base_pos = g_base_pos;
    a.g_base_nrm = g_base_nrm;
    a.g_disp = g_disp;
    ADMS_STAGE_CHECK(tess_backward(a, (cudaStream_t)cuda_stream));
    return ADMS_OK;
}

adms_status adms_mip_fwd(float* chain, int32_t h, int32_t w, int32_t levels, void* cuda_stream) {
    adms_stage_texture t{chain, nullptr, h, w, levels};
    if (!tex_ok(t)) return ADMS_ERR_ARG;
    ADMS_STAGE_CHECK(mip_build(tex_dev(t), (cudaStream_t)cuda_stream));
    return ADMS_OK;
}

adms_status adms_mip_bwd(const float* g_chain, int32_t h, int32_t w, int32_t levels, float* g_level0,
                         void* cuda_stream) {
    adms_stage_texture t{g_chain, nullptr, h, w, levels};
    if (!tex_ok(t) || !g_level0) return ADMS_ERR_ARG;
    TexDev d = tex_dev(t);
    d.grad = reinterpret_cast<float4*>(const_cast<float*>(g_chain));
    ADMS_STAGE_CHECK(fold_mip_gradient(d, reinterpret_cast<float4*>(g_level0), (cudaStream_t)cuda_stream));
    return ADMS_OK;
}

}  // extern "C"
