// Optimizer step (Sec. 5.3): lambda and learning-rate schedules, Adam with
// default parameters fused with the adjoint of the mip chain and the range
// clamps, and the mip rebuild of the updated textures.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "kernels.cuh"
#include "bulk.cuh"

namespace adms {

constexpr float kLog2_10 = 3.32192809488736234787f;

// lambda_t (Eq. 5 text, recursive reading), lambda_0 heuristic, lr_t, bias corrections
__global__ void k_schedule(SchedArgs a) {
    JobState* s = a.st;
    int t = s->t;
    double l_img = s->img_loss;
    double l_lap = a.has_pos ? s->lap_sum / (double)a.n_verts : 0.0;
    if (a.has_pos) {
        if (t == 0) {
            double lam0 = a.lambda0_user;
            if (!(lam0 > 0.0)) {
                if (l_lap > 0.0) {
                    lam0 = 0.25 * l_img / l_lap;
                } else {
                    lam0 = 0.0;
                    s->status = ADMS_ERR_ARG;
                }
            }
            s->lam0 = (float)lam0;
            s->lam = (float)lam0;
        } else {
            double lmin = 0.02 * (double)s->lam0;
            s->lam = (float)(((double)s->lam - lmin) * (double)exp2f(-1e-6f * kLog2_10 * (float)t) + lmin);
        }
    }
    // float32 transcendentals: float64 ones cost ~10 us on one thread here; the
    // results are float32 and within a few ulp of the float64 values
    s->lr = a.lr0 * exp2f(-0.0002f * kLog2_10 * (float)t);
    s->bc1 = -expm1f((float)(t + 1) * log1pf(-0.1f));   // 1 - 0.9^(t+1)
    s->bc2 = -expm1f((float)(t + 1) * log1pf(-0.001f)); // 1 - 0.999^(t+1)
    s->last_img_loss = (float)l_img;
    s->last_lap = (float)l_lap;
    s->img_loss = 0.0;
}

cudaError_t schedule_step(const SchedArgs& a, cudaStream_t st) {
    k_schedule<<<1, 1, 0, st>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

__global__ void k_advance(JobState* s) {
    s->t += 1;
    if (s->status_next) s->status = s->status_next;
}

__global__ void k_finish_call(JobState* s, float* out) {
    if (out) *out = (float)s->call_loss;
    s->img_loss += s->call_loss;
    if (!isfinite(s->call_loss)) s->status = ADMS_ERR_NONFINITE;  // latched: the optimizer skips the job
}

struct StatusPtrs {
    JobState* p[ADMS_STATUS_MAX];
};
__global__ void k_gather_status(const StatusPtrs P, int n, int* out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = P.p[k]->status;
}
cudaError_t gather_status(JobState* const* js, int n, int* out, cudaStream_t st) {
    if (n <= 0 || n > ADMS_STATUS_MAX) return cudaErrorInvalidValue;
    StatusPtrs P;
    for (int k = 0; k < n; ++k) P.p[k] = js[k];
    k_gather_status<<<(n + 127) / 128, 128, 0, st>>>(P, n, out);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t finish_call_loss(JobState* js, float* out, cudaStream_t st) {
    k_finish_call<<<1, 1, 0, st>>>(js, out);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t advance_step(JobState* js, cudaStream_t st) {
    k_advance<<<1, 1, 0, st>>>(js);
    count_launches(1);
    return cudaGetLastError();
}

// One Adam update. A job whose status is latched (a non-finite loss or gradient
// was seen) is skipped whole by its kernels; a non-finite gradient element met
// here (one the earlier checks missed) leaves its latent and moments unchanged
// and latches status_next (status itself stays constant while the step's
// kernels run, so every tile of a texture takes the same branch), so no NaN or
// infinity is ever written into a latent.
__device__ __forceinline__ float adam1(float p, float g, float& m, float& v, float lr, float bc1, float bc2) {
    bool ok = isfinite(g);
    float m1 = 0.9f * m + 0.1f * g;
    float v1 = 0.999f * v + 0.001f * g * g;
    float mh = m1 / bc1, vh = v1 / bc2;
    float p1 = p - lr * mh / (sqrtf(vh) + 1e-8f);
    m = ok ? m1 : m;
    v = ok ? v1 : v;
    return ok ? p1 : p;
}
__device__ __forceinline__ void latch_nonfinite(const JobState* js, float a, float b = 0.f, float c = 0.f,
                                                float d = 0.f) {
    if (!(isfinite(a) && isfinite(b) && isfinite(c) && isfinite(d)))
        atomicExch(&const_cast<JobState*>(js)->status_next, (int)ADMS_ERR_NONFINITE);
}

__global__ void k_adam_flat(float* __restrict__ p, float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                            long long n, const JobState* __restrict__ js, float lr_scale) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || js->status) return;
    float lr = js->lr * lr_scale, bc1 = js->bc1, bc2 = js->bc2;
    float mm = m[i], vv = v[i], gi = g[i];
    latch_nonfinite(js, gi);
    p[i] = adam1(p[i], gi, mm, vv, lr, bc1, bc2);
    m[i] = mm;
    v[i] = vv;
    g[i] = 0.f;
}

cudaError_t adam_flat(float* p, float* g, float* m, float* v, long long n, const JobState* js, cudaStream_t st,
                      float lr_scale) {
    if (n <= 0) return cudaSuccess;
    k_adam_flat<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, g, m, v, n, js, lr_scale);
    count_launches(1);
    return cudaGetLastError();
}

__device__ __forceinline__ float clampf(float x, float lo, float hi) { return fminf(fmaxf(x, lo), hi); }

// range clamps after an update (Sec. 5.3 reading): kd in [0,1]; (gamma, r, m) in
// [0,1] x [0.08,1] x [0,1]; normal xy in [-1,1], z in [0,1]
__device__ __forceinline__ float4 clamp_texel(float4 p, int clamp_kind) {
    if (clamp_kind == 0) {
        p = make_float4(clampf(p.x, 0.f, 1.f), clampf(p.y, 0.f, 1.f), clampf(p.z, 0.f, 1.f), clampf(p.w, 0.f, 1.f));
    } else if (clamp_kind == 1) {
        p.x = clampf(p.x, 0.f, 1.f);
        p.y = clampf(p.y, ADMS_ROUGH_MIN, 1.f);
        p.z = clampf(p.z, 0.f, 1.f);
    } else if (clamp_kind == 2) {
        p.x = clampf(p.x, -1.f, 1.f);
        p.y = clampf(p.y, -1.f, 1.f);
        p.z = clampf(p.z, 0.f, 1.f);
    }
    return p;
}

// Adam on every texel of every level of a texture whose levels are independent
// latents (Sec. 6 prefiltering): each level keeps its own gradient and moments,
// and nothing is folded or rebuilt
__global__ void k_adam_tex_levels(TexDev t, float4* __restrict__ m, float4* __restrict__ v, long long n,
                                  int clamp_kind, const JobState* __restrict__ js) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || js->status) return;
    float lr = js->lr, bc1 = js->bc1, bc2 = js->bc2;
    float4 g = t.grad[i], p = t.tex[i], mm = m[i], vv = v[i];
    latch_nonfinite(js, g.x, g.y, g.z, g.w);
    p.x = adam1(p.x, g.x, mm.x, vv.x, lr, bc1, bc2);
    p.y = adam1(p.y, g.y, mm.y, vv.y, lr, bc1, bc2);
    p.z = adam1(p.z, g.z, mm.z, vv.z, lr, bc1, bc2);
    p.w = adam1(p.w, g.w, mm.w, vv.w, lr, bc1, bc2);
    const_cast<float4*>(t.tex)[i] = clamp_texel(p, clamp_kind);
    m[i] = mm;
    v[i] = vv;
    t.grad[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

cudaError_t adam_texture_levels(const TexDev& t, float4* m, float4* v, int clamp_kind, const JobState* js,
                                cudaStream_t st) {
    long long n = t.off[t.levels - 1] + (long long)max(t.w0 >> (t.levels - 1), 1) * max(t.h0 >> (t.levels - 1), 1);
    k_adam_tex_levels<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(t, m, v, n, clamp_kind, js);
    count_launches(1);
    return cudaGetLastError();
}

__global__ void k_adam_tex(TexDev t, float4* __restrict__ m, float4* __restrict__ v, int clamp_kind,
                           const JobState* __restrict__ js) {
    int n = t.w0 * t.h0;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || js->status) return;
    int x = i % t.w0, y = i / t.w0;
    float4 g = t.grad[i];
    // adjoint of the box-filter chain: level k texel = mean of its children
    float wgt = 1.f;
    for (int k = 1; k < t.levels; ++k) {
        int wp = max(t.w0 >> (k - 1), 1), hp = max(t.h0 >> (k - 1), 1);
        wgt *= 1.f / (float)((wp > 1 ? 2 : 1) * (hp > 1 ? 2 : 1));
        int wk = max(t.w0 >> k, 1);
        float4 gk = t.grad[t.off[k] + (y >> k) * wk + (x >> k)];
        g = f4madd(g, wgt, gk);
    }
    float lr = js->lr, bc1 = js->bc1, bc2 = js->bc2;
    latch_nonfinite(js, g.x, g.y, g.z, g.w);
    float4 p = t.tex[i], mm = m[i], vv = v[i];
    p.x = adam1(p.x, g.x, mm.x, vv.x, lr, bc1, bc2);
    p.y = adam1(p.y, g.y, mm.y, vv.y, lr, bc1, bc2);
    p.z = adam1(p.z, g.z, mm.z, vv.z, lr, bc1, bc2);
    p.w = adam1(p.w, g.w, mm.w, vv.w, lr, bc1, bc2);
    p = clamp_texel(p, clamp_kind);
    const_cast<float4*>(t.tex)[i] = p;
    m[i] = mm;
    v[i] = vv;
    t.grad[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// weight of a level-k texel's gradient in each of its level-0 texels (product of
// the 2x2 / 2x1 box-filter factors down the chain)
__device__ __forceinline__ float level_weight(const TexDev& t, int k) {
    float w = 1.f;
    for (int j = 1; j <= k; ++j) {
        int wp = max(t.w0 >> (j - 1), 1), hp = max(t.h0 >> (j - 1), 1);
        w *= 1.f / (float)((wp > 1 ? 2 : 1) * (hp > 1 ? 2 : 1));
    }
    return w;
}

// Adam on the 32x32 texel tiles of level 0 of every texture of a launch (up to
// ADMS_ADAM_TEX textures of any jobs, tile ranges from tile0), each followed by
// levels 1..5 of its tile from the updated texels (2x2 box average, same order of
// summation as k_mip_level), so level 0 is read once for both.
//
// Streaming: one persistent block per SM walks tiles blockIdx.x, + gridDim.x, ...
// Thread 0 moves a tile's four level-0 arrays (gradient, latent, moments: one
// 32 x 32-texel box of each texture's tensor maps, 16 KB) into one of three
// shared-memory stages with TMA copies completing on that stage's mbarrier, two
// tiles ahead of the arithmetic, and writes the cleared gradient, the updated
// latent and the moments back with TMA stores from shared memory.
//
// Thread t owns the 2x2 level-0 quad under level-1 texel (cx, cy) of the tile,
// t interleaving the bits of cx (even bits) and cy (odd bits): the four children
// of a level-2 texel are lanes 4j..4j+3, those of a level-3 texel lanes 16j + {0,
// 4, 8, 12}, those of a level-4 texel threads 64j + {0, 16, 32, 48}, each time in
// the order (0,0), (1,0), (0,1), (1,1). Levels 1-3 are formed in registers and by
// shuffles, level 4 through shared memory after the tile's one block barrier,
// level 5 by shuffles in warp 0.
//
// The mip adjoint: each level-0 texel receives sum_k w_k g_k over its ancestors
// (w_k = 1/4^k up to level 5, the product of the box factors beyond), formed by
// each thread from its own loads (issued a tile ahead into registers) as
// g0 + ((((c + w5 g5) + w4 g4) + w3 g3) + w2 g2) + w1 g1, c the sum over levels
// 6.. . A gradient texel of levels 1..5 is cleared by its owner after every reader
// in the block has consumed it; k_adam_mip_top, launched after, builds levels 6..
// and clears their gradients.
struct AdamStage {
    float4 g[32][32], p[32][32], m[32][32], v[32][32];
};
// shared-memory stages of the streamed Adam (tiles in flight: the one being updated and
// STAGES - 1 fetched ahead), whether a tile's fetch is issued before (EARLY) or after the
// arithmetic of the tile STAGES - 1 ahead of it, and the resident blocks per SM the
// register allocation must allow
#ifndef ADMS_ADAM_STAGES
#define ADMS_ADAM_STAGES 3
#endif
#ifndef ADMS_ADAM_EARLY_FETCH
#define ADMS_ADAM_EARLY_FETCH 0
#endif
#ifndef ADMS_ADAM_MIN_BLOCKS
#define ADMS_ADAM_MIN_BLOCKS 1
#endif
static_assert(ADMS_ADAM_STAGES == 2 || ADMS_ADAM_STAGES == 3, "two or three Adam stages");
#define ADMS_ADAM_THREADS 256
struct AdamSmem {
    AdamStage st[ADMS_ADAM_STAGES];
    float4 s3[2][16];  // a tile's level-3 texels in thread (interleaved-bit) order, by tile parity
    uint64_t bar[ADMS_ADAM_STAGES];
};
#define ADMS_ADAM_WAIT_NS 2000000000ull  // a tile's wait gives up after 2 s
// persistent blocks of the streamed Adam, in percent of the SMs (one block per SM at 100)
#ifndef ADMS_ADAM_GRID_PCT
#define ADMS_ADAM_GRID_PCT 100
#endif

__device__ __forceinline__ int even_bits(int t) {  // bits 0, 2, 4, 6 of t, packed
    return (t & 1) | ((t >> 1) & 2) | ((t >> 2) & 4) | ((t >> 3) & 8);
}
__device__ __forceinline__ float4 quad_mean(float4 a, float4 b, float4 c, float4 d) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    acc = f4madd(acc, 1.f, a);
    acc = f4madd(acc, 1.f, b);
    acc = f4madd(acc, 1.f, c);
    acc = f4madd(acc, 1.f, d);
    return f4scale(acc, 0.25f);
}
__device__ __forceinline__ float4 shfl_down4(float4 v, int d, unsigned mask = 0xffffffffu) {
    return make_float4(__shfl_down_sync(mask, v.x, d), __shfl_down_sync(mask, v.y, d), __shfl_down_sync(mask, v.z, d),
                       __shfl_down_sync(mask, v.w, d));
}
// Adam on four components with the bias corrections as reciprocals and the step's
// division approximate (2 ulp)
__device__ __forceinline__ float4 adam4(float4 p, float4 g, float4& m, float4& v, float lr, float ibc1, float ibc2) {
    float pv[4] = {p.x, p.y, p.z, p.w}, gv[4] = {g.x, g.y, g.z, g.w};
    float mv[4] = {m.x, m.y, m.z, m.w}, vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        bool ok = isfinite(gv[c]);
        float m1 = 0.9f * mv[c] + 0.1f * gv[c];
        float v1 = 0.999f * vv[c] + 0.001f * gv[c] * gv[c];
        float p1 = pv[c] - __fdividef(lr * (m1 * ibc1), sqrtf(v1 * ibc2) + 1e-8f);
        mv[c] = ok ? m1 : mv[c];
        vv[c] = ok ? v1 : vv[c];
        pv[c] = ok ? p1 : pv[c];
    }
    m = make_float4(mv[0], mv[1], mv[2], mv[3]);
    v = make_float4(vv[0], vv[1], vv[2], vv[3]);
    return make_float4(pv[0], pv[1], pv[2], pv[3]);
}
// the texture entry of flattened tile index `tile`: last entry with tile0 <= tile
__device__ __forceinline__ int adam_entry(const TexAdamBatch& P, int tile) {
    int lo = 0, hi = P.n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (P.a[mid].tile0 <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ void adam_tile_xy(const TexAdam& A, int tile, int& bx, int& by) {
    int tb = tile - A.tile0, tiles_x = A.t.w0 >> 5;
    bx = tb % tiles_x;
    by = tb / tiles_x;
}
// one thread: the tile's four level-0 arrays into stage S (four boxes of the
// texture's tensor maps), completing on bar
__device__ __forceinline__ void adam_fetch(const TexAdamBatch& P, int tile, AdamStage& S, uint64_t* bar) {
    int e = adam_entry(P, tile);
    int bx, by;
    adam_tile_xy(P.a[e], tile, bx, by);
    const CUtensorMap* tm = P.maps[e];
    if (bx < 0 || by < 0 || 32 * bx >= P.a[e].t.w0 || 32 * by >= P.a[e].t.h0) {
        // never taken for a launcher-built batch: record it and complete the phase without copies
        atomicExch(&const_cast<JobState*>(P.a[e].js)->status_next, (int)ADMS_ERR_STATE);
        mbar_arrive_expect_tx(bar, 0);
        return;
    }
    mbar_arrive_expect_tx(bar, (uint32_t)sizeof(AdamStage) + P.extra_tx);
    tile2d_g2s(&S.g[0][0], &tm[0], bx * 128, by * 32, bar);
    tile2d_g2s(&S.p[0][0], &tm[1], bx * 128, by * 32, bar);
    tile2d_g2s(&S.m[0][0], &tm[2], bx * 128, by * 32, bar);
    tile2d_g2s(&S.v[0][0], &tm[3], bx * 128, by * 32, bar);
}

// the pyramid gradients of levels 1..5 above level-0 texel (x, y) of `tile` (and
// its quad) into
// g[1..5] and the tile's ancestors' gradients (levels 6..) into anc[0..]: a tile's
// loads, issued a tile ahead into registers (the ancestors are the same address
// for every thread of the block: broadcast loads)
#define ADMS_ADAM_ANC (ADMS_MAX_LEVELS - 6)
__device__ __forceinline__ void adam_pyramid(const TexAdamBatch& P, int tile, int x, int y, float4 g[6],
                                             float4 anc[ADMS_ADAM_ANC]) {
    const TexAdam& A = P.a[adam_entry(P, tile)];
    if (A.js->status) return;
    const TexDev& t = A.t;
    int bx, by;
    adam_tile_xy(A, tile, bx, by);
#pragma unroll
    for (int l = 1; l <= 5; ++l)
        g[l] = t.grad[t.off[l] + (((by << 5) + y) >> l) * (t.w0 >> l) + (((bx << 5) + x) >> l)];
#pragma unroll
    for (int i = 0; i < ADMS_ADAM_ANC; ++i) {
        int l = 6 + i;
        if (l < t.levels) anc[i] = t.grad[t.off[l] + ((by << 5) >> l) * max(t.w0 >> l, 1) + ((bx << 5) >> l)];
    }
}

// tid 0, during tile k (index `tile`): fetch the tile STAGES - 1 ahead into the stage
// that tile k - 1 used, once tile k - 1's stores have read it; *fetched: the highest
// tile ordinal fetched so far
__device__ __forceinline__ void adam_fetch_ahead(const TexAdamBatch& P, AdamSmem& S, int tile, int k, int total,
                                                 int* fetched) {
    int ahead = tile + (ADMS_ADAM_STAGES - 1) * (int)gridDim.x;
    if (ahead >= total) return;
    int sa = (k + ADMS_ADAM_STAGES - 1) % ADMS_ADAM_STAGES;
    bulk_wait_read0();
    adam_fetch(P, ahead, S.st[sa], &S.bar[sa]);
    *fetched = k + ADMS_ADAM_STAGES - 1;
}

__global__ void __launch_bounds__(ADMS_ADAM_THREADS, ADMS_ADAM_MIN_BLOCKS)
    k_adam_tex_stream(const __grid_constant__ TexAdamBatch P, int total) {
    extern __shared__ __align__(128) unsigned char adam_raw[];
    AdamSmem& S = *reinterpret_cast<AdamSmem*>(adam_raw);
    int tid = threadIdx.x, lane = tid & 31;
    if (smem_u32(adam_raw) & 127u) {  // the TMA boxes need 128-byte-aligned stages
        if (tid == 0) atomicExch(&const_cast<JobState*>(P.a[0].js)->status_next, (int)ADMS_ERR_STATE);
        return;
    }
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    if (tid == 0) {
        for (int q = 0; q < ADMS_ADAM_STAGES; ++q) mbar_init(&S.bar[q], 1);
        fence_barrier_init();
    }
    __syncthreads();
    // tile j of this block (tile blockIdx.x + j gridDim.x) goes through stage j % STAGES,
    // whose (j / STAGES)-th phase its copies complete; tiles 0 .. STAGES - 2 are fetched
    // here, tile j + STAGES - 1 during tile j, once tile j - 1's stores (same stage) have
    // read it
    int tile = blockIdx.x;
    int fetched = -1;  // tid 0: the highest tile ordinal whose copies were issued
    if (tid == 0)
        for (int j = 0; j < ADMS_ADAM_STAGES - 1; ++j)
            if (tile + j * (int)gridDim.x < total) {
                adam_fetch(P, tile + j * gridDim.x, S.st[j], &S.bar[j]);
                fetched = j;
            }
    // the thread's quad: level-0 texels (x, y) .. (x + 1, y + 1) of the tile
    int cx = even_bits(tid), cy = even_bits(tid >> 1);  // its level-1 texel
    int x = 2 * cx, y = 2 * cy;
    float4 gk[6], anc[ADMS_ADAM_ANC];
    if (tile < total) adam_pyramid(P, tile, x, y, gk, anc);
    int k = 0;
    for (; tile < total; tile += gridDim.x, ++k) {
        int s = k % ADMS_ADAM_STAGES;
        int ent = adam_entry(P, tile);
        const TexAdam& A = P.a[ent];
        const TexDev& t = A.t;
        int bx, by;
        adam_tile_xy(A, tile, bx, by);
        bool live = A.js->status == 0;  // a latched job's tiles change nothing
        float4* grad = t.grad;
        float4* tex = const_cast<float4*>(t.tex);
        // one block barrier per tile: each thread waits for the stage itself; the
        // barrier after the arithmetic orders its shared-memory writes before the
        // stores, and the shared array a tile writes alternates with the tile's parity
        // (agreed per warp: the shuffles below need every lane)
        bool ok = __all_sync(0xffffffffu, mbar_wait(&S.bar[s], (uint32_t)(k / ADMS_ADAM_STAGES) & 1u, ADMS_ADAM_WAIT_NS));
        AdamStage& T = S.st[s];
#if ADMS_ADAM_EARLY_FETCH
        if (tid == 0 && ok) adam_fetch_ahead(P, S, tile, k, total, &fetched);
#endif
        if (live && ok) {
            float4 c = zero;
            float w = 1.f / 1024.f;  // 1/4^5
#pragma unroll
            for (int i = 0; i < ADMS_ADAM_ANC; ++i) {
                int l = 6 + i;
                if (l < t.levels) {
                    int wp = max(t.w0 >> (l - 1), 1), hp = max(t.h0 >> (l - 1), 1);
                    w *= 1.f / (float)((wp > 1 ? 2 : 1) * (hp > 1 ? 2 : 1));
                    c = f4madd(c, w, anc[i]);
                }
            }
            float4 push = f4madd(c, 1.f / 1024.f, gk[5]);
            push = f4madd(push, 1.f / 256.f, gk[4]);
            push = f4madd(push, 1.f / 64.f, gk[3]);
            push = f4madd(push, 1.f / 16.f, gk[2]);
            push = f4madd(push, 0.25f, gk[1]);
            float lr = A.js->lr, ibc1 = 1.f / A.js->bc1, ibc2 = 1.f / A.js->bc2;
            float4 pq[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int qx = x + (q & 1), qy = y + (q >> 1);
                float4 g = f4madd(T.g[qy][qx], 1.f, push);
                latch_nonfinite(A.js, g.x, g.y, g.z, g.w);
                float4 mm = T.m[qy][qx], vv = T.v[qy][qx];
                pq[q] = clamp_texel(adam4(T.p[qy][qx], g, mm, vv, lr, ibc1, ibc2), A.clamp_kind);
                T.p[qy][qx] = pq[q];
                T.m[qy][qx] = mm;
                T.v[qy][qx] = vv;
                T.g[qy][qx] = zero;  // stored back: the cleared gradient
            }
            // level 1: the thread's own quad; levels 2 and 3: lanes 4j and 16j gather by shuffles
            float4 l = quad_mean(pq[0], pq[1], pq[2], pq[3]);
            {
                int o = t.off[1] + ((by << 4) + cy) * (t.w0 >> 1) + (bx << 4) + cx;
                tex[o] = l;
                grad[o] = zero;
            }
#pragma unroll
            for (int lv = 2; lv <= 3; ++lv) {
                int d = lv == 2 ? 1 : 4;  // lane distance of the x neighbour
                float4 a1 = shfl_down4(l, d), a2 = shfl_down4(l, 2 * d), a3 = shfl_down4(l, 3 * d);
                l = quad_mean(l, a1, a2, a3);
                if ((lane & (4 * d - 1)) == 0) {
                    int n = 32 >> lv;
                    int o = t.off[lv] + (by * n + (y >> lv)) * (t.w0 >> lv) + bx * n + (x >> lv);
                    tex[o] = l;
                    grad[o] = zero;
                }
            }
            if ((lane & 15) == 0) S.s3[k & 1][tid >> 4] = l;
        }
        if (tile + (int)gridDim.x < total) adam_pyramid(P, tile + gridDim.x, x, y, gk, anc);
        fence_proxy_async();  // the stage's updated rows, before the stores read them
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(&const_cast<JobState*>(A.js)->status_next, (int)ADMS_ERR_TIMEOUT);
            break;
        }
#if !ADMS_ADAM_EARLY_FETCH
        if (tid == 0) adam_fetch_ahead(P, S, tile, k, total, &fetched);
#endif
        if (live) {
            if (tid == 0) {
                const CUtensorMap* tm = P.maps[ent];
                tile2d_s2g(&tm[0], bx * 128, by * 32, &T.g[0][0]);
                tile2d_s2g(&tm[1], bx * 128, by * 32, &T.p[0][0]);
                tile2d_s2g(&tm[2], bx * 128, by * 32, &T.m[0][0]);
                tile2d_s2g(&tm[3], bx * 128, by * 32, &T.v[0][0]);
                bulk_commit();
            }
            // level 4 in threads 0..3 (texel (q & 1, q >> 1)), level 5 in thread 0
            if (tid < 4) {
                const float4* s3 = S.s3[k & 1];
                float4 l4 = quad_mean(s3[4 * tid], s3[4 * tid + 1], s3[4 * tid + 2], s3[4 * tid + 3]);
                int o = t.off[4] + (by * 2 + (tid >> 1)) * (t.w0 >> 4) + bx * 2 + (tid & 1);
                tex[o] = l4;
                grad[o] = zero;
                float4 a1 = shfl_down4(l4, 1, 0xfu), a2 = shfl_down4(l4, 2, 0xfu), a3 = shfl_down4(l4, 3, 0xfu);
                if (tid == 0) {
                    int o5 = t.off[5] + by * (t.w0 >> 5) + bx;
                    tex[o5] = quad_mean(l4, a1, a2, a3);
                    grad[o5] = zero;
                }
            }
        }
    }
    if (tid == 0 && tile < total) {
        // gave up on tile k's wait: let the copies issued for later tiles land before the
        // block's memory is released
        for (int q = k + 1; q <= fetched; ++q)
            mbar_wait(&S.bar[q % ADMS_ADAM_STAGES], (uint32_t)(q / ADMS_ADAM_STAGES) & 1u, ADMS_ADAM_WAIT_NS);
    }
    if (tid == 0) bulk_wait0();
}

// Levels 6.. of every texture of a streamed-Adam launch, one block per texture,
// from the level 5 that the tiles wrote (2x2 box average, same order as
// k_mip_level); their gradients, read by every tile above, are cleared here.
__global__ void k_adam_mip_top(const __grid_constant__ TexAdamBatch P) {
    const TexAdam& A = P.a[blockIdx.x];
    if (A.js->status) return;
    const TexDev& t = A.t;
    float4* tex = const_cast<float4*>(t.tex);
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int lv = 6; lv < t.levels; ++lv) {
        int ws = max(t.w0 >> (lv - 1), 1), hs = max(t.h0 >> (lv - 1), 1);
        int wd = max(t.w0 >> lv, 1), hd = max(t.h0 >> lv, 1);
        int sx = ws > 1 ? 2 : 1, sy = hs > 1 ? 2 : 1;
        for (int i = threadIdx.x; i < wd * hd; i += blockDim.x) {
            int x = i % wd, y = i / wd;
            float4 acc = zero;
            for (int dy = 0; dy < sy; ++dy)
                for (int dx = 0; dx < sx; ++dx) acc = f4madd(acc, 1.f, tex[t.off[lv - 1] + (y * sy + dy) * ws + (x * sx + dx)]);
            tex[t.off[lv] + i] = f4scale(acc, 1.f / (float)(sx * sy));
            t.grad[t.off[lv] + i] = zero;
        }
        __syncthreads();
    }
}

bool adam_tiled(const TexDev& t) { return t.levels > 5 && (t.w0 % 32) == 0 && (t.h0 % 32) == 0; }

cudaError_t adam_prepare() {
    return cudaFuncSetAttribute(k_adam_tex_stream, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(AdamSmem));
}

cudaError_t adam_encode_maps(const TexDev& t, const float4* m, const float4* v, CUtensorMap out[4]) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const void* base[4] = {t.grad, t.tex, m, v};
    cuuint64_t dim[2] = {(cuuint64_t)4 * t.w0, (cuuint64_t)t.h0};
    cuuint64_t stride[1] = {(cuuint64_t)t.w0 * sizeof(float4)};
    cuuint32_t box[2] = {128, 32}, estride[2] = {1, 1};
    for (int k = 0; k < 4; ++k) {
        CUresult r = encode(&out[k],
                            CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base[k]), dim, stride, box, estride,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

cudaError_t adam_textures_tiled(std::vector<TexAdam>& list, cudaStream_t st, uint32_t extra_tx) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (!e) e = adam_prepare();
        if (e) {
            sms = 0;
            return e;
        }
    }
    thread_local TexAdamBatch P;  // 26 KB of kernel parameters: not on the host stack
    for (size_t e0 = 0; e0 < list.size(); e0 += ADMS_ADAM_TEX) {
        size_t e1 = std::min(list.size(), e0 + ADMS_ADAM_TEX);
        int tiles = 0;
        for (size_t e = e0; e < e1; ++e) {
            P.a[e - e0] = list[e];
            P.a[e - e0].tile0 = tiles;
            for (int k = 0; k < 4; ++k) P.maps[e - e0][k] = list[e].tmaps[k];
            tiles += (list[e].t.w0 >> 5) * (list[e].t.h0 >> 5);
        }
        P.n = (int)(e1 - e0);
        P.extra_tx = extra_tx;
        int blocks = std::min(tiles, std::max(1, sms * ADMS_ADAM_GRID_PCT / 100));
        k_adam_tex_stream<<<blocks, ADMS_ADAM_THREADS, sizeof(AdamSmem), st>>>(P, tiles);
        k_adam_mip_top<<<P.n, 256, 0, st>>>(P);
        count_launches(2);
        cudaError_t e = cudaGetLastError();
        if (e) return e;
    }
    return cudaSuccess;
}

cudaError_t adam_texture_and_mips(const TexDev& t, float4* m, float4* v, int clamp_kind, const JobState* js,
                                  cudaStream_t st) {
    cudaError_t e = adam_texture(t, m, v, clamp_kind, js, st);
    if (e) return e;
    return mip_build(t, st);
}

// level-0 gradient including the adjoint of the mip chain, written to out (no update)
__global__ void k_fold_mips(TexDev t, float4* __restrict__ out) {
    int n = t.w0 * t.h0;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int x = i % t.w0, y = i / t.w0;
    float4 g = t.grad[i];
    for (int k = 1; k < t.levels; ++k) {
        int wk = max(t.w0 >> k, 1);
        g = f4madd(g, level_weight(t, k), t.grad[t.off[k] + (y >> k) * wk + (x >> k)]);
    }
    out[i] = g;
}

cudaError_t fold_mip_gradient(const TexDev& t, float4* out, cudaStream_t st) {
    int n = t.w0 * t.h0;
    k_fold_mips<<<(n + 255) / 256, 256, 0, st>>>(t, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t adam_texture(const TexDev& t, float4* m, float4* v, int clamp_kind, const JobState* js, cudaStream_t st) {
    int n = t.w0 * t.h0;
    k_adam_tex<<<(n + 255) / 256, 256, 0, st>>>(t, m, v, clamp_kind, js);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    if (t.levels > 1) {
        size_t coarse = 0;
        for (int k = 1; k < t.levels; ++k) coarse += (size_t)max(t.w0 >> k, 1) * max(t.h0 >> k, 1);
        e = cudaMemsetAsync(t.grad + t.off[1], 0, coarse * sizeof(float4), st);
    }
    return e;
}

__global__ void k_mip_level(float4* __restrict__ tex, int src_off, int ws, int hs, int dst_off, int wd, int hd) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= wd * hd) return;
    int x = i % wd, y = i / wd;
    int sx = ws > 1 ? 2 : 1, sy = hs > 1 ? 2 : 1;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int dy = 0; dy < sy; ++dy)
        for (int dx = 0; dx < sx; ++dx) acc = f4madd(acc, 1.f, tex[src_off + (y * sy + dy) * ws + (x * sx + dx)]);
    tex[dst_off + i] = f4scale(acc, 1.f / (float)(sx * sy));
}

cudaError_t mip_build(const TexDev& t, cudaStream_t st) {
    for (int k = 1; k < t.levels; ++k) {
        int ws = max(t.w0 >> (k - 1), 1), hs = max(t.h0 >> (k - 1), 1);
        int wd = max(t.w0 >> k, 1), hd = max(t.h0 >> k, 1);
        k_mip_level<<<(wd * hd + 255) / 256, 256, 0, st>>>(const_cast<float4*>(t.tex), t.off[k - 1], ws, hs, t.off[k],
                                                          wd, hd);
        count_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace adms
