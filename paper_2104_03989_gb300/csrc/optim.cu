// Optimizer step (Sec. 5.3): lambda and learning-rate schedules, Adam with
// default parameters fused with the adjoint of the mip chain and the range
// clamps, and the mip rebuild of the updated textures.
#include "kernels.cuh"

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

// Adam + clamps on one level-0 texel whose gradient g already includes the mip adjoint
__device__ __forceinline__ float4 adam_texel(const TexDev& t, float4* __restrict__ m, float4* __restrict__ v, int i,
                                             float4 g, int clamp_kind, float lr, float bc1, float bc2) {
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
    return p;
}

// adam_texel with the texel's latent and moments already loaded
__device__ __forceinline__ float4 adam_texel_v(const TexDev& t, float4* __restrict__ m, float4* __restrict__ v, int i,
                                               float4 g, float4 p, float4 mm, float4 vv, int clamp_kind, float lr,
                                               float bc1, float bc2) {
    p.x = adam1(p.x, g.x, mm.x, vv.x, lr, bc1, bc2);
    p.y = adam1(p.y, g.y, mm.y, vv.y, lr, bc1, bc2);
    p.z = adam1(p.z, g.z, mm.z, vv.z, lr, bc1, bc2);
    p.w = adam1(p.w, g.w, mm.w, vv.w, lr, bc1, bc2);
    p = clamp_texel(p, clamp_kind);
    const_cast<float4*>(t.tex)[i] = p;
    m[i] = mm;
    v[i] = vv;
    t.grad[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    return p;
}

// Adam on one 32x32 texel tile of level 0 per block, for every texture of a
// launch (up to ADMS_ADAM_TEX textures of any jobs, block ranges from tile0),
// then levels 1..5 of that tile built in shared memory from the updated texels
// (2x2 box average, same order of summation as k_mip_level), so level 0 is read
// once for both. The mip adjoint is pushed down the tile's pyramid first; each
// gradient texel of levels 1..5 belongs to one tile, which zeroes it with the
// mip writes at the end (a store right after each push-down read held the
// reads back: Adam took 0.23 instead of 0.11 ms per step). All of a tile's reads
// are issued before its first barrier (one memory round trip instead of one per
// pyramid level). The last tile of a texture to finish (a counter per texture)
// builds levels 6.. from level 5, zeroes their gradients and resets the counter.
// resident blocks per SM of the tiled Adam (register cap 65536 / (256 x this)): the
// thread keeps its 16 level-0 loads in flight at once
#ifndef ADMS_ADAM_BLOCKS
#define ADMS_ADAM_BLOCKS 3
#endif
__global__ void __launch_bounds__(256, ADMS_ADAM_BLOCKS) k_adam_tex_batch(const TexAdamBatch P) {
    __shared__ float4 tile[32][32];
    // push level k (k = 1..5): first the raw level-k gradient texels of this tile, then
    // in place sum_{j >= k} weight_j * grad_j at those texels
    __shared__ float4 push[256 + 64 + 16 + 4 + 1];
    __shared__ float4 anc[ADMS_MAX_LEVELS];  // gradients of the tile's ancestors at levels 6..
    __shared__ int s_last;
    const int poff[6] = {0, 0, 256, 320, 336, 340};
    int lo = 0, hi = P.n - 1;  // the texture: last entry with tile0 <= blockIdx.x
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (P.a[mid].tile0 <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const TexAdam& A = P.a[lo];
    if (A.js->status) return;  // every tile of a latched job's texture leaves (its tile counter stays 0)
    const TexDev& t = A.t;
    int tb = (int)blockIdx.x - A.tile0;
    int tiles_x = t.w0 >> 5, n_tiles = tiles_x * (t.h0 >> 5);
    int bx = tb % tiles_x, by = tb / tiles_x;
    int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    float lr = A.js->lr, bc1 = A.js->bc1, bc2 = A.js->bc2;
    // every global read of the tile issued up front: the thread's four level-0 texels
    // (gradient, latent, moments) and the raw gradients of the tile's pyramid and
    // ancestors, so that one memory round trip covers them all
    float4 g0[4], p0[4], m0[4], v0[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        int i = ((by << 5) + ty + 8 * r) * t.w0 + (bx << 5) + tx;
        g0[r] = t.grad[i];
        p0[r] = t.tex[i];
        m0[r] = A.m[i];
        v0[r] = A.v[i];
    }
#pragma unroll
    for (int k = 1; k <= 5; ++k) {
        int n = 32 >> k, wk = t.w0 >> k;
        for (int idx = threadIdx.x; idx < n * n; idx += 256)
            push[poff[k] + idx] = t.grad[t.off[k] + (((by << 5) >> k) + idx / n) * wk + ((bx << 5) >> k) + idx % n];
    }
    {
        int k = threadIdx.x;
        if (k >= 6 && k < t.levels)
            anc[k] = t.grad[t.off[k] + ((by << 5) >> k) * max(t.w0 >> k, 1) + ((bx << 5) >> k)];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int k = 6; k < t.levels; ++k) c = f4madd(c, level_weight(t, k), anc[k]);
        push[poff[5]] = f4madd(c, level_weight(t, 5), push[poff[5]]);
    }
    for (int k = 4; k >= 1; --k) {
        __syncthreads();
        int n = 32 >> k;
        float wl = level_weight(t, k);
        for (int idx = threadIdx.x; idx < n * n; idx += 256) {
            int cx = idx % n, cy = idx / n;
            push[poff[k] + idx] = f4madd(push[poff[k + 1] + (cy >> 1) * (n >> 1) + (cx >> 1)], wl, push[poff[k] + idx]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        int lx = tx, ly = ty + 8 * r;
        int i = ((by << 5) + ly) * t.w0 + (bx << 5) + lx;
        float4 g = f4madd(g0[r], 1.f, push[(ly >> 1) * 16 + (lx >> 1)]);
        latch_nonfinite(A.js, g.x, g.y, g.z, g.w);
        tile[ly][lx] = adam_texel_v(t, A.m, A.v, i, g, p0[r], m0[r], v0[r], A.clamp_kind, lr, bc1, bc2);
    }
    int top = min(5, t.levels - 1);
    float4* tex = const_cast<float4*>(t.tex);
    for (int k = 1; k <= top; ++k) {
        int n = 32 >> k;
        __syncthreads();
        float4 acc;
        int cx = 0, cy = 0;
        bool act = (int)threadIdx.x < n * n;
        if (act) {
            cx = threadIdx.x % n;
            cy = threadIdx.x / n;
            acc = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) acc = f4madd(acc, 1.f, tile[2 * cy + dy][2 * cx + dx]);
            acc = f4scale(acc, 0.25f);
        }
        __syncthreads();
        if (act) {
            tile[cy][cx] = acc;
            int o = t.off[k] + (by * n + cy) * (t.w0 >> k) + bx * n + cx;
            tex[o] = acc;
            t.grad[o] = make_float4(0.f, 0.f, 0.f, 0.f);  // read in the push-down above
        }
    }
    if (t.levels <= 6) return;
    // the last tile of this texture builds levels 6..
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(A.done, 1) == n_tiles - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int k = 6; k < t.levels; ++k) {
        int ws = max(t.w0 >> (k - 1), 1), hs = max(t.h0 >> (k - 1), 1);
        int wd = max(t.w0 >> k, 1), hd = max(t.h0 >> k, 1);
        int sx = ws > 1 ? 2 : 1, sy = hs > 1 ? 2 : 1;
        for (int i = threadIdx.x; i < wd * hd; i += blockDim.x) {
            int x = i % wd, y = i / wd;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int dy = 0; dy < sy; ++dy)
                for (int dx = 0; dx < sx; ++dx)
                    acc = f4madd(acc, 1.f, __ldcg(tex + t.off[k - 1] + (y * sy + dy) * ws + (x * sx + dx)));
            tex[t.off[k] + i] = f4scale(acc, 1.f / (float)(sx * sy));
            t.grad[t.off[k] + i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *A.done = 0;
}

bool adam_tiled(const TexDev& t) { return t.levels > 5 && (t.w0 % 32) == 0 && (t.h0 % 32) == 0; }

cudaError_t adam_textures_tiled(std::vector<TexAdam>& list, cudaStream_t st) {
    TexAdamBatch P;
    for (size_t e0 = 0; e0 < list.size(); e0 += ADMS_ADAM_TEX) {
        size_t e1 = std::min(list.size(), e0 + ADMS_ADAM_TEX);
        int blocks = 0;
        for (size_t e = e0; e < e1; ++e) {
            P.a[e - e0] = list[e];
            P.a[e - e0].tile0 = blocks;
            blocks += (list[e].t.w0 >> 5) * (list[e].t.h0 >> 5);
        }
        P.n = (int)(e1 - e0);
        k_adam_tex_batch<<<blocks, 256, 0, st>>>(P);
        count_launches(1);
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
