// C ABI: contexts, jobs with resident state, and the step calls.
//
// Host-side preprocessing (topology is fixed, Sec. 3): edge adjacency for the
// silhouette test, vertex -> face and one-ring CSR tables, mip-chain layout.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "kernels.cuh"

using namespace adms;

namespace {

struct TexState {
    float4* data = nullptr;  // mip chain
    float4* grad = nullptr;  // mip chain (when optimized)
    float4* m = nullptr;     // level 0
    float4* v = nullptr;
    CUtensorMap tmaps[4];  // tensor maps of level 0 for the tiled Adam (grad, tex, m, v)
    bool per_level = false;  // every level is a latent: m, v span the chain
    int w = 0, h = 0, levels = 0;
    int off[ADMS_MAX_LEVELS] = {0};
    size_t total = 0;
    bool opt = false;

    TexDev dev() const {
        TexDev t;
        t.tex = data;
        t.grad = opt ? grad : nullptr;
        t.w0 = w;
        t.h0 = h;
        t.levels = levels;
        for (int k = 0; k < ADMS_MAX_LEVELS; ++k) t.off[k] = off[k];
        return t;
    }
};

struct Job {
    bool alive = false;
    bool frozen = true;
    adms_opt_params opt{};
    uint64_t seed = 0;
    int V = 0, T = 0, F = 0;  // render mesh (the tessellation for tessellated jobs)
    int LV = 0;               // latent (base) vertices
    // latents and their optimizer state (base positions for tessellated jobs)
    float* pos = nullptr;
    float* g_pos = nullptr;
    float* m_pos = nullptr;
    float* v_pos = nullptr;
    TexState kd, orm, nrm;
    // render-mesh positions and their gradient (alias pos / g_pos without tessellation)
    float* rpos = nullptr;
    float* g_rpos = nullptr;
    // tessellation + displacement (Sec. 5.1)
    bool tess = false;
    int Fb = 0, n_seg = 0, dh = 0, dw = 0;
    int *btri = nullptr, *btri_uv = nullptr, *bvf_off = nullptr, *bvf_face = nullptr, *owner = nullptr, *wts = nullptr;
    float2 *vert_uv = nullptr, *buv = nullptr;
    float* bnrm = nullptr;
    double *g_bnrm = nullptr, *g_btan0 = nullptr, *g_bpos_acc = nullptr;
    float4 *b_vpos = nullptr, *b_vnrm = nullptr, *b_vtan = nullptr, *b_tmp_n = nullptr, *b_tmp_t = nullptr;
    float *disp = nullptr, *g_disp = nullptr, *m_disp = nullptr, *v_disp = nullptr;
    // dense skinning (Eq. 2): render positions = skinned rest positions
    bool skin = false;
    int SB = 0;  // bones
    float *skin_w = nullptr, *g_skin_w = nullptr, *m_skin_w = nullptr, *v_skin_w = nullptr, *bones = nullptr;
    float skin_lr_scale = 0.f;  // the weights' learning rate is lr_t times this (0: frozen)
    // topology
    float2* uv = nullptr;
    int* tri = nullptr;
    int* tri_uv = nullptr;
    int* adj = nullptr;
    int* vf_off = nullptr;
    int* vf_face = nullptr;
    int* ring_off = nullptr;
    int* ring = nullptr;
    float* delta_ref = nullptr;
    // per-step derived state
    float4 *vpos = nullptr, *vnrm = nullptr, *vtan = nullptr, *tmp_n = nullptr, *tmp_t = nullptr;
    float2* frame_inv = nullptr;  // the frame's normalisations (one-launch frame adjoint)
    double *g_nrm = nullptr, *g_tan = nullptr, *g_pos_acc = nullptr;
    float* delta = nullptr;
    JobState* st = nullptr;
    bool frame_valid = false;
    bool lap_valid = false;  // delta and lap_sum hold the Laplacian of the current positions
    // a pipelined context's deferred texture step (the texture latents' Adam updates
    // and the step counter of the last optimizer_step), not yet issued
    bool tex_pending = false;
    // per-call scratch
    size_t px_cap = 0, view_cap = 0, tile_cap = 0, rec_cap = 0;
    unsigned long long* keys = nullptr;
    float4* pre = nullptr;
    float4* gprime = nullptr;
    int* refine = nullptr;
    adms_view* views = nullptr;
    RasterScratch rs{};
    // latest forward
    bool have_fwd = false;
    int B = 0, H = 0, W = 0;  // views and the grid the kernels work on (the sample grid when S > 1)
    // supersampled rendering (Sec. 5.2): S x S samples per pixel; MSAA shades once per
    // pixel (at its centre), ssaa shades every sample; the resolve averages them
    int S = 1;
    bool ssaa = false;
    int PH = 0, PW = 0;        // pixels per view
    float4* acol = nullptr;    // antialiased sample colours (+ blend masks) for the resolve
    // depth-peeled transparency (Sec. 5.2): L layers; keys and pre hold L slices of
    // B H W (front to back), acc the composites A_1 .. A_{L-1} of the layers behind
    // each layer (xyz; w: blend mask bits), gprime2 the second dL/d(composite) buffer
    int L = 0;
    float4* acc = nullptr;
    float4* gprime2 = nullptr;
    const float* ref = nullptr;
    float loss_scale = 0.f;
    std::vector<void*> allocs;
    size_t bytes = 0;
};

}  // namespace

enum Stage {
    ST_FRAME = 0,
    ST_RASTER_SETUP,
    ST_RASTER,
    ST_SHADE,
    ST_AA_LOSS,
    ST_SHADE_BWD,
    ST_FRAME_BWD,
    ST_LAPLACIAN,
    ST_ADAM,
    ST_MIP,
    ST_SMALL,
    ST_COUNT
};
static const char* kStageNames[ST_COUNT] = {"frame",     "raster_setup", "raster", "shade",     "aa_loss", "shade_bwd",
                                            "frame_bwd", "laplacian",    "adam",   "mip_build", "scalars"};

struct StageRec {
    int stage;
    cudaEvent_t a, b;
};

struct adms_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // jobs with a deferred texture step when the capture began / ended (sorted): a
    // replay issues the steps of the first set and leaves those of the second
    std::vector<adms_job> pend_begin, pend_end;
};

// device-side arguments and work items of the batched (many-job) launches
struct BatchState {
    std::vector<long long> key;  // (job, B, H, W) per job + tile width: the item lists depend on it
    std::vector<ShadeArgs> h_args;   // passed to each launch as kernel parameters
    std::vector<RasterJob> h_rargs;
    std::vector<int> px_off, rt_off;  // job k's items: [off[k], off[k + 1])
    WorkItem* d_px = nullptr;
    WorkItem* d_rt = nullptr;
    size_t cap_px = 0, cap_rt = 0;
    std::vector<void*> allocs;
    size_t bytes = 0;
    bool has_job(long long job) const {  // key layout: 4 entries per job, then the tile width
        for (size_t k = 0; k + 4 < key.size(); k += 4)
            if (key[k] == job) return true;
        return false;
    }
};

struct adms_ctx {
    cudaStream_t stream = 0;
    // a second stream for the independent branches of a call (the vertex frame and
    // the Laplacian beside the raster, the flat latents' Adam beside the textures'),
    // forked from and joined back into `stream` within the call, so that a graph
    // captured on `stream` holds both
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // pipelined optimizer steps (adms_ctx_set_pipelining): a job's texture step is
    // deferred to its next forward_loss, which issues it on `late` beside its frame
    // and raster and waits for it before the shading; any other call naming the job
    // issues it first, in line
    bool pipeline = false;
    cudaStream_t late = nullptr;
    cudaEvent_t ev_late_fork = nullptr, ev_late_join = nullptr;
    // failure-detection test hook: bytes added to each Adam tile's expected copy
    // count, so that its bounded waits run out (adms_ctx_test_wait_timeout)
    uint32_t adam_extra_tx = 0;
    // the reference images of forward_loss calls are complete once this event has
    // completed (recorded on another stream that renders them), or null
    cudaEvent_t ref_event = nullptr;
    size_t budget = 0;
    size_t in_use = 0;
    std::string err;
    std::vector<Job> jobs;
    bool capturing = false;
    std::vector<adms_job> cap_pending;  // jobs with a deferred texture step when the capture began
    // one argument / work-item state per job set (and tile width): a graph recorded
    // for one batch keeps valid device arguments while other batches run
    std::vector<BatchState> batches;
    int sm_count = 148;
    // tile width (pixels; tiles are tw x 256/tw) and persistent blocks per SM of the
    // batched launches: [shade, aa+loss, backward, raster]; set by adms_autotune
    int tune_tw = 16;
    // (0: one block per item, the default: the ~4k-instruction pixel kernels lose
    // instruction-cache locality when persistent blocks drift apart in the loop)
    int tune_bpsm[4] = {0, 0, 0, 0};
    int occ[4] = {4, 4, 2, 4};  // resident blocks per SM of each persistent kernel
    // optional per-stage timing with CUDA events on the context's stream
    bool profile = false;
    std::vector<cudaEvent_t> pool;
    size_t pool_used = 0;
    std::vector<StageRec> recs;
    double stage_ms[ST_COUNT] = {0};
    long long stage_n[ST_COUNT] = {0};

    cudaEvent_t event() {
        if (pool_used == pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool.push_back(e);
        }
        return pool[pool_used++];
    }
};

namespace {

adms_status fail(adms_ctx* c, adms_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(ctx, ADMS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// run one launcher, bracketed by events when the context profiles
template <typename F>
cudaError_t timed(adms_ctx* ctx, int stage, F&& f) {
    if (!ctx->profile) return f();
    cudaEvent_t a = ctx->event();
    cudaEventRecord(a, ctx->stream);
    cudaError_t e = f();
    cudaEvent_t b = ctx->event();
    cudaEventRecord(b, ctx->stream);
    ctx->recs.push_back({stage, a, b});
    return e;
}

#define TIMED(stage, call) timed(ctx, stage, [&]() { return (call); })

// the stream of a branch: the side stream, ordered after everything issued on the
// context's stream so far (with per-stage profiling the branch stays on the
// context's stream, where the stage events time it)
cudaStream_t fork_branch(adms_ctx* ctx, cudaError_t& e) {
    e = cudaSuccess;
    if (ctx->profile || !ctx->side) return ctx->stream;
    e = cudaEventRecord(ctx->ev_fork, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0);
    return ctx->side;
}

// the context's stream waits for everything issued on the side stream
cudaError_t join_branch(adms_ctx* ctx) {
    if (ctx->profile || !ctx->side) return cudaSuccess;
    cudaError_t e = cudaEventRecord(ctx->ev_join, ctx->side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0);
    return e;
}

template <typename T>
adms_status job_alloc(adms_ctx* ctx, Job& j, T** out, size_t count) {
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    bytes = (bytes + 255) & ~size_t(255);
    if (ctx->capturing)
        return fail(ctx, ADMS_ERR_STATE, "a call inside graph capture needs new scratch: run it once before capturing");
    if (ctx->budget && ctx->in_use + bytes > ctx->budget)
        return fail(ctx, ADMS_ERR_BUDGET, "HBM budget exceeded (" + std::to_string(ctx->in_use + bytes) + " > " +
                                              std::to_string(ctx->budget) + " bytes)");
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return fail(ctx, ADMS_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    e = cudaMemsetAsync(p, 0, bytes, ctx->stream);
    if (e != cudaSuccess) return fail(ctx, ADMS_ERR_CUDA, std::string("cudaMemset: ") + cudaGetErrorString(e));
    j.allocs.push_back(p);
    j.bytes += bytes;
    ctx->in_use += bytes;
    *out = static_cast<T*>(p);
    return ADMS_OK;
}

#define AL(ptr, n)                                             \
    do {                                                       \
        adms_status s_ = job_alloc(ctx, j, &(ptr), (size_t)(n)); \
        if (s_ != ADMS_OK) return s_;                          \
    } while (0)

void job_free(adms_ctx* ctx, Job& j) {
    for (void* p : j.allocs) cudaFree(p);
    ctx->in_use -= std::min(ctx->in_use, j.bytes);
    j = Job();
}

Job* get_job(adms_ctx* ctx, adms_job h) {
    if (!ctx || h < 0 || h >= (adms_job)ctx->jobs.size() || !ctx->jobs[h].alive) return nullptr;
    return &ctx->jobs[h];
}

bool pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

// copy from host or device memory into a host vector
template <typename T>
adms_status to_host(adms_ctx* ctx, const T* src, size_t n, std::vector<T>& dst) {
    dst.resize(n);
    if (n) CK(cudaMemcpy(dst.data(), src, n * sizeof(T), cudaMemcpyDefault));
    return ADMS_OK;
}

adms_status tex_create(adms_ctx* ctx, Job& j, TexState& t, const float* src, int h, int w, bool mips, bool opt,
                       bool per_level) {
    if (!src || !pow2(h) || !pow2(w)) return fail(ctx, ADMS_ERR_ARG, "texture sizes must be powers of two");
    t.w = w;
    t.h = h;
    t.opt = opt;
    int lw = 0, lh = 0;
    while ((1 << lw) < w) ++lw;
    while ((1 << lh) < h) ++lh;
    t.levels = mips ? 1 + std::max(lw, lh) : 1;
    if (t.levels > ADMS_MAX_LEVELS) return fail(ctx, ADMS_ERR_ARG, "texture too large");
    size_t off = 0;
    for (int k = 0; k < t.levels; ++k) {
        t.off[k] = (int)off;
        off += (size_t)std::max(w >> k, 1) * std::max(h >> k, 1);
    }
    t.total = off;
    AL(t.data, t.total);
    CK(cudaMemcpyAsync(t.data, src, (size_t)w * h * sizeof(float4), cudaMemcpyDefault, ctx->stream));
    t.per_level = opt && per_level && t.levels > 1;
    if (opt) {
        size_t nm = t.per_level ? t.total : (size_t)w * h;
        AL(t.grad, t.total);
        AL(t.m, nm);
        AL(t.v, nm);
        if (!t.per_level && adam_tiled(t.dev())) CK(adam_encode_maps(t.dev(), t.m, t.v, t.tmaps));
    }
    CK(mip_build(t.dev(), ctx->stream));
    return ADMS_OK;
}

// grow per-call scratch to B views of H x W
adms_status ensure_scratch(adms_ctx* ctx, Job& j, int B, int H, int W) {
    size_t px = (size_t)B * H * W;
    int tiles = ((W + ADMS_TILE - 1) / ADMS_TILE) * ((H + ADMS_TILE - 1) / ADMS_TILE);
    size_t ntiles = (size_t)B * tiles;
    if (px > j.px_cap) {
        size_t nl = (size_t)std::max(j.L, 1);
        AL(j.keys, px * nl);
        AL(j.pre, px * nl);
        AL(j.gprime, px);
        AL(j.refine, px + 1);
        if (j.S > 1) AL(j.acol, px);
        if (j.L > 1) {
            AL(j.acc, px * (nl - 1));
            AL(j.gprime2, px);
        }
        j.px_cap = px;
    }
    if ((size_t)B > j.view_cap) {
        AL(j.views, B);
        AL(j.rs.clip, (size_t)B * j.V);
        AL(j.rs.scr, (size_t)B * j.V);
        AL(j.rs.vs, (size_t)B * j.V);
        AL(j.rs.rec, (size_t)B * j.F);
        AL(j.rs.bin, (size_t)B * j.F);
        AL(j.rs.asign, (size_t)B * j.F);
        AL(j.rs.silmask, (size_t)B * j.F);
        j.view_cap = B;
    }
    if (ntiles > j.tile_cap) {
        AL(j.rs.tile_count, 2 * ntiles);  // the fill cursors follow: one clear per raster pass
        AL(j.rs.tile_off, ntiles);
        j.rs.tile_cursor = j.rs.tile_count + ntiles;
        j.tile_cap = ntiles;
    }
    // tile-list capacity: 8 entries per triangle and view, at least 4 per tile
    size_t want = std::max<size_t>((size_t)8 * B * j.F, 4 * ntiles);
    if ((long long)want > j.rs.list_capacity) {
        AL(j.rs.list, want);
        j.rs.list_capacity = (long long)want;
    }
    if (!j.rs.total_pairs) {
        AL(j.rs.total_pairs, 1);
        AL(j.rs.overflow_ctr, 1);
    }
    return ADMS_OK;
}

// the Laplacian of Eq. 4 over the optimized (base) positions, its gradient added into g_pos
LapArgs lap_args(Job& j) { return LapArgs{j.LV, j.pos, j.ring_off, j.ring, j.delta_ref, j.delta, j.g_pos, j.st}; }

FrameArgs frame_args(Job& j) {
    FrameArgs f;
    f.V = j.V;
    f.F = j.F;
    f.pos = j.rpos;
    f.uv = j.uv;
    f.tri = j.tri;
    f.tri_uv = j.tri_uv;
    f.vf_off = j.vf_off;
    f.vf_face = j.vf_face;
    f.vpos = j.vpos;
    f.vnrm = j.vnrm;
    f.vtan = j.vtan;
    f.g_nrm = j.g_nrm;
    f.g_tan = j.g_tan;
    f.tmp_n = j.tmp_n;
    f.tmp_t = j.tmp_t;
    f.g_pos_acc = j.g_pos_acc;
    f.g_pos = j.g_rpos;
    f.status = &j.st->status;
    f.inv = j.frame_inv;
    return f;
}

// frame of the base mesh of a tessellated job (its normals feed the displacement)
FrameArgs base_frame_args(Job& j) {
    FrameArgs f;
    f.V = j.LV;
    f.F = j.Fb;
    f.pos = j.pos;
    f.uv = j.buv;
    f.tri = j.btri;
    f.tri_uv = j.btri_uv;
    f.vf_off = j.bvf_off;
    f.vf_face = j.bvf_face;
    f.vpos = j.b_vpos;
    f.vnrm = j.b_vnrm;
    f.vtan = j.b_vtan;
    f.g_nrm = j.g_bnrm;
    f.g_tan = j.g_btan0;
    f.tmp_n = j.b_tmp_n;
    f.tmp_t = j.b_tmp_t;
    f.g_pos_acc = j.g_bpos_acc;
    f.g_pos = j.g_pos;
    f.status = &j.st->status;
    return f;
}

TessArgs tess_args(Job& j) {
    TessArgs a;
    a.Vb = j.LV;
    a.Fb = j.Fb;
    a.Vt = j.V;
    a.n_seg = j.n_seg;
    a.base_pos = j.pos;
    a.base_tri = j.btri;
    a.bvf_off = j.bvf_off;
    a.bvf_face = j.bvf_face;
    a.base_nrm = j.bnrm;
    a.owner = j.owner;
    a.wts = j.wts;
    a.vert_uv = j.vert_uv;
    a.disp = j.disp;
    a.dh = j.dh;
    a.dw = j.dw;
    a.pos_out = j.rpos;
    a.g_pos_t = j.g_rpos;
    a.g_base_pos = j.g_bpos_acc;
    a.g_base_nrm = j.g_bnrm;
    a.g_disp = j.g_disp;
    return a;
}

ShadeArgs shade_args(Job& j) {
    ShadeArgs a;
    memset(&a, 0, sizeof(a));
    a.B = j.B;
    a.H = j.H;
    a.W = j.W;
    a.V = j.V;
    a.F = j.F;
    a.views = j.views;
    a.clip = j.rs.clip;
    a.scr = j.rs.scr;
    a.vpos = j.vpos;
    a.vnrm = j.vnrm;
    a.vtan = j.vtan;
    a.uv = j.uv;
    a.tri = j.tri;
    a.tri_uv = j.tri_uv;
    a.status = &j.st->status;
    a.silmask = j.rs.silmask;
    a.keys = j.keys;
    a.kd = j.kd.dev();
    a.orm = j.orm.dev();
    a.nrm = j.nrm.dev();
    a.pre = j.pre;
    a.gprime = j.gprime;
    a.refine = j.refine;
    a.msaa = (j.S > 1 && !j.ssaa) ? j.S : 0;
    a.acol = j.S > 1 ? j.acol : nullptr;
    a.peel = j.L > 0;
    a.loss_kind = j.opt.loss;
    a.loss_scale = j.loss_scale;
    a.aa = j.opt.aa;
    a.g_pos = j.g_pos_acc;
    a.g_nrm = j.g_nrm;
    a.g_tan = j.g_tan;
    return a;
}

// AA on the sample grid, then the per-pixel resolve of a supersampled job: the
// loss and each sample's dL/d(colour) when ref is given, the image into out_img
adms_status aa_resolve(adms_ctx* ctx, Job& j, const float* ref, double* loss_acc, float* out_img);

// arguments of layer l of a depth-peeled job: its keys and colours, the
// composite behind it (A_{l+1}, none behind the last layer)
ShadeArgs layer_args(Job& j, int l) {
    ShadeArgs a = shade_args(j);
    size_t px = (size_t)j.B * j.H * j.W;
    a.keys = j.keys + (size_t)l * px;
    a.pre = j.pre + (size_t)l * px;
    a.under = l + 1 < j.L ? j.acc + (size_t)l * px : nullptr;
    return a;
}

// back-to-front composite of a depth-peeled job, each layer antialiased with its own
// visibility: A_l = AA_l(alpha_l c_l + (1 - alpha_l) A_{l+1}); layer 0 takes the loss
// (and dL/dA_0 into gprime) when ref is given and writes the image into out_img
adms_status peel_composite(adms_ctx* ctx, Job& j, const float* ref, double* loss_acc, float* out_img);
// the adjoint of peel_composite and of every layer's shading, front to back
adms_status peel_backward(adms_ctx* ctx, Job& j);

// frame, raster and pre-AA shading of B views already copied to j.views
SkinArgs skin_args(Job& j) {
    SkinArgs a;
    a.V = j.V;
    a.B = j.SB;
    a.pos = j.pos;
    a.w = j.skin_w;
    a.bones = j.bones;
    a.out = j.rpos;
    a.g_out = j.g_rpos;
    a.g_pos = j.g_pos;
    a.g_w = j.g_skin_w;
    return a;
}

// The render positions (tessellated, skinned) on the context's stream, then the
// vertex frame and, once per set of positions, the Laplacian on a branch beside
// the raster: both need only the positions. *forked tells the caller to join the
// branch before the shading.
adms_status frame_branch(adms_ctx* ctx, Job& j, bool* forked) {
    *forked = false;
    if (j.frame_valid) return ADMS_OK;
    if (j.tess) CK(TIMED(ST_FRAME, tess_forward(tess_args(j), ctx->stream)));
    if (j.skin) CK(TIMED(ST_FRAME, skin_forward(skin_args(j), ctx->stream)));
    cudaError_t e;
    cudaStream_t bs = fork_branch(ctx, e);
    CK(e);
    *forked = true;
    CK(TIMED(ST_FRAME, frame_forward(frame_args(j), bs)));
    if (j.opt.optimize_pos && !j.lap_valid) {
        CK(TIMED(ST_LAPLACIAN, laplacian_forward(lap_args(j), bs)));
        j.lap_valid = true;
    }
    j.frame_valid = true;
    return ADMS_OK;
}

// join_late: the context's stream waits for the late stream (the job's deferred
// texture step) before the shading, the first kernel that reads the textures
adms_status render_core(adms_ctx* ctx, Job& j, bool join_late = false) {
    bool forked = false;
    adms_status fs = frame_branch(ctx, j, &forked);
    if (fs) return fs;
    RasterIn in;
    in.pos = j.rpos;
    in.tri = j.tri;
    in.adj = j.adj;
    in.views = j.views;
    in.B = j.B;
    in.V = j.V;
    in.F = j.F;
    in.W = j.W;
    in.H = j.H;
    in.keys = j.keys;
    if (j.L > 0) {
        // all L peeling layers in one tile pass (a k-buffer per sample): every triangle binned
        in.small_px = 0;
        CK(TIMED(ST_RASTER_SETUP, raster_prepare(in, j.rs, ctx->stream)));
        CK(TIMED(ST_RASTER, raster_tiles_peeled(in, j.rs, j.L, ctx->stream)));
        if (forked) CK(join_branch(ctx));
        if (join_late) CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_late_join, 0));
        for (int l = 0; l < j.L; ++l) CK(TIMED(ST_SHADE, shade_forward(layer_args(j, l), ctx->stream)));
        return ADMS_OK;
    }
    in.small_px = j.opt.raster_direct_px > 0 ? j.opt.raster_direct_px : ADMS_SMALL_PX;
    in.zfilter = j.opt.raster_depth_filter;
    CK(TIMED(ST_RASTER_SETUP, raster_prepare(in, j.rs, ctx->stream)));
    CK(TIMED(ST_RASTER, raster_tiles(in, j.rs, ctx->stream)));
    if (forked) CK(join_branch(ctx));
    if (join_late) CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_late_join, 0));
    CK(TIMED(ST_SHADE, shade_forward(shade_args(j), ctx->stream)));
    return ADMS_OK;
}

adms_status peel_composite(adms_ctx* ctx, Job& j, const float* ref, double* loss_acc, float* out_img) {
    size_t px = (size_t)j.B * j.H * j.W;
    for (int l = j.L - 1; l >= 0; --l) {
        ShadeArgs a = layer_args(j, l);
        a.ref = l == 0 ? ref : nullptr;
        a.loss_acc = l == 0 ? loss_acc : nullptr;
        a.out_img = l == 0 ? out_img : nullptr;
        a.acol = l > 0 ? j.acc + (size_t)(l - 1) * px : nullptr;
        CK(TIMED(ST_AA_LOSS, aa_loss_forward(a, ctx->stream)));
    }
    return ADMS_OK;
}

adms_status peel_backward(adms_ctx* ctx, Job& j) {
    for (int l = 0; l < j.L; ++l) {
        ShadeArgs a = layer_args(j, l);
        a.ref = j.ref;
        a.gprime = l % 2 == 0 ? j.gprime : j.gprime2;
        a.g_under = l + 1 < j.L ? (l % 2 == 0 ? j.gprime2 : j.gprime) : nullptr;
        CK(TIMED(ST_SHADE_BWD, shade_backward(a, ctx->stream)));
    }
    return ADMS_OK;
}

adms_status aa_resolve(adms_ctx* ctx, Job& j, const float* ref, double* loss_acc, float* out_img) {
    ShadeArgs a = shade_args(j);
    a.ref = nullptr;
    a.loss_acc = nullptr;
    a.out_img = nullptr;
    CK(TIMED(ST_AA_LOSS, aa_loss_forward(a, ctx->stream)));
    ResolveArgs r;
    r.B = j.B;
    r.H = j.PH;
    r.W = j.PW;
    r.S = j.S;
    r.acol = j.acol;
    r.ref = ref;
    r.gprime = j.gprime;
    r.out_img = out_img;
    r.loss_acc = loss_acc;
    r.loss_kind = j.opt.loss;
    r.loss_scale = j.loss_scale;
    CK(TIMED(ST_AA_LOSS, resolve_loss(r, ctx->stream)));
    return ADMS_OK;
}

void build_topology(const std::vector<int>& tri, int V, int F, std::vector<int>& adj, std::vector<int>& vf_off,
                    std::vector<int>& vf_face, std::vector<int>& ring_off, std::vector<int>& ring) {
    adj.assign((size_t)F * 3, -1);
    std::unordered_map<uint64_t, std::vector<int>> edges;
    edges.reserve((size_t)F * 2);
    for (int f = 0; f < F; ++f)
        for (int k = 0; k < 3; ++k) {
            uint32_t a = tri[3 * f + k], b = tri[3 * f + (k + 1) % 3];
            uint64_t key = ((uint64_t)std::min(a, b) << 32) | std::max(a, b);
            edges[key].push_back(3 * f + k);
        }
    for (auto& kv : edges)
        if (kv.second.size() == 2) {
            adj[kv.second[0]] = kv.second[1] / 3;
            adj[kv.second[1]] = kv.second[0] / 3;
        }
    vf_off.assign(V + 1, 0);
    for (int f = 0; f < F; ++f)
        for (int k = 0; k < 3; ++k) vf_off[tri[3 * f + k] + 1]++;
    for (int v = 0; v < V; ++v) vf_off[v + 1] += vf_off[v];
    vf_face.assign(vf_off[V], 0);
    std::vector<int> cur(vf_off.begin(), vf_off.end() - 1);
    for (int f = 0; f < F; ++f)
        for (int k = 0; k < 3; ++k) vf_face[cur[tri[3 * f + k]]++] = f;
    std::vector<std::vector<int>> nb(V);
    for (int f = 0; f < F; ++f)
        for (int k = 0; k < 3; ++k) {
            int a = tri[3 * f + k], b = tri[3 * f + (k + 1) % 3];
            nb[a].push_back(b);
            nb[b].push_back(a);
        }
    ring_off.assign(V + 1, 0);
    ring.clear();
    for (int v = 0; v < V; ++v) {
        auto& n = nb[v];
        std::sort(n.begin(), n.end());
        n.erase(std::unique(n.begin(), n.end()), n.end());
        ring.insert(ring.end(), n.begin(), n.end());
        ring_off[v + 1] = (int)ring.size();
    }
}

template <typename T>
adms_status upload(adms_ctx* ctx, Job& j, T** dst, const std::vector<T>& src) {
    AL(*dst, src.size());
    if (!src.empty()) CK(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    return ADMS_OK;
}

#define UP(dst, src)                               \
    do {                                           \
        adms_status s_ = upload(ctx, j, &(dst), src); \
        if (s_ != ADMS_OK) return s_;              \
    } while (0)

// Host side of the tessellation (Sec. 5.1): the lattice of n = 2^levels segments
// per base edge. Tessellated triangles are ordered base face by base face, and
// within a face by lattice row a and column b (the "up" triangle of cell (a, b),
// then its "down" triangle). A vertex shared by several base faces is owned by
// the lowest-numbered one, which fixes its weights and displacement UV.
struct TessHost {
    int n = 0, L = 0, NT = 0, Vt = 0;
    std::vector<int> rtri, rtri_uv, owner, wts;
    std::vector<float> corner_uv, vert_uv;
};

void build_tessellation(const std::vector<int>& tri, const std::vector<int>& tri_uv, const std::vector<float>& uv,
                        int F, int levels, TessHost& t) {
    int n = 1 << levels;
    t.n = n;
    std::vector<int> loc((n + 1) * (n + 1), -1), li, lj;
    for (int i = 0; i <= n; ++i)
        for (int jj = 0; jj <= n - i; ++jj) {
            loc[i * (n + 1) + jj] = (int)li.size();
            li.push_back(i);
            lj.push_back(jj);
        }
    t.L = (int)li.size();
    std::vector<int> lt;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n - a; ++b) {
            lt.insert(lt.end(), {loc[a * (n + 1) + b], loc[(a + 1) * (n + 1) + b], loc[a * (n + 1) + b + 1]});
            if (a + b + 1 < n)
                lt.insert(lt.end(), {loc[(a + 1) * (n + 1) + b], loc[(a + 1) * (n + 1) + b + 1], loc[a * (n + 1) + b + 1]});
        }
    t.NT = (int)lt.size() / 3;
    struct Key {
        long long a, b, c;
        bool operator==(const Key& o) const { return a == o.a && b == o.b && c == o.c; }
    };
    struct KH {
        size_t operator()(const Key& k) const { return std::hash<long long>()(k.a * 1000003LL ^ k.b * 998244353LL ^ k.c); }
    };
    std::unordered_map<Key, int, KH> index;
    std::vector<int> gidx((size_t)F * t.L);
    for (int f = 0; f < F; ++f) {
        for (int l = 0; l < t.L; ++l) {
            int w[3] = {n - li[l] - lj[l], li[l], lj[l]};
            long long id[3] = {tri[3 * f], tri[3 * f + 1], tri[3 * f + 2]};
            // canonical key: (vertex id, weight) pairs with weight > 0, sorted by id
            long long pr[3];
            int m = 0;
            for (int k = 0; k < 3; ++k)
                if (w[k] > 0) pr[m++] = id[k] * 4096 + w[k];
            std::sort(pr, pr + m);
            Key key{m > 0 ? pr[0] : -1, m > 1 ? pr[1] : -1, m > 2 ? pr[2] : -1};
            auto it = index.find(key);
            if (it == index.end()) {
                int v = (int)index.size();
                index.emplace(key, v);
                t.owner.insert(t.owner.end(), {tri[3 * f], tri[3 * f + 1], tri[3 * f + 2]});
                t.wts.insert(t.wts.end(), {w[0], w[1], w[2]});
                double u = 0.0, vv = 0.0;
                for (int k = 0; k < 3; ++k) {
                    double wk = (double)w[k] / (double)n;
                    u += wk * (double)uv[2 * tri_uv[3 * f + k]];
                    vv += wk * (double)uv[2 * tri_uv[3 * f + k] + 1];
                }
                t.vert_uv.push_back((float)u);
                t.vert_uv.push_back((float)vv);
                gidx[(size_t)f * t.L + l] = v;
            } else {
                gidx[(size_t)f * t.L + l] = it->second;
            }
            double u = 0.0, vv = 0.0;
            for (int k = 0; k < 3; ++k) {
                double wk = (double)w[k] / (double)n;
                u += wk * (double)uv[2 * tri_uv[3 * f + k]];
                vv += wk * (double)uv[2 * tri_uv[3 * f + k] + 1];
            }
            t.corner_uv.push_back((float)u);
            t.corner_uv.push_back((float)vv);
        }
        for (int k = 0; k < t.NT * 3; ++k) {
            t.rtri.push_back(gidx[(size_t)f * t.L + lt[k]]);
            t.rtri_uv.push_back(f * t.L + lt[k]);
        }
    }
    t.Vt = (int)index.size();
}

adms_status job_create_impl(adms_ctx* ctx, const adms_mesh_desc* mesh, const adms_material_desc* mat,
                            const adms_opt_params* opt, uint64_t seed, Job& j) {
    if (!mesh || !mat || !mesh->pos || !mesh->uv || !mesh->tri_pos || !mesh->tri_uv || mesh->n_verts <= 0 ||
        mesh->n_tris <= 0 || mesh->n_uv <= 0)
        return fail(ctx, ADMS_ERR_ARG, "invalid mesh description");
    j.alive = true;
    j.seed = seed;
    j.frozen = opt == nullptr;
    if (opt) j.opt = *opt;
    else {
        memset(&j.opt, 0, sizeof(j.opt));
        j.opt.aa = 1;
    }
    if (j.opt.tess_levels < 0 || j.opt.tess_levels > 6) return fail(ctx, ADMS_ERR_ARG, "tess_levels must be in [0, 6]");
    if (j.opt.samples < 0 || j.opt.samples > 8) return fail(ctx, ADMS_ERR_ARG, "samples must be in [0, 8]");
    if (j.opt.layers < 0 || j.opt.layers > 16) return fail(ctx, ADMS_ERR_ARG, "layers must be in [0, 16]");
    if (j.opt.raster_direct_px < 0 || j.opt.raster_direct_px > 4096)
        return fail(ctx, ADMS_ERR_ARG, "raster_direct_px must be in [0, 4096]");
    if (j.opt.raster_depth_filter != 0 && j.opt.raster_depth_filter != 1)
        return fail(ctx, ADMS_ERR_ARG, "raster_depth_filter must be 0 or 1");
    if (j.opt.layers > 0 && (j.opt.samples > 1 || j.opt.tess_levels > 0))
        return fail(ctx, ADMS_ERR_ARG, "depth peeling runs on plain meshes at one sample per pixel");
    j.L = j.opt.layers;
    j.S = std::max(1, (int)j.opt.samples);
    j.ssaa = j.opt.shade_samples != 0;
    j.tess = j.opt.tess_levels > 0;
    if (j.tess && (!mat->disp || !pow2(mat->disp_h) || !pow2(mat->disp_w)))
        return fail(ctx, ADMS_ERR_ARG, "a tessellated job needs a power-of-two displacement map");
    int Vb = mesh->n_verts, Tb = mesh->n_uv, Fb = mesh->n_tris;
    j.LV = Vb;
    std::vector<int> tri, tri_uv;
    adms_status s;
    if ((s = to_host(ctx, mesh->tri_pos, (size_t)Fb * 3, tri))) return s;
    if ((s = to_host(ctx, mesh->tri_uv, (size_t)Fb * 3, tri_uv))) return s;
    for (int x : tri)
        if (x < 0 || x >= Vb) return fail(ctx, ADMS_ERR_ARG, "position index out of range");
    for (int x : tri_uv)
        if (x < 0 || x >= Tb) return fail(ctx, ADMS_ERR_ARG, "uv index out of range");
    // latent (base) positions, their Laplacian topology and optimizer state
    std::vector<int> badj, bvf_off, bvf_face, ring_off, ring;
    build_topology(tri, Vb, Fb, badj, bvf_off, bvf_face, ring_off, ring);
    UP(j.ring_off, ring_off);
    UP(j.ring, ring);
    AL(j.pos, (size_t)Vb * 3);
    CK(cudaMemcpyAsync(j.pos, mesh->pos, (size_t)Vb * 3 * sizeof(float), cudaMemcpyDefault, ctx->stream));
    AL(j.g_pos, (size_t)Vb * 3);
    if (j.opt.optimize_pos) {
        AL(j.m_pos, (size_t)Vb * 3);
        AL(j.v_pos, (size_t)Vb * 3);
    }
    AL(j.delta, (size_t)Vb * 3);
    // render mesh: the base mesh itself, or its tessellation
    std::vector<int> rtri = tri, rtri_uv = tri_uv;
    if (!j.tess) {
        j.V = Vb;
        j.T = Tb;
        j.F = Fb;
        AL(j.uv, j.T);
        CK(cudaMemcpyAsync(j.uv, mesh->uv, (size_t)j.T * 2 * sizeof(float), cudaMemcpyDefault, ctx->stream));
        j.rpos = j.pos;
        j.g_rpos = j.g_pos;
    } else {
        std::vector<float> uvh;
        if ((s = to_host(ctx, mesh->uv, (size_t)Tb * 2, uvh))) return s;
        TessHost th;
        build_tessellation(tri, tri_uv, uvh, Fb, j.opt.tess_levels, th);
        j.V = th.Vt;
        j.F = Fb * th.NT;
        j.T = Fb * th.L;
        j.n_seg = th.n;
        rtri = th.rtri;
        rtri_uv = th.rtri_uv;
        AL(j.uv, j.T);
        CK(cudaMemcpyAsync(j.uv, th.corner_uv.data(), th.corner_uv.size() * sizeof(float), cudaMemcpyHostToDevice,
                           ctx->stream));
        UP(j.btri, tri);
        UP(j.btri_uv, tri_uv);
        UP(j.bvf_off, bvf_off);
        UP(j.bvf_face, bvf_face);
        UP(j.owner, th.owner);
        UP(j.wts, th.wts);
        AL(j.vert_uv, j.V);
        CK(cudaMemcpyAsync(j.vert_uv, th.vert_uv.data(), th.vert_uv.size() * sizeof(float), cudaMemcpyHostToDevice,
                           ctx->stream));
        AL(j.buv, Tb);
        CK(cudaMemcpyAsync(j.buv, mesh->uv, (size_t)Tb * 2 * sizeof(float), cudaMemcpyDefault, ctx->stream));
        AL(j.bnrm, (size_t)Vb * 3);
        AL(j.rpos, (size_t)j.V * 3);
        AL(j.g_rpos, (size_t)j.V * 3);
        AL(j.g_bnrm, (size_t)Vb * 3);
        AL(j.g_btan0, (size_t)Vb * 3);
        AL(j.g_bpos_acc, (size_t)Vb * 3);
        AL(j.b_vpos, Vb);
        AL(j.b_vnrm, Vb);
        AL(j.b_vtan, Vb);
        AL(j.b_tmp_n, Vb);
        AL(j.b_tmp_t, Vb);
        j.Fb = Fb;
        j.dh = mat->disp_h;
        j.dw = mat->disp_w;
        AL(j.disp, (size_t)j.dh * j.dw);
        CK(cudaMemcpyAsync(j.disp, mat->disp, (size_t)j.dh * j.dw * sizeof(float), cudaMemcpyDefault, ctx->stream));
        if (j.opt.optimize_disp) {
            AL(j.g_disp, (size_t)j.dh * j.dw);
            AL(j.m_disp, (size_t)j.dh * j.dw);
            AL(j.v_disp, (size_t)j.dh * j.dw);
        }
    }
    std::vector<int> adj, vf_off, vf_face, rring_off, rring;
    build_topology(rtri, j.V, j.F, adj, vf_off, vf_face, rring_off, rring);
    UP(j.tri, rtri);
    UP(j.tri_uv, rtri_uv);
    UP(j.adj, adj);
    UP(j.vf_off, vf_off);
    UP(j.vf_face, vf_face);
    AL(j.vpos, j.V);
    AL(j.vnrm, j.V);
    AL(j.vtan, j.V);
    AL(j.tmp_n, j.V);
    AL(j.tmp_t, j.V);
    AL(j.frame_inv, j.V);
    AL(j.g_nrm, (size_t)j.V * 6);  // the tangents' gradient follows: one clear per backward
    j.g_tan = j.g_nrm + (size_t)j.V * 3;
    AL(j.g_pos_acc, (size_t)j.V * 3);
    AL(j.st, 1);
    bool mips = mat->mips != 0;
    bool pl = j.opt.per_level_textures != 0;
    if (pl && !mips) return fail(ctx, ADMS_ERR_ARG, "per-level textures need mip chains");
    if ((s = tex_create(ctx, j, j.kd, mat->kd, mat->kd_h, mat->kd_w, mips, j.opt.optimize_kd, pl))) return s;
    if ((s = tex_create(ctx, j, j.orm, mat->orm, mat->orm_h, mat->orm_w, mips, j.opt.optimize_orm, pl))) return s;
    if ((s = tex_create(ctx, j, j.nrm, mat->nrm, mat->nrm_h, mat->nrm_w, mips, j.opt.optimize_nrm, pl))) return s;
    if (j.opt.relative_laplacian) {
        AL(j.delta_ref, (size_t)Vb * 3);
        LapArgs la{Vb, j.pos, j.ring_off, j.ring, nullptr, j.delta_ref, j.g_pos, j.st};
        CK(laplacian_forward(la, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return ADMS_OK;
}

// frame (and tessellation) plus the per-job raster preparation of a batched call
// frame_branch and the raster setup of one job of a batch (*forked: join before
// the batch's shading)
adms_status frame_and_prepare(adms_ctx* ctx, Job& j, bool* forked) {
    bool f = false;
    adms_status fs = frame_branch(ctx, j, &f);
    if (fs) return fs;
    *forked = *forked || f;
    RasterIn in;
    in.pos = j.rpos;
    in.tri = j.tri;
    in.adj = j.adj;
    in.views = j.views;
    in.B = j.B;
    in.V = j.V;
    in.F = j.F;
    in.W = j.W;
    in.H = j.H;
    in.keys = j.keys;
    in.small_px = j.opt.raster_direct_px > 0 ? j.opt.raster_direct_px : ADMS_SMALL_PX;
    in.zfilter = j.opt.raster_depth_filter;
    CK(TIMED(ST_RASTER_SETUP, raster_prepare(in, j.rs, ctx->stream)));
    return ADMS_OK;
}

template <typename T>
adms_status batch_alloc(adms_ctx* ctx, BatchState& bs, T** out, size_t count) {
    size_t bytes = ((std::max<size_t>(count, 1) * sizeof(T)) + 255) & ~size_t(255);
    if (ctx->capturing) return fail(ctx, ADMS_ERR_STATE, "batched launch needs new scratch during capture");
    if (ctx->budget && ctx->in_use + bytes > ctx->budget) return fail(ctx, ADMS_ERR_BUDGET, "HBM budget exceeded");
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return fail(ctx, ADMS_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    bs.allocs.push_back(p);
    bs.bytes += bytes;
    ctx->in_use += bytes;
    *out = static_cast<T*>(p);
    return ADMS_OK;
}

void batch_free(adms_ctx* ctx, BatchState& bs) {
    for (void* p : bs.allocs) cudaFree(p);
    ctx->in_use -= std::min(ctx->in_use, bs.bytes);
    bs = BatchState();
}

// grid of a batched launch: SMs x blocks per SM (persistent), or one block per
// item when the tuning says 0 (the launchers clamp the grid to the item count)
int batch_grid(const adms_ctx* ctx, int kind) {
    return ctx->tune_bpsm[kind] > 0 ? ctx->sm_count * ctx->tune_bpsm[kind] : INT32_MAX;
}

// drop the batched argument lists of every job set that holds this job (the
// caller has synchronized the stream)
void batch_release(adms_ctx* ctx, long long job) {
    std::vector<BatchState> keep;
    for (BatchState& b : ctx->batches) {
        if (b.has_job(job))
            batch_free(ctx, b);
        else
            keep.push_back(std::move(b));
    }
    ctx->batches = std::move(keep);
}

// Arguments and work items of a batched call. Uploaded only when the job set,
// their image sizes, the tile width or the jobs' buffers change, so a warmed-up
// batched step records into a CUDA graph without host-to-device copies.
adms_status batch_upload(adms_ctx* ctx, const std::vector<Job*>& js, float* const* out_img, BatchState** out_bs,
                         bool backward = false) {
    int n = (int)js.size();
    std::vector<long long> key;
    for (Job* j : js) {
        key.push_back((long long)(j - ctx->jobs.data()));
        key.push_back(j->B);
        key.push_back(j->H);
        key.push_back(j->W);
    }
    key.push_back(ctx->tune_tw);
    BatchState* found = nullptr;
    for (BatchState& b : ctx->batches)
        if (b.key == key) found = &b;
    if (!found) {
        if (ctx->capturing) return fail(ctx, ADMS_ERR_STATE, "new batch during capture: make the same call once before");
        ctx->batches.emplace_back();
        found = &ctx->batches.back();
    }
    BatchState& bs = *found;
    *out_bs = found;
    bool same = key == bs.key;
    if (backward && same) return ADMS_OK;  // the forward's arguments serve the backward
    std::vector<ShadeArgs> args(n);
    std::vector<RasterJob> rargs(n);
    for (int k = 0; k < n; ++k) {
        Job& j = *js[k];
        args[k] = shade_args(j);
        args[k].ref = j.ref;
        args[k].loss_acc = &j.st->call_loss;
        args[k].out_img = out_img ? out_img[k] : nullptr;
        RasterJob& r = rargs[k];
        memset(&r, 0, sizeof(r));
        r.rec = j.rs.rec;
        r.bin = j.rs.bin;
        r.F = j.F;
        r.W = j.W;
        r.H = j.H;
        r.tiles_x = (j.W + ADMS_TILE - 1) / ADMS_TILE;
        r.tiles_y = (j.H + ADMS_TILE - 1) / ADMS_TILE;
        r.tile_off = j.rs.tile_off;
        r.tile_count = j.rs.tile_count;
        r.list = j.rs.list;
        r.capacity = j.rs.list_capacity;
        r.keys = j.keys;
        r.overflow_ctr = j.rs.overflow_ctr;
    }
    bs.h_args = args;
    bs.h_rargs = rargs;
    adms_status s;
    if (!same) {
        if (ctx->capturing)
            return fail(ctx, ADMS_ERR_STATE, "new batched work items during capture: make the same call once before");
        int tw = ctx->tune_tw, th = 256 / tw;
        std::vector<WorkItem> px, rt;
        bs.px_off.assign(1, 0);
        bs.rt_off.assign(1, 0);
        for (int k = 0; k < n; ++k) {
            const Job& j = *js[k];
            for (int b = 0; b < j.B; ++b) {
                for (int y0 = 0; y0 < j.H; y0 += th)
                    for (int x0 = 0; x0 < j.W; x0 += tw) px.push_back({k, b, x0, y0});
                for (int y0 = 0; y0 < j.H; y0 += ADMS_TILE)
                    for (int x0 = 0; x0 < j.W; x0 += ADMS_TILE) rt.push_back({k, b, x0, y0});
            }
            bs.px_off.push_back((int)px.size());
            bs.rt_off.push_back((int)rt.size());
        }
        if (px.size() > bs.cap_px) {
            if ((s = batch_alloc(ctx, bs, &bs.d_px, px.size()))) return s;
            bs.cap_px = px.size();
        }
        if (rt.size() > bs.cap_rt) {
            if ((s = batch_alloc(ctx, bs, &bs.d_rt, rt.size()))) return s;
            bs.cap_rt = rt.size();
        }
        CK(cudaMemcpy(bs.d_px, px.data(), px.size() * sizeof(WorkItem), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(bs.d_rt, rt.data(), rt.size() * sizeof(WorkItem), cudaMemcpyHostToDevice));
        bs.key = key;
    }
    return ADMS_OK;
}

// ------------------------------------------------------------------ checkpoints
// A job's resumable state as one host blob: a fixed header (shapes and options,
// so a blob is only loaded into a job of the same layout) and the device
// buffers below, in this order. Gradients and per-step scratch are not kept:
// export between optimizer steps.
const char kCkptMagic[8] = {'A', 'D', 'M', 'S', 'C', 'K', 'P', 'T'};
const uint32_t kCkptVersion = 3;  // 2: per-level, skinning and multisampling fields; 3: layers

struct CkptHeader {
    char magic[8];
    uint32_t version, n_sections;
    uint64_t seed;
    int32_t LV, V, F, tess_levels, dh, dw;
    int32_t tex_w[3], tex_h[3], tex_levels[3], tex_opt[3];
    int32_t optimize[5];  // pos, kd, orm, nrm, disp
    int32_t loss, relative_laplacian, batch_views, aa, per_level_textures, n_bones, samples, shade_samples, layers;
    float lr0, lambda0, skin_lr_scale;
    uint64_t section_bytes[16];
};

struct CkptSection {
    void* ptr;
    size_t bytes;
};

void ckpt_describe(Job& j, CkptHeader& h, std::vector<CkptSection>& secs) {
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kCkptMagic, 8);
    h.version = kCkptVersion;
    h.seed = j.seed;
    h.LV = j.LV;
    h.V = j.V;
    h.F = j.F;
    h.tess_levels = j.opt.tess_levels;
    h.dh = j.dh;
    h.dw = j.dw;
    const TexState* tx[3] = {&j.kd, &j.orm, &j.nrm};
    for (int k = 0; k < 3; ++k) {
        h.tex_w[k] = tx[k]->w;
        h.tex_h[k] = tx[k]->h;
        h.tex_levels[k] = tx[k]->levels;
        h.tex_opt[k] = tx[k]->opt;
    }
    h.optimize[0] = j.opt.optimize_pos;
    h.optimize[1] = j.opt.optimize_kd;
    h.optimize[2] = j.opt.optimize_orm;
    h.optimize[3] = j.opt.optimize_nrm;
    h.optimize[4] = j.opt.optimize_disp;
    h.loss = j.opt.loss;
    h.relative_laplacian = j.opt.relative_laplacian;
    h.batch_views = j.opt.batch_views;
    h.aa = j.opt.aa;
    h.per_level_textures = j.opt.per_level_textures;
    h.n_bones = j.SB;
    h.samples = j.S;
    h.shade_samples = j.ssaa;
    h.layers = j.L;
    h.skin_lr_scale = j.skin_lr_scale;
    h.lr0 = j.opt.lr0;
    h.lambda0 = j.opt.lambda0;
    secs.clear();
    auto add = [&](void* p, size_t n) {
        if (p && n) secs.push_back({p, n});
    };
    size_t pv = (size_t)j.LV * 3 * sizeof(float);
    add(j.pos, pv);
    add(j.m_pos, pv);
    add(j.v_pos, pv);
    for (int k = 0; k < 3; ++k) {
        TexState& t = *const_cast<TexState*>(tx[k]);
        add(t.data, t.total * sizeof(float4));  // the whole chain: resumes without a rebuild
        if (t.opt) {
            size_t nm = (t.per_level ? t.total : (size_t)t.w * t.h) * sizeof(float4);
            add(t.m, nm);
            add(t.v, nm);
        }
    }
    size_t pd = (size_t)j.dh * j.dw * sizeof(float);
    add(j.disp, pd);
    add(j.m_disp, pd);
    add(j.v_disp, pd);
    add(j.delta_ref, pv);
    size_t psw = (size_t)j.LV * j.SB * sizeof(float);
    add(j.skin_w, psw);
    add(j.m_skin_w, psw);
    add(j.v_skin_w, psw);
    add(j.bones, (size_t)j.SB * 16 * sizeof(float));
    add(j.st, sizeof(JobState));
    h.n_sections = (uint32_t)secs.size();
    for (size_t k = 0; k < secs.size() && k < 16; ++k) h.section_bytes[k] = secs[k].bytes;
}

}  // namespace

// ============================================================================ C ABI

extern "C" {

// ------------------------------------------------------------------ texture steps
// the Adam updates of the texture latents of jobs js (Eq. 4 moments, clamps, the mip
// chain rebuilt) on stream st: every job's tiled textures in one launch
static adms_status texture_adams(adms_ctx* ctx, const std::vector<Job*>& js, cudaStream_t st) {
    std::vector<TexAdam> tiled;
    for (Job* jp : js) {
        Job& j = *jp;
        TexState* maps[3] = {&j.kd, &j.orm, &j.nrm};
        for (int m = 0; m < 3; ++m) {
            if (!maps[m]->opt) continue;
            TexDev td = maps[m]->dev();
            if (maps[m]->per_level) {
                CK(TIMED(ST_ADAM, adam_texture_levels(td, maps[m]->m, maps[m]->v, m, j.st, st)));
            } else if (adam_tiled(td)) {
                TexAdam ta{td, maps[m]->m, maps[m]->v, j.st, m, 0};
                ta.tmaps = maps[m]->tmaps;
                tiled.push_back(ta);
            } else {
                CK(TIMED(ST_ADAM, adam_texture_and_mips(td, maps[m]->m, maps[m]->v, m, j.st, st)));
            }
        }
    }
    if (!tiled.empty()) CK(TIMED(ST_ADAM, adam_textures_tiled(tiled, st, ctx->adam_extra_tx)));
    return ADMS_OK;
}

// a job's deferred texture step and step counter, in line on the context's stream
static adms_status flush_job(adms_ctx* ctx, Job& j) {
    if (!j.tex_pending) return ADMS_OK;
    j.tex_pending = false;
    adms_status s = texture_adams(ctx, {&j}, ctx->stream);
    if (s) return s;
    CK(TIMED(ST_SMALL, advance_step(j.st, ctx->stream)));
    return ADMS_OK;
}
static adms_status flush_all(adms_ctx* ctx) {
    for (auto& j : ctx->jobs)
        if (j.alive) {
            adms_status s = flush_job(ctx, j);
            if (s) return s;
        }
    return ADMS_OK;
}

// forward_loss of one job: its deferred texture step on the late stream, ordered
// after everything issued on the context's stream so far; *forked tells the caller
// to wait for it before the shading (in line when profiling: the stage events time
// it on the context's stream)
static adms_status fork_texture_step(adms_ctx* ctx, Job& j, bool* forked) {
    *forked = false;
    if (!j.tex_pending) return ADMS_OK;
    if (ctx->profile) return flush_job(ctx, j);
    j.tex_pending = false;
    CK(cudaEventRecord(ctx->ev_late_fork, ctx->stream));
    CK(cudaStreamWaitEvent(ctx->late, ctx->ev_late_fork, 0));
    adms_status s = texture_adams(ctx, {&j}, ctx->late);
    if (s) return s;
    CK(advance_step(j.st, ctx->late));
    CK(cudaEventRecord(ctx->ev_late_join, ctx->late));
    *forked = true;
    return ADMS_OK;
}

static std::vector<adms_job> pending_jobs(adms_ctx* ctx) {
    std::vector<adms_job> out;
    for (size_t h = 0; h < ctx->jobs.size(); ++h)
        if (ctx->jobs[h].alive && ctx->jobs[h].tex_pending) out.push_back((adms_job)h);
    return out;
}

adms_status adms_ctx_create(adms_ctx** out, size_t hbm_budget_bytes, void* cuda_stream) {
    if (!out) return ADMS_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ADMS_ERR_CUDA;
    adms_ctx* c = new adms_ctx();
    c->stream = (cudaStream_t)cuda_stream;
    c->budget = hbm_budget_bytes;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0) c->sm_count = sms;
    for (int k = 0; k < 4; ++k) c->occ[k] = adms::batched_occupancy(k);
    if (adms::adam_prepare() != cudaSuccess) {
        delete c;
        return ADMS_ERR_CUDA;
    }
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->late, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_late_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_late_join, cudaEventDisableTiming) != cudaSuccess) {
        if (c->ev_late_fork) cudaEventDestroy(c->ev_late_fork);
        if (c->late) cudaStreamDestroy(c->late);
        if (c->ev_join) cudaEventDestroy(c->ev_join);
        if (c->ev_fork) cudaEventDestroy(c->ev_fork);
        if (c->side) cudaStreamDestroy(c->side);
        delete c;
        return ADMS_ERR_CUDA;
    }
    *out = c;
    return ADMS_OK;
}

adms_status adms_ctx_destroy(adms_ctx* ctx) {
    if (!ctx) return ADMS_ERR_ARG;
    cudaStreamSynchronize(ctx->stream);
    for (auto& j : ctx->jobs)
        if (j.alive) job_free(ctx, j);
    for (BatchState& b : ctx->batches) batch_free(ctx, b);
    for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
    cudaStreamSynchronize(ctx->side);
    cudaStreamSynchronize(ctx->late);
    cudaEventDestroy(ctx->ev_fork);
    cudaEventDestroy(ctx->ev_join);
    cudaEventDestroy(ctx->ev_late_fork);
    cudaEventDestroy(ctx->ev_late_join);
    cudaStreamDestroy(ctx->side);
    cudaStreamDestroy(ctx->late);
    delete ctx;
    return ADMS_OK;
}

adms_status adms_autotune(adms_ctx* ctx, const adms_job* jobs, int32_t n_jobs, const adms_view* views,
                          const int32_t* views_per_job, const int32_t* hw, const float* const* ref_rgb) {
    if (!ctx || n_jobs < 2) return fail(ctx, ADMS_ERR_ARG, "autotune needs a batch of at least two jobs");
    if (ctx->capturing || ctx->profile) return fail(ctx, ADMS_ERR_STATE, "autotune while capturing or profiling");
    const int tws[3] = {8, 16, 32};
    float best_total = 1e30f;
    int best_tw = ctx->tune_tw, best_b[4] = {ctx->tune_bpsm[0], ctx->tune_bpsm[1], ctx->tune_bpsm[2], ctx->tune_bpsm[3]};
    std::vector<Job*> js;
    for (int k = 0; k < n_jobs; ++k) {
        Job* j = get_job(ctx, jobs[k]);
        if (!j) return fail(ctx, ADMS_ERR_ARG, "invalid job handle");
        if (adms_status fs = flush_job(ctx, *j)) return fs;  // its deferred texture step first
        js.push_back(j);
    }
    // timing events, destroyed on every return path; the tile width is restored
    // if a timing run fails
    struct Timing {
        cudaEvent_t ev[2] = {nullptr, nullptr};
        adms_ctx* ctx;
        int tw0;
        bool done = false;
        ~Timing() {
            for (auto& e : ev)
                if (e) cudaEventDestroy(e);
            if (!done) ctx->tune_tw = tw0;
        }
    } timing{{nullptr, nullptr}, ctx, ctx->tune_tw};
    cudaEvent_t* ev = timing.ev;
    for (int k = 0; k < 2; ++k) CK(cudaEventCreate(&ev[k]));
    // a forward sizes every job's scratch; then time each kernel at each tile
    // width with one block per item and with persistent grids of occ/2 .. occ
    // resident blocks per SM (second of two runs; every kernel here is
    // idempotent or accumulates into buffers reset below)
    adms_status s = adms_forward_loss(ctx, jobs, n_jobs, views, views_per_job, hw, ref_rgb, nullptr, nullptr);
    if (s) return s;
    for (int tw : tws) {
        ctx->tune_tw = tw;
        BatchState* bsp = nullptr;
        if ((s = batch_upload(ctx, js, nullptr, &bsp))) return s;
        BatchState& bs = *bsp;
        float total = 0.f;
        int b_kind[4] = {best_b[0], best_b[1], best_b[2], best_b[3]};
        for (int kind = 0; kind < 4; ++kind) {
            if (kind == 3 && tw != tws[0]) continue;  // the raster's items do not depend on tw
            float t_best = 1e30f;
            std::vector<int> cands(1, 0);  // 0: one block per item
            for (int bp = std::max(1, ctx->occ[kind] / 2); bp <= ctx->occ[kind]; ++bp) cands.push_back(bp);
            for (int bp : cands) {
                for (int rep = 0; rep < 2; ++rep) {
                    int blocks = bp ? ctx->sm_count * bp : INT32_MAX;
                    CK(cudaEventRecord(ev[0], ctx->stream));
                    if (kind == 3)
                        CK(raster_tiles_batched(bs.h_rargs.data(), bs.rt_off.data(), n_jobs, bs.d_rt, blocks,
                                                ctx->stream));
                    else
                        CK(pixels_batched(kind, bs.h_args.data(), bs.px_off.data(), n_jobs, bs.d_px, tw, blocks,
                                          ctx->stream));
                    CK(cudaEventRecord(ev[1], ctx->stream));
                    CK(cudaEventSynchronize(ev[1]));
                    float t = 0.f;
                    CK(cudaEventElapsedTime(&t, ev[0], ev[1]));
                    if (rep == 1 && t < t_best) {
                        t_best = t;
                        b_kind[kind] = bp;
                    }
                }
            }
            if (kind == 3) best_b[3] = b_kind[3];
            else total += t_best;
        }
        if (total < best_total) {
            best_total = total;
            best_tw = tw;
            for (int kk = 0; kk < 3; ++kk) best_b[kk] = b_kind[kk];
        }
    }
    timing.done = true;
    ctx->tune_tw = best_tw;
    for (int kk = 0; kk < 4; ++kk) ctx->tune_bpsm[kk] = best_b[kk];
    // leave the jobs as they were: no gradients, no pending forward, no loss recorded
    for (Job* j : js) {
        if ((s = adms_job_zero_gradients(ctx, (adms_job)(j - ctx->jobs.data())))) return s;
        CK(cudaMemsetAsync(j->st, 0, 2 * sizeof(double), ctx->stream));  // call_loss, img_loss
        j->have_fwd = false;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return ADMS_OK;
}

adms_status adms_ctx_set_tuning(adms_ctx* ctx, const int32_t* in5) {
    if (!ctx || !in5) return ADMS_ERR_ARG;
    if (in5[0] != 8 && in5[0] != 16 && in5[0] != 32) return fail(ctx, ADMS_ERR_ARG, "tile width must be 8, 16 or 32");
    ctx->tune_tw = in5[0];
    for (int k = 0; k < 4; ++k) ctx->tune_bpsm[k] = in5[1 + k] <= 0 ? 0 : std::min(in5[1 + k], ctx->occ[k]);
    return ADMS_OK;
}

adms_status adms_ctx_tuning(adms_ctx* ctx, int32_t* out5) {
    if (!ctx || !out5) return ADMS_ERR_ARG;
    out5[0] = ctx->tune_tw;
    for (int k = 0; k < 4; ++k) out5[1 + k] = ctx->tune_bpsm[k];
    return ADMS_OK;
}

adms_status adms_ctx_set_stream(adms_ctx* ctx, void* cuda_stream) {
    if (!ctx) return ADMS_ERR_ARG;
    ctx->stream = (cudaStream_t)cuda_stream;
    return ADMS_OK;
}

adms_status adms_ctx_set_ref_event(adms_ctx* ctx, void* cuda_event) {
    if (!ctx) return ADMS_ERR_ARG;
    ctx->ref_event = (cudaEvent_t)cuda_event;
    return ADMS_OK;
}

// the context's stream waits for the reference images, right before the first
// kernel that reads them
static cudaError_t wait_ref(adms_ctx* ctx) {
    return ctx->ref_event ? cudaStreamWaitEvent(ctx->stream, ctx->ref_event, 0) : cudaSuccess;
}

adms_status adms_sync(adms_ctx* ctx) {
    if (!ctx) return ADMS_ERR_ARG;
    if (adms_status fs = flush_all(ctx)) return fs;
    CK(cudaStreamSynchronize(ctx->stream));
    return ADMS_OK;
}

const char* adms_last_error(adms_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

size_t adms_bytes_in_use(adms_ctx* ctx) { return ctx ? ctx->in_use : 0; }

adms_status adms_job_create(adms_ctx* ctx, const adms_mesh_desc* mesh, const adms_material_desc* mat,
                            const adms_opt_params* opt, uint64_t seed, adms_job* out) {
    if (!ctx || !out) return fail(ctx, ADMS_ERR_ARG, "null argument");
    ctx->jobs.emplace_back();
    Job& j = ctx->jobs.back();
    adms_status s = job_create_impl(ctx, mesh, mat, opt, seed, j);
    if (s != ADMS_OK) {
        cudaStreamSynchronize(ctx->stream);
        job_free(ctx, ctx->jobs.back());
        return s;
    }
    *out = (adms_job)(ctx->jobs.size() - 1);
    return ADMS_OK;
}

adms_status adms_job_destroy(adms_ctx* ctx, adms_job job) {
    Job* j = get_job(ctx, job);
    if (!j) return fail(ctx, ADMS_ERR_ARG, "invalid job handle");
    j->tex_pending = false;  // a destroyed job's deferred texture step is dropped
    CK(cudaStreamSynchronize(ctx->stream));
    job_free(ctx, *j);
    batch_release(ctx, job);
    return ADMS_OK;
}

adms_status adms_ctx_release_batches(adms_ctx* ctx) {
    if (!ctx) return ADMS_ERR_ARG;
    if (ctx->capturing) return fail(ctx, ADMS_ERR_STATE, "cannot release batched state during capture");
    CK(cudaStreamSynchronize(ctx->stream));
    for (BatchState& b : ctx->batches) batch_free(ctx, b);
    ctx->batches.clear();
    return ADMS_OK;
}

adms_status adms_job_reserve(adms_ctx* ctx, adms_job job, int32_t n_views, int32_t H, int32_t W) {
    Job* j = get_job(ctx, job);
    if (!j || n_views <= 0 || H <= 0 || W <= 0 || H > 16384 || W > 16384)
        return fail(ctx, ADMS_ERR_ARG, "invalid job handle or size");
    if (adms_status fs = flush_job(ctx, *j)) return fs;  // its deferred texture step first
    return ensure_scratch(ctx, *j, n_views, H, W);
}

adms_status adms_job_params(adms_ctx* ctx, adms_job job, adms_param_view* out) {
    Job* j = get_job(ctx, job);
    if (!j || !out) return fail(ctx, ADMS_ERR_ARG, "invalid job handle");
    if (adms_status fs = flush_job(ctx, *j)) return fs;  // its deferred texture step first
    memset(out, 0, sizeof(*out));
    out->pos = j->pos;
    out->kd = (float*)j->kd.data;
    out->orm = (float*)j->orm.data;
    out->nrm = (float*)j->nrm.data;
    out->g_pos = j->g_pos;
    out->g_kd = (float*)j->kd.grad;
    out->g_orm = (float*)j->orm.grad;
    out->g_nrm = (float*)j->nrm.grad;
    out->disp = j->disp;
    out->g_disp = j->g_disp;
    out->disp_h = j->dh;
    out->disp_w = j->dw;
    out->n_verts = j->LV;
    out->n_tris_render = j->F;
    out->kd_h = j->kd.h;
    out->kd_w = j->kd.w;
    out->orm_h = j->orm.h;
    out->orm_w = j->orm.w;
    out->nrm_h = j->nrm.h;
    out->nrm_w = j->nrm.w;
    out->kd_levels = j->kd.levels;
    out->orm_levels = j->orm.levels;
    out->nrm_levels = j->nrm.levels;
    JobState hs;
    CK(cudaMemcpyAsync(&hs, j->st, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    out->t = hs.t;
    out->skin_w = j->skin_w;
    out->g_skin_w = j->g_skin_w;
    out->n_bones = j->SB;
    return ADMS_OK;
}

adms_status adms_job_skinning(adms_ctx* ctx, adms_job job, const float* weights, int32_t n_bones, float lr_scale) {
    Job* jp = get_job(ctx, job);
    if (!jp || !weights || n_bones < 1 || n_bones > ADMS_MAX_BONES || !(lr_scale >= 0.f))
        return fail(ctx, ADMS_ERR_ARG, "invalid job, weights, bone count (1..1024) or learning-rate scale");
    if (adms_status fs = flush_job(ctx, *jp)) return fs;  // its deferred texture step first
    Job& j = *jp;
    if (j.tess) return fail(ctx, ADMS_ERR_STATE, "skinning of a tessellated job is not supported");
    if (j.L > 0) return fail(ctx, ADMS_ERR_STATE, "skinning of a depth-peeled job is not supported");
    if (j.skin) return fail(ctx, ADMS_ERR_STATE, "skinning is already set for this job");
    size_t nw = (size_t)j.LV * n_bones;
    AL(j.skin_w, nw);
    CK(cudaMemcpyAsync(j.skin_w, weights, nw * sizeof(float), cudaMemcpyDefault, ctx->stream));
    if (lr_scale > 0.f && !j.frozen) {
        AL(j.g_skin_w, nw);
        AL(j.m_skin_w, nw);
        AL(j.v_skin_w, nw);
        j.skin_lr_scale = lr_scale;
    }
    AL(j.bones, (size_t)n_bones * 16);
    std::vector<float> eye((size_t)n_bones * 16, 0.f);
    for (int b = 0; b < n_bones; ++b)
        for (int r = 0; r < 4; ++r) eye[(size_t)b * 16 + 5 * r] = 1.f;
    CK(cudaMemcpyAsync(j.bones, eye.data(), eye.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    AL(j.rpos, (size_t)j.V * 3);  // render positions no longer alias the rest positions
    AL(j.g_rpos, (size_t)j.V * 3);
    j.SB = n_bones;
    j.skin = true;
    j.frame_valid = false;
    CK(cudaStreamSynchronize(ctx->stream));
    return ADMS_OK;
}

adms_status adms_job_set_bones(adms_ctx* ctx, adms_job job, const float* bones) {
    Job* j = get_job(ctx, job);
    if (!j || !bones) return fail(ctx, ADMS_ERR_ARG, "invalid job handle or bones");
    if (adms_status fs = flush_job(ctx, *j)) return fs;  // its deferred texture step first
    if (!j->skin) return fail(ctx, ADMS_ERR_STATE, "the job has no skinning (adms_job_skinning)");
    CK(cudaMemcpyAsync(j->bones, bones, sizeof(float) * 16 * j->SB, cudaMemcpyDefault, ctx->stream));
    j->frame_valid = false;
    return ADMS_OK;
}

adms_status adms_jobs_status(adms_ctx* ctx, const adms_job* jobs, int32_t n_jobs, int32_t* out) {
    if (!ctx || !jobs || !out || n_jobs <= 0 || n_jobs > ADMS_STATUS_MAX)
        return fail(ctx, ADMS_ERR_ARG, "invalid jobs_status arguments");
    std::vector<JobState*> sts;
    for (int k = 0; k < n_jobs; ++k) {
        Job* j = get_job(ctx, jobs[k]);
        if (!j) return fail(ctx, ADMS_ERR_ARG, "invalid job handle");
        if (adms_status fs = flush_job(ctx, *j)) return fs;  // its deferred texture step first
        sts.push_back(j->st);
    }
    CK(gather_status(sts.data(), n_jobs, out, ctx->stream));
    return ADMS_OK;
}

adms_status adms_job_stats(adms_ctx* ctx, adms_job job, adms_stats* out) {
    Job* j = get_job(ctx, job);
    if (!j || !out) return fail(ctx, ADMS_ERR_ARG, "invalid job handle");
    if (adms_status fs = flush_job(ctx, *j)) return fs;  // its deferred texture step first
    JobState hs;
    unsigned long long ovf = 0;
    CK(cudaMemcpyAsync(&hs, j->st, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
    if (j->rs.overflow_ctr)
        CK(cudaMemcpyAsync(&ovf, j->rs.overflow_ctr, sizeof(ovf), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    out->image_loss = hs.last_img_loss;
    out->laplacian = hs.last_lap;
    out->lambda = hs.lam;
    out->lr = hs.lr;
    out->t = hs.t;
    out->status = hs.status;
    out->tile_overflows = (int64_t)ovf;
    out->call_loss = hs.call_loss;
    return ADMS_OK;
}

adms_status adms_render_reference(adms_ctx* ctx, adms_job job, const adms_view* views, int32_t n_views, int32_t H,
                                  int32_t W, float* out_rgb) {
    Job* jp = get_job(ctx, job);
    if (!jp || !views || !out_rgb || n_views <= 0 || H <= 0 || W <= 0 || H > 16384 || W > 16384)
        return fail(ctx, ADMS_ERR_ARG, "invalid render_reference arguments");
    if (adms_status fs = flush_job(ctx, *jp)) return fs;  // its deferred texture step first
    Job& j = *jp;
    adms_status s = ensure_scratch(ctx, j, n_views, H * j.S, W * j.S);
    if (s) return s;
    j.B = n_views;
    j.H = H * j.S;
    j.W = W * j.S;
    j.PH = H;
    j.PW = W;
    CK(cudaMemcpyAsync(j.views, views, sizeof(adms_view) * n_views, cudaMemcpyDefault, ctx->stream));
    if ((s = render_core(ctx, j))) return s;
    if (j.S > 1 || j.L > 0) {
        if ((s = j.L > 0 ? peel_composite(ctx, j, nullptr, nullptr, out_rgb)
                         : aa_resolve(ctx, j, nullptr, nullptr, out_rgb)))
            return s;
        j.have_fwd = false;
        return ADMS_OK;
    }
    ShadeArgs a = shade_args(j);
    a.ref = nullptr;
    a.loss_acc = nullptr;
    a.out_img = out_rgb;
    a.aa = 1;
    CK(TIMED(ST_AA_LOSS, aa_loss_forward(a, ctx->stream)));
    j.have_fwd = false;
    return ADMS_OK;
}

adms_status adms_forward_loss(adms_ctx* ctx, const adms_job* jobs, int32_t n_jobs, const adms_view* views,
                              const int32_t* views_per_job, const int32_t* hw, const float* const* ref_rgb,
                              float* out_loss, float* const* out_img) {
    if (!ctx || !jobs || n_jobs <= 0 || !views || !views_per_job || !hw || !ref_rgb)
        return fail(ctx, ADMS_ERR_ARG, "invalid forward_loss arguments");
    size_t vofs = 0;
    bool forked = false;  // a batch's frame branches, joined before its shading
    std::vector<Job*> js;
    for (int k = 0; k < n_jobs; ++k) {
        Job* jp = get_job(ctx, jobs[k]);
        int B = views_per_job[k], H = hw[2 * k], W = hw[2 * k + 1];
        if (!jp || B <= 0 || H <= 0 || W <= 0 || H > 16384 || W > 16384 || !ref_rgb[k])
            return fail(ctx, ADMS_ERR_ARG, "invalid job, view count, size or reference pointer");
        for (Job* o : js)
            if (o == jp) return fail(ctx, ADMS_ERR_ARG, "a job appears twice in one call");
        js.push_back(jp);
        Job& j = *jp;
        if (n_jobs > 1 && (j.S > 1 || j.L > 0))
            return fail(ctx, ADMS_ERR_STATE,
                        "supersampled (MSAA) and depth-peeled jobs run one per call, not in a batch");
        if ((long long)H * j.S > 16384 || (long long)W * j.S > 16384)
            return fail(ctx, ADMS_ERR_ARG, "sample grid larger than 16384 per side");
        adms_status s = ensure_scratch(ctx, j, B, H * j.S, W * j.S);
        if (s) return s;
        j.B = B;
        j.H = H * j.S;
        j.W = W * j.S;
        j.PH = H;
        j.PW = W;
        j.ref = ref_rgb[k];
        int norm_views = j.opt.batch_views > 0 ? j.opt.batch_views : B;
        j.loss_scale = (float)(1.0 / (3.0 * (double)norm_views * H * W));
        CK(cudaMemcpyAsync(j.views, views + vofs, sizeof(adms_view) * B, cudaMemcpyDefault, ctx->stream));
        vofs += B;
        CK(cudaMemsetAsync(&j.st->call_loss, 0, sizeof(double), ctx->stream));
        if (n_jobs == 1) {
            bool late = false;  // the job's deferred texture step runs beside its frame and raster
            if ((s = fork_texture_step(ctx, j, &late))) return s;
            if ((s = render_core(ctx, j, late))) return s;
            CK(wait_ref(ctx));
            if (j.L > 0) {
                if ((s = peel_composite(ctx, j, j.ref, &j.st->call_loss, out_img ? out_img[k] : nullptr))) return s;
            } else if (j.S > 1) {
                if ((s = aa_resolve(ctx, j, j.ref, &j.st->call_loss, out_img ? out_img[k] : nullptr))) return s;
            } else {
                ShadeArgs a = shade_args(j);
                a.ref = j.ref;
                a.loss_acc = &j.st->call_loss;
                a.out_img = out_img ? out_img[k] : nullptr;
                CK(TIMED(ST_AA_LOSS, aa_loss_forward(a, ctx->stream)));
            }
        } else {
            if ((s = flush_job(ctx, j))) return s;
            if ((s = frame_and_prepare(ctx, j, &forked))) return s;
        }
    }
    if (n_jobs > 1) {
        // one persistent launch per stage over the tiles of every job and view
        BatchState* bsp = nullptr;
        adms_status s = batch_upload(ctx, js, out_img, &bsp);
        if (s) return s;
        BatchState& bs = *bsp;
        CK(TIMED(ST_RASTER, raster_tiles_batched(bs.h_rargs.data(), bs.rt_off.data(), n_jobs, bs.d_rt,
                                                 batch_grid(ctx, 3), ctx->stream)));
        if (forked) CK(join_branch(ctx));
        CK(TIMED(ST_SHADE, pixels_batched(0, bs.h_args.data(), bs.px_off.data(), n_jobs, bs.d_px, ctx->tune_tw,
                                          batch_grid(ctx, 0), ctx->stream)));
        CK(wait_ref(ctx));
        CK(TIMED(ST_AA_LOSS, pixels_batched(1, bs.h_args.data(), bs.px_off.data(), n_jobs, bs.d_px, ctx->tune_tw,
                                            batch_grid(ctx, 1), ctx->stream)));
    }
    for (int k = 0; k < n_jobs; ++k) {
        CK(TIMED(ST_SMALL, finish_call_loss(js[k]->st, out_loss ? out_loss + k : nullptr, ctx->stream)));
        js[k]->have_fwd = true;
    }
    return ADMS_OK;
}

adms_status adms_backward(adms_ctx* ctx, const adms_job* jobs, int32_t n_jobs, int32_t recompute_raster) {
    if (!ctx || !jobs || n_jobs <= 0) return fail(ctx, ADMS_ERR_ARG, "invalid backward arguments");
    std::vector<Job*> js;
    for (int k = 0; k < n_jobs; ++k) {
        Job* jp = get_job(ctx, jobs[k]);
        if (!jp) return fail(ctx, ADMS_ERR_ARG, "invalid job handle");
        if (adms_status fs = flush_job(ctx, *jp)) return fs;  // its deferred texture step first
        for (Job* o : js)
            if (o == jp) return fail(ctx, ADMS_ERR_ARG, "a job appears twice in one call");
        js.push_back(jp);
        Job& j = *jp;
        if (!j.have_fwd) return fail(ctx, ADMS_ERR_STATE, "backward without a preceding forward_loss");
        if (recompute_raster) {
            // rebuild keys, pre-AA colours and dL/d(AA colour) from the latents and the
            // caller's reference images instead of reading what the forward kept
            adms_status s = render_core(ctx, j);
            if (s) return s;
            CK(wait_ref(ctx));
            if (j.L > 0) {
                if ((s = peel_composite(ctx, j, j.ref, nullptr, nullptr))) return s;
            } else if (j.S > 1) {
                if ((s = aa_resolve(ctx, j, j.ref, nullptr, nullptr))) return s;
            } else {
                ShadeArgs r = shade_args(j);
                r.ref = j.ref;
                r.loss_acc = nullptr;
                CK(TIMED(ST_AA_LOSS, aa_loss_forward(r, ctx->stream)));
            }
        }
        CK(cudaMemsetAsync(j.g_nrm, 0, sizeof(double) * 6 * j.V, ctx->stream));  // g_nrm and g_tan
        if (j.tess || j.skin) CK(cudaMemsetAsync(j.g_rpos, 0, sizeof(float) * 3 * j.V, ctx->stream));
        if (n_jobs == 1 && j.L > 0) {
            adms_status s = peel_backward(ctx, j);
            if (s) return s;
        } else if (n_jobs == 1) {
            ShadeArgs a = shade_args(j);
            a.ref = j.ref;
            CK(TIMED(ST_SHADE_BWD, shade_backward(a, ctx->stream)));
        }
    }
    if (n_jobs > 1) {
        BatchState* bsp = nullptr;
        adms_status s = batch_upload(ctx, js, nullptr, &bsp, true);
        if (s) return s;
        BatchState& bs = *bsp;
        CK(TIMED(ST_SHADE_BWD, pixels_batched(2, bs.h_args.data(), bs.px_off.data(), n_jobs, bs.d_px, ctx->tune_tw,
                                              batch_grid(ctx, 2), ctx->stream)));
    }
    for (int k = 0; k < n_jobs; ++k) {
        Job& j = *js[k];
        CK(TIMED(ST_FRAME_BWD, frame_backward(frame_args(j), ctx->stream)));
        if (j.tess) {
            // render positions -> base positions, base normals and displacement texels,
            // then the base normals' adjoint back to base positions
            CK(cudaMemsetAsync(j.g_bnrm, 0, sizeof(double) * 3 * j.LV, ctx->stream));
            CK(TIMED(ST_FRAME_BWD, tess_backward(tess_args(j), ctx->stream)));
            CK(TIMED(ST_FRAME_BWD, frame_backward(base_frame_args(j), ctx->stream)));
        }
        // skinned positions -> rest positions and weights
        if (j.skin) CK(TIMED(ST_FRAME_BWD, skin_backward(skin_args(j), ctx->stream)));
        j.have_fwd = false;
    }
    return ADMS_OK;
}

adms_status adms_optimizer_step(adms_ctx* ctx, const adms_job* jobs, int32_t n_jobs) {
    if (!ctx || !jobs || n_jobs <= 0) return fail(ctx, ADMS_ERR_ARG, "invalid optimizer_step arguments");
    std::vector<Job*> js;
    for (int k = 0; k < n_jobs; ++k) {
        Job* jp = get_job(ctx, jobs[k]);
        if (!jp) return fail(ctx, ADMS_ERR_ARG, "invalid job handle");
        if (jp->frozen) return fail(ctx, ADMS_ERR_STATE, "optimizer_step on a frozen job");
        js.push_back(jp);
    }
    for (Job* jp : js) {
        adms_status s = flush_job(ctx, *jp);  // a step not yet consumed by a forward_loss
        if (s) return s;
    }
    // schedules per job (after the Laplacian when no forward computed it for these
    // positions); then the flat latents (positions with the Laplacian term, skin
    // weights, displacement) on a branch beside the textures: every job's tiled
    // textures in one launch; then, joined, the step counters. A pipelined context
    // issues the flat latents' updates here and defers the texture step.
    for (Job* jp : js) {
        Job& j = *jp;
        if (j.opt.optimize_pos && !j.lap_valid) CK(TIMED(ST_LAPLACIAN, laplacian_forward(lap_args(j), ctx->stream)));
        SchedArgs sa{j.st, j.opt.lr0, j.opt.lambda0, j.opt.optimize_pos, j.LV};
        CK(TIMED(ST_SMALL, schedule_step(sa, ctx->stream)));
    }
    cudaStream_t bs = ctx->stream;
    if (!ctx->pipeline) {
        cudaError_t fe;
        bs = fork_branch(ctx, fe);
        CK(fe);
    }
    for (Job* jp : js) {
        Job& j = *jp;
        if (j.opt.optimize_pos) {
            CK(TIMED(ST_LAPLACIAN, laplacian_backward(lap_args(j), bs)));
            CK(TIMED(ST_ADAM, adam_flat(j.pos, j.g_pos, j.m_pos, j.v_pos, (long long)j.LV * 3, j.st, bs)));
        } else {
            CK(cudaMemsetAsync(j.g_pos, 0, sizeof(float) * 3 * j.LV, bs));
        }
        if (j.g_skin_w)
            CK(TIMED(ST_ADAM, adam_flat(j.skin_w, j.g_skin_w, j.m_skin_w, j.v_skin_w, (long long)j.LV * j.SB, j.st,
                                        bs, j.skin_lr_scale)));
        if (j.tess) {
            if (j.opt.optimize_disp)
                CK(TIMED(ST_ADAM, adam_flat(j.disp, j.g_disp, j.m_disp, j.v_disp, (long long)j.dh * j.dw, j.st, bs)));
        }
    }
    for (Job* jp : js) {
        jp->frame_valid = false;
        jp->lap_valid = false;
    }
    if (ctx->pipeline) {
        for (Job* jp : js) jp->tex_pending = true;
        return ADMS_OK;
    }
    adms_status s = texture_adams(ctx, js, ctx->stream);
    if (s) return s;
    CK(join_branch(ctx));
    for (Job* jp : js) CK(TIMED(ST_SMALL, advance_step(jp->st, ctx->stream)));
    return ADMS_OK;
}

adms_status adms_job_fold_gradients(adms_ctx* ctx, adms_job job, float* g_kd, float* g_orm, float* g_nrm) {
    Job* j = get_job(ctx, job);
    if (!j) return fail(ctx, ADMS_ERR_ARG, "invalid job handle");
    if (adms_status fs = flush_job(ctx, *j)) return fs;  // its deferred texture step first
    TexState* maps[3] = {&j->kd, &j->orm, &j->nrm};
    float* outs[3] = {g_kd, g_orm, g_nrm};
    for (int m = 0; m < 3; ++m) {
        if (!outs[m]) continue;
        if (!maps[m]->opt) return fail(ctx, ADMS_ERR_STATE, "texture is not optimized: no gradient");
        if (maps[m]->per_level)
            CK(cudaMemcpyAsync(outs[m], maps[m]->grad, sizeof(float4) * maps[m]->w * maps[m]->h,
                               cudaMemcpyDeviceToDevice, ctx->stream));
        else
            CK(fold_mip_gradient(maps[m]->dev(), reinterpret_cast<float4*>(outs[m]), ctx->stream));
    }
    return ADMS_OK;
}

adms_status adms_job_zero_gradients(adms_ctx* ctx, adms_job job) {
    Job* jp = get_job(ctx, job);
    if (!jp) return fail(ctx, ADMS_ERR_ARG, "invalid job handle");
    if (adms_status fs = flush_job(ctx, *jp)) return fs;  // its deferred texture step first
    Job& j = *jp;
    CK(cudaMemsetAsync(j.g_pos, 0, sizeof(float) * 3 * j.LV, ctx->stream));
    CK(cudaMemsetAsync(j.g_pos_acc, 0, sizeof(double) * 3 * j.V, ctx->stream));
    if (j.tess) {
        CK(cudaMemsetAsync(j.g_rpos, 0, sizeof(float) * 3 * j.V, ctx->stream));
        CK(cudaMemsetAsync(j.g_bpos_acc, 0, sizeof(double) * 3 * j.LV, ctx->stream));
    }
    if (j.skin) CK(cudaMemsetAsync(j.g_rpos, 0, sizeof(float) * 3 * j.V, ctx->stream));
    if (j.g_skin_w) CK(cudaMemsetAsync(j.g_skin_w, 0, sizeof(float) * j.LV * j.SB, ctx->stream));
    if (j.g_disp) CK(cudaMemsetAsync(j.g_disp, 0, sizeof(float) * j.dh * j.dw, ctx->stream));
    TexState* maps[3] = {&j.kd, &j.orm, &j.nrm};
    for (int m = 0; m < 3; ++m)
        if (maps[m]->grad) CK(cudaMemsetAsync(maps[m]->grad, 0, sizeof(float4) * maps[m]->total, ctx->stream));
    return ADMS_OK;
}

adms_status adms_job_invalidate(adms_ctx* ctx, adms_job job) {
    Job* j = get_job(ctx, job);
    if (!j) return fail(ctx, ADMS_ERR_ARG, "invalid job handle");
    if (adms_status fs = flush_job(ctx, *j)) return fs;  // its deferred texture step first
    TexState* maps[3] = {&j->kd, &j->orm, &j->nrm};
    for (int m = 0; m < 3; ++m)
        if (!maps[m]->per_level) CK(TIMED(ST_MIP, mip_build(maps[m]->dev(), ctx->stream)));
    j->frame_valid = false;
    j->lap_valid = false;
    return ADMS_OK;
}

adms_status adms_laplacian(adms_ctx* ctx, adms_job job, float* out_loss, float* g_pos) {
    Job* jp = get_job(ctx, job);
    if (!jp || !out_loss) return fail(ctx, ADMS_ERR_ARG, "invalid laplacian arguments");
    if (adms_status fs = flush_job(ctx, *jp)) return fs;  // its deferred texture step first
    Job& j = *jp;
    LapArgs la{j.LV, j.pos, j.ring_off, j.ring, j.delta_ref, j.delta, g_pos, j.st};
    CK(TIMED(ST_LAPLACIAN, laplacian_forward(la, ctx->stream)));
    CK(TIMED(ST_LAPLACIAN, laplacian_value(la, out_loss, ctx->stream)));
    if (g_pos) CK(TIMED(ST_LAPLACIAN, laplacian_gradient(la, 1.0f, ctx->stream)));
    return ADMS_OK;
}

adms_status adms_job_keys(adms_ctx* ctx, adms_job job, uint64_t* out_keys, size_t capacity) {
    Job* j = get_job(ctx, job);
    if (!j || !out_keys) return fail(ctx, ADMS_ERR_ARG, "invalid job handle");
    if (adms_status fs = flush_job(ctx, *j)) return fs;  // its deferred texture step first
    size_t n = (size_t)j->B * j->H * j->W * std::max(j->L, 1);
    if (capacity < n) return fail(ctx, ADMS_ERR_ARG, "key buffer too small");
    CK(cudaMemcpyAsync(out_keys, j->keys, n * sizeof(uint64_t), cudaMemcpyDefault, ctx->stream));
    return ADMS_OK;
}

adms_status adms_job_export(adms_ctx* ctx, adms_job job, void* host_buf, size_t* bytes) {
    Job* j = get_job(ctx, job);
    if (!j || !bytes) return fail(ctx, ADMS_ERR_ARG, "invalid job handle");
    if (adms_status fs = flush_job(ctx, *j)) return fs;  // its deferred texture step first
    CkptHeader h;
    std::vector<CkptSection> secs;
    ckpt_describe(*j, h, secs);
    size_t total = sizeof(CkptHeader);
    for (const CkptSection& c : secs) total += c.bytes;
    if (!host_buf) {
        *bytes = total;
        return ADMS_OK;
    }
    if (*bytes < total) return fail(ctx, ADMS_ERR_ARG, "checkpoint buffer too small");
    CK(cudaStreamSynchronize(ctx->stream));
    unsigned char* out = static_cast<unsigned char*>(host_buf);
    memcpy(out, &h, sizeof(h));
    size_t off = sizeof(h);
    for (const CkptSection& c : secs) {
        CK(cudaMemcpy(out + off, c.ptr, c.bytes, cudaMemcpyDeviceToHost));
        off += c.bytes;
    }
    *bytes = total;
    return ADMS_OK;
}

adms_status adms_job_import(adms_ctx* ctx, const adms_mesh_desc* mesh, const adms_material_desc* mat,
                            const adms_opt_params* opt, const void* host_buf, size_t bytes, adms_job* out) {
    if (!ctx || !host_buf || !out) return fail(ctx, ADMS_ERR_ARG, "null argument");
    if (bytes < sizeof(CkptHeader)) return fail(ctx, ADMS_ERR_ARG, "checkpoint shorter than its header");
    CkptHeader want;
    memcpy(&want, host_buf, sizeof(want));
    if (memcmp(want.magic, kCkptMagic, 8) != 0 || want.version != kCkptVersion)
        return fail(ctx, ADMS_ERR_ARG, "not an adms checkpoint of this version");
    adms_job h = -1;
    adms_status s = adms_job_create(ctx, mesh, mat, opt, want.seed, &h);
    if (s) return s;
    if (want.n_bones > 0) {  // skinning is set after creation: set it up, the blob brings its weights
        std::vector<float> zeros((size_t)ctx->jobs[h].LV * want.n_bones, 0.f);
        s = adms_job_skinning(ctx, h, zeros.data(), want.n_bones, want.skin_lr_scale);
        if (s) {
            adms_job_destroy(ctx, h);
            return s;
        }
    }
    Job& j = ctx->jobs[h];
    CkptHeader got;
    std::vector<CkptSection> secs;
    ckpt_describe(j, got, secs);
    size_t total = sizeof(CkptHeader);
    for (const CkptSection& c : secs) total += c.bytes;
    if (memcmp(&got, &want, sizeof(CkptHeader)) != 0 || total != bytes) {
        adms_job_destroy(ctx, h);
        return fail(ctx, ADMS_ERR_ARG, "checkpoint does not match the mesh, textures or options given");
    }
    const unsigned char* in = static_cast<const unsigned char*>(host_buf);
    size_t off = sizeof(CkptHeader);
    for (const CkptSection& c : secs) {
        cudaError_t e = cudaMemcpy(c.ptr, in + off, c.bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            adms_job_destroy(ctx, h);
            return fail(ctx, ADMS_ERR_CUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
        }
        off += c.bytes;
    }
    j.frame_valid = false;
    j.lap_valid = false;
    j.have_fwd = false;
    *out = h;
    return ADMS_OK;
}

adms_status adms_graph_begin(adms_ctx* ctx) {
    if (!ctx || ctx->capturing) return fail(ctx, ADMS_ERR_STATE, "already capturing");
    if (!ctx->stream) return fail(ctx, ADMS_ERR_STATE, "graph capture needs a non-default stream");
    if (ctx->profile) return fail(ctx, ADMS_ERR_STATE, "disable stage profiling before capturing");
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    ctx->capturing = true;
    ctx->cap_pending = pending_jobs(ctx);
    return ADMS_OK;
}

adms_status adms_graph_end(adms_ctx* ctx, adms_graph** out) {
    if (!ctx || !out || !ctx->capturing) return fail(ctx, ADMS_ERR_STATE, "not capturing");
    ctx->capturing = false;
    adms_graph* g = new adms_graph();
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g->graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) {
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return fail(ctx, ADMS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    g->pend_begin = ctx->cap_pending;
    g->pend_end = pending_jobs(ctx);
    *out = g;
    return ADMS_OK;
}

adms_status adms_graph_launch(adms_ctx* ctx, adms_graph* g) {
    if (!ctx || !g) return fail(ctx, ADMS_ERR_ARG, "null graph");
    if (pending_jobs(ctx) != g->pend_begin)
        return fail(ctx, ADMS_ERR_STATE,
                    "the graph was captured with another set of jobs holding a deferred texture step");
    CK(cudaGraphLaunch(g->exec, ctx->stream));
    for (adms_job h : g->pend_begin) ctx->jobs[h].tex_pending = false;
    for (adms_job h : g->pend_end) ctx->jobs[h].tex_pending = true;
    return ADMS_OK;
}

adms_status adms_ctx_set_pipelining(adms_ctx* ctx, int32_t enable) {
    if (!ctx) return ADMS_ERR_ARG;
    if (ctx->capturing) return fail(ctx, ADMS_ERR_STATE, "cannot change pipelining during capture");
    if (!enable)
        if (adms_status fs = flush_all(ctx)) return fs;
    ctx->pipeline = enable != 0;
    return ADMS_OK;
}

adms_status adms_graph_destroy(adms_graph* g) {
    if (!g) return ADMS_ERR_ARG;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return ADMS_OK;
}

adms_status adms_ctx_test_wait_timeout(adms_ctx* ctx, int32_t enable) {
    if (!ctx) return ADMS_ERR_ARG;
    ctx->adam_extra_tx = enable ? 16u : 0u;
    return ADMS_OK;
}

adms_status adms_ctx_profile(adms_ctx* ctx, int32_t enable) {
    if (!ctx) return ADMS_ERR_ARG;
    ctx->profile = enable != 0;
    return ADMS_OK;
}

adms_status adms_ctx_stage_times(adms_ctx* ctx, double* ms_out, int64_t* launches_out, int32_t n_stages) {
    if (!ctx || !ms_out || n_stages < ST_COUNT) return fail(ctx, ADMS_ERR_ARG, "stage buffer too small");
    CK(cudaStreamSynchronize(ctx->stream));
    for (const StageRec& r : ctx->recs) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, r.a, r.b));
        ctx->stage_ms[r.stage] += ms;
        ctx->stage_n[r.stage] += 1;
    }
    ctx->recs.clear();
    ctx->pool_used = 0;
    for (int s = 0; s < ST_COUNT; ++s) {
        ms_out[s] = ctx->stage_ms[s];
        if (launches_out) launches_out[s] = ctx->stage_n[s];
        ctx->stage_ms[s] = 0.0;
        ctx->stage_n[s] = 0;
    }
    return ADMS_OK;
}

adms_status adms_mesh_topology(const int32_t* tri, int32_t n_verts, int32_t n_tris, int32_t* adj, int32_t* vf_off,
                               int32_t* vf_face) {
    if (!tri || !adj || !vf_off || !vf_face || n_verts <= 0 || n_tris <= 0) return ADMS_ERR_ARG;
    std::vector<int> t(tri, tri + (size_t)3 * n_tris);
    for (int x : t)
        if (x < 0 || x >= n_verts) return ADMS_ERR_ARG;
    std::vector<int> a, off, face, ring_off, ring;
    build_topology(t, n_verts, n_tris, a, off, face, ring_off, ring);
    std::copy(a.begin(), a.end(), adj);
    std::copy(off.begin(), off.end(), vf_off);
    std::copy(face.begin(), face.end(), vf_face);
    return ADMS_OK;
}

adms_status adms_tessellation(const int32_t* tri, const int32_t* tri_uv, const float* uv, int32_t n_verts, int32_t n_uv,
                              int32_t n_tris, int32_t levels, int32_t* counts, int32_t* rtri, int32_t* rtri_uv,
                              float* ruv, int32_t* owner, int32_t* wts, float* vert_uv) {
    if (!tri || !tri_uv || !uv || !counts || n_verts <= 0 || n_uv <= 0 || n_tris <= 0 || levels < 1 || levels > 8)
        return ADMS_ERR_ARG;
    std::vector<int> t(tri, tri + (size_t)3 * n_tris), tu(tri_uv, tri_uv + (size_t)3 * n_tris);
    for (int x : t)
        if (x < 0 || x >= n_verts) return ADMS_ERR_ARG;
    for (int x : tu)
        if (x < 0 || x >= n_uv) return ADMS_ERR_ARG;
    TessHost h;
    build_tessellation(t, tu, std::vector<float>(uv, uv + (size_t)2 * n_uv), n_tris, levels, h);
    int Ft = (int)h.rtri.size() / 3;
    bool fill = rtri || rtri_uv || ruv || owner || wts || vert_uv;
    if (fill) {
        if (!rtri || !rtri_uv || !ruv || !owner || !wts || !vert_uv) return ADMS_ERR_ARG;
        if (counts[0] < h.Vt || counts[1] < Ft || counts[2] < (int)h.corner_uv.size() / 2) return ADMS_ERR_ARG;
        std::copy(h.rtri.begin(), h.rtri.end(), rtri);
        std::copy(h.rtri_uv.begin(), h.rtri_uv.end(), rtri_uv);
        std::copy(h.corner_uv.begin(), h.corner_uv.end(), ruv);
        std::copy(h.owner.begin(), h.owner.end(), owner);
        std::copy(h.wts.begin(), h.wts.end(), wts);
        std::copy(h.vert_uv.begin(), h.vert_uv.end(), vert_uv);
    }
    counts[0] = h.Vt;
    counts[1] = Ft;
    counts[2] = (int)h.corner_uv.size() / 2;
    return ADMS_OK;
}

int32_t adms_stage_count(void) { return ST_COUNT; }

const char* adms_stage_name(int32_t i) { return (i >= 0 && i < ST_COUNT) ? kStageNames[i] : ""; }

int64_t adms_launch_count(void) { return (int64_t)g_launches.load(); }

}  // extern "C"
