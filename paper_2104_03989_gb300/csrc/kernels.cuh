// Kernel-side data structures and host launchers of the render-and-compare step.
#pragma once

#include <algorithm>
#include <atomic>
#include <cstring>
#include <vector>

#include <cuda.h>  // CUtensorMap

#include "common.cuh"

namespace adms {

// kernels launched by this library in this process (counted on the host at each launch)
inline std::atomic<long long> g_launches{0};
inline void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// transformed vertex of one view: snapped sub-pixel position, depth, usable flag
struct VtxS {
    int X, Y;
    float z;
    int ok;
};

// triangle setup record of one view: oriented edge functions s E_k = ea Sx + eb Sy + ec
// (s = sign of the snapped area), fill-rule thresholds, depth plane, pixel bbox
struct TriRec {
    long long ec[3];
    int ea[3], eb[3];
    int thr[3];
    float fA, z0, dz1, dz2;
    int sg, id, valid;
    short bx0, bx1, by0, by1;
};

// pixel bounding box of a binned triangle of one view; empty (bx0 > bx1) for
// triangles rasterized by the small-triangle pass or not drawn at all
struct TriBin {
    short bx0, bx1, by0, by1;
};

// triangles with at most this many samples in their pixel bbox skip binning (default)
#define ADMS_SMALL_PX 16

struct RasterIn {
    const float* pos;          // [V][3] render positions
    const int* tri;            // [F][3]
    const int* adj;            // [F][3] face across edge k, or -1
    const adms_view* views;    // device, [B]
    int B, V, F, W, H;
    unsigned long long* keys;  // [B][H][W]
    int small_px = ADMS_SMALL_PX;  // triangles with at most this many samples in their bbox are
                                   // rasterized directly (atomicMin), the rest binned into tiles
    int zfilter = 0;  // small_px > ADMS_SMALL_PX: read each sample's stored key before its test
};

// scratch of the raster (global memory beyond inputs and outputs)
struct RasterScratch {
    float4* clip;       // [B][V]
    float4* scr;        // [B][V] screen position as (x_hi, x_lo, y_hi, y_lo) float pairs
    VtxS* vs;           // [B][V]
    TriRec* rec;        // [B][F] (written for binned triangles only)
    TriBin* bin;        // [B][F]
    int8_t* asign;      // [B][F]
    uint8_t* silmask;   // [B][F] bit e: edge e is a silhouette edge in that view
    int* tile_count;    // [B * tiles]
    int* tile_off;      // [B * tiles]
    int* tile_cursor;   // [B * tiles]
    int* list;          // [list_capacity]
    long long list_capacity;
    long long* total_pairs;               // device scalar
    unsigned long long* overflow_ctr;     // device scalar
};

cudaError_t raster_views(const RasterIn& in, RasterScratch& s, cudaStream_t st);
// transform, setup, tile counts, scan and tile lists (in.keys may be null when
// in.small_px is 0: nothing is then rasterized directly and the keys are untouched)
cudaError_t raster_prepare(const RasterIn& in, RasterScratch& s, cudaStream_t st);
// the per-tile z-buffer pass
cudaError_t raster_tiles(const RasterIn& in, RasterScratch& s, cudaStream_t st);
// depth peeling (Sec. 5.2) in one tile pass: in.keys receives L slices of [B][H][W],
// slice l the (l+1)-th nearest fragment per sample (EMPTY beyond the last); needs
// raster_prepare with small_px = 0 (every triangle binned); L in [1, 16]
cudaError_t raster_tiles_peeled(const RasterIn& in, RasterScratch& s, int L, cudaStream_t st);

// everything the per-pixel shading, AA, loss and backward kernels read
struct ShadeArgs {
    int B, H, W, V, F;
    const adms_view* views;          // [B]
    const float4* clip;              // [B][V]
    const float4* scr;               // [B][V] (x_hi, x_lo, y_hi, y_lo)
    const float4* vpos;              // [V] xyz
    const float4* vnrm;              // [V] unit smooth normals
    const float4* vtan;              // [V] unit tangents
    const float2* uv;                // [T]
    const int* tri;                  // [F][3]
    const int* tri_uv;               // [F][3]
    int* status;                     // the job's latched status word (JobState::status), or null: set to
                                     // ADMS_ERR_NONFINITE when a vertex gradient sum is NaN or infinite
    const uint8_t* silmask;          // [B][F]
    const unsigned long long* keys;  // [B][H][W]
    TexDev kd, orm, nrm;
    float4* pre;                     // [B][H][W] pre-AA colour
    const float* ref;                // [B][H][W][3]
    int msaa;                        // s > 1: keys, pre, gprime are on an s x s sample grid per pixel
                                     // and each sample is shaded at its pixel's centre, LOD of the pixel
    int peel;                        // a layer of a depth-peeled composite: pre.w is the layer's opacity
                                     // and the colour AA acts on is opacity x pre + (1 - opacity) x under
    float4* acol;                    // [B][H][W] antialiased sample colours (w: the blend mask bits) for
                                     // the per-pixel resolve, or null
    int* refine;                     // [0]: count, then pixel indices shaded again with a refined
                                     // texture coordinate (null: none)
    float4* gprime;                  // [B][H][W] dL/d(AA colour) in xyz; w: bit n set (as raw bits)
                                     // when the pair with neighbour n (-x, +x, -y, +y) blended
    const float4* under;             // peel: [B][H][W] the composite of the layers behind (xyz; w: its
                                     // blend mask bits), or null for the black background
    float4* g_under;                 // peel backward: [B][H][W] dL/d(under) with under's blend mask in
                                     // w (the next layer's gprime), or null for the last layer
    float* out_img;                  // [B][H][W][3] or null
    int loss_kind;
    float loss_scale;                // 1 / (3 P)
    int aa;
    double* loss_acc;                // device scalar (sum of per-pixel losses times loss_scale)
    double* g_pos;                   // [V][3] accumulated in float64
    double* g_nrm;                   // [V][3] d/d(unit normal)
    double* g_tan;                   // [V][3] d/d(unit tangent)
    double* g_clip;                  // per-stage calls: [B][V][4] d/d(clip coordinates), or null
};

cudaError_t shade_forward(const ShadeArgs& a, cudaStream_t st);
cudaError_t aa_loss_forward(const ShadeArgs& a, cudaStream_t st);
cudaError_t shade_backward(const ShadeArgs& a, cudaStream_t st);

// per-pixel resolve of a supersampled render: pixel = mean of its s x s antialiased
// samples; with a reference, the loss per pixel and each sample's share of
// dL/d(colour) (into gprime.xyz; gprime.w keeps the sample's blend mask)
struct ResolveArgs {
    int B, H, W, S;        // pixels per view H x W, samples per axis S
    const float4* acol;    // [B][S H][S W]
    const float* ref;      // [B][H][W][3] or null
    float4* gprime;        // [B][S H][S W]
    float* out_img;        // [B][H][W][3] or null
    double* loss_acc;      // or null
    int loss_kind;
    float loss_scale;      // 1 / (3 P), P pixels
};
cudaError_t resolve_loss(const ResolveArgs& r, cudaStream_t st);

// one unit of work of a batched launch: a tile of one view of one job
struct WorkItem {
    int job, view, x0, y0;
};
// Jobs per batched launch: their arguments travel in the launch's parameter
// space (60 x 536 B, under the 32 KB limit), read-only and captured with the
// launch by a graph; larger job sets take one launch per 60 jobs.
#define ADMS_BATCH_JOBS 60
struct ShadeBatch {
    ShadeArgs a[ADMS_BATCH_JOBS];
};
static_assert(sizeof(ShadeBatch) + 64 <= 32764, "batched launch parameters exceed the kernel parameter space");
// persistent launch over work items of many jobs; kind 0 shade, 1 AA + loss, 2 backward.
// args: host array of n_jobs arguments; items (device) are ordered by job, job k's
// items being [item_off[k], item_off[k+1]) (item_off: host, n_jobs + 1 entries);
// tiles are tw x (256 / tw) pixels; blocks should not exceed the resident count
cudaError_t pixels_batched(int kind, const ShadeArgs* args, const int* item_off, int n_jobs, const WorkItem* items,
                           int tw, int blocks, cudaStream_t st);
// resident blocks per SM of the persistent launches: kind 0-2 as above, 3 the raster
int batched_occupancy(int kind);

// per-job arguments of the tile raster
struct RasterJob {
    const TriRec* rec;
    const TriBin* bin;
    int F, W, H, tiles_x, tiles_y;
    const int* tile_off;
    const int* tile_count;
    const int* list;
    long long capacity;
    unsigned long long* keys;
    unsigned long long* overflow_ctr;
};
struct RasterBatch {
    RasterJob a[ADMS_BATCH_JOBS];
};
// persistent launch of the 16x16-tile raster over (job, view, tile) items; arguments
// and item ranges as for pixels_batched
cudaError_t raster_tiles_batched(const RasterJob* args, const int* item_off, int n_jobs, const WorkItem* items,
                                 int blocks, cudaStream_t st);
int raster_batch_occupancy();

// mesh frame (smooth normals, tangents) and its adjoint
struct FrameArgs {
    int V, F;
    const float* pos;     // [V][3]
    const float2* uv;     // [T]
    const int* tri;       // [F][3]
    const int* tri_uv;    // [F][3]
    const int* vf_off;    // [V+1] vertex -> incident faces CSR
    const int* vf_face;   // [sum]
    float4* vpos;         // out [V]
    float4* vnrm;         // out [V]
    float4* vtan;         // out [V]
    const double* g_nrm;  // in  [V][3]
    const double* g_tan;  // in  [V][3]
    float4* tmp_n;        // scratch [V]
    float4* tmp_t;        // scratch [V]
    double* g_pos_acc;    // in  [V][3] pixel-stage position gradient; read and zeroed
    float* g_pos;         // accumulated [V][3]
    int* status = nullptr; // latched ADMS_ERR_NONFINITE when a position gradient is NaN or infinite
    // optional [V]: 1/|sum| of each vertex's normal (x) and tangent (y) sums, negated
    // where the squared sum is at or below the normalisation floor; written by
    // frame_forward when set, after which frame_backward is one launch
    float2* inv = nullptr;
};
cudaError_t frame_forward(const FrameArgs& a, cudaStream_t st);
cudaError_t frame_backward(const FrameArgs& a, cudaStream_t st);

// tessellation + displacement (latent base mesh -> render mesh) and its adjoint
// dense skinning (Eq. 2) of the rest positions by the frame's bones
#define ADMS_MAX_BONES 1024  // 12 floats of shared memory per bone
struct SkinArgs {
    int V, B;
    const float* pos;    // [V][3] rest positions (latent)
    const float* w;      // [V][B] weights (latent)
    const float* bones;  // [B][16] row-major affine bone matrices of the frame
    float* out;          // [V][3] skinned (render) positions
    const float* g_out;  // [V][3] dL/d(skinned positions)
    float* g_pos;        // [V][3] += dL/d(rest positions)
    float* g_w;          // [V][B] += dL/dw (null: weights not optimized)
};
cudaError_t skin_forward(const SkinArgs& a, cudaStream_t st);
cudaError_t skin_backward(const SkinArgs& a, cudaStream_t st);

struct TessArgs {
    int Vb, Fb, Vt, n_seg;
    const float* base_pos;   // [Vb][3] latent
    const int* base_tri;     // [Fb][3]
    const int* bvf_off;      // [Vb+1] base vertex -> incident faces (ascending)
    const int* bvf_face;
    float* base_nrm;         // [Vb][3] base normals (float32 contract)
    const int* owner;        // [Vt][3] base vertices of the owning base face
    const int* wts;          // [Vt][3] integer lattice weights (sum n_seg)
    const float2* vert_uv;   // [Vt] displacement lookup coordinates
    const float* disp;       // [dh][dw] latent displacement map
    int dh, dw;
    float* pos_out;          // [Vt][3] render positions
    const float* g_pos_t;    // [Vt][3] gradient w.r.t. render positions
    double* g_base_pos;      // [Vb][3] accumulated
    double* g_base_nrm;      // [Vb][3] accumulated
    float* g_disp;           // [dh][dw] accumulated, or null
};
cudaError_t tess_forward(const TessArgs& a, cudaStream_t st);
cudaError_t tess_backward(const TessArgs& a, cudaStream_t st);

// device-side per-job scalars
struct JobState {
    double call_loss;    // L_image of the current forward call
    double img_loss;     // accumulated L_image since the last optimizer step
    double lap_sum;      // sum_i |delta_i - delta'_i|^2
    float lam, lam0, lr, bc1, bc2;
    float last_img_loss, last_lap;
    int t;
    int status;        // 0 or a latched adms_status; constant during an optimizer step
    int status_next;   // latched by the optimizer step's kernels, folded into status when t advances
};

struct LapArgs {
    int V;
    const float* pos;       // [V][3]
    const int* ring_off;    // [V+1]
    const int* ring;        // one-ring CSR
    const float* delta_ref; // [V][3] or null (absolute)
    float* delta;           // scratch [V][3]
    float* g_pos;           // [V][3]
    JobState* st;
};
cudaError_t laplacian_forward(const LapArgs& a, cudaStream_t st);
cudaError_t laplacian_backward(const LapArgs& a, cudaStream_t st);
// *out = L_delta after laplacian_forward
cudaError_t laplacian_value(const LapArgs& a, float* out, cudaStream_t st);
// a.g_pos = scale * dL_delta/dpos (overwrites) after laplacian_forward
cudaError_t laplacian_gradient(const LapArgs& a, float scale, cudaStream_t st);
// level-0 texture gradient with the mip-chain adjoint folded in
cudaError_t fold_mip_gradient(const TexDev& t, float4* out, cudaStream_t st);

struct SchedArgs {
    JobState* st;
    float lr0, lambda0_user;  // <= 0: heuristic
    int has_pos;
    int n_verts;
};
cudaError_t schedule_step(const SchedArgs& a, cudaStream_t st);

// Adam on a flat float array (positions, displacement): no clamps
cudaError_t adam_flat(float* p, float* g, float* m, float* v, long long n, const JobState* js, cudaStream_t st,
                      float lr_scale = 1.f);
// Adam on a float4 texture (level 0) with the mip-chain adjoint folded in; clamp_kind 0 kd, 1 orm, 2 nrm
cudaError_t adam_texture(const TexDev& t, float4* m, float4* v, int clamp_kind, const JobState* js, cudaStream_t st);
// Adam on every level of a texture whose mip levels are independent latents (m, v
// hold the whole chain); no mip adjoint, no rebuild
cudaError_t adam_texture_levels(const TexDev& t, float4* m, float4* v, int clamp_kind, const JobState* js,
                                cudaStream_t st);
// rebuild levels 1.. of a mip chain from level 0 (2x2 box average)
cudaError_t mip_build(const TexDev& t, cudaStream_t st);
// Adam on a texture, then the rebuild of its mip chain (textures that do not tile)
cudaError_t adam_texture_and_mips(const TexDev& t, float4* m, float4* v, int clamp_kind, const JobState* js,
                                  cudaStream_t st);
// one optimized texture of a tiled Adam launch
struct TexAdam {
    TexDev t;
    float4* m;
    float4* v;
    const JobState* js;
    int clamp_kind;  // 0 kd, 1 orm, 2 nrm
    int tile0;       // set by the launcher
    const CUtensorMap* tmaps = nullptr;  // host CUtensorMap[4]: level 0 of grad, tex, m, v (adam_encode_maps)
};
// textures per launch: their arguments and tensor maps are kernel parameters (< 32 KB)
#define ADMS_ADAM_TEX 40
struct TexAdamBatch {
    CUtensorMap maps[ADMS_ADAM_TEX][4];  // grad, tex, m, v of texture k
    TexAdam a[ADMS_ADAM_TEX];
    int n;
    uint32_t extra_tx;  // test hook: bytes each tile's wait expects beyond its copies (0)
};
// whether a texture takes the tiled path (both sides multiples of 32, at least 6 levels)
bool adam_tiled(const TexDev& t);
// the streamed Adam's shared-memory limit (called once per process before its first launch)
cudaError_t adam_prepare();
// host: the tensor maps of level 0 of a tiled texture's gradient, latents and
// moments (float4 texels as float32 x 4, boxes of 32 texels x 32 rows)
cudaError_t adam_encode_maps(const TexDev& t, const float4* m, const float4* v, CUtensorMap out[4]);
// Adam + mip rebuild of every listed texture (all adam_tiled, any jobs), one 32x32-texel
// tile per block, one launch per ADMS_ADAM_TEX textures
cudaError_t adam_textures_tiled(std::vector<TexAdam>& list, cudaStream_t st, uint32_t extra_tx = 0);
cudaError_t advance_step(JobState* js, cudaStream_t st);
// out[k] = the latched status of job k (stream-ordered; out: device [n])
#define ADMS_STATUS_MAX 512
cudaError_t gather_status(JobState* const* js, int n, int* out, cudaStream_t st);
// out[j] = call_loss; img_loss += call_loss
cudaError_t finish_call_loss(JobState* js, float* out, cudaStream_t st);

}  // namespace adms
