/*
 * adms.h — C ABI of the GB300 (sm_103a) render-and-compare library for
 * appearance-driven mesh simplification (Hasselgren et al., "Appearance-Driven
 * Automatic 3D Model Simplification").
 *
 * The calls follow the paper's statement of the problem (Sec. 3, Eq. 1):
 * a latent mesh with textures is rendered under random cameras and lights,
 * compared with renders of a reference, differentiated, and updated by Adam.
 *
 *   adms_render_reference  — forward render of a (frozen) job        (Sec. 3, reference renderer)
 *   adms_forward_loss      — render + silhouette AA + image loss      (Sec. 5.1, 5.2, 5.3)
 *   adms_backward          — gradients w.r.t. every latent            (Sec. 3: dL/dtheta)
 *   adms_optimizer_step    — Laplacian term, lambda/lr schedules, Adam (Eq. 4, Eq. 5, Sec. 5.3)
 *
 * Conventions
 *   - Every call returns an adms_status; nothing throws across the ABI.
 *     adms_last_error() describes the latest failure of a context.
 *   - Pointers: "device" = CUDA device memory of the context's GPU; "any" =
 *     host or device memory (copied with cudaMemcpyDefault). The caller owns
 *     every buffer it passes; the library owns each job's resident state
 *     (mesh, textures with mip chains, gradients, Adam moments, scratch).
 *   - All GPU work is ordered on the context's CUDA stream and asynchronous
 *     unless stated otherwise. Inputs passed to adms_forward_loss (reference
 *     images) must stay valid until the matching adms_backward has been
 *     enqueued; views are copied in.
 *   - A context is used by one host thread at a time.
 *
 * Layouts
 *   - positions: float32 [V][3]; UV corners: float32 [T][2];
 *     triangles: int32 [F][3] position indices and int32 [F][3] UV indices
 *     (separate index buffers, so UV seams do not split positions).
 *   - textures: float32 [h][w][4] (row = v, column = u), level 0 only;
 *     h and w powers of two. Base colour (r, g, b, alpha); specular
 *     (gamma, r, m, unused); tangent-space normal (x, y, z, unused).
 *     displacement: float32 [h][w] (tessellated jobs only).
 *   - images: float32 [B][H][W][3], row 0 at the top.
 *   - keys: uint64 [B][H][W]; (float_bits(depth) << 32) | triangle id, all
 *     ones for an empty pixel.
 */
#ifndef ADMS_H
#define ADMS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ADMS_OK = 0,
    ADMS_ERR_ARG = -1,       /* invalid argument (null pointer, size, handle) */
    ADMS_ERR_BUDGET = -2,    /* allocation would exceed the context's HBM budget */
    ADMS_ERR_CUDA = -3,      /* a CUDA runtime call failed */
    ADMS_ERR_TIMEOUT = -4,   /* a bounded device wait gave up */
    ADMS_ERR_NONFINITE = -5, /* a loss or gradient was NaN/Inf: latched in the job's status on the
                                device (see adms_jobs_status), its optimizer steps are skipped */
    ADMS_ERR_STATE = -6      /* call out of order (e.g. backward before forward) */
} adms_status;

typedef struct adms_ctx adms_ctx;
typedef int32_t adms_job;

/* One camera and its lights, 112 bytes. clip = mvp * [x y z 1]^T (row-major,
 * OpenGL conventions); screen x = (clip.x/clip.w)(W/2) + W/2,
 * y = H/2 - (clip.y/clip.w)(H/2). A light with zero strength is off. */
typedef struct {
    float mvp[16];
    float eye[3];
    float pad0;
    float light_pos[3]; /* point light position */
    float light_I;      /* point light intensity; irradiance I / d^2 */
    float light_dir[3]; /* unit vector towards the directional light */
    float light_E;      /* directional irradiance */
} adms_view;

typedef struct {
    int32_t n_verts, n_uv, n_tris;
    const float* pos;       /* any, [n_verts][3] */
    const float* uv;        /* any, [n_uv][2] */
    const int32_t* tri_pos; /* any, [n_tris][3] */
    const int32_t* tri_uv;  /* any, [n_tris][3] */
} adms_mesh_desc;

typedef struct {
    const float* kd;   /* any, [kd_h][kd_w][4] */
    const float* orm;  /* any, [orm_h][orm_w][4] */
    const float* nrm;  /* any, [nrm_h][nrm_w][4] */
    const float* disp; /* any, [disp_h][disp_w] or NULL */
    int32_t kd_h, kd_w, orm_h, orm_w, nrm_h, nrm_w, disp_h, disp_w;
    int32_t mips;      /* 1: full mip chains and trilinear filtering; 0: level 0 only */
} adms_material_desc;

enum { ADMS_LOSS_L1 = 0, ADMS_LOSS_LOGL1 = 1, ADMS_LOSS_L2 = 2 };

typedef struct {
    int32_t optimize_pos, optimize_kd, optimize_orm, optimize_nrm, optimize_disp; /* 0/1 */
    int32_t loss;            /* ADMS_LOSS_* */
    int32_t tess_levels;     /* edge-midpoint subdivisions of the base mesh (0 = none) */
    int32_t batch_views;     /* views per optimizer step for the loss mean (0 = views of each call) */
    int32_t relative_laplacian; /* 1: delta' = delta of the initial mesh; 0: absolute (delta' = 0) */
    int32_t aa;              /* 1: silhouette antialiasing (default), 0: off */
    float lr0;               /* initial learning rate (Sec. 5.3), e.g. 0.01 */
    float lambda0;           /* initial Laplacian weight; <= 0 selects 0.25 L_image / L_delta at t = 0 */
    int32_t per_level_textures; /* 1: every mip level of each optimized texture is its own latent
                                  (Sec. 6, prefiltering for several rendering resolutions): the
                                  levels start as the box-filter chain of the given level 0, each
                                  level takes its own gradient and Adam moments, and nothing is
                                  folded or rebuilt; needs mips. 0: one latent per texture (level
                                  0), coarser levels are its box-filter chain */
    int32_t samples;         /* s in [2, 8]: s x s visibility samples per pixel (Sec. 5.2,
                                antialiasing): raster, shading and silhouette antialiasing on the
                                sample grid, each pixel the mean of its samples, the loss per
                                pixel; 0 or 1: one sample per pixel. Such a job runs one per
                                forward_loss / backward call (not batched); adms_job_keys returns
                                the sample grid's keys */
    int32_t shade_samples;   /* with samples > 1: 0 = MSAA, each sample takes its triangle shaded
                                once per pixel at the pixel's centre with the pixel's LOD (the
                                training render); 1 = every sample shaded at its own position (a
                                supersampled render, e.g. for reference images) */
    int32_t layers;          /* L in [1, 16]: order-independent transparency by L depth-peeling
                                passes (Sec. 5.2; the aggregate-geometry application of Sec. 6).
                                Layer 0 is the nearest fragment per pixel, layer l the nearest
                                one whose depth|id key is strictly greater than layer l-1's; each
                                layer is shaded and takes its opacity from the base colour's
                                fourth channel; blending runs back to front from a black
                                background, each layer's composite antialiased with that layer's
                                visibility, and the loss is taken on the front composite.
                                Plain meshes only (no tessellation, skinning or samples > 1); runs
                                one job per forward_loss / backward call; adms_job_keys returns
                                the L layers' keys, layer after layer. 0: opaque rendering, the
                                fourth channel unused */
    int32_t raster_direct_px; /* raster tuning (no counterpart in the paper; results do not depend on
                                it): triangles whose pixel bounding box holds at most this many
                                samples are rasterized one thread per triangle with a 64-bit atomicMin
                                per covered sample, larger ones binned into 16x16 tiles. 0 = 16.
                                Dense clouds of small triangles (e.g. a 1.2M-triangle foliage
                                reference) run faster with a few hundred. Ignored with layers > 0
                                (every triangle is binned). In [0, 4096] */
    int32_t raster_depth_filter; /* raster tuning with raster_direct_px > 16 (results do not depend on
                                it): 1 = the direct raster reads each sample's stored key first and
                                skips the coverage test when the triangle's depth floor cannot beat
                                it (pays where many fragments land on each sample, e.g. foliage);
                                0 = every covered sample goes straight to atomicMin (closed
                                surfaces, about two fragments per sample). 0 or 1 */
} adms_opt_params;

/* Device pointers into a job's resident state (owned by the library, valid
 * until adms_job_destroy). Texture and texture-gradient pointers address the
 * whole mip chain, level after level (level k is [max(h>>k,1)][max(w>>k,1)][4]);
 * gradients hold the latest backward's result per level until the next
 * optimizer step folds the coarser levels into level 0 (the adjoint of the
 * box filter) and zeroes them. */
typedef struct {
    float *pos, *kd, *orm, *nrm, *disp;
    float *g_pos, *g_kd, *g_orm, *g_nrm, *g_disp;
    int32_t n_verts, n_tris_render, kd_h, kd_w, orm_h, orm_w, nrm_h, nrm_w, disp_h, disp_w;
    int32_t kd_levels, orm_levels, nrm_levels; /* mip levels held per texture (1 = level 0 only) */
    int32_t t;            /* optimizer steps taken */
    float *skin_w, *g_skin_w; /* skinning weights [n_verts][n_bones] and their gradient (NULL if none) */
    int32_t n_bones;      /* 0 without skinning */
} adms_param_view;

/* Job state scalars, read back with adms_job_stats (synchronises the stream). */
typedef struct {
    float image_loss;     /* L_image of the latest step's forward calls (summed over calls) */
    float laplacian;      /* L_delta at the latest optimizer step */
    float lambda;         /* lambda_t used at the latest optimizer step */
    float lr;             /* lr_t used at the latest optimizer step */
    int32_t t;            /* optimizer steps taken */
    int32_t status;       /* 0, or an adms_status latched on the device */
    int64_t tile_overflows; /* raster tiles that fell back to a full triangle scan */
    double call_loss;     /* L_image of the latest forward_loss call, float64 accumulation */
} adms_stats;

/* ---- context ------------------------------------------------------------- */

/* Create a context on the current CUDA device. hbm_budget_bytes bounds the
 * library's own allocations (0 = no bound). cuda_stream: a cudaStream_t or
 * NULL for the legacy default stream. */
adms_status adms_ctx_create(adms_ctx** out, size_t hbm_budget_bytes, void* cuda_stream);
adms_status adms_ctx_destroy(adms_ctx* ctx);
adms_status adms_ctx_set_stream(adms_ctx* ctx, void* cuda_stream);
/* Overlap of reference rendering with the candidate's forward (no counterpart in
 * the paper, which renders the reference as a black box before each comparison):
 * cuda_event (a cudaEvent_t, or NULL for none) completes when the reference
 * images that later forward_loss calls read are written, typically recorded
 * after adms_render_reference on another stream (adms_ctx_set_stream switches the
 * stream between calls). Each forward_loss, and a backward that recomputes its
 * raster, makes the context's stream wait on it right before the first kernel
 * that reads a reference image, so the candidate's frame, raster and shading run
 * alongside the reference render. The event is read at those calls (and captured
 * into a graph with them); the caller keeps it alive. */
adms_status adms_ctx_set_ref_event(adms_ctx* ctx, void* cuda_event);
/* Pipelined optimizer steps (enable = 1; 0, the default, turns them off and
 * issues what is deferred). No counterpart in the paper; the results are those of
 * unpipelined steps. adms_optimizer_step then issues the schedules and the flat
 * latents' updates (positions, skin weights, displacement) and defers the job's
 * texture step (the texture latents' Adam updates with their mip chains, and the
 * advance of t). The job's next adms_forward_loss (one job per call) issues it on
 * a third stream of the context beside its vertex frame and raster, which read
 * only the positions, and makes the context's stream wait for it before the
 * shading, the first kernel that reads a texture. Any other call naming the job
 * (render_reference, backward, a second optimizer_step, job_params, job_stats,
 * export, gradient access, a batched forward_loss, ...) and adms_sync issue it
 * first, in line, so every call sees the latents of the sequential schedule;
 * memory read directly through adms_job_params pointers is current only after
 * such a call. A graph records which jobs held a deferred step when its capture
 * began and ended; adms_graph_launch refuses (ADMS_ERR_STATE) to replay it unless
 * the same jobs hold one now. Not during a capture (ADMS_ERR_STATE). */
adms_status adms_ctx_set_pipelining(adms_ctx* ctx, int32_t enable);
/* Issue every deferred texture step, then block until the context's stream is
 * idle; surfaces latched device errors. */
adms_status adms_sync(adms_ctx* ctx);
const char* adms_last_error(adms_ctx* ctx);
/* Bytes of HBM currently held by the context's jobs and scratch. */
size_t adms_bytes_in_use(adms_ctx* ctx);

/* ---- jobs ------------------------------------------------------------------ */

/* Copy a mesh and its textures in and allocate the job's resident state
 * (Sec. 3: the latent representation; Sec. 5.1: topology fixed, tessellation
 * precomputed). opt may be NULL for a frozen job (e.g. a reference model).
 * seed is kept with the job (checkpointed). Synchronises the stream. */
adms_status adms_job_create(adms_ctx* ctx, const adms_mesh_desc* mesh, const adms_material_desc* mat,
                            const adms_opt_params* opt, uint64_t seed, adms_job* out);
/* Free a job's resident state and the batched argument lists of every job set
 * it was part of; graphs that recorded calls on this job must not be launched
 * afterwards. Synchronises the stream. */
adms_status adms_job_destroy(adms_ctx* ctx, adms_job job);
/* Free the cached argument and work-item lists of all batched (n_jobs > 1)
 * calls; the next batched call rebuilds its own. Graphs that recorded a batched
 * call must not be launched afterwards. For schedulers whose job set changes
 * (a set's lists live until one of its jobs is destroyed otherwise).
 * Synchronises the stream. */
adms_status adms_ctx_release_batches(adms_ctx* ctx);
/* Dense linear-blend skinning (Sec. 5.1, Eq. 2): from now on the job renders
 * v^s_i = sum_b w_ib M_b [v_i; 1] instead of its rest positions v_i, with the
 * affine bone matrices M_b of the current frame (adms_job_set_bones; identity
 * until set). weights: [n_verts][n_bones] float32, host or device, copied;
 * every vertex-bone pair is its own weight (the dense operator), used as given
 * (no normalisation). lr_scale > 0 makes the weights a latent: the backward
 * accumulates their gradient beside the rest positions' and the optimizer
 * step applies Adam to them with learning rate lr_t * lr_scale (no clamps);
 * 0 keeps them fixed. Adam moves every weight by about its learning rate per
 * step, and the weights of a vertex tend to move together, so its skinned
 * position moves up to n_bones times faster than a rest position: 1/n_bones
 * keeps the two in step. The skinned positions feed the
 * bit-exact visibility through a fixed float32 evaluation (bones ascending,
 * each row ((m0 x + m1 y) + m2 z) + m3, weighted sum from 0, no FMA).
 * ADMS_ERR_ARG: n_bones outside [1, 1024], lr_scale < 0 or a null pointer; ADMS_ERR_STATE:
 * a tessellated job or skinning already set. Synchronises the stream. */
adms_status adms_job_skinning(adms_ctx* ctx, adms_job job, const float* weights, int32_t n_bones, float lr_scale);
/* The bone matrices of the frame the next calls render: [n_bones][4][4]
 * row-major float32 (last row 0 0 0 1), host or device; copied on the stream
 * (from device memory it records into a graph like the views). */
adms_status adms_job_set_bones(adms_ctx* ctx, adms_job job, const float* bones);
/* Allocate the job's per-call render scratch for n_views views of H x W now
 * (keys, per-pixel buffers, per-view transforms, bins), so that later calls of
 * that size or smaller allocate nothing for this job. Lets a scheduler admit
 * work against the HBM budget up front: ADMS_ERR_BUDGET if it does not fit
 * (the job stays valid), ADMS_ERR_ARG for non-positive or > 16384 sizes. */
adms_status adms_job_reserve(adms_ctx* ctx, adms_job job, int32_t n_views, int32_t H, int32_t W);
adms_status adms_job_params(adms_ctx* ctx, adms_job job, adms_param_view* out);
adms_status adms_job_stats(adms_ctx* ctx, adms_job job, adms_stats* out);
/* The latched status of each job (0, or e.g. ADMS_ERR_NONFINITE) into out
 * (device, [n_jobs] int32), ordered on the context's stream like the step
 * calls, without synchronising: a scheduler reads it back with the losses.
 * n_jobs in [1, 512]. */
adms_status adms_jobs_status(adms_ctx* ctx, const adms_job* jobs, int32_t n_jobs, int32_t* out);

/* ---- the step (Sec. 3, Eq. 1) --------------------------------------------- */

/* Forward render of n_views views at H x W with silhouette AA (Sec. 3: the
 * reference renderer is a black box that only sees camera and light; here it
 * is this library's own forward path applied to a frozen job).
 * views: any, [n_views]; out_rgb: device, [n_views][H][W][3]. */
adms_status adms_render_reference(adms_ctx* ctx, adms_job job, const adms_view* views, int32_t n_views,
                                  int32_t H, int32_t W, float* out_rgb);

/* Render each job under its views, antialias silhouettes, and take the image
 * loss against its reference images (Sec. 5.3: L1 on Gamma(log(x + 1))).
 *   jobs: host, [n_jobs]; views: any, all jobs' views back to back;
 *   views_per_job, hw: host, [n_jobs] and [n_jobs][2] (H, W);
 *   ref_rgb: host array of n_jobs device pointers, each [B_j][H_j][W_j][3];
 *   out_loss: device, [n_jobs] (L_image of this call); out_img: NULL, or a
 *   host array of n_jobs device pointers (NULL entries allowed) receiving the
 *   antialiased images [B_j][H_j][W_j][3].
 * Keeps what backward needs in the job's scratch. */
adms_status adms_forward_loss(adms_ctx* ctx, const adms_job* jobs, int32_t n_jobs, const adms_view* views,
                              const int32_t* views_per_job, const int32_t* hw, const float* const* ref_rgb,
                              float* out_loss, float* const* out_img);

/* Accumulate dL_image/dtheta for every latent of each job from its latest
 * forward_loss (Sec. 3, Sec. 5.1-5.2 chained backward: AA, shading, texture,
 * interpolation, transform, tangent frame, tessellation). recompute_raster:
 * 1 re-rasterizes and re-shades instead of reading the forward's buffers. */
adms_status adms_backward(adms_ctx* ctx, const adms_job* jobs, int32_t n_jobs, int32_t recompute_raster);

/* Per job: L_delta and its gradient (Eq. 4), lambda_t (Eq. 5, with the
 * lambda_0 heuristic at t = 0), lr_t = lr0 10^(-0.0002 t) and one Adam step
 * (beta = 0.9, 0.999, eps = 1e-8) on every optimized latent, fused with the
 * adjoint of the mip chain and followed by clamping and a mip rebuild; zeroes
 * the gradients and advances t.
 * Failure detection (no counterpart in the paper): a job whose status is
 * latched is not updated (its latents, moments and gradients are left as they
 * are). The status latches ADMS_ERR_NONFINITE on the device when a forward's
 * loss is NaN or infinite, when a vertex-stage gradient sum of the backward is,
 * or (from the next step on) when this step meets a non-finite gradient
 * element, which it leaves unapplied; no latent ever receives a NaN or an
 * infinity from an update. The other jobs of a batched call are unaffected. */
adms_status adms_optimizer_step(adms_ctx* ctx, const adms_job* jobs, int32_t n_jobs);

/* Level-0 gradient of each optimized texture with the adjoint of the box-filter
 * mip chain folded in (what the optimizer step applies), written to device
 * buffers [h][w][4] (NULL entries skipped); nothing is updated or zeroed. With
 * per-level textures, level 0's own gradient (the coarser levels' gradients
 * stay in the chain behind adms_param_view's gradient pointers).
 * ADMS_ERR_STATE for a texture that is not optimized. */
adms_status adms_job_fold_gradients(adms_ctx* ctx, adms_job job, float* g_kd, float* g_orm, float* g_nrm);
/* Zero every gradient buffer of a job (positions, displacement, textures). */
adms_status adms_job_zero_gradients(adms_ctx* ctx, adms_job job);
/* Rebuild the mip chains from level 0 (not for per-level textures, whose levels
 * are latents) and recompute the vertex frame at the next forward: call after
 * writing latents through adms_job_params pointers. */
adms_status adms_job_invalidate(adms_ctx* ctx, adms_job job);
/* L_delta of the job's current positions (Eq. 4; delta' = 0 unless the job
 * was created with relative_laplacian) into out_loss (device scalar), and
 * dL_delta/dpos into g_pos (device [V][3], overwritten; NULL skips it). */
adms_status adms_laplacian(adms_ctx* ctx, adms_job job, float* out_loss, float* g_pos);

/* Raw visibility of the latest forward_loss / render_reference of a job:
 * copies [B][H][W] keys into out_keys (device); a depth-peeled job's are
 * [L][B][H][W]. ADMS_ERR_ARG when capacity (in keys) is smaller. */
adms_status adms_job_keys(adms_ctx* ctx, adms_job job, uint64_t* out_keys, size_t capacity);

/* ---- checkpoint / resume --------------------------------------------------- */

/* Serialise a job's resumable state into host memory: a versioned header
 * (shapes, options, seed) followed by the positions and their Adam moments,
 * each texture's whole mip chain and level-0 moments, the displacement map and
 * its moments, the relative-Laplacian reference and the job state (t, lambda_0,
 * lambda, lr, bias corrections, latched status). Gradients are not kept:
 * export between optimizer steps. With host_buf == NULL only *bytes is set;
 * otherwise *bytes is the buffer's capacity on entry (ADMS_ERR_ARG if too
 * small) and the blob's size on return. Synchronises the stream. */
adms_status adms_job_export(adms_ctx* ctx, adms_job job, void* host_buf, size_t* bytes);
/* Recreate a job from adms_job_export output (checkpoint/resume): mesh, mat and
 * opt must describe the job that was exported (same topology, texture sizes,
 * options); their latent values are replaced by the blob's. ADMS_ERR_ARG if
 * the blob is not a checkpoint of this version or does not match them. A
 * skinned job comes back skinned (weights, moments and the last bones from the
 * blob). */
adms_status adms_job_import(adms_ctx* ctx, const adms_mesh_desc* mesh, const adms_material_desc* mat,
                            const adms_opt_params* opt, const void* host_buf, size_t bytes, adms_job* out);

/* ---- batched jobs ------------------------------------------------------------- */

/* adms_forward_loss and adms_backward with n_jobs > 1 run the per-pixel stages
 * (tile raster, shading, AA + loss, fused backward) as one launch each over
 * (job, view, tile) work items of every job, whatever their meshes, textures,
 * view counts and resolutions. The default grid is one block per item; a
 * persistent grid (block k takes items k, k + grid, ...; SMs x blocks per SM
 * blocks, at most the resident count) is the other choice. adms_autotune
 * times those launches on the given batch for tile widths 8, 16, 32 pixels
 * (tiles of 256 pixels) with one block per item and with half the resident
 * blocks per SM up to all of them, and keeps the fastest choice. It leaves the
 * jobs as it found them (gradients zeroed, no pending forward, no recorded
 * loss) and synchronises the stream. Arguments as for adms_forward_loss. */
adms_status adms_autotune(adms_ctx* ctx, const adms_job* jobs, int32_t n_jobs, const adms_view* views,
                          const int32_t* views_per_job, const int32_t* hw, const float* const* ref_rgb);
/* The context's batched-launch choices: out5 = {tile width, blocks per SM for
 * shading, AA + loss, backward, raster}. */
adms_status adms_ctx_tuning(adms_ctx* ctx, int32_t* out5);
/* Set those choices (same layout); blocks per SM <= 0 select one block per
 * item, others are clamped to the resident count. ADMS_ERR_ARG for a tile width other than 8, 16 or 32. Calls already
 * recorded into a graph keep the choices they were recorded with. */
adms_status adms_ctx_set_tuning(adms_ctx* ctx, const int32_t* in5);

/* ---- per-stage calls -------------------------------------------------------------
 *
 * The renderer as separate differentiable primitives, each with its adjoint, for
 * an autograd system that chains them (Sec. 5.2 builds the renderer from a
 * rasterizer, attribute interpolation, filtered texture lookups and an
 * antialiasing pass; Sec. 3 differentiates the image loss through all of them):
 *
 *   frame   (Sec. 5.1)      positions -> unit smooth vertex normals and tangents
 *   setup   (Sec. 5.2)      positions -> clip coordinates (+ triangle setup, tile bins)
 *   raster  (Sec. 5.2)      -> visibility keys, perspective-correct barycentrics
 *   shade   (Sec. 5.2)      barycentrics, vertex attributes, textures -> colour
 *   aa_loss (Sec. 5.2, 5.3) silhouette antialiasing and the image loss
 *
 * The arithmetic is the step calls' own; the one difference is that raster hands
 * shade its barycentrics as a buffer, so that dL/d(barycentrics) -> dL/d(clip)
 * (raster_bwd) and dL/d(colour) -> texels, vertex attributes and dL/d(barycentrics)
 * (shade_bwd) are separate calls. One sample per pixel, opaque meshes, the same
 * readings as the step calls. Stateless: every pointer is the caller's device
 * memory on the current device, nothing is allocated and nothing is kept between
 * calls; work is enqueued on cuda_stream (NULL: legacy default stream) and the
 * calls return before it runs. Gradient outputs marked "+=" are accumulated into
 * (the caller zeroes them); the others are overwritten. ADMS_ERR_ARG for null
 * pointers, non-positive or > 16384 image sizes, textures that are not power-of-
 * two mip chains, or a workspace that is too small or not 256-byte aligned;
 * ADMS_ERR_CUDA when a launch fails.
 *
 * Workspace: setup_fwd writes the views' screen positions, triangle setup
 * records, tile lists and silhouette masks into `work` (adms_stage_workspace_bytes,
 * 256-byte aligned). raster_fwd, raster_bwd, aa_loss_fwd and aa_loss_bwd read
 * them: pass the same workspace after a setup_fwd of the same positions, views
 * and sizes. Tiles whose triangle list does not fit it scan every triangle of
 * their view (same keys, slower). */
typedef struct {
    int32_t n_verts, n_uv, n_tris;
    const float* pos;       /* [V][3] render positions */
    const float* uv;        /* [T][2] UV corners */
    const int32_t* tri;     /* [F][3] position indices */
    const int32_t* tri_uv;  /* [F][3] UV indices */
    const int32_t* adj;     /* [F][3] face across edge (tri[f][k], tri[f][(k+1)%3]), -1 if none (adms_mesh_topology) */
    const int32_t* vf_off;  /* [V+1] vertex -> incident faces, CSR offsets (adms_mesh_topology) */
    const int32_t* vf_face; /* [vf_off[V]] incident faces, ascending per vertex */
} adms_stage_mesh;

/* A texture with its whole mip chain: float32 texels of 4 channels, level k
 * ([max(h>>k,1)][max(w>>k,1)][4]) right after level k-1; h, w powers of two,
 * 1 <= levels <= the full chain. */
typedef struct {
    const float* tex;  /* device, the chain */
    float* grad;       /* device, same layout, += in shade_bwd; NULL: no texel gradient */
    int32_t h, w, levels;
} adms_stage_texture;

/* Host helper (Sec. 3: the topology is fixed during optimization): the edge
 * adjacency adj [F][3] and the vertex -> face CSR (vf_off [V+1], vf_face [3F],
 * faces ascending) of a triangle list; all host memory, caller-owned. An edge
 * shared by more than two faces counts as open (-1). ADMS_ERR_ARG for an index
 * outside [0, n_verts). */
adms_status adms_mesh_topology(const int32_t* tri, int32_t n_verts, int32_t n_tris, int32_t* adj, int32_t* vf_off,
                               int32_t* vf_face);
/* Bytes of workspace for the setup / raster / aa_loss calls of one problem, with
 * room for list_entries (>= 4) tile-list entries; 0 for invalid sizes. */
size_t adms_stage_workspace_bytes(int32_t n_verts, int32_t n_tris, int32_t n_views, int32_t H, int32_t W,
                                  int64_t list_entries);

/* Sec. 5.1, smooth normals and tangents, recomputed from the positions: vertex
 * normal = normalised sum of the unnormalised face normals, vertex tangent =
 * normalised sum of sign(det duv) normalize(e1 dv2 - e2 dv1) over the faces.
 * Outputs [V][4] (fourth component 0): vpos4 = the positions, vnrm4, vtan4. */
adms_status adms_frame_fwd(const adms_stage_mesh* mesh, float* vpos4, float* vnrm4, float* vtan4, void* cuda_stream);
/* Adjoint of adms_frame_fwd: g_pos [V][3] += dL/dpos from dL/d(vpos4 xyz)
 * (g_vpos [V][3] float64, read and then zeroed), dL/d(vnrm4 xyz) and
 * dL/d(vtan4 xyz) (g_vnrm, g_vtan [V][3] float64); tmp: [2V][4] float scratch. */
adms_status adms_frame_bwd(const adms_stage_mesh* mesh, double* g_vpos, const double* g_vnrm, const double* g_vtan,
                           float* g_pos, float* tmp, void* cuda_stream);

/* Sec. 5.2, vertex transform and triangle setup of n_views views at H x W: clip
 * [B][V][4] = mvp [x y z 1]^T in float32 (fixed operation order, no FMA: the
 * bit-exact visibility contract), and into the workspace the snapped 8-bit
 * sub-pixel positions, the double-float screen positions used for shading, the
 * setup records, tile bins and the silhouette masks (an edge is a silhouette
 * edge in a view when it has one face or its faces' snapped areas differ in
 * sign). views: device [B]. */
adms_status adms_setup_fwd(const adms_stage_mesh* mesh, const adms_view* views, int32_t n_views, int32_t H, int32_t W,
                           float* clip, void* work, size_t work_bytes, void* cuda_stream);
/* Adjoint of the transform: g_pos [V][3] += sum over views of mvp[:, :3]^T
 * g_clip (g_clip: [B][V][4] float64). */
adms_status adms_setup_bwd(const adms_view* views, int32_t n_views, int32_t n_verts, const double* g_clip,
                           float* g_pos, void* cuda_stream);

/* Sec. 5.2 rasterization: keys [B][H][W] (as adms_job_keys: depth bits << 32 |
 * triangle id, minimum per pixel, all ones when empty; top-left fill rule on the
 * snapped positions), and for each covered pixel the perspective-correct
 * barycentrics of corners 1 and 2, rast [B][H][W][2], and their screen
 * derivatives d/dx b1, d/dx b2, d/dy b1, d/dy b2, rast_db [B][H][W][4] (texture
 * LOD only); zeros at empty pixels. clip: adms_setup_fwd's output. keep_keys = 1:
 * keys and rast_db are inputs, read and not written (visibility and texture LOD
 * held fixed while the positions move, as the adjoints assume, e.g. for finite
 * differences); 0: both are computed. */
adms_status adms_raster_fwd(const adms_stage_mesh* mesh, const adms_view* views, int32_t n_views, int32_t H, int32_t W,
                            const float* clip, uint64_t* keys, int32_t keep_keys, float* rast, float* rast_db,
                            void* work, size_t work_bytes, void* cuda_stream);
/* Adjoint of the barycentrics (the keys are piecewise constant in the positions
 * and have none; the visibility gradient is aa_loss_bwd's): g_clip [B][V][4]
 * float64 += dL/d(clip) from g_rast [B][H][W][2] = dL/d(rast). */
adms_status adms_raster_bwd(const adms_stage_mesh* mesh, const adms_view* views, int32_t n_views, int32_t H, int32_t W,
                            const float* clip, const uint64_t* keys, const float* g_rast, double* g_clip, void* work,
                            size_t work_bytes, void* cuda_stream);

/* Sec. 5.2 shading of every covered pixel: position, normal, tangent and uv
 * interpolated at (1 - b1 - b2, b1, b2) from vpos4 / vnrm4 / vtan4 [V][4] and the
 * UV corners; trilinear lookups of maps[0] base colour, maps[1] (gamma, r, m),
 * maps[2] tangent-space normal at the LOD of the uv footprint (u wraps, v
 * clamps); normal mapping and diffuse + GGX under the view's lights (the
 * readings of adms_forward_loss). pre [B][H][W][4]: colour, 1 (0 when empty). */
adms_status adms_shade_fwd(const adms_stage_mesh* mesh, const adms_view* views, int32_t n_views, int32_t H, int32_t W,
                           const uint64_t* keys, const float* rast, const float* rast_db, const float* vpos4,
                           const float* vnrm4, const float* vtan4, const adms_stage_texture* maps, float* pre,
                           void* cuda_stream);
/* Adjoint of adms_shade_fwd for g_pre [B][H][W][4] = dL/d(pre) (fourth channel
 * ignored; the LOD held fixed): maps[i].grad += the texel gradients (whole chain),
 * g_vpos, g_vnrm, g_vtan [V][3] float64 += dL/d(vpos4, vnrm4, vtan4 xyz), and
 * g_rast [B][H][W][2] = dL/d(rast). */
adms_status adms_shade_bwd(const adms_stage_mesh* mesh, const adms_view* views, int32_t n_views, int32_t H, int32_t W,
                           const uint64_t* keys, const float* rast, const float* rast_db, const float* vpos4,
                           const float* vnrm4, const float* vtan4, const adms_stage_texture* maps, const float* g_pre,
                           double* g_vpos, double* g_vnrm, double* g_vtan, float* g_rast, void* cuda_stream);

/* Sec. 5.2 silhouette antialiasing and the Sec. 5.3 image loss (the readings of
 * adms_forward_loss: pairs of 4-neighbours with different triangles blend by the
 * crossing of the owner's silhouette edge; L1, log-tone-mapped L1 or L2 per
 * channel, times loss_scale, e.g. 1 / (3 B H W)). pre: [B][H][W][4] from shade.
 * With ref ([B][H][W][3]): *loss (float64 device scalar) += the loss and gprime
 * [B][H][W][4] = dL/d(antialiased colour) in xyz (w: the pair bits the adjoint
 * reads). img [B][H][W][3]: the antialiased image, or NULL (needed without ref). */
adms_status adms_aa_loss_fwd(const adms_stage_mesh* mesh, const adms_view* views, int32_t n_views, int32_t H, int32_t W,
                             const float* clip, const uint64_t* keys, const float* pre, const float* ref,
                             int32_t loss_kind, float loss_scale, float* img, double* loss, float* gprime, void* work,
                             size_t work_bytes, void* cuda_stream);
/* Adjoint of adms_aa_loss_fwd for dL/d(loss) = *g_loss (device scalar; NULL = 1):
 * g_pre [B][H][W][4] = dL/d(pre) (fourth channel 0), and g_clip [B][V][4]
 * float64 += the silhouette crossings' gradient w.r.t. their edges' clip
 * coordinates. gprime: adms_aa_loss_fwd's. */
adms_status adms_aa_loss_bwd(const adms_stage_mesh* mesh, const adms_view* views, int32_t n_views, int32_t H, int32_t W,
                             const float* clip, const uint64_t* keys, const float* pre, const float* gprime,
                             const float* g_loss, float* g_pre, double* g_clip, void* work, size_t work_bytes,
                             void* cuda_stream);

/* Tessellation with displacement (Sec. 5.1, Eq. 3) as a stage: a base mesh split
 * `levels` times at edge midpoints (the (2^levels)-segment lattice of every base
 * triangle; vertices shared along base edges merged), each render vertex
 * v = sum_k w_k p_k displaced along the normalised interpolated smooth base
 * normal by the bilinear level-0 lookup of a scalar map at the vertex's UV. */
typedef struct {
    int32_t n_base_verts, n_base_tris, n_verts, n_segments; /* n_segments = 2^levels */
    const int32_t* base_tri; /* [Fb][3] */
    const int32_t* bvf_off;  /* [Vb+1] base vertex -> incident faces (adms_mesh_topology of the base mesh) */
    const int32_t* bvf_face;
    const int32_t* owner;    /* [Vt][3] the base vertices of the render vertex's owning base face */
    const int32_t* wts;      /* [Vt][3] its integer lattice weights (summing to n_segments) */
    const float* vert_uv;    /* [Vt][2] the UV its displacement is looked up at */
} adms_tess_desc;

/* Host helper: the tessellation tables of a base mesh (host memory, caller-
 * owned). counts [3] = {render vertices Vt, render triangles Ft, render UV
 * corners Tt}: with every table pointer NULL only counts is written; otherwise
 * counts holds the capacities on entry (ADMS_ERR_ARG if too small) and rtri
 * [Ft][3], rtri_uv [Ft][3], ruv [Tt][2] (the render mesh, sub-triangles keeping
 * their base face's UV corners interpolated), owner, wts [Vt][3] and vert_uv
 * [Vt][2] (a shared vertex takes the UV of its lowest-numbered owning base face)
 * are filled. levels in [1, 8]. */
adms_status adms_tessellation(const int32_t* tri, const int32_t* tri_uv, const float* uv, int32_t n_verts, int32_t n_uv,
                              int32_t n_tris, int32_t levels, int32_t* counts, int32_t* rtri, int32_t* rtri_uv,
                              float* ruv, int32_t* owner, int32_t* wts, float* vert_uv);
/* Render positions pos [Vt][3] from base positions [Vb][3] and the displacement
 * map disp [dh][dw] (dh, dw powers of two; u wraps, v clamps), and the smooth base normals base_nrm
 * [Vb][3] they use, in the float32 contract of the step calls (visibility is
 * decided on these positions). */
adms_status adms_tess_fwd(const adms_tess_desc* tess, const float* base_pos, const float* disp, int32_t dh, int32_t dw,
                          float* base_nrm, float* pos, void* cuda_stream);
/* Adjoint for g_pos [Vt][3] = dL/d(pos): g_base_pos and g_base_nrm [Vb][3]
 * float64 += the direct position and base-normal gradients, g_disp [dh][dw] +=
 * the displacement texels' (NULL: skipped). The base normals' own adjoint is
 * adms_frame_bwd on the base mesh (normal gradient g_base_nrm, no tangent
 * gradient), which also folds g_base_pos into the base positions. */
adms_status adms_tess_bwd(const adms_tess_desc* tess, const float* base_pos, const float* base_nrm, const float* disp,
                          int32_t dh, int32_t dw, const float* g_pos, double* g_base_pos, double* g_base_nrm,
                          float* g_disp, void* cuda_stream);

/* Sec. 5.2 filtered lookups: rebuild levels 1 .. levels-1 of a chain from level 0
 * (each texel the mean of its 2 x 2 parents), in place. */
adms_status adms_mip_fwd(float* chain, int32_t h, int32_t w, int32_t levels, void* cuda_stream);
/* Adjoint of adms_mip_fwd: g_level0 [h][w][4] = level 0's gradient plus every
 * coarser level's gradient spread evenly over the level-0 texels under it. */
adms_status adms_mip_bwd(const float* g_chain, int32_t h, int32_t w, int32_t levels, float* g_level0,
                         void* cuda_stream);

/* ---- visibility without allocation -------------------------------------------- */

/* Visibility keys of n_views views, for callers that cannot call cudaMalloc
 * (code inside another framework's memory pool or a fixed arena, or a frame
 * loop where an allocation and the synchronisation it brings are not
 * allowed). The paper has no counterpart: it is a deployment variant of the
 * raster that adms_render_reference and adms_forward_loss run.
 *
 * Inputs (device): pos [n_verts][3] float32, tri [n_tris][3] int32 with every
 * index in [0, n_verts), views [n_views] adms_view. Output (device, caller-
 * owned): keys [n_views][H][W] with the same bits as the context path's keys.
 * Work is enqueued on cuda_stream (NULL: legacy default stream).
 *
 * Allocates nothing: no cudaMalloc, no cudaFree, no allocating library call.
 * Its scratch is one file-scope device array of 32 MiB that every GPU loading
 * this library holds until the process exits. It must hold
 *   n_views * n_verts * 48 + n_views * n_tris * 106 + n_tris * 12
 *   + tiles * 28 bytes (tiles = n_views * ceil(W/16) * ceil(H/16)), plus
 * 256-byte rounding per part; larger problems return ADMS_ERR_ARG, decided with
 * overflow-checked arithmetic before any CUDA call. Tile lists
 * use whatever space is left; a tile whose list does not fit scans every
 * triangle, with the same keys. The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current:
 * make that first call before any stream capture. Every call shares the one
 * array, so calls that overlap on the GPU (different streams, or threads
 * using different streams) race: serialise them. Returns ADMS_ERR_CUDA if a
 * CUDA call fails. */
adms_status adms_visibility_noalloc(const float* pos, int32_t n_verts, const int32_t* tri, int32_t n_tris,
                                    const adms_view* views, int32_t n_views, int32_t H, int32_t W,
                                    uint64_t* keys, void* cuda_stream);

/* ---- CUDA graphs ----------------------------------------------------------- */

typedef struct adms_graph adms_graph;

/* Record, rather than run, the adms calls made on this context's stream until
 * adms_graph_end (CUDA stream capture, thread-local mode), so a whole step
 * (render_reference, forward_loss, backward, optimizer_step) replays as one
 * graph launch. The stream must not be the legacy default stream. Recorded
 * calls must not need new scratch (ADMS_ERR_STATE): make the same calls once
 * before capturing. Pointers passed while capturing are baked into the graph:
 * views and reference images must live at fixed device addresses whose
 * contents the caller refreshes between launches. */
adms_status adms_graph_begin(adms_ctx* ctx);
adms_status adms_graph_end(adms_ctx* ctx, adms_graph** out);
/* Enqueue one replay of a recorded graph on the context's stream. With pipelined
 * steps (adms_ctx_set_pipelining) the jobs holding a deferred texture step must be
 * those at the capture's start (else ADMS_ERR_STATE, nothing enqueued); after the
 * launch they are those at its end. */
adms_status adms_graph_launch(adms_ctx* ctx, adms_graph* graph);
adms_status adms_graph_destroy(adms_graph* graph);

/* ---- tracing ------------------------------------------------------------- */

/* Bracket every stage launched through this context with CUDA events on its
 * stream (enable = 1) or stop doing so (0). No paper counterpart: tooling. */
adms_status adms_ctx_profile(adms_ctx* ctx, int32_t enable);
/* Synchronise, then return and reset the GPU milliseconds and stage launch
 * counts accumulated per stage since the previous call. ms_out and
 * launches_out (nullable) hold n_stages >= adms_stage_count() entries. */
adms_status adms_ctx_stage_times(adms_ctx* ctx, double* ms_out, int64_t* launches_out, int32_t n_stages);
int32_t adms_stage_count(void);
/* Name of stage i ("raster", "shade_bwd", ...), "" if out of range. */
const char* adms_stage_name(int32_t i);
/* Kernels this library has launched in this process (host-side count). */
int64_t adms_launch_count(void);

/* ---- failure-detection test hook ----------------------------------------- */

/* The one wait on the device, the texture Adam's wait for each tile's TMA copies
 * (adms_optimizer_step), gives up after 2 s of the GPU's global timer, latches
 * ADMS_ERR_TIMEOUT in the job's status (read by adms_jobs_status / adms_job_stats
 * after the step) and leaves that texture's latents unchanged. With enable = 1
 * every such wait of this context's later optimizer steps expects 16 bytes more
 * than its copies deliver, so that it runs out (each launch then takes about
 * 4 s); 0 restores normal steps. For tests only; no paper counterpart. */
adms_status adms_ctx_test_wait_timeout(adms_ctx* ctx, int32_t enable);

#ifdef __cplusplus
}
#endif
#endif /* ADMS_H */
