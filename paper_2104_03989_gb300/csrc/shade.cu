// Per-pixel deferred shading, silhouette antialiasing, image loss and the fused
// backward (Sec. 5.2 renderer, Sec. 5.3 objective).
//
// No G-buffer is stored: every per-pixel kernel recomputes the perspective-
// correct barycentrics and the interpolated attributes from the visibility
// key (triangle id) and the per-view vertex data.
//
// Precision: screen positions arrive as float-float pairs computed in float64
// per vertex, so offsets from the pixel centre keep float32 relative
// precision; attributes are interpolated as corner-0 value + weighted corner
// differences, which keeps texel coordinates of large textures accurate and
// lets the barycentric adjoint use (a_j - a) without cancellation. Vertex
// gradients are accumulated in float64.
#include "pixel.cuh"

namespace adms {

// ------------------------------------------------------------------ single-job kernels (16x16 tiles)
// the listed pixels of one job (A.refine[0] of them), grid-stride
__global__ void __launch_bounds__(256) k_shade_refine(ShadeArgs A) {
    int n = A.refine[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        shade_refine_px(A, A.refine[1 + i]);
}

// A 16x16 tile of pixels is shaded by 256 / THREADS blocks, each a band of
// 16 x (THREADS / 16) rows; thread t takes column t % 16 of row t / 16 of its band.
template <int THREADS>
__device__ __forceinline__ void band_pixel(int W, int& px, int& py) {
    constexpr int PARTS = 256 / THREADS;
    int tiles_x = (W + ADMS_TILE - 1) / ADMS_TILE;
    int tile = blockIdx.x / PARTS, part = blockIdx.x % PARTS;
    px = (tile % tiles_x) * ADMS_TILE + (threadIdx.x & 15);
    py = (tile / tiles_x) * ADMS_TILE + part * (ADMS_TILE / PARTS) + (threadIdx.x >> 4);
}

// block shapes measured on the plain-method step (threads per block x resident
// blocks per SM, i.e. the register cap 65536 / (threads x blocks)); shading: 256 x 5
// 0.0928 ms, 256 x 4 0.0919, 256 x 6 0.0902, 128 x 10 0.0903, 128 x 8 0.0882, 128 x 12
// 0.0882; AA + loss: 256 x 8 0.0612, 256 x 6 0.0672, 128 x 12 0.0631, 128 x 16 0.0593;
// the backward's below (a few hundred bytes of spills cost less than the latency the
// extra resident warps hide)
#ifndef ADMS_FWD_THREADS
#define ADMS_FWD_THREADS 128
#endif
#ifndef ADMS_FWD_BLOCKS
#define ADMS_FWD_BLOCKS 8
#endif
#ifndef ADMS_AA_THREADS
#define ADMS_AA_THREADS 128
#endif
#ifndef ADMS_AA_BLOCKS
#define ADMS_AA_BLOCKS 16
#endif
template <bool INLINE>
__global__ void __launch_bounds__(ADMS_FWD_THREADS, ADMS_FWD_BLOCKS) k_shade_fwd(ShadeArgs A) {
    int px, py;
    band_pixel<ADMS_FWD_THREADS>(A.W, px, py);
    shade_fwd_px<INLINE>(A, blockIdx.y, px, py);
}

template <bool PEEL>
__global__ void __launch_bounds__(ADMS_AA_THREADS, ADMS_AA_BLOCKS) k_aa_loss(ShadeArgs A) {
    __shared__ double red[ADMS_AA_THREADS / 32];
    int px, py;
    band_pixel<ADMS_AA_THREADS>(A.W, px, py);
    aa_loss_block<PEEL>(A, blockIdx.y, px, py, red);
}

// resident blocks per SM of the fused backward (register cap 65536 / (threads x this))
// (the plain-method step: 256 threads x 3 blocks 0.174 ms; 128 x 5: 0.175; 128 x 6:
// 0.171; 128 x 7: 0.171)
#ifndef ADMS_BWD_BLOCKS
#define ADMS_BWD_BLOCKS 6
#endif
#ifndef ADMS_BWD_THREADS
#define ADMS_BWD_THREADS 128  // 256: a block per 16x16 tile; 128: two blocks of 16x8 pixels
#endif
template <bool PEEL>
__global__ void __launch_bounds__(ADMS_BWD_THREADS, ADMS_BWD_BLOCKS) k_shade_bwd(ShadeArgs A) {
    __shared__ float rows[(ADMS_BWD_THREADS / 32) * 32 * ADMS_VROW];
    int px, py;
    band_pixel<ADMS_BWD_THREADS>(A.W, px, py);
    shade_bwd_px<PEEL>(A, blockIdx.y, px, py, rows + (threadIdx.x >> 5) * 32 * ADMS_VROW);
}

// MSAA forward: a block takes a 32x32-sample region (four samples per thread), its
// (pixel, triangle) groups are compacted into a shared-memory list and each group is
// shaded by one thread; every sample copies its group's colour. (A 16x16 region holds
// only ~70 groups at 2x2 MSAA, which left most of a block's warps waiting while three
// shaded.)
#define ADMS_MSAA_REGION 32
__global__ void __launch_bounds__(256, 4) k_shade_fwd_msaa(ShadeArgs A) {
    constexpr int R = ADMS_MSAA_REGION, N = R * R, PER = N / 256;
    __shared__ int tri[N];
    __shared__ short list[N];
    __shared__ float4 col[N];
    __shared__ int count;
    int rx = (A.W + R - 1) / R;
    int b = blockIdx.y, tid = threadIdx.x;
    int x0 = (blockIdx.x % rx) * R, y0 = (blockIdx.x / rx) * R;
    if (tid == 0) count = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        int t = tid + 256 * k, px = x0 + (t % R), py = y0 + (t / R);
        bool inside = px < A.W && py < A.H;
        tri[t] = inside ? key_tri(A.keys[((size_t)b * A.H + py) * A.W + px]) : -1;
    }
    __syncthreads();
    int lead[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        int t = tid + 256 * k;
        lead[k] = group_leader(A.msaa, x0, y0, R, x0 + (t % R), y0 + (t / R), tri[t], tri);
        if (lead[k] == t) list[atomicAdd(&count, 1)] = (short)t;
    }
    __syncthreads();
    int n = count;
    for (int i = tid; i < n; i += 256) {
        int t = list[i];
        int sx = x0 + (t % R), sy = y0 + (t / R);
        col[t] = shade_covered(A, b, sx, sy, tri[t], ((size_t)b * A.H + sy) * A.W + sx);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        int t = tid + 256 * k, px = x0 + (t % R), py = y0 + (t / R);
        if (px < A.W && py < A.H)
            A.pre[((size_t)b * A.H + py) * A.W + px] = lead[k] >= 0 ? col[lead[k]] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// MSAA backward over a 32x32-sample region (four samples per thread): the AA
// adjoint runs per sample; the shading adjoint of a (pixel, triangle) group is
// linear in its colour gradient and its samples share the shading, so the group's
// leader takes the sum of its samples' gradients (in a fixed order) and the
// compacted leaders run the adjoint once per group
__global__ void __launch_bounds__(256, 3) k_shade_bwd_msaa(ShadeArgs A) {
    constexpr int R = ADMS_MSAA_REGION, N = R * R, PER = N / 256;
    __shared__ int tri[N];
    __shared__ float3 gsum[N];
    __shared__ short list[N];
    __shared__ int count;
    __shared__ float rows[8 * 32 * ADMS_VROW];
    int rx = (A.W + R - 1) / R;
    int b = blockIdx.y, tid = threadIdx.x;
    int x0 = (blockIdx.x % rx) * R, y0 = (blockIdx.x / rx) * R;
    if (tid == 0) count = 0;
    for (int k = 0; k < PER; ++k) {
        int t = tid + 256 * k, px = x0 + (t % R), py = y0 + (t / R);
        int f = -1;
        float3 gc = zero3();
        if (px < A.W && py < A.H) {
            size_t pix = ((size_t)b * A.H + py) * A.W + px;
            unsigned long long kp = A.keys[pix];
            f = key_tri(kp);
            gc = aa_adjoint<false>(A, b, px, py, pix, kp);
        }
        tri[t] = f;
        gsum[t] = gc;
    }
    __syncthreads();
    // leaders sum their groups (registers first: other leaders still read gsum)
    float3 g[PER];
    bool leader[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        int t = tid + 256 * k, px = x0 + (t % R), py = y0 + (t / R);
        int f = tri[t];
        g[k] = zero3();
        leader[k] = false;
        if (f < 0) continue;
        int sm = A.msaa, ox = (px / sm) * sm, oy = (py / sm) * sm;
        int first = -1;
        for (int y = max(oy, y0); y < min(oy + sm, y0 + R); ++y)
            for (int x = max(ox, x0); x < min(ox + sm, x0 + R); ++x) {
                int u = (y - y0) * R + (x - x0);
                if (tri[u] != f) continue;
                if (first < 0) first = u;
                g[k] += gsum[u];
            }
        leader[k] = first == t;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        int t = tid + 256 * k;
        if (leader[k] && (g[k].x != 0.f || g[k].y != 0.f || g[k].z != 0.f)) {
            gsum[t] = g[k];
            list[atomicAdd(&count, 1)] = (short)t;
        }
    }
    __syncthreads();
    int n = count;
    // warp-uniform trips: the vertex scatter is warp-collective
    for (int base = tid & ~31; base < n; base += 256) {
        int i = base + (tid & 31);
        int fl = -1;
        float* wrows = rows + (tid >> 5) * 32 * ADMS_VROW;
        if (i < n) {
            int t = list[i];
            fl = tri[t];
            shading_adjoint<false>(A, b, x0 + (t % R), y0 + (t / R), fl, gsum[t], 0.f, wrows + (tid & 31) * ADMS_VROW);
        }
        scatter_vertex_rows(A, fl, wrows);
    }
}

// ------------------------------------------------------------------ persistent batched kernels
// One launch covers (job, view, tile) work items of up to 64 jobs with
// different meshes, textures, view counts and resolutions. Block k takes items
// k, k + gridDim.x, ... (equal tiles of tw x (256 / tw) pixels, so a static
// stride balances them without a shared counter). The jobs' arguments are
// kernel parameters: read-only, no copy per block, and no aliasing with the
// stores and atomics of the pixel code.
// refinement lists of a batch (see k_shade_refine): reset before the shading
// launch, then one grid-stride pass per job (blockIdx.y)
__global__ void k_refine_reset(const ShadeBatch P, int n) {
    int k = threadIdx.x;
    if (k < n && P.a[k].refine) P.a[k].refine[0] = 0;
}
__global__ void __launch_bounds__(256) k_refine_batch(const ShadeBatch P) {
    const ShadeArgs& A = P.a[blockIdx.y];
    if (!A.refine) return;
    int n = A.refine[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        shade_refine_px(A, A.refine[1 + i]);
}

template <int KIND>
__global__ void __launch_bounds__(256, KIND == 2 ? 3 : (KIND == 1 ? 8 : 5))
    k_pixels_batch(const ShadeBatch P, const WorkItem* __restrict__ items, int n, int tw, int job0) {
    __shared__ double red[8];
    __shared__ float rows[KIND == 2 ? 8 * 32 * ADMS_VROW : 1];
    for (int it = blockIdx.x; it < n; it += gridDim.x) {
        WorkItem w = items[it];
        const ShadeArgs& A = P.a[w.job - job0];
        int px = w.x0 + (int)threadIdx.x % tw, py = w.y0 + (int)threadIdx.x / tw;
        if (KIND == 0) shade_fwd_px(A, w.view, px, py);
        else if (KIND == 1) aa_loss_block(A, w.view, px, py, red);
        else shade_bwd_px(A, w.view, px, py, rows + (threadIdx.x >> 5) * 32 * ADMS_VROW);
    }
}

// ------------------------------------------------------------------ supersample resolve
__global__ void __launch_bounds__(256) k_resolve(ResolveArgs r) {
    __shared__ double red[8];
    long long n = (long long)r.B * r.H * r.W;
    long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double lsum = 0.0;
    if (pix < n) {
        int b = (int)(pix / ((long long)r.H * r.W));
        int rem = (int)(pix - (long long)b * r.H * r.W);
        int py = rem / r.W, px = rem - py * r.W;
        int SW = r.S * r.W;
        size_t base = ((size_t)b * r.S * r.H + (size_t)py * r.S) * SW + (size_t)px * r.S;
        float3 c = zero3();
        for (int sy = 0; sy < r.S; ++sy)
            for (int sx = 0; sx < r.S; ++sx) c += f3of(r.acol[base + (size_t)sy * SW + sx]);
        float inv = 1.f / (float)(r.S * r.S);
        c = inv * c;
        if (r.out_img) {
            r.out_img[pix * 3] = c.x;
            r.out_img[pix * 3 + 1] = c.y;
            r.out_img[pix * 3 + 2] = c.z;
        }
        if (r.ref) {
            const float* y = r.ref + pix * 3;
            float g0, g1, g2;
            lsum = (double)loss_term(r.loss_kind, c.x, y[0], &g0) + (double)loss_term(r.loss_kind, c.y, y[1], &g1) +
                   (double)loss_term(r.loss_kind, c.z, y[2], &g2);
            float k = r.loss_scale * inv;  // each sample carries 1 / s^2 of its pixel
            for (int sy = 0; sy < r.S; ++sy)
                for (int sx = 0; sx < r.S; ++sx) {
                    size_t q = base + (size_t)sy * SW + sx;
                    r.gprime[q] = make_float4(g0 * k, g1 * k, g2 * k, r.acol[q].w);
                }
        }
    }
    lsum = warp_sum_d(lsum);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lsum;
    __syncthreads();
    if (threadIdx.x == 0 && r.loss_acc) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        atomicAdd(r.loss_acc, s * (double)r.loss_scale);
    }
}

cudaError_t resolve_loss(const ResolveArgs& r, cudaStream_t st) {
    long long n = (long long)r.B * r.H * r.W;
    k_resolve<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(r);
    count_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ launchers
static dim3 pix_grid(const ShadeArgs& a) {
    int tx = (a.W + ADMS_TILE - 1) / ADMS_TILE, ty = (a.H + ADMS_TILE - 1) / ADMS_TILE;
    return dim3(tx * ty, a.B);
}
// the grid of band_pixel<threads>: 256 / threads blocks per tile
static dim3 band_grid(const ShadeArgs& a, int threads) {
    dim3 g = pix_grid(a);
    g.x *= 256 / threads;
    return g;
}

// grids of up to this many samples refine their bright pixels in the shading
// kernel itself (no list, no second launch)
#ifndef ADMS_INLINE_REFINE_PX
#define ADMS_INLINE_REFINE_PX (1 << 20)
#endif

cudaError_t shade_forward(const ShadeArgs& a, cudaStream_t st) {
    bool inline_refine = a.msaa <= 1 && (size_t)a.B * a.H * a.W <= ADMS_INLINE_REFINE_PX;
    bool list = a.refine && !inline_refine;
    if (list) {
        cudaError_t e = cudaMemsetAsync(a.refine, 0, sizeof(int), st);
        if (e) return e;
    }
    if (a.msaa > 1) {
        int R = ADMS_MSAA_REGION;
        k_shade_fwd_msaa<<<dim3(((a.W + R - 1) / R) * ((a.H + R - 1) / R), a.B), 256, 0, st>>>(a);
    } else if (inline_refine) {
        k_shade_fwd<true><<<band_grid(a, ADMS_FWD_THREADS), ADMS_FWD_THREADS, 0, st>>>(a);
    } else {
        k_shade_fwd<false><<<band_grid(a, ADMS_FWD_THREADS), ADMS_FWD_THREADS, 0, st>>>(a);
    }
    count_launches(1);
    if (list) {
        k_shade_refine<<<128, 256, 0, st>>>(a);
        count_launches(1);
    }
    return cudaGetLastError();
}
cudaError_t aa_loss_forward(const ShadeArgs& a, cudaStream_t st) {
    if (a.peel) k_aa_loss<true><<<band_grid(a, ADMS_AA_THREADS), ADMS_AA_THREADS, 0, st>>>(a);
    else k_aa_loss<false><<<band_grid(a, ADMS_AA_THREADS), ADMS_AA_THREADS, 0, st>>>(a);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t shade_backward(const ShadeArgs& a, cudaStream_t st) {
    if (a.msaa > 1) {
        int R = ADMS_MSAA_REGION;
        k_shade_bwd_msaa<<<dim3(((a.W + R - 1) / R) * ((a.H + R - 1) / R), a.B), 256, 0, st>>>(a);
    } else if (a.peel) {
        k_shade_bwd<true><<<band_grid(a, ADMS_BWD_THREADS), ADMS_BWD_THREADS, 0, st>>>(a);
    } else {
        k_shade_bwd<false><<<band_grid(a, ADMS_BWD_THREADS), ADMS_BWD_THREADS, 0, st>>>(a);
    }
    count_launches(1);
    return cudaGetLastError();
}

int batched_occupancy(int kind) {
    if (kind == 3) return raster_batch_occupancy();
    int n = 0;
    cudaError_t e = kind == 0   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pixels_batch<0>, 256, 0)
                    : kind == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pixels_batch<1>, 256, 0)
                                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pixels_batch<2>, 256, 0);
    return e == cudaSuccess && n > 0 ? n : 1;
}

cudaError_t pixels_batched(int kind, const ShadeArgs* args, const int* item_off, int n_jobs, const WorkItem* items,
                           int tw, int blocks, cudaStream_t st) {
    ShadeBatch P;
    for (int j0 = 0; j0 < n_jobs; j0 += ADMS_BATCH_JOBS) {
        int j1 = std::min(n_jobs, j0 + ADMS_BATCH_JOBS);
        int s0 = item_off[j0], n = item_off[j1] - s0;
        if (n <= 0) continue;
        memcpy(P.a, args + j0, sizeof(ShadeArgs) * (j1 - j0));
        int g = std::min(blocks, n);
        if (kind == 0) {
            k_refine_reset<<<1, ADMS_BATCH_JOBS, 0, st>>>(P, j1 - j0);
            k_pixels_batch<0><<<g, 256, 0, st>>>(P, items + s0, n, tw, j0);
            k_refine_batch<<<dim3(64, j1 - j0), 256, 0, st>>>(P);
            count_launches(2);
        }
        else if (kind == 1) k_pixels_batch<1><<<g, 256, 0, st>>>(P, items + s0, n, tw, j0);
        else k_pixels_batch<2><<<g, 256, 0, st>>>(P, items + s0, n, tw, j0);
        count_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e) return e;
    }
    return cudaSuccess;
}

}  // namespace adms
