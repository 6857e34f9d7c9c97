// Mesh operations (Sec. 5.1): smooth vertex normals and tangents from positions
// and UVs, recomputed every step, with their adjoint; the uniform Laplacian
// regularizer of Eq. 4.
//
// Both run one thread per vertex and gather over a vertex -> face (or one-ring)
// CSR table, so results do not depend on atomic ordering.
#include "kernels.cuh"

namespace adms {

struct FaceFrame {
    float3 e1, e2, fn, tv;
    float d1y, d2y;
    int sgn;
    int idx[3];
};

__device__ __forceinline__ FaceFrame face_frame(const FrameArgs& a, int f) {
    FaceFrame r;
    int i0 = a.tri[3 * f], i1 = a.tri[3 * f + 1], i2 = a.tri[3 * f + 2];
    r.idx[0] = i0;
    r.idx[1] = i1;
    r.idx[2] = i2;
    float3 p0 = f3(a.pos[3 * i0], a.pos[3 * i0 + 1], a.pos[3 * i0 + 2]);
    float3 p1 = f3(a.pos[3 * i1], a.pos[3 * i1 + 1], a.pos[3 * i1 + 2]);
    float3 p2 = f3(a.pos[3 * i2], a.pos[3 * i2 + 1], a.pos[3 * i2 + 2]);
    float2 u0 = a.uv[a.tri_uv[3 * f]], u1 = a.uv[a.tri_uv[3 * f + 1]], u2 = a.uv[a.tri_uv[3 * f + 2]];
    r.e1 = p1 - p0;
    r.e2 = p2 - p0;
    r.fn = cross3(r.e1, r.e2);
    float d1x = u1.x - u0.x, d2x = u2.x - u0.x;
    r.d1y = u1.y - u0.y;
    r.d2y = u2.y - u0.y;
    float det = d1x * r.d2y - d2x * r.d1y;
    r.sgn = det > 0.f ? 1 : (det < 0.f ? -1 : 0);
    r.tv = r.d2y * r.e1 - r.d1y * r.e2;
    return r;
}

// The gathers over a vertex's faces (or one-ring) run in batches of ADMS_GATHER:
// the batch's loads are issued together (the last entry repeated past the end)
// and summed in list order, so each sum keeps the order of a plain loop while the
// dependent loads of a vertex take ceil(valence / ADMS_GATHER) round trips
// instead of one per face.
#define ADMS_GATHER 4

// unnormalised vertex normal (sum of face normals) and tangent (sum of signed unit face tangents)
__device__ __forceinline__ void vertex_sums(const FrameArgs& a, int v, float3& n, float3& t) {
    n = zero3();
    t = zero3();
    int lo = a.vf_off[v], hi = a.vf_off[v + 1];
    for (int j0 = lo; j0 < hi; j0 += ADMS_GATHER) {
        FaceFrame ff[ADMS_GATHER];
#pragma unroll
        for (int q = 0; q < ADMS_GATHER; ++q) ff[q] = face_frame(a, a.vf_face[min(j0 + q, hi - 1)]);
#pragma unroll
        for (int q = 0; q < ADMS_GATHER; ++q) {
            if (j0 + q < hi) {
                n += ff[q].fn;
                if (ff[q].sgn != 0) t += (float)ff[q].sgn * nrm3(ff[q].tv).y;
            }
        }
    }
}

__global__ void k_frame_fwd(FrameArgs a) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.V) return;
    float3 n, t;
    vertex_sums(a, v, n, t);
    Nrm3 nn = nrm3(n), tn = nrm3(t);
    a.vpos[v] = make_float4(a.pos[3 * v], a.pos[3 * v + 1], a.pos[3 * v + 2], 0.f);
    a.vnrm[v] = make_float4(nn.y.x, nn.y.y, nn.y.z, 0.f);
    a.vtan[v] = make_float4(tn.y.x, tn.y.y, tn.y.z, 0.f);
    if (a.inv) a.inv[v] = make_float2(nn.big ? nn.inv : -nn.inv, tn.big ? tn.inv : -tn.inv);
}

// the normalisation of vertex c's normal (k = 0) or tangent (k = 1) sum as the
// forward left it: the unit vector and the signed inverse length
__device__ __forceinline__ Nrm3 stored_nrm3(const FrameArgs& a, int c, int k) {
    float4 y = k == 0 ? a.vnrm[c] : a.vtan[c];
    float2 iv = a.inv[c];
    float s = k == 0 ? iv.x : iv.y;
    Nrm3 r;
    r.y = f3(y.x, y.y, y.z);
    r.inv = fabsf(s);
    r.big = s > 0.f;
    return r;
}

// dL/d(normal sum) of vertex c: the adjoint of its normalisation (k_frame_bwd1's tmp_n)
__device__ __forceinline__ float3 sum_grad(const FrameArgs& a, int c, int k) {
    const double* g = (k == 0 ? a.g_nrm : a.g_tan) + 3 * c;
    return nrm3_bwd(stored_nrm3(a, c, k), f3((float)g[0], (float)g[1], (float)g[2]));
}

// phase 1: gradients w.r.t. the unnormalised sums
__global__ void k_frame_bwd1(FrameArgs a) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.V) return;
    float3 n, t;
    vertex_sums(a, v, n, t);
    float3 gn = nrm3_bwd(nrm3(n), f3((float)a.g_nrm[3 * v], (float)a.g_nrm[3 * v + 1], (float)a.g_nrm[3 * v + 2]));
    float3 gt = nrm3_bwd(nrm3(t), f3((float)a.g_tan[3 * v], (float)a.g_tan[3 * v + 1], (float)a.g_tan[3 * v + 2]));
    a.tmp_n[v] = make_float4(gn.x, gn.y, gn.z, 0.f);
    a.tmp_t[v] = make_float4(gt.x, gt.y, gt.z, 0.f);
}

// g_pos[v] += the pixel stage's float64 position gradient + g (the frame adjoint);
// the float64 accumulator is zeroed for the next backward
__device__ __forceinline__ void fold_position_grad(const FrameArgs& a, int v, float3 g) {
    double* acc = a.g_pos_acc + 3 * v;
    double g0 = acc[0] + (double)g.x, g1 = acc[1] + (double)g.y, g2 = acc[2] + (double)g.z;
    if (a.status && !(isfinite(g0) && isfinite(g1) && isfinite(g2))) atomicExch(a.status, (int)ADMS_ERR_NONFINITE);
    a.g_pos[3 * v] += (float)g0;
    a.g_pos[3 * v + 1] += (float)g1;
    a.g_pos[3 * v + 2] += (float)g2;
    acc[0] = 0.0;
    acc[1] = 0.0;
    acc[2] = 0.0;
}

// phase 2: each vertex gathers its share of every incident face's adjoint
__global__ void k_frame_bwd2(FrameArgs a) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.V) return;
    float3 g = zero3();
    int lo = a.vf_off[v], hi = a.vf_off[v + 1];
    for (int j0 = lo; j0 < hi; j0 += ADMS_GATHER) {
        FaceFrame ff[ADMS_GATHER];
        float3 Gfn[ADMS_GATHER], Gft[ADMS_GATHER];
#pragma unroll
        for (int q = 0; q < ADMS_GATHER; ++q) {
            ff[q] = face_frame(a, a.vf_face[min(j0 + q, hi - 1)]);
            Gfn[q] = f3(a.tmp_n[ff[q].idx[0]]) + f3(a.tmp_n[ff[q].idx[1]]) + f3(a.tmp_n[ff[q].idx[2]]);
            Gft[q] = f3(a.tmp_t[ff[q].idx[0]]) + f3(a.tmp_t[ff[q].idx[1]]) + f3(a.tmp_t[ff[q].idx[2]]);
        }
#pragma unroll
        for (int q = 0; q < ADMS_GATHER; ++q) {
            if (j0 + q >= hi) continue;
            float3 ge1 = cross3(ff[q].e2, Gfn[q]), ge2 = cross3(Gfn[q], ff[q].e1);
            if (ff[q].sgn != 0) {
                float3 gtv = (float)ff[q].sgn * nrm3_bwd(nrm3(ff[q].tv), Gft[q]);
                ge1 += ff[q].d2y * gtv;
                ge2 -= ff[q].d1y * gtv;
            }
            if (ff[q].idx[0] == v) g -= ge1 + ge2;
            if (ff[q].idx[1] == v) g += ge1;
            if (ff[q].idx[2] == v) g += ge2;
        }
    }
    fold_position_grad(a, v, g);
}

// k_frame_bwd1 and k_frame_bwd2 in one launch, after a frame_forward that kept the
// normalisations (a.inv): eight threads per vertex, slot s taking the vertex's
// incident faces s, s + 8, ... and forming their corners' normalisation adjoints
// itself; the slots' sums are combined by shuffles in a fixed order
#define ADMS_FRAME_SLOTS 8
__global__ void k_frame_bwd_fused(FrameArgs a) {
    int gid = blockIdx.x * blockDim.x + threadIdx.x;
    int v = gid / ADMS_FRAME_SLOTS, slot = gid % ADMS_FRAME_SLOTS;
    bool valid = v < a.V;
    float3 g = zero3();
    if (valid) {
        int lo = a.vf_off[v], hi = a.vf_off[v + 1];
        for (int j = lo + slot; j < hi; j += ADMS_FRAME_SLOTS) {
            FaceFrame ff = face_frame(a, a.vf_face[j]);
            float3 Gfn = sum_grad(a, ff.idx[0], 0) + sum_grad(a, ff.idx[1], 0) + sum_grad(a, ff.idx[2], 0);
            float3 ge1 = cross3(ff.e2, Gfn), ge2 = cross3(Gfn, ff.e1);
            if (ff.sgn != 0) {
                float3 Gft = sum_grad(a, ff.idx[0], 1) + sum_grad(a, ff.idx[1], 1) + sum_grad(a, ff.idx[2], 1);
                float3 gtv = (float)ff.sgn * nrm3_bwd(nrm3(ff.tv), Gft);
                ge1 += ff.d2y * gtv;
                ge2 -= ff.d1y * gtv;
            }
            if (ff.idx[0] == v) g -= ge1 + ge2;
            if (ff.idx[1] == v) g += ge1;
            if (ff.idx[2] == v) g += ge2;
        }
    }
    // the eight slots of a vertex are consecutive lanes of one warp
#pragma unroll
    for (int o = ADMS_FRAME_SLOTS / 2; o > 0; o >>= 1) {
        g.x += __shfl_down_sync(0xffffffffu, g.x, o, ADMS_FRAME_SLOTS);
        g.y += __shfl_down_sync(0xffffffffu, g.y, o, ADMS_FRAME_SLOTS);
        g.z += __shfl_down_sync(0xffffffffu, g.z, o, ADMS_FRAME_SLOTS);
    }
    if (valid && slot == 0) fold_position_grad(a, v, g);
}

cudaError_t frame_forward(const FrameArgs& a, cudaStream_t st) {
    k_frame_fwd<<<(a.V + 127) / 128, 128, 0, st>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t frame_backward(const FrameArgs& a, cudaStream_t st) {
    if (a.inv) {
        k_frame_bwd_fused<<<(a.V * ADMS_FRAME_SLOTS + 127) / 128, 128, 0, st>>>(a);
        count_launches(1);
        return cudaGetLastError();
    }
    k_frame_bwd1<<<(a.V + 127) / 128, 128, 0, st>>>(a);
    k_frame_bwd2<<<(a.V + 127) / 128, 128, 0, st>>>(a);
    count_launches(2);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ Laplacian (Eq. 4)
__global__ void k_lap_fwd(LapArgs a) {
    __shared__ double red[4];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (i < a.V) {
        int lo = a.ring_off[i], hi = a.ring_off[i + 1];
        float3 m = zero3();
        for (int j0 = lo; j0 < hi; j0 += ADMS_GATHER) {
            float3 pk[ADMS_GATHER];
#pragma unroll
            for (int q = 0; q < ADMS_GATHER; ++q) {
                int k = a.ring[min(j0 + q, hi - 1)];
                pk[q] = f3(a.pos[3 * k], a.pos[3 * k + 1], a.pos[3 * k + 2]);
            }
#pragma unroll
            for (int q = 0; q < ADMS_GATHER; ++q)
                if (j0 + q < hi) m += pk[q];
        }
        float inv = hi > lo ? 1.f / (float)(hi - lo) : 0.f;
        float3 d = f3(a.pos[3 * i], a.pos[3 * i + 1], a.pos[3 * i + 2]) - inv * m;
        if (a.delta_ref) d -= f3(a.delta_ref[3 * i], a.delta_ref[3 * i + 1], a.delta_ref[3 * i + 2]);
        a.delta[3 * i] = d.x;
        a.delta[3 * i + 1] = d.y;
        a.delta[3 * i + 2] = d.z;
        s = (double)dot3(d, d);
    }
    s = warp_sum_d(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(&a.st->lap_sum, red[0] + red[1] + red[2] + red[3]);
}

// g -= sum over the one-ring i of vertex k of delta_i / |ring(i)| (the adjoint of
// the one-ring means, gathered per vertex)
__device__ __forceinline__ void ring_adjoint(const LapArgs& a, int k, float3& g) {
    int lo = a.ring_off[k], hi = a.ring_off[k + 1];
    for (int j0 = lo; j0 < hi; j0 += ADMS_GATHER) {
        float inv[ADMS_GATHER];
        float3 d[ADMS_GATHER];
#pragma unroll
        for (int q = 0; q < ADMS_GATHER; ++q) {
            int i = a.ring[min(j0 + q, hi - 1)];
            inv[q] = 1.f / (float)(a.ring_off[i + 1] - a.ring_off[i]);
            d[q] = f3(a.delta[3 * i], a.delta[3 * i + 1], a.delta[3 * i + 2]);
        }
#pragma unroll
        for (int q = 0; q < ADMS_GATHER; ++q)
            if (j0 + q < hi) g -= inv[q] * d[q];
    }
}

__global__ void k_lap_bwd(LapArgs a) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.V) return;
    float lam = a.st->lam;
    float scale = 2.f * lam / (float)a.V;
    float3 g = f3(a.delta[3 * k], a.delta[3 * k + 1], a.delta[3 * k + 2]);
    ring_adjoint(a, k, g);
    a.g_pos[3 * k] += scale * g.x;
    a.g_pos[3 * k + 1] += scale * g.y;
    a.g_pos[3 * k + 2] += scale * g.z;
}

cudaError_t laplacian_forward(const LapArgs& a, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(&a.st->lap_sum, 0, sizeof(double), st);
    if (e) return e;
    k_lap_fwd<<<(a.V + 127) / 128, 128, 0, st>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

__global__ void k_lap_value(LapArgs a, float* out) { *out = (float)(a.st->lap_sum / (double)a.V); }

// g = scale * dL_delta/dpos, written (not accumulated) into a.g_pos
__global__ void k_lap_grad_out(LapArgs a, float scale) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.V) return;
    float s = 2.f * scale / (float)a.V;
    float3 g = f3(a.delta[3 * k], a.delta[3 * k + 1], a.delta[3 * k + 2]);
    ring_adjoint(a, k, g);
    a.g_pos[3 * k] = s * g.x;
    a.g_pos[3 * k + 1] = s * g.y;
    a.g_pos[3 * k + 2] = s * g.z;
}

cudaError_t laplacian_value(const LapArgs& a, float* out, cudaStream_t st) {
    k_lap_value<<<1, 1, 0, st>>>(a, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t laplacian_gradient(const LapArgs& a, float scale, cudaStream_t st) {
    k_lap_grad_out<<<(a.V + 127) / 128, 128, 0, st>>>(a, scale);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t laplacian_backward(const LapArgs& a, cudaStream_t st) {
    k_lap_bwd<<<(a.V + 127) / 128, 128, 0, st>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace adms
