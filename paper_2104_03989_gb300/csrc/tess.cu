// Edge-midpoint tessellation with displacement mapping (Sec. 5.1, Eq. 3) and
// its adjoint. The topology is fixed at job creation (constant tessellation
// factor); every step recomputes the displaced positions from the latent base
// positions and the scalar displacement map:
//   v = sum_k w_k p_k, n = normalize(sum_k w_k nhat_k), v^d = v + tex2d(t) n
// with nhat the smooth base normals and w the lattice weights of the vertex on
// its owning base face.
//
// The forward follows a float32 contract operation by operation (IEEE RN, no
// FMA, fixed order): these positions decide visibility, and the keys must
// match bit for bit. Base normals: face normals summed over incident faces in
// increasing face order, l2 = (x*x + y*y) + z*z, n = s / sqrt(max(l2, 1e-20));
// positions: v = (w0 pa + w1 pb) + w2 pc, same for the normal sum; bilinear
// displacement d = ((gx gy) t00 + (fx gy) t10) + ((gx fy) t01 + (fx fy) t11).
#include "kernels.cuh"

namespace adms {

__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }

__global__ void k_base_normals_exact(TessArgs a) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.Vb) return;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    for (int j = a.bvf_off[v]; j < a.bvf_off[v + 1]; ++j) {
        const int* t = a.base_tri + 3 * a.bvf_face[j];
        const float* p0 = a.base_pos + 3 * t[0];
        const float* p1 = a.base_pos + 3 * t[1];
        const float* p2 = a.base_pos + 3 * t[2];
        float e1x = sub(p1[0], p0[0]), e1y = sub(p1[1], p0[1]), e1z = sub(p1[2], p0[2]);
        float e2x = sub(p2[0], p0[0]), e2y = sub(p2[1], p0[1]), e2z = sub(p2[2], p0[2]);
        s0 = add(s0, sub(mul(e1y, e2z), mul(e1z, e2y)));
        s1 = add(s1, sub(mul(e1z, e2x), mul(e1x, e2z)));
        s2 = add(s2, sub(mul(e1x, e2y), mul(e1y, e2x)));
    }
    float l2 = add(add(mul(s0, s0), mul(s1, s1)), mul(s2, s2));
    float len = __fsqrt_rn(l2 > 1e-20f ? l2 : 1e-20f);
    a.base_nrm[3 * v] = __fdiv_rn(s0, len);
    a.base_nrm[3 * v + 1] = __fdiv_rn(s1, len);
    a.base_nrm[3 * v + 2] = __fdiv_rn(s2, len);
}

struct TessEval {
    float w[3];
    float v[3], ns[3], len, l2, d;
    float fx, fy;
    int idx[4];
};

__device__ __forceinline__ void tess_eval(const TessArgs& a, int t, TessEval& e) {
    const int* o = a.owner + 3 * t;
    float fn = (float)a.n_seg;
#pragma unroll
    for (int k = 0; k < 3; ++k) e.w[k] = __fdiv_rn((float)a.wts[3 * t + k], fn);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        e.v[c] = add(add(mul(e.w[0], a.base_pos[3 * o[0] + c]), mul(e.w[1], a.base_pos[3 * o[1] + c])),
                     mul(e.w[2], a.base_pos[3 * o[2] + c]));
        e.ns[c] = add(add(mul(e.w[0], a.base_nrm[3 * o[0] + c]), mul(e.w[1], a.base_nrm[3 * o[1] + c])),
                      mul(e.w[2], a.base_nrm[3 * o[2] + c]));
    }
    e.l2 = add(add(mul(e.ns[0], e.ns[0]), mul(e.ns[1], e.ns[1])), mul(e.ns[2], e.ns[2]));
    e.len = __fsqrt_rn(e.l2 > 1e-20f ? e.l2 : 1e-20f);
    float2 uv = a.vert_uv[t];
    float x = sub(mul(uv.x, (float)a.dw), 0.5f), y = sub(mul(uv.y, (float)a.dh), 0.5f);
    float x0 = floorf(x), y0 = floorf(y);
    e.fx = sub(x, x0);
    e.fy = sub(y, y0);
    int ix = (int)x0, iy = (int)y0;
    int ixa = ix & (a.dw - 1);  // u wraps: dw is a power of two
    int ixb = (ixa + 1) & (a.dw - 1);
    int iya = min(max(iy, 0), a.dh - 1), iyb = min(max(iy + 1, 0), a.dh - 1);
    e.idx[0] = iya * a.dw + ixa;
    e.idx[1] = iya * a.dw + ixb;
    e.idx[2] = iyb * a.dw + ixa;
    e.idx[3] = iyb * a.dw + ixb;
    float gx = sub(1.f, e.fx), gy = sub(1.f, e.fy);
    float q0 = mul(mul(gx, gy), a.disp[e.idx[0]]);
    float q1 = mul(mul(e.fx, gy), a.disp[e.idx[1]]);
    float q2 = mul(mul(gx, e.fy), a.disp[e.idx[2]]);
    float q3 = mul(mul(e.fx, e.fy), a.disp[e.idx[3]]);
    e.d = add(add(q0, q1), add(q2, q3));
}

__global__ void k_tess_fwd(TessArgs a) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.Vt) return;
    TessEval e;
    tess_eval(a, t, e);
#pragma unroll
    for (int c = 0; c < 3; ++c) a.pos_out[3 * t + c] = add(e.v[c], mul(e.d, __fdiv_rn(e.ns[c], e.len)));
}

// adjoint: out = v + d n, n = ns / |ns|, v = sum w p, ns = sum w nhat, d = bilinear(disp)
__global__ void k_tess_bwd(TessArgs a) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.Vt) return;
    TessEval e;
    tess_eval(a, t, e);
    float3 g = f3(a.g_pos_t[3 * t], a.g_pos_t[3 * t + 1], a.g_pos_t[3 * t + 2]);
    Nrm3 nn;
    nn.inv = 1.f / e.len;
    nn.big = e.l2 > 1e-20f;
    nn.y = f3(e.ns[0], e.ns[1], e.ns[2]) * nn.inv;
    float g_d = dot3(g, nn.y);
    float3 g_ns = nrm3_bwd(nn, e.d * g);
    const int* o = a.owner + 3 * t;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double* gp = a.g_base_pos + 3 * o[k];
        double* gn = a.g_base_nrm + 3 * o[k];
        atomicAdd(gp, (double)(e.w[k] * g.x));
        atomicAdd(gp + 1, (double)(e.w[k] * g.y));
        atomicAdd(gp + 2, (double)(e.w[k] * g.z));
        atomicAdd(gn, (double)(e.w[k] * g_ns.x));
        atomicAdd(gn + 1, (double)(e.w[k] * g_ns.y));
        atomicAdd(gn + 2, (double)(e.w[k] * g_ns.z));
    }
    if (a.g_disp) {
        float gx = 1.f - e.fx, gy = 1.f - e.fy;
        atomicAdd(a.g_disp + e.idx[0], g_d * gx * gy);
        atomicAdd(a.g_disp + e.idx[1], g_d * e.fx * gy);
        atomicAdd(a.g_disp + e.idx[2], g_d * gx * e.fy);
        atomicAdd(a.g_disp + e.idx[3], g_d * e.fx * e.fy);
    }
}

cudaError_t tess_forward(const TessArgs& a, cudaStream_t st) {
    k_base_normals_exact<<<(a.Vb + 127) / 128, 128, 0, st>>>(a);
    k_tess_fwd<<<(a.Vt + 127) / 128, 128, 0, st>>>(a);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t tess_backward(const TessArgs& a, cudaStream_t st) {
    k_tess_bwd<<<(a.Vt + 127) / 128, 128, 0, st>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace adms
