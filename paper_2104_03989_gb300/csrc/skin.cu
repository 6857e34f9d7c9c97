// Dense linear-blend skinning (Eq. 2): v^s_i = sum_b w_ib M_b [v_i; 1] with affine
// bone matrices of the frame being rendered, and its adjoint to the rest
// positions and to every vertex-bone weight.
//
// The skinned positions feed the bit-exact visibility, so their arithmetic is
// fixed: bones in ascending order; row r of M_b v is ((M[r][0] x + M[r][1] y) +
// M[r][2] z) + M[r][3]; the weighted sum starts at 0 and adds w_ib * t_r; every
// operation rounded once (no FMA).
//
// A (V x B) x (B x 12) contraction per call, but a few MFLOP at the sizes the
// path meets (thousands of vertices, tens of bones): one thread per vertex with
// the frame's bones staged in shared memory; no tensor-core tiling pays here.
#include "kernels.cuh"

namespace adms {

__global__ void k_skin_fwd(SkinArgs a) {
    extern __shared__ float sb[];  // [B][12]: the first three rows of each bone
    for (int k = threadIdx.x; k < a.B * 12; k += blockDim.x) sb[k] = a.bones[(k / 12) * 16 + k % 12];
    __syncthreads();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.V) return;
    float x = a.pos[3 * i], y = a.pos[3 * i + 1], z = a.pos[3 * i + 2];
    float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
    const float* w = a.w + (size_t)i * a.B;
    for (int b = 0; b < a.B; ++b) {
        const float* M = sb + 12 * b;
        float wb = w[b];
        float t0 = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(M[0], x), __fmul_rn(M[1], y)), __fmul_rn(M[2], z)), M[3]);
        float t1 = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(M[4], x), __fmul_rn(M[5], y)), __fmul_rn(M[6], z)), M[7]);
        float t2 = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(M[8], x), __fmul_rn(M[9], y)), __fmul_rn(M[10], z)), M[11]);
        acc0 = __fadd_rn(acc0, __fmul_rn(wb, t0));
        acc1 = __fadd_rn(acc1, __fmul_rn(wb, t1));
        acc2 = __fadd_rn(acc2, __fmul_rn(wb, t2));
    }
    a.out[3 * i] = acc0;
    a.out[3 * i + 1] = acc1;
    a.out[3 * i + 2] = acc2;
}

// dL/dw_ib = g_i . (M_b [v_i; 1])[0..2]; dL/dv_i = sum_b w_ib M_b[0..2][0..2]^T g_i
// (both accumulated: several backward calls may precede an optimizer step)
__global__ void k_skin_bwd(SkinArgs a) {
    extern __shared__ float sb[];
    for (int k = threadIdx.x; k < a.B * 12; k += blockDim.x) sb[k] = a.bones[(k / 12) * 16 + k % 12];
    __syncthreads();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.V) return;
    float x = a.pos[3 * i], y = a.pos[3 * i + 1], z = a.pos[3 * i + 2];
    float g0 = a.g_out[3 * i], g1 = a.g_out[3 * i + 1], g2 = a.g_out[3 * i + 2];
    float gx = 0.f, gy = 0.f, gz = 0.f;
    const float* w = a.w + (size_t)i * a.B;
    float* gw = a.g_w ? a.g_w + (size_t)i * a.B : nullptr;
    for (int b = 0; b < a.B; ++b) {
        const float* M = sb + 12 * b;
        float wb = w[b];
        if (gw) {
            float t0 = M[0] * x + M[1] * y + M[2] * z + M[3];
            float t1 = M[4] * x + M[5] * y + M[6] * z + M[7];
            float t2 = M[8] * x + M[9] * y + M[10] * z + M[11];
            gw[b] += g0 * t0 + g1 * t1 + g2 * t2;
        }
        gx += wb * (M[0] * g0 + M[4] * g1 + M[8] * g2);
        gy += wb * (M[1] * g0 + M[5] * g1 + M[9] * g2);
        gz += wb * (M[2] * g0 + M[6] * g1 + M[10] * g2);
    }
    a.g_pos[3 * i] += gx;
    a.g_pos[3 * i + 1] += gy;
    a.g_pos[3 * i + 2] += gz;
}

cudaError_t skin_forward(const SkinArgs& a, cudaStream_t st) {
    if (a.V <= 0) return cudaSuccess;
    k_skin_fwd<<<(a.V + 127) / 128, 128, sizeof(float) * 12 * a.B, st>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t skin_backward(const SkinArgs& a, cudaStream_t st) {
    if (a.V <= 0) return cudaSuccess;
    k_skin_bwd<<<(a.V + 127) / 128, 128, sizeof(float) * 12 * a.B, st>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace adms
