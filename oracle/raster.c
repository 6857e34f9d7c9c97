/*
 * Oracle visibility: vertex transform, fixed-point snapping, scanline coverage
 * with the top-left fill rule, and packed depth|triangle-id keys.
 *
 * TEST INFRASTRUCTURE ONLY. This file is part of the CPU oracle that checks the
 * CUDA path; only the tests, the smoke check and the bench's CPU-baseline leg
 * may load it. It shares no code with the CUDA kernels.
 *
 * The paper rasterizes with the primitives of Laine et al. 2020 (Sec. 5.2,
 * "Differentiable Renderer") and states no fill rule, precision or depth
 * encoding; this file fixes one reading bit for bit:
 *   - clip_r = ((M[r][0] x + M[r][1] y) + M[r][2] z) + M[r][3] in float32,
 *     every operation rounded to nearest (build with -ffp-contract=off);
 *   - sx = (clip.x / clip.w) * (W/2) + W/2, sy = H/2 - (clip.y / clip.w) * (H/2),
 *     X = rint(sx * 256), Y = rint(sy * 256) (8 sub-pixel bits, ties to even);
 *   - a vertex is unusable when clip.w <= 1e-6 or |sx*256|, |sy*256| > 2^27;
 *   - pixel (i, j) samples S = (256 i + 128, 256 j + 128);
 *     E_ab(S) = (X_b - X_a)(S_y - Y_a) - (Y_b - Y_a)(S_x - X_a) in int64;
 *   - both windings are drawn; a sample is covered when every edge of the
 *     positively wound triangle has E > 0, or E == 0 on a top or left edge;
 *   - depth d = (z0 + b1 (z1 - z0)) + b2 (z2 - z0), b1 = (float)E_20 / (float)A,
 *     b2 = (float)E_01 / (float)A in the triangle's own vertex order;
 *     samples with d outside [0, 1] are dropped;
 *   - key = (float_bits(d) << 32) | triangle id, minimum per pixel (equal depth:
 *     lower id wins), empty pixel = all ones.
 * Coverage here is computed per row as an interval of pixels solved from each
 * edge inequality (a scanline), not by testing pixels one at a time.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define GUARD 134217728.0f /* 2^27 sub-pixel units */

static int64_t floor_div(int64_t a, int64_t b) /* b > 0 */
{
    int64_t q = a / b;
    if ((a % b != 0) && (a < 0)) q -= 1;
    return q;
}

static int64_t ceil_div(int64_t a, int64_t b) /* b > 0 */
{
    return -floor_div(-a, b);
}

/* Transform V vertices by one view. Outputs (all caller-owned):
 * clip[V*4], XY[V*2] snapped sub-pixel coordinates, z01[V], ok[V]. */
void oracle_transform(const float* mvp, const float* pos, int V, int W, int H,
                      float* clip, int32_t* XY, float* z01, int8_t* ok)
{
    const float hW = 0.5f * (float)W, hH = 0.5f * (float)H;
    for (int v = 0; v < V; ++v) {
        const float x = pos[3 * v], y = pos[3 * v + 1], z = pos[3 * v + 2];
        float c[4];
        for (int r = 0; r < 4; ++r) {
            const float* m = mvp + 4 * r;
            float a = m[0] * x;
            float b = m[1] * y;
            float s = a + b;
            float t = m[2] * z;
            s = s + t;
            c[r] = s + m[3];
        }
        clip[4 * v + 0] = c[0];
        clip[4 * v + 1] = c[1];
        clip[4 * v + 2] = c[2];
        clip[4 * v + 3] = c[3];
        XY[2 * v] = 0;
        XY[2 * v + 1] = 0;
        z01[v] = 0.0f;
        ok[v] = 0;
        if (!(c[3] > 1e-6f)) continue;
        float qx = c[0] / c[3];
        float qy = c[1] / c[3];
        float sx = qx * hW;
        sx = sx + hW;
        float sy = qy * hH;
        sy = hH - sy;
        float fx = sx * 256.0f, fy = sy * 256.0f;
        if (!(fabsf(fx) <= GUARD) || !(fabsf(fy) <= GUARD)) continue;
        XY[2 * v] = (int32_t)rintf(fx);
        XY[2 * v + 1] = (int32_t)rintf(fy);
        float qz = c[2] / c[3];
        float zz = qz * 0.5f;
        z01[v] = zz + 0.5f;
        ok[v] = 1;
    }
}

/* Displaced tessellated positions in float32 (Sec. 5.1, Eq. 3), the positions
 * that visibility sees for tessellated meshes. Every operation is one IEEE
 * float32 operation, rounded to nearest, in the order written:
 *   face normal fn = e1 x e2 (e1 = p1 - p0, e2 = p2 - p0), component
 *     x = e1.y*e2.z - e1.z*e2.y (and cyclic);
 *   base vertex normal: sum of fn over its incident faces in increasing face
 *     order, starting from 0; l2 = (x*x + y*y) + z*z; n = sum / sqrt(max(l2, 1e-20));
 *   tessellated vertex with integer weights (i0, i1, i2) / n_seg on base face
 *     (a, b, c): w_k = (float)i_k / (float)n_seg,
 *     v = (w0*pa + w1*pb) + w2*pc, s = (w0*na + w1*nb) + w2*nc, normalised as above;
 *   displacement d = bilinear level-0 lookup at (u, v): x = u*W - 0.5,
 *     x0 = floor(x), fx = x - x0 (u wraps, v clamps),
 *     d = ((1-fx)(1-fy) t00 + fx(1-fy) t10) + ((1-fx) fy t01 + fx fy t11);
 *   out = v + d*n.
 * vf_off/vf_face: vertex -> incident faces, faces ascending. */
void oracle_tess_positions(const float* base_pos, const int32_t* base_tri, const int32_t* vf_off,
                           const int32_t* vf_face, int n_base,
                           int n_tess, const int32_t* owner_idx /* [n_tess][3] base vertex ids */,
                           const int32_t* weights /* [n_tess][3] */, int n_seg,
                           const float* vert_uv /* [n_tess][2] */, const float* disp, int dh, int dw,
                           float* base_nrm /* out [n_base][3] */, float* out_pos /* out [n_tess][3] */)
{
    for (int v = 0; v < n_base; ++v) {
        float s[3] = {0.0f, 0.0f, 0.0f};
        for (int j = vf_off[v]; j < vf_off[v + 1]; ++j) {
            const int32_t* t = base_tri + 3 * vf_face[j];
            const float* p0 = base_pos + 3 * t[0];
            const float* p1 = base_pos + 3 * t[1];
            const float* p2 = base_pos + 3 * t[2];
            float e1[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
            float e2[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]};
            float a, b;
            a = e1[1] * e2[2]; b = e1[2] * e2[1]; s[0] = s[0] + (a - b);
            a = e1[2] * e2[0]; b = e1[0] * e2[2]; s[1] = s[1] + (a - b);
            a = e1[0] * e2[1]; b = e1[1] * e2[0]; s[2] = s[2] + (a - b);
        }
        float l2 = s[0] * s[0];
        l2 = l2 + s[1] * s[1];
        l2 = l2 + s[2] * s[2];
        float len = sqrtf(l2 > 1e-20f ? l2 : 1e-20f);
        base_nrm[3 * v] = s[0] / len;
        base_nrm[3 * v + 1] = s[1] / len;
        base_nrm[3 * v + 2] = s[2] / len;
    }
    const float fn = (float)n_seg;
    for (int t = 0; t < n_tess; ++t) {
        const int32_t* o = owner_idx + 3 * t;
        float w0 = (float)weights[3 * t] / fn, w1 = (float)weights[3 * t + 1] / fn, w2 = (float)weights[3 * t + 2] / fn;
        float vv[3], ns[3];
        for (int c = 0; c < 3; ++c) {
            float x = w0 * base_pos[3 * o[0] + c];
            float y = w1 * base_pos[3 * o[1] + c];
            float z = w2 * base_pos[3 * o[2] + c];
            vv[c] = (x + y) + z;
            x = w0 * base_nrm[3 * o[0] + c];
            y = w1 * base_nrm[3 * o[1] + c];
            z = w2 * base_nrm[3 * o[2] + c];
            ns[c] = (x + y) + z;
        }
        float l2 = ns[0] * ns[0];
        l2 = l2 + ns[1] * ns[1];
        l2 = l2 + ns[2] * ns[2];
        float len = sqrtf(l2 > 1e-20f ? l2 : 1e-20f);
        float u = vert_uv[2 * t], vc = vert_uv[2 * t + 1];
        float x = u * (float)dw - 0.5f, y = vc * (float)dh - 0.5f;
        float x0 = floorf(x), y0 = floorf(y);
        float fx = x - x0, fy = y - y0;
        int ix = (int)x0, iy = (int)y0;
        int ixa = ix % dw;
        if (ixa < 0) ixa += dw;
        int ixb = ixa + 1 == dw ? 0 : ixa + 1;
        int iya = iy < 0 ? 0 : (iy > dh - 1 ? dh - 1 : iy);
        int iyb = iy + 1 < 0 ? 0 : (iy + 1 > dh - 1 ? dh - 1 : iy + 1);
        float gx = 1.0f - fx, gy = 1.0f - fy;
        float t00 = disp[iya * dw + ixa], t10 = disp[iya * dw + ixb];
        float t01 = disp[iyb * dw + ixa], t11 = disp[iyb * dw + ixb];
        float q0 = (gx * gy) * t00;
        float q1 = (fx * gy) * t10;
        float q2 = (gx * fy) * t01;
        float q3 = (fx * fy) * t11;
        float d = (q0 + q1) + (q2 + q3);
        for (int c = 0; c < 3; ++c) {
            float nc = ns[c] / len;
            out_pos[3 * t + c] = vv[c] + d * nc;
        }
    }
}

static int64_t edge_fn(int64_t xa, int64_t ya, int64_t xb, int64_t yb, int64_t sx, int64_t sy)
{
    return (xb - xa) * (sy - ya) - (yb - ya) * (sx - xa);
}

/* Rasterize F triangles of one view into keys[H*W] (caller initialises to all
 * ones; keys already present are min-merged). area_sign[F] receives the sign
 * of the snapped signed area (0 for unusable or degenerate triangles).
 * floor_keys (or NULL): a fragment is kept only when its key is strictly
 * greater than floor_keys at its pixel (the two-sided depth test of a depth
 * peeling pass, Sec. 5.2, with the previous layer's keys as the floor). */
static void raster_into(const int32_t* XY, const float* z01, const int8_t* ok,
                        const int32_t* tri, int F, int W, int H, const uint64_t* floor_keys,
                        uint64_t* keys, int8_t* area_sign)
{
    for (int f = 0; f < F; ++f) {
        const int32_t i0 = tri[3 * f], i1 = tri[3 * f + 1], i2 = tri[3 * f + 2];
        area_sign[f] = 0;
        if (!ok[i0] || !ok[i1] || !ok[i2]) continue;
        const int64_t X0 = XY[2 * i0], Y0 = XY[2 * i0 + 1];
        const int64_t X1 = XY[2 * i1], Y1 = XY[2 * i1 + 1];
        const int64_t X2 = XY[2 * i2], Y2 = XY[2 * i2 + 1];
        const int64_t A = edge_fn(X0, Y0, X1, Y1, X2, Y2);
        if (A == 0) continue;
        area_sign[f] = (int8_t)(A > 0 ? 1 : -1);

        /* positively wound vertex order for the coverage test */
        int64_t px[3] = {X0, X1, X2}, py[3] = {Y0, Y1, Y2};
        if (A < 0) {
            px[1] = X2; py[1] = Y2;
            px[2] = X1; py[2] = Y1;
        }
        int64_t ex[3], ey[3], dx[3], dy[3];
        int incl[3];
        for (int k = 0; k < 3; ++k) {
            /* edge k runs from vertex (k+1)%3 to (k+2)%3 */
            const int a = (k + 1) % 3, b = (k + 2) % 3;
            ex[k] = px[a];
            ey[k] = py[a];
            dx[k] = px[b] - px[a];
            dy[k] = py[b] - py[a];
            /* top edge: horizontal, interior below; left edge: going up */
            incl[k] = (dy[k] < 0) || (dy[k] == 0 && dx[k] > 0);
        }
        int64_t minX = X0, maxX = X0, minY = Y0, maxY = Y0;
        if (X1 < minX) minX = X1;
        if (X2 < minX) minX = X2;
        if (X1 > maxX) maxX = X1;
        if (X2 > maxX) maxX = X2;
        if (Y1 < minY) minY = Y1;
        if (Y2 < minY) minY = Y2;
        if (Y1 > maxY) maxY = Y1;
        if (Y2 > maxY) maxY = Y2;
        int64_t ilo = ceil_div(minX - 128, 256), ihi = floor_div(maxX - 128, 256);
        int64_t jlo = ceil_div(minY - 128, 256), jhi = floor_div(maxY - 128, 256);
        if (ilo < 0) ilo = 0;
        if (jlo < 0) jlo = 0;
        if (ihi > W - 1) ihi = W - 1;
        if (jhi > H - 1) jhi = H - 1;

        const float z0 = z01[i0], z1 = z01[i1], z2 = z01[i2];
        const float fA = (float)A;
        const float dz1 = z1 - z0, dz2 = z2 - z0;

        for (int64_t j = jlo; j <= jhi; ++j) {
            const int64_t Sy = 256 * j + 128;
            int64_t lo = ilo, hi = ihi;
            for (int k = 0; k < 3 && lo <= hi; ++k) {
                /* E(i) = K - D i with S_x = 256 i + 128; need E(i) >= t */
                const int64_t K = dx[k] * (Sy - ey[k]) - dy[k] * (128 - ex[k]);
                const int64_t D = 256 * dy[k];
                const int64_t t = incl[k] ? 0 : 1;
                if (D == 0) {
                    if (K < t) hi = lo - 1;
                } else if (D > 0) {
                    const int64_t m = floor_div(K - t, D);
                    if (m < hi) hi = m;
                } else {
                    const int64_t m = ceil_div(t - K, -D);
                    if (m > lo) lo = m;
                }
            }
            for (int64_t i = lo; i <= hi; ++i) {
                const int64_t Sx = 256 * i + 128;
                const int64_t e20 = edge_fn(X2, Y2, X0, Y0, Sx, Sy);
                const int64_t e01 = edge_fn(X0, Y0, X1, Y1, Sx, Sy);
                const float b1 = (float)e20 / fA;
                const float b2 = (float)e01 / fA;
                float u = b1 * dz1;
                float s = z0 + u;
                float w = b2 * dz2;
                float d = s + w;
                if (!(d >= 0.0f && d <= 1.0f)) continue;
                if (d == 0.0f) d = 0.0f; /* canonical +0 */
                uint32_t bits;
                memcpy(&bits, &d, 4);
                const uint64_t key = ((uint64_t)bits << 32) | (uint32_t)f;
                uint64_t* kp = keys + j * (int64_t)W + i;
                if (floor_keys && !(key > floor_keys[j * (int64_t)W + i])) continue;
                if (key < *kp) *kp = key;
            }
        }
    }
}

void oracle_raster(const int32_t* XY, const float* z01, const int8_t* ok,
                   const int32_t* tri, int F, int W, int H,
                   uint64_t* keys, int8_t* area_sign)
{
    raster_into(XY, z01, ok, tri, F, W, H, NULL, keys, area_sign);
}

/* One depth-peeling pass: the nearest fragment behind floor_keys at every pixel. */
void oracle_raster_layer(const int32_t* XY, const float* z01, const int8_t* ok,
                         const int32_t* tri, int F, int W, int H, const uint64_t* floor_keys,
                         uint64_t* keys, int8_t* area_sign)
{
    raster_into(XY, z01, ok, tri, F, W, H, floor_keys, keys, area_sign);
}

/* Skinned positions (Eq. 2) under the float32 contract that visibility uses:
 *   v^s_i = sum over bones b in ascending order of w_ib * (M_b [v_i; 1])[0..2],
 *   where row r of M_b v is ((M[r][0] x + M[r][1] y) + M[r][2] z) + M[r][3],
 *   and the weighted sum starts at 0 and adds w_ib * t_r for b = 0, 1, ...;
 *   every operation rounded once (no FMA; built with -ffp-contract=off).
 * pos [V][3], w [V][B] (row per vertex), bones [B][16] row-major 4x4. */
void oracle_skin_positions(const float* pos, int V, const float* w, int B, const float* bones, float* out)
{
    for (int i = 0; i < V; ++i) {
        float x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
        float acc[3] = {0.0f, 0.0f, 0.0f};
        for (int b = 0; b < B; ++b) {
            const float* M = bones + 16 * b;
            float wb = w[(size_t)i * B + b];
            for (int r = 0; r < 3; ++r) {
                float t = M[4 * r] * x;
                t = t + M[4 * r + 1] * y;
                t = t + M[4 * r + 2] * z;
                t = t + M[4 * r + 3];
                acc[r] = acc[r] + wb * t;
            }
        }
        out[3 * i] = acc[0];
        out[3 * i + 1] = acc[1];
        out[3 * i + 2] = acc[2];
    }
}
