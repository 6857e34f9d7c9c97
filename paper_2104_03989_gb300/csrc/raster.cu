// Vertex transform, triangle setup, binning and tiled fixed-point rasterization
// with a packed depth|triangle-id z-buffer (Sec. 5.2: rasterization primitive).
//
// The visibility arithmetic is fixed bit for bit so that the keys are exact:
//   clip_r = ((M[r][0] x + M[r][1] y) + M[r][2] z) + M[r][3]   (float32, each op RN, no FMA)
//   sx = (clip.x / clip.w)(W/2) + W/2, sy = H/2 - (clip.y / clip.w)(H/2), X = rint(256 sx)
//   E_ab(S) = (X_b - X_a)(S_y - Y_a) - (Y_b - Y_a)(S_x - X_a) in int64 at S = (256 i + 128, 256 j + 128)
//   covered: every edge of the positively wound triangle has E > 0, or E = 0 on a top/left edge
//   d = (z0 + b1 (z1 - z0)) + b2 (z2 - z0), b1 = (float)E_20 / (float)A, b2 = (float)E_01 / (float)A
//   key = (float_bits(d) << 32) | triangle id, minimum per pixel.
#include "kernels.cuh"

namespace adms {

__device__ __forceinline__ long long floor_div_ll(long long a, long long b) {  // b > 0
    long long q = a / b;
    if ((a % b != 0) && (a < 0)) q -= 1;
    return q;
}
__device__ __forceinline__ long long ceil_div_ll(long long a, long long b) { return -floor_div_ll(-a, b); }

// m0 x + m1 y + m2 z + m3 (float inputs, double-float result)
__device__ __forceinline__ DF df_row(const float* m, float x, float y, float z) {
    DF p0 = df_two_prod(m[0], x), p1 = df_two_prod(m[1], y), p2 = df_two_prod(m[2], z);
    DF s = df_two_sum(p0.hi, p1.hi);
    float t = __fadd_rn(s.lo, __fadd_rn(p0.lo, p1.lo));
    DF u = df_two_sum(s.hi, p2.hi);
    t = __fadd_rn(t, __fadd_rn(u.lo, p2.lo));
    DF v = df_two_sum(u.hi, m[3]);
    t = __fadd_rn(t, v.lo);
    return df_fast_two_sum(v.hi, t);
}
// a / b
__device__ __forceinline__ DF df_div(DF a, DF b) {
    float q1 = __fdiv_rn(a.hi, b.hi);
    DF p = df_two_prod(q1, b.hi);
    // r = a - q1 b, the leading terms cancel exactly up to p.lo
    float r = __fsub_rn(__fadd_rn(__fsub_rn(__fsub_rn(a.hi, p.hi), p.lo), a.lo), __fmul_rn(q1, b.lo));
    return df_fast_two_sum(q1, __fdiv_rn(r, b.hi));
}
// c0 + s q (float c0, s; double-float q)
__device__ __forceinline__ DF df_affine(float c0, float s, DF q) {
    DF p = df_two_prod(q.hi, s);
    float e = __fmaf_rn(q.lo, s, p.lo);
    DF u = df_two_sum(c0, p.hi);
    return df_fast_two_sum(u.hi, __fadd_rn(u.lo, e));
}

// ---------------------------------------------------------------- transform
__global__ void k_transform(const float* __restrict__ pos, int V, const adms_view* __restrict__ views, int B, int W,
                            int H, float4* __restrict__ clip, VtxS* __restrict__ vs, float4* __restrict__ scr,
                            long long* __restrict__ zero_total) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && zero_total) *zero_total = 0;  // the tile-list allocation's counter (k_list_alloc)
    if (i >= B * V) return;
    int b = i / V, v = i - b * V;
    const float* M = views[b].mvp;
    float x = pos[3 * v], y = pos[3 * v + 1], z = pos[3 * v + 2];
    {
        // shading-side screen position to ~48 bits as a (hi, lo) float pair:
        // sx = (W/2) (cx / cw) + W/2, sy = H/2 - (H/2) (cy / cw) in double-float
        // arithmetic (float64 runs at a small fraction of the float32 rate here)
        DF cx = df_row(M, x, y, z), cy = df_row(M + 4, x, y, z), cw = df_row(M + 12, x, y, z);
        float hW = 0.5f * (float)W, hH = 0.5f * (float)H;
        DF sx = df_affine(hW, hW, df_div(cx, cw));
        DF sy = df_affine(hH, -hH, df_div(cy, cw));
        scr[i] = make_float4(sx.hi, sx.lo, sy.hi, sy.lo);
    }
    float c[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        float s = __fadd_rn(__fmul_rn(M[4 * r], x), __fmul_rn(M[4 * r + 1], y));
        s = __fadd_rn(s, __fmul_rn(M[4 * r + 2], z));
        c[r] = __fadd_rn(s, M[4 * r + 3]);
    }
    clip[i] = make_float4(c[0], c[1], c[2], c[3]);
    VtxS o;
    o.X = 0;
    o.Y = 0;
    o.z = 0.f;
    o.ok = 0;
    if (c[3] > 1e-6f) {
        float hW = 0.5f * (float)W, hH = 0.5f * (float)H;
        float sx = __fadd_rn(__fmul_rn(__fdiv_rn(c[0], c[3]), hW), hW);
        float sy = __fsub_rn(hH, __fmul_rn(__fdiv_rn(c[1], c[3]), hH));
        float fx = __fmul_rn(sx, 256.f), fy = __fmul_rn(sy, 256.f);
        if (fabsf(fx) <= 134217728.f && fabsf(fy) <= 134217728.f) {
            o.X = __float2int_rn(fx);
            o.Y = __float2int_rn(fy);
            o.z = __fadd_rn(__fmul_rn(__fdiv_rn(c[2], c[3]), 0.5f), 0.5f);
            o.ok = 1;
        }
    }
    vs[i] = o;
}

// ---------------------------------------------------------------- tile-list allocation
// Each tile's list segment [off, off + count) in the list buffer: a warp scans its 32
// tiles' counts by shuffles and reserves their segments together with one 64-bit
// atomicAdd on *total (zeroed by k_transform), so the segments lie in no particular
// order, as the entries inside a segment already do (the raster's per-pixel minimum
// does not depend on either). Offsets saturate at INT_MAX (the list-capacity check
// catches an overflow); *total ends exact. Many small blocks rather than one large
// scan block: a 1024-thread block does not fit on an SM beside a resident
// streamed-Adam block, which a pipelined step runs at the same time.
__global__ void __launch_bounds__(256) k_list_alloc(const int* __restrict__ count, int n, int* __restrict__ off,
                                                    unsigned long long* __restrict__ total) {
    int i = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31;
    long long c = i < n ? count[i] : 0;
    long long x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    unsigned long long base = 0;
    if (lane == 31 && x > 0) base = atomicAdd(total, (unsigned long long)x);
    base = __shfl_sync(0xffffffffu, base, 31);
    if (i < n) off[i] = (int)min((long long)base + x - c, (long long)0x7fffffff);
}

// ---------------------------------------------------------------- coverage test
// coverage + depth key of one triangle at a sample with oriented edge values
// e0, e1, e2 there, or ADMS_EMPTY_KEY
__device__ __forceinline__ unsigned long long key_of(const TriRec& r, long long e0, long long e1, long long e2) {
    if (e0 < r.thr[0] || e1 < r.thr[1] || e2 < r.thr[2]) return ADMS_EMPTY_KEY;
    // back to the triangle's own vertex order: E_20 = s e1, E_01 = s e2
    long long E20 = r.sg > 0 ? e1 : -e1;
    long long E01 = r.sg > 0 ? e2 : -e2;
    float b1 = __fdiv_rn(__ll2float_rn(E20), r.fA);
    float b2 = __fdiv_rn(__ll2float_rn(E01), r.fA);
    float d = __fadd_rn(__fadd_rn(r.z0, __fmul_rn(b1, r.dz1)), __fmul_rn(b2, r.dz2));
    if (!(d >= 0.f && d <= 1.f)) return ADMS_EMPTY_KEY;
    if (d == 0.f) d = 0.f;
    return ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)r.id;
}

// coverage + depth key of one triangle at one sample, or ADMS_EMPTY_KEY
__device__ __forceinline__ unsigned long long tri_key(const TriRec& r, int Sx, int Sy) {
    return key_of(r, (long long)r.ea[0] * Sx + (long long)r.eb[0] * Sy + r.ec[0],
                  (long long)r.ea[1] * Sx + (long long)r.eb[1] * Sy + r.ec[1],
                  (long long)r.ea[2] * Sx + (long long)r.eb[2] * Sy + r.ec[2]);
}

// keeps the minimum in best
__device__ __forceinline__ void test_tri(const TriRec& r, int Sx, int Sy, unsigned long long& best) {
    unsigned long long key = tri_key(r, Sx, Sy);
    if (key < best) best = key;
}

// keeps the KB smallest keys in kb[0] < kb[1] < ... (a per-sample k-buffer; the
// keys of one sample are distinct, each triangle giving at most one): the
// fragment sinks into place and the largest falls out
template <int KB>
__device__ __forceinline__ void test_tri_kbuf(const TriRec& r, int Sx, int Sy, unsigned long long (&kb)[KB]) {
    unsigned long long key = tri_key(r, Sx, Sy);
    if (key >= kb[KB - 1]) return;
#pragma unroll
    for (int i = 0; i < KB; ++i) {
        unsigned long long lo = key < kb[i] ? key : kb[i];
        key = key < kb[i] ? kb[i] : key;
        kb[i] = lo;
    }
}

// z-buffer update of the direct raster, for dense clouds of small triangles (a
// foliage canopy puts ~160 fragments on each sample). The stored key is read
// first: zlo is a lower bound on every key the triangle can produce, so when it
// is above the stored key the sample is skipped without its coverage test; else
// the key goes in only if it is below the stored one. The stored key only ever
// decreases, so a read that lags behind other threads' updates is never below the
// current minimum and can only let an unneeded test or atomicMin through.
// Without the filter (zfilter = 0: closed surfaces, about two fragments per sample)
// the read would only add a dependent round trip: the key goes straight to atomicMin.
__device__ __forceinline__ void zmin_test(unsigned long long* a, const TriRec& r, int Sx, int Sy,
                                          unsigned long long zlo, int zfilter) {
    if (!zfilter) {
        unsigned long long key = tri_key(r, Sx, Sy);
        if (key != ADMS_EMPTY_KEY) atomicMin(a, key);
        return;
    }
    unsigned long long cur = __ldcg(a);
    if (zlo > cur) return;
    unsigned long long key = tri_key(r, Sx, Sy);
    if (key != ADMS_EMPTY_KEY && key < cur) atomicMin(a, key);
}

// A lower bound on the keys of a triangle with vertex depths z0, z1, z2: its
// interpolated depth d = z0 + b1 (z1 - z0) + b2 (z2 - z0) (b1, b2 >= 0, b1 + b2 <= 1,
// each operation rounded once) is at least min z less a few units of rounding of
// the largest |z| (1e-6 x max(1, |z|) covers them with room), and a key needs d >= 0.
__device__ __forceinline__ unsigned long long key_floor(float z0, float z1, float z2) {
    float zmn = fminf(z0, fminf(z1, z2));
    float zmx = fmaxf(fabsf(z0), fmaxf(fabsf(z1), fabsf(z2)));
    float lo = fmaxf(zmn - 1e-6f * fmaxf(1.f, zmx), 0.f);
    return (unsigned long long)__float_as_uint(lo) << 32;
}

// the setup record of lane src, for every lane of the warp
__device__ __forceinline__ TriRec shfl_rec(const TriRec& r, int src) {
    const unsigned full = 0xffffffffu;
    TriRec o;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        o.ec[k] = __shfl_sync(full, r.ec[k], src);
        o.ea[k] = __shfl_sync(full, r.ea[k], src);
        o.eb[k] = __shfl_sync(full, r.eb[k], src);
        o.thr[k] = __shfl_sync(full, r.thr[k], src);
    }
    o.fA = __shfl_sync(full, r.fA, src);
    o.z0 = __shfl_sync(full, r.z0, src);
    o.dz1 = __shfl_sync(full, r.dz1, src);
    o.dz2 = __shfl_sync(full, r.dz2, src);
    o.sg = __shfl_sync(full, r.sg, src);
    o.id = __shfl_sync(full, r.id, src);
    o.valid = 1;
    int bx = __shfl_sync(full, ((int)(unsigned short)r.bx0) | ((int)r.bx1 << 16), src);
    int by = __shfl_sync(full, ((int)(unsigned short)r.by0) | ((int)r.by1 << 16), src);
    o.bx0 = (short)(bx & 0xffff);
    o.bx1 = (short)(bx >> 16);
    o.by0 = (short)(by & 0xffff);
    o.by1 = (short)(by >> 16);
    return o;
}

// ---------------------------------------------------------------- setup, small triangles, tile counts
// One thread per (view, triangle). Triangles whose pixel bounding box holds at
// most small_px samples are rasterized here directly, one 64-bit atomicMin per
// covered sample (the minimum does not depend on the order); larger ones get a
// setup record and are counted into the tiles they overlap. Direct triangles of
// up to ADMS_SMALL_PX samples loop over their box in their own thread; larger
// direct ones are rasterized by the whole warp, one triangle after another with
// the lanes striding over its box (a thread per triangle left three quarters of
// the lanes idle on a canopy of leaves of 20-300 samples each).
// COOP: the instantiation with the warp-wide path and the filtered z-buffer
// updates, launched when small_px exceeds ADMS_SMALL_PX; the other keeps the
// common case (small_px = ADMS_SMALL_PX) to its own registers.
template <bool COOP>
__global__ void __launch_bounds__(256, COOP ? 3 : 1) k_setup(const int* __restrict__ tri, int F, const VtxS* __restrict__ vs, int V, int B, int W, int H,
                        int tiles_x, int tiles_y, TriRec* __restrict__ rec, TriBin* __restrict__ bin,
                        int8_t* __restrict__ asign, int* __restrict__ tile_count, unsigned long long* __restrict__ keys,
                        int small_px, int zfilter) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool coop = false;  // this lane's triangle goes to the warp-wide direct raster
    TriRec r;
    int b = 0;
    unsigned long long zlo = 0ull;  // lower bound on the triangle's keys (COOP)
    if (i < B * F) {
        b = i / F;
        int f = i - b * F;
        int i0 = tri[3 * f], i1 = tri[3 * f + 1], i2 = tri[3 * f + 2];
        const VtxS* vb = vs + (size_t)b * V;
        VtxS a0 = vb[i0], a1 = vb[i1], a2 = vb[i2];
        TriBin tb;
        tb.bx0 = 1;
        tb.bx1 = 0;
        tb.by0 = 1;
        tb.by1 = 0;
        int8_t sgn = 0;
        if (a0.ok && a1.ok && a2.ok) {
            long long X0 = a0.X, Y0 = a0.Y, X1 = a1.X, Y1 = a1.Y, X2 = a2.X, Y2 = a2.Y;
            long long A = (X1 - X0) * (Y2 - Y0) - (Y1 - Y0) * (X2 - X0);
            if (A != 0) {
                int sg = A > 0 ? 1 : -1;
                sgn = (int8_t)sg;
                long long minX = min(X0, min(X1, X2)), maxX = max(X0, max(X1, X2));
                long long minY = min(Y0, min(Y1, Y2)), maxY = max(Y0, max(Y1, Y2));
                long long ilo = max(ceil_div_ll(minX - 128, 256), 0ll), ihi = min(floor_div_ll(maxX - 128, 256), (long long)W - 1);
                long long jlo = max(ceil_div_ll(minY - 128, 256), 0ll), jhi = min(floor_div_ll(maxY - 128, 256), (long long)H - 1);
                if (ilo <= ihi && jlo <= jhi) {
                    // original-order edges: e0 = 1->2, e1 = 2->0, e2 = 0->1
                    long long px[3] = {X0, X1, X2}, py[3] = {Y0, Y1, Y2};
    #pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        int a = (k + 1) % 3, c = (k + 2) % 3;
                        long long dx = px[c] - px[a], dy = py[c] - py[a];
                        // oriented value s E = a Sx + b Sy + cst with s = sign(A)
                        r.ea[k] = (int)(-sg * dy);
                        r.eb[k] = (int)(sg * dx);
                        r.ec[k] = sg * (dy * px[a] - dx * py[a]);
                        long long odx = sg * dx, ody = sg * dy;
                        r.thr[k] = ((ody < 0) || (ody == 0 && odx > 0)) ? 0 : 1;
                    }
                    r.fA = __ll2float_rn(A);
                    r.sg = sg;
                    r.z0 = a0.z;
                    r.dz1 = __fsub_rn(a1.z, a0.z);
                    r.dz2 = __fsub_rn(a2.z, a0.z);
                    r.id = f;
                    r.valid = 1;
                    r.bx0 = (short)ilo;
                    r.bx1 = (short)ihi;
                    r.by0 = (short)jlo;
                    r.by1 = (short)jhi;
                    long long npx = (ihi - ilo + 1) * (jhi - jlo + 1);
                    if (COOP) zlo = key_floor(a0.z, a1.z, a2.z);
                    if (COOP && npx <= small_px && npx > ADMS_SMALL_PX) {
                        coop = true;
                    } else if (npx <= small_px) {
                        unsigned long long* kb = keys + (size_t)b * H * W;
                        for (int y = (int)jlo; y <= (int)jhi; ++y)
                            for (int x = (int)ilo; x <= (int)ihi; ++x) {
                                if (COOP) {
                                    zmin_test(kb + (size_t)y * W + x, r, 256 * x + 128, 256 * y + 128, zlo, zfilter);
                                } else {
                                    unsigned long long key = tri_key(r, 256 * x + 128, 256 * y + 128);
                                    if (key != ADMS_EMPTY_KEY) atomicMin(kb + (size_t)y * W + x, key);
                                }
                            }
                    } else {
                        rec[i] = r;
                        tb.bx0 = r.bx0;
                        tb.bx1 = r.bx1;
                        tb.by0 = r.by0;
                        tb.by1 = r.by1;
                        int tx0 = (int)ilo / ADMS_TILE, tx1 = (int)ihi / ADMS_TILE;
                        int ty0 = (int)jlo / ADMS_TILE, ty1 = (int)jhi / ADMS_TILE;
                        int* tc = tile_count + (size_t)b * tiles_x * tiles_y;
                        for (int ty = ty0; ty <= ty1; ++ty)
                            for (int tx = tx0; tx <= tx1; ++tx) atomicAdd(tc + ty * tiles_x + tx, 1);
                    }
                }
            }
        }
        asign[i] = sgn;
        bin[i] = tb;
    }
    if (!COOP) return;
    // warp-wide direct raster of the lanes' mid-sized triangles (every lane of the
    // warp reaches this point: none returned early)
    unsigned todo = __ballot_sync(0xffffffffu, coop);
    int lane = threadIdx.x & 31;
    while (todo) {
        int src = __ffs(todo) - 1;
        todo &= todo - 1;
        TriRec t = shfl_rec(r, src);
        int tb_ = __shfl_sync(0xffffffffu, b, src);
        unsigned long long tlo = __shfl_sync(0xffffffffu, zlo, src);
        int bw = t.bx1 - t.bx0 + 1, n = bw * (t.by1 - t.by0 + 1);
        unsigned long long* kb = keys + (size_t)tb_ * H * W;
        for (int q = lane; q < n; q += 32) {
            int y = t.by0 + q / bw, x = t.bx0 + q - (q / bw) * bw;
            zmin_test(kb + (size_t)y * W + x, t, 256 * x + 128, 256 * y + 128, tlo, zfilter);
        }
    }
}

// ---------------------------------------------------------------- tile lists
// Per (view, triangle), after the scan of the tile counts: the triangle's
// silhouette-edge mask, then its entries in the tile lists. Bit e of
// silmask[b][f] is set when edge e of triangle f is a silhouette edge in view b:
// no neighbour across it, or a neighbour whose snapped area has another sign.
__global__ void k_bin_fill(const TriBin* __restrict__ bin, int F, int B, int tiles_x, int tiles_y,
                           const int* __restrict__ tile_off, int* __restrict__ tile_cursor, int* __restrict__ list,
                           long long capacity, const int* __restrict__ adj, const int8_t* __restrict__ asign,
                           uint8_t* __restrict__ silmask) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * F) return;
    int b = i / F, f = i - b * F;
    {
        const int8_t* sg = asign + (size_t)b * F;
        int sf = sg[f];
        uint8_t msk = 0;
        if (sf != 0) {
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                int nb = adj[3 * f + e];
                if (nb < 0 || sg[nb] != sf) msk |= (uint8_t)(1u << e);
            }
        }
        silmask[i] = msk;
    }
    TriBin tb = bin[i];
    if (tb.bx0 > tb.bx1) return;
    size_t tbase = (size_t)b * tiles_x * tiles_y;
    int tx0 = tb.bx0 / ADMS_TILE, tx1 = tb.bx1 / ADMS_TILE, ty0 = tb.by0 / ADMS_TILE, ty1 = tb.by1 / ADMS_TILE;
    for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) {
            size_t t = tbase + ty * tiles_x + tx;
            long long p = (long long)tile_off[t] + atomicAdd(tile_cursor + t, 1);
            if (p < capacity) list[p] = f;
        }
}

// ---------------------------------------------------------------- tiled raster
// One block per (view, 16x16 tile), one pixel per thread; the tile's triangle
// records are staged through shared memory in chunks of 256. Each pixel starts
// from the key left by the small-triangle pass. A tile whose list did not fit
// the list buffer scans every binned triangle of its view instead.
__device__ __forceinline__ void raster_tile_body(const TriRec* __restrict__ rec, const TriBin* __restrict__ bin, int F,
                                                 int W, int H, int tiles_x, int tiles_y,
                                                 const int* __restrict__ tile_off, const int* __restrict__ tile_count,
                                                 const int* __restrict__ list, long long capacity,
                                                 unsigned long long* __restrict__ keys,
                                                 unsigned long long* __restrict__ overflow_ctr, int b, int tile,
                                                 TriRec* sm) {
    int tx = tile % tiles_x, ty = tile / tiles_x;
    int lx = threadIdx.x & 15, ly = threadIdx.x >> 4;
    int px = tx * ADMS_TILE + lx, py = ty * ADMS_TILE + ly;
    int Sx = 256 * px + 128, Sy = 256 * py + 128;
    bool inside = px < W && py < H;
    size_t pix = ((size_t)b * H + py) * W + px;
    size_t t = (size_t)b * tiles_x * tiles_y + tile;
    long long off = tile_off[t];
    int cnt = tile_count[t];
    const TriRec* rb = rec + (size_t)b * F;
    const TriBin* bb = bin + (size_t)b * F;
    bool overflow = off + cnt > capacity;
    int n = overflow ? F : cnt;
    if (n == 0) return;  // no binned triangle: the small-triangle pass left the final keys
    unsigned long long best = inside ? keys[pix] : ADMS_EMPTY_KEY;
    if (overflow && threadIdx.x == 0) atomicAdd(overflow_ctr, 1ull);
    // Each warp shades a 16 x 2 strip of the tile (rows 2w, 2w + 1): the staged records
    // whose pixel box meets a warp's rows go to that warp's list, and each warp walks
    // only its own. The key is a minimum over the same triangles in any order.
    __shared__ unsigned char wlist[8][256];
    __shared__ int wcount[8];
    int warp = threadIdx.x >> 5;
    int row0 = ty * ADMS_TILE;
    for (int c0 = 0; c0 < n; c0 += 256) {
        int m = min(256, n - c0);
        __syncthreads();
        if (threadIdx.x < 8) wcount[threadIdx.x] = 0;
        if ((int)threadIdx.x < m) {
            if (overflow) {
                int id = c0 + threadIdx.x;
                TriBin tb = bb[id];
                if (tb.bx0 <= tb.bx1) sm[threadIdx.x] = rb[id];
                else sm[threadIdx.x].valid = 0;
            } else {
                sm[threadIdx.x] = rb[list[off + c0 + threadIdx.x]];
            }
        }
        __syncthreads();
        unsigned wmask = 0;
        if ((int)threadIdx.x < m && sm[threadIdx.x].valid) {
            int r0 = max((int)sm[threadIdx.x].by0 - row0, 0), r1 = min((int)sm[threadIdx.x].by1 - row0, ADMS_TILE - 1);
            for (int w = r0 >> 1; w <= (r1 >> 1); ++w) wmask |= 1u << w;  // empty when r1 < r0
        }
        for (unsigned mm = wmask; mm; mm &= mm - 1) {
            int w = __ffs(mm) - 1;
            wlist[w][atomicAdd(&wcount[w], 1)] = (unsigned char)threadIdx.x;
        }
        __syncthreads();
        int cntw = wcount[warp];
        for (int j = 0; j < cntw; ++j) {
            const TriRec& r = sm[wlist[warp][j]];
            if (px < r.bx0 || px > r.bx1 || py < r.by0 || py > r.by1) continue;
            test_tri(r, Sx, Sy, best);
        }
    }
    if (inside) keys[pix] = best;
}

__global__ void __launch_bounds__(256) k_raster(const TriRec* __restrict__ rec, const TriBin* __restrict__ bin, int F,
                                                int W, int H, int tiles_x, int tiles_y,
                                                const int* __restrict__ tile_off, const int* __restrict__ tile_count,
                                                const int* __restrict__ list, long long capacity,
                                                unsigned long long* __restrict__ keys,
                                                unsigned long long* __restrict__ overflow_ctr) {
    __shared__ TriRec sm[256];
    raster_tile_body(rec, bin, F, W, H, tiles_x, tiles_y, tile_off, tile_count, list, capacity, keys, overflow_ctr,
                     blockIdx.y, blockIdx.x, sm);
}

// Depth peeling in one pass (Sec. 5.2): per sample the L nearest fragments,
// front to back, which are exactly the layers that L peeling passes with a
// two-sided test on the packed depth|id key would find (the keys of a sample are
// distinct). One block per (view, 16x16 tile) as in k_raster, the tile's records
// staged through shared memory, a KB-entry k-buffer per thread in registers
// (KB >= L); every triangle must be binned (no small-triangle pass). keys holds
// L slices of [B][H][W].
template <int KB>
__global__ void __launch_bounds__(256) k_raster_kbuf(const TriRec* __restrict__ rec, const TriBin* __restrict__ bin,
                                                     int F, int W, int H, int tiles_x, int tiles_y,
                                                     const int* __restrict__ tile_off,
                                                     const int* __restrict__ tile_count, const int* __restrict__ list,
                                                     long long capacity, unsigned long long* __restrict__ keys, int L,
                                                     int B, unsigned long long* __restrict__ overflow_ctr) {
    __shared__ TriRec sm[256];
    int b = blockIdx.y, tile = blockIdx.x;
    int tx = tile % tiles_x, ty = tile / tiles_x;
    int lx = threadIdx.x & 15, ly = threadIdx.x >> 4;
    int px = tx * ADMS_TILE + lx, py = ty * ADMS_TILE + ly;
    int Sx = 256 * px + 128, Sy = 256 * py + 128;
    bool inside = px < W && py < H;
    unsigned long long kb[KB];
#pragma unroll
    for (int i = 0; i < KB; ++i) kb[i] = ADMS_EMPTY_KEY;
    size_t t = (size_t)b * tiles_x * tiles_y + tile;
    long long off = tile_off[t];
    int cnt = tile_count[t];
    const TriRec* rb = rec + (size_t)b * F;
    const TriBin* bb = bin + (size_t)b * F;
    bool overflow = off + cnt > capacity;
    int n = overflow ? F : cnt;
    if (overflow && threadIdx.x == 0) atomicAdd(overflow_ctr, 1ull);
    for (int c0 = 0; c0 < n; c0 += 256) {
        int m = min(256, n - c0);
        __syncthreads();
        if ((int)threadIdx.x < m) {
            if (overflow) {
                int id = c0 + threadIdx.x;
                TriBin tb = bb[id];
                if (tb.bx0 <= tb.bx1) sm[threadIdx.x] = rb[id];
                else sm[threadIdx.x].valid = 0;
            } else {
                sm[threadIdx.x] = rb[list[off + c0 + threadIdx.x]];
            }
        }
        __syncthreads();
        for (int k = 0; k < m; ++k) {
            const TriRec& r = sm[k];
            if (!r.valid) continue;
            if (px < r.bx0 || px > r.bx1 || py < r.by0 || py > r.by1) continue;
            test_tri_kbuf<KB>(r, Sx, Sy, kb);
        }
    }
    if (!inside) return;
    size_t pix = ((size_t)b * H + py) * W + px, layer = (size_t)B * H * W;
#pragma unroll
    for (int i = 0; i < KB; ++i)
        if (i < L) keys[pix + (size_t)i * layer] = kb[i];
}
// persistent: block k takes items k, k + gridDim.x, ... (the items are equal
// 16x16 tiles, so a static stride balances them without a shared counter); the
// jobs' arguments are kernel parameters (up to 64 jobs per launch)
__global__ void __launch_bounds__(256) k_raster_batch(const RasterBatch P, const WorkItem* __restrict__ items, int n,
                                                      int job0) {
    __shared__ TriRec sm[256];
    for (int it = blockIdx.x; it < n; it += gridDim.x) {
        WorkItem w = items[it];
        const RasterJob& R = P.a[w.job - job0];
        int tile = (w.y0 / ADMS_TILE) * R.tiles_x + w.x0 / ADMS_TILE;
        raster_tile_body(R.rec, R.bin, R.F, R.W, R.H, R.tiles_x, R.tiles_y, R.tile_off, R.tile_count, R.list,
                         R.capacity, R.keys, R.overflow_ctr, w.view, tile, sm);
    }
}

int raster_batch_occupancy() {
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_raster_batch, 256, 0);
    return e == cudaSuccess && n > 0 ? n : 1;
}

cudaError_t raster_tiles_batched(const RasterJob* args, const int* item_off, int n_jobs, const WorkItem* items,
                                 int blocks, cudaStream_t st) {
    RasterBatch P;
    for (int j0 = 0; j0 < n_jobs; j0 += ADMS_BATCH_JOBS) {
        int j1 = std::min(n_jobs, j0 + ADMS_BATCH_JOBS);
        int s0 = item_off[j0], n = item_off[j1] - s0;
        if (n <= 0) continue;
        memcpy(P.a, args + j0, sizeof(RasterJob) * (j1 - j0));
        k_raster_batch<<<std::min(blocks, n), 256, 0, st>>>(P, items + s0, n, j0);
        count_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------- host launchers
cudaError_t raster_prepare(const RasterIn& in, RasterScratch& s, cudaStream_t st) {
    int B = in.B, V = in.V, F = in.F, W = in.W, H = in.H;
    int tiles_x = (W + ADMS_TILE - 1) / ADMS_TILE, tiles_y = (H + ADMS_TILE - 1) / ADMS_TILE;
    int ntiles = B * tiles_x * tiles_y;
    cudaError_t e;
    // without a key buffer (every triangle binned: small_px = 0) the keys are left to raster_tiles' caller
    if (in.keys && (e = cudaMemsetAsync(in.keys, 0xFF, sizeof(unsigned long long) * B * H * W, st))) return e;
    if (s.tile_cursor == s.tile_count + ntiles) {  // one buffer: counts, then cursors
        if ((e = cudaMemsetAsync(s.tile_count, 0, sizeof(int) * 2 * ntiles, st))) return e;
    } else {
        if ((e = cudaMemsetAsync(s.tile_count, 0, sizeof(int) * ntiles, st))) return e;
        if ((e = cudaMemsetAsync(s.tile_cursor, 0, sizeof(int) * ntiles, st))) return e;
    }
    int bs = 256;
    k_transform<<<(B * V + bs - 1) / bs, bs, 0, st>>>(in.pos, V, in.views, B, W, H, s.clip, s.vs, s.scr,
                                                    s.total_pairs);
    if (in.small_px > ADMS_SMALL_PX)
        k_setup<true><<<(B * F + bs - 1) / bs, bs, 0, st>>>(in.tri, F, s.vs, V, B, W, H, tiles_x, tiles_y, s.rec,
                                                          s.bin, s.asign, s.tile_count, in.keys, in.small_px, in.zfilter);
    else
        k_setup<false><<<(B * F + bs - 1) / bs, bs, 0, st>>>(in.tri, F, s.vs, V, B, W, H, tiles_x, tiles_y, s.rec,
                                                           s.bin, s.asign, s.tile_count, in.keys, in.small_px, 0);
    k_list_alloc<<<(ntiles + bs - 1) / bs, bs, 0, st>>>(s.tile_count, ntiles, s.tile_off,
                                                       reinterpret_cast<unsigned long long*>(s.total_pairs));
    k_bin_fill<<<(B * F + bs - 1) / bs, bs, 0, st>>>(s.bin, F, B, tiles_x, tiles_y, s.tile_off, s.tile_cursor,
                                                   s.list, s.list_capacity, in.adj, s.asign, s.silmask);
    count_launches(4);
    return cudaGetLastError();
}

cudaError_t raster_tiles(const RasterIn& in, RasterScratch& s, cudaStream_t st) {
    int tiles_x = (in.W + ADMS_TILE - 1) / ADMS_TILE, tiles_y = (in.H + ADMS_TILE - 1) / ADMS_TILE;
    dim3 grid(tiles_x * tiles_y, in.B);
    k_raster<<<grid, 256, 0, st>>>(s.rec, s.bin, in.F, in.W, in.H, tiles_x, tiles_y, s.tile_off, s.tile_count, s.list,
                                   s.list_capacity, in.keys, s.overflow_ctr);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t raster_tiles_peeled(const RasterIn& in, RasterScratch& s, int L, cudaStream_t st) {
    if (L < 1 || L > 16) return cudaErrorInvalidValue;
    int tiles_x = (in.W + ADMS_TILE - 1) / ADMS_TILE, tiles_y = (in.H + ADMS_TILE - 1) / ADMS_TILE;
    dim3 grid(tiles_x * tiles_y, in.B);
#define ADMS_KBUF_LAUNCH(KB)                                                                                        \
    k_raster_kbuf<KB><<<grid, 256, 0, st>>>(s.rec, s.bin, in.F, in.W, in.H, tiles_x, tiles_y, s.tile_off,           \
                                            s.tile_count, s.list, s.list_capacity, in.keys, L, in.B, s.overflow_ctr)
    if (L <= 2) ADMS_KBUF_LAUNCH(2);
    else if (L <= 4) ADMS_KBUF_LAUNCH(4);
    else if (L <= 8) ADMS_KBUF_LAUNCH(8);
    else ADMS_KBUF_LAUNCH(16);
#undef ADMS_KBUF_LAUNCH
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t raster_views(const RasterIn& in, RasterScratch& s, cudaStream_t st) {
    cudaError_t e = raster_prepare(in, s, st);
    if (e) return e;
    return raster_tiles(in, s, st);
}

}  // namespace adms
