// Visibility keys without any allocation, for callers that cannot call
// cudaMalloc: code running inside another framework's memory pool or a
// pre-sized arena, or a real-time loop where allocation (and the
// synchronisation it implies) is not allowed. It runs the same transform,
// setup, small-triangle, binning and tile kernels as the context-based path,
// with their scratch carved out of one file-scope device array.
#include <mutex>

#include "kernels.cuh"

using namespace adms;

namespace {

constexpr size_t kScratchBytes = 32u << 20;  // every GPU that loads the library holds this until exit
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

unsigned char* g_scratch_dev[kMaxDevices] = {nullptr};  // device address of the array, per device
std::mutex g_scratch_mu;

// Offsets of the scratch parts in the array, computed with checked arithmetic:
// false when a product or sum overflows or the fixed-size parts (plus four tile-list
// entries per tile) do not fit, so no request can wrap around the size check.
struct Layout {
    size_t clip, scr, vs, rec, bin, asign, silmask, adj, tile_count, tile_off, tile_cursor, total, overflow, list;
};

bool add_part(size_t& off, size_t n, size_t elem, size_t& at) {
    size_t bytes;
    if (__builtin_mul_overflow(n, elem, &bytes) || bytes > kScratchBytes) return false;
    at = off;
    off += (bytes + 255) & ~size_t(255);  // both below 2^26 here: no overflow
    return off <= kScratchBytes;
}

bool plan_layout(size_t B, size_t V, size_t F, size_t ntiles, Layout& L) {
    size_t BV, BF, F3, off = 0;
    if (__builtin_mul_overflow(B, V, &BV) || __builtin_mul_overflow(B, F, &BF) || __builtin_mul_overflow(F, (size_t)3, &F3))
        return false;
    bool ok = add_part(off, BV, sizeof(float4), L.clip) && add_part(off, BV, sizeof(float4), L.scr) &&
              add_part(off, BV, sizeof(VtxS), L.vs) && add_part(off, BF, sizeof(TriRec), L.rec) &&
              add_part(off, BF, sizeof(TriBin), L.bin) && add_part(off, BF, 1, L.asign) &&
              add_part(off, BF, 1, L.silmask) && add_part(off, F3, sizeof(int), L.adj) &&
              add_part(off, ntiles, sizeof(int), L.tile_count) && add_part(off, ntiles, sizeof(int), L.tile_off) &&
              add_part(off, ntiles, sizeof(int), L.tile_cursor) && add_part(off, 1, sizeof(long long), L.total) &&
              add_part(off, 1, sizeof(unsigned long long), L.overflow);
    // at least 4 list entries per tile; a tile whose list does not fit scans every triangle instead
    if (!ok || ntiles > (kScratchBytes - off) / (4 * sizeof(int))) return false;
    L.list = off;
    return true;
}

}  // namespace

extern "C" adms_status adms_visibility_noalloc(const float* pos, int32_t n_verts, const int32_t* tri, int32_t n_tris,
                                               const adms_view* views, int32_t n_views, int32_t H, int32_t W,
                                               uint64_t* keys, void* cuda_stream) {
    if (!pos || !tri || !views || !keys || n_verts <= 0 || n_tris <= 0 || n_views <= 0 || H <= 0 || W <= 0 ||
        H > 16384 || W > 16384)
        return ADMS_ERR_ARG;
    size_t B = (size_t)n_views, V = (size_t)n_verts, F = (size_t)n_tris;
    int tiles_x = (W + ADMS_TILE - 1) / ADMS_TILE, tiles_y = (H + ADMS_TILE - 1) / ADMS_TILE;
    size_t ntiles = B * (size_t)tiles_x * (size_t)tiles_y;  // < 2^31 * 2^20: no overflow
    Layout L;
    if (!plan_layout(B, V, F, ntiles, L)) return ADMS_ERR_ARG;  // checked before any CUDA call
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ADMS_ERR_CUDA;
    unsigned char* base;
    {
        // first call on a device: look up the array's device address with that device current
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_dev[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ADMS_ERR_CUDA;
            g_scratch_dev[dev] = static_cast<unsigned char*>(p);
        }
        base = g_scratch_dev[dev];
    }
    RasterScratch s{};
    s.clip = reinterpret_cast<float4*>(base + L.clip);
    s.scr = reinterpret_cast<float4*>(base + L.scr);
    s.vs = reinterpret_cast<VtxS*>(base + L.vs);
    s.rec = reinterpret_cast<TriRec*>(base + L.rec);
    s.bin = reinterpret_cast<TriBin*>(base + L.bin);
    s.asign = reinterpret_cast<int8_t*>(base + L.asign);
    // the shared setup pass also derives silhouette masks; with no adjacency given
    // (all -1) they are computed and left unused
    s.silmask = reinterpret_cast<uint8_t*>(base + L.silmask);
    int* adj = reinterpret_cast<int*>(base + L.adj);
    s.tile_count = reinterpret_cast<int*>(base + L.tile_count);
    s.tile_off = reinterpret_cast<int*>(base + L.tile_off);
    s.tile_cursor = reinterpret_cast<int*>(base + L.tile_cursor);
    s.total_pairs = reinterpret_cast<long long*>(base + L.total);
    s.overflow_ctr = reinterpret_cast<unsigned long long*>(base + L.overflow);
    s.list = reinterpret_cast<int*>(base + L.list);
    s.list_capacity = (long long)((kScratchBytes - L.list) / sizeof(int));

    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the array keeps the previous call's contents: clear what must start at zero (or -1)
    if (cudaMemsetAsync(s.overflow_ctr, 0, sizeof(unsigned long long), st) != cudaSuccess) return ADMS_ERR_CUDA;
    if (cudaMemsetAsync(adj, 0xFF, F * 3 * sizeof(int), st) != cudaSuccess) return ADMS_ERR_CUDA;
    RasterIn in;
    in.pos = pos;
    in.tri = tri;
    in.adj = adj;
    in.views = views;
    in.B = n_views;
    in.V = n_verts;
    in.F = n_tris;
    in.W = W;
    in.H = H;
    in.keys = reinterpret_cast<unsigned long long*>(keys);
    if (raster_views(in, s, st) != cudaSuccess) return ADMS_ERR_CUDA;
    return ADMS_OK;
}
