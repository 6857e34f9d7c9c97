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

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" adms_status adms_visibility_noalloc(const float* pos, int32_t n_verts, const int32_t* tri, int32_t n_tris,
                                               const adms_view* views, int32_t n_views, int32_t H, int32_t W,
                                               uint64_t* keys, void* cuda_stream) {
    if (!pos || !tri || !views || !keys || n_verts <= 0 || n_tris <= 0 || n_views <= 0 || H <= 0 || W <= 0 ||
        H > 16384 || W > 16384)
        return ADMS_ERR_ARG;
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
    size_t B = (size_t)n_views, V = (size_t)n_verts, F = (size_t)n_tris;
    int tiles_x = (W + ADMS_TILE - 1) / ADMS_TILE, tiles_y = (H + ADMS_TILE - 1) / ADMS_TILE;
    size_t ntiles = B * tiles_x * tiles_y;
    // carve the fixed-size parts; whatever is left holds the tile lists
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return base + o;
    };
    RasterScratch s{};
    s.clip = reinterpret_cast<float4*>(carve(B * V * sizeof(float4)));
    s.scr = reinterpret_cast<float4*>(carve(B * V * sizeof(float4)));
    s.vs = reinterpret_cast<VtxS*>(carve(B * V * sizeof(VtxS)));
    s.rec = reinterpret_cast<TriRec*>(carve(B * F * sizeof(TriRec)));
    s.bin = reinterpret_cast<TriBin*>(carve(B * F * sizeof(TriBin)));
    s.asign = reinterpret_cast<int8_t*>(carve(B * F));
    // the shared setup pass also derives silhouette masks; with no adjacency given
    // (all -1) they are computed and left unused
    s.silmask = reinterpret_cast<uint8_t*>(carve(B * F));
    int* adj = reinterpret_cast<int*>(carve(F * 3 * sizeof(int)));
    s.tile_count = reinterpret_cast<int*>(carve(ntiles * sizeof(int)));
    s.tile_off = reinterpret_cast<int*>(carve(ntiles * sizeof(int)));
    s.tile_cursor = reinterpret_cast<int*>(carve(ntiles * sizeof(int)));
    s.total_pairs = reinterpret_cast<long long*>(carve(sizeof(long long)));
    s.overflow_ctr = reinterpret_cast<unsigned long long*>(carve(sizeof(unsigned long long)));
    // at least 4 list entries per tile; a tile whose list does not fit scans every triangle instead
    if (off + 4 * ntiles * sizeof(int) > kScratchBytes) return ADMS_ERR_ARG;
    s.list = reinterpret_cast<int*>(base + off);
    s.list_capacity = (long long)((kScratchBytes - off) / sizeof(int));

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
