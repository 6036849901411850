// gs_bin_and_sort_static: gs_bin_and_sort with its scratch in a fixed
// file-scope device array, for callers that cannot allocate device memory
// (see gsplat103.h).  It only supplies that array as the workspace of the
// ordinary entry point.
#include <mutex>

#include "gs_common.cuh"

namespace gs {

// gs_sort.cu: the argument checks gs_bin_and_sort makes before its workspace check.
int bin_and_sort_check_args(const char* who, const GsView* views, int32_t V, int64_t P, int32_t T_total,
                            const int16_t* rects, const float* depths, const int32_t* touched, int64_t K_capacity,
                            const int32_t* isect_ids, const int32_t* isect_pos, const int32_t* emit_start,
                            const int32_t* tile_ranges, const int32_t* K_out, const uint32_t* flags);

// Workspace bytes gs_bin_and_sort needs at the static limits, rounded up.
// The entry point re-checks the exact requirement before every call.
constexpr size_t kStaticScratchBytes = size_t(24) << 20;  // 24 MiB

static __device__ __align__(256) unsigned char g_sort_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_scratch_mutex;
static void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_sort_scratch on the current device, looked up once per
// device with that device current.
static int scratch_address(void** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(GS_ERR_CUDA, "gs_bin_and_sort_static: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return fail(GS_ERR_INVALID_ARG, "gs_bin_and_sort_static: device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess || !p)
            return fail(GS_ERR_CUDA, "gs_bin_and_sort_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return GS_OK;
}

}  // namespace gs

using namespace gs;

extern "C" int gs_bin_and_sort_static(const GsView* views, int32_t V, int64_t P, int32_t T_total, const int16_t* rects,
                                      const float* depths, const int32_t* touched, int64_t K_capacity,
                                      int32_t* isect_ids, int32_t* isect_pos, int32_t* emit_start,
                                      int32_t* tile_ranges, int32_t* K_out, uint32_t* flags, void* stream)
{
    gs::NvtxRange nvtx("gs_bin_and_sort_static");
    // argument errors are reported before the first CUDA call (the scratch address lookup)
    const int checked = bin_and_sort_check_args("gs_bin_and_sort_static", views, V, P, T_total, rects, depths, touched,
                                                K_capacity, isect_ids, isect_pos, emit_start, tile_ranges, K_out, flags);
    if (checked != GS_OK) return checked;
    if (P > GS_STATIC_MAX_PROJECTIONS || K_capacity > GS_STATIC_MAX_INTERSECTIONS)
        return fail(GS_ERR_INVALID_ARG,
                    "gs_bin_and_sort_static: P=%lld and K_capacity=%lld must not exceed %d and %d "
                    "(use gs_bin_and_sort with a caller workspace for larger problems)",
                    (long long)P, (long long)K_capacity, GS_STATIC_MAX_PROJECTIONS, GS_STATIC_MAX_INTERSECTIONS);
    const size_t need = gs_bin_and_sort_workspace_size(P, K_capacity, T_total);
    if (need > kStaticScratchBytes)
        return fail(GS_ERR_INVALID_ARG, "gs_bin_and_sort_static: needs %zu bytes of scratch, has %zu", need,
                    kStaticScratchBytes);
    void* scratch = nullptr;
    const int rc = scratch_address(&scratch);
    if (rc != GS_OK) return rc;
    return gs_bin_and_sort(views, V, P, T_total, rects, depths, touched, K_capacity, scratch, kStaticScratchBytes,
                           isect_ids, isect_pos, emit_start, tile_ranges, K_out, flags, stream);
}
