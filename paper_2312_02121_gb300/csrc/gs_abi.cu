// Error reporting, version and batch layout of the C ABI (gsplat103.h).
#include <atomic>
#include <cstdarg>
#include <cstdio>

#include "gs_common.cuh"

namespace gs {

static thread_local char g_last_error[512] = "";
static std::atomic<int64_t> g_launches{0};

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return code;
}

int launch_status(const char* what)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(GS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return GS_OK;
}

}  // namespace gs

extern "C" int gs_version(void) { return 200; }

extern "C" const char* gs_last_error(void) { return gs::g_last_error; }

extern "C" int64_t gs_kernel_launches(void) { return gs::g_launches.load(std::memory_order_relaxed); }

extern "C" int gs_views_layout(GsView* views, int32_t V, int64_t* P_total, int32_t* T_total, int64_t* pix_total)
{
    if (V < 0 || (V > 0 && !views) || !P_total || !T_total || !pix_total)
        return gs::fail(GS_ERR_INVALID_ARG, "gs_views_layout: bad arguments (V=%d)", V);
    int64_t P = 0, T = 0, pix = 0;
    for (int32_t v = 0; v < V; ++v) {
        GsView& w = views[v];
        if (w.cam.width <= 0 || w.cam.height <= 0 || w.g_count < 0 || w.g_begin < 0)
            return gs::fail(GS_ERR_INVALID_ARG, "gs_views_layout: view %d has size %dx%d, g_begin %d, g_count %d", v,
                            w.cam.width, w.cam.height, w.g_begin, w.g_count);
        w.tiles_x = (w.cam.width + GS_TILE - 1) / GS_TILE;
        w.tiles_y = (w.cam.height + GS_TILE - 1) / GS_TILE;
        w.proj_offset = P;
        w.pixel_offset = pix;
        w.tile_offset = static_cast<int32_t>(T);
        w.reserved = 0;
        P += w.g_count;
        T += static_cast<int64_t>(w.tiles_x) * w.tiles_y;
        pix += static_cast<int64_t>(w.cam.width) * w.cam.height;
        if (T >= (int64_t(1) << 31) || P >= (int64_t(1) << 31))
            return gs::fail(GS_ERR_INVALID_ARG, "gs_views_layout: more than 2^31 tiles or projections");
    }
    *P_total = P;
    *T_total = static_cast<int32_t>(T);
    *pix_total = pix;
    return GS_OK;
}
