// Shared device helpers and host error plumbing of the sm_103a rasteriser.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gsplat103.h"

namespace gs {

constexpr int kTile = GS_TILE;
constexpr unsigned kFull = 0xffffffffu;

// Records a message for gs_last_error() and returns `code`.
int fail(int code, const char* fmt, ...);
// GS_OK, or GS_ERR_CUDA with the launch error of the kernels just enqueued.
int launch_status(const char* what);
// Adds n to the library-wide count of enqueued kernels.
void count_launches(int n);

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Index of the view that owns projection p: the largest v with
// proj_offset <= p (views are laid out in increasing offsets; an empty view
// shares its offset with the next one, so the largest match is the owner).
__device__ __forceinline__ int view_of_projection(const GsView* __restrict__ views, int V, int64_t p)
{
    int lo = 0, hi = V - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (views[mid].proj_offset <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Index of the view that owns global tile id `tile`.
__device__ __forceinline__ int view_of_tile(const GsView* __restrict__ views, int V, int tile)
{
    int lo = 0, hi = V - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (views[mid].tile_offset <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Carves consecutive 256-byte aligned sub-buffers out of a workspace.
struct Carver {
    char* base;
    size_t used = 0;
    explicit Carver(void* b) : base(static_cast<char*>(b)) {}
    template <typename T>
    T* take(size_t count)
    {
        T* p = reinterpret_cast<T*>(base ? base + used : nullptr);
        used += align256(count * sizeof(T));
        return p;
    }
};

}  // namespace gs
