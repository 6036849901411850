// Shared device helpers and host error plumbing of the sm_103a rasteriser.
#pragma once

#include <cuda_runtime.h>
#include <climits>
#include <stdint.h>

#include "gsplat103.h"

#include <nvtx3/nvToolsExt.h>

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

// Programmatic dependent launch.  A kernel enqueued with launch_pdl may be
// scheduled while the kernel before it in the stream is still draining, so
// its launch latency and block start-up overlap that tail.  Every kernel of
// the library therefore begins with pdl_wait() -- which returns once all work
// it depends on has completed and its writes are visible -- before it reads
// anything, and then calls pdl_trigger() so that the next kernel may be
// scheduled in turn.  Both are no-ops for a kernel launched the usual way.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl_smem(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                                   Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t stream, Args... args)
{
    return launch_pdl_smem(kernel, grid, block, 0, stream, args...);
}

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

// An NVTX range over one C-ABI call, named after it: profilers that collect NVTX
// (Nsight Systems, ncu's --nvtx filters) see every stage; without one attached
// the push and pop return at once.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Vector types for the fp32 and fp64 instantiations of the kernels: V2/V4 have
// the size and alignment of 2/4 scalars, so they load and store as one vector.
// fp32 uses CUDA's own float2/float4; fp64 uses aligned structs.
struct alignas(16) Double2 {
    double x, y;
};
struct alignas(32) Double4 {
    double x, y, z, w;
};
template <typename S> struct VecOf;
template <> struct VecOf<float> {
    using V2 = float2;
    using V4 = float4;
};
template <> struct VecOf<double> {
    using V2 = Double2;
    using V4 = Double4;
};
template <typename S> using V2 = typename VecOf<S>::V2;
template <typename S> using V4 = typename VecOf<S>::V4;

// d[0..2] += (x, y, z) and d[0..3] += (x, y, z, w) with reduction atomics: in
// fp32 an 8-byte (16-byte) aligned run goes as one 2-vector (4-vector) atomic,
// each component still added on its own, so the results are those of the
// scalar atomics.
__device__ __forceinline__ void atomic_add3(float* d, float x, float y, float z)
{
    if ((reinterpret_cast<uintptr_t>(d) & 7u) == 0) {
        atomicAdd(reinterpret_cast<float2*>(d), make_float2(x, y));
        atomicAdd(d + 2, z);
    } else {
        atomicAdd(d, x);
        atomicAdd(reinterpret_cast<float2*>(d + 1), make_float2(y, z));
    }
}
__device__ __forceinline__ void atomic_add3(double* d, double x, double y, double z)
{
    atomicAdd(d, x);
    atomicAdd(d + 1, y);
    atomicAdd(d + 2, z);
}
__device__ __forceinline__ void atomic_add4(float* d, float x, float y, float z, float w)
{
    if ((reinterpret_cast<uintptr_t>(d) & 15u) == 0) {
        atomicAdd(reinterpret_cast<float4*>(d), make_float4(x, y, z, w));
    } else {
        atomic_add3(d, x, y, z);
        atomicAdd(d + 3, w);
    }
}
__device__ __forceinline__ void atomic_add4(double* d, double x, double y, double z, double w)
{
    atomic_add3(d, x, y, z);
    atomicAdd(d + 3, w);
}

template <typename S>
__device__ __forceinline__ V4<S> mk4(S x, S y, S z, S w)
{
    V4<S> v;
    v.x = x; v.y = y; v.z = z; v.w = w;
    return v;
}

// Correctly rounded product that the compiler may not fuse into an FMA.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

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
