// Device helpers shared by the compositing kernels (Sec. 2.2, Eq. 7 and its
// backward, Sec. 3.1): per-scalar constants, the staged form of a projected
// Gaussian, the factored quadratic form sigma, the exact per-warp box cull,
// the tile context of a CTA and the launch-grid helpers.
#pragma once

#include <algorithm>
#include <cstdlib>

#include "gs_common.cuh"

namespace gs {

constexpr int kWarps = 8;

template <typename S> struct RT;  // per-scalar constants and primitives
template <> struct RT<float> {
    static constexpr int kFwdBatch = 256;
    static constexpr int kBwdBatch = 96;   // Gaussians per backward batch (per-warp partial slots)
    static constexpr float kLog2e = 1.4426950408889634f;
    __device__ static float alpha_min() { return GS_ALPHA_MIN; }
    __device__ static float alpha_max() { return GS_ALPHA_MAX; }
    __device__ static float t_min() { return GS_T_MIN; }
    // 2^x on the SFU (PTX ex2.approx.ftz.f32)
    __device__ static float ex2(float x)
    {
        float y;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    __device__ static float rcp(float x) { return __fdividef(1.f, x); }
    __device__ static float stash(int p) { return __int_as_float(p); }
    __device__ static int unstash(float v) { return __float_as_int(v); }
};
template <> struct RT<double> {
    static constexpr int kFwdBatch = 128;
    static constexpr int kBwdBatch = 32;
    static constexpr double kLog2e = 1.4426950408889634;
    __device__ static double alpha_min() { return 1.0 / 255.0; }
    __device__ static double alpha_max() { return 0.99; }
    __device__ static double t_min() { return 1e-4; }
    __device__ static double ex2(double x) { return exp2(x); }
    __device__ static double rcp(double x) { return 1.0 / x; }
    __device__ static double stash(int p) { return (double)p; }
    __device__ static int unstash(double v) { return (int)v; }
};

// One staged Gaussian (4 x V4 = 64 bytes in fp32).  The conic arrives in the
// factored form of the ABI, (a, k, D) with sigma = (a (dx + k dy)^2 + D dy^2) / 2
// (Y = [[a, b], [b, c]] with b = a k, c = a k^2 + D):
//   xy  : mu'.x, mu'.y, opacity, a
//   q   : -log2e/2 * a, k, -log2e/2 * D, b
//   col : r, g, b, D
//   cull: sigma threshold (<0: never reaches 1/255; +inf: never culled),
//         -b/c, c, (backward: the projection index)
template <typename S>
struct Staged {
    V4<S> xy, q, col, cull;
};

// log2(e) * (-sigma) at Delta = (dx, dy); u = dx + k dy is returned too.
// Explicit roundings keep forward and backward bit-identical.
template <typename S>
__device__ __forceinline__ S neg_sigma_log2(const V4<S>& q, S dx, S dy, S& u)
{
    u = fma(q.y, dy, dx);
    return fma(mul_rn(q.x, u), u, mul_rn(mul_rn(q.z, dy), dy));
}

template <typename S>
__device__ __forceinline__ void stage_gaussian(V4<S>* sh_xy, V4<S>* sh_q, V4<S>* sh_col, V4<S>* sh_cull, int j,
                                               V2<S> m, S a, S k, S D, S o, S r, S g, S bl, bool need_cull = true)
{
    const S b = a * k;
    sh_xy[j] = mk4<S>(m.x, m.y, o, a);
    sh_q[j] = mk4<S>(S(-0.5) * RT<S>::kLog2e * a, k, S(-0.5) * RT<S>::kLog2e * D, b);
    sh_col[j] = mk4<S>(r, g, bl, D);
    if (!need_cull) return;  // a walk that takes its cull from elsewhere
    const S c = fma(b, k, D);
    S thr;
    if (!(o >= RT<S>::alpha_min())) {
        thr = S(-1);  // o e^-sigma < 1/255 everywhere
    } else if (!(a > S(0) && D > S(0)) || S(4) * c > S(1e7) * D) {
        thr = S(INFINITY);  // degenerate or extremely elongated conic: never culled
    } else {
        thr = S(1.05) * log(S(255) * o) + S(1e-3);
    }
    sh_cull[j] = mk4<S>(thr, -b / c, c, S(0));
}

// Can the Gaussian reach alpha >= 1/255 at a pixel centre of the box
// [X0, X1] x [Y0, Y1]?  Minimum of sigma over the box: zero when mu' is
// inside, otherwise the least of the four edge minima (on an edge sigma is a
// parabola; its vertex is clamped to the edge).
template <typename S>
__device__ __forceinline__ bool reaches_box(const Staged<S>& g, S X0, S X1, S Y0, S Y1)
{
    const S thr = g.cull.x;
    if (thr < S(0)) return false;
    if (!(thr < S(INFINITY))) return true;
    const S mx = g.xy.x, my = g.xy.y;
    if (mx >= X0 && mx <= X1 && my >= Y0 && my <= Y1) return true;
    const S a = g.xy.w, k = g.q.y, D = g.col.w, kv = g.cull.y;
    auto sig = [&](S dx, S dy) {
        const S u = fma(k, dy, dx);
        return S(0.5) * fma(a * u, u, D * dy * dy);
    };
    const S dxl = mx - X0, dxr = mx - X1, dyt = my - Y0, dyb = my - Y1;
    S smin = sig(dxl, fmin(fmax(kv * dxl, dyb), dyt));
    smin = fmin(smin, sig(dxr, fmin(fmax(kv * dxr, dyb), dyt)));
    smin = fmin(smin, sig(fmin(fmax(-k * dyt, dxr), dxl), dyt));
    smin = fmin(smin, sig(fmin(fmax(-k * dyb, dxr), dxl), dyb));
    return smin <= thr;
}

// The tuned compositing kernels for C channels, run on chunks of up to 3 of them (gs_raster.cu); the
// channel entry points hand small C to them.
int rasterize_fwd_chunks3(const char* who, int C, const GsView* views, int32_t V, int32_t T_total,
                          const float* means2d, const float* conics, const float* opacities, const float* colors,
                          const int32_t* isect_ids, const int32_t* tile_ranges, const float* background, float* out,
                          float* T_final, int32_t* last_idx, int32_t* n_contrib, const GsRasterConfig* config,
                          void* stream);
int rasterize_bwd_chunks3(const char* who, int C, const GsView* views, int32_t V, int64_t P, int32_t T_total,
                          const float* means2d, const float* conics, const float* opacities, const float* colors,
                          const int32_t* isect_ids, const int32_t* tile_ranges, const float* background,
                          const float* T_final, const int32_t* last_idx, const float* dL_dout, float* dL_dmeans2d,
                          float* dL_dconics, float* dL_dopacities, float* dL_dcolors, const GsRasterConfig* config,
                          void* stream);

template <typename S>
struct TileCtx {
    const GsView* view;
    int tx, ty, px, py;
    bool inside;
    int64_t pix;         // packed pixel index
    S cx, cy;            // pixel centre
    S wx0, wx1, wy0, wy1;  // warp's pixel-centre box
    int64_t g_shift;     // g = p + g_shift
};

template <typename S>
__device__ __forceinline__ TileCtx<S> tile_ctx(const GsView* __restrict__ views, int V, int tile)
{
    TileCtx<S> t;
    t.view = views + view_of_tile(views, V, tile);
    const int local = tile - t.view->tile_offset;
    t.tx = local % t.view->tiles_x;
    t.ty = local / t.view->tiles_x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int bx = t.tx * kTile + (w & 1) * 8, by = t.ty * kTile + (w >> 1) * 4;
    t.px = bx + (lane & 7);
    t.py = by + (lane >> 3);
    const int W = t.view->cam.width, H = t.view->cam.height;
    t.inside = t.px < W && t.py < H;
    t.pix = t.view->pixel_offset + (int64_t)t.py * W + t.px;
    t.cx = S(t.px) + S(0.5);
    t.cy = S(t.py) + S(0.5);
    t.wx0 = S(bx) + S(0.5);
    t.wx1 = S(bx) + S(7.5);
    t.wy0 = S(by) + S(0.5);
    t.wy1 = S(by) + S(3.5);
    t.g_shift = (int64_t)t.view->g_begin - t.view->proj_offset;
    return t;
}

template <typename S>
__device__ __forceinline__ Staged<S> load_staged(const V4<S>* sh_xy, const V4<S>* sh_q, const V4<S>* sh_col,
                                                 const V4<S>* sh_cull, int j)
{
    return Staged<S>{sh_xy[j], sh_q[j], sh_col[j], sh_cull[j]};
}

__device__ __forceinline__ void atomic_add2(float2* a, float x, float y)
{
    atomicAdd(a, make_float2(x, y));
}
__device__ __forceinline__ void atomic_add2(Double2* a, double x, double y)
{
    atomicAdd(&a->x, x);
    atomicAdd(&a->y, y);
}

// GS_NO_CULL=1 in the environment visits every (pixel, Gaussian) pair; the
// results must not change (checked by the test-suite).
inline bool cull_enabled()
{
    const char* e = getenv("GS_NO_CULL");
    return !(e && e[0] == '1');
}

// Grid for a launch of `kernel` with `threads` per CTA: one CTA per tile, or a persistent grid.
template <typename K>
inline int raster_grid(K kernel, const GsRasterConfig* cfg, int32_t T_total, unsigned* grid, int threads = 256)
{
    if (!cfg || !cfg->persistent) {
        *grid = (unsigned)T_total;
        return GS_OK;
    }
    int dev = 0, sms = 0, fit = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
        cudaSuccess || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kernel, threads, 0) != cudaSuccess)
        return launch_status("raster grid");
    int per = cfg->ctas_per_sm > 0 ? std::min(cfg->ctas_per_sm, fit) : fit;
    per = std::max(per, 1);
    *grid = (unsigned)std::min<int64_t>((int64_t)per * sms, T_total);
    return GS_OK;
}

inline int check_config(const GsRasterConfig* cfg, const char* who)
{
    if (cfg && cfg->persistent && !cfg->queue) return fail(GS_ERR_INVALID_ARG, "%s: persistent needs a queue", who);
    return GS_OK;
}

}  // namespace gs
