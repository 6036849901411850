// Front-to-back compositing (Sec. 2.2, Eq. 7) and its backward (Sec. 3.1) for
// any number of channels per Gaussian (features, depth, ...), fp32.
//
// Eq. 7 composites every channel with the same alpha_n T_n, and Sec. 3.1
// derives every gradient term per channel k, with dL/dalpha_n summed over the
// channels.  So C channels split into chunks that are composited by separate
// launches: each launch rebuilds the same alpha and T (bit-identical
// arithmetic) and writes its chunk of the output.  In the backward each chunk
// adds its share of dL/dalpha, and with it its share of the mu', conic and
// opacity gradients, with atomics.  A chunk has at most 32 channels and is
// handled by a kernel compiled for NC in {1, 2, 4, 8, 16, 32} lanes of
// colour, the smallest that holds it (unused lanes carry zeros).
//
// The tile walk is that of the 3-channel kernels: one 256-thread CTA per 16x16
// tile, one pixel per thread, warps on 8x4 pixel boxes, the exact per-warp box
// cull, branchless bodies.  Colours are staged in shared memory beside the
// geometry.  The backward sums a Gaussian's 6 + NC per-pixel terms over the
// warp through a shared-memory transpose, 16 terms at a time (or takes the
// lone contributing lane's terms), adds them into a per-(tile, Gaussian) slot
// with shared atomics, and flushes the slots to the outputs with global
// atomics.  The deterministic reduction
// of the 3-channel path is not offered here.
#include "gs_raster_common.cuh"

namespace gs {

template <int NC>
struct Nc {
    static constexpr int kB = NC >= 16 ? 128 : 256;  // Gaussians per staged batch (forward)
    // backward batches: smaller, so that the per-warp reduction buffers fit the 48 KB of static
    // shared memory beside the slots
    static constexpr int kBwdB = NC >= 32 ? 64 : NC >= 4 ? 128 : 256;
    static constexpr int kR = 6 + NC;                // dmu'(2) dconic(3) dopacity(1) dcolor(NC)
};

// The warp's sums of r[0..kR) added into slot[0..kR) (shared memory, shared by the CTA's warps),
// kG terms at a time through the warp's 32 x kGS buffer: every lane stores its kG terms as a row,
// lane L then sums column L % kG over rows 16 (L / 16) .. +15, and one shuffle adds the two halves.
// With rows kGS = 17 floats apart the row stores and the column loads are conflict-free.  The
// order is fixed within the warp: 16 adds, then the other half.  (Butterfly shuffles cost 5
// shuffles and 5 adds per term.)
constexpr int kG = 16, kGS = 17;

template <int kR>
__device__ __forceinline__ void warp_add_terms(const float (&r)[kR], float* buf, float* slot, int lane)
{
    float* row = buf + lane * kGS;
    const int col = lane & 15, half = lane >> 4;
    const float* colp = buf + half * 16 * kGS + col;
#pragma unroll
    for (int g0 = 0; g0 < kR; g0 += kG) {
#pragma unroll
        for (int q = 0; q < kG; ++q)
            if (g0 + q < kR) row[q] = r[g0 + q];
        __syncwarp();
        float acc = 0.f;
        if (g0 + col < kR) {
#pragma unroll
            for (int i = 0; i < 16; ++i) acc += colp[i * kGS];
        }
        acc += __shfl_xor_sync(kFull, acc, 16);
        if (half == 0 && g0 + col < kR) atomicAdd(slot + g0 + col, acc);
        __syncwarp();  // the buffer is free again
    }
}

// Stages the colour chunk [c0, c0 + nc) of the batch's Gaussians (sh_g holds
// their Gaussian indices) into sh_c[j][0..NC), zero-padded; coalesced over k.
template <int NC>
__device__ __forceinline__ void stage_colors(float (*sh_c)[NC], const int* sh_g, int n, const float* __restrict__ colors,
                                             int C, int c0, int nc)
{
    for (int i = threadIdx.x; i < n * NC; i += blockDim.x) {
        const int j = i / NC, k = i - j * NC;
        sh_c[j][k] = k < nc ? colors[(int64_t)C * sh_g[j] + c0 + k] : 0.f;
    }
}

template <int NC, bool kCull, bool kPersistent>
__global__ void __launch_bounds__(256)
k_raster_fwd_nc(const GsView* __restrict__ views, int V, int T_total, const int32_t* __restrict__ tile_order,
                int* __restrict__ queue, const float2* __restrict__ means2d, const float* __restrict__ conics,
                const float* __restrict__ opacities, const float* __restrict__ colors, int C, int c0, int nc,
                const int32_t* __restrict__ isect_ids, const int2* __restrict__ tile_ranges,
                const float* __restrict__ background, float* __restrict__ out, float* __restrict__ T_final,
                int32_t* __restrict__ last_idx, int32_t* __restrict__ n_contrib)
{
    pdl_wait();
    pdl_trigger();
    constexpr int kB = Nc<NC>::kB;
    __shared__ float4 sh_xy[kB], sh_q[kB], sh_col[kB], sh_cull[kB];
    __shared__ __align__(16) float sh_c[kB][NC];
    __shared__ int sh_g[kB];
    __shared__ int s_next;
    for (int qi = blockIdx.x;;) {
        if (kPersistent) {
            __syncthreads();
            if (threadIdx.x == 0) s_next = atomicAdd(queue, 1);
            __syncthreads();
            qi = s_next;
            if (qi >= T_total) break;
        }
        const int tile = tile_order ? tile_order[qi] : qi;
        const TileCtx<float> t = tile_ctx<float>(views, V, tile);
        const int lane = threadIdx.x & 31;
        const int2 range = tile_ranges[tile];

        float T = 1.f, acc[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) acc[k] = 0.f;
        int last = range.x - 1, count = 0;
        bool done = !t.inside;

        for (int b0 = range.x; b0 < range.y; b0 += kB) {
            if (__syncthreads_count(done) == (int)blockDim.x) break;  // also guards the stage below
            const int n = min(kB, range.y - b0);
            if (threadIdx.x < n) {
                const int p = isect_ids[b0 + threadIdx.x];
                const int64_t g = p + t.g_shift;
                stage_gaussian<float>(sh_xy, sh_q, sh_col, sh_cull, threadIdx.x, means2d[p], conics[3 * p],
                                      conics[3 * p + 1], conics[3 * p + 2], opacities[g], 0.f, 0.f, 0.f);
                sh_g[threadIdx.x] = (int)g;
            }
            __syncthreads();
            stage_colors<NC>(sh_c, sh_g, n, colors, C, c0, nc);
            __syncthreads();
            for (int s = 0; s < n; s += 32) {
                if (__all_sync(kFull, done)) break;  // a finished warp walks no further chunk
                bool hit = s + lane < n;
                if (kCull && hit)
                    hit = reaches_box(load_staged<float>(sh_xy, sh_q, sh_col, sh_cull, s + lane), t.wx0, t.wx1,
                                      t.wy0, t.wy1);
                unsigned m = __ballot_sync(kFull, hit);
                while (m) {
                    const int j = s + __ffs(m) - 1;
                    m &= m - 1;
                    const float4 xy = sh_xy[j];
                    float u;
                    const float p2 = neg_sigma_log2(sh_q[j], xy.x - t.cx, xy.y - t.cy, u);
                    const float raw = mul_rn(xy.z, RT<float>::ex2(p2));
                    const float alpha = fminf(RT<float>::alpha_max(), raw);
                    const float Tn = fmaf(-T, alpha, T);  // as the 3-channel kernel: T (1 - alpha), one rounding
                    const bool take = !done && p2 <= 0.f && raw >= RT<float>::alpha_min();
                    const bool stop = take && Tn < RT<float>::t_min();
                    const bool comp = take && !stop;
                    done = done || stop;
                    const float wgt = comp ? alpha * T : 0.f;
#pragma unroll
                    for (int k = 0; k < NC; ++k) acc[k] = fmaf(wgt, sh_c[j][k], acc[k]);
                    T = comp ? Tn : T;
                    last = comp ? b0 + j : last;
                    count += comp;
                }
            }
        }
        if (t.inside) {
            float* o = out + (int64_t)C * t.pix + c0;
#pragma unroll
            for (int k = 0; k < NC; ++k)
                if (k < nc) o[k] = fmaf(T, background ? background[c0 + k] : 0.f, acc[k]);
            if (c0 == 0) {  // every chunk computes the same T and last index
                T_final[t.pix] = T;
                last_idx[t.pix] = last;
                if (n_contrib) n_contrib[t.pix] = count;
            }
        }
        if (!kPersistent) break;
    }
}

template <int NC, bool kCull, bool kPersistent>
__global__ void __launch_bounds__(256)
k_raster_bwd_nc(const GsView* __restrict__ views, int V, int T_total, const int32_t* __restrict__ tile_order,
                int* __restrict__ queue, const float2* __restrict__ means2d, const float* __restrict__ conics,
                const float* __restrict__ opacities, const float* __restrict__ colors, int C, int c0, int nc,
                const int32_t* __restrict__ isect_ids, const int2* __restrict__ tile_ranges,
                const float* __restrict__ background, const float* __restrict__ T_final,
                const int32_t* __restrict__ last_idx, const float* __restrict__ dL_dout,
                float2* __restrict__ dL_dmeans2d, float* __restrict__ dL_dconics, float* __restrict__ dL_dopacities,
                float* __restrict__ dL_dcolors)
{
    pdl_wait();
    pdl_trigger();
    constexpr int kB = Nc<NC>::kBwdB, kR = Nc<NC>::kR;
    __shared__ float4 sh_xy[kB], sh_q[kB], sh_col[kB], sh_cull[kB];
    __shared__ float s_red[kWarps][32 * kGS];
    __shared__ __align__(16) float sh_c[kB][NC];
    __shared__ int sh_g[kB];
    __shared__ float s_grad[kB][kR];
    __shared__ unsigned s_mask[(kB + 31) / 32];
    __shared__ int s_maxlast[kWarps];
    __shared__ int s_next;
    for (int qi = blockIdx.x;;) {
        if (kPersistent) {
            __syncthreads();
            if (threadIdx.x == 0) s_next = atomicAdd(queue, 1);
            __syncthreads();
            qi = s_next;
            if (qi >= T_total) break;
        }
        const int tile = tile_order ? tile_order[qi] : qi;
        const TileCtx<float> t = tile_ctx<float>(views, V, tile);
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        const int2 range = tile_ranges[tile];

        float T = 1.f, bgT = 0.f, g[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) g[k] = 0.f;
        int last = range.x - 1;
        if (t.inside) {
            T = T_final[t.pix];
            last = last_idx[t.pix];
            const float* gp = dL_dout + (int64_t)C * t.pix + c0;
#pragma unroll
            for (int k = 0; k < NC; ++k)
                if (k < nc) {
                    g[k] = gp[k];
                    if (background) bgT = fmaf(background[c0 + k], g[k], bgT);
                }
            bgT *= T;
        }
        float SdL = bgT;  // S_n . dL/dC + T_final b . dL/dC over the chunk's channels

        int wl = last;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) wl = max(wl, __shfl_xor_sync(kFull, wl, d));
        if (lane == 0) s_maxlast[w] = wl;
        __syncthreads();
        int maxlast = s_maxlast[0];
#pragma unroll
        for (int i = 1; i < kWarps; ++i) maxlast = max(maxlast, s_maxlast[i]);

        const int nbatch = maxlast >= range.x ? (maxlast - range.x) / kB + 1 : 0;
        for (int kb = nbatch - 1; kb >= 0; --kb) {
            const int b0 = range.x + kb * kB;
            const int n = min(kB, maxlast - b0 + 1);
            for (int i = threadIdx.x; i < kB * kR; i += blockDim.x) (&s_grad[0][0])[i] = 0.f;
            if (threadIdx.x < (kB + 31) / 32) s_mask[threadIdx.x] = 0u;
            if (threadIdx.x < n) {
                const int p = isect_ids[b0 + threadIdx.x];
                const int64_t gg = p + t.g_shift;
                stage_gaussian<float>(sh_xy, sh_q, sh_col, sh_cull, threadIdx.x, means2d[p], conics[3 * p],
                                      conics[3 * p + 1], conics[3 * p + 2], opacities[gg], 0.f, 0.f, 0.f);
                sh_cull[threadIdx.x].w = RT<float>::stash(p);
                sh_g[threadIdx.x] = (int)gg;
            }
            __syncthreads();
            stage_colors<NC>(sh_c, sh_g, n, colors, C, c0, nc);
            __syncthreads();
            const int nw = min(n, wl - b0 + 1);
            for (int s = ((kB - 1) >> 5) << 5; s >= 0; s -= 32) {
                unsigned chunk_mask = 0u;
                if (s < nw) {
                    bool hit = s + lane < nw;
                    if (kCull && hit)
                        hit = reaches_box(load_staged<float>(sh_xy, sh_q, sh_col, sh_cull, s + lane), t.wx0, t.wx1,
                                          t.wy0, t.wy1);
                    unsigned m = __ballot_sync(kFull, hit);
                    while (m) {
                        const int hb = 31 - __clz(m);
                        m ^= 1u << hb;
                        const int j = s + hb;  // back to front
                        const float4 xy = sh_xy[j];
                        const float4 qq = sh_q[j];
                        const float D = sh_col[j].w;
                        const float dx = xy.x - t.cx, dy = xy.y - t.cy;
                        float u;
                        const float p2 = neg_sigma_log2(qq, dx, dy, u);
                        const float ge = RT<float>::ex2(p2);
                        const float raw = mul_rn(xy.z, ge);
                        const float alpha = fminf(RT<float>::alpha_max(), raw);
                        const bool contrib = (b0 + j <= last) && (p2 <= 0.f) && (raw >= RT<float>::alpha_min());
                        const unsigned cm = __ballot_sync(kFull, contrib);
                        if (cm == 0u) continue;
                        const float inv1ma = RT<float>::rcp(1.f - alpha);
                        const float Tn = T * inv1ma;
                        const float wgt = contrib ? alpha * Tn : 0.f;
                        float cdot = 0.f;
#pragma unroll
                        for (int k = 0; k < NC; ++k) cdot = fmaf(sh_c[j][k], g[k], cdot);
                        const float dL_dalpha = fmaf(Tn, cdot, -SdL * inv1ma);
                        const float gd = (contrib && raw < RT<float>::alpha_max()) ? ge * dL_dalpha : 0.f;
                        SdL = fmaf(wgt, cdot, SdL);
                        T = contrib ? Tn : T;
                        const float ds = -xy.z * gd;
                        // sums the flush turns into dL/dmu' = (a S_u, b S_u + D S_dy) and the factored
                        // conic's dL/d(a, k, D) = (S_u2 / 2, a S_udy, S_dy2 / 2)
                        float r[kR];
                        r[0] = ds * u;
                        r[1] = ds * dy;
                        r[2] = r[0] * u;
                        r[3] = r[0] * dy;
                        r[4] = r[1] * dy;
                        r[5] = gd;
#pragma unroll
                        for (int k = 0; k < NC; ++k) r[6 + k] = wgt * g[k];
                        chunk_mask |= 1u << hb;
                        float* slot = s_grad[j];
                        if (__popc(cm) == 1) {
                            if (contrib) {
#pragma unroll
                                for (int q = 0; q < kR; ++q) atomicAdd(slot + q, r[q]);
                            }
                        } else {
                            warp_add_terms<kR>(r, s_red[w], slot, lane);
                        }
                    }
                }
                if (lane == 0 && chunk_mask) atomicOr(&s_mask[s >> 5], chunk_mask);
            }
            __syncthreads();
            if (threadIdx.x < n) {
                const int j = threadIdx.x;
                if (s_mask[j >> 5] & (1u << (j & 31))) {
                    const int p = RT<float>::unstash(sh_cull[j].w);
                    const int64_t gg = sh_g[j];
                    const float* a = s_grad[j];
                    const float ca = sh_xy[j].w, cb = sh_q[j].w, D = sh_col[j].w;
                    atomicAdd(dL_dmeans2d + p, make_float2(ca * a[0], fmaf(cb, a[0], D * a[1])));
                    atomicAdd(dL_dconics + 3 * p + 0, 0.5f * a[2]);
                    atomicAdd(dL_dconics + 3 * p + 1, ca * a[3]);
                    atomicAdd(dL_dconics + 3 * p + 2, 0.5f * a[4]);
                    atomicAdd(dL_dopacities + gg, a[5]);
                    float* dc = dL_dcolors + (int64_t)C * gg + c0;
                    for (int k = 0; k < nc; ++k) atomicAdd(dc + k, a[6 + k]);
                }
            }
            __syncthreads();
        }
        if (!kPersistent) break;
    }
}

// The kernel variant for a chunk of nc <= 32 channels.
template <int NC>
using FwdNc = decltype(&k_raster_fwd_nc<NC, true, true>);
template <int NC>
using BwdNc = decltype(&k_raster_bwd_nc<NC, true, true>);

template <int NC>
static FwdNc<NC> fwd_kernel(bool cull, bool pers)
{
    return cull ? (pers ? k_raster_fwd_nc<NC, true, true> : k_raster_fwd_nc<NC, true, false>)
                : (pers ? k_raster_fwd_nc<NC, false, true> : k_raster_fwd_nc<NC, false, false>);
}

template <int NC>
static BwdNc<NC> bwd_kernel(bool cull, bool pers)
{
    return cull ? (pers ? k_raster_bwd_nc<NC, true, true> : k_raster_bwd_nc<NC, true, false>)
                : (pers ? k_raster_bwd_nc<NC, false, true> : k_raster_bwd_nc<NC, false, false>);
}

struct ChunkArgs {
    const GsView* views;
    int V, T_total;
    const GsRasterConfig* cfg;
    cudaStream_t s;
};

template <int NC>
static int launch_fwd(const ChunkArgs& a, const float* means2d, const float* conics, const float* opacities,
                      const float* colors, int C, int c0, int nc, const int32_t* isect_ids, const int32_t* tile_ranges,
                      const float* background, float* out, float* T_final, int32_t* last_idx, int32_t* n_contrib)
{
    const bool pers = a.cfg && a.cfg->persistent;
    auto kern = fwd_kernel<NC>(cull_enabled(), pers);
    unsigned grid;
    if (int rc = raster_grid(kern, a.cfg, a.T_total, &grid)) return rc;
    int* queue = pers ? a.cfg->queue : nullptr;
    if (pers && cudaMemsetAsync(queue, 0, sizeof(int), a.s) != cudaSuccess) return launch_status("gs_rasterize_fwd_nc");
    launch_pdl(kern, grid, 256, a.s, a.views, a.V, a.T_total, a.cfg ? a.cfg->tile_order : nullptr, queue,
                                reinterpret_cast<const float2*>(means2d), conics, opacities, colors, C, c0, nc,
                                isect_ids, reinterpret_cast<const int2*>(tile_ranges), background, out, T_final,
                                last_idx, n_contrib);
    count_launches(1);
    return launch_status("gs_rasterize_fwd_nc");
}

template <int NC>
static int launch_bwd(const ChunkArgs& a, const float* means2d, const float* conics, const float* opacities,
                      const float* colors, int C, int c0, int nc, const int32_t* isect_ids, const int32_t* tile_ranges,
                      const float* background, const float* T_final, const int32_t* last_idx, const float* dL_dout,
                      float* dL_dmeans2d, float* dL_dconics, float* dL_dopacities, float* dL_dcolors)
{
    const bool pers = a.cfg && a.cfg->persistent;
    auto kern = bwd_kernel<NC>(cull_enabled(), pers);
    unsigned grid;
    if (int rc = raster_grid(kern, a.cfg, a.T_total, &grid)) return rc;
    int* queue = pers ? a.cfg->queue : nullptr;
    if (pers && cudaMemsetAsync(queue, 0, sizeof(int), a.s) != cudaSuccess) return launch_status("gs_rasterize_bwd_nc");
    launch_pdl(kern, grid, 256, a.s, a.views, a.V, a.T_total, a.cfg ? a.cfg->tile_order : nullptr, queue,
                                reinterpret_cast<const float2*>(means2d), conics, opacities, colors, C, c0, nc,
                                isect_ids, reinterpret_cast<const int2*>(tile_ranges), background, T_final, last_idx,
                                dL_dout, reinterpret_cast<float2*>(dL_dmeans2d), dL_dconics, dL_dopacities,
                                dL_dcolors);
    count_launches(1);
    return launch_status("gs_rasterize_bwd_nc");
}

// Chunk c0.. of nc channels goes to the smallest compiled width that holds it.
template <typename F>
static int for_each_chunk(int C, F&& f)
{
    for (int c0 = 0; c0 < C; c0 += 32) {
        const int nc = std::min(32, C - c0);
        int rc;
        if (nc <= 1) rc = f.template operator()<1>(c0, nc);
        else if (nc <= 2) rc = f.template operator()<2>(c0, nc);
        else if (nc <= 4) rc = f.template operator()<4>(c0, nc);
        else if (nc <= 8) rc = f.template operator()<8>(c0, nc);
        else if (nc <= 16) rc = f.template operator()<16>(c0, nc);
        else rc = f.template operator()<32>(c0, nc);
        if (rc) return rc;
    }
    return GS_OK;
}

static bool misaligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7) != 0; }

struct FwdChunks {
    const ChunkArgs& a;
    const float *means2d, *conics, *opacities, *colors;
    int C;
    const int32_t *isect_ids, *tile_ranges;
    const float* background;
    float *out, *T_final;
    int32_t *last_idx, *n_contrib;
    template <int NC>
    int operator()(int c0, int nc) const
    {
        return launch_fwd<NC>(a, means2d, conics, opacities, colors, C, c0, nc, isect_ids, tile_ranges, background,
                              out, T_final, last_idx, n_contrib);
    }
};

struct BwdChunks {
    const ChunkArgs& a;
    const float *means2d, *conics, *opacities, *colors;
    int C;
    const int32_t *isect_ids, *tile_ranges;
    const float *background, *T_final;
    const int32_t* last_idx;
    const float* dL_dout;
    float *dL_dmeans2d, *dL_dconics, *dL_dopacities, *dL_dcolors;
    template <int NC>
    int operator()(int c0, int nc) const
    {
        return launch_bwd<NC>(a, means2d, conics, opacities, colors, C, c0, nc, isect_ids, tile_ranges, background,
                              T_final, last_idx, dL_dout, dL_dmeans2d, dL_dconics, dL_dopacities, dL_dcolors);
    }
};

}  // namespace gs

using namespace gs;

// Up to this many channels the tuned 3-channel kernels run the image (one chunk).  Beyond, the kernels
// below are faster than the tuned ones run once per chunk of 3 (fwd+bwd at 1080p, 1M Gaussians:
// 4 channels 1.52 against 2.62 ms, 8 channels 1.83 against 4.08, 12 channels 2.88 against 5.51).
constexpr int kChunked3MaxC = 3;

extern "C" int gs_rasterize_fwd_nc(const GsView* views, int32_t V, int32_t T_total, int32_t C, const float* means2d,
                                   const float* conics, const float* opacities, const float* colors,
                                   const int32_t* isect_ids, const int32_t* tile_ranges, const float* background,
                                   float* out, float* T_final, int32_t* last_idx, int32_t* n_contrib,
                                   const GsRasterConfig* config, void* stream)
{
    gs::NvtxRange nvtx("gs_rasterize_fwd_nc");
    const char* who = "gs_rasterize_fwd_nc";
    if (V <= 0 || T_total < 0 || C <= 0) return fail(GS_ERR_INVALID_ARG, "%s: V=%d T_total=%d C=%d", who, V, T_total, C);
    if (C <= kChunked3MaxC)  // the tuned kernels, on chunks of up to 3 channels
        return rasterize_fwd_chunks3(who, C, views, V, T_total, means2d, conics, opacities, colors, isect_ids,
                                     tile_ranges, background, out, T_final, last_idx, n_contrib, config, stream);
    if (!views || !tile_ranges || !out || !T_final || !last_idx)
        return fail(GS_ERR_INVALID_ARG, "%s: null pointer argument", who);
    if (misaligned8(means2d) || misaligned8(tile_ranges))
        return fail(GS_ERR_INVALID_ARG, "%s: means2d and tile_ranges need 8-byte alignment", who);
    if (int rc = check_config(config, who)) return rc;
    if (T_total == 0) return GS_OK;
    const ChunkArgs a{views, V, T_total, config, as_stream(stream)};
    return for_each_chunk(C, FwdChunks{a, means2d, conics, opacities, colors, C, isect_ids, tile_ranges, background,
                                       out, T_final, last_idx, n_contrib});
}

extern "C" int gs_rasterize_bwd_nc(const GsView* views, int32_t V, int64_t P, int32_t T_total, int32_t C,
                                   const float* means2d, const float* conics, const float* opacities,
                                   const float* colors, const int32_t* isect_ids, const int32_t* tile_ranges,
                                   const float* background, const float* T_final, const int32_t* last_idx,
                                   const float* dL_dout, float* dL_dmeans2d, float* dL_dconics, float* dL_dopacities,
                                   float* dL_dcolors, const GsRasterConfig* config, void* stream)
{
    gs::NvtxRange nvtx("gs_rasterize_bwd_nc");
    const char* who = "gs_rasterize_bwd_nc";
    if (V <= 0 || P < 0 || T_total < 0 || C <= 0)
        return fail(GS_ERR_INVALID_ARG, "%s: V=%d P=%lld T_total=%d C=%d", who, V, (long long)P, T_total, C);
    if (C <= kChunked3MaxC)
        return rasterize_bwd_chunks3(who, C, views, V, P, T_total, means2d, conics, opacities, colors, isect_ids,
                                     tile_ranges, background, T_final, last_idx, dL_dout, dL_dmeans2d, dL_dconics,
                                     dL_dopacities, dL_dcolors, config, stream);
    if (!views || !tile_ranges || !T_final || !last_idx || !dL_dout ||
        (P > 0 && (!dL_dmeans2d || !dL_dconics || !dL_dopacities || !dL_dcolors)))
        return fail(GS_ERR_INVALID_ARG, "%s: null pointer argument", who);
    if (misaligned8(means2d) || misaligned8(dL_dmeans2d) || misaligned8(tile_ranges))
        return fail(GS_ERR_INVALID_ARG, "%s: 2-vector arrays need 8-byte alignment", who);
    if (int rc = check_config(config, who)) return rc;
    if (T_total == 0 || P == 0) return GS_OK;
    const ChunkArgs a{views, V, T_total, config, as_stream(stream)};
    return for_each_chunk(C, BwdChunks{a, means2d, conics, opacities, colors, C, isect_ids, tile_ranges, background,
                                       T_final, last_idx, dL_dout, dL_dmeans2d, dL_dconics, dL_dopacities,
                                       dL_dcolors});
}
