// Front-to-back compositing (Sec. 2.2, Eq. 7) and its backward (Sec. 3.1) over
// 16x16 tiles, written for sm_103a.
//
// One 256-thread CTA per tile, one pixel per thread; warp w covers the 8x4
// pixel block (w & 1, w >> 1) of the tile, so a warp's pixels form a compact
// box.  The tile's depth-sorted Gaussians are staged in shared memory in
// batches.  Before a warp walks 32 staged Gaussians, each lane tests one of
// them against the warp's box: the minimum of sigma over the box (exact for
// the quadratic form, evaluated edge by edge) against the alpha >= 1/255
// threshold sigma <= ln(255 o), widened by 5% + 1e-3 -- far beyond fp32
// rounding.  The warp then walks only the Gaussians that can reach one of its
// pixels.  Skipped pairs would fail the alpha test anyway, so results are
// identical to visiting every pair; the cull only removes work.  Warps whose
// pixels have all terminated stop early.  Inside the walk every lane
// evaluates and predicates decide, so the warp does not diverge.
//
// sigma is evaluated in the factored form sigma = (a u^2 + (det/a) dy^2) / 2
// with u = dx + (b/a) dy: both terms are non-negative, so elongated conics do
// not lose digits to cancellation (det is computed with a compensated
// product).
//
// The backward walks the same batches in reverse from each pixel's last
// composited Gaussian, rebuilding T_n from the saved T_final (Sec. 3.1).  When
// given a GsRasterConfig.warp_hits buffer, the forward stores each warp's
// 32-bit cull ballot of every chunk of 32 pairs it walks, and the backward
// walks those bits instead of repeating the test.  The
// nine per-pixel gradient terms of a Gaussian are summed over the warp
// through a shared-memory transpose into the warp's own slot for that
// Gaussian (plain stores), and the slots of the tile's warps are summed in a
// fixed order, giving one partial per (tile, Gaussian).  The fast mode adds
// the partials straight into the per-projection outputs with global atomics;
// the deterministic mode writes them as records that a second kernel sums per
// projection in emission order.
//
// Everything is templated on the scalar type: fp32 is the fast path, fp64
// (smaller batches, exp2 instead of the SFU) serves the gs_*_f64 entry points
// used to check the analytic backward against finite differences.  The
// colours have 3 channels (RGB), or 1 to 3 channels C apart in a separate
// instantiation that the multi-channel entry points use.
#include "gs_raster_bwd.cuh"

namespace gs {

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------

// kPersistent: a grid of a few CTAs per SM pops tiles from the global queue
// counter `queue` (zeroed before launch) until T_total tiles are taken;
// otherwise CTA i renders queue slot i.  Slot qi renders tile tile_order[qi]
// (identity when tile_order is NULL).  kCount: also count each pixel's
// composited Gaussians into n_contrib (a separate instantiation, so that the
// usual walk carries no counter).  kAnyC: W_arg channels of colours C_arg
// apart; otherwise 3 channels 3 apart (a separate instantiation: the runtime
// stride cost the 3-channel walk 2 %).  kLoss (3 channels): each pixel's L2
// loss against lo.target is taken as soon as its colour is known -- dL/dC =
// 2 inv_norm (C - target) into lo.dL and inv_norm (C - target)^2 summed into
// lo.loss -- so that no second kernel reads the image back.
template <typename S>
struct FwdLoss {
    const S* target;
    S* dL;    // nullable
    S* loss;  // nullable (accumulated: one atomic per CTA)
    S inv_norm;
};

template <typename S, bool kCull, bool kPersistent, bool kCount, bool kAnyC, bool kLoss = false>
__global__ void __launch_bounds__(256, 6)  // 6 CTAs per SM (40 registers) measured fastest
k_raster_fwd(const GsView* __restrict__ views, int V, int T_total, const int32_t* __restrict__ tile_order,
             int* __restrict__ queue, const V2<S>* __restrict__ means2d, const S* __restrict__ conics,
             const S* __restrict__ opacities, const S* __restrict__ colors, const int32_t* __restrict__ isect_ids,
             const int2* __restrict__ tile_ranges, const S* __restrict__ background, S* __restrict__ out_rgb,
             S* __restrict__ T_final, int32_t* __restrict__ last_idx, int32_t* __restrict__ n_contrib,
             uint32_t* __restrict__ warp_hits, int C_arg, int W_arg, FwdLoss<S> lo)
{
    static_assert(!kLoss || !kAnyC, "the folded loss takes 3 channels 3 apart");
    pdl_wait();
    pdl_trigger();
    const int C = kAnyC ? C_arg : 3, CW = kAnyC ? W_arg : 3;
    constexpr int kB = RT<S>::kFwdBatch;
    __shared__ V4<S> sh_xy[kB], sh_q[kB], sh_col[kB], sh_cull[kB];
    __shared__ int s_next;
    S lsum = 0;  // this thread's share of the loss (kLoss)
    for (int qi = blockIdx.x;;) {
        if (kPersistent) {
            __syncthreads();  // the previous tile is done with shared memory
            if (threadIdx.x == 0) s_next = atomicAdd(queue, 1);
            __syncthreads();
            qi = s_next;
            if (qi >= T_total) break;
        }
        const int tile = tile_order ? tile_order[qi] : qi;
        const TileCtx<S> t = tile_ctx<S>(views, V, tile);
        const int lane = threadIdx.x & 31;
        const int2 range = tile_ranges[tile];

        S T = 1, C0 = 0, C1 = 0, C2 = 0;
        int last = range.x - 1, count = 0;
        bool done = !t.inside;
        const int w = threadIdx.x >> 5;
        for (int b0 = range.x; b0 < range.y; b0 += kB) {
            if (__syncthreads_count(done) == (int)blockDim.x) break;  // also guards the stage below
            if (threadIdx.x < kB) {
                const int i = b0 + threadIdx.x;
                if (i < range.y) {
                    const int p = isect_ids[i];
                    const int64_t g = p + t.g_shift;
                    S c0, c1, c2;
                    load_c3(colors, g, C, CW, c0, c1, c2);
                    stage_gaussian<S>(sh_xy, sh_q, sh_col, sh_cull, threadIdx.x, means2d[p], conics[3 * p],
                                      conics[3 * p + 1], conics[3 * p + 2], opacities[g], c0, c1, c2);
                }
            }
            __syncthreads();
            const int n = min(kB, range.y - b0);
            int lastj = -1;  // this batch's last composited entry (the batch offset is added once, below)
            for (int s = 0; s < n; s += 32) {
                // a warp whose pixels are all finished walks no further chunk (nor culls it: the backward
                // reads no ballot past a warp's last composited entry)
                if (__all_sync(kFull, done)) break;
                bool hit = s + lane < n;
                if (kCull && hit)
                    hit = reaches_box(load_staged<S>(sh_xy, sh_q, sh_col, sh_cull, s + lane), t.wx0, t.wx1, t.wy0,
                                      t.wy1);
                unsigned m = __ballot_sync(kFull, hit);
                // the chunk's ballot of warp w goes to word w of the chunk (a chunk shorter than 8
                // entries has room for the first warps' words only)
                if (warp_hits && lane == 0 && w < n - s) warp_hits[b0 + s + w] = m;
                while (m) {
                    const int j = s + __ffs(m) - 1;
                    m &= m - 1;
                    // every lane evaluates; predicates decide (no divergent branches)
                    const V4<S> xy = sh_xy[j];
                    S u;
                    const S p2 = neg_sigma_log2(sh_q[j], xy.x - t.cx, xy.y - t.cy, u);
                    const S raw = mul_rn(xy.z, RT<S>::ex2(p2));
                    const S alpha = fmin(RT<S>::alpha_max(), raw);
                    const S Tn = fma(-T, alpha, T);  // T (1 - alpha) in one rounding
                    // p2 > 0 means sigma < 0 (not a positive-definite conic): skipped; the alpha test
                    // is on o e^-sigma before the clamp, so a NaN opacity is skipped too
                    const bool take = !done && p2 <= S(0) && raw >= RT<S>::alpha_min();
                    const bool stop = take && Tn < RT<S>::t_min();  // not composited; the pixel is finished
                    const bool comp = take && !stop;
                    done = done || stop;
                    const V4<S> c = sh_col[j];
                    const S wgt = comp ? alpha * T : S(0);
                    C0 = fma(wgt, c.x, C0);
                    C1 = fma(wgt, c.y, C1);
                    C2 = fma(wgt, c.z, C2);
                    T = comp ? Tn : T;
                    lastj = comp ? j : lastj;
                    if (kCount) count += comp;
                }
            }
            if (lastj >= 0) last = b0 + lastj;
        }
        if (t.inside) {
            S bg0 = 0, bg1 = 0, bg2 = 0;
            if (background) load_c3(background, 0, C, CW, bg0, bg1, bg2);
            S* o = out_rgb + (int64_t)C * t.pix;
            const S r0 = fma(T, bg0, C0), r1 = fma(T, bg1, C1), r2 = fma(T, bg2, C2);
            o[0] = r0;
            if (CW > 1) o[1] = r1;
            if (CW > 2) o[2] = r2;
            T_final[t.pix] = T;
            last_idx[t.pix] = last;
            if (kCount) n_contrib[t.pix] = count;
            if (kLoss) {  // as gs_l2_loss computes it from the stored image
                const S* tg = lo.target + 3 * t.pix;
                const S d0 = r0 - tg[0], d1 = r1 - tg[1], d2 = r2 - tg[2];
                if (lo.dL) {
                    const S two = S(2) * lo.inv_norm;
                    S* g = lo.dL + 3 * t.pix;
                    g[0] = two * d0;
                    g[1] = two * d1;
                    g[2] = two * d2;
                }
                lsum += (d0 * d0 + d1 * d1) + d2 * d2;
            }
        }
        if (!kPersistent) break;
    }
    if (kLoss && lo.loss) {  // one atomic per CTA
        __shared__ S s_loss[kWarps];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) lsum += __shfl_xor_sync(kFull, lsum, d);
        if ((threadIdx.x & 31) == 0) s_loss[threadIdx.x >> 5] = lsum;
        __syncthreads();
        if (threadIdx.x == 0) {
            S tot = 0;
#pragma unroll
            for (int i = 0; i < kWarps; ++i) tot += s_loss[i];
            atomicAdd(lo.loss, tot * lo.inv_norm);
        }
    }
}

// Per projection: sum of its (tile, Gaussian) records in emission order.
template <typename S>
__global__ void __launch_bounds__(256)
k_reduce_records(const GsView* __restrict__ views, int V, int64_t P, const int32_t* __restrict__ touched,
                 const int32_t* __restrict__ emit_start, const int32_t* __restrict__ isect_pos,
                 const int32_t* __restrict__ K_dev, int64_t cap, const S* __restrict__ records,
                 V2<S>* __restrict__ dL_dmeans2d, S* __restrict__ dL_dconics, S* __restrict__ dL_dopacities,
                 S* __restrict__ dL_dcolors, int C, int CW)
{
    pdl_wait();
    pdl_trigger();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int n = touched[p];
    if (n <= 0) return;
    const int64_t K = min((int64_t)*K_dev, cap);
    const int64_t e0 = emit_start[p];
    if (e0 < 0 || e0 + n > K) return;  // capacity overflow: outputs are flagged invalid
    S acc[kRec];
#pragma unroll
    for (int q = 0; q < kRec; ++q) acc[q] = S(0);
    for (int j = 0; j < n; ++j) {
        const S* rec = records + (size_t)isect_pos[e0 + j] * kRec;
#pragma unroll
        for (int q = 0; q < kRec; ++q) acc[q] += rec[q];
    }
    V2<S> m = dL_dmeans2d[p];
    m.x += acc[0];
    m.y += acc[1];
    dL_dmeans2d[p] = m;
    dL_dconics[3 * p + 0] += acc[2];
    dL_dconics[3 * p + 1] += acc[3];
    dL_dconics[3 * p + 2] += acc[4];
    const GsView& view = views[view_of_projection(views, V, p)];
    const int64_t g = view.g_begin + (p - view.proj_offset);
    atomicAdd(dL_dopacities + g, acc[5]);
    S* dc = dL_dcolors + (int64_t)C * g;
    if (CW == 3) {
        atomic_add3(dc, acc[6], acc[7], acc[8]);
    } else {
        atomicAdd(dc, acc[6]);
        if (CW > 1) atomicAdd(dc + 1, acc[7]);
    }
}

template <typename S>
static int rasterize_fwd_impl(const char* who, int C, int CW, const GsView* views, int32_t V, int32_t T_total, const S* means2d,
                              const S* conics, const S* opacities, const S* colors, const int32_t* isect_ids,
                              const int32_t* tile_ranges, const S* background, S* out_rgb, S* T_final,
                              int32_t* last_idx, int32_t* n_contrib, uint32_t* warp_hits,
                              const GsRasterConfig* config, void* stream, const FwdLoss<S>* loss = nullptr)
{
    if (V <= 0 || T_total < 0 || CW < 1 || CW > 3 || C < CW)
        return fail(GS_ERR_INVALID_ARG, "%s: V=%d T_total=%d C=%d", who, V, T_total, C);
    if (!views || !tile_ranges || !out_rgb || !T_final || !last_idx)
        return fail(GS_ERR_INVALID_ARG, "%s: null pointer argument", who);
    if ((reinterpret_cast<uintptr_t>(means2d) & (2 * sizeof(S) - 1)) || (reinterpret_cast<uintptr_t>(tile_ranges) & 7))
        return fail(GS_ERR_INVALID_ARG, "%s: means2d needs %zu-byte, tile_ranges 8-byte alignment", who,
                    2 * sizeof(S));
    if (int rc = check_config(config, who)) return rc;
    if (T_total == 0) return GS_OK;
    cudaStream_t s = as_stream(stream);
    const bool cull = cull_enabled(), pers = config && config->persistent;
    // the any-channel instantiations exist for fp32 only (the fp64 entry points composite 3 channels)
    constexpr bool kA = std::is_same<S, float>::value;
    using KF = decltype(&k_raster_fwd<S, true, true, true, false>);
    static const KF table[2][2][2][2] = {
        {{{k_raster_fwd<S, false, false, false, false>, k_raster_fwd<S, false, false, false, kA>},
          {k_raster_fwd<S, false, false, true, false>, k_raster_fwd<S, false, false, true, kA>}},
         {{k_raster_fwd<S, false, true, false, false>, k_raster_fwd<S, false, true, false, kA>},
          {k_raster_fwd<S, false, true, true, false>, k_raster_fwd<S, false, true, true, kA>}}},
        {{{k_raster_fwd<S, true, false, false, false>, k_raster_fwd<S, true, false, false, kA>},
          {k_raster_fwd<S, true, false, true, false>, k_raster_fwd<S, true, false, true, kA>}},
         {{k_raster_fwd<S, true, true, false, false>, k_raster_fwd<S, true, true, false, kA>},
          {k_raster_fwd<S, true, true, true, false>, k_raster_fwd<S, true, true, true, kA>}}}};
    KF kern = table[cull][pers][n_contrib != nullptr][C != 3 || CW != 3];
    if (loss) {
        if constexpr (kA) {
            static const KF with_loss[2][2] = {
                {k_raster_fwd<S, false, false, false, false, true>, k_raster_fwd<S, false, true, false, false, true>},
                {k_raster_fwd<S, true, false, false, false, true>, k_raster_fwd<S, true, true, false, false, true>}};
            if (n_contrib || C != 3 || CW != 3) return fail(GS_ERR_INVALID_ARG, "%s: the folded loss takes 3 channels "
                                                            "and no contributor count", who);
            kern = with_loss[cull][pers];
        } else {
            return fail(GS_ERR_INVALID_ARG, "%s: no folded loss in this precision", who);
        }
    }
    unsigned grid;
    if (int rc = raster_grid(kern, config, T_total, &grid)) return rc;
    int* queue = pers ? config->queue : nullptr;
    if (pers && cudaMemsetAsync(queue, 0, sizeof(int), s) != cudaSuccess) return launch_status(who);
    launch_pdl(kern, grid, 256, s, views, V, T_total, config ? config->tile_order : nullptr, queue,
                              reinterpret_cast<const V2<S>*>(means2d), conics, opacities, colors, isect_ids,
                              reinterpret_cast<const int2*>(tile_ranges), background, out_rgb, T_final, last_idx,
                              n_contrib, warp_hits, C, CW, loss ? *loss : FwdLoss<S>{nullptr, nullptr, nullptr, S(0)});
    count_launches(1);
    return launch_status(who);
}

// The backward's batch shape from the config: pixels per thread and staged batch.  fp32 takes the
// config's fields (0 = defaults); fp64 has one shape.
template <typename S>
static int bwd_shape(const GsRasterConfig* cfg, const char* who, int* px, int* batch)
{
    if (!std::is_same<S, float>::value) {
        *px = 1;
        *batch = RT<S>::kBwdBatch;
        return GS_OK;
    }
    const int p = cfg && cfg->bwd_pixels ? cfg->bwd_pixels : GS_BWD_PIXELS_DEFAULT;
    const int b = cfg && cfg->bwd_batch ? cfg->bwd_batch : (p == 1 ? RT<float>::kBwdBatch : 64);
    const bool ok = (p == 1 && (b == 64 || b == 96)) || (p == 2 && (b == 64 || b == 128));
    if (!ok)
        return fail(GS_ERR_INVALID_ARG, "%s: backward batch shape %d pixels per thread, batch %d is not compiled "
                    "(one pixel: 64 or 96; two: 64 or 128)", who, p, b);
    *px = p;
    *batch = b;
    return GS_OK;
}

// The backward kernel for a shape and its variant flags.  The default batch of each pixel count has
// every variant; the other batches only the culling ones, and a non-culling request (GS_NO_CULL)
// falls back to the default batch of that pixel count.
template <typename S>
static RasterBwdKernel<S> pick_bwd(bool cull, bool atomic, bool pers, bool any_c, int px, int batch)
{
    constexpr bool kA = std::is_same<S, float>::value;  // the any-channel variants exist for fp32 only
    constexpr int kB0 = RT<S>::kBwdBatch;
#define GS_BWD1(CULL, AT, PE, AC, B) k_raster_bwd<S, CULL, AT, PE, (AC) && kA, 1, B>
    static const RasterBwdKernel<S> full[2][2][2][2] = {
        {{{GS_BWD1(false, false, false, false, kB0), GS_BWD1(false, false, false, true, kB0)},
          {GS_BWD1(false, false, true, false, kB0), GS_BWD1(false, false, true, true, kB0)}},
         {{GS_BWD1(false, true, false, false, kB0), GS_BWD1(false, true, false, true, kB0)},
          {GS_BWD1(false, true, true, false, kB0), GS_BWD1(false, true, true, true, kB0)}}},
        {{{GS_BWD1(true, false, false, false, kB0), GS_BWD1(true, false, false, true, kB0)},
          {GS_BWD1(true, false, true, false, kB0), GS_BWD1(true, false, true, true, kB0)}},
         {{GS_BWD1(true, true, false, false, kB0), GS_BWD1(true, true, false, true, kB0)},
          {GS_BWD1(true, true, true, false, kB0), GS_BWD1(true, true, true, true, kB0)}}}};
    if (px == 1 && batch == kB0) return full[cull][atomic][pers][any_c];
    if constexpr (kA) {
    if (px == 1 && batch == 64) {
        static const RasterBwdKernel<S> b64[2][2][2] = {
            {{GS_BWD1(true, false, false, false, 64), GS_BWD1(true, false, false, true, 64)},
             {GS_BWD1(true, false, true, false, 64), GS_BWD1(true, false, true, true, 64)}},
            {{GS_BWD1(true, true, false, false, 64), GS_BWD1(true, true, false, true, 64)},
             {GS_BWD1(true, true, true, false, 64), GS_BWD1(true, true, true, true, 64)}}};
        return cull ? b64[atomic][pers][any_c] : full[cull][atomic][pers][any_c];
    }
    if (px == 2) {
        RasterBwdKernel<float> k = raster_bwd_px2_kernel(cull, atomic, pers, any_c, batch);
        return k ? k : raster_bwd_px2_kernel(cull, atomic, pers, any_c, 64);
    }
    }
#undef GS_BWD1
    return nullptr;
}

template <typename S>
static size_t bwd_workspace(int64_t K_capacity, int32_t deterministic)
{
    if (K_capacity < 0) return 0;
    return deterministic ? align256((size_t)K_capacity * kRec * sizeof(S)) : 0;
}

template <typename S>
static int rasterize_bwd_impl(const char* who, int C, int CW, const GsView* views, int32_t V, int64_t P, int32_t T_total,
                              const S* means2d, const S* conics, const S* opacities, const S* colors,
                              const int32_t* isect_ids, const int32_t* isect_pos, const int32_t* emit_start,
                              const int32_t* touched, const int32_t* tile_ranges, const int32_t* K, int64_t K_capacity,
                              const S* background, const S* T_final, const int32_t* last_idx,
                              const uint32_t* warp_hits, const S* dL_drgb,
                              int32_t deterministic, void* workspace, size_t workspace_bytes, S* dL_dmeans2d,
                              S* dL_dconics, S* dL_dopacities, S* dL_dcolors, const GsRasterConfig* config,
                              void* stream)
{
    if (V <= 0 || P < 0 || T_total < 0 || K_capacity < 0 || K_capacity >= (int64_t(1) << 31) || CW < 1 || CW > 3 ||
        C < CW)
        return fail(GS_ERR_INVALID_ARG, "%s: V=%d P=%lld T_total=%d K_capacity=%lld C=%d", who, V, (long long)P,
                    T_total, (long long)K_capacity, C);
    if (!views || !tile_ranges || !T_final || !last_idx || !dL_drgb ||
        (P > 0 && (!dL_dmeans2d || !dL_dconics || !dL_dopacities || !dL_dcolors)) ||
        (deterministic && P > 0 && (!K || !touched || !emit_start || !isect_pos)))
        return fail(GS_ERR_INVALID_ARG, "%s: null pointer argument", who);
    if ((reinterpret_cast<uintptr_t>(means2d) & (2 * sizeof(S) - 1)) ||
        (reinterpret_cast<uintptr_t>(dL_dmeans2d) & (2 * sizeof(S) - 1)) || (reinterpret_cast<uintptr_t>(tile_ranges) & 7))
        return fail(GS_ERR_INVALID_ARG, "%s: 2-vector arrays need %zu-byte alignment", who, 2 * sizeof(S));
    const size_t need = bwd_workspace<S>(K_capacity, deterministic);
    if (workspace_bytes < need || (need > 0 && !workspace))
        return fail(GS_ERR_INVALID_ARG, "%s: workspace of %zu bytes, need %zu", who, workspace_bytes, need);
    if (int rc = check_config(config, who)) return rc;
    if (T_total == 0 || P == 0) return GS_OK;
    cudaStream_t s = as_stream(stream);
    S* records = static_cast<S*>(workspace);
    const bool cull = cull_enabled(), pers = config && config->persistent;
    int px = 1, batch = RT<S>::kBwdBatch;
    if (int rc = bwd_shape<S>(config, who, &px, &batch)) return rc;
    const RasterBwdKernel<S> kern = pick_bwd<S>(cull, !deterministic, pers, C != 3 || CW != 3, px, batch);
    if (!kern) return fail(GS_ERR_INVALID_ARG, "%s: no backward compiled for %d pixels per thread, batch %d", who, px,
                           batch);
    const int threads = px == 1 ? bwd_threads<1>() : bwd_threads<2>();
    unsigned grid;
    if (int rc = raster_grid(kern, config, T_total, &grid, threads)) return rc;
    int* queue = pers ? config->queue : nullptr;
    if (pers && cudaMemsetAsync(queue, 0, sizeof(int), s) != cudaSuccess) return launch_status(who);
    launch_pdl(kern, grid, threads, s, views, V, T_total, config ? config->tile_order : nullptr, queue,
                              reinterpret_cast<const V2<S>*>(means2d), conics, opacities, colors, isect_ids,
                              reinterpret_cast<const int2*>(tile_ranges), background, T_final, last_idx, warp_hits,
                              dL_drgb,
                              records, reinterpret_cast<V2<S>*>(dL_dmeans2d), dL_dconics, dL_dopacities, dL_dcolors, C,
                              CW);
    count_launches(1);
    if (deterministic) {
        launch_pdl(k_reduce_records<S>, (unsigned)((P + 255) / 256), 256, s,
            views, V, P, touched, emit_start, isect_pos, K, K_capacity, records,
            reinterpret_cast<V2<S>*>(dL_dmeans2d), dL_dconics, dL_dopacities, dL_dcolors, C, CW);
        count_launches(1);
    }
    return launch_status(who);
}

int rasterize_fwd_chunks3(const char* who, int C, const GsView* views, int32_t V, int32_t T_total,
                          const float* means2d, const float* conics, const float* opacities, const float* colors,
                          const int32_t* isect_ids, const int32_t* tile_ranges, const float* background, float* out,
                          float* T_final, int32_t* last_idx, int32_t* n_contrib, const GsRasterConfig* config,
                          void* stream)
{
    if (C < 1) return fail(GS_ERR_INVALID_ARG, "%s: C=%d", who, C);
    // every chunk rebuilds the same alpha, T, last index and warp-box ballots
    for (int c0 = 0; c0 < C; c0 += 3) {
        const int cw = std::min(3, C - c0);
        if (int rc = rasterize_fwd_impl<float>(who, C, cw, views, V, T_total, means2d, conics, opacities,
                                               colors ? colors + c0 : nullptr, isect_ids, tile_ranges,
                                               background ? background + c0 : nullptr, out ? out + c0 : nullptr,
                                               T_final, last_idx, n_contrib, config ? config->warp_hits : nullptr,
                                               config, stream))
            return rc;
    }
    return GS_OK;
}

int rasterize_bwd_chunks3(const char* who, int C, const GsView* views, int32_t V, int64_t P, int32_t T_total,
                          const float* means2d, const float* conics, const float* opacities, const float* colors,
                          const int32_t* isect_ids, const int32_t* tile_ranges, const float* background,
                          const float* T_final, const int32_t* last_idx, const float* dL_dout, float* dL_dmeans2d,
                          float* dL_dconics, float* dL_dopacities, float* dL_dcolors, const GsRasterConfig* config,
                          void* stream)
{
    if (C < 1) return fail(GS_ERR_INVALID_ARG, "%s: C=%d", who, C);
    // each chunk adds its channels' share of every gradient (dL/dalpha is a sum over the channels)
    for (int c0 = 0; c0 < C; c0 += 3) {
        const int cw = std::min(3, C - c0);
        if (int rc = rasterize_bwd_impl<float>(
                who, C, cw, views, V, P, T_total, means2d, conics, opacities, colors ? colors + c0 : nullptr,
                isect_ids, nullptr, nullptr, nullptr, tile_ranges, nullptr, 0, background ? background + c0 : nullptr,
                T_final, last_idx, config ? config->warp_hits : nullptr, dL_dout ? dL_dout + c0 : nullptr, 0,
                nullptr, 0, dL_dmeans2d, dL_dconics, dL_dopacities, dL_dcolors ? dL_dcolors + c0 : nullptr, config,
                stream))
            return rc;
    }
    return GS_OK;
}

}  // namespace gs

using namespace gs;

extern "C" int gs_rasterize_fwd(const GsView* views, int32_t V, int32_t T_total, const float* means2d,
                                const float* conics, const float* opacities, const float* colors,
                                const int32_t* isect_ids, const int32_t* tile_ranges, const float* background,
                                float* out_rgb, float* T_final, int32_t* last_idx, int32_t* n_contrib,
                                const GsRasterConfig* config, void* stream)
{
    gs::NvtxRange nvtx("gs_rasterize_fwd");
    return rasterize_fwd_impl<float>("gs_rasterize_fwd", 3, 3, views, V, T_total, means2d, conics, opacities, colors,
                                     isect_ids, tile_ranges, background, out_rgb, T_final, last_idx, n_contrib,
                                     config ? config->warp_hits : nullptr, config, stream);
}

extern "C" int gs_rasterize_fwd_l2(const GsView* views, int32_t V, int32_t T_total, const float* means2d,
                                   const float* conics, const float* opacities, const float* colors,
                                   const int32_t* isect_ids, const int32_t* tile_ranges, const float* background,
                                   float* out_rgb, float* T_final, int32_t* last_idx, const float* target,
                                   float inv_norm, float* dL_drgb, float* loss, const GsRasterConfig* config,
                                   void* stream)
{
    gs::NvtxRange nvtx("gs_rasterize_fwd_l2");
    if (!target || (!dL_drgb && !loss))
        return fail(GS_ERR_INVALID_ARG, "gs_rasterize_fwd_l2: null target, or neither dL_drgb nor loss");
    const FwdLoss<float> lo{target, dL_drgb, loss, inv_norm};
    return rasterize_fwd_impl<float>("gs_rasterize_fwd_l2", 3, 3, views, V, T_total, means2d, conics, opacities,
                                     colors, isect_ids, tile_ranges, background, out_rgb, T_final, last_idx, nullptr,
                                     config ? config->warp_hits : nullptr, config, stream, &lo);
}

extern "C" int gs_rasterize_fwd_f64(const GsView* views, int32_t V, int32_t T_total, const double* means2d,
                                    const double* conics, const double* opacities, const double* colors,
                                    const int32_t* isect_ids, const int32_t* tile_ranges, const double* background,
                                    double* out_rgb, double* T_final, int32_t* last_idx, int32_t* n_contrib,
                                    const GsRasterConfig* config, void* stream)
{
    gs::NvtxRange nvtx("gs_rasterize_fwd_f64");
    return rasterize_fwd_impl<double>("gs_rasterize_fwd_f64", 3, 3, views, V, T_total, means2d, conics, opacities, colors,
                                      isect_ids, tile_ranges, background, out_rgb, T_final, last_idx, n_contrib,
                                      config ? config->warp_hits : nullptr, config, stream);
}

extern "C" size_t gs_rasterize_bwd_workspace_size(int64_t K_capacity, int32_t deterministic)
{
    return bwd_workspace<float>(K_capacity, deterministic);
}

extern "C" size_t gs_rasterize_bwd_f64_workspace_size(int64_t K_capacity, int32_t deterministic)
{
    return bwd_workspace<double>(K_capacity, deterministic);
}

extern "C" int gs_rasterize_bwd(const GsView* views, int32_t V, int64_t P, int32_t T_total, const float* means2d,
                                const float* conics, const float* opacities, const float* colors,
                                const int32_t* isect_ids, const int32_t* isect_pos, const int32_t* emit_start,
                                const int32_t* touched, const int32_t* tile_ranges, const int32_t* K,
                                int64_t K_capacity, const float* background, const float* T_final,
                                const int32_t* last_idx, const float* dL_drgb, int32_t deterministic,
                                void* workspace, size_t workspace_bytes, float* dL_dmeans2d, float* dL_dconics,
                                float* dL_dopacities, float* dL_dcolors, const GsRasterConfig* config, void* stream)
{
    gs::NvtxRange nvtx("gs_rasterize_bwd");
    return rasterize_bwd_impl<float>("gs_rasterize_bwd", 3, 3, views, V, P, T_total, means2d, conics, opacities, colors,
                                     isect_ids, isect_pos, emit_start, touched, tile_ranges, K, K_capacity,
                                     background, T_final, last_idx, config ? config->warp_hits : nullptr, dL_drgb,
                                     deterministic, workspace,
                                     workspace_bytes, dL_dmeans2d, dL_dconics, dL_dopacities, dL_dcolors, config,
                                     stream);
}

extern "C" int gs_rasterize_bwd_f64(const GsView* views, int32_t V, int64_t P, int32_t T_total,
                                    const double* means2d, const double* conics, const double* opacities,
                                    const double* colors, const int32_t* isect_ids, const int32_t* isect_pos,
                                    const int32_t* emit_start, const int32_t* touched, const int32_t* tile_ranges,
                                    const int32_t* K, int64_t K_capacity, const double* background,
                                    const double* T_final, const int32_t* last_idx, const double* dL_drgb,
                                    int32_t deterministic, void* workspace, size_t workspace_bytes,
                                    double* dL_dmeans2d, double* dL_dconics, double* dL_dopacities,
                                    double* dL_dcolors, const GsRasterConfig* config, void* stream)
{
    gs::NvtxRange nvtx("gs_rasterize_bwd_f64");
    return rasterize_bwd_impl<double>("gs_rasterize_bwd_f64", 3, 3, views, V, P, T_total, means2d, conics, opacities,
                                      colors, isect_ids, isect_pos, emit_start, touched, tile_ranges, K, K_capacity,
                                      background, T_final, last_idx, config ? config->warp_hits : nullptr, dL_drgb,
                                      deterministic, workspace,
                                      workspace_bytes, dL_dmeans2d, dL_dconics, dL_dopacities, dL_dcolors, config,
                                      stream);
}
