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
// pixels have all terminated stop early.
//
// sigma is evaluated in the factored form sigma = (a u^2 + (det/a) dy^2) / 2
// with u = dx + (b/a) dy: both terms are non-negative, so elongated conics do
// not lose digits to cancellation (det is computed with a compensated
// product).
//
// The backward walks the same batches in reverse from each pixel's last
// composited Gaussian, rebuilding T_n from the saved T_final (Sec. 3.1).  The
// nine per-pixel gradient terms of a Gaussian are summed over the warp with a
// reduce-scatter (each shuffle level halves the vector a lane carries), then
// over the eight warps in a fixed order, giving one record per (tile,
// Gaussian) pair.  A second kernel sums each projection's records over its
// tiles in emission order.  No floating-point atomics touch per-projection
// outputs, so gradients are run-to-run identical.
#include <algorithm>

#include "gs_common.cuh"

namespace gs {

constexpr int kFwdBatch = 256;
constexpr int kBwdBatch = 64;  // deterministic mode (per-warp partial slots)
constexpr int kWarps = 8;
constexpr int kRec = 9;  // dmu'(2) dconic(3) dopacity(1) dcolor(3)
constexpr float kLog2e = 1.4426950408889634f;

// 2^x on the SFU (PTX ex2.approx.ftz.f32).
__device__ __forceinline__ float ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// One staged Gaussian (4 x float4 = 64 bytes):
//   g.xy  : mu'.x, mu'.y, opacity, a
//   g.q   : -log2e/2 * a, k = b/a, -log2e/2 * D, b     (D = det/a = c - b^2/a)
//   g.col : r, g, b, D
//   g.cull: sigma threshold (<0: never reaches 1/255; +inf: never culled),
//           -b/c, c, (backward: the projection index, as int bits)
struct Staged {
    float4 xy, q, col, cull;
};

// log2(e) * (-sigma) at Delta = (dx, dy); u = dx + k dy is returned too.
// Explicit roundings keep forward and backward bit-identical.
__device__ __forceinline__ float neg_sigma_log2(const float4& q, float dx, float dy, float& u)
{
    u = fmaf(q.y, dy, dx);
    return fmaf(__fmul_rn(q.x, u), u, __fmul_rn(__fmul_rn(q.z, dy), dy));
}

__device__ __forceinline__ void stage_gaussian(float4* sh_xy, float4* sh_q, float4* sh_col, float4* sh_cull, int j,
                                               float2 m, float a, float b, float c, float o, float r, float g,
                                               float bl)
{
    // det with the rounding error of b^2 compensated (Kahan's 2x2 determinant)
    const float bb = b * b;
    const float det = fmaf(a, c, -bb) - fmaf(b, b, -bb);
    const float k = b / a;
    const float D = det / a;
    sh_xy[j] = make_float4(m.x, m.y, o, a);
    sh_q[j] = make_float4(-0.5f * kLog2e * a, k, -0.5f * kLog2e * D, b);
    sh_col[j] = make_float4(r, g, bl, D);
    float thr;
    if (!(o >= GS_ALPHA_MIN)) {
        thr = -1.f;  // o e^-sigma < 1/255 everywhere
    } else if (!(a > 0.f && det > 0.f) || 4.f * a * c > 1e7f * det) {
        thr = INFINITY;  // degenerate or extremely elongated conic: never culled
    } else {
        thr = 1.05f * logf(255.f * o) + 1e-3f;
    }
    sh_cull[j] = make_float4(thr, -b / c, c, 0.f);
}

// Can the Gaussian reach alpha >= 1/255 at a pixel centre of the box
// [X0, X1] x [Y0, Y1]?  Minimum of sigma over the box: zero when mu' is
// inside, otherwise the least of the four edge minima (on an edge sigma is a
// parabola; its vertex is clamped to the edge).
__device__ __forceinline__ bool reaches_box(const Staged& g, float X0, float X1, float Y0, float Y1)
{
    const float thr = g.cull.x;
    if (thr < 0.f) return false;
    if (!(thr < INFINITY)) return true;
    const float mx = g.xy.x, my = g.xy.y;
    if (mx >= X0 && mx <= X1 && my >= Y0 && my <= Y1) return true;
    const float a = g.xy.w, k = g.q.y, D = g.col.w, kv = g.cull.y;
    auto sig = [&](float dx, float dy) {
        const float u = fmaf(k, dy, dx);
        return 0.5f * fmaf(a * u, u, D * dy * dy);
    };
    const float dxl = mx - X0, dxr = mx - X1, dyt = my - Y0, dyb = my - Y1;
    float smin = sig(dxl, fminf(fmaxf(kv * dxl, dyb), dyt));
    smin = fminf(smin, sig(dxr, fminf(fmaxf(kv * dxr, dyb), dyt)));
    smin = fminf(smin, sig(fminf(fmaxf(-k * dyt, dxr), dxl), dyt));
    smin = fminf(smin, sig(fminf(fmaxf(-k * dyb, dxr), dxl), dyb));
    return smin <= thr;
}

struct TileCtx {
    const GsView* view;
    int tx, ty, px, py;
    bool inside;
    int64_t pix;       // packed pixel index
    float cx, cy;      // pixel centre
    float wx0, wx1, wy0, wy1;  // warp's pixel-centre box
    int64_t g_shift;   // g = p + g_shift
};

__device__ __forceinline__ TileCtx tile_ctx(const GsView* __restrict__ views, int V, int tile)
{
    TileCtx t;
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
    t.cx = t.px + 0.5f;
    t.cy = t.py + 0.5f;
    t.wx0 = bx + 0.5f;
    t.wx1 = bx + 7.5f;
    t.wy0 = by + 0.5f;
    t.wy1 = by + 3.5f;
    t.g_shift = (int64_t)t.view->g_begin - t.view->proj_offset;
    return t;
}

__device__ __forceinline__ Staged load_staged(const float4* sh_xy, const float4* sh_q, const float4* sh_col,
                                              const float4* sh_cull, int j)
{
    return Staged{sh_xy[j], sh_q[j], sh_col[j], sh_cull[j]};
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------

// kPersistent: a grid of a few CTAs per SM pops tiles from the global queue
// counter `queue` (zeroed before launch) until T_total tiles are taken;
// otherwise CTA i renders queue slot i.  Slot qi renders tile tile_order[qi]
// (identity when tile_order is NULL).
template <bool kCull, bool kPersistent>
__global__ void __launch_bounds__(256)
k_raster_fwd(const GsView* __restrict__ views, int V, int T_total, const int32_t* __restrict__ tile_order,
             int* __restrict__ queue, const float2* __restrict__ means2d,
             const float* __restrict__ conics, const float* __restrict__ opacities, const float* __restrict__ colors,
             const int32_t* __restrict__ isect_ids, const int2* __restrict__ tile_ranges,
             const float* __restrict__ background, float* __restrict__ out_rgb, float* __restrict__ T_final,
             int32_t* __restrict__ last_idx, int32_t* __restrict__ n_contrib)
{
    __shared__ float4 sh_xy[kFwdBatch], sh_q[kFwdBatch], sh_col[kFwdBatch], sh_cull[kFwdBatch];
    __shared__ int s_next;
    for (int qi = blockIdx.x;;) {
        if (kPersistent) {
            __syncthreads();  // the previous tile is done with shared memory
            if (threadIdx.x == 0) s_next = atomicAdd(queue, 1);
            __syncthreads();
            qi = s_next;
            if (qi >= T_total) break;
        }
        const int tile = tile_order ? tile_order[qi] : qi;
        const TileCtx t = tile_ctx(views, V, tile);
        const int lane = threadIdx.x & 31;
        const int2 range = tile_ranges[tile];

        float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
        int last = range.x - 1, count = 0;
        bool done = !t.inside;

        for (int b0 = range.x; b0 < range.y; b0 += kFwdBatch) {
            if (__syncthreads_count(done) == (int)blockDim.x) break;  // also guards the stage below
            {
                const int i = b0 + threadIdx.x;
                if (i < range.y) {
                    const int p = isect_ids[i];
                    const int64_t g = p + t.g_shift;
                    stage_gaussian(sh_xy, sh_q, sh_col, sh_cull, threadIdx.x, means2d[p], conics[3 * p],
                                   conics[3 * p + 1], conics[3 * p + 2], opacities[g], colors[3 * g], colors[3 * g + 1],
                                   colors[3 * g + 2]);
                }
            }
            __syncthreads();
            const int n = min(kFwdBatch, range.y - b0);
            for (int s = 0; s < n; s += 32) {
                bool hit = s + lane < n;
                if (kCull && hit)
                    hit = reaches_box(load_staged(sh_xy, sh_q, sh_col, sh_cull, s + lane), t.wx0, t.wx1, t.wy0, t.wy1);
                unsigned m = __ballot_sync(kFull, hit);
                while (m) {
                    const int j = s + __ffs(m) - 1;
                    m &= m - 1;
                    // every lane evaluates; predicates decide (no divergent branches)
                    const float4 xy = sh_xy[j];
                    float u;
                    const float p2 = neg_sigma_log2(sh_q[j], xy.x - t.cx, xy.y - t.cy, u);
                    const float alpha = fminf(GS_ALPHA_MAX, __fmul_rn(xy.z, ex2(p2)));
                    const float Tn = T * (1.f - alpha);
                    // p2 > 0 means sigma < 0 (not a positive-definite conic): skipped
                    const bool take = !done && p2 <= 0.f && alpha >= GS_ALPHA_MIN;
                    const bool stop = take && Tn < GS_T_MIN;  // not composited; the pixel is finished
                    const bool comp = take && !stop;
                    done = done || stop;
                    const float4 c = sh_col[j];
                    const float wgt = comp ? alpha * T : 0.f;
                    C0 = fmaf(wgt, c.x, C0);
                    C1 = fmaf(wgt, c.y, C1);
                    C2 = fmaf(wgt, c.z, C2);
                    T = comp ? Tn : T;
                    last = comp ? b0 + j : last;
                    count += comp;
                }
                if (__all_sync(kFull, done)) break;
            }
        }
        if (t.inside) {
            float bg0 = 0.f, bg1 = 0.f, bg2 = 0.f;
            if (background) { bg0 = background[0]; bg1 = background[1]; bg2 = background[2]; }
            out_rgb[3 * t.pix + 0] = fmaf(T, bg0, C0);
            out_rgb[3 * t.pix + 1] = fmaf(T, bg1, C1);
            out_rgb[3 * t.pix + 2] = fmaf(T, bg2, C2);
            T_final[t.pix] = T;
            last_idx[t.pix] = last;
            if (n_contrib) n_contrib[t.pix] = count;
        }
        if (!kPersistent) break;
    }
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------

// Sum of r[0..8] over the warp through shared memory.  Every lane stores its
// nine terms as one 10-float row of the warp's buffer (four 8-byte stores and
// one 4-byte store; at a 10-word row stride the 8-byte stores of a half-warp
// hit 32 distinct banks).  Lane L < 27 then sums column L / 3 over the rows
// congruent to L % 3 modulo 3 (11 or 10 rows); the three parts of a column
// start 10 banks apart, so each of those loads is conflict-free.  Two
// shuffles fold the parts: lane 3q returns the total of term q.  The
// summation order is fixed, so results are deterministic.
constexpr int kRedStride = 10;

struct RedLane {
    int q, part;  // column and row residue this lane sums
};

__device__ __forceinline__ RedLane red_lane(int lane)
{
    return RedLane{lane / 3, lane % 3};
}

__device__ __forceinline__ float warp_sum9(const float (&r)[kRec], float* buf, int lane, RedLane rl)
{
    float* row = buf + lane * kRedStride;
    *reinterpret_cast<float2*>(row + 0) = make_float2(r[0], r[1]);
    *reinterpret_cast<float2*>(row + 2) = make_float2(r[2], r[3]);
    *reinterpret_cast<float2*>(row + 4) = make_float2(r[4], r[5]);
    *reinterpret_cast<float2*>(row + 6) = make_float2(r[6], r[7]);
    row[8] = r[8];
    __syncwarp();
    float acc = 0.f;
    if (lane < 3 * kRec) {
        const float* col = buf + rl.part * kRedStride + rl.q;
#pragma unroll
        for (int i = 0; i < 11; ++i)
            if (rl.part + 3 * i < 32) acc += col[3 * i * kRedStride];
    }
    __syncwarp();  // the buffer is free again
    const float a1 = __shfl_down_sync(kFull, acc, 1);
    const float a2 = __shfl_down_sync(kFull, acc, 2);
    return acc + (a1 + a2);  // lane 3q: part 0 + (part 1 + part 2)
}

// kAtomic: each (tile, Gaussian) sum is added straight into the per-projection
// outputs with vector reduction atomics (fast; fp32 summation order across
// tiles varies).  Otherwise it is written as a record for k_reduce_records
// (deterministic).
template <bool kCull, bool kAtomic, bool kPersistent>
__global__ void __launch_bounds__(256, 4)
k_raster_bwd(const GsView* __restrict__ views, int V, int T_total, const int32_t* __restrict__ tile_order,
             int* __restrict__ queue, const float2* __restrict__ means2d,
             const float* __restrict__ conics, const float* __restrict__ opacities, const float* __restrict__ colors,
             const int32_t* __restrict__ isect_ids, const int2* __restrict__ tile_ranges,
             const float* __restrict__ background, const float* __restrict__ T_final,
             const int32_t* __restrict__ last_idx, const float* __restrict__ dL_drgb, float* __restrict__ records,
             float2* __restrict__ dL_dmeans2d, float* __restrict__ dL_dconics, float* __restrict__ dL_dopacities,
             float* __restrict__ dL_dcolors)
{
    // deterministic: one partial slot per warp, summed in warp order; atomic:
    // one slot per Gaussian, accumulated with shared-memory atomics (less
    // shared memory, so larger batches)
    constexpr int kB = kAtomic ? 256 : kBwdBatch;
    constexpr int kSlots = kAtomic ? 1 : kWarps;
    __shared__ float4 sh_xy[kB], sh_q[kB], sh_col[kB], sh_cull[kB];
    __shared__ float s_grad[kSlots][kB][kRec];
    __shared__ unsigned s_mask[kSlots][kB / 32];
    __shared__ __align__(16) float s_red[kWarps][32 * kRedStride];
    __shared__ int s_maxlast[kWarps];
    __shared__ int s_next;
    for (int qi = blockIdx.x;;) {
        if (kPersistent) {
            __syncthreads();  // the previous tile is done with shared memory
            if (threadIdx.x == 0) s_next = atomicAdd(queue, 1);
            __syncthreads();
            qi = s_next;
            if (qi >= T_total) break;
        }
        const int tile = tile_order ? tile_order[qi] : qi;
        const TileCtx t = tile_ctx(views, V, tile);
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        const int2 range = tile_ranges[tile];

        float T = 1.f, g0 = 0.f, g1 = 0.f, g2 = 0.f, bgT = 0.f;
        int last = range.x - 1;
        if (t.inside) {
            T = T_final[t.pix];
            last = last_idx[t.pix];
            g0 = dL_drgb[3 * t.pix + 0];
            g1 = dL_drgb[3 * t.pix + 1];
            g2 = dL_drgb[3 * t.pix + 2];
            if (background) bgT = T * (background[0] * g0 + background[1] * g1 + background[2] * g2);
        }
        float SdL = 0.f;  // S_n . dL/dC, S_n = sum_{m>n} c_m alpha_m T_m
        const RedLane rl = red_lane(lane);

        // the warp's and the tile's largest last index bound the work
        int wl = last;
    #pragma unroll
        for (int d = 16; d > 0; d >>= 1) wl = max(wl, __shfl_xor_sync(kFull, wl, d));
        if (lane == 0) s_maxlast[w] = wl;
        __syncthreads();
        int maxlast = s_maxlast[0];
    #pragma unroll
        for (int i = 1; i < kWarps; ++i) maxlast = max(maxlast, s_maxlast[i]);

        const int nbatch = maxlast >= range.x ? (maxlast - range.x) / kB + 1 : 0;
        for (int k = nbatch - 1; k >= 0; --k) {
            const int b0 = range.x + k * kB;
            const int n = min(kB, maxlast - b0 + 1);
            if (kAtomic) {
                for (int i = threadIdx.x; i < kB * kRec; i += blockDim.x) (&s_grad[0][0][0])[i] = 0.f;
                if (threadIdx.x < kB / 32) s_mask[0][threadIdx.x] = 0u;
            }
            if (threadIdx.x < n) {
                const int p = isect_ids[b0 + threadIdx.x];
                const int64_t g = p + t.g_shift;
                stage_gaussian(sh_xy, sh_q, sh_col, sh_cull, threadIdx.x, means2d[p], conics[3 * p], conics[3 * p + 1],
                               conics[3 * p + 2], opacities[g], colors[3 * g], colors[3 * g + 1], colors[3 * g + 2]);
                sh_cull[threadIdx.x].w = __int_as_float(p);  // the projection, for the atomic flush
            }
            __syncthreads();
            // this warp only needs entries up to its own last index
            const int nw = min(n, wl - b0 + 1);
            for (int s = ((kB - 1) >> 5) << 5; s >= 0; s -= 32) {
                unsigned chunk_mask = 0u;  // Gaussians of this chunk the warp wrote a partial for
                if (s < nw) {
                    bool hit = s + lane < nw;
                    if (kCull && hit)
                        hit = reaches_box(load_staged(sh_xy, sh_q, sh_col, sh_cull, s + lane), t.wx0, t.wx1, t.wy0,
                                          t.wy1);
                    unsigned m = __ballot_sync(kFull, hit);
                    while (m) {
                        const int hb = 31 - __clz(m);
                        m ^= 1u << hb;
                        const int j = s + hb;  // back to front
                        // every lane evaluates; lanes that do not composite this
                        // Gaussian carry zero terms (selects, no branches)
                        const float4 xy = sh_xy[j];
                        const float4 qq = sh_q[j];
                        const float4 col = sh_col[j];
                        const float dx = xy.x - t.cx, dy = xy.y - t.cy;
                        float u;
                        const float p2 = neg_sigma_log2(qq, dx, dy, u);
                        const float ge = ex2(p2);  // exp(-sigma)
                        const float raw = __fmul_rn(xy.z, ge);
                        const float alpha = fminf(GS_ALPHA_MAX, raw);
                        const bool contrib = (b0 + j <= last) && (p2 <= 0.f) && (alpha >= GS_ALPHA_MIN);
                        const unsigned cm = __ballot_sync(kFull, contrib);
                        if (cm == 0u) continue;
                        const float inv1ma = __fdividef(1.f, 1.f - alpha);
                        const float Tn = T * inv1ma;  // T before this Gaussian
                        const float wgt = contrib ? alpha * Tn : 0.f;
                        const float cdot = fmaf(col.x, g0, fmaf(col.y, g1, col.z * g2));
                        const float dL_dalpha = fmaf(Tn, cdot, -(SdL + bgT) * inv1ma);
                        const float gd = (contrib && raw < GS_ALPHA_MAX) ? ge * dL_dalpha : 0.f;  // dL/do
                        SdL = fmaf(wgt, cdot, SdL);
                        T = contrib ? Tn : T;
                        const float ds = -xy.z * gd;  // dL/dsigma
                        const float hds = 0.5f * ds;
                        float r[kRec];
                        r[0] = ds * (xy.w * u);                    // Y Delta = (a u, b u + D dy)
                        r[1] = ds * fmaf(qq.w, u, col.w * dy);
                        r[2] = hds * dx * dx;
                        r[3] = ds * dx * dy;
                        r[4] = hds * dy * dy;
                        r[5] = gd;
                        r[6] = wgt * g0;
                        r[7] = wgt * g1;
                        r[8] = wgt * g2;
                        chunk_mask |= 1u << hb;
                        float* slot = s_grad[kAtomic ? 0 : w][j];
                        if (__popc(cm) == 1) {
                            // one contributing pixel: its terms are the warp's sum
                            if (contrib) {
    #pragma unroll
                                for (int q = 0; q < kRec; ++q) {
                                    if (kAtomic) atomicAdd(slot + q, r[q]);
                                    else slot[q] = r[q];
                                }
                            }
                        } else {
                            const float tot = warp_sum9(r, s_red[w], lane, rl);
                            if (lane < 3 * kRec && rl.part == 0) {
                                if (kAtomic) atomicAdd(slot + rl.q, tot);
                                else slot[rl.q] = tot;
                            }
                        }
                    }
                }
                if (lane == 0) {
                    if (kAtomic) {
                        if (chunk_mask) atomicOr(&s_mask[0][s >> 5], chunk_mask);
                    } else {
                        s_mask[w][s >> 5] = chunk_mask;
                    }
                }
            }
            __syncthreads();
            // fixed-order sum over warps: one (tile, Gaussian) partial
            if (threadIdx.x < n) {
                const int j = threadIdx.x;
                float acc[kRec];
    #pragma unroll
                for (int q = 0; q < kRec; ++q) acc[q] = 0.f;
                bool any = false;
    #pragma unroll
                for (int ww = 0; ww < kSlots; ++ww)
                    if (s_mask[ww][j >> 5] & (1u << (j & 31))) {
                        any = true;
    #pragma unroll
                        for (int q = 0; q < kRec; ++q) acc[q] += s_grad[ww][j][q];
                    }
                if (kAtomic) {
                    if (any) {
                        const int p = __float_as_int(sh_cull[j].w);
                        const int64_t g = p + t.g_shift;
                        atomicAdd(dL_dmeans2d + p, make_float2(acc[0], acc[1]));
                        atomicAdd(dL_dconics + 3 * p + 0, acc[2]);
                        atomicAdd(dL_dconics + 3 * p + 1, acc[3]);
                        atomicAdd(dL_dconics + 3 * p + 2, acc[4]);
                        atomicAdd(dL_dopacities + g, acc[5]);
                        atomicAdd(dL_dcolors + 3 * g + 0, acc[6]);
                        atomicAdd(dL_dcolors + 3 * g + 1, acc[7]);
                        atomicAdd(dL_dcolors + 3 * g + 2, acc[8]);
                    }
                } else {
                    float* rec = records + (size_t)(b0 + j) * kRec;
    #pragma unroll
                    for (int q = 0; q < kRec; ++q) rec[q] = acc[q];
                }
            }
            __syncthreads();
        }
        if (!kAtomic) {
            // Gaussians after every pixel's last one received nothing
            const int first_unused = max(range.x, maxlast + 1);
            for (int i = first_unused + threadIdx.x; i < range.y; i += blockDim.x) {
                float* rec = records + (size_t)i * kRec;
    #pragma unroll
                for (int q = 0; q < kRec; ++q) rec[q] = 0.f;
            }
        }
        if (!kPersistent) break;
    }
}

// Per projection: sum of its (tile, Gaussian) records in emission order.
__global__ void __launch_bounds__(256)
k_reduce_records(const GsView* __restrict__ views, int V, int64_t P, const int32_t* __restrict__ touched,
                 const int32_t* __restrict__ emit_start, const int32_t* __restrict__ isect_pos,
                 const int32_t* __restrict__ K_dev, int64_t cap, const float* __restrict__ records,
                 float2* __restrict__ dL_dmeans2d, float* __restrict__ dL_dconics, float* __restrict__ dL_dopacities,
                 float* __restrict__ dL_dcolors)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int n = touched[p];
    if (n <= 0) return;
    const int64_t K = min((int64_t)*K_dev, cap);
    const int64_t e0 = emit_start[p];
    if (e0 < 0 || e0 + n > K) return;  // capacity overflow: outputs are flagged invalid
    float acc[kRec];
#pragma unroll
    for (int q = 0; q < kRec; ++q) acc[q] = 0.f;
    for (int j = 0; j < n; ++j) {
        const float* rec = records + (size_t)isect_pos[e0 + j] * kRec;
#pragma unroll
        for (int q = 0; q < kRec; ++q) acc[q] += rec[q];
    }
    float2 m = dL_dmeans2d[p];
    m.x += acc[0];
    m.y += acc[1];
    dL_dmeans2d[p] = m;
    dL_dconics[3 * p + 0] += acc[2];
    dL_dconics[3 * p + 1] += acc[3];
    dL_dconics[3 * p + 2] += acc[4];
    const GsView& view = views[view_of_projection(views, V, p)];
    const int64_t g = view.g_begin + (p - view.proj_offset);
    atomicAdd(dL_dopacities + g, acc[5]);
    atomicAdd(dL_dcolors + 3 * g + 0, acc[6]);
    atomicAdd(dL_dcolors + 3 * g + 1, acc[7]);
    atomicAdd(dL_dcolors + 3 * g + 2, acc[8]);
}

// GS_NO_CULL=1 in the environment visits every (pixel, Gaussian) pair; the
// results must not change (checked by the test-suite).
static bool cull_enabled()
{
    const char* e = getenv("GS_NO_CULL");
    return !(e && e[0] == '1');
}

}  // namespace gs

using namespace gs;

// Grid for a launch of `kernel`: one CTA per tile, or a persistent grid.
template <typename K>
static int raster_grid(K kernel, const GsRasterConfig* cfg, int32_t T_total, unsigned* grid)
{
    if (!cfg || !cfg->persistent) {
        *grid = (unsigned)T_total;
        return GS_OK;
    }
    int dev = 0, sms = 0, fit = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
        cudaSuccess || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kernel, 256, 0) != cudaSuccess)
        return launch_status("raster grid");
    int per = cfg->ctas_per_sm > 0 ? std::min(cfg->ctas_per_sm, fit) : fit;
    per = std::max(per, 1);
    *grid = (unsigned)std::min<int64_t>((int64_t)per * sms, T_total);
    return GS_OK;
}

static int check_config(const GsRasterConfig* cfg, const char* who)
{
    if (cfg && cfg->persistent && !cfg->queue) return fail(GS_ERR_INVALID_ARG, "%s: persistent needs a queue", who);
    return GS_OK;
}

extern "C" int gs_rasterize_fwd(const GsView* views, int32_t V, int32_t T_total, const float* means2d,
                                const float* conics, const float* opacities, const float* colors,
                                const int32_t* isect_ids, const int32_t* tile_ranges, const float* background,
                                float* out_rgb, float* T_final, int32_t* last_idx, int32_t* n_contrib,
                                const GsRasterConfig* config, void* stream)
{
    if (V <= 0 || T_total < 0)
        return fail(GS_ERR_INVALID_ARG, "gs_rasterize_fwd: V=%d T_total=%d", V, T_total);
    if (!views || !tile_ranges || !out_rgb || !T_final || !last_idx)
        return fail(GS_ERR_INVALID_ARG, "gs_rasterize_fwd: null pointer argument");
    if ((reinterpret_cast<uintptr_t>(means2d) & 7) || (reinterpret_cast<uintptr_t>(tile_ranges) & 7))
        return fail(GS_ERR_INVALID_ARG, "gs_rasterize_fwd: means2d and tile_ranges need 8-byte alignment");
    if (int rc = check_config(config, "gs_rasterize_fwd")) return rc;
    if (T_total == 0) return GS_OK;
    cudaStream_t s = as_stream(stream);
    const bool cull = cull_enabled(), pers = config && config->persistent;
    auto kern = cull ? (pers ? k_raster_fwd<true, true> : k_raster_fwd<true, false>)
                     : (pers ? k_raster_fwd<false, true> : k_raster_fwd<false, false>);
    unsigned grid;
    if (int rc = raster_grid(kern, config, T_total, &grid)) return rc;
    int* queue = pers ? config->queue : nullptr;
    if (pers && cudaMemsetAsync(queue, 0, sizeof(int), s) != cudaSuccess) return launch_status("gs_rasterize_fwd");
    kern<<<grid, 256, 0, s>>>(views, V, T_total, config ? config->tile_order : nullptr, queue,
                              reinterpret_cast<const float2*>(means2d), conics, opacities, colors, isect_ids,
                              reinterpret_cast<const int2*>(tile_ranges), background, out_rgb, T_final, last_idx,
                              n_contrib);
    count_launches(1);
    return launch_status("gs_rasterize_fwd");
}

extern "C" size_t gs_rasterize_bwd_workspace_size(int64_t K_capacity, int32_t deterministic)
{
    if (K_capacity < 0) return 0;
    return deterministic ? align256((size_t)K_capacity * kRec * sizeof(float)) : 0;
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
    if (V <= 0 || P < 0 || T_total < 0 || K_capacity < 0 || K_capacity >= (int64_t(1) << 31))
        return fail(GS_ERR_INVALID_ARG, "gs_rasterize_bwd: V=%d P=%lld T_total=%d K_capacity=%lld", V, (long long)P,
                    T_total, (long long)K_capacity);
    if (!views || !tile_ranges || !T_final || !last_idx || !dL_drgb ||
        (P > 0 && (!dL_dmeans2d || !dL_dconics || !dL_dopacities || !dL_dcolors)) ||
        (deterministic && P > 0 && (!K || !touched || !emit_start || !isect_pos)))
        return fail(GS_ERR_INVALID_ARG, "gs_rasterize_bwd: null pointer argument");
    if ((reinterpret_cast<uintptr_t>(means2d) & 7) || (reinterpret_cast<uintptr_t>(dL_dmeans2d) & 7) ||
        (reinterpret_cast<uintptr_t>(tile_ranges) & 7))
        return fail(GS_ERR_INVALID_ARG, "gs_rasterize_bwd: float2 arrays need 8-byte alignment");
    const size_t need = gs_rasterize_bwd_workspace_size(K_capacity, deterministic);
    if (workspace_bytes < need || (need > 0 && !workspace))
        return fail(GS_ERR_INVALID_ARG, "gs_rasterize_bwd: workspace of %zu bytes, need %zu", workspace_bytes, need);
    if (int rc = check_config(config, "gs_rasterize_bwd")) return rc;
    if (T_total == 0 || P == 0) return GS_OK;
    cudaStream_t s = as_stream(stream);
    float* records = static_cast<float*>(workspace);
    const bool cull = cull_enabled(), pers = config && config->persistent;
    using KB = decltype(&k_raster_bwd<true, true, true>);
    static const KB table[2][2][2] = {
        {{k_raster_bwd<false, false, false>, k_raster_bwd<false, false, true>},
         {k_raster_bwd<false, true, false>, k_raster_bwd<false, true, true>}},
        {{k_raster_bwd<true, false, false>, k_raster_bwd<true, false, true>},
         {k_raster_bwd<true, true, false>, k_raster_bwd<true, true, true>}}};
    const KB kern = table[cull][!deterministic][pers];
    unsigned grid;
    if (int rc = raster_grid(kern, config, T_total, &grid)) return rc;
    int* queue = pers ? config->queue : nullptr;
    if (pers && cudaMemsetAsync(queue, 0, sizeof(int), s) != cudaSuccess) return launch_status("gs_rasterize_bwd");
    kern<<<grid, 256, 0, s>>>(views, V, T_total, config ? config->tile_order : nullptr, queue,
                              reinterpret_cast<const float2*>(means2d), conics, opacities, colors, isect_ids,
                              reinterpret_cast<const int2*>(tile_ranges), background, T_final, last_idx, dL_drgb,
                              records, reinterpret_cast<float2*>(dL_dmeans2d), dL_dconics, dL_dopacities,
                              dL_dcolors);
    count_launches(1);
    if (deterministic) {
        k_reduce_records<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(
            views, V, P, touched, emit_start, isect_pos, K, K_capacity, records,
            reinterpret_cast<float2*>(dL_dmeans2d), dL_dconics, dL_dopacities, dL_dcolors);
        count_launches(1);
    }
    return launch_status("gs_rasterize_bwd");
}
