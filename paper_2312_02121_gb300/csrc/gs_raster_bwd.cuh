// The compositing backward of Sec. 3.1 (3 channels, or 1-3 channels C apart),
// templated on the scalar type, on how many pixels each thread owns and on
// the staging batch -- the batch shape the autotuner chooses between.  The
// kernels are instantiated in gs_raster.cu (one pixel per thread, and every
// fp64 variant) and gs_raster_bwd2.cu (two pixels per thread), so that the
// two groups compile in parallel.
//
// Layout of a CTA: one 16x16 tile.  With one pixel per thread the CTA has 8
// warps, warp w on the 8x4 pixel box (w & 1, w >> 1) -- the boxes of the
// forward's warps, whose cull ballots the backward reads.  With two pixels per
// thread it has 4 warps, warp w on the 8x8 box (w & 1, w >> 1); lane L owns
// pixel (L & 7, L >> 3) of the box's upper 8x4 half and the pixel 4 rows
// below it, in the lower half.  The two halves are the boxes of forward warps
// w' and w' + 2 (w' = (w & 1) + 4 (w >> 1)), so each half walks the forward's
// ballots of its own box, and a Gaussian that reaches both halves is
// evaluated for both pixels and reduced over the warp once: the reduction
// costs the same per event but now covers 64 pixels.
//
// The walk is back to front from each pixel's last composited Gaussian,
// rebuilding T_n from the saved T_final (Sec. 3.1).  The nine per-pixel
// gradient terms of a Gaussian are summed over the warp through a
// shared-memory transpose into the warp's own slot for that Gaussian (plain
// stores), and the slots of the tile's warps are summed in a fixed order,
// giving one partial per (tile, Gaussian).  The fast mode adds the partials
// straight into the per-projection outputs with global atomics; the
// deterministic mode writes them as records that a second kernel sums per
// projection in emission order.
#pragma once

#include "gs_raster_common.cuh"

namespace gs {

constexpr int kRec = 9;  // dmu'(2) dconic(3: a, k, D) dopacity(1) dcolor(3)

// These kernels composite up to 3 channels (the RGB of Eq. 7) of colours whose values are C apart
// per Gaussian or pixel: CW = 1, 2 or 3 of them, from the pointers given (a chunk of a C-channel
// image starts at an offset).  A channel past CW reads as zero (zero colour, zero dL/dC, so it adds
// nothing to alpha's gradient) and is never written.
template <typename S>
__device__ __forceinline__ void load_c3(const S* __restrict__ a, int64_t i, int C, int CW, S& x, S& y, S& z)
{
    const S* b = a + (int64_t)C * i;
    x = b[0];
    y = CW > 1 ? b[1] : S(0);
    z = CW > 2 ? b[2] : S(0);
}

// Sum of r[0..8] over the warp through shared memory.  Every lane stores its
// nine terms as one 10-scalar row of the warp's buffer (four 2-vector stores
// and one scalar store; in fp32 the 8-byte stores of a half-warp hit 32
// distinct banks at this stride).  Lane L < 27 then sums column L / 3 over the
// rows congruent to L % 3 modulo 3 (11 or 10 rows); the three parts of a
// column start 10 banks apart, so each of those loads is conflict-free in
// fp32.  Two shuffles fold the parts: lane 3q returns the total of term q.
// The summation order is fixed, so results are deterministic.
constexpr int kRedStride = 10;

struct RedLane {
    int q, part;  // column and row residue this lane sums
};

__device__ __forceinline__ RedLane red_lane(int lane)
{
    return RedLane{lane / 3, lane % 3};
}

template <typename S>
__device__ __forceinline__ S warp_sum9(const S (&r)[kRec], S* buf, int lane, RedLane rl)
{
    S* row = buf + lane * kRedStride;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        V2<S> v;
        v.x = r[2 * i];
        v.y = r[2 * i + 1];
        *reinterpret_cast<V2<S>*>(row + 2 * i) = v;
    }
    row[8] = r[8];
    __syncwarp();
    // lanes 27-31 sum a valid column too (their result is not used): no branch
    const S* col = buf + rl.part * kRedStride + min(rl.q, kRec - 1);
    S acc = 0;
#pragma unroll
    for (int i = 0; i < 10; ++i) acc += col[3 * i * kRedStride];
    const S tail = col[(rl.part < 2 ? 30 : 27) * kRedStride];  // rows 30, 31 exist for residues 0, 1
    acc += rl.part < 2 ? tail : S(0);
    __syncwarp();  // the buffer is free again
    const S a1 = __shfl_down_sync(kFull, acc, 1);
    const S a2 = __shfl_down_sync(kFull, acc, 2);
    return acc + (a1 + a2);  // lane 3q: part 0 + (part 1 + part 2)
}

// One (tile, Gaussian) partial of a walked batch: the fixed-order sum of the
// kNW warps' slots, turned into dL/dmu' and dL/dconic, added to the
// outputs (fast mode) or written as a record (deterministic mode).  fl holds
// the Gaussian's (a, b, D, stashed projection) from its staging.
template <typename S, bool kAtomic, int kNW, int kB>
__device__ __forceinline__ void flush_partial(int j, int b0, const S (*s_grad)[kB][kRec],
                                              const unsigned (*s_mask)[(kB + 31) / 32], V4<S> fl,
                                              int64_t g_shift, S* __restrict__ records,
                                              V2<S>* __restrict__ dL_dmeans2d, S* __restrict__ dL_dconics,
                                              S* __restrict__ dL_dopacities, S* __restrict__ dL_dcolors, int C,
                                              int CW)
{
    S acc[kRec];
#pragma unroll
    for (int q = 0; q < kRec; ++q) acc[q] = S(0);
    bool any = false;
#pragma unroll
    for (int ww = 0; ww < kNW; ++ww)
        if (s_mask[ww][j >> 5] & (1u << (j & 31))) {
            any = true;
#pragma unroll
            for (int q = 0; q < kRec; ++q) acc[q] += s_grad[ww][j][q];
        }
    // from the reduced sums to dL/dmu' and dL/d(a, k, D) of the factored conic (see the walk)
    const S su = acc[0], sdy = acc[1];
    acc[0] = fl.x * su;
    acc[1] = fma(fl.y, su, fl.z * sdy);
    acc[2] *= S(0.5);
    acc[3] *= fl.x;
    acc[4] *= S(0.5);
    if (kAtomic) {
        if (any) {
            const int p = RT<S>::unstash(fl.w);
            const int64_t g = p + g_shift;
            atomic_add2(dL_dmeans2d + p, acc[0], acc[1]);
            // scalar atomics: 2-vector ones for the 3-float runs were measured 0.4 % slower here
            atomicAdd(dL_dconics + 3 * p + 0, acc[2]);
            atomicAdd(dL_dconics + 3 * p + 1, acc[3]);
            atomicAdd(dL_dconics + 3 * p + 2, acc[4]);
            atomicAdd(dL_dopacities + g, acc[5]);
            S* dc = dL_dcolors + (int64_t)C * g;
            atomicAdd(dc, acc[6]);
            if (CW > 1) atomicAdd(dc + 1, acc[7]);
            if (CW > 2) atomicAdd(dc + 2, acc[8]);
        }
    } else {
        S* rec = records + (size_t)(b0 + j) * kRec;
#pragma unroll
        for (int q = 0; q < kRec; ++q) rec[q] = acc[q];
    }
}

// Threads of a backward CTA with kPx pixels per thread.
template <int kPx>
constexpr int bwd_threads() { return 32 * (kWarps / kPx); }

// kAtomic: each (tile, Gaussian) partial is added straight into the
// per-projection outputs with reduction atomics (fast; the summation order
// across tiles varies).  Otherwise it is written as a record for
// k_reduce_records (deterministic).  kPersistent / kAnyC as for the forward.
// kPx: pixels per thread (1 or 2); kB: Gaussians per staged batch (a multiple
// of 32, at most the CTA's threads).
template <typename S, bool kCull, bool kAtomic, bool kPersistent, bool kAnyC, int kPx, int kB>
__global__ void __launch_bounds__(bwd_threads<kPx>(), kPx == 1 ? 4 : 7)  // measured: 4, and 7 (72 registers; 8 CTAs at 63 was 5 % slower)
k_raster_bwd(const GsView* __restrict__ views, int V, int T_total, const int32_t* __restrict__ tile_order,
             int* __restrict__ queue, const V2<S>* __restrict__ means2d, const S* __restrict__ conics,
             const S* __restrict__ opacities, const S* __restrict__ colors, const int32_t* __restrict__ isect_ids,
             const int2* __restrict__ tile_ranges, const S* __restrict__ background, const S* __restrict__ T_final,
             const int32_t* __restrict__ last_idx, const uint32_t* __restrict__ warp_hits,
             const S* __restrict__ dL_drgb, S* __restrict__ records,
             V2<S>* __restrict__ dL_dmeans2d, S* __restrict__ dL_dconics, S* __restrict__ dL_dopacities,
             S* __restrict__ dL_dcolors, int C_arg, int W_arg)
{
    static_assert(kPx == 1 || kPx == 2, "one or two pixels per thread");
    constexpr int kNW = kWarps / kPx;  // warps per CTA, one partial slot each per Gaussian
    constexpr int kThreads = 32 * kNW;
    static_assert(kB % 32 == 0 && kB <= kThreads, "one staging thread per batch entry, whole chunks");
    static_assert(kWarps * (kB / 32) <= kThreads, "one thread per forward ballot word of a batch");
    // the flush of a walked batch runs on threads [kFlushOff, kFlushOff + kB) while threads [0, kB)
    // stage the next one, so that it costs no barrier of its own (the same threads when the block
    // has no room for both)
    constexpr int kFlushOff = 2 * kB <= kThreads ? kB : 0;
    pdl_wait();
    pdl_trigger();
    const int C = kAnyC ? C_arg : 3, CW = kAnyC ? W_arg : 3;
    __shared__ V4<S> sh_xy[kB], sh_q[kB], sh_col[kB], sh_cull[kB];
    // one partial slot per (warp, Gaussian), written with plain stores and summed in warp order at
    // the flush (shared-memory atomics into one slot per Gaussian were measured 8 % slower)
    __shared__ S s_grad[kNW][kB][kRec];
    __shared__ unsigned s_mask[kNW][(kB + 31) / 32];
    __shared__ V4<S> s_fl[2][kB];  // (a, b, D, projection) of the last two staged batches, for the flush
    __shared__ uint32_t s_hitw[(kB + 31) / 32][kWarps];  // box ballots of the staged chunks (word b: box b)
    __shared__ __align__(16) S s_red[kNW][32 * kRedStride];
    __shared__ int s_maxlast[kNW];
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
        const GsView* view = views + view_of_tile(views, V, tile);
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        const int2 range = tile_ranges[tile];
        const int64_t g_shift = (int64_t)view->g_begin - view->proj_offset;
        const int local = tile - view->tile_offset;
        const int Wd = view->cam.width, Hd = view->cam.height;
        // this warp's box: 8 pixels wide, 4 kPx high; pixel i of the lane sits 4 i rows below the first
        const int tx0 = (local % view->tiles_x) * kTile, ty0 = (local / view->tiles_x) * kTile;
        const int bx = tx0 + (w & 1) * 8;
        const int by = ty0 + (w >> 1) * 4 * kPx;
        const int px = bx + (lane & 7);
        const S cx = S(px) + S(0.5);
        S T[kPx], g0[kPx], g1[kPx], g2[kPx], cy[kPx], SdL[kPx];
        int last[kPx];
#pragma unroll
        for (int i = 0; i < kPx; ++i) {
            const int py = by + (lane >> 3) + 4 * i;
            cy[i] = S(py) + S(0.5);
            T[i] = 1;
            g0[i] = g1[i] = g2[i] = 0;
            last[i] = range.x - 1;
            S bgT = 0;
            if (px < Wd && py < Hd) {
                const int64_t pix = view->pixel_offset + (int64_t)py * Wd + px;
                T[i] = T_final[pix];
                last[i] = last_idx[pix];
                load_c3(dL_drgb, pix, C, CW, g0[i], g1[i], g2[i]);
                if (background) {
                    S b0, b1, b2;
                    load_c3(background, 0, C, CW, b0, b1, b2);
                    bgT = T[i] * (b0 * g0[i] + b1 * g1[i] + b2 * g2[i]);
                }
            }
            // S_n . dL/dC + T_final b . dL/dC, with S_n = sum_{m>n} c_m alpha_m T_m: the numerator of
            // the suffix term of dL/dalpha_n (the background part is constant per pixel, so it starts
            // the sum)
            SdL[i] = bgT;
        }
        const RedLane rl = red_lane(lane);

        // the largest last index of each half-box of the warp (whose forward ballots are valid up to
        // it), of the warp and of the tile bound the work
        int wl[kPx], wlall = range.x - 1;
#pragma unroll
        for (int i = 0; i < kPx; ++i) {
            wl[i] = last[i];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) wl[i] = max(wl[i], __shfl_xor_sync(kFull, wl[i], d));
            wlall = max(wlall, wl[i]);
        }
        if (lane == 0) s_maxlast[w] = wlall;
        __syncthreads();
        int maxlast = s_maxlast[0];
#pragma unroll
        for (int i = 1; i < kNW; ++i) maxlast = max(maxlast, s_maxlast[i]);

        // batches walk back to front
        const int nbatch = maxlast >= range.x ? (maxlast - range.x) / kB + 1 : 0;
        int prev_b0 = 0, prev_n = 0;
        for (int k = nbatch - 1; k >= 0; --k) {
            const int b0 = range.x + k * kB;
            const int n = min(kB, maxlast - b0 + 1);
            // word ww of a chunk is forward warp ww's ballot; a chunk of fewer than 8 entries kept the
            // first warps' words only, and the other boxes walk all of it (loaded first, so that its
            // latency overlaps the staging loads)
            const bool put_hits = warp_hits && threadIdx.x < kWarps * ((n + 31) >> 5);
            uint32_t hw = kFull;
            if (put_hits) {
                const int e0 = b0 + 32 * (threadIdx.x / kWarps), ww = threadIdx.x % kWarps;
                if (ww < range.y - e0) hw = warp_hits[e0 + ww];
            }
            if (threadIdx.x < n) {
                const int p = isect_ids[b0 + threadIdx.x];
                const int64_t g = p + g_shift;
                S c0, c1, c2;
                load_c3(colors, g, C, CW, c0, c1, c2);
                // with the forward's ballots the backward never reads the cull thresholds
                stage_gaussian<S>(sh_xy, sh_q, sh_col, sh_cull, threadIdx.x, means2d[p], conics[3 * p],
                                  conics[3 * p + 1], conics[3 * p + 2], opacities[g], c0, c1, c2, !warp_hits);
                s_fl[k & 1][threadIdx.x] = mk4<S>(sh_xy[threadIdx.x].w, sh_q[threadIdx.x].w, sh_col[threadIdx.x].w,
                                                  RT<S>::stash(p));
            }
            if (kCull && !warp_hits && threadIdx.x < kB) {
                // without the forward's ballots: the same box test for each staged Gaussian against the
                // tile's 8 boxes, turned into the forward's word layout by one ballot per box over each
                // staging warp (whole warps: kB is a multiple of 32)
                unsigned reach = 0u;
                if (threadIdx.x < n) {
                    const Staged<S> st = load_staged<S>(sh_xy, sh_q, sh_col, sh_cull, threadIdx.x);
#pragma unroll
                    for (int b = 0; b < kWarps; ++b) {
                        const S x0 = S(tx0 + (b & 1) * 8) + S(0.5), y0 = S(ty0 + (b >> 1) * 4) + S(0.5);
                        reach |= (unsigned)reaches_box(st, x0, x0 + S(7), y0, y0 + S(3)) << b;
                    }
                }
#pragma unroll
                for (int b = 0; b < kWarps; ++b) {
                    const unsigned word = __ballot_sync(kFull, (reach >> b) & 1u);
                    if (lane == b) s_hitw[threadIdx.x >> 5][b] = word;
                }
            }
            if (kFlushOff == 0 || threadIdx.x >= kFlushOff) {
                const int j = threadIdx.x - kFlushOff;
                if (j < prev_n)
                    flush_partial<S, kAtomic, kNW, kB>(j, prev_b0, s_grad, s_mask, s_fl[(k + 1) & 1][j], g_shift,
                                                       records, dL_dmeans2d, dL_dconics, dL_dopacities, dL_dcolors,
                                                       C, CW);
            }
            if (put_hits) (&s_hitw[0][0])[threadIdx.x] = hw;
            __syncthreads();
            int lastj[kPx];  // each pixel's last index, relative to the batch
#pragma unroll
            for (int i = 0; i < kPx; ++i) lastj[i] = last[i] - b0;
            for (int s = ((kB - 1) >> 5) << 5; s >= 0; s -= 32) {
                unsigned chunk_mask = 0u;  // Gaussians of this chunk the warp wrote a partial for
                // the entries of this chunk each half-box may need: up to its own largest last index
                unsigned mi[kPx], m = 0u;
#pragma unroll
                for (int i = 0; i < kPx; ++i) {
                    const int lim = min(n, wl[i] - b0 + 1) - s;
                    const unsigned valid = lim <= 0 ? 0u : lim >= 32 ? kFull : (1u << lim) - 1u;
                    // the box's ballot of this chunk (the forward's, or the staging's box test)
                    mi[i] = (kCull || warp_hits) ? s_hitw[s >> 5][(w & 1) + 2 * (kPx * (w >> 1) + i)] & valid
                                                 : valid;
                    m |= mi[i];
                }
                while (m) {
                    const int hb = 31 - __clz(m);
                    m ^= 1u << hb;
                    const int j = s + hb;  // back to front
                    // each box the Gaussian can reach is evaluated and, when one of its pixels composites
                    // it, turned into gradient terms at once (lanes whose pixel does not composite it carry
                    // zero terms: selects, no branches); the warp then reduces once for all its pixels
                    const V4<S> xy = sh_xy[j];
                    const V4<S> qq = sh_q[j];
                    const V4<S> col = sh_col[j];
                    const S dx = xy.x - cx;
                    S r[kRec];
#pragma unroll
                    for (int q = 0; q < kRec; ++q) r[q] = S(0);
                    bool any = false;
#pragma unroll
                    for (int i = 0; i < kPx; ++i) {
                        if (kPx > 1 && !((mi[i] >> hb) & 1u)) continue;  // warp-uniform
                        const S dy = xy.y - cy[i];
                        S u;
                        const S p2 = neg_sigma_log2(qq, dx, dy, u);
                        const S ge = RT<S>::ex2(p2);  // exp(-sigma)
                        const S raw = mul_rn(xy.z, ge);
                        const S alpha = fmin(RT<S>::alpha_max(), raw);
                        const bool ctb = (j <= lastj[i]) && (p2 <= S(0)) && (raw >= RT<S>::alpha_min());
                        if (__ballot_sync(kFull, ctb) == 0u) continue;  // warp-uniform
                        const S inv1ma = RT<S>::rcp(S(1) - alpha);
                        const S Tn = T[i] * inv1ma;  // T before this Gaussian
                        const S wgt = ctb ? alpha * Tn : S(0);
                        const S cdot = fma(col.x, g0[i], fma(col.y, g1[i], col.z * g2[i]));
                        const S dL_dalpha = fma(Tn, cdot, -SdL[i] * inv1ma);
                        const S gd = (ctb && raw < RT<S>::alpha_max()) ? ge * dL_dalpha : S(0);  // dL/do
                        SdL[i] = fma(wgt, cdot, SdL[i]);
                        T[i] = ctb ? Tn : T[i];
                        const S ds = -xy.z * gd;  // dL/dsigma
                        // the sums the warp reduces; the flush turns them into the gradients: with
                        // sigma = (a u^2 + D dy^2) / 2, u = dx + k dy,
                        // dL/dmu' = (a sum ds u, b sum ds u + D sum ds dy) and
                        // dL/d(a, k, D) = (sum ds u^2 / 2, a sum ds u dy, sum ds dy^2 / 2)
                        const S dsu = ds * u;
                        const S dsdy = ds * dy;
                        const S t[kRec] = {dsu, dsdy, dsu * u, dsu * dy, dsdy * dy, gd,
                                           wgt * g0[i], wgt * g1[i], wgt * g2[i]};
#pragma unroll
                        for (int q = 0; q < kRec; ++q) r[q] = i == 0 ? t[q] : r[q] + t[q];
                        any = true;
                    }
                    if (!any) continue;
                    chunk_mask |= 1u << hb;
                    // the warp's sum of each term, into the warp's own slot for this Gaussian (a
                    // lone contributing lane is not special-cased: the transpose is cheaper than its
                    // nine dependent stores)
                    const S tot = warp_sum9<S>(r, s_red[w], lane, rl);
                    if (lane < 3 * kRec && rl.part == 0) s_grad[w][j][rl.q] = tot;
                }
                if (lane == 0) s_mask[w][s >> 5] = chunk_mask;
            }
            __syncthreads();  // the walk's slots and masks are complete before the next flush reads them
            prev_b0 = b0;
            prev_n = n;
        }
        if (threadIdx.x < prev_n)  // the last walked batch (batch 0)
            flush_partial<S, kAtomic, kNW, kB>(threadIdx.x, prev_b0, s_grad, s_mask, s_fl[0][threadIdx.x], g_shift,
                                               records, dL_dmeans2d, dL_dconics, dL_dopacities, dL_dcolors, C, CW);
        if (!kAtomic) {
            // Gaussians after every pixel's last one received nothing
            const int first_unused = max(range.x, maxlast + 1);
            for (int i = first_unused + threadIdx.x; i < range.y; i += blockDim.x) {
                S* rec = records + (size_t)i * kRec;
#pragma unroll
                for (int q = 0; q < kRec; ++q) rec[q] = S(0);
            }
        }
        if (!kPersistent) break;
    }
}

// The kernel type every backward instantiation shares.
template <typename S>
using RasterBwdKernel = void (*)(const GsView*, int, int, const int32_t*, int*, const V2<S>*, const S*, const S*,
                                 const S*, const int32_t*, const int2*, const S*, const S*, const int32_t*,
                                 const uint32_t*, const S*, S*, V2<S>*, S*, S*, S*, int, int);

// Two-pixel kernels (gs_raster_bwd2.cu): the instantiation for (cull, atomic,
// persistent, any-channel, batch), or nullptr when that combination is not
// compiled (batches of 64 have every variant; other batches only the culling
// ones).
RasterBwdKernel<float> raster_bwd_px2_kernel(bool cull, bool atomic, bool persistent, bool any_c, int batch);

}  // namespace gs
