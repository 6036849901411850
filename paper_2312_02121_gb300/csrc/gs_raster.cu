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
#include "gs_raster_common.cuh"

namespace gs {

constexpr int kRec = 9;  // dmu'(2) dconic(3) dopacity(1) dcolor(3)

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
// stride cost the 3-channel walk 2 %).
template <typename S, bool kCull, bool kPersistent, bool kCount, bool kAnyC>
__global__ void __launch_bounds__(256, 6)  // 6 CTAs per SM (40 registers) measured fastest
k_raster_fwd(const GsView* __restrict__ views, int V, int T_total, const int32_t* __restrict__ tile_order,
             int* __restrict__ queue, const V2<S>* __restrict__ means2d, const S* __restrict__ conics,
             const S* __restrict__ opacities, const S* __restrict__ colors, const int32_t* __restrict__ isect_ids,
             const int2* __restrict__ tile_ranges, const S* __restrict__ background, S* __restrict__ out_rgb,
             S* __restrict__ T_final, int32_t* __restrict__ last_idx, int32_t* __restrict__ n_contrib,
             uint32_t* __restrict__ warp_hits, int C_arg, int W_arg)
{
    pdl_wait();
    pdl_trigger();
    const int C = kAnyC ? C_arg : 3, CW = kAnyC ? W_arg : 3;
    constexpr int kB = RT<S>::kFwdBatch;
    __shared__ V4<S> sh_xy[kB], sh_q[kB], sh_col[kB], sh_cull[kB];
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
                if (__all_sync(kFull, done)) break;
            }
            if (lastj >= 0) last = b0 + lastj;
        }
        if (t.inside) {
            S bg0 = 0, bg1 = 0, bg2 = 0;
            if (background) load_c3(background, 0, C, CW, bg0, bg1, bg2);
            S* o = out_rgb + (int64_t)C * t.pix;
            o[0] = fma(T, bg0, C0);
            if (CW > 1) o[1] = fma(T, bg1, C1);
            if (CW > 2) o[2] = fma(T, bg2, C2);
            T_final[t.pix] = T;
            last_idx[t.pix] = last;
            if (kCount) n_contrib[t.pix] = count;
        }
        if (!kPersistent) break;
    }
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------

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
// warps' slots, turned into dL/dmu' and the packed dL/dconic, added to the
// outputs (fast mode) or written as a record (deterministic mode).  fl holds
// the Gaussian's (a, b, D, stashed projection) from its staging.
template <typename S, bool kAtomic, int kB>
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
    for (int ww = 0; ww < kWarps; ++ww)
        if (s_mask[ww][j >> 5] & (1u << (j & 31))) {
            any = true;
#pragma unroll
            for (int q = 0; q < kRec; ++q) acc[q] += s_grad[ww][j][q];
        }
    // from the reduced sums to dL/dmu' and the packed dL/dconic (see the walk)
    const S su = acc[0], sdy = acc[1];
    acc[0] = fl.x * su;
    acc[1] = fma(fl.y, su, fl.z * sdy);
    acc[2] *= S(0.5);
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

// kAtomic: each (tile, Gaussian) partial is added straight into the
// per-projection outputs with reduction atomics (fast; the summation order
// across tiles varies).  Otherwise it is written as a record for
// k_reduce_records (deterministic).  kAnyC as for the forward.
template <typename S, bool kCull, bool kAtomic, bool kPersistent, bool kAnyC>
__global__ void __launch_bounds__(256, 4)
k_raster_bwd(const GsView* __restrict__ views, int V, int T_total, const int32_t* __restrict__ tile_order,
             int* __restrict__ queue, const V2<S>* __restrict__ means2d, const S* __restrict__ conics,
             const S* __restrict__ opacities, const S* __restrict__ colors, const int32_t* __restrict__ isect_ids,
             const int2* __restrict__ tile_ranges, const S* __restrict__ background, const S* __restrict__ T_final,
             const int32_t* __restrict__ last_idx, const uint32_t* __restrict__ warp_hits,
             const S* __restrict__ dL_drgb, S* __restrict__ records,
             V2<S>* __restrict__ dL_dmeans2d, S* __restrict__ dL_dconics, S* __restrict__ dL_dopacities,
             S* __restrict__ dL_dcolors, int C_arg, int W_arg)
{
    pdl_wait();
    pdl_trigger();
    const int C = kAnyC ? C_arg : 3, CW = kAnyC ? W_arg : 3;
    // one partial slot per (warp, Gaussian), written with plain stores and summed in warp order at
    // the flush (shared-memory atomics into one slot per Gaussian were measured 8 % slower)
    constexpr int kB = RT<S>::kBwdBatch;
    constexpr int kSlots = kWarps;
    __shared__ V4<S> sh_xy[kB], sh_q[kB], sh_col[kB], sh_cull[kB];
    __shared__ S s_grad[kSlots][kB][kRec];
    __shared__ unsigned s_mask[kSlots][(kB + 31) / 32];
    __shared__ V4<S> s_fl[2][kB];  // (a, b, D, projection) of the last two staged batches, for the flush
    __shared__ uint32_t s_hitw[(kB + 31) / 32][kWarps];  // the forward's cull ballots of the staged chunks
    __shared__ __align__(16) S s_red[kWarps][32 * kRedStride];
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
        const TileCtx<S> t = tile_ctx<S>(views, V, tile);
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        const int2 range = tile_ranges[tile];

        S T = 1, g0 = 0, g1 = 0, g2 = 0, bgT = 0;
        int last = range.x - 1;
        if (t.inside) {
            T = T_final[t.pix];
            last = last_idx[t.pix];
            load_c3(dL_drgb, t.pix, C, CW, g0, g1, g2);
            if (background) {
                S b0, b1, b2;
                load_c3(background, 0, C, CW, b0, b1, b2);
                bgT = T * (b0 * g0 + b1 * g1 + b2 * g2);
            }
        }
        // S_n . dL/dC + T_final b . dL/dC, with S_n = sum_{m>n} c_m alpha_m T_m: the numerator of the
        // suffix term of dL/dalpha_n (the background part is constant per pixel, so it starts the sum)
        S SdL = bgT;
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

        // batches walk back to front; the flush of a walked batch runs on threads [kB, 2 kB) while
        // threads [0, kB) stage the next one, so that it costs no barrier of its own
        static_assert(2 * kB <= 256, "staging and flush share the block");
        const int nbatch = maxlast >= range.x ? (maxlast - range.x) / kB + 1 : 0;
        int prev_b0 = 0, prev_n = 0;
        for (int k = nbatch - 1; k >= 0; --k) {
            const int b0 = range.x + k * kB;
            const int n = min(kB, maxlast - b0 + 1);
            // word ww of a chunk is warp ww's forward ballot; a chunk of fewer than 8 entries kept the
            // first warps' words only, and the other warps walk all of it (loaded first, so that its
            // latency overlaps the staging loads)
            const bool put_hits = warp_hits && threadIdx.x < kWarps * ((n + 31) >> 5);
            uint32_t hw = kFull;
            if (put_hits) {
                const int e0 = b0 + 32 * (threadIdx.x / kWarps), ww = threadIdx.x % kWarps;
                if (ww < range.y - e0) hw = warp_hits[e0 + ww];
            }
            if (threadIdx.x < n) {
                const int p = isect_ids[b0 + threadIdx.x];
                const int64_t g = p + t.g_shift;
                S c0, c1, c2;
                load_c3(colors, g, C, CW, c0, c1, c2);
                // with the forward's ballots the backward never reads the cull thresholds
                stage_gaussian<S>(sh_xy, sh_q, sh_col, sh_cull, threadIdx.x, means2d[p], conics[3 * p],
                                  conics[3 * p + 1], conics[3 * p + 2], opacities[g], c0, c1, c2, !warp_hits);
                s_fl[k & 1][threadIdx.x] = mk4<S>(sh_xy[threadIdx.x].w, sh_q[threadIdx.x].w, sh_col[threadIdx.x].w,
                                                  RT<S>::stash(p));
            } else if (threadIdx.x >= kB && threadIdx.x < kB + prev_n) {
                const int j = threadIdx.x - kB;
                flush_partial<S, kAtomic, kB>(j, prev_b0, s_grad, s_mask, s_fl[(k + 1) & 1][j], t.g_shift, records,
                                              dL_dmeans2d, dL_dconics, dL_dopacities, dL_dcolors, C, CW);
            }
            if (put_hits) (&s_hitw[0][0])[threadIdx.x] = hw;
            __syncthreads();
            // this warp only needs entries up to its own last index
            const int nw = min(n, wl - b0 + 1);
            const int lastj = last - b0;  // this pixel's last index, relative to the batch
            for (int s = ((kB - 1) >> 5) << 5; s >= 0; s -= 32) {
                unsigned chunk_mask = 0u;  // Gaussians of this chunk the warp wrote a partial for
                if (s < nw) {
                    bool hit = s + lane < nw;
                    if (warp_hits)  // the forward's cull of the same entry against the same box
                        hit = hit && ((s_hitw[s >> 5][w] >> lane) & 1u);
                    else if (kCull && hit)
                        hit = reaches_box(load_staged<S>(sh_xy, sh_q, sh_col, sh_cull, s + lane), t.wx0, t.wx1,
                                          t.wy0, t.wy1);
                    unsigned m = __ballot_sync(kFull, hit);
                    while (m) {
                        const int hb = 31 - __clz(m);
                        m ^= 1u << hb;
                        const int j = s + hb;  // back to front
                        // every lane evaluates; lanes that do not composite this
                        // Gaussian carry zero terms (selects, no branches)
                        const V4<S> xy = sh_xy[j];
                        const V4<S> qq = sh_q[j];
                        const V4<S> col = sh_col[j];
                        const S dx = xy.x - t.cx, dy = xy.y - t.cy;
                        S u;
                        const S p2 = neg_sigma_log2(qq, dx, dy, u);
                        const S ge = RT<S>::ex2(p2);  // exp(-sigma)
                        const S raw = mul_rn(xy.z, ge);
                        const S alpha = fmin(RT<S>::alpha_max(), raw);
                        const bool contrib = (j <= lastj) && (p2 <= S(0)) && (raw >= RT<S>::alpha_min());
                        const unsigned cm = __ballot_sync(kFull, contrib);
                        if (cm == 0u) continue;
                        const S inv1ma = RT<S>::rcp(S(1) - alpha);
                        const S Tn = T * inv1ma;  // T before this Gaussian
                        const S wgt = contrib ? alpha * Tn : S(0);
                        const S cdot = fma(col.x, g0, fma(col.y, g1, col.z * g2));
                        const S dL_dalpha = fma(Tn, cdot, -SdL * inv1ma);
                        const S gd = (contrib && raw < RT<S>::alpha_max()) ? ge * dL_dalpha : S(0);  // dL/do
                        SdL = fma(wgt, cdot, SdL);
                        T = contrib ? Tn : T;
                        const S ds = -xy.z * gd;  // dL/dsigma
                        const S dsdx = ds * dx;
                        // the sums the warp reduces; the flush turns them into the gradients:
                        // dL/dmu' = sum ds Y Delta = (a sum ds u, b sum ds u + D sum ds dy) and
                        // dL/dconic = (sum ds dx^2 / 2, sum ds dx dy, sum ds dy^2 / 2)
                        S r[kRec];
                        r[0] = ds * u;
                        r[1] = ds * dy;
                        r[2] = dsdx * dx;
                        r[3] = dsdx * dy;
                        r[4] = r[1] * dy;
                        r[5] = gd;
                        r[6] = wgt * g0;
                        r[7] = wgt * g1;
                        r[8] = wgt * g2;
                        chunk_mask |= 1u << hb;
                        // the warp's sum of each term, into the warp's own slot for this Gaussian (a
                        // lone contributing lane is not special-cased: the transpose is cheaper than its
                        // nine dependent stores)
                        const S tot = warp_sum9<S>(r, s_red[w], lane, rl);
                        if (lane < 3 * kRec && rl.part == 0) s_grad[w][j][rl.q] = tot;
                    }
                }
                if (lane == 0) s_mask[w][s >> 5] = chunk_mask;
            }
            __syncthreads();  // the walk's slots and masks are complete before the next flush reads them
            prev_b0 = b0;
            prev_n = n;
        }
        if (threadIdx.x < prev_n)  // the last walked batch (batch 0)
            flush_partial<S, kAtomic, kB>(threadIdx.x, prev_b0, s_grad, s_mask, s_fl[0][threadIdx.x], t.g_shift,
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
                              const GsRasterConfig* config, void* stream)
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
    const KF kern = table[cull][pers][n_contrib != nullptr][C != 3 || CW != 3];
    unsigned grid;
    if (int rc = raster_grid(kern, config, T_total, &grid)) return rc;
    int* queue = pers ? config->queue : nullptr;
    if (pers && cudaMemsetAsync(queue, 0, sizeof(int), s) != cudaSuccess) return launch_status(who);
    launch_pdl(kern, grid, 256, s, views, V, T_total, config ? config->tile_order : nullptr, queue,
                              reinterpret_cast<const V2<S>*>(means2d), conics, opacities, colors, isect_ids,
                              reinterpret_cast<const int2*>(tile_ranges), background, out_rgb, T_final, last_idx,
                              n_contrib, warp_hits, C, CW);
    count_launches(1);
    return launch_status(who);
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
    constexpr bool kA = std::is_same<S, float>::value;
    using KB = decltype(&k_raster_bwd<S, true, true, true, false>);
    static const KB table[2][2][2][2] = {
        {{{k_raster_bwd<S, false, false, false, false>, k_raster_bwd<S, false, false, false, kA>},
          {k_raster_bwd<S, false, false, true, false>, k_raster_bwd<S, false, false, true, kA>}},
         {{k_raster_bwd<S, false, true, false, false>, k_raster_bwd<S, false, true, false, kA>},
          {k_raster_bwd<S, false, true, true, false>, k_raster_bwd<S, false, true, true, kA>}}},
        {{{k_raster_bwd<S, true, false, false, false>, k_raster_bwd<S, true, false, false, kA>},
          {k_raster_bwd<S, true, false, true, false>, k_raster_bwd<S, true, false, true, kA>}},
         {{k_raster_bwd<S, true, true, false, false>, k_raster_bwd<S, true, true, false, kA>},
          {k_raster_bwd<S, true, true, true, false>, k_raster_bwd<S, true, true, true, kA>}}}};
    const KB kern = table[cull][!deterministic][pers][C != 3 || CW != 3];
    unsigned grid;
    if (int rc = raster_grid(kern, config, T_total, &grid)) return rc;
    int* queue = pers ? config->queue : nullptr;
    if (pers && cudaMemsetAsync(queue, 0, sizeof(int), s) != cudaSuccess) return launch_status(who);
    launch_pdl(kern, grid, 256, s, views, V, T_total, config ? config->tile_order : nullptr, queue,
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
