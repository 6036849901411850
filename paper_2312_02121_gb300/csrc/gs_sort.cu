// Tile binning and per-tile depth order (Sec. 2.2), written for sm_103a.
//
// The paper sorts (tile, depth) keys of every Gaussian-tile pair (the tile
// sort of Kerbl et al., App. C).  The same order is produced here in two
// cheaper sorts:
//   1. a stable LSD radix sort of the projections on their (positive) fp32
//      depth -- this gives (depth, p) order, ties by p.  The keys are sorted
//      relative to the smallest visible one, on the bits the spread of the
//      visible keys needs (24 of 31 at the 1080p benchmark frame: 3 passes
//      of 8 bits instead of 4);
//   2. the pairs are emitted in that order (scan of `touched` in depth order,
//      then each block's pairs are written by all its threads), and a stable
//      LSD radix sort on the global tile id alone (ceil(log2 T_total) bits,
//      e.g. 13 for one 1080p view) groups them by tile while keeping depth
//      order.
// Result: pairs ordered exactly by (tile, depth, p), as if the 64-bit
// (tile | depth) keys had been sorted stably in p order, but sorting 31 bits
// of P keys plus ~13 bits of K keys instead of ~44 bits of K keys.
//
// The radix sort is a classic three-kernel LSD pass (per-block digit
// histograms, per-digit scan across blocks, stable scatter with warp-level
// ranking and a shared-memory reorder for coalesced writes).  Item counts may
// live in device memory, so the whole pipeline is graph-capturable.
#include <algorithm>

#include "gs_common.cuh"

namespace gs {

constexpr int kRT = 256;              // threads per radix block
// Items per thread of a radix pass (a template parameter): 16 for long
// sorts, 8 for short ones, whose blocks are then small enough to fill the GPU.
constexpr int kRIShort = 8, kRILong = 16;
constexpr int kRTileMin = kRT * kRIShort;  // the smallest radix block (sizes the histogram)
constexpr int64_t kDepthLongFrom = (int64_t(1) << 22);  // projections from which the depth sort takes long blocks
constexpr int kRWarps = kRT / 32;
constexpr int kMaxBins = 256;         // digits of at most 8 bits
constexpr int kScanThreads = 1024;
constexpr int kEmitItems = 2;         // projections per thread in scan/emit (2 measured faster than 3-6)
constexpr int kEmitTile = 256 * kEmitItems;
// binary-search steps over a block's first slots
constexpr int kEmitSearch = kEmitTile <= 512 ? 9 : kEmitTile <= 1024 ? 10 : 11;
static_assert(kEmitTile <= (1 << kEmitSearch), "the emission's search covers the block");

__device__ __forceinline__ int item_count(const int32_t* count_dev, int64_t count_static, int64_t cap)
{
    int64_t c = count_dev ? (int64_t)*count_dev : count_static;
    if (c > cap) c = cap;
    return c < 0 ? 0 : (int)c;
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive scan over a 256-thread block; returns the block total in *total.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan_256(T x, T* total)
{
    __shared__ T warp_tot[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T incl = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T y = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    T before = 0, all = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const T t = warp_tot[i];
        if (i < w) before += t;
        all += t;
    }
    __syncthreads();
    if (total) *total = all;
    return before + incl - x;
}

// ---------------------------------------------------------------------------
// radix sort passes (uint32 keys, uint32 values)
// ---------------------------------------------------------------------------

// What pass `pass` of `passes` does.  With a key range krange = {smallest key,
// ~largest key} in device memory (an adaptive sort), the keys are sorted
// relative to the smallest, on the bits their spread needs, in passes of 8
// bits: the first pass subtracts the smallest key, passes past the needed ones
// do nothing, and the last needed one writes its values to the final buffer.
// At least one pass runs, so the values always come out as a permutation.
struct PassPlan {
    bool run, last;
    uint32_t sub;
};

__device__ __forceinline__ PassPlan pass_plan(const uint32_t* krange, int pass, int passes)
{
    if (!krange) return PassPlan{true, pass == passes - 1, 0u};
    const uint32_t lo = krange[0], hi = ~krange[1];
    const int need = hi > lo ? 32 - __clz(hi - lo) : 1;  // bits of the spread
    const int np = min((need + 7) / 8, passes);
    return PassPlan{pass < np, pass == np - 1, pass == 0 ? lo : 0u};
}

template <int kRI>
__global__ void __launch_bounds__(kRT)
k_radix_hist(const uint32_t* __restrict__ keys, const int32_t* __restrict__ count_dev, int64_t count_static,
             int64_t cap, int shift, int bits, uint32_t* __restrict__ hist, const uint32_t* __restrict__ krange,
             int pass, int passes)
{
    constexpr int kRTile = kRT * kRI;
    pdl_wait();
    pdl_trigger();
    const PassPlan plan = pass_plan(krange, pass, passes);
    if (!plan.run) return;
    __shared__ uint32_t h[kRWarps][kMaxBins];
    const int count = item_count(count_dev, count_static, cap);
    const int nb = (count + kRTile - 1) / kRTile;
    const int b = blockIdx.x;
    if (b >= nb) return;
    const int bins = 1 << bits;
    const unsigned mask = bins - 1;
    const int w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRWarps * kMaxBins; i += kRT) (&h[0][0])[i] = 0;
    __syncthreads();
    const int base = b * kRTile;
    // all loads first (kRI in flight per thread), then the shared-memory counts
    uint32_t key[kRI];
#pragma unroll
    for (int k = 0; k < kRI; ++k) {
        const int idx = base + k * kRT + threadIdx.x;
        key[k] = idx < count ? keys[idx] - plan.sub : 0u;
    }
#pragma unroll
    for (int k = 0; k < kRI; ++k)
        if (base + k * kRT + (int)threadIdx.x < count) atomicAdd(&h[w][(key[k] >> shift) & mask], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < bins; d += kRT) {
        uint32_t s = 0;
#pragma unroll
        for (int i = 0; i < kRWarps; ++i) s += h[i][d];
        hist[(size_t)d * nb + b] = s;
    }
}

// Exclusive scan of a row of counts by the 256 threads of a block, thread t
// taking the slice [lo, hi) of at most H counts, held in registers between the
// sum and the write-back; the row's total into *tot.
template <int H>
__device__ __forceinline__ void scan_row_held(uint32_t* __restrict__ row, int lo, int hi, uint32_t* tot)
{
    uint32_t held[H];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < H; ++i) held[i] = lo + i < hi ? row[lo + i] : 0u;
#pragma unroll
    for (int i = 0; i < H; ++i) s += held[i];
    uint32_t run = block_exclusive_scan_256<uint32_t>(s, tot);
#pragma unroll
    for (int i = 0; i < H; ++i)
        if (lo + i < hi) {
            row[lo + i] = run;
            run += held[i];
        }
}

// One block per digit: exclusive scan of that digit's per-block counts (in
// place) and the digit total.
template <int kRI>
__global__ void __launch_bounds__(kRT)
k_radix_scan_rows(uint32_t* __restrict__ hist, const int32_t* __restrict__ count_dev, int64_t count_static,
                  int64_t cap, uint32_t* __restrict__ digit_total, const uint32_t* __restrict__ krange, int pass,
                  int passes)
{
    constexpr int kRTile = kRT * kRI;
    pdl_wait();
    pdl_trigger();
    if (!pass_plan(krange, pass, passes).run) return;
    const int count = item_count(count_dev, count_static, cap);
    const int nb = (count + kRTile - 1) / kRTile;
    const int d = blockIdx.x;
    uint32_t* row = hist + (size_t)d * nb;
    const int per = (nb + kRT - 1) / kRT;
    const int lo = min(nb, (int)threadIdx.x * per), hi = min(nb, lo + per);
    uint32_t tot;
    // a thread's slice is held in registers between the sum and the write-back (all its loads in flight
    // at once) when it has at most 64 counts, i.e. up to 16384 radix blocks
    if (per <= 8) {
        scan_row_held<8>(row, lo, hi, &tot);
    } else if (per <= 64) {
        scan_row_held<64>(row, lo, hi, &tot);
    } else {
        uint32_t s = 0;
#pragma unroll 8
        for (int i = lo; i < hi; ++i) s += row[i];
        uint32_t run = block_exclusive_scan_256<uint32_t>(s, &tot);
#pragma unroll 8
        for (int i = lo; i < hi; ++i) {
            const uint32_t x = row[i];
            row[i] = run;
            run += x;
        }
    }
    if (threadIdx.x == 0) digit_total[d] = tot;
}

// Stable scatter of one block of items by digit.  vals_in == nullptr means
// "value = input position" (the first pass of a sort of indices).
template <int kRI>
__global__ void __launch_bounds__(kRT)
k_radix_scatter(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                const int32_t* __restrict__ count_dev, int64_t count_static, int64_t cap, int shift, int bits,
                const uint32_t* __restrict__ hist, const uint32_t* __restrict__ digit_total,
                const uint32_t* __restrict__ krange, int pass, int passes, uint32_t* __restrict__ vals_last)
{
    pdl_wait();
    pdl_trigger();
    const PassPlan plan = pass_plan(krange, pass, passes);
    if (!plan.run) return;
    if (plan.last && vals_last) vals_out = vals_last;
    constexpr int kRTile = kRT * kRI;
    __shared__ uint32_t s_keys[kRTile];
    __shared__ uint32_t s_vals[kRTile];
    __shared__ uint32_t s_warp[kRWarps][kMaxBins];  // per-warp digit counts, then per-warp offsets
    __shared__ uint32_t s_base[kMaxBins];           // global position of the block's first item of each digit
    __shared__ uint32_t s_local[kMaxBins];          // local position of the block's first item of each digit

    const int count = item_count(count_dev, count_static, cap);
    const int nb = (count + kRTile - 1) / kRTile;
    const int b = blockIdx.x;
    if (b >= nb) return;
    const int bins = 1 << bits;
    const unsigned mask = bins - 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int base = b * kRTile;
    const int n_here = min(kRTile, count - base);

    // every global load first, so that their latencies overlap: the block's items (warp-striped: warp w
    // owns items [w * 32 kRI, (w + 1) * 32 kRI) of the block), the digit totals and this block's count
    // of each digit
    uint32_t key[kRI], val[kRI], rank[kRI] = {};
#pragma unroll
    for (int k = 0; k < kRI; ++k) {
        const int li = w * (kRI * 32) + k * 32 + lane;
        const int idx = base + li;
        const bool valid = li < n_here;
        key[k] = valid ? keys_in[idx] - plan.sub : 0u;
        val[k] = valid ? (vals_in ? vals_in[idx] : (uint32_t)idx) : 0u;
    }
    // digit offsets: exclusive scan of digit totals + this block's row prefix
    {
        const int d = threadIdx.x;
        const uint32_t tot = d < bins ? digit_total[d] : 0u;
        const uint32_t mine = d < bins ? hist[(size_t)d * nb + b] : 0u;
        const uint32_t ex = block_exclusive_scan_256<uint32_t>(tot, nullptr);
        if (d < bins) s_base[d] = ex + mine;
    }
    for (int i = lane; i < kMaxBins; i += 32) s_warp[w][i] = 0;
    __syncwarp();

    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int k = 0; k < kRI; ++k) {
        const int li = w * (kRI * 32) + k * 32 + lane;
        const bool valid = li < n_here;
        const uint32_t d = (key[k] >> shift) & mask;
        // lanes holding the same digit, via one ballot per digit bit (__match_any_sync was measured slower)
        unsigned peers = __ballot_sync(kFull, valid);
        for (int bit = 0; bit < bits; ++bit) {
            const unsigned bal = __ballot_sync(kFull, (d >> bit) & 1u);
            peers &= ((d >> bit) & 1u) ? bal : ~bal;
        }
        uint32_t before = 0;
        if (valid) before = s_warp[w][d];
        __syncwarp();
        if (valid) {
            rank[k] = before + __popc(peers & lt);
            if ((peers & lt) == 0) s_warp[w][d] = before + __popc(peers);  // lowest peer updates
        }
        __syncwarp();
    }
    __syncthreads();
    // per-digit: offsets of each warp inside the block, and block totals
    {
        const int d = threadIdx.x;
        uint32_t run = 0;
        if (d < bins) {
#pragma unroll
            for (int i = 0; i < kRWarps; ++i) {
                const uint32_t c = s_warp[i][d];
                s_warp[i][d] = run;
                run += c;
            }
        }
        const uint32_t ex = block_exclusive_scan_256<uint32_t>(d < bins ? run : 0u, nullptr);
        if (d < bins) s_local[d] = ex;
    }
    __syncthreads();
    // reorder the block in shared memory by digit (stable)
#pragma unroll
    for (int k = 0; k < kRI; ++k) {
        const int li = w * (kRI * 32) + k * 32 + lane;
        if (li < n_here) {
            const uint32_t d = (key[k] >> shift) & mask;
            const uint32_t lp = s_local[d] + s_warp[w][d] + rank[k];
            s_keys[lp] = key[k];
            s_vals[lp] = val[k];
        }
    }
    __syncthreads();
    // coalesced write-out: consecutive items of a digit go to consecutive positions
    for (int j = threadIdx.x; j < n_here; j += kRT) {
        const uint32_t k2 = s_keys[j];
        const uint32_t d = (k2 >> shift) & mask;
        const uint32_t gp = s_base[d] + (uint32_t)j - s_local[d];
        keys_out[gp] = k2;
        vals_out[gp] = s_vals[j];
    }
}

struct RadixBufs {
    uint32_t* hist;
    uint32_t* digit_total;
};

// Stable LSD sort of (key, value) pairs on key bits [0, total_bits), in
// passes of at most 8 bits.  Keys ping-pong between k1 and k2, values between
// v1 and v2; the values start as vals0, or as the input positions when vals0
// is null.  The item count is *count_dev (device, clamped to cap) or
// count_static.  The last pass writes its values to vals_last when that is
// given.  With krange (device {smallest key, ~largest key}) the sort is
// adaptive (see pass_plan): it needs vals_last, which then always receives
// the values.  Returns the buffers holding the result (for an adaptive sort
// only the values: the keys are left relative and in either buffer).
template <int kRI>
static void lsd_sort(uint32_t* k1, uint32_t* k2, uint32_t* v1, uint32_t* v2, const uint32_t* vals0,
                     const int32_t* count_dev, int64_t count_static, int64_t cap, int total_bits,
                     const RadixBufs& rb, cudaStream_t s, uint32_t** keys_out, uint32_t** vals_out,
                     uint32_t* vals_last = nullptr, const uint32_t* krange = nullptr)
{
    constexpr int kRTile = kRT * kRI;
    uint32_t *kin = k1, *kout = k2, *vout = v1;
    const uint32_t* vin = vals0;
    if (total_bits > 0 && cap > 0) {
        const int passes = (total_bits + 7) / 8;
        const int per = (total_bits + passes - 1) / passes;
        const unsigned grid = (unsigned)((cap + kRTile - 1) / kRTile);
        for (int pass = 0, shift = 0; pass < passes; ++pass, shift += per) {
            const int bits = std::min(per, total_bits - shift);
            // the device picks vals_last for the last pass that runs (the host's last one when not adaptive)
            launch_pdl(k_radix_hist<kRI>, grid, kRT, s, kin, count_dev, count_static, cap, shift, bits, rb.hist, krange,
                       pass, passes);
            launch_pdl(k_radix_scan_rows<kRI>, 1u << bits, kRT, s, rb.hist, count_dev, count_static, cap,
                       rb.digit_total, krange, pass, passes);
            launch_pdl(k_radix_scatter<kRI>, grid, kRT, s, kin, vin, kout, vout, count_dev, count_static, cap, shift,
                       bits, rb.hist, rb.digit_total, krange, pass, passes, vals_last);
            count_launches(3);
            std::swap(kin, kout);
            vin = (vals_last && pass == passes - 1) ? vals_last : vout;
            vout = (vout == v1) ? v2 : v1;
        }
    }
    *keys_out = kin;
    *vals_out = const_cast<uint32_t*>(krange ? vals_last : vin);  // vals0 itself when no pass ran
}

// ---------------------------------------------------------------------------
// binning kernels
// ---------------------------------------------------------------------------

// Depth keys: the fp32 bit pattern of t_z (> near > 0, so monotone in 31
// bits); culled projections get the largest key.  The smallest key and the
// complement of the largest one over the visible projections go to krange
// (both by atomicMin, one pair per block of kKeyItems x 256 keys; the caller
// sets both words to ~0 first): the depth sort then sorts only the bits their
// spread needs.  A culled projection's key may fall outside that range; its
// place in the order does not matter, as it has no pairs.
//
// The blocks also zero tile_ranges (T entries): the finalization writes only
// the ranges of tiles that have pairs, and this is the call's first kernel.
constexpr int kKeyItems = 8;
__global__ void __launch_bounds__(256)
k_depth_keys(int64_t P, const float* __restrict__ depths, const int32_t* __restrict__ touched,
             uint32_t* __restrict__ keys, uint32_t* __restrict__ krange, int2* __restrict__ tile_ranges, int32_t T)
{
    pdl_wait();
    pdl_trigger();
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < T; i += (int64_t)gridDim.x * 256)
        tile_ranges[i] = make_int2(0, 0);
    __shared__ uint32_t s_lo[8], s_hi[8];
    uint32_t lo = 0xffffffffu, hi_c = 0xffffffffu;
    const int64_t base = (int64_t)blockIdx.x * (256 * kKeyItems) + threadIdx.x;
    // both loads of every item first (the depth unconditionally), so that no load waits for another
    int32_t tc[kKeyItems];
    float dz[kKeyItems];
#pragma unroll
    for (int k = 0; k < kKeyItems; ++k) {
        const int64_t p = base + k * 256;
        tc[k] = p < P ? touched[p] : 0;
        dz[k] = p < P ? depths[p] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < kKeyItems; ++k) {
        const int64_t p = base + k * 256;
        if (p < P) {
            const bool vis = tc[k] > 0;
            const uint32_t key = vis ? __float_as_uint(dz[k]) : 0x7fffffffu;
            keys[p] = key;
            if (vis) {
                lo = min(lo, key);
                hi_c = min(hi_c, ~key);
            }
        }
    }
    lo = __reduce_min_sync(kFull, lo);
    hi_c = __reduce_min_sync(kFull, hi_c);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        s_lo[w] = lo;
        s_hi[w] = hi_c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < 8; ++i) {
            lo = min(lo, s_lo[i]);
            hi_c = min(hi_c, s_hi[i]);
        }
        if (lo != 0xffffffffu) {
            atomicMin(krange, lo);
            atomicMin(krange + 1, hi_c);
        }
    }
}

// Per block of kEmitTile projections in depth order: sum of touched.  The
// counts are also stored in depth order (cnt_sorted[r] = touched[order[r]]),
// so that the emission reads them contiguously instead of gathering again.
__global__ void __launch_bounds__(256)
k_touched_block_sums(int64_t P, const uint32_t* __restrict__ order, const int32_t* __restrict__ touched,
                     int64_t* __restrict__ block_sums, int32_t* __restrict__ cnt_sorted)
{
    pdl_wait();
    pdl_trigger();
    const int64_t base = (int64_t)blockIdx.x * kEmitTile;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kEmitItems; ++k) {
        const int64_t r = base + k * 256 + threadIdx.x;
        if (r < P) {
            const int32_t c = touched[order[r]];
            cnt_sorted[r] = c;
            s += c;
        }
    }
    int64_t tot;
    block_exclusive_scan_256<int64_t>(s, &tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// Single block: exclusive scan of the block sums in place; K and the
// capacity flag.
__global__ void __launch_bounds__(kScanThreads)
k_scan_block_sums(int64_t nblk, int64_t* __restrict__ block_sums, int64_t cap, int32_t* __restrict__ K_out,
                  uint32_t* __restrict__ flags)
{
    pdl_wait();
    pdl_trigger();
    __shared__ int64_t warp_tot[kScanThreads / 32];
    const int64_t per = (nblk + kScanThreads - 1) / kScanThreads;
    const int64_t lo = min(nblk, (int64_t)threadIdx.x * per), hi = min(nblk, lo + per);
    int64_t s = 0;
#pragma unroll 8
    for (int64_t i = lo; i < hi; ++i) s += block_sums[i];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t incl = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t y = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    int64_t before = 0, all = 0;
    for (int i = 0; i < kScanThreads / 32; ++i) {
        if (i < w) before += warp_tot[i];
        all += warp_tot[i];
    }
    int64_t run = before + incl - s;
#pragma unroll 8
    for (int64_t i = lo; i < hi; ++i) {
        const int64_t x = block_sums[i];
        block_sums[i] = run;
        run += x;
    }
    if (threadIdx.x == 0) {
        *K_out = (int32_t)min(all, (int64_t)INT32_MAX);
        if (all > cap) atomicOr(flags, GS_FLAG_CAPACITY);
    }
}

// Emission of the (tile, projection) pairs in depth order: pair j of the
// projection at depth rank r gets emission index off[r] + j; its key is the
// global tile id (row-major inside the rectangle), its owner the projection.
// A block takes kEmitTile consecutive ranks and scans their pair counts into
// shared memory.  Its threads then write the block's slots round-robin, each
// finding the slot's owner by a ten-step binary search over the block's first
// slots -- so the stores are contiguous and the work is spread over the block
// whatever the rectangle sizes.
//
// kOwnPrefix: block_prefix holds each block's total (not yet scanned), and
// every block sums its predecessors' itself (at most kEmitOwnPrefixMax blocks,
// so at most that many loads per block); the last block writes K and the
// capacity flag.  This saves the single-block scan launch.
constexpr int64_t kEmitOwnPrefixMax = 4096;
template <bool kOwnPrefix>
__global__ void __launch_bounds__(256)
k_emit(const GsView* __restrict__ views, int V, int64_t P, const uint32_t* __restrict__ order,
       const int32_t* __restrict__ cnt_sorted, const short4* __restrict__ rects, const int64_t* __restrict__ block_prefix,
       int64_t cap, uint32_t* __restrict__ tile_keys, uint32_t* __restrict__ owner, int32_t* __restrict__ emit_start,
       int32_t* __restrict__ K_out, uint32_t* __restrict__ flags)
{
    pdl_wait();
    pdl_trigger();
    __shared__ int s_off[kEmitTile + 1];  // block-local first slot of each rank
    __shared__ uint32_t s_p[kEmitTile];
    __shared__ int s_x0[kEmitTile], s_w[kEmitTile];
    __shared__ int s_row0[kEmitTile];      // tile id of the rectangle's first row start (x = 0)
    __shared__ int s_tx[kEmitTile];        // tiles_x of the projection's view
    __shared__ float s_iw[kEmitTile];      // 1 / rectangle width
    const int64_t base = (int64_t)blockIdx.x * kEmitTile;
    int64_t gbase;
    if (kOwnPrefix) {
        int64_t part = 0;
        for (int b = threadIdx.x; b < (int)blockIdx.x; b += 256) part += block_prefix[b];
        block_exclusive_scan_256<int64_t>(part, &gbase);
    } else {
        gbase = block_prefix[blockIdx.x];
    }
    int cnt[kEmitItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kEmitItems; ++k) {
        const int li = threadIdx.x * kEmitItems + k;
        const int64_t r = base + li;
        uint32_t p = 0u;
        cnt[k] = 0;
        if (r < P) {
            p = order[r];
            cnt[k] = cnt_sorted[r];
            if (cnt[k] > 0) {
                const GsView& view = views[view_of_projection(views, V, (int64_t)p)];
                const short4 rc = rects[p];
                s_x0[li] = rc.x;
                s_w[li] = rc.z - rc.x;
                s_iw[li] = 1.f / (float)(rc.z - rc.x);
                s_row0[li] = view.tile_offset + rc.y * view.tiles_x;
                s_tx[li] = view.tiles_x;
            }
        }
        s_p[li] = p;
        s += cnt[k];
    }
    int total;
    int off = block_exclusive_scan_256<int>(s, &total);
#pragma unroll
    for (int k = 0; k < kEmitItems; ++k) {
        const int li = threadIdx.x * kEmitItems + k;
        s_off[li] = off;
        if (emit_start && cnt[k] > 0) emit_start[s_p[li]] = (int32_t)min(gbase + off, (int64_t)INT32_MAX);
        off += cnt[k];
    }
    if (threadIdx.x == 0) s_off[kEmitTile] = total;
    if (kOwnPrefix && threadIdx.x == 0 && blockIdx.x == gridDim.x - 1) {
        const int64_t all = gbase + total;
        *K_out = (int32_t)min(all, (int64_t)INT32_MAX);
        if (all > cap) atomicOr(flags, GS_FLAG_CAPACITY);
    }
    __syncthreads();
    // the block's slots go round-robin over all its threads (consecutive threads, consecutive slots),
    // so that a projection with thousands of tiles is shared by the block instead of one warp
#pragma unroll 1
    for (int e = threadIdx.x; e < total; e += 256) {
        const int64_t ge = gbase + e;
        if (ge >= cap) break;
        // the last rank whose first slot is <= e (ranks with no pairs share it with the next one; the last
        // of them owns the slot): s_off[lo] <= e < s_off[hi] throughout
        int lo = 0, hi = kEmitTile;
#pragma unroll
        for (int step = 0; step < kEmitSearch; ++step) {  // 2^kEmitSearch >= kEmitTile
            const int mid = (lo + hi) >> 1;
            if (s_off[mid] <= e) lo = mid; else hi = mid;
        }
        const int r = lo;
        const int j = e - s_off[r];
        const int w = s_w[r];
        // j / w through the reciprocal: the estimate is within one of the quotient (j / w is at most the
        // rectangle height, < 2^15), and the two integer checks make it exact
        int dy = (int)((float)j * s_iw[r]);
        dy -= dy * w > j;
        dy += (dy + 1) * w <= j;
        tile_keys[ge] = (uint32_t)(s_row0[r] + dy * s_tx[r] + s_x0[r] + (j - dy * w));
        owner[ge] = s_p[r];
    }
}

// Sorted pairs -> projection ids, inverse positions and per-tile ranges.  The
// sorted values are emission indices when isect_pos is wanted (their owners
// are gathered and the inverse permutation is scattered), else the owners
// themselves, which the last radix pass already wrote into isect_ids.  Each
// thread takes kFinItems consecutive pairs (16-byte loads of their keys, all
// issued before any is used).
constexpr int kFinItems = 16;
__global__ void k_finalize(const int32_t* __restrict__ K_dev, int64_t cap, const uint32_t* __restrict__ keys,
                           const uint32_t* __restrict__ vals, const uint32_t* __restrict__ owner,
                           int32_t* __restrict__ isect_ids, int32_t* __restrict__ isect_pos,
                           int2* __restrict__ tile_ranges)
{
    pdl_wait();
    pdl_trigger();
    const int K = item_count(K_dev, 0, cap);
    const int i0 = kFinItems * (blockIdx.x * blockDim.x + threadIdx.x);
    if (i0 >= K) return;
    const int n = min(kFinItems, K - i0);
    uint32_t t[kFinItems];
    if (n == kFinItems) {  // keys comes from the workspace (16-byte aligned) and i0 is a multiple of 4
#pragma unroll
        for (int q = 0; q < kFinItems / 4; ++q) {
            const uint4 v = reinterpret_cast<const uint4*>(keys + i0)[q];
            t[4 * q + 0] = v.x;
            t[4 * q + 1] = v.y;
            t[4 * q + 2] = v.z;
            t[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kFinItems; ++k) t[k] = k < n ? keys[i0 + k] : 0u;
    }
    // tile ids are below 2^31, so ~0 marks "no neighbour"
    uint32_t prev = i0 > 0 ? keys[i0 - 1] : ~0u;
    const uint32_t next = i0 + n < K ? keys[i0 + n] : ~0u;
#pragma unroll
    for (int k = 0; k < kFinItems; ++k) {
        if (k >= n) break;
        const int i = i0 + k;
        if (isect_pos) {
            const uint32_t e = vals[i];
            isect_ids[i] = (int32_t)owner[e];
            isect_pos[e] = i;
        } else if (vals != reinterpret_cast<const uint32_t*>(isect_ids)) {
            isect_ids[i] = (int32_t)vals[i];  // only when no pass ran (a single tile: zero key bits)
        }
        const uint32_t cur = t[k];
        const uint32_t nx = k + 1 < n ? t[k + 1] : next;
        if (cur != prev) tile_ranges[cur].x = i;
        if (nx != cur) tile_ranges[cur].y = i + 1;
        prev = cur;
    }
}

// Longest-first key of each tile: 65535 - min(list length, 65535).
__global__ void k_tile_len_keys(int32_t T, const int2* __restrict__ tile_ranges, uint32_t* __restrict__ keys)
{
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < T) {
        const int2 r = tile_ranges[i];
        keys[i] = 65535u - (uint32_t)min(max(r.y - r.x, 0), 65535);
    }
}

// The same order for up to kOrderRankMax tiles in one launch, by counting: a
// tile's key packs its length key above its id (unique keys, so the order is
// the rank of each key among all of them, ties by id included), and each group
// of kOrderSplit threads counts the keys below its tile's over interleaved
// quads of the whole key array, staged in shared memory by every CTA.  O(T^2)
// compares, spread over ceil(T / 64) CTAs of 1024 threads; larger batches take
// the radix sort.
constexpr int kOrderRankMax = 12288;
constexpr int kOrderSplit = 16;
constexpr int kOrderThreads = 1024;

__device__ __forceinline__ uint32_t order_key(int2 r, int t)
{
    return ((65535u - (uint32_t)min(max(r.y - r.x, 0), 65535)) << 16) | (uint32_t)t;
}

__global__ void __launch_bounds__(kOrderThreads)
k_tile_order_rank(int32_t T, const int2* __restrict__ tile_ranges, int32_t* __restrict__ order)
{
    extern __shared__ uint4 s_keys4[];
    uint32_t* s_key = reinterpret_cast<uint32_t*>(s_keys4);
    pdl_wait();
    pdl_trigger();
    const int n4 = (T + 3) & ~3;  // padded with keys above every real one (ids < 2^14)
#pragma unroll 4
    for (int i = threadIdx.x; i < n4; i += kOrderThreads) s_key[i] = i < T ? order_key(tile_ranges[i], i) : ~0u;
    __syncthreads();
    const int sub = threadIdx.x % kOrderSplit;
    const int t = blockIdx.x * (kOrderThreads / kOrderSplit) + threadIdx.x / kOrderSplit;
    const uint32_t mine = t < T ? s_key[t] : 0u;
    // the 16 threads of a group read 16 consecutive quads; the warp's two groups the same ones
    int c0 = 0, c1 = 0, c2 = 0, c3 = 0;
#pragma unroll 4
    for (int i = sub; i < n4 / 4; i += kOrderSplit) {
        const uint4 k = s_keys4[i];
        c0 += k.x < mine;
        c1 += k.y < mine;
        c2 += k.z < mine;
        c3 += k.w < mine;
    }
    int c = (c0 + c1) + (c2 + c3);
#pragma unroll
    for (int d = 1; d < kOrderSplit; d <<= 1) c += __shfl_xor_sync(kFull, c, d);
    if (sub == 0 && t < T) order[c] = t;
}

__global__ void k_copy_u32(int32_t n, const uint32_t* __restrict__ src, int32_t* __restrict__ dst)
{
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (int32_t)src[i];
}

struct OrderLayout {
    uint32_t *ka, *kb, *va, *vb, *hist, *digit_total;
    size_t bytes;
};

static OrderLayout carve_order(void* ws, int64_t T)
{
    Carver c(ws);
    OrderLayout L;
    L.ka = c.take<uint32_t>(T);
    L.kb = c.take<uint32_t>(T);
    L.va = c.take<uint32_t>(T);
    L.vb = c.take<uint32_t>(T);
    L.hist = c.take<uint32_t>((size_t)((T + kRTileMin - 1) / kRTileMin) * kMaxBins + 1);
    L.digit_total = c.take<uint32_t>(kMaxBins);
    L.bytes = c.used;
    return L;
}

struct SortLayout {
    uint32_t *dkey_a, *dkey_b, *dval_a, *dval_b, *order, *krange;
    int32_t* cnt_sorted;
    int64_t* block_sums;
    uint32_t *tkey_a, *tkey_b, *tval_a, *tval_b, *owner;
    uint32_t *hist, *digit_total;
    size_t bytes;
};

static SortLayout carve(void* ws, int64_t P, int64_t cap)
{
    Carver c(ws);
    SortLayout L;
    L.dkey_a = c.take<uint32_t>(P);
    L.dkey_b = c.take<uint32_t>(P);
    L.dval_a = c.take<uint32_t>(P);
    L.dval_b = c.take<uint32_t>(P);
    L.order = c.take<uint32_t>(P);
    L.krange = c.take<uint32_t>(2);
    L.cnt_sorted = c.take<int32_t>(P);
    L.block_sums = c.take<int64_t>((P + kEmitTile - 1) / kEmitTile + 1);
    L.tkey_a = c.take<uint32_t>(cap);
    L.tkey_b = c.take<uint32_t>(cap);
    L.tval_a = c.take<uint32_t>(cap);
    L.tval_b = c.take<uint32_t>(cap);
    L.owner = c.take<uint32_t>(cap);
    // radix blocks of the depth sort (short blocks) and of the tile sort (long blocks)
    const int64_t nb = std::max((P + kRTileMin - 1) / kRTileMin, (cap + kRT * kRILong - 1) / (kRT * kRILong));
    L.hist = c.take<uint32_t>((size_t)nb * kMaxBins + 1);
    L.digit_total = c.take<uint32_t>(kMaxBins);
    L.bytes = c.used;
    return L;
}

static int bit_length(int64_t x)
{
    int b = 0;
    while (x > 0) { ++b; x >>= 1; }
    return b;
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_bin_and_sort_workspace_size(int64_t P, int64_t K_capacity, int32_t T_total)
{
    (void)T_total;
    if (P < 0 || K_capacity < 0) return 0;
    return carve(nullptr, P, K_capacity).bytes;
}

namespace gs {

// The host checks of the binning arguments other than the workspace, shared by
// gs_bin_and_sort and gs_bin_and_sort_static (`who` names the entry point in
// the message).  Nothing is read through the pointers.
int bin_and_sort_check_args(const char* who, const GsView* views, int32_t V, int64_t P, int32_t T_total,
                            const int16_t* rects, const float* depths, const int32_t* touched, int64_t K_capacity,
                            const int32_t* isect_ids, const int32_t* isect_pos, const int32_t* emit_start,
                            const int32_t* tile_ranges, const int32_t* K_out, const uint32_t* flags)
{
    if (V <= 0 || P < 0 || T_total <= 0 || K_capacity < 0 || P >= (int64_t(1) << 31) ||
        K_capacity >= (int64_t(1) << 31))
        return fail(GS_ERR_INVALID_ARG, "%s: V=%d P=%lld T_total=%d K_capacity=%lld", who, V, (long long)P, T_total,
                    (long long)K_capacity);
    if (!views || !tile_ranges || !K_out || !flags || (P > 0 && (!rects || !depths || !touched)) ||
        (K_capacity > 0 && !isect_ids) || (isect_pos && !emit_start))
        return fail(GS_ERR_INVALID_ARG, "%s: null pointer argument", who);
    if ((reinterpret_cast<uintptr_t>(rects) & 7) || (reinterpret_cast<uintptr_t>(tile_ranges) & 7))
        return fail(GS_ERR_INVALID_ARG, "%s: rects and tile_ranges need 8-byte alignment", who);
    return GS_OK;
}

}  // namespace gs

extern "C" int gs_bin_and_sort(const GsView* views, int32_t V, int64_t P, int32_t T_total, const int16_t* rects,
                               const float* depths, const int32_t* touched, int64_t K_capacity, void* workspace,
                               size_t workspace_bytes, int32_t* isect_ids, int32_t* isect_pos, int32_t* emit_start,
                               int32_t* tile_ranges, int32_t* K_out, uint32_t* flags, void* stream)
{
    gs::NvtxRange nvtx("gs_bin_and_sort");
    const int checked = gs::bin_and_sort_check_args("gs_bin_and_sort", views, V, P, T_total, rects, depths, touched,
                                                    K_capacity, isect_ids, isect_pos, emit_start, tile_ranges, K_out,
                                                    flags);
    if (checked != GS_OK) return checked;
    const SortLayout need = carve(nullptr, P, K_capacity);
    if (!workspace || workspace_bytes < need.bytes)
        return fail(GS_ERR_INVALID_ARG, "gs_bin_and_sort: workspace of %zu bytes, need %zu", workspace_bytes,
                    need.bytes);
    if (reinterpret_cast<uintptr_t>(workspace) & 15)
        return fail(GS_ERR_INVALID_ARG, "gs_bin_and_sort: workspace needs 16-byte alignment");
    cudaStream_t s = as_stream(stream);
    const SortLayout L = carve(workspace, P, K_capacity);
    if (P == 0) {
        if (cudaMemsetAsync(tile_ranges, 0, sizeof(int32_t) * 2 * (size_t)T_total, s) != cudaSuccess ||
            cudaMemsetAsync(K_out, 0, sizeof(int32_t), s) != cudaSuccess)
            return launch_status("gs_bin_and_sort memset");
        return launch_status("gs_bin_and_sort");
    }
    // otherwise k_depth_keys zeroes tile_ranges, and the emission (or the block-sum scan) writes K_out
    const RadixBufs rb{L.hist, L.digit_total};

    // 1. projections in (depth, p) order: an adaptive sort on the spread of the visible depth keys
    if (cudaMemsetAsync(L.krange, 0xff, 2 * sizeof(uint32_t), s) != cudaSuccess)
        return launch_status("gs_bin_and_sort memset");
    launch_pdl(k_depth_keys, (unsigned)((P + 256 * kKeyItems - 1) / (256 * kKeyItems)), 256, s, P, depths, touched,
               L.dkey_a, L.krange, reinterpret_cast<int2*>(tile_ranges), T_total);
    count_launches(1);
    uint32_t *dk, *order;
    // short radix blocks fill the GPU for a frame's million projections; long ones write longer runs of
    // each digit (and scan fewer blocks) once there are millions of blocks' worth
    if (P >= kDepthLongFrom)
        lsd_sort<kRILong>(L.dkey_a, L.dkey_b, L.dval_a, L.dval_b, nullptr, nullptr, P, P, 31, rb, s, &dk, &order,
                          L.order, L.krange);
    else
        lsd_sort<kRIShort>(L.dkey_a, L.dkey_b, L.dval_a, L.dval_b, nullptr, nullptr, P, P, 31, rb, s, &dk, &order,
                           L.order, L.krange);

    // 2. scan of touched in depth order, K, emission
    const int64_t nblk = (P + kEmitTile - 1) / kEmitTile;
    launch_pdl(k_touched_block_sums, (unsigned)nblk, 256, s, P, order, touched, L.block_sums, L.cnt_sorted);
    if (nblk <= kEmitOwnPrefixMax) {
        launch_pdl(k_emit<true>, (unsigned)nblk, 256, s, views, V, P, order, L.cnt_sorted,
                   reinterpret_cast<const short4*>(rects), L.block_sums, K_capacity, L.tkey_a, L.owner, emit_start,
                   K_out, flags);
        count_launches(2);
    } else {
        launch_pdl(k_scan_block_sums, 1, kScanThreads, s, nblk, L.block_sums, K_capacity, K_out, flags);
        launch_pdl(k_emit<false>, (unsigned)nblk, 256, s, views, V, P, order, L.cnt_sorted,
                   reinterpret_cast<const short4*>(rects), L.block_sums, K_capacity, L.tkey_a, L.owner, emit_start,
                   K_out, flags);
        count_launches(3);
    }
    if (K_capacity == 0) return launch_status("gs_bin_and_sort");

    // 3. stable sort of the pairs by global tile id; the values are the emission indices when the
    //    inverse positions are wanted, else directly the owning projections
    //    (in the latter case the last pass writes them straight into isect_ids)
    uint32_t *tk, *tv;
    lsd_sort<kRILong>(L.tkey_a, L.tkey_b, L.tval_a, L.tval_b, isect_pos ? nullptr : L.owner, K_out, 0, K_capacity,
                      bit_length((int64_t)T_total - 1), rb, s, &tk, &tv,
                      isect_pos ? nullptr : reinterpret_cast<uint32_t*>(isect_ids));
    // 4. projection ids, inverse positions, tile ranges
    launch_pdl(k_finalize, (unsigned)((K_capacity + 256 * kFinItems - 1) / (256 * kFinItems)), 256, s, K_out, K_capacity, tk, tv, L.owner,
               isect_ids, isect_pos, reinterpret_cast<int2*>(tile_ranges));
    count_launches(1);
    return launch_status("gs_bin_and_sort");
}

extern "C" size_t gs_tile_order_workspace_size(int32_t T_total)
{
    return T_total < 0 ? 0 : carve_order(nullptr, T_total).bytes;
}

extern "C" int gs_tile_order(const int32_t* tile_ranges, int32_t T_total, void* workspace, size_t workspace_bytes,
                             int32_t* order, void* stream)
{
    gs::NvtxRange nvtx("gs_tile_order");
    if (T_total < 0) return fail(GS_ERR_INVALID_ARG, "gs_tile_order: T_total=%d", T_total);
    if (T_total == 0) return GS_OK;
    if (!tile_ranges || !order || (reinterpret_cast<uintptr_t>(tile_ranges) & 7))
        return fail(GS_ERR_INVALID_ARG, "gs_tile_order: null or misaligned pointer argument");
    const OrderLayout need = carve_order(nullptr, T_total);
    if (!workspace || workspace_bytes < need.bytes)
        return fail(GS_ERR_INVALID_ARG, "gs_tile_order: workspace of %zu bytes, need %zu", workspace_bytes,
                    need.bytes);
    cudaStream_t s = as_stream(stream);
    if (T_total <= kOrderRankMax) {
        const size_t smem = sizeof(uint32_t) * (size_t)((T_total + 3) & ~3);  // at most 48 KB: no opt-in
        launch_pdl_smem(k_tile_order_rank, (unsigned)((T_total + kOrderThreads / kOrderSplit - 1) /
                                                      (kOrderThreads / kOrderSplit)),
                        kOrderThreads, smem, s, T_total, reinterpret_cast<const int2*>(tile_ranges), order);
        count_launches(1);
        return launch_status("gs_tile_order");
    }
    const OrderLayout L = carve_order(workspace, T_total);
    const unsigned g = (unsigned)((T_total + 255) / 256);
    launch_pdl(k_tile_len_keys, g, 256, s, T_total, reinterpret_cast<const int2*>(tile_ranges), L.ka);
    uint32_t *k, *v;
    lsd_sort<kRIShort>(L.ka, L.kb, L.va, L.vb, nullptr, nullptr, T_total, T_total, 16, RadixBufs{L.hist, L.digit_total}, s, &k,
             &v);
    launch_pdl(k_copy_u32, g, 256, s, T_total, v, order);
    count_launches(2);
    return launch_status("gs_tile_order");
}
