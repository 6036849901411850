// gs_autotune: picks the tile walk and the backward's batch shape for a frame
// by timing the compositing forward and backward (Sec. 2.2 Eq. 7, Sec. 3.1) of
// every candidate on the caller's stream, in scratch the caller provides.
// None of the candidates changes any result (beyond the fp32 order of the
// fast backward's atomics), so the choice is purely a matter of speed.  The
// tile size is not a candidate: it is part of the method's result (a
// Gaussian is composited in every pixel of every tile its 3-sigma box
// touches, Sec. 2.2), not a free parameter.
#include <algorithm>
#include <vector>

#include "gs_common.cuh"

namespace gs {

// The built-in candidates: five tile walks x four backward batch shapes.
static const GsTuning kWalks[] = {
    {0, 0, 0, 0, 0, 0.f},  // one CTA per tile, tile id order
    {0, 0, 1, 0, 0, 0.f},  // one CTA per tile, longest list first
    {1, 0, 1, 0, 0, 0.f},  // persistent grid (as many CTAs as fit), longest first
    {1, 4, 1, 0, 0, 0.f},  // persistent grid of 4 CTAs per SM, longest first
    {1, 3, 1, 0, 0, 0.f},  // persistent grid of 3 CTAs per SM, longest first
};
static const int kShapes[][2] = {{1, 96}, {2, 64}, {2, 128}, {1, 64}};
constexpr int kNumDefault = 5 * 4;

struct TuneLayout {
    float *rgb, *T_final, *dL, *g2, *gc, *go, *gcol;
    int32_t *last, *order, *queue;
    uint32_t* hits;
    void* order_ws;
    size_t order_ws_bytes, bytes;
};

static TuneLayout carve_tune(void* ws, int64_t P, int64_t N, int32_t T, int64_t K_capacity, int64_t pix)
{
    Carver c(ws);
    TuneLayout L;
    L.rgb = c.take<float>(3 * pix);
    L.T_final = c.take<float>(pix);
    L.last = c.take<int32_t>(pix);
    L.dL = c.take<float>(3 * pix);
    L.g2 = c.take<float>(2 * P);
    L.gc = c.take<float>(3 * P);
    L.go = c.take<float>(N);
    L.gcol = c.take<float>(3 * N);
    L.order = c.take<int32_t>(T);
    L.queue = c.take<int32_t>(1);
    L.hits = c.take<uint32_t>(K_capacity);
    L.order_ws_bytes = gs_tile_order_workspace_size(T);
    L.order_ws = c.take<unsigned char>(L.order_ws_bytes);
    L.bytes = c.used;
    return L;
}

// Events for one timed interval, destroyed on every path out.
struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

}  // namespace gs

using namespace gs;

extern "C" int gs_autotune_default_candidates(GsTuning* out, int32_t capacity, int32_t* count)
{
    if (!count || capacity < 0 || (capacity > 0 && !out))
        return fail(GS_ERR_INVALID_ARG, "gs_autotune_default_candidates: null pointer or negative capacity");
    int n = 0;
    for (const GsTuning& w : kWalks)
        for (const auto& sh : kShapes) {
            if (n < capacity) {
                GsTuning t = w;
                t.bwd_pixels = sh[0];
                t.bwd_batch = sh[1];
                out[n] = t;
            }
            ++n;
        }
    *count = n;
    return GS_OK;
}

extern "C" size_t gs_autotune_workspace_size(int64_t P, int64_t N, int32_t T_total, int64_t K_capacity,
                                             int64_t pixels)
{
    if (P < 0 || N < 0 || T_total < 0 || K_capacity < 0 || pixels < 0) return 0;
    return carve_tune(nullptr, P, N, T_total, K_capacity, pixels).bytes;
}

extern "C" int gs_autotune(const GsView* views, int32_t V, int64_t P, int64_t N, int32_t T_total, int64_t pixels,
                           const float* means2d, const float* conics, const float* opacities, const float* colors,
                           const int32_t* isect_ids, const int32_t* tile_ranges, const int32_t* K, int64_t K_capacity,
                           const GsTuning* candidates, int32_t n_candidates, int32_t repeats, void* workspace,
                           size_t workspace_bytes, GsTuning* results, GsTuning* best, void* stream)
{
    gs::NvtxRange nvtx("gs_autotune");
    const char* who = "gs_autotune";
    if (V <= 0 || P < 0 || N < 0 || T_total <= 0 || pixels <= 0 || K_capacity < 0 || n_candidates < 0 ||
        repeats < 1 || repeats > 1000)
        return fail(GS_ERR_INVALID_ARG, "%s: V=%d P=%lld N=%lld T_total=%d pixels=%lld K_capacity=%lld "
                    "n_candidates=%d repeats=%d", who, V, (long long)P, (long long)N, T_total, (long long)pixels,
                    (long long)K_capacity, n_candidates, repeats);
    if (!views || !means2d || !conics || !opacities || !colors || !isect_ids || !tile_ranges || !K || !best ||
        (n_candidates > 0 && !candidates))
        return fail(GS_ERR_INVALID_ARG, "%s: null pointer argument", who);
    const TuneLayout need = carve_tune(nullptr, P, N, T_total, K_capacity, pixels);
    if (!workspace || workspace_bytes < need.bytes)
        return fail(GS_ERR_INVALID_ARG, "%s: workspace of %zu bytes, need %zu", who, workspace_bytes, need.bytes);
    if (reinterpret_cast<uintptr_t>(workspace) & 15)
        return fail(GS_ERR_INVALID_ARG, "%s: workspace needs 16-byte alignment", who);
    std::vector<GsTuning> cands;
    if (n_candidates > 0) {
        cands.assign(candidates, candidates + n_candidates);
    } else {
        int32_t n = 0;
        cands.resize(kNumDefault);
        gs_autotune_default_candidates(cands.data(), kNumDefault, &n);
    }
    cudaStream_t s = as_stream(stream);
    const TuneLayout L = carve_tune(workspace, P, N, T_total, K_capacity, pixels);
    // dL/dC = 0: the backward's work depends on the forward's state only (which pairs composite), so
    // its time is that of any other dL/dC, and the accumulated outputs stay finite
    if (cudaMemsetAsync(L.dL, 0, sizeof(float) * 3 * (size_t)pixels, s) != cudaSuccess ||
        cudaMemsetAsync(L.g2, 0, sizeof(float) * 2 * (size_t)P, s) != cudaSuccess ||
        cudaMemsetAsync(L.gc, 0, sizeof(float) * 3 * (size_t)P, s) != cudaSuccess ||
        cudaMemsetAsync(L.go, 0, sizeof(float) * (size_t)N, s) != cudaSuccess ||
        cudaMemsetAsync(L.gcol, 0, sizeof(float) * 3 * (size_t)N, s) != cudaSuccess)
        return launch_status(who);
    EventPair ev;
    if (cudaEventCreate(&ev.a) != cudaSuccess || cudaEventCreate(&ev.b) != cudaSuccess) return launch_status(who);

    // one run of candidate c: its tile order (when longest first), the forward and the backward
    auto once = [&](const GsTuning& c) -> int {
        GsRasterConfig cfg{};
        cfg.persistent = c.persistent;
        cfg.ctas_per_sm = c.ctas_per_sm;
        cfg.tile_order = c.longest_first ? L.order : nullptr;
        cfg.queue = L.queue;
        cfg.warp_hits = L.hits;
        cfg.bwd_pixels = c.bwd_pixels;
        cfg.bwd_batch = c.bwd_batch;
        if (c.longest_first)
            if (int rc = gs_tile_order(tile_ranges, T_total, L.order_ws, L.order_ws_bytes, L.order, stream)) return rc;
        if (int rc = gs_rasterize_fwd(views, V, T_total, means2d, conics, opacities, colors, isect_ids, tile_ranges,
                                      nullptr, L.rgb, L.T_final, L.last, nullptr, &cfg, stream))
            return rc;
        return gs_rasterize_bwd(views, V, P, T_total, means2d, conics, opacities, colors, isect_ids, nullptr, nullptr,
                                nullptr, tile_ranges, K, K_capacity, nullptr, L.T_final, L.last, L.dL, 0, nullptr, 0,
                                L.g2, L.gc, L.go, L.gcol, &cfg, stream);
    };
    // a warm-up of every candidate (and its argument checks), then the repeats round-robin over the
    // candidates, so that a drift of the clocks during the tuning weighs on all of them alike
    for (const GsTuning& c : cands)
        if (int rc = once(c)) return rc;
    std::vector<std::vector<float>> times(cands.size());
    for (int r = 0; r < repeats; ++r)
        for (size_t ci = 0; ci < cands.size(); ++ci) {
            if (cudaEventRecord(ev.a, s) != cudaSuccess) return launch_status(who);
            if (int rc = once(cands[ci])) return rc;
            if (cudaEventRecord(ev.b, s) != cudaSuccess || cudaEventSynchronize(ev.b) != cudaSuccess)
                return launch_status(who);
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev.a, ev.b) != cudaSuccess) return launch_status(who);
            times[ci].push_back(ms);
        }
    int best_i = -1;
    for (size_t ci = 0; ci < cands.size(); ++ci) {
        GsTuning& c = cands[ci];
        std::sort(times[ci].begin(), times[ci].end());
        c.ms = times[ci][times[ci].size() / 2];
        if (results) results[ci] = c;
        if (best_i < 0 || c.ms < cands[best_i].ms) best_i = (int)ci;
    }
    *best = cands[best_i];
    return GS_OK;
}
