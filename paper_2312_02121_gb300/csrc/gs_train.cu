// Training-step kernels around the rasteriser: the L2 image loss with its
// gradient dL/dC (the input of Sec. 3.1), and a fused Adam update of the raw
// Gaussian parameters with the activations the renderer consumes (scale =
// exp(log-scale), opacity = sigmoid(logit)).  The paper derives gradients
// only; these kernels close the loop of an optimisation step so that a whole
// step runs on the GPU and can be captured into one CUDA graph.  Both are
// bound by HBM traffic.
#include <algorithm>

#include "gs_common.cuh"

namespace gs {

// ---------------------------------------------------------------------------
// L2 loss
// ---------------------------------------------------------------------------

template <typename S>
__device__ __forceinline__ S block_sum(S x, S* sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = x;
    __syncthreads();
    x = S(0);
    if (w == 0) {
        x = lane < (int)(blockDim.x >> 5) ? sh[lane] : S(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    }
    return x;  // valid in thread 0
}

// L = inv_norm * sum (rgb - target)^2 ; dL/drgb = 2 inv_norm (rgb - target).
// A grid-stride loop over 4-element groups (vector loads when the pointers
// allow), one atomic per block into *loss.
template <typename S>
__global__ void __launch_bounds__(256)
k_l2_loss(const S* __restrict__ rgb, const S* __restrict__ target, int64_t n, S inv_norm, S* __restrict__ dL,
          S* __restrict__ loss, bool vec)
{
    pdl_wait();
    pdl_trigger();
    __shared__ S sh[8];
    S acc = S(0);
    const S two = S(2) * inv_norm;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n4 = vec ? n / 4 : 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const V4<S> a = reinterpret_cast<const V4<S>*>(rgb)[i];
        const V4<S> b = reinterpret_cast<const V4<S>*>(target)[i];
        const S d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
        acc += (d0 * d0 + d1 * d1) + (d2 * d2 + d3 * d3);
        if (dL) reinterpret_cast<V4<S>*>(dL)[i] = mk4<S>(two * d0, two * d1, two * d2, two * d3);
    }
    for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const S d = rgb[i] - target[i];
        acc += d * d;
        if (dL) dL[i] = two * d;
    }
    acc = block_sum<S>(acc, sh);
    if (threadIdx.x == 0 && loss) atomicAdd(loss, acc * inv_norm);
}

static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

template <typename S>
static int l2_loss_impl(const char* who, const S* rgb, const S* target, int64_t n, S inv_norm, S* dL, S* loss,
                        void* stream)
{
    if (n < 0) return fail(GS_ERR_INVALID_ARG, "%s: n=%lld", who, (long long)n);
    if (n > 0 && (!rgb || !target || (!dL && !loss))) return fail(GS_ERR_INVALID_ARG, "%s: null pointer argument", who);
    if (n == 0) return GS_OK;
    const bool vec = aligned(rgb, 4 * sizeof(S)) && aligned(target, 4 * sizeof(S)) && (!dL || aligned(dL, 4 * sizeof(S)));
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t groups = (n + 3) / 4;
    const unsigned blocks = (unsigned)std::min<int64_t>((groups + 255) / 256, (int64_t)std::max(sms, 1) * 8);
    launch_pdl(k_l2_loss<S>, blocks, 256, as_stream(stream), rgb, target, n, inv_norm, dL, loss, vec);
    count_launches(1);
    return launch_status(who);
}

// ---------------------------------------------------------------------------
// Adam
// ---------------------------------------------------------------------------

// State header (first 256 bytes): the step count and the bias corrections of
// the current step; then m and v, 11 + C floats per Gaussian each, field after
// field (means 3, quats 4, log-scales 3, logits 1, colors C).
struct AdamHeader {
    int32_t step;
    float bc1, bc2;  // 1 - beta1^t, 1 - beta2^t
};
constexpr int kAdamGeom = 11;  // means 3, quats 4, log-scales 3, logit 1

__global__ void k_adam_prepare(AdamHeader* h, float beta1, float beta2, const int32_t* __restrict__ skip)
{
    pdl_wait();
    pdl_trigger();
    if (skip && *skip) return;
    const int t = h->step + 1;
    h->step = t;
    h->bc1 = 1.f - powf(beta1, (float)t);
    h->bc2 = 1.f - powf(beta2, (float)t);
}

struct AdamArgs {
    float lr[5], beta1, beta2, eps;
};

__device__ __forceinline__ float adam_one(float& p, float g, float& m, float& v, float lr, const AdamArgs& a,
                                          float bc1, float bc2)
{
    m = fmaf(a.beta1, m, (1.f - a.beta1) * g);
    v = fmaf(a.beta2, v, (1.f - a.beta2) * g * g);
    const float mh = m / bc1, vh = v / bc2;
    p -= lr * mh / (sqrtf(vh) + a.eps);
    return p;
}

// One thread per Gaussian: its 11 + C values, moments and activations.
__global__ void __launch_bounds__(256)
k_adam_step(int64_t N, int C, AdamArgs a, const AdamHeader* __restrict__ h, float* __restrict__ m, float* __restrict__ v,
            float* __restrict__ means, float* __restrict__ quats, float* __restrict__ log_scales,
            float* __restrict__ logits, float* __restrict__ colors, const float* __restrict__ g_means,
            const float* __restrict__ g_quats, const float* __restrict__ g_scales, const float* __restrict__ g_op,
            const float* __restrict__ g_colors, float* __restrict__ scales, float* __restrict__ opacities,
            const int32_t* __restrict__ skip)
{
    pdl_wait();
    pdl_trigger();
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N || (skip && *skip)) return;
    const float bc1 = h->bc1, bc2 = h->bc2;
    // moments: field-major blocks of N x width
    float* m_means = m;
    float* m_quats = m + 3 * N;
    float* m_scales = m + 7 * N;
    float* m_op = m + 10 * N;
    float* m_col = m + 11 * N;
    float* v_means = v;
    float* v_quats = v + 3 * N;
    float* v_scales = v + 7 * N;
    float* v_op = v + 10 * N;
    float* v_col = v + 11 * N;
#pragma unroll
    for (int j = 0; j < 3; ++j)
        adam_one(means[3 * n + j], g_means[3 * n + j], m_means[3 * n + j], v_means[3 * n + j], a.lr[0], a, bc1, bc2);
#pragma unroll
    for (int j = 0; j < 4; ++j)
        adam_one(quats[4 * n + j], g_quats[4 * n + j], m_quats[4 * n + j], v_quats[4 * n + j], a.lr[1], a, bc1, bc2);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        // d/dlog s = d/ds * s
        const float s = scales[3 * n + j];
        const float ls = adam_one(log_scales[3 * n + j], g_scales[3 * n + j] * s, m_scales[3 * n + j],
                                  v_scales[3 * n + j], a.lr[2], a, bc1, bc2);
        scales[3 * n + j] = expf(ls);
    }
    {
        // d/dlogit = d/do * o (1 - o)
        const float o = opacities[n];
        const float lg = adam_one(logits[n], g_op[n] * o * (1.f - o), m_op[n], v_op[n], a.lr[3], a, bc1, bc2);
        opacities[n] = 1.f / (1.f + expf(-lg));
    }
    for (int j = 0; j < C; ++j) {
        const int64_t i = (int64_t)C * n + j;
        adam_one(colors[i], g_colors[i], m_col[i], v_col[i], a.lr[4], a, bc1, bc2);
    }
}

__global__ void __launch_bounds__(256)
k_activate(int64_t N, const float* __restrict__ log_scales, const float* __restrict__ logits,
           float* __restrict__ scales, float* __restrict__ opacities)
{
    pdl_wait();
    pdl_trigger();
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
#pragma unroll
    for (int j = 0; j < 3; ++j) scales[3 * n + j] = expf(log_scales[3 * n + j]);
    opacities[n] = 1.f / (1.f + expf(-logits[n]));
}

}  // namespace gs

using namespace gs;

extern "C" int gs_l2_loss(const float* rgb, const float* target, int64_t n, float inv_norm, float* dL_drgb,
                          float* loss, void* stream)
{
    gs::NvtxRange nvtx("gs_l2_loss");
    return l2_loss_impl<float>("gs_l2_loss", rgb, target, n, inv_norm, dL_drgb, loss, stream);
}

extern "C" int gs_l2_loss_f64(const double* rgb, const double* target, int64_t n, double inv_norm, double* dL_drgb,
                              double* loss, void* stream)
{
    gs::NvtxRange nvtx("gs_l2_loss_f64");
    return l2_loss_impl<double>("gs_l2_loss_f64", rgb, target, n, inv_norm, dL_drgb, loss, stream);
}

extern "C" size_t gs_adam_state_size(int64_t N, int32_t C)
{
    return N < 0 || C < 1 ? 0 : 256 + align256(sizeof(float) * (kAdamGeom + C) * (size_t)N) * 2;
}

extern "C" int gs_adam_step(int64_t N, int32_t C, const GsAdamConfig* cfg, void* state, size_t state_bytes, float* means,
                            float* quats, float* log_scales, float* opacity_logits, float* colors,
                            const float* dL_dmeans, const float* dL_dquats, const float* dL_dscales,
                            const float* dL_dopacities, const float* dL_dcolors, float* scales, float* opacities,
                            const int32_t* skip_if_set, void* stream)
{
    gs::NvtxRange nvtx("gs_adam_step");
    const char* who = "gs_adam_step";
    if (N < 0 || C < 1 || !cfg)
        return fail(GS_ERR_INVALID_ARG, "%s: N=%lld, C=%d or null config", who, (long long)N, C);
    if (!state || state_bytes < gs_adam_state_size(N, C))
        return fail(GS_ERR_INVALID_ARG, "%s: state needs %zu bytes, got %zu", who, gs_adam_state_size(N, C),
                    state_bytes);
    if (N > 0 && (!means || !quats || !log_scales || !opacity_logits || !colors || !dL_dmeans || !dL_dquats ||
                  !dL_dscales || !dL_dopacities || !dL_dcolors || !scales || !opacities))
        return fail(GS_ERR_INVALID_ARG, "%s: null pointer argument", who);
    if (!(cfg->beta1 >= 0.f && cfg->beta1 < 1.f && cfg->beta2 >= 0.f && cfg->beta2 < 1.f && cfg->eps > 0.f))
        return fail(GS_ERR_INVALID_ARG, "%s: need 0 <= beta < 1 and eps > 0", who);
    cudaStream_t s = as_stream(stream);
    AdamHeader* h = reinterpret_cast<AdamHeader*>(state);
    float* m = reinterpret_cast<float*>(static_cast<char*>(state) + 256);
    float* v = reinterpret_cast<float*>(static_cast<char*>(state) + 256 +
                                        align256(sizeof(float) * (kAdamGeom + C) * (size_t)N));
    launch_pdl(k_adam_prepare, 1, 1, s, h, cfg->beta1, cfg->beta2, skip_if_set);
    AdamArgs a;
    for (int i = 0; i < 5; ++i) a.lr[i] = cfg->lr[i];
    a.beta1 = cfg->beta1;
    a.beta2 = cfg->beta2;
    a.eps = cfg->eps;
    int launched = 1;
    if (N > 0) {
        launch_pdl(k_adam_step, (unsigned)((N + 255) / 256), 256, s, N, C, a, h, m, v, means, quats, log_scales,
                                                                opacity_logits, colors, dL_dmeans, dL_dquats,
                                                                dL_dscales, dL_dopacities, dL_dcolors, scales,
                                                                opacities, skip_if_set);
        ++launched;
    }
    count_launches(launched);
    return launch_status(who);
}

extern "C" int gs_activate(int64_t N, const float* log_scales, const float* opacity_logits, float* scales,
                           float* opacities, void* stream)
{
    gs::NvtxRange nvtx("gs_activate");
    if (N < 0) return fail(GS_ERR_INVALID_ARG, "gs_activate: N=%lld", (long long)N);
    if (N == 0) return GS_OK;
    if (!log_scales || !opacity_logits || !scales || !opacities)
        return fail(GS_ERR_INVALID_ARG, "gs_activate: null pointer argument");
    launch_pdl(k_activate, (unsigned)((N + 255) / 256), 256, as_stream(stream), N, log_scales, opacity_logits, scales,
                                                                          opacities);
    count_launches(1);
    return launch_status("gs_activate");
}
