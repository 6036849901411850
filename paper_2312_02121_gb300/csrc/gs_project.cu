// Projection of 3D Gaussians (Sec. 2.1, Eq. 2-6, tile box of Sec. 2.2) and its
// backward (Sec. 3.2, Eq. 16-20, and Sec. 3.2.1).  One thread per projection
// (view, Gaussian); both kernels are bound by HBM traffic (~50 B in / 36 B out
// per projection forward).
#include "gs_common.cuh"

namespace gs {

// Eq. 5 for a unit quaternion (w, x, y, z), with R_11 = 1 - 2(x^2 + z^2)
// (the orthonormal form; the printed minus sign is a typo, see the dR/dz
// Jacobian of Sec. 3.2.1).
__device__ __forceinline__ void quat_to_rot(float w, float x, float y, float z, float R[9])
{
    R[0] = 1.f - 2.f * (y * y + z * z);
    R[1] = 2.f * (x * y - w * z);
    R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);
    R[4] = 1.f - 2.f * (x * x + z * z);
    R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);
    R[7] = 2.f * (y * z + w * x);
    R[8] = 1.f - 2.f * (x * x + y * y);
}

// Forward quantities shared by both kernels.
struct Proj {
    float t[3];       // camera-space mean
    float J00, J02, J11, J12;
    float rz;         // 1 / t_z
    float q[4];       // unit quaternion
    float qinv;       // 1 / |q|
    float R[9];       // rotation of the Gaussian
    float M[9];       // R S
    float Sig[6];     // Sigma: 00 01 02 11 12 22
    float T[6];       // J R_cw (2x3)
    float a, b, c;    // Sigma' + eps2d I
};

__device__ __forceinline__ void project_one(const GsCamera& cam, const float* __restrict__ means,
                                            const float4* __restrict__ quats, const float* __restrict__ scales,
                                            int64_t g, float eps2d, Proj& o, float& u, float& v)
{
    const float mx = means[3 * g + 0], my = means[3 * g + 1], mz = means[3 * g + 2];
    const float* W = cam.R;
    // Eq. 2: t = T_cw [mu; 1]
    o.t[0] = fmaf(W[0], mx, fmaf(W[1], my, fmaf(W[2], mz, cam.t[0])));
    o.t[1] = fmaf(W[3], mx, fmaf(W[4], my, fmaf(W[5], mz, cam.t[1])));
    o.t[2] = fmaf(W[6], mx, fmaf(W[7], my, fmaf(W[8], mz, cam.t[2])));
    o.rz = 1.f / o.t[2];
    u = cam.fx * o.t[0] * o.rz + cam.cx;
    v = cam.fy * o.t[1] * o.rz + cam.cy;
    // Eq. 3: J
    o.J00 = cam.fx * o.rz;
    o.J11 = cam.fy * o.rz;
    o.J02 = -cam.fx * o.t[0] * o.rz * o.rz;
    o.J12 = -cam.fy * o.t[1] * o.rz * o.rz;
    // Eq. 5-6: Sigma = R S S^T R^T with q normalised
    const float4 q = quats[g];
    o.qinv = 1.f / sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    o.q[0] = q.x * o.qinv; o.q[1] = q.y * o.qinv; o.q[2] = q.z * o.qinv; o.q[3] = q.w * o.qinv;
    quat_to_rot(o.q[0], o.q[1], o.q[2], o.q[3], o.R);
    const float s0 = scales[3 * g + 0], s1 = scales[3 * g + 1], s2 = scales[3 * g + 2];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        o.M[3 * i + 0] = o.R[3 * i + 0] * s0;
        o.M[3 * i + 1] = o.R[3 * i + 1] * s1;
        o.M[3 * i + 2] = o.R[3 * i + 2] * s2;
    }
    const float* M = o.M;
    o.Sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    o.Sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    o.Sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    o.Sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    o.Sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    o.Sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    // Eq. 4: Sigma' = T Sigma T^T with T = J R_cw
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        o.T[j] = o.J00 * W[j] + o.J02 * W[6 + j];
        o.T[3 + j] = o.J11 * W[3 + j] + o.J12 * W[6 + j];
    }
    const float* S = o.Sig;
    float U[6];  // T Sigma
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const float* Tr = o.T + 3 * r;
        U[3 * r + 0] = Tr[0] * S[0] + Tr[1] * S[1] + Tr[2] * S[2];
        U[3 * r + 1] = Tr[0] * S[1] + Tr[1] * S[3] + Tr[2] * S[4];
        U[3 * r + 2] = Tr[0] * S[2] + Tr[1] * S[4] + Tr[2] * S[5];
    }
    o.a = U[0] * o.T[0] + U[1] * o.T[1] + U[2] * o.T[2] + eps2d;
    o.b = U[0] * o.T[3] + U[1] * o.T[4] + U[2] * o.T[5];
    o.c = U[3] * o.T[3] + U[4] * o.T[4] + U[5] * o.T[5] + eps2d;
}

// a c - b^2 with the rounding error of b^2 compensated (Kahan's 2x2 determinant).
__device__ __forceinline__ float det2(float a, float b, float c)
{
    const float bb = b * b;
    const float e = fmaf(b, b, -bb);
    return fmaf(a, c, -bb) - e;
}

__global__ void __launch_bounds__(256)
k_project_fwd(const GsView* __restrict__ views, int V, int64_t P, const float* __restrict__ means,
              const float4* __restrict__ quats, const float* __restrict__ scales, float eps2d,
              float2* __restrict__ means2d, float* __restrict__ conics, float* __restrict__ depths,
              short4* __restrict__ rects, int32_t* __restrict__ touched, unsigned long long* __restrict__ K_total)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int count = 0;
    if (p < P) {
        const GsView& view = views[view_of_projection(views, V, p)];
        const GsCamera& cam = view.cam;
        const int64_t g = view.g_begin + (p - view.proj_offset);
        Proj o;
        float u, v;
        project_one(cam, means, quats, scales, g, eps2d, o, u, v);
        const float det = det2(o.a, o.b, o.c);
        bool ok = o.t[2] > cam.near_plane && o.t[2] < cam.far_plane && det > 0.f &&
                  isfinite(u) && isfinite(v) && isfinite(o.a) && isfinite(o.c) && isfinite(det);
        float ca = 0.f, cb = 0.f, cc = 0.f;
        short4 r = make_short4(0, 0, 0, 0);
        if (ok) {
            const float inv = 1.f / det;
            ca = o.c * inv;
            cb = -o.b * inv;
            cc = o.a * inv;
            // Sec. 2.2: tight 3-sigma box and the tiles it touches (1/16 is exact)
            const float rx = 3.f * sqrtf(o.a), ry = 3.f * sqrtf(o.c);
            const float TX = (float)view.tiles_x, TY = (float)view.tiles_y;
            const float x0 = fminf(fmaxf(floorf((u - rx) * (1.f / kTile)), 0.f), TX);
            const float x1 = fminf(fmaxf(floorf((u + rx) * (1.f / kTile)) + 1.f, 0.f), TX);
            const float y0 = fminf(fmaxf(floorf((v - ry) * (1.f / kTile)), 0.f), TY);
            const float y1 = fminf(fmaxf(floorf((v + ry) * (1.f / kTile)) + 1.f, 0.f), TY);
            if (x0 < x1 && y0 < y1) {
                r = make_short4((short)x0, (short)y0, (short)x1, (short)y1);
                count = (int)((x1 - x0) * (y1 - y0));
            } else {
                ok = false;
            }
        }
        means2d[p] = make_float2(u, v);
        conics[3 * p + 0] = ca;
        conics[3 * p + 1] = cb;
        conics[3 * p + 2] = cc;
        depths[p] = o.t[2];
        rects[p] = r;
        touched[p] = count;
    }
    if (K_total) {
        __shared__ unsigned long long warp_sum[8];
        unsigned long long s = (unsigned long long)count;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(kFull, s, d);
        if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long tot = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += warp_sum[w];
            if (tot) atomicAdd(K_total, tot);
        }
    }
}

__global__ void __launch_bounds__(256)
k_project_bwd(const GsView* __restrict__ views, int V, int64_t P, const float* __restrict__ means,
              const float4* __restrict__ quats, const float* __restrict__ scales, float eps2d,
              const int32_t* __restrict__ touched, const float2* __restrict__ dL_dmeans2d,
              const float* __restrict__ dL_dconics, float* __restrict__ dL_dmeans, float* __restrict__ dL_dquats,
              float* __restrict__ dL_dscales)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P || touched[p] == 0) return;
    const GsView& view = views[view_of_projection(views, V, p)];
    const GsCamera& cam = view.cam;
    const int64_t g = view.g_begin + (p - view.proj_offset);
    Proj o;
    float u, v;
    project_one(cam, means, quats, scales, g, eps2d, o, u, v);
    const float inv = 1.f / det2(o.a, o.b, o.c);
    const float Y0 = o.c * inv, Y1 = -o.b * inv, Y2 = o.a * inv;  // Y = [[Y0, Y1], [Y1, Y2]]

    // Sec. 3.1: G = dL/dY from the packed conic gradient (the b gradient covers both off-diagonals)
    const float ga = dL_dconics[3 * p + 0], gb = 0.5f * dL_dconics[3 * p + 1], gc = dL_dconics[3 * p + 2];
    // dL/dSigma' = -Y G Y
    const float YG00 = Y0 * ga + Y1 * gb, YG01 = Y0 * gb + Y1 * gc;
    const float YG10 = Y1 * ga + Y2 * gb, YG11 = Y1 * gb + Y2 * gc;
    const float D00 = -(YG00 * Y0 + YG01 * Y1);
    const float D01 = -(YG00 * Y1 + YG01 * Y2);
    const float D10 = -(YG10 * Y0 + YG11 * Y1);
    const float D11 = -(YG10 * Y1 + YG11 * Y2);
    const float Ds = 0.5f * (D01 + D10);  // symmetric part

    // Sec. 3.2: dL/dSigma = T^T D T ; dL/dT = D T Sigma^T + D^T T Sigma = 2 D T Sigma
    float Vm[6];  // D T (2x3)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        Vm[j] = D00 * o.T[j] + Ds * o.T[3 + j];
        Vm[3 + j] = Ds * o.T[j] + D11 * o.T[3 + j];
    }
    float dSig[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) dSig[3 * i + j] = o.T[i] * Vm[j] + o.T[3 + i] * Vm[3 + j];
    const float* S = o.Sig;
    const float Sf[9] = {S[0], S[1], S[2], S[1], S[3], S[4], S[2], S[4], S[5]};
    float dT[6];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            dT[3 * r + j] = 2.f * (Vm[3 * r + 0] * Sf[j] + Vm[3 * r + 1] * Sf[3 + j] + Vm[3 * r + 2] * Sf[6 + j]);
    // dL/dJ = dL/dT R_cw^T (only the four non-constant entries of J matter)
    const float* W = cam.R;
    const float dJ00 = dT[0] * W[0] + dT[1] * W[1] + dT[2] * W[2];
    const float dJ02 = dT[0] * W[6] + dT[1] * W[7] + dT[2] * W[8];
    const float dJ11 = dT[3] * W[3] + dT[4] * W[4] + dT[5] * W[5];
    const float dJ12 = dT[3] * W[6] + dT[4] * W[7] + dT[5] * W[8];
    // dJ/dt as printed in Sec. 3.2, plus the 2D-mean term J^T dL/dmu' (Eq. 16-17)
    const float rz2 = o.rz * o.rz, rz3 = rz2 * o.rz;
    const float2 gm = dL_dmeans2d[p];
    const float dtx = -cam.fx * rz2 * dJ02 + o.J00 * gm.x;
    const float dty = -cam.fy * rz2 * dJ12 + o.J11 * gm.y;
    const float dtz = -cam.fx * rz2 * dJ00 + 2.f * cam.fx * o.t[0] * rz3 * dJ02 - cam.fy * rz2 * dJ11 +
                      2.f * cam.fy * o.t[1] * rz3 * dJ12 + o.J02 * gm.x + o.J12 * gm.y;
    // Eq. 20: dL/dmu = R_cw^T dL/dt
    atomicAdd(dL_dmeans + 3 * g + 0, W[0] * dtx + W[3] * dty + W[6] * dtz);
    atomicAdd(dL_dmeans + 3 * g + 1, W[1] * dtx + W[4] * dty + W[7] * dtz);
    atomicAdd(dL_dmeans + 3 * g + 2, W[2] * dtx + W[5] * dty + W[8] * dtz);

    // Sec. 3.2.1: dL/dM = (G + G^T) M = 2 dSigma M (dSigma is symmetric)
    float dM[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            dM[3 * i + j] = 2.f * (dSig[3 * i + 0] * o.M[j] + dSig[3 * i + 1] * o.M[3 + j] + dSig[3 * i + 2] * o.M[6 + j]);
    const float s[3] = {scales[3 * g + 0], scales[3 * g + 1], scales[3 * g + 2]};
    float dR[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) dR[3 * i + j] = dM[3 * i + j] * s[j];
#pragma unroll
    for (int j = 0; j < 3; ++j)
        atomicAdd(dL_dscales + 3 * g + j, o.R[j] * dM[j] + o.R[3 + j] * dM[3 + j] + o.R[6 + j] * dM[6 + j]);
    // <dL/dR, dR/dq> with the four Jacobians of Sec. 3.2.1 at the unit quaternion
    const float w = o.q[0], x = o.q[1], y = o.q[2], z = o.q[3];
    const float gw = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    const float gx = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] -
                            2.f * x * dR[8]);
    const float gy = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] -
                            2.f * y * dR[8]);
    const float gz = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] + y * dR[5] +
                            x * dR[6] + y * dR[7]);
    // through q_hat = q / |q|: dq = (I - q_hat q_hat^T) dq_hat / |q|
    const float dot = gw * w + gx * x + gy * y + gz * z;
    atomicAdd(dL_dquats + 4 * g + 0, (gw - w * dot) * o.qinv);
    atomicAdd(dL_dquats + 4 * g + 1, (gx - x * dot) * o.qinv);
    atomicAdd(dL_dquats + 4 * g + 2, (gy - y * dot) * o.qinv);
    atomicAdd(dL_dquats + 4 * g + 3, (gz - z * dot) * o.qinv);
}

static bool misaligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) != 0; }

}  // namespace gs

using namespace gs;

extern "C" int gs_project(const GsView* views, int32_t V, int64_t P, const float* means, const float* quats,
                          const float* scales, float eps2d, float* means2d, float* conics, float* depths,
                          int16_t* rects, int32_t* touched, int64_t* K_total, void* stream)
{
    if (V < 0 || P < 0 || (P > 0 && V == 0))
        return fail(GS_ERR_INVALID_ARG, "gs_project: V=%d P=%lld", V, (long long)P);
    if (P > 0 && (!views || !means || !quats || !scales || !means2d || !conics || !depths || !rects || !touched))
        return fail(GS_ERR_INVALID_ARG, "gs_project: null pointer argument");
    if (misaligned(quats, 16) || misaligned(means2d, 8) || misaligned(rects, 8))
        return fail(GS_ERR_INVALID_ARG, "gs_project: quats need 16-byte, means2d/rects 8-byte alignment");
    if (!(eps2d >= 0.f)) return fail(GS_ERR_INVALID_ARG, "gs_project: eps2d must be >= 0");
    cudaStream_t s = as_stream(stream);
    if (K_total && cudaMemsetAsync(K_total, 0, sizeof(int64_t), s) != cudaSuccess)
        return launch_status("gs_project memset");
    if (P == 0) return GS_OK;
    const int threads = 256;
    const unsigned blocks = (unsigned)((P + threads - 1) / threads);
    k_project_fwd<<<blocks, threads, 0, s>>>(views, V, P, means, reinterpret_cast<const float4*>(quats), scales, eps2d,
                                             reinterpret_cast<float2*>(means2d), conics, depths,
                                             reinterpret_cast<short4*>(rects), touched,
                                             reinterpret_cast<unsigned long long*>(K_total));
    count_launches(1);
    return launch_status("gs_project");
}

extern "C" int gs_project_bwd(const GsView* views, int32_t V, int64_t P, const float* means, const float* quats,
                              const float* scales, float eps2d, const int32_t* touched, const float* dL_dmeans2d,
                              const float* dL_dconics, float* dL_dmeans, float* dL_dquats, float* dL_dscales,
                              void* stream)
{
    if (V < 0 || P < 0 || (P > 0 && V == 0))
        return fail(GS_ERR_INVALID_ARG, "gs_project_bwd: V=%d P=%lld", V, (long long)P);
    if (P > 0 && (!views || !means || !quats || !scales || !touched || !dL_dmeans2d || !dL_dconics || !dL_dmeans ||
                  !dL_dquats || !dL_dscales))
        return fail(GS_ERR_INVALID_ARG, "gs_project_bwd: null pointer argument");
    if (misaligned(quats, 16) || misaligned(dL_dmeans2d, 8))
        return fail(GS_ERR_INVALID_ARG, "gs_project_bwd: quats need 16-byte, dL_dmeans2d 8-byte alignment");
    if (P == 0) return GS_OK;
    const int threads = 256;
    const unsigned blocks = (unsigned)((P + threads - 1) / threads);
    k_project_bwd<<<blocks, threads, 0, as_stream(stream)>>>(
        views, V, P, means, reinterpret_cast<const float4*>(quats), scales, eps2d, touched,
        reinterpret_cast<const float2*>(dL_dmeans2d), dL_dconics, dL_dmeans, dL_dquats, dL_dscales);
    count_launches(1);
    return launch_status("gs_project_bwd");
}
