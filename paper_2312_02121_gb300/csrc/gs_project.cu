// Projection of 3D Gaussians (Sec. 2.1, Eq. 2-6, tile box of Sec. 2.2) and its
// backward (Sec. 3.2, Eq. 16-20, and Sec. 3.2.1).  One thread per projection
// (view, Gaussian); both kernels are bound by HBM traffic (~50 B in / 36 B out
// per projection forward).  Instantiated for fp32 (the fast path) and fp64
// (the gs_*_f64 entry points, used to check the analytic backward against
// finite differences).
#include <type_traits>

#include "gs_common.cuh"

namespace gs {

// Eq. 5 for a unit quaternion (w, x, y, z), with R_11 = 1 - 2(x^2 + z^2)
// (the orthonormal form; the printed minus sign is a typo, see the dR/dz
// Jacobian of Sec. 3.2.1).
template <typename S>
__device__ __forceinline__ void quat_to_rot(S w, S x, S y, S z, S R[9])
{
    R[0] = S(1) - S(2) * (y * y + z * z);
    R[1] = S(2) * (x * y - w * z);
    R[2] = S(2) * (x * z + w * y);
    R[3] = S(2) * (x * y + w * z);
    R[4] = S(1) - S(2) * (x * x + z * z);
    R[5] = S(2) * (y * z - w * x);
    R[6] = S(2) * (x * z - w * y);
    R[7] = S(2) * (y * z + w * x);
    R[8] = S(1) - S(2) * (x * x + y * y);
}

// Forward quantities shared by both kernels.
//
// Sigma' is formed from the images of the Gaussian's scaled axes, A = T R S
// (T = J R_cw, 2x3), as Sigma' = A A^T + eps2d I -- the same matrix as
// T Sigma T^T of Eq. 4 with Sigma = R S S^T R^T of Eq. 6, but without
// forming Sigma: the product M M^T buries the variance of a thin Gaussian's
// short axes under the long one (fp32 keeps about 7 digits of the largest
// entry), A A^T keeps every axis to full relative precision.  Its
// determinant comes from Cauchy-Binet, det(A A^T) = sum_{i<j} (a_i ^ a_j)^2
// over the columns a_i of A, plus eps2d (|row 0|^2 + |row 1|^2) + eps2d^2: a
// sum of non-negative terms, where a c - b^2 cancels for a thin Gaussian.
template <typename S>
struct Proj {
    S t[3];       // camera-space mean
    S J00, J02, J11, J12;
    S rz;         // 1 / t_z
    S q[4];       // unit quaternion
    S qinv;       // 1 / |q|
    S R[9];       // rotation of the Gaussian
    S s[3];       // scales
    S T[6];       // J R_cw (2x3)
    S Bx[3], By[3];  // T R: the image of each unit axis (column j: (Bx[j], By[j])); A = B S
    S a, b, c;    // Sigma' + eps2d I = [[a, b], [b, c]]
    S det;        // det of that
};

template <typename S>
__device__ __forceinline__ void project_one(const GsCamera& cam, const S* __restrict__ means,
                                            const V4<S>* __restrict__ quats, const S* __restrict__ scales, int64_t g,
                                            S eps2d, Proj<S>& o, S& u, S& v)
{
    const S mx = means[3 * g + 0], my = means[3 * g + 1], mz = means[3 * g + 2];
    S W[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) W[i] = S(cam.R[i]);
    const S fx = S(cam.fx), fy = S(cam.fy);
    // Eq. 2: t = T_cw [mu; 1]
    o.t[0] = fma(W[0], mx, fma(W[1], my, fma(W[2], mz, S(cam.t[0]))));
    o.t[1] = fma(W[3], mx, fma(W[4], my, fma(W[5], mz, S(cam.t[1]))));
    o.t[2] = fma(W[6], mx, fma(W[7], my, fma(W[8], mz, S(cam.t[2]))));
    o.rz = S(1) / o.t[2];
    u = fx * o.t[0] * o.rz + S(cam.cx);
    v = fy * o.t[1] * o.rz + S(cam.cy);
    // Eq. 3: J
    o.J00 = fx * o.rz;
    o.J11 = fy * o.rz;
    o.J02 = -fx * o.t[0] * o.rz * o.rz;
    o.J12 = -fy * o.t[1] * o.rz * o.rz;
    // Eq. 5: R of the normalised quaternion
    const V4<S> q = quats[g];
    o.qinv = S(1) / sqrt(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    o.q[0] = q.x * o.qinv; o.q[1] = q.y * o.qinv; o.q[2] = q.z * o.qinv; o.q[3] = q.w * o.qinv;
    quat_to_rot(o.q[0], o.q[1], o.q[2], o.q[3], o.R);
    o.s[0] = scales[3 * g + 0];
    o.s[1] = scales[3 * g + 1];
    o.s[2] = scales[3 * g + 2];
    // Eq. 4 and 6: T = J R_cw, A = T R S, Sigma' = A A^T + eps2d I
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        o.T[j] = o.J00 * W[j] + o.J02 * W[6 + j];
        o.T[3 + j] = o.J11 * W[3 + j] + o.J12 * W[6 + j];
    }
    S Ax[3], Ay[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        o.Bx[j] = o.T[0] * o.R[j] + o.T[1] * o.R[3 + j] + o.T[2] * o.R[6 + j];
        o.By[j] = o.T[3] * o.R[j] + o.T[4] * o.R[3 + j] + o.T[5] * o.R[6 + j];
        Ax[j] = o.Bx[j] * o.s[j];
        Ay[j] = o.By[j] * o.s[j];
    }
    const S rx2 = Ax[0] * Ax[0] + Ax[1] * Ax[1] + Ax[2] * Ax[2];
    const S ry2 = Ay[0] * Ay[0] + Ay[1] * Ay[1] + Ay[2] * Ay[2];
    o.a = rx2 + eps2d;
    o.c = ry2 + eps2d;
    o.b = Ax[0] * Ay[0] + Ax[1] * Ay[1] + Ax[2] * Ay[2];
    const S w01 = Ax[0] * Ay[1] - Ay[0] * Ax[1], w02 = Ax[0] * Ay[2] - Ay[0] * Ax[2], w12 = Ax[1] * Ay[2] - Ay[1] * Ax[2];
    o.det = w01 * w01 + w02 * w02 + w12 * w12 + eps2d * (rx2 + ry2) + eps2d * eps2d;
}

// The conic Y = Sigma'^-1 in the factored form (ya, yk, yd) of the ABI:
// sigma = (ya (dx + yk dy)^2 + yd dy^2) / 2, i.e. Y = [[ya, ya yk], [ya yk, ya yk^2 + yd]] -- the LDL^T
// factors of Y.  ya = c / det, yk = -b / c, yd = 1 / c: quotients only, no cancellation, so both axes of a
// thin Gaussian keep their digits (the packed entries of Y lose the long axis: yd = Y_11 - Y_01^2 / Y_00
// cancels).
template <typename S>
__device__ __forceinline__ void conic_factors(const Proj<S>& o, S& ya, S& yk, S& yd)
{
    ya = o.c / o.det;
    yk = -o.b / o.c;
    yd = S(1) / o.c;
}

template <typename S>
__global__ void __launch_bounds__(256)
k_project_fwd(const GsView* __restrict__ views, int V, int64_t P, const S* __restrict__ means,
              const V4<S>* __restrict__ quats, const S* __restrict__ scales, S eps2d, V2<S>* __restrict__ means2d,
              S* __restrict__ conics, float* __restrict__ depths, short4* __restrict__ rects,
              int32_t* __restrict__ touched, unsigned long long* __restrict__ K_total)
{
    pdl_wait();
    pdl_trigger();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int count = 0;
    if (p < P) {
        const GsView& view = views[view_of_projection(views, V, p)];
        const GsCamera& cam = view.cam;
        const int64_t g = view.g_begin + (p - view.proj_offset);
        Proj<S> o;
        S u, v;
        project_one(cam, means, quats, scales, g, eps2d, o, u, v);
        bool ok = o.t[2] > S(cam.near_plane) && o.t[2] < S(cam.far_plane) && o.det > S(0) && o.c > S(0) &&
                  isfinite(u) && isfinite(v) && isfinite(o.a) && isfinite(o.c) && isfinite(o.det);
        S ca = 0, cb = 0, cc = 0;
        short4 r = make_short4(0, 0, 0, 0);
        if (ok) {
            conic_factors(o, ca, cb, cc);
            // Sec. 2.2: tight 3-sigma box and the tiles it touches (1/16 is exact)
            const S rx = S(3) * sqrt(o.a), ry = S(3) * sqrt(o.c);
            const S TX = (S)view.tiles_x, TY = (S)view.tiles_y;
            const S x0 = fmin(fmax(floor((u - rx) * (S(1) / kTile)), S(0)), TX);
            const S x1 = fmin(fmax(floor((u + rx) * (S(1) / kTile)) + S(1), S(0)), TX);
            const S y0 = fmin(fmax(floor((v - ry) * (S(1) / kTile)), S(0)), TY);
            const S y1 = fmin(fmax(floor((v + ry) * (S(1) / kTile)) + S(1), S(0)), TY);
            if (x0 < x1 && y0 < y1) {
                r = make_short4((short)x0, (short)y0, (short)x1, (short)y1);
                count = (int)((x1 - x0) * (y1 - y0));
            } else {
                ok = false;
            }
        }
        V2<S> m2;
        m2.x = u;
        m2.y = v;
        means2d[p] = m2;
        conics[3 * p + 0] = ca;
        conics[3 * p + 1] = cb;
        conics[3 * p + 2] = cc;
        depths[p] = (float)o.t[2];  // sort key (fp32 in both instantiations)
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

// The backward of one projection p of view `view`.  With kView it also returns
// this projection's share of dL/dT_cw (rows 0-2 of the 4x4, row-major) in vg.
//
// Sec. 3.2 (Eq. 16-20) and 3.2.1, arranged so that fp32 keeps its digits for a
// thin Gaussian.  The conic gradient arrives as dL/d(ya, yk, yd), the factored
// conic of the forward.  Through ya = c / det, yk = -b / c, yd = 1 / c it gives
// dL/dSigma' (the -Y G Y of Sec. 3.2, written in the factors):
//   dL/dSigma' = al [[1, yk], [yk, yk^2]] + be [[0, 1], [1, 2 yk]] + ga [[0, 0], [0, 1]],
//   al = -ya^2 dL/dya,  be = -yd dL/dyk / 2,  ga = -yd^2 dL/dyd.
// Each unit axis image b_j = (Bx_j, By_j) (column j of T R) is written in the
// conic's coordinates u_j = Bx_j + yk By_j, y_j = By_j; the bilinear form of
// dL/dSigma' is then Q_ij = b_i^T dL/dSigma' b_j = u_i p_j + y_i r_j with
// p_j = al u_j + be y_j and r_j = be u_j + ga y_j.  With A = B S and
// Sigma' = A A^T + eps2d I:
//   dL/dA_j = 2 dL/dSigma' a_j = 2 s_j (p_j, yk p_j + r_j)
//   dL/dT   = dL/dA (R S)^T          (-> dL/dJ = dL/dT R_cw^T, dL/dt, dL/dmu)
//   dL/ds_j = (R^T dL/dM)_jj = 2 s_j Q_jj
//   R^T dL/dR = E S with E = R^T dL/dM, E_ij = 2 s_j Q_ij, whose antisymmetric
//   part is the gradient of a rotation of the Gaussian about its own axes:
//   dL/domega = 2 (Q_12 (s_1^2 - s_2^2), Q_20 (s_2^2 - s_0^2), Q_01 (s_0^2 - s_1^2)).
// Since R(q (x) r) = R(q) R(r), such a rotation moves the unit quaternion by
// q_hat (x) (0, omega) / 2, so dL/dq = 2 q_hat (x) (0, dL/domega) / |q|: the
// gradient the printed dR/dq matrices of Sec. 3.2.1 give, projected on the
// sphere (dL/dq = (I - q_hat q_hat^T) dL/dq_hat / |q|), but without the large
// component along q_hat that the projection would cancel.
//
// u_j of the longest axis image cancels when that axis lies along the
// conic's direction (1, -1 / yk); it is then taken from the identity
// sum_j s_j^2 u_j y_j = -eps2d yk (the off-diagonal of P Sigma' P^T, which is
// diagonal for the factor P = [[1, yk], [0, 1]] of Y = P^T diag(ya, yd) P),
// whose other terms are small and exact.
// kStore: every Gaussian has this one projection only, so its gradients are
// written instead of accumulated (zeros for a culled projection).
template <typename S, bool kView, bool kStore = false>
__device__ __forceinline__ void project_bwd_one(const GsView& view, int64_t p, const S* __restrict__ means,
                                                const V4<S>* __restrict__ quats, const S* __restrict__ scales,
                                                S eps2d, const V2<S>* __restrict__ dL_dmeans2d,
                                                const S* __restrict__ dL_dconics, S* __restrict__ dL_dmeans,
                                                S* __restrict__ dL_dquats, S* __restrict__ dL_dscales, S vg[12],
                                                bool live = true)
{
    const GsCamera& cam = view.cam;
    const int64_t g = view.g_begin + (p - view.proj_offset);
    Proj<S> o;
    S u2, v2;
    project_one(cam, means, quats, scales, g, eps2d, o, u2, v2);
    S ya, yk, yd;
    conic_factors(o, ya, yk, yd);
    const S al = -ya * ya * dL_dconics[3 * p + 0];
    const S be = S(-0.5) * yd * dL_dconics[3 * p + 1];
    const S ga = -yd * yd * dL_dconics[3 * p + 2];

    const S* s = o.s;
    S ut[3], yt[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        ut[j] = fma(yk, o.By[j], o.Bx[j]);
        yt[j] = o.By[j];
    }
    {  // the longest axis image, from the identity when its u cancels
        S mag[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) mag[j] = s[j] * (fabs(o.Bx[j]) + fabs(o.By[j]));
        const int L = mag[0] >= mag[1] ? (mag[0] >= mag[2] ? 0 : 2) : (mag[1] >= mag[2] ? 1 : 2);
        S uL = ut[0], yL = yt[0], bxL = o.Bx[0], sL = s[0];
        if (L == 1) { uL = ut[1]; yL = yt[1]; bxL = o.Bx[1]; sL = s[1]; }
        if (L == 2) { uL = ut[2]; yL = yt[2]; bxL = o.Bx[2]; sL = s[2]; }
        if (fabs(uL) < S(0.25) * (fabs(bxL) + fabs(yk * yL)) && yL != S(0) && sL != S(0)) {
            S num = eps2d * yk;
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (j != L) num = fma(s[j] * s[j] * ut[j], yt[j], num);
            const S uf = -num / (sL * sL * yL);
            if (isfinite(uf)) {
                if (L == 0) ut[0] = uf;
                if (L == 1) ut[1] = uf;
                if (L == 2) ut[2] = uf;
            }
        }
    }
    S pt[3], rt[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        pt[j] = fma(al, ut[j], be * yt[j]);
        rt[j] = fma(be, ut[j], ga * yt[j]);
    }
    auto Q = [&](int i, int j) { return fma(ut[i], pt[j], yt[i] * rt[j]); };

    // dL/dT = dL/dA (R S)^T
    S dT[6] = {S(0), S(0), S(0), S(0), S(0), S(0)};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const S w0 = S(2) * s[j] * s[j] * pt[j];
        const S w1 = S(2) * s[j] * s[j] * fma(yk, pt[j], rt[j]);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            dT[i] = fma(w0, o.R[3 * i + j], dT[i]);
            dT[3 + i] = fma(w1, o.R[3 * i + j], dT[3 + i]);
        }
    }
    // dL/dJ = dL/dT R_cw^T (only the four non-constant entries of J matter)
    S W[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) W[i] = S(cam.R[i]);
    const S fx = S(cam.fx), fy = S(cam.fy);
    const S dJ00 = dT[0] * W[0] + dT[1] * W[1] + dT[2] * W[2];
    const S dJ02 = dT[0] * W[6] + dT[1] * W[7] + dT[2] * W[8];
    const S dJ11 = dT[3] * W[3] + dT[4] * W[4] + dT[5] * W[5];
    const S dJ12 = dT[3] * W[6] + dT[4] * W[7] + dT[5] * W[8];
    // dJ/dt as printed in Sec. 3.2, plus the 2D-mean term J^T dL/dmu' (Eq. 16-17)
    const S rz2 = o.rz * o.rz, rz3 = rz2 * o.rz;
    const V2<S> gm = dL_dmeans2d[p];
    const S dtx = -fx * rz2 * dJ02 + o.J00 * gm.x;
    const S dty = -fy * rz2 * dJ12 + o.J11 * gm.y;
    const S dtz = -fx * rz2 * dJ00 + S(2) * fx * o.t[0] * rz3 * dJ02 - fy * rz2 * dJ11 +
                  S(2) * fy * o.t[1] * rz3 * dJ12 + o.J02 * gm.x + o.J12 * gm.y;
    // Eq. 20: dL/dmu = R_cw^T dL/dt
    if (kStore) {
        const S z = S(0);
        dL_dmeans[3 * g + 0] = live ? W[0] * dtx + W[3] * dty + W[6] * dtz : z;
        dL_dmeans[3 * g + 1] = live ? W[1] * dtx + W[4] * dty + W[7] * dtz : z;
        dL_dmeans[3 * g + 2] = live ? W[2] * dtx + W[5] * dty + W[8] * dtz : z;
    } else if (live) {
        atomic_add3(dL_dmeans + 3 * g, W[0] * dtx + W[3] * dty + W[6] * dtz, W[1] * dtx + W[4] * dty + W[7] * dtz,
                W[2] * dtx + W[5] * dty + W[8] * dtz);
    }
    if constexpr (kView) {
        // Eq. 20: dL/dT_cw = dL/dt [mu; 1]^T; the R_cw block also gains J^T dL/dT, the covariance route
        // (Sigma' = T Sigma T^T with T = J R_cw), for which the rows of J are (J00, 0, J02), (0, J11, J12)
        const S mu[3] = {means[3 * g + 0], means[3 * g + 1], means[3 * g + 2]};
        const S dt[3] = {dtx, dty, dtz};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            vg[0 * 4 + j] = dt[0] * mu[j] + o.J00 * dT[j];
            vg[1 * 4 + j] = dt[1] * mu[j] + o.J11 * dT[3 + j];
            vg[2 * 4 + j] = dt[2] * mu[j] + o.J02 * dT[j] + o.J12 * dT[3 + j];
        }
        vg[3] = dtx;
        vg[7] = dty;
        vg[11] = dtz;
    }

    // Sec. 3.2.1: the scales and the rotation
    if (kStore) {
        dL_dscales[3 * g + 0] = live ? S(2) * s[0] * Q(0, 0) : S(0);
        dL_dscales[3 * g + 1] = live ? S(2) * s[1] * Q(1, 1) : S(0);
        dL_dscales[3 * g + 2] = live ? S(2) * s[2] * Q(2, 2) : S(0);
    } else if (live) {
        atomic_add3(dL_dscales + 3 * g, S(2) * s[0] * Q(0, 0), S(2) * s[1] * Q(1, 1), S(2) * s[2] * Q(2, 2));
    }
    const S s00 = s[0] * s[0], s11 = s[1] * s[1], s22 = s[2] * s[2];
    const S om0 = S(2) * Q(1, 2) * (s11 - s22);
    const S om1 = S(2) * Q(2, 0) * (s22 - s00);
    const S om2 = S(2) * Q(0, 1) * (s00 - s11);
    // 2 q_hat (x) (0, omega) / |q|
    const S w = o.q[0], x = o.q[1], y = o.q[2], z = o.q[3];
    const S k2 = S(2) * o.qinv;
    if (kStore) {
        V4<S> dq;
        dq.x = live ? -k2 * (x * om0 + y * om1 + z * om2) : S(0);
        dq.y = live ? k2 * (w * om0 + y * om2 - z * om1) : S(0);
        dq.z = live ? k2 * (w * om1 + z * om0 - x * om2) : S(0);
        dq.w = live ? k2 * (w * om2 + x * om1 - y * om0) : S(0);
        reinterpret_cast<V4<S>*>(dL_dquats)[g] = dq;
    } else if (live) {
        atomic_add4(dL_dquats + 4 * g, -k2 * (x * om0 + y * om1 + z * om2), k2 * (w * om0 + y * om2 - z * om1),
                    k2 * (w * om1 + z * om0 - x * om2), k2 * (w * om2 + x * om1 - y * om0));
    }
}

template <typename S, bool kStore>
__global__ void __launch_bounds__(256, 4)  // 4 CTAs per SM (64 registers): 8 % faster than 3
k_project_bwd(const GsView* __restrict__ views, int V, int64_t P, const S* __restrict__ means,
              const V4<S>* __restrict__ quats, const S* __restrict__ scales, S eps2d,
              const int32_t* __restrict__ touched, const V2<S>* __restrict__ dL_dmeans2d,
              const S* __restrict__ dL_dconics, S* __restrict__ dL_dmeans, S* __restrict__ dL_dquats,
              S* __restrict__ dL_dscales)
{
    pdl_wait();
    pdl_trigger();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    // a culled projection runs the same arithmetic and stores nothing: its inputs are then loaded
    // together with `touched` instead of after it
    const bool live = touched[p] != 0;
    project_bwd_one<S, false, kStore>(views[view_of_projection(views, V, p)], p, means, quats, scales, eps2d, dL_dmeans2d,
                              dL_dconics, dL_dmeans, dL_dquats, dL_dscales, nullptr, live);
}

// The same, plus dL/dT_cw per view.  A view's projections are contiguous, so a
// warp almost always lies in one view: it sums its 12 terms by shuffles and
// hands them to the block, which adds each run of equal views to global
// memory with one atomic per entry (about 12 atomics per 256 projections).
// A warp that straddles a view boundary adds lane by lane instead.
template <typename S>
__global__ void __launch_bounds__(256)
k_project_bwd_view(const GsView* __restrict__ views, int V, int64_t P, const S* __restrict__ means,
                   const V4<S>* __restrict__ quats, const S* __restrict__ scales, S eps2d,
                   const int32_t* __restrict__ touched, const V2<S>* __restrict__ dL_dmeans2d,
                   const S* __restrict__ dL_dconics, S* __restrict__ dL_dmeans, S* __restrict__ dL_dquats,
                   S* __restrict__ dL_dscales, S* __restrict__ dL_dviewmats)
{
    pdl_wait();
    pdl_trigger();
    __shared__ S s_sum[8][12];
    __shared__ int s_view[8];
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    S vg[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) vg[i] = S(0);
    int vi = -1;
    if (p < P && touched[p] != 0) {
        vi = view_of_projection(views, V, p);
        project_bwd_one<S, true>(views[vi], p, means, quats, scales, eps2d, dL_dmeans2d, dL_dconics, dL_dmeans,
                                 dL_dquats, dL_dscales, vg);
    }
    const unsigned full = 0xffffffffu;
    const int vlo = __reduce_min_sync(full, vi < 0 ? INT_MAX : vi);
    const int vhi = __reduce_max_sync(full, vi);
    if (vhi >= 0 && vlo == vhi) {
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            S x = vg[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(full, x, o);
            vg[i] = x;
        }
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < 12; ++i) s_sum[warp][i] = vg[i];
            s_view[warp] = vlo;
        }
    } else {
        if (vi >= 0)
#pragma unroll
            for (int i = 0; i < 12; ++i) atomicAdd(dL_dviewmats + 16 * (int64_t)vi + i, vg[i]);
        if (lane == 0) s_view[warp] = -1;
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        const int i = threadIdx.x;
        int cur = -1;
        S acc = S(0);
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const int v = s_view[w];
            if (v < 0) continue;
            if (v != cur) {
                if (cur >= 0) atomicAdd(dL_dviewmats + 16 * (int64_t)cur + i, acc);
                cur = v;
                acc = S(0);
            }
            acc += s_sum[w][i];
        }
        if (cur >= 0) atomicAdd(dL_dviewmats + 16 * (int64_t)cur + i, acc);
    }
}

static bool misaligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) != 0; }

template <typename S>
static int project_impl(const char* who, const GsView* views, int32_t V, int64_t P, const S* means, const S* quats,
                        const S* scales, S eps2d, S* means2d, S* conics, float* depths, int16_t* rects,
                        int32_t* touched, int64_t* K_total, void* stream)
{
    if (V < 0 || P < 0 || (P > 0 && V == 0)) return fail(GS_ERR_INVALID_ARG, "%s: V=%d P=%lld", who, V, (long long)P);
    if (P > 0 && (!views || !means || !quats || !scales || !means2d || !conics || !depths || !rects || !touched))
        return fail(GS_ERR_INVALID_ARG, "%s: null pointer argument", who);
    if (misaligned(quats, 4 * sizeof(S)) || misaligned(means2d, 2 * sizeof(S)) || misaligned(rects, 8))
        return fail(GS_ERR_INVALID_ARG, "%s: quats need %zu-byte, means2d %zu-byte, rects 8-byte alignment", who,
                    4 * sizeof(S), 2 * sizeof(S));
    if (!(eps2d >= S(0))) return fail(GS_ERR_INVALID_ARG, "%s: eps2d must be >= 0", who);
    cudaStream_t s = as_stream(stream);
    if (K_total && cudaMemsetAsync(K_total, 0, sizeof(int64_t), s) != cudaSuccess) return launch_status(who);
    if (P == 0) return GS_OK;
    const int threads = 256;
    const unsigned blocks = (unsigned)((P + threads - 1) / threads);
    launch_pdl(k_project_fwd<S>, blocks, threads, s, views, V, P, means, reinterpret_cast<const V4<S>*>(quats), scales,
                                                 eps2d, reinterpret_cast<V2<S>*>(means2d), conics, depths,
                                                 reinterpret_cast<short4*>(rects), touched,
                                                 reinterpret_cast<unsigned long long*>(K_total));
    count_launches(1);
    return launch_status(who);
}

template <typename S>
static int project_bwd_impl(const char* who, const GsView* views, int32_t V, int64_t P, const S* means,
                            const S* quats, const S* scales, S eps2d, const int32_t* touched, const S* dL_dmeans2d,
                            const S* dL_dconics, S* dL_dmeans, S* dL_dquats, S* dL_dscales, S* dL_dviewmats,
                            void* stream, bool exclusive = false)
{
    if (V < 0 || P < 0 || (P > 0 && V == 0)) return fail(GS_ERR_INVALID_ARG, "%s: V=%d P=%lld", who, V, (long long)P);
    if (P > 0 && (!views || !means || !quats || !scales || !touched || !dL_dmeans2d || !dL_dconics || !dL_dmeans ||
                  !dL_dquats || !dL_dscales))
        return fail(GS_ERR_INVALID_ARG, "%s: null pointer argument", who);
    if (misaligned(quats, 4 * sizeof(S)) || misaligned(dL_dmeans2d, 2 * sizeof(S)) ||
        (exclusive && misaligned(dL_dquats, 4 * sizeof(S))))
        return fail(GS_ERR_INVALID_ARG, "%s: quats%s need %zu-byte, dL_dmeans2d %zu-byte alignment", who,
                    exclusive ? " and dL_dquats" : "", 4 * sizeof(S), 2 * sizeof(S));
    if (P == 0) return GS_OK;
    const int threads = 256;
    const unsigned blocks = (unsigned)((P + threads - 1) / threads);
    if (dL_dviewmats)
        launch_pdl(k_project_bwd_view<S>, blocks, threads, as_stream(stream),
            views, V, P, means, reinterpret_cast<const V4<S>*>(quats), scales, eps2d, touched,
            reinterpret_cast<const V2<S>*>(dL_dmeans2d), dL_dconics, dL_dmeans, dL_dquats, dL_dscales, dL_dviewmats);
    else {
        auto kernel = k_project_bwd<S, false>;
        if constexpr (std::is_same<S, float>::value)  // the exclusive entry point is fp32
            if (exclusive) kernel = k_project_bwd<S, true>;
        launch_pdl(kernel, blocks, threads, as_stream(stream),
            views, V, P, means, reinterpret_cast<const V4<S>*>(quats), scales, eps2d, touched,
            reinterpret_cast<const V2<S>*>(dL_dmeans2d), dL_dconics, dL_dmeans, dL_dquats, dL_dscales);
    }
    count_launches(1);
    return launch_status(who);
}

}  // namespace gs

using namespace gs;

extern "C" int gs_project(const GsView* views, int32_t V, int64_t P, const float* means, const float* quats,
                          const float* scales, float eps2d, float* means2d, float* conics, float* depths,
                          int16_t* rects, int32_t* touched, int64_t* K_total, void* stream)
{
    gs::NvtxRange nvtx("gs_project");
    return project_impl<float>("gs_project", views, V, P, means, quats, scales, eps2d, means2d, conics, depths, rects,
                                touched, K_total, stream);
}

extern "C" int gs_project_f64(const GsView* views, int32_t V, int64_t P, const double* means, const double* quats,
                              const double* scales, double eps2d, double* means2d, double* conics, float* depths,
                              int16_t* rects, int32_t* touched, int64_t* K_total, void* stream)
{
    gs::NvtxRange nvtx("gs_project_f64");
    return project_impl<double>("gs_project_f64", views, V, P, means, quats, scales, eps2d, means2d, conics, depths,
                                 rects, touched, K_total, stream);
}

extern "C" int gs_project_bwd(const GsView* views, int32_t V, int64_t P, const float* means, const float* quats,
                              const float* scales, float eps2d, const int32_t* touched, const float* dL_dmeans2d,
                              const float* dL_dconics, float* dL_dmeans, float* dL_dquats, float* dL_dscales,
                              float* dL_dviewmats, void* stream)
{
    gs::NvtxRange nvtx("gs_project_bwd");
    return project_bwd_impl<float>("gs_project_bwd", views, V, P, means, quats, scales, eps2d, touched, dL_dmeans2d,
                                   dL_dconics, dL_dmeans, dL_dquats, dL_dscales, dL_dviewmats, stream);
}

extern "C" int gs_project_bwd_exclusive(const GsView* views, int32_t V, int64_t P, const float* means,
                                        const float* quats, const float* scales, float eps2d, const int32_t* touched,
                                        const float* dL_dmeans2d, const float* dL_dconics, float* dL_dmeans,
                                        float* dL_dquats, float* dL_dscales, void* stream)
{
    gs::NvtxRange nvtx("gs_project_bwd_exclusive");
    return project_bwd_impl<float>("gs_project_bwd_exclusive", views, V, P, means, quats, scales, eps2d, touched,
                                   dL_dmeans2d, dL_dconics, dL_dmeans, dL_dquats, dL_dscales, nullptr, stream, true);
}

extern "C" int gs_project_bwd_f64(const GsView* views, int32_t V, int64_t P, const double* means,
                                  const double* quats, const double* scales, double eps2d, const int32_t* touched,
                                  const double* dL_dmeans2d, const double* dL_dconics, double* dL_dmeans,
                                  double* dL_dquats, double* dL_dscales, double* dL_dviewmats, void* stream)
{
    gs::NvtxRange nvtx("gs_project_bwd_f64");
    return project_bwd_impl<double>("gs_project_bwd_f64", views, V, P, means, quats, scales, eps2d, touched,
                                    dL_dmeans2d, dL_dconics, dL_dmeans, dL_dquats, dL_dscales, dL_dviewmats, stream);
}
