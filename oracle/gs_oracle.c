/*
 * gs_oracle.c -- FP64 CPU oracle for differentiable 3D Gaussian splatting,
 * written from "Mathematical Supplement for the gsplat Library"
 * (Ye & Kanazawa, arXiv 2312.02121).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * constant table or helper with the CUDA library and includes nothing of it.
 *
 * Every function follows one passage of the paper, named in its comment:
 *   Sec. 2.1, Eq. 1-6    projection of a Gaussian (t, mu', J, R, Sigma, Sigma')
 *   Sec. 2.2, Eq. 7      tile binning, depth order and front-to-back compositing
 *   Sec. 3.1             compositing gradients (colour, alpha, opacity, sigma,
 *                        2D mean, conic)
 *   Sec. 3.2, Eq. 16-20  projection gradients (t, Sigma, T, J, mu)
 *   Sec. 3.2.1           scale and rotation gradients (M, R, S, q)
 *
 * Where the paper is silent, garbled or inconsistent the oracle takes one
 * fixed reading; each is marked "Reading Ox" below:
 *   O1  conic = closed-form 2x2 inverse of Sigma'; cull when t_z <= near,
 *       t_z >= far, det Sigma' <= 0, the tile rectangle is empty, or a value is
 *       not finite.
 *   O2  mu' = (fx t_x / t_z + cx, fy t_y / t_z + cy); pixel (px, py) has its
 *       centre at (px + 1/2, py + 1/2).  (The printed mu' of Eq. 2 mixes an
 *       NDC map with c_x; this reading is the one whose derivative is J of
 *       Eq. 3.)
 *   O3  quaternions are stored (w, x, y, z).
 *   O4  R_11 = 1 - 2(x^2 + z^2).  Eq. 5 prints 1 - 2(x^2 - z^2), which is not
 *       orthonormal; the printed dR/dz (entry (1,1) = -4z) fixes the sign.
 *   O5  the forward normalises q; the rotation Jacobians are applied at the
 *       unit quaternion and chained through the normalisation.
 *   O6  Delta = mu' - pixel centre, so that d sigma / d mu' = Y Delta holds as
 *       printed in Sec. 3.1.
 *   O7  alpha = min(ALPHA_MAX, o exp(-sigma)); a Gaussian is skipped unless
 *       o exp(-sigma) >= ALPHA_MIN (so a NaN opacity is skipped rather than
 *       clamped to ALPHA_MAX); compositing stops before a Gaussian whose
 *       T (1 - alpha) would fall below T_MIN (that Gaussian is not
 *       composited); sigma < 0 is skipped.  d alpha/d(o, sigma) = 0 where the
 *       clamp is active.  Background b adds T_final * b.
 *   O8  d mu' / d t_xyz = J and d mu' / d t_w = 0 (the printed 2x4 matrix
 *       of Eq. 17 is garbled).
 *   O9  the 3-sigma box is the tight axis-aligned box r_x = 3 sqrt(Sigma'_00),
 *       r_y = 3 sqrt(Sigma'_11); tile rectangle x in
 *       [clamp(floor((mu'_x - r_x)/16), 0, TX), clamp(floor((mu'_x + r_x)/16) + 1, 0, TX)),
 *       likewise y; Gaussian n is in the list of the tile of pixel p iff that
 *       tile lies in rect(n).
 *   O11 eps2d is added to the diagonal of Sigma' (a low-pass dilation; 0 gives
 *       the paper's Sigma' exactly).
 *   O12 equal depths are ordered by Gaussian index.
 *   O13 conics are packed (a, b, c) for Y = [[a, b], [b, c]]; the gradient of
 *       the packed b is dL/dY_01 + dL/dY_10.
 *   O14 dL/dT_cw.  Eq. 20 gives dL/dT_cw = (dL/dt) [mu; 1]^T, which follows
 *       T_cw through t only.  Sigma' = T Sigma T^T with T = J R_cw (Sec. 3.2)
 *       also depends on R_cw, so the 3x3 rotation block gains
 *       J^T dL/dT; the paper computes dL/dT but carries it only into J.
 *       The 16 entries are treated as independent (no SE(3) projection);
 *       the bottom row stays zero because d mu'/d t_w = 0 (O8) and
 *       dJ/dt_w = 0.
 *
 * All arithmetic is double precision.  OpenMP (when available) only splits
 * independent pixels or Gaussians across threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Reading O7: compositing thresholds. */
#define OR_ALPHA_MIN (1.0 / 255.0)
#define OR_ALPHA_MAX 0.99
#define OR_T_MIN 1e-4

/* Camera of Sec. 2.1: extrinsics T_cw = [R_cw t_cw; 0 1] (R row-major) and
 * intrinsics (fx, fy, cx, cy); near/far clipping planes; image size. */
typedef struct {
    double R[9];
    double t[3];
    double fx, fy, cx, cy;
    double near_plane, far_plane;
    int32_t width, height;
} or_camera;

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* small dense helpers (row-major)                                           */
/* ------------------------------------------------------------------------ */

/* C (m x n) = A (m x p) B (p x n) */
static void mm(const double* A, const double* B, double* C, int m, int p, int n)
{
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < p; ++k) s += A[i * p + k] * B[k * n + j];
            C[i * n + j] = s;
        }
}

/* B (n x m) = A^T for A (m x n) */
static void tr(const double* A, double* B, int m, int n)
{
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) B[j * m + i] = A[i * n + j];
}

/* Frobenius inner product <X, Y> = Tr(X^T Y), Sec. 3 (Eq. 8). */
static double fprod(const double* X, const double* Y, int count)
{
    double s = 0.0;
    for (int i = 0; i < count; ++i) s += X[i] * Y[i];
    return s;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.1 -- projection                                                    */
/* ------------------------------------------------------------------------ */

/* Eq. 5 (with Reading O4): rotation matrix of a unit quaternion q = (w,x,y,z). */
void or_quat_to_rotmat(const double* q, double* R)
{
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.0 - 2.0 * (y * y + z * z);
    R[1] = 2.0 * (x * y - w * z);
    R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);
    R[4] = 1.0 - 2.0 * (x * x + z * z);
    R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);
    R[7] = 2.0 * (y * z + w * x);
    R[8] = 1.0 - 2.0 * (x * x + y * y);
}

/* Sec. 3.2.1: dR/dw, dR/dx, dR/dy, dR/dz (each 3x3 row-major) at q = (w,x,y,z). */
void or_rotmat_jacobians(const double* q, double* dRdw, double* dRdx, double* dRdy, double* dRdz)
{
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    const double a[9] = {0, -z, y, z, 0, -x, -y, x, 0};
    const double b[9] = {0, y, z, y, -2 * x, -w, z, w, -2 * x};
    const double c[9] = {-2 * y, x, w, x, 0, z, -w, z, -2 * y};
    const double d[9] = {-2 * z, -w, x, w, -2 * z, y, x, y, 0};
    for (int i = 0; i < 9; ++i) {
        dRdw[i] = 2.0 * a[i];
        dRdx[i] = 2.0 * b[i];
        dRdy[i] = 2.0 * c[i];
        dRdz[i] = 2.0 * d[i];
    }
}

/* Eq. 6: Sigma = R S S^T R^T with S = diag(s), q normalised first (O5).
 * Also returns R and M = R S when the pointers are non-null. */
void or_covariance3d(const double* q_raw, const double* s, double* Sigma, double* R_out, double* M_out)
{
    double qn = sqrt(q_raw[0] * q_raw[0] + q_raw[1] * q_raw[1] + q_raw[2] * q_raw[2] + q_raw[3] * q_raw[3]);
    double q[4] = {q_raw[0] / qn, q_raw[1] / qn, q_raw[2] / qn, q_raw[3] / qn};
    double R[9], S[9] = {s[0], 0, 0, 0, s[1], 0, 0, 0, s[2]}, M[9], Mt[9];
    or_quat_to_rotmat(q, R);
    mm(R, S, M, 3, 3, 3);
    tr(M, Mt, 3, 3);
    mm(M, Mt, Sigma, 3, 3, 3);
    if (R_out) memcpy(R_out, R, sizeof(R));
    if (M_out) memcpy(M_out, M, sizeof(M));
}

/* Eq. 3: the EWA local-affine Jacobian J (2x3) at camera-space point t. */
void or_ewa_jacobian(const or_camera* cam, const double* t, double* J)
{
    const double tz = t[2], tz2 = t[2] * t[2];
    J[0] = cam->fx / tz;
    J[1] = 0.0;
    J[2] = -cam->fx * t[0] / tz2;
    J[3] = 0.0;
    J[4] = cam->fy / tz;
    J[5] = -cam->fy * t[1] / tz2;
}

/* Sec. 3.2: the printed dJ/dt_x, dJ/dt_y, dJ/dt_z (each 2x3, stacked into
 * out[18]); dJ/dt_w = 0. */
void or_ewa_jacobian_dt(const or_camera* cam, const double* t, double* out)
{
    const double tx = t[0], ty = t[1], tz = t[2];
    const double tz2 = tz * tz, tz3 = tz2 * tz;
    const double dJx[6] = {0, 0, -cam->fx / tz2, 0, 0, 0};
    const double dJy[6] = {0, 0, 0, 0, 0, -cam->fy / tz2};
    const double dJz[6] = {-cam->fx / tz2, 0, 2 * cam->fx * tx / tz3, 0, -cam->fy / tz2, 2 * cam->fy * ty / tz3};
    memcpy(out, dJx, sizeof(dJx));
    memcpy(out + 6, dJy, sizeof(dJy));
    memcpy(out + 12, dJz, sizeof(dJz));
}

/* Eq. 2 (Reading O2): camera-space point t and pixel-space mean mu'. */
void or_world_to_pixel(const or_camera* cam, const double* mu, double* t, double* mu2d)
{
    for (int i = 0; i < 3; ++i)
        t[i] = cam->R[3 * i + 0] * mu[0] + cam->R[3 * i + 1] * mu[1] + cam->R[3 * i + 2] * mu[2] + cam->t[i];
    mu2d[0] = cam->fx * t[0] / t[2] + cam->cx;
    mu2d[1] = cam->fy * t[1] / t[2] + cam->cy;
}

static int tiles_across(int pixels, int tile) { return (pixels + tile - 1) / tile; }

static int clampi(long v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : (int)v); }

/* Distance (pixels) from v to the nearest tile boundary k*tile, k in [0, ntiles]. */
static double boundary_margin(double v, int tile, int ntiles)
{
    double k = floor(v / tile + 0.5);
    if (k < 0) k = 0;
    if (k > ntiles) k = ntiles;
    return fabs(v - k * tile);
}

/*
 * Sec. 2.1 (Eq. 2-6) and Sec. 2.2 (3-sigma box, Readings O1, O9, O11):
 * projects N Gaussians into one camera.
 * Inputs : means[N,3], quats[N,4] (w,x,y,z), scales[N,3].
 * Outputs: means2d[N,2], cov2d[N,3] (Sigma'_00, Sigma'_01, Sigma'_11, with
 *          eps2d), conics[N,3] (a, b, c), depths[N] (t_z), rects[N,4]
 *          (x0, y0, x1, y1 tile indices, half-open), valid[N] (1 = kept),
 *          rect_margin[N] (pixels from the nearest tile boundary of the box
 *          edges; +inf when culled).  Any output pointer except valid may be NULL.
 */
void or_project(const or_camera* cam, int64_t N, const double* means, const double* quats,
                const double* scales, double eps2d, int32_t tile,
                double* means2d, double* cov2d, double* conics, double* depths,
                int32_t* rects, int32_t* valid, double* rect_margin)
{
    const int TX = tiles_across(cam->width, tile), TY = tiles_across(cam->height, tile);
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        double t[3], mu2d[2], J[6], Sigma[9], T[6], Tt[6], TS[6], cov[4];
        int ok = 1;
        or_world_to_pixel(cam, means + 3 * n, t, mu2d);
        or_ewa_jacobian(cam, t, J);
        or_covariance3d(quats + 4 * n, scales + 3 * n, Sigma, NULL, NULL);
        /* Eq. 4: Sigma' = J R_cw Sigma R_cw^T J^T (+ eps2d I, O11) */
        mm(J, cam->R, T, 2, 3, 3);
        tr(T, Tt, 2, 3);
        mm(T, Sigma, TS, 2, 3, 3);
        mm(TS, Tt, cov, 2, 3, 2);
        cov[0] += eps2d;
        cov[3] += eps2d;
        const double s00 = cov[0], s01 = 0.5 * (cov[1] + cov[2]), s11 = cov[3];
        const double det = s00 * s11 - s01 * s01;
        if (!(t[2] > cam->near_plane) || !(t[2] < cam->far_plane)) ok = 0;
        if (!(det > 0.0)) ok = 0;
        if (!isfinite(mu2d[0]) || !isfinite(mu2d[1]) || !isfinite(det)) ok = 0;
        double ca = 0, cb = 0, cc = 0;
        int32_t r4[4] = {0, 0, 0, 0};
        double margin = INFINITY;
        if (ok) {
            ca = s11 / det;
            cb = -s01 / det;
            cc = s00 / det;
            const double rx = 3.0 * sqrt(s00), ry = 3.0 * sqrt(s11);
            const double ex0 = mu2d[0] - rx, ex1 = mu2d[0] + rx;
            const double ey0 = mu2d[1] - ry, ey1 = mu2d[1] + ry;
            r4[0] = clampi((long)floor(ex0 / tile), 0, TX);
            r4[2] = clampi((long)floor(ex1 / tile) + 1, 0, TX);
            r4[1] = clampi((long)floor(ey0 / tile), 0, TY);
            r4[3] = clampi((long)floor(ey1 / tile) + 1, 0, TY);
            if (r4[0] >= r4[2] || r4[1] >= r4[3]) ok = 0;
            margin = fmin(fmin(boundary_margin(ex0, tile, TX), boundary_margin(ex1, tile, TX)),
                          fmin(boundary_margin(ey0, tile, TY), boundary_margin(ey1, tile, TY)));
        }
        if (!ok) {
            r4[0] = r4[1] = r4[2] = r4[3] = 0;
            margin = INFINITY;
        }
        valid[n] = ok;
        if (means2d) { means2d[2 * n] = mu2d[0]; means2d[2 * n + 1] = mu2d[1]; }
        if (cov2d) { cov2d[3 * n] = s00; cov2d[3 * n + 1] = s01; cov2d[3 * n + 2] = s11; }
        if (conics) { conics[3 * n] = ca; conics[3 * n + 1] = cb; conics[3 * n + 2] = cc; }
        if (depths) depths[n] = t[2];
        if (rects) memcpy(rects + 4 * n, r4, sizeof(r4));
        if (rect_margin) rect_margin[n] = margin;
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2 -- binning, depth order, compositing (Eq. 7)                      */
/* ------------------------------------------------------------------------ */

typedef struct { double depth; int64_t id; } depth_key;

static int cmp_depth_key(const void* a, const void* b)
{
    const depth_key* x = (const depth_key*)a;
    const depth_key* y = (const depth_key*)b;
    if (x->depth < y->depth) return -1;
    if (x->depth > y->depth) return 1;
    return (x->id > y->id) - (x->id < y->id); /* Reading O12 */
}

/* Valid Gaussians in (depth, index) order; returns their count. */
static int64_t depth_order(int64_t N, const double* depths, const int32_t* valid, int64_t* order)
{
    depth_key* keys = (depth_key*)malloc(sizeof(depth_key) * (N > 0 ? N : 1));
    int64_t m = 0;
    for (int64_t n = 0; n < N; ++n)
        if (valid[n]) { keys[m].depth = depths[n]; keys[m].id = n; ++m; }
    qsort(keys, (size_t)m, sizeof(depth_key), cmp_depth_key);
    for (int64_t i = 0; i < m; ++i) order[i] = keys[i].id;
    free(keys);
    return m;
}

/* Reading O9: does rect(n) contain tile (tx, ty)? */
static int rect_has_tile(const int32_t* r, int tx, int ty)
{
    return tx >= r[0] && tx < r[2] && ty >= r[1] && ty < r[3];
}

/* One compositing step of Eq. 7 for pixel centre (x, y) and Gaussian n.
 * Returns 0 = skipped, 1 = composited; *alpha / *g receive alpha and exp(-sigma),
 * *clamped whether alpha was clamped, *margin the smallest relative margin of
 * the threshold tests met here. */
static double sigma_of(const double* mu2d, const double* conic, double x, double y, double* dx, double* dy)
{
    *dx = mu2d[0] - x; /* Reading O6 */
    *dy = mu2d[1] - y;
    return 0.5 * (conic[0] * *dx * *dx + 2.0 * conic[1] * *dx * *dy + conic[2] * *dy * *dy);
}

typedef struct {
    int64_t id;
    double alpha, T, g; /* alpha_n, T_n (before n), exp(-sigma_n) */
    double dx, dy;
    int clamped;
} contrib;

/* Composites pixel (px, py) over the Gaussians of list[0..m) in order.
 * Fills out[] with the composited Gaussians (may be NULL), returns their count.
 * With depth_gap (and depths) it also reports the smallest relative depth
 * difference between consecutive Gaussians that pass the alpha test, up to
 * the one that stops the pixel: where it is tiny, a lower-precision depth key
 * may order them the other way (Readings O10, O12). */
static int64_t composite_pixel(int px, int py, const int64_t* list, int64_t m,
                               const double* means2d, const double* conics, const double* opac,
                               const double* colors, int nc, const double* bg,
                               double* rgb, double* T_final, int64_t* last_id, double* margin,
                               const double* depths, double* depth_gap, contrib* out)
{
    const double x = px + 0.5, y = py + 0.5; /* Reading O2: pixel centres */
    double T = 1.0, mg = INFINITY, gap = INFINITY, prev_depth = 0.0;
    int have_prev = 0;
    if (rgb)
        for (int k = 0; k < nc; ++k) rgb[k] = 0.0;
    int64_t last = -1, cnt = 0;
    for (int64_t i = 0; i < m; ++i) {
        const int64_t n = list[i];
        double dx, dy;
        const double sigma = sigma_of(means2d + 2 * n, conics + 3 * n, x, y, &dx, &dy);
        if (sigma < 0.0) continue;
        const double g = exp(-sigma);
        const double raw = opac[n] * g;
        const double alpha = raw < OR_ALPHA_MAX ? raw : OR_ALPHA_MAX;
        mg = fmin(mg, fabs(raw - OR_ALPHA_MIN) / OR_ALPHA_MIN);
        mg = fmin(mg, fabs(raw - OR_ALPHA_MAX) / OR_ALPHA_MAX);
        if (!(raw >= OR_ALPHA_MIN)) continue; /* O7: also skips a non-finite o e^-sigma */
        if (depth_gap) {
            const double d = depths[n];
            if (have_prev) gap = fmin(gap, fabs(d - prev_depth) / fmax(fabs(prev_depth), 1e-300));
            prev_depth = d;
            have_prev = 1;
        }
        const double Tn = T * (1.0 - alpha);
        mg = fmin(mg, fabs(Tn - OR_T_MIN) / OR_T_MIN);
        if (Tn < OR_T_MIN) break;
        if (rgb)
            for (int k = 0; k < nc; ++k) rgb[k] += colors[(int64_t)nc * n + k] * alpha * T;
        if (out) {
            out[cnt].id = n;
            out[cnt].alpha = alpha;
            out[cnt].T = T;
            out[cnt].g = g;
            out[cnt].dx = dx;
            out[cnt].dy = dy;
            out[cnt].clamped = raw >= OR_ALPHA_MAX;
        }
        T = Tn;
        last = n;
        ++cnt;
    }
    if (bg && rgb)
        for (int k = 0; k < nc; ++k) rgb[k] += T * bg[k];
    if (T_final) *T_final = T;
    if (last_id) *last_id = last;
    if (margin) *margin = mg;
    if (depth_gap) *depth_gap = gap;
    return cnt;
}

typedef struct { int64_t tile; int64_t pos; int64_t pix; } pix_key;

static int cmp_pix_key(const void* a, const void* b)
{
    const pix_key* x = (const pix_key*)a;
    const pix_key* y = (const pix_key*)b;
    if (x->tile != y->tile) return (x->tile > y->tile) - (x->tile < y->tile);
    return (x->pos > y->pos) - (x->pos < y->pos);
}

/* Groups the pixel list by tile (so that a tile's Gaussian list is built
 * once): groups[] holds (tile, position in the caller's list, pixel id) in
 * tile order; starts[g]..starts[g+1] delimit group g; returns the group count. */
static int64_t group_by_tile(int64_t npix, const int64_t* pix, int W, int tile, int TX,
                             pix_key* groups, int64_t* starts)
{
    for (int64_t i = 0; i < npix; ++i) {
        const int64_t p = pix[i];
        const int px = (int)(p % W), py = (int)(p / W);
        groups[i].pix = p;
        groups[i].pos = i;
        groups[i].tile = (int64_t)(py / tile) * TX + px / tile;
    }
    qsort(groups, (size_t)npix, sizeof(pix_key), cmp_pix_key);
    int64_t ng = 0;
    for (int64_t i = 0; i < npix; ++i)
        if (i == 0 || groups[i].tile != groups[i - 1].tile) starts[ng++] = i;
    starts[ng] = npix;
    return ng;
}

/* Sec. 2.2: the list of tile (tx, ty) -- valid Gaussians whose rectangle
 * contains it, in global depth order. */
static int64_t tile_list(const int64_t* order, int64_t m, const int32_t* rects, int tx, int ty, int64_t* list)
{
    int64_t k = 0;
    for (int64_t i = 0; i < m; ++i)
        if (rect_has_tile(rects + 4 * order[i], tx, ty)) list[k++] = order[i];
    return k;
}

/* Eq. 7 for one pixel, with its whole record: the composited Gaussians of the
 * tile list in order -- ids[c], alpha[c], T[c] (transmittance before each,
 * the running product) -- and the final transmittance.  Returns c.
 * Capacity of the output arrays: N. */
int64_t or_pixel_trace(int64_t N, const double* means2d, const double* conics, const double* opac,
                       const double* colors, int32_t nc, const double* depths, const int32_t* rects,
                       const int32_t* valid, int32_t tile, int32_t px, int32_t py,
                       int64_t* ids, double* alpha, double* T, double* T_final)
{
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (N > 0 ? N : 1));
    int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (N > 0 ? N : 1));
    contrib* cs = (contrib*)malloc(sizeof(contrib) * (N > 0 ? N : 1));
    const int64_t m = depth_order(N, depths, valid, order);
    const int64_t k = tile_list(order, m, rects, px / tile, py / tile, list);
    const int64_t c = composite_pixel(px, py, list, k, means2d, conics, opac, colors, nc, NULL,
                                      NULL, T_final, NULL, NULL, NULL, NULL, cs);
    for (int64_t j = 0; j < c; ++j) { ids[j] = cs[j].id; alpha[j] = cs[j].alpha; T[j] = cs[j].T; }
    free(order); free(list); free(cs);
    return c;
}

/*
 * Sec. 2.2, Eq. 7 (Readings O6, O7, O9, O12): front-to-back compositing of
 * nc channels (colors[N,nc]; Eq. 7 composites each channel alike).
 * Pixels rendered: pix[0..npix) (linear index y*W + x); pix == NULL means all
 * W*H pixels in order.  Outputs are indexed by position in that list:
 * rgb[npix,nc], T_final[npix], last_id[npix] (index of the last composited
 * Gaussian or -1), n_contrib[npix], margin[npix] (smallest relative margin
 * of any alpha/T threshold test met; +inf if none), depth_gap[npix] (may be
 * NULL: smallest relative depth difference between consecutive Gaussians that
 * pass the alpha test, up to the one that stops the pixel; +inf if fewer than
 * two).  bg (nc values) may be NULL.
 */
void or_rasterize(int64_t N, const double* means2d, const double* conics, const double* opac,
                  const double* colors, int32_t nc, const double* depths, const int32_t* rects,
                  const int32_t* valid, int32_t W, int32_t H, int32_t tile, const double* bg,
                  int64_t npix, const int64_t* pix,
                  double* rgb, double* T_final, int64_t* last_id, int64_t* n_contrib, double* margin,
                  double* depth_gap)
{
    const int TX = tiles_across(W, tile);
    int64_t* all = NULL;
    if (!pix) {
        npix = (int64_t)W * H;
        all = (int64_t*)malloc(sizeof(int64_t) * (npix > 0 ? npix : 1));
        for (int64_t i = 0; i < npix; ++i) all[i] = i;
        pix = all;
    }
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (N > 0 ? N : 1));
    const int64_t m = depth_order(N, depths, valid, order);
    pix_key* groups = (pix_key*)malloc(sizeof(pix_key) * (npix > 0 ? npix : 1));
    int64_t* starts = (int64_t*)malloc(sizeof(int64_t) * (npix + 1));
    const int64_t ng = group_by_tile(npix, pix, W, tile, TX, groups, starts);
#pragma omp parallel
    {
        int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (m > 0 ? m : 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t g = 0; g < ng; ++g) {
            const int64_t t = groups[starts[g]].tile;
            const int tx = (int)(t % TX), ty = (int)(t / TX);
            const int64_t k = tile_list(order, m, rects, tx, ty, list);
            for (int64_t i = starts[g]; i < starts[g + 1]; ++i) {
                const int64_t p = groups[i].pix, o = groups[i].pos;
                const int64_t c = composite_pixel((int)(p % W), (int)(p / W), list, k, means2d, conics, opac, colors, nc,
                                                  bg, rgb ? rgb + (int64_t)nc * o : NULL, T_final ? T_final + o : NULL,
                                                  last_id ? last_id + o : NULL, margin ? margin + o : NULL, depths,
                                                  depth_gap ? depth_gap + o : NULL, NULL);
                if (n_contrib) n_contrib[o] = c;
            }
        }
        free(list);
    }
    free(order); free(groups); free(starts); free(all);
}

/*
 * Sec. 3.1: gradients of L w.r.t. the 2D parameters, given dL/dC for the
 * pixels pix[0..npix) (dL_drgb[npix,nc], same order; pix == NULL = all).
 * Sec. 3.1 derives every term per channel k; dL/dalpha sums them over the nc
 * channels.
 * Written as the plain definition: for each pixel the composited Gaussians,
 * their T_n as the running product of Eq. 7 and S_n = sum_{m>n} c_m alpha_m T_m
 * as an explicit suffix sum, then
 *   dC/dc_n(k)     = alpha_n T_n
 *   dC(k)/dalpha_n = c_n(k) T_n - S_n(k)/(1 - alpha_n) - b(k) T_final/(1 - alpha_n)
 *   dalpha/do      = exp(-sigma),   dalpha/dsigma = -o exp(-sigma)   (0 if clamped)
 *   dsigma/dmu'    = Y Delta,       dsigma/dY = Delta Delta^T / 2   (packed: O13)
 * Outputs (accumulated, caller zeroes): dL_dmeans2d[N,2], dL_dconics[N,3],
 * dL_dopac[N], dL_dcolors[N,nc].
 */
void or_rasterize_bwd(int64_t N, const double* means2d, const double* conics, const double* opac,
                      const double* colors, int32_t nc, const double* depths, const int32_t* rects,
                      const int32_t* valid, int32_t W, int32_t H, int32_t tile, const double* bg,
                      int64_t npix, const int64_t* pix, const double* dL_drgb,
                      double* dL_dmeans2d, double* dL_dconics, double* dL_dopac, double* dL_dcolors)
{
    int64_t* all = NULL;
    if (!pix) {
        npix = (int64_t)W * H;
        all = (int64_t*)malloc(sizeof(int64_t) * (npix > 0 ? npix : 1));
        for (int64_t i = 0; i < npix; ++i) all[i] = i;
        pix = all;
    }
    const int TX = tiles_across(W, tile);
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (N > 0 ? N : 1));
    const int64_t m = depth_order(N, depths, valid, order);
    pix_key* groups = (pix_key*)malloc(sizeof(pix_key) * (npix > 0 ? npix : 1));
    int64_t* starts = (int64_t*)malloc(sizeof(int64_t) * (npix + 1));
    const int64_t ng = group_by_tile(npix, pix, W, tile, TX, groups, starts);
    const int nth = or_num_threads();
    /* one private accumulator per thread (6 geometry terms + nc colours per
     * Gaussian), summed in thread order at the end */
    const int64_t R = 6 + nc;
    double* acc = (double*)calloc((size_t)nth * (N > 0 ? N : 1) * R, sizeof(double));
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* my = acc + (size_t)tid * (N > 0 ? N : 1) * R;
        int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (m > 0 ? m : 1));
        contrib* cs = (contrib*)malloc(sizeof(contrib) * (m > 0 ? m : 1));
        double* S = (double*)malloc(sizeof(double) * nc * (m + 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t gi = 0; gi < ng; ++gi) {
            const int64_t tl = groups[starts[gi]].tile;
            const int64_t k = tile_list(order, m, rects, (int)(tl % TX), (int)(tl / TX), list);
            for (int64_t pi = starts[gi]; pi < starts[gi + 1]; ++pi) {
                const int64_t p = groups[pi].pix, i = groups[pi].pos;
                const int px = (int)(p % W), py = (int)(p / W);
                double Tf;
                const int64_t c = composite_pixel(px, py, list, k, means2d, conics, opac, colors, nc, bg,
                                                  NULL, &Tf, NULL, NULL, NULL, NULL, cs);
                const double* G = dL_drgb + (int64_t)nc * i;
                /* S_n as explicit suffix sums */
                for (int q = 0; q < nc; ++q) S[(int64_t)nc * c + q] = 0.0;
                for (int64_t j = c - 1; j >= 0; --j)
                    for (int q = 0; q < nc; ++q)
                        S[nc * j + q] = S[nc * (j + 1) + q] + colors[(int64_t)nc * cs[j].id + q] * cs[j].alpha * cs[j].T;
                for (int64_t j = 0; j < c; ++j) {
                    const contrib* e = cs + j;
                    const int64_t n = e->id;
                    double dL_dalpha = 0.0;
                    for (int q = 0; q < nc; ++q) {
                        double dC_dalpha = colors[(int64_t)nc * n + q] * e->T - S[nc * (j + 1) + q] / (1.0 - e->alpha);
                        if (bg) dC_dalpha -= bg[q] * Tf / (1.0 - e->alpha);
                        dL_dalpha += G[q] * dC_dalpha;
                        my[R * n + 6 + q] += G[q] * e->alpha * e->T;
                    }
                    if (e->clamped) continue;
                    const double dL_do = e->g * dL_dalpha;
                    const double dL_dsigma = -opac[n] * e->g * dL_dalpha;
                    const double* Y = conics + 3 * n;
                    my[R * n + 0] += dL_dsigma * (Y[0] * e->dx + Y[1] * e->dy);
                    my[R * n + 1] += dL_dsigma * (Y[1] * e->dx + Y[2] * e->dy);
                    my[R * n + 2] += dL_dsigma * 0.5 * e->dx * e->dx;
                    my[R * n + 3] += dL_dsigma * e->dx * e->dy;
                    my[R * n + 4] += dL_dsigma * 0.5 * e->dy * e->dy;
                    my[R * n + 5] += dL_do;
                }
            }
        }
        free(list); free(cs); free(S);
    }
    for (int t = 0; t < nth; ++t) {
        const double* my = acc + (size_t)t * (N > 0 ? N : 1) * R;
        for (int64_t n = 0; n < N; ++n) {
            dL_dmeans2d[2 * n + 0] += my[R * n + 0];
            dL_dmeans2d[2 * n + 1] += my[R * n + 1];
            dL_dconics[3 * n + 0] += my[R * n + 2];
            dL_dconics[3 * n + 1] += my[R * n + 3];
            dL_dconics[3 * n + 2] += my[R * n + 4];
            dL_dopac[n] += my[R * n + 5];
            for (int q = 0; q < nc; ++q) dL_dcolors[(int64_t)nc * n + q] += my[R * n + 6 + q];
        }
    }
    free(acc); free(order); free(groups); free(starts); free(all);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2 -- projection gradients                                          */
/* ------------------------------------------------------------------------ */

/*
 * Sec. 3.2 and 3.2.1 (Eq. 16-20, Readings O5, O8, O13): given dL/dmu'[N,2] and
 * dL/dconic[N,3] (packed), returns dL/dmu[N,3], dL/dq[N,4] (w.r.t. the raw,
 * unnormalised quaternion) and dL/ds[N,3].  Culled Gaussians (valid == 0) get 0.
 */
void or_project_bwd(const or_camera* cam, int64_t N, const double* means, const double* quats,
                    const double* scales, double eps2d, const int32_t* valid,
                    const double* dL_dmeans2d, const double* dL_dconics,
                    double* dL_dmeans, double* dL_dquats, double* dL_dscales, double* dL_dviewmat)
{
    (void)eps2d; /* d Sigma' / d Sigma does not depend on the dilation (O11) */
    /* per-Gaussian terms of dL/dT_cw (rows 0-2 of the 4x4), summed in index order below */
    double* vterm = dL_dviewmat ? (double*)calloc((size_t)(N > 0 ? N : 1) * 12, sizeof(double)) : NULL;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        double* gm = dL_dmeans + 3 * n;
        double* gq = dL_dquats + 4 * n;
        double* gs = dL_dscales + 3 * n;
        memset(gm, 0, 3 * sizeof(double));
        memset(gq, 0, 4 * sizeof(double));
        memset(gs, 0, 3 * sizeof(double));
        if (!valid[n]) continue;
        /* forward quantities, recomputed */
        double t[3], mu2d[2], J[6], Sigma[9], R[9], M[9], T[6], Tt[6], TS[6], cov[4];
        or_world_to_pixel(cam, means + 3 * n, t, mu2d);
        or_ewa_jacobian(cam, t, J);
        or_covariance3d(quats + 4 * n, scales + 3 * n, Sigma, R, M);
        mm(J, cam->R, T, 2, 3, 3);
        tr(T, Tt, 2, 3);
        mm(T, Sigma, TS, 2, 3, 3);
        mm(TS, Tt, cov, 2, 3, 2);
        cov[0] += eps2d;
        cov[3] += eps2d;
        const double s01 = 0.5 * (cov[1] + cov[2]);
        const double det = cov[0] * cov[3] - s01 * s01;
        const double Y[4] = {cov[3] / det, -s01 / det, -s01 / det, cov[0] / det};

        /* Sec. 3.1: G = dL/dY from the packed conic gradient (O13) */
        const double* gc = dL_dconics + 3 * n;
        const double GY[4] = {gc[0], 0.5 * gc[1], 0.5 * gc[1], gc[2]};
        /* dL/dSigma' = -Y^T G Y^T */
        double tmp[4], Gs[4], Yt[4];
        tr(Y, Yt, 2, 2);
        mm(Yt, GY, tmp, 2, 2, 2);
        mm(tmp, Yt, Gs, 2, 2, 2);
        for (int i = 0; i < 4; ++i) Gs[i] = -Gs[i];

        /* dL/dSigma = T^T (dL/dSigma') T */
        double TtG[6], GSig[9];
        mm(Tt, Gs, TtG, 3, 2, 2);
        mm(TtG, T, GSig, 3, 2, 3);

        /* dL/dT = G T Sigma^T + G^T T Sigma ; dL/dJ = dL/dT R_cw^T */
        double Gst[4], SigT[9], a1[6], a2[6], GT[6], Rcwt[9], GJ[6];
        tr(Gs, Gst, 2, 2);
        tr(Sigma, SigT, 3, 3);
        {
            double GsT[6], GstT[6];
            mm(Gs, T, GsT, 2, 2, 3);
            mm(GsT, SigT, a1, 2, 3, 3);
            mm(Gst, T, GstT, 2, 2, 3);
            mm(GstT, Sigma, a2, 2, 3, 3);
        }
        for (int i = 0; i < 6; ++i) GT[i] = a1[i] + a2[i];
        tr(cam->R, Rcwt, 3, 3);
        mm(GT, Rcwt, GJ, 2, 3, 3);

        /* dJ/dt_x, dJ/dt_y, dJ/dt_z as printed in Sec. 3.2 (dJ/dt_w = 0) */
        double dJ[18];
        or_ewa_jacobian_dt(cam, t, dJ);
        double gt[3] = {fprod(GJ, dJ, 6), fprod(GJ, dJ + 6, 6), fprod(GJ, dJ + 12, 6)};

        /* Eq. 16 with Reading O8: the 2D-mean term J^T dL/dmu' */
        const double* gmu2 = dL_dmeans2d + 2 * n;
        for (int i = 0; i < 3; ++i) gt[i] += J[i] * gmu2[0] + J[3 + i] * gmu2[1];

        /* Eq. 20: dL/dmu = R_cw^T dL/dt_xyz */
        for (int i = 0; i < 3; ++i)
            gm[i] = cam->R[0 * 3 + i] * gt[0] + cam->R[1 * 3 + i] * gt[1] + cam->R[2 * 3 + i] * gt[2];

        /* Eq. 20 with Reading O14: dL/dT_cw = (dL/dt) [mu; 1]^T, plus J^T dL/dT in the R_cw block */
        if (vterm) {
            double JtGT[9], Jt[6];
            tr(J, Jt, 2, 3);
            mm(Jt, GT, JtGT, 3, 2, 3);
            const double* mu = means + 3 * n;
            double* v = vterm + 12 * n;
            for (int i = 0; i < 3; ++i) {
                for (int j = 0; j < 3; ++j) v[4 * i + j] = gt[i] * mu[j] + JtGT[3 * i + j];
                v[4 * i + 3] = gt[i];
            }
        }

        /* Sec. 3.2.1: dL/dM = G M + G^T M ; dL/dR = dL/dM S^T ; dL/dS = R^T dL/dM */
        double GSt[9], GM1[9], GM2[9], GM[9], S[9] = {scales[3 * n], 0, 0, 0, scales[3 * n + 1], 0, 0, 0, scales[3 * n + 2]};
        double GR[9], GS[9], Rt[9];
        tr(GSig, GSt, 3, 3);
        mm(GSig, M, GM1, 3, 3, 3);
        mm(GSt, M, GM2, 3, 3, 3);
        for (int i = 0; i < 9; ++i) GM[i] = GM1[i] + GM2[i];
        mm(GM, S, GR, 3, 3, 3); /* S is diagonal: S^T = S */
        tr(R, Rt, 3, 3);
        mm(Rt, GM, GS, 3, 3, 3);
        gs[0] = GS[0];
        gs[1] = GS[4];
        gs[2] = GS[8];

        /* dL/dq_hat via the printed rotation Jacobians, then through q_hat = q/|q| (O5) */
        const double* qr = quats + 4 * n;
        const double qn = sqrt(qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]);
        const double qh[4] = {qr[0] / qn, qr[1] / qn, qr[2] / qn, qr[3] / qn};
        double dRw[9], dRx[9], dRy[9], dRz[9];
        or_rotmat_jacobians(qh, dRw, dRx, dRy, dRz);
        const double gqh[4] = {fprod(GR, dRw, 9), fprod(GR, dRx, 9), fprod(GR, dRy, 9), fprod(GR, dRz, 9)};
        const double dot = gqh[0] * qh[0] + gqh[1] * qh[1] + gqh[2] * qh[2] + gqh[3] * qh[3];
        for (int i = 0; i < 4; ++i) gq[i] = (gqh[i] - qh[i] * dot) / qn;
    }
    if (dL_dviewmat) {
        for (int i = 0; i < 16; ++i) dL_dviewmat[i] = 0.0;
        for (int64_t n = 0; n < N; ++n)
            for (int i = 0; i < 12; ++i) dL_dviewmat[i] += vterm[12 * n + i];
        free(vterm);
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2 -- brute-force binning for bit-exact list comparison              */
/* ------------------------------------------------------------------------ */

typedef struct { int64_t tile; float depth; int64_t id; } bin_key;

static int cmp_bin_key(const void* a, const void* b)
{
    const bin_key* x = (const bin_key*)a;
    const bin_key* y = (const bin_key*)b;
    if (x->tile != y->tile) return (x->tile > y->tile) - (x->tile < y->tile);
    if (x->depth < y->depth) return -1;
    if (x->depth > y->depth) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

/*
 * Sec. 2.2 (tile binning and per-tile depth sort) by brute force: every
 * (Gaussian, tile) pair of the TX x TY grid is tested against rect(n); the
 * pairs found are ordered by (tile, depth, index).  Takes the single-precision
 * depths and integer rectangles the caller supplies, so the result is exact
 * integer data.  rects[N,4] = (x0, y0, x1, y1); valid[N].
 * Writes ids[K] (Gaussian index per list entry, tile-major) and
 * ranges[TX*TY, 2] ([start, end) per tile) when non-null; returns K.
 * Call with ids == NULL first to learn K.
 */
int64_t or_bin(int64_t N, const int32_t* rects, const float* depths, const int32_t* valid,
               int32_t TX, int32_t TY, int64_t* ids, int64_t* ranges)
{
    int64_t K = 0;
    for (int64_t n = 0; n < N; ++n) {
        if (!valid[n]) continue;
        for (int ty = 0; ty < TY; ++ty)
            for (int tx = 0; tx < TX; ++tx)
                if (rect_has_tile(rects + 4 * n, tx, ty)) ++K;
    }
    if (!ids && !ranges) return K;
    bin_key* keys = (bin_key*)malloc(sizeof(bin_key) * (K > 0 ? K : 1));
    int64_t k = 0;
    for (int64_t n = 0; n < N; ++n) {
        if (!valid[n]) continue;
        for (int ty = 0; ty < TY; ++ty)
            for (int tx = 0; tx < TX; ++tx)
                if (rect_has_tile(rects + 4 * n, tx, ty)) {
                    keys[k].tile = (int64_t)ty * TX + tx;
                    keys[k].depth = depths[n];
                    keys[k].id = n;
                    ++k;
                }
    }
    qsort(keys, (size_t)K, sizeof(bin_key), cmp_bin_key);
    if (ids)
        for (int64_t i = 0; i < K; ++i) ids[i] = keys[i].id;
    if (ranges) {
        const int64_t nt = (int64_t)TX * TY;
        for (int64_t t = 0; t < nt; ++t) ranges[2 * t] = ranges[2 * t + 1] = 0;
        for (int64_t i = 0; i < K; ++i) {
            const int64_t t = keys[i].tile;
            if (i == 0 || keys[i - 1].tile != t) ranges[2 * t] = i;
            ranges[2 * t + 1] = i + 1;
        }
    }
    free(keys);
    return K;
}
