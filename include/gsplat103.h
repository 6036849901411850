/*
 * gsplat103.h -- C ABI of a GB300 (sm_103a) differentiable 3D Gaussian-splatting
 * rasteriser, after "Mathematical Supplement for the gsplat Library"
 * (Ye & Kanazawa, arXiv 2312.02121).  The paper exposes each stage of the
 * forward and backward pass on its own (Sec. 1, Sec. 4); so does this ABI:
 *
 *   gs_project        Sec. 2.1, Eq. 1-6, plus the 3-sigma tile box of Sec. 2.2
 *   gs_bin_and_sort   Sec. 2.2: 16x16 tile binning and per-tile depth order
 *   gs_rasterize_fwd  Sec. 2.2, Eq. 7: front-to-back compositing
 *   gs_rasterize_bwd  Sec. 3.1: compositing gradients
 *   gs_project_bwd    Sec. 3.2, 3.2.1: projection, scale and rotation gradients
 *   gs_autotune       the tile walk and batch shape of the compositing stages
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns GS_OK (0) or a GS_ERR_* code; gs_last_error()
 *    gives a message for the calling thread's last failure.  Argument errors
 *    are detected on the host before anything is launched: null required
 *    pointers, negative or oversized counts, too small a workspace, and the
 *    alignment of the vector-typed arrays and workspaces named below.  The
 *    natural alignment of the scalar arrays is the caller's duty and is not
 *    checked (a tensor whose storage offset counts whole elements has it).
 *  - All array arguments are caller-owned DEVICE memory (plain pointers), fp32
 *    unless stated, C-contiguous, 4-byte aligned at least; float2/short4 data
 *    (means2d, rects) must be 8-byte aligned and quaternions 16-byte aligned.
 *    The library never allocates or frees memory and never synchronises: all
 *    work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and the call returns before it completes.  Results are only
 *    valid after the caller synchronises the stream.
 *  - Calls enqueue only kernels and cudaMemsetAsync, so a sequence of them can
 *    be captured into a CUDA graph when the sizes (P, T_total, K_capacity) are
 *    fixed.  (gs_bin_and_sort_static is not covered by this statement.)
 *  - Quaternions are stored (w, x, y, z) and need not be unit length; the
 *    forward normalises them.  Scales are linear (not log) and opacities are
 *    in [0, 1]; activations belong to the caller.
 *  - Thresholds: a Gaussian whose alpha at a pixel is below 1/255 is skipped,
 *    alpha is clamped to 0.99, and compositing stops before a Gaussian that
 *    would take the transmittance below 1e-4 (GS_ALPHA_MIN, GS_ALPHA_MAX,
 *    GS_T_MIN).  The paper fixes none of these values.
 *
 * Views and batches
 * -----------------
 * One call processes V views at once.  The parameter arrays (means, quats,
 * scales, opacities, colors) hold the Gaussians of every scene back to back;
 * view v renders the scene occupying Gaussians [g_begin, g_begin + g_count)
 * through its camera.  Its projected entries ("projections", one per
 * Gaussian of its scene) occupy [proj_offset, proj_offset + g_count) of the
 * per-projection arrays, its tiles the global tile ids
 * [tile_offset, tile_offset + tiles_x * tiles_y), and its pixels
 * [pixel_offset, pixel_offset + width * height) of the packed image buffers
 * (row-major inside a view).  A single view is a batch of one with all
 * offsets 0.  gs_views_layout() fills the offsets and tile counts on a host
 * copy; the `views` argument of the other entry points is a device copy of
 * that array (kernels read it), with views in increasing offset order.
 */
#ifndef GSPLAT103_H
#define GSPLAT103_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GS_OK 0
#define GS_ERR_INVALID_ARG 1
#define GS_ERR_CAPACITY 2
#define GS_ERR_TIMEOUT 3
#define GS_ERR_CUDA 4

#define GS_TILE 16            /* tile edge in pixels (Sec. 2.2: 16x16 tiles) */
#define GS_ALPHA_MIN (1.0f / 255.0f)
#define GS_ALPHA_MAX 0.99f
#define GS_T_MIN 1e-4f

/* bits of the device error word written by gs_bin_and_sort */
#define GS_FLAG_CAPACITY 1u   /* more intersections than K_capacity */

/* Camera of Sec. 2.1, Eq. 1: world-to-camera extrinsics T_cw = [R_cw t_cw; 0 1]
 * (R row-major) and pinhole intrinsics; pixel (x, y) has its centre at
 * (x + 0.5, y + 0.5).  A Gaussian is culled unless near < t_z < far.  80 bytes. */
typedef struct GsCamera {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    float near_plane, far_plane;
    int32_t width, height;
} GsCamera;

/* One view of a batch (see "Views and batches").  120 bytes. */
typedef struct GsView {
    GsCamera cam;
    int32_t g_begin;       /* first Gaussian of the rendered scene */
    int32_t g_count;       /* number of Gaussians of that scene */
    int64_t proj_offset;   /* first projection of this view */
    int64_t pixel_offset;  /* first pixel of this view in packed images */
    int32_t tile_offset;   /* first global tile id of this view */
    int32_t tiles_x;       /* ceil(width / 16) */
    int32_t tiles_y;       /* ceil(height / 16) */
    int32_t reserved;
} GsView;

/* Version of this ABI (major * 100 + minor). */
int gs_version(void);

/* Message describing the calling thread's last error ("" if none). */
const char* gs_last_error(void);

/* Number of CUDA kernels this library has enqueued since it was loaded
 * (all threads; a monotonic counter for instrumentation). */
int64_t gs_kernel_launches(void);

/*
 * Fills proj_offset, pixel_offset, tile_offset, tiles_x, tiles_y of views[0..V)
 * (host memory) from g_count and the camera sizes, in view order, and returns
 * the totals: *P_total projections, *T_total tiles, *pix_total pixels.
 * GS_ERR_INVALID_ARG on V < 0, non-positive image sizes, negative counts or
 * totals that overflow the 32-bit tile / projection index space.
 */
int gs_views_layout(GsView* views, int32_t V, int64_t* P_total, int32_t* T_total, int64_t* pix_total);

/*
 * Sec. 2.1 (Eq. 2-6) and the tile box of Sec. 2.2.  For every projection p of
 * every view: t = T_cw [mu; 1]; mu' = (fx t_x/t_z + cx, fy t_y/t_z + cy);
 * J of Eq. 3; R(q/|q|) of Eq. 5 (with R_11 = 1 - 2(x^2 + z^2), the orthonormal
 * form); Sigma = R S S^T R^T; Sigma' = J R_cw Sigma R_cw^T J^T + eps2d I;
 * the conic Y = Sigma'^-1; the tight box r = 3 (sqrt(Sigma'_00),
 * sqrt(Sigma'_11)) and its tile rectangle [floor((mu' - r)/16),
 * floor((mu' + r)/16) + 1) clamped to the tile grid.
 * A projection is culled (touched = 0, zero rect) when t_z <= near,
 * t_z >= far, det Sigma' <= 0, the rectangle is empty, or a value is not
 * finite.
 *
 * The conic is stored FACTORED, as (a, k, d) with
 *     sigma = 1/2 Delta^T Y Delta = 1/2 (a (Delta_x + k Delta_y)^2 + d Delta_y^2),
 * i.e. Y = [[a, a k], [a k, a k^2 + d]] (the LDL^T factors of Y):
 * a = Sigma'_11 / det Sigma', k = -Sigma'_01 / Sigma'_11, d = 1 / Sigma'_11.
 * The packed entries (Y_00, Y_01, Y_11) of a thin Gaussian lose the long
 * axis in fp32 (d = Y_11 - Y_01^2 / Y_00 cancels); the factors keep both axes
 * to full precision.  Sigma' is formed as A A^T + eps2d I from the images
 * A = J R_cw R S of the scaled axes, and det Sigma' by Cauchy-Binet (a sum of
 * non-negative terms), so no step cancels.
 *   in : views[V] (device), means[N,3], quats[N,4], scales[N,3]
 *   out: means2d[P,2], conics[P,3] = (a, k, d), depths[P] (t_z), rects[P,4]
 *        int16 (x0, y0, x1, y1 tile indices, half-open), touched[P] int32
 *        (tiles in the rectangle), K_total (device int64, nullable): set to
 *        the sum of touched (the intersection count).
 */
int gs_project(const GsView* views, int32_t V, int64_t P, const float* means, const float* quats,
               const float* scales, float eps2d, float* means2d, float* conics, float* depths,
               int16_t* rects, int32_t* touched, int64_t* K_total, void* stream);

/* Bytes of scratch gs_bin_and_sort needs for P projections, at most
 * K_capacity intersections and T_total tiles (256-byte aligned sub-buffers). */
size_t gs_bin_and_sort_workspace_size(int64_t P, int64_t K_capacity, int32_t T_total);

/*
 * Sec. 2.2: binning and per-tile depth order (the tile sort of Kerbl et al.,
 * App. C, realised as a depth sort of the projections followed by a stable
 * tile-id sort of the intersections).  Every projection p is paired with each
 * tile of its rectangle; the pairs are ordered by (global tile id, depth,
 * p) -- exactly, equal depths by p.
 *   in : views (device), P, T_total, rects, depths, touched (from gs_project),
 *        K_capacity (size of the isect arrays), workspace (device, >=
 *        gs_bin_and_sort_workspace_size bytes, 16-byte aligned, contents
 *        irrelevant)
 *   out: isect_ids[K_capacity]   projection of each sorted pair
 *        isect_pos[K_capacity]   sorted position of each pair in emission
 *                                order (the order p's pairs are generated:
 *                                pair j of p is emission emit_start[p] + j);
 *                                nullable -- only the deterministic
 *                                gs_rasterize_bwd reads it
 *        emit_start[P]           first emission index of each projection;
 *                                nullable unless isect_pos is given (it is
 *                                read only with it)
 *        tile_ranges[T_total,2]  [start, end) of each tile's sorted pairs
 *        K_out                   (device int32) number of pairs K
 *        flags                   (device uint32) GS_FLAG_CAPACITY is OR-ed in
 *                                when K > K_capacity; the outputs are then
 *                                incomplete but no write leaves its buffer.
 * Outputs past K are left untouched.  Needs P < 2^31 and K_capacity < 2^31.
 */
int gs_bin_and_sort(const GsView* views, int32_t V, int64_t P, int32_t T_total, const int16_t* rects,
                    const float* depths, const int32_t* touched, int64_t K_capacity, void* workspace,
                    size_t workspace_bytes, int32_t* isect_ids, int32_t* isect_pos, int32_t* emit_start,
                    int32_t* tile_ranges, int32_t* K_out, uint32_t* flags, void* stream);

/* Size limits of gs_bin_and_sort_static. */
#define GS_STATIC_MAX_PROJECTIONS 131072
#define GS_STATIC_MAX_INTERSECTIONS 1048576

/*
 * gs_bin_and_sort without a workspace argument, for callers that cannot
 * allocate device memory themselves: code that receives device pointers from a
 * host application that owns all allocations (a plugin, an embedded renderer)
 * and has no allocator of its own to call, or a real-time loop that must not
 * call cudaMalloc/cudaFree after start-up because they synchronise the device.
 * The paper has no counterpart; it is an interface convenience.
 *
 * The scratch gs_bin_and_sort needs lives in one fixed array in this
 * library's device memory (a file-scope __device__ array of 24 MiB =
 * 25,165,824 bytes), which every GPU that loads the library holds until the
 * process exits.  So:
 *  - P must be <= GS_STATIC_MAX_PROJECTIONS and K_capacity <=
 *    GS_STATIC_MAX_INTERSECTIONS; larger sizes return GS_ERR_INVALID_ARG.
 *  - All calls share that one array and it keeps the previous call's
 *    contents; nothing in it needs to start at zero (every kernel writes what
 *    it later reads).  Calls whose work overlaps on the GPU (different
 *    streams, or several host threads) race on it and give wrong results:
 *    serialise them, e.g. on one stream.
 *  - The first call on each device looks up the array's device address with
 *    cudaGetSymbolAddress while that device is current, and later calls reuse
 *    it; make that first call before any stream capture begins.  The address
 *    is kept for the life of the process: after a cudaDeviceReset it may be
 *    stale, so a process that resets a device must not call this entry point
 *    on that device again.
 * The call allocates nothing: no cudaMalloc, cudaFree or allocating library
 * routine.  Arguments and outputs are those of gs_bin_and_sort.
 */
int gs_bin_and_sort_static(const GsView* views, int32_t V, int64_t P, int32_t T_total, const int16_t* rects,
                           const float* depths, const int32_t* touched, int64_t K_capacity, int32_t* isect_ids,
                           int32_t* isect_pos, int32_t* emit_start, int32_t* tile_ranges, int32_t* K_out,
                           uint32_t* flags, void* stream);

/* How the two compositing kernels walk the tiles and the shape of the
 * backward's work (NULL or zeroed fields = defaults: one CTA per tile, in
 * tile id order, the default batch shape).  None of these choices changes
 * any result beyond the fp32 summation order of the fast backward's atomics;
 * in the deterministic mode the results are identical. */
typedef struct GsRasterConfig {
    int32_t persistent;         /* 1: a persistent grid pops tiles from a global queue */
    int32_t ctas_per_sm;        /* persistent grid = ctas_per_sm x SMs (<= 0: as many as fit) */
    const int32_t* tile_order;  /* device [T_total]: the order tiles are taken in (a permutation
                                   of tile ids, e.g. longest list first from gs_tile_order);
                                   NULL = tile id order */
    int32_t* queue;             /* device int32 counter the persistent grid pops from; required
                                   when persistent; the call zeroes it on its stream */
    uint32_t* warp_hits;        /* device [K_capacity] 32-bit words, nullable (up to 3-channel
                                   kernels): the forward records, for every chunk of 32 sorted
                                   pairs of a tile, which of them each of the tile's 8 warp boxes
                                   (8x4 pixels each) can be reached by (word w of the chunk holds
                                   box w's 32 bits), and the backward reads that instead of
                                   repeating the same test.  Give the backward the buffer the
                                   forward of the same frame filled; words the forward had no
                                   use for are left as they were. */
    int32_t bwd_pixels;         /* pixels per thread of gs_rasterize_bwd (fp32, up to 3 channels):
                                   0 = the default (GS_BWD_PIXELS_DEFAULT), 1 = one (8 warps per
                                   tile, each on an 8x4 box), 2 = two (4 warps, each on an 8x8 box:
                                   a Gaussian that reaches both 8x4 halves is reduced over the warp
                                   once for 64 pixels) */
    int32_t bwd_batch;          /* Gaussians per staged batch of gs_rasterize_bwd: 0 = the default
                                   for the pixel count; otherwise one of the compiled shapes -- 64 or
                                   96 with one pixel per thread, 64 or 128 with two.  The fp64 entry
                                   points ignore both fields (one pixel, batches of 32). */
} GsRasterConfig;

/* The backward's default pixels per thread. */
#define GS_BWD_PIXELS_DEFAULT 2

/* Bytes of scratch gs_tile_order needs for T_total tiles. */
size_t gs_tile_order_workspace_size(int32_t T_total);

/*
 * Orders the tiles by decreasing list length (end - start of tile_ranges,
 * clamped to 65535), ties by tile id: a longest-first queue for
 * GsRasterConfig.tile_order, so the longest tiles start first and the tail of
 * a launch is short.  order[T_total] receives tile ids.
 */
int gs_tile_order(const int32_t* tile_ranges, int32_t T_total, void* workspace, size_t workspace_bytes,
                  int32_t* order, void* stream);

/*
 * Sec. 2.2, Eq. 7: for every pixel of every view, walks its tile's sorted list
 * front to back: sigma = 1/2 Delta^T Y Delta with Delta = mu' - pixel centre,
 * alpha = min(0.99, o exp(-sigma)), skip alpha < 1/255 (and sigma < 0), stop
 * before T (1 - alpha) < 1e-4, C += c alpha T, T *= (1 - alpha).  Finally
 * C += T * background.
 *   in : views (device), T_total, means2d, conics (from gs_project),
 *        opacities[N], colors[N,3], isect_ids, tile_ranges (from
 *        gs_bin_and_sort), background[3] (device, nullable = black),
 *        config (host, nullable: how tiles are walked; see GsRasterConfig)
 *   out: out_rgb[pix,3], T_final[pix] (transmittance after the last
 *        composited Gaussian), last_idx[pix] int32 (sorted position of the last
 *        composited Gaussian; tile start - 1 when none), n_contrib[pix] int32
 *        (nullable: number of Gaussians composited into the pixel).
 */
int gs_rasterize_fwd(const GsView* views, int32_t V, int32_t T_total, const float* means2d,
                     const float* conics, const float* opacities, const float* colors,
                     const int32_t* isect_ids, const int32_t* tile_ranges, const float* background,
                     float* out_rgb, float* T_final, int32_t* last_idx, int32_t* n_contrib,
                     const GsRasterConfig* config, void* stream);

/*
 * gs_rasterize_fwd with the L2 loss of gs_l2_loss folded in (the paper has no
 * loss; this is the training step's common case).  Each pixel's colour C is
 * composited exactly as gs_rasterize_fwd does it and written to out_rgb; the
 * same kernel then reads target and writes dL_drgb = 2 inv_norm (C - target),
 * bit-identical to gs_l2_loss on the stored image, and adds inv_norm (C -
 * target)^2 to *loss (one atomic per CTA, so fp32 sums vary in the last bits
 * run to run).  Three channels, no contributor count.
 *   in : as gs_rasterize_fwd, plus target[pix,3] (device), inv_norm
 *   out: as gs_rasterize_fwd (n_contrib omitted), plus dL_drgb[pix,3] (device,
 *        nullable) and loss (device scalar, nullable, ACCUMULATED: the caller
 *        zeroes it); at least one of the two.
 */
int gs_rasterize_fwd_l2(const GsView* views, int32_t V, int32_t T_total, const float* means2d,
                        const float* conics, const float* opacities, const float* colors,
                        const int32_t* isect_ids, const int32_t* tile_ranges, const float* background,
                        float* out_rgb, float* T_final, int32_t* last_idx, const float* target,
                        float inv_norm, float* dL_drgb, float* loss, const GsRasterConfig* config,
                        void* stream);

/* Bytes of scratch gs_rasterize_bwd needs for K_capacity intersections:
 * 0 unless deterministic. */
size_t gs_rasterize_bwd_workspace_size(int64_t K_capacity, int32_t deterministic);

/*
 * Sec. 3.1: back to front from each pixel's last composited Gaussian,
 * rebuilding T_{n-1} = T_n / (1 - alpha_{n-1}) from the saved T_final and
 * S_{n-1} = c_n alpha_n T_n + S_n, with
 *   dC/dc_n = alpha_n T_n,
 *   dC/dalpha_n = c_n T_n - S_n/(1 - alpha_n) - background T_final/(1 - alpha_n),
 *   dalpha/do = exp(-sigma), dalpha/dsigma = -o exp(-sigma) (both 0 where the
 *   0.99 clamp was active), dsigma/dmu' = Y Delta, and for the factored conic
 *   (a, k, d) of gs_project, with u = Delta_x + k Delta_y,
 *   dsigma/d(a, k, d) = (u^2/2, a u Delta_y, Delta_y^2/2).
 * Per-pixel terms are first summed per (tile, Gaussian) inside each tile (warp
 * reduce-scatter, then a fixed-order sum over the tile's warps).  The tile sums
 * then reach the per-projection outputs in one of two ways:
 *   deterministic == 0: vector reduction atomics (fast; the fp32 order of the
 *     tile sums varies from run to run);
 *   deterministic != 0: written as records in workspace and summed per
 *     projection in emission order by a second kernel -- run-to-run identical
 *     for a single view (opacities/colors of a scene seen by several views are
 *     still summed over views with atomics).
 *   in : the forward's inputs and outputs, dL_drgb[pix,3], K_capacity,
 *        K (device int32 from gs_bin_and_sort), isect_pos, emit_start, touched
 *        (these four are read only when deterministic; may be NULL otherwise),
 *        workspace (>= gs_rasterize_bwd_workspace_size bytes)
 *   out (ACCUMULATED: += into caller-initialised buffers):
 *        dL_dmeans2d[P,2], dL_dconics[P,3] = dL/d(a, k, d) (per projection),
 *        dL_dopacities[N], dL_dcolors[N,3] (per Gaussian, summed over views).
 */
int gs_rasterize_bwd(const GsView* views, int32_t V, int64_t P, int32_t T_total, const float* means2d,
                     const float* conics, const float* opacities, const float* colors,
                     const int32_t* isect_ids, const int32_t* isect_pos, const int32_t* emit_start,
                     const int32_t* touched, const int32_t* tile_ranges, const int32_t* K,
                     int64_t K_capacity, const float* background, const float* T_final,
                     const int32_t* last_idx, const float* dL_drgb, int32_t deterministic, void* workspace,
                     size_t workspace_bytes, float* dL_dmeans2d, float* dL_dconics, float* dL_dopacities,
                     float* dL_dcolors, const GsRasterConfig* config, void* stream);

/*
 * Sec. 3.2 (Eq. 16-20) and 3.2.1: for every projection with touched > 0,
 * recomputes the forward and maps dL/dmu' and dL/dconic (w.r.t. the factored
 * conic (a, k, d) of gs_project) to
 *   dL/dSigma' (-Y G Y of Sec. 3.2 with G = dL/dY, written in the factors),
 *   dL/dSigma = T^T dL/dSigma' T with T = J R_cw, dL/dT, dL/dJ = dL/dT R_cw^T,
 *   dL/dt = J^T dL/dmu' + <dL/dJ, dJ/dt>, dL/dmu = R_cw^T dL/dt,
 *   dL/dM = 2 dL/dSigma M, dL/dR = dL/dM S, dL/ds = diag(R^T dL/dM),
 *   dL/dq from dL/dR through R(q/|q|) (Sec. 3.2.1; the kernel takes the
 *   equivalent route through the rotation about the Gaussian's own axes,
 *   which keeps fp32 precision for thin Gaussians).
 *   in : views, P, means, quats, scales, eps2d, touched, dL_dmeans2d,
 *        dL_dconics (dL/d(a, k, d))
 *   out (ACCUMULATED, summed over views): dL_dmeans[N,3], dL_dquats[N,4]
 *        (w.r.t. the raw quaternion), dL_dscales[N,3].
 *   out (optional, may be NULL; ACCUMULATED): dL_dviewmats[V,4,4], dL/dT_cw of
 *        each view, row-major, summed over the view's projections.  Eq. 20
 *        gives dL/dT_cw = dL/dt [mu; 1]^T, which follows T_cw through t only;
 *        because Sigma' = T Sigma T^T with T = J R_cw also depends on R_cw,
 *        the rotation block adds J^T dL/dT.  The 16 entries are treated as
 *        independent (the caller projects onto SE(3) if it wants a pose
 *        update); row 3 stays zero.  Asking for it selects a kernel variant
 *        that also reduces the 12 terms per view (one atomic per entry per
 *        256 projections), so fp32 results vary in the last bits run to run.
 */
int gs_project_bwd(const GsView* views, int32_t V, int64_t P, const float* means, const float* quats,
                   const float* scales, float eps2d, const int32_t* touched, const float* dL_dmeans2d,
                   const float* dL_dconics, float* dL_dmeans, float* dL_dquats, float* dL_dscales,
                   float* dL_dviewmats, void* stream);

/*
 * gs_project_bwd for batches in which every Gaussian has exactly one
 * projection: the views' Gaussian ranges [g_begin, g_begin + g_count) do not
 * overlap (one view, or views of distinct scenes).  The caller guarantees this
 * (the views live in device memory and are not read on the host).  The paper
 * has no counterpart; it saves the fill of the 3D gradients before the step.
 *   in : as gs_project_bwd (no view-matrix gradient)
 *   out (WRITTEN, not accumulated): dL_dmeans[N,3], dL_dquats[N,4] (16-byte
 *        aligned), dL_dscales[N,3] of every Gaussian of the views -- zeros for
 *        a culled projection (touched == 0).  Gaussians outside every view are
 *        left untouched.  The values are those gs_project_bwd adds to zeroed
 *        outputs, bit for bit.
 */
int gs_project_bwd_exclusive(const GsView* views, int32_t V, int64_t P, const float* means, const float* quats,
                             const float* scales, float eps2d, const int32_t* touched, const float* dL_dmeans2d,
                             const float* dL_dconics, float* dL_dmeans, float* dL_dquats, float* dL_dscales,
                             void* stream);

/* One candidate of gs_autotune: a tile walk and a backward batch shape (the
 * GsRasterConfig fields the tuner chooses, plus the tile order).  24 bytes. */
typedef struct GsTuning {
    int32_t persistent;     /* GsRasterConfig.persistent */
    int32_t ctas_per_sm;    /* GsRasterConfig.ctas_per_sm */
    int32_t longest_first;  /* 1: tiles in gs_tile_order's longest-first order */
    int32_t bwd_pixels;     /* GsRasterConfig.bwd_pixels */
    int32_t bwd_batch;      /* GsRasterConfig.bwd_batch */
    float ms;               /* out: median device time of one compositing forward + backward, ms */
} GsTuning;

/* The built-in candidates of gs_autotune: *count receives how many there are
 * and out[0..min(count, capacity)) the candidates (out may be NULL when
 * capacity is 0): five tile walks (one CTA per tile in id order or longest
 * first; a persistent grid of as many CTAs as fit, 4 or 3 per SM, longest
 * first) times the four backward batch shapes. */
int gs_autotune_default_candidates(GsTuning* out, int32_t capacity, int32_t* count);

/* Bytes of scratch gs_autotune needs: a frame's images, per-pixel state and
 * gradients, the tile order and the ballot buffer (256-byte aligned parts). */
size_t gs_autotune_workspace_size(int64_t P, int64_t N, int32_t T_total, int64_t K_capacity, int64_t pixels);

/*
 * Picks how to composite a frame fastest.  The paper exposes each stage on its
 * own and fixes no launch shape; the tile size is not tuned, because it is part
 * of the result (Sec. 2.2: a Gaussian is composited in every pixel of every
 * tile its 3-sigma box touches).  For every candidate (NULL / n_candidates = 0:
 * the built-in ones) it runs gs_tile_order when longest_first, then
 * gs_rasterize_fwd and the fast gs_rasterize_bwd with that walk and batch shape
 * on `stream`: every candidate once to warm up, then `repeats` rounds that
 * time every candidate in turn with CUDA events (so a drift of the clocks
 * weighs on all of them alike), and records each one's median.  No candidate
 * changes any result.
 *   in : the frame as gs_project and gs_bin_and_sort left it: views (device),
 *        P projections, N Gaussians (the largest g_begin + g_count of the
 *        views), T_total tiles, pixels (total), means2d, conics, opacities,
 *        colors (3 channels), isect_ids, tile_ranges, K (device), K_capacity;
 *        workspace (device, >= gs_autotune_workspace_size bytes, 16-byte
 *        aligned, contents irrelevant)
 *   out: results[n] (host, nullable) every candidate with its time, *best
 *        (host) the fastest.
 * Unlike the other entry points it WAITS for the stream (it reads the event
 * times after each candidate), so it cannot be captured into a CUDA graph; it
 * creates and destroys two CUDA events and allocates no device memory.  An
 * invalid candidate (a batch shape that is not compiled) returns the error of
 * the compositing call it was given to.
 */
int gs_autotune(const GsView* views, int32_t V, int64_t P, int64_t N, int32_t T_total, int64_t pixels,
                const float* means2d, const float* conics, const float* opacities, const float* colors,
                const int32_t* isect_ids, const int32_t* tile_ranges, const int32_t* K, int64_t K_capacity,
                const GsTuning* candidates, int32_t n_candidates, int32_t repeats, void* workspace,
                size_t workspace_bytes, GsTuning* results, GsTuning* best, void* stream);

/*
 * Sec. 2.2 (Eq. 7) and Sec. 3.1 for C channels per Gaussian (features, depth
 * as a channel, ...): Eq. 7 composites every channel with the same alpha and
 * T, and Sec. 3.1 derives every gradient term per channel, with dL/dalpha
 * summed over the channels.  Arguments are those of gs_rasterize_fwd /
 * gs_rasterize_bwd (fast mode) with colors[N,C], background[C] (nullable),
 * out[pixels,C], dL_dout[pixels,C] and dL_dcolors[N,C]; T_final, last_idx and
 * n_contrib as there.  C <= 3 runs the kernels of gs_rasterize_fwd /
 * gs_rasterize_bwd with a channel stride of C (missing channels count as zero
 * colour and zero dL/dC, which adds nothing), GsRasterConfig.warp_hits
 * included.  Larger C are composited in chunks of up to 32 channels on
 * kernels with a lane per channel (these ignore warp_hits): every chunk
 * rebuilds the same alpha and T, and the backward adds every chunk's share
 * with atomics.  Either way the backward's fp32 sums vary in the last bits run to
 * run (the deterministic mode is gs_rasterize_bwd's).  Outputs of the
 * backward are ACCUMULATED (the caller zeroes them).
 */
int gs_rasterize_fwd_nc(const GsView* views, int32_t V, int32_t T_total, int32_t C, const float* means2d,
                        const float* conics, const float* opacities, const float* colors, const int32_t* isect_ids,
                        const int32_t* tile_ranges, const float* background, float* out, float* T_final,
                        int32_t* last_idx, int32_t* n_contrib, const GsRasterConfig* config, void* stream);

int gs_rasterize_bwd_nc(const GsView* views, int32_t V, int64_t P, int32_t T_total, int32_t C,
                        const float* means2d, const float* conics, const float* opacities, const float* colors,
                        const int32_t* isect_ids, const int32_t* tile_ranges, const float* background,
                        const float* T_final, const int32_t* last_idx, const float* dL_dout, float* dL_dmeans2d,
                        float* dL_dconics, float* dL_dopacities, float* dL_dcolors, const GsRasterConfig* config,
                        void* stream);

/*
 * Training-step helpers (the paper has no counterpart: it derives gradients
 * only).  They let a whole optimisation step -- forward, loss, backward,
 * update -- run on the GPU and be captured into one CUDA graph.
 *
 * gs_l2_loss: L = inv_norm * sum_i (rgb_i - target_i)^2 over n scalars and
 * its gradient dL/drgb_i = 2 inv_norm (rgb_i - target_i), the dL/dC that
 * gs_rasterize_bwd takes.  For the mean over all pixels and channels pass
 * inv_norm = 1 / n.
 *   in : rgb[n], target[n]
 *   out: dL_drgb[n] (nullable), loss (device scalar, nullable; ACCUMULATED:
 *        the caller zeroes it; blocks add with atomics, so fp32 sums vary in
 *        the last bits run to run).  At least one output must be given.
 */
int gs_l2_loss(const float* rgb, const float* target, int64_t n, float inv_norm, float* dL_drgb, float* loss,
               void* stream);
int gs_l2_loss_f64(const double* rgb, const double* target, int64_t n, double inv_norm, double* dL_drgb,
                   double* loss, void* stream);

/* Adam hyper-parameters: one learning rate per parameter group (means,
 * quaternions, log-scales, opacity logits, colours), the moment decay rates
 * and the denominator offset. */
typedef struct GsAdamConfig {
    float lr[5];
    float beta1, beta2, eps;
} GsAdamConfig;

/* Bytes of optimiser state for N Gaussians of C colour channels (a 256-byte
 * header holding the step count, then the first and second moments, 11 + C
 * floats per Gaussian each). */
size_t gs_adam_state_size(int64_t N, int32_t C);

/*
 * One Adam step (Kingma & Ba, bias-corrected) on the raw parameters of N
 * Gaussians, in place: means[N,3], quats[N,4] (raw; the renderer normalises
 * them), log_scales[N,3], opacity_logits[N], colors[N,C].  The gradients are
 * those of the projection and compositing backward, i.e. with respect to the
 * ACTIVATED values scale = exp(log-scale) and opacity = sigmoid(logit); the
 * step chains them through the activations using scales[N,3] and
 * opacities[N] (the activated values the forward used) and then rewrites
 * scales and opacities from the updated raw values, ready for the next
 * forward.  `state` (gs_adam_state_size bytes, device) must be zeroed before
 * the first step; the step count lives in it, so repeated launches (or graph
 * replays) advance the bias correction.  When skip_if_set (device int32,
 * nullable) is non-zero at run time -- e.g. the flags of gs_bin_and_sort after
 * an intersection overflow made the gradients incomplete -- the step changes
 * nothing, not even the step count.  Two kernels are enqueued.
 */
int gs_adam_step(int64_t N, int32_t C, const GsAdamConfig* cfg, void* state, size_t state_bytes, float* means,
                 float* quats,
                 float* log_scales, float* opacity_logits, float* colors, const float* dL_dmeans,
                 const float* dL_dquats, const float* dL_dscales, const float* dL_dopacities,
                 const float* dL_dcolors, float* scales, float* opacities, const int32_t* skip_if_set,
                 void* stream);

/* scales = exp(log_scales) [N,3], opacities = sigmoid(opacity_logits) [N]. */
int gs_activate(int64_t N, const float* log_scales, const float* opacity_logits, float* scales, float* opacities,
                void* stream);

/*
 * FP64 instantiations of the four arithmetic stages, for checking the analytic
 * backward of Sec. 3 against finite differences (e.g. torch.autograd.gradcheck)
 * and against an fp64 reference.  Arguments are those of the fp32 entry points
 * with double in place of float, except that depths stay fp32 (they are the
 * sort key of gs_bin_and_sort, which both precisions share).  Thresholds are
 * 1/255, 0.99 and 1e-4 in double.  The fp64 kernels use smaller batches and
 * are not tuned for speed.
 */
int gs_project_f64(const GsView* views, int32_t V, int64_t P, const double* means, const double* quats,
                   const double* scales, double eps2d, double* means2d, double* conics, float* depths,
                   int16_t* rects, int32_t* touched, int64_t* K_total, void* stream);

int gs_rasterize_fwd_f64(const GsView* views, int32_t V, int32_t T_total, const double* means2d,
                         const double* conics, const double* opacities, const double* colors,
                         const int32_t* isect_ids, const int32_t* tile_ranges, const double* background,
                         double* out_rgb, double* T_final, int32_t* last_idx, int32_t* n_contrib,
                         const GsRasterConfig* config, void* stream);

size_t gs_rasterize_bwd_f64_workspace_size(int64_t K_capacity, int32_t deterministic);

int gs_rasterize_bwd_f64(const GsView* views, int32_t V, int64_t P, int32_t T_total, const double* means2d,
                         const double* conics, const double* opacities, const double* colors,
                         const int32_t* isect_ids, const int32_t* isect_pos, const int32_t* emit_start,
                         const int32_t* touched, const int32_t* tile_ranges, const int32_t* K,
                         int64_t K_capacity, const double* background, const double* T_final,
                         const int32_t* last_idx, const double* dL_drgb, int32_t deterministic, void* workspace,
                         size_t workspace_bytes, double* dL_dmeans2d, double* dL_dconics, double* dL_dopacities,
                         double* dL_dcolors, const GsRasterConfig* config, void* stream);

int gs_project_bwd_f64(const GsView* views, int32_t V, int64_t P, const double* means, const double* quats,
                       const double* scales, double eps2d, const int32_t* touched, const double* dL_dmeans2d,
                       const double* dL_dconics, double* dL_dmeans, double* dL_dquats, double* dL_dscales,
                       double* dL_dviewmats, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GSPLAT103_H */
