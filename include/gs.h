/*
 * gs.h -- C ABI of the GB300 (sm_103a) differentiable 3D-Gaussian-splatting mapping step.
 *
 * The step is the global Gaussian-map optimisation of RMGS-SLAM (arXiv 2604.12942, §III-C):
 * Gaussians + keyframe poses/intrinsics + target images -> rendered colour and depth, an
 * L1 photometric + depth loss, its gradients (to every Gaussian parameter and to each
 * keyframe's SE(3) pose) and a masked Adam update of the "visible and unfrozen" Gaussians.
 *
 * Conventions shared by every entry point
 *   - All tensor arguments are DEVICE pointers unless stated otherwise; the caller owns and
 *     allocates every buffer, including the workspace sized by gs_workspace_size().  The
 *     library never allocates device memory and never frees caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Every call
 *     is asynchronous on that stream; host-side argument errors are returned synchronously,
 *     device-side conditions (pair-capacity overflow, timeouts) are written to the status
 *     word of the workspace and read with gs_read_counters() after the stream is synced.
 *   - Camera arrays (gs_camera*, n_views = L->n_views entries) are HOST memory.  Their poses
 *     and intrinsics are copied into the workspace by each call (a by-value kernel argument,
 *     so calls can be captured in a CUDA graph); image sizes must match the layout's.
 *   - Gaussian parameters are structure-of-arrays float32 planes, each plane contiguous
 *     over the n Gaussians: means [3][n], log_scales [3][n], quats [4][n] (w, x, y, z,
 *     unnormalised), opacity_logits [n], sh [3K][n] with K = (sh_degree+1)^2 and plane
 *     k*3 + c holding SH coefficient k of colour channel c.
 *   - Images of the n_views views are packed one after another in view order; view v starts
 *     at pixel offset pix_off(v) = sum_{u<v} W_u H_u.  Colour is planar: channel c of view v
 *     is the W_v*H_v plane at rgb + 3*pix_off(v) + c*W_v*H_v.  Depth, T, masks: one plane
 *     per view at + pix_off(v).  Row-major, pixel (x, y) at y*W + x, sampled at its centre
 *     (x + 0.5, y + 0.5).
 *   - Functions return GS_OK or an error; gs_last_error() gives a message (thread-local).
 *
 * Readings of the paper's "standard differentiable Gaussian splatting" (§III-C), fixed by
 * gs_render_opts (defaults from gs_default_opts):
 *   alpha = min(alpha_max, o * exp(-q/2)), q = d^T Sigma'^-1 d; fragments with
 *   alpha < alpha_min are skipped; when T * (1 - alpha) < T_min the fragment is not added
 *   and the pixel stops.  C = sum_i c_i alpha_i T_i + T_final * bg, and depth
 *   D = sum_i z_i alpha_i T_i with the same weights (§III-C depth equation), z_i the
 *   camera-frame depth of the Gaussian centre.
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1,  /* bad pointer, size, view count, tile size, ... */
    GS_ERR_CUDA = 2,         /* a CUDA runtime call failed (message in gs_last_error) */
    GS_ERR_CAPACITY = 3,     /* more (tile, Gaussian) pairs than the workspace holds */
    GS_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
    GS_ERR_NONFINITE = 5,    /* a non-finite value was detected: a camera value (returned by
                                the call) or a Gaussian parameter (the projection sets the
                                status word; the later stages of the step then do nothing) */
    GS_ERR_UNSUPPORTED = 6   /* a valid request this build does not implement */
} gs_status;

#define GS_MAX_VIEWS 32
#define GS_MAX_SH_DEGREE 3

/* Pinhole keyframe camera.  R_cw, t_cw map world to camera (row-major): p_c = R_cw p + t_cw,
 * camera looking along +z with +x right and +y down; u = fx x/z + cx, v = fy y/z + cy. */
typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float R_cw[9];
    float t_cw[3];
} gs_camera;

/* The Gaussian map (§III-B: one Gaussian per LiDAR point with mean, log-space scale,
 * rotation quaternion, opacity and SH colour).  Device planes as described above. */
typedef struct {
    int64_t n;
    int32_t sh_degree;      /* 0..3 */
    float *means;           /* [3][n] */
    float *log_scales;      /* [3][n] */
    float *quats;           /* [4][n] */
    float *opacity_logits;  /* [n]    */
    float *sh;              /* [3K][n] */
} gs_gaussians;

/* Compositing constants, loss weights (§III-C total-loss equation, SSIM weight 0) and the
 * kernel shape.  tile: 8 or 16 (pixels per tile side); chunk: Gaussians staged per
 * shared-memory batch, one of 32, 64, 128, 256. */
typedef struct {
    float near_z;       /* cull if z <= near_z (default 0.2 m) */
    float dilation;     /* added to the 2-D covariance diagonal (default 0.3 px^2) */
    float alpha_min;    /* default 1/255 */
    float alpha_max;    /* default 0.99 */
    float T_min;        /* default 1e-4 */
    float clamp_fov;    /* x/z, y/z clamp inside the EWA Jacobian, x tan(half fov) (1.3) */
    float bg[3];        /* background colour (default black) */
    float lambda_rgb;   /* default 1 */
    float lambda_depth; /* default 0.1 */
    int32_t tile;       /* default 16 */
    int32_t chunk;      /* default 64 */
    int32_t count_fragments; /* 1: the compositing kernels fill the frag_* and visits_* counters
                                of gs_counters (a few percent slower); 0 (default): those
                                counters stay 0 */
    /* The rest of the §III-C objective (total-loss equation, SSIM term, interior mask):   */
    float lambda_ssim;       /* weight of 1 - SSIM over the mask (default 0: no SSIM term); a
                                workspace laid out with lambda_ssim > 0 holds its scratch */
    float mask_opacity;      /* M_geo = [1 - T_final >= mask_opacity] (default 0.5) */
    int32_t mask_erode;      /* >= 0: the step supervises inside M_int = Erode(M_geo, disk of this
                                radius, 0..16) of its own rendering, intersected with the caller's
                                mask; -1 (default): the caller's mask alone */
    /* Launch form of gs_step's compositing, backward and update stages (a9):                   */
    int32_t persistent;      /* 1: forward compositing, backward compositing, projection backward
                                and Adam run as ONE cooperative persistent kernel whose phases are
                                separated by bounded grid barriers (needs tile 16, chunk 256, the
                                fused L1 loss and optimize = 1; else gs_step returns
                                GS_ERR_UNSUPPORTED); 0 (default): one kernel per stage */
    int32_t sync_spin_limit; /* polls (about 0.1 us apart) before a grid-barrier wait gives up and
                                sets GS_ERR_TIMEOUT; 0 (default): 10,000,000 (about a second) */
    int32_t sync_skip_block; /* diagnostic: this block of the persistent kernel does not arrive at
                                its first grid barrier, so that the others' waits time out (tests
                                the bounded wait); -1 (default): none */
} gs_render_opts;

/* Byte offsets of the workspace regions (all 256-byte aligned) -- exposed so callers and
 * tests can inspect intermediate state; the layout is an implementation detail otherwise. */
typedef struct {
    size_t views;        /* internal per-view table */
    size_t counters;     /* gs_counters-compatible block: status, n_pairs, ... */
    size_t loss_acc;     /* double [GS_MAX_VIEWS][3] masked L1 colour / L1 depth / SSIM sums,
                            uint32 [GS_MAX_VIEWS][2] counts |M|, |M and D~ > 0| */
    size_t proj;         /* [n_views*n] records of 12 floats: (u, v, z, opacity),
                            (a, b, c, rx bits), (r, g, b, ry bits); (a, b, c) is the inverse
                            2-D covariance times -log2(e)/2, so alpha = o * 2^(a dx^2 +
                            2 b dx dy + c dy^2); rx, ry are the box half-extents (int32) */
    size_t vis_bits;     /* uint32 [n_views][ceil(n/32)]: bit i % 32 of word
                            v * ceil(n/32) + i / 32 is set when Gaussian i covers a tile of
                            view v (its record in proj is then valid); other bits are 0 */
    size_t scan_tmp;     /* uint32 scratch of the scans */
    size_t ekeys0, ekeys1; /* uint32 [n_views*n] ping-pong: bits(z) of the visible entries */
    size_t evals0, evals1; /* uint32 [n_views*n] ping-pong: their compact indices (positions
                              in `entries`); after gs_bin_sort evals0 lists the entries by depth */
    size_t keys0, keys1; /* uint32 [max_pairs] ping-pong: global tile id of each pair */
    size_t vals0, vals1; /* uint32 [max_pairs] ping-pong: view * n + Gaussian index; after
                            gs_bin_sort buffer sorted_buf holds the pairs ordered by (tile,
                            depth, view, index) */
    size_t pair_mask;    /* uint8 [max_pairs] per sorted pair: the 8x4-pixel warp regions of
                            its tile that hold pixels with alpha >= alpha_min (written by
                            gs_render_fwd, read by the backward) */
    size_t emit_tmp;     /* uint32 scratch of the pair emission */
    size_t sort_tmp;     /* uint32 scratch of the radix sorts */
    size_t ranges;       /* uint32 [total_tiles][2] [first, last+1) in the sorted pairs */
    size_t T_final;      /* float [total_pixels] */
    size_t n_contrib;    /* uint32 [total_pixels] tile-list position after the last added */
    size_t grad2d;       /* [n_views*n] records of 12 floats (screen-space gradient sums of
                            gs_composite_bwd); only the records of visible entries are defined */
    size_t geo2d;        /* [n_views*n] records of 12 floats: per visible entry, the gradients
                            w.r.t. the mean and the world covariance (projection backward);
                            before that, the binning's scratch (the depth-sorted entries' tile
                            rectangles and indices) */
    size_t dirgrad;      /* float [3][n]: per visible row, the gradient of the mean through the SH
                            view directions (projection backward: SH part -> geometry part) */
    size_t visible;      /* uint8 [n]: 1 if the Gaussian covers a tile of any view */
    size_t entries;      /* uint32 [n_views*n]: the visible entries in (view, Gaussian) order */
    size_t erect;        /* uint32 [n_views*n][2]: per visible entry, in the order of `entries`,
                            its tile rectangle (first global tile id, wx | wy << 16) */
    size_t tile_order;   /* uint32 [total_tiles]: compositing work order, largest pair count
                            first (power-of-two buckets), then scratch */
    size_t render_mask;  /* uint8 [total_pixels]: the step's interior mask (mask_erode >= 0) */
    size_t ssim_tmp;     /* float [9 * total_pixels] SSIM partials (only if has_ssim) */
    size_t total;        /* workspace bytes */
    int32_t has_ssim;    /* laid out with lambda_ssim > 0 */
    int32_t sorted_buf;  /* 0 or 1: which ping-pong buffer holds the sorted pairs */
    int32_t total_tiles;
    int64_t total_pixels;
    int64_t max_pairs;
    int64_t n;           /* Gaussians the workspace was laid out for */
    int32_t n_views;
    int32_t tile;
} gs_ws_layout;

/* Device-side counters copied back by gs_read_counters. */
typedef struct {
    uint32_t status;     /* gs_status of the device work since the last reset */
    uint32_t n_entries;  /* visible (view, Gaussian) entries of the last gs_bin_sort */
    uint64_t n_pairs;    /* (tile, Gaussian) pairs of the last gs_bin_sort */
    uint64_t adam_step;  /* Adam steps taken by gs_step / a captured graph */
    uint64_t frag_fwd_eval, frag_fwd_add;  /* (pixel, Gaussian) fragments tested / added by the */
    uint64_t frag_bwd_eval, frag_bwd_add;  /* forward and the backward compositing of the step  */
    uint32_t visits_fwd, visits_bwd;       /* (record, warp) pairs the compositing loops walked;
                                              these six only with opts.count_fragments = 1 */
} gs_counters;

/* Inputs and outputs of one batched step (gs_step / gs_graph_create).  Device pointers,
 * packed per view as for gs_render_fwd. */
typedef struct {
    const float *target_rgb;    /* [3*P] required */
    const float *target_depth;  /* [P] or NULL (no depth term) */
    const uint8_t *mask;        /* [P] or NULL (all pixels) */
    float *out_rgb, *out_depth; /* [3*P], [P] rendered colour and depth */
    float *dl_drgb, *dl_ddepth; /* [3*P], [P] dL/dC, dL/dD (dl_ddepth needed with target_depth) */
    float *loss_out;            /* [n_views + 1] per-view loss terms and their mean */
    float *grad_twist;          /* [n_views][6] or NULL; zeroed, then the pose gradients */
    const uint8_t *update_mask; /* [n] or NULL: rows allowed to change (unfrozen segments) */
    float lr[6];                /* means, log-scales, quats, opacity, SH DC, SH rest */
    float b1, b2, eps;
    int32_t optimize;           /* 0: stop after the backward (gradients left in grads) */
    /* Optional HOST buffers (pinned memory; NULL = not used) for a step fed from the host: the
     * step starts by copying host_target_rgb [3*P], host_target_depth [P] and host_mask [P]
     * into target_rgb, target_depth and mask (which must then be given: the device buffers the
     * step reads) and ends by copying loss_out [n_views + 1] into host_loss_out.  In a graph of
     * gs_graph_create the upload runs on a second branch, overlapped with the projection and
     * the binning (which do not read the targets); gs_step copies in stream order.  The host
     * buffers must stay valid until the step has completed on the stream. */
    const float *host_target_rgb, *host_target_depth;
    const uint8_t *host_mask;
    float *host_loss_out;
} gs_step_io;

typedef struct gs_graph_s *gs_graph;

void gs_default_opts(gs_render_opts *opts);
const char *gs_last_error(void);
const char *gs_version(void);

/* Workspace size and layout for n Gaussians seen by n_views cameras (host array) with at
 * most max_pairs (tile, Gaussian) pairs.  The layout is a plain host-side descriptor: the
 * caller computes it once per (n, views, image sizes, tile, max_pairs) and passes it, with
 * a device buffer of at least layout.total bytes (256-byte aligned), to every stage call.
 * gs_workspace_size returns 0 on invalid arguments. */
size_t gs_workspace_size(int64_t n, int32_t n_views, const gs_camera *cams,
                         const gs_render_opts *opts, int64_t max_pairs);
gs_status gs_workspace_layout(int64_t n, int32_t n_views, const gs_camera *cams,
                              const gs_render_opts *opts, int64_t max_pairs, gs_ws_layout *out);

/* Copies the device counters into *out (host memory); synchronises `stream`. */
gs_status gs_read_counters(const gs_ws_layout *L, const void *ws, gs_counters *out, void *stream);
/* Clears the device counters (status, pair count, the Adam step of gs_step).  Call once after
 * allocating a workspace (asynchronous on `stream`). */
gs_status gs_workspace_init(const gs_ws_layout *L, void *ws, void *stream);

/* Device-side failures.  The projection clears the status word; a stage that fails sets it
 * (GS_ERR_CAPACITY from the binning, GS_ERR_NONFINITE from the projection on a NaN or infinite
 * parameter) and every later stage of the step -- binning, compositing, backward, projection
 * backward, the fused Adam update and its step counter -- then does nothing, so a failed
 * step leaves the parameters, moments and Adam step unchanged.  gs_read_counters reports it. */

/* a1 -- EWA projection with SH colour (§III-C "standard differentiable Gaussian splatting";
 * tile-based rasterizer of §II-A).  For every view v and Gaussian i: q = q/|q| -> R,
 * Sigma = R S S^T R^T with S = diag(exp(log_scale)); p_c = R_cw mu + t_cw, culled if
 * z <= near_z; Sigma' = J R_cw Sigma R_cw^T J^T + dilation*I with the perspective
 * Jacobian J at (x/z, y/z) clamped to +-clamp_fov*(W/2)/fx (resp. H, fy); o =
 * sigmoid(logit), culled if o < alpha_min; rgb = max(0, sum_k sh_k Y_k(dir) + 0.5),
 * dir = normalize(mu - camera centre); box half-extents rx = ceil(sqrt(tau Sigma'_xx)), ry = ceil(sqrt(tau
 * Sigma'_yy)), tau = 2 ln(o/alpha_min) (the bounding box of the ellipse outside which
 * alpha < alpha_min).  Writes the proj, vis_bits and visible regions of the workspace. */
gs_status gs_project(const gs_gaussians *g, const gs_camera *cams, const gs_render_opts *opts,
                     const gs_ws_layout *L, void *ws, void *stream);

/* a2-a4 -- Tile binning, (tile, depth) radix sort and tile ranges (§II-A tile-based
 * rasterizer).  A record with box half-extents rx, ry covers tiles x in
 * [floor((u-rx)/T), floor((u+rx)/T)] and y in [floor((v-ry)/T), floor((v+ry)/T)], clamped to
 * the view's grid, computed in FP32 exactly as written.  The pairs (global tile id
 * tile_offset(v) + ty*tiles_x + tx, value v*n + i) come out in the order of the key
 * (tile id << 32) | float_bits(z) sorted stably from emission in ascending (v, i) then
 * row-major tile order -- computed as a stable sort of the visible (v, i) entries by
 * float_bits(z) followed by a stable sort of their pairs by tile id.  If the pairs exceed
 * max_pairs the status word becomes GS_ERR_CAPACITY, n_pairs holds the required count and
 * the later stages of the step do nothing.  Reads the proj and vis_bits regions that
 * gs_project writes. */
gs_status gs_bin_sort(const gs_camera *cams, const gs_render_opts *opts, const gs_ws_layout *L,
                      void *ws, void *stream);

/* a5 -- Front-to-back compositing of colour and depth (§III-C, depth equation) with the
 * fused L1 loss (§III-C loss equations, SSIM weight 0).  With opts.lambda_ssim > 0 or
 * opts.mask_erode >= 0 the compositing only renders and the loss is that of gs_objective, on
 * gs_render_mask's mask when mask_erode >= 0 (else on `mask`).  Outputs (packed per view, see
 * above): out_rgb [3*P], out_depth [P]; out_T [P] (final transmittance) may be NULL.
 * When target_rgb is non-NULL the loss is evaluated:
 *   L = 1/V sum_v [ lambda_rgb/|M_v| sum_{x in M_v} ||C - C~||_1
 *                 + lambda_depth/|M_v,D| sum_{x in M_v,D} |D - D~| ]
 * where M_v = {mask != 0} (mask may be NULL = all ones) and M_v,D = M_v and {D~ > 0};
 * dl_drgb [3*P] / dl_ddepth [P] receive dL/dC and dL/dD (sign(0) = 0) and loss_out (device,
 * n_views + 1 floats) the per-view terms and their mean.  target_depth may be NULL (no
 * depth term). */
gs_status gs_render_fwd(const gs_camera *cams, const gs_render_opts *opts, const gs_ws_layout *L,
                        void *ws, float *out_rgb, float *out_depth, float *out_T,
                        const float *target_rgb, const float *target_depth, const uint8_t *mask,
                        float *dl_drgb, float *dl_ddepth, float *loss_out, void *stream);

/* f1 -- Interior mask (§III-C, optimization: a geometric support mask from the accumulated
 * opacity of the current rendering, eroded morphologically; supervision is evaluated inside
 * it).  mask_out[p] = [1 - T_final(q) >= opts.mask_opacity for every pixel q of the view with
 * |q - p| <= r] and caller_mask[p] != 0 (caller_mask may be NULL), r = max(0, opts.mask_erode);
 * pixels outside the image count as outside the support.  T_final is the workspace's, from
 * the last gs_render_fwd.  The threshold is decided on the FP32 value, 1 - T computed in
 * FP32.  mask_out: device uint8 [P], packed per view; the caller owns it. */
gs_status gs_render_mask(const gs_camera *cams, const gs_render_opts *opts, const gs_ws_layout *L,
                         void *ws, const uint8_t *caller_mask, uint8_t *mask_out, void *stream);

/* f1 -- The full §III-C objective over a mask M (total-loss, L_rgb, L_ssim and L_depth
 * equations): per view lambda_rgb L_rgb + lambda_ssim (1 - SSIM) + lambda_depth L_depth,
 * averaged over the views.  L_rgb and L_depth are as in gs_render_fwd; SSIM is taken on
 * x = C M and y = C~ M per channel with an 11 x 11 Gaussian window (sigma 1.5, normalised,
 * zeros outside the image), C1 = 0.01^2, C2 = 0.03^2, and averaged over the pixels of M and
 * the three channels (an empty M contributes 0).  rgb [3*P], depth [P]: rendered images (from
 * gs_render_fwd); target_depth may be NULL (then depth and dl_ddepth may be too); mask may be
 * NULL (all pixels).  dl_drgb / dl_ddepth are overwritten with dL/dC, dL/dD (the mask is a
 * constant: no gradient flows through it); loss_out (device, n_views + 1 floats) receives the
 * per-view terms and their mean.  lambda_ssim > 0 needs a workspace laid out with
 * lambda_ssim > 0 (it holds 9 floats of scratch per pixel). */
gs_status gs_objective(const gs_camera *cams, const gs_render_opts *opts, const gs_ws_layout *L,
                       void *ws, const float *rgb, const float *depth, const float *target_rgb,
                       const float *target_depth, const uint8_t *mask, float *dl_drgb,
                       float *dl_ddepth, float *loss_out, void *stream);

/* f2 -- Map-size updates between mapping iterations (§III-C, optimization: new Gaussians pass
 * a 3-D Euclidean proximity test before insertion; low-opacity Gaussians are pruned under a
 * bounded removal ratio).  The three calls below read counts back and so synchronize `stream`.
 * They share one caller-owned device scratch buffer of gs_map_update_scratch_bytes(n_map,
 * n_new) bytes (256-byte multiple); calls that overlap on the GPU must not share it. */
size_t gs_map_update_scratch_bytes(int64_t n_map, int64_t n_new);

/* Prune plan: rows with sigmoid(logit) < opacity_min (decided on the FP32 logit against the
 * FP32 logit of opacity_min) are candidates; at most floor(max_ratio * n) of them (in double
 * precision) are removed,
 * those with the smallest (logit, row index).  keep: device uint8 [n] (1 = stays); *n_keep
 * (host) receives the rows kept.  Only g->opacity_logits is read. */
gs_status gs_prune_plan(const gs_gaussians *g, float opacity_min, double max_ratio, uint8_t *keep,
                        void *scratch, size_t scratch_bytes, int64_t *n_keep, void *stream);

/* Proximity plan: accept[j] = 1 unless a mean of `map` lies strictly within `radius` of
 * new_means[:, j] (squared distance summed in FP32 in x, y, z order; new means are not tested
 * against each other).  new_means: device [3][n_new] planes; accept: device uint8 [n_new];
 * *n_accept (host) receives the count accepted.  Only map->means is read. */
gs_status gs_dedup_plan(const gs_gaussians *map, const float *new_means, int64_t n_new, float radius,
                        uint8_t *accept, void *scratch, size_t scratch_bytes, int64_t *n_accept,
                        void *stream);

/* Update: out = the rows of `in` with keep != 0, in order, then the rows of new_rows (may be
 * NULL) with accept != 0 (accept may be NULL = all), in order; m_out / v_out carry the kept
 * rows' Adam moments and zeros for the new rows; tags_out (may be NULL) the kept rows' tags_in
 * and the new rows' new_tags (either may be NULL = 0).  out->n (= m_out->n = v_out->n) must
 * equal the rows kept plus accepted; all maps share sh_degree; outputs must not alias inputs. */
gs_status gs_map_update(const gs_gaussians *in, const gs_gaussians *m_in, const gs_gaussians *v_in,
                        const uint8_t *keep, const gs_gaussians *new_rows, const uint8_t *accept,
                        const uint32_t *tags_in, const uint32_t *new_tags, gs_gaussians *out,
                        gs_gaussians *m_out, gs_gaussians *v_out, uint32_t *tags_out, void *scratch,
                        size_t scratch_bytes, void *stream);

/* f3 -- Gaussian-GICP loop registration (§III-D: target-set, residual, covariance and loop-pose
 * equations).  Calls synchronize `stream`; their scratch is a caller-owned device buffer of
 * gs_gicp_scratch_bytes(n of the target map) bytes. */
size_t gs_gicp_scratch_bytes(int64_t n_target_map);

/* Target set around a historical loopframe: target_flag[i] = 1 if, for some query view k,
 * the mean projects inside its image (z > near_z, 0 <= u < width, 0 <= v < height, u = fx x/z
 * + cx, v = fy y/z + cy, all in FP32) and lies closer than d_max to the view's camera centre
 * (squared distance in FP32), and source_flag[i] == 0 (source_flag may be NULL).  views: host
 * array of 1..GS_MAX_VIEWS cameras; target_flag: device uint8 [n]; *n_target: host count. */
gs_status gs_gicp_target_set(const gs_gaussians *map, const gs_camera *views, int32_t n_views,
                             float near_z, float d_max, const uint8_t *source_flag,
                             uint8_t *target_flag, void *scratch, size_t scratch_bytes,
                             int64_t *n_target, void *stream);

typedef struct {
    double T[12];      /* row-major 3 x 4 [R | t]: maps source means onto target means */
    double cost;       /* sum of r^T Omega r at the final correspondences */
    int64_t n_corr;    /* correspondences at the final T */
    int32_t iters;     /* Gauss-Newton iterations taken */
    int32_t converged; /* 1 if the last update was below eps */
} gs_gicp_result;

/* Registration of the source rows (src_flag != 0, or all if NULL) of `src` onto the target rows
 * of `tar`: Gauss-Newton on sum r^T (Sigma~_n + R Sigma~_m R^T)^-1 r, r = mu_n - T mu_m, with
 * Sigma~ the planar form of each covariance (eigenvalues 1, 1, 1e-3, the smallest-scale axis
 * getting 1e-3) and the weights held fixed within an iteration; correspondences: the nearest
 * target mean within d_corr of T mu_m (FP32 squared distance; lower row on ties); update
 * T <- Exp(xi) T, xi = (rho, phi); stops when |xi| < eps or after max_iters.  T_init: host
 * row-major 3 x 4; result: host. */
gs_status gs_gicp_register(const gs_gaussians *src, const uint8_t *src_flag, const gs_gaussians *tar,
                           const uint8_t *tar_flag, const double T_init[12], float d_corr,
                           int32_t max_iters, double eps, gs_gicp_result *result, void *scratch,
                           size_t scratch_bytes, void *stream);

/* a6-a7 -- Analytic backward of gs_render_fwd and gs_project for upstream per-pixel
 * gradients dl_drgb [3*P], dl_ddepth [P] (dl_ddepth may be NULL).  Transmittance is
 * recomputed back to front from the stored final T (T_i = T_{i+1} / (1 - alpha_i)); no
 * per-fragment state is stored.  Gradients are ADDED to `grads` (same layout as g) and, if
 * grad_twist is non-NULL, to grad_twist [n_views][6]: the derivative w.r.t. the twist
 * xi = (rho, phi) of a left perturbation T_cw <- Exp(xi) T_cw of each view's pose.
 * Only rows with a nonzero `visible` flag of the workspace (the Gaussian covers a tile of
 * some view) are read and written; the other gradient rows are left as they are. */
gs_status gs_render_bwd(const gs_gaussians *g, const gs_camera *cams, const gs_render_opts *opts,
                        const gs_ws_layout *L, void *ws, const float *dl_drgb,
                        const float *dl_ddepth, gs_gaussians *grads, float *grad_twist,
                        void *stream);

/* a6 and a7 separately (gs_render_bwd = gs_composite_bwd then gs_project_bwd): the backward
 * compositing into the workspace's per-(view, Gaussian) screen-space sums (cleared first), and
 * the chain rule from those sums to the parameter gradients (added to grads) and the twists
 * (added to grad_twist, may be NULL). */
gs_status gs_composite_bwd(const gs_camera *cams, const gs_render_opts *opts, const gs_ws_layout *L,
                           void *ws, const float *dl_drgb, const float *dl_ddepth, void *stream);
gs_status gs_project_bwd(const gs_gaussians *g, const gs_camera *cams, const gs_render_opts *opts,
                         const gs_ws_layout *L, void *ws, gs_gaussians *grads, float *grad_twist,
                         void *stream);

/* Pose twists of the differentiable rendering (§III-C: the optimisation refines keyframe
 * poses with the map; here a pose increment xi = (rho, phi), rho the translation part, acts on
 * the left, T_cw <- Exp(xi) T_cw).  Host-side helpers of the autograd form, all arrays HOST
 * memory, n_views in 1..GS_MAX_VIEWS.
 *   gs_twist_cameras: out[v] = cams[v] with (R_cw, t_cw) replaced by Exp(xi_v) (R_cw, t_cw),
 *     computed in double (Rodrigues rotation, t = V(phi) rho) and rounded to float; out may
 *     equal cams.  xi: [n_views][6].
 *   gs_twist_grad: g_xi_v = J(xi_v)^T g_left_v, with J the left Jacobian of SE(3)
 *     (Exp(xi + d) = Exp(J(xi) d) Exp(xi) to first order, summed as its power series in the
 *     6 x 6 adjoint of xi) and g_left the gradient w.r.t. a left perturbation of the already
 *     moved pose (gs_render_bwd's grad_twist); so g_xi is the gradient w.r.t. xi itself
 *     (J = I at xi = 0).  xi, g_left, g_xi: [n_views][6]; g_xi may equal g_left.
 * A non-finite xi returns GS_ERR_NONFINITE. */
gs_status gs_twist_cameras(const gs_camera *cams, const float *xi, int32_t n_views, gs_camera *out);
gs_status gs_twist_grad(const float *xi, const float *g_left, int32_t n_views, float *g_xi);

/* a8 -- Fused masked Adam (§III-C: visible and unfrozen Gaussians are refined by a sparse
 * gradient-based optimiser; only the most recent segments are updated).  Row i is updated
 * iff (update_mask == NULL or update_mask[i]) and (visible == NULL or visible[i]);
 * other rows keep p, m and v unchanged.  m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr_group * m_hat / (sqrt(v_hat) + eps) with bias correction by `step` (>= 1).
 * lr[6]: means, log-scales, quats, opacity, SH DC, SH rest.  Zeroes the gradient rows
 * with visible[i] != 0 (all rows when visible == NULL) afterwards; rows with visible[i] ==
 * 0 are neither read nor written -- gs_project_bwd leaves exactly those rows untouched,
 * so after a step of gs_project_bwd + gs_adam_step every gradient row is zero again. */
gs_status gs_adam_step(gs_gaussians *params, gs_gaussians *grads, gs_gaussians *m, gs_gaussians *v,
                       const uint8_t *update_mask, const uint8_t *visible, const float lr[6],
                       float b1, float b2, float eps, int64_t step, void *stream);

/* a7 + a8 fused -- gs_project_bwd followed by gs_adam_step (with the workspace's visible
 * flags) in one kernel: every visible row's gradient is formed in registers and applied by
 * the masked Adam update directly, so the gradient planes are never written or read.
 * Gives the same parameters, moments and twists as the two calls in sequence on zeroed
 * gradients.  `params` is read and updated in place; step as for gs_adam_step. */
gs_status gs_project_bwd_adam(gs_gaussians *params, const gs_camera *cams, const gs_render_opts *opts,
                              const gs_ws_layout *L, void *ws, gs_gaussians *m, gs_gaussians *v,
                              const uint8_t *update_mask, const float lr[6], float b1, float b2,
                              float eps, int64_t step, float *grad_twist, void *stream);

/* a9 -- The batched mapping step (§III-C: each iteration samples keyframes from the recent and
 * history windows and updates the visible, unfrozen Gaussians): gs_project, gs_bin_sort,
 * gs_render_fwd with the fused L1 loss, gs_render_bwd and, if io->optimize, the masked Adam
 * step, for every view of the batch, on one stream without host synchronisation.  With
 * io->optimize the projection backward and Adam run fused (gs_project_bwd_adam): each row's
 * gradient goes straight into its Adam update and `grads` is neither read nor written;
 * without it the gradients are added to `grads`.  The Adam step counter is a device
 * counter in the workspace (gs_workspace_init sets it to 0), so the sequence can be
 * captured once and replayed. */
gs_status gs_step(gs_gaussians *params, gs_gaussians *grads, gs_gaussians *m, gs_gaussians *v,
                  const gs_camera *cams, const gs_render_opts *opts, const gs_ws_layout *L, void *ws,
                  const gs_step_io *io, void *stream);

/* CUDA graph of one gs_step, captured on `stream` (must not be the legacy default stream).
 * All pointers are baked into the graph; write new targets into the same buffers.  New poses
 * (same image sizes) go in with gs_graph_set_cameras, which rewrites the by-value camera
 * argument of the captured view-table upload -- no re-capture.  The handle owns only host
 * and driver objects; gs_graph_destroy releases them. */
gs_status gs_graph_create(gs_graph *out, gs_gaussians *params, gs_gaussians *grads, gs_gaussians *m,
                          gs_gaussians *v, const gs_camera *cams, const gs_render_opts *opts,
                          const gs_ws_layout *L, void *ws, const gs_step_io *io, void *stream);
gs_status gs_graph_launch(gs_graph g, void *stream);
gs_status gs_graph_set_cameras(gs_graph g, const gs_camera *cams);
gs_status gs_graph_destroy(gs_graph g);

/* ---------------------------------------------------------------------------------------
 * The learned Gaussian initialiser (a10-a12).  RMGS-SLAM §III-B initialises one Gaussian per
 * LiDAR point by a cascade -- a learned model where its prediction is valid, else the
 * voxel-PCA prior (§III-A) where it is geometrically reliable, else an isotropic depth
 * heuristic.  The paper's model (a pretrained feed-forward network) is not available; here
 * it is a small MLP over the voxel-PCA features.
 * --------------------------------------------------------------------------------------- */

/* Voxel-PCA constants (§III-A; the paper fixes tau_p, tau_l but does not state them). */
typedef struct {
    float voxel;      /* voxel side (0.5 m) */
    int32_t min_pts;  /* points needed for a feature (5) */
    float tau_p;      /* planar if lambda_min < tau_p (2.5e-3 m^2) */
    float tau_l;      /* else linear if lambda_max / lambda_min > tau_l (10) */
    float sigma;      /* per-point noise, Sigma_i = sigma^2 I (0.02 m) */
    float tau_trace;  /* reliable iff trace of the directional block of Sigma_g < tau_trace (1e-2) */
} gs_pca_opts;

/* a10 -- Voxel-PCA features (§III-A): points [3][n] (world, FP32) and colours [3][n] are
 * grouped into voxels by key (floor(p/voxel) per axis, FP32, sorted with the radix sort); per
 * voxel with >= min_pts points: mean, covariance, sorted eigen-decomposition (each eigenvector's
 * largest component positive, v_max = v_min x v_mid), planar / linear / unreliable class and
 * reliability from the descriptor covariance Sigma_g = sum_i J_i Sigma_i J_i^T.  Per point:
 *   x_out [n][16] = [ln max(lambda, 1e-4) (3), V row-major (9), rgb (3), ln(d / fx)] (zero rows
 *   without a feature), has_feature, reliable, s_pca [n][3] = ln sqrt(max(lambda, 1e-4)),
 *   q_pca [n][4] (w, x, y, z; w >= 0) of V; depth [n] and inside [n]: among the n_frames host
 *   cameras (the segment's loopframes / keyframes, <= 32) the closest one whose image the point
 *   projects into gives d (the "closer view" of §III-B) and inside = 1; with none, d is the
 *   depth in frames[0] and inside = 0; fx is frames[0].fx.  ws: gs_pca_workspace_size(n)
 *   bytes, 256-aligned. */
size_t gs_pca_workspace_size(int64_t n);
gs_status gs_voxel_pca(const float *pts, const float *rgb, int64_t n, const gs_camera *frames,
                       int32_t n_frames, const gs_pca_opts *opts, void *ws, size_t ws_bytes, float *x_out,
                       uint8_t *has_feature, uint8_t *reliable, float *s_pca, float *q_pca,
                       float *depth, uint8_t *inside, void *stream);

/* a11 -- MLP inference y [n][16] = f(x [n][16]): 16 -> 128 -> 128 -> 128 -> 16 with GELU
 * (erf form) after the hidden layers; BF16 weights (w_bf16 [36864] = W1 128x16 | W2 128x128 |
 * W3 128x128 | W4 16x128, row-major [out][in]), FP32 biases [400] (b1 | b2 | b3 | b4), BF16
 * input and hidden activations, FP32 accumulation (tensor cores).  Outputs 0..10 are the
 * residuals: log-scale (3), quaternion (4), opacity logit (1), colour (3). */
gs_status gs_mlp_infer(const uint16_t *w_bf16, const float *bias, const float *x, int64_t n,
                       float *y, void *stream);

/* a12 -- One training step on n (x, y_target) rows: forward, loss = mean over rows and the
 * 11 used outputs of (y - y_target)^2, backward GEMMs (BF16 operands, FP32 accumulate), Adam
 * on the FP32 master weights w_master [36864] and biases [400] (both updated in place), BF16
 * copy into w_bf16.  grad_w [36864], grad_b [400] must be zero on entry and are zeroed again;
 * adam_m, adam_v [37264] (weights then biases).  scratch: gs_mlp_train_scratch_size(n) bytes.
 * loss_out (device float, may be NULL) receives the loss of this step's forward. */
size_t gs_mlp_train_scratch_size(int64_t n);
gs_status gs_mlp_train_step(float *w_master, uint16_t *w_bf16, float *bias, float *grad_w, float *grad_b,
                            float *adam_m, float *adam_v, const float *x, const float *y_target,
                            int64_t n, float lr, float b1, float b2, float eps, int64_t step,
                            void *scratch, size_t scratch_bytes, float *loss_out, void *stream);

/* a12 -- Training pairs of the initialiser from the plain mapping loop (§III-B's learned
 * branch; its targets here are what the plain loop changes).  For every row i with
 * has_feature[i] != 0 and inside[i] != 0 (either may be NULL = every row), in row order, row
 * k of the outputs is x_out[k] = x[i] (16 features, as gs_voxel_pca writes them) and
 * y_out[k] = the residual of the optimised map `opt` against the initial map `init` in the
 * MLP's output units (FP32, each operation rounded once):
 *   y[0..2] = log-scale(opt) - log-scale(init);
 *   y[3..6] = q(opt)/|q(opt)| - q(init)/|q(init)|, each normalised quaternion multiplied by -1
 *             first if its w component is negative (w >= 0 forms);
 *   y[7] = logit(opt) - logit(init);  y[8..10] = (SH DC(opt) - SH DC(init)) * Y00 (colour
 *   units, Y00 = 1 / (2 sqrt(pi)));  y[11..15] = 0.
 * init, opt: the same n and sh_degree; x [n][16], x_out / y_out [n][16] device, 16-byte
 * aligned; *n_out (host) receives the rows written.  scratch: gs_init_residuals_scratch_bytes(n)
 * device bytes.  Synchronises `stream` (to read the count). */
size_t gs_init_residuals_scratch_bytes(int64_t n);
gs_status gs_init_residuals(const gs_gaussians *init, const gs_gaussians *opt, const float *x,
                            const uint8_t *has_feature, const uint8_t *inside, float *x_out, float *y_out,
                            int64_t *n_out, void *scratch, size_t scratch_bytes, void *stream);

/* Cascaded initialisation (§III-B equations): per point, the model branch where the MLP output
 * y (may be NULL: no model) is valid -- the point has a feature, lies inside the loopframe,
 * the outputs are finite and |log-scale residual| < 3 -- giving log-scale s_pca + dy,
 * quaternion normalize(q_pca + dq), opacity logit logit(opacity_init) + do, colour rgb + dc;
 * else the PCA branch where reliable: s_pca + log(beta), q_pca; else the heuristic ln(d/fx)
 * isotropic with identity rotation.  beta = clamp(#(reliable and not valid) / n, 0.25, 1).
 * Non-model branches take opacity_init; SH DC from the colour, higher SH zero.  Writes every
 * plane of `out` (n Gaussians), branch [n] (2 model, 1 PCA, 0 heuristic; may be NULL) and
 * beta_out (device float, may be NULL); count_tmp is one device uint32 of scratch. */
gs_status gs_init_cascade(const float *pts, const float *rgb, int64_t n, const float *y,
                          const uint8_t *has_feature, const uint8_t *reliable, const float *s_pca,
                          const float *q_pca, const float *depth, const uint8_t *inside, float fx,
                          float opacity_init, gs_gaussians *out, int32_t *branch,
                          unsigned int *count_tmp, float *beta_out, void *stream);

/* Allocation-free sort (the paper has no counterpart; it is a service of this library).
 * Stable LSD radix sort of n (key, value) pairs by the low key_bits bits of the key (8 bits
 * per pass), the same sort gs_bin_sort applies to its (tile, depth) pairs, for callers that
 * cannot allocate device memory -- e.g. code running under a no-allocation policy, inside
 * a host callback, or as a plug-in of an application that owns all device allocations.
 * Its scratch is a fixed array inside the library (13,108,480 bytes = 12.5 MiB per device,
 * held by every GPU that loads the library until the process exits), so a call sorts at
 * most 1048576 pairs; larger n returns GS_ERR_INVALID_ARG.  The call allocates nothing.
 *   keys_in [n], vals_in [n]   device input, not modified
 *   keys_out [n], vals_out [n] device output; the byte ranges of the two outputs must not
 *                              overlap each other or either input (GS_ERR_INVALID_ARG)
 * The first call on a device (with that device current) looks up the scratch address with
 * cudaGetSymbolAddress, which can load the library's device code; make that first call
 * before any stream capture.  All calls share the scratch and it keeps the previous call's
 * contents, so calls that may overlap on the GPU (other streams, other host threads)
 * race and must be serialised by the caller. */
gs_status gs_sort_pairs_noalloc(const uint64_t *keys_in, const uint32_t *vals_in, int64_t n,
                                int32_t key_bits, uint64_t *keys_out, uint32_t *vals_out,
                                void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GS_H */
