// extern "C" entry points declared in include/gs.h: argument checks, workspace layout and
// the launch sequence of each stage.  Host code only; all arithmetic of the step runs in
// the kernels of project.cu, binsort.cu, render.cu and adam.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "gs_kernels.cuh"

namespace gs {

static thread_local std::string g_err;

static gs_status fail(gs_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define GS_CUDA(call)                                                                           \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return fail(GS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// loss accumulators: double [GS_MAX_VIEWS][3] sums, then uint32 [GS_MAX_VIEWS][2] counts
constexpr size_t kLossAccBytes = sizeof(double) * 3 * GS_MAX_VIEWS + sizeof(uint32_t) * 2 * GS_MAX_VIEWS;

struct Geometry {
    int total_tiles = 0;
    int64_t total_pixels = 0;
    View views[GS_MAX_VIEWS];
    int64_t pix[GS_MAX_VIEWS];
};

static gs_status check_opts(const gs_render_opts* o) {
    if (!o) return fail(GS_ERR_INVALID_ARG, "opts is NULL");
    if (o->tile != 8 && o->tile != 16) return fail(GS_ERR_INVALID_ARG, "tile must be 8 or 16 (got %d)", o->tile);
    if (o->chunk != 32 && o->chunk != 64 && o->chunk != 128 && o->chunk != 256)
        return fail(GS_ERR_INVALID_ARG, "chunk must be 32, 64, 128 or 256 (got %d)", o->chunk);
    if (!(o->alpha_min > 0.f) || !(o->alpha_max <= 1.f) || !(o->alpha_min < o->alpha_max))
        return fail(GS_ERR_INVALID_ARG, "need 0 < alpha_min < alpha_max <= 1");
    if (!(o->T_min >= 0.f) || !(o->near_z >= 0.f) || !(o->dilation >= 0.f) || !(o->clamp_fov > 0.f))
        return fail(GS_ERR_INVALID_ARG, "invalid compositing constants");
    if (!(o->lambda_ssim >= 0.f) || !(o->mask_opacity >= 0.f && o->mask_opacity <= 1.f) || o->mask_erode < -1 ||
        o->mask_erode > 16)
        return fail(GS_ERR_INVALID_ARG, "need lambda_ssim >= 0, mask_opacity in [0, 1], mask_erode in [-1, 16]");
    if (o->persistent != 0 && o->persistent != 1) return fail(GS_ERR_INVALID_ARG, "persistent must be 0 or 1");
    if (o->sync_spin_limit < 0 || o->sync_skip_block < -1)
        return fail(GS_ERR_INVALID_ARG, "need sync_spin_limit >= 0 and sync_skip_block >= -1");
    return GS_OK;
}

static gs_status make_geometry(int32_t n_views, const gs_camera* cams, const gs_render_opts* o, Geometry& G) {
    if (n_views < 1 || n_views > GS_MAX_VIEWS)
        return fail(GS_ERR_INVALID_ARG, "n_views must be in [1, %d] (got %d)", GS_MAX_VIEWS, n_views);
    if (!cams) return fail(GS_ERR_INVALID_ARG, "cams is NULL");
    gs_status s = check_opts(o);
    if (s != GS_OK) return s;
    int64_t toff = 0, poff = 0;
    for (int v = 0; v < n_views; v++) {
        const gs_camera& c = cams[v];
        if (c.width <= 0 || c.height <= 0 || c.width > 16384 || c.height > 16384)
            return fail(GS_ERR_INVALID_ARG, "view %d: bad size %dx%d", v, c.width, c.height);
        if (!(c.fx > 0.f) || !(c.fy > 0.f)) return fail(GS_ERR_INVALID_ARG, "view %d: focal lengths must be > 0", v);
        bool finite = std::isfinite(c.fx) && std::isfinite(c.fy) && std::isfinite(c.cx) && std::isfinite(c.cy);
        for (int k = 0; k < 9; k++) finite = finite && std::isfinite(c.R_cw[k]);
        for (int k = 0; k < 3; k++) finite = finite && std::isfinite(c.t_cw[k]);
        if (!finite) return fail(GS_ERR_NONFINITE, "view %d: a camera value is not finite", v);
        View& V = G.views[v];
        memset(&V, 0, sizeof(V));
        V.W = c.width;
        V.H = c.height;
        V.tiles_x = (c.width + o->tile - 1) / o->tile;
        V.tiles_y = (c.height + o->tile - 1) / o->tile;
        V.n_tiles = V.tiles_x * V.tiles_y;
        V.tile_off = (int32_t)toff;
        V.pix_off = poff;
        V.fx = c.fx; V.fy = c.fy; V.cx = c.cx; V.cy = c.cy;
        memcpy(V.R, c.R_cw, sizeof(V.R));
        memcpy(V.t, c.t_cw, sizeof(V.t));
        for (int i = 0; i < 3; i++)
            V.cw[i] = -(c.R_cw[0 * 3 + i] * c.t_cw[0] + c.R_cw[1 * 3 + i] * c.t_cw[1] + c.R_cw[2 * 3 + i] * c.t_cw[2]);
        V.limx = o->clamp_fov * (0.5f * (float)c.width) / c.fx;
        V.limy = o->clamp_fov * (0.5f * (float)c.height) / c.fy;
        G.pix[v] = (int64_t)c.width * c.height;
        toff += V.n_tiles;
        poff += G.pix[v];
    }
    if (toff > (int64_t)1 << 30) return fail(GS_ERR_INVALID_ARG, "too many tiles");
    G.total_tiles = (int)toff;
    G.total_pixels = poff;
    return GS_OK;
}

static int tile_bits(int total_tiles) {
    int b = 0;
    while (b < 31 && ((int64_t)1 << b) < total_tiles) b++;
    return b;
}

// Passes of the pair sort over the global tile id bits tb (0 passes when there is one tile):
// as few as 8- or 9-bit digits allow, P = min(ceil(tb / 8), ceil(tb / 9)).  The tb - 8 P
// passes that need a ninth bit are the last ones: the first pass's input, in emission order,
// spreads over all digits, and fewer digits give longer runs per digit in each chunk's
// scatter (17 tile bits: an 8-bit then a 9-bit pass).
static int pair_sort_passes(int total_tiles, int* shifts, int* bits) {
    const int tb = tile_bits(total_tiles);
    const int P = (tb + 7) / 8 < (tb + 8) / 9 ? (tb + 7) / 8 : (tb + 8) / 9;
    const int nine = tb - 8 * P > 0 ? tb - 8 * P : 0;
    int s = 0;
    for (int p = 0; p < P; p++) {
        bits[p] = p >= P - nine ? 9 : 8;
        shifts[p] = s;
        s += bits[p];
    }
    return P;
}

static gs_status layout(int64_t n, int32_t n_views, const gs_camera* cams, const gs_render_opts* o, int64_t max_pairs,
                        gs_ws_layout& L, Geometry& G) {
    if (n < 0) return fail(GS_ERR_INVALID_ARG, "n must be >= 0");
    if (max_pairs < 0 || max_pairs > (int64_t)0xFFFFFFFFll) return fail(GS_ERR_INVALID_ARG, "max_pairs out of range");
    gs_status s = make_geometry(n_views, cams, o, G);
    if (s != GS_OK) return s;
    const int64_t VN = (int64_t)n_views * n;
    if (VN >= (int64_t)0xFFFFFFFFll) return fail(GS_ERR_INVALID_ARG, "n_views * n must be < 2^32");
    memset(&L, 0, sizeof(L));
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t r = off; off = align256(off + bytes); return r; };
    L.views = take(sizeof(View) * GS_MAX_VIEWS);
    L.counters = take(sizeof(Counters));
    L.loss_acc = take(kLossAccBytes);
    L.proj = take(sizeof(float) * 12 * (size_t)VN);
    L.vis_bits = take(sizeof(uint32_t) * (size_t)n_views * (size_t)((n + 31) / 32));
    L.scan_tmp = take(sizeof(uint32_t) * ((size_t)VN / kScanBlock + 2));
    L.ekeys0 = take(sizeof(uint32_t) * (size_t)VN);
    L.ekeys1 = take(sizeof(uint32_t) * (size_t)VN);
    L.evals0 = take(sizeof(uint32_t) * (size_t)VN);
    L.evals1 = take(sizeof(uint32_t) * (size_t)VN);
    L.keys0 = take(sizeof(uint32_t) * (size_t)max_pairs);
    L.keys1 = take(sizeof(uint32_t) * (size_t)max_pairs);
    L.vals0 = take(sizeof(uint32_t) * (size_t)max_pairs);
    L.vals1 = take(sizeof(uint32_t) * (size_t)max_pairs);
    L.pair_mask = take((size_t)max_pairs);
    L.emit_tmp = take(sizeof(uint32_t) * ((size_t)max_pairs / kEmitChunk + 2));
    L.sort_tmp = take(sizeof(uint32_t) * ((size_t)kSortMaxBins * kSortMaxGrid + kSortMaxBins));
    L.ranges = take(sizeof(uint32_t) * 2 * (size_t)G.total_tiles);
    L.T_final = take(sizeof(float) * (size_t)G.total_pixels);
    L.n_contrib = take(sizeof(uint32_t) * (size_t)G.total_pixels);
    L.grad2d = take(sizeof(float) * 12 * (size_t)VN);
    L.geo2d = take(sizeof(float) * 12 * (size_t)VN);
    L.dirgrad = take(sizeof(float) * 3 * (size_t)n);
    L.entries = take(sizeof(uint32_t) * (size_t)VN);
    L.erect = take(sizeof(uint32_t) * 2 * (size_t)VN);
    L.visible = take((size_t)n);
    L.tile_order = take(sizeof(uint32_t) * ((size_t)G.total_tiles + 2 * 34));
    L.render_mask = take((size_t)G.total_pixels);
    L.has_ssim = o->lambda_ssim > 0.f ? 1 : 0;
    L.ssim_tmp = take(L.has_ssim ? sizeof(float) * 9 * (size_t)G.total_pixels : 0);
    L.total = off;
    int shifts[16], bits[16];
    L.sorted_buf = pair_sort_passes(G.total_tiles, shifts, bits) & 1;
    L.total_tiles = G.total_tiles;
    L.total_pixels = G.total_pixels;
    L.max_pairs = max_pairs;
    L.n = n;
    L.n_views = n_views;
    L.tile = o->tile;
    return GS_OK;
}

template <typename T>
static T* at(void* ws, size_t off) { return reinterpret_cast<T*>(reinterpret_cast<char*>(ws) + off); }

static Opts to_opts(const gs_render_opts* o) {
    Opts r;
    r.near_z = o->near_z; r.dilation = o->dilation; r.alpha_min = o->alpha_min; r.alpha_max = o->alpha_max;
    r.T_min = o->T_min; r.clamp_fov = o->clamp_fov;
    r.bg0 = o->bg[0]; r.bg1 = o->bg[1]; r.bg2 = o->bg[2];
    r.lambda_rgb = o->lambda_rgb; r.lambda_depth = o->lambda_depth;
    r.tile = o->tile; r.chunk = o->chunk;
    r.count = o->count_fragments != 0;
    return r;
}

struct ViewsParam {
    int n;
    View v[GS_MAX_VIEWS];
};

__global__ void setup_views_kernel(View* dst, const __grid_constant__ ViewsParam p) {
    for (int i = threadIdx.x; i < p.n; i += blockDim.x) dst[i] = p.v[i];
}

static gs_status upload_views(void* ws, const gs_ws_layout& L, const Geometry& G, int n_views, cudaStream_t st) {
    ViewsParam p;
    memset(&p, 0, sizeof(p));
    p.n = n_views;
    memcpy(p.v, G.views, sizeof(View) * n_views);
    setup_views_kernel<<<1, 32, 0, st>>>(at<View>(ws, L.views), p);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

static gs_status check_ws(const void* ws, const gs_ws_layout* L) {
    if (!L) return fail(GS_ERR_INVALID_ARG, "layout is NULL");
    if (!ws) return fail(GS_ERR_INVALID_ARG, "workspace is NULL");
    if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return fail(GS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    return GS_OK;
}

static gs_status check_gaussians(const gs_gaussians* g, bool need) {
    if (!g) return fail(GS_ERR_INVALID_ARG, "gaussians is NULL");
    if (g->n < 0) return fail(GS_ERR_INVALID_ARG, "n must be >= 0");
    if (g->sh_degree < 0 || g->sh_degree > GS_MAX_SH_DEGREE) return fail(GS_ERR_INVALID_ARG, "sh_degree must be 0..3");
    if (need && g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh))
        return fail(GS_ERR_INVALID_ARG, "a parameter plane pointer is NULL");
    return GS_OK;
}

// Geometry of the cameras, checked against the layout the workspace was made for.
static gs_status geometry_for(const gs_ws_layout* L, const gs_camera* cams, const gs_render_opts* opts, Geometry& G) {
    gs_status s = make_geometry(L->n_views, cams, opts, G);
    if (s != GS_OK) return s;
    if (G.total_tiles != L->total_tiles || G.total_pixels != L->total_pixels || opts->tile != L->tile)
        return fail(GS_ERR_INVALID_ARG, "cameras / tile size do not match the workspace layout");
    if (opts->lambda_ssim > 0.f && !L->has_ssim)
        return fail(GS_ERR_INVALID_ARG, "lambda_ssim > 0 needs a workspace laid out with lambda_ssim > 0");
    return GS_OK;
}


// ---------------------------------------------------------------------------------------
// Stage runners: launch sequences without argument checks or camera upload.  The public
// entry points (and gs_step) validate, upload the view table, then call these.
// ---------------------------------------------------------------------------------------
static cudaError_t run_project(const gs_gaussians* g, const gs_render_opts* opts, const gs_ws_layout* L, void* ws,
                               cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(at<Counters>(ws, L->counters), 0, kCountersResetBytes, st);
    if (e != cudaSuccess) return e;
    ProjectArgs a;
    a.n = g->n;
    a.n_views = L->n_views;
    a.views = at<View>(ws, L->views);
    a.op = to_opts(opts);
    a.means = g->means; a.log_scales = g->log_scales; a.quats = g->quats; a.logits = g->opacity_logits; a.sh = g->sh;
    a.proj = at<float4>(ws, L->proj);
    a.vis_bits = at<uint32_t>(ws, L->vis_bits);
    a.visible = at<uint8_t>(ws, L->visible);
    a.counters = at<Counters>(ws, L->counters);
    return launch_project(a, g->sh_degree, st);
}

static cudaError_t run_bin_sort(const gs_render_opts* opts, const gs_ws_layout* L, void* ws, cudaStream_t st) {
    Counters* cnt = at<Counters>(ws, L->counters);
    BinArgs b;
    b.n = L->n;
    b.n_views = L->n_views;
    b.views = at<View>(ws, L->views);
    b.tile = opts->tile;
    b.max_pairs = L->max_pairs;
    b.proj = at<float4>(ws, L->proj);
    b.vis_bits = at<uint32_t>(ws, L->vis_bits);
    b.scan_tmp = at<uint32_t>(ws, L->scan_tmp);
    b.ekeys = at<uint32_t>(ws, L->ekeys0);
    b.evals = at<uint32_t>(ws, L->evals0);
    b.entries = at<uint32_t>(ws, L->entries);
    b.erect = at<uint2>(ws, L->erect);
    b.sorted_evals = at<uint32_t>(ws, L->evals0);   // 4 passes: the entry sort ends in buffer 0
    b.pkeys = at<uint32_t>(ws, L->keys0);
    b.pvals = at<uint32_t>(ws, L->vals0);
    b.poff = at<uint32_t>(ws, L->ekeys1);           // free once the entries are sorted
    b.chunk_first = at<uint32_t>(ws, L->emit_tmp);
    b.srt = at<uint32_t>(ws, L->geo2d);              // free until the projection backward
    b.counters = cnt;
    cudaError_t e = launch_entries(b, st);
    if (e != cudaSuccess) return e;
    SortArgs sa;
    sa.hist = at<uint32_t>(ws, L->sort_tmp);
    sa.digit_tot = sa.hist + (size_t)kSortMaxBins * kSortMaxGrid;
    sa.counters = cnt;
    sa.grid = sort_grid();
    // 1. entries by depth
    sa.keys[0] = at<uint32_t>(ws, L->ekeys0);
    sa.keys[1] = at<uint32_t>(ws, L->ekeys1);
    sa.vals[0] = at<uint32_t>(ws, L->evals0);
    sa.vals[1] = at<uint32_t>(ws, L->evals1);
    sa.count = &cnt->n_entries;
    const int depth_shifts[4] = {0, 8, 16, 24}, depth_bits[4] = {8, 8, 8, 8};
    if ((e = launch_sort32(sa, 4, depth_shifts, depth_bits, st)) != cudaSuccess) return e;
    // 2. pairs emitted in depth order, then by tile
    if ((e = launch_emit(b, st)) != cudaSuccess) return e;
    sa.keys[0] = at<uint32_t>(ws, L->keys0);
    sa.keys[1] = at<uint32_t>(ws, L->keys1);
    sa.vals[0] = at<uint32_t>(ws, L->vals0);
    sa.vals[1] = at<uint32_t>(ws, L->vals1);
    sa.count = &cnt->n_pairs;
    int shifts[16], bits[16];
    const int np = pair_sort_passes(L->total_tiles, shifts, bits);
    if ((e = launch_sort32(sa, np, shifts, bits, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(at<uint32_t>(ws, L->ranges), 0, sizeof(uint32_t) * 2 * (size_t)L->total_tiles, st)) !=
        cudaSuccess)
        return e;
    RangeArgs r;
    r.keys = static_cast<const uint32_t*>(sa.keys[np & 1]);
    r.ranges = at<uint2>(ws, L->ranges);
    r.counters = cnt;
    if ((e = launch_ranges(r, L->total_tiles, st)) != cudaSuccess) return e;
    uint32_t* order = at<uint32_t>(ws, L->tile_order);
    return launch_tile_order(r.ranges, L->total_tiles, order, order + L->total_tiles, cnt, st);
}

static ObjArgs obj_args(const gs_render_opts* opts, const gs_ws_layout* L, const Geometry& G, void* ws) {
    ObjArgs o;
    memset(&o, 0, sizeof(o));
    o.n_views = L->n_views;
    o.views = at<View>(ws, L->views);
    for (int v = 0; v < L->n_views; v++) {
        o.max_w = G.views[v].W > o.max_w ? G.views[v].W : o.max_w;
        o.max_h = G.views[v].H > o.max_h ? G.views[v].H : o.max_h;
    }
    o.T_final = at<float>(ws, L->T_final);
    o.tau = opts->mask_opacity;
    o.r_erode = opts->mask_erode > 0 ? opts->mask_erode : 0;
    double* sums = at<double>(ws, L->loss_acc);
    o.sums = sums;
    o.counts = reinterpret_cast<uint32_t*>(sums + 3 * GS_MAX_VIEWS);
    o.ssim_part = L->has_ssim ? at<float>(ws, L->ssim_tmp) : nullptr;
    o.lambda_rgb = opts->lambda_rgb;
    o.lambda_depth = opts->lambda_depth;
    o.lambda_ssim = opts->lambda_ssim;
    ssim_window(o.win);
    return o;
}

// M_int of the last forward's transmittance (and the caller's mask) into mask_out.
static cudaError_t run_render_mask(const gs_render_opts* opts, const gs_ws_layout* L, const Geometry& G, void* ws,
                                   const uint8_t* caller_mask, uint8_t* mask_out, cudaStream_t st) {
    ObjArgs o = obj_args(opts, L, G, ws);
    o.caller_mask = caller_mask;
    o.mask_out = mask_out;
    return launch_render_mask(o, st);
}

// The objective over `mask`: counts, masked L1 terms, SSIM (if lambda_ssim > 0), per-view
// losses and their mean.
static cudaError_t run_objective(const gs_render_opts* opts, const gs_ws_layout* L, const Geometry& G, void* ws,
                                 const float* rgb, const float* depth, const float* target_rgb,
                                 const float* target_depth, const uint8_t* mask, float* dl_drgb, float* dl_ddepth,
                                 float* loss_out, cudaStream_t st) {
    ObjArgs o = obj_args(opts, L, G, ws);
    cudaError_t e;
    if ((e = cudaMemsetAsync(o.sums, 0, kLossAccBytes, st)) != cudaSuccess) return e;
    if ((e = launch_loss_count(o.views, L->n_views, G.pix, target_depth, mask, const_cast<uint32_t*>(o.counts), st)) !=
        cudaSuccess)
        return e;
    o.rgb = rgb; o.depth = depth; o.tgt_rgb = target_rgb; o.tgt_depth = target_depth; o.mask = mask;
    o.dl_drgb = dl_drgb;
    o.dl_ddepth = target_depth ? dl_ddepth : nullptr;
    if ((e = launch_objective(o, st)) != cudaSuccess) return e;
    return launch_loss_finalize(o.sums, o.counts, L->n_views, opts->lambda_rgb, opts->lambda_depth, opts->lambda_ssim,
                                target_depth != nullptr, loss_out, st);
}

// Arguments of the forward compositing (its loss epilogue is off when tgt_rgb is NULL).
static FwdArgs fwd_args(const gs_render_opts* opts, const gs_ws_layout* L, void* ws, float* out_rgb, float* out_depth,
                        float* out_T, const float* tgt_rgb, const float* tgt_depth, const uint8_t* mask,
                        float* dl_drgb, float* dl_ddepth) {
    double* sums = at<double>(ws, L->loss_acc);
    FwdArgs a;
    a.n_views = L->n_views;
    a.views = at<View>(ws, L->views);
    a.op = to_opts(opts);
    a.proj = at<float4>(ws, L->proj);
    a.vals = at<uint32_t>(ws, L->sorted_buf ? L->vals1 : L->vals0);
    a.ranges = at<uint2>(ws, L->ranges);
    a.order = at<uint32_t>(ws, L->tile_order);
    a.counters = at<Counters>(ws, L->counters);
    a.pair_mask = at<uint8_t>(ws, L->pair_mask);
    a.T_final = at<float>(ws, L->T_final);
    a.n_contrib = at<uint32_t>(ws, L->n_contrib);
    a.out_rgb = out_rgb;
    a.out_depth = out_depth;
    a.out_T = out_T;
    a.tgt_rgb = tgt_rgb;
    a.tgt_depth = tgt_depth;
    a.mask = mask;
    a.dl_drgb = dl_drgb;
    a.dl_ddepth = dl_ddepth;
    a.loss_sums = sums;
    a.loss_counts = reinterpret_cast<uint32_t*>(sums + 3 * GS_MAX_VIEWS);
    return a;
}

// Arguments of the backward compositing for upstream gradients dl_drgb, dl_ddepth.
static BwdArgs bwd_args(const gs_render_opts* opts, const gs_ws_layout* L, void* ws, const float* dl_drgb,
                        const float* dl_ddepth) {
    BwdArgs b;
    b.n_views = L->n_views;
    b.views = at<View>(ws, L->views);
    b.op = to_opts(opts);
    b.proj = at<float4>(ws, L->proj);
    b.vals = at<uint32_t>(ws, L->sorted_buf ? L->vals1 : L->vals0);
    b.ranges = at<uint2>(ws, L->ranges);
    b.order = at<uint32_t>(ws, L->tile_order);
    b.counters = at<Counters>(ws, L->counters);
    b.pair_mask = at<uint8_t>(ws, L->pair_mask);
    b.entries = at<uint32_t>(ws, L->entries);
    b.T_final = at<float>(ws, L->T_final);
    b.n_contrib = at<uint32_t>(ws, L->n_contrib);
    b.dl_drgb = dl_drgb;
    b.dl_ddepth = dl_ddepth;
    b.grad2d = at<float4>(ws, L->grad2d);
    return b;
}

// Forward compositing.  With a target and neither the SSIM term nor the render-derived mask,
// the L1 loss is fused into the compositing epilogue; otherwise the forward only renders and
// the mask and the objective follow as separate kernels.
static cudaError_t run_fwd(const gs_render_opts* opts, const gs_ws_layout* L, const Geometry& G, void* ws,
                           float* out_rgb, float* out_depth, float* out_T, const float* target_rgb,
                           const float* target_depth, const uint8_t* mask, float* dl_drgb, float* dl_ddepth,
                           float* loss_out, cudaStream_t st, LossFinal* defer = nullptr) {
    double* sums = at<double>(ws, L->loss_acc);
    uint32_t* counts = reinterpret_cast<uint32_t*>(sums + 3 * GS_MAX_VIEWS);
    const bool separate = target_rgb && (opts->lambda_ssim > 0.f || opts->mask_erode >= 0);
    const bool fused = target_rgb && !separate;
    cudaError_t e;
    if (fused) {
        if ((e = cudaMemsetAsync(sums, 0, kLossAccBytes, st)) != cudaSuccess) return e;
        if ((e = launch_loss_count(at<View>(ws, L->views), L->n_views, G.pix, target_depth, mask, counts, st)) !=
            cudaSuccess)
            return e;
    }
    const FwdArgs a = fwd_args(opts, L, ws, out_rgb, out_depth, out_T, fused ? target_rgb : nullptr,
                               fused ? target_depth : nullptr, fused ? mask : nullptr, fused ? dl_drgb : nullptr,
                               fused ? dl_ddepth : nullptr);
    if ((e = launch_render_fwd(a, L->total_tiles, st)) != cudaSuccess) return e;
    if (fused && defer) {   // the caller's next kernel writes the loss terms
        *defer = LossFinal{sums, counts, L->n_views, opts->lambda_rgb, opts->lambda_depth, target_depth != nullptr,
                           loss_out};
        return cudaSuccess;
    }
    if (fused)
        return launch_loss_finalize(sums, counts, L->n_views, opts->lambda_rgb, opts->lambda_depth, 0.f,
                                    target_depth != nullptr, loss_out, st);
    if (separate) {
        const uint8_t* m = mask;
        if (opts->mask_erode >= 0) {
            uint8_t* rm = at<uint8_t>(ws, L->render_mask);
            if ((e = run_render_mask(opts, L, G, ws, mask, rm, st)) != cudaSuccess) return e;
            m = rm;
        }
        return run_objective(opts, L, G, ws, out_rgb, out_depth, target_rgb, target_depth, m, dl_drgb, dl_ddepth,
                             loss_out, st);
    }
    return cudaSuccess;
}

static cudaError_t run_composite_bwd(const gs_render_opts* opts, const gs_ws_layout* L, void* ws, const float* dl_drgb,
                                     const float* dl_ddepth, cudaStream_t st, Counters* adam_ctr = nullptr,
                                     float b1 = 0.f, float b2 = 0.f, const LossFinal& lf = LossFinal()) {
    return launch_render_bwd(bwd_args(opts, L, ws, dl_drgb, dl_ddepth), L->total_tiles, st, adam_ctr, b1, b2, lf);
}

// Adam settings of the fused projection backward (a7 + a8).
struct FusedAdam {
    gs_gaussians *params, *m, *v;
    const uint8_t* update_mask;
    const float* lr;
    float b1, b2, eps;
    int64_t step;                // host step (used when step_dev is null)
    const Counters* step_dev;
};

static ProjectBwdArgs pbwd_args(const gs_gaussians* g, const gs_render_opts* opts, const gs_ws_layout* L, void* ws,
                                gs_gaussians* grads, float* grad_twist, const FusedAdam* fa) {
    ProjectBwdArgs p;
    memset(&p, 0, sizeof(p));
    p.n = L->n;
    p.n_views = L->n_views;
    p.views = at<View>(ws, L->views);
    p.op = to_opts(opts);
    p.means = g->means; p.log_scales = g->log_scales; p.quats = g->quats; p.logits = g->opacity_logits; p.sh = g->sh;
    p.vis_bits = at<uint32_t>(ws, L->vis_bits);
    p.visible = at<uint8_t>(ws, L->visible);
    p.entries = at<uint32_t>(ws, L->entries);
    p.counters = at<Counters>(ws, L->counters);
    p.grad2d = at<float4>(ws, L->grad2d);
    p.geo2d = at<float4>(ws, L->geo2d);
    p.dirgrad = at<float>(ws, L->dirgrad);
    if (grads) {
        p.g_means = grads->means; p.g_log_scales = grads->log_scales; p.g_quats = grads->quats;
        p.g_logits = grads->opacity_logits; p.g_sh = grads->sh;
    }
    p.grad_twist = grad_twist;
    if (fa) {
        p.fused_adam = 1;
        p.p_means = fa->params->means; p.p_log_scales = fa->params->log_scales; p.p_quats = fa->params->quats;
        p.p_logits = fa->params->opacity_logits; p.p_sh = fa->params->sh;
        const gs_gaussians* mv[2] = {fa->m, fa->v};
        float** dst[2] = {p.m, p.v};
        for (int k = 0; k < 2; k++) {
            dst[k][0] = mv[k]->means; dst[k][1] = mv[k]->log_scales; dst[k][2] = mv[k]->quats;
            dst[k][3] = mv[k]->opacity_logits; dst[k][4] = mv[k]->sh;
        }
        p.update_mask = fa->update_mask;
        for (int k = 0; k < 6; k++) p.lr[k] = fa->lr[k];
        p.b1 = fa->b1; p.b2 = fa->b2; p.eps = fa->eps;
        p.bc1 = fa->step > 0 ? (float)(1.0 - pow((double)fa->b1, (double)fa->step)) : 1.f;
        p.bc2 = fa->step > 0 ? (float)(1.0 - pow((double)fa->b2, (double)fa->step)) : 1.f;
        p.step_dev = fa->step_dev;
    }
    return p;
}

static cudaError_t run_project_bwd(const gs_gaussians* g, const gs_render_opts* opts, const gs_ws_layout* L, void* ws,
                                   gs_gaussians* grads, float* grad_twist, cudaStream_t st,
                                   const FusedAdam* fa = nullptr) {
    return launch_project_bwd(pbwd_args(g, opts, L, ws, grads, grad_twist, fa), g->sh_degree, st);
}

static cudaError_t run_bwd(const gs_gaussians* g, const gs_render_opts* opts, const gs_ws_layout* L, void* ws,
                           const float* dl_drgb, const float* dl_ddepth, gs_gaussians* grads, float* grad_twist,
                           cudaStream_t st) {
    cudaError_t e = run_composite_bwd(opts, L, ws, dl_drgb, dl_ddepth, st);
    if (e != cudaSuccess) return e;
    return run_project_bwd(g, opts, L, ws, grads, grad_twist, st);
}

static gs_status check_adam(gs_gaussians* params, gs_gaussians* grads, gs_gaussians* m, gs_gaussians* v,
                            const float* lr, float b1, float b2, float eps) {
    gs_status s;
    gs_gaussians* all[4] = {params, grads, m, v};
    for (auto* x : all)
        if ((s = check_gaussians(x, true)) != GS_OK) return s;
    for (auto* x : all)
        if (x->n != params->n || x->sh_degree != params->sh_degree)
            return fail(GS_ERR_INVALID_ARG, "params / grads / m / v differ in n or sh_degree");
    if (!lr) return fail(GS_ERR_INVALID_ARG, "lr is NULL");
    if (!(b1 >= 0.f && b1 < 1.f && b2 >= 0.f && b2 < 1.f && eps >= 0.f))
        return fail(GS_ERR_INVALID_ARG, "need 0 <= b1, b2 < 1 and eps >= 0");
    return GS_OK;
}

static cudaError_t run_adam(gs_gaussians* params, gs_gaussians* grads, gs_gaussians* m, gs_gaussians* v,
                            const uint8_t* update_mask, const uint8_t* visible, const float* lr, float b1, float b2,
                            float eps, int64_t step, const Counters* step_dev, cudaStream_t st) {
    const int K = (params->sh_degree + 1) * (params->sh_degree + 1);
    AdamArgs a;
    a.n = params->n;
    a.n_planes = 11 + 3 * K;
    gs_gaussians* src[4] = {params, grads, m, v};
    float** dst[4] = {a.p, a.g, a.m, a.v};
    for (int k = 0; k < 4; k++) {
        dst[k][0] = src[k]->means;
        dst[k][1] = src[k]->log_scales;
        dst[k][2] = src[k]->quats;
        dst[k][3] = src[k]->opacity_logits;
        dst[k][4] = src[k]->sh;
    }
    a.planes_of[0] = 3; a.planes_of[1] = 3; a.planes_of[2] = 4; a.planes_of[3] = 1; a.planes_of[4] = 3 * K;
    a.update_mask = update_mask;
    a.visible = visible;
    for (int k = 0; k < 6; k++) a.lr[k] = lr[k];
    a.b1 = b1; a.b2 = b2; a.eps = eps;
    a.bc1 = step > 0 ? (float)(1.0 - pow((double)b1, (double)step)) : 1.f;
    a.bc2 = step > 0 ? (float)(1.0 - pow((double)b2, (double)step)) : 1.f;
    a.step_dev = step_dev;
    return launch_adam(a, st);
}

static gs_status check_step_io(const gs_step_io* io) {
    if (!io) return fail(GS_ERR_INVALID_ARG, "io is NULL");
    if (!io->target_rgb || !io->out_rgb || !io->out_depth || !io->dl_drgb || !io->loss_out)
        return fail(GS_ERR_INVALID_ARG, "target_rgb, out_rgb, out_depth, dl_drgb and loss_out are required");
    if (io->target_depth && !io->dl_ddepth) return fail(GS_ERR_INVALID_ARG, "the depth loss needs dl_ddepth");
    if ((io->host_target_depth && !io->target_depth) || (io->host_mask && !io->mask))
        return fail(GS_ERR_INVALID_ARG, "host targets need the device buffers they are copied into");
    return GS_OK;
}

// Copies the step's host targets into its device buffers on stream `st`.
static cudaError_t upload_targets(const gs_step_io* io, const gs_ws_layout* L, cudaStream_t st) {
    const size_t P = (size_t)L->total_pixels;
    cudaError_t e = cudaSuccess;
    if (io->host_target_rgb)
        e = cudaMemcpyAsync(const_cast<float*>(io->target_rgb), io->host_target_rgb, sizeof(float) * 3 * P,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && io->host_target_depth)
        e = cudaMemcpyAsync(const_cast<float*>(io->target_depth), io->host_target_depth, sizeof(float) * P,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && io->host_mask)
        e = cudaMemcpyAsync(const_cast<uint8_t*>(io->mask), io->host_mask, P, cudaMemcpyHostToDevice, st);
    return e;
}

// A second stream and fork / join events: the upload branch of a captured step.
struct CopyBranch {
    cudaStream_t st = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

static gs_status run_step_tail(gs_gaussians* params, gs_gaussians* grads, gs_gaussians* m, gs_gaussians* v,
                               const gs_render_opts* opts, const gs_ws_layout* L, const Geometry& G, void* ws,
                               const gs_step_io* io, cudaStream_t st);

// The whole step on one stream (no host synchronisation, capturable).
static gs_status run_step(gs_gaussians* params, gs_gaussians* grads, gs_gaussians* m, gs_gaussians* v,
                          const gs_render_opts* opts, const gs_ws_layout* L, const Geometry& G, void* ws,
                          const gs_step_io* io, cudaStream_t st, const CopyBranch* cb = nullptr) {
    gs_status s;
    const bool host_in = io->host_target_rgb || io->host_target_depth || io->host_mask;
    const bool branch = host_in && cb && cb->st;
    if (branch) {
        GS_CUDA(cudaEventRecord(cb->fork, st));
        GS_CUDA(cudaStreamWaitEvent(cb->st, cb->fork, 0));
        GS_CUDA(upload_targets(io, L, cb->st));
        GS_CUDA(cudaEventRecord(cb->join, cb->st));
    } else if (host_in) {
        GS_CUDA(upload_targets(io, L, st));
    }
    if ((s = upload_views(ws, *L, G, L->n_views, st)) != GS_OK) return s;
    GS_CUDA(run_project(params, opts, L, ws, st));
    GS_CUDA(run_bin_sort(opts, L, ws, st));
    if (branch) GS_CUDA(cudaStreamWaitEvent(st, cb->join, 0));   // targets needed from here on
    s = run_step_tail(params, grads, m, v, opts, L, G, ws, io, st);
    if (s == GS_OK && io->host_loss_out)
        GS_CUDA(cudaMemcpyAsync(io->host_loss_out, io->loss_out, sizeof(float) * (L->n_views + 1),
                                cudaMemcpyDeviceToHost, st));
    return s;
}

// The step after the binning: compositing with the loss, backward and update.
static gs_status run_step_tail(gs_gaussians* params, gs_gaussians* grads, gs_gaussians* m, gs_gaussians* v,
                               const gs_render_opts* opts, const gs_ws_layout* L, const Geometry& G, void* ws,
                               const gs_step_io* io, cudaStream_t st) {
    if (opts->persistent) {
        // loss normalisers first (the forward's epilogue reads them), then one persistent
        // kernel for forward, backward, projection backward and Adam
        double* sums = at<double>(ws, L->loss_acc);
        uint32_t* counts = reinterpret_cast<uint32_t*>(sums + 3 * GS_MAX_VIEWS);
        GS_CUDA(cudaMemsetAsync(sums, 0, kLossAccBytes, st));
        GS_CUDA(launch_loss_count(at<View>(ws, L->views), L->n_views, G.pix, io->target_depth, io->mask, counts, st));
        if (io->grad_twist) GS_CUDA(cudaMemsetAsync(io->grad_twist, 0, sizeof(float) * 6 * L->n_views, st));
        const float* dl_dd = io->target_depth ? io->dl_ddepth : nullptr;
        const FwdArgs fa_ = fwd_args(opts, L, ws, io->out_rgb, io->out_depth, nullptr, io->target_rgb, io->target_depth,
                                     io->mask, io->dl_drgb, io->target_depth ? io->dl_ddepth : nullptr);
        Counters* c = at<Counters>(ws, L->counters);
        FusedAdam fad{params, m, v, io->update_mask, io->lr, io->b1, io->b2, io->eps, 0, c};
        GS_CUDA(launch_step_persistent(fa_, bwd_args(opts, L, ws, io->dl_drgb, dl_dd),
                                       pbwd_args(params, opts, L, ws, nullptr, io->grad_twist, &fad), params->sh_degree,
                                       L->total_tiles, opts->lambda_rgb, opts->lambda_depth, io->target_depth != nullptr,
                                       io->loss_out, io->b1, io->b2, opts->sync_spin_limit, opts->sync_skip_block, st,
                                       nullptr));
        return GS_OK;
    }
    // with the update, the fused loss's terms are written by the record clear that starts the
    // backward (one kernel fewer)
    LossFinal lf;
    GS_CUDA(run_fwd(opts, L, G, ws, io->out_rgb, io->out_depth, nullptr, io->target_rgb, io->target_depth, io->mask,
                    io->dl_drgb, io->target_depth ? io->dl_ddepth : nullptr, io->loss_out, st,
                    io->optimize ? &lf : nullptr));
    if (io->grad_twist) GS_CUDA(cudaMemsetAsync(io->grad_twist, 0, sizeof(float) * 6 * L->n_views, st));
    const float* dl_dd = io->target_depth ? io->dl_ddepth : nullptr;
    if (io->optimize) {
        Counters* c = at<Counters>(ws, L->counters);
        // (the record clear before the compositing also advances the Adam step counter)
        GS_CUDA(run_composite_bwd(opts, L, ws, io->dl_drgb, dl_dd, st, c, io->b1, io->b2, lf));
        FusedAdam fa{params, m, v, io->update_mask, io->lr, io->b1, io->b2, io->eps, 0, c};
        GS_CUDA(run_project_bwd(params, opts, L, ws, nullptr, io->grad_twist, st, &fa));
    } else {
        GS_CUDA(run_bwd(params, opts, L, ws, io->dl_drgb, dl_dd, grads, io->grad_twist, st));
    }
    return GS_OK;
}

static gs_status check_step(gs_gaussians* params, gs_gaussians* grads, gs_gaussians* m, gs_gaussians* v,
                            const gs_camera* cams, const gs_render_opts* opts, const gs_ws_layout* L, void* ws,
                            const gs_step_io* io, Geometry& G) {
    gs_status s;
    if ((s = check_ws(ws, L)) != GS_OK) return s;
    if ((s = check_step_io(io)) != GS_OK) return s;
    if ((s = check_adam(params, grads, m, v, io->lr, io->b1, io->b2, io->eps)) != GS_OK) return s;
    if (params->n != L->n) return fail(GS_ERR_INVALID_ARG, "n does not match the layout");
    if (opts->persistent &&
        (opts->tile != 16 || opts->chunk != 256 || !io->optimize || opts->lambda_ssim > 0.f || opts->mask_erode >= 0 ||
         opts->count_fragments))
        return fail(GS_ERR_UNSUPPORTED, "the persistent step needs tile 16, chunk 256, optimize = 1, the fused L1 loss "
                                        "and no fragment counters");
    return geometry_for(L, cams, opts, G);
}

// Captured step: the graph, its executable and the node of the view-table upload, whose
// by-value camera argument gs_graph_set_cameras rewrites.
struct GraphState {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t views_node = nullptr;
    cudaKernelNodeParams views_params;
    gs_render_opts opts;
    gs_ws_layout layout;
    void* ws = nullptr;
    CopyBranch copy;   // the host-target upload branch (created only when the step has one)
};

static void release_copy_branch(CopyBranch& c) {
    if (c.fork) cudaEventDestroy(c.fork);
    if (c.join) cudaEventDestroy(c.join);
    if (c.st) cudaStreamDestroy(c.st);
    c = CopyBranch();
}

// Error recording for entry points defined in other translation units.
gs_status record_error(gs_status s, const char* msg) { return fail(s, "%s", msg); }

}  // namespace gs

using namespace gs;

extern "C" {

const char* gs_last_error(void) { return g_err.c_str(); }
const char* gs_version(void) { return "gs-gb300 0.1 (sm_103a)"; }

void gs_default_opts(gs_render_opts* o) {
    if (!o) return;
    o->near_z = 0.2f;
    o->dilation = 0.3f;
    o->alpha_min = 1.0f / 255.0f;
    o->alpha_max = 0.99f;
    o->T_min = 1e-4f;
    o->clamp_fov = 1.3f;
    o->bg[0] = o->bg[1] = o->bg[2] = 0.f;
    o->lambda_rgb = 1.0f;
    o->lambda_depth = 0.1f;
    o->tile = 16;
    o->chunk = 64;
    o->count_fragments = 0;
    o->lambda_ssim = 0.0f;
    o->mask_opacity = 0.5f;
    o->mask_erode = -1;
    o->persistent = 0;
    o->sync_spin_limit = 0;
    o->sync_skip_block = -1;
}

size_t gs_workspace_size(int64_t n, int32_t n_views, const gs_camera* cams, const gs_render_opts* opts,
                         int64_t max_pairs) {
    gs_ws_layout L;
    Geometry G;
    if (layout(n, n_views, cams, opts, max_pairs, L, G) != GS_OK) return 0;
    return L.total;
}

gs_status gs_workspace_layout(int64_t n, int32_t n_views, const gs_camera* cams, const gs_render_opts* opts,
                              int64_t max_pairs, gs_ws_layout* out) {
    if (!out) return fail(GS_ERR_INVALID_ARG, "out is NULL");
    Geometry G;
    return layout(n, n_views, cams, opts, max_pairs, *out, G);
}

gs_status gs_read_counters(const gs_ws_layout* L, const void* ws, gs_counters* out, void* stream) {
    if (!ws || !out || !L) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    Counters c;
    GS_CUDA(cudaMemcpyAsync(&c, at<Counters>(const_cast<void*>(ws), L->counters), sizeof(c), cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    out->status = c.status;
    out->n_entries = c.n_entries32;
    out->n_pairs = c.n_pairs;
    out->adam_step = c.adam_step;
    out->frag_fwd_eval = c.frag_fwd_eval;
    out->frag_fwd_add = c.frag_fwd_add;
    out->frag_bwd_eval = c.frag_bwd_eval;
    out->frag_bwd_add = c.frag_bwd_add;
    out->visits_fwd = c.visits_fwd;
    out->visits_bwd = c.visits_bwd;
    return GS_OK;
}

gs_status gs_workspace_init(const gs_ws_layout* L, void* ws, void* stream) {
    gs_status s;
    if ((s = check_ws(ws, L)) != GS_OK) return s;
    GS_CUDA(cudaMemsetAsync(at<Counters>(ws, L->counters), 0, sizeof(Counters), (cudaStream_t)stream));
    return GS_OK;
}

gs_status gs_project(const gs_gaussians* g, const gs_camera* cams, const gs_render_opts* opts, const gs_ws_layout* L,
                     void* ws, void* stream) {
    gs_status s = check_gaussians(g, true);
    if (s != GS_OK) return s;
    if ((s = check_ws(ws, L)) != GS_OK) return s;
    if (g->n != L->n) return fail(GS_ERR_INVALID_ARG, "n = %lld does not match the layout (%lld)", (long long)g->n, (long long)L->n);
    Geometry G;
    if ((s = geometry_for(L, cams, opts, G)) != GS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = upload_views(ws, *L, G, L->n_views, st)) != GS_OK) return s;
    GS_CUDA(run_project(g, opts, L, ws, st));
    return GS_OK;
}

gs_status gs_bin_sort(const gs_camera* cams, const gs_render_opts* opts, const gs_ws_layout* L, void* ws, void* stream) {
    gs_status s;
    if ((s = check_ws(ws, L)) != GS_OK) return s;
    Geometry G;
    if ((s = geometry_for(L, cams, opts, G)) != GS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = upload_views(ws, *L, G, L->n_views, st)) != GS_OK) return s;
    GS_CUDA(run_bin_sort(opts, L, ws, st));
    return GS_OK;
}

gs_status gs_render_fwd(const gs_camera* cams, const gs_render_opts* opts, const gs_ws_layout* L, void* ws,
                        float* out_rgb, float* out_depth, float* out_T, const float* target_rgb,
                        const float* target_depth, const uint8_t* mask, float* dl_drgb, float* dl_ddepth,
                        float* loss_out, void* stream) {
    gs_status s;
    if ((s = check_ws(ws, L)) != GS_OK) return s;
    Geometry G;
    if ((s = geometry_for(L, cams, opts, G)) != GS_OK) return s;
    if (!out_rgb || !out_depth) return fail(GS_ERR_INVALID_ARG, "out_rgb and out_depth are required");
    if (target_rgb && (!dl_drgb || !loss_out)) return fail(GS_ERR_INVALID_ARG, "the loss needs dl_drgb and loss_out");
    if (target_depth && !target_rgb) return fail(GS_ERR_INVALID_ARG, "target_depth needs target_rgb");
    if (target_depth && !dl_ddepth) return fail(GS_ERR_INVALID_ARG, "the depth loss needs dl_ddepth");
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = upload_views(ws, *L, G, L->n_views, st)) != GS_OK) return s;
    GS_CUDA(run_fwd(opts, L, G, ws, out_rgb, out_depth, out_T, target_rgb, target_depth, mask, dl_drgb, dl_ddepth,
                    loss_out, st));
    return GS_OK;
}

gs_status gs_render_mask(const gs_camera* cams, const gs_render_opts* opts, const gs_ws_layout* L, void* ws,
                         const uint8_t* caller_mask, uint8_t* mask_out, void* stream) {
    gs_status s;
    if ((s = check_ws(ws, L)) != GS_OK) return s;
    Geometry G;
    if ((s = geometry_for(L, cams, opts, G)) != GS_OK) return s;
    if (!mask_out) return fail(GS_ERR_INVALID_ARG, "mask_out is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = upload_views(ws, *L, G, L->n_views, st)) != GS_OK) return s;
    GS_CUDA(run_render_mask(opts, L, G, ws, caller_mask, mask_out, st));
    return GS_OK;
}

gs_status gs_objective(const gs_camera* cams, const gs_render_opts* opts, const gs_ws_layout* L, void* ws,
                       const float* rgb, const float* depth, const float* target_rgb, const float* target_depth,
                       const uint8_t* mask, float* dl_drgb, float* dl_ddepth, float* loss_out, void* stream) {
    gs_status s;
    if ((s = check_ws(ws, L)) != GS_OK) return s;
    Geometry G;
    if ((s = geometry_for(L, cams, opts, G)) != GS_OK) return s;
    if (!rgb || !target_rgb || !dl_drgb || !loss_out) return fail(GS_ERR_INVALID_ARG, "rgb, target_rgb, dl_drgb and loss_out are required");
    if (target_depth && (!depth || !dl_ddepth)) return fail(GS_ERR_INVALID_ARG, "the depth term needs depth and dl_ddepth");
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = upload_views(ws, *L, G, L->n_views, st)) != GS_OK) return s;
    GS_CUDA(run_objective(opts, L, G, ws, rgb, depth, target_rgb, target_depth, mask, dl_drgb, dl_ddepth, loss_out, st));
    return GS_OK;
}

gs_status gs_render_bwd(const gs_gaussians* g, const gs_camera* cams, const gs_render_opts* opts, const gs_ws_layout* L,
                        void* ws, const float* dl_drgb, const float* dl_ddepth, gs_gaussians* grads, float* grad_twist,
                        void* stream) {
    gs_status s = check_gaussians(g, true);
    if (s != GS_OK) return s;
    if ((s = check_gaussians(grads, true)) != GS_OK) return s;
    if ((s = check_ws(ws, L)) != GS_OK) return s;
    if (g->n != L->n || grads->n != L->n || grads->sh_degree != g->sh_degree)
        return fail(GS_ERR_INVALID_ARG, "gaussians / grads do not match the layout");
    if (!dl_drgb) return fail(GS_ERR_INVALID_ARG, "dl_drgb is required");
    Geometry G;
    if ((s = geometry_for(L, cams, opts, G)) != GS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = upload_views(ws, *L, G, L->n_views, st)) != GS_OK) return s;
    GS_CUDA(run_bwd(g, opts, L, ws, dl_drgb, dl_ddepth, grads, grad_twist, st));
    return GS_OK;
}

gs_status gs_composite_bwd(const gs_camera* cams, const gs_render_opts* opts, const gs_ws_layout* L, void* ws,
                           const float* dl_drgb, const float* dl_ddepth, void* stream) {
    gs_status s;
    if ((s = check_ws(ws, L)) != GS_OK) return s;
    if (!dl_drgb) return fail(GS_ERR_INVALID_ARG, "dl_drgb is required");
    Geometry G;
    if ((s = geometry_for(L, cams, opts, G)) != GS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = upload_views(ws, *L, G, L->n_views, st)) != GS_OK) return s;
    GS_CUDA(run_composite_bwd(opts, L, ws, dl_drgb, dl_ddepth, st));
    return GS_OK;
}

gs_status gs_project_bwd(const gs_gaussians* g, const gs_camera* cams, const gs_render_opts* opts,
                         const gs_ws_layout* L, void* ws, gs_gaussians* grads, float* grad_twist, void* stream) {
    gs_status s = check_gaussians(g, true);
    if (s != GS_OK) return s;
    if ((s = check_gaussians(grads, true)) != GS_OK) return s;
    if ((s = check_ws(ws, L)) != GS_OK) return s;
    if (g->n != L->n || grads->n != L->n || grads->sh_degree != g->sh_degree)
        return fail(GS_ERR_INVALID_ARG, "gaussians / grads do not match the layout");
    Geometry G;
    if ((s = geometry_for(L, cams, opts, G)) != GS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = upload_views(ws, *L, G, L->n_views, st)) != GS_OK) return s;
    GS_CUDA(run_project_bwd(g, opts, L, ws, grads, grad_twist, st));
    return GS_OK;
}

gs_status gs_project_bwd_adam(gs_gaussians* params, const gs_camera* cams, const gs_render_opts* opts,
                              const gs_ws_layout* L, void* ws, gs_gaussians* m, gs_gaussians* v,
                              const uint8_t* update_mask, const float lr[6], float b1, float b2, float eps,
                              int64_t step, float* grad_twist, void* stream) {
    gs_status s;
    // the parameter planes stand in for the (unused) gradient planes in the shape checks
    if ((s = check_adam(params, params, m, v, lr, b1, b2, eps)) != GS_OK) return s;
    if (step < 1) return fail(GS_ERR_INVALID_ARG, "step must be >= 1");
    if ((s = check_ws(ws, L)) != GS_OK) return s;
    if (params->n != L->n) return fail(GS_ERR_INVALID_ARG, "gaussians do not match the layout");
    Geometry G;
    if ((s = geometry_for(L, cams, opts, G)) != GS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = upload_views(ws, *L, G, L->n_views, st)) != GS_OK) return s;
    FusedAdam fa{params, m, v, update_mask, lr, b1, b2, eps, step, nullptr};
    GS_CUDA(run_project_bwd(params, opts, L, ws, nullptr, grad_twist, st, &fa));
    return GS_OK;
}

gs_status gs_adam_step(gs_gaussians* params, gs_gaussians* grads, gs_gaussians* m, gs_gaussians* v,
                       const uint8_t* update_mask, const uint8_t* visible, const float lr[6], float b1, float b2,
                       float eps, int64_t step, void* stream) {
    gs_status s;
    if ((s = check_adam(params, grads, m, v, lr, b1, b2, eps)) != GS_OK) return s;
    if (step < 1) return fail(GS_ERR_INVALID_ARG, "step must be >= 1");
    GS_CUDA(run_adam(params, grads, m, v, update_mask, visible, lr, b1, b2, eps, step, nullptr, (cudaStream_t)stream));
    return GS_OK;
}

gs_status gs_step(gs_gaussians* params, gs_gaussians* grads, gs_gaussians* m, gs_gaussians* v, const gs_camera* cams,
                  const gs_render_opts* opts, const gs_ws_layout* L, void* ws, const gs_step_io* io, void* stream) {
    Geometry G;
    gs_status s = check_step(params, grads, m, v, cams, opts, L, ws, io, G);
    if (s != GS_OK) return s;
    return run_step(params, grads, m, v, opts, L, G, ws, io, (cudaStream_t)stream);
}

gs_status gs_graph_create(gs_graph* out, gs_gaussians* params, gs_gaussians* grads, gs_gaussians* m, gs_gaussians* v,
                          const gs_camera* cams, const gs_render_opts* opts, const gs_ws_layout* L, void* ws,
                          const gs_step_io* io, void* stream) {
    if (!out) return fail(GS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!stream) return fail(GS_ERR_INVALID_ARG, "capture needs a non-default stream");
    Geometry G;
    gs_status s = check_step(params, grads, m, v, cams, opts, L, ws, io, G);
    if (s != GS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    GraphState* gst = new GraphState();
    gst->opts = *opts;
    gst->layout = *L;
    gst->ws = ws;
    if (io->host_target_rgb || io->host_target_depth || io->host_mask) {
        cudaError_t e = cudaStreamCreateWithFlags(&gst->copy.st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&gst->copy.fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&gst->copy.join, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            release_copy_branch(gst->copy);
            delete gst;
            return fail(GS_ERR_CUDA, "copy branch: %s", cudaGetErrorString(e));
        }
    }
    {
        const cudaError_t eb = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (eb != cudaSuccess) {
            release_copy_branch(gst->copy);
            delete gst;
            return fail(GS_ERR_CUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(eb));
        }
    }
    s = run_step(params, grads, m, v, opts, L, G, ws, io, st, &gst->copy);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(st, &graph);
    if (s != GS_OK || ec != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        release_copy_branch(gst->copy);
        delete gst;
        return s != GS_OK ? s : fail(GS_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(ec));
    }
    gst->graph = graph;
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    cudaGraphNode_t* nodes = new cudaGraphNode_t[nn ? nn : 1];
    cudaGraphGetNodes(graph, nodes, &nn);
    for (size_t i = 0; i < nn; i++) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp;
        if (cudaGraphKernelNodeGetParams(nodes[i], &kp) != cudaSuccess) continue;
        if (kp.func == reinterpret_cast<void*>(setup_views_kernel)) {
            gst->views_node = nodes[i];
            gst->views_params = kp;
        }
    }
    delete[] nodes;
    const cudaError_t ei = cudaGraphInstantiate(&gst->exec, graph, 0);
    if (ei != cudaSuccess || !gst->views_node) {
        cudaGraphDestroy(graph);
        release_copy_branch(gst->copy);
        delete gst;
        return fail(GS_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ei));
    }
    *out = reinterpret_cast<gs_graph>(gst);
    return GS_OK;
}

gs_status gs_graph_launch(gs_graph g, void* stream) {
    if (!g) return fail(GS_ERR_INVALID_ARG, "graph is NULL");
    GraphState* gst = reinterpret_cast<GraphState*>(g);
    GS_CUDA(cudaGraphLaunch(gst->exec, (cudaStream_t)stream));
    return GS_OK;
}

gs_status gs_graph_set_cameras(gs_graph g, const gs_camera* cams) {
    if (!g) return fail(GS_ERR_INVALID_ARG, "graph is NULL");
    GraphState* gst = reinterpret_cast<GraphState*>(g);
    Geometry G;
    gs_status s = geometry_for(&gst->layout, cams, &gst->opts, G);
    if (s != GS_OK) return s;
    ViewsParam p;
    memset(&p, 0, sizeof(p));
    p.n = gst->layout.n_views;
    memcpy(p.v, G.views, sizeof(View) * p.n);
    View* dst = at<View>(gst->ws, gst->layout.views);
    void* args[2] = {&dst, &p};
    cudaKernelNodeParams kp = gst->views_params;
    kp.kernelParams = args;
    kp.extra = nullptr;
    GS_CUDA(cudaGraphExecKernelNodeSetParams(gst->exec, gst->views_node, &kp));
    return GS_OK;
}

gs_status gs_graph_destroy(gs_graph g) {
    if (!g) return GS_OK;
    GraphState* gst = reinterpret_cast<GraphState*>(g);
    if (gst->exec) cudaGraphExecDestroy(gst->exec);
    if (gst->graph) cudaGraphDestroy(gst->graph);
    release_copy_branch(gst->copy);
    delete gst;
    return GS_OK;
}


// ---------------------------------------------------------------------------------------
// f2: map-size updates between mapping iterations (mapupdate.cu).
// ---------------------------------------------------------------------------------------
static int map_planes(const gs_gaussians* g, int64_t stride, const float** out) {
    const int K = (g->sh_degree + 1) * (g->sh_degree + 1);
    int p = 0;
    for (int k = 0; k < 3; k++) out[p++] = g->means + k * stride;
    for (int k = 0; k < 3; k++) out[p++] = g->log_scales + k * stride;
    for (int k = 0; k < 4; k++) out[p++] = g->quats + k * stride;
    out[p++] = g->opacity_logits;
    for (int k = 0; k < 3 * K; k++) out[p++] = g->sh + k * stride;
    return p;
}

// The plans and the update read their counts back: they synchronize the caller's stream.
static gs_status sync_counts(cudaStream_t st) {
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(GS_ERR_CUDA, "%s", cudaGetErrorString(e));
    return GS_OK;
}

size_t gs_map_update_scratch_bytes(int64_t n_map, int64_t n_new) {
    if (n_map < 0 || n_new < 0) return 0;
    return map_update_scratch_bytes(n_map, n_new);
}

gs_status gs_prune_plan(const gs_gaussians* g, float opacity_min, double max_ratio, uint8_t* keep, void* scratch,
                        size_t scratch_bytes, int64_t* n_keep, void* stream) {
    gs_status s = check_gaussians(g, true);
    if (s != GS_OK) return s;
    if (!keep || !scratch || !n_keep) return fail(GS_ERR_INVALID_ARG, "keep, scratch and n_keep are required");
    if (!(opacity_min > 0.f && opacity_min < 1.f) || !(max_ratio >= 0.0 && max_ratio <= 1.0))
        return fail(GS_ERR_INVALID_ARG, "need 0 < opacity_min < 1 and 0 <= max_ratio <= 1");
    if (g->n >= (int64_t)0xFFFFFFFFll) return fail(GS_ERR_INVALID_ARG, "n must be < 2^32");
    if (scratch_bytes < map_update_scratch_bytes(g->n, 0)) return fail(GS_ERR_INVALID_ARG, "scratch too small");
    // the FP32 logit of opacity_min: sigmoid(logit) < opacity_min iff logit < it
    const float thr = (float)log((double)opacity_min / (1.0 - (double)opacity_min));
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long kept = 0;
    GS_CUDA(launch_prune_plan(g->opacity_logits, g->n, thr, max_ratio, keep, scratch, &kept, st));
    if ((s = sync_counts(st)) != GS_OK) return s;
    *n_keep = (int64_t)kept;
    return GS_OK;
}

gs_status gs_dedup_plan(const gs_gaussians* map, const float* new_means, int64_t n_new, float radius,
                        uint8_t* accept, void* scratch, size_t scratch_bytes, int64_t* n_accept, void* stream) {
    gs_status s = check_gaussians(map, false);
    if (s != GS_OK) return s;
    if (map->n > 0 && !map->means) return fail(GS_ERR_INVALID_ARG, "map means are NULL");
    if (n_new < 0 || (n_new > 0 && (!new_means || !accept)) || !scratch || !n_accept)
        return fail(GS_ERR_INVALID_ARG, "new_means, accept, scratch and n_accept are required");
    if (!(radius > 0.f)) return fail(GS_ERR_INVALID_ARG, "radius must be > 0");
    if (map->n >= (int64_t)0x7FFFFFFFll || n_new >= (int64_t)0x7FFFFFFFll) return fail(GS_ERR_INVALID_ARG, "sizes must be < 2^31");
    if (scratch_bytes < map_update_scratch_bytes(map->n, n_new)) return fail(GS_ERR_INVALID_ARG, "scratch too small");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long acc = 0;
    GS_CUDA(launch_dedup_plan(map->means, map->n, new_means, n_new, radius, accept, scratch, &acc, st));
    if ((s = sync_counts(st)) != GS_OK) return s;
    *n_accept = (int64_t)acc;
    return GS_OK;
}

gs_status gs_map_update(const gs_gaussians* in, const gs_gaussians* m_in, const gs_gaussians* v_in, const uint8_t* keep,
                        const gs_gaussians* new_rows, const uint8_t* accept, const uint32_t* tags_in,
                        const uint32_t* new_tags, gs_gaussians* out, gs_gaussians* m_out, gs_gaussians* v_out,
                        uint32_t* tags_out, void* scratch, size_t scratch_bytes, void* stream) {
    gs_status s;
    const gs_gaussians* need[6] = {in, m_in, v_in, out, m_out, v_out};
    for (const gs_gaussians* g : need)
        if ((s = check_gaussians(g, true)) != GS_OK) return s;
    if (new_rows && (s = check_gaussians(new_rows, true)) != GS_OK) return s;
    const int deg = in->sh_degree;
    if (m_in->n != in->n || v_in->n != in->n || m_out->n != out->n || v_out->n != out->n ||
        m_in->sh_degree != deg || v_in->sh_degree != deg || out->sh_degree != deg || m_out->sh_degree != deg ||
        v_out->sh_degree != deg || (new_rows && new_rows->sh_degree != deg))
        return fail(GS_ERR_INVALID_ARG, "the maps, moments and new rows must agree in n and sh_degree");
    if (!keep || !scratch) return fail(GS_ERR_INVALID_ARG, "keep and scratch are required");
    const int64_t n_new = new_rows ? new_rows->n : 0;
    if (in->n >= (int64_t)0x7FFFFFFFll || n_new >= (int64_t)0x7FFFFFFFll) return fail(GS_ERR_INVALID_ARG, "sizes must be < 2^31");
    if (scratch_bytes < map_update_scratch_bytes(in->n, n_new)) return fail(GS_ERR_INVALID_ARG, "scratch too small");
    cudaStream_t st = (cudaStream_t)stream;
    MapUpdateArgs a;
    memset(&a, 0, sizeof(a));
    uint32_t totals[2] = {0, 0};
    uint32_t *pk = nullptr, *pn = nullptr;
    GS_CUDA(launch_map_scan(keep, in->n, new_rows ? accept : nullptr, n_new, scratch, &pk, &pn, totals, st));
    if ((s = sync_counts(st)) != GS_OK) return s;
    const int64_t n_acc = new_rows ? (accept ? (int64_t)totals[1] : n_new) : 0;
    if (out->n != (int64_t)totals[0] + n_acc)
        return fail(GS_ERR_INVALID_ARG, "out->n must be %lld (kept %u + accepted %lld), got %lld",
                    (long long)((int64_t)totals[0] + n_acc), totals[0], (long long)n_acc, (long long)out->n);
    a.n = in->n; a.n_new = n_new; a.n_out = out->n; a.n_keep = totals[0];
    a.keep = keep; a.accept = new_rows ? accept : nullptr; a.pos_keep = pk; a.pos_new = pn;
    a.n_planes = map_planes(in, in->n, a.in);
    map_planes(m_in, in->n, a.m_in);
    map_planes(v_in, in->n, a.v_in);
    if (new_rows) map_planes(new_rows, n_new, a.nw);
    map_planes(out, out->n, const_cast<const float**>(a.out));
    map_planes(m_out, out->n, const_cast<const float**>(a.m_out));
    map_planes(v_out, out->n, const_cast<const float**>(a.v_out));
    a.tags_in = tags_in; a.new_tags = new_tags; a.tags_out = tags_out;
    GS_CUDA(launch_compact(a, st));
    return GS_OK;
}


// ---------------------------------------------------------------------------------------
// f3: Gaussian-GICP loop registration (gicp.cu); host side: 6 x 6 solves and SE(3) updates.
// ---------------------------------------------------------------------------------------
static GicpMap gicp_map(const gs_gaussians* g) {
    GicpMap m;
    m.n = g->n; m.means = g->means; m.log_scales = g->log_scales; m.quats = g->quats;
    return m;
}

size_t gs_gicp_scratch_bytes(int64_t n_target_map) {
    if (n_target_map < 0) return 0;
    return gicp_scratch_bytes(n_target_map);
}

gs_status gs_gicp_target_set(const gs_gaussians* map, const gs_camera* views, int32_t n_views, float near_z,
                             float d_max, const uint8_t* source_flag, uint8_t* target_flag, void* scratch,
                             size_t scratch_bytes, int64_t* n_target, void* stream) {
    gs_status s = check_gaussians(map, false);
    if (s != GS_OK) return s;
    if (map->n > 0 && !map->means) return fail(GS_ERR_INVALID_ARG, "map means are NULL");
    if (n_views < 1 || n_views > GS_MAX_VIEWS || !views) return fail(GS_ERR_INVALID_ARG, "need 1..%d views", GS_MAX_VIEWS);
    if (!target_flag || !scratch || !n_target) return fail(GS_ERR_INVALID_ARG, "target_flag, scratch and n_target are required");
    if (!(d_max > 0.f) || !(near_z >= 0.f)) return fail(GS_ERR_INVALID_ARG, "need d_max > 0 and near_z >= 0");
    if (scratch_bytes < gicp_scratch_bytes(0)) return fail(GS_ERR_INVALID_ARG, "scratch too small");
    GicpView gv[GS_MAX_VIEWS];
    for (int k = 0; k < n_views; k++) {
        const gs_camera& c = views[k];
        for (int j = 0; j < 9; j++) gv[k].R[j] = c.R_cw[j];
        for (int j = 0; j < 3; j++) gv[k].t[j] = c.t_cw[j];
        // camera centre -R^T t in FP64, rounded once
        for (int j = 0; j < 3; j++) {
            double v = 0;
            for (int r = 0; r < 3; r++) v -= (double)c.R_cw[3 * r + j] * (double)c.t_cw[r];
            gv[k].c[j] = (float)v;
        }
        gv[k].fx = c.fx; gv[k].fy = c.fy; gv[k].cx = c.cx; gv[k].cy = c.cy;
        gv[k].W = (float)c.width; gv[k].H = (float)c.height;
    }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long cnt = 0;
    GS_CUDA(launch_gicp_target_set(gicp_map(map), gv, n_views, near_z, d_max * d_max, source_flag, target_flag, scratch,
                                   &cnt, st));
    if ((s = sync_counts(st)) != GS_OK) return s;
    *n_target = (int64_t)cnt;
    return GS_OK;
}

// (rho, phi) -> 4 x 4 rigid transform
static void se3_exp(const double xi[6], double T[16]) {
    const double* rho = xi;
    const double* phi = xi + 3;
    const double th = sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
    const double K[9] = {0, -phi[2], phi[1], phi[2], 0, -phi[0], -phi[1], phi[0], 0};
    double K2[9];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) K2[3 * r + c] = K[3 * r] * K[c] + K[3 * r + 1] * K[3 + c] + K[3 * r + 2] * K[6 + c];
    double A, B, C;
    if (th < 1e-12) { A = 1.0; B = 0.5; C = 1.0 / 6.0; }
    else { A = sin(th) / th; B = (1 - cos(th)) / (th * th); C = (1 - A) / (th * th); }
    double R[9], V[9];
    for (int k = 0; k < 9; k++) {
        const double I = (k % 4 == 0) ? 1.0 : 0.0;
        R[k] = I + A * K[k] + B * K2[k];
        V[k] = I + B * K[k] + C * K2[k];
    }
    if (th < 1e-12) for (int k = 0; k < 9; k++) { R[k] = ((k % 4 == 0) ? 1.0 : 0.0) + K[k]; V[k] = ((k % 4 == 0) ? 1.0 : 0.0) + 0.5 * K[k]; }
    for (int k = 0; k < 16; k++) T[k] = 0;
    for (int r = 0; r < 3; r++) {
        for (int c = 0; c < 3; c++) T[4 * r + c] = R[3 * r + c];
        T[4 * r + 3] = V[3 * r] * rho[0] + V[3 * r + 1] * rho[1] + V[3 * r + 2] * rho[2];
    }
    T[15] = 1;
}

// Left Jacobian of SE(3) at xi = (rho, phi): J = sum_k ad^k / (k+1)! with the 6 x 6 adjoint
// ad = [[phi^, rho^], [0, phi^]], so that Exp(xi + d) = Exp(J d) Exp(xi) to first order.
// The series is summed until its terms fall below double rounding (at most 120 terms: the
// k-th term is bounded by |xi|^k / (k+1)!).
static void se3_left_jacobian(const double xi[6], double J[36]) {
    double ad[36] = {0};
    auto hat = [&](const double* w, int r0, int c0) {
        ad[6 * (r0 + 0) + c0 + 1] = -w[2]; ad[6 * (r0 + 0) + c0 + 2] = w[1];
        ad[6 * (r0 + 1) + c0 + 0] = w[2];  ad[6 * (r0 + 1) + c0 + 2] = -w[0];
        ad[6 * (r0 + 2) + c0 + 0] = -w[1]; ad[6 * (r0 + 2) + c0 + 1] = w[0];
    };
    hat(xi + 3, 0, 0);
    hat(xi, 0, 3);
    hat(xi + 3, 3, 3);
    double term[36], next[36];
    for (int k = 0; k < 36; k++) term[k] = J[k] = (k % 7 == 0) ? 1.0 : 0.0;
    for (int m = 1; m <= 120; m++) {
        double mx = 0;
        for (int r = 0; r < 6; r++)
            for (int c = 0; c < 6; c++) {
                double s = 0;
                for (int e = 0; e < 6; e++) s += term[6 * r + e] * ad[6 * e + c];
                next[6 * r + c] = s / (double)(m + 1);
                mx = fmax(mx, fabs(next[6 * r + c]));
            }
        for (int k = 0; k < 36; k++) { term[k] = next[k]; J[k] += next[k]; }
        if (mx < 1e-18) break;
    }
}

static bool finite_twist(const float* xi, int32_t n_views) {
    for (int k = 0; k < 6 * n_views; k++)
        if (!std::isfinite(xi[k])) return false;
    return true;
}

gs_status gs_twist_cameras(const gs_camera* cams, const float* xi, int32_t n_views, gs_camera* out) {
    if (!cams || !xi || !out) return fail(GS_ERR_INVALID_ARG, "cams, xi and out are required");
    if (n_views < 1 || n_views > GS_MAX_VIEWS) return fail(GS_ERR_INVALID_ARG, "need 1..%d views", GS_MAX_VIEWS);
    if (!finite_twist(xi, n_views)) return fail(GS_ERR_NONFINITE, "a twist component is not finite");
    for (int v = 0; v < n_views; v++) {
        double x[6], E[16];
        for (int k = 0; k < 6; k++) x[k] = xi[6 * v + k];
        se3_exp(x, E);
        gs_camera c = cams[v];
        for (int r = 0; r < 3; r++) {
            double t = E[4 * r + 3];
            for (int e = 0; e < 3; e++) t += E[4 * r + e] * (double)cams[v].t_cw[e];
            c.t_cw[r] = (float)t;
            for (int col = 0; col < 3; col++) {
                double s = 0;
                for (int e = 0; e < 3; e++) s += E[4 * r + e] * (double)cams[v].R_cw[3 * e + col];
                c.R_cw[3 * r + col] = (float)s;
            }
        }
        out[v] = c;
    }
    return GS_OK;
}

gs_status gs_twist_grad(const float* xi, const float* g_left, int32_t n_views, float* g_xi) {
    if (!xi || !g_left || !g_xi) return fail(GS_ERR_INVALID_ARG, "xi, g_left and g_xi are required");
    if (n_views < 1 || n_views > GS_MAX_VIEWS) return fail(GS_ERR_INVALID_ARG, "need 1..%d views", GS_MAX_VIEWS);
    if (!finite_twist(xi, n_views)) return fail(GS_ERR_NONFINITE, "a twist component is not finite");
    for (int v = 0; v < n_views; v++) {
        double x[6], J[36];
        for (int k = 0; k < 6; k++) x[k] = xi[6 * v + k];
        se3_left_jacobian(x, J);
        for (int c = 0; c < 6; c++) {
            double s = 0;
            for (int r = 0; r < 6; r++) s += J[6 * r + c] * (double)g_left[6 * v + r];
            g_xi[6 * v + c] = (float)s;
        }
    }
    return GS_OK;
}

// Solves H x = b (6 x 6, symmetric positive definite) by Cholesky; false if not positive.
static bool solve6(const double H[36], const double b[6], double x[6]) {
    double L[36] = {0};
    for (int i = 0; i < 6; i++)
        for (int j = 0; j <= i; j++) {
            double s = H[6 * i + j];
            for (int k = 0; k < j; k++) s -= L[6 * i + k] * L[6 * j + k];
            if (i == j) {
                if (!(s > 0)) return false;
                L[6 * i + i] = sqrt(s);
            } else {
                L[6 * i + j] = s / L[6 * j + j];
            }
        }
    double y[6];
    for (int i = 0; i < 6; i++) {
        double s = b[i];
        for (int k = 0; k < i; k++) s -= L[6 * i + k] * y[k];
        y[i] = s / L[6 * i + i];
    }
    for (int i = 5; i >= 0; i--) {
        double s = y[i];
        for (int k = i + 1; k < 6; k++) s -= L[6 * k + i] * x[k];
        x[i] = s / L[6 * i + i];
    }
    return true;
}

gs_status gs_gicp_register(const gs_gaussians* src, const uint8_t* src_flag, const gs_gaussians* tar,
                           const uint8_t* tar_flag, const double T_init[12], float d_corr, int32_t max_iters,
                           double eps, gs_gicp_result* result, void* scratch, size_t scratch_bytes, void* stream) {
    gs_status s;
    if ((s = check_gaussians(src, true)) != GS_OK) return s;
    if ((s = check_gaussians(tar, true)) != GS_OK) return s;
    if (!T_init || !result || !scratch) return fail(GS_ERR_INVALID_ARG, "T_init, result and scratch are required");
    if (!(d_corr > 0.f) || max_iters < 1 || !(eps > 0.0)) return fail(GS_ERR_INVALID_ARG, "need d_corr > 0, max_iters >= 1, eps > 0");
    if (tar->n >= (int64_t)0x7FFFFFFFll || src->n >= (int64_t)0x7FFFFFFFll) return fail(GS_ERR_INVALID_ARG, "sizes must be < 2^31");
    if (scratch_bytes < gicp_scratch_bytes(tar->n)) return fail(GS_ERR_INVALID_ARG, "scratch too small");
    cudaStream_t st = (cudaStream_t)stream;
    const GicpMap gs_src = gicp_map(src), gs_tar = gicp_map(tar);
    GS_CUDA(launch_gicp_build(gs_tar, tar_flag, d_corr, scratch, st));
    double T[16];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 4; c++) T[4 * r + c] = T_init[4 * r + c];
    T[12] = T[13] = T[14] = 0; T[15] = 1;
    double acc[29];
    auto evaluate = [&]() -> cudaError_t {
        const double R[9] = {T[0], T[1], T[2], T[4], T[5], T[6], T[8], T[9], T[10]};
        const double t[3] = {T[3], T[7], T[11]};
        return launch_gicp_normal_eq(gs_src, src_flag, gs_tar, d_corr, R, t, scratch, acc, st);
    };
    int it = 0;
    bool converged = false;
    for (it = 1; it <= max_iters; it++) {
        GS_CUDA(evaluate());
        if (acc[28] < 6) break;
        double H[36], g[6], xi[6];
        int k = 0;
        for (int r = 0; r < 6; r++)
            for (int c = r; c < 6; c++) { H[6 * r + c] = acc[k]; H[6 * c + r] = acc[k]; k++; }
        for (int r = 0; r < 6; r++) g[r] = -acc[21 + r];
        if (!solve6(H, g, xi)) break;
        double E[16], Tn[16];
        se3_exp(xi, E);
        for (int r = 0; r < 4; r++)
            for (int c = 0; c < 4; c++) {
                double v = 0;
                for (int e = 0; e < 4; e++) v += E[4 * r + e] * T[4 * e + c];
                Tn[4 * r + c] = v;
            }
        for (int k2 = 0; k2 < 16; k2++) T[k2] = Tn[k2];
        double nrm = 0;
        for (int r = 0; r < 6; r++) nrm += xi[r] * xi[r];
        if (sqrt(nrm) < eps) { converged = true; break; }
    }
    GS_CUDA(evaluate());
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 4; c++) result->T[4 * r + c] = T[4 * r + c];
    result->cost = acc[27];
    result->n_corr = (int64_t)acc[28];
    result->iters = it > max_iters ? max_iters : it;
    result->converged = converged ? 1 : 0;
    return GS_OK;
}

}  // extern "C"
