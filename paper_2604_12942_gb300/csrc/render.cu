// a5-a6: front-to-back compositing of colour and depth with the fused L1 loss, and its
// backward with transmittance recomputed back to front.  RMGS-SLAM §III-C: colour by
// standard alpha compositing, depth D = sum z_i T_i alpha_i with the same weights, loss
// lambda_rgb L_rgb + lambda_depth L_depth over the mask (SSIM weight 0).
//
// One CTA per (view, tile) work item, one or two pixels per thread.  The tile's depth-sorted pair
// list is walked in chunks staged in shared memory (records gathered once per chunk by
// the whole CTA); the inner loop then reads broadcast shared memory only.
#include "gs_kernels.cuh"
#include "project_bwd.cuh"

namespace gs {

// View of global tile gt: the number of views whose first tile is <= gt, minus one.  Every lane
// of the warp tests one view (n_views <= 32), so the lookup is one parallel load.
__device__ __forceinline__ int view_of_tile(const View* views, int n_views, int gt) {
    const int lane = threadIdx.x & 31;
    const bool le = lane < n_views && views[lane].tile_off <= gt;
    return __popc(__ballot_sync(0xffffffffu, le)) - 1;
}

// ----------------------------------------------------------------------------------------
// Loss normalisers: |M_v| and |M_v and D~ > 0| per view.
// ----------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) loss_count_kernel(const View* views, const float* tgt_depth,
                                                         const uint8_t* mask, uint32_t* counts) {
    const int v = blockIdx.y;
    const View& V = views[v];
    const int64_t P = (int64_t)V.W * V.H;
    uint32_t cm = 0, cd = 0;
    // four independent pixels per iteration, so that their loads are in flight together
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p0 < P; p0 += 4 * stride) {
        bool in[4];
        float d[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int64_t p = p0 + u * stride;
            const int64_t g = V.pix_off + p;
            in[u] = p < P && (mask ? mask[g] != 0 : true);
            d[u] = (p < P && tgt_depth) ? tgt_depth[g] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            cm += in[u];
            cd += (in[u] && d[u] > 0.f);
        }
    }
    // block sums first: the counters of a view take one atomic per block, not one per warp
    // (same-address atomics are applied one after another)
    __shared__ uint32_t s_c[2][8];
    cm = warp_sum(cm);
    cd = warp_sum(cd);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_c[0][w] = cm;
        s_c[1][w] = cd;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t tm = 0, td = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) {
            tm += s_c[0][k];
            td += s_c[1][k];
        }
        if (tm) atomicAdd(&counts[2 * v], tm);
        if (td) atomicAdd(&counts[2 * v + 1], td);
    }
}

cudaError_t launch_loss_count(const View* views, int n_views, const int64_t* pix_counts_host, const float* tgt_depth,
                              const uint8_t* mask, uint32_t* counts, cudaStream_t st) {
    int64_t mx = 0;
    for (int v = 0; v < n_views; v++) mx = pix_counts_host[v] > mx ? pix_counts_host[v] : mx;
    int bx = (int)((mx + 255) / 256);
    if (bx > 256) bx = 256;
    if (bx < 1) bx = 1;
    loss_count_kernel<<<dim3(bx, n_views), 256, 0, st>>>(views, tgt_depth, mask, counts);
    return cudaGetLastError();
}

__global__ void loss_finalize_kernel(const double* sums, const uint32_t* counts, int n_views, float lambda_rgb,
                                     float lambda_depth, float lambda_ssim, int has_depth, float* loss_out) {
    if (threadIdx.x == 0)
        loss_finalize_one(sums, counts, n_views, lambda_rgb, lambda_depth, lambda_ssim, has_depth, loss_out);
}

cudaError_t launch_loss_finalize(const double* sums, const uint32_t* counts, int n_views, float lambda_rgb,
                                 float lambda_depth, float lambda_ssim, int has_depth, float* loss_out, cudaStream_t st) {
    loss_finalize_kernel<<<1, 32, 0, st>>>(sums, counts, n_views, lambda_rgb, lambda_depth, lambda_ssim, has_depth,
                                           loss_out);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------------------
// Work decomposition shared by the forward and the backward compositing kernels.
//
// A CTA owns one (view, tile) item.  Each warp owns an 8 x (4 PPT) pixel sub-region of the
// tile and each lane PPT pixels of it, (x, y + 4q) for q < PPT with x = lane % 8,
// y = lane / 8.  The CTA stages CHUNK records of the tile's list in shared memory; every
// warp then walks the chunk and skips, warp-uniformly, every Gaussian whose
// alpha >= alpha_min box misses its sub-region (outside the box alpha < alpha_min, so
// nothing is lost).  The forward uses one pixel per thread (its per-fragment work is small,
// occupancy matters more); the backward two, which halves its warp reductions per pixel.
// ----------------------------------------------------------------------------------------
constexpr int kFwdPPT = 1;
constexpr int kBwdPPT = 2;
// Backward visits with at most this many contributing lanes skip the warp reduction: those
// lanes add their sums to the record directly.
constexpr int kBwdDirectLanes = 20;
static_assert(kFwdPPT == 1 && kBwdPPT == 2, "bwd_mask_from_fwd maps 8 x 4 forward regions to 8 x 8 ones");

template <int TILE, int PPT>
struct TileMap {
    static constexpr int NT = TILE * TILE / PPT;    // threads per CTA
    static constexpr int WX = TILE / 8;             // warp regions per tile row
    static constexpr int RH = 4 * PPT;              // warp region height
};

// Bit r of the result is set when warp region r of the tile whose top-left pixel is (X0, Y0)
// may hold a fragment of the record with alpha >= alpha_min.  Regions are first tested
// against the record's alpha box, then exactly: alpha = o 2^e >= alpha_min needs
// Q = -e <= thr = log2(o / alpha_min) with Q(d) = A dx^2 + 2 B dx dy + C dy^2 (positive
// definite), so a region is dropped when the least Q over the rectangle spanned by its pixel
// centres exceeds thr by more than a margin that covers the FP32 rounding of e in the
// compositing loops (well above 10 ulp of the largest term).  The least Q is 0 when the
// rectangle holds the mean; otherwise it lies on an edge that faces the mean (at the
// minimiser the gradient of Q points into the rectangle, so the mean is on the outer side of
// that edge's line): at most one vertical edge (x = x0 if x0 > 0, x = x1 if x1 < 0) and one
// horizontal edge, each minimised at its stationary point clamped to the edge.  The
// stationary points and the margin's terms depend on the column or the row only and are
// computed once per column and row.  Computed once per staged record; warps then test one
// bit per fragment.
template <int TILE, int PPT>
__device__ __forceinline__ uint32_t region_mask(float u, float v, float rx, float ry, float a, float b, float c,
                                                float o, float alpha_min, float X0, float Y0) {
    using TM = TileMap<TILE, PPT>;
    constexpr int NC = TM::WX, NR = TILE / TM::RH;
    uint32_t cols = 0, rows = 0;
#pragma unroll
    for (int cc = 0; cc < NC; cc++) {
        const float x0 = X0 + 8.f * cc;
        if (u - rx <= x0 + 7.5f && u + rx >= x0 + 0.5f) cols |= 1u << cc;
    }
#pragma unroll
    for (int r = 0; r < NR; r++) {
        const float y0 = Y0 + (float)(TM::RH * r);
        if (v - ry <= y0 + ((float)TM::RH - 0.5f) && v + ry >= y0 + 0.5f) rows |= 1u << r;
    }
    if (!(cols && rows)) return 0u;
    const float A = -a, B = -b, C = -c;   // e = -(A dx^2 + 2 B dx dy + C dy^2)
    const float iA = 1.f / A, iC = 1.f / C;
    const float thr = __log2f(o / alpha_min);
    const float B2 = 2.f * B, aB2 = 2.f * fabsf(B);
    // per column: its edges, the facing vertical edge X (if any) with A X and the stationary
    // dy of Q on x = X, and A Xm^2 for the margin (Xm the farther edge)
    float cx0[NC], cx1[NC], cX[NC], cAX[NC], cDy[NC], cXm[NC], cM[NC];
    bool cF[NC];
#pragma unroll
    for (int cc = 0; cc < NC; cc++) {
        const float x0 = X0 + 8.f * cc + 0.5f - u, x1 = x0 + 7.f;
        cx0[cc] = x0;
        cx1[cc] = x1;
        cF[cc] = x0 > 0.f || x1 < 0.f;
        const float X = x0 > 0.f ? x0 : x1;
        cX[cc] = X;
        cAX[cc] = A * X;
        cDy[cc] = -B * X * iC;
        const float Xm = fmaxf(fabsf(x0), fabsf(x1));
        cXm[cc] = Xm;
        cM[cc] = A * Xm * Xm;
    }
    uint32_t m = 0;
#pragma unroll
    for (int r = 0; r < NR; r++) {
        const float y0 = Y0 + (float)(TM::RH * r) + 0.5f - v, y1 = y0 + (float)(TM::RH - 1);
        const bool rF = y0 > 0.f || y1 < 0.f;
        const float Y = y0 > 0.f ? y0 : y1;
        const float CY = C * Y, dxs = -B * Y * iA;
        const float Ym = fmaxf(fabsf(y0), fabsf(y1));
        const float rM = C * Ym * Ym;
#pragma unroll
        for (int cc = 0; cc < NC; cc++) {
            float q = 0.f;   // the rectangle holds the mean
            if (cF[cc] || rF) {
                float qv = INFINITY, qh = INFINITY;
                if (cF[cc]) {
                    const float dy = fminf(fmaxf(cDy[cc], y0), y1);
                    qv = (cAX[cc] + B2 * dy) * cX[cc] + C * dy * dy;
                }
                if (rF) {
                    const float dx = fminf(fmaxf(dxs, cx0[cc]), cx1[cc]);
                    qh = (CY + B2 * dx) * Y + A * dx * dx;
                }
                q = fminf(qv, qh);
            }
            const float margin = 1e-5f * (cM[cc] + aB2 * cXm[cc] * Ym + rM) + 1e-3f;
            if (!(q > thr + margin)) m |= 1u << (r * NC + cc);
        }
    }
    // regions outside the alpha box hold no fragment with alpha >= alpha_min
    uint32_t box = 0;
#pragma unroll
    for (int r = 0; r < NR; r++)
        if (rows & (1u << r)) box |= cols << (r * NC);
    return m & box;
}

// Backward warp regions (8 x 8) from the forward ones (8 x 4): region (c, r) is the union of
// forward regions (c, 2r) and (c, 2r + 1).
template <int TILE>
__device__ __forceinline__ uint32_t bwd_mask_from_fwd(uint32_t m) {
    constexpr int WX = TILE / 8;
    uint32_t out = 0;
#pragma unroll
    for (int r = 0; r < TILE / 8; r++)
        out |= (((m >> (2 * r * WX)) | (m >> ((2 * r + 1) * WX))) & ((1u << WX) - 1u)) << (r * WX);
    return out;
}

__device__ __forceinline__ void load_record(const float4* proj, uint32_t gid, float2& uv, float4& co, float4& cz,
                                            float& rx, float& ry) {
    const float4* r = proj + 3 * (size_t)gid;
    const float4 f0 = __ldg(r), f1 = __ldg(r + 1), f2 = __ldg(r + 2);
    uv = make_float2(f0.x, f0.y);
    co = make_float4(f1.x, f1.y, f1.z, f0.w);
    cz = make_float4(f2.x, f2.y, f2.z, f0.z);
    rx = (float)__float_as_int(f1.w);
    ry = (float)__float_as_int(f2.w);
}

// ----------------------------------------------------------------------------------------
// Forward compositing.
// ----------------------------------------------------------------------------------------
// 40 resident warps per SM (at most 51 registers a thread): the compositing loop is latency
// bound and gains more from occupancy than from the few registers the staging code wants.
constexpr int kFwdThreadsPerSM = 1280;

// Shared memory of one forward tile: two chunk buffers of raw records (u, v, z, o),
// (a, b, c, rx), (r, g, b, ry) -- while the warps composite one, cp.async fills the other --,
// the chunk's region masks, per-warp record lists, loss partials and the pixels' targets.
template <int TILE, int CHUNK>
struct FwdSmem {
    static constexpr int NT = TileMap<TILE, kFwdPPT>::NT;
    static constexpr int NW = NT / 32;
    float4 rec[2][CHUNK][3];
    uint32_t mask[CHUNK];
    uint16_t list[NW][CHUNK];   // per warp: the chunk's records that reach its region
    double red[2][NW];
    float tgt[4][NT];           // target r, g, b, depth of each thread's pixel
};

// The forward of work item `item` (the item-th tile of the work order), by the CTA's NT threads.
// COUNT: fill the fragment and visit counters (a diagnostic option; off in the step).
template <int TILE, int CHUNK, bool COUNT>
__device__ __forceinline__ void render_fwd_tile(const FwdArgs& a, int item, FwdSmem<TILE, CHUNK>& S) {
    using TM = TileMap<TILE, kFwdPPT>;
    constexpr int NT = TM::NT;
    constexpr int NW = NT / 32;
    auto& s_rec = S.rec;
    auto& s_mask = S.mask;
    auto& s_list = S.list;
    auto& s_red = S.red;
    auto& s_tgt = S.tgt;
    // (loads ordered so that the dependent chain order -> ranges / view -> ids -> records is
    // as short as possible: CTAs are short and this latency is paid once per tile)
    const uint32_t status = a.counters->status;
    const int gt = a.order ? (int)a.order[item] : item;
    if (status != 0) return;
    const uint2 rg = a.ranges[gt];
    const int v = view_of_tile(a.views, a.n_views, gt);
    const int n = (int)(rg.y - rg.x);
    const View& V = a.views[v];
    const int lt = gt - V.tile_off;
    const int tx = lt % V.tiles_x, ty = lt / V.tiles_x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t ltm;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(ltm));
    // one pixel per thread
    const int x = tx * TILE + (w % TM::WX) * 8 + (lane & 7), y = ty * TILE + (w / TM::WX) * TM::RH + (lane >> 3);
    const float pxc = (float)x + 0.5f, pyc = (float)y + 0.5f;
    const bool inside = x < V.W && y < V.H;
    bool done = !inside;
    float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, dep = 0.f;
    uint32_t last = 0;
    // this pixel's targets, copied to shared memory now (cp.async, no registers held) so that
    // the loss epilogue does not wait for them
    if (inside && a.tgt_rgb) {
        const int64_t P = (int64_t)V.W * V.H, p = (int64_t)y * V.W + x;
        const float* t = a.tgt_rgb + 3 * V.pix_off;
        cp_async4(&s_tgt[0][threadIdx.x], t + p);
        cp_async4(&s_tgt[1][threadIdx.x], t + P + p);
        cp_async4(&s_tgt[2][threadIdx.x], t + 2 * P + p);
        if (a.tgt_depth) cp_async4(&s_tgt[3][threadIdx.x], a.tgt_depth + V.pix_off + p);
    }
    cp_async_commit();
    const float amin = a.op.alpha_min, amax = a.op.alpha_max, tmin = a.op.T_min;
    uint32_t n_eval = 0, n_add = 0, n_visit = 0;
    int b = 0;   // buffer holding the chunk being composited
    // composite one fragment with opacity alpha of chunk record k (front to back), branch-free:
    // a fragment that is skipped (alpha < alpha_min), stops the pixel (T (1 - alpha) < T_min)
    // or comes after the stop adds exact zeros
    auto add = [&](float alpha, int k, int base) {
        const bool act = !done;
        const bool pass = act && !(alpha < amin);
        const float test_T = T * (1.f - alpha);
        const bool stop = pass && test_T < tmin;
        const bool c = pass && !stop;
        if constexpr (COUNT) {
            n_eval += act;
            n_add += c;
        }
        done = done || stop;
        const float wgt = c ? alpha * T : 0.f;
        const float4 r2 = s_rec[b][k][2];
        c0 = fmaf(wgt, r2.x, c0);
        c1 = fmaf(wgt, r2.y, c1);
        c2 = fmaf(wgt, r2.z, c2);
        dep = fmaf(wgt, s_rec[b][k][0].z, dep);
        T = c ? test_T : T;
        last = c ? (uint32_t)(base + k + 1) : last;
    };
    auto alpha_of = [&](int k) {
        const float4 r0 = s_rec[b][k][0], r1 = s_rec[b][k][1];
        const float G = ex2_approx(frag_exponent(pxc - r0.x, pyc - r0.y, r1.x, r1.y, r1.z).e);
        return fminf(amax, r0.w * G);
    };
    // Pipeline over chunks c = [c CHUNK, (c + 1) CHUNK): the pair ids of chunk c + 2 are loaded
    // into registers and the records of chunk c + 1 copied asynchronously while chunk c is
    // composited.
    const int nchunks = (n + CHUNK - 1) / CHUNK;
    constexpr int R = (CHUNK + NT - 1) / NT;   // staged records per thread
    uint32_t pid[R];
    auto fetch_ids = [&](int c) {
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int j = c * CHUNK + (int)threadIdx.x + r * NT;
            if (c < nchunks && (int)threadIdx.x + r * NT < CHUNK && j < n) pid[r] = a.vals[rg.x + j];
        }
    };
    auto stage = [&](int c, int bb) {
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int k = (int)threadIdx.x + r * NT;
            const int j = c * CHUNK + k;
            if (c < nchunks && k < CHUNK && j < n) {
                const float4* src = a.proj + 3 * (size_t)pid[r];
#pragma unroll
                for (int h = 0; h < 3; h++) cp_async16(&s_rec[bb][k][h], src + h);
            }
        }
        cp_async_commit();
    };
    fetch_ids(0);
    stage(0, 0);
    fetch_ids(1);
    for (int c = 0; c < nchunks; c++) {
        b = c & 1;
        const int base = c * CHUNK;
        if (__syncthreads_count(!done) == 0) break;   // (also: every warp is done with buffer b ^ 1)
        stage(c + 1, b ^ 1);
        fetch_ids(c + 2);
        cp_async_wait_prior();   // this thread's copies of chunk c have landed (c + 1 may be in flight)
        const int m = min(CHUNK, n - base);
        // warp-region masks of the chunk's records, kept per pair for the backward.  Thread t
        // takes the records it copied itself (stage gives record k to thread k mod NT), which
        // its own wait has made visible to it: no barrier before this loop.
        for (int k = threadIdx.x; k < m; k += NT) {
            const float4 r0 = s_rec[b][k][0], r1 = s_rec[b][k][1];
            const float rxf = (float)__float_as_int(r1.w), ryf = (float)__float_as_int(s_rec[b][k][2].w);
            const uint32_t msk = region_mask<TILE, kFwdPPT>(r0.x, r0.y, rxf, ryf, r1.x, r1.y, r1.z, r0.w, amin,
                                                           (float)(tx * TILE), (float)(ty * TILE));
            s_mask[k] = msk;
            a.pair_mask[rg.x + base + k] = (uint8_t)msk;
        }
        __syncthreads();
        if (__any_sync(0xffffffffu, !done)) {
            // compact the records whose alpha >= alpha_min region reaches this warp's pixels
            int cnt = 0;
            for (int k0 = 0; k0 < m; k0 += 32) {
                const int k = k0 + lane;
                const bool hit = k < m && ((s_mask[k] >> w) & 1u);
                const uint32_t bal = __ballot_sync(0xffffffffu, hit);
                if (hit) s_list[w][cnt + __popc(bal & ltm)] = (uint16_t)k;
                cnt += __popc(bal);
            }
            __syncwarp();
            if constexpr (COUNT) n_visit += cnt;
            // eight, four, then two records per iteration: their alphas are independent, the
            // compositing is not (four per iteration: 0.936 -> 0.908 ms at 2M Gaussians, 8 views;
            // eight: 0.882)
            int t = 0;
            for (; t + 7 < cnt; t += 8) {
                if (__all_sync(0xffffffffu, done)) break;
                int kk[8];
                float al[8];
#pragma unroll
                for (int u = 0; u < 8; u++) kk[u] = s_list[w][t + u];
#pragma unroll
                for (int u = 0; u < 8; u++) al[u] = alpha_of(kk[u]);
#pragma unroll
                for (int u = 0; u < 8; u++) add(al[u], kk[u], base);
            }
            for (; t + 3 < cnt; t += 4) {
                if (__all_sync(0xffffffffu, done)) break;
                const int ka = s_list[w][t], kb = s_list[w][t + 1], kc = s_list[w][t + 2], kd = s_list[w][t + 3];
                const float alpha_a = alpha_of(ka), alpha_b = alpha_of(kb);
                const float alpha_c = alpha_of(kc), alpha_d = alpha_of(kd);
                add(alpha_a, ka, base);
                add(alpha_b, kb, base);
                add(alpha_c, kc, base);
                add(alpha_d, kd, base);
            }
            for (; t + 1 < cnt; t += 2) {
                if (__all_sync(0xffffffffu, done)) break;
                const int ka = s_list[w][t], kb = s_list[w][t + 1];
                const float alpha_a = alpha_of(ka), alpha_b = alpha_of(kb);
                add(alpha_a, ka, base);
                add(alpha_b, kb, base);
            }
            if (t < cnt) {
                const int k = s_list[w][t];
                add(alpha_of(k), k, base);
            }
        }
    }
    cp_async_wait_all();
    if constexpr (COUNT) {
        warp_count_add(&a.counters->frag_fwd_eval, n_eval);
        warp_count_add(&a.counters->frag_fwd_add, n_add);
        if (lane == 0 && n_visit) atomicAdd(&a.counters->visits_fwd, n_visit);
    }
    // L1 sums: FP32 within a warp (32 pixels), FP64 across warps and CTAs (the FP64 pipe is
    // narrow: it only sees the per-warp totals)
    float lr = 0.f, ld = 0.f;
    if (inside) {
        const int64_t P = (int64_t)V.W * V.H;
        const int64_t p = (int64_t)y * V.W + x;
        const int64_t g = V.pix_off + p;
        const float o0 = c0 + T * a.op.bg0, o1 = c1 + T * a.op.bg1, o2 = c2 + T * a.op.bg2;
        float* rgb = a.out_rgb + 3 * V.pix_off;
        rgb[p] = o0;
        rgb[P + p] = o1;
        rgb[2 * P + p] = o2;
        a.out_depth[g] = dep;
        if (a.out_T) a.out_T[g] = T;
        a.T_final[g] = T;
        a.n_contrib[g] = last;
        if (a.tgt_rgb) {
            const bool in = a.mask ? a.mask[g] != 0 : true;
            const float tr = s_tgt[0][threadIdx.x], tgr = s_tgt[1][threadIdx.x], tbl = s_tgt[2][threadIdx.x];
            const float cm = (float)a.loss_counts[2 * v], cd = (float)a.loss_counts[2 * v + 1];
            const float inv_v = 1.0f / (float)a.n_views;
            const float krgb = (in && cm > 0.f) ? a.op.lambda_rgb * inv_v / cm : 0.f;
            const float r0 = o0 - tr, r1 = o1 - tgr, r2 = o2 - tbl;
            float* dl = a.dl_drgb + 3 * V.pix_off;
            dl[p] = krgb * (float)((r0 > 0.f) - (r0 < 0.f));
            dl[P + p] = krgb * (float)((r1 > 0.f) - (r1 < 0.f));
            dl[2 * P + p] = krgb * (float)((r2 > 0.f) - (r2 < 0.f));
            if (in) lr += fabsf(r0) + fabsf(r1) + fabsf(r2);
            if (a.dl_ddepth) {
                const float td = a.tgt_depth ? s_tgt[3][threadIdx.x] : 0.f;
                const bool ind = in && td > 0.f;
                const float kd = (ind && cd > 0.f) ? a.op.lambda_depth * inv_v / cd : 0.f;
                const float rd = dep - td;
                a.dl_ddepth[g] = kd * (float)((rd > 0.f) - (rd < 0.f));
                if (ind) ld += fabsf(rd);
            }
        }
    }
    if (a.tgt_rgb) {
        // block reduction of the two L1 sums, one atomic per CTA
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lr += __shfl_xor_sync(0xffffffffu, lr, o);
            ld += __shfl_xor_sync(0xffffffffu, ld, o);
        }
        if (lane == 0) { s_red[0][w] = (double)lr; s_red[1][w] = (double)ld; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double sr = 0, sd = 0;
            for (int k = 0; k < NW; k++) { sr += s_red[0][k]; sd += s_red[1][k]; }
            if (sr != 0.0) atomicAdd(&a.loss_sums[3 * v], sr);
            if (sd != 0.0) atomicAdd(&a.loss_sums[3 * v + 1], sd);
        }
    }
}

template <int TILE, int CHUNK, bool COUNT>
__global__ void __launch_bounds__(TileMap<TILE, kFwdPPT>::NT, kFwdThreadsPerSM / TileMap<TILE, kFwdPPT>::NT)
    render_fwd_kernel(FwdArgs a) {
    __shared__ FwdSmem<TILE, CHUNK> S;
    render_fwd_tile<TILE, CHUNK, COUNT>(a, blockIdx.x, S);
}

// ----------------------------------------------------------------------------------------
// Backward compositing.
//
// For a pixel with upstream gradients g_C (3) and g_D, walking its contributing fragments
// back to front with T_i = T_{i+1} / (1 - alpha_i):
//   w_i = alpha_i T_i;  dL/dc_i = g_C w_i;  dL/dz_i = g_D w_i
//   dL/dalpha_i = T_i (g_C.c_i + g_D z_i) - S_i / (1 - alpha_i)
// with S_i = g_C.bg T_final + sum_{j>i} (g_C.c_j + g_D z_j) w_j (one running scalar).
// If o G < alpha_max (the clamp is inactive), alpha = o 2^e gives dalpha/do = G and
// dalpha/de = ln2 o G.  Per (view, Gaussian) the kernel accumulates, with h = dL/dalpha o G:
//   r0 = (sum h h_x, sum h h_y, sum h dx^2, sum h dx dy)
//   r1 = (sum h dy^2, sum dL/dalpha G, sum g_D w, 0), r2 = (sum g_C w, 0)
// (h_x, h_y from frag_exponent) and the projection backward applies the constant factors.
// A lane first sums its two pixels; the warp's 10 sums are then reduced (warp_reduce10) and
// written by 10 lanes with one atomic each -- or, when at most kBwdDirectLanes lanes
// contribute, added by those lanes directly with vector atomics.
// ----------------------------------------------------------------------------------------
// Warp sums of 10 per-lane values by transpose reductions: values 0..7 halve their count at
// each of the lane-xor 16, 8, 4 exchanges and finish with two butterflies (lane l ends with
// the total of value (l >> 2) & 7); values 8..9 take one exchange and four butterflies (lane
// l ends with value 8 + (l >> 4)).  44 shuffle / select / add instructions instead of 62 for
// a 16-padded transpose.
__device__ __forceinline__ void warp_reduce10(float (&v)[10], float& out8, float& out2) {
    const int lane = threadIdx.x & 31;
    {
        const bool hi = lane & 16;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float mine = hi ? v[4 + k] : v[k];
            const float other = hi ? v[k] : v[4 + k];
            v[k] = mine + __shfl_xor_sync(0xffffffffu, other, 16);
        }
    }
    {
        const bool hi = lane & 8;
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const float mine = hi ? v[2 + k] : v[k];
            const float other = hi ? v[k] : v[2 + k];
            v[k] = mine + __shfl_xor_sync(0xffffffffu, other, 8);
        }
    }
    {
        const bool hi = lane & 4;
        const float mine = hi ? v[1] : v[0];
        const float other = hi ? v[0] : v[1];
        v[0] = mine + __shfl_xor_sync(0xffffffffu, other, 4);
    }
    float a = v[0];
    a += __shfl_xor_sync(0xffffffffu, a, 2);
    a += __shfl_xor_sync(0xffffffffu, a, 1);
    out8 = a;
    const bool hi = lane & 16;
    const float mine = hi ? v[9] : v[8];
    const float other = hi ? v[8] : v[9];
    float b = mine + __shfl_xor_sync(0xffffffffu, other, 16);
    b += __shfl_xor_sync(0xffffffffu, b, 8);
    b += __shfl_xor_sync(0xffffffffu, b, 4);
    b += __shfl_xor_sync(0xffffffffu, b, 2);
    b += __shfl_xor_sync(0xffffffffu, b, 1);
    out2 = b;
}

template <int TILE, int CHUNK, bool COUNT>
__global__ void __launch_bounds__(TileMap<TILE, kBwdPPT>::NT) render_bwd_kernel(BwdArgs a) {
    constexpr int kPPT = kBwdPPT;
    using TM = TileMap<TILE, kPPT>;
    constexpr int NT = TM::NT;
    // two chunk buffers: while the warps walk one, cp.async fills the other
    __shared__ float4 s_rec[2][CHUNK][3];   // raw projected records (u, v, z, o), (a, b, c, rx), (r, g, b, ry)
    __shared__ uint32_t s_id[2][CHUNK];
    __shared__ uint32_t s_mask[2][CHUNK];
    __shared__ uint16_t s_list[NT / 32][CHUNK];   // per warp: the chunk's records that reach its region
    __shared__ uint32_t s_max;
    const uint32_t status = a.counters->status;
    const int gt = a.order ? (int)a.order[blockIdx.x] : (int)blockIdx.x;
    if (status != 0) return;
    const uint2 rg = a.ranges[gt];
    const int v = view_of_tile(a.views, a.n_views, gt);
    const View& V = a.views[v];
    const int lt = gt - V.tile_off;
    const int tx = lt % V.tiles_x, ty = lt / V.tiles_x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int rx0 = tx * TILE + (w % TM::WX) * 8, ry0 = ty * TILE + (w / TM::WX) * TM::RH;
    const float amin = a.op.alpha_min, amax = a.op.alpha_max;
    uint32_t n_eval = 0, n_add = 0, n_visit = 0;
    float px[kPPT], py[kPPT], T[kPPT], S[kPPT], gc0[kPPT], gc1[kPPT], gc2[kPPT], gd[kPPT];
    uint32_t last[kPPT];
    uint32_t mylast = 0;
#pragma unroll
    for (int q = 0; q < kPPT; q++) {
        const int xi = rx0 + (lane & 7), yi = ry0 + (lane >> 3) + 4 * q;
        px[q] = (float)xi + 0.5f;
        py[q] = (float)yi + 0.5f;
        T[q] = 0.f; gc0[q] = gc1[q] = gc2[q] = gd[q] = 0.f;
        last[q] = 0;
        if (xi < V.W && yi < V.H) {
            const int64_t P = (int64_t)V.W * V.H;
            const int64_t p = (int64_t)yi * V.W + xi;
            const int64_t g = V.pix_off + p;
            T[q] = a.T_final[g];
            last[q] = a.n_contrib[g];
            const float* d = a.dl_drgb + 3 * V.pix_off;
            gc0[q] = d[p];
            gc1[q] = d[P + p];
            gc2[q] = d[2 * P + p];
            gd[q] = a.dl_ddepth ? a.dl_ddepth[g] : 0.f;
            if (gc0[q] == 0.f && gc1[q] == 0.f && gc2[q] == 0.f && gd[q] == 0.f) last[q] = 0;
        }
        S[q] = (gc0[q] * a.op.bg0 + gc1[q] * a.op.bg1 + gc2[q] * a.op.bg2) * T[q];
        mylast = max(mylast, last[q]);
    }
    const uint32_t wtop = __reduce_max_sync(0xffffffffu, mylast);
    int top_all;
    if constexpr (NT == 32) {
        top_all = (int)wtop;   // one warp: no block reduction
    } else {
        if (threadIdx.x == 0) s_max = 0;
        __syncthreads();
        if (lane == 0 && wtop) atomicMax(&s_max, wtop);
        __syncthreads();
        top_all = (int)s_max;
    }
    // Chunk c covers list positions [max(0, top_all - (c + 1) CHUNK), top_all - c CHUNK).
    // Pipeline: the ids and masks of chunk c + 2 are loaded into registers and the records of
    // chunk c + 1 are copied asynchronously while chunk c is composited.
    const int nchunks = (top_all + CHUNK - 1) / CHUNK;
    constexpr int R = (CHUNK + NT - 1) / NT;   // staged records per thread
    uint32_t pid[R];
    uint32_t pmsk[R];
    auto fetch_ids = [&](int c) {
        const int top = top_all - c * CHUNK, lo = max(0, top - CHUNK);
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int k = (int)threadIdx.x + r * NT;
            if (c < nchunks && k < top - lo) {
                pid[r] = a.vals[rg.x + lo + k];
                pmsk[r] = a.pair_mask[rg.x + lo + k];
            }
        }
    };
    auto stage = [&](int c, int b) {
        const int top = top_all - c * CHUNK, lo = max(0, top - CHUNK);
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int k = (int)threadIdx.x + r * NT;
            if (c < nchunks && k < top - lo) {
                s_id[b][k] = pid[r];
                s_mask[b][k] = bwd_mask_from_fwd<TILE>(pmsk[r]);
                const float4* src = a.proj + 3 * (size_t)pid[r];
#pragma unroll
                for (int h = 0; h < 3; h++) cp_async16(&s_rec[b][k][h], src + h);
            }
        }
        cp_async_commit();
    };
    fetch_ids(0);
    stage(0, 0);
    fetch_ids(1);
    for (int c = 0; c < nchunks; c++) {
        const int b = c & 1;
        const int top = top_all - c * CHUNK, lo = max(0, top - CHUNK);
        stage(c + 1, b ^ 1);
        fetch_ids(c + 2);
        cp_async_wait_prior();   // chunk c has landed (chunk c + 1 may still be in flight)
        __syncthreads();
        uint32_t ltm;
        asm("mov.u32 %0, %%lanemask_lt;" : "=r"(ltm));
        // this warp's records of the chunk, back to front: positions below its pixels' last
        // added fragment whose alpha >= alpha_min region reaches the warp's pixels
        const int kstart = min(top, (int)wtop) - 1 - lo;
        int cnt = 0;
        for (int k0 = kstart; k0 >= 0; k0 -= 32) {
            const int kk = k0 - lane;
            const bool hit = kk >= 0 && ((s_mask[b][kk] >> w) & 1u);
            const uint32_t bal = __ballot_sync(0xffffffffu, hit);
            if (hit) s_list[w][cnt + __popc(bal & ltm)] = (uint16_t)kk;
            cnt += __popc(bal);
        }
        __syncwarp();
        if constexpr (COUNT) n_visit += cnt;
        for (int t = 0; t < cnt; t++) {
            const int k = s_list[w][t];
            const int j = lo + k;
            const float4 r0 = s_rec[b][k][0], r1 = s_rec[b][k][1];
            const float2 bx = make_float2(r0.x, r0.y);
            const float4 co = make_float4(r1.x, r1.y, r1.z, r0.w);
            float val[10];
#pragma unroll
            for (int q = 0; q < 10; q++) val[q] = 0.f;
            bool contrib = false;
            const float4 r2 = s_rec[b][k][2];
            const float4 cz = make_float4(r2.x, r2.y, r2.z, r0.z);
            // Branch-free per pixel: every lane computes the fragment and commits it with
            // selects (adding exact zeros where it does not contribute), so the warp runs one
            // straight path instead of re-converging around per-pixel branches.
#pragma unroll
            for (int q = 0; q < kPPT; q++) {
                const bool live = (uint32_t)j < last[q];
                const float dx = px[q] - bx.x, dy = py[q] - bx.y;
                const FragE fe = frag_exponent(dx, dy, co.x, co.y, co.z);
                const float G = ex2_approx(fe.e);
                const float a0 = co.w * G;
                const float alpha = fminf(amax, a0);
                const bool c = live && !(alpha < amin);
                if constexpr (COUNT) {
                    n_eval += live;
                    n_add += c;
                }
                contrib |= c;
                const float rom = rcp_approx(1.f - alpha);
                const float Tn = T[q] * rom;
                const float wgt = alpha * Tn;
                const float gcz = gc0[q] * cz.x + gc1[q] * cz.y + gc2[q] * cz.z + gd[q] * cz.w;
                const float dLda = Tn * gcz - S[q] * rom;
                S[q] = c ? fmaf(gcz, wgt, S[q]) : S[q];
                T[q] = c ? Tn : T[q];
                const float wc = c ? wgt : 0.f;
                val[7] = fmaf(gc0[q], wc, val[7]);
                val[8] = fmaf(gc1[q], wc, val[8]);
                val[9] = fmaf(gc2[q], wc, val[9]);
                val[6] = fmaf(gd[q], wc, val[6]);
                const float gl = (c && a0 < amax) ? dLda : 0.f;   // the 0.99 clamp stops the gradient
                const float h = gl * a0;
                const float hdx = h * dx;
                val[0] = fmaf(h, fe.hx, val[0]);
                val[1] = fmaf(h, fe.hy, val[1]);
                val[2] = fmaf(hdx, dx, val[2]);
                val[3] = fmaf(hdx, dy, val[3]);
                val[4] = fmaf(h * dy, dy, val[4]);
                val[5] = fmaf(gl, G, val[5]);
            }
            const uint32_t cmask = __ballot_sync(0xffffffffu, contrib);
            if (cmask) {
                float4* rec4 = a.grad2d + 3 * (size_t)s_id[b][k];
                if (__popc(cmask) <= kBwdDirectLanes) {
                    // few contributing lanes: each adds its own sums with three vector atomics
                    // (slots 7 and 11 of the record are padding and receive zeros)
                    if (contrib) {
                        atomicAdd(rec4, make_float4(val[0], val[1], val[2], val[3]));
                        atomicAdd(rec4 + 1, make_float4(val[4], val[5], val[6], 0.f));
                        atomicAdd(rec4 + 2, make_float4(val[7], val[8], val[9], 0.f));
                    }
                } else {
                    float t8, t2;
                    warp_reduce10(val, t8, t2);
                    float* rec = reinterpret_cast<float*>(rec4);
                    // value index -> record slot: 0..6 -> 0..6, 7..9 -> 8..10
                    if ((lane & 3) == 0) {
                        const int idx = lane >> 2;
                        atomicAdd(rec + (idx < 7 ? idx : idx + 1), t8);
                    }
                    if ((lane & 15) == 0) atomicAdd(rec + 9 + (lane >> 4), t2);
                }
            }
        }
        __syncthreads();   // buffer b is refilled with chunk c + 2 in the next iteration
    }
    cp_async_wait_all();
    if constexpr (COUNT) {
        warp_count_add(&a.counters->frag_bwd_eval, n_eval);
        warp_count_add(&a.counters->frag_bwd_add, n_add);
        if (lane == 0 && n_visit) atomicAdd(&a.counters->visits_bwd, n_visit);
    }
}

// ----------------------------------------------------------------------------------------
// Backward compositing, one independent warp per (16 x 16 tile, 8 x 8 region).  The warp walks
// the tile's list back to front 32 positions at a time: each lane tests the stored region mask
// of one position, the hits are compacted in order (a ballot) and only their records are
// copied (cp.async) into the warp's own double buffer while the previous window's records are
// composited.  No block barrier: every warp proceeds at its own pace.  The per-record
// arithmetic is that of render_bwd_kernel.
// ----------------------------------------------------------------------------------------
constexpr int kWin = 32;   // list positions per window

// A warp's shared memory: its two windows of staged records, their ids and list positions.
struct BwdWarpSmem {
    float4 rec[2][kWin][3];
    uint32_t id[2][kWin];
    int pos[2][kWin];
};

// The backward of work item `item` = 4 t + w: region w of the t-th tile of the work order, by
// one warp with its own shared memory S.
template <bool COUNT>
__device__ __forceinline__ void render_bwd_region(const BwdArgs& a, int item, BwdWarpSmem& W) {
    constexpr int TILE = 16, kPPT = kBwdPPT;
    auto& s_rec = W.rec;
    auto& s_id = W.id;
    auto& s_pos = W.pos;
    const uint32_t status = a.counters->status;
    const int gt = a.order ? (int)a.order[item >> 2] : (item >> 2);
    const int w = item & 3;   // region: column w % 2, row w / 2 (the forward's mask order)
    if (status != 0) return;
    const uint2 rg = a.ranges[gt];
    const int v = view_of_tile(a.views, a.n_views, gt);
    const View& V = a.views[v];
    const int lt = gt - V.tile_off;
    const int tx = lt % V.tiles_x, ty = lt / V.tiles_x;
    const int lane = threadIdx.x & 31;
    const int rx0 = tx * TILE + (w & 1) * 8, ry0 = ty * TILE + (w >> 1) * 8;
    const float amin = a.op.alpha_min, amax = a.op.alpha_max;
    uint32_t n_eval = 0, n_add = 0, n_visit = 0;
    float px[kPPT], py[kPPT], T[kPPT], S[kPPT], gc0[kPPT], gc1[kPPT], gc2[kPPT], gd[kPPT];
    uint32_t last[kPPT];
    uint32_t mylast = 0;
#pragma unroll
    for (int q = 0; q < kPPT; q++) {
        const int xi = rx0 + (lane & 7), yi = ry0 + (lane >> 3) + 4 * q;
        px[q] = (float)xi + 0.5f;
        py[q] = (float)yi + 0.5f;
        T[q] = 0.f; gc0[q] = gc1[q] = gc2[q] = gd[q] = 0.f;
        last[q] = 0;
        if (xi < V.W && yi < V.H) {
            const int64_t P = (int64_t)V.W * V.H;
            const int64_t p = (int64_t)yi * V.W + xi;
            const int64_t g = V.pix_off + p;
            T[q] = a.T_final[g];
            last[q] = a.n_contrib[g];
            const float* d = a.dl_drgb + 3 * V.pix_off;
            gc0[q] = d[p];
            gc1[q] = d[P + p];
            gc2[q] = d[2 * P + p];
            gd[q] = a.dl_ddepth ? a.dl_ddepth[g] : 0.f;
            if (gc0[q] == 0.f && gc1[q] == 0.f && gc2[q] == 0.f && gd[q] == 0.f) last[q] = 0;
        }
        S[q] = (gc0[q] * a.op.bg0 + gc1[q] * a.op.bg1 + gc2[q] * a.op.bg2) * T[q];
        mylast = max(mylast, last[q]);
    }
    const int wtop = (int)__reduce_max_sync(0xffffffffu, mylast);
    // the lane's two pixels (rows y and y + 4 of the region) as packed pairs
    const float2 px2 = make_float2(px[0], px[1]), py2 = make_float2(py[0], py[1]);
    const float2 g0 = make_float2(gc0[0], gc0[1]), g1 = make_float2(gc1[0], gc1[1]);
    const float2 g2 = make_float2(gc2[0], gc2[1]), gd2 = make_float2(gd[0], gd[1]);
    float2 T2 = make_float2(T[0], T[1]), S2 = make_float2(S[0], S[1]);
    uint32_t ltm;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(ltm));
    // window starting (from the back) at position k0: this warp's hits, copied into buffer b
    auto gather = [&](int k0, int b) -> int {
        const int k = k0 - lane;
        bool hit = false;
        if (k >= 0) hit = (bwd_mask_from_fwd<TILE>(a.pair_mask[rg.x + k]) >> w) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, hit);
        if (hit) {
            const int slot = __popc(bal & ltm);
            const uint32_t id = a.vals[rg.x + k];
            s_id[b][slot] = id;
            s_pos[b][slot] = k;
            const float4* src = a.proj + 3 * (size_t)id;
#pragma unroll
            for (int h = 0; h < 3; h++) cp_async16(&s_rec[b][slot][h], src + h);
        }
        cp_async_commit();
        return __popc(bal);
    };
    // windows start at wtop - 1, wtop - 1 - kWin, ... (while >= 0); one commit group each
    int next = wtop - 1;
    bool have = next >= 0;
    int cnt = have ? gather(next, 0) : 0;
    next -= kWin;
    for (int b = 0; have; b ^= 1) {
        // the next window into the other buffer (or an empty group), then this window's records
        const bool have_next = next >= 0;
        int cnt_next = 0;
        if (have_next) cnt_next = gather(next, b ^ 1);
        else cp_async_commit();
        next -= kWin;
        cp_async_wait_prior();   // this window's copies (all lanes') have landed after the syncwarp
        __syncwarp();
        // each record's depth into its colour word's last slot (r_y is not needed here), so that
        // the adjoint reads colour and depth with one 16-byte load
        if (lane < cnt) s_rec[b][lane][2].w = s_rec[b][lane][0].z;
        __syncwarp();
        if constexpr (COUNT) n_visit += cnt;
        // the alphas of the lane's two pixels of record t, as one packed pair: a record that no
        // pixel of the warp adds (all below alpha_min or past their pixels' last fragment)
        // changes nothing and is skipped whole
        struct Alphas {
            float2 dx, dy, hx, hy, G, a0, al;
            bool c0, c1;
        };
        auto alphas = [&](int t, Alphas& P) {
            const uint32_t j = (uint32_t)s_pos[b][t];
            const float4 r0 = s_rec[b][t][0], r1 = s_rec[b][t][1];
            P.dx = __fadd2_rn(px2, dup2(-r0.x));
            P.dy = __fadd2_rn(py2, dup2(-r0.y));
            const FragE2 fe = frag_exponent2(P.dx, P.dy, dup2(r1.x), dup2(r1.y), dup2(r1.z));
            P.hx = fe.hx;
            P.hy = fe.hy;
            P.G = make_float2(ex2_approx(fe.e.x), ex2_approx(fe.e.y));
            P.a0 = __fmul2_rn(dup2(r0.w), P.G);
            P.al = make_float2(fminf(amax, P.a0.x), fminf(amax, P.a0.y));
            P.c0 = j < last[0] && !(P.al.x < amin);
            P.c1 = j < last[1] && !(P.al.y < amin);
            if constexpr (COUNT) {
                n_eval += (j < last[0]) + (j < last[1]);
                n_add += P.c0 + P.c1;
            }
        };
        // back to front, each pixel of the lane in turn: T in front of the fragment from the one
        // behind it, weight, the colour / depth adjoint and dL/dalpha; pixels that do not add it
        // keep T and S (scalar arithmetic: packing these pairs measured slower)
        auto adjoint = [&](int t, const Alphas& P) {
            const bool contrib = P.c0 || P.c1;
            const float dxs[2] = {P.dx.x, P.dx.y}, dys[2] = {P.dy.x, P.dy.y}, hxs[2] = {P.hx.x, P.hx.y},
                        hys[2] = {P.hy.x, P.hy.y};
            const float Gs[2] = {P.G.x, P.G.y}, a0s[2] = {P.a0.x, P.a0.y}, als[2] = {P.al.x, P.al.y};
            const float4 r2 = s_rec[b][t][2];
            const float4 cz = r2;   // colour and depth
            float val[10];
#pragma unroll
            for (int q = 0; q < 10; q++) val[q] = 0.f;
            const float Ts[2] = {T2.x, T2.y}, Ss[2] = {S2.x, S2.y};
            const float g0s[2] = {g0.x, g0.y}, g1s[2] = {g1.x, g1.y}, g2s[2] = {g2.x, g2.y}, gds[2] = {gd2.x, gd2.y};
            float Tn_[2], Sn_[2];
            const bool cq[2] = {P.c0, P.c1};
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const float dxv = dxs[q], dyv = dys[q], Gv = Gs[q], a0v = a0s[q], alpha = als[q];
                const bool c = cq[q];
                const float rom = rcp_approx(1.f - alpha);
                const float Tn = Ts[q] * rom;
                const float wgt = alpha * Tn;
                const float gcz = g0s[q] * cz.x + g1s[q] * cz.y + g2s[q] * cz.z + gds[q] * cz.w;
                const float dLda = Tn * gcz - Ss[q] * rom;
                Sn_[q] = c ? fmaf(gcz, wgt, Ss[q]) : Ss[q];
                Tn_[q] = c ? Tn : Ts[q];
                const float wc = c ? wgt : 0.f;
                val[7] = fmaf(g0s[q], wc, val[7]);
                val[8] = fmaf(g1s[q], wc, val[8]);
                val[9] = fmaf(g2s[q], wc, val[9]);
                val[6] = fmaf(gds[q], wc, val[6]);
                const float gl = (c && a0v < amax) ? dLda : 0.f;   // the 0.99 clamp stops the gradient
                const float h = gl * a0v;
                const float hdx = h * dxv;
                val[0] = fmaf(h, hxs[q], val[0]);
                val[1] = fmaf(h, hys[q], val[1]);
                val[2] = fmaf(hdx, dxv, val[2]);
                val[3] = fmaf(hdx, dyv, val[3]);
                val[4] = fmaf(h * dyv, dyv, val[4]);
                val[5] = fmaf(gl, Gv, val[5]);
            }
            S2 = make_float2(Sn_[0], Sn_[1]);
            T2 = make_float2(Tn_[0], Tn_[1]);
            const uint32_t cmask = __ballot_sync(0xffffffffu, contrib);
            float4* rec4 = a.grad2d + 3 * (size_t)s_id[b][t];
            if (__popc(cmask) <= kBwdDirectLanes) {
                if (contrib) {
                    atomicAdd(rec4, make_float4(val[0], val[1], val[2], val[3]));
                    atomicAdd(rec4 + 1, make_float4(val[4], val[5], val[6], 0.f));
                    atomicAdd(rec4 + 2, make_float4(val[7], val[8], val[9], 0.f));
                }
            } else {
                float t8, t2;
                warp_reduce10(val, t8, t2);
                float* rec = reinterpret_cast<float*>(rec4);
                if ((lane & 3) == 0) {
                    const int idx = lane >> 2;
                    atomicAdd(rec + (idx < 7 ? idx : idx + 1), t8);
                }
                if ((lane & 15) == 0) atomicAdd(rec + 9 + (lane >> 4), t2);
            }
        };
        // two records per iteration: their alphas are independent (the adjoints are not)
        int t = 0;
        for (; t + 1 < cnt; t += 2) {
            Alphas A, B;
            alphas(t, A);
            alphas(t + 1, B);
            if (__any_sync(0xffffffffu, A.c0 || A.c1)) adjoint(t, A);
            if (__any_sync(0xffffffffu, B.c0 || B.c1)) adjoint(t + 1, B);
        }
        if (t < cnt) {
            Alphas A;
            alphas(t, A);
            if (__any_sync(0xffffffffu, A.c0 || A.c1)) adjoint(t, A);
        }
        __syncwarp();   // every lane is done with buffer b before it is refilled
        cnt = cnt_next;
        have = have_next;
    }
    cp_async_wait_all();
    if constexpr (COUNT) {
        warp_count_add(&a.counters->frag_bwd_eval, n_eval);
        warp_count_add(&a.counters->frag_bwd_add, n_add);
        if (lane == 0 && n_visit) atomicAdd(&a.counters->visits_bwd, n_visit);
    }
}

template <bool COUNT>
__global__ void __launch_bounds__(32, 32) render_bwd_warp_kernel(BwdArgs a) {
    __shared__ BwdWarpSmem S;
    render_bwd_region<COUNT>(a, blockIdx.x, S);
}

template <int TILE, int CHUNK>
static void launch_fwd_c(const FwdArgs& a, int total_tiles, cudaStream_t st) {
    constexpr int NT = TileMap<TILE, kFwdPPT>::NT;
    if (a.op.count) render_fwd_kernel<TILE, CHUNK, true><<<total_tiles, NT, 0, st>>>(a);
    else render_fwd_kernel<TILE, CHUNK, false><<<total_tiles, NT, 0, st>>>(a);
}

template <int TILE>
static cudaError_t launch_fwd_t(const FwdArgs& a, int total_tiles, int chunk, cudaStream_t st) {
    switch (chunk) {
        case 32: launch_fwd_c<TILE, 32>(a, total_tiles, st); break;
        case 64: launch_fwd_c<TILE, 64>(a, total_tiles, st); break;
        case 128: launch_fwd_c<TILE, 128>(a, total_tiles, st); break;
        default: launch_fwd_c<TILE, 256>(a, total_tiles, st); break;
    }
    return cudaGetLastError();
}

template <int TILE, int CHUNK>
static void launch_bwd_c(const BwdArgs& a, int total_tiles, cudaStream_t st) {
    constexpr int NT = TileMap<TILE, kBwdPPT>::NT;
    if (a.op.count) render_bwd_kernel<TILE, CHUNK, true><<<total_tiles, NT, 0, st>>>(a);
    else render_bwd_kernel<TILE, CHUNK, false><<<total_tiles, NT, 0, st>>>(a);
}

template <int TILE>
static cudaError_t launch_bwd_t(const BwdArgs& a, int total_tiles, int chunk, cudaStream_t st) {
    switch (chunk) {
        case 32: launch_bwd_c<TILE, 32>(a, total_tiles, st); break;
        case 64: launch_bwd_c<TILE, 64>(a, total_tiles, st); break;
        case 128: launch_bwd_c<TILE, 128>(a, total_tiles, st); break;
        default: launch_bwd_c<TILE, 256>(a, total_tiles, st); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_render_fwd(const FwdArgs& a, int total_tiles, cudaStream_t st) {
    if (total_tiles <= 0) return cudaSuccess;
    return a.op.tile == 8 ? launch_fwd_t<8>(a, total_tiles, a.op.chunk, st)
                          : launch_fwd_t<16>(a, total_tiles, a.op.chunk, st);
}

// Zeroes the screen-space gradient records of the visible entries -- the only records the
// backward compositing adds to and the projection backward reads.
// Also, one thread each: the fused step's loss terms (lf.loss_out non-null; whatever the status,
// as the separate loss kernel) and its Adam step counter (adam_ctr non-null).
__global__ void __launch_bounds__(256) clear_grad2d_kernel(BwdArgs a, Counters* adam_ctr, float b1, float b2,
                                                           LossFinal lf) {
    if (lf.loss_out && blockIdx.x == 0 && threadIdx.x == 0)
        loss_finalize_one(lf.sums, lf.counts, lf.n_views, lf.lambda_rgb, lf.lambda_depth, 0.f, lf.has_depth,
                          lf.loss_out);
    if (a.counters->status != 0) return;
    if (adam_ctr && blockIdx.x == 0 && threadIdx.x == 0) adam_step_advance(adam_ctr, b1, b2);
    const int64_t E = (int64_t)a.counters->n_entries;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    // three threads per entry, one 16-byte word each (a warp's stores then cover about 11 whole
    // records); 32-bit index arithmetic while 3 E fits
    if (3 * E <= (int64_t)0xFFFFFFFFu) {
        const uint32_t n3 = (uint32_t)(3 * E);
        for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n3; e += gridDim.x * blockDim.x) {
            const uint32_t ent = e / 3u;
            a.grad2d[3 * (size_t)a.entries[ent] + (e - 3u * ent)] = z;
        }
    } else {
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < 3 * E; e += (int64_t)gridDim.x * blockDim.x)
            a.grad2d[3 * (size_t)a.entries[e / 3] + (size_t)(e % 3)] = z;
    }
}

cudaError_t launch_render_bwd(const BwdArgs& a, int total_tiles, cudaStream_t st, Counters* adam_ctr, float b1,
                              float b2, const LossFinal& lf) {
    clear_grad2d_kernel<<<sort_grid() * 4, 256, 0, st>>>(a, adam_ctr, b1, b2, lf);
    if (total_tiles <= 0) return cudaGetLastError();
    // 16 x 16 tiles: one independent warp per 8 x 8 region (8 x 8 tiles are one warp already)
    if (a.op.tile == 16) {
        if (a.op.count) render_bwd_warp_kernel<true><<<4 * total_tiles, 32, 0, st>>>(a);
        else render_bwd_warp_kernel<false><<<4 * total_tiles, 32, 0, st>>>(a);
        return cudaGetLastError();
    }
    return a.op.tile == 8 ? launch_bwd_t<8>(a, total_tiles, a.op.chunk, st)
                          : launch_bwd_t<16>(a, total_tiles, a.op.chunk, st);
}

// ----------------------------------------------------------------------------------------
// a9, persistent form of the step's last stages: forward compositing (with the fused L1 loss),
// backward compositing, the projection backward's entry and row parts and the fused Adam update
// as ONE cooperative kernel whose blocks are all resident, the phases separated by grid
// barriers:
//   phase 0  zero the screen-space gradient records of the visible entries
//   phase 1  forward tiles, taken from a queue in the largest-first work order
//   -- barrier --  (one thread: the loss terms and the Adam step counter)
//   phase 2  backward (tile, 8 x 8 region) items, one per warp, from a second queue
//   -- barrier --
//   phase 3  projection backward, entry part (grid-stride over the visible entries)
//   -- barrier --
//   phase 4a projection backward, row part: SH planes (with their Adam update)
//   -- barrier --
//   phase 4b projection backward, row part: geometry planes (with their Adam update)
// Every wait at a barrier is bounded: after `spin_limit` polls the block sets GS_ERR_TIMEOUT
// in the status word and returns, and so does every block that then finds the status set, so
// the kernel always ends.  The phases are the same device code as the stage kernels; the
// register budget of the kernel is that of its heaviest phase.
// ----------------------------------------------------------------------------------------
struct GridSync {
    unsigned int count;   // blocks arrived at the current barrier
    unsigned int gen;     // barriers completed
    unsigned int q_fwd;   // next forward work item
    unsigned int q_bwd;   // next backward work item
};
static_assert(sizeof(Counters) + sizeof(GridSync) <= 256, "the grid state follows the counters in their slot");

struct PersistentArgs {
    FwdArgs fwd;
    BwdArgs bwd;
    ProjectBwdArgs pb;
    Counters* counters;
    GridSync* sync;
    int total_tiles;
    float lambda_rgb, lambda_depth;
    int has_depth;
    float* loss_out;
    float b1, b2;
    unsigned long long spin_limit;
    int skip_block;   // diagnostic: this block does not arrive at the first barrier (-1: none)
};

constexpr int kPersistThreads = 256;
constexpr int kPersistWarps = kPersistThreads / 32;
static_assert(kPersistThreads == kEntryThreads, "the entry part runs with the persistent block");
static_assert(kPersistThreads == TileMap<16, kFwdPPT>::NT, "a forward tile is one persistent block");

template <int DEG>
struct PersistSmem {
    union {
        FwdSmem<16, 256> fwd;
        BwdWarpSmem bwd[kPersistWarps];
        float mv[sh_mv_floats<DEG, kPersistThreads>()];
        float gmv[geo_mv_floats<kPersistThreads>()];
    } u;
    float tw[GS_MAX_VIEWS * 6];
    float cam[GS_MAX_VIEWS * 12];
    unsigned int item;
    int ok;
};

// Grid barrier with a bounded wait.  Thread 0 of each block reads the generation, arrives
// (unless `arrive` is false), and the last block to arrive resets the count and advances the
// generation; the others poll it, at most spin_limit times, about 0.1 us apart.  Returns false
// (for the whole block) if the wait gave up or the status word is set.
template <int DEG>
__device__ __forceinline__ bool grid_barrier(const PersistentArgs& P, bool arrive, PersistSmem<DEG>& S) {
    __syncthreads();
    if (threadIdx.x == 0) {
        GridSync* g = P.sync;
        volatile unsigned int* vgen = &g->gen;
        const unsigned int g0 = *vgen;
        __threadfence();
        bool released = false;
        if (arrive && atomicAdd(&g->count, 1u) + 1u == gridDim.x) {
            atomicExch(&g->count, 0u);
            __threadfence();
            atomicAdd(&g->gen, 1u);
            released = true;
        }
        int ok = 1;
        if (!released) {
            unsigned long long polls = 0;
            while (*vgen == g0) {
                if (++polls > P.spin_limit) {
                    set_status(P.counters, GS_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        S.ok = ok && *(volatile uint32_t*)&P.counters->status == 0u;
    }
    __syncthreads();
    return S.ok != 0;
}

template <int DEG>
__global__ void __launch_bounds__(kPersistThreads, 2) step_persistent_kernel(PersistentArgs P) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    PersistSmem<DEG>& S = *reinterpret_cast<PersistSmem<DEG>*>(s_raw);
    if (P.counters->status != 0) return;   // failed earlier stage: every block leaves at once
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    {   // phase 0
        const int64_t E = (int64_t)P.counters->n_entries;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int64_t e = (int64_t)blockIdx.x * kPersistThreads + threadIdx.x; e < E;
             e += (int64_t)gridDim.x * kPersistThreads) {
            float4* rec = P.bwd.grad2d + 3 * (size_t)P.bwd.entries[e];
            rec[0] = z;
            rec[1] = z;
            rec[2] = z;
        }
    }
    for (;;) {   // phase 1
        if (threadIdx.x == 0) S.item = atomicAdd(&P.sync->q_fwd, 1u);
        __syncthreads();
        const unsigned int t = S.item;
        __syncthreads();
        if (t >= (unsigned int)P.total_tiles) break;
        render_fwd_tile<16, 256, false>(P.fwd, (int)t, S.u.fwd);
    }
    if (!grid_barrier<DEG>(P, (int)blockIdx.x != P.skip_block, S)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (P.loss_out)
            loss_finalize_one(P.fwd.loss_sums, P.fwd.loss_counts, P.fwd.n_views, P.lambda_rgb, P.lambda_depth, 0.f,
                              P.has_depth, P.loss_out);
        adam_step_advance(P.counters, P.b1, P.b2);
    }
    for (;;) {   // phase 2
        unsigned int item = 0;
        if (lane == 0) item = atomicAdd(&P.sync->q_bwd, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= 4u * (unsigned int)P.total_tiles) break;
        render_bwd_region<false>(P.bwd, (int)item, S.u.bwd[warp]);
    }
    if (!grid_barrier<DEG>(P, true, S)) return;
    project_bwd_entry_part(P.pb, blockIdx.x, gridDim.x, S.tw);   // phase 3
    if (!grid_barrier<DEG>(P, true, S)) return;
    for (int64_t blk = blockIdx.x; blk * kPersistThreads < P.pb.n; blk += gridDim.x) {   // phase 4a
        project_bwd_sh_rows<DEG, true, kPersistThreads>(P.pb, blk, S.tw, S.u.mv, S.cam);
        __syncthreads();
    }
    if (!grid_barrier<DEG>(P, true, S)) return;
    for (int64_t blk = blockIdx.x; blk * kPersistThreads < P.pb.n; blk += gridDim.x)   // phase 4b
        project_bwd_geo_rows<DEG, true, kPersistThreads>(P.pb, blk, S.u.gmv);
}

template <int DEG>
static cudaError_t launch_persistent_d(const PersistentArgs& P, cudaStream_t st, int* grid_out) {
    const size_t smem = sizeof(PersistSmem<DEG>);
    static bool attr_set[kMaxDevices] = {};
    cudaError_t e = once_per_device(attr_set, [&] {
        return cudaFuncSetAttribute(step_persistent_kernel<DEG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    });
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_persistent_kernel<DEG>, kPersistThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    const int grid = per_sm * device_sms();
    if (grid_out) *grid_out = grid;
    if ((e = cudaMemsetAsync(P.sync, 0, sizeof(GridSync), st)) != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kPersistThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, step_persistent_kernel<DEG>, P);
}

cudaError_t launch_step_persistent(const FwdArgs& fwd, const BwdArgs& bwd, const ProjectBwdArgs& pb, int deg,
                                   int total_tiles, float lambda_rgb, float lambda_depth, int has_depth,
                                   float* loss_out, float b1, float b2, long long spin_limit, int skip_block,
                                   cudaStream_t st, int* grid_out) {
    PersistentArgs P;
    P.fwd = fwd;
    P.bwd = bwd;
    P.pb = pb;
    P.counters = fwd.counters;
    P.sync = reinterpret_cast<GridSync*>(reinterpret_cast<char*>(fwd.counters) + 128);
    P.total_tiles = total_tiles;
    P.lambda_rgb = lambda_rgb;
    P.lambda_depth = lambda_depth;
    P.has_depth = has_depth;
    P.loss_out = loss_out;
    P.b1 = b1;
    P.b2 = b2;
    P.spin_limit = spin_limit > 0 ? (unsigned long long)spin_limit : 10000000ull;
    P.skip_block = skip_block;
    switch (deg) {
        case 0: return launch_persistent_d<0>(P, st, grid_out);
        case 1: return launch_persistent_d<1>(P, st, grid_out);
        case 2: return launch_persistent_d<2>(P, st, grid_out);
        default: return launch_persistent_d<3>(P, st, grid_out);
    }
}

}  // namespace gs
