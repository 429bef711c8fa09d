// The rest of the mapping objective (RMGS-SLAM §III-C, "Optimization"): the interior mask
// M_int = Erode(M_geo, r_erode) with M_geo the accumulated-opacity support of the current
// rendering, and lambda_rgb L_rgb + lambda_ssim (1 - SSIM) + lambda_depth L_depth evaluated
// inside it, with dL/dC and dL/dD for the backward.  Used by the step instead of the forward's
// fused L1 epilogue when the SSIM term or the render-derived mask is switched on (the mask
// needs every neighbour's transmittance, so it cannot be taken inside the forward).
//
// SSIM (per channel): x = C * M, y = C~ * M, 11 x 11 Gaussian window (sigma 1.5) with zeros
// outside the image, C1 = 0.01^2, C2 = 0.03^2; the SSIM map is averaged over M and the three
// channels.  The window is separable: each kernel makes a horizontal pass over a tile with a
// 5-pixel halo in shared memory, then a vertical one.  The forward writes, per pixel and
// channel, the three partial derivatives of the weighted SSIM map with respect to the local
// mean, second moment and cross moment; the backward convolves them back onto the pixels.
#include "gs_kernels.cuh"

namespace gs {

constexpr int kObjTX = 32, kObjTY = 8;          // threads of a block
constexpr int kObjRows = 2;                      // output rows per thread
constexpr int kObjH = kObjTY * kObjRows;         // output tile: 32 x 16 pixels
constexpr int kHalo = 5;                         // window radius
constexpr int kInW = kObjTX + 2 * kHalo, kInH = kObjH + 2 * kHalo;
constexpr float kSsimC1 = 0.01f * 0.01f, kSsimC2 = 0.03f * 0.03f;

// Interior mask: [1 - T >= tau] eroded by the radius-r disk (outside the image counts as
// outside the support), and the caller's mask.  The block thresholds its 32 x 8 pixels and a
// halo of r once into shared memory, then every pixel tests the disk there.
constexpr int kMaskMaxR = 16;
__global__ void __launch_bounds__(kObjTX * kObjTY) render_mask_kernel(ObjArgs a) {
    __shared__ uint8_t s_geo[kObjTY + 2 * kMaskMaxR][kObjTX + 2 * kMaskMaxR];
    __shared__ int s_w[2 * kMaskMaxR + 1];   // half-width of the disk in each row
    const View& V = a.views[blockIdx.z];
    const int x0 = blockIdx.x * kObjTX, y0 = blockIdx.y * kObjTY;
    if (x0 >= V.W || y0 >= V.H) return;   // (the whole block)
    const int r = a.r_erode;
    const int tw = kObjTX + 2 * r, th = kObjTY + 2 * r;
    const float* T = a.T_final + V.pix_off;
    const int t = threadIdx.y * kObjTX + threadIdx.x;
    if (t <= 2 * r) {
        const int dy = t - r;
        int w = 0;
        while ((w + 1) * (w + 1) + dy * dy <= r * r) w++;
        s_w[t] = w;
    }
    for (int i = t; i < tw * th; i += kObjTX * kObjTY) {
        const int iy = i / tw, ix = i - iy * tw;
        const int gx = x0 - r + ix, gy = y0 - r + iy;
        const bool inside = gx >= 0 && gx < V.W && gy >= 0 && gy < V.H;
        s_geo[iy][ix] = inside && __fsub_rn(1.f, __ldg(T + (int64_t)gy * V.W + gx)) >= a.tau;
    }
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= V.W || y >= V.H) return;
    bool in = true;
    for (int dy = -r; dy <= r; dy++) {
        const int w = s_w[dy + r];   // the largest w with w^2 + dy^2 <= r^2
        const uint8_t* row = &s_geo[threadIdx.y + r + dy][threadIdx.x + r];
        for (int dx = -w; dx <= w; dx++) in = in && row[dx];
    }
    const int64_t g = V.pix_off + (int64_t)y * V.W + x;
    if (a.caller_mask) in = in && a.caller_mask[g] != 0;
    a.mask_out[g] = in ? 1 : 0;
}

// Block sums of two per-thread values, one FP64 atomic each (every thread of the block calls
// it; the leading barrier lets it be called again right after).
__device__ __forceinline__ void block_add2(float s0, float s1, double* dst0, double* dst1) {
    __shared__ double s_r[2][kObjTX * kObjTY / 32];
    const int t = threadIdx.y * kObjTX + threadIdx.x, lane = t & 31, w = t >> 5;
    __syncthreads();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if (lane == 0) { s_r[0][w] = (double)s0; s_r[1][w] = (double)s1; }
    __syncthreads();
    if (t == 0) {
        double a0 = 0, a1 = 0;
        for (int k = 0; k < kObjTX * kObjTY / 32; k++) { a0 += s_r[0][k]; a1 += s_r[1][k]; }
        if (a0 != 0.0) atomicAdd(dst0, a0);
        if (dst1 && a1 != 0.0) atomicAdd(dst1, a1);
    }
}

// Masked L1 terms: the same arithmetic as the forward's fused epilogue, on a given mask.
__global__ void __launch_bounds__(kObjTX * kObjTY) masked_l1_kernel(ObjArgs a) {
    const int v = blockIdx.z;
    const View& V = a.views[v];
    const int x = blockIdx.x * kObjTX + threadIdx.x, y = blockIdx.y * kObjTY + threadIdx.y;
    float lr = 0.f, ld = 0.f;
    if (x < V.W && y < V.H) {
        const int64_t P = (int64_t)V.W * V.H, p = (int64_t)y * V.W + x, g = V.pix_off + p;
        const float* c = a.rgb + 3 * V.pix_off;
        const float* t = a.tgt_rgb + 3 * V.pix_off;
        const bool in = a.mask ? a.mask[g] != 0 : true;
        const float cm = (float)a.counts[2 * v], cd = (float)a.counts[2 * v + 1];
        const float inv_v = 1.0f / (float)a.n_views;
        const float krgb = (in && cm > 0.f) ? a.lambda_rgb * inv_v / cm : 0.f;
        float* dl = a.dl_drgb + 3 * V.pix_off;
#pragma unroll
        for (int ch = 0; ch < 3; ch++) {
            const float r = c[ch * P + p] - t[ch * P + p];
            dl[ch * P + p] = krgb * (float)((r > 0.f) - (r < 0.f));
            if (in) lr += fabsf(r);
        }
        if (a.dl_ddepth) {
            const float td = a.tgt_depth ? a.tgt_depth[g] : 0.f;
            const bool ind = in && td > 0.f;
            const float kd = (ind && cd > 0.f) ? a.lambda_depth * inv_v / cd : 0.f;
            const float rd = a.depth[g] - td;
            a.dl_ddepth[g] = kd * (float)((rd > 0.f) - (rd < 0.f));
            if (ind) ld += fabsf(rd);
        }
    }
    block_add2(lr, ld, &a.sums[3 * v], &a.sums[3 * v + 1]);
}

// Register-blocked separable passes over a tile (kInH x kInW inputs -> kObjH x kObjTX outputs):
// a horizontal task makes 4 consecutive outputs of one row from 14 inputs (four 16-byte shared
// loads; rows padded to kInS floats keep the quarter-warp phases conflict-free), a vertical
// task 2 consecutive rows of one column from 12.  All three channels of a tile are loaded in
// one phase, so the global loads of a block are in flight together.
constexpr int kSeg = 4;                       // horizontal outputs per task
constexpr int kSegs = kObjTX / kSeg;          // tasks per row
constexpr int kHIn = kSeg + 2 * kHalo;        // inputs per horizontal task (14)
constexpr int kInS = 44;                      // padded row stride of the input tiles
static_assert(kInS >= kInW && kInS % 4 == 0 && kInS >= 4 * ((kHIn + 3) / 4) + kObjTX - kSeg, "tile row stride");

__device__ __forceinline__ void load_row16(const float* row, float (&v)[16]) {
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const float4 q = *reinterpret_cast<const float4*>(row + 4 * j);
        v[4 * j] = q.x; v[4 * j + 1] = q.y; v[4 * j + 2] = q.z; v[4 * j + 3] = q.w;
    }
}

__device__ __forceinline__ void hconv(const float (&win)[11], const float (&v)[16], float* out) {
    float o[kSeg];
#pragma unroll
    for (int k = 0; k < kSeg; k++) {
        float acc = 0.f;
#pragma unroll
        for (int q = 0; q < 2 * kHalo + 1; q++) acc = fmaf(win[q], v[k + q], acc);
        o[k] = acc;
    }
    *reinterpret_cast<float4*>(out) = make_float4(o[0], o[1], o[2], o[3]);
}

// SSIM forward, fused with the masked L1 terms.  Per channel: the local means of x = C M and
// y = C~ M, E[x^2 + y^2] and E[xy] (SSIM uses the two variances only summed), the SSIM map (summed over M), and the partials
// k(q) dS/dmu_x, k(q) dS/dE[x^2], k(q) dS/dE[xy], k(q) = -lambda_ssim M(q) / (3 |M| views)
// (the gradient of lambda_ssim (1 - SSIM) / views); and at the same output pixels the L1
// colour terms (and, with the first channel, the depth term) with the epilogue's arithmetic.
__global__ void __launch_bounds__(kObjTX * kObjTY) ssim_fwd_kernel(ObjArgs a) {
    __shared__ __align__(16) float s_x[3][kInH][kInS];
    __shared__ __align__(16) float s_y[3][kInH][kInS];
    // horizontal sums of x, y, x^2 + y^2 and xy (SSIM needs E[x^2] and E[y^2] only summed)
    __shared__ __align__(16) float s_h[4][kInH][kObjTX];
    __shared__ uint8_t s_m[kInH][kInW];
    const int v = blockIdx.z;
    const View& V = a.views[v];
    const int x0 = blockIdx.x * kObjTX, y0 = blockIdx.y * kObjH;
    if (x0 >= V.W || y0 >= V.H) return;   // (the whole block: no barrier is skipped by part of it)
    const int t = threadIdx.y * kObjTX + threadIdx.x;
    const int64_t P = (int64_t)V.W * V.H;
    const uint32_t cm = a.counts[2 * v];
    const float cd = (float)a.counts[2 * v + 1];
    const float inv_v = 1.0f / (float)a.n_views;
    const float k = cm > 0 ? -a.lambda_ssim / (3.f * (float)cm * (float)a.n_views) : 0.f;
    const float kr = cm > 0 ? a.lambda_rgb * inv_v / (float)cm : 0.f;
    const int ox = t & 31, oy0 = (t >> 5) * kObjRows;   // vertical task: column, first row
    const float* c = a.rgb + 3 * V.pix_off;
    const float* tc = a.tgt_rgb + 3 * V.pix_off;
    for (int i = t; i < kInH * kInW; i += kObjTX * kObjTY) {
        const int iy = i / kInW, ix = i - iy * kInW;
        const int gx = x0 - kHalo + ix, gy = y0 - kHalo + iy;
        float xv[3] = {0.f, 0.f, 0.f}, yv[3] = {0.f, 0.f, 0.f};
        bool in = false;
        if (gx >= 0 && gx < V.W && gy >= 0 && gy < V.H) {
            const int64_t p = (int64_t)gy * V.W + gx;
            in = a.mask ? a.mask[V.pix_off + p] != 0 : true;
#pragma unroll
            for (int ch = 0; ch < 3; ch++) {
                xv[ch] = in ? c[ch * P + p] : 0.f;
                yv[ch] = in ? tc[ch * P + p] : 0.f;
            }
        }
#pragma unroll
        for (int ch = 0; ch < 3; ch++) { s_x[ch][iy][ix] = xv[ch]; s_y[ch][iy][ix] = yv[ch]; }
        s_m[iy][ix] = in ? 1 : 0;
    }
    __syncthreads();
    float ssum = 0.f, lr = 0.f, ld = 0.f;
    for (int ch = 0; ch < 3; ch++) {
        for (int task = t; task < kInH * kSegs; task += kObjTX * kObjTY) {
            const int iy = task / kSegs, cx = (task - iy * kSegs) * kSeg;
            float xs[16], ys[16], tmp[16];
            load_row16(&s_x[ch][iy][cx], xs);
            load_row16(&s_y[ch][iy][cx], ys);
            hconv(a.win, xs, &s_h[0][iy][cx]);
            hconv(a.win, ys, &s_h[1][iy][cx]);
#pragma unroll
            for (int q = 0; q < kHIn; q++) tmp[q] = fmaf(xs[q], xs[q], ys[q] * ys[q]);
            hconv(a.win, tmp, &s_h[2][iy][cx]);
#pragma unroll
            for (int q = 0; q < kHIn; q++) tmp[q] = xs[q] * ys[q];
            hconv(a.win, tmp, &s_h[3][iy][cx]);
        }
        __syncthreads();
        float mo[4][kObjRows];
#pragma unroll
        for (int m = 0; m < 4; m++) {
            float col[kObjRows + 2 * kHalo];
#pragma unroll
            for (int q = 0; q < kObjRows + 2 * kHalo; q++) col[q] = s_h[m][oy0 + q][ox];
#pragma unroll
            for (int rr = 0; rr < kObjRows; rr++) {
                float acc = 0.f;
#pragma unroll
                for (int q = 0; q < 2 * kHalo + 1; q++) acc = fmaf(a.win[q], col[rr + q], acc);
                mo[m][rr] = acc;
            }
        }
#pragma unroll
        for (int rr = 0; rr < kObjRows; rr++) {
            const int gx = x0 + ox, gy = y0 + oy0 + rr;
            if (gx >= V.W || gy >= V.H) continue;
            const float mx = mo[0][rr], my = mo[1][rr], e2 = mo[2][rr], exy = mo[3][rr];
            const float sxy = exy - mx * my;
            const float A1 = 2.f * mx * my + kSsimC1, A2 = 2.f * sxy + kSsimC2;
            const float B1 = mx * mx + my * my + kSsimC1, B2 = e2 - mx * mx - my * my + kSsimC2;
            const float inv = 1.f / (B1 * B2);
            const float S = A1 * A2 * inv;
            const int64_t p = (int64_t)gy * V.W + gx;
            const bool in = s_m[oy0 + rr + kHalo][ox + kHalo] != 0;
            const float kq = in ? k : 0.f;
            if (in) ssum += S;
            const float d_mu = 2.f * my * (A2 - A1) * inv - 2.f * mx * S * (1.f / B1 - 1.f / B2);
            float* part = a.ssim_part + 9 * V.pix_off + (3 * ch) * P + p;
            part[0] = kq * d_mu;
            part[P] = kq * (-S / B2);
            part[2 * P] = kq * (2.f * A1 * inv);
            // L1 colour term of this channel (x, y are C, C~ inside the mask)
            const float r = s_x[ch][oy0 + rr + kHalo][ox + kHalo] - s_y[ch][oy0 + rr + kHalo][ox + kHalo];
            const float krgb = in ? kr : 0.f;
            a.dl_drgb[3 * V.pix_off + ch * P + p] = krgb * (float)((r > 0.f) - (r < 0.f));
            if (in) lr += fabsf(r);
            if (ch == 0 && a.dl_ddepth) {
                const int64_t g = V.pix_off + p;
                const float td = a.tgt_depth ? a.tgt_depth[g] : 0.f;
                const bool ind = in && td > 0.f;
                const float kd = (ind && cd > 0.f) ? a.lambda_depth * inv_v / cd : 0.f;
                const float rd = a.depth[g] - td;
                a.dl_ddepth[g] = kd * (float)((rd > 0.f) - (rd < 0.f));
                if (ind) ld += fabsf(rd);
            }
        }
        __syncthreads();   // s_h is refilled for the next channel
    }
    block_add2(lr, ld, &a.sums[3 * v], &a.sums[3 * v + 1]);
    block_add2(ssum, 0.f, &a.sums[3 * v + 2], nullptr);
}

// SSIM backward: dL/dx(p) = sum_q w(q - p) [P_mu(q) + 2 x(p) P_xx(q) + y(p) P_xy(q)], and
// dL/dC = M dL/dx, added to the L1 gradient already in dl_drgb.  The three partial maps of a
// channel are loaded together; channels are processed one after the other.
__global__ void __launch_bounds__(kObjTX * kObjTY) ssim_bwd_kernel(ObjArgs a) {
    __shared__ __align__(16) float s_p[3][kInH][kInS];
    __shared__ __align__(16) float s_h[3][kInH][kObjTX];
    const View& V = a.views[blockIdx.z];
    const int x0 = blockIdx.x * kObjTX, y0 = blockIdx.y * kObjH;
    if (x0 >= V.W || y0 >= V.H) return;
    const int t = threadIdx.y * kObjTX + threadIdx.x;
    const int64_t P = (int64_t)V.W * V.H;
    const int ox = t & 31, oy0 = (t >> 5) * kObjRows;
    for (int ch = 0; ch < 3; ch++) {
        const float* part = a.ssim_part + 9 * V.pix_off + (3 * ch) * P;
        for (int i = t; i < kInH * kInW; i += kObjTX * kObjTY) {
            const int iy = i / kInW, ix = i - iy * kInW;
            const int gx = x0 - kHalo + ix, gy = y0 - kHalo + iy;
            float p0 = 0.f, p1 = 0.f, p2 = 0.f;
            if (gx >= 0 && gx < V.W && gy >= 0 && gy < V.H) {
                const int64_t p = (int64_t)gy * V.W + gx;
                p0 = part[p]; p1 = part[P + p]; p2 = part[2 * P + p];
            }
            s_p[0][iy][ix] = p0; s_p[1][iy][ix] = p1; s_p[2][iy][ix] = p2;
        }
        __syncthreads();
        for (int task = t; task < 3 * kInH * kSegs; task += kObjTX * kObjTY) {
            const int m = task / (kInH * kSegs), rest = task - m * (kInH * kSegs);
            const int iy = rest / kSegs, cx = (rest - iy * kSegs) * kSeg;
            float v16[16];
            load_row16(&s_p[m][iy][cx], v16);
            hconv(a.win, v16, &s_h[m][iy][cx]);
        }
        __syncthreads();
        float cv[3][kObjRows];
#pragma unroll
        for (int m = 0; m < 3; m++) {
            float col[kObjRows + 2 * kHalo];
#pragma unroll
            for (int q = 0; q < kObjRows + 2 * kHalo; q++) col[q] = s_h[m][oy0 + q][ox];
#pragma unroll
            for (int rr = 0; rr < kObjRows; rr++) {
                float acc = 0.f;
#pragma unroll
                for (int q = 0; q < 2 * kHalo + 1; q++) acc = fmaf(a.win[q], col[rr + q], acc);
                cv[m][rr] = acc;
            }
        }
#pragma unroll
        for (int rr = 0; rr < kObjRows; rr++) {
            const int gx = x0 + ox, gy = y0 + oy0 + rr;
            if (gx >= V.W || gy >= V.H) continue;
            const int64_t p = (int64_t)gy * V.W + gx;
            const bool in = a.mask ? a.mask[V.pix_off + p] != 0 : true;
            if (!in) continue;
            const float xv = a.rgb[3 * V.pix_off + ch * P + p], yv = a.tgt_rgb[3 * V.pix_off + ch * P + p];
            float* dl = a.dl_drgb + 3 * V.pix_off + ch * P + p;
            *dl += cv[0][rr] + 2.f * xv * cv[1][rr] + yv * cv[2][rr];
        }
        __syncthreads();
    }
}

static dim3 obj_grid(const ObjArgs& a, int tile_h) {
    return dim3((unsigned)((a.max_w + kObjTX - 1) / kObjTX), (unsigned)((a.max_h + tile_h - 1) / tile_h),
                (unsigned)a.n_views);
}

cudaError_t launch_render_mask(const ObjArgs& a, cudaStream_t st) {
    if (a.n_views <= 0) return cudaSuccess;
    render_mask_kernel<<<obj_grid(a, kObjTY), dim3(kObjTX, kObjTY), 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_objective(const ObjArgs& a, cudaStream_t st) {
    if (a.n_views <= 0) return cudaSuccess;
    if (a.lambda_ssim > 0.f) {
        // (the L1 terms ride along in the SSIM forward, which holds C and C~ at every pixel)
        ssim_fwd_kernel<<<obj_grid(a, kObjH), dim3(kObjTX, kObjTY), 0, st>>>(a);
        ssim_bwd_kernel<<<obj_grid(a, kObjH), dim3(kObjTX, kObjTY), 0, st>>>(a);
    } else {
        masked_l1_kernel<<<obj_grid(a, kObjTY), dim3(kObjTX, kObjTY), 0, st>>>(a);
    }
    return cudaGetLastError();
}

// 1-D weights of the normalised 11-tap Gaussian (sigma 1.5), rounded once to FP32.
void ssim_window(float (&w)[11]) {
    double g[11], s = 0;
    for (int i = 0; i < 11; i++) {
        const double d = i - 5;
        g[i] = exp(-d * d / (2.0 * 1.5 * 1.5));
        s += g[i];
    }
    for (int i = 0; i < 11; i++) w[i] = (float)(g[i] / s);
}

}  // namespace gs
