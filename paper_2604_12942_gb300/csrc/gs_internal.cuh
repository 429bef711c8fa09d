// Internal device-side definitions of the sm_103a 3DGS mapping-step library.
// The math here follows §III-C of RMGS-SLAM (standard differentiable Gaussian splatting,
// depth composited with the colour weights) under the readings documented in gs.h.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gs.h"

namespace gs {

constexpr float kLn2 = 0.69314718055994530942f;
constexpr float kLog2e = 1.44269504088896340736f;
constexpr int kSortBins = 256;                    // 8-bit digits (64-bit keys)
constexpr int kSortMaxBins = 512;                 // up to 9-bit digits (32-bit keys)
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;                     // per thread per chunk
constexpr int kSortChunk = kSortThreads * kSortItems;
constexpr int kSortMaxGrid = 512;                 // blocks of a sort pass (at most)
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanBlock = kScanThreads * kScanItems;
constexpr int kEmitThreads = 256;
constexpr int kEmitChunk = 2048;                  // pairs per chunk of the balanced emission

// Launch attributes (a kernel's dynamic shared-memory limit) and grid sizes taken from device
// properties belong to one device: the library keeps them per device, so it works on every
// device it is used on.  Concurrent first calls may both set an attribute (harmless).
constexpr int kMaxDevices = 64;
inline int current_device() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return -1;
    return d;
}
// Runs set() once per device; a failed attempt is retried on the next call.
template <class F>
inline cudaError_t once_per_device(bool (&done)[kMaxDevices], F set) {
    const int d = current_device();
    if (d >= 0 && done[d]) return cudaSuccess;
    const cudaError_t e = set();
    if (e == cudaSuccess && d >= 0) done[d] = true;
    return e;
}
inline int device_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 148;
}

// Per-view table held in the workspace.
struct View {
    int32_t W, H, tiles_x, tiles_y;
    int32_t tile_off, n_tiles;
    int64_t pix_off;
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    float cw[3];          // camera centre -R^T t
    float limx, limy;     // clamp of x/z, y/z in the Jacobian
};

struct Counters {
    uint32_t status;
    uint32_t n_entries32;  // copy of n_entries for the host-side counter block
    unsigned long long n_pairs;
    // fragments (pixel, Gaussian) evaluated / added by the forward and backward compositing
    unsigned long long frag_fwd_eval, frag_fwd_add, frag_bwd_eval, frag_bwd_add;
    uint32_t visits_fwd, visits_bwd;   // (record, warp) visits of the compositing loops
    unsigned long long adam_step;   // Adam step counter of gs_step (device-side, graph-safe)
    float adam_bc1, adam_bc2;       // 1 - b1^t, 1 - b2^t for that step
    unsigned long long n_entries;   // visible (view, Gaussian) entries of the last binning
};
constexpr size_t kCountersResetBytes = 56;   // status .. visit counters: cleared per step

// One Adam update of a parameter p with gradient g, given the inverse bias corrections
// ibc1 = 1 / (1 - b1^t), ibc2 = 1 / (1 - b2^t); shared by the Adam kernel and the fused
// projection backward.  Every operation is an explicitly rounded intrinsic, so the compiler
// cannot contract it differently in the two kernels and both give bit-identical results; the
// bias corrections are multiplications and the step a correctly rounded square root and
// reciprocal (one rounding more than three divisions, several times fewer instructions).
__device__ __forceinline__ void adam_update(float& p, float g, float& m, float& v, float lr, float b1, float b2,
                                            float eps, float ibc1, float ibc2) {
    m = __fmaf_rn(b1, m, __fmul_rn(__fsub_rn(1.f, b1), g));
    v = __fmaf_rn(b2, v, __fmul_rn(__fmul_rn(__fsub_rn(1.f, b2), g), g));
    const float mh = __fmul_rn(m, ibc1), vh = __fmul_rn(v, ibc2);
    p = __fsub_rn(p, __fmul_rn(__fmul_rn(lr, mh), __frcp_rn(__fadd_rn(__fsqrt_rn(vh), eps))));
}

// Asynchronous 16-byte global -> shared copies (cp.async, L2 only), in commit groups.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// all but the most recently committed group have completed
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Adds a warp's per-lane counts to a device counter (one atomic per warp).
__device__ __forceinline__ void warp_count_add(unsigned long long* dst, uint32_t v) {
    unsigned long long s = v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(dst, s);
}

struct Opts {
    float near_z, dilation, alpha_min, alpha_max, T_min, clamp_fov;
    float bg0, bg1, bg2;
    float lambda_rgb, lambda_depth;
    int tile, chunk;
    int count;   // fill the fragment / visit counters
};

__device__ __forceinline__ void set_status(Counters* c, uint32_t s) { atomicCAS(&c->status, 0u, s); }

// Advances the device-side Adam step counter and stores the bias corrections of that step
// (one thread); a failed step (status set) takes no Adam step.
__device__ __forceinline__ void adam_step_advance(Counters* c, float b1, float b2) {
    if (c->status != 0) return;
    const unsigned long long t = c->adam_step + 1;
    c->adam_step = t;
    c->adam_bc1 = (float)(1.0 - pow((double)b1, (double)t));
    c->adam_bc2 = (float)(1.0 - pow((double)b2, (double)t));
}

// The loss terms of every view and their mean from the accumulated masked sums (one thread):
// lambda_rgb L1 / |M| + lambda_depth L1_D / |M_D| + lambda_ssim (1 - mean SSIM over M).
__device__ __forceinline__ void loss_finalize_one(const double* sums, const uint32_t* counts, int n_views,
                                                  float lambda_rgb, float lambda_depth, float lambda_ssim,
                                                  int has_depth, float* loss_out) {
    double tot = 0;
    for (int v = 0; v < n_views; v++) {
        const double cm = counts[2 * v], cd = counts[2 * v + 1];
        double l = cm > 0 ? lambda_rgb * sums[3 * v] / cm : 0.0;
        if (has_depth && cd > 0) l += lambda_depth * sums[3 * v + 1] / cd;
        if (lambda_ssim > 0.f && cm > 0) l += lambda_ssim * (1.0 - sums[3 * v + 2] / (3.0 * cm));
        loss_out[v] = (float)l;
        tot += l;
    }
    loss_out[n_views] = (float)(tot / n_views);
}

// ---------------------------------------------------------------------------------------
// Compositing exponent.  The record stores the inverse 2-D covariance [[A, B], [B, C]]
// scaled by k = -log2(e)/2, (a, b, c) = k (A, B, C), so that alpha = o * 2^e with
//   h_x = a dx + b dy,  h_y = b dx + c dy,  e = dx h_x + dy h_y  (= -q/2 * log2(e)).
// (h_x, h_y) is also -1/2 of de/d(u, v), which the backward reuses.  The forward and the
// backward kernels call exactly this sequence of correctly rounded operations, so both take
// the same skip / stop decisions.
// ---------------------------------------------------------------------------------------
struct FragE {
    float hx, hy, e;
};

__device__ __forceinline__ FragE frag_exponent(float dx, float dy, float a, float b, float c) {
    FragE f;
    f.hx = __fmaf_rn(a, dx, __fmul_rn(b, dy));
    f.hy = __fmaf_rn(c, dy, __fmul_rn(b, dx));
    f.e = __fmaf_rn(dx, f.hx, __fmul_rn(dy, f.hy));
    return f;
}

// Two exponents at once in packed FP32 pairs (sm_100+ f32x2 arithmetic): component by
// component the same correctly rounded operations as frag_exponent, so bit-identical.
struct FragE2 {
    float2 hx, hy, e;
};

__device__ __forceinline__ float2 dup2(float x) { return make_float2(x, x); }

__device__ __forceinline__ FragE2 frag_exponent2(float2 dx, float2 dy, float2 a, float2 b, float2 c) {
    FragE2 f;
    f.hx = __ffma2_rn(a, dx, __fmul2_rn(b, dy));
    f.hy = __ffma2_rn(c, dy, __fmul2_rn(b, dx));
    f.e = __ffma2_rn(dx, f.hx, __fmul2_rn(dy, f.hy));
    return f;
}

constexpr float kConicScale = -0.5f * kLog2e;

// 2^x by the hardware ex2 instruction (flush-to-zero for tiny results).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/x by the hardware rcp instruction.
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Tiles covered along one axis by centre c and integer radius r: [floor((c-r)/T),
// floor((c+r)/T)] clamped to [0, n-1]; false if empty.  FP32, correctly rounded, as gs.h
// defines it.
__device__ __forceinline__ bool tile_span(float c, int r, int tile, int n, int& lo, int& hi) {
    const float rf = (float)r;
    const float tf = (float)tile;
    float a = floorf(__fdiv_rn(__fsub_rn(c, rf), tf));
    float b = floorf(__fdiv_rn(__fadd_rn(c, rf), tf));
    if (!(b >= 0.0f) || !(a <= (float)(n - 1))) return false;
    a = fmaxf(a, 0.0f);
    b = fminf(b, (float)(n - 1));
    lo = (int)a;
    hi = (int)b;
    return hi >= lo;
}

// ---------------------------------------------------------------------------------------
// Real spherical harmonics, degree <= 3 (orthonormal, Condon-Shortley phase).
// ---------------------------------------------------------------------------------------
constexpr float SH0 = 0.28209479177387814f;
constexpr float SH1 = 0.48860251190291992f;
constexpr float SH2a = 1.09254843059207907f;
constexpr float SH2b = 0.31539156525252005f;
constexpr float SH2c = 0.54627421529603959f;
constexpr float SH3a = 0.59004358992664352f;
constexpr float SH3b = 2.89061144264055405f;
constexpr float SH3c = 0.45704579946446573f;
constexpr float SH3d = 0.37317633259011540f;
constexpr float SH3e = 1.44530572132027702f;

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
    Y[0] = SH0;
    if (DEG >= 1) {
        Y[1] = -SH1 * y;
        Y[2] = SH1 * z;
        Y[3] = -SH1 * x;
    }
    if (DEG >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = SH2a * x * y;
        Y[5] = -SH2a * y * z;
        Y[6] = SH2b * (2.f * zz - xx - yy);
        Y[7] = -SH2a * x * z;
        Y[8] = SH2c * (xx - yy);
        if (DEG >= 3) {
            Y[9] = -SH3a * y * (3.f * xx - yy);
            Y[10] = SH3b * x * y * z;
            Y[11] = -SH3c * y * (4.f * zz - xx - yy);
            Y[12] = SH3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -SH3c * x * (4.f * zz - xx - yy);
            Y[14] = SH3e * z * (xx - yy);
            Y[15] = -SH3a * x * (xx - 3.f * yy);
        }
    }
}

// g += w_k * grad Y_k for every k (gradients of the polynomial forms above).
template <int DEG>
__device__ __forceinline__ void sh_basis_grad_acc(float x, float y, float z, const float* w, float& gx,
                                                  float& gy, float& gz) {
    if (DEG >= 1) {
        gy += -SH1 * w[1];
        gz += SH1 * w[2];
        gx += -SH1 * w[3];
    }
    if (DEG >= 2) {
        gx += SH2a * y * w[4];
        gy += SH2a * x * w[4];
        gy += -SH2a * z * w[5];
        gz += -SH2a * y * w[5];
        gx += -2.f * SH2b * x * w[6];
        gy += -2.f * SH2b * y * w[6];
        gz += 4.f * SH2b * z * w[6];
        gx += -SH2a * z * w[7];
        gz += -SH2a * x * w[7];
        gx += 2.f * SH2c * x * w[8];
        gy += -2.f * SH2c * y * w[8];
        if (DEG >= 3) {
            const float xx = x * x, yy = y * y, zz = z * z;
            gx += -6.f * SH3a * x * y * w[9];
            gy += -3.f * SH3a * (xx - yy) * w[9];
            gx += SH3b * y * z * w[10];
            gy += SH3b * x * z * w[10];
            gz += SH3b * x * y * w[10];
            gx += 2.f * SH3c * x * y * w[11];
            gy += -SH3c * (4.f * zz - xx - 3.f * yy) * w[11];
            gz += -8.f * SH3c * y * z * w[11];
            gx += -6.f * SH3d * x * z * w[12];
            gy += -6.f * SH3d * y * z * w[12];
            gz += SH3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
            gx += -SH3c * (4.f * zz - 3.f * xx - yy) * w[13];
            gy += 2.f * SH3c * x * y * w[13];
            gz += -8.f * SH3c * x * z * w[13];
            gx += 2.f * SH3e * x * z * w[14];
            gy += -2.f * SH3e * y * z * w[14];
            gz += SH3e * (xx - yy) * w[14];
            gx += -3.f * SH3a * (xx - yy) * w[15];
            gy += 6.f * SH3a * x * y * w[15];
        }
    }
}

// ---------------------------------------------------------------------------------------
// Gaussian geometry: world covariance Sigma = M M^T with M = R(q/|q|) diag(exp(s)).
// ---------------------------------------------------------------------------------------
struct Cov3 {
    float qn[4], qinv;   // normalised quaternion, 1/|q|
    float Rq[9];
    float s[3];
    float M[9];
    float S[6];          // Sigma: xx, xy, xz, yy, yz, zz
};

__device__ __forceinline__ void cov3_forward(const float* q, const float* ls, Cov3& c) {
    const float n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    c.qinv = rsqrtf(n2);
    const float w = q[0] * c.qinv, x = q[1] * c.qinv, y = q[2] * c.qinv, z = q[3] * c.qinv;
    c.qn[0] = w; c.qn[1] = x; c.qn[2] = y; c.qn[3] = z;
    c.Rq[0] = 1.f - 2.f * (y * y + z * z); c.Rq[1] = 2.f * (x * y - w * z); c.Rq[2] = 2.f * (x * z + w * y);
    c.Rq[3] = 2.f * (x * y + w * z); c.Rq[4] = 1.f - 2.f * (x * x + z * z); c.Rq[5] = 2.f * (y * z - w * x);
    c.Rq[6] = 2.f * (x * z - w * y); c.Rq[7] = 2.f * (y * z + w * x); c.Rq[8] = 1.f - 2.f * (x * x + y * y);
#pragma unroll
    for (int k = 0; k < 3; k++) c.s[k] = expf(ls[k]);
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int k = 0; k < 3; k++) c.M[r * 3 + k] = c.Rq[r * 3 + k] * c.s[k];
    const float* M = c.M;
    c.S[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    c.S[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    c.S[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    c.S[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    c.S[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    c.S[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
}

// Per-view projection of one Gaussian (everything the backward needs again).
struct ProjV {
    bool culled;
    float pc[3];
    float tx, ty;
    bool clx, cly;
    float J00, J02, J11, J12;   // J = [[J00, 0, J02], [0, J11, J12]]
    float T[6];                 // J W, 2x3 row-major
    float a, b, c;              // dilated 2-D covariance
    float det;
    float o;
    float u, v;
    int rx, ry;          // half-extents of the alpha >= alpha_min box (pixels)
};

__device__ __forceinline__ void project_view(const float* mu, const Cov3& cv, float logit, const View& V,
                                             const Opts& op, ProjV& P) {
    // Every field is computed (no early exit) so the backward, which recomputes this for
    // the pairs the forward kept, never reads an unset value.
    const float* W = V.R;
    // Camera-frame centre, each row as fma(R_k2, mu_z, fma(R_k1, mu_y, R_k0 mu_x)) + t_k with
    // every operation rounded once.  The depth's FP32 bits are the compositing order's sort
    // key, so its operation order is part of the definition of that order; the intrinsics
    // keep the compiler from contracting it any other way.
#pragma unroll
    for (int k = 0; k < 3; k++)
        P.pc[k] = __fadd_rn(__fmaf_rn(W[3 * k + 2], mu[2], __fmaf_rn(W[3 * k + 1], mu[1], __fmul_rn(W[3 * k], mu[0]))),
                            V.t[k]);
    const float x = P.pc[0], y = P.pc[1], z = P.pc[2];
    const bool front = z > op.near_z;
    const float iz = 1.0f / (front ? z : 1.0f);
    const float rx = x * iz, ry = y * iz;
    P.tx = fminf(V.limx, fmaxf(-V.limx, rx));
    P.ty = fminf(V.limy, fmaxf(-V.limy, ry));
    P.clx = (rx < -V.limx) || (rx > V.limx);
    P.cly = (ry < -V.limy) || (ry > V.limy);
    P.J00 = V.fx * iz;
    P.J02 = -V.fx * P.tx * iz;
    P.J11 = V.fy * iz;
    P.J12 = -V.fy * P.ty * iz;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        P.T[k] = P.J00 * W[k] + P.J02 * W[6 + k];
        P.T[3 + k] = P.J11 * W[3 + k] + P.J12 * W[6 + k];
    }
    // T Sigma (2x3) then (T Sigma) T^T
    const float* S = cv.S;
    float TS[6];
#pragma unroll
    for (int r = 0; r < 2; r++) {
        const float* t = &P.T[3 * r];
        TS[3 * r + 0] = t[0] * S[0] + t[1] * S[1] + t[2] * S[2];
        TS[3 * r + 1] = t[0] * S[1] + t[1] * S[3] + t[2] * S[4];
        TS[3 * r + 2] = t[0] * S[2] + t[1] * S[4] + t[2] * S[5];
    }
    P.a = TS[0] * P.T[0] + TS[1] * P.T[1] + TS[2] * P.T[2] + op.dilation;
    P.b = TS[0] * P.T[3] + TS[1] * P.T[4] + TS[2] * P.T[5];
    P.c = TS[3] * P.T[3] + TS[4] * P.T[4] + TS[5] * P.T[5] + op.dilation;
    P.det = P.a * P.c - P.b * P.b;
    P.o = 1.0f / (1.0f + expf(-logit));
    const bool opaque = P.o >= op.alpha_min;
    // alpha >= alpha_min only inside d^T Sigma'^-1 d <= tau, tau = 2 ln(o / alpha_min), whose
    // bounding box has half-extents sqrt(tau Sigma'_xx), sqrt(tau Sigma'_yy)
    const float tau = 2.0f * logf(fmaxf(P.o, op.alpha_min) / op.alpha_min);
    const bool ok = front && P.det > 0.f && opaque && tau > 0.f;
    P.rx = ok ? (int)ceilf(fminf(sqrtf(tau * P.a), 1e9f)) : 0;
    P.ry = ok ? (int)ceilf(fminf(sqrtf(tau * P.c), 1e9f)) : 0;
    P.u = V.fx * x * iz + V.cx;
    P.v = V.fy * y * iz + V.cy;
    P.culled = !(ok && P.rx > 0 && P.ry > 0);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace gs
