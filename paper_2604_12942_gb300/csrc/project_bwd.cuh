// a7 (and a8 fused): the projection backward's device code, shared by its standalone kernels
// (project.cu) and the persistent form of the step (render.cu).
// RMGS-SLAM §III-C ("standard differentiable Gaussian splatting"); the chain rule to the
// Gaussian parameters and to each view's SE(3) pose twist.
#pragma once

#include "gs_kernels.cuh"

namespace gs {

// Backward of the projection.  Screen-space sums per (view, Gaussian) come from the
// backward compositing kernel (see render.cu for their definition):
//   r0 = (sum h h_x, sum h h_y, sum h dx^2, sum h dx dy)
//   r1 = (sum h dy^2, dL/do, dL/dz, 0), r2 = (dL/dr, dL/dg, dL/db, 0)
// with h = dL/dalpha * o * G and e = dx h_x + dy h_y.  Since dalpha/de = ln2 o G and
// de/du = -2 h_x, de/dv = -2 h_y, de/dA = k dx^2, de/dB = 2 k dx dy, de/dC = k dy^2
// (k = -log2(e)/2, ln2 log2(e) = 1): dL/du = -2 ln2 r0.x, dL/dv = -2 ln2 r0.y,
// dL/dA = -r0.z / 2, dL/dB = -r0.w, dL/dC = -r1.x / 2.  Pose: xi = (rho, phi), T_cw <- Exp(xi) T_cw, so
// dp_c = rho + phi x p_c, dW = [phi]x W and the camera centre moves by -W^T rho.
// Geometry part of the projection backward for one (view, Gaussian) entry: from the entry's
// screen-space sums r0, r1 (see render.cu) to the mean through p_c, to the world covariance
// and to the view's twist.  The opacity sum r1.y and the colour sums pass through unchanged.
__device__ __forceinline__ void entry_geometry_bwd(const float (&mu)[3], const Cov3& cv, float logit, const View& V,
                                                   const Opts& op, const float4 r0, const float4 r1,
                                                   float (&g_mu)[3], float (&gS)[6], float (&tw)[6]) {
#pragma unroll
    for (int k = 0; k < 3; k++) g_mu[k] = 0.f;
#pragma unroll
    for (int k = 0; k < 6; k++) gS[k] = 0.f;
    ProjV P;
    project_view(mu, cv, logit, V, op, P);
    const float* W = V.R;
    // screen-space gradients
    const float gu = -2.f * kLn2 * r0.x, gv = -2.f * kLn2 * r0.y;
    const float gA = -0.5f * r0.z, gB = -r0.w, gC = -0.5f * r1.x;
    float g_pc[3] = {0.f, 0.f, r1.z};
    // conic = inverse(cov), cov = [[a, b], [b, c]]
    const float pa = P.a, pb = P.b, pc = P.c;
    const float id2 = 1.0f / (P.det * P.det);
    const float ga = (-pc * pc * gA + pb * pc * gB - pb * pb * gC) * id2;
    const float gb = (2.f * pb * pc * gA - (pa * pc + pb * pb) * gB + 2.f * pa * pb * gC) * id2;
    const float gc = (-pb * pb * gA + pa * pb * gB - pa * pa * gC) * id2;
    const float G00 = ga, G01 = 0.5f * gb, G11 = gc;
    // T Sigma
    const float* S = cv.S;
    float TS[6];
#pragma unroll
    for (int r = 0; r < 2; r++) {
        const float* t = &P.T[3 * r];
        TS[3 * r + 0] = t[0] * S[0] + t[1] * S[1] + t[2] * S[2];
        TS[3 * r + 1] = t[0] * S[1] + t[1] * S[3] + t[2] * S[4];
        TS[3 * r + 2] = t[0] * S[2] + t[1] * S[4] + t[2] * S[5];
    }
    // g_T = 2 G T Sigma
    float gT[6];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        gT[k] = 2.f * (G00 * TS[k] + G01 * TS[3 + k]);
        gT[3 + k] = 2.f * (G01 * TS[k] + G11 * TS[3 + k]);
    }
    // g_Sigma += T^T G T
    {
        float GT[6];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            GT[k] = G00 * P.T[k] + G01 * P.T[3 + k];
            GT[3 + k] = G01 * P.T[k] + G11 * P.T[3 + k];
        }
        gS[0] += P.T[0] * GT[0] + P.T[3] * GT[3];
        gS[1] += P.T[0] * GT[1] + P.T[3] * GT[4];
        gS[2] += P.T[0] * GT[2] + P.T[3] * GT[5];
        gS[3] += P.T[1] * GT[1] + P.T[4] * GT[4];
        gS[4] += P.T[1] * GT[2] + P.T[4] * GT[5];
        gS[5] += P.T[2] * GT[2] + P.T[5] * GT[5];
    }
    // T = J W : g_J = g_T W^T, g_W = J^T g_T
    const float gJ00 = gT[0] * W[0] + gT[1] * W[1] + gT[2] * W[2];
    const float gJ02 = gT[0] * W[6] + gT[1] * W[7] + gT[2] * W[8];
    const float gJ11 = gT[3] * W[3] + gT[4] * W[4] + gT[5] * W[5];
    const float gJ12 = gT[3] * W[6] + gT[4] * W[7] + gT[5] * W[8];
    float gW[9];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        gW[k] = P.J00 * gT[k];
        gW[3 + k] = P.J11 * gT[3 + k];
        gW[6 + k] = P.J02 * gT[k] + P.J12 * gT[3 + k];
    }
    const float x = P.pc[0], y = P.pc[1], z = P.pc[2];
    const float iz = 1.0f / z, iz2 = iz * iz;
    const float fx = V.fx, fy = V.fy;
    const float dtx_dx = P.clx ? 0.f : iz, dtx_dz = P.clx ? 0.f : -x * iz2;
    const float dty_dy = P.cly ? 0.f : iz, dty_dz = P.cly ? 0.f : -y * iz2;
    g_pc[2] += -gJ00 * fx * iz2 - gJ11 * fy * iz2;
    g_pc[2] += gJ02 * (fx * P.tx * iz2 - fx * iz * dtx_dz);
    g_pc[0] += gJ02 * (-fx * iz * dtx_dx);
    g_pc[2] += gJ12 * (fy * P.ty * iz2 - fy * iz * dty_dz);
    g_pc[1] += gJ12 * (-fy * iz * dty_dy);
    g_pc[0] += gu * fx * iz;
    g_pc[1] += gv * fy * iz;
    g_pc[2] += -(gu * fx * x + gv * fy * y) * iz2;
#pragma unroll
    for (int k = 0; k < 3; k++) g_mu[k] += W[k] * g_pc[0] + W[3 + k] * g_pc[1] + W[6 + k] * g_pc[2];
    // pose: rho <- g_pc, phi <- p_c x g_pc + vee(g_W W^T)
    tw[0] = g_pc[0]; tw[1] = g_pc[1]; tw[2] = g_pc[2];
    tw[3] = y * g_pc[2] - z * g_pc[1];
    tw[4] = z * g_pc[0] - x * g_pc[2];
    tw[5] = x * g_pc[1] - y * g_pc[0];
    {
        // A = g_W W^T; need A21 - A12, A02 - A20, A10 - A01
        auto Arc = [&](int r, int c) { return gW[3 * r] * W[3 * c] + gW[3 * r + 1] * W[3 * c + 1] + gW[3 * r + 2] * W[3 * c + 2]; };
        tw[3] += Arc(2, 1) - Arc(1, 2);
        tw[4] += Arc(0, 2) - Arc(2, 0);
        tw[5] += Arc(1, 0) - Arc(0, 1);
    }
}

// a7, entry part: one thread per visible (view, Gaussian) entry, entries in (view, Gaussian)
// order (so a warp mostly reads consecutive rows of one view).  Writes the entry's geometry
// gradients to its geo record -- (g_mu, gS_xx), (gS_xy, gS_xz, gS_yy, gS_yz), (gS_zz, 0, 0, 0)
// -- and adds its geometric twist to the view's (sums over the lanes of one view, then per CTA).
// The screen-space sums are only read, so the backward can be repeated on them.
constexpr int kEntryThreads = 256;

// The entry part over the block's share of the entries (block `blk` of `nblk`, kEntryThreads
// threads); s_tw: the block's GS_MAX_VIEWS * 6 floats of shared memory.
__device__ __forceinline__ void project_bwd_entry_part(const ProjectBwdArgs& a, int64_t blk, int64_t nblk,
                                                       float* s_tw) {
    // a failed earlier stage (capacity, non-finite input) leaves the screen-space sums undefined
    if (a.counters->status != 0) return;
    for (int t = threadIdx.x; t < a.n_views * 6; t += kEntryThreads) s_tw[t] = 0.f;
    __syncthreads();
    const int64_t E = (int64_t)a.counters->n_entries;
    const int64_t n = a.n;
    const int lane = threadIdx.x & 31;
    const Opts op = a.op;
    for (int64_t base = blk * kEntryThreads; base < E; base += nblk * kEntryThreads) {
        const int64_t e = base + threadIdx.x;
        const bool valid = e < E;
        int v = -1;
        float tw[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (valid) {
            const uint32_t idx = a.entries[e];
            v = (int)(idx / (uint64_t)n);
            const int64_t i = (int64_t)idx - (int64_t)v * n;
            float mu[3], ls[3], q[4];
#pragma unroll
            for (int k = 0; k < 3; k++) { mu[k] = __ldg(a.means + k * n + i); ls[k] = __ldg(a.log_scales + k * n + i); }
#pragma unroll
            for (int k = 0; k < 4; k++) q[k] = __ldg(a.quats + k * n + i);
            const float logit = __ldg(a.logits + i);
            const float4* rec = a.grad2d + 3 * (size_t)idx;
            const float4 r0 = rec[0], r1 = rec[1];
            Cov3 cv;
            cov3_forward(q, ls, cv);
            float g_mu[3], gS[6];
            entry_geometry_bwd(mu, cv, logit, a.views[v], op, r0, r1, g_mu, gS, tw);
            float4* geo = a.geo2d + 3 * (size_t)idx;
            geo[0] = make_float4(g_mu[0], g_mu[1], g_mu[2], gS[0]);
            geo[1] = make_float4(gS[1], gS[2], gS[3], gS[4]);
            geo[2] = make_float4(gS[5], 0.f, 0.f, 0.f);
        }
        if (a.grad_twist) {
            // lanes with the same view: one warp sum per view present in the warp
            uint32_t pending = __ballot_sync(0xffffffffu, valid);
            while (pending) {
                const int leader = __ffs(pending) - 1;
                const int vl = __shfl_sync(0xffffffffu, v, leader);
                const uint32_t grp = __ballot_sync(0xffffffffu, valid && v == vl);
#pragma unroll
                for (int k = 0; k < 6; k++) {
                    const float x = warp_sum(((grp >> lane) & 1u) ? tw[k] : 0.f);
                    if (lane == leader) atomicAdd(&s_tw[vl * 6 + k], x);
                }
                pending &= ~grp;
            }
        }
    }
    if (a.grad_twist) {
        __syncthreads();
        for (int t = threadIdx.x; t < a.n_views * 6; t += kEntryThreads)
            if (s_tw[t] != 0.f) atomicAdd(&a.grad_twist[t], s_tw[t]);
    }
}

// ----------------------------------------------------------------------------------------
// The row part in two kernels, each with fewer live registers than the combined row part (so
// more resident warps for their memory latency):
//   SH part        one colour channel at a time: the channel's K coefficients and their
//                  gradient sums in registers (no shared memory), the row's views walked once
//                  per channel; the SH planes' gradient (or, fused, their Adam step), the
//                  view-direction gradient of the mean into dirgrad [3][n] and the
//                  view-direction twist (rho) of every view
//   geometry part  the entry part's geometry gradients and the opacity sums over the row's
//                  views, plus dirgrad; the covariance -> scale and rotation chain; the 11
//                  geometry planes' gradient (or, fused, their Adam step)
// ----------------------------------------------------------------------------------------
// Fused: each thread's Adam moments of a channel's K planes are copied asynchronously (cp.async,
// 4 bytes each, no registers held while in flight) into s_mv [2 buffers][m, v][K][T] of shared
// memory while the thread walks the previous channel's views, so the moment loads of a row are
// in flight together with its other work; a thread reads only the slots it copied itself.
template <int DEG, int T>
constexpr int sh_mv_floats() { return 2 * 2 * (DEG + 1) * (DEG + 1) * T; }

// s_cam: GS_MAX_VIEWS * 12 floats of shared memory, each view's camera centre and rotation
// (cw, R) copied there when the block starts, so the walk over a row's views reads them without
// a trip to L2 (the streamed planes keep little of the view table in L1).
template <int DEG, bool FUSED_ADAM, int T>
__device__ __forceinline__ void project_bwd_sh_rows(const ProjectBwdArgs& a, int64_t blk, float* s_tw, float* s_mv,
                                                    float* s_cam) {
    if (a.counters->status != 0) return;   // no gradient (and no Adam update) after a failed stage
    constexpr int K = (DEG + 1) * (DEG + 1);
    for (int t = threadIdx.x; t < a.n_views * 6; t += T) s_tw[t] = 0.f;
    for (int t = threadIdx.x; t < a.n_views * 12; t += T) {
        const View& V = a.views[t / 12];
        const int f = t % 12;
        s_cam[t] = f < 3 ? V.cw[f] : V.R[f - 3];
    }
    __syncthreads();
    const int64_t n = a.n;
    const int64_t i = blk * T + threadIdx.x;
    const bool live = i < n && a.visible[i] != 0;
    const int64_t ii = live ? i : 0;
    uint64_t vmask = 0;
    if (live) {
        // the row's bit of each view's visibility word (one word for the 32 rows of a warp)
        const int64_t nw = (n + 31) >> 5;
#pragma unroll 8
        for (int v = 0; v < a.n_views; v++)
            vmask |= (uint64_t)((__ldg(a.vis_bits + v * nw + (ii >> 5)) >> (ii & 31)) & 1u) << v;
    }
    if (__all_sync(0xffffffffu, !live) && a.grad_twist == nullptr) return;
    float mu[3];
#pragma unroll
    for (int k = 0; k < 3; k++) mu[k] = live ? __ldg(a.means + k * n + ii) : 0.f;
    const int lane = threadIdx.x & 31;
    const bool upd = live && (!FUSED_ADAM || !a.update_mask || a.update_mask[i]);
    // moments of channel c into buffer c & 1 (an empty commit group when there is nothing to copy)
    auto prefetch = [&](int c) {
        if (FUSED_ADAM && upd) {
            float* dst = s_mv + (c & 1) * 2 * K * T + threadIdx.x;
#pragma unroll
            for (int k = 0; k < K; k++) {
                cp_async4(dst + k * T, a.m[4] + (int64_t)(k * 3 + c) * n + i);
                cp_async4(dst + (K + k) * T, a.v[4] + (int64_t)(k * 3 + c) * n + i);
            }
        }
        cp_async_commit();
    };
    if (FUSED_ADAM) prefetch(0);
    float gdir[3] = {0.f, 0.f, 0.f};
#pragma unroll 1
    for (int c = 0; c < 3; c++) {
        if (FUSED_ADAM) {
            if (c < 2) prefetch(c + 1);
            else cp_async_commit();
        }
        float shc[K], gc[K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            shc[k] = live ? __ldg(a.sh + (int64_t)(k * 3 + c) * n + ii) : 0.f;
            gc[k] = 0.f;
        }
        // the walk over the row's views loads the next view's dL/d colour c while it evaluates
        // the current one
        auto colour_grad = [&](int v) {
            return __ldg(reinterpret_cast<const float*>(a.grad2d + 3 * ((int64_t)v * n + ii) + 2) + c);
        };
        uint64_t todo = vmask;
        int v_nx = todo != 0 ? __ffsll((long long)todo) - 1 : -1;
        float g_nx = v_nx >= 0 ? colour_grad(v_nx) : 0.f;
        while (__any_sync(0xffffffffu, v_nx >= 0)) {
            const bool act = v_nx >= 0;
            const int v = act ? v_nx : 0;
            const float g = g_nx;   // dL/d colour c in view v
            todo &= todo - 1;
            v_nx = todo != 0 ? __ffsll((long long)todo) - 1 : -1;
            if (v_nx >= 0) g_nx = colour_grad(v_nx);
            float tw[3] = {0.f, 0.f, 0.f};
            if (act) {
                const float* cam = s_cam + v * 12;   // cw, then R row-major
                // rgb_c = max(0, sum_k sh_kc Y_k(dir) + 0.5), dir = (mu - cw)/|mu - cw|
                const float d[3] = {mu[0] - cam[0], mu[1] - cam[1], mu[2] - cam[2]};
                const float rn = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                const float dir[3] = {d[0] * rn, d[1] * rn, d[2] * rn};
                float Y[16];
                sh_basis<DEG>(dir[0], dir[1], dir[2], Y);
                float s = 0.5f;
#pragma unroll
                for (int k = 0; k < K; k++) s += shc[k] * Y[k];
                if (!(s < 0.f)) {   // a clamped channel has no gradient
#pragma unroll
                    for (int k = 0; k < K; k++) gc[k] += g * Y[k];
                    if (DEG > 0) {
                        float gd[3] = {0.f, 0.f, 0.f};
                        sh_basis_grad_acc<DEG>(dir[0], dir[1], dir[2], shc, gd[0], gd[1], gd[2]);
                        const float dd = gd[0] * dir[0] + gd[1] * dir[1] + gd[2] * dir[2];
#pragma unroll
                        for (int k = 0; k < 3; k++) gd[k] = g * (gd[k] - dir[k] * dd) * rn;
#pragma unroll
                        for (int k = 0; k < 3; k++) gdir[k] += gd[k];
                        const float* W = cam + 3;
#pragma unroll
                        for (int r = 0; r < 3; r++) tw[r] = W[3 * r] * gd[0] + W[3 * r + 1] * gd[1] + W[3 * r + 2] * gd[2];
                    }
                }
            }
            if (DEG > 0 && a.grad_twist) {
                // the view-direction term moves only rho: one warp sum per view among the lanes
                uint32_t pending = __ballot_sync(0xffffffffu, act);
                while (pending) {
                    const int leader = __ffs(pending) - 1;
                    const int vl = __shfl_sync(0xffffffffu, v, leader);
                    const uint32_t grp = __ballot_sync(0xffffffffu, act && v == vl);
#pragma unroll
                    for (int k = 0; k < 3; k++) {
                        const float x = warp_sum(((grp >> lane) & 1u) ? tw[k] : 0.f);
                        if (lane == leader) atomicAdd(&s_tw[vl * 6 + k], x);
                    }
                    pending &= ~grp;
                }
            }
        }
        if (upd) {
            if constexpr (FUSED_ADAM) {
                // a8 on the channel's planes: the gradient goes straight into Adam
                const float bc1 = __frcp_rn(a.step_dev ? a.step_dev->adam_bc1 : a.bc1);
                const float bc2 = __frcp_rn(a.step_dev ? a.step_dev->adam_bc2 : a.bc2);
                cp_async_wait_prior();   // this channel's moments have landed (the next may be in flight)
                const float* mv = s_mv + (c & 1) * 2 * K * T + threadIdx.x;
#pragma unroll
                for (int k = 0; k < K; k++) {
                    float p = shc[k], mm = mv[k * T], vv = mv[(K + k) * T];
                    adam_update(p, gc[k], mm, vv, k == 0 ? a.lr[4] : a.lr[5], a.b1, a.b2, a.eps, bc1, bc2);
                    a.p_sh[(int64_t)(k * 3 + c) * n + i] = p;
                    a.m[4][(int64_t)(k * 3 + c) * n + i] = mm;
                    a.v[4][(int64_t)(k * 3 + c) * n + i] = vv;
                }
            } else {
#pragma unroll
                for (int k = 0; k < K; k++) {
                    float* gp = a.g_sh + (int64_t)(k * 3 + c) * n + i;
                    *gp = __fadd_rn(*gp, gc[k]);
                }
            }
        }
    }
    if (FUSED_ADAM) cp_async_wait_all();
    if (live && DEG > 0) {
#pragma unroll
        for (int k = 0; k < 3; k++) a.dirgrad[k * n + i] = gdir[k];
    }
    if (a.grad_twist) {
        __syncthreads();
        for (int t = threadIdx.x; t < a.n_views * 6; t += T)
            if (s_tw[t] != 0.f) atomicAdd(&a.grad_twist[t], s_tw[t]);
    }
}

// Adam on NP consecutive planes of one parameter group at row i (planes k n + i), the moments
// read from shared memory (sm[k * stride], sv[k * stride]) and written back to global memory.
template <int NP>
__device__ __forceinline__ void adam_planes(float* P, float* M, float* V, int64_t n, int64_t i, const float* p0,
                                            const float* g, const float* sm, const float* sv, int stride, float lr,
                                            const ProjectBwdArgs& a, float bc1, float bc2) {
    float mm[NP], vv[NP];
#pragma unroll
    for (int k = 0; k < NP; k++) { mm[k] = sm[k * stride]; vv[k] = sv[k * stride]; }
#pragma unroll
    for (int k = 0; k < NP; k++) {
        float p = p0[k];
        adam_update(p, g[k], mm[k], vv[k], lr, a.b1, a.b2, a.eps, bc1, bc2);
        P[k * n + i] = p;
        M[k * n + i] = mm[k];
        V[k * n + i] = vv[k];
    }
}

// Fused: the row's 22 Adam moments of the geometry planes are copied asynchronously into
// s_mv [2][11][T] of shared memory when the thread starts, so they are in flight during the
// walk over its views and the covariance chain; a thread reads only its own slots.
template <int T>
constexpr int geo_mv_floats() { return 2 * 11 * T; }

template <int DEG, bool FUSED_ADAM, int T>
__device__ __forceinline__ void project_bwd_geo_rows(const ProjectBwdArgs& a, int64_t blk, float* s_mv) {
    if (a.counters->status != 0) return;
    const int64_t n = a.n;
    const int64_t i = blk * T + threadIdx.x;
    const bool live = i < n && a.visible[i] != 0;
    if (!live) return;   // no block-wide synchronisation below
    const bool upd = !FUSED_ADAM || !a.update_mask || a.update_mask[i];
    if (FUSED_ADAM && upd) {
        float* dst = s_mv + threadIdx.x;
        const float* const mg[2][4] = {{a.m[0], a.m[1], a.m[2], a.m[3]}, {a.v[0], a.v[1], a.v[2], a.v[3]}};
#pragma unroll
        for (int h = 0; h < 2; h++) {
#pragma unroll
            for (int k = 0; k < 11; k++) {
                const float* src = k < 3 ? mg[h][0] + k * n : k < 6 ? mg[h][1] + (k - 3) * n
                                 : k < 10 ? mg[h][2] + (k - 6) * n : mg[h][3];
                cp_async4(dst + (h * 11 + k) * T, src + i);
            }
        }
        cp_async_commit();
    }
    uint64_t vmask = 0;
    const int64_t nw = (n + 31) >> 5;
#pragma unroll 8
    for (int v = 0; v < a.n_views; v++)
        vmask |= (uint64_t)((__ldg(a.vis_bits + v * nw + (i >> 5)) >> (i & 31)) & 1u) << v;
    float mu[3], ls[3], q[4];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        mu[k] = __ldg(a.means + k * n + i);
        ls[k] = __ldg(a.log_scales + k * n + i);
    }
#pragma unroll
    for (int k = 0; k < 4; k++) q[k] = __ldg(a.quats + k * n + i);
    const float logit = __ldg(a.logits + i);
    float g_mu[3] = {0.f, 0.f, 0.f};
    if (DEG > 0) {
#pragma unroll
        for (int k = 0; k < 3; k++) g_mu[k] = a.dirgrad[k * n + i];
    }
    float gS[6] = {0, 0, 0, 0, 0, 0};   // dL/dSigma as a symmetric matrix: xx xy xz yy yz zz
    float g_o = 0.f;
    for (uint64_t todo = vmask; todo; todo &= todo - 1) {
        const int v = __ffsll((long long)todo) - 1;
        const int64_t idx = (int64_t)v * n + i;
        const float4* geo = a.geo2d + 3 * idx;
        const float4 q0 = geo[0], q1 = geo[1], q2 = geo[2];
        g_o += reinterpret_cast<const float*>(a.grad2d + 3 * idx + 1)[1];
        g_mu[0] += q0.x; g_mu[1] += q0.y; g_mu[2] += q0.z;
        gS[0] += q0.w; gS[1] += q1.x; gS[2] += q1.y; gS[3] += q1.z; gS[4] += q1.w; gS[5] += q2.x;
    }
    Cov3 cv;
    cov3_forward(q, ls, cv);
    // Sigma = M M^T -> g_M = 2 gSigma M (symmetric gSigma); M = Rq diag(s)
    const float Gs[9] = {gS[0], gS[1], gS[2], gS[1], gS[3], gS[4], gS[2], gS[4], gS[5]};
    float gM[9];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++)
            gM[3 * r + c] = 2.f * (Gs[3 * r] * cv.M[c] + Gs[3 * r + 1] * cv.M[3 + c] + Gs[3 * r + 2] * cv.M[6 + c]);
    float gls[3], gR[9];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        gls[c] = (cv.Rq[c] * gM[c] + cv.Rq[3 + c] * gM[3 + c] + cv.Rq[6 + c] * gM[6 + c]) * cv.s[c];
#pragma unroll
        for (int r = 0; r < 3; r++) gR[3 * r + c] = gM[3 * r + c] * cv.s[c];
    }
    const float w = cv.qn[0], x = cv.qn[1], y = cv.qn[2], z = cv.qn[3];
    float gq[4];
    gq[0] = 2.f * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
    gq[1] = 2.f * (y * gR[1] + z * gR[2] + y * gR[3] - 2.f * x * gR[4] - w * gR[5] + z * gR[6] + w * gR[7] - 2.f * x * gR[8]);
    gq[2] = 2.f * (-2.f * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] - w * gR[6] + z * gR[7] - 2.f * y * gR[8]);
    gq[3] = 2.f * (-2.f * z * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] - 2.f * z * gR[4] + y * gR[5] + x * gR[6] + y * gR[7]);
    const float dq = gq[0] * w + gq[1] * x + gq[2] * y + gq[3] * z;
    const float qn[4] = {w, x, y, z};
    const float o = 1.0f / (1.0f + expf(-logit));
    float g[11];
#pragma unroll
    for (int k = 0; k < 3; k++) { g[k] = g_mu[k]; g[3 + k] = gls[k]; }
#pragma unroll
    for (int k = 0; k < 4; k++) g[6 + k] = (gq[k] - qn[k] * dq) * cv.qinv;
    g[10] = g_o * o * (1.f - o);
    // element i of geometry plane k (means 0-2, log-scales 3-5, quats 6-9, logit 10)
    auto at = [&](float* const* grp, int k) -> float& {
        return k < 3 ? grp[0][k * n + i] : k < 6 ? grp[1][(k - 3) * n + i] : k < 10 ? grp[2][(k - 6) * n + i]
                                                                                     : grp[3][i];
    };
    if constexpr (FUSED_ADAM) {
        if (!upd) return;
        const float bc1 = __frcp_rn(a.step_dev ? a.step_dev->adam_bc1 : a.bc1);   // inverse bias corrections
        const float bc2 = __frcp_rn(a.step_dev ? a.step_dev->adam_bc2 : a.bc2);
        cp_async_wait_all();
        const float* mv = s_mv + threadIdx.x;
        // by parameter group (means, log-scales, quaternion, logit)
        adam_planes<3>(a.p_means, a.m[0], a.v[0], n, i, mu, g, mv, mv + 11 * T, T, a.lr[0], a, bc1, bc2);
        adam_planes<3>(a.p_log_scales, a.m[1], a.v[1], n, i, ls, g + 3, mv + 3 * T, mv + 14 * T, T, a.lr[1], a, bc1,
                       bc2);
        adam_planes<4>(a.p_quats, a.m[2], a.v[2], n, i, q, g + 6, mv + 6 * T, mv + 17 * T, T, a.lr[2], a, bc1, bc2);
        adam_planes<1>(a.p_logits, a.m[3], a.v[3], n, i, &logit, g + 10, mv + 10 * T, mv + 21 * T, T, a.lr[3], a, bc1,
                       bc2);
    } else {
        // (explicit adds: the accumulation is never contracted into the last product of the
        // gradient, which keeps it equal to the value the fused variant feeds to Adam)
        float* const gg[4] = {a.g_means, a.g_log_scales, a.g_quats, a.g_logits};
#pragma unroll
        for (int k = 0; k < 11; k++) at(gg, k) = __fadd_rn(at(gg, k), g[k]);
    }
}

}  // namespace gs
