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

// a7, row part, and a8 when fused.
// One thread per Gaussian, kProjBwdThreads per block.  The 3K SH coefficients and their
// gradient sums live in shared memory (one column per thread) rather than registers, which
// keeps the kernel within 128 registers at SH degree 3.
constexpr int kProjBwdThreads = 128;   // row block of the standalone kernel

// FUSED_ADAM: apply the masked Adam step of a8 to the row with its finished gradient instead
// of adding the gradient to the gradient planes (same arithmetic as adam_kernel).
// Row block `blk` (rows blk * T .. blk * T + T - 1, T threads): s_tw is the block's
// GS_MAX_VIEWS * 6 floats, s_dyn its 2 * 3K * T floats of shared memory.
template <int DEG, bool FUSED_ADAM, int T>
__device__ __forceinline__ void project_bwd_rows(const ProjectBwdArgs& a, int64_t blk, float* s_tw, float* s_dyn) {
    if (a.counters->status != 0) return;   // no gradient (and no Adam update) after a failed stage
    constexpr int K = (DEG + 1) * (DEG + 1);
    constexpr int kProjBwdThreads = T;   // the row-block size within this function
    // dynamic shared memory: SH gradient sums [3K][threads], then SH coefficients [3K][threads]
    for (int t = threadIdx.x; t < a.n_views * 6; t += T) s_tw[t] = 0.f;
    float* g_sh = s_dyn + threadIdx.x;                           // g_sh[k * kProjBwdThreads]
    float* sh = s_dyn + 3 * K * kProjBwdThreads + threadIdx.x;   // sh[k * kProjBwdThreads]
#pragma unroll
    for (int k = 0; k < 3 * K; k++) g_sh[k * kProjBwdThreads] = 0.f;
    __syncthreads();
    const int64_t n = a.n;
    const int64_t i = blk * T + threadIdx.x;
    // Rows that cover no tile of any view have no gradient: they read and write nothing.
    const bool live = i < n && a.visible[i] != 0;
    const int64_t ii = live ? i : 0;
    // views whose tiles the row covers, loaded together
    uint64_t vmask = 0;
    if (live) {
#pragma unroll 8
        for (int v = 0; v < a.n_views; v++)
            if (__ldg(a.touched + (int64_t)v * n + ii) != 0u) vmask |= 1ull << v;
    }
    if (__all_sync(0xffffffffu, !live)) {
        if (a.grad_twist == nullptr) return;
    }
    float mu[3], ls[3], q[4];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        mu[k] = live ? __ldg(a.means + k * n + ii) : 0.f;
        ls[k] = live ? __ldg(a.log_scales + k * n + ii) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < 4; k++) q[k] = live ? __ldg(a.quats + k * n + ii) : (k == 0 ? 1.f : 0.f);
    const float logit = live ? __ldg(a.logits + ii) : 0.f;
#pragma unroll
    for (int k = 0; k < 3 * K; k++) sh[k * kProjBwdThreads] = live ? __ldg(a.sh + k * n + ii) : 0.f;
    Cov3 cv;
    cov3_forward(q, ls, cv);
    float g_mu[3] = {0, 0, 0};
    float gS[6] = {0, 0, 0, 0, 0, 0};   // dL/dSigma as a symmetric matrix: xx xy xz yy yz zz
    float g_o = 0.f;
    const int lane = threadIdx.x & 31;
    // Each lane walks its own views in increasing order, so the warp iterates as often as its
    // busiest Gaussian has views, not once per view any of its Gaussians has.
    uint64_t todo = vmask;
    while (__any_sync(0xffffffffu, todo != 0)) {
        const bool act = todo != 0;
        const int v = act ? __ffsll((long long)todo) - 1 : 0;
        todo &= todo - 1;
        const View& V = a.views[v];
        const int64_t idx = (int64_t)v * n + ii;
        float tw[6] = {0, 0, 0, 0, 0, 0};
        if (act) {
            // geometry gradients of the entry (entry part), opacity and colour sums
            const float4* geo = a.geo2d + 3 * idx;
            const float4 q0 = geo[0], q1 = geo[1], q2 = geo[2];
            const float4* gr = a.grad2d + 3 * idx;
            const float o_sum = reinterpret_cast<const float*>(gr + 1)[1];
            const float4 r2 = gr[2];
            g_mu[0] += q0.x; g_mu[1] += q0.y; g_mu[2] += q0.z;
            gS[0] += q0.w; gS[1] += q1.x; gS[2] += q1.y; gS[3] += q1.z; gS[4] += q1.w; gS[5] += q2.x;
            g_o += o_sum;
            const float* W = V.R;
            // SH colour: rgb_c = max(0, sum_k sh_kc Y_k(dir) + 0.5), dir = (mu - cw)/|mu - cw|
            float d[3] = {mu[0] - V.cw[0], mu[1] - V.cw[1], mu[2] - V.cw[2]};
            const float rn = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            const float dir[3] = {d[0] * rn, d[1] * rn, d[2] * rn};
            float Y[16];
            sh_basis<DEG>(dir[0], dir[1], dir[2], Y);
            const float grgb[3] = {r2.x, r2.y, r2.z};
            float wk[16];
#pragma unroll
            for (int k = 0; k < K; k++) wk[k] = 0.f;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                float s = 0.5f;
#pragma unroll
                for (int k = 0; k < K; k++) s += sh[(k * 3 + c) * kProjBwdThreads] * Y[k];
                if (s < 0.f) continue;   // clamped channel: no gradient
#pragma unroll
                for (int k = 0; k < K; k++) {
                    g_sh[(k * 3 + c) * kProjBwdThreads] += grgb[c] * Y[k];
                    wk[k] += grgb[c] * sh[(k * 3 + c) * kProjBwdThreads];
                }
            }
            if (DEG > 0) {
                float gd[3] = {0.f, 0.f, 0.f};
                sh_basis_grad_acc<DEG>(dir[0], dir[1], dir[2], wk, gd[0], gd[1], gd[2]);
                const float dd = gd[0] * dir[0] + gd[1] * dir[1] + gd[2] * dir[2];
#pragma unroll
                for (int k = 0; k < 3; k++) gd[k] = (gd[k] - dir[k] * dd) * rn;
#pragma unroll
                for (int k = 0; k < 3; k++) g_mu[k] += gd[k];
#pragma unroll
                for (int r = 0; r < 3; r++) tw[r] += W[3 * r] * gd[0] + W[3 * r + 1] * gd[1] + W[3 * r + 2] * gd[2];
            }
        }
        if (DEG > 0 && a.grad_twist) {
            // the view-direction term moves only rho (the geometric twist came from the entry
            // part): one warp sum per view present among the active lanes
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
    if (live) {
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
        if constexpr (FUSED_ADAM) {
            // a8 on this row: the gradient goes straight into Adam (never stored)
            if (!a.update_mask || a.update_mask[i]) {
                const float bc1 = __frcp_rn(a.step_dev ? a.step_dev->adam_bc1 : a.bc1);   // inverse bias corrections
                const float bc2 = __frcp_rn(a.step_dev ? a.step_dev->adam_bc2 : a.bc2);
                // Moments are loaded a group of planes at a time, all loads of a group before
                // its stores, so that a row waits for a few memory round trips, not 11 + 3K.
                {
                    float p[11], g[11], mm[11], vv[11];
                    // element i of geometry plane k (means 0-2, log-scales 3-5, quats 6-9, logit 10)
                    auto at = [&](float* const* grp, int k) -> float& {
                        return k < 3 ? grp[0][k * n + i] : k < 6 ? grp[1][(k - 3) * n + i]
                             : k < 10 ? grp[2][(k - 6) * n + i] : grp[3][i];
                    };
                    float* const pg[4] = {a.p_means, a.p_log_scales, a.p_quats, a.p_logits};
#pragma unroll
                    for (int k = 0; k < 11; k++) { mm[k] = at(a.m, k); vv[k] = at(a.v, k); }
#pragma unroll
                    for (int k = 0; k < 3; k++) { p[k] = mu[k]; g[k] = g_mu[k]; p[3 + k] = ls[k]; g[3 + k] = gls[k]; }
#pragma unroll
                    for (int k = 0; k < 4; k++) { p[6 + k] = q[k]; g[6 + k] = (gq[k] - qn[k] * dq) * cv.qinv; }
                    p[10] = logit;
                    g[10] = g_o * o * (1.f - o);
#pragma unroll
                    for (int k = 0; k < 11; k++) {
                        const float lr = k < 3 ? a.lr[0] : k < 6 ? a.lr[1] : k < 10 ? a.lr[2] : a.lr[3];
                        adam_update(p[k], g[k], mm[k], vv[k], lr, a.b1, a.b2, a.eps, bc1, bc2);
                        at(pg, k) = p[k];
                        at(a.m, k) = mm[k];
                        at(a.v, k) = vv[k];
                    }
                }
                constexpr int GS = 3 * K < 16 ? 3 * K : 16;
                // (the group loop stays rolled: an unrolled tail of 3K planes would crowd the
                // instruction cache of this already long kernel)
#pragma unroll 1
                for (int k0 = 0; k0 < 3 * K; k0 += GS) {
                    float mm[GS], vv[GS];
#pragma unroll
                    for (int k = 0; k < GS; k++) {
                        mm[k] = a.m[4][(k0 + k) * n + i];
                        vv[k] = a.v[4][(k0 + k) * n + i];
                    }
#pragma unroll
                    for (int k = 0; k < GS; k++) {
                        float p = sh[(k0 + k) * kProjBwdThreads];
                        adam_update(p, g_sh[(k0 + k) * kProjBwdThreads], mm[k], vv[k], k0 + k < 3 ? a.lr[4] : a.lr[5],
                                    a.b1, a.b2, a.eps, bc1, bc2);
                        a.p_sh[(k0 + k) * n + i] = p;
                        a.m[4][(k0 + k) * n + i] = mm[k];
                        a.v[4][(k0 + k) * n + i] = vv[k];
                    }
                }
            }
        } else {
            // (explicit adds: the accumulation is never contracted into the last product of
            // the gradient, which keeps it equal to the value the fused variant feeds to Adam)
#pragma unroll
            for (int k = 0; k < 3; k++) a.g_means[k * n + i] = __fadd_rn(a.g_means[k * n + i], g_mu[k]);
#pragma unroll
            for (int k = 0; k < 3; k++) a.g_log_scales[k * n + i] = __fadd_rn(a.g_log_scales[k * n + i], gls[k]);
#pragma unroll
            for (int k = 0; k < 4; k++)
                a.g_quats[k * n + i] = __fadd_rn(a.g_quats[k * n + i], (gq[k] - qn[k] * dq) * cv.qinv);
            a.g_logits[i] = __fadd_rn(a.g_logits[i], g_o * o * (1.f - o));
#pragma unroll
            for (int k = 0; k < 3 * K; k++) a.g_sh[k * n + i] = __fadd_rn(a.g_sh[k * n + i], g_sh[k * kProjBwdThreads]);
        }
    }
    if (a.grad_twist) {
        __syncthreads();
        for (int t = threadIdx.x; t < a.n_views * 6; t += T)
            if (s_tw[t] != 0.f) atomicAdd(&a.grad_twist[t], s_tw[t]);
    }
}

}  // namespace gs
