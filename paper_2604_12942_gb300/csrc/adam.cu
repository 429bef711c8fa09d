// a8: fused masked Adam over the parameter planes, zeroing the gradients it consumed.
// RMGS-SLAM §III-C: visible and unfrozen Gaussians are refined by a sparse gradient-based
// optimiser (only Gaussians of the most recent segments are updated).
#include "gs_kernels.cuh"

namespace gs {

// One row of one plane: update p, m, v if `upd`, consume (zero) the gradient if `vis`.
__device__ __forceinline__ void adam_one(float& p, float& g, float& m, float& v, bool upd, bool vis, float lr,
                                         const AdamArgs& a, float bc1, float bc2) {
    if (upd) adam_update(p, g, m, v, lr, a.b1, a.b2, a.eps, bc1, bc2);
    if (vis) g = 0.f;
}

// grid: (blocks over n in steps of 4*256, total planes).  Plane k of the packed layout
// (means 3, log-scales 3, quats 4, opacity 1, SH 3K) maps to group pointer and row.
__global__ void __launch_bounds__(256) adam_kernel(AdamArgs a) {
    int k = blockIdx.y;
    int grp = 0;
    while (k >= a.planes_of[grp]) { k -= a.planes_of[grp]; grp++; }
    const int gplane = blockIdx.y;
    const int lr_idx = gplane < 3 ? 0 : gplane < 6 ? 1 : gplane < 10 ? 2 : gplane < 11 ? 3 : gplane < 14 ? 4 : 5;
    const float lr = a.lr[lr_idx];
    const int64_t n = a.n;
    float* P = a.p[grp] + (int64_t)k * n;
    float* G = a.g[grp] + (int64_t)k * n;
    float* M = a.m[grp] + (int64_t)k * n;
    float* V = a.v[grp] + (int64_t)k * n;
    const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (i0 >= n) return;
    const float bc1 = __frcp_rn(a.step_dev ? a.step_dev->adam_bc1 : a.bc1);   // inverse bias corrections
    const float bc2 = __frcp_rn(a.step_dev ? a.step_dev->adam_bc2 : a.bc2);
    bool upd[4], vis[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int64_t i = i0 + q;
        vis[q] = i < n && (!a.visible || a.visible[i]);
        upd[q] = vis[q] && (!a.update_mask || a.update_mask[i]);
    }
    // Rows outside `visible` received no gradient this step: nothing to read or write.
    if (!(vis[0] | vis[1] | vis[2] | vis[3])) return;
    const bool any_upd = upd[0] | upd[1] | upd[2] | upd[3];
    const bool vec = ((n & 3) == 0) && (((uintptr_t)P | (uintptr_t)G | (uintptr_t)M | (uintptr_t)V) & 15) == 0;
    if (vec) {
        if (!any_upd) {   // visible but frozen: only consume the gradient
            if (vis[0] & vis[1] & vis[2] & vis[3]) {
                *reinterpret_cast<float4*>(G + i0) = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
#pragma unroll
                for (int q = 0; q < 4; q++)
                    if (vis[q]) G[i0 + q] = 0.f;
            }
            return;
        }
        float4 p = *reinterpret_cast<float4*>(P + i0), g = *reinterpret_cast<float4*>(G + i0);
        float4 m = *reinterpret_cast<float4*>(M + i0), v = *reinterpret_cast<float4*>(V + i0);
        adam_one(p.x, g.x, m.x, v.x, upd[0], vis[0], lr, a, bc1, bc2);
        adam_one(p.y, g.y, m.y, v.y, upd[1], vis[1], lr, a, bc1, bc2);
        adam_one(p.z, g.z, m.z, v.z, upd[2], vis[2], lr, a, bc1, bc2);
        adam_one(p.w, g.w, m.w, v.w, upd[3], vis[3], lr, a, bc1, bc2);
        *reinterpret_cast<float4*>(P + i0) = p;
        *reinterpret_cast<float4*>(G + i0) = g;
        *reinterpret_cast<float4*>(M + i0) = m;
        *reinterpret_cast<float4*>(V + i0) = v;
    } else {
        for (int q = 0; q < 4 && i0 + q < n; q++) {
            if (!vis[q]) continue;
            const int64_t i = i0 + q;
            if (!upd[q]) {
                G[i] = 0.f;
                continue;
            }
            float p = P[i], g = G[i], m = M[i], v = V[i];
            adam_one(p, g, m, v, true, true, lr, a, bc1, bc2);
            P[i] = p;
            G[i] = g;
            M[i] = m;
            V[i] = v;
        }
    }
}

cudaError_t launch_adam(const AdamArgs& a, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    const int64_t bx = (a.n + 4 * 256 - 1) / (4 * 256);
    adam_kernel<<<dim3((unsigned)bx, a.n_planes), 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gs
