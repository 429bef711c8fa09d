// a8: fused masked Adam over the parameter planes, zeroing the gradients it consumed.
// RMGS-SLAM §III-C: visible and unfrozen Gaussians are refined by a sparse gradient-based
// optimiser (only Gaussians of the most recent segments are updated).
#include "gs_kernels.cuh"

namespace gs {

__device__ __forceinline__ void adam_one(float& p, float& g, float& m, float& v, bool upd, float lr, const AdamArgs& a,
                                         float bc1, float bc2) {
    if (upd) {
        m = a.b1 * m + (1.f - a.b1) * g;
        v = a.b2 * v + (1.f - a.b2) * g * g;
        const float mh = m / bc1, vh = v / bc2;
        p -= lr * mh / (sqrtf(vh) + a.eps);
    }
    g = 0.f;
}

// Advances the device-side Adam step counter and stores the bias corrections of that step
// (one thread; lets a captured graph run many steps without host-side parameters).
__global__ void adam_step_counter_kernel(Counters* c, float b1, float b2) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const unsigned long long t = c->adam_step + 1;
    c->adam_step = t;
    c->adam_bc1 = (float)(1.0 - pow((double)b1, (double)t));
    c->adam_bc2 = (float)(1.0 - pow((double)b2, (double)t));
}

cudaError_t launch_adam_step_counter(Counters* c, float b1, float b2, cudaStream_t st) {
    adam_step_counter_kernel<<<1, 32, 0, st>>>(c, b1, b2);
    return cudaGetLastError();
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
    const float bc1 = a.step_dev ? a.step_dev->adam_bc1 : a.bc1;
    const float bc2 = a.step_dev ? a.step_dev->adam_bc2 : a.bc2;
    bool upd[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int64_t i = i0 + q;
        upd[q] = i < n && (!a.update_mask || a.update_mask[i]) && (!a.visible || a.visible[i]);
    }
    const bool vec = ((n & 3) == 0) && (((uintptr_t)P | (uintptr_t)G | (uintptr_t)M | (uintptr_t)V) & 15) == 0;
    if (vec) {
        float4 p = *reinterpret_cast<float4*>(P + i0), g = *reinterpret_cast<float4*>(G + i0);
        float4 m = *reinterpret_cast<float4*>(M + i0), v = *reinterpret_cast<float4*>(V + i0);
        adam_one(p.x, g.x, m.x, v.x, upd[0], lr, a, bc1, bc2);
        adam_one(p.y, g.y, m.y, v.y, upd[1], lr, a, bc1, bc2);
        adam_one(p.z, g.z, m.z, v.z, upd[2], lr, a, bc1, bc2);
        adam_one(p.w, g.w, m.w, v.w, upd[3], lr, a, bc1, bc2);
        *reinterpret_cast<float4*>(P + i0) = p;
        *reinterpret_cast<float4*>(G + i0) = g;
        if (upd[0] | upd[1] | upd[2] | upd[3]) {
            *reinterpret_cast<float4*>(M + i0) = m;
            *reinterpret_cast<float4*>(V + i0) = v;
        }
    } else {
        for (int q = 0; q < 4 && i0 + q < n; q++) {
            const int64_t i = i0 + q;
            float p = P[i], g = G[i], m = M[i], v = V[i];
            adam_one(p, g, m, v, upd[q], lr, a, bc1, bc2);
            P[i] = p;
            G[i] = g;
            if (upd[q]) { M[i] = m; V[i] = v; }
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
