// Gaussian-GICP loop registration (RMGS-SLAM §III-D): the frustum target set around a
// historical loopframe, planar-regularised covariances, nearest-mean correspondences and the
// Gauss-Newton normal equations of sum r^T (Sigma~_n + R Sigma~_m R^T)^-1 r, r = mu_n - T mu_m.
//
// The target set's decisions (in front of the near plane, inside the image, within d_max of
// the view's centre) are taken in FP32 with a fixed operation order.  Correspondences are found
// in FP32 through a spatial hash of the target means (cells 0.1% wider than d_corr, computed in
// FP64, so the nearest target within d_corr is always in the 27 cells around the query's).
// The weights, residuals and normal equations are evaluated in FP64 and summed in FP64; the
// host solves the 6 x 6 system and updates T (api.cu).
#include "gs_kernels.cuh"

namespace gs {

constexpr int kGThreads = 256;

struct GicpState {
    unsigned long long count;
    double acc[29];   // H upper triangle (21), g (6), cost, correspondences
};

static int g_grid(int64_t n) {
    int64_t b = (n + kGThreads - 1) / kGThreads;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

__global__ void __launch_bounds__(kGThreads) gicp_target_kernel(GicpMap map, const GicpView* views, int nv,
                                                                float near_z, float dmax2, const uint8_t* src_flag,
                                                                uint8_t* flag, GicpState* s) {
    uint32_t cnt = 0;
    const int64_t n = map.n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float m0 = map.means[i], m1 = map.means[n + i], m2 = map.means[2 * n + i];
        bool in = false;
        for (int k = 0; k < nv && !in; k++) {
            const GicpView& V = views[k];
            float pc[3];
#pragma unroll
            for (int r = 0; r < 3; r++)
                pc[r] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(V.R[3 * r], m0), __fmul_rn(V.R[3 * r + 1], m1)),
                                            __fmul_rn(V.R[3 * r + 2], m2)), V.t[r]);
            const float z = pc[2];
            const float u = __fadd_rn(__fdiv_rn(__fmul_rn(V.fx, pc[0]), z), V.cx);
            const float v = __fadd_rn(__fdiv_rn(__fmul_rn(V.fy, pc[1]), z), V.cy);
            const bool img = z > near_z && u >= 0.f && u < V.W && v >= 0.f && v < V.H;
            const float d0 = __fsub_rn(m0, V.c[0]), d1 = __fsub_rn(m1, V.c[1]), d2 = __fsub_rn(m2, V.c[2]);
            const float dd = __fadd_rn(__fadd_rn(__fmul_rn(d0, d0), __fmul_rn(d1, d1)), __fmul_rn(d2, d2));
            in = img && dd < dmax2;
        }
        if (src_flag && src_flag[i]) in = false;
        flag[i] = in ? 1 : 0;
        cnt += in;
    }
    cnt = warp_sum(cnt);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&s->count, (unsigned long long)cnt);
}

// ---------------------------------------------------------------------------------------
// Target hash: row ids of the flagged target means by cell hash (counting sort).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t g_hash(int cx, int cy, int cz, uint32_t mask) {
    return ((uint32_t)cx * 73856093u ^ (uint32_t)cy * 19349663u ^ (uint32_t)cz * 83492791u) & mask;
}
__device__ __forceinline__ int g_cell(float p, double inv) { return (int)floor((double)p * inv); }

// pts: the flagged target means in hash order, (x, y, z, row index bits), so that a candidate
// of the nearest-mean search is one 16-byte load from a contiguous run of its cell
struct GicpHash {
    uint64_t T;
    uint32_t *count, *start, *cursor, *cell, *bsum;
    float4* pts;
    double* Rt;   // R (9) and t (3) of the current iteration
    GicpState* state;
};

static size_t hash_words(uint64_t T, int64_t n_tar) { return 3 * (size_t)T + (size_t)n_tar + (size_t)(T / 1024) + 2; }

static GicpHash hash_layout(void* scratch, int64_t n_tar) {
    GicpHash h;
    h.T = 1;
    while (h.T < (uint64_t)(2 * (n_tar > 0 ? n_tar : 1))) h.T <<= 1;
    h.state = static_cast<GicpState*>(scratch);
    uint32_t* b = reinterpret_cast<uint32_t*>(h.state + 1);
    h.count = b;
    h.start = h.count + h.T;
    h.cursor = h.start + h.T;
    h.cell = h.cursor + h.T;
    h.bsum = h.cell + n_tar;
    uintptr_t q = reinterpret_cast<uintptr_t>(b + hash_words(h.T, n_tar));
    q = (q + 15) & ~(uintptr_t)15;
    h.pts = reinterpret_cast<float4*>(q);
    h.Rt = reinterpret_cast<double*>(h.pts + n_tar);
    return h;
}

size_t gicp_scratch_bytes(int64_t n_tar) {
    uint64_t T = 1;
    while (T < (uint64_t)(2 * (n_tar > 0 ? n_tar : 1))) T <<= 1;
    // hash words, then (16-byte aligned) the means in hash order, then 12 doubles (R, t)
    const size_t reg = sizeof(GicpState) + sizeof(uint32_t) * hash_words(T, n_tar) + 15 +
                       sizeof(float4) * (size_t)(n_tar > 0 ? n_tar : 0) + 12 * sizeof(double);
    // target set: the state, then the view table
    const size_t tgt = ((sizeof(GicpState) + 255) & ~(size_t)255) + sizeof(GicpView) * GS_MAX_VIEWS;
    return ((reg > tgt ? reg : tgt) + 255) & ~(size_t)255;
}

__global__ void __launch_bounds__(kGThreads) gicp_hash_count(GicpMap tar, const uint8_t* flag, double inv,
                                                             uint32_t mask, uint32_t* count, uint32_t* cell) {
    const int64_t n = tar.n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (flag && !flag[i]) continue;
        const uint32_t h = g_hash(g_cell(tar.means[i], inv), g_cell(tar.means[n + i], inv),
                                  g_cell(tar.means[2 * n + i], inv), mask);
        cell[i] = h;
        atomicAdd(&count[h], 1u);
    }
}

__global__ void __launch_bounds__(kGThreads) gicp_hash_fill(GicpMap tar, const uint8_t* flag, const uint32_t* cell,
                                                            const uint32_t* start, uint32_t* cursor, float4* pts) {
    const int64_t n = tar.n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (flag && !flag[i]) continue;
        const uint32_t h = cell[i];
        pts[start[h] + atomicAdd(&cursor[h], 1u)] =
            make_float4(tar.means[i], tar.means[n + i], tar.means[2 * n + i], __int_as_float((int)i));
    }
}

// ---------------------------------------------------------------------------------------
// Normal equations.
// ---------------------------------------------------------------------------------------
// Planar covariance R diag(l) R^T (l = 1e-3 on the smallest log-scale axis, the first on ties,
// 1 on the others), R from the normalised quaternion; upper triangle xx xy xz yy yz zz.
__device__ void planar_cov(const GicpMap& g, int64_t i, double (&S)[6]) {
    const int64_t n = g.n;
    double w = g.quats[i], x = g.quats[n + i], y = g.quats[2 * n + i], z = g.quats[3 * n + i];
    const double in = 1.0 / sqrt(w * w + x * x + y * y + z * z);
    w *= in; x *= in; y *= in; z *= in;
    const double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                         2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                         2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
    const float l0 = g.log_scales[i], l1 = g.log_scales[n + i], l2 = g.log_scales[2 * n + i];
    const int a = (l0 <= l1 && l0 <= l2) ? 0 : (l1 <= l2 ? 1 : 2);
    const double lam[3] = {a == 0 ? 1e-3 : 1.0, a == 1 ? 1e-3 : 1.0, a == 2 ? 1e-3 : 1.0};
    int k = 0;
    for (int r = 0; r < 3; r++)
        for (int c = r; c < 3; c++) {
            double v = 0;
            for (int e = 0; e < 3; e++) v += R[3 * r + e] * lam[e] * R[3 * c + e];
            S[k++] = v;
        }
}

// ---------------------------------------------------------------------------------------
// Source list: the flagged source rows of [lo, hi) (hi - lo <= the hash size T), compacted
// into the hash's cursor words, which are free once the hash is built, with their count in
// the first scan word.  The normal equations then run on full warps: the FP64 pipe takes a
// warp instruction at the same cost however few of its lanes are active, so a grid over every
// row of the map (most not flagged) would pay about 32 times for each flagged row.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kGThreads) gicp_src_compact(const uint8_t* flag, int64_t lo, int64_t hi,
                                                              uint32_t* list, uint32_t* count) {
    const int lane = threadIdx.x & 31;
    uint32_t ltm;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(ltm));
    // (base is the same for the 32 lanes of a warp, so the loop and the ballot are warp-uniform)
    for (int64_t base = lo + (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < hi;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = base + lane;
        const bool f = m < hi && (!flag || flag[m] != 0);
        const uint32_t bal = __ballot_sync(0xffffffffu, f);
        if (!bal) continue;
        uint32_t b = 0;
        if (lane == 0) b = atomicAdd(count, (uint32_t)__popc(bal));
        b = __shfl_sync(0xffffffffu, b, 0);
        if (f) list[b + __popc(bal & ltm)] = (uint32_t)(m - lo);
    }
}

__global__ void __launch_bounds__(kGThreads) gicp_normal_kernel(GicpMap src, const uint32_t* list,
                                                                const uint32_t* list_count, int64_t lo, GicpMap tar,
                                                                double inv, uint32_t mask, float r2,
                                                                GicpHash h, const double* Rd, const double* td,
                                                                float Rf0, float Rf1, float Rf2, float Rf3, float Rf4,
                                                                float Rf5, float Rf6, float Rf7, float Rf8, float tf0,
                                                                float tf1, float tf2) {
    const float Rf[9] = {Rf0, Rf1, Rf2, Rf3, Rf4, Rf5, Rf6, Rf7, Rf8};
    const float tf[3] = {tf0, tf1, tf2};
    double acc[29];
#pragma unroll
    for (int k = 0; k < 29; k++) acc[k] = 0.0;
    const int64_t ns = src.n, nt = tar.n;
    const int64_t cnt = (int64_t)*list_count;
    for (int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; li < cnt; li += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = lo + list[li];
        const float s0 = src.means[m], s1 = src.means[ns + m], s2 = src.means[2 * ns + m];
        float q[3];
#pragma unroll
        for (int r = 0; r < 3; r++)
            q[r] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(Rf[3 * r], s0), __fmul_rn(Rf[3 * r + 1], s1)),
                                       __fmul_rn(Rf[3 * r + 2], s2)), tf[r]);
        const int cx = g_cell(q[0], inv), cy = g_cell(q[1], inv), cz = g_cell(q[2], inv);
        float best = r2;
        int64_t bi = -1;
        for (int dz = -1; dz <= 1; dz++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    const uint32_t hh = g_hash(cx + dx, cy + dy, cz + dz, mask);
                    const uint32_t b = h.start[hh], e = b + h.count[hh];
                    for (uint32_t t = b; t < e; t++) {
                        const float4 P = h.pts[t];
                        const int64_t j = __float_as_int(P.w);
                        const float ex = __fsub_rn(q[0], P.x), ey = __fsub_rn(q[1], P.y), ez = __fsub_rn(q[2], P.z);
                        const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
                        if (d2 < best || (d2 == best && bi >= 0 && j < bi)) { best = d2; bi = j; }
                    }
                }
        if (bi < 0) continue;
        // FP64: residual, weight, Jacobian J = [-I | [q]x]
        double qd[3], res[3];
        for (int r = 0; r < 3; r++) qd[r] = Rd[3 * r] * s0 + Rd[3 * r + 1] * s1 + Rd[3 * r + 2] * s2 + td[r];
        res[0] = (double)tar.means[bi] - qd[0];
        res[1] = (double)tar.means[nt + bi] - qd[1];
        res[2] = (double)tar.means[2 * nt + bi] - qd[2];
        double Sm[6], Sn[6];
        planar_cov(src, m, Sm);
        planar_cov(tar, bi, Sn);
        const double Smf[9] = {Sm[0], Sm[1], Sm[2], Sm[1], Sm[3], Sm[4], Sm[2], Sm[4], Sm[5]};
        double A[9];   // Sigma~_n + R Sigma~_m R^T
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) {
                double v = 0;
                for (int e = 0; e < 3; e++)
                    for (int f = 0; f < 3; f++) v += Rd[3 * r + e] * Smf[3 * e + f] * Rd[3 * c + f];
                A[3 * r + c] = v;
            }
        A[0] += Sn[0]; A[1] += Sn[1]; A[2] += Sn[2]; A[3] += Sn[1]; A[4] += Sn[3]; A[5] += Sn[4];
        A[6] += Sn[2]; A[7] += Sn[4]; A[8] += Sn[5];
        // inverse by the adjugate
        const double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
        const double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
        const double id = 1.0 / det;
        const double O[9] = {c00 * id, (A[2] * A[7] - A[1] * A[8]) * id, (A[1] * A[5] - A[2] * A[4]) * id,
                             c01 * id, (A[0] * A[8] - A[2] * A[6]) * id, (A[2] * A[3] - A[0] * A[5]) * id,
                             c02 * id, (A[1] * A[6] - A[0] * A[7]) * id, (A[0] * A[4] - A[1] * A[3]) * id};
        const double J[3][6] = {{-1, 0, 0, 0, -qd[2], qd[1]}, {0, -1, 0, qd[2], 0, -qd[0]}, {0, 0, -1, -qd[1], qd[0], 0}};
        double OJ[3][6], Or[3];
        for (int r = 0; r < 3; r++) {
            Or[r] = O[3 * r] * res[0] + O[3 * r + 1] * res[1] + O[3 * r + 2] * res[2];
            for (int c = 0; c < 6; c++) OJ[r][c] = O[3 * r] * J[0][c] + O[3 * r + 1] * J[1][c] + O[3 * r + 2] * J[2][c];
        }
        int k = 0;
        for (int r = 0; r < 6; r++)
            for (int c = r; c < 6; c++) acc[k++] += J[0][r] * OJ[0][c] + J[1][r] * OJ[1][c] + J[2][r] * OJ[2][c];
        for (int r = 0; r < 6; r++) acc[21 + r] += J[0][r] * Or[0] + J[1][r] * Or[1] + J[2][r] * Or[2];
        acc[27] += res[0] * Or[0] + res[1] * Or[1] + res[2] * Or[2];
        acc[28] += 1.0;
    }
    // warp sums, then one FP64 atomic per value per warp (warps without a correspondence add
    // nothing)
    if (!__any_sync(0xffffffffu, acc[28] != 0.0)) return;
#pragma unroll
    for (int k = 0; k < 29; k++) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(&h.state->acc[k], v);
    }
}

cudaError_t launch_gicp_target_set(const GicpMap& map, const GicpView* views, int n_views, float near_z, float dmax2,
                                   const uint8_t* source_flag, uint8_t* target_flag, void* scratch,
                                   unsigned long long* count_host, cudaStream_t st) {
    GicpState* s = static_cast<GicpState*>(scratch);
    GicpView* dv = reinterpret_cast<GicpView*>(reinterpret_cast<char*>(scratch) + ((sizeof(GicpState) + 255) & ~(size_t)255));
    cudaError_t e = cudaMemsetAsync(s, 0, sizeof(GicpState), st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(dv, views, sizeof(GicpView) * n_views, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    gicp_target_kernel<<<g_grid(map.n), kGThreads, 0, st>>>(map, dv, n_views, near_z, dmax2, source_flag, target_flag, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaMemcpyAsync(count_host, &s->count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
}

cudaError_t launch_gicp_build(const GicpMap& tar, const uint8_t* tar_flag, float d_corr, void* scratch, cudaStream_t st) {
    GicpHash h = hash_layout(scratch, tar.n);
    cudaError_t e;
    if ((e = cudaMemsetAsync(h.count, 0, sizeof(uint32_t) * h.T, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(h.cursor, 0, sizeof(uint32_t) * h.T, st)) != cudaSuccess) return e;
    const double inv = 1.0 / (1.001 * (double)d_corr);
    const uint32_t mask = (uint32_t)(h.T - 1);
    if (tar.n > 0) gicp_hash_count<<<g_grid(tar.n), kGThreads, 0, st>>>(tar, tar_flag, inv, mask, h.count, h.cell);
    if ((e = exclusive_scan_u32(h.count, (int64_t)h.T, h.start, h.bsum, nullptr, st)) != cudaSuccess) return e;
    if (tar.n > 0) gicp_hash_fill<<<g_grid(tar.n), kGThreads, 0, st>>>(tar, tar_flag, h.cell, h.start, h.cursor, h.pts);
    return cudaGetLastError();
}

cudaError_t launch_gicp_normal_eq(const GicpMap& src, const uint8_t* src_flag, const GicpMap& tar, float d_corr,
                                  const double* R, const double* t, void* scratch, double* acc_host, cudaStream_t st) {
    GicpHash h = hash_layout(scratch, tar.n);
    // R and t (FP64) travel after the hashed means, written from the host each iteration
    cudaError_t e = cudaMemsetAsync(h.state, 0, sizeof(GicpState), st);
    if (e != cudaSuccess) return e;
    double* Rt = h.Rt;
    double host[12];
    for (int k = 0; k < 9; k++) host[k] = R[k];
    for (int k = 0; k < 3; k++) host[9 + k] = t[k];
    if ((e = cudaMemcpyAsync(Rt, host, sizeof(host), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    const double inv = 1.0 / (1.001 * (double)d_corr);
    const uint32_t mask = (uint32_t)(h.T - 1);
    const float r2 = d_corr * d_corr;
    // the source rows in segments of at most T rows (one segment when the source map is no
    // larger than twice the target map)
    for (int64_t lo = 0; lo < src.n; lo += (int64_t)h.T) {
        const int64_t hi = src.n - lo < (int64_t)h.T ? src.n : lo + (int64_t)h.T;
        if ((e = cudaMemsetAsync(h.bsum, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
        gicp_src_compact<<<g_grid(hi - lo), kGThreads, 0, st>>>(src_flag, lo, hi, h.cursor, h.bsum);
        gicp_normal_kernel<<<g_grid(hi - lo), kGThreads, 0, st>>>(
            src, h.cursor, h.bsum, lo, tar, inv, mask, r2, h, Rt, Rt + 9, (float)R[0], (float)R[1], (float)R[2],
            (float)R[3], (float)R[4], (float)R[5], (float)R[6], (float)R[7], (float)R[8], (float)t[0], (float)t[1],
            (float)t[2]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = cudaMemcpyAsync(acc_host, h.state->acc, sizeof(double) * 29, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return e;
    return cudaStreamSynchronize(st);   // the host array must not go out of scope before the copy
}

}  // namespace gs
