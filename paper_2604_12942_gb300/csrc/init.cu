// a10-a11: voxel-PCA geometric fitting (RMGS-SLAM §III-A) and the cascaded Gaussian
// initialisation (§III-B equations).  Points are grouped into cubic voxels by sorting their
// voxel keys with the library's radix sort; one thread per voxel then computes the mean,
// the covariance, a 3x3 Jacobi eigen-decomposition, the planar / linear classification and
// the trace of the descriptor covariance, and writes the per-point features the learned
// initialiser consumes.
#include <cstring>

#include "gs_kernels.cuh"

namespace gs {

constexpr float kLambdaFloor = 1e-4f;   // (0.01 m)^2 floor of eigenvalues before the log
constexpr float kY00 = 0.28209479177387814f;

struct PcaArgs {
    int64_t n;
    const float* pts;      // [3][n]
    const float* rgb;      // [3][n]
    float voxel, tau_p, tau_l, sigma2, tau_trace;
    int min_pts;
    unsigned long long* keys;   // sorted keys
    const uint32_t* idx;        // sorted point indices
    float* x;              // [n][16]
    uint8_t* has_feature;
    uint8_t* reliable;
    float* s_pca;          // [n][3]
    float* q_pca;          // [n][4]
    const float* depth;    // [n]
    float fx;
};

// voxel key of an FP32 point: floor(p / s) per axis (IEEE division), 21 bits each, +2^20
__device__ __forceinline__ unsigned long long voxel_key(float x, float y, float z, float s) {
    unsigned long long k = 0;
    const float c[3] = {x, y, z};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float q = floorf(__fdiv_rn(c[a], s));
        q = fminf(fmaxf(q, -1048576.0f), 1048575.0f);
        k = (k << 21) | (unsigned long long)((int)q + 1048576);
    }
    return k;
}

__global__ void voxel_key_kernel(const float* pts, int64_t n, float s, unsigned long long* keys, uint32_t* idx,
                                 Counters* c) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        c->status = 0;
        c->n_pairs = (unsigned long long)n;
    }
    if (i >= n) return;
    keys[i] = voxel_key(pts[i], pts[n + i], pts[2 * n + i], s);
    idx[i] = (uint32_t)i;
}

// Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix; columns of V are eigenvectors.
__device__ void jacobi3(float A[9], float lam[3], float V[9]) {
#pragma unroll
    for (int i = 0; i < 9; i++) V[i] = (i % 4 == 0) ? 1.f : 0.f;
    for (int sweep = 0; sweep < 12; sweep++) {
        const float off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
        const float diag = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
        if (off <= 1e-14f * diag || off == 0.f) break;
#pragma unroll
        for (int pq = 0; pq < 3; pq++) {
            const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
            const float apq = A[p * 3 + q];
            if (apq == 0.f) continue;
            const float theta = 0.5f * (A[q * 3 + q] - A[p * 3 + p]) / apq;
            const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
            const float cth = rsqrtf(t * t + 1.f), sth = t * cth;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float akp = A[k * 3 + p], akq = A[k * 3 + q];
                A[k * 3 + p] = cth * akp - sth * akq;
                A[k * 3 + q] = sth * akp + cth * akq;
            }
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float apk = A[p * 3 + k], aqk = A[q * 3 + k];
                A[p * 3 + k] = cth * apk - sth * aqk;
                A[q * 3 + k] = sth * apk + cth * aqk;
            }
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float vkp = V[k * 3 + p], vkq = V[k * 3 + q];
                V[k * 3 + p] = cth * vkp - sth * vkq;
                V[k * 3 + q] = sth * vkp + cth * vkq;
            }
        }
    }
    lam[0] = A[0];
    lam[1] = A[4];
    lam[2] = A[8];
}

// Rotation matrix -> unit quaternion (w, x, y, z) with w >= 0 (largest-pivot form).
__device__ void matrix_to_quat(const float R[9], float q[4]) {
    const float tr = R[0] + R[4] + R[8];
    const float c0 = 1.f + tr, c1 = 1.f + R[0] - R[4] - R[8], c2 = 1.f - R[0] + R[4] - R[8], c3 = 1.f - R[0] - R[4] + R[8];
    int k = 0;
    float best = c0;
    if (c1 > best) { best = c1; k = 1; }
    if (c2 > best) { best = c2; k = 2; }
    if (c3 > best) { best = c3; k = 3; }
    const float s = 2.f * sqrtf(fmaxf(best, 1e-30f)), is = 1.f / s;
    if (k == 0) { q[0] = 0.25f * s; q[1] = (R[7] - R[5]) * is; q[2] = (R[2] - R[6]) * is; q[3] = (R[3] - R[1]) * is; }
    else if (k == 1) { q[0] = (R[7] - R[5]) * is; q[1] = 0.25f * s; q[2] = (R[1] + R[3]) * is; q[3] = (R[2] + R[6]) * is; }
    else if (k == 2) { q[0] = (R[2] - R[6]) * is; q[1] = (R[1] + R[3]) * is; q[2] = 0.25f * s; q[3] = (R[5] + R[7]) * is; }
    else { q[0] = (R[3] - R[1]) * is; q[1] = (R[2] + R[6]) * is; q[2] = (R[5] + R[7]) * is; q[3] = 0.25f * s; }
    const float nrm = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float sg = q[0] < 0.f ? -nrm : nrm;
#pragma unroll
    for (int i = 0; i < 4; i++) q[i] *= sg;
}

// One thread per sorted position; the first point of each voxel processes the voxel.
__global__ void __launch_bounds__(128) voxel_stats_kernel(PcaArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = a.n;
    if (i >= n) return;
    const unsigned long long key = a.keys[i];
    if (i > 0 && a.keys[i - 1] == key) return;
    int64_t e = i + 1;
    while (e < n && a.keys[e] == key) e++;
    const int64_t N = e - i;
    const float* P = a.pts;
    float mu[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f}, V[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    bool has = N >= a.min_pts, rel = false;
    if (has) {
        // centre on the first point for precision, then the two-pass mean / covariance
        const uint32_t p0 = a.idx[i];
        const float o[3] = {P[p0], P[n + p0], P[2 * n + p0]};
        float m[3] = {0.f, 0.f, 0.f};
        for (int64_t j = i; j < e; j++) {
            const uint32_t pj = a.idx[j];
#pragma unroll
            for (int k = 0; k < 3; k++) m[k] += P[(int64_t)k * n + pj] - o[k];
        }
#pragma unroll
        for (int k = 0; k < 3; k++) m[k] /= (float)N;
        float C[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int64_t j = i; j < e; j++) {
            const uint32_t pj = a.idx[j];
            float d[3];
#pragma unroll
            for (int k = 0; k < 3; k++) d[k] = P[(int64_t)k * n + pj] - o[k] - m[k];
#pragma unroll
            for (int r = 0; r < 3; r++)
#pragma unroll
                for (int c = 0; c < 3; c++) C[r * 3 + c] += d[r] * d[c];
        }
#pragma unroll
        for (int k = 0; k < 9; k++) C[k] /= (float)N;
#pragma unroll
        for (int k = 0; k < 3; k++) mu[k] = o[k] + m[k];
        float W[9], lw[3];
        jacobi3(C, lw, W);
        // ascending order
        int id[3] = {0, 1, 2};
        if (lw[id[1]] < lw[id[0]]) { int t = id[0]; id[0] = id[1]; id[1] = t; }
        if (lw[id[2]] < lw[id[1]]) { int t = id[1]; id[1] = id[2]; id[2] = t; }
        if (lw[id[1]] < lw[id[0]]) { int t = id[0]; id[0] = id[1]; id[1] = t; }
#pragma unroll
        for (int c = 0; c < 3; c++) {
            l[c] = lw[id[c]];
#pragma unroll
            for (int r = 0; r < 3; r++) V[r * 3 + c] = W[r * 3 + id[c]];
        }
        // sign: largest-magnitude component positive; v_max = v_min x v_mid
#pragma unroll
        for (int c = 0; c < 2; c++) {
            int big = 0;
            if (fabsf(V[3 + c]) > fabsf(V[big * 3 + c])) big = 1;
            if (fabsf(V[6 + c]) > fabsf(V[big * 3 + c])) big = 2;
            if (V[big * 3 + c] < 0.f)
#pragma unroll
                for (int r = 0; r < 3; r++) V[r * 3 + c] = -V[r * 3 + c];
        }
        V[2] = V[3] * V[7] - V[6] * V[4];
        V[5] = V[6] * V[1] - V[0] * V[7];
        V[8] = V[0] * V[4] - V[3] * V[1];
        const int cls = (l[0] < a.tau_p) ? 1 : ((l[2] > a.tau_l * l[0]) ? 2 : 0);
        const float g1 = (l[1] - l[0]) / fmaxf(l[2], 1e-30f), g2 = (l[2] - l[1]) / fmaxf(l[2], 1e-30f);
        if (cls != 0 && g1 > 1e-6f && g2 > 1e-6f) {
            // trace of the directional block of Sigma_g = sigma^2 sum_i ||F_i||_F^2, where row m
            // of F_i is (d.v_m v_k + d.v_k v_m) / (N (l_k - l_m)) and the two terms are orthogonal
            const int k = cls == 1 ? 0 : 2;
            float tr = 0.f;
            for (int64_t j = i; j < e; j++) {
                const uint32_t pj = a.idx[j];
                float d[3];
#pragma unroll
                for (int q = 0; q < 3; q++) d[q] = P[(int64_t)q * n + pj] - mu[q];
                const float dk = d[0] * V[k] + d[1] * V[3 + k] + d[2] * V[6 + k];
#pragma unroll
                for (int mm = 0; mm < 3; mm++) {
                    if (mm == k) continue;
                    const float dm = d[0] * V[mm] + d[1] * V[3 + mm] + d[2] * V[6 + mm];
                    const float den = (float)N * (l[k] - l[mm]);
                    tr += (dm * dm + dk * dk) / (den * den);
                }
            }
            rel = tr * a.sigma2 < a.tau_trace;
        }
    }
    float qv[4] = {1.f, 0.f, 0.f, 0.f};
    if (has) matrix_to_quat(V, qv);
    for (int64_t j = i; j < e; j++) {
        const uint32_t p = a.idx[j];
        float* x = a.x + 16 * (size_t)p;
        if (has) {
#pragma unroll
            for (int k = 0; k < 3; k++) x[k] = logf(fmaxf(l[k], kLambdaFloor));
#pragma unroll
            for (int k = 0; k < 9; k++) x[3 + k] = V[k];
#pragma unroll
            for (int k = 0; k < 3; k++) x[12 + k] = a.rgb[(int64_t)k * n + p];
            x[15] = logf(fmaxf(a.depth[p], 1e-6f) / a.fx);
        } else {
#pragma unroll
            for (int k = 0; k < 16; k++) x[k] = 0.f;
        }
        a.has_feature[p] = has;
        a.reliable[p] = rel;
#pragma unroll
        for (int k = 0; k < 3; k++) a.s_pca[3 * (size_t)p + k] = has ? 0.5f * logf(fmaxf(l[k], kLambdaFloor)) : 0.f;
#pragma unroll
        for (int k = 0; k < 4; k++) a.q_pca[4 * (size_t)p + k] = qv[k];
    }
}

// Frames a point may be seen from (the segment's keyframes / loopframes), by value.
struct FrameSet {
    int n;
    gs_camera cam[GS_MAX_VIEWS];
};

// Per point: the camera-frame depth in the closest frame whose image it projects into (the
// "closer view" of §III-B), and whether there is one; if none, the depth in frame 0.
__global__ void point_depth_kernel(const float* pts, int64_t n, const __grid_constant__ FrameSet fs, float* depth,
                                   uint8_t* inside) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = pts[i], y = pts[n + i], z = pts[2 * n + i];
    float best = 0.f, first = 0.f;
    bool found = false;
    for (int f = 0; f < fs.n; f++) {
        const gs_camera& cam = fs.cam[f];
        const float* R = cam.R_cw;
        const float cx = R[0] * x + R[1] * y + R[2] * z + cam.t_cw[0];
        const float cy = R[3] * x + R[4] * y + R[5] * z + cam.t_cw[1];
        const float cz = R[6] * x + R[7] * y + R[8] * z + cam.t_cw[2];
        if (f == 0) first = cz;
        if (!(cz > 0.f)) continue;
        const float u = cam.fx * cx / cz + cam.cx, v = cam.fy * cy / cz + cam.cy;
        if (u >= 0.f && u < (float)cam.width && v >= 0.f && v < (float)cam.height && (!found || cz < best)) {
            best = cz;
            found = true;
        }
    }
    depth[i] = found ? best : first;
    inside[i] = found;
}



struct PcaWs {
    size_t counters, keys0, keys1, vals0, vals1, hist, total;
};

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

static PcaWs pca_layout(int64_t n) {
    PcaWs L;
    size_t off = 0;
    auto take = [&](size_t b) { const size_t r = off; off = al256(off + b); return r; };
    L.counters = take(sizeof(Counters));
    L.keys0 = take(8 * (size_t)n);
    L.keys1 = take(8 * (size_t)n);
    L.vals0 = take(4 * (size_t)n);
    L.vals1 = take(4 * (size_t)n);
    L.hist = take(sizeof(uint32_t) * ((size_t)kSortMaxBins * kSortMaxGrid + kSortMaxBins));
    L.total = off;
    return L;
}

size_t pca_workspace_size(int64_t n) { return pca_layout(n).total; }

cudaError_t launch_voxel_pca(const float* pts, const float* rgb, int64_t n, const FrameSet& fs, float voxel,
                             int min_pts, float tau_p, float tau_l, float sigma, float tau_trace, void* ws,
                             float* x, uint8_t* has_feature, uint8_t* reliable, float* s_pca, float* q_pca,
                             float* depth, uint8_t* inside, cudaStream_t st) {
    const PcaWs L = pca_layout(n);
    char* b = static_cast<char*>(ws);
    Counters* cnt = reinterpret_cast<Counters*>(b + L.counters);
    SortArgs sa;
    unsigned long long* vkeys = reinterpret_cast<unsigned long long*>(b + L.keys0);
    sa.keys[0] = vkeys;
    sa.keys[1] = b + L.keys1;
    sa.vals[0] = reinterpret_cast<uint32_t*>(b + L.vals0);
    sa.vals[1] = reinterpret_cast<uint32_t*>(b + L.vals1);
    sa.hist = reinterpret_cast<uint32_t*>(b + L.hist);
    sa.digit_tot = sa.hist + (size_t)kSortMaxBins * kSortMaxGrid;
    sa.counters = cnt;
    sa.count = &cnt->n_pairs;
    sa.grid = sort_grid();
    const int blocks = (int)((n + 255) / 256);
    point_depth_kernel<<<blocks, 256, 0, st>>>(pts, n, fs, depth, inside);
    voxel_key_kernel<<<blocks, 256, 0, st>>>(pts, n, voxel, vkeys, sa.vals[0], cnt);
    int shifts[8] = {0, 8, 16, 24, 32, 40, 48, 56};
    cudaError_t e = launch_sort64(sa, 8, shifts, st);   // 63-bit keys, result back in buffer 0
    if (e != cudaSuccess) return e;
    PcaArgs a;
    a.n = n;
    a.pts = pts;
    a.rgb = rgb;
    a.voxel = voxel;
    a.tau_p = tau_p;
    a.tau_l = tau_l;
    a.sigma2 = sigma * sigma;
    a.tau_trace = tau_trace;
    a.min_pts = min_pts;
    a.keys = vkeys;
    a.idx = sa.vals[0];
    a.x = x;
    a.has_feature = has_feature;
    a.reliable = reliable;
    a.s_pca = s_pca;
    a.q_pca = q_pca;
    a.depth = depth;
    a.fx = fs.cam[0].fx;
    voxel_stats_kernel<<<(int)((n + 127) / 128), 128, 0, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Cascade (§III-B): model where the MLP prediction is valid, else PCA where reliable, else
// the isotropic depth heuristic.
// ---------------------------------------------------------------------------------------
struct CascadeArgs {
    int64_t n;
    int K;                  // SH coefficients per channel of the output map
    const float* pts;       // [3][n]
    const float* rgb;       // [3][n]
    const float* y;         // [n][16] or null
    const uint8_t* has_feature;
    const uint8_t* reliable;
    const float* s_pca;
    const float* q_pca;
    const float* depth;
    const uint8_t* inside;
    float fx;
    unsigned int* count;    // #(reliable and not valid)
    float opacity_logit0;
    float *means, *log_scales, *quats, *logits, *sh;   // output planes
    int32_t* branch;
    float* beta_out;
};

__device__ __forceinline__ bool model_valid(const CascadeArgs& a, int64_t i) {
    if (!a.y || !a.has_feature[i] || !a.inside[i]) return false;
    const float* y = a.y + 16 * (size_t)i;
#pragma unroll
    for (int k = 0; k < 11; k++)
        if (!isfinite(y[k])) return false;
#pragma unroll
    for (int k = 0; k < 3; k++)
        if (!(fabsf(y[k]) < 3.f)) return false;
    return true;
}

__global__ void cascade_count_kernel(CascadeArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned int c = 0;
    if (i < a.n) c = (a.reliable[i] && !model_valid(a, i)) ? 1u : 0u;
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(a.count, c);
}

__global__ void cascade_assign_kernel(CascadeArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = a.n;
    const float beta = fminf(1.f, fmaxf(0.25f, (float)(*a.count) / (float)(n > 0 ? n : 1)));
    if (i == 0 && a.beta_out) *a.beta_out = beta;
    if (i >= n) return;
    float ls[3], q[4] = {1.f, 0.f, 0.f, 0.f}, col[3], lo = a.opacity_logit0;
#pragma unroll
    for (int k = 0; k < 3; k++) col[k] = a.rgb[(int64_t)k * n + i];
    int br = 0;
    if (model_valid(a, i)) {
        const float* y = a.y + 16 * (size_t)i;
        float qq[4], nq = 0.f;
#pragma unroll
        for (int k = 0; k < 4; k++) { qq[k] = a.q_pca[4 * (size_t)i + k] + y[3 + k]; nq += qq[k] * qq[k]; }
        nq = rsqrtf(nq);
#pragma unroll
        for (int k = 0; k < 4; k++) q[k] = qq[k] * nq;
#pragma unroll
        for (int k = 0; k < 3; k++) { ls[k] = a.s_pca[3 * (size_t)i + k] + y[k]; col[k] += y[8 + k]; }
        lo += y[7];
        br = 2;
    } else if (a.reliable[i]) {
        const float lb = logf(beta);
#pragma unroll
        for (int k = 0; k < 3; k++) ls[k] = a.s_pca[3 * (size_t)i + k] + lb;
#pragma unroll
        for (int k = 0; k < 4; k++) q[k] = a.q_pca[4 * (size_t)i + k];
        br = 1;
    } else {
        const float s = logf(fmaxf(a.depth[i], 1e-6f) / a.fx);
#pragma unroll
        for (int k = 0; k < 3; k++) ls[k] = s;
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        a.means[(int64_t)k * n + i] = a.pts[(int64_t)k * n + i];
        a.log_scales[(int64_t)k * n + i] = ls[k];
    }
#pragma unroll
    for (int k = 0; k < 4; k++) a.quats[(int64_t)k * n + i] = q[k];
    a.logits[i] = lo;
#pragma unroll
    for (int c = 0; c < 3; c++) a.sh[(int64_t)c * n + i] = (col[c] - 0.5f) / kY00;
    for (int k = 3; k < 3 * a.K; k++) a.sh[(int64_t)k * n + i] = 0.f;
    if (a.branch) a.branch[i] = br;
}

cudaError_t launch_cascade(const CascadeArgs& a, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(a.count, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    const int blocks = (int)((a.n + 255) / 256);
    if (blocks > 0) cascade_count_kernel<<<blocks, 256, 0, st>>>(a);
    cascade_assign_kernel<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gs

using namespace gs;

namespace gs {
gs_status record_error(gs_status s, const char* msg);
}

extern "C" size_t gs_pca_workspace_size(int64_t n) { return n > 0 ? pca_workspace_size(n) : 256; }

extern "C" gs_status gs_voxel_pca(const float* pts, const float* rgb, int64_t n, const gs_camera* frames,
                                  int32_t n_frames, const gs_pca_opts* opts, void* ws, size_t ws_bytes, float* x_out,
                                  uint8_t* has_feature, uint8_t* reliable, float* s_pca, float* q_pca, float* depth,
                                  uint8_t* inside, void* stream) {
    if (n < 0 || n > 0xFFFFFFFFll) return record_error(GS_ERR_INVALID_ARG, "n out of range");
    if (!frames || !opts) return record_error(GS_ERR_INVALID_ARG, "frames / opts is NULL");
    if (n_frames < 1 || n_frames > GS_MAX_VIEWS) return record_error(GS_ERR_INVALID_ARG, "n_frames must be in [1, 32]");
    FrameSet fs;
    memset(&fs, 0, sizeof(fs));
    fs.n = n_frames;
    for (int f = 0; f < n_frames; f++) {
        if (!(frames[f].fx > 0.f) || !(frames[f].fy > 0.f)) return record_error(GS_ERR_INVALID_ARG, "focal lengths must be > 0");
        fs.cam[f] = frames[f];
    }
    if (n == 0) return GS_OK;
    if (!pts || !rgb || !ws || !x_out || !has_feature || !reliable || !s_pca || !q_pca || !depth || !inside)
        return record_error(GS_ERR_INVALID_ARG, "NULL buffer");
    if (ws_bytes < pca_workspace_size(n)) return record_error(GS_ERR_INVALID_ARG, "PCA workspace too small");
    if (!(opts->voxel > 0.f) || opts->min_pts < 1) return record_error(GS_ERR_INVALID_ARG, "bad PCA options");
    cudaError_t e = launch_voxel_pca(pts, rgb, n, fs, opts->voxel, opts->min_pts, opts->tau_p, opts->tau_l,
                                     opts->sigma, opts->tau_trace, ws, x_out, has_feature, reliable, s_pca, q_pca,
                                     depth, inside, (cudaStream_t)stream);
    if (e != cudaSuccess) return record_error(GS_ERR_CUDA, cudaGetErrorString(e));
    return GS_OK;
}

extern "C" gs_status gs_init_cascade(const float* pts, const float* rgb, int64_t n, const float* y,
                                     const uint8_t* has_feature, const uint8_t* reliable, const float* s_pca,
                                     const float* q_pca, const float* depth, const uint8_t* inside, float fx,
                                     float opacity_init, gs_gaussians* out, int32_t* branch, unsigned int* count_tmp,
                                     float* beta_out, void* stream) {
    if (!out || out->n != n || n < 0) return record_error(GS_ERR_INVALID_ARG, "output map must have n Gaussians");
    if (out->sh_degree < 0 || out->sh_degree > 3) return record_error(GS_ERR_INVALID_ARG, "sh_degree must be 0..3");
    if (!(opacity_init > 0.f && opacity_init < 1.f)) return record_error(GS_ERR_INVALID_ARG, "opacity_init in (0,1)");
    if (n > 0 && (!pts || !rgb || !has_feature || !reliable || !s_pca || !q_pca || !depth || !inside || !count_tmp ||
                  !out->means || !out->log_scales || !out->quats || !out->opacity_logits || !out->sh))
        return record_error(GS_ERR_INVALID_ARG, "NULL buffer");
    CascadeArgs a;
    a.n = n;
    a.K = (out->sh_degree + 1) * (out->sh_degree + 1);
    a.pts = pts; a.rgb = rgb; a.y = y; a.has_feature = has_feature; a.reliable = reliable;
    a.s_pca = s_pca; a.q_pca = q_pca; a.depth = depth; a.inside = inside; a.fx = fx;
    a.count = count_tmp;
    a.opacity_logit0 = logf(opacity_init / (1.f - opacity_init));
    a.means = out->means; a.log_scales = out->log_scales; a.quats = out->quats; a.logits = out->opacity_logits;
    a.sh = out->sh;
    a.branch = branch;
    a.beta_out = beta_out;
    cudaError_t e = launch_cascade(a, (cudaStream_t)stream);
    if (e != cudaSuccess) return record_error(GS_ERR_CUDA, cudaGetErrorString(e));
    return GS_OK;
}
