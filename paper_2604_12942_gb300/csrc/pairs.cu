// a12, pair generation: training pairs of the learned initialiser from the plain mapping loop.
// RMGS-SLAM §III-B's learned branch predicts Gaussian attributes; here the model (the MLP of
// mlp.cu) predicts residuals on top of the voxel-PCA / heuristic initialisation, and its
// targets are what the plain loop changed: the optimised map minus the initial map, in the
// model's output units.  Rows whose point has a voxel feature and lies inside the loopframe
// (the rows whose model prediction the cascade can use) are kept, in row order.
//
// Per kept row i (FP32, every operation rounded once):
//   y[0..2]  = s_opt - s_init                     (log-scales)
//   y[3..6]  = q_opt / |q_opt| - q_init / |q_init| after giving both w >= 0 (sign flip of
//              the whole normalised quaternion when w < 0)
//   y[7]     = logit_opt - logit_init
//   y[8..10] = (sh_opt[c] - sh_init[c]) * Y00     (DC colour, c = r, g, b)
//   y[11..15] = 0
// and x_out = the row's 16 features.
#include "gs_kernels.cuh"

namespace gs {

constexpr int kPairThreads = 256;

struct PairArgs {
    int64_t n;
    const float* init[5];      // means, log_scales, quats, logits, sh of the initial map
    const float* opt[5];       // the same planes of the optimised map
    const float* x;            // [n][16]
    const uint8_t* has_feature;
    const uint8_t* inside;
    float* x_out;              // [n_kept][16]
    float* y_out;              // [n_kept][16]
    uint32_t* block_count;     // [blocks]
    uint32_t* block_off;       // [blocks + 1]
};

__device__ __forceinline__ bool pair_kept(const PairArgs& a, int64_t i) {
    return i < a.n && (!a.has_feature || a.has_feature[i]) && (!a.inside || a.inside[i]);
}

__global__ void __launch_bounds__(kPairThreads) pair_count_kernel(PairArgs a) {
    const int64_t i = (int64_t)blockIdx.x * kPairThreads + threadIdx.x;
    const int c = __syncthreads_count(pair_kept(a, i));
    if (threadIdx.x == 0) a.block_count[blockIdx.x] = (uint32_t)c;
}

// exclusive scan of the block counts by one block (the counts are few: n / 256)
__global__ void __launch_bounds__(1024) pair_scan_kernel(PairArgs a, int blocks) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int b0 = 0; b0 < blocks; b0 += 1024) {
        const int b = b0 + (int)threadIdx.x;
        const uint32_t c = b < blocks ? a.block_count[b] : 0u;
        uint32_t inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) s_warp[w] = inc;
        __syncthreads();
        if (w == 0) {
            uint32_t s = s_warp[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += t;
            }
            s_warp[lane] = s;   // inclusive over warps
        }
        __syncthreads();
        const uint32_t before = s_carry + (w > 0 ? s_warp[w - 1] : 0u) + inc - c;
        if (b < blocks) a.block_off[b] = before;
        __syncthreads();
        if (threadIdx.x == 1023) s_carry = before + c;
        __syncthreads();
    }
    if (threadIdx.x == 0) a.block_off[blocks] = s_carry;
}

__global__ void __launch_bounds__(kPairThreads) pair_write_kernel(PairArgs a) {
    __shared__ uint32_t s_warp[kPairThreads / 32];
    const int64_t i = (int64_t)blockIdx.x * kPairThreads + threadIdx.x;
    const bool keep = pair_kept(a, i);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) s_warp[w] = __popc(bal);
    __syncthreads();
    uint32_t off = a.block_off[blockIdx.x];
    for (int k = 0; k < w; k++) off += s_warp[k];
    off += __popc(bal & ((1u << lane) - 1u));
    if (!keep) return;
    const int64_t n = a.n;
    float y[16];
#pragma unroll
    for (int k = 0; k < 16; k++) y[k] = 0.f;
#pragma unroll
    for (int k = 0; k < 3; k++) y[k] = __fsub_rn(a.opt[1][k * n + i], a.init[1][k * n + i]);
    float qi[4], qo[4];
#pragma unroll
    for (int k = 0; k < 4; k++) { qi[k] = a.init[2][k * n + i]; qo[k] = a.opt[2][k * n + i]; }
    auto unit_w_pos = [](float (&q)[4]) {
        const float nrm = __fsqrt_rn(__fmaf_rn(q[3], q[3], __fmaf_rn(q[2], q[2], __fmaf_rn(q[1], q[1], __fmul_rn(q[0], q[0])))));
        const float s = q[0] < 0.f ? -1.f : 1.f;   // the sign of w is that of the stored component
#pragma unroll
        for (int k = 0; k < 4; k++) q[k] = __fdiv_rn(s * q[k], nrm);
    };
    unit_w_pos(qi);
    unit_w_pos(qo);
#pragma unroll
    for (int k = 0; k < 4; k++) y[3 + k] = __fsub_rn(qo[k], qi[k]);
    y[7] = __fsub_rn(a.opt[3][i], a.init[3][i]);
#pragma unroll
    for (int c = 0; c < 3; c++) y[8 + c] = __fmul_rn(__fsub_rn(a.opt[4][c * n + i], a.init[4][c * n + i]), SH0);
    const float4* xs = reinterpret_cast<const float4*>(a.x + 16 * i);
    float4* xd = reinterpret_cast<float4*>(a.x_out + 16 * (size_t)off);
    float4* yd = reinterpret_cast<float4*>(a.y_out + 16 * (size_t)off);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        xd[k] = __ldg(xs + k);
        yd[k] = make_float4(y[4 * k], y[4 * k + 1], y[4 * k + 2], y[4 * k + 3]);
    }
}

gs_status record_error(gs_status s, const char* msg);

static int64_t pair_blocks(int64_t n) { return (n + kPairThreads - 1) / kPairThreads; }

}  // namespace gs

using namespace gs;

extern "C" size_t gs_init_residuals_scratch_bytes(int64_t n) {
    if (n < 0) return 0;
    const int64_t b = pair_blocks(n);
    return (size_t)(((2 * b + 1) * sizeof(uint32_t) + 255) & ~(size_t)255) + 256;
}

extern "C" gs_status gs_init_residuals(const gs_gaussians* init, const gs_gaussians* opt, const float* x,
                                       const uint8_t* has_feature, const uint8_t* inside, float* x_out, float* y_out,
                                       int64_t* n_out, void* scratch, size_t scratch_bytes, void* stream) {
    if (!init || !opt || !n_out) return record_error(GS_ERR_INVALID_ARG, "init, opt and n_out are required");
    if (init->n != opt->n || init->n < 0) return record_error(GS_ERR_INVALID_ARG, "init and opt must have the same n");
    if (init->sh_degree < 0 || init->sh_degree > GS_MAX_SH_DEGREE || opt->sh_degree != init->sh_degree)
        return record_error(GS_ERR_INVALID_ARG, "bad or different sh_degree");
    const int64_t n = init->n;
    *n_out = 0;
    if (n == 0) return GS_OK;
    if (n >= (int64_t)1 << 31) return record_error(GS_ERR_INVALID_ARG, "n must be < 2^31");
    if (!x || !x_out || !y_out || !scratch) return record_error(GS_ERR_INVALID_ARG, "x, x_out, y_out and scratch are required");
    if (!init->log_scales || !init->quats || !init->opacity_logits || !init->sh || !opt->log_scales || !opt->quats ||
        !opt->opacity_logits || !opt->sh)
        return record_error(GS_ERR_INVALID_ARG, "a parameter plane is NULL");
    if (scratch_bytes < gs_init_residuals_scratch_bytes(n)) return record_error(GS_ERR_INVALID_ARG, "scratch too small");
    if (reinterpret_cast<uintptr_t>(x) % 16 || reinterpret_cast<uintptr_t>(x_out) % 16 ||
        reinterpret_cast<uintptr_t>(y_out) % 16)
        return record_error(GS_ERR_INVALID_ARG, "x, x_out and y_out must be 16-byte aligned");
    PairArgs a;
    a.n = n;
    const gs_gaussians* src[2] = {init, opt};
    for (int s = 0; s < 2; s++) {
        const float** d = s ? a.opt : a.init;
        d[0] = src[s]->means; d[1] = src[s]->log_scales; d[2] = src[s]->quats;
        d[3] = src[s]->opacity_logits; d[4] = src[s]->sh;
    }
    a.x = x; a.has_feature = has_feature; a.inside = inside; a.x_out = x_out; a.y_out = y_out;
    const int64_t blocks = pair_blocks(n);
    a.block_count = static_cast<uint32_t*>(scratch);
    a.block_off = a.block_count + blocks;
    cudaStream_t st = (cudaStream_t)stream;
    pair_count_kernel<<<(unsigned)blocks, kPairThreads, 0, st>>>(a);
    pair_scan_kernel<<<1, 1024, 0, st>>>(a, (int)blocks);
    pair_write_kernel<<<(unsigned)blocks, kPairThreads, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return record_error(GS_ERR_CUDA, cudaGetErrorString(e));
    uint32_t total = 0;
    e = cudaMemcpyAsync(&total, a.block_off + blocks, sizeof(total), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return record_error(GS_ERR_CUDA, cudaGetErrorString(e));
    *n_out = (int64_t)total;
    return GS_OK;
}
