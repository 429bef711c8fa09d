// a11-a12: the learned Gaussian initialiser's MLP (16 -> 128 -> 128 -> 128 -> 16, GELU),
// BF16 weights and activations with FP32 accumulation on the tensor cores
// (mma.sync m16n8k16), inference and one training step (MSE, backward GEMMs, Adam on FP32
// master weights).  It stands in for the paper's pretrained feed-forward model (§III-B).
//
// Parameters, packed:  weights BF16 [36864] = W1 (128x16) | W2 (128x128) | W3 (128x128) |
// W4 (16x128), each row-major [out][in];  biases FP32 [400] = b1 (128) | b2 | b3 | b4 (16).
#include <cuda_bf16.h>

#include "gs_kernels.cuh"

namespace gs {

constexpr int kIn = 16, kHid = 128, kOut = 16, kOutUsed = 11;
constexpr int kNW = 2048 + 32768 + 2048;
constexpr int kNB = 400;
__host__ __device__ __forceinline__ int woff(int l) { return l == 0 ? 0 : l == 1 ? 2048 : l == 2 ? 2048 + 16384 : 2048 + 32768; }
__host__ __device__ __forceinline__ int boff(int l) { return 128 * l; }
constexpr int kRows = 128;   // rows per CTA iteration (8 warps x 16)
constexpr int kThreads = 256;
constexpr int kLdIn = kIn + 8, kLdHid = kHid + 8;   // padded smem strides (bf16 elements)

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// acc += A (16x16) * B (16x8) with A(m, k) = A0[m*sam + k*sak] and B(k, n) = B0[k*sbk + n*sbn]
// (BF16 in shared memory), FP32 accumulate.  Fragment layout of mma.m16n8k16 (row.col):
// lane = 4 g + t; A regs {(g, 2t..2t+1), (g+8, 2t..), (g, 2t+8..), (g+8, 2t+8..)}, B regs
// {(2t..2t+1, g), (2t+8.., g)}, C {(g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1)}.
__device__ __forceinline__ void mma_tile(float acc[4], const bf16* A0, int sam, int sak, const bf16* B0, int sbk,
                                         int sbn) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    auto A = [&](int m, int k) { return A0[m * sam + k * sak]; };
    auto B = [&](int k, int n) { return B0[k * sbk + n * sbn]; };
    const uint32_t a0 = pack2(A(g, 2 * t), A(g, 2 * t + 1));
    const uint32_t a1 = pack2(A(g + 8, 2 * t), A(g + 8, 2 * t + 1));
    const uint32_t a2 = pack2(A(g, 2 * t + 8), A(g, 2 * t + 9));
    const uint32_t a3 = pack2(A(g + 8, 2 * t + 8), A(g + 8, 2 * t + 9));
    const uint32_t b0 = pack2(B(2 * t, g), B(2 * t + 1, g));
    const uint32_t b1 = pack2(B(2 * t + 8, g), B(2 * t + 9, g));
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(acc[0]), "+f"(acc[1]), "+f"(acc[2]), "+f"(acc[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.3989422804014327f;
}

struct MlpSmem {
    bf16 w1[kHid * kLdIn];
    bf16 w2[kHid * kLdHid];
    bf16 w3[kHid * kLdHid];
    bf16 w4[kOut * kLdHid];
    float b[kNB];
    bf16 a0[kRows * kLdIn];
    bf16 a1[kRows * kLdHid];
    bf16 a2[kRows * kLdHid];
    bf16 a3[kRows * kLdHid];
};

__device__ void load_weights(MlpSmem& S, const bf16* w, const float* b) {
    for (int e = threadIdx.x; e < kHid * kIn; e += blockDim.x) S.w1[(e / kIn) * kLdIn + e % kIn] = w[woff(0) + e];
    for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x) {
        S.w2[(e / kHid) * kLdHid + e % kHid] = w[woff(1) + e];
        S.w3[(e / kHid) * kLdHid + e % kHid] = w[woff(2) + e];
    }
    for (int e = threadIdx.x; e < kOut * kHid; e += blockDim.x) S.w4[(e / kHid) * kLdHid + e % kHid] = w[woff(3) + e];
    for (int e = threadIdx.x; e < kNB; e += blockDim.x) S.b[e] = b[e];
}

// One layer for the warp's 16 rows: out[r][n] = sum_k in[r][k] W[n][k] + bias[n].  The
// result goes through `epi(row, col, value)` (each lane owns 4 values per 8-column tile).
template <int K, int N, typename Epi>
__device__ __forceinline__ void warp_layer(const bf16* in, int ldin, const bf16* W, int ldw, const float* bias, int r0,
                                           Epi epi) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll 2
    for (int n0 = 0; n0 < N; n0 += 8) {
        float acc[4] = {bias[n0 + 2 * t], bias[n0 + 2 * t + 1], bias[n0 + 2 * t], bias[n0 + 2 * t + 1]};
#pragma unroll
        for (int k0 = 0; k0 < K; k0 += 16) mma_tile(acc, in + r0 * ldin + k0, ldin, 1, W + n0 * ldw + k0, 1, ldw);
        epi(r0 + g, n0 + 2 * t, acc[0]);
        epi(r0 + g, n0 + 2 * t + 1, acc[1]);
        epi(r0 + g + 8, n0 + 2 * t, acc[2]);
        epi(r0 + g + 8, n0 + 2 * t + 1, acc[3]);
    }
}

// Forward of the warp's 16 rows from S.a0; hidden activations (BF16) kept in S.a1..a3,
// pre-activations optionally stored (FP32) for the backward, outputs through `out`.
template <typename Out>
__device__ __forceinline__ void warp_forward(MlpSmem& S, int r0, float* z1, float* z2, float* z3, int64_t row_base,
                                             int64_t n, Out out) {
    auto hid = [&](bf16* dst, float* zst) {
        return [=, &S](int r, int c, float v) {
            dst[r * kLdHid + c] = __float2bfloat16_rn(gelu(v));
            if (zst && row_base + r < n) zst[(row_base + r) * kHid + c] = v;
        };
    };
    warp_layer<kIn, kHid>(S.a0, kLdIn, S.w1, kLdIn, S.b + boff(0), r0, hid(S.a1, z1));
    __syncwarp();
    warp_layer<kHid, kHid>(S.a1, kLdHid, S.w2, kLdHid, S.b + boff(1), r0, hid(S.a2, z2));
    __syncwarp();
    warp_layer<kHid, kHid>(S.a2, kLdHid, S.w3, kLdHid, S.b + boff(2), r0, hid(S.a3, z3));
    __syncwarp();
    warp_layer<kHid, kOut>(S.a3, kLdHid, S.w4, kLdHid, S.b + boff(3), r0, out);
}

__device__ __forceinline__ void load_input_rows(MlpSmem& S, const float* x, int64_t row_base, int64_t n) {
    for (int e = threadIdx.x; e < kRows * kIn; e += blockDim.x) {
        const int r = e / kIn, c = e % kIn;
        const int64_t row = row_base + r;
        S.a0[r * kLdIn + c] = __float2bfloat16_rn(row < n ? x[row * kIn + c] : 0.f);
    }
}

__global__ void __launch_bounds__(kThreads) mlp_infer_kernel(const bf16* w, const float* b, const float* x, int64_t n,
                                                             float* y) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpSmem& S = *reinterpret_cast<MlpSmem*>(smem_raw);
    load_weights(S, w, b);
    const int r0 = (threadIdx.x >> 5) * 16;
    for (int64_t base = (int64_t)blockIdx.x * kRows; base < n; base += (int64_t)gridDim.x * kRows) {
        __syncthreads();
        load_input_rows(S, x, base, n);
        __syncthreads();
        warp_forward(S, r0, nullptr, nullptr, nullptr, base, n, [&](int r, int c, float v) {
            if (base + r < n) y[(base + r) * kOut + c] = v;
        });
    }
}

// Training, pass 1: forward with stored pre-activations and hidden activations; output
// gradient g4 = 2 (y - t) / (n * 11) on the 11 used outputs; loss sum.
__global__ void __launch_bounds__(kThreads) mlp_train_fwd_kernel(const bf16* w, const float* b, const float* x,
                                                                 const float* t, int64_t n, float* z1, float* z2,
                                                                 float* z3, float* g4, double* loss_sum) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpSmem& S = *reinterpret_cast<MlpSmem*>(smem_raw);
    load_weights(S, w, b);
    const int r0 = (threadIdx.x >> 5) * 16;
    double lsum = 0.0;
    const float scale = 2.f / ((float)n * (float)kOutUsed);
    for (int64_t base = (int64_t)blockIdx.x * kRows; base < n; base += (int64_t)gridDim.x * kRows) {
        __syncthreads();
        load_input_rows(S, x, base, n);
        __syncthreads();
        warp_forward(S, r0, z1, z2, z3, base, n, [&](int r, int c, float v) {
            const int64_t row = base + r;
            if (row >= n) return;
            float gv = 0.f;
            if (c < kOutUsed) {
                const float d = v - t[row * kOut + c];
                lsum += (double)d * (double)d;
                gv = scale * d;
            }
            g4[row * kOut + c] = gv;
        });
    }
    lsum = warp_sum(lsum);
    if ((threadIdx.x & 31) == 0 && lsum != 0.0) atomicAdd(loss_sum, lsum);
}

struct BwdSmem {
    bf16 w1[kHid * kLdIn];
    bf16 w2[kHid * kLdHid];
    bf16 w3[kHid * kLdHid];
    bf16 w4[kOut * kLdHid];
    bf16 act[kRows * kLdHid];     // a_{l-1} of the current layer (BF16, recomputed input side)
    bf16 g[kRows * kLdHid];       // g_l (BF16 operand)
    bf16 gn[kRows * kLdHid];      // g_{l-1} being formed
};

// Training, pass 2: per CTA rows, layer by layer from the output: weight / bias gradients
// (g_l^T a_{l-1}, reduced over the CTA's rows and added atomically) and the gradient of the
// previous layer's pre-activation g_{l-1} = (g_l W_l) * gelu'(z_{l-1}).
__global__ void __launch_bounds__(kThreads) mlp_train_bwd_kernel(const bf16* w, const float* x, int64_t n,
                                                                 const float* z1, const float* z2, const float* z3,
                                                                 const float* g4, float* gw, float* gb) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdSmem& S = *reinterpret_cast<BwdSmem*>(smem_raw);
    for (int e = threadIdx.x; e < kHid * kIn; e += blockDim.x) S.w1[(e / kIn) * kLdIn + e % kIn] = w[woff(0) + e];
    for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x) {
        S.w2[(e / kHid) * kLdHid + e % kHid] = w[woff(1) + e];
        S.w3[(e / kHid) * kLdHid + e % kHid] = w[woff(2) + e];
    }
    for (int e = threadIdx.x; e < kOut * kHid; e += blockDim.x) S.w4[(e / kHid) * kLdHid + e % kHid] = w[woff(3) + e];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
    const float* zs[4] = {nullptr, z1, z2, z3};
    const bf16* Ws[4] = {S.w1, S.w2, S.w3, S.w4};
    const int lds[4] = {kLdIn, kLdHid, kLdHid, kLdHid};
    for (int64_t base = (int64_t)blockIdx.x * kRows; base < n; base += (int64_t)gridDim.x * kRows) {
        __syncthreads();
        // g4 of the rows (16 columns)
        for (int e = threadIdx.x; e < kRows * kOut; e += blockDim.x) {
            const int r = e / kOut, c = e % kOut;
            const int64_t row = base + r;
            S.g[r * kLdHid + c] = __float2bfloat16_rn(row < n ? g4[row * kOut + c] : 0.f);
        }
        for (int l = 3; l >= 0; l--) {
            const int out_dim = l == 3 ? kOut : kHid, in_dim = l == 0 ? kIn : kHid;
            // a_{l-1}: the network input (l = 0) or gelu(z_l) of the previous layer, as BF16
            for (int e = threadIdx.x; e < kRows * in_dim; e += blockDim.x) {
                const int r = e / in_dim, c = e % in_dim;
                const int64_t row = base + r;
                float v = 0.f;
                if (row < n) v = (l == 0) ? x[row * kIn + c] : gelu(zs[l][row * kHid + c]);
                S.act[r * kLdHid + c] = __float2bfloat16_rn(v);
            }
            __syncthreads();
            // bias gradient: column sums of g_l
            for (int c = threadIdx.x; c < out_dim; c += blockDim.x) {
                float s = 0.f;
                for (int r = 0; r < kRows; r++) s += __bfloat162float(S.g[r * kLdHid + c]);
                if (s != 0.f) atomicAdd(&gb[boff(l) + c], s);
            }
            // weight gradient gW[o][i] = sum_r g[r][o] a[r][i]: M = out, N = in, K = rows
            const int mt = out_dim / 16, nt = in_dim / 8;
            for (int tile = warp; tile < mt * nt; tile += kThreads / 32) {
                const int o0 = (tile / nt) * 16, i0 = (tile % nt) * 8;
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
                for (int r0 = 0; r0 < kRows; r0 += 16)
                    mma_tile(acc, S.g + r0 * kLdHid + o0, 1, kLdHid, S.act + r0 * kLdHid + i0, kLdHid, 1);
                float* dst = gw + woff(l);
                atomicAdd(&dst[(o0 + gq) * in_dim + i0 + 2 * tq], acc[0]);
                atomicAdd(&dst[(o0 + gq) * in_dim + i0 + 2 * tq + 1], acc[1]);
                atomicAdd(&dst[(o0 + gq + 8) * in_dim + i0 + 2 * tq], acc[2]);
                atomicAdd(&dst[(o0 + gq + 8) * in_dim + i0 + 2 * tq + 1], acc[3]);
            }
            if (l == 0) break;
            // g_{l-1} = (g_l W_l) * gelu'(z_l): rows x in_dim, K = out_dim (each warp its 16 rows)
            const int r0 = warp * 16;
            for (int i0 = 0; i0 < in_dim; i0 += 8) {
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
                for (int k0 = 0; k0 < out_dim; k0 += 16)
                    mma_tile(acc, S.g + r0 * kLdHid + k0, kLdHid, 1, Ws[l] + k0 * lds[l] + i0, lds[l], 1);
                const int rr[4] = {r0 + gq, r0 + gq, r0 + gq + 8, r0 + gq + 8};
                const int cc[4] = {i0 + 2 * tq, i0 + 2 * tq + 1, i0 + 2 * tq, i0 + 2 * tq + 1};
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int64_t row = base + rr[q];
                    const float zz = row < n ? zs[l][row * kHid + cc[q]] : 0.f;
                    S.gn[rr[q] * kLdHid + cc[q]] = __float2bfloat16_rn(acc[q] * gelu_grad(zz));
                }
            }
            __syncthreads();
            for (int e = threadIdx.x; e < kRows * kHid; e += blockDim.x) {
                const int r = e / kHid, c = e % kHid;
                S.g[r * kLdHid + c] = S.gn[r * kLdHid + c];
            }
            __syncthreads();
        }
    }
}

// Adam on the FP32 master parameters (weights then biases), BF16 copy of the weights,
// gradients cleared.
__global__ void mlp_adam_kernel(float* master, bf16* wq, float* bias, float* gw, float* gb, float* m, float* v, float lr,
                                float b1, float b2, float eps, float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNW + kNB) return;
    const bool is_w = i < kNW;
    float g = is_w ? gw[i] : gb[i - kNW];
    float p = is_w ? master[i] : bias[i - kNW];
    const float mm = b1 * m[i] + (1.f - b1) * g;
    const float vv = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mm;
    v[i] = vv;
    p -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
    if (is_w) {
        master[i] = p;
        wq[i] = __float2bfloat16_rn(p);
        gw[i] = 0.f;
    } else {
        bias[i - kNW] = p;
        gb[i - kNW] = 0.f;
    }
}

static int mlp_grid(int64_t n) {
    const int sms = device_sms();
    const int64_t blocks = (n + kRows - 1) / kRows;
    return (int)(blocks < sms ? (blocks > 0 ? blocks : 1) : sms);
}

static bool g_mlp_attr[kMaxDevices] = {};
static cudaError_t mlp_attrs() {
    return once_per_device(g_mlp_attr, [] {
        cudaError_t e = cudaFuncSetAttribute(mlp_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(MlpSmem));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(mlp_train_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(MlpSmem));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(mlp_train_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(BwdSmem));
        return e;
    });
}

__global__ void mlp_loss_finalize_kernel(const double* s, int64_t n, float* out) {
    if (threadIdx.x == 0) *out = (float)(*s / ((double)n * kOutUsed));
}

gs_status record_error(gs_status s, const char* msg);

}  // namespace gs

using namespace gs;

extern "C" gs_status gs_mlp_infer(const uint16_t* w_bf16, const float* bias, const float* x, int64_t n, float* y,
                                  void* stream) {
    if (n < 0) return record_error(GS_ERR_INVALID_ARG, "n must be >= 0");
    if (n == 0) return GS_OK;
    if (!w_bf16 || !bias || !x || !y) return record_error(GS_ERR_INVALID_ARG, "NULL buffer");
    cudaError_t e = mlp_attrs();
    if (e != cudaSuccess) return record_error(GS_ERR_CUDA, cudaGetErrorString(e));
    mlp_infer_kernel<<<mlp_grid(n), kThreads, sizeof(MlpSmem), (cudaStream_t)stream>>>(
        reinterpret_cast<const bf16*>(w_bf16), bias, x, n, y);
    e = cudaGetLastError();
    return e == cudaSuccess ? GS_OK : record_error(GS_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" size_t gs_mlp_train_scratch_size(int64_t n) {
    // z1..z3 [n][128] FP32, g4 [n][16] FP32, loss sum (double)
    return sizeof(float) * (size_t)n * (3 * 128 + 16) + 256;
}

extern "C" gs_status gs_mlp_train_step(float* w_master, uint16_t* w_bf16, float* bias, float* grad_w, float* grad_b,
                                       float* adam_m, float* adam_v, const float* x, const float* y_target, int64_t n,
                                       float lr, float b1, float b2, float eps, int64_t step, void* scratch,
                                       size_t scratch_bytes, float* loss_out, void* stream) {
    if (n < 1) return record_error(GS_ERR_INVALID_ARG, "n must be >= 1");
    if (step < 1) return record_error(GS_ERR_INVALID_ARG, "step must be >= 1");
    if (!w_master || !w_bf16 || !bias || !grad_w || !grad_b || !adam_m || !adam_v || !x || !y_target || !scratch)
        return record_error(GS_ERR_INVALID_ARG, "NULL buffer");
    if (scratch_bytes < gs_mlp_train_scratch_size(n)) return record_error(GS_ERR_INVALID_ARG, "scratch too small");
    cudaError_t e = mlp_attrs();
    if (e != cudaSuccess) return record_error(GS_ERR_CUDA, cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)stream;
    float* z1 = static_cast<float*>(scratch);
    float* z2 = z1 + (size_t)n * 128;
    float* z3 = z2 + (size_t)n * 128;
    float* g4 = z3 + (size_t)n * 128;
    double* lsum = reinterpret_cast<double*>(
        (reinterpret_cast<uintptr_t>(g4 + (size_t)n * 16) + 15) & ~(uintptr_t)15);
    cudaMemsetAsync(lsum, 0, sizeof(double), st);
    const bf16* wq = reinterpret_cast<const bf16*>(w_bf16);
    const int grid = mlp_grid(n);
    mlp_train_fwd_kernel<<<grid, kThreads, sizeof(MlpSmem), st>>>(wq, bias, x, y_target, n, z1, z2, z3, g4, lsum);
    mlp_train_bwd_kernel<<<grid, kThreads, sizeof(BwdSmem), st>>>(wq, x, n, z1, z2, z3, g4, grad_w, grad_b);
    const float bc1 = (float)(1.0 - pow((double)b1, (double)step)), bc2 = (float)(1.0 - pow((double)b2, (double)step));
    mlp_adam_kernel<<<(kNW + kNB + 255) / 256, 256, 0, st>>>(w_master, reinterpret_cast<bf16*>(w_bf16), bias, grad_w,
                                                            grad_b, adam_m, adam_v, lr, b1, b2, eps, bc1, bc2);
    if (loss_out) mlp_loss_finalize_kernel<<<1, 32, 0, st>>>(lsum, n, loss_out);
    e = cudaGetLastError();
    return e == cudaSuccess ? GS_OK : record_error(GS_ERR_CUDA, cudaGetErrorString(e));
}

