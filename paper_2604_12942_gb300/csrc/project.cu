// a1 and a7: per-Gaussian EWA projection with SH colour, and its backward (chain rule to
// the Gaussian parameters and to each view's SE(3) pose twist).
// RMGS-SLAM §III-C ("standard differentiable Gaussian splatting"); gs.h documents the
// readings (near plane, dilation, Jacobian clamp, opacity-aware radius, SH convention).
#include "gs_kernels.cuh"

namespace gs {

// 8 blocks of 128 threads per SM (at most 64 registers a thread): the kernel waits on memory
// and gains more from resident warps than it loses to the few spilled values (3 blocks of 256
// without spills: 0.149 ms against 0.133 at 2M Gaussians, 8 views; 4 of 256: 0.136).
static_assert(sizeof(View) % 4 == 0, "the view table is copied in 4-byte words");

template <int DEG>
__global__ void __launch_bounds__(128, 8) project_kernel(ProjectArgs a) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    // the view table in shared memory: every thread walks all views, and the streamed planes
    // leave little of it in L1 (0.142 -> 0.136 ms at 2M Gaussians, 8 views)
    __shared__ View s_views[GS_MAX_VIEWS];
    {
        const int words = a.n_views * (int)(sizeof(View) / 4);
        const uint32_t* src = reinterpret_cast<const uint32_t*>(a.views);
        uint32_t* dst = reinterpret_cast<uint32_t*>(s_views);
        for (int t = threadIdx.x; t < words; t += blockDim.x) dst[t] = src[t];
    }
    __syncthreads();
    const int64_t n = a.n;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // Every lane reaches the ballots after the view loop (they build the visibility words);
    // lanes past n read row n - 1 and see nothing.  Blocks of 128 rows start on a word, so
    // the 32 lanes of a warp are the 32 rows of word i / 32 of each view.
    const bool in = i < n;
    const int64_t ii = in ? i : n - 1;
    float mu[3], ls[3], q[4];
#pragma unroll
    for (int k = 0; k < 3; k++) { mu[k] = __ldg(a.means + k * n + ii); ls[k] = __ldg(a.log_scales + k * n + ii); }
#pragma unroll
    for (int k = 0; k < 4; k++) q[k] = __ldg(a.quats + k * n + ii);
    const float logit = __ldg(a.logits + ii);
    // A non-finite parameter invalidates the step: the row is treated as unseen and the status
    // word becomes GS_ERR_NONFINITE, so the later stages of the step do nothing.
    bool finite = isfinite(logit);
#pragma unroll
    for (int k = 0; k < 3; k++) finite = finite && isfinite(mu[k]) && isfinite(ls[k]);
#pragma unroll
    for (int k = 0; k < 4; k++) finite = finite && isfinite(q[k]);
    if (in && !finite) set_status(a.counters, GS_ERR_NONFINITE);
    // geometry of every view first; the SH coefficients are then loaded only by rows that
    // some view sees (a row no view sees reads 11 of its 11 + 3K floats)
    uint32_t vis = 0;
    const Opts op = a.op;
    if (in && finite) {
        Cov3 cv;
        cov3_forward(q, ls, cv);
        for (int v = 0; v < a.n_views; v++) {
            const View& V = s_views[v];
            ProjV P;
            project_view(mu, cv, logit, V, op, P);
            if (P.culled) continue;
            int x0, x1, y0, y1;
            if (!tile_span(P.u, P.rx, op.tile, V.tiles_x, x0, x1) ||
                !tile_span(P.v, P.ry, op.tile, V.tiles_y, y0, y1))
                continue;
            const float idet = 1.0f / P.det;
            const float A = P.c * idet, B = -P.b * idet, C = P.a * idet;
            float4* rec = a.proj + 3 * ((int64_t)v * n + i);
            rec[0] = make_float4(P.u, P.v, P.pc[2], P.o);
            rec[1] = make_float4(kConicScale * A, kConicScale * B, kConicScale * C, __int_as_float(P.rx));
            rec[2].w = __int_as_float(P.ry);
            vis |= 1u << v;
        }
    }
    // view v's word of the warp's 32 rows goes to lane v, which stores it
    {
        const int lane = threadIdx.x & 31;
        const int64_t nw = (n + 31) >> 5;   // words per view
        const int64_t word = i >> 5;
        uint32_t mine = 0;
        for (int v = 0; v < a.n_views; v++) {
            const uint32_t bits = __ballot_sync(0xffffffffu, (vis >> v) & 1u);
            if (lane == v) mine = bits;
        }
        if (lane < a.n_views && word < nw) a.vis_bits[lane * nw + word] = mine;
    }
    if (in) a.visible[i] = vis ? 1 : 0;
    if (!vis) return;
    float sh[3 * K];
    bool sh_finite = true;
#pragma unroll
    for (int k = 0; k < 3 * K; k++) {
        sh[k] = __ldg(a.sh + k * n + i);
        sh_finite = sh_finite && isfinite(sh[k]);
    }
    if (!sh_finite) set_status(a.counters, GS_ERR_NONFINITE);
    // colour along each seeing view's direction
    for (uint32_t m = vis; m; m &= m - 1) {
        const int v = __ffs(m) - 1;
        const View& V = s_views[v];
        float d[3] = {mu[0] - V.cw[0], mu[1] - V.cw[1], mu[2] - V.cw[2]};
        const float rn = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        float Y[16];
        sh_basis<DEG>(d[0] * rn, d[1] * rn, d[2] * rn, Y);
        float rgb[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            float s = 0.5f;
#pragma unroll
            for (int k = 0; k < K; k++) s += sh[k * 3 + c] * Y[k];
            rgb[c] = fmaxf(s, 0.0f);
        }
        float* r2 = reinterpret_cast<float*>(a.proj + 3 * ((int64_t)v * n + i) + 2);
        r2[0] = rgb[0];
        r2[1] = rgb[1];
        r2[2] = rgb[2];
    }
}

}  // namespace gs

#include "project_bwd.cuh"

namespace gs {

__global__ void __launch_bounds__(kEntryThreads) project_bwd_entry_kernel(ProjectBwdArgs a) {
    __shared__ float s_tw[GS_MAX_VIEWS * 6];
    project_bwd_entry_part(a, blockIdx.x, gridDim.x, s_tw);
}

// The row part as two kernels (SH part, then geometry part; see project_bwd.cuh).  Blocks of
// 64 rows: a block whose rows no view sees ends at once, and small blocks keep the SMs' warp
// slots filled through the ragged end of the grid (128-row blocks: 0.549 ms against 0.539 at
// 2M Gaussians, 8 views).
constexpr int kRowThreads = 64;

template <int DEG, bool FUSED_ADAM>
__global__ void __launch_bounds__(kRowThreads, 10) project_bwd_sh_kernel(ProjectBwdArgs a) {
    __shared__ float s_tw[GS_MAX_VIEWS * 6];
    __shared__ float s_cam[GS_MAX_VIEWS * 12];
    __shared__ float s_mv[FUSED_ADAM ? sh_mv_floats<DEG, kRowThreads>() : 1];
    project_bwd_sh_rows<DEG, FUSED_ADAM, kRowThreads>(a, blockIdx.x, s_tw, s_mv, s_cam);
}

template <int DEG, bool FUSED_ADAM>
__global__ void __launch_bounds__(kRowThreads, 16) project_bwd_geo_kernel(ProjectBwdArgs a) {
    __shared__ float s_mv[FUSED_ADAM ? geo_mv_floats<kRowThreads>() : 1];
    project_bwd_geo_rows<DEG, FUSED_ADAM, kRowThreads>(a, blockIdx.x, s_mv);
}


cudaError_t launch_project(const ProjectArgs& a, int deg, cudaStream_t st) {
    const int threads = 128;
    const unsigned blocks = (unsigned)((a.n + threads - 1) / threads);
    if (blocks == 0) return cudaSuccess;
    switch (deg) {
        case 0: project_kernel<0><<<blocks, threads, 0, st>>>(a); break;
        case 1: project_kernel<1><<<blocks, threads, 0, st>>>(a); break;
        case 2: project_kernel<2><<<blocks, threads, 0, st>>>(a); break;
        default: project_kernel<3><<<blocks, threads, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

template <int DEG, bool FUSED_ADAM>
static cudaError_t launch_project_bwd_d(const ProjectBwdArgs& a, unsigned blocks, cudaStream_t st) {
    project_bwd_sh_kernel<DEG, FUSED_ADAM><<<blocks, kRowThreads, 0, st>>>(a);
    project_bwd_geo_kernel<DEG, FUSED_ADAM><<<blocks, kRowThreads, 0, st>>>(a);
    return cudaGetLastError();
}

template <bool FUSED_ADAM>
static cudaError_t launch_project_bwd_t(const ProjectBwdArgs& a, int deg, cudaStream_t st) {
    const unsigned blocks = (unsigned)((a.n + kRowThreads - 1) / kRowThreads);
    if (blocks == 0) return cudaSuccess;
    switch (deg) {
        case 0: return launch_project_bwd_d<0, FUSED_ADAM>(a, blocks, st);
        case 1: return launch_project_bwd_d<1, FUSED_ADAM>(a, blocks, st);
        case 2: return launch_project_bwd_d<2, FUSED_ADAM>(a, blocks, st);
        default: return launch_project_bwd_d<3, FUSED_ADAM>(a, blocks, st);
    }
}

cudaError_t launch_project_bwd(const ProjectBwdArgs& a, int deg, cudaStream_t st) {
    // entry part (persistent grid over the device-side entry count), then the row part's SH
    // and geometry kernels
    project_bwd_entry_kernel<<<sort_grid() * 4, kEntryThreads, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return a.fused_adam ? launch_project_bwd_t<true>(a, deg, st) : launch_project_bwd_t<false>(a, deg, st);
}

}  // namespace gs
