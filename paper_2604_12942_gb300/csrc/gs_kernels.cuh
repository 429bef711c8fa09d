// Kernel argument blocks and launchers shared between the translation units.
#pragma once

#include "gs_internal.cuh"

namespace gs {

struct ProjectArgs {
    int64_t n;
    int n_views;
    const View* views;
    Opts op;
    const float *means, *log_scales, *quats, *logits, *sh;
    float4* proj;          // [V*n][3]
    uint32_t* touched;     // [V*n]
    uint8_t* visible;      // [n]
};

struct ProjectBwdArgs {
    int64_t n;
    int n_views;
    const View* views;
    Opts op;
    const float *means, *log_scales, *quats, *logits, *sh;
    const uint32_t* touched;
    const float4* grad2d;  // [V*n][3]
    float *g_means, *g_log_scales, *g_quats, *g_logits, *g_sh;
    float* grad_twist;     // [V][6] or null
};

struct BinArgs {
    int64_t n;
    int n_views;
    const View* views;
    int tile;
    int64_t max_pairs;
    const float4* proj;
    const uint32_t* touched;
    uint32_t* offsets;
    uint32_t* scan_tmp;
    unsigned long long* keys;   // emission output (keys0)
    uint32_t* vals;
    Counters* counters;
};

struct SortArgs {
    unsigned long long* keys[2];
    uint32_t* vals[2];
    uint32_t* hist;            // [grid][256] block histograms, then offsets
    uint32_t* digit_tot;       // [256]
    Counters* counters;
    int grid;
};

struct RangeArgs {
    const unsigned long long* keys;
    uint2* ranges;
    Counters* counters;
};

struct FwdArgs {
    int n_views;
    const View* views;
    Opts op;
    const float4* proj;
    const uint32_t* vals;
    const uint2* ranges;
    const uint32_t* order;     // work order of the (view, tile) items, or null (identity)
    const Counters* counters;
    float* T_final;
    uint32_t* n_contrib;
    float *out_rgb, *out_depth, *out_T;
    const float *tgt_rgb, *tgt_depth;
    const uint8_t* mask;
    float *dl_drgb, *dl_ddepth;
    double* loss_sums;         // [V][2]
    const uint32_t* loss_counts;  // [V][2]
};

struct BwdArgs {
    int n_views;
    const View* views;
    Opts op;
    const float4* proj;
    const uint32_t* vals;
    const uint2* ranges;
    const uint32_t* order;
    const Counters* counters;
    const float* T_final;
    const uint32_t* n_contrib;
    const float *dl_drgb, *dl_ddepth;
    float4* grad2d;
};

struct AdamArgs {
    int64_t n;
    int n_planes;
    float* p[5];
    float* g[5];
    float* m[5];
    float* v[5];
    int planes_of[5];          // planes in each group pointer (3, 3, 4, 1, 3K)
    const uint8_t* update_mask;
    const uint8_t* visible;
    float lr[6];
    float b1, b2, eps, bc1, bc2;
    const Counters* step_dev;   // if set, bias corrections come from this device counter block
};

cudaError_t launch_project(const ProjectArgs& a, int deg, cudaStream_t st);
cudaError_t launch_project_bwd(const ProjectBwdArgs& a, int deg, cudaStream_t st);
cudaError_t launch_bin(const BinArgs& a, cudaStream_t st);
// Exclusive scan of n uint32 values; the total goes to c->n_pairs (status GS_ERR_CAPACITY if it
// exceeds max_total).  tmp holds n / 4096 + 2 values.
cudaError_t launch_exclusive_scan(const uint32_t* in, int64_t n, uint32_t* out, uint32_t* tmp, Counters* c,
                                  int64_t max_total, cudaStream_t st);
cudaError_t launch_sort(const SortArgs& a, int n_passes, const int* shifts, cudaStream_t st);
cudaError_t launch_ranges(const RangeArgs& a, int n_tiles, cudaStream_t st);
cudaError_t launch_tile_order(const uint2* ranges, int n_tiles, uint32_t* order, uint32_t* tmp, const Counters* c,
                              cudaStream_t st);
cudaError_t launch_loss_count(const View* views, int n_views, const int64_t* pix_counts_host,
                              const float* tgt_depth, const uint8_t* mask, uint32_t* counts, cudaStream_t st);
cudaError_t launch_render_fwd(const FwdArgs& a, int total_tiles, cudaStream_t st);
cudaError_t launch_loss_finalize(const double* sums, const uint32_t* counts, int n_views, float lambda_rgb,
                                 float lambda_depth, int has_depth, float* loss_out, cudaStream_t st);
cudaError_t launch_render_bwd(const BwdArgs& a, int total_tiles, cudaStream_t st);
cudaError_t launch_adam(const AdamArgs& a, cudaStream_t st);
cudaError_t launch_adam_step_counter(Counters* c, float b1, float b2, cudaStream_t st);
cudaError_t launch_setup_views(View* dst, const View* src_host, int n_views, cudaStream_t st);

int sort_grid();

}  // namespace gs
