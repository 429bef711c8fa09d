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
    uint32_t* vis_bits;    // [V][ceil(n/32)] bit i % 32 of word v * ceil(n/32) + i / 32: view v
                           //   covers a tile of Gaussian i
    uint8_t* visible;      // [n]
    Counters* counters;    // status word: GS_ERR_NONFINITE on a non-finite parameter
};

struct ProjectBwdArgs {
    int64_t n;
    int n_views;
    const View* views;
    Opts op;
    const float *means, *log_scales, *quats, *logits, *sh;
    const uint32_t* vis_bits; // [V][ceil(n/32)] per-view visibility words (ProjectArgs)
    const uint8_t* visible;   // [n] covers a tile of some view (rows without it are skipped)
    const uint32_t* entries;  // visible (view, Gaussian) entries in (view, Gaussian) order
    const Counters* counters; // n_entries
    const float4* grad2d;  // [V*n][3] screen-space sums
    float4* geo2d;         // [V*n][3] per-entry geometry gradients (entry part -> row part)
    float* dirgrad;        // [3][n] view-direction gradient of the mean (SH part -> geometry part)
    float *g_means, *g_log_scales, *g_quats, *g_logits, *g_sh;
    float* grad_twist;     // [V][6] or null
    // fused Adam (fused_adam != 0): parameters updated in place, gradients not stored
    int fused_adam;
    float *p_means, *p_log_scales, *p_quats, *p_logits, *p_sh;
    float* m[5];
    float* v[5];
    const uint8_t* update_mask;
    float lr[6];
    float b1, b2, eps, bc1, bc2;
    const Counters* step_dev;   // if set, bias corrections come from this device counter block
};

// Binning in two sorts: the visible (view, Gaussian) entries by depth, then their pairs by tile.
struct BinArgs {
    int64_t n;
    int n_views;
    const View* views;
    int tile;
    int64_t max_pairs;
    const float4* proj;
    const uint32_t* vis_bits;     // [V][ceil(n/32)] per-view visibility words (ProjectArgs)
    uint32_t* scan_tmp;           // block sums of the scans
    uint32_t* ekeys;              // compaction output: bits(z) of each entry
    uint32_t* evals;              //   and its compact index (the value the depth sort carries)
    uint32_t* entries;            //   view * n + Gaussian index of each entry, (view, Gaussian) order
    uint2* erect;                 //   its tile rectangle: (first global tile id, wx | wy << 16)
    const uint32_t* sorted_evals; // compact indices of the entries in depth order
    uint32_t* pkeys;              // emission output: global tile id of each pair
    uint32_t* pvals;              //   and the entry's view * n + Gaussian index
    uint32_t* poff;               // [n_views * n] pair offset of each depth-sorted entry
    uint32_t* chunk_first;        // [max_pairs / kEmitChunk + 2] entry of each chunk's first pair
    uint32_t* srt;                // [3][n_views * n] the depth-sorted entries' first tile ids,
                                  //   tile spans (wx | wy << 16) and view * n + index (scratch)
    Counters* counters;
};

// Stable LSD radix sort of (key, value) pairs with 8-bit digits; pass p reads buffer
// (p & 1) of keys / vals and writes the other.  Keys are uint32 or uint64 per the launcher.
struct SortArgs {
    void* keys[2];
    uint32_t* vals[2];
    uint32_t* hist;            // [256][grid] block histograms, then block offsets
    uint32_t* digit_tot;       // [256] digit totals
    const Counters* counters;  // status word (a set status skips the sort)
    const unsigned long long* count;   // element count, read on the device
    int grid;
    uint32_t digit_mask = 0xFFFFFFFFu;  // ANDed into every digit of the pass (a partial top digit)
};

struct RangeArgs {
    const uint32_t* keys;      // sorted global tile ids
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
    Counters* counters;
    uint8_t* pair_mask;        // [max_pairs] out: warp regions of its tile each pair can reach
    float* T_final;
    uint32_t* n_contrib;
    float *out_rgb, *out_depth, *out_T;
    const float *tgt_rgb, *tgt_depth;
    const uint8_t* mask;
    float *dl_drgb, *dl_ddepth;
    double* loss_sums;         // [V][3] (L1 rgb, L1 depth, SSIM)
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
    Counters* counters;
    const uint8_t* pair_mask;  // [max_pairs] from the forward
    const uint32_t* entries;   // visible (view, Gaussian) entries (counters->n_entries of them)
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

// The render-derived mask and the masked objective (objective.cu).
struct ObjArgs {
    int n_views;
    const View* views;
    int max_w, max_h;            // largest view size (grid extent)
    // interior mask
    const float* T_final;        // [P] from the forward
    const uint8_t* caller_mask;  // [P] or null
    uint8_t* mask_out;           // [P]
    float tau;                   // accumulated-opacity threshold
    int r_erode;                 // erosion disk radius (pixels)
    // objective over `mask`
    const float *rgb, *depth;    // rendered [3P] planar per view, [P]
    const float *tgt_rgb, *tgt_depth;
    const uint8_t* mask;         // [P] or null (all pixels)
    const uint32_t* counts;      // [V][2] |M|, |M and D~ > 0|
    double* sums;                // [V][3] L1 rgb, L1 depth, SSIM sums
    float *dl_drgb, *dl_ddepth;  // outputs (overwritten by the L1 terms, SSIM added)
    float* ssim_part;            // [9P] scratch, planar per view
    float lambda_rgb, lambda_depth, lambda_ssim;
    float win[11];               // 1-D Gaussian window
};
cudaError_t launch_render_mask(const ObjArgs& a, cudaStream_t st);
cudaError_t launch_objective(const ObjArgs& a, cudaStream_t st);
void ssim_window(float (&w)[11]);

// Map-size updates (mapupdate.cu).
constexpr int kMapMaxPlanes = 11 + 3 * 16;
struct MapUpdateArgs {
    int64_t n, n_new, n_out, n_keep;
    int n_planes;
    const uint8_t* keep;         // [n]
    const uint8_t* accept;       // [n_new] or null (all accepted)
    const uint32_t* pos_keep;    // exclusive scan of keep
    const uint32_t* pos_new;     // exclusive scan of accept (null: identity)
    const float* in[kMapMaxPlanes];
    const float* m_in[kMapMaxPlanes];
    const float* v_in[kMapMaxPlanes];
    const float* nw[kMapMaxPlanes];
    float* out[kMapMaxPlanes];
    float* m_out[kMapMaxPlanes];
    float* v_out[kMapMaxPlanes];
    const uint32_t *tags_in, *new_tags;
    uint32_t* tags_out;
};
size_t map_update_scratch_bytes(int64_t n_map, int64_t n_new);
cudaError_t launch_prune_plan(const float* logits, int64_t n, float thr, double max_ratio, uint8_t* keep,
                              void* scratch, unsigned long long* kept_host, cudaStream_t st);
cudaError_t launch_dedup_plan(const float* map_means, int64_t n, const float* new_means, int64_t nq, float radius,
                              uint8_t* accept, void* scratch, unsigned long long* accepted_host, cudaStream_t st);
cudaError_t launch_map_scan(const uint8_t* keep, int64_t n, const uint8_t* accept, int64_t n_new, void* scratch,
                            uint32_t** pos_keep, uint32_t** pos_new, uint32_t* totals_host, cudaStream_t st);
cudaError_t launch_compact(const MapUpdateArgs& a, cudaStream_t st);
// exclusive scan of n uint32 (bsum: ceil(n / 1024) + 1 words of scratch; total may be null)
cudaError_t exclusive_scan_u32(const uint32_t* x, int64_t n, uint32_t* out, uint32_t* bsum, uint32_t* total,
                               cudaStream_t st);

// Gaussian-GICP loop registration (gicp.cu).
struct GicpView {
    float R[9], t[3], c[3];       // world -> camera, and the camera centre (FP32)
    float fx, fy, cx, cy, W, H;
};
struct GicpMap {
    int64_t n;
    const float *means, *log_scales, *quats;   // [3][n], [3][n], [4][n]
};
size_t gicp_scratch_bytes(int64_t n_tar);
cudaError_t launch_gicp_target_set(const GicpMap& map, const GicpView* views, int n_views, float near_z, float dmax2,
                                   const uint8_t* source_flag, uint8_t* target_flag, void* scratch,
                                   unsigned long long* count_host, cudaStream_t st);
// builds the target hash (once per registration)
cudaError_t launch_gicp_build(const GicpMap& tar, const uint8_t* tar_flag, float d_corr, void* scratch, cudaStream_t st);
// accumulates H (21, upper triangle row-major), g (6), cost, count for transform (R, t) into
// 29 doubles copied to acc_host
cudaError_t launch_gicp_normal_eq(const GicpMap& src, const uint8_t* src_flag, const GicpMap& tar, float d_corr,
                                  const double* R, const double* t, void* scratch, double* acc_host, cudaStream_t st);

cudaError_t launch_project(const ProjectArgs& a, int deg, cudaStream_t st);
cudaError_t launch_project_bwd(const ProjectBwdArgs& a, int deg, cudaStream_t st);
// Compaction of the visible entries (their vis_bits set) in (view, Gaussian) order with their
// depth keys; the count goes to c->n_entries.
cudaError_t launch_entries(const BinArgs& a, cudaStream_t st);
// Pair offsets over the depth-sorted entries (total to c->n_pairs, GS_ERR_CAPACITY above
// max_pairs) and emission of one (tile id, entry) pair per covered tile.
cudaError_t launch_emit(const BinArgs& a, cudaStream_t st);
// 32-bit keys: pass p takes bits[p]-bit digits (8 or 9) at shifts[p]; 64-bit keys: 8-bit digits.
cudaError_t launch_sort32(const SortArgs& a, int n_passes, const int* shifts, const int* bits, cudaStream_t st);
cudaError_t launch_sort64(const SortArgs& a, int n_passes, const int* shifts, cudaStream_t st);
cudaError_t launch_ranges(const RangeArgs& a, int n_tiles, cudaStream_t st);
cudaError_t launch_tile_order(const uint2* ranges, int n_tiles, uint32_t* order, uint32_t* tmp, const Counters* c,
                              cudaStream_t st);
cudaError_t launch_loss_count(const View* views, int n_views, const int64_t* pix_counts_host,
                              const float* tgt_depth, const uint8_t* mask, uint32_t* counts, cudaStream_t st);
cudaError_t launch_render_fwd(const FwdArgs& a, int total_tiles, cudaStream_t st);
cudaError_t launch_loss_finalize(const double* sums, const uint32_t* counts, int n_views, float lambda_rgb,
                                 float lambda_depth, float lambda_ssim, int has_depth, float* loss_out,
                                 cudaStream_t st);
// The loss terms of the fused L1 loss (loss_finalize_one's arguments); loss_out null: none.
struct LossFinal {
    const double* sums = nullptr;
    const uint32_t* counts = nullptr;
    int n_views = 0;
    float lambda_rgb = 0.f, lambda_depth = 0.f;
    int has_depth = 0;
    float* loss_out = nullptr;
};
// Clears the gradient records of the visible entries (and, with adam_ctr, advances the fused
// step's Adam counter with adam_step_advance; with lf.loss_out, writes the loss terms as
// launch_loss_finalize does), then the backward compositing.
cudaError_t launch_render_bwd(const BwdArgs& a, int total_tiles, cudaStream_t st, Counters* adam_ctr = nullptr,
                              float b1 = 0.f, float b2 = 0.f, const LossFinal& lf = LossFinal());
cudaError_t launch_adam(const AdamArgs& a, cudaStream_t st);
// The persistent form of forward -> backward -> projection backward + Adam (render.cu); the
// grid state lives 128 bytes into the counters' 256-byte slot of the workspace.
cudaError_t launch_step_persistent(const FwdArgs& fwd, const BwdArgs& bwd, const ProjectBwdArgs& pb, int deg,
                                   int total_tiles, float lambda_rgb, float lambda_depth, int has_depth,
                                   float* loss_out, float b1, float b2, long long spin_limit, int skip_block,
                                   cudaStream_t st, int* grid_out);
cudaError_t launch_setup_views(View* dst, const View* src_host, int n_views, cudaStream_t st);

int sort_grid();

}  // namespace gs
