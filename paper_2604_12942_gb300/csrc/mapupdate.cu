// Map-size updates between mapping iterations (RMGS-SLAM §III-C): low-opacity pruning under a
// bounded removal ratio, the 3-D proximity test that filters redundant new Gaussians before
// insertion, and the compaction that applies both to the parameter planes, the Adam moments
// and an optional per-row tag (e.g. the segment id that decides which rows are frozen).
//
// Pruning picks, among the rows with opacity below opacity_min (decided on the FP32 logit),
// at most floor(max_ratio * n) rows with the smallest (logit, row index): a radix select of the
// k-th smallest 64-bit key (ordered logit bits, row index) in eight 8-bit rounds, each a
// histogram over the rows still matching the key prefix, then one marking pass.  No sort.
//
// The proximity test hashes the map means into cubic cells of side 1.001 * radius (a counting
// sort of row ids by cell hash); a new mean looks at the 27 cells around its own and is
// redundant if any map mean there lies strictly within radius (squared distance summed in FP32
// in x, y, z order).  Cells are computed in FP64 (a few operations per point) and are 0.1%
// wider than the radius, so two means closer than the radius never end up two cells apart.
#include "gs_kernels.cuh"

namespace gs {

constexpr int kMuThreads = 256;

struct SelectState {
    unsigned long long prefix;   // key bits decided so far
    unsigned long long count;    // candidates
    unsigned long long k;        // rows to remove
    unsigned long long rank;     // rank (1-based) of the threshold key inside the current prefix group
    unsigned long long kept;     // rows kept / new rows accepted
    uint32_t hist[256];
};

__device__ __forceinline__ unsigned long long prune_key(float logit, int64_t i) {
    const uint32_t b = __float_as_uint(logit);
    const uint32_t ord = (b >> 31) ? ~b : (b | 0x80000000u);   // monotone in the float value
    return ((unsigned long long)ord << 32) | (unsigned long long)(uint32_t)i;
}

__global__ void __launch_bounds__(kMuThreads) prune_count_kernel(const float* lg, int64_t n, float thr,
                                                                 SelectState* s) {
    uint32_t c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += lg[i] < thr;
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&s->count, (unsigned long long)c);
}

__global__ void prune_init_kernel(SelectState* s, unsigned long long k_max) {
    if (threadIdx.x < 256) s->hist[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        s->k = s->count < k_max ? s->count : k_max;
        s->rank = s->k;
        s->prefix = 0;
    }
}

// Round r: histogram of digit (7 - r) of the candidates' keys whose higher digits equal the
// prefix.
__global__ void __launch_bounds__(kMuThreads) prune_hist_kernel(const float* lg, int64_t n, float thr, int round,
                                                                SelectState* s) {
    __shared__ uint32_t h[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) h[t] = 0;
    __syncthreads();
    const int shift = 56 - 8 * round;
    const unsigned long long hi_mask = round == 0 ? 0ull : (~0ull << (shift + 8));
    const unsigned long long prefix = s->prefix;
    if (s->k > 0) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            const float x = lg[i];
            if (!(x < thr)) continue;
            const unsigned long long key = prune_key(x, i);
            if ((key & hi_mask) == (prefix & hi_mask)) atomicAdd(&h[(key >> shift) & 255u], 1u);
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 256; t += blockDim.x)
        if (h[t]) atomicAdd(&s->hist[t], h[t]);
}

// Picks the digit holding the rank-th key of the prefix group and clears the histogram.
__global__ void prune_pick_kernel(int round, SelectState* s) {
    if (threadIdx.x != 0) return;
    if (s->k > 0) {
        const int shift = 56 - 8 * round;
        unsigned long long below = 0;
        int d = 0;
        for (; d < 255; d++) {
            if (below + s->hist[d] >= s->rank) break;
            below += s->hist[d];
        }
        s->rank -= below;
        s->prefix |= (unsigned long long)d << shift;
    }
    for (int t = 0; t < 256; t++) s->hist[t] = 0;
}

__global__ void __launch_bounds__(kMuThreads) prune_mark_kernel(const float* lg, int64_t n, float thr,
                                                                SelectState* s, uint8_t* keep) {
    const unsigned long long k = s->k, t = s->prefix;
    uint32_t kept = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float x = lg[i];
        const bool drop = k > 0 && x < thr && prune_key(x, i) <= t;
        keep[i] = drop ? 0 : 1;
        kept += !drop;
    }
    kept = warp_sum(kept);
    if ((threadIdx.x & 31) == 0 && kept) atomicAdd(&s->kept, (unsigned long long)kept);
}

// ---------------------------------------------------------------------------------------
// Proximity test.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cell_hash(int cx, int cy, int cz, uint32_t mask) {
    // three large odd multipliers, XOR-combined, then the table's low bits
    return ((uint32_t)cx * 73856093u ^ (uint32_t)cy * 19349663u ^ (uint32_t)cz * 83492791u) & mask;
}

__device__ __forceinline__ int cell_of(float p, double inv_cell) { return (int)floor((double)p * inv_cell); }

__global__ void __launch_bounds__(kMuThreads) hash_count_kernel(const float* mm, int64_t n, double inv_cell,
                                                                uint32_t mask, uint32_t* count, uint32_t* cell_of_row) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t h = cell_hash(cell_of(mm[i], inv_cell), cell_of(mm[n + i], inv_cell),
                                     cell_of(mm[2 * n + i], inv_cell), mask);
        cell_of_row[i] = h;
        atomicAdd(&count[h], 1u);
    }
}

__global__ void __launch_bounds__(kMuThreads) hash_fill_kernel(int64_t n, const uint32_t* cell_of_row,
                                                               const uint32_t* start, uint32_t* cursor,
                                                               uint32_t* rows) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t h = cell_of_row[i];
        rows[start[h] + atomicAdd(&cursor[h], 1u)] = (uint32_t)i;
    }
}

__global__ void __launch_bounds__(kMuThreads) dedup_query_kernel(const float* mm, int64_t n, const float* qm,
                                                                 int64_t nq, double inv_cell, float r2, uint32_t mask,
                                                                 const uint32_t* start, const uint32_t* count,
                                                                 const uint32_t* rows, uint8_t* accept,
                                                                 SelectState* s) {
    uint32_t acc = 0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nq; j += (int64_t)gridDim.x * blockDim.x) {
        const float qx = qm[j], qy = qm[nq + j], qz = qm[2 * nq + j];
        const int cx = cell_of(qx, inv_cell), cy = cell_of(qy, inv_cell), cz = cell_of(qz, inv_cell);
        bool near = false;
        for (int dz = -1; dz <= 1 && !near; dz++)
            for (int dy = -1; dy <= 1 && !near; dy++)
                for (int dx = -1; dx <= 1 && !near; dx++) {
                    const uint32_t h = cell_hash(cx + dx, cy + dy, cz + dz, mask);
                    const uint32_t b = start[h], e = b + count[h];
                    for (uint32_t t = b; t < e; t++) {
                        const uint32_t i = rows[t];
                        const float ex = __fsub_rn(qx, mm[i]), ey = __fsub_rn(qy, mm[n + i]), ez = __fsub_rn(qz, mm[2 * n + i]);
                        const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
                        if (d2 < r2) { near = true; break; }
                    }
                }
        accept[j] = near ? 0 : 1;
        acc += !near;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(&s->kept, (unsigned long long)acc);
}

// ---------------------------------------------------------------------------------------
// Exclusive scan of uint32 (or uint8 flags) over up to 2^31 items: per-block totals, a scan of
// the totals in one block, then the per-item offsets.
// ---------------------------------------------------------------------------------------
constexpr int kScanT = 1024;

__device__ __forceinline__ uint32_t block_scan_excl(uint32_t x, uint32_t& total) {
    __shared__ uint32_t s_w[33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_w[w] = inc;
    __syncthreads();
    if (w == 0) {
        const uint32_t t = lane < (int)(blockDim.x >> 5) ? s_w[lane] : 0u;
        uint32_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        s_w[lane] = ti - t;
        if (lane == 31) s_w[32] = ti;
    }
    __syncthreads();
    total = s_w[32];
    const uint32_t r = s_w[w] + inc - x;
    __syncthreads();
    return r;
}

template <typename T>
__global__ void __launch_bounds__(kScanT) scan_totals_kernel(const T* x, int64_t n, uint32_t* bsum) {
    const int64_t i = (int64_t)blockIdx.x * kScanT + threadIdx.x;
    uint32_t tot;
    block_scan_excl(i < n ? (uint32_t)x[i] : 0u, tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanT) scan_bsum_kernel(uint32_t* bsum, int nb, uint32_t* total) {
    uint32_t carry = 0;
    for (int b0 = 0; b0 < nb; b0 += kScanT) {
        const int b = b0 + threadIdx.x;
        uint32_t tot;
        const uint32_t ex = block_scan_excl(b < nb ? bsum[b] : 0u, tot);
        if (b < nb) bsum[b] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

template <typename T>
__global__ void __launch_bounds__(kScanT) scan_apply_kernel(const T* x, int64_t n, const uint32_t* bsum,
                                                            uint32_t* out) {
    const int64_t i = (int64_t)blockIdx.x * kScanT + threadIdx.x;
    uint32_t tot;
    const uint32_t ex = block_scan_excl(i < n ? (uint32_t)x[i] : 0u, tot);
    if (i < n) out[i] = bsum[blockIdx.x] + ex;
}

template <typename T>
static cudaError_t exclusive_scan(const T* x, int64_t n, uint32_t* out, uint32_t* bsum, uint32_t* total,
                                  cudaStream_t st) {
    const int nb = (int)((n + kScanT - 1) / kScanT);
    if (nb > 0) scan_totals_kernel<T><<<nb, kScanT, 0, st>>>(x, n, bsum);
    scan_bsum_kernel<<<1, kScanT, 0, st>>>(bsum, nb, total);
    if (nb > 0) scan_apply_kernel<T><<<nb, kScanT, 0, st>>>(x, n, bsum, out);
    return cudaGetLastError();
}

cudaError_t exclusive_scan_u32(const uint32_t* x, int64_t n, uint32_t* out, uint32_t* bsum, uint32_t* total,
                               cudaStream_t st) {
    return exclusive_scan(x, n, out, bsum, total, st);
}

// ---------------------------------------------------------------------------------------
// Compaction: kept rows to their scanned positions, accepted new rows after them (with zero
// moments).  Every plane is passed by its own base pointer (input stride n, new rows n_new,
// output n_out).  One thread per row; the planes go in groups of 8, all 24 loads of a group
// (parameters, m, v) before its stores, so that a row has that many reads in flight instead
// of the three a plane at a time would give (the stores may alias later loads as far as the
// compiler knows, so it cannot reorder them itself).
// ---------------------------------------------------------------------------------------
constexpr int kCompactGroup = 8;

__global__ void __launch_bounds__(kMuThreads) compact_kernel(MapUpdateArgs a) {
    const int64_t total = a.n + a.n_new;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < total; r += (int64_t)gridDim.x * blockDim.x) {
        const bool old = r < a.n;
        const int64_t i = old ? r : r - a.n;
        if (old ? !a.keep[i] : (a.accept && !a.accept[i])) continue;
        const int64_t o = old ? (int64_t)a.pos_keep[i] : (int64_t)a.n_keep + (a.pos_new ? (int64_t)a.pos_new[i] : i);
        for (int p0 = 0; p0 < a.n_planes; p0 += kCompactGroup) {
            float x[kCompactGroup], mm[kCompactGroup], vv[kCompactGroup];
#pragma unroll
            for (int k = 0; k < kCompactGroup; k++) {
                const int p = p0 + k;
                if (p < a.n_planes) {
                    x[k] = old ? a.in[p][i] : a.nw[p][i];
                    mm[k] = old ? a.m_in[p][i] : 0.f;
                    vv[k] = old ? a.v_in[p][i] : 0.f;
                }
            }
#pragma unroll
            for (int k = 0; k < kCompactGroup; k++) {
                const int p = p0 + k;
                if (p < a.n_planes) {
                    a.out[p][o] = x[k];
                    a.m_out[p][o] = mm[k];
                    a.v_out[p][o] = vv[k];
                }
            }
        }
        if (a.tags_out) a.tags_out[o] = old ? (a.tags_in ? a.tags_in[i] : 0u) : (a.new_tags ? a.new_tags[i] : 0u);
    }
}

static int mu_grid(int64_t n) {
    int64_t b = (n + kMuThreads - 1) / kMuThreads;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

size_t map_update_scratch_bytes(int64_t n_map, int64_t n_new) {
    const int64_t m = n_map > n_new ? n_map : n_new;
    uint64_t T = 1;
    while (T < (uint64_t)(2 * (n_map > 0 ? n_map : 1))) T <<= 1;
    const size_t nb = (size_t)((m + kScanT - 1) / kScanT) + 1;
    const size_t nbT = (size_t)((T + kScanT - 1) / kScanT) + 1;
    const size_t prune = sizeof(SelectState);
    const size_t dedup = sizeof(SelectState) + sizeof(uint32_t) * (3 * (size_t)T + 2 * (size_t)n_map + nbT + 2);
    const size_t update = sizeof(uint32_t) * ((size_t)n_map + (size_t)n_new + 2 * nb + 4);
    size_t r = prune > dedup ? prune : dedup;
    r = r > update ? r : update;
    return (r + 255) & ~(size_t)255;
}

cudaError_t launch_prune_plan(const float* logits, int64_t n, float thr, double max_ratio, uint8_t* keep,
                              void* scratch, unsigned long long* kept_dev, cudaStream_t st) {
    SelectState* s = static_cast<SelectState*>(scratch);
    cudaError_t e = cudaMemsetAsync(s, 0, sizeof(SelectState), st);
    if (e != cudaSuccess) return e;
    const int g = mu_grid(n);
    prune_count_kernel<<<g, kMuThreads, 0, st>>>(logits, n, thr, s);
    const unsigned long long k_max = (unsigned long long)floor(max_ratio * (double)n);
    prune_init_kernel<<<1, 256, 0, st>>>(s, k_max);
    for (int r = 0; r < 8; r++) {
        prune_hist_kernel<<<g, kMuThreads, 0, st>>>(logits, n, thr, r, s);
        prune_pick_kernel<<<1, 32, 0, st>>>(r, s);
    }
    prune_mark_kernel<<<g, kMuThreads, 0, st>>>(logits, n, thr, s, keep);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaMemcpyAsync(kept_dev, &s->kept, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
}

cudaError_t launch_dedup_plan(const float* map_means, int64_t n, const float* new_means, int64_t nq, float radius,
                              uint8_t* accept, void* scratch, unsigned long long* accepted_host, cudaStream_t st) {
    SelectState* s = static_cast<SelectState*>(scratch);
    uint64_t T = 1;
    while (T < (uint64_t)(2 * (n > 0 ? n : 1))) T <<= 1;
    uint32_t* base = reinterpret_cast<uint32_t*>(s + 1);
    uint32_t* count = base;
    uint32_t* start = count + T;
    uint32_t* cursor = start + T;
    uint32_t* rows = cursor + T;
    uint32_t* cell = rows + n;
    uint32_t* bsum = cell + n;
    cudaError_t e = cudaMemsetAsync(s, 0, sizeof(SelectState), st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(count, 0, sizeof(uint32_t) * T, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(cursor, 0, sizeof(uint32_t) * T, st)) != cudaSuccess) return e;
    const double inv_cell = 1.0 / (1.001 * (double)radius);
    const uint32_t mask = (uint32_t)(T - 1);
    if (n > 0) hash_count_kernel<<<mu_grid(n), kMuThreads, 0, st>>>(map_means, n, inv_cell, mask, count, cell);
    if ((e = exclusive_scan(count, (int64_t)T, start, bsum, nullptr, st)) != cudaSuccess) return e;
    if (n > 0) hash_fill_kernel<<<mu_grid(n), kMuThreads, 0, st>>>(n, cell, start, cursor, rows);
    if (nq > 0)
        dedup_query_kernel<<<mu_grid(nq), kMuThreads, 0, st>>>(map_means, n, new_means, nq, inv_cell,
                                                               radius * radius, mask, start, count, rows, accept, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaMemcpyAsync(accepted_host, &s->kept, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
}

cudaError_t launch_map_scan(const uint8_t* keep, int64_t n, const uint8_t* accept, int64_t n_new, void* scratch,
                            uint32_t** pos_keep, uint32_t** pos_new, uint32_t* totals_host, cudaStream_t st) {
    uint32_t* base = static_cast<uint32_t*>(scratch);
    uint32_t* tot = base;                 // [2]
    uint32_t* pk = base + 4;
    uint32_t* pn = pk + n;
    uint32_t* bsum = pn + n_new;
    cudaError_t e = cudaMemsetAsync(tot, 0, sizeof(uint32_t) * 2, st);
    if (e != cudaSuccess) return e;
    if ((e = exclusive_scan(keep, n, pk, bsum, tot, st)) != cudaSuccess) return e;
    *pos_keep = pk;
    *pos_new = nullptr;
    if (accept && n_new > 0) {
        if ((e = exclusive_scan(accept, n_new, pn, bsum, tot + 1, st)) != cudaSuccess) return e;
        *pos_new = pn;
    }
    return cudaMemcpyAsync(totals_host, tot, sizeof(uint32_t) * 2, cudaMemcpyDeviceToHost, st);
}

cudaError_t launch_compact(const MapUpdateArgs& a, cudaStream_t st) {
    const int64_t total = a.n + a.n_new;
    if (total > 0) compact_kernel<<<mu_grid(total), kMuThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gs
