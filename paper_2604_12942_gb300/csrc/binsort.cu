// a2-a4: tile binning (scan of tiles-touched, pair emission), the stable LSD radix sort of
// the (tile, depth) keys and the per-tile ranges.  Tile-based rasterizer of §II-A / §III-C.
//
// The sort runs on a fixed grid (a multiple of the SM count) whose blocks each own a
// contiguous run of chunks; the pair count is read on the device, so no host round trip
// or re-launch is needed between binning and sorting and the whole sequence can be
// captured in a CUDA graph.  Every pass: per-block digit histograms (upsweep), a scan of
// the histograms (one block, one warp per digit), then a stable scatter (downsweep) that
// ranks each chunk with warp match/ballot counting and writes digit runs contiguously.
#include "gs_kernels.cuh"

namespace gs {

// ----------------------------------------------------------------------------------------
// Exclusive scan of tiles-touched -> pair offsets and the pair count.
// ----------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t block_exclusive_scan_1024(uint32_t x, uint32_t* s_warp, uint32_t& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0u;
        uint32_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        s_warp[lane] = ti - t;
        if (lane == 31) s_warp[32] = ti;
    }
    __syncthreads();
    total = s_warp[32];
    const uint32_t r = s_warp[w] + inc - x;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const uint32_t* __restrict__ in, int64_t n,
                                                                  uint32_t* __restrict__ bsum) {
    __shared__ uint32_t s[33];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        const int64_t j = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (j < n) sum += in[j];
    }
    sum = warp_sum(sum);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t t = threadIdx.x < (kScanThreads >> 5) ? s[threadIdx.x] : 0u;
        t = warp_sum(t);
        if (threadIdx.x == 0) bsum[blockIdx.x] = t;
    }
}

// One block: exclusive scan of the block sums, the pair count and the capacity check.
__global__ void __launch_bounds__(kScanThreads) scan_blocks_kernel(uint32_t* __restrict__ bsum, int nb,
                                                                  Counters* c, int64_t max_pairs) {
    __shared__ uint32_t s[33];
    unsigned long long carry = 0;
    for (int base = 0; base < nb; base += kScanThreads) {
        const int j = base + threadIdx.x;
        const uint32_t x = j < nb ? bsum[j] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan_1024(x, s, tot);
        if (j < nb) bsum[j] = (uint32_t)(carry + ex);
        carry += tot;
    }
    if (threadIdx.x == 0) {
        c->n_pairs = carry;
        if (carry > (unsigned long long)max_pairs) set_status(c, GS_ERR_CAPACITY);
    }
}

__global__ void __launch_bounds__(kScanThreads) scan_down_kernel(const uint32_t* __restrict__ in, int64_t n,
                                                                const uint32_t* __restrict__ bsum,
                                                                uint32_t* __restrict__ out) {
    __shared__ uint32_t s[33];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
    uint32_t x[kScanItems], sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        x[k] = (base + k < n) ? in[base + k] : 0u;
        sum += x[k];
    }
    uint32_t tot;
    uint32_t run = block_exclusive_scan_1024(sum, s, tot) + bsum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        if (base + k < n) out[base + k] = run;
        run += x[k];
    }
}

// One thread per (view, Gaussian): write its pairs at its scanned offset.
__global__ void __launch_bounds__(256) emit_kernel(BinArgs a) {
    if (a.counters->status != 0) return;
    const int64_t total = (int64_t)a.n_views * a.n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = a.touched[idx];
        if (t == 0) continue;
        const int v = (int)(idx / a.n);
        const View& V = a.views[v];
        const float4 r0 = a.proj[3 * idx];
        const int rx = __float_as_int(a.proj[3 * idx + 1].w);
        const int ry = __float_as_int(a.proj[3 * idx + 2].w);
        int x0, x1, y0, y1;
        if (!tile_span(r0.x, rx, a.tile, V.tiles_x, x0, x1) || !tile_span(r0.y, ry, a.tile, V.tiles_y, y0, y1))
            continue;
        const unsigned long long zb = (unsigned long long)__float_as_uint(r0.z);
        uint32_t off = a.offsets[idx];
        for (int ty = y0; ty <= y1; ty++) {
            for (int tx = x0; tx <= x1; tx++) {
                const unsigned long long tileid = (unsigned long long)(V.tile_off + ty * V.tiles_x + tx);
                a.keys[off] = (tileid << 32) | zb;
                a.vals[off] = (uint32_t)idx;
                off++;
            }
        }
    }
}

cudaError_t launch_exclusive_scan(const uint32_t* in, int64_t n, uint32_t* out, uint32_t* tmp, Counters* c,
                                  int64_t max_total, cudaStream_t st) {
    const int nb = (int)((n + kScanBlock - 1) / kScanBlock);
    if (nb > 0) scan_reduce_kernel<<<nb, kScanThreads, 0, st>>>(in, n, tmp);
    scan_blocks_kernel<<<1, kScanThreads, 0, st>>>(tmp, nb, c, max_total);
    if (nb > 0) scan_down_kernel<<<nb, kScanThreads, 0, st>>>(in, n, tmp, out);
    return cudaGetLastError();
}

cudaError_t launch_bin(const BinArgs& a, cudaStream_t st) {
    const int64_t total = (int64_t)a.n_views * a.n;
    cudaError_t e = launch_exclusive_scan(a.touched, total, a.offsets, a.scan_tmp, a.counters, a.max_pairs, st);
    if (e != cudaSuccess) return e;
    const int64_t eb64 = (total + 255) / 256;
    const int eb = (int)(eb64 < 152 * 32 ? eb64 : 152 * 32);
    if (eb > 0) emit_kernel<<<eb, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------------------
// Radix sort.
// ----------------------------------------------------------------------------------------
__device__ __forceinline__ void chunk_span(const Counters* c, int grid, int b, int64_t& lo, int64_t& hi) {
    const int64_t P = (int64_t)c->n_pairs;
    const int64_t nch = (P + kSortChunk - 1) / kSortChunk;
    const int64_t c0 = nch * b / grid, c1 = nch * (b + 1) / grid;
    lo = c0 * kSortChunk;
    hi = min(c1 * kSortChunk, P);
}

__global__ void __launch_bounds__(kSortThreads) sort_upsweep_kernel(SortArgs a, int in_buf, int shift) {
    // one private histogram per warp keeps shared-memory atomics on a digit to one warp
    __shared__ uint32_t h[kSortThreads / 32][kSortBins];
    if (a.counters->status != 0) return;
    for (int t = threadIdx.x; t < (kSortThreads / 32) * kSortBins; t += blockDim.x) (&h[0][0])[t] = 0;
    __syncthreads();
    int64_t lo, hi;
    chunk_span(a.counters, a.grid, blockIdx.x, lo, hi);
    const unsigned long long* keys = a.keys[in_buf];
    uint32_t* hw = h[threadIdx.x >> 5];
    for (int64_t j = lo + threadIdx.x; j < hi; j += blockDim.x) {
        const uint32_t d = (uint32_t)(keys[j] >> shift) & (kSortBins - 1);
        atomicAdd(&hw[d], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kSortBins; d += blockDim.x) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; w++) s += h[w][d];
        a.hist[(int64_t)d * a.grid + blockIdx.x] = s;
    }
}

// One block of 1024 threads: per digit (one warp per 8 digits) exclusive prefix over the
// blocks; digit totals scanned into digit_tot as the start of each digit's output run.
__global__ void __launch_bounds__(1024) sort_scan_kernel(SortArgs a) {
    __shared__ uint32_t s_tot[kSortBins];
    __shared__ uint32_t s_w[33];
    if (a.counters->status != 0) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = w; d < kSortBins; d += 32) {
        uint32_t* row = a.hist + (int64_t)d * a.grid;
        uint32_t carry = 0;
        for (int b0 = 0; b0 < a.grid; b0 += 32) {
            const int b = b0 + lane;
            const uint32_t x = b < a.grid ? row[b] : 0u;
            uint32_t inc = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (b < a.grid) row[b] = carry + inc - x;
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (lane == 0) s_tot[d] = carry;
    }
    __syncthreads();
    uint32_t tot;
    const uint32_t x = threadIdx.x < kSortBins ? s_tot[threadIdx.x] : 0u;
    const uint32_t ex = block_exclusive_scan_1024(x, s_w, tot);
    if (threadIdx.x < kSortBins) a.digit_tot[threadIdx.x] = ex;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

constexpr int kSortWarps = kSortThreads / 32;
constexpr int kItemsPerWarp = kSortChunk / kSortWarps;   // 512

struct SortSmem {
    unsigned long long keys[kSortChunk];
    uint32_t vals[kSortChunk];
    uint32_t wcnt[kSortWarps][kSortBins];
    uint32_t run[kSortBins];
    uint32_t tot[kSortBins];
    uint32_t cstart[kSortBins];
    uint32_t scan_w[33];
};

__global__ void __launch_bounds__(kSortThreads) sort_downsweep_kernel(SortArgs a, int in_buf, int shift) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem& S = *reinterpret_cast<SortSmem*>(smem_raw);
    if (a.counters->status != 0) return;
    int64_t lo, hi;
    chunk_span(a.counters, a.grid, blockIdx.x, lo, hi);
    const unsigned long long* kin = a.keys[in_buf];
    const uint32_t* vin = a.vals[in_buf];
    unsigned long long* kout = a.keys[in_buf ^ 1];
    uint32_t* vout = a.vals[in_buf ^ 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kSortBins; d += blockDim.x)
        S.run[d] = a.digit_tot[d] + a.hist[(int64_t)d * a.grid + blockIdx.x];
    const uint32_t ltm = lanemask_lt();
    for (int64_t base = lo; base < hi; base += kSortChunk) {
        const int m = (int)(hi - base < kSortChunk ? hi - base : kSortChunk);
        for (int t = threadIdx.x; t < kSortWarps * kSortBins; t += blockDim.x) (&S.wcnt[0][0])[t] = 0;
        __syncthreads();
        unsigned long long key[kSortItems];
        uint32_t val[kSortItems];
        uint32_t rank[kSortItems];
#pragma unroll
        for (int j = 0; j < kSortItems; j++) {
            const int item = w * kItemsPerWarp + j * 32 + lane;
            const bool valid = item < m;
            key[j] = valid ? kin[base + item] : 0ull;
            val[j] = valid ? vin[base + item] : 0u;
            const uint32_t d = valid ? ((uint32_t)(key[j] >> shift) & (kSortBins - 1)) : (uint32_t)kSortBins;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            uint32_t r = __popc(peers & ltm);
            if (valid) r += S.wcnt[w][d];
            __syncwarp();
            if (valid && lane == 31 - __clz(peers)) S.wcnt[w][d] += __popc(peers);
            __syncwarp();
            rank[j] = r;
        }
        __syncthreads();
        // per digit: prefix over warps, chunk totals
        for (int d = threadIdx.x; d < kSortBins; d += blockDim.x) {
            uint32_t run = 0;
#pragma unroll
            for (int ww = 0; ww < kSortWarps; ww++) {
                const uint32_t c = S.wcnt[ww][d];
                S.wcnt[ww][d] = run;
                run += c;
            }
            S.tot[d] = run;
        }
        __syncthreads();
        {
            // exclusive scan of the chunk totals over digits (kSortThreads == kSortBins)
            const uint32_t x = S.tot[threadIdx.x];
            uint32_t inc = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane == 31) S.scan_w[w] = inc;
            __syncthreads();
            if (w == 0) {
                const uint32_t t0 = lane < kSortWarps ? S.scan_w[lane] : 0u;
                uint32_t ti = t0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
                    if (lane >= o) ti += y;
                }
                if (lane < kSortWarps) S.scan_w[lane] = ti - t0;
            }
            __syncthreads();
            S.cstart[threadIdx.x] = S.scan_w[w] + inc - x;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kSortItems; j++) {
            const int item = w * kItemsPerWarp + j * 32 + lane;
            if (item < m) {
                const uint32_t d = (uint32_t)(key[j] >> shift) & (kSortBins - 1);
                const uint32_t pos = S.cstart[d] + S.wcnt[w][d] + rank[j];
                S.keys[pos] = key[j];
                S.vals[pos] = val[j];
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            const unsigned long long kk = S.keys[k];
            const uint32_t d = (uint32_t)(kk >> shift) & (kSortBins - 1);
            const int64_t g = (int64_t)S.run[d] + (k - (int)S.cstart[d]);
            kout[g] = kk;
            vout[g] = S.vals[k];
        }
        __syncthreads();
        for (int d = threadIdx.x; d < kSortBins; d += blockDim.x) S.run[d] += S.tot[d];
        __syncthreads();
    }
}

static int g_sort_grid = 0;
int sort_grid() {
    if (g_sort_grid == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        g_sort_grid = (sms > 0 ? sms : 148) * 2;
    }
    return g_sort_grid;
}

cudaError_t launch_sort(const SortArgs& a, int n_passes, const int* shifts, cudaStream_t st) {
    static bool attr_set = false;
    const size_t smem = sizeof(SortSmem);
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(sort_downsweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    for (int p = 0; p < n_passes; p++) {
        const int in_buf = p & 1;
        sort_upsweep_kernel<<<a.grid, kSortThreads, 0, st>>>(a, in_buf, shifts[p]);
        sort_scan_kernel<<<1, 1024, 0, st>>>(a);
        sort_downsweep_kernel<<<a.grid, kSortThreads, smem, st>>>(a, in_buf, shifts[p]);
    }
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------------------
// Tile ranges.
// ----------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) ranges_kernel(RangeArgs a) {
    if (a.counters->status != 0) return;
    const int64_t P = (int64_t)a.counters->n_pairs;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = (uint32_t)(a.keys[i] >> 32);
        if (i == 0 || (uint32_t)(a.keys[i - 1] >> 32) != t) a.ranges[t].x = (uint32_t)i;
        if (i == P - 1 || (uint32_t)(a.keys[i + 1] >> 32) != t) a.ranges[t].y = (uint32_t)(i + 1);
    }
}

cudaError_t launch_ranges(const RangeArgs& a, int n_tiles, cudaStream_t st) {
    (void)n_tiles;
    ranges_kernel<<<sort_grid() * 4, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------------------
// Work order of the compositing kernels: (view, tile) items by decreasing pair count, in
// power-of-two buckets (bucket b holds counts in [2^(b-1), 2^b)), so that the largest tiles
// are scheduled first and the tail of the launch is made of short items.
// ----------------------------------------------------------------------------------------
constexpr int kOrderBuckets = 34;

__device__ __forceinline__ int order_bucket(uint2 r) {
    const uint32_t c = r.y - r.x;
    return c ? 33 - __clz(c) : 0;   // 0 = empty, 1..33
}

__global__ void tile_order_hist_kernel(const uint2* ranges, int n_tiles, uint32_t* cnt, const Counters* c) {
    __shared__ uint32_t h[kOrderBuckets];
    for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x) h[b] = 0;
    __syncthreads();
    if (c->status == 0)
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += gridDim.x * blockDim.x)
            atomicAdd(&h[order_bucket(ranges[t])], 1u);
    __syncthreads();
    for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x)
        if (h[b]) atomicAdd(&cnt[b], h[b]);
}

// cursor[b] = number of items in buckets above b (largest counts first)
__global__ void tile_order_scan_kernel(const uint32_t* cnt, uint32_t* cursor) {
    if (threadIdx.x != 0) return;
    uint32_t run = 0;
    for (int b = kOrderBuckets - 1; b >= 0; b--) {
        cursor[b] = run;
        run += cnt[b];
    }
}

__global__ void tile_order_scatter_kernel(const uint2* ranges, int n_tiles, uint32_t* cursor, uint32_t* order,
                                          const Counters* c) {
    const int lane = threadIdx.x & 31;
    for (int t0 = blockIdx.x * blockDim.x; t0 < n_tiles; t0 += gridDim.x * blockDim.x) {
        const int t = t0 + threadIdx.x;
        const bool ok = t < n_tiles;
        const int b = ok ? (c->status == 0 ? order_bucket(ranges[t]) : 0) : kOrderBuckets;
        // one atomic per bucket per warp
        const uint32_t peers = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (ok && lane == leader) base = atomicAdd(&cursor[b], (uint32_t)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (ok) order[base + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)t;
    }
}

cudaError_t launch_tile_order(const uint2* ranges, int n_tiles, uint32_t* order, uint32_t* tmp, const Counters* c,
                              cudaStream_t st) {
    if (n_tiles <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(tmp, 0, sizeof(uint32_t) * 2 * kOrderBuckets, st);
    if (e != cudaSuccess) return e;
    const int blocks = (n_tiles + 255) / 256 < 1024 ? (n_tiles + 255) / 256 : 1024;
    tile_order_hist_kernel<<<blocks, 256, 0, st>>>(ranges, n_tiles, tmp, c);
    tile_order_scan_kernel<<<1, 32, 0, st>>>(tmp, tmp + kOrderBuckets);
    tile_order_scatter_kernel<<<blocks, 256, 0, st>>>(ranges, n_tiles, tmp + kOrderBuckets, order, c);
    return cudaGetLastError();
}

}  // namespace gs
