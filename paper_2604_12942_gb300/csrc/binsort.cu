// a2-a4: tile binning, the stable LSD radix sorts and the per-tile ranges.  Tile-based
// rasterizer of §II-A / §III-C: every Gaussian is listed, in depth order, in each tile its
// alpha >= alpha_min box covers.
//
// The required order is (global tile, depth, view, Gaussian index).  Instead of one sort on
// a (tile << 32 | bits(z)) key over all pairs, the binning sorts twice:
//   1. the visible (view, Gaussian) entries -- compacted in (view, index) order -- by the
//      32-bit depth key (4 passes over the entries, about a fifth of the pairs);
//   2. the pairs, emitted from the depth-sorted entries, by the global tile id alone
//      (ceil(tile bits / 8) passes with 32-bit keys).
// Both sorts are stable, so pass 2 keeps the depth order within a tile and pass 1 keeps
// (view, index) order between equal depths: the result is the order above.
//
// The sorts run on a fixed grid (a multiple of the SM count) whose blocks each own a
// contiguous run of chunks; element counts are read on the device, so no host round trip
// is needed between the stages and the whole sequence can be captured in a CUDA graph.
// Every pass: per-block digit histograms (upsweep), a per-digit scan over the blocks (one
// warp per digit), then a stable scatter (downsweep) that ranks each chunk with warp
// ballot counting and writes digit runs contiguously.
#include "gs_kernels.cuh"

namespace gs {

// ----------------------------------------------------------------------------------------
// Block-wide scans.
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

// One block: exclusive scan of nb block sums in place; the total goes to *total_out and
// sets GS_ERR_CAPACITY when it exceeds max_total (max_total < 0: no limit).
__global__ void __launch_bounds__(kScanThreads) scan_blocks_kernel(uint32_t* __restrict__ bsum, int nb,
                                                                  unsigned long long* total_out,
                                                                  uint32_t* total32_out, Counters* c,
                                                                  int64_t max_total) {
    __shared__ uint32_t s[33];
    if (c->status != 0) return;
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
        *total_out = carry;
        if (total32_out) *total32_out = (uint32_t)carry;
        if (max_total >= 0 && carry > (unsigned long long)max_total) set_status(c, GS_ERR_CAPACITY);
    }
}

// ----------------------------------------------------------------------------------------
// Entry compaction.  The projection leaves one bit word per view and 32 Gaussians (vis_bits,
// each view padded to whole words).  A block of kEntryThreads threads covers as many words:
// the count kernel writes the block's entry total; the totals are scanned; the compaction
// kernel gives each word its offset by a block scan of the word counts, and each warp writes
// the entries of 32 words, one word at a time with a lane per slot, so entries stay in (view,
// index) order.  Blocks of 256 (four resident per SM) rather than 1024 (one, at the
// compaction's registers) shorten the ragged end of the grid.
// ----------------------------------------------------------------------------------------
constexpr int kEntryThreads = 256;

__global__ void __launch_bounds__(kEntryThreads) entry_count_kernel(const uint32_t* __restrict__ bits, int64_t n_words,
                                                                   uint32_t* __restrict__ bsum) {
    __shared__ uint32_t s[kEntryThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t word = (int64_t)blockIdx.x * kEntryThreads + threadIdx.x;
    const uint32_t sum = warp_sum((uint32_t)__popc(word < n_words ? bits[word] : 0u));
    if (lane == 0) s[w] = sum;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t t = threadIdx.x < (kEntryThreads >> 5) ? s[threadIdx.x] : 0u;
        t = warp_sum(t);
        if (threadIdx.x == 0) bsum[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kEntryThreads, 4) entry_compact_kernel(BinArgs a, int64_t n_words) {
    __shared__ uint32_t s[33];
    __shared__ uint32_t s_off[kEntryThreads], s_word[kEntryThreads];
    if (a.counters->status != 0) return;
    const int64_t word = (int64_t)blockIdx.x * kEntryThreads + threadIdx.x;
    const uint32_t b = word < n_words ? a.vis_bits[word] : 0u;
    const uint32_t nw = (uint32_t)((a.n + 31) >> 5);   // words per view
    uint32_t tot;
    const uint32_t off = block_exclusive_scan_1024((uint32_t)__popc(b), s, tot) + a.scan_tmp[blockIdx.x];
    s_off[threadIdx.x] = off;
    s_word[threadIdx.x] = b;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t ltm;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(ltm));
    // four bit words per iteration: their record gathers are issued together
    for (int k = 0; k < 32; k += 4) {
        bool hit[4];
        float4 g0[4];
        int grx[4], gry[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int lw = w * 32 + k + u;
            hit[u] = (s_word[lw] >> lane) & 1u;
            const uint32_t gw = (uint32_t)blockIdx.x * kEntryThreads + lw;   // < V * nw
            const uint32_t v = gw / nw;
            const uint32_t idx = v * (uint32_t)a.n + (gw - v * nw) * 32 + lane;
            if (hit[u]) {
                g0[u] = __ldg(a.proj + 3 * (size_t)idx);
                grx[u] = __float_as_int(__ldg(a.proj + 3 * (size_t)idx + 1).w);
                gry[u] = __float_as_int(__ldg(a.proj + 3 * (size_t)idx + 2).w);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int lw = w * 32 + k + u;
            const uint32_t bw = s_word[lw];
            if (hit[u]) {
                const uint32_t pos = s_off[lw] + (uint32_t)__popc(bw & ltm);
                const uint32_t gw = (uint32_t)blockIdx.x * kEntryThreads + lw;
                const uint32_t v = gw / nw;
                const uint32_t idx = v * (uint32_t)a.n + (gw - v * nw) * 32 + lane;
                const float4 r0 = g0[u];
                const int rx = grx[u];
                const int ry = gry[u];
                const View& V = a.views[v];
                // the rectangle the projection found non-empty
                int xa = 0, xb = 0, ya = 0, yb = 0;
                tile_span(r0.x, rx, a.tile, V.tiles_x, xa, xb);
                tile_span(r0.y, ry, a.tile, V.tiles_y, ya, yb);
                a.ekeys[pos] = __float_as_uint(r0.z);   // z > 0: bits are monotone
                a.evals[pos] = pos;
                a.entries[pos] = idx;
                a.erect[pos] = make_uint2((uint32_t)(V.tile_off + ya * V.tiles_x + xa),
                                          (uint32_t)(xb - xa + 1) | ((uint32_t)(yb - ya + 1) << 16));
            }
        }
    }
}

cudaError_t launch_entries(const BinArgs& a, cudaStream_t st) {
    const int64_t n_words = (int64_t)a.n_views * ((a.n + 31) >> 5);
    const int nb = (int)((n_words + kEntryThreads - 1) / kEntryThreads);
    if (nb > 0) entry_count_kernel<<<nb, kEntryThreads, 0, st>>>(a.vis_bits, n_words, a.scan_tmp);
    scan_blocks_kernel<<<1, kScanThreads, 0, st>>>(a.scan_tmp, nb, &a.counters->n_entries, &a.counters->n_entries32,
                                                   a.counters, -1);
    if (nb > 0) entry_compact_kernel<<<nb, kEntryThreads, 0, st>>>(a, n_words);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------------------
// Pair emission from the depth-sorted entries: the tile counts of their rectangles, taken
// in that order, are scanned into pair offsets (total = pair count), then each entry writes
// one (global tile id, view * n + index) pair per covered tile, tiles in row-major order.
// The rectangles and indices are read from the compact per-entry arrays of the compaction
// (12 bytes an entry, which stay in L2), not from the projected records.
// ----------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t rect_count(uint2 r) { return (r.y & 0xFFFFu) * (r.y >> 16); }

// The entry count is known only on the device, so the scans over the depth-sorted entries
// cover the capacity (n_views * n) in chunks of kScanBlock entries, taken in turn by a grid of
// resident blocks: a chunk past the last entry costs one store, not a block launch.
//
// Pair count of each chunk.  Also writes, in depth order, each entry's tile rectangle and
// index (srt), which the offsets and the emission then read without the gather through the
// sorted compact indices.
__global__ void __launch_bounds__(kScanThreads) pair_count_kernel(BinArgs a, int nb) {
    __shared__ uint32_t s[33];
    const int64_t E = (int64_t)a.counters->n_entries;
    const int64_t VN = (int64_t)a.n_views * a.n;
    for (int ch = blockIdx.x; ch < nb; ch += gridDim.x) {
        const int64_t base = (int64_t)ch * kScanBlock;
        if (base >= E) {   // (the same for the whole block)
            if (threadIdx.x == 0) a.scan_tmp[ch] = 0u;
            continue;
        }
        uint32_t sum = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            const int64_t j = base + (int64_t)k * kScanThreads + threadIdx.x;
            if (j < E) {
                const uint32_t c = a.sorted_evals[j];
                const uint2 r = a.erect[c];
                a.srt[j] = r.x;
                a.srt[VN + j] = r.y;
                a.srt[2 * VN + j] = a.entries[c];
                sum += rect_count(r);
            }
        }
        sum = warp_sum(sum);
        if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = sum;
        __syncthreads();
        if (threadIdx.x < 32) {
            uint32_t t = threadIdx.x < (kScanThreads >> 5) ? s[threadIdx.x] : 0u;
            t = warp_sum(t);
            if (threadIdx.x == 0) a.scan_tmp[ch] = t;
        }
        __syncthreads();   // s is written again for the next chunk
    }
}

// Pair offsets of the depth-sorted entries (poff[e] = pairs of the entries before e), and
// for every output chunk of kEmitChunk pairs the entry holding its first pair.
__global__ void __launch_bounds__(kScanThreads) pair_offsets_kernel(BinArgs a, int nb) {
    __shared__ uint32_t s[33];
    if (a.counters->status != 0) return;
    const int64_t E = (int64_t)a.counters->n_entries;
    for (int ch = blockIdx.x; ch < nb && (int64_t)ch * kScanBlock < E; ch += gridDim.x) {
        const int64_t base = (int64_t)ch * kScanBlock + (int64_t)threadIdx.x * kScanItems;
        uint32_t t[kScanItems], sum = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            t[k] = base + k < E ? rect_count(make_uint2(0u, a.srt[(int64_t)a.n_views * a.n + base + k])) : 0u;
            sum += t[k];
        }
        uint32_t tot;
        uint32_t off = block_exclusive_scan_1024(sum, s, tot) + a.scan_tmp[ch];   // (ends with a barrier)
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            if (base + k < E) {
                a.poff[base + k] = off;
                // chunk starts c * kEmitChunk inside [off, off + t)
                for (uint32_t c = (off + kEmitChunk - 1) / kEmitChunk; c * (uint64_t)kEmitChunk < (uint64_t)off + t[k];
                     c++)
                    a.chunk_first[c] = (uint32_t)(base + k);
            }
            off += t[k];
        }
    }
}

// Emission balanced over the output: a block takes a chunk of kEmitChunk consecutive pairs,
// stages the entries they come from (at most kEmitChunk + 1) with their tile rectangles in
// shared memory, marks the slot where each entry starts, and finds every slot's entry with a
// running maximum over the chunk.  A few entries
// with very many tiles no longer serialise on one warp.
__global__ void __launch_bounds__(kEmitThreads) pair_emit_kernel(BinArgs a) {
    static_assert(kEmitChunk == 8 * kEmitThreads, "each thread owns 8 consecutive slots of the chunk");
    __shared__ uint32_t s_off[kEmitChunk + 1], s_t0[kEmitChunk + 1], s_id[kEmitChunk + 1];
    __shared__ uint16_t s_wx[kEmitChunk + 1], s_tx[kEmitChunk + 1];
    __shared__ __align__(16) uint16_t s_own[kEmitChunk];   // slot -> local entry index
    __shared__ uint32_t s_wmax[kEmitThreads / 32];
    __shared__ uint16_t s_view_tx[GS_MAX_VIEWS];   // tiles per row of each view
    if (a.counters->status != 0) return;
    for (int v = threadIdx.x; v < a.n_views; v += blockDim.x) s_view_tx[v] = (uint16_t)a.views[v].tiles_x;
    const uint64_t P = a.counters->n_pairs;
    const int64_t E = (int64_t)a.counters->n_entries;
    const uint64_t n_chunks = (P + kEmitChunk - 1) / kEmitChunk;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // the chunks in turn over the grid (a resident grid: the pair count is known only here)
    for (uint64_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        const uint64_t p0 = c * kEmitChunk, p1 = p0 + kEmitChunk < P ? p0 + kEmitChunk : P;
        const int64_t e0 = a.chunk_first[c];
        const int64_t e1 = c + 1 < n_chunks ? (int64_t)a.chunk_first[c + 1] : E - 1;
        const int ne = (int)(e1 - e0 + 1);   // <= kEmitChunk + 1: every entry has >= 1 pair
        for (int i = threadIdx.x; i < kEmitChunk; i += blockDim.x) s_own[i] = 0;
        __syncthreads();
        const int64_t VN = (int64_t)a.n_views * a.n;
        for (int j = threadIdx.x; j < ne; j += blockDim.x) {
            const int64_t e = e0 + j;
            const uint32_t idx = a.srt[2 * VN + e];
            const uint2 r = make_uint2(a.srt[e], a.srt[VN + e]);
            const uint32_t off = a.poff[e];
            s_off[j] = off;
            s_t0[j] = r.x;
            s_id[j] = idx;
            s_wx[j] = (uint16_t)(r.y & 0xFFFFu);
            s_tx[j] = s_view_tx[idx / (uint32_t)a.n];
            // the entry's first pair slot in this chunk (entry 0 starts at or before p0)
            if (j > 0 && off < p1) s_own[off - p0] = (uint16_t)j;
        }
        __syncthreads();
        // slot owner = the last entry starting at or before the slot: a running maximum over
        // the chunk (8 slots per thread, then warp and block maxima of the thread maxima)
        uint32_t own[8], mx = 0;
        {
            const uint4 q = *reinterpret_cast<const uint4*>(s_own + 8 * threadIdx.x);
            const uint32_t wd[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int h = 0; h < 4; h++) {
                mx = max(mx, wd[h] & 0xFFFFu);
                own[2 * h] = mx;
                mx = max(mx, wd[h] >> 16);
                own[2 * h + 1] = mx;
            }
        }
        uint32_t inc = mx;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc = max(inc, y);
        }
        if (lane == 31) s_wmax[w] = inc;
        uint32_t before = __shfl_up_sync(0xffffffffu, inc, 1);
        if (lane == 0) before = 0;
        __syncthreads();
        for (int ww = 0; ww < w; ww++) before = max(before, s_wmax[ww]);
        __syncthreads();   // every thread has read its slots
#pragma unroll
        for (int h = 0; h < 8; h++) s_own[8 * threadIdx.x + h] = (uint16_t)max(before, own[h]);
        __syncthreads();
        // coalesced writes: thread t writes slots t, t + 256, ...
        for (uint64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            const uint32_t j = s_own[p - p0];
            const uint32_t kk = (uint32_t)p - s_off[j], wx = s_wx[j];
            const uint32_t ty = kk / wx, tx = kk - ty * wx;
            a.pkeys[p] = s_t0[j] + ty * (uint32_t)s_tx[j] + tx;
            a.pvals[p] = s_id[j];
        }
        __syncthreads();
    }
}

// Blocks of `kernel` resident on the device at once (occupancy times SMs), kept per device.
template <class Kernel>
static int resident_grid(int (&cache)[kMaxDevices], Kernel kernel, int threads) {
    const int d = current_device();
    if (d >= 0 && cache[d] > 0) return cache[d];
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int g = per_sm * device_sms();
    if (d >= 0) cache[d] = g;
    return g;
}

cudaError_t launch_emit(const BinArgs& a, cudaStream_t st) {
    static int g_count[kMaxDevices] = {}, g_offsets[kMaxDevices] = {}, g_emit[kMaxDevices] = {};
    const int64_t total = (int64_t)a.n_views * a.n;   // upper bound of the entry count
    const int nb = (int)((total + kScanBlock - 1) / kScanBlock);
    if (nb > 0) {
        const int g = resident_grid(g_count, pair_count_kernel, kScanThreads);
        pair_count_kernel<<<g < nb ? g : nb, kScanThreads, 0, st>>>(a, nb);
    }
    scan_blocks_kernel<<<1, kScanThreads, 0, st>>>(a.scan_tmp, nb, &a.counters->n_pairs, nullptr, a.counters,
                                                   a.max_pairs);
    if (nb > 0) {
        const int g = resident_grid(g_offsets, pair_offsets_kernel, kScanThreads);
        pair_offsets_kernel<<<g < nb ? g : nb, kScanThreads, 0, st>>>(a, nb);
    }
    // one chunk of kEmitChunk pairs per block and turn; the pair count is known only on the
    // device, so the grid is the resident one (capped by the capacity's chunks)
    const int64_t emit_chunks = (a.max_pairs + kEmitChunk - 1) / kEmitChunk;
    const int64_t ge = resident_grid(g_emit, pair_emit_kernel, kEmitThreads);
    const int64_t emit_grid = emit_chunks < ge ? emit_chunks : ge;
    pair_emit_kernel<<<(unsigned)(emit_grid > 0 ? emit_grid : 1), kEmitThreads, 0, st>>>(a);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------------------
// Radix sort with BITS-bit digits (8 or 9), keys K = uint32_t or unsigned long long.
// ----------------------------------------------------------------------------------------
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kItemsPerWarp = kSortChunk / kSortWarps;   // 512
constexpr int kUpThreads = 512;                          // upsweep block (same chunk range, more warps)
constexpr int kUpWarps = kUpThreads / 32;
constexpr int kUpItems = kSortChunk / kUpThreads;        // 8

__device__ __forceinline__ void chunk_span(unsigned long long count, int grid, int b, int64_t& lo, int64_t& hi) {
    const int64_t P = (int64_t)count;
    const int64_t nch = (P + kSortChunk - 1) / kSortChunk;
    const int64_t c0 = nch * b / grid, c1 = nch * (b + 1) / grid;
    lo = c0 * kSortChunk;
    hi = min(c1 * kSortChunk, P);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// The pass's digit: BITS bits of the key from `shift`, restricted by the pass's digit mask (a
// sort by the low b bits ends with a pass whose mask keeps only the bits below b).
template <int BITS, typename K>
__device__ __forceinline__ uint32_t digit_of(K k, int shift, uint32_t mask) {
    return (uint32_t)(k >> shift) & ((1u << BITS) - 1u) & mask;
}

// Per-block digit histograms over the block's chunks: every thread loads its kUpItems keys of
// a chunk first, then adds them to its warp's private histogram with shared-memory atomics.
template <typename K, int BITS>
__global__ void __launch_bounds__(kUpThreads) sort_upsweep_kernel(SortArgs a, int in_buf, int shift) {
    constexpr int BINS = 1 << BITS;
    __shared__ uint32_t h[kUpWarps][BINS];
    if (a.counters->status != 0) return;
    for (int t = threadIdx.x; t < kUpWarps * BINS; t += blockDim.x) (&h[0][0])[t] = 0;
    __syncthreads();
    int64_t lo, hi;
    chunk_span(*a.count, a.grid, blockIdx.x, lo, hi);
    const K* keys = static_cast<const K*>(in_buf ? a.keys[1] : a.keys[0]);
    uint32_t* hw = h[threadIdx.x >> 5];
    for (int64_t base = lo; base < hi; base += kSortChunk) {
        K k[kUpItems];
#pragma unroll
        for (int j = 0; j < kUpItems; j++) {
            const int64_t idx = base + (int64_t)j * kUpThreads + threadIdx.x;
            k[j] = idx < hi ? keys[idx] : (K)0;
        }
#pragma unroll
        for (int j = 0; j < kUpItems; j++) {
            const int64_t idx = base + (int64_t)j * kUpThreads + threadIdx.x;
            if (idx < hi) atomicAdd(&hw[digit_of<BITS>(k[j], shift, a.digit_mask)], 1u);
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < BINS; d += blockDim.x) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kUpWarps; w++) s += h[w][d];
        a.hist[(int64_t)d * a.grid + blockIdx.x] = s;
    }
}

// One warp per digit: exclusive prefix of the digit's block counts (in place) and the
// digit total.  8 warps per block.
__global__ void __launch_bounds__(256) sort_scan_kernel(SortArgs a) {
    if (a.counters->status != 0) return;
    const int lane = threadIdx.x & 31;
    const int d = blockIdx.x * 8 + (threadIdx.x >> 5);
    uint32_t* row = a.hist + (int64_t)d * a.grid;
    constexpr int C = kSortMaxGrid / 32;
    uint32_t x[C];
#pragma unroll
    for (int c = 0; c < C; c++) {
        const int b = c * 32 + lane;
        x[c] = b < a.grid ? row[b] : 0u;
    }
    uint32_t carry = 0;
#pragma unroll
    for (int c = 0; c < C; c++) {
        if (c * 32 >= a.grid) break;
        uint32_t inc = x[c];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const int b = c * 32 + lane;
        if (b < a.grid) row[b] = carry + inc - x[c];
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) a.digit_tot[d] = carry;
}

// Digit-indexed shared arrays are stored at dix(d) = d with its low 5 bits XORed with the next
// ones: digits 32 m apart (tile ids one or more tile rows apart, which a warp step often holds)
// then fall in different banks.  A bijection on [0, 2^BITS).
__device__ __forceinline__ int dix(uint32_t d) { return (int)(d ^ ((d >> 5) & 31u)); }

// Chunk position k is stored at k + k / 32: ranked keys of one warp step often land at a
// fixed stride (consecutive digits with similar counts), which without the skew would hit the
// same few shared-memory banks.
__device__ __forceinline__ int skew(int k) { return k + (k >> 5); }

template <typename K, int BITS>
struct SortSmem {
    static constexpr int BINS = 1 << BITS;
    K keys[kSortChunk + kSortChunk / 32];
    uint32_t vals[kSortChunk + kSortChunk / 32];
    uint32_t wcnt[kSortWarps][BINS];
    uint32_t run[BINS];
    uint32_t tot[BINS];
    uint32_t cstart[BINS];
    uint32_t scan_w[33];
};

// Exclusive scan of DPT consecutive values per thread over the block (kSortThreads threads);
// out[q] receives the prefix of value q.
template <int DPT>
__device__ __forceinline__ void block_exclusive_scan_dpt(const uint32_t (&x)[DPT], uint32_t (&out)[DPT],
                                                         uint32_t* scan_w) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t sum = 0;
#pragma unroll
    for (int q = 0; q < DPT; q++) sum += x[q];
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) scan_w[w] = inc;
    __syncthreads();
    if (w == 0) {
        const uint32_t t0 = lane < kSortWarps ? scan_w[lane] : 0u;
        uint32_t ti = t0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < kSortWarps) scan_w[lane] = ti - t0;
    }
    __syncthreads();
    uint32_t r = scan_w[w] + inc - sum;
#pragma unroll
    for (int q = 0; q < DPT; q++) {
        out[q] = r;
        r += x[q];
    }
    __syncthreads();
}

// resident downsweep blocks per SM (and the grid of every sort pass: this many per SM)
constexpr int kSortBlocksPerSM = 3;   // (2 and 4 measured slower on GB300)

template <typename K, int BITS>
__global__ void __launch_bounds__(kSortThreads, kSortBlocksPerSM) sort_downsweep_kernel(SortArgs a, int in_buf, int shift) {
    constexpr int BINS = 1 << BITS;
    constexpr int DPT = BINS / kSortThreads;   // digits per thread: 1 or 2
    static_assert(DPT * kSortThreads == BINS, "whole digits per thread");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem<K, BITS>& S = *reinterpret_cast<SortSmem<K, BITS>*>(smem_raw);
    if (a.counters->status != 0) return;
    int64_t lo, hi;
    chunk_span(*a.count, a.grid, blockIdx.x, lo, hi);
    // (selects, not a runtime index into the parameter arrays, which would go to local memory)
    const K* kin = static_cast<const K*>(in_buf ? a.keys[1] : a.keys[0]);
    const uint32_t* vin = in_buf ? a.vals[1] : a.vals[0];
    K* kout = static_cast<K*>(in_buf ? a.keys[0] : a.keys[1]);
    uint32_t* vout = in_buf ? a.vals[0] : a.vals[1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int d0 = threadIdx.x * DPT;   // this thread's digits d0 .. d0 + DPT - 1
    {
        // start of this block's run of each digit: digit offset + count in earlier blocks
        uint32_t x[DPT], ex[DPT];
#pragma unroll
        for (int q = 0; q < DPT; q++) x[q] = a.digit_tot[d0 + q];
        block_exclusive_scan_dpt<DPT>(x, ex, S.scan_w);
#pragma unroll
        for (int q = 0; q < DPT; q++) S.run[dix(d0 + q)] = ex[q] + a.hist[(int64_t)(d0 + q) * a.grid + blockIdx.x];
    }
    const uint32_t ltm = lanemask_lt();
    for (int64_t base = lo; base < hi; base += kSortChunk) {
        const int m = (int)(hi - base < kSortChunk ? hi - base : kSortChunk);
        for (int t = threadIdx.x; t < kSortWarps * BINS; t += blockDim.x) (&S.wcnt[0][0])[t] = 0;
        K key[kSortItems];
        uint32_t val[kSortItems];
        uint32_t rank[kSortItems];
        // all loads first: the chunk's reads are in flight together
#pragma unroll
        for (int j = 0; j < kSortItems; j++) {
            const int item = w * kItemsPerWarp + j * 32 + lane;
            const bool valid = item < m;
            key[j] = valid ? kin[base + item] : (K)0;
            val[j] = valid ? vin[base + item] : 0u;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kSortItems; j++) {
            const int item = w * kItemsPerWarp + j * 32 + lane;
            const bool valid = item < m;
            const uint32_t d = valid ? digit_of<BITS>(key[j], shift, a.digit_mask) : (uint32_t)BINS;
            // lanes holding the same digit: one ballot per digit bit, and one for validity (a
            // fixed cost; __match_any_sync is slower when a warp holds many distinct digits)
            uint32_t peers = __ballot_sync(0xffffffffu, valid);
            if (!valid) peers = ~peers;
#pragma unroll
            for (int bit = 0; bit < BITS; bit++) {
                const bool set = (d >> bit) & 1u;
                const uint32_t bb = __ballot_sync(0xffffffffu, set);
                peers &= set ? bb : ~bb;
            }
            uint32_t r = __popc(peers & ltm);
            if (valid) r += S.wcnt[w][dix(d)];
            __syncwarp();
            if (valid && lane == 31 - __clz(peers)) S.wcnt[w][dix(d)] += __popc(peers);
            __syncwarp();
            rank[j] = r;
        }
        __syncthreads();
        {
            // per digit: prefix over warps and the chunk total, then the chunk's digit starts
            uint32_t tot[DPT], cs[DPT];
#pragma unroll
            for (int q = 0; q < DPT; q++) {
                uint32_t run = 0;
#pragma unroll
                for (int ww = 0; ww < kSortWarps; ww++) {
                    const uint32_t c = S.wcnt[ww][dix(d0 + q)];
                    S.wcnt[ww][dix(d0 + q)] = run;
                    run += c;
                }
                tot[q] = run;
                S.tot[dix(d0 + q)] = run;
            }
            block_exclusive_scan_dpt<DPT>(tot, cs, S.scan_w);
#pragma unroll
            for (int q = 0; q < DPT; q++) S.cstart[dix(d0 + q)] = cs[q];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kSortItems; j++) {
            const int item = w * kItemsPerWarp + j * 32 + lane;
            if (item < m) {
                const uint32_t d = digit_of<BITS>(key[j], shift, a.digit_mask);
                const int pos = skew((int)(S.cstart[dix(d)] + S.wcnt[w][dix(d)] + rank[j]));
                S.keys[pos] = key[j];
                S.vals[pos] = val[j];
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            const K kk = S.keys[skew(k)];
            const uint32_t d = digit_of<BITS>(kk, shift, a.digit_mask);
            const int64_t g = (int64_t)S.run[dix(d)] + (k - (int)S.cstart[dix(d)]);
            kout[g] = kk;
            vout[g] = S.vals[skew(k)];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < DPT; q++) S.run[dix(d0 + q)] += S.tot[dix(d0 + q)];
    }
}

static int g_sort_grid[kMaxDevices] = {};
int sort_grid() {
    const int d = current_device();
    if (d >= 0 && g_sort_grid[d] > 0) return g_sort_grid[d];
    const int g = device_sms() * kSortBlocksPerSM;
    const int grid = g < kSortMaxGrid ? g : kSortMaxGrid;
    if (d >= 0) g_sort_grid[d] = grid;
    return grid;
}

// One pass (in_buf -> in_buf ^ 1) with BITS-bit digits at `shift`.
template <typename K, int BITS>
static cudaError_t launch_pass(const SortArgs& a, int in_buf, int shift, cudaStream_t st) {
    static bool attr_set[kMaxDevices] = {};
    const size_t smem = sizeof(SortSmem<K, BITS>);
    if (a.grid < 1 || a.grid > kSortMaxGrid) return cudaErrorInvalidValue;
    cudaError_t e = once_per_device(attr_set, [&] {
        return cudaFuncSetAttribute(sort_downsweep_kernel<K, BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    });
    if (e != cudaSuccess) return e;
    sort_upsweep_kernel<K, BITS><<<a.grid, kUpThreads, 0, st>>>(a, in_buf, shift);
    sort_scan_kernel<<<(1 << BITS) / 8, 256, 0, st>>>(a);
    sort_downsweep_kernel<K, BITS><<<a.grid, kSortThreads, smem, st>>>(a, in_buf, shift);
    return cudaGetLastError();
}

cudaError_t launch_sort32(const SortArgs& a, int n_passes, const int* shifts, const int* bits, cudaStream_t st) {
    for (int p = 0; p < n_passes; p++) {
        const cudaError_t e = bits[p] == 9 ? launch_pass<uint32_t, 9>(a, p & 1, shifts[p], st)
                                           : launch_pass<uint32_t, 8>(a, p & 1, shifts[p], st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_sort64(const SortArgs& a, int n_passes, const int* shifts, cudaStream_t st) {
    for (int p = 0; p < n_passes; p++) {
        const cudaError_t e = launch_pass<unsigned long long, 8>(a, p & 1, shifts[p], st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ----------------------------------------------------------------------------------------
// Tile ranges.
// ----------------------------------------------------------------------------------------
// Each thread takes 4 consecutive sorted tile ids (one 16-byte load) and the id before them
// (from the previous lane, or loaded by lane 0); a start boundary j (key[j] != key[j - 1])
// opens key[j]'s range and closes key[j - 1]'s.
__global__ void __launch_bounds__(256) ranges_kernel(RangeArgs a) {
    if (a.counters->status != 0) return;
    const int64_t P = (int64_t)a.counters->n_pairs;
    const int64_t groups = (P + 3) / 4;
    const int lane = threadIdx.x & 31;
    for (int64_t g0 = (int64_t)blockIdx.x * blockDim.x; g0 < groups; g0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = g0 + threadIdx.x;
        const int64_t i0 = 4 * g;
        uint32_t k[4] = {0u, 0u, 0u, 0u};
        if (i0 + 3 < P) {
            const uint4 q = *reinterpret_cast<const uint4*>(a.keys + i0);
            k[0] = q.x; k[1] = q.y; k[2] = q.z; k[3] = q.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; j++) k[j] = i0 + j < P ? a.keys[i0 + j] : 0u;
        }
        uint32_t prev = __shfl_up_sync(0xffffffffu, k[3], 1);
        if (lane == 0 && i0 > 0 && i0 < P) prev = a.keys[i0 - 1];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int64_t i = i0 + j;
            if (i >= P) break;
            const uint32_t before = j == 0 ? prev : k[j - 1];
            if (i == 0 || before != k[j]) {
                a.ranges[k[j]].x = (uint32_t)i;
                if (i > 0) a.ranges[before].y = (uint32_t)i;
            }
            if (i == P - 1) a.ranges[k[j]].y = (uint32_t)P;
        }
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
