// gs_sort_pairs_noalloc: the library's stable LSD radix sort of (key, value) pairs for
// callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or forbidden -- e.g. inside
// a host callback or a real-time loop with a no-allocation policy, a plug-in whose host
// application owns every device allocation, or a process that has already reserved all of
// its memory up front.  The regular sort (gs_bin_sort) keeps its scratch in the
// caller-allocated workspace; this entry point keeps it in a fixed array compiled into the
// library instead, so the caller passes only the input and output buffers.
//
// The scratch is one file-scope __device__ array of kNoAllocBytes (13,108,480 bytes, 12.5 MiB),
// which every GPU that loads the library holds until the process exits.  It bounds a call to
// kNoAllocMaxPairs pairs.  All calls share it and it keeps the last call's contents, so
// calls that overlap on the GPU (different streams, or different host threads without
// ordering) race with each other and must be serialised by the caller.
#include <mutex>

#include "gs_kernels.cuh"

namespace gs {

constexpr int64_t kNoAllocMaxPairs = int64_t(1) << 20;
// The sort grid never exceeds kSortMaxGrid blocks (sort_grid() caps it), and each block of a
// pass owns one histogram row: the scratch holds exactly that many rows.
constexpr int kNoAllocMaxGrid = kSortMaxGrid;
constexpr size_t kNoAllocCounters = 256;
constexpr size_t kNoAllocHist = sizeof(uint32_t) * ((size_t)kSortBins * kNoAllocMaxGrid + kSortBins);
constexpr size_t kNoAllocKeys = sizeof(unsigned long long) * (size_t)kNoAllocMaxPairs;
constexpr size_t kNoAllocVals = sizeof(uint32_t) * (size_t)kNoAllocMaxPairs;
constexpr size_t kNoAllocBytes = kNoAllocCounters + kNoAllocHist + kNoAllocKeys + kNoAllocVals;

static_assert(kNoAllocBytes == 13108480, "the size stated in gs.h");
static_assert(sizeof(Counters) <= kNoAllocCounters, "counter block");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch per device, looked up on the first call made with
// that device current.  In host code the array's name is only a host-side stand-in; the
// kernels get the address returned by cudaGetSymbolAddress.
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[128] = {nullptr};

static cudaError_t noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

// The sort kernels read the pair count and the status word from a Counters block; here it
// lives at the start of the scratch and is rewritten by every call.
__global__ void noalloc_init_kernel(Counters* c, unsigned long long n) {
    if (threadIdx.x == 0) {
        c->status = 0;
        c->n_entries32 = 0;
        c->n_pairs = n;
    }
}

gs_status record_error(gs_status s, const char* msg);

// True if the byte ranges [a, a + na) and [b, b + nb) share a byte.
static bool overlap(const void* a, size_t na, const void* b, size_t nb) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

}  // namespace gs

using namespace gs;

extern "C" gs_status gs_sort_pairs_noalloc(const uint64_t* keys_in, const uint32_t* vals_in, int64_t n,
                                           int32_t key_bits, uint64_t* keys_out, uint32_t* vals_out,
                                           void* stream) {
    if (n < 0) return record_error(GS_ERR_INVALID_ARG, "n must be >= 0");
    if (n > kNoAllocMaxPairs)
        return record_error(GS_ERR_INVALID_ARG,
                               "n exceeds the 1048576-pair limit of the allocation-free sort; use gs_bin_sort with "
                               "a caller-allocated workspace");
    if (key_bits < 1 || key_bits > 64) return record_error(GS_ERR_INVALID_ARG, "key_bits must be in [1, 64]");
    if (n == 0) return GS_OK;
    if (!keys_in || !vals_in || !keys_out || !vals_out) return record_error(GS_ERR_INVALID_ARG, "NULL buffer");
    {
        const size_t kb = sizeof(uint64_t) * (size_t)n, vb = sizeof(uint32_t) * (size_t)n;
        if (overlap(keys_out, kb, keys_in, kb) || overlap(keys_out, kb, vals_in, vb) ||
            overlap(vals_out, vb, keys_in, kb) || overlap(vals_out, vb, vals_in, vb) ||
            overlap(keys_out, kb, vals_out, vb))
            return record_error(GS_ERR_INVALID_ARG,
                                "the output buffers must not overlap each other or the inputs");
    }
    void* base = nullptr;
    cudaError_t e = noalloc_scratch(&base);
    if (e != cudaSuccess) return record_error(GS_ERR_CUDA, cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* b = static_cast<unsigned char*>(base);
    Counters* cnt = reinterpret_cast<Counters*>(b);
    uint32_t* hist = reinterpret_cast<uint32_t*>(b + kNoAllocCounters);
    unsigned long long* k_tmp = reinterpret_cast<unsigned long long*>(b + kNoAllocCounters + kNoAllocHist);
    uint32_t* v_tmp = reinterpret_cast<uint32_t*>(b + kNoAllocCounters + kNoAllocHist + kNoAllocKeys);
    noalloc_init_kernel<<<1, 32, 0, st>>>(cnt, (unsigned long long)n);
    const int passes = (key_bits + 7) / 8;
    // Pass 0 reads the caller's input; the passes then alternate between the output and
    // the scratch copy so that the last one writes the output.
    unsigned long long* kout = reinterpret_cast<unsigned long long*>(keys_out);
    unsigned long long* kdst[2] = {(passes & 1) ? kout : k_tmp, (passes & 1) ? k_tmp : kout};
    uint32_t* vdst[2] = {(passes & 1) ? vals_out : v_tmp, (passes & 1) ? v_tmp : vals_out};
    SortArgs a;
    a.hist = hist;
    a.digit_tot = hist + (size_t)kSortBins * kNoAllocMaxGrid;
    a.counters = cnt;
    a.count = &cnt->n_pairs;
    a.grid = sort_grid();   // <= kSortMaxGrid = kNoAllocMaxGrid
    for (int p = 0; p < passes; p++) {
        const int shift = 8 * p;
        if (p == 0) {
            a.keys[0] = const_cast<unsigned long long*>(reinterpret_cast<const unsigned long long*>(keys_in));
            a.vals[0] = const_cast<uint32_t*>(vals_in);
        } else {
            a.keys[0] = kdst[(p - 1) & 1];
            a.vals[0] = vdst[(p - 1) & 1];
        }
        a.keys[1] = kdst[p & 1];
        a.vals[1] = vdst[p & 1];
        // the last pass takes only the key bits below key_bits
        const int top = key_bits - shift;
        a.digit_mask = top >= 8 ? 0xFFFFFFFFu : (1u << top) - 1u;
        e = launch_sort64(a, 1, &shift, st);
        if (e != cudaSuccess) return record_error(GS_ERR_CUDA, cudaGetErrorString(e));
    }
    return GS_OK;
}
