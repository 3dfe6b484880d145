// Stable LSD radix sort of (uint32 key, uint32 value) pairs, 8-bit digits.
//
// Each pass is reduce-then-scan over a FIXED grid of kSortBlocks blocks, so
// the launch shape never depends on the element count; the count may live in
// device memory (the tile-instance count is only known on the device), which
// keeps the whole binning stage free of host synchronisation.
//   upsweep:   block b histograms the digits of its contiguous chunk
//   scan:      one block per digit scans that digit's block counts and
//              writes the digit total; the downsweep adds the prefix of
//              the lower digits' totals
//   downsweep: block b ranks its chunk tile by tile (warp ranking by ballots,
//              stable), reorders each tile by digit in shared memory and
//              writes it out with coalesced runs per digit.
#include "gs_internal.cuh"

namespace gs {

constexpr int kWarps = kSortThreads / 32;
constexpr int kItems = 8;                            // per thread per tile
constexpr int kTileItems = kSortThreads * kItems;    // 2048
constexpr int kHist = kRadix * kSortBlocks;
static_assert(kRadix == kSortThreads, "one thread per digit");

size_t sort_scratch_bytes() { return (size_t)(kHist + kRadix) * sizeof(uint32_t); }

__global__ void __launch_bounds__(kSortThreads)
k_upsweep(const uint32_t *__restrict__ keys, int64_t n_host, const uint32_t *n_dev, int shift,
          uint32_t mask, uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[kWarps][kRadix];
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kWarps * kRadix; i += kSortThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    const int64_t n = sort_count(n_host, n_dev);
    const int64_t chunk = (n + kSortBlocks - 1) / kSortBlocks;
    const int64_t beg = (int64_t)blockIdx.x * chunk;
    const int64_t end = beg + chunk < n ? beg + chunk : n;
    int64_t i = beg + threadIdx.x;
    for (; i + 3 * kSortThreads < end; i += 4 * kSortThreads) {
        uint32_t k0 = __ldg(keys + i), k1 = __ldg(keys + i + kSortThreads);
        uint32_t k2 = __ldg(keys + i + 2 * kSortThreads), k3 = __ldg(keys + i + 3 * kSortThreads);
        atomicAdd(&h[warp][(k0 >> shift) & mask], 1u);
        atomicAdd(&h[warp][(k1 >> shift) & mask], 1u);
        atomicAdd(&h[warp][(k2 >> shift) & mask], 1u);
        atomicAdd(&h[warp][(k3 >> shift) & mask], 1u);
    }
    for (; i < end; i += kSortThreads) atomicAdd(&h[warp][(__ldg(keys + i) >> shift) & mask], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s += h[w][d];
        hist[(size_t)d * kSortBlocks + blockIdx.x] = s;
    }
}

// Per digit d (one block each): exclusive scan, in place, of the kSortBlocks
// block counts of digit d, and the digit's total into totals[d].
__global__ void __launch_bounds__(kSortThreads)
k_scan_digit(uint32_t *__restrict__ hist, uint32_t *__restrict__ totals) {
    constexpr int kPer = (kSortBlocks + kSortThreads - 1) / kSortThreads;
    __shared__ uint32_t warp_sums[kWarps];
    uint32_t *h = hist + (size_t)blockIdx.x * kSortBlocks;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t c[kPer];
    uint32_t local = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int idx = tid * kPer + j;
        c[j] = idx < kSortBlocks ? h[idx] : 0u;
        local += c[j];
    }
    uint32_t x = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    uint32_t before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        before += w < warp ? warp_sums[w] : 0u;
        all += warp_sums[w];
    }
    uint32_t run = x - local + before;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int idx = tid * kPer + j;
        if (idx < kSortBlocks) h[idx] = run;
        run += c[j];
    }
    if (tid == 0) totals[blockIdx.x] = all;
}

__global__ void __launch_bounds__(kSortThreads)
k_downsweep(const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
            uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, int64_t n_host,
            const uint32_t *n_dev, int shift, uint32_t mask, const uint32_t *__restrict__ hist,
            const uint32_t *__restrict__ totals) {
    __shared__ uint32_t wcnt[kWarps][kRadix];   // per-warp digit counts of the tile
    __shared__ uint32_t tile_start[kRadix];     // tile-local start of each digit
    __shared__ uint32_t gbase[kRadix];          // global start of each digit for this block
    __shared__ uint32_t gshift[kRadix];         // gbase - tile_start: output position - tile slot
    __shared__ uint2 skv[kTileItems];           // the tile reordered by digit: (key, value)
    __shared__ uint32_t scan_tmp[kWarps];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int nbits = 32 - __clz(mask);  // digit width; the value 1 << nbits marks "no item"
    const int64_t n = sort_count(n_host, n_dev);
    const int64_t chunk = (n + kSortBlocks - 1) / kSortBlocks;
    const int64_t beg = (int64_t)blockIdx.x * chunk;
    const int64_t end = beg + chunk < n ? beg + chunk : n;
    {
        // global start of digit tid = (sum of all lower digits' totals) + this
        // block's exclusive prefix within digit tid
        const uint32_t tot = totals[tid];
        uint32_t x = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) scan_tmp[warp] = x;
        __syncthreads();
        uint32_t before = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) before += w < warp ? scan_tmp[w] : 0u;
        gbase[tid] = x - tot + before + hist[(size_t)tid * kSortBlocks + blockIdx.x];
        __syncthreads();
    }

    for (int64_t t0 = beg; t0 < end; t0 += kTileItems) {
        const int tile_n = (int)((end - t0) < kTileItems ? (end - t0) : kTileItems);
        for (int i = tid; i < kWarps * kRadix; i += kSortThreads) (&wcnt[0][0])[i] = 0;
        uint32_t k[kItems], v[kItems], rank[kItems];
        int dig[kItems];
#pragma unroll
        for (int r = 0; r < kItems; ++r) {
            const int li = warp * (32 * kItems) + r * 32 + lane;  // warp owns a contiguous run
            if (li < tile_n) {
                k[r] = __ldg(keys_in + t0 + li);
                v[r] = __ldg(vals_in + t0 + li);
                dig[r] = (int)((k[r] >> shift) & mask);
            } else {
                dig[r] = 1 << nbits;  // no digit: matches only other lanes past the end
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kItems; ++r) {
            const bool has = dig[r] < (1 << nbits);
            const uint32_t peers = warp_peers((uint32_t)dig[r], nbits);
            const int leader = __ffs(peers) - 1;
            uint32_t base = 0;
            if (has) base = wcnt[warp][dig[r]];
            __syncwarp();
            if (lane == leader && has) wcnt[warp][dig[r]] = base + __popc(peers);
            __syncwarp();
            rank[r] = base + __popc(peers & lt_mask);
        }
        __syncthreads();
        // per digit: exclusive prefix over warps, and the tile total
        uint32_t total = 0;
        if (tid < kRadix) {
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                uint32_t c = wcnt[w][tid];
                wcnt[w][tid] = total;
                total += c;
            }
        }
        // exclusive scan of the digit totals (kRadix == kSortThreads)
        uint32_t x = total;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) scan_tmp[warp] = x;
        __syncthreads();
        if (tid < 32) {
            uint32_t s = tid < kWarps ? scan_tmp[tid] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            if (tid < kWarps) scan_tmp[tid] = s;
        }
        __syncthreads();
        if (tid < kRadix) {
            const uint32_t ts = x - total + (warp > 0 ? scan_tmp[warp - 1] : 0u);
            tile_start[tid] = ts;
            gshift[tid] = gbase[tid] - ts;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kItems; ++r) {
            if (dig[r] < (1 << nbits)) {
                const uint32_t pos = tile_start[dig[r]] + wcnt[warp][dig[r]] + rank[r];
                skv[pos] = make_uint2(k[r], v[r]);
            }
        }
        __syncthreads();
        for (int i = tid; i < tile_n; i += kSortThreads) {
            const uint2 kv = skv[i];
            const int d = (int)((kv.x >> shift) & mask);
            const uint32_t g = gshift[d] + (uint32_t)i;  // (unsigned wrap-around is exact)
            keys_out[g] = kv.x;
            vals_out[g] = kv.y;
        }
        __syncthreads();
        if (tid < kRadix) gbase[tid] += total;
        __syncthreads();
    }
}

int sort_pairs(uint32_t *keys_a, uint32_t *vals_a, uint32_t *keys_b, uint32_t *vals_b,
               int64_t n_host, const uint32_t *n_dev, int begin_bit, int end_bit, void *scratch,
               cudaStream_t s, int *final_buf) {
    uint32_t *hist = (uint32_t *)scratch;
    uint32_t *totals = hist + kHist;
    uint32_t *kin = keys_a, *vin = vals_a, *kout = keys_b, *vout = vals_b;
    int cur = 0;
    // as many passes as 8-bit digits need, the bits spread evenly over them
    // (13 tile bits: 7 + 6 rather than 8 + 5), which lengthens the per-digit
    // runs each block writes in the pass with the most digits
    const int passes = (end_bit - begin_bit + kRadixBits - 1) / kRadixBits;
    for (int bit = begin_bit, p = 0; bit < end_bit; ++p) {
        const int nb = (end_bit - bit + (passes - p) - 1) / (passes - p);
        const uint32_t mask = (1u << nb) - 1u;
        k_upsweep<<<kSortBlocks, kSortThreads, 0, s>>>(kin, n_host, n_dev, bit, mask, hist);
        k_scan_digit<<<kRadix, kSortThreads, 0, s>>>(hist, totals);
        k_downsweep<<<kSortBlocks, kSortThreads, 0, s>>>(kin, vin, kout, vout, n_host, n_dev, bit,
                                                         mask, hist, totals);
        bit += nb;
        uint32_t *tk = kin, *tv = vin;
        kin = kout;
        vin = vout;
        kout = tk;
        vout = tv;
        cur ^= 1;
    }
    if (final_buf) *final_buf = cur;
    return launch_error();
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_sort_scratch_bytes(int64_t n) {
    (void)n;
    return sort_scratch_bytes();
}

extern "C" int gs_sort_pairs_u32(uint32_t *keys_in, uint32_t *vals_in, uint32_t *keys_out,
                                 uint32_t *vals_out, int64_t n, int32_t begin_bit, int32_t end_bit,
                                 void *scratch, void *stream) {
    if (n < 0 || n >= (1ll << 31) || begin_bit < 0 || end_bit > 32 || begin_bit > end_bit)
        return GS_ERR_ARG;
    if (n == 0) return GS_OK;
    if (!keys_in || !vals_in || !keys_out || !vals_out || !scratch) return GS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (begin_bit == end_bit) {
        int rc = check_cuda(cudaMemcpyAsync(keys_out, keys_in, n * 4, cudaMemcpyDeviceToDevice, s));
        if (rc) return rc;
        return check_cuda(cudaMemcpyAsync(vals_out, vals_in, n * 4, cudaMemcpyDeviceToDevice, s));
    }
    int final_buf = 0;
    int rc = sort_pairs(keys_in, vals_in, keys_out, vals_out, n, nullptr, begin_bit, end_bit,
                        scratch, s, &final_buf);
    if (rc) return rc;
    if (final_buf == 0) {  // an even number of passes ends in the input buffers
        rc = check_cuda(cudaMemcpyAsync(keys_out, keys_in, n * 4, cudaMemcpyDeviceToDevice, s));
        if (rc) return rc;
        rc = check_cuda(cudaMemcpyAsync(vals_out, vals_in, n * 4, cudaMemcpyDeviceToDevice, s));
    }
    return rc;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of gs_sort_pairs_u32.
//
// Some callers cannot hand the sort a scratch buffer: plug-ins living
// inside a framework whose memory pool owns all device memory, code that
// runs under a fixed device-memory budget, and latency-critical loops that
// cannot afford cudaMalloc's implicit device synchronisation.  This entry
// point keeps its scratch in a file-scope __device__ array instead.  The
// array holds the per-pass digit histogram of the fixed-grid sort,
// kRadix * kSortBlocks + kRadix 32-bit counters (609 KiB); it does not grow
// with n, and every GPU that loads the library keeps it until the process
// exits.
#include <mutex>

namespace gs {

__device__ __align__(256) uint32_t g_noalloc_sort_scratch[kHist + kRadix];

constexpr int kNoallocMaxDevices = 64;
static uint32_t *g_noalloc_ptr[kNoallocMaxDevices];
static std::mutex g_noalloc_mutex;

// Device address of the scratch array for the current device, looked up once
// per device (with that device current) and cached for the life of the
// process (a cudaDeviceReset invalidates it; the header says so).
static int noalloc_scratch(uint32_t **out) {
    int dev = 0;
    int rc = check_cuda(cudaGetDevice(&dev));
    if (rc) return rc;
    if (dev < 0 || dev >= kNoallocMaxDevices) return GS_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        rc = check_cuda(cudaGetSymbolAddress(&p, g_noalloc_sort_scratch));
        if (rc) return rc;
        g_noalloc_ptr[dev] = (uint32_t *)p;
    }
    *out = g_noalloc_ptr[dev];
    return GS_OK;
}

}  // namespace gs

extern "C" int gs_sort_pairs_u32_noalloc(uint32_t *keys_in, uint32_t *vals_in, uint32_t *keys_out,
                                         uint32_t *vals_out, int64_t n, int32_t begin_bit,
                                         int32_t end_bit, void *stream) {
    if (n < 0 || n > GS_SORT_NOALLOC_MAX_N || begin_bit < 0 || end_bit > 32 || begin_bit > end_bit)
        return GS_ERR_ARG;
    if (n == 0) return GS_OK;
    if (!keys_in || !vals_in || !keys_out || !vals_out) return GS_ERR_ARG;
    uint32_t *scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    // The histogram is fully rewritten by every pass, so no clearing is needed.
    return gs_sort_pairs_u32(keys_in, vals_in, keys_out, vals_out, n, begin_bit, end_bit, scratch,
                             stream);
}
