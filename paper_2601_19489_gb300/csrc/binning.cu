// a2-a4: binning (Sec. 2.1).
//
//  1. depth sort: radix sort of the (view, Gaussian) items by camera depth
//     (float bits of z > 0 order like the floats; culled items carry the
//     largest key).  Items of different views interleave, which is harmless:
//     an item only ever writes tiles of its own view.
//  2. scan of the tile counts in depth order (fixed grid, no host sync): the
//     block sums, scanned by the block that finishes last (which also
//     publishes the instance count and the capacity overflow flag), and the
//     key-write pass that rescans inside each block.
//  3. key write, one (global tile id, item) instance per touched tile:
//     load-balanced (Fig. 2): the SnugBox columns of a warp's 32 Gaussians
//     form one flat list that the lanes walk one column each, so every lane
//     evaluates a per-column ellipse test whatever the Gaussians' sizes, and
//     a segmented warp scan places each column's tiles;
//     sequential ("Sq"): one thread walks its Gaussian's columns.
//     Each round of Gaussians writes its (contiguous) run of instances.
//  4. stable radix sort of the instances by tile id: every tile's list keeps
//     the depth order of step 1, ties in depth by ascending Gaussian index.
//  5. tile ranges by binary search in the sorted ids.  (Each tile's first
//     checkpoint bucket is taken by the forward, one atomic per tile.)
// Steps 2-5 are the radix path (load_balanced = 0, or the plan's bin_radix);
// the default path replaces them with the counting binning further below,
// which writes every instance once, straight to its place in its tile's
// list, with no key array and no sort of the instances.
#include "gs_internal.cuh"

namespace gs {

constexpr int kScanThreads = 256;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t *warp_tmp,
                                                         uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tmp[warp] = inc;
    __syncthreads();
    uint32_t before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) {
        const uint32_t s = warp_tmp[w];
        before += w < warp ? s : 0u;
        all += s;
    }
    __syncthreads();
    *total = all;
    return inc - x + before;
}

__device__ __forceinline__ void chunk_of(int64_t n, int64_t *beg, int64_t *end) {
    const int64_t chunk = (n + kBinBlocks - 1) / kBinBlocks;
    *beg = (int64_t)blockIdx.x * chunk;
    *end = *beg + chunk < n ? *beg + chunk : n;
}

// Block b sums the tile counts of its chunk of depth ranks into
// block_sums[b]; the block that finishes last (a counter in the status
// words, cleared by gs_bin_sort) then scans the block sums (64-bit) into
// block_offs and publishes the instance count (saturated to 32 bits) and the
// overflow flag.  Thread t of that block owns the kCountPer consecutive sums
// from t * kCountPer.
constexpr int kCountPer = (kBinBlocks + kScanThreads - 1) / kScanThreads;

// The (Gaussian, block) entries of the counting binning: the 8 x 8-tile
// blocks its tile rectangle meets (none for a culled Gaussian).
__device__ __forceinline__ uint32_t coarse_blocks(const uint32_t *__restrict__ touched,
                                                  const uint2 *__restrict__ rects, uint32_t item) {
    if (!touched[item]) return 0u;
    int tx0, ty0, tx1, ty1;
    unpack_rect(rects[item], &tx0, &ty0, &tx1, &ty1);
    return (uint32_t)((((tx1 - 1) / kBlk) - tx0 / kBlk + 1) * (((ty1 - 1) / kBlk) - ty0 / kBlk + 1));
}

// kCoarse = false: scans the tile instances (touched) and publishes n_inst
// (and the overflow flag against capacity).  kCoarse = true: scans the
// (Gaussian, block) entries into block_offs and publishes n_coarse; the
// tile instances are only summed (their block sums in inst_sums) and
// published as n_inst, so the instance count is exact even when the entries
// overflow; the overflow flag covers both (capacity holds both).
template <bool kCoarse>
__global__ void __launch_bounds__(kScanThreads)
k_count(const uint32_t *__restrict__ order, const uint32_t *__restrict__ touched, const uint2 *__restrict__ rects,
        int64_t n, uint32_t *__restrict__ block_sums, unsigned long long *__restrict__ block_offs, StatusDev *st,
        int64_t capacity, uint32_t *__restrict__ inst_sums) {
    __shared__ uint32_t tmp[kScanThreads / 32];
    __shared__ unsigned long long tmp64[kScanThreads / 32];
    __shared__ bool s_last;
    int64_t beg, end;
    chunk_of(n, &beg, &end);
    uint32_t s = 0, si = 0;
    for (int64_t r = beg + threadIdx.x; r < end; r += kScanThreads) {
        const uint32_t item = order[r];
        if (kCoarse) {
            s += coarse_blocks(touched, rects, item);
            si += touched[item];
        } else {
            s += touched[item];
        }
    }
    uint32_t total, total_i = 0;
    block_exclusive_scan(s, tmp, &total);
    if (kCoarse) block_exclusive_scan(si, tmp, &total_i);
    if (threadIdx.x == 0) {
        block_sums[blockIdx.x] = total;
        if (kCoarse) inst_sums[blockIdx.x] = total_i;
        __threadfence();  // the sums are visible before this block counts as done
        s_last = atomicAdd(&st->done_blocks, 1u) == (uint32_t)kBinBlocks - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long own[kCountPer];
    unsigned long long x = 0;
#pragma unroll
    for (int k = 0; k < kCountPer; ++k) {
        const int b = tid * kCountPer + k;
        own[k] = b < kBinBlocks ? __ldcg(block_sums + b) : 0ull;
        x += own[k];
    }
    unsigned long long inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) tmp64[warp] = inc;
    __syncthreads();
    unsigned long long before = 0, all = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) {
        before += w < warp ? tmp64[w] : 0ull;
        all += tmp64[w];
    }
    unsigned long long run = inc - x + before;
#pragma unroll
    for (int k = 0; k < kCountPer; ++k) {
        const int b = tid * kCountPer + k;
        if (b < kBinBlocks) block_offs[b] = run;
        run += own[k];
    }
    unsigned long long all_i = all;
    if (kCoarse) {
        // the instance total: the block sums of touched, summed
        unsigned long long xi = 0;
#pragma unroll
        for (int k = 0; k < kCountPer; ++k) {
            const int b = tid * kCountPer + k;
            xi += b < kBinBlocks ? __ldcg(inst_sums + b) : 0ull;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) xi += __shfl_xor_sync(0xffffffffu, xi, o);
        __syncthreads();
        if (lane == 0) tmp64[warp] = xi;
        __syncthreads();
        all_i = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) all_i += tmp64[w];
    }
    if (tid == 0) {
        const auto sat = [](unsigned long long v) { return v > 0xffffffffull ? 0xffffffffu : (uint32_t)v; };
        if (kCoarse) st->n_coarse = sat(all);
        st->n_inst = sat(all_i);
        st->overflow = (all > (unsigned long long)capacity || all_i > (unsigned long long)capacity) ? 1u : 0u;
        st->done_blocks = 0;
    }
}

// Instance key write.  Block b takes the chunk of depth ranks whose count it
// summed, in rounds of kWriteRound ranks: a block scan of their tile counts
// gives each Gaussian its slot range, and the round's instances (one
// contiguous run of the output) are written straight to global memory, where
// L2 merges the lanes' neighbouring writes.  (Assembling each run in shared
// memory first was measured slower: it limited the blocks per SM.)
constexpr int kWriteRound = 128;

__device__ __forceinline__ uint32_t block_exclusive_scan128(uint32_t x, uint32_t *warp_tmp, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tmp[warp] = inc;
    __syncthreads();
    uint32_t before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kWriteRound / 32; ++w) {
        const uint32_t v = warp_tmp[w];
        before += w < warp ? v : 0u;
        all += v;
    }
    __syncthreads();
    *total = all;
    return inc - x + before;
}

struct WriteSink {
    uint32_t *g_tile, *g_item;       // output (global)
    unsigned long long round_base;   // global position of the round's first instance
    unsigned long long capacity;
    __device__ __forceinline__ void put(uint32_t local, uint32_t tile, uint32_t item) const {
        const unsigned long long pos = round_base + local;
        if (pos < capacity) {
            g_tile[pos] = tile;
            g_item[pos] = item;
        }
    }
};

template <bool kLB>
__global__ void __launch_bounds__(kWriteRound)
k_write_keys(ViewsDev views, int64_t n_per_view, const uint32_t *__restrict__ order,
             const uint32_t *__restrict__ touched, const float4 *__restrict__ rec,
             const float2 *__restrict__ bin, const uint2 *__restrict__ rects,
             const unsigned long long *__restrict__ block_offs, int64_t n, int64_t capacity,
             uint32_t *__restrict__ inst_tile, uint32_t *__restrict__ inst_item, StatusDev *st, int box3) {
    __shared__ uint32_t tmp[kWriteRound / 32];
    int64_t beg, end;
    chunk_of(n, &beg, &end);
    unsigned long long base = block_offs[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t r0 = beg; r0 < end; r0 += kWriteRound) {
        const int64_t r = r0 + threadIdx.x;
        uint32_t item = 0, cnt = 0;
        if (r < end) {
            item = order[r];
            cnt = touched[item];
        }
        uint32_t total;
        const uint32_t off = block_exclusive_scan128(cnt, tmp, &total);
        WriteSink sink{inst_tile, inst_item, base, (unsigned long long)capacity};
        if (!kLB) {
            // one thread per Gaussian walks its columns
            if (cnt) {
                const int v = (int)(item / (uint32_t)n_per_view);
                const ViewDev &cam = views.v[v];
                const float4 r0v = rec[3 * (size_t)item];
                const float2 bv = bin[item];
                BinGeom bg{};
                if (!box3) bin_geom(r0v.x, r0v.y, r0v.z, r0v.w, rec[3 * (size_t)item + 1].x, bv.y, bv.x, bg);
                int tx0, ty0, tx1, ty1;
                unpack_rect(rects[item], &tx0, &ty0, &tx1, &ty1);
                uint32_t w = 0;
                for (int tx = tx0; tx < tx1; ++tx) {
                    float xa, xb;
                    column_span(tx, (float)cam.W, &xa, &xb);
                    int lo = ty0, hi = ty1 - 1;  // the whole box column (3-sigma box)
                    if (!box3 && !column_rows(bg, xa, xb, (float)cam.H, ty0, ty1, &lo, &hi)) continue;
                    for (int ty = lo; ty <= hi; ++ty, ++w)
                        if (w < cnt) sink.put(off + w, (uint32_t)(cam.tile_off + ty * cam.tiles_x + tx), item);
                }
                if (w != cnt) {
                    // keep every slot valid (cannot happen while the count and
                    // the write share column_rows)
                    atomicCAS(&st->error, 0, GS_ERR_INTERNAL);
                    for (; w < cnt; ++w) sink.put(off + w, (uint32_t)(cam.tile_off + ty0 * cam.tiles_x + tx0), item);
                }
            }
        } else {
            // load-balanced: the columns of the warp's 32 Gaussians are laid out
            // in one flat list and every lane takes one column at a time, so
            // all lanes work whatever the Gaussians' sizes; a segmented warp
            // scan of the row counts places each column's tiles.
            __shared__ uint32_t s_carry[kWriteRound];  // tiles placed so far, per Gaussian
            BinGeom my{};
            int mtx0 = 0, mty0 = 0, mtx1 = 0, mty1 = 0, mtoff = 0, mtiles_x = 0, mW = 0, mH = 0;
            if (cnt) {
                const int v = (int)(item / (uint32_t)n_per_view);
                const ViewDev &cam = views.v[v];
                const float4 r0v = rec[3 * (size_t)item];
                const float2 bv = bin[item];
                if (!box3) bin_geom(r0v.x, r0v.y, r0v.z, r0v.w, rec[3 * (size_t)item + 1].x, bv.y, bv.x, my);
                unpack_rect(rects[item], &mtx0, &mty0, &mtx1, &mty1);
                mtoff = cam.tile_off;
                mtiles_x = cam.tiles_x;
                mW = cam.W;
                mH = cam.H;
            }
            s_carry[threadIdx.x] = 0;
            const uint32_t ncols = cnt ? (uint32_t)(mtx1 - mtx0) : 0u;
            uint32_t colpref = ncols;  // inclusive, then exclusive scan of column counts
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, colpref, o);
                if (lane >= o) colpref += y;
            }
            const uint32_t n_cols = __shfl_sync(0xffffffffu, colpref, 31);
            colpref -= ncols;
            __syncwarp();
            for (uint32_t c0 = 0; c0 < n_cols; c0 += 32) {
                const uint32_t f = c0 + lane;
                const bool has = f < n_cols;
                // owner: the last lane j with colpref_j <= f (binary search)
                int j = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const uint32_t cp = __shfl_sync(0xffffffffu, colpref, j + step);
                    if (cp <= f) j += step;
                }
                BinGeom bg;
                bg.mx = __shfl_sync(0xffffffffu, my.mx, j);
                bg.my = __shfl_sync(0xffffffffu, my.my, j);
                bg.B = __shfl_sync(0xffffffffu, my.B, j);
                bg.detc = __shfl_sync(0xffffffffu, my.detc, j);
                bg.tC = __shfl_sync(0xffffffffu, my.tC, j);
                bg.invC = __shfl_sync(0xffffffffu, my.invC, j);
                bg.dx_top = __shfl_sync(0xffffffffu, my.dx_top, j);
                bg.rx = __shfl_sync(0xffffffffu, my.rx, j);
                bg.ry = __shfl_sync(0xffffffffu, my.ry, j);
                const int tx0 = __shfl_sync(0xffffffffu, mtx0, j), ty0 = __shfl_sync(0xffffffffu, mty0, j);
                const int ty1 = __shfl_sync(0xffffffffu, mty1, j);
                const int toff = __shfl_sync(0xffffffffu, mtoff, j);
                const int tiles_x = __shfl_sync(0xffffffffu, mtiles_x, j);
                const float fW = (float)__shfl_sync(0xffffffffu, mW, j);
                const float fH = (float)__shfl_sync(0xffffffffu, mH, j);
                const uint32_t cp_j = __shfl_sync(0xffffffffu, colpref, j);
                const uint32_t it = __shfl_sync(0xffffffffu, item, j);
                const uint32_t o0 = __shfl_sync(0xffffffffu, off, j);
                const uint32_t c_j = __shfl_sync(0xffffffffu, cnt, j);
                const int tx = tx0 + (int)(f - cp_j);
                int lo = 0, hi = -1, rows = 0;
                if (has) {
                    if (box3) {  // the whole box column (3-sigma box)
                        lo = ty0;
                        hi = ty1 - 1;
                        rows = ty1 - ty0;
                    } else {
                        float xa, xb;
                        column_span(tx, fW, &xa, &xb);
                        rows = column_rows(bg, xa, xb, fH, ty0, ty1, &lo, &hi);
                    }
                }
                // segmented exclusive scan of rows over the chunk (segments =
                // runs of equal owner)
                uint32_t inc = (uint32_t)rows;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += y;
                }
                const bool head = lane == 0 || f == cp_j;
                const uint32_t heads = __ballot_sync(0xffffffffu, head);
                const int seg_lane = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
                const uint32_t before_seg = __shfl_sync(0xffffffffu, inc, seg_lane > 0 ? seg_lane - 1 : 0);
                const uint32_t seg_excl = inc - (uint32_t)rows - (seg_lane > 0 ? before_seg : 0u);
                const uint32_t w0 = s_carry[warp * 32 + j] + seg_excl;
                for (int ty = lo; ty <= hi; ++ty) {
                    const uint32_t w = w0 + (uint32_t)(ty - lo);
                    if (w < c_j) sink.put(o0 + w, (uint32_t)(toff + ty * tiles_x + tx), it);
                }
                __syncwarp();
                // the last column of each segment advances its Gaussian's count
                const bool tail = has && (lane == 31 || ((heads >> (lane + 1)) & 1u) || f + 1 == n_cols);
                if (tail) s_carry[warp * 32 + j] += seg_excl + (uint32_t)rows;
                __syncwarp();
            }
            if (cnt && s_carry[threadIdx.x] != cnt) {
                // keep every slot valid (cannot happen while the count and the
                // write share column_rows)
                atomicCAS(&st->error, 0, GS_ERR_INTERNAL);
                for (uint32_t w = s_carry[threadIdx.x]; w < cnt; ++w)
                    sink.put(off + w, (uint32_t)(mtoff + mty0 * mtiles_x + mtx0), item);
            }
        }
        base += total;
    }
}

// [start, end) of every tile in the sorted tile ids by binary search (one
// thread per tile): every range is written, empty tiles get start == end.
__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t *__restrict__ a, uint32_t n, uint32_t v) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(256)
k_tile_ranges(const uint32_t *__restrict__ keys, const StatusDev *st, int64_t capacity,
              uint32_t total_tiles, uint2 *__restrict__ ranges) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total_tiles) return;
    int64_t n64 = st->n_inst;
    if (n64 > capacity) n64 = capacity;
    const uint32_t n = (uint32_t)n64;
    ranges[t] = make_uint2(lower_bound_u32(keys, n, t), lower_bound_u32(keys, n, t + 1));
}

// ============================================================================
// Counting binning (the default path of gs_bin_sort).
//
// The tiles are grouped in blocks of kBlk x kBlk.  After the depth sort:
//  1. k_count<true>: each visible Gaussian's number of blocks its tile
//     rectangle meets, scanned in depth order (n_coarse);
//  2. k_coarse_write: one (block id, item) entry per such block, in depth
//     order;
//  3. a stable radix sort of the entries by block id (block_bits bits): every
//     block's entries stay in depth order;
//  4. k_block_bounds: each block's [start, end) among the sorted entries;
//  5. k_chunk_scan: each block's entries cut into chunks of kChunk, the
//     chunks of all blocks numbered by a scan;
//  6. k_fine_mask: a warp per chunk (claimed from a counter) computes every
//     entry's 64-bit mask of
//     the block's tiles its Gaussian touches (exact column test), stores it
//     and counts the chunk's instances per tile;
//  7. k_fine_offsets: a CTA per block turns the counts into each chunk's
//     first position per tile (the block's tiles in column-major order, each
//     tile's chunks in order); the CTA that finishes last scans the block
//     totals into block bases and checks their sum against the instance
//     count;
//  8. k_fine_scatter: a warp per chunk (claimed from a counter), a lane per
//     two tiles, walks the chunk's entries in order and writes each item at the next position of every
//     tile in its mask; the tile ranges come from the block bases.
// Each tile's list therefore keeps the entries' order, which is the depth
// order: the same lists as the radix path's.

__device__ __forceinline__ int view_of_block(const ViewsDev &vd, int b) {
    int v = 0;
    while (v + 1 < vd.V && b >= vd.v[v + 1].block_off) ++v;
    return v;
}

__global__ void __launch_bounds__(kWriteRound)
k_coarse_write(ViewsDev views, int64_t n_per_view, const uint32_t *__restrict__ order,
               const uint32_t *__restrict__ touched, const uint2 *__restrict__ rects,
               const unsigned long long *__restrict__ block_offs, int64_t n, int64_t capacity,
               uint32_t *__restrict__ ckey, uint32_t *__restrict__ cval) {
    __shared__ uint32_t tmp[kWriteRound / 32];
    int64_t beg, end;
    chunk_of(n, &beg, &end);
    unsigned long long base = block_offs[blockIdx.x];
    for (int64_t r0 = beg; r0 < end; r0 += kWriteRound) {
        const int64_t r = r0 + threadIdx.x;
        uint32_t item = 0, cnt = 0;
        if (r < end) {
            item = order[r];
            cnt = coarse_blocks(touched, rects, item);
        }
        uint32_t total;
        const uint32_t off = block_exclusive_scan128(cnt, tmp, &total);
        if (cnt) {
            const ViewDev &cam = views.v[item / (uint32_t)n_per_view];
            int tx0, ty0, tx1, ty1;
            unpack_rect(rects[item], &tx0, &ty0, &tx1, &ty1);
            uint32_t w = 0;
            for (int by = ty0 / kBlk; by <= (ty1 - 1) / kBlk; ++by)
                for (int bx = tx0 / kBlk; bx <= (tx1 - 1) / kBlk; ++bx, ++w) {
                    const unsigned long long pos = base + off + w;
                    if (pos < (unsigned long long)capacity) {
                        ckey[pos] = (uint32_t)(cam.block_off + by * cam.blocks_x + bx);
                        cval[pos] = item;
                    }
                }
        }
        base += total;
    }
}

// [start, end) of every block that has entries (the caller zeroes brange).
__global__ void __launch_bounds__(256)
k_block_bounds(const uint32_t *__restrict__ ckey, const StatusDev *st, int64_t capacity, uint2 *__restrict__ brange) {
    int64_t n = st->n_coarse;
    if (n > capacity) n = capacity;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        const uint32_t k = ckey[i];
        if (i == 0 || ckey[i - 1] != k) brange[k].x = (uint32_t)i;
        if (i + 1 == n || ckey[i + 1] != k) brange[k].y = (uint32_t)(i + 1);
    }
}

// One CTA: bchunk[b] = chunks of the blocks before b, bchunk[nblocks] = all
// chunks (also published as n_chunks).  Thread t owns a contiguous range of
// blocks.
constexpr int kChunkScanThreads = 1024;

// Exclusive scan of x over the CTA (kChunkScanThreads threads).
__device__ __forceinline__ uint32_t cta_exclusive_scan1024(uint32_t x, uint32_t *warp_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = warp_tot[lane], wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        warp_tot[lane] = wi - w;
    }
    __syncthreads();
    const uint32_t r = inc - x + warp_tot[warp];
    __syncthreads();  // warp_tot is free again
    return r;
}

// With totals (the entries per block, when the entries were sorted in one
// pass whose digit is the block id: the sort's digit totals), brange is
// written here from their scan; otherwise k_block_bounds wrote it.
__global__ void __launch_bounds__(kChunkScanThreads)
k_chunk_scan(uint2 *__restrict__ brange, const uint32_t *__restrict__ totals, int nblocks,
             uint32_t *__restrict__ bchunk, StatusDev *st) {
    __shared__ uint32_t warp_tot[kChunkScanThreads / 32];
    const int tid = threadIdx.x;
    const int per = (nblocks + kChunkScanThreads - 1) / kChunkScanThreads;
    const int b0 = min(tid * per, nblocks), b1 = min(b0 + per, nblocks);
    if (totals) {
        uint32_t sum = 0;
        for (int b = b0; b < b1; ++b) sum += totals[b];
        uint32_t run = cta_exclusive_scan1024(sum, warp_tot);
        for (int b = b0; b < b1; ++b) {
            brange[b] = make_uint2(run, run + totals[b]);
            run += totals[b];
        }
        __syncthreads();  // brange is read back below by other threads
    }
    uint32_t local = 0;
    for (int b = b0; b < b1; ++b) {
        const uint2 r = brange[b];
        local += (r.y - r.x + kChunk - 1) / kChunk;
    }
    uint32_t run = cta_exclusive_scan1024(local, warp_tot);
    for (int b = b0; b < b1; ++b) {
        bchunk[b] = run;
        const uint2 r = brange[b];
        run += (r.y - r.x + kChunk - 1) / kChunk;
    }
    if (tid == kChunkScanThreads - 1) {
        bchunk[nblocks] = run;
        st->n_chunks = run;
    }
}

constexpr int kFineWarps = 4;
constexpr int kFineCtas = 152 * 16;

// The chunk c of a warp: its block b (bchunk[b] <= c < bchunk[b + 1]) and
// its entries [e0, e1).
__device__ __forceinline__ int chunk_block(const uint32_t *__restrict__ bchunk, int nblocks, uint32_t c) {
    int lo = 0, hi = nblocks;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (bchunk[mid] <= c) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Tiles of a block are numbered column-major, t = 8 cx + cy, so an entry's
// tile set is a 64-bit mask whose byte cx holds the rows of column cx; it is
// kept as two words (columns 0-3, columns 4-7).

// 32 x 32 bit-matrix transpose across a warp: lane i holds row i (bit j =
// element (i, j)); afterwards lane j holds column j (bit i = element (i, j)).
// Five butterfly stages: at stage s, lanes i and i ^ s exchange the s x s
// blocks whose row and column bit s differ.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
    uint32_t m = 0x0000ffffu;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, s);
        x = (lane & s) ? ((x & ~m) | ((y & ~m) >> s)) : ((x & m) | ((y & m) << s));
        m ^= m << (s >> 1);
    }
    return x;
}

// Pass 1: a warp per chunk; its entries go 32 at a time, one per lane.  A
// lane computes its entry's mask — for every in-block column of the
// entry's tile rectangle, the rows of the exact column test (the same test
// as the tile count) — and stores it; then the warp counts the chunk's
// instances per tile (lane l: tiles l and l + 32) into ccnt[chunk][64].
// The columns are visited in lockstep over the union of the lanes'
// column ranges, so the lanes share one loop.
__global__ void __launch_bounds__(kFineWarps * 32)
k_fine_mask(ViewsDev views, const uint32_t *__restrict__ cval, const uint2 *__restrict__ brange,
            const uint32_t *__restrict__ bchunk, const float4 *__restrict__ rec, const float2 *__restrict__ bin,
            const uint2 *__restrict__ rects, uint32_t *__restrict__ mlo, uint32_t *__restrict__ mhi,
            uint32_t *__restrict__ ccnt, StatusDev *st, int box3) {
    const int lane = threadIdx.x & 31;
    const int nblocks = views.total_blocks;
    const uint32_t n_chunks = st->n_chunks;
    // chunks claimed one at a time from a counter: their instance counts
    // differ widely, so a fixed assignment leaves some SMs working long
    // after the others
    for (;;) {
        uint32_t c = 0;
        if (lane == 0) c = atomicAdd(&st->next_mask_chunk, 1u);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= n_chunks) break;
        const int b = chunk_block(bchunk, nblocks, c);
        const uint2 br = brange[b];
        const uint32_t e0 = br.x + (c - bchunk[b]) * (uint32_t)kChunk;
        const uint32_t e1 = min(e0 + (uint32_t)kChunk, br.y);
        const ViewDev &cam = views.v[view_of_block(views, b)];
        const int lb = b - cam.block_off;
        const int btx0 = (lb % cam.blocks_x) * kBlk, bty0 = (lb / cam.blocks_x) * kBlk;
        const float fW = (float)cam.W, fH = (float)cam.H;
        uint32_t cnt0 = 0, cnt1 = 0;
        for (uint32_t s0 = e0; s0 < e1; s0 += 32) {
            const uint32_t e = s0 + (uint32_t)lane;
            BinGeom g{};
            int xa = kBlk, xb = 0, ry0 = 0, ry1 = 0;  // in-block column range [xa, xb)
            if (e < e1) {
                const uint32_t item = cval[e];
                const float4 r0v = rec[3 * (size_t)item];
                const float2 bv = bin[item];
                if (!box3) bin_geom(r0v.x, r0v.y, r0v.z, r0v.w, rec[3 * (size_t)item + 1].x, bv.y, bv.x, g);
                int tx0, ty0, tx1, ty1;
                unpack_rect(rects[item], &tx0, &ty0, &tx1, &ty1);
                ry0 = max(ty0, bty0);
                ry1 = min(ty1, bty0 + kBlk);
                if (ry1 > ry0) {
                    xa = max(tx0, btx0) - btx0;
                    xb = min(tx1, btx0 + kBlk) - btx0;
                }
            }
            const int xmin = (int)__reduce_min_sync(0xffffffffu, (unsigned)xa);
            const int xmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)xb);
            uint32_t lo32 = 0, hi32 = 0;
            for (int X = xmin; X < xmax; ++X) {
                if (X >= xa && X < xb) {
                    int rlo = ry0, rhi = ry1 - 1;
                    bool any = true;
                    if (!box3) {
                        float pa, pb;
                        column_span(btx0 + X, fW, &pa, &pb);
                        any = column_rows(g, pa, pb, fH, ry0, ry1, &rlo, &rhi) > 0;
                    }
                    if (any) {
                        const uint32_t rowbits = ((2u << (rhi - rlo)) - 1u) << (rlo - bty0);
                        if (X < 4) lo32 |= rowbits << (8 * X);
                        else hi32 |= rowbits << (8 * (X - 4));
                    }
                }
            }
            if (e < e1) {
                mlo[e] = lo32;
                mhi[e] = hi32;
            }
            // lane l: the step's entries that touch tiles l and l + 32
            cnt0 += __popc(warp_transpose32(lo32, lane));
            cnt1 += __popc(warp_transpose32(hi32, lane));
        }
        ccnt[(size_t)c * kBlkTiles + lane] = cnt0;
        ccnt[(size_t)c * kBlkTiles + 32 + lane] = cnt1;
    }
}

// Pass 2: ccnt holds each chunk's first block-local position per tile and
// bbase the block bases.  A warp per chunk, lane l owning tiles l and
// l + 32: 32 entries at a time, the warp transposes their masks so that lane
// l holds, as bits, which of the entries touch its tiles, and appends those
// entries' items to its runs in entry order, so each run keeps the entries'
// (depth) order by construction.  The runs are
// staged in shared memory a 32-byte sector at a time: a lane writes a
// sector once it is full (two 16-byte stores), and only the sectors its run
// shares with a neighbour's (its first and last) word by word, so the
// instance list is written in whole sectors rather than one scattered word
// per instance.  The warps also write the tile ranges (a block per warp).
struct RunStage {
    uint32_t r;    // next position of the run
    uint32_t lo;   // first slot of the current sector that belongs to the run
};

__device__ __forceinline__ void run_flush_partial(const RunStage &rs, const uint32_t *slot, uint32_t cap,
                                                  uint32_t *__restrict__ out) {
    const uint32_t sec = rs.r & ~7u;
    for (uint32_t j = rs.lo; j < (rs.r & 7u); ++j)
        if (sec + j < cap) out[sec + j] = slot[j];
}

__device__ __forceinline__ void run_append(RunStage &rs, uint32_t *slot, uint32_t x, uint32_t cap,
                                           uint32_t *__restrict__ out) {
    slot[rs.r & 7u] = x;
    ++rs.r;
    if ((rs.r & 7u) == 0u) {  // the sector [r - 8, r) is complete
        const uint32_t sec = rs.r - 8u;
        if (rs.lo == 0u && rs.r <= cap) {
            uint4 *o = reinterpret_cast<uint4 *>(out + sec);
            o[0] = make_uint4(slot[0], slot[1], slot[2], slot[3]);
            o[1] = make_uint4(slot[4], slot[5], slot[6], slot[7]);
        } else {
            for (uint32_t j = rs.lo; j < 8u; ++j)
                if (sec + j < cap) out[sec + j] = slot[j];
        }
        rs.lo = 0u;
    }
}

constexpr int kStageStride = 9;  // words per staged sector (8 + 1 against bank conflicts)

__global__ void __launch_bounds__(kFineWarps * 32)
k_fine_scatter(ViewsDev views, const uint32_t *__restrict__ cval, const uint2 *__restrict__ brange,
               const uint32_t *__restrict__ bchunk, const uint32_t *__restrict__ mlo,
               const uint32_t *__restrict__ mhi, const uint32_t *__restrict__ ccnt,
               const uint32_t *__restrict__ bbase, const uint2 *__restrict__ btile, StatusDev *st,
               int64_t capacity, uint32_t *__restrict__ inst_item, uint2 *__restrict__ ranges) {
    __shared__ uint32_t s_stage[kFineWarps][kBlkTiles * kStageStride];
    __shared__ uint32_t s_item[kFineWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * kFineWarps + warp, nw = gridDim.x * kFineWarps;
    const int nblocks = views.total_blocks;
    const uint32_t cap = (uint32_t)capacity;
    for (int b = gw; b < nblocks; b += nw) {
        const ViewDev &cam = views.v[view_of_block(views, b)];
        const int lb = b - cam.block_off;
        const int bx = lb % cam.blocks_x, by = lb / cam.blocks_x;
        const uint32_t base = bbase[b];
        for (int t = lane; t < kBlkTiles; t += 32) {
            const int tx = bx * kBlk + t / kBlk, ty = by * kBlk + t % kBlk;
            if (tx < cam.tiles_x && ty < cam.tiles_y) {
                const uint2 bt = btile[(size_t)b * kBlkTiles + t];
                const uint32_t s = min(base + bt.x, cap), e = min(base + bt.x + bt.y, cap);
                ranges[cam.tile_off + ty * cam.tiles_x + tx] = make_uint2(s, e);
            }
        }
    }
    uint32_t *slot0 = s_stage[warp] + lane * kStageStride;
    uint32_t *slot1 = s_stage[warp] + (lane + 32) * kStageStride;
    const uint32_t n_chunks = st->n_chunks;
    for (;;) {  // chunks claimed one at a time, as in k_fine_mask
        uint32_t c = 0;
        if (lane == 0) c = atomicAdd(&st->next_scatter_chunk, 1u);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= n_chunks) break;
        const int b = chunk_block(bchunk, nblocks, c);
        const uint2 br = brange[b];
        const uint32_t e0 = br.x + (c - bchunk[b]) * (uint32_t)kChunk;
        const uint32_t e1 = min(e0 + (uint32_t)kChunk, br.y);
        const uint32_t base = bbase[b];
        // the runs of tiles lane and lane + 32 (a base parked at the capacity
        // keeps every position there or beyond: no write)
        RunStage rs0, rs1;
        rs0.r = min(base + ccnt[(size_t)c * kBlkTiles + lane], cap);
        rs1.r = min(base + ccnt[(size_t)c * kBlkTiles + 32 + lane], cap);
        rs0.lo = rs0.r & 7u;
        rs1.lo = rs1.r & 7u;
        uint32_t *items = s_item[warp];
        for (uint32_t s0 = e0; s0 < e1; s0 += 32) {
            const uint32_t e = s0 + (uint32_t)lane;
            uint32_t lo = 0, hi = 0, it = 0;
            if (e < e1) {
                lo = mlo[e];
                hi = mhi[e];
                it = cval[e];
            }
            items[lane] = it;
            // lane l: bit k set when the step's entry k touches tile l (w0)
            // or l + 32 (w1); the set bits in order are the run's entries
            uint32_t w0 = warp_transpose32(lo, lane), w1 = warp_transpose32(hi, lane);
            __syncwarp();
            while (w0) {
                const int k = __ffs(w0) - 1;
                w0 &= w0 - 1u;
                run_append(rs0, slot0, items[k], cap, inst_item);
            }
            while (w1) {
                const int k = __ffs(w1) - 1;
                w1 &= w1 - 1u;
                run_append(rs1, slot1, items[k], cap, inst_item);
            }
            __syncwarp();  // the next step overwrites items
        }
        run_flush_partial(rs0, slot0, cap, inst_item);
        run_flush_partial(rs1, slot1, cap, inst_item);
        __syncwarp();  // the next chunk reuses the staging
    }
}

// A CTA per block: group g (of kOffGroups) of threads owns a contiguous run
// of the block's chunks, thread (g, t) tile t.  ccnt[chunk][t] becomes the
// chunk's first block-local position for tile t; btile[b][t] = (tile start
// in the block, tile total); bbase[b] is written by the CTA that finishes
// last, which scans the block totals (64-bit) and publishes n_inst.
constexpr int kOffThreads = 1024;
constexpr int kOffGroups = kOffThreads / kBlkTiles;

__global__ void __launch_bounds__(kOffThreads)
k_fine_offsets(const uint32_t *__restrict__ bchunk, uint32_t *__restrict__ ccnt, uint2 *__restrict__ btile,
               uint32_t *__restrict__ btot, uint32_t *__restrict__ bbase, StatusDev *st, int nblocks,
               int64_t capacity) {
    __shared__ uint32_t s_part[kOffGroups][kBlkTiles];
    __shared__ uint32_t s_tstart[kBlkTiles];
    __shared__ uint32_t s_w0;
    __shared__ bool s_last;
    __shared__ unsigned long long s_scan[kOffThreads / 32];
    const int tid = threadIdx.x, t = tid % kBlkTiles, g = tid / kBlkTiles;
    const int b = blockIdx.x;
    const uint32_t c0 = bchunk[b], nch = bchunk[b + 1] - c0;
    const uint32_t per = (nch + kOffGroups - 1) / kOffGroups;
    const uint32_t ga = c0 + min((uint32_t)g * per, nch), gb = c0 + min((uint32_t)(g + 1) * per, nch);
    uint32_t sum = 0;
#pragma unroll 4
    for (uint32_t c = ga; c < gb; ++c) sum += ccnt[(size_t)c * kBlkTiles + t];
    s_part[g][t] = sum;
    __syncthreads();
    uint32_t tot = 0, inc = 0;
    if (tid < kBlkTiles) {
        // exclusive prefix over the groups, per tile
        for (int gg = 0; gg < kOffGroups; ++gg) {
            const uint32_t x = s_part[gg][t];
            s_part[gg][t] = tot;
            tot += x;
        }
        inc = tot;  // inclusive scan over the 64 tiles (two warps)
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if ((tid & 31) >= o) inc += y;
        }
        if (tid == 31) s_w0 = inc;
    }
    __syncthreads();
    if (tid < kBlkTiles) {
        if (tid >= 32) inc += s_w0;
        s_tstart[t] = inc - tot;
        btile[(size_t)b * kBlkTiles + t] = make_uint2(inc - tot, tot);
        if (tid == kBlkTiles - 1) btot[b] = inc;
    }
    __syncthreads();
    uint32_t run = s_tstart[t] + s_part[g][t];
    for (uint32_t c = ga; c < gb; ++c) {
        const uint32_t x = ccnt[(size_t)c * kBlkTiles + t];
        ccnt[(size_t)c * kBlkTiles + t] = run;
        run += x;
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();  // btot[b] is visible before this CTA counts as done
        s_last = atomicAdd(&st->done_offsets, 1u) == (uint32_t)nblocks - 1u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the last CTA: exclusive scan of the block totals, thread tid owning a
    // contiguous run of blocks
    const int lane = tid & 31, warp = tid >> 5;
    const int bper = (nblocks + kOffThreads - 1) / kOffThreads;
    const int b0 = min(tid * bper, nblocks), b1 = min(b0 + bper, nblocks);
    unsigned long long local = 0;
    for (int k = b0; k < b1; ++k) local += __ldcg(btot + k);
    unsigned long long x = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_scan[warp] = x;
    __syncthreads();
    unsigned long long before = 0, all = 0;
    for (int w = 0; w < kOffThreads / 32; ++w) {
        before += w < warp ? s_scan[w] : 0ull;
        all += s_scan[w];
    }
    unsigned long long runb = x - local + before;
    for (int k = b0; k < b1; ++k) {
        // a base at or past the capacity parks the whole block there (every
        // position is then rejected by the writes)
        bbase[k] = runb < (unsigned long long)capacity ? (uint32_t)runb : (uint32_t)capacity;
        runb += __ldcg(btot + k);
    }
    if (tid == 0) {
        // without an overflow, the walks placed exactly the instances the
        // tile counts of the preprocess promised
        if (!st->overflow && all != (unsigned long long)st->n_inst) atomicCAS(&st->error, 0, GS_ERR_INTERNAL);
        st->done_offsets = 0;
    }
}

// Steps 2-8 of the counting binning (after the depth sort).
static int bin_counting(const gs_plan *plan, void *ws, const uint32_t *order, uint32_t *block_sums,
                        unsigned long long *block_offs, cudaStream_t s) {
    StatusDev *st = ws_at<StatusDev>(ws, plan->o_status);
    const ViewsDev vd = make_views(plan, nullptr);
    const uint32_t *touched = ws_at<uint32_t>(ws, plan->o_touched);
    const uint2 *rects = ws_at<uint2>(ws, plan->o_rect);
    const int64_t ccap = plan->coarse_cap;
    const int nblocks = plan->total_blocks;
    // the entries ping-pong through the instance buffers the radix path
    // uses and one more of the same size, never through the output buffer
    uint32_t *ckA = ws_at<uint32_t>(ws, plan->o_ikey[0]), *cvA = ws_at<uint32_t>(ws, plan->o_ikey[1]);
    uint32_t *ckB = ws_at<uint32_t>(ws, plan->o_ival[1 - plan->inst_final]), *cvB = ws_at<uint32_t>(ws, plan->o_cval);
    uint32_t *out = ws_at<uint32_t>(ws, plan->o_ival[plan->inst_final]);
    uint32_t *inst_sums = reinterpret_cast<uint32_t *>(block_offs + kBinBlocks);
    k_count<true><<<kBinBlocks, kScanThreads, 0, s>>>(order, touched, rects, plan->VN, block_sums, block_offs, st,
                                                      ccap, inst_sums);
    k_coarse_write<<<kBinBlocks, kWriteRound, 0, s>>>(vd, plan->n, order, touched, rects, block_offs, plan->VN, ccap,
                                                      ckA, cvA);
    int rc = launch_error();
    if (rc) return rc;
    int cfinal = 0;
    rc = sort_pairs(ckA, cvA, ckB, cvB, ccap, &st->n_coarse, 0, plan->block_bits,
                    ws_at<uint32_t>(ws, plan->o_sort_scratch), s, &cfinal);
    if (rc) return rc;
    const uint32_t *ckey = cfinal ? ckB : ckA, *cval = cfinal ? cvB : cvA;
    uint2 *brange = ws_at<uint2>(ws, plan->o_brange);
    uint32_t *bchunk = ws_at<uint32_t>(ws, plan->o_bchunk);
    const uint32_t *totals = nullptr;
    if (plan->block_bits <= kRadixBits) {
        // one sort pass with the block id as its digit: its digit totals are
        // the entries per block
        totals = ws_at<uint32_t>(ws, plan->o_sort_scratch) + kRadix * kSortBlocks;
    } else {
        rc = check_cuda(cudaMemsetAsync(brange, 0, (size_t)nblocks * sizeof(uint2), s));
        if (rc) return rc;
        k_block_bounds<<<kSortBlocks, 256, 0, s>>>(ckey, st, ccap, brange);
    }
    k_chunk_scan<<<1, kChunkScanThreads, 0, s>>>(brange, totals, nblocks, bchunk, st);
    uint32_t *ccnt = ws_at<uint32_t>(ws, plan->o_ccnt);
    uint2 *btile = ws_at<uint2>(ws, plan->o_btile);
    uint32_t *bbase = ws_at<uint32_t>(ws, plan->o_bbase);
    uint32_t *btot = bbase + nblocks;  // block totals
    const float4 *rec = ws_at<float4>(ws, plan->o_rec);
    const float2 *bin = ws_at<float2>(ws, plan->o_bin);
    uint2 *ranges = ws_at<uint2>(ws, plan->o_ranges);
    // the entries' tile masks go to the pair of buffers the sort left free
    uint32_t *mlo = cfinal ? ckA : ckB, *mhi = cfinal ? cvA : cvB;
    k_fine_mask<<<kFineCtas, kFineWarps * 32, 0, s>>>(vd, cval, brange, bchunk, rec, bin, rects, mlo, mhi, ccnt, st,
                                                      plan->bbox_3sigma);
    k_fine_offsets<<<nblocks, kOffThreads, 0, s>>>(bchunk, ccnt, btile, btot, bbase, st, nblocks, plan->inst_cap);
    k_fine_scatter<<<kFineCtas, kFineWarps * 32, 0, s>>>(vd, cval, brange, bchunk, mlo, mhi, ccnt, bbase, btile, st,
                                                         plan->inst_cap, out, ranges);
    return launch_error();
}

}  // namespace gs

using namespace gs;

extern "C" int gs_bin_sort(const gs_plan *plan, void *ws, int load_balanced, void *stream) {
    if (!plan || !ws) return GS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t VN = plan->VN;
    StatusDev *st = ws_at<StatusDev>(ws, plan->o_status);
    uint32_t *scratch = ws_at<uint32_t>(ws, plan->o_sort_scratch);
    // the error word, the finished-block counter of k_count, the entry and
    // chunk counts, the finished-CTA counter of k_fine_offsets, the
    // backward's unit counter (cleared again by its launch) and the chunk
    // counters of k_fine_mask and k_fine_scatter (adjacent)
    static_assert(offsetof(StatusDev, next_scatter_chunk) - offsetof(StatusDev, error) == 7 * sizeof(int32_t),
                  "status words cleared together must be adjacent");
    int rc = check_cuda(cudaMemsetAsync(&st->error, 0, 8 * sizeof(int32_t), s));
    if (rc) return rc;

    // 1. depth order of the items (keys were written by gs_preprocess)
    int dfinal = 0;
    rc = sort_pairs(ws_at<uint32_t>(ws, plan->o_dkey[0]), ws_at<uint32_t>(ws, plan->o_dval[0]),
                    ws_at<uint32_t>(ws, plan->o_dkey[1]), ws_at<uint32_t>(ws, plan->o_dval[1]), VN,
                    nullptr, 0, 32, scratch, s, &dfinal);
    if (rc) return rc;
    const uint32_t *order = ws_at<uint32_t>(ws, plan->o_dval[dfinal]);

    uint32_t *block_sums = ws_at<uint32_t>(ws, plan->o_block_sums);
    unsigned long long *block_offs = reinterpret_cast<unsigned long long *>(block_sums + kBinBlocks + 32);
    const uint32_t *touched = ws_at<uint32_t>(ws, plan->o_touched);
    if (load_balanced && !plan->bin_radix) return bin_counting(plan, ws, order, block_sums, block_offs, s);

    // 2. scan of tile counts in depth order
    k_count<false><<<kBinBlocks, kScanThreads, 0, s>>>(order, touched, nullptr, VN, block_sums, block_offs, st,
                                                       plan->inst_cap, nullptr);

    // 3. instance keys
    const ViewsDev vd = make_views(plan, nullptr);
    uint32_t *ik0 = ws_at<uint32_t>(ws, plan->o_ikey[0]), *iv0 = ws_at<uint32_t>(ws, plan->o_ival[0]);
    uint32_t *ik1 = ws_at<uint32_t>(ws, plan->o_ikey[1]), *iv1 = ws_at<uint32_t>(ws, plan->o_ival[1]);
    if (load_balanced)
        k_write_keys<true><<<kBinBlocks, kWriteRound, 0, s>>>(
            vd, plan->n, order, touched, ws_at<float4>(ws, plan->o_rec), ws_at<float2>(ws, plan->o_bin),
            ws_at<uint2>(ws, plan->o_rect),
            block_offs, VN, plan->inst_cap, ik0, iv0, st, plan->bbox_3sigma);
    else
        k_write_keys<false><<<kBinBlocks, kWriteRound, 0, s>>>(
            vd, plan->n, order, touched, ws_at<float4>(ws, plan->o_rec), ws_at<float2>(ws, plan->o_bin),
            ws_at<uint2>(ws, plan->o_rect),
            block_offs, VN, plan->inst_cap, ik0, iv0, st, plan->bbox_3sigma);
    rc = launch_error();
    if (rc) return rc;

    // 4. stable sort by tile id (count read on the device)
    int ifinal = 0;
    rc = sort_pairs(ik0, iv0, ik1, iv1, plan->inst_cap, &st->n_inst, 0, plan->tile_bits, scratch, s,
                    &ifinal);
    if (rc) return rc;

    // 5. ranges and buckets
    uint2 *ranges = ws_at<uint2>(ws, plan->o_ranges);
    k_tile_ranges<<<(plan->total_tiles + 255) / 256, 256, 0, s>>>(
        ws_at<uint32_t>(ws, plan->o_ikey[ifinal]), st, plan->inst_cap, (uint32_t)plan->total_tiles, ranges);
    return launch_error();
}
