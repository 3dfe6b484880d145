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

__global__ void __launch_bounds__(kScanThreads)
k_count(const uint32_t *__restrict__ order, const uint32_t *__restrict__ touched, int64_t n,
        uint32_t *__restrict__ block_sums, unsigned long long *__restrict__ block_offs, StatusDev *st,
        int64_t capacity) {
    __shared__ uint32_t tmp[kScanThreads / 32];
    __shared__ unsigned long long tmp64[kScanThreads / 32];
    __shared__ bool s_last;
    int64_t beg, end;
    chunk_of(n, &beg, &end);
    uint32_t s = 0;
    for (int64_t r = beg + threadIdx.x; r < end; r += kScanThreads) s += touched[order[r]];
    uint32_t total;
    block_exclusive_scan(s, tmp, &total);
    if (threadIdx.x == 0) {
        block_sums[blockIdx.x] = total;
        __threadfence();  // the sum is visible before this block counts as done
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
    if (tid == 0) {
        st->n_inst = all > 0xffffffffull ? 0xffffffffu : (uint32_t)all;
        st->overflow = all > (unsigned long long)capacity ? 1u : 0u;
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

}  // namespace gs

using namespace gs;

extern "C" int gs_bin_sort(const gs_plan *plan, void *ws, int load_balanced, void *stream) {
    if (!plan || !ws) return GS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t VN = plan->VN;
    StatusDev *st = ws_at<StatusDev>(ws, plan->o_status);
    uint32_t *scratch = ws_at<uint32_t>(ws, plan->o_sort_scratch);
    // the error word and the finished-block counter of k_count (adjacent)
    int rc = check_cuda(cudaMemsetAsync(&st->error, 0, 2 * sizeof(int32_t), s));
    if (rc) return rc;

    // 1. depth order of the items (keys were written by gs_preprocess)
    int dfinal = 0;
    rc = sort_pairs(ws_at<uint32_t>(ws, plan->o_dkey[0]), ws_at<uint32_t>(ws, plan->o_dval[0]),
                    ws_at<uint32_t>(ws, plan->o_dkey[1]), ws_at<uint32_t>(ws, plan->o_dval[1]), VN,
                    nullptr, 0, 32, scratch, s, &dfinal);
    if (rc) return rc;
    const uint32_t *order = ws_at<uint32_t>(ws, plan->o_dval[dfinal]);

    // 2. scan of tile counts in depth order
    uint32_t *block_sums = ws_at<uint32_t>(ws, plan->o_block_sums);
    unsigned long long *block_offs = reinterpret_cast<unsigned long long *>(block_sums + kBinBlocks + 32);
    const uint32_t *touched = ws_at<uint32_t>(ws, plan->o_touched);
    k_count<<<kBinBlocks, kScanThreads, 0, s>>>(order, touched, VN, block_sums, block_offs, st, plan->inst_cap);

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
