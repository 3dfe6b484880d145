// a2-a4: binning (Sec. 2.1).
//
//  1. depth sort: radix sort of the (view, Gaussian) items by camera depth
//     (float bits of z > 0 order like the floats; culled items carry the
//     largest key).  Items of different views interleave, which is harmless:
//     an item only ever writes tiles of its own view.
//  2. scan of the tile counts in depth order (fixed grid, no host sync): the
//     block sums, one block scanning them (also publishing the instance count
//     and the capacity overflow flag), and the key-write pass that rescans
//     inside each block.
//  3. key write, one (global tile id, item) instance per touched tile:
//     load-balanced (Fig. "LB"): a warp takes one Gaussian at a time, its
//     lanes test one candidate tile of the SnugBox each (per-column ellipse
//     test) and compact the hits with ballot/popc;
//     sequential ("Sq"): one thread walks its Gaussian's columns.
//  4. stable radix sort of the instances by tile id: every tile's list keeps
//     the depth order of step 1, ties in depth by ascending Gaussian index.
//  5. tile ranges from the run boundaries, and the 32-splat bucket offsets.
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
    const int64_t chunk = (n + kSortBlocks - 1) / kSortBlocks;
    *beg = (int64_t)blockIdx.x * chunk;
    *end = *beg + chunk < n ? *beg + chunk : n;
}

__global__ void __launch_bounds__(kScanThreads)
k_count_reduce(const uint32_t *__restrict__ order, const uint32_t *__restrict__ touched, int64_t n,
               uint32_t *__restrict__ block_sums) {
    __shared__ uint32_t tmp[kScanThreads / 32];
    int64_t beg, end;
    chunk_of(n, &beg, &end);
    uint32_t s = 0;
    for (int64_t r = beg + threadIdx.x; r < end; r += kScanThreads) s += touched[order[r]];
    uint32_t total;
    block_exclusive_scan(s, tmp, &total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// One block: exclusive scan (64-bit) of the block sums into block_offs;
// publishes the instance count (saturated to 32 bits) and the overflow flag.
__global__ void __launch_bounds__(1024)
k_count_top(const uint32_t *__restrict__ block_sums, unsigned long long *__restrict__ block_offs,
            StatusDev *st, int64_t capacity) {
    __shared__ unsigned long long tmp[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned long long x = tid < kSortBlocks ? block_sums[tid] : 0ull;
    unsigned long long inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) tmp[warp] = inc;
    __syncthreads();
    unsigned long long before = 0, all = 0;
    for (int w = 0; w < 32; ++w) {
        before += w < warp ? tmp[w] : 0ull;
        all += tmp[w];
    }
    if (tid < kSortBlocks) block_offs[tid] = inc - x + before;
    if (tid == 0) {
        st->n_inst = all > 0xffffffffull ? 0xffffffffu : (uint32_t)all;
        st->overflow = all > (unsigned long long)capacity ? 1u : 0u;
        st->bucket_next = 0;
    }
}

// Instance key write.  Block b rescans the counts of its chunk of depth ranks
// in rounds of kScanThreads and writes each Gaussian's touched tiles.
template <bool kLB>
__global__ void __launch_bounds__(kScanThreads)
k_write_keys(ViewsDev views, int64_t n_per_view, const uint32_t *__restrict__ order,
             const uint32_t *__restrict__ touched, const float4 *__restrict__ rec,
             const float2 *__restrict__ bin,
             const uint2 *__restrict__ rects, const unsigned long long *__restrict__ block_offs, int64_t n,
             int64_t capacity, uint32_t *__restrict__ inst_tile, uint32_t *__restrict__ inst_item,
             StatusDev *st) {
    __shared__ uint32_t tmp[kScanThreads / 32];
    __shared__ uint32_t s_item[kScanThreads];
    __shared__ unsigned long long s_off[kScanThreads];
    __shared__ uint32_t s_cnt[kScanThreads];
    int64_t beg, end;
    chunk_of(n, &beg, &end);
    unsigned long long base = block_offs[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t r0 = beg; r0 < end; r0 += kScanThreads) {
        const int64_t r = r0 + threadIdx.x;
        uint32_t item = 0, cnt = 0;
        if (r < end) {
            item = order[r];
            cnt = touched[item];
        }
        uint32_t total;
        const unsigned long long off = base + block_exclusive_scan(cnt, tmp, &total);
        base += total;
        if (!kLB) {
            if (cnt == 0) continue;
            const int v = (int)(item / (uint32_t)n_per_view);
            const ViewDev &cam = views.v[v];
            const float4 r0v = rec[3 * (size_t)item];
            const float Cc = rec[3 * (size_t)item + 1].x;
            const float2 bv = bin[item];
            const float tb = bv.x, detc = bv.y;
            int tx0, ty0, tx1, ty1;
            unpack_rect(rects[item], &tx0, &ty0, &tx1, &ty1);
            float rx, ry;
            ellipse_extent(r0v.z, Cc, detc, tb, &rx, &ry);
            uint32_t w = 0;
            for (int tx = tx0; tx < tx1; ++tx) {
                float xa, xb;
                column_span(tx, (float)cam.W, &xa, &xb);
                int lo, hi;
                if (!column_rows(r0v.x, r0v.y, r0v.z, r0v.w, Cc, detc, tb, rx, ry, xa, xb,
                                 (float)cam.H, ty0, ty1, &lo, &hi))
                    continue;
                for (int ty = lo; ty <= hi; ++ty, ++w) {
                    const unsigned long long pos = off + w;
                    if (w < cnt && pos < (unsigned long long)capacity) {
                        inst_tile[pos] = (uint32_t)(cam.tile_off + ty * cam.tiles_x + tx);
                        inst_item[pos] = item;
                    }
                }
            }
            if (w != cnt) {
                // keep every slot of this Gaussian valid (never happens when the
                // count and the write agree, which the shared column test ensures)
                atomicCAS(&st->error, 0, GS_ERR_INTERNAL);
                for (; w < cnt; ++w) {
                    const unsigned long long pos = off + w;
                    if (pos < (unsigned long long)capacity) {
                        inst_tile[pos] = (uint32_t)(cam.tile_off + ty0 * cam.tiles_x + tx0);
                        inst_item[pos] = item;
                    }
                }
            }
        } else {
            s_item[threadIdx.x] = item;
            s_off[threadIdx.x] = off;
            s_cnt[threadIdx.x] = cnt;
            __syncthreads();
            // warp `warp` takes the Gaussians of lanes warp*32 .. warp*32+31 in turn
            for (int j = 0; j < 32; ++j) {
                const int slot = warp * 32 + j;
                const uint32_t c = s_cnt[slot];
                if (c == 0) continue;
                const uint32_t it = s_item[slot];
                const unsigned long long o0 = s_off[slot];
                const int v = (int)(it / (uint32_t)n_per_view);
                const ViewDev &cam = views.v[v];
                const float4 r0v = rec[3 * (size_t)it];
                const float Cc = rec[3 * (size_t)it + 1].x;
                const float2 bv = bin[it];
                const float tb = bv.x, detc = bv.y;
                int tx0, ty0, tx1, ty1;
                unpack_rect(rects[it], &tx0, &ty0, &tx1, &ty1);
                float rx, ry;
                ellipse_extent(r0v.z, Cc, detc, tb, &rx, &ry);
                const int wdt = tx1 - tx0;
                const int cand = wdt * (ty1 - ty0);
                uint32_t written = 0;
                for (int c0 = 0; c0 < cand; c0 += 32) {
                    const int ci = c0 + lane;
                    bool hit = false;
                    int tx = 0, ty = 0;
                    if (ci < cand) {
                        tx = tx0 + ci % wdt;
                        ty = ty0 + ci / wdt;
                        float xa, xb;
                        column_span(tx, (float)cam.W, &xa, &xb);
                        int lo, hi;
                        if (column_rows(r0v.x, r0v.y, r0v.z, r0v.w, Cc, detc, tb, rx, ry, xa, xb,
                                        (float)cam.H, ty0, ty1, &lo, &hi))
                            hit = ty >= lo && ty <= hi;
                    }
                    const uint32_t ballot = __ballot_sync(0xffffffffu, hit);
                    if (hit) {
                        const uint32_t w = written + __popc(ballot & ((1u << lane) - 1u));
                        const unsigned long long pos = o0 + w;
                        if (w < c && pos < (unsigned long long)capacity) {
                            inst_tile[pos] = (uint32_t)(cam.tile_off + ty * cam.tiles_x + tx);
                            inst_item[pos] = it;
                        }
                    }
                    written += __popc(ballot);
                }
                if (written != c) {  // see the sequential path
                    if (lane == 0) atomicCAS(&st->error, 0, GS_ERR_INTERNAL);
                    for (uint32_t w = written + lane; w < c; w += 32) {
                        const unsigned long long pos = o0 + w;
                        if (pos < (unsigned long long)capacity) {
                            inst_tile[pos] = (uint32_t)(cam.tile_off + ty0 * cam.tiles_x + tx0);
                            inst_item[pos] = it;
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Run boundaries of the sorted tile ids -> [start, end) per tile.
__global__ void __launch_bounds__(256)
k_tile_ranges(const uint32_t *__restrict__ keys, const StatusDev *st, int64_t capacity,
              uint32_t total_tiles, uint2 *__restrict__ ranges) {
    int64_t n = st->n_inst;
    if (n > capacity) n = capacity;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        if (k >= total_tiles) continue;  // cannot happen for keys written by k_write_keys
        if (i == 0 || keys[i - 1] != k) ranges[k].x = (uint32_t)i;
        if (i == n - 1 || keys[i + 1] != k) ranges[k].y = (uint32_t)(i + 1);
    }
}

// One block: bucket_off[t] = sum over tiles before t of ceil(len / 32).
__global__ void __launch_bounds__(1024)
k_bucket_offsets(const uint2 *__restrict__ ranges, int total_tiles, uint32_t *__restrict__ bucket_off,
                 StatusDev *st) {
    __shared__ uint32_t tmp[32];
    __shared__ uint32_t carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int t0 = 0; t0 < total_tiles; t0 += 1024) {
        const int t = t0 + tid;
        uint32_t nb = 0;
        if (t < total_tiles) {
            const uint2 r = ranges[t];
            nb = (r.y - r.x + kBucket - 1) / kBucket;
        }
        uint32_t inc = nb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) tmp[warp] = inc;
        __syncthreads();
        uint32_t before = 0, all = 0;
        for (int w = 0; w < 32; ++w) {
            before += w < warp ? tmp[w] : 0u;
            all += tmp[w];
        }
        if (t < total_tiles) bucket_off[t] = carry + inc - nb + before;
        __syncthreads();
        if (tid == 0) carry += all;
        __syncthreads();
    }
    if (tid == 0) {
        bucket_off[total_tiles] = carry;
        st->n_buckets = carry;
    }
}

}  // namespace gs

using namespace gs;

extern "C" int gs_bin_sort(const gs_plan *plan, void *ws, int load_balanced, void *stream) {
    if (!plan || !ws) return GS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t VN = plan->VN;
    StatusDev *st = ws_at<StatusDev>(ws, plan->o_status);
    uint32_t *scratch = ws_at<uint32_t>(ws, plan->o_sort_scratch);
    int rc = check_cuda(cudaMemsetAsync(&st->error, 0, sizeof(int32_t), s));
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
    unsigned long long *block_offs = reinterpret_cast<unsigned long long *>(block_sums + kSortBlocks + 32);
    const uint32_t *touched = ws_at<uint32_t>(ws, plan->o_touched);
    k_count_reduce<<<kSortBlocks, kScanThreads, 0, s>>>(order, touched, VN, block_sums);
    k_count_top<<<1, 1024, 0, s>>>(block_sums, block_offs, st, plan->inst_cap);

    // 3. instance keys
    const ViewsDev vd = make_views(plan, nullptr);
    uint32_t *ik0 = ws_at<uint32_t>(ws, plan->o_ikey[0]), *iv0 = ws_at<uint32_t>(ws, plan->o_ival[0]);
    uint32_t *ik1 = ws_at<uint32_t>(ws, plan->o_ikey[1]), *iv1 = ws_at<uint32_t>(ws, plan->o_ival[1]);
    if (load_balanced)
        k_write_keys<true><<<kSortBlocks, kScanThreads, 0, s>>>(
            vd, plan->n, order, touched, ws_at<float4>(ws, plan->o_rec), ws_at<float2>(ws, plan->o_bin),
            ws_at<uint2>(ws, plan->o_rect),
            block_offs, VN, plan->inst_cap, ik0, iv0, st);
    else
        k_write_keys<false><<<kSortBlocks, kScanThreads, 0, s>>>(
            vd, plan->n, order, touched, ws_at<float4>(ws, plan->o_rec), ws_at<float2>(ws, plan->o_bin),
            ws_at<uint2>(ws, plan->o_rect),
            block_offs, VN, plan->inst_cap, ik0, iv0, st);
    rc = launch_error();
    if (rc) return rc;

    // 4. stable sort by tile id (count read on the device)
    int ifinal = 0;
    rc = sort_pairs(ik0, iv0, ik1, iv1, plan->inst_cap, &st->n_inst, 0, plan->tile_bits, scratch, s,
                    &ifinal);
    if (rc) return rc;

    // 5. ranges and buckets
    uint2 *ranges = ws_at<uint2>(ws, plan->o_ranges);
    rc = check_cuda(cudaMemsetAsync(ranges, 0, (size_t)plan->total_tiles * sizeof(uint2), s));
    if (rc) return rc;
    k_tile_ranges<<<4 * 152, 256, 0, s>>>(ws_at<uint32_t>(ws, plan->o_ikey[ifinal]), st, plan->inst_cap,
                                          (uint32_t)plan->total_tiles, ranges);
    k_bucket_offsets<<<1, 1024, 0, s>>>(ranges, plan->total_tiles, ws_at<uint32_t>(ws, plan->o_bucket_off),
                                        st);
    return launch_error();
}
