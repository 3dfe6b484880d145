// Host side of the C ABI: plans (workspace layout), camera marshalling,
// status read-back and error strings.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "gs_internal.cuh"

namespace gs {

int check_cuda(cudaError_t e) { return e == cudaSuccess ? GS_OK : GS_ERR_CUDA; }

int launch_error() { return check_cuda(cudaGetLastError()); }

ViewsDev make_views(const gs_plan *plan, const gs_camera *cams) {
    ViewsDev vd;
    memset(&vd, 0, sizeof(vd));
    vd.V = plan->V;
    vd.total_tiles = plan->total_tiles;
    vd.total_blocks = plan->total_blocks;
    for (int v = 0; v < plan->V; ++v) {
        ViewDev &d = vd.v[v];
        d.W = plan->W[v];
        d.H = plan->H[v];
        d.tiles_x = plan->tiles_x[v];
        d.tiles_y = plan->tiles_y[v];
        d.tile_off = plan->tile_off[v];
        d.pix_off = (int)plan->pix_off[v];
        d.blocks_x = plan->blocks_x[v];
        d.block_off = plan->block_off[v];
        if (!cams) continue;  // image geometry only
        const gs_camera &c = cams[v];
        d.fx = c.fx;
        d.fy = c.fy;
        d.cx = c.cx;
        d.cy = c.cy;
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) d.R[i * 3 + j] = c.w2c[i * 4 + j];
            d.t[i] = c.w2c[i * 4 + 3];
        }
        // camera centre = -R^T t (host, double precision, rounded once)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int i = 0; i < 3; ++i) s -= (double)c.w2c[i * 4 + j] * (double)c.w2c[i * 4 + 3];
            d.campos[j] = (float)s;
        }
        d.limx = 1.3f * (0.5f * (float)c.width / c.fx);
        d.limy = 1.3f * (0.5f * (float)c.height / c.fy);
        d.near_z = c.near_z;
    }
    return vd;
}

}  // namespace gs

using namespace gs;

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

extern "C" gs_plan *gs_plan_create_tuned(int64_t n, int32_t sh_degree, int32_t n_views,
                                         const int32_t *widths, const int32_t *heights,
                                         int64_t inst_capacity, const gs_tuning *tuning) {
    const int32_t bucket = tuning && tuning->bucket ? tuning->bucket : kBucket;
    const int32_t bwd_warps = tuning && tuning->bwd_warps ? tuning->bwd_warps : 4;
    const int32_t chains = tuning ? tuning->bwd_chains : 0;
    const int32_t fwd_pixels = tuning && tuning->fwd_pixels ? tuning->fwd_pixels : 1;
    if ((bucket != 32 && bucket != 64) || (bwd_warps != 1 && bwd_warps != 2 && bwd_warps != 4 && bwd_warps != 8) ||
        chains < 0 || chains > 2 || (fwd_pixels != 1 && fwd_pixels != 2))
        return nullptr;
    if (n <= 0 || n >= (1ll << 31) || sh_degree < 0 || sh_degree > 3 || n_views < 1 ||
        n_views > GS_MAX_VIEWS || !widths || !heights || inst_capacity <= 0 ||
        inst_capacity >= (1ll << 31))
        return nullptr;
    gs_plan *p = (gs_plan *)calloc(1, sizeof(gs_plan));
    if (!p) return nullptr;
    p->n = n;
    p->sh_degree = sh_degree;
    p->K = (sh_degree + 1) * (sh_degree + 1);
    p->V = n_views;
    p->VN = (int64_t)n_views * n;
    int64_t tiles = 0, pix = 0;
    for (int v = 0; v < n_views; ++v) {
        if (widths[v] <= 0 || heights[v] <= 0 || widths[v] > 16384 || heights[v] > 16384) {
            free(p);
            return nullptr;
        }
        p->W[v] = widths[v];
        p->H[v] = heights[v];
        p->tiles_x[v] = (widths[v] + kTile - 1) / kTile;
        p->tiles_y[v] = (heights[v] + kTile - 1) / kTile;
        p->tile_off[v] = (int32_t)tiles;
        p->pix_off[v] = pix;
        tiles += (int64_t)p->tiles_x[v] * p->tiles_y[v];
        pix += (int64_t)widths[v] * heights[v];
    }
    p->tile_off[n_views] = (int32_t)tiles;
    p->pix_off[n_views] = pix;
    int64_t blocks = 0;
    for (int v = 0; v < n_views; ++v) {
        p->blocks_x[v] = (p->tiles_x[v] + kBlk - 1) / kBlk;
        p->block_off[v] = (int32_t)blocks;
        blocks += (int64_t)p->blocks_x[v] * ((p->tiles_y[v] + kBlk - 1) / kBlk);
    }
    p->block_off[n_views] = (int32_t)blocks;
    if (p->VN >= (1ll << 31) || tiles >= (1ll << 24)) {
        free(p);
        return nullptr;
    }
    p->total_tiles = (int32_t)tiles;
    p->total_pixels = pix;
    int bits = 1;
    while ((1ll << bits) < tiles) ++bits;
    p->tile_bits = bits;
    p->total_blocks = (int32_t)blocks;
    bits = 1;
    while ((1ll << bits) < blocks) ++bits;
    p->block_bits = bits;
    p->inst_cap = inst_capacity;
    p->bucket = bucket;
    p->bucket_shift = bucket == 64 ? 6 : 5;
    p->bwd_warps = bwd_warps;
    p->two_chain_min = chains == 2 ? 0 : chains == 1 ? (1 << 30) : kTwoChainAuto;
    p->bbox_3sigma = tuning && tuning->bbox_3sigma ? 1 : 0;
    p->bwd_per_pixel = tuning && tuning->bwd_per_pixel ? 1 : 0;
    p->bin_radix = tuning && tuning->bin_radix ? 1 : 0;
    p->fwd_pixels = fwd_pixels;
    // the counting binning's (Gaussian, block) entries: at most one per
    // instance of capacity (an entry whose block holds no tile of its
    // Gaussian is rare), in the radix path's instance buffers and o_cval
    p->coarse_cap = inst_capacity;
    p->chunk_cap = p->coarse_cap / kChunk + blocks + 1;
    p->bucket_cap = inst_capacity / bucket + tiles + 1;
    p->sort_scratch_bytes = sort_scratch_bytes();

    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    const size_t VN = (size_t)p->VN, I = (size_t)inst_capacity, T = (size_t)tiles;
    p->o_status = take(sizeof(StatusDev));
    p->o_rec = take(VN * 3 * sizeof(float4));
    p->o_touched = take(VN * sizeof(uint32_t));
    p->o_rect = take(VN * sizeof(uint2));
    p->o_bin = take(VN * sizeof(float2));
    for (int b = 0; b < 2; ++b) {
        p->o_dkey[b] = take(VN * sizeof(uint32_t));
        p->o_dval[b] = take(VN * sizeof(uint32_t));
    }
    for (int b = 0; b < 2; ++b) {
        p->o_ikey[b] = take(I * sizeof(uint32_t));
        p->o_ival[b] = take(I * sizeof(uint32_t));
    }
    p->o_ranges = take(T * sizeof(uint2));
    p->o_tile_maxc = take(T * sizeof(uint32_t));
    p->o_bucket_off = take((T + 1) * sizeof(uint32_t));
    p->unit_cap = T + p->bucket_cap / kBwdChunk + 1;
    p->o_tile_order = take((size_t)kTileClasses * p->unit_cap * sizeof(uint2));
    p->o_tile_count = take((size_t)kTileClasses * sizeof(uint32_t));
    p->o_ncontrib = take((size_t)pix * sizeof(uint32_t));
    p->o_final = take(p->bwd_per_pixel ? ((size_t)pix + 4) * sizeof(float) : 16);
    p->o_ckpt = take((size_t)p->bucket_cap * kCkptCh * kTilePix * sizeof(float));
    p->o_grad2d = take(VN * 3 * sizeof(float4));
    p->o_posed = take(GS_MAX_VIEWS * sizeof(ViewDev));
    p->o_sort_scratch = take(p->sort_scratch_bytes);
    // uint32 block sums, then (8-byte aligned) uint64 block offsets, then the
    // uint32 instance block sums of the counting binning's count
    p->o_block_sums = take((kBinBlocks + 32) * sizeof(uint32_t) + kBinBlocks * sizeof(uint64_t) +
                           kBinBlocks * sizeof(uint32_t));
    const size_t NB = (size_t)blocks;
    p->o_brange = take(NB * sizeof(uint2));
    p->o_bchunk = take((NB + 1) * sizeof(uint32_t));
    p->o_btile = take(NB * kBlkTiles * sizeof(uint2));
    p->o_bbase = take(2 * NB * sizeof(uint32_t));  // block bases, then block totals
    p->o_ccnt = take((size_t)p->chunk_cap * kBlkTiles * sizeof(uint32_t));
    p->o_cval = take(I * sizeof(uint32_t));
    p->bytes = o;
    // the radix sort ping-pongs: after P passes the data is in buffer P % 2
    p->depth_final = (32 / kRadixBits) % 2;
    p->inst_final = ((p->tile_bits + kRadixBits - 1) / kRadixBits) % 2;
    return p;
}

extern "C" gs_plan *gs_plan_create(int64_t n, int32_t sh_degree, int32_t n_views, const int32_t *widths,
                                   const int32_t *heights, int64_t inst_capacity) {
    return gs_plan_create_tuned(n, sh_degree, n_views, widths, heights, inst_capacity, nullptr);
}

extern "C" void gs_plan_destroy(gs_plan *plan) { free(plan); }

extern "C" size_t gs_plan_workspace_bytes(const gs_plan *plan) { return plan ? plan->bytes : 0; }

extern "C" int64_t gs_plan_pixels(const gs_plan *plan) { return plan ? plan->total_pixels : 0; }

extern "C" int gs_workspace_view(const gs_plan *p, void *ws, int which, void **ptr, size_t *bytes) {
    if (!p || !ptr || !bytes) return GS_ERR_ARG;
    size_t off = 0, nb = 0;
    const size_t VN = (size_t)p->VN;
    switch (which) {
        case GS_WS_RECORDS: off = p->o_rec; nb = VN * 3 * sizeof(float4); break;
        case GS_WS_TILES_TOUCHED: off = p->o_touched; nb = VN * 4; break;
        case GS_WS_RECTS: off = p->o_rect; nb = VN * 8; break;
        case GS_WS_DEPTH_ORDER: off = p->o_dval[p->depth_final]; nb = VN * 4; break;
        case GS_WS_INST_TILE: off = p->o_ikey[p->inst_final]; nb = (size_t)p->inst_cap * 4; break;
        case GS_WS_INST_GID: off = p->o_ival[p->inst_final]; nb = (size_t)p->inst_cap * 4; break;
        case GS_WS_TILE_RANGES: off = p->o_ranges; nb = (size_t)p->total_tiles * 8; break;
        case GS_WS_N_CONTRIB: off = p->o_ncontrib; nb = (size_t)p->total_pixels * 4; break;
        case GS_WS_GRAD2D: off = p->o_grad2d; nb = VN * 3 * sizeof(float4); break;
        case GS_WS_STATUS: off = p->o_status; nb = sizeof(StatusDev); break;
        case GS_WS_BIN: off = p->o_bin; nb = VN * sizeof(float2); break;
        default: return GS_ERR_ARG;
    }
    *ptr = (char *)ws + off;
    *bytes = nb;
    return GS_OK;
}

extern "C" int gs_read_status(const gs_plan *p, const void *ws, gs_status *out, void *stream) {
    if (!p || !ws || !out) return GS_ERR_ARG;
    StatusDev st;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = check_cuda(cudaMemcpyAsync(&st, (const char *)ws + p->o_status, sizeof(st),
                                        cudaMemcpyDeviceToHost, s));
    if (rc) return rc;
    rc = check_cuda(cudaStreamSynchronize(s));
    if (rc) return rc;
    out->n_instances = st.n_inst;
    out->n_buckets = st.n_buckets;
    out->inst_capacity = p->inst_cap;
    out->overflow = (int32_t)st.overflow;
    out->error = st.error;
    if (st.error) return st.error;
    if (st.overflow) return GS_ERR_CAPACITY;
    return GS_OK;
}

extern "C" const char *gs_error_string(int code) {
    switch (code) {
        case GS_OK: return "ok";
        case GS_ERR_ARG: return "invalid argument";
        case GS_ERR_CAPACITY: return "tile-instance capacity exceeded";
        case GS_ERR_CUDA: return "CUDA runtime error";
        case GS_ERR_TIMEOUT: return "bounded device wait timed out";
        case GS_ERR_INTERNAL: return "device-side consistency check failed";
        default: return "unknown error";
    }
}
