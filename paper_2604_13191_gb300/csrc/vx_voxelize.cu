// vx_voxelize.cu -- level 0 of the pyramid: sparse voxelization of capsules (fiber
// segments) and triangles with 8^3 sub-cell occupancy, mass and second moments.
//
// Pipeline (one stream):
//   prep      per primitive: grid coordinates (Sec. 3.1, P_volume), weights
//   count     warp per primitive: conservative voxel test over its bounding box
//   scan      exclusive offsets of the per-primitive candidate counts
//   emit      warp per primitive: (Morton key, primitive id) pairs, ballot-compacted
//   sort      stable LSD radix sort by key (Sec. 3.3: samples ordered by block id)
//   heads     segment starts where the key changes (Sec. 3.3)
//   reduce    warp per voxel: exact sub-cell masks (OR over primitives), mass and
//             moment summed in primitive order (Sec. 3.4-3.5, 4.1)
//   finalize  compaction of the non-empty voxels, occupancy counts, S = M / m and
//             the compact SGGX parameters (Eq. compact-sggx)
//
// Arithmetic: every FP32 quantity that decides a bit, and every per-voxel sum, is
// evaluated with the operation order written below and no contraction (the library
// is compiled with -fmad=false); the per-voxel sums run sequentially in primitive
// order so the result does not depend on scheduling.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "vx_internal.cuh"

#include "vx_level0.cuh"

namespace {

// exact 64-bit total of the per-primitive candidate counts (the 32-bit scan total wraps)
__global__ void k_sum_u64(const uint32_t* __restrict__ cnt, uint32_t n, unsigned long long* __restrict__ total) {
    unsigned long long acc = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc += cnt[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(total, acc);
}

// The count pass's ballot store (WS_BALLOTS, CAND_BALLOTS words per primitive) in *out, or
// NULL when it would take more than 256 MB (the emit pass then tests every voxel again).
// Errors: VX_ERR_OUT_OF_MEMORY, as for any workspace.
vx_status window_ballots(vx_context* ctx, uint32_t np, cudaStream_t s, uint32_t** out) {
    *out = nullptr;
    const size_t bytes = (size_t)np * CAND_BALLOTS * 4;
    if (bytes > ((size_t)256 << 20)) return VX_OK;
    VX_TRY(vx_ws_ensure(ctx, WS_BALLOTS, bytes, s));
    *out = (uint32_t*)ctx->ws[WS_BALLOTS].p;
    return VX_OK;
}

// Candidate counts and offsets of the primitives over one window (WS_COUNT, WS_OFFS), and
// the hit ballots of their ranges (WS_BALLOTS, see window_ballots); the exact total goes to
// *total.  Synchronises the stream once.
vx_status count_window(vx_context* ctx, bool fiber, uint32_t np, const Window& win, float4* r0, float4* r1,
                       float4* r2, uint32_t* misc, cudaStream_t s, uint64_t* total) {
    VX_TRY(vx_ws_ensure(ctx, WS_COUNT, (size_t)np * 4, s));
    VX_TRY(vx_ws_ensure(ctx, WS_OFFS, (size_t)np * 4, s));
    uint32_t* cnt = (uint32_t*)ctx->ws[WS_COUNT].p;
    uint32_t* offs = (uint32_t*)ctx->ws[WS_OFFS].p;
    ctx->ballots = nullptr;
    uint32_t* ballots = nullptr;
    VX_TRY(window_ballots(ctx, np, s, &ballots));
    ctx->ballots = ballots;
    ctx->ballots_np = np;
    for (int i = 0; i < 3; ++i) {
        ctx->ballots_win[i] = win.lo[i];
        ctx->ballots_win[3 + i] = win.hi[i];
    }
    const unsigned cblocks = (unsigned)std::min<size_t>((np + EMIT_WARPS - 1) / EMIT_WARPS, (size_t)vx::kSMs * 64);
    if (fiber)
        VX_LAUNCH(ctx, ST_COUNT, s, k_candidates<true, false><<<cblocks, EMIT_WARPS * 32, 0, s>>>(
                                        r0, r1, r2, np, win, cnt, nullptr, nullptr, nullptr, ballots));
    else
        VX_LAUNCH(ctx, ST_COUNT, s, k_candidates<false, false><<<cblocks, EMIT_WARPS * 32, 0, s>>>(
                                        r0, r1, r2, np, win, cnt, nullptr, nullptr, nullptr, ballots));
    VX_TRY(vx_scan_u32(ctx, cnt, offs, np, misc + 1, s));
    unsigned long long* t64 = (unsigned long long*)(misc + 8);
    VX_CUDA_TRY(cudaMemsetAsync(t64, 0, 8, s));
    VX_LAUNCH(ctx, ST_COUNT, s, k_sum_u64<<<(unsigned)std::min<size_t>(grid_for(np, 256), (size_t)vx::kSMs * 8), 256, 0, s>>>(
                                    cnt, np, t64));
    VX_TRY(vx_readback_async(ctx, 0, misc, 48, s));
    VX_CUDA_TRY(cudaStreamSynchronize(s));
    if (((uint32_t*)ctx->host_pin)[0]) return VX_ERR_INVALID_ARG;
    *total = ((const uint64_t*)ctx->host_pin)[4];
    return VX_OK;
}

// Candidate pairs of one pass at most (31-bit pair indices).
constexpr int64_t kMaxPassPairs = 0x7fffffffll;

// A window of the grid in the planning of a voxelization: its corner and size (2^lg voxels
// per side) and, once counted, its candidate-pair total.
struct Leaf {
    int lo[3];
    int lg;
    uint64_t pairs;
};

inline Window window_of(const Leaf& w) {
    Window win;
    for (int i = 0; i < 3; ++i) { win.lo[i] = w.lo[i]; win.hi[i] = w.lo[i] + (1 << w.lg) - 1; }
    return win;
}

inline uint64_t key_hi_of(const Leaf& w) {
    return vx_morton3_64((uint32_t)(w.lo[0] >> w.lg), (uint32_t)(w.lo[1] >> w.lg), (uint32_t)(w.lo[2] >> w.lg))
           << (3 * w.lg);
}

// Emit, sort and segment heads of one window whose candidate counts and offsets are in
// WS_COUNT / WS_OFFS (count_window ran on it last) and whose pair total fits 31 bits.  On
// return the sorted keys / primitive ids are in *k0 / *v0, the run starts in WS_STARTS and
// the number of candidate voxels in *nseg.  Synchronises the stream once.
vx_status window_segments(vx_context* ctx, bool fiber, uint32_t np, const Window& win, int bits, uint32_t npairs,
                          float4* r0, float4* r1, float4* r2, uint32_t* misc, cudaStream_t s, uint32_t** k0,
                          uint32_t** v0, uint32_t** k1, uint32_t** v1, uint32_t* nseg) {
    uint32_t* offs = (uint32_t*)ctx->ws[WS_OFFS].p;
    const unsigned cblocks = (unsigned)std::min<size_t>((np + EMIT_WARPS - 1) / EMIT_WARPS, (size_t)vx::kSMs * 64);
    VX_TRY(vx_ws_ensure(ctx, WS_KEYS0, (size_t)npairs * 4, s));
    VX_TRY(vx_ws_ensure(ctx, WS_VALS0, (size_t)npairs * 4, s));
    VX_TRY(vx_ws_ensure(ctx, WS_KEYS1, (size_t)npairs * 4, s));
    VX_TRY(vx_ws_ensure(ctx, WS_VALS1, (size_t)npairs * 4, s));
    *k0 = (uint32_t*)ctx->ws[WS_KEYS0].p;
    *v0 = (uint32_t*)ctx->ws[WS_VALS0].p;
    *k1 = (uint32_t*)ctx->ws[WS_KEYS1].p;
    *v1 = (uint32_t*)ctx->ws[WS_VALS1].p;
    // the ballots the count pass of this window stored, if it stored any
    bool same = ctx->ballots != nullptr && ctx->ballots_np == np;
    for (int i = 0; i < 3; ++i)
        same = same && ctx->ballots_win[i] == win.lo[i] && ctx->ballots_win[3 + i] == win.hi[i];
    uint32_t* ballots = same ? ctx->ballots : nullptr;
    if (fiber)
        VX_LAUNCH(ctx, ST_EMIT, s, k_candidates<true, true><<<cblocks, EMIT_WARPS * 32, 0, s>>>(
                                       r0, r1, r2, np, win, nullptr, offs, *k0, *v0, ballots));
    else
        VX_LAUNCH(ctx, ST_EMIT, s, k_candidates<false, true><<<cblocks, EMIT_WARPS * 32, 0, s>>>(
                                       r0, r1, r2, np, win, nullptr, offs, *k0, *v0, ballots));
    VX_CUDA_TRY(cudaGetLastError());
    VX_TRY(vx_radix_sort_u32(ctx, k0, v0, k1, v1, npairs, 3 * bits, s, misc));
    VX_TRY(vx_ws_ensure(ctx, WS_FLAGS, (size_t)npairs * 4, s));
    VX_TRY(vx_ws_ensure(ctx, WS_STARTS, (size_t)npairs * 4 + 8, s));
    uint32_t* starts = (uint32_t*)ctx->ws[WS_STARTS].p;
    VX_TRY(vx_segment_starts(ctx, *k0, npairs, misc + 2, starts, s));
    VX_TRY(vx_readback_async(ctx, 0, misc, 12, s));
    VX_CUDA_TRY(cudaStreamSynchronize(s));
    if (((uint32_t*)ctx->host_pin)[0] & 4u) return VX_ERR_TIMEOUT;   // a bounded wait of the sort gave up
    *nseg = ((uint32_t*)ctx->host_pin)[2];
    return VX_OK;
}

// Per-voxel reduction and compaction of one window after window_segments: the non-empty
// voxels are written to `dst`, a level or a view into one at the window's first row, with
// room for at least nseg rows (dst == NULL: a new level block of exactly the window's
// voxels is allocated into *alloc_out).  *nvox receives the window's voxel count.
// Keys are key_hi | the Morton key relative to the window's corner.  Synchronises once.
vx_status window_reduce(vx_context* ctx, bool fiber, uint32_t np, uint32_t nseg, uint64_t key_hi, int res,
                        uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, const Window& win, float4* r0,
                        float4* r1, float4* r2, uint32_t* misc, cudaStream_t s, const vx_level* dst,
                        vx_level* alloc_out, uint32_t* nvox_out) {
    const int bx = win.lo[0], by = win.lo[1], bz = win.lo[2];
    uint32_t* flags = (uint32_t*)ctx->ws[WS_FLAGS].p;
    uint32_t* starts = (uint32_t*)ctx->ws[WS_STARTS].p;
    vx_stage_units(ctx, ST_FINALIZE, nseg);
    // temp outputs per candidate voxel: mask 64 + mass 4 + moment 24 bytes; the sort's
    // alternate buffers are free now and hold the key and the non-empty flag.
    VX_TRY(vx_ws_ensure(ctx, WS_SEG_OUT, (size_t)std::max<uint32_t>(nseg, 1) * (64 + 4 + 24), s));
    char* so = (char*)ctx->ws[WS_SEG_OUT].p;
    SegOut seg;
    seg.mask = (uint64_t*)so;
    seg.moment = (float*)(so + (size_t)nseg * 64);   // 8-byte aligned rows
    seg.mass = (float*)(so + (size_t)nseg * 88);
    seg.key = k1;
    seg.nonzero = v1;
    const unsigned rblocks = (unsigned)std::min<size_t>((nseg + RED_WARPS - 1) / RED_WARPS, (size_t)vx::kSMs * 32);
    VX_CUDA_TRY(cudaMemsetAsync(misc + 6, 0, 4, s));
    if (fiber) {
        // resident blocks (7 per SM) taking voxels from a counter
        const unsigned fblocks = (unsigned)std::min<size_t>((nseg + RED_WARPS - 1) / RED_WARPS, (size_t)vx::kSMs * 7);
        VX_LAUNCH(ctx, ST_REDUCE_FIBERS, s, k_reduce_fibers<<<fblocks, RED_WARPS * 32, 0, s>>>(
                                                k0, v0, starts, misc + 2, r0, r1, r2, seg, bx, by, bz, misc + 6));
    } else {
        VX_LAUNCH(ctx, ST_REDUCE_TRIS, s, k_reduce_tris<<<rblocks, RED_WARPS * 32, 0, s>>>(
                                              k0, v0, starts, misc + 2, r0, r1, r2, seg, bx, by, bz, misc + 6));
    }
    VX_CUDA_TRY(cudaGetLastError());
    // compaction: dst index = exclusive scan of the non-empty flags (the head flags are free)
    VX_TRY(vx_scan_u32(ctx, seg.nonzero, flags, nseg, misc + 3, s));
    VX_TRY(vx_readback_async(ctx, 0, misc + 3, 4, s));
    VX_CUDA_TRY(cudaStreamSynchronize(s));
    const uint32_t nvox = ((uint32_t*)ctx->host_pin)[0];
    *nvox_out = nvox;
    vx_level view;
    if (dst) {
        view = *dst;
    } else {
        VX_TRY(vx_level_alloc(ctx, alloc_out, nvox, 1, 0, res, s));
        view = *alloc_out;
    }
    if (nvox > 0) {
        VX_LAUNCH(ctx, ST_FINALIZE, s, k_finalize<<<grid_for(nseg, 256), 256, 0, s>>>(seg, misc + 2, flags, view, key_hi));
        VX_CUDA_TRY(cudaGetLastError());
    }
    return VX_OK;
}

// The level arrays of L from row `at` on (a view for k_finalize; K = 1 rows).
inline vx_level level_view(const vx_level& L, int64_t at) {
    vx_level v = L;
    v.keys += at;
    v.mask += (size_t)at * 8;
    v.mass += at;
    v.moment += (size_t)at * 6;
    v.occ += at;
    v.occ_proj += (size_t)at * 3;
    v.lobe_count += at;
    v.lobes += (size_t)at * 7 * L.K;
    v.compact += (size_t)at * 6 * L.K;
    return v;
}

// Prepared primitives of one voxelization: records in grid coordinates (WS_REC_A/B/C).
struct Prepared {
    bool fiber;
    uint32_t np;
    int bits_R;
    int R;
    float4 *r0, *r1, *r2;   // r2: triangles' third records, fibers' tangent terms
    uint32_t* misc;
};

vx_status prepare(vx_context* ctx, const vx_primitives* prims, const vx_grid* grid, cudaStream_t s, Prepared* P) {
    const uint32_t R = grid->resolution;
    if (R == 0 || (R & (R - 1)) != 0) return VX_ERR_INVALID_ARG;
    if (R > 2048 || grid->sub_res != 8) return VX_ERR_UNSUPPORTED;
    if (!(grid->voxel_size > 0.0f) || !isfinite(grid->voxel_size)) return VX_ERR_INVALID_ARG;
    if (prims->num_prims < 0 || prims->num_prims > 0xfffffffell) return VX_ERR_CAPACITY;
    const bool fiber = prims->kind == VX_FIBERS;
    if (!fiber && prims->kind != VX_TRIANGLES) return VX_ERR_INVALID_ARG;
    const uint32_t np = (uint32_t)prims->num_prims;
    P->fiber = fiber;
    P->np = np;
    P->R = (int)R;
    P->bits_R = 0;
    while ((1u << P->bits_R) < R) ++P->bits_R;
    P->r0 = P->r1 = P->r2 = nullptr;
    P->misc = nullptr;
    if (np == 0) return VX_OK;
    if (fiber) {
        if (!prims->ctrl || !prims->fiber_offsets || prims->num_fibers <= 0 || prims->num_ctrl < 0)
            return VX_ERR_INVALID_ARG;
        if (((uintptr_t)prims->ctrl & 15) != 0) return VX_ERR_INVALID_ARG;
    } else {
        if (!prims->tri_verts || ((uintptr_t)prims->tri_verts & 15) != 0) return VX_ERR_INVALID_ARG;
    }
    GridDev g;
    g.o[0] = grid->origin[0]; g.o[1] = grid->origin[1]; g.o[2] = grid->origin[2];
    g.s = 1.0f / grid->voxel_size;
    g.R = (int)R;
    VX_TRY(vx_ws_ensure(ctx, WS_REC_A, (size_t)np * 16, s));
    VX_TRY(vx_ws_ensure(ctx, WS_REC_B, (size_t)np * 16, s));
    // triangles: the third vertex records; fibers: the tangent terms (two float4 each)
    VX_TRY(vx_ws_ensure(ctx, WS_REC_C, (size_t)np * (fiber ? 32 : 16), s));
    VX_TRY(vx_ws_ensure(ctx, WS_MISC, 256, s));
    uint32_t* misc = (uint32_t*)ctx->ws[WS_MISC].p;   // [0] err, [1] npairs, [2] nseg, [3] nvox, [4] segtotal
    VX_CUDA_TRY(cudaMemsetAsync(misc, 0, 64, s));
    float4* r0 = (float4*)ctx->ws[WS_REC_A].p;
    float4* r1 = (float4*)ctx->ws[WS_REC_B].p;
    float4* r2 = (float4*)ctx->ws[WS_REC_C].p;
    if (fiber) {
        const int64_t F = prims->num_fibers;
        if (F > 0x7fffffff) return VX_ERR_CAPACITY;
        VX_TRY(vx_ws_ensure(ctx, WS_FIBER_START, (size_t)F * 4 + 256, s));
        uint32_t* fs = (uint32_t*)ctx->ws[WS_FIBER_START].p;
        VX_LAUNCH(ctx, ST_PREP, s, k_fiber_seg_counts<<<grid_for((size_t)F, 256), 256, 0, s>>>(prims->fiber_offsets, F, prims->num_ctrl, fs, misc));
        VX_TRY(vx_scan_u32(ctx, fs, fs, (uint32_t)F, misc + 4, s));
        VX_LAUNCH(ctx, ST_PREP, s, k_prep_fibers<<<grid_for(np, 256), 256, 0, s>>>((const float4*)prims->ctrl, prims->num_ctrl, prims->fiber_offsets, fs, F,
                                                         misc + 4, prims->weights, np, g, r0, r1, misc));
        VX_LAUNCH(ctx, ST_PREP, s, k_tangent_terms<<<grid_for(np, 256), 256, 0, s>>>(r0, r1, np, r2));
    } else {
        VX_LAUNCH(ctx, ST_PREP, s, k_prep_tris<<<grid_for(np, 256), 256, 0, s>>>((const float4*)prims->tri_verts, prims->weights, np, g, r0,
                                                       r1, r2, misc));
    }
    VX_CUDA_TRY(cudaGetLastError());
    vx_stage_units(ctx, ST_PREP, np);
    P->r0 = r0; P->r1 = r1; P->r2 = r2; P->misc = misc;
    return VX_OK;
}

// Windows of the region [lo, lo + 2^lg)^3 in Morton order: a window is split into its
// eight octants while it is wider than 2^max_lg voxels (max_lg <= 10: keys of one pass are
// 30-bit) or holds more candidate pairs than one pass may; octants without pairs are
// dropped.  Each window is counted (one synchronisation); the list holds every window that
// is kept, with its pair total.  VX_ERR_CAPACITY when a single voxel is over the limit.
// *counted (optional) receives the index of the leaf whose counts and offsets are still in
// the workspace (the last window counted was that leaf), or -1.
vx_status plan_windows(vx_context* ctx, const Prepared& P, const int lo[3], int lg, int max_lg, cudaStream_t s,
                       std::vector<Leaf>* leaves, int* counted) {
    if (counted) *counted = -1;
    struct Pending { int lo[3]; int lg; };
    std::vector<Pending> stack;
    stack.push_back(Pending{{lo[0], lo[1], lo[2]}, lg});
    const uint64_t limit = (uint64_t)std::min<int64_t>(ctx->max_pairs, kMaxPassPairs);
    while (!stack.empty()) {
        const Pending w = stack.back();
        stack.pop_back();
        Leaf leaf{{w.lo[0], w.lo[1], w.lo[2]}, w.lg, 0};
        uint64_t total = 0;
        VX_TRY(count_window(ctx, P.fiber, P.np, window_of(leaf), P.r0, P.r1, P.r2, P.misc, s, &total));
        if (counted) *counted = -1;
        if (total == 0) continue;                                 // an empty window adds nothing
        if (w.lg <= max_lg && total <= limit) {
            leaf.pairs = total;
            leaves->push_back(leaf);
            if (counted) *counted = (int)leaves->size() - 1;
            continue;
        }
        if (w.lg == 0) return VX_ERR_CAPACITY;                    // one voxel over the limit
        const int half = 1 << (w.lg - 1);
        for (int o = 7; o >= 0; --o) {                            // pushed in reverse: popped in Morton order
            Pending c;
            c.lg = w.lg - 1;
            c.lo[0] = w.lo[0] + ((o & 1) ? half : 0);
            c.lo[1] = w.lo[1] + ((o & 2) ? half : 0);
            c.lo[2] = w.lo[2] + ((o & 4) ? half : 0);
            stack.push_back(c);
        }
    }
    return VX_OK;
}

// Level 0 of the planned windows (Morton order), as one level block.  One window: its
// pipeline allocates the block.  Several: a first pass counts each window's candidate
// voxels (emit, sort, heads), one block is allocated for their sum, and a second pass
// reduces every window straight into its rows, so that no window is held twice.
// `counted`: index of the leaf whose counts and offsets are in the workspace (or -1).
vx_status voxelize_leaves(vx_context* ctx, const Prepared& P, const std::vector<Leaf>& leaves, int counted,
                          cudaStream_t s, vx_level* out0) {
    const int res = P.R;
    uint32_t *k0, *v0, *k1, *v1;
    for (const Leaf& w : leaves) {
        vx_stage_units(ctx, ST_COUNT, (int64_t)w.pairs);
        vx_stage_units(ctx, ST_EMIT, (int64_t)w.pairs);
        vx_stage_units(ctx, ST_SORT_SCATTER, (int64_t)w.pairs);
        vx_stage_units(ctx, ST_SORT_HIST, (int64_t)w.pairs);
        vx_stage_units(ctx, ST_REDUCE_FIBERS + (P.fiber ? 0 : 1), (int64_t)w.pairs);
    }
    if (leaves.empty()) return vx_level_alloc(ctx, out0, 0, 1, 0, res, s);
    if (leaves.size() == 1) {
        const Leaf& w = leaves[0];
        const Window win = window_of(w);
        uint64_t total = w.pairs;
        if (counted != 0) VX_TRY(count_window(ctx, P.fiber, P.np, win, P.r0, P.r1, P.r2, P.misc, s, &total));
        uint32_t nseg = 0, nvox = 0;
        VX_TRY(window_segments(ctx, P.fiber, P.np, win, w.lg, (uint32_t)total, P.r0, P.r1, P.r2, P.misc, s, &k0, &v0,
                               &k1, &v1, &nseg));
        vx_status st = window_reduce(ctx, P.fiber, P.np, nseg, key_hi_of(w), res, k0, v0, k1, v1, win, P.r0, P.r1,
                                     P.r2, P.misc, s, nullptr, out0, &nvox);
        if (st != VX_OK) vx_level_release(ctx, out0, s);
        return st;
    }
    // pass 1: candidate voxels per window (an upper bound of its voxels)
    std::vector<uint32_t> nsegs(leaves.size());
    int64_t cap = 0;
    for (size_t i = 0; i < leaves.size(); ++i) {
        const Window win = window_of(leaves[i]);
        uint64_t total = leaves[i].pairs;
        if (counted != (int)i) VX_TRY(count_window(ctx, P.fiber, P.np, win, P.r0, P.r1, P.r2, P.misc, s, &total));
        counted = (int)i;
        VX_TRY(window_segments(ctx, P.fiber, P.np, win, leaves[i].lg, (uint32_t)total, P.r0, P.r1, P.r2, P.misc, s,
                               &k0, &v0, &k1, &v1, &nsegs[i]));
        cap += nsegs[i];
    }
    VX_TRY(vx_level_alloc(ctx, out0, cap, 1, 0, res, s));
    // pass 2: every window reduced into its rows
    int64_t at = 0;
    vx_status st = VX_OK;
    for (size_t i = 0; i < leaves.size() && st == VX_OK; ++i) {
        const Window win = window_of(leaves[i]);
        uint64_t total = leaves[i].pairs;
        uint32_t nseg = 0, nvox = 0;
        if (counted != (int)i) st = count_window(ctx, P.fiber, P.np, win, P.r0, P.r1, P.r2, P.misc, s, &total);
        counted = (int)i;
        if (st == VX_OK)
            st = window_segments(ctx, P.fiber, P.np, win, leaves[i].lg, (uint32_t)total, P.r0, P.r1, P.r2, P.misc, s,
                                 &k0, &v0, &k1, &v1, &nseg);
        if (st == VX_OK && nseg != nsegs[i]) st = VX_ERR_CUDA;    // the two passes must agree
        if (st == VX_OK) {
            const vx_level view = level_view(*out0, at);
            st = window_reduce(ctx, P.fiber, P.np, nseg, key_hi_of(leaves[i]), res, k0, v0, k1, v1, win, P.r0, P.r1,
                               P.r2, P.misc, s, &view, nullptr, &nvox);
        }
        at += nvox;
    }
    if (st != VX_OK) {
        vx_level_release(ctx, out0, s);
        return st;
    }
    out0->num_voxels = at;
    return VX_OK;
}

}  // namespace

extern "C" vx_status vx_voxelize(vx_context* ctx, const vx_primitives* prims, const vx_grid* grid,
                                 void* stream, vx_level* out0) {
    if (!ctx || !prims || !grid || !out0) return VX_ERR_INVALID_ARG;
    memset(out0, 0, sizeof(*out0));
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    Prepared P;
    VX_TRY(prepare(ctx, prims, grid, s, &P));
    if (P.np == 0) return vx_level_alloc(ctx, out0, 0, 1, 0, P.R, s);
    std::vector<Leaf> leaves;
    const int lo[3] = {0, 0, 0};
    int counted = -1;
    VX_TRY(plan_windows(ctx, P, lo, P.bits_R, 10, s, &leaves, &counted));
    return voxelize_leaves(ctx, P, leaves, counted, s, out0);
}

// Copies row 0 of `src` (one voxel) into row i of `dst` (same K).
static vx_status copy_root(vx_context* ctx, const vx_level& src, const vx_level& dst, int64_t i, cudaStream_t s) {
    const int K = src.K;
    VX_CUDA_TRY(cudaMemcpyAsync(dst.keys + i, src.keys, 8, cudaMemcpyDeviceToDevice, s));
    VX_CUDA_TRY(cudaMemcpyAsync(dst.mask + (size_t)i * 8, src.mask, 64, cudaMemcpyDeviceToDevice, s));
    VX_CUDA_TRY(cudaMemcpyAsync(dst.mass + i, src.mass, 4, cudaMemcpyDeviceToDevice, s));
    VX_CUDA_TRY(cudaMemcpyAsync(dst.moment + (size_t)i * 6, src.moment, 24, cudaMemcpyDeviceToDevice, s));
    VX_CUDA_TRY(cudaMemcpyAsync(dst.occ + i, src.occ, 2, cudaMemcpyDeviceToDevice, s));
    VX_CUDA_TRY(cudaMemcpyAsync(dst.occ_proj + (size_t)i * 3, src.occ_proj, 3, cudaMemcpyDeviceToDevice, s));
    VX_CUDA_TRY(cudaMemcpyAsync(dst.lobe_count + i, src.lobe_count, 1, cudaMemcpyDeviceToDevice, s));
    VX_CUDA_TRY(cudaMemcpyAsync(dst.lobes + (size_t)i * 7 * K, src.lobes, (size_t)28 * K, cudaMemcpyDeviceToDevice, s));
    VX_CUDA_TRY(cudaMemcpyAsync(dst.compact + (size_t)i * 6 * K, src.compact, (size_t)24 * K, cudaMemcpyDeviceToDevice,
                                s));
    return VX_OK;
}

extern "C" vx_status vx_voxelize_lod_windowed(vx_context* ctx, const vx_primitives* prims, const vx_grid* grid,
                                              const vx_lod_params* lod, int window_log2, vx_window_fn on_window,
                                              void* user, void* stream, vx_level* top, int* num_top) {
    if (!ctx || !prims || !grid || !lod || !on_window || !top || !num_top) return VX_ERR_INVALID_ARG;
    *num_top = 0;
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    Prepared P;
    VX_TRY(prepare(ctx, prims, grid, s, &P));
    const int L = P.bits_R, w = window_log2;
    if (w < 1 || w > L) return VX_ERR_INVALID_ARG;
    if (lod->num_levels != 0) return VX_ERR_INVALID_ARG;
    if (lod->K < 1 || lod->K > vx::kMaxK) return VX_ERR_UNSUPPORTED;
    if (lod->K > 1 && (!lod->dirs || lod->n_samples < 1 || lod->n_samples > 65536)) return VX_ERR_INVALID_ARG;
    if (lod->merge != 0 && lod->merge != 1) return VX_ERR_INVALID_ARG;
    if (3 * (L - w) > 21) return VX_ERR_UNSUPPORTED;              // at most 2^21 windows
    const int K = lod->K;
    for (int l = 0; l <= L - w; ++l) memset(&top[l], 0, sizeof(vx_level));
    // the window roots (level w) are gathered here, one row per non-empty window
    vx_level roots;
    VX_TRY(vx_level_alloc(ctx, &roots, P.np ? (int64_t)1 << (3 * (L - w)) : 0, K, w, P.R >> w, s));
    vx_status st = VX_OK;
    int64_t nroots = 0;
    std::vector<Leaf> leaves;
    if (P.np) {
        const int lo[3] = {0, 0, 0};
        st = plan_windows(ctx, P, lo, P.bits_R, std::min(w, 10), s, &leaves, nullptr);
    }
    // leaves are in Morton order, so the leaves of one 2^w window are contiguous
    size_t i = 0;
    int64_t index = 0;
    while (st == VX_OK && i < leaves.size()) {
        const int sh = w;
        size_t j = i;
        while (j < leaves.size() && (leaves[j].lo[0] >> sh) == (leaves[i].lo[0] >> sh) &&
               (leaves[j].lo[1] >> sh) == (leaves[i].lo[1] >> sh) && (leaves[j].lo[2] >> sh) == (leaves[i].lo[2] >> sh))
            ++j;
        const std::vector<Leaf> group(leaves.begin() + i, leaves.begin() + j);
        vx_window info;
        for (int a = 0; a < 3; ++a) info.lo[a] = (leaves[i].lo[a] >> sh) << sh;
        info.log2_size = w;
        info.index = index;
        vx_level lv[12];
        memset(lv, 0, sizeof(lv));
        st = voxelize_leaves(ctx, P, group, -1, s, &lv[0]);
        if (st == VX_OK && lv[0].num_voxels > 0) {
            vx_lod_params wp = *lod;
            wp.num_levels = w;
            st = vx_build_lod(ctx, &lv[0], &wp, stream, &lv[1]);
            if (st == VX_OK) st = copy_root(ctx, lv[w], roots, nroots, s);
            if (st == VX_OK) {
                ++nroots;
                ++index;
                vx_level_release(ctx, &lv[w], s);
                // ownership of levels 0 .. w-1 passes to the callee, whatever it returns
                st = on_window(user, &info, lv, w, stream);
            } else {
                for (int l = 0; l <= w; ++l) vx_level_release(ctx, &lv[l], s);
            }
        } else {
            vx_level_release(ctx, &lv[0], s);
        }
        i = j;
    }
    if (st != VX_OK) {
        vx_level_release(ctx, &roots, s);
        return st;
    }
    roots.num_voxels = nroots;
    top[0] = roots;
    if (L > w) {
        vx_lod_params tp = *lod;
        tp.num_levels = L - w;
        st = vx_build_lod(ctx, &roots, &tp, stream, &top[1]);
        if (st != VX_OK) {
            vx_level_release(ctx, &top[0], s);
            return st;
        }
    }
    *num_top = L - w + 1;
    return VX_OK;
}

// =====================================================================================
// Adjoint (vx_backward)
// =====================================================================================
namespace {

__global__ void k_key_shift_flags(const uint64_t* __restrict__ keys, uint32_t n, int shift, uint32_t* __restrict__ flags) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flags[i] = (i == 0 || (keys[i] >> shift) != (keys[i - 1] >> shift)) ? 1u : 0u;
}

// level-0 adjoints (FP64): g = grad_0 (init) or g += grad_l[parent index]
__global__ void k_bcast(const uint32_t* __restrict__ excl, const uint32_t* __restrict__ flags, uint32_t n,
                        const float* __restrict__ gmass, const float* __restrict__ gmom, int init,
                        double* __restrict__ gm, double* __restrict__ gM) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t p = init ? i : excl[i] + flags[i] - 1u;
    if (init) {
        gm[i] = (double)gmass[p];
#pragma unroll
        for (int c = 0; c < 6; ++c) gM[(size_t)i * 6 + c] = (double)gmom[(size_t)p * 6 + c];
    } else {
        gm[i] = gm[i] + (double)gmass[p];
#pragma unroll
        for (int c = 0; c < 6; ++c) gM[(size_t)i * 6 + c] = gM[(size_t)i * 6 + c] + (double)gmom[(size_t)p * 6 + c];
    }
}

// Per-segment constants of the fiber adjoint (grid units, FP64): endpoints, direction,
// its length and reciprocal components, unit tangent, radius and weight.
struct SegAdj {
    double A[3], d[3], inv[3], t[3];
    double dn, r, w;
};
__device__ __forceinline__ SegAdj seg_adj(float4 Af, float4 Bf) {
    SegAdj g;
    g.A[0] = Af.x; g.A[1] = Af.y; g.A[2] = Af.z;
    g.d[0] = (double)Bf.x - Af.x; g.d[1] = (double)Bf.y - Af.y; g.d[2] = (double)Bf.z - Af.z;
    g.dn = sqrt(g.d[0] * g.d[0] + g.d[1] * g.d[1] + g.d[2] * g.d[2]);
    const double idn = g.dn > 0.0 ? 1.0 / g.dn : 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        g.inv[i] = g.d[i] != 0.0 ? 1.0 / g.d[i] : 0.0;
        g.t[i] = g.d[i] * idn;
    }
    g.r = Af.w;
    g.w = Bf.w;
    return g;
}

// d/d(A, B, r, w) of  w * pi r^2 len * (gm + gM . T(t))  for one (segment, voxel) pair
// (grid units); out: dA[3], dB[3], dr, dw.  FP64: the end-point terms of a piece that
// crosses a plane almost parallel to it are large and cancel between the two voxels
// sharing the plane, so FP32 would leave an error of a few 1e-6 of their size.
__device__ __forceinline__ void pair_grad(const SegAdj& g, int vi, int vj, int vk, double gm, const double* gM,
                                          double* out) {
#pragma unroll
    for (int c = 0; c < 8; ++c) out[c] = 0.0;
    const double a[3] = {g.A[0] - vi, g.A[1] - vj, g.A[2] - vk};
    double t0 = 0.0, t1 = 1.0;
    int ax0 = -1, ax1 = -1;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (g.d[i] == 0.0) {
            if (a[i] < 0.0 || a[i] > 1.0) return;
        } else {
            const double ta = -a[i] * g.inv[i], tb = (1.0 - a[i]) * g.inv[i];
            const double tn = g.d[i] > 0.0 ? ta : tb, tf = g.d[i] > 0.0 ? tb : ta;
            if (tn > t0) { t0 = tn; ax0 = i; }
            if (tf < t1) { t1 = tf; ax1 = i; }
        }
    }
    if (t1 <= t0) return;
    // (no bit-exact contract here: the multiply-adds are fused explicitly)
    const double pi = 3.14159265358979323846;
    const double* t = g.t;
    const double dn = g.dn;
    const double len = (t1 - t0) * dn;
    const double pr2 = pi * g.r * g.r;
    const double mu = pr2 * len;
    double gt[3];
    gt[0] = fma(2.0 * gM[0], t[0], fma(gM[3], t[1], gM[4] * t[2]));
    gt[1] = fma(gM[3], t[0], fma(2.0 * gM[1], t[1], gM[5] * t[2]));
    gt[2] = fma(gM[4], t[0], fma(gM[5], t[1], 2.0 * gM[2] * t[2]));
    // gm + gM . T(t) = gm + (t . gt) / 2 (T(t) pairs each off-diagonal once)
    const double tg = fma(t[0], gt[0], fma(t[1], gt[1], t[2] * gt[2]));
    const double G = fma(0.5, tg, gm);
    out[7] = mu * G;                       // d/dw
    out[6] = g.w * (2.0 * mu / g.r) * G;   // d/dr
    // d len / d A, d B: the clipped ends (1 - t_e) A + t_e B move with both endpoints, and an
    // end on a voxel plane also slides along the segment (its t_e depends on the endpoints)
    double cA[3], cB[3];
    const double dte = t1 - t0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        cA[k] = -dte * t[k];
        cB[k] = dte * t[k];
    }
    if (ax0 >= 0) {
        const double f = dn * g.inv[ax0];
        cA[ax0] = fma((1.0 - t0), f, cA[ax0]);
        cB[ax0] = fma(t0, f, cB[ax0]);
    }
    if (ax1 >= 0) {
        const double f = dn * g.inv[ax1];
        cA[ax1] = fma(-(1.0 - t1), f, cA[ax1]);
        cB[ax1] = fma(-t1, f, cB[ax1]);
    }
    const double kmu = g.w * pr2 * G;
    const double wmd = g.w * mu / dn;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double gd = wmd * fma(-t[k], tg, gt[k]);
        out[k] = fma(kmu, cA[k], -gd);
        out[3 + k] = fma(kmu, cB[k], gd);
    }
}

// first index in keys[lo, hi) whose key is >= k (hi when none)
__device__ __forceinline__ uint32_t lower_key(const uint64_t* __restrict__ keys, uint32_t lo, uint32_t hi, uint64_t k) {
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (keys[mid] < k) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// warp per segment: sum of its pair gradients (lane j takes pairs j, j+32, ...; fixed tree).
// The segment's candidate keys lie between their minimum and maximum, so the voxels are
// looked up in the slice of keys0 between those two keys.
// The window of one pass of the adjoint: pair keys are relative to its corner (wx, wy, wz),
// global keys are key_hi | key; per-primitive gradients are added to (accumulate) or written.
struct AdjWin {
    uint64_t key_hi;
    int wx, wy, wz;
    int accumulate;
};

__global__ void __launch_bounds__(EMIT_WARPS * 32) k_adjoint_fibers(const float4* __restrict__ ra,
                                                                    const float4* __restrict__ rb, uint32_t np,
                                                                    const uint32_t* __restrict__ offs,
                                                                    const uint32_t* __restrict__ cnt,
                                                                    const uint32_t* __restrict__ pkeys,
                                                                    const uint64_t* __restrict__ keys0, uint32_t V0,
                                                                    const double* __restrict__ gm,
                                                                    const double* __restrict__ gM,
                                                                    double* __restrict__ seg_grad, AdjWin W) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * EMIT_WARPS;
    for (uint32_t p = blockIdx.x * EMIT_WARPS + (threadIdx.x >> 5); p < np; p += warps) {
        const uint32_t beg = offs[p], n = cnt[p];
        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (n > 0) {
            const SegAdj g = seg_adj(ra[p], rb[p]);
            uint32_t kmin = 0xffffffffu, kmax = 0u;
            for (uint32_t j = lane; j < n; j += 32) {
                const uint32_t key = pkeys[beg + j];
                kmin = min(kmin, key);
                kmax = max(kmax, key);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
                kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
            }
            uint32_t bound = 0;
            if (lane == 0) bound = lower_key(keys0, 0, V0, W.key_hi | kmin);
            if (lane == 1) bound = lower_key(keys0, 0, V0, (W.key_hi | kmax) + 1);
            const uint32_t lo = __shfl_sync(0xffffffffu, bound, 0), hi = __shfl_sync(0xffffffffu, bound, 1);
            for (uint32_t j = lane; j < n; j += 32) {
                const uint32_t key = pkeys[beg + j];
                const uint64_t gk = W.key_hi | key;
                const uint32_t v = lower_key(keys0, lo, hi, gk);
                if (v >= hi || keys0[v] != gk) continue;
                double gr[8];
                double gMv[6];
#pragma unroll
                for (int c = 0; c < 6; ++c) gMv[c] = gM[(size_t)v * 6 + c];
                pair_grad(g, W.wx + (int)vx_compact1by2(key), W.wy + (int)vx_compact1by2(key >> 1),
                          W.wz + (int)vx_compact1by2(key >> 2), gm[v], gMv, gr);
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[c] = acc[c] + gr[c];
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = acc[c] + __shfl_xor_sync(0xffffffffu, acc[c], o);
        if (lane < 8) {
            double* o = seg_grad + (size_t)p * 8 + lane;
            *o = W.accumulate ? *o + acc[lane] : acc[lane];
        }
    }
}

// thread per control point: world-unit gradients from the segment before and after it
__global__ void k_adjoint_ctrl(const int64_t* __restrict__ off, int64_t F, const uint32_t* __restrict__ seg_start,
                               int64_t P, const double* __restrict__ seg_grad, float s, float4* __restrict__ gctrl) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P) return;
    int64_t lo = 0, hi = F;       // last fiber with off[f] <= c
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= c) lo = mid + 1; else hi = mid;
    }
    const int64_t f = lo - 1;
    float4 g = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (f >= 0 && c < off[f + 1]) {
        const bool has_prev = c > off[f];
        const bool has_next = c + 1 < off[f + 1];
        double px = 0.0, py = 0.0, pz = 0.0, pr = 0.0, nx = 0.0, ny = 0.0, nz = 0.0, nr = 0.0;
        if (has_prev) {
            const double* q = seg_grad + (size_t)(seg_start[f] + (uint32_t)(c - 1 - off[f])) * 8;
            px = q[3]; py = q[4]; pz = q[5]; pr = q[6];
        }
        if (has_next) {
            const double* q = seg_grad + (size_t)(seg_start[f] + (uint32_t)(c - off[f])) * 8;
            nx = q[0]; ny = q[1]; nz = q[2]; nr = q[6];
        }
        g.x = (float)((px + nx) * (double)s);
        g.y = (float)((py + ny) * (double)s);
        g.z = (float)((pz + nz) * (double)s);
        g.w = (float)((pr + nr) * (0.5 * (double)s));
    }
    gctrl[c] = g;
}

// d/d(U0, U1, U2, w) of  w * area(T ∩ voxel) * (gm + gM . T(n))  for one (triangle, voxel)
// pair (grid units, FP64); out[3j + k] = d/dU_j[k], out[9] = d/dw.
// The triangle is the image of the reference triangle {s, t >= 0, s + t <= 1} under
// (s, t) -> U0 + s e1 + t e2, so area(T ∩ voxel) = J * A, J = |e1 x e2|, A the area of
// the reference polygon cut out by the six voxel half-planes.  A box constraint
// g(s, t) <= 0 whose value changes by dg when a vertex moves shifts its polygon edge
// outward by -dg / |grad g|, so dA = -sum over the polygon's edges on box planes of
// (edge length / |grad g|) * dg(edge midpoint) (dg is affine in s, t).  The clip
// decisions are taken on voxel-local coordinates, as the forward's clip takes them: a
// vertex or an edge lying exactly on a voxel plane (a heightfield's border row) stays
// inside, and its derivative is that of the piece it belongs to.
__device__ void tri_pair_grad(const float4 P0, const float4 P1, const float4 P2, int vi, int vj, int vk, double gm,
                              const double* gM, double* out) {
#pragma unroll
    for (int c = 0; c < 10; ++c) out[c] = 0.0;
    const double e1[3] = {(double)P1.x - P0.x, (double)P1.y - P0.y, (double)P1.z - P0.z};
    const double e2[3] = {(double)P2.x - P0.x, (double)P2.y - P0.y, (double)P2.z - P0.z};
    // polygon vertices carry their voxel-local coordinates (x, y, z: every clip decision is
    // taken on them, exact for the triangle's own vertices) and their reference-domain
    // coordinates (s, t); lab[i] labels the edge i -> i+1: -1 a triangle edge, 2k + side a
    // voxel plane
    double px[12], py[12], pz[12], ps[12], pt[12];
    double qx[12], qy[12], qz[12], qs[12], qt[12];
    int lab[12], qlab[12];
    px[0] = (double)P0.x - vi; py[0] = (double)P0.y - vj; pz[0] = (double)P0.z - vk;
    px[1] = (double)P1.x - vi; py[1] = (double)P1.y - vj; pz[1] = (double)P1.z - vk;
    px[2] = (double)P2.x - vi; py[2] = (double)P2.y - vj; pz[2] = (double)P2.z - vk;
    ps[0] = 0.0; pt[0] = 0.0; ps[1] = 1.0; pt[1] = 0.0; ps[2] = 0.0; pt[2] = 1.0;
    lab[0] = lab[1] = lab[2] = -1;
    int n = 3;
    for (int c = 0; c < 6 && n > 0; ++c) {
        const int k = c >> 1;
        const bool hi = c & 1;
        const double bound = hi ? 1.0 : 0.0;
        int m = 0;
        for (int i = 0; i < n; ++i) {
            const int j = (i + 1 == n) ? 0 : i + 1;
            const double xi = k == 0 ? px[i] : (k == 1 ? py[i] : pz[i]);
            const double xj = k == 0 ? px[j] : (k == 1 ? py[j] : pz[j]);
            const bool sin_ = hi ? (xi <= 1.0) : (xi >= 0.0);
            const bool ein = hi ? (xj <= 1.0) : (xj >= 0.0);
            if (sin_) {
                qx[m] = px[i]; qy[m] = py[i]; qz[m] = pz[i]; qs[m] = ps[i]; qt[m] = pt[i]; qlab[m] = lab[i];
                ++m;
            }
            if (sin_ != ein) {
                const double l = (bound - xi) / (xj - xi);
                qx[m] = k == 0 ? bound : px[i] + l * (px[j] - px[i]);
                qy[m] = k == 1 ? bound : py[i] + l * (py[j] - py[i]);
                qz[m] = k == 2 ? bound : pz[i] + l * (pz[j] - pz[i]);
                qs[m] = ps[i] + l * (ps[j] - ps[i]);
                qt[m] = pt[i] + l * (pt[j] - pt[i]);
                qlab[m] = sin_ ? c : lab[i];
                ++m;
            }
        }
        n = m;
        for (int i = 0; i < n; ++i) {
            px[i] = qx[i]; py[i] = qy[i]; pz[i] = qz[i]; ps[i] = qs[i]; pt[i] = qt[i]; lab[i] = qlab[i];
        }
    }
    if (n < 3) return;
    double A = 0.0;
    double dA[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int i = 0; i < n; ++i) {
        const int j = (i + 1 == n) ? 0 : i + 1;
        A += ps[i] * pt[j] - ps[j] * pt[i];
        const int c = lab[i];
        if (c < 0) continue;
        const int k = c >> 1;
        const double gn = sqrt(e1[k] * e1[k] + e2[k] * e2[k]);
        if (gn == 0.0) continue;
        const double ds = ps[j] - ps[i], dt = pt[j] - pt[i];
        const double f = -sqrt(ds * ds + dt * dt) / gn * ((c & 1) ? 1.0 : -1.0);
        const double sm = 0.5 * (ps[i] + ps[j]), tm = 0.5 * (pt[i] + pt[j]);
        dA[0][k] += f * (1.0 - sm - tm);
        dA[1][k] += f * sm;
        dA[2][k] += f * tm;
    }
    A *= 0.5;
    const double nr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const double J = sqrt(nr[0] * nr[0] + nr[1] * nr[1] + nr[2] * nr[2]);
    if (!(J > 0.0) || !(A > 0.0)) return;
    const double nh[3] = {nr[0] / J, nr[1] / J, nr[2] / J};
    const double mu = J * A;
    const double G = gm + gM[0] * nh[0] * nh[0] + gM[1] * nh[1] * nh[1] + gM[2] * nh[2] * nh[2] +
                     gM[3] * nh[0] * nh[1] + gM[4] * nh[0] * nh[2] + gM[5] * nh[1] * nh[2];
    double gt[3];
    gt[0] = 2.0 * gM[0] * nh[0] + gM[3] * nh[1] + gM[4] * nh[2];
    gt[1] = gM[3] * nh[0] + 2.0 * gM[1] * nh[1] + gM[5] * nh[2];
    gt[2] = gM[4] * nh[0] + gM[5] * nh[1] + 2.0 * gM[2] * nh[2];
    const double ng = nh[0] * gt[0] + nh[1] * gt[1] + nh[2] * gt[2];
    // q = d G / d (raw normal)
    const double q[3] = {(gt[0] - nh[0] * ng) / J, (gt[1] - nh[1] * ng) / J, (gt[2] - nh[2] * ng) / J};
    const double w = P0.w;
    const double U[3][3] = {{P0.x, P0.y, P0.z}, {P1.x, P1.y, P1.z}, {P2.x, P2.y, P2.z}};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        // d J / d U_j = (U_j+1 - U_j+2) x nh,  d G / d U_j = (U_j+1 - U_j+2) x q
        const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        const double d[3] = {U[j1][0] - U[j2][0], U[j1][1] - U[j2][1], U[j1][2] - U[j2][2]};
        const double dJ[3] = {d[1] * nh[2] - d[2] * nh[1], d[2] * nh[0] - d[0] * nh[2], d[0] * nh[1] - d[1] * nh[0]};
        const double dG[3] = {d[1] * q[2] - d[2] * q[1], d[2] * q[0] - d[0] * q[2], d[0] * q[1] - d[1] * q[0]};
#pragma unroll
        for (int k = 0; k < 3; ++k) out[3 * j + k] = w * ((dJ[k] * A + J * dA[j][k]) * G + mu * dG[k]);
    }
    out[9] = mu * G;
}

// warp per triangle: sum of its pair gradients (lane j takes pairs j, j+32, ...; fixed tree)
__global__ void __launch_bounds__(EMIT_WARPS * 32) k_adjoint_tris(const float4* __restrict__ r0,
                                                                  const float4* __restrict__ r1,
                                                                  const float4* __restrict__ r2, uint32_t np,
                                                                  const uint32_t* __restrict__ offs,
                                                                  const uint32_t* __restrict__ cnt,
                                                                  const uint32_t* __restrict__ pkeys,
                                                                  const uint64_t* __restrict__ keys0, uint32_t V0,
                                                                  const double* __restrict__ gm,
                                                                  const double* __restrict__ gM,
                                                                  double* __restrict__ tri_grad, AdjWin W) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * EMIT_WARPS;
    for (uint32_t p = blockIdx.x * EMIT_WARPS + (threadIdx.x >> 5); p < np; p += warps) {
        const float4 A = r0[p], B = r1[p], Cv = r2[p];
        const uint32_t beg = offs[p], n = cnt[p];
        double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        // the triangle's voxels lie in the slice of keys0 between its smallest and largest key
        uint32_t kmin = 0xffffffffu, kmax = 0u;
        for (uint32_t j = lane; j < n; j += 32) {
            const uint32_t key = pkeys[beg + j];
            kmin = min(kmin, key);
            kmax = max(kmax, key);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
            kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        }
        uint32_t bound = 0;
        if (n > 0 && lane == 0) bound = lower_key(keys0, 0, V0, W.key_hi | kmin);
        if (n > 0 && lane == 1) bound = lower_key(keys0, 0, V0, (W.key_hi | kmax) + 1);
        const uint32_t lo = __shfl_sync(0xffffffffu, bound, 0), hi = __shfl_sync(0xffffffffu, bound, 1);
        for (uint32_t j = lane; j < n; j += 32) {
            const uint32_t key = pkeys[beg + j];
            const uint64_t gk = W.key_hi | key;
            const uint32_t v = lower_key(keys0, lo, hi, gk);
            if (v >= hi || keys0[v] != gk) continue;
            double g[10];
            double gMv[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) gMv[c] = gM[(size_t)v * 6 + c];
            tri_pair_grad(A, B, Cv, W.wx + (int)vx_compact1by2(key), W.wy + (int)vx_compact1by2(key >> 1),
                          W.wz + (int)vx_compact1by2(key >> 2), gm[v], gMv, g);
#pragma unroll
            for (int c = 0; c < 10; ++c) acc[c] = acc[c] + g[c];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int c = 0; c < 10; ++c) acc[c] = acc[c] + __shfl_xor_sync(0xffffffffu, acc[c], o);
        if (lane < 10) {
            double* o = tri_grad + (size_t)p * 10 + lane;
            *o = W.accumulate ? *o + acc[lane] : acc[lane];
        }
    }
}

// thread per triangle: world-unit vertex gradients ([T][3] float4, w = 0) and weights
__global__ void k_adjoint_tri_out(const double* __restrict__ tri_grad, uint32_t np, float s,
                                  float4* __restrict__ gverts, float* __restrict__ gw) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const double* q = tri_grad + (size_t)p * 10;
#pragma unroll
    for (int j = 0; j < 3; ++j)
        gverts[(size_t)p * 3 + j] = make_float4((float)(q[3 * j] * (double)s), (float)(q[3 * j + 1] * (double)s),
                                                (float)(q[3 * j + 2] * (double)s), 0.0f);
    if (gw) gw[p] = (float)q[9];
}

__global__ void k_adjoint_weights(const double* __restrict__ seg_grad, uint32_t np, float* __restrict__ gw) {
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < np) gw[p] = (float)seg_grad[(size_t)p * 8 + 7];
}

}  // namespace

extern "C" vx_status vx_backward(vx_context* ctx, const vx_primitives* prims, const vx_grid* grid,
                                 const uint64_t* keys0, int64_t num_voxels0, int num_levels,
                                 const float* const* grad_mass, const float* const* grad_moment, void* stream,
                                 float* grad_ctrl, float* grad_weights) {
    if (!ctx || !prims || !grid || !grad_mass || !grad_moment || !grad_ctrl) return VX_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    const bool fiber = prims->kind == VX_FIBERS;
    if (!fiber && prims->kind != VX_TRIANGLES) return VX_ERR_INVALID_ARG;
    const uint32_t R = grid->resolution;
    if (R == 0 || (R & (R - 1)) != 0) return VX_ERR_INVALID_ARG;
    if (R > 2048 || grid->sub_res != 8) return VX_ERR_UNSUPPORTED;
    if (num_voxels0 < 0 || num_voxels0 > 0xffffffffll || num_levels < 0 || num_levels > 11) return VX_ERR_INVALID_ARG;
    if ((num_voxels0 > 0 && !keys0) || !(grid->voxel_size > 0.0f) || !isfinite(grid->voxel_size))
        return VX_ERR_INVALID_ARG;
    if (fiber && prims->num_ctrl < 0) return VX_ERR_INVALID_ARG;
    if (prims->num_prims < 0 || prims->num_prims > 0xfffffffell) return VX_ERR_CAPACITY;
    if (((uintptr_t)grad_ctrl & 15) != 0) return VX_ERR_INVALID_ARG;
    if (fiber && (!prims->ctrl || !prims->fiber_offsets || prims->num_fibers <= 0 || ((uintptr_t)prims->ctrl & 15) != 0))
        return VX_ERR_INVALID_ARG;
    if (!fiber && prims->num_prims > 0 && (!prims->tri_verts || ((uintptr_t)prims->tri_verts & 15) != 0))
        return VX_ERR_INVALID_ARG;
    for (int l = 0; l <= num_levels; ++l)
        if (!grad_mass[l] || !grad_moment[l]) return VX_ERR_INVALID_ARG;
    const uint32_t np = (uint32_t)prims->num_prims;
    const uint32_t V0 = (uint32_t)num_voxels0;
    const int64_t P = fiber ? prims->num_ctrl : 3 * (int64_t)np, F = prims->num_fibers;
    GridDev g;
    g.o[0] = grid->origin[0]; g.o[1] = grid->origin[1]; g.o[2] = grid->origin[2];
    g.s = 1.0f / grid->voxel_size;
    g.R = (int)R;
    if (P) VX_CUDA_TRY(cudaMemsetAsync(grad_ctrl, 0, (size_t)P * 16, s));
    if (grad_weights && np) VX_CUDA_TRY(cudaMemsetAsync(grad_weights, 0, (size_t)np * 4, s));
    if (np == 0) return VX_OK;

    // ---- level-0 adjoints (coarse adjoints broadcast down) ------------------------------
    VX_TRY(vx_ws_ensure(ctx, WS_LOD_FLAGS, (size_t)std::max<uint32_t>(V0, 1) * 4, s));
    VX_TRY(vx_ws_ensure(ctx, WS_LOD_IDX, (size_t)std::max<uint32_t>(V0, 1) * 4, s));
    VX_TRY(vx_ws_ensure(ctx, WS_LOD_TMP, (size_t)std::max<uint32_t>(V0, 1) * 56, s));
    uint32_t* flags = (uint32_t*)ctx->ws[WS_LOD_FLAGS].p;
    uint32_t* excl = (uint32_t*)ctx->ws[WS_LOD_IDX].p;
    double* gm = (double*)ctx->ws[WS_LOD_TMP].p;
    double* gM = gm + V0;
    if (V0) {
        VX_LAUNCH(ctx, ST_LOD_HEADS, s, k_bcast<<<grid_for(V0, 256), 256, 0, s>>>(excl, flags, V0, grad_mass[0],
                                                                                 grad_moment[0], 1, gm, gM));
        for (int l = 1; l <= num_levels; ++l) {
            VX_LAUNCH(ctx, ST_LOD_HEADS, s, k_key_shift_flags<<<grid_for(V0, 256), 256, 0, s>>>(keys0, V0, 3 * l, flags));
            VX_TRY(vx_scan_u32(ctx, flags, excl, V0, nullptr, s));
            VX_LAUNCH(ctx, ST_LOD_HEADS, s, k_bcast<<<grid_for(V0, 256), 256, 0, s>>>(excl, flags, V0, grad_mass[l],
                                                                                     grad_moment[l], 0, gm, gM));
        }
    }
    // ---- recompute the candidate pairs (primitive-major order), window by window ----------
    // Windows as in vx_voxelize: at most 1024 voxels wide and one pass of pairs each.  Every
    // window adds its pairs' terms to the per-primitive gradients (FP64).
    Prepared Pp;
    VX_TRY(prepare(ctx, prims, grid, s, &Pp));
    std::vector<Leaf> leaves;
    int counted = -1;
    const int lo0[3] = {0, 0, 0};
    VX_TRY(plan_windows(ctx, Pp, lo0, Pp.bits_R, 10, s, &leaves, &counted));
    float4 *r0 = Pp.r0, *r1 = Pp.r1, *r2 = Pp.r2;
    uint32_t* misc = Pp.misc;
    uint32_t* fs = fiber ? (uint32_t*)ctx->ws[WS_FIBER_START].p : nullptr;
    const size_t per_prim = fiber ? 64 : 80;
    VX_TRY(vx_ws_ensure(ctx, WS_SEG_OUT, (size_t)np * per_prim, s));
    double* pgrad = (double*)ctx->ws[WS_SEG_OUT].p;
    VX_CUDA_TRY(cudaMemsetAsync(pgrad, 0, (size_t)np * per_prim, s));
    const unsigned cblocks = (unsigned)std::min<size_t>((np + EMIT_WARPS - 1) / EMIT_WARPS, (size_t)vx::kSMs * 64);
    for (size_t i = 0; i < leaves.size(); ++i) {
        const Leaf& w = leaves[i];
        const Window win = window_of(w);
        uint64_t total = w.pairs;
        if (counted != (int)i) VX_TRY(count_window(ctx, fiber, np, win, r0, r1, r2, misc, s, &total));
        counted = (int)i;
        const uint32_t npairs = (uint32_t)total;
        uint32_t* cnt = (uint32_t*)ctx->ws[WS_COUNT].p;
        uint32_t* offs = (uint32_t*)ctx->ws[WS_OFFS].p;
        VX_TRY(vx_ws_ensure(ctx, WS_KEYS0, (size_t)std::max<uint32_t>(npairs, 1) * 4, s));
        VX_TRY(vx_ws_ensure(ctx, WS_VALS0, (size_t)std::max<uint32_t>(npairs, 1) * 4, s));
        uint32_t* k0 = (uint32_t*)ctx->ws[WS_KEYS0].p;
        uint32_t* v0 = (uint32_t*)ctx->ws[WS_VALS0].p;
        AdjWin W;
        W.key_hi = key_hi_of(w);
        W.wx = w.lo[0]; W.wy = w.lo[1]; W.wz = w.lo[2];
        W.accumulate = 1;
        if (fiber) {
            VX_LAUNCH(ctx, ST_EMIT, s, k_candidates<true, true><<<cblocks, EMIT_WARPS * 32, 0, s>>>(
                                           r0, r1, nullptr, np, win, nullptr, offs, k0, v0));
            VX_LAUNCH(ctx, ST_REDUCE_FIBERS, s, k_adjoint_fibers<<<cblocks, EMIT_WARPS * 32, 0, s>>>(
                                                    r0, r1, np, offs, cnt, k0, keys0, V0, gm, gM, pgrad, W));
        } else {
            VX_LAUNCH(ctx, ST_EMIT, s, k_candidates<false, true><<<cblocks, EMIT_WARPS * 32, 0, s>>>(
                                           r0, r1, r2, np, win, nullptr, offs, k0, v0));
            VX_LAUNCH(ctx, ST_REDUCE_TRIS, s, k_adjoint_tris<<<cblocks, EMIT_WARPS * 32, 0, s>>>(
                                                  r0, r1, r2, np, offs, cnt, k0, keys0, V0, gm, gM, pgrad, W));
        }
        VX_CUDA_TRY(cudaGetLastError());
    }
    if (!fiber) {
        // per-triangle gradients (no sharing between triangles: no scatter)
        VX_LAUNCH(ctx, ST_FINALIZE, s, k_adjoint_tri_out<<<grid_for(np, 256), 256, 0, s>>>(
                                           pgrad, np, g.s, (float4*)grad_ctrl, grad_weights));
        VX_CUDA_TRY(cudaGetLastError());
        return VX_OK;
    }
    // per-segment gradients, then the control-point scatter
    VX_LAUNCH(ctx, ST_FINALIZE, s, k_adjoint_ctrl<<<grid_for((size_t)P, 256), 256, 0, s>>>(
                                       prims->fiber_offsets, F, fs, P, pgrad, g.s, (float4*)grad_ctrl));
    if (grad_weights)
        VX_LAUNCH(ctx, ST_FINALIZE, s, k_adjoint_weights<<<grid_for(np, 256), 256, 0, s>>>(pgrad, np, grad_weights));
    VX_CUDA_TRY(cudaGetLastError());
    return VX_OK;
}

// =====================================================================================
// vx_backward_noalloc: the adjoint with its scratch in a fixed device array
// =====================================================================================
// For callers that cannot allocate device memory.  The scratch is one file-scope device
// array, sized for the limits below, held by every device that loads the library until
// the process exits.  Host code must not pass the array's name to a kernel (on the host
// it names a host-side stand-in): its device address is fetched once per device with
// cudaGetSymbolAddress and cached.
namespace {

constexpr uint32_t NA_MAX_PRIMS = 1u << 16;    // 65,536 segments
constexpr uint32_t NA_MAX_FIBERS = 1u << 13;   // 8,192 fibers
constexpr uint32_t NA_MAX_PAIRS = 1u << 21;    // 2,097,152 candidate (voxel, segment) pairs
constexpr uint32_t NA_MAX_VOXELS = 1u << 18;   // 262,144 level-0 voxels

constexpr size_t na_al(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t NA_RA = 0;
constexpr size_t NA_RB = NA_RA + na_al(16ull * NA_MAX_PRIMS);
constexpr size_t NA_CNT = NA_RB + na_al(16ull * NA_MAX_PRIMS);
constexpr size_t NA_OFFS = NA_CNT + na_al(4ull * NA_MAX_PRIMS);
constexpr size_t NA_FS = NA_OFFS + na_al(4ull * NA_MAX_PRIMS);
constexpr size_t NA_MISC = NA_FS + na_al(4ull * NA_MAX_FIBERS + 4);
constexpr size_t NA_KEYS = NA_MISC + 256;
constexpr size_t NA_VALS = NA_KEYS + na_al(4ull * NA_MAX_PAIRS);
constexpr size_t NA_SEG = NA_VALS + na_al(4ull * NA_MAX_PAIRS);
constexpr size_t NA_FLAGS = NA_SEG + na_al(64ull * NA_MAX_PRIMS);
constexpr size_t NA_EXCL = NA_FLAGS + na_al(4ull * NA_MAX_VOXELS);
constexpr size_t NA_GM = NA_EXCL + na_al(4ull * NA_MAX_VOXELS);
constexpr size_t NA_GMM = NA_GM + na_al(8ull * NA_MAX_VOXELS);
constexpr size_t NA_PART = NA_GMM + na_al(48ull * NA_MAX_VOXELS);
constexpr size_t NA_BYTES = NA_PART + na_al(4ull * (NA_MAX_VOXELS / 2048 + 64));   // ~39 MB

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

std::mutex g_na_mutex;
unsigned char* g_na_ptr[256] = {};

// device address of the scratch array on the current device (set up on first use); the
// stream must belong to that device, or the address would be another device's
vx_status na_scratch(cudaStream_t s, unsigned char** out) {
    int dev = 0, sdev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VX_ERR_CUDA;
    if (cudaStreamGetDevice(s, &sdev) != cudaSuccess) return VX_ERR_INVALID_ARG;
    if (sdev != dev) return VX_ERR_INVALID_ARG;
    if (dev < 0 || dev >= 256) return VX_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return VX_ERR_CUDA;
        g_na_ptr[dev] = (unsigned char*)p;
    }
    *out = g_na_ptr[dev];
    return VX_OK;
}

}  // namespace

#define NA_TRY(expr)                                   \
    do {                                               \
        if ((expr) != cudaSuccess) return VX_ERR_CUDA; \
    } while (0)

extern "C" vx_status vx_backward_noalloc(const vx_primitives* prims, const vx_grid* grid, const uint64_t* keys0,
                                         int64_t num_voxels0, int num_levels, const float* const* grad_mass,
                                         const float* const* grad_moment, void* stream, float* grad_ctrl,
                                         float* grad_weights) {
    if (!prims || !grid || !grad_mass || !grad_moment || !grad_ctrl) return VX_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (prims->kind != VX_FIBERS) return VX_ERR_UNSUPPORTED;
    const uint32_t R = grid->resolution;
    if (R == 0 || (R & (R - 1)) != 0) return VX_ERR_INVALID_ARG;
    if (R > 1024 || grid->sub_res != 8) return VX_ERR_UNSUPPORTED;
    if (num_voxels0 < 0 || num_levels < 0 || num_levels > 11 || prims->num_prims < 0 || prims->num_fibers <= 0 ||
        prims->num_ctrl < 0 || (num_voxels0 > 0 && !keys0) || !(grid->voxel_size > 0.0f) ||
        !isfinite(grid->voxel_size))
        return VX_ERR_INVALID_ARG;
    if (prims->num_prims > (int64_t)NA_MAX_PRIMS || prims->num_fibers > (int64_t)NA_MAX_FIBERS ||
        num_voxels0 > (int64_t)NA_MAX_VOXELS)
        return VX_ERR_CAPACITY;
    if (!prims->ctrl || !prims->fiber_offsets || ((uintptr_t)prims->ctrl & 15) != 0 ||
        ((uintptr_t)grad_ctrl & 15) != 0)
        return VX_ERR_INVALID_ARG;
    for (int l = 0; l <= num_levels; ++l)
        if (!grad_mass[l] || !grad_moment[l]) return VX_ERR_INVALID_ARG;
    unsigned char* base = nullptr;
    VX_TRY(na_scratch(s, &base));
    const uint32_t np = (uint32_t)prims->num_prims;
    const uint32_t V0 = (uint32_t)num_voxels0;
    const int64_t P = prims->num_ctrl, F = prims->num_fibers;
    GridDev g;
    g.o[0] = grid->origin[0]; g.o[1] = grid->origin[1]; g.o[2] = grid->origin[2];
    g.s = 1.0f / grid->voxel_size;
    g.R = (int)R;
    float4* r0 = (float4*)(base + NA_RA);
    float4* r1 = (float4*)(base + NA_RB);
    uint32_t* cnt = (uint32_t*)(base + NA_CNT);
    uint32_t* offs = (uint32_t*)(base + NA_OFFS);
    uint32_t* fs = (uint32_t*)(base + NA_FS);
    uint32_t* misc = (uint32_t*)(base + NA_MISC);
    uint32_t* k0 = (uint32_t*)(base + NA_KEYS);
    uint32_t* v0 = (uint32_t*)(base + NA_VALS);
    double* seg_grad = (double*)(base + NA_SEG);
    uint32_t* flags = (uint32_t*)(base + NA_FLAGS);
    uint32_t* excl = (uint32_t*)(base + NA_EXCL);
    double* gm = (double*)(base + NA_GM);
    double* gM = (double*)(base + NA_GMM);
    uint32_t* part = (uint32_t*)(base + NA_PART);

    // the array keeps the previous call's contents: clear the counters and error flag
    NA_TRY(cudaMemsetAsync(misc, 0, 64, s));
    if (np == 0) {
        if (P) NA_TRY(cudaMemsetAsync(grad_ctrl, 0, (size_t)P * 16, s));
        return VX_OK;
    }

    // level-0 adjoints (coarse adjoints broadcast down)
    if (V0) {
        k_bcast<<<grid_for(V0, 256), 256, 0, s>>>(excl, flags, V0, grad_mass[0], grad_moment[0], 1, gm, gM);
        for (int l = 1; l <= num_levels; ++l) {
            k_key_shift_flags<<<grid_for(V0, 256), 256, 0, s>>>(keys0, V0, 3 * l, flags);
            NA_TRY(vx_scan_u32_scratch(flags, excl, V0, nullptr, part, s));
            k_bcast<<<grid_for(V0, 256), 256, 0, s>>>(excl, flags, V0, grad_mass[l], grad_moment[l], 0, gm, gM);
        }
    }
    // candidate pairs, primitive-major
    k_fiber_seg_counts<<<grid_for((size_t)F, 256), 256, 0, s>>>(prims->fiber_offsets, F, prims->num_ctrl, fs, misc);
    NA_TRY(vx_scan_u32_scratch(fs, fs, (uint32_t)F, misc + 4, part, s));
    k_prep_fibers<<<grid_for(np, 256), 256, 0, s>>>((const float4*)prims->ctrl, prims->num_ctrl, prims->fiber_offsets, fs, F, misc + 4,
                                                     prims->weights, np, g, r0, r1, misc);
    const unsigned cblocks = (unsigned)std::min<size_t>((np + EMIT_WARPS - 1) / EMIT_WARPS, (size_t)vx::kSMs * 64);
    k_candidates<true, false><<<cblocks, EMIT_WARPS * 32, 0, s>>>(r0, r1, nullptr, np, full_window((int)R), cnt,
                                                                  nullptr, nullptr, nullptr);
    NA_TRY(vx_scan_u32_scratch(cnt, offs, np, misc + 1, part, s));
    // the exact 64-bit total (the 32-bit scan total wraps)
    k_sum_u64<<<(unsigned)std::min<size_t>(grid_for(np, 256), (size_t)vx::kSMs * 8), 256, 0, s>>>(
        cnt, np, (unsigned long long*)(misc + 8));
    uint32_t host[12] = {0};
    NA_TRY(cudaMemcpyAsync(host, misc, 48, cudaMemcpyDeviceToHost, s));
    NA_TRY(cudaStreamSynchronize(s));
    if (host[0]) return VX_ERR_INVALID_ARG;
    uint64_t npairs64 = 0;
    memcpy(&npairs64, host + 8, 8);
    if (npairs64 > NA_MAX_PAIRS) return VX_ERR_CAPACITY;
    const uint32_t npairs = (uint32_t)npairs64;
    // the caller's outputs are written only once every limit has passed
    NA_TRY(cudaMemsetAsync(grad_ctrl, 0, (size_t)P * 16, s));
    if (grad_weights) NA_TRY(cudaMemsetAsync(grad_weights, 0, (size_t)np * 4, s));
    if (npairs)
        k_candidates<true, true><<<cblocks, EMIT_WARPS * 32, 0, s>>>(r0, r1, nullptr, np, full_window((int)R), nullptr,
                                                                     offs, k0, v0);
    AdjWin W0;
    W0.key_hi = 0;
    W0.wx = W0.wy = W0.wz = 0;
    W0.accumulate = 0;
    k_adjoint_fibers<<<cblocks, EMIT_WARPS * 32, 0, s>>>(r0, r1, np, offs, cnt, k0, keys0, V0, gm, gM, seg_grad, W0);
    k_adjoint_ctrl<<<grid_for((size_t)P, 256), 256, 0, s>>>(prims->fiber_offsets, F, fs, P, seg_grad, g.s,
                                                             (float4*)grad_ctrl);
    if (grad_weights) k_adjoint_weights<<<grid_for(np, 256), 256, 0, s>>>(seg_grad, np, grad_weights);
    NA_TRY(cudaGetLastError());
    return VX_OK;
}
