// vx_internal.cuh -- shared declarations of the CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/vx.h"

#define VX_CUDA_TRY(expr)                                                   \
    do {                                                                    \
        cudaError_t e_ = (expr);                                            \
        if (e_ != cudaSuccess) {                                            \
            vx_record_cuda_error(ctx, e_, #expr);                           \
            return VX_ERR_CUDA;                                             \
        }                                                                   \
    } while (0)

#define VX_TRY(expr)                    \
    do {                                \
        vx_status s_ = (expr);          \
        if (s_ != VX_OK) return s_;     \
    } while (0)

namespace vx {

constexpr int kWarp = 32;
constexpr int kSMs = 152;        // GB300: 152 SMs on two dies
constexpr int kMaxK = 8;         // lobe cap
constexpr int kMaxCand = 8 * kMaxK;

struct Buf {
    void* p = nullptr;
    size_t cap = 0;
};

}  // namespace vx

// Pipeline stages (for launch counts and optional event timing).
enum VxStage {
    ST_PREP = 0, ST_COUNT, ST_EMIT, ST_SCAN, ST_SORT_HIST, ST_SORT_SCATTER, ST_HEADS,
    ST_REDUCE_FIBERS, ST_REDUCE_TRIS, ST_FINALIZE, ST_LOD_COUNTS, ST_LOD_HEADS, ST_LOD_REDUCE,
    ST_SGGX_CLUSTER, ST_BATCH, ST_READBACK, ST_NSTAGES
};
extern const char* const kStageNames[ST_NSTAGES];

namespace vx {
constexpr int kEventPool = 4096;
struct EventRec {
    int stage;
    cudaEvent_t a, b;
};
}  // namespace vx

struct vx_context {
    vx_allocator alloc;
    bool own_alloc;               // NULL allocator given: cudaMallocAsync
    cudaStream_t last_stream = nullptr;
    char last_err[256] = {0};
    // workspace slots (grow-only)
    vx::Buf ws[32];
    uint64_t* host_pin = nullptr; // pinned readback buffer (64 words), mapped
    uint64_t* host_pin_dev = nullptr;   // its device address
    // hit ballots stored by the last candidate count pass: the buffer (NULL: none stored),
    // its primitive count and window (lo xyz, hi xyz); an emit pass uses them only on a match
    uint32_t* ballots = nullptr;
    uint32_t ballots_np = 0;
    int ballots_win[6] = {0, 0, 0, 0, 0, 0};
    // profiling
    bool prof = false;
    int64_t launches[ST_NSTAGES] = {0};
    double stage_ms[ST_NSTAGES] = {0};
    int64_t units[ST_NSTAGES] = {0};
    unsigned long long* dev_lobe_count = nullptr;   // device counter of lobe samplings
    int64_t max_pairs = 0x7fffffffll;  // candidate pairs per voxelization pass (window)
    vx::EventRec* ev = nullptr;   // pool of kEventPool records
    int nev = 0;
};

// Brackets one kernel launch: counts it and, with profiling on, records events.
void vx_stage_begin(vx_context* ctx, int stage, cudaStream_t s);
void vx_stage_end(vx_context* ctx, cudaStream_t s);
inline void vx_stage_units(vx_context* ctx, int stage, int64_t n) { ctx->units[stage] += n; }
#define VX_LAUNCH(ctx, stage, s, ...)          \
    do {                                       \
        vx_stage_begin((ctx), (stage), (s));   \
        __VA_ARGS__;                           \
        vx_stage_end((ctx), (s));              \
    } while (0)

enum WsSlot {
    WS_REC_A = 0, WS_REC_B, WS_REC_C, WS_COUNT, WS_OFFS, WS_SCAN_TMP,
    WS_KEYS0, WS_VALS0, WS_KEYS1, WS_VALS1, WS_SORT_HIST,
    WS_FLAGS, WS_SEGIDX, WS_STARTS, WS_SEG_OUT, WS_MISC, WS_FIBER_START,
    WS_LOD_FLAGS, WS_LOD_IDX, WS_LOD_STARTS, WS_LOD_WORK, WS_LOD_TMP, WS_LOD_STATS0, WS_LOD_STATS1, WS_BALLOTS,
    WS_NSLOTS
};
static_assert(WS_NSLOTS <= 32, "workspace slot table");

void vx_record_cuda_error(vx_context* ctx, cudaError_t e, const char* what);
// Copies `bytes` (a multiple of 4; src 4-byte aligned) of device memory into the context's
// pinned readback buffer at byte offset `off` (off + bytes <= 512), with a one-block kernel
// that stores into the mapped buffer.  No copy engine is involved, so the readback does not
// queue behind the caller's large transfers on other streams.  The buffer holds the values
// once `s` is synchronised.
vx_status vx_readback_async(vx_context* ctx, size_t off, const void* src, size_t bytes, cudaStream_t s);
vx_status vx_ws_ensure(vx_context* ctx, int slot, size_t bytes, cudaStream_t s);
void* vx_dev_alloc(vx_context* ctx, size_t bytes, cudaStream_t s);
void vx_dev_free(vx_context* ctx, void* p, cudaStream_t s);

// ---- scan / sort primitives (vx_sort.cu) -----------------------------------
// Exclusive prefix sum of n uint32 values; out may alias in.  total (device, may be
// NULL) receives the sum.  Needs scan workspace slot WS_SCAN_TMP.
vx_status vx_scan_u32(vx_context* ctx, const uint32_t* in, uint32_t* out, uint32_t n,
                      uint32_t* total, cudaStream_t s);
// Stable LSD radix sort of (key, value) uint32 pairs on the low `bits` bits.  The
// function ping-pongs between the two buffer pairs and leaves *keys / *vals pointing
// at the sorted data.  err (device): bit 4 is set when a bounded wait of the scatter's
// copy pipeline gave up (the result is then incomplete; report VX_ERR_TIMEOUT).
vx_status vx_radix_sort_u32(vx_context* ctx, uint32_t** keys, uint32_t** vals, uint32_t** keys_alt,
                            uint32_t** vals_alt, uint32_t n, int bits, cudaStream_t s, uint32_t* err);

// Starts of the runs of equal keys in the sorted keys[0, n): starts[r] = first index of run
// r, starts[*nseg] = n; *nseg (device) receives the number of runs.  starts needs room for
// the number of runs + 1 words.  Uses scan workspace slot WS_SCAN_TMP.
vx_status vx_segment_starts(vx_context* ctx, const uint32_t* keys, uint32_t n, uint32_t* nseg, uint32_t* starts,
                            cudaStream_t s);

// Exclusive prefix sum with caller-provided partials (>= ceil(n / 2048) words).
cudaError_t vx_scan_u32_scratch(const uint32_t* in, uint32_t* out, uint32_t n, uint32_t* total,
                                uint32_t* partials, cudaStream_t s);

// Stable LSD radix sort with caller-provided scratch (graph-capturable); optional final
// pass on the digit lut[value] (255 for the padding value 0xffffffff).
cudaError_t vx_radix_sort_u32_scratch(uint32_t** keys, uint32_t** vals, uint32_t** keys_alt, uint32_t** vals_alt,
                                      uint32_t n, int bits, const uint8_t* lut, uint32_t* hist,
                                      uint32_t* partials, cudaStream_t s);

// One batched LoD step (K = 1) with device-side counts (vx_lod.cu); see its definition.
cudaError_t vx_lod_step_batched(const vx_level* in, const uint16_t* inst_in, const uint32_t* n_dev, uint32_t cap_in,
                                vx_level* out, uint16_t* inst_out, uint32_t* np_dev, uint32_t cap_out,
                                uint32_t* flags, uint32_t* idx, uint32_t* starts, uint32_t* partials, uint32_t* tmp,
                                uint32_t* err, const float4* dirs4, int n_dirs, uint32_t* work, uint32_t* wcnt,
                                const void* cst, void* pst, int merge, int tier, cudaStream_t s);
// The clustering of a batched LoD step again, alone, with a given tier (0 warp per parent,
// 1 block of 8 warps, 2 block of 16 warps): for timing the tiers while a batch is planned.
cudaError_t vx_lod_cluster_batched(const vx_level* in, const vx_level* out, const uint32_t* starts,
                                   const uint32_t* work, uint32_t* wcnt, const float4* dirs4, int n_dirs,
                                   const void* cst, void* pst, uint32_t cap_out, int merge, int tier,
                                   cudaStream_t s);
cudaError_t vx_lod_batched_prepare(int K, const float* dirs, int n, float4* dirs4, cudaStream_t s);
constexpr size_t kLobeStatsBytes = 48;   // per-lobe histogram + sample moment kept between levels
// Direction table of the lobe sampling: n float4 directions, then the whole pairs of them
// ({x0, x1, y0, y1}, {z0, z1, 0, 0} for directions 2j, 2j + 1) for the packed FP32 loop.
inline size_t vx_dirs_bytes(int n) { return (size_t)n * 16 + (size_t)(n / 2) * 32; }

// ---- Morton ------------------------------------------------------------------
__host__ __device__ inline uint32_t vx_part1by2(uint32_t x) {
    x &= 0x000003ffu;
    x = (x | (x << 16)) & 0xff0000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}
__host__ __device__ inline uint32_t vx_compact1by2(uint32_t x) {
    x &= 0x09249249u;
    x = (x | (x >> 2)) & 0x030c30c3u;
    x = (x | (x >> 4)) & 0x0300f00fu;
    x = (x | (x >> 8)) & 0xff0000ffu;
    x = (x | (x >> 16)) & 0x000003ffu;
    return x;
}
__host__ __device__ inline uint32_t vx_morton3(uint32_t x, uint32_t y, uint32_t z) {
    return vx_part1by2(x) | (vx_part1by2(y) << 1) | (vx_part1by2(z) << 2);
}
// 64-bit Morton key of coordinates below 2^21 (host and device)
__host__ __device__ inline uint64_t vx_morton3_64(uint32_t x, uint32_t y, uint32_t z) {
    uint64_t k = 0;
    for (int b = 0; b < 21; ++b)
        k |= ((uint64_t)((x >> b) & 1u) << (3 * b)) | ((uint64_t)((y >> b) & 1u) << (3 * b + 1)) |
             ((uint64_t)((z >> b) & 1u) << (3 * b + 2));
    return k;
}

// ---- level layout --------------------------------------------------------------
// Byte offsets of each array inside one level block (256-byte aligned sections).
struct LevelLayout {
    size_t keys, mask, mass, moment, occ, proj, lobe_count, lobes, compact, total;
};
inline size_t vx_align256(size_t x) { return (x + 255) & ~size_t(255); }
inline LevelLayout vx_level_layout(int64_t n, int K) {
    LevelLayout L;
    size_t o = 0;
    size_t nn = (size_t)n;
    L.keys = o; o += vx_align256(nn * 8);
    L.mask = o; o += vx_align256(nn * 64);
    L.mass = o; o += vx_align256(nn * 4);
    L.moment = o; o += vx_align256(nn * 24);
    L.occ = o; o += vx_align256(nn * 2);
    L.proj = o; o += vx_align256(nn * 3);
    L.lobe_count = o; o += vx_align256(nn);
    L.lobes = o; o += vx_align256(nn * (size_t)K * 28);
    L.compact = o; o += vx_align256(nn * (size_t)K * 24);
    L.total = o;
    return L;
}
vx_status vx_level_alloc(vx_context* ctx, vx_level* L, int64_t n, int K, int level, int res,
                         cudaStream_t s);
