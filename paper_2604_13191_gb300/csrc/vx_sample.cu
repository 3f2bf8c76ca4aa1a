// vx_sample.cu -- sample-based voxelization of fiber segments: the paper's vertex-map
// sampling (Sec. 3.2-3.3: equally spaced samples along t, gathered per voxel) as a second
// workload, to compare occupancy and mass with the exact path of vx_voxelize.
//
// Segment p (grid units A, B, radius r, weight w) gives S samples on its axis at
// t_j = (j + 1/2) / S.  A sample at u = A + t_j (B - A) marks the sub-cell
// floor(8 (u - floor(u))) of voxel floor(u) (dropped outside [0, R)^3) and adds
// c = (w pi r^2 |B - A|) / S and c T(t) to that voxel; a voxel's sums run in sample order
// (p S + j ascending), FP32 in the order written here.
#include <math.h>

#include "vx_internal.cuh"
#include "vx_level0.cuh"

namespace {

// per sample id q = p S + j: the key of its voxel (1 << kbits when outside the grid)
__global__ void k_sample_keys(const float4* __restrict__ ra, const float4* __restrict__ rb, uint32_t n, int S,
                              int R, int kbits, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const uint32_t p = q / (uint32_t)S;
    const int j = (int)(q - p * (uint32_t)S);
    const float4 A = ra[p], B = rb[p];
    const float tj = ((float)j + 0.5f) / (float)S;
    const float u[3] = {A.x + tj * (B.x - A.x), A.y + tj * (B.y - A.y), A.z + tj * (B.z - A.z)};
    bool inside = true;
    uint32_t v[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (!(u[i] >= 0.0f) || !(u[i] < (float)R)) inside = false;
        v[i] = inside ? (uint32_t)floorf(u[i]) : 0u;
    }
    keys[q] = inside ? vx_morton3(v[0], v[1], v[2]) : (1u << kbits);
    vals[q] = q;
}

// thread per voxel (a run of equal keys): mask, sums in sample order, occupancy, K = 1 lobe
__global__ void k_sample_reduce(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                                const uint32_t* __restrict__ starts, uint32_t nvox, const float4* __restrict__ ra,
                                const float4* __restrict__ rb, int S, vx_level out) {
    const uint32_t vx_i = blockIdx.x * blockDim.x + threadIdx.x;
    if (vx_i >= nvox) return;
    const uint32_t beg = starts[vx_i], end = starts[vx_i + 1];
    uint64_t mk[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    float m = 0.0f;
    float M[6] = {0, 0, 0, 0, 0, 0};
    for (uint32_t i = beg; i < end; ++i) {
        const uint32_t q = vals[i];
        const uint32_t p = q / (uint32_t)S;
        const int j = (int)(q - p * (uint32_t)S);
        const float4 A = ra[p], B = rb[p];
        const float d[3] = {B.x - A.x, B.y - A.y, B.z - A.z};
        const float tj = ((float)j + 0.5f) / (float)S;
        const float u[3] = {A.x + tj * d[0], A.y + tj * d[1], A.z + tj * d[2]};
        int sc[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int c = (int)((u[k] - floorf(u[k])) * 8.0f);
            sc[k] = c > 7 ? 7 : c;
        }
        mk[sc[2]] |= 1ull << (sc[0] + 8 * sc[1]);
        const float dn = sqrtf((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
        float t[3] = {0.0f, 0.0f, 0.0f};
        if (dn > 0.0f) { t[0] = d[0] / dn; t[1] = d[1] / dn; t[2] = d[2] / dn; }
        const float mu = (kPi * (A.w * A.w)) * dn;
        const float c = (B.w * mu) / (float)S;
        m = m + c;
        M[0] = M[0] + c * (t[0] * t[0]);
        M[1] = M[1] + c * (t[1] * t[1]);
        M[2] = M[2] + c * (t[2] * t[2]);
        M[3] = M[3] + c * (t[0] * t[1]);
        M[4] = M[4] + c * (t[0] * t[2]);
        M[5] = M[5] + c * (t[1] * t[2]);
    }
    out.keys[vx_i] = (uint64_t)keys[beg];
#pragma unroll
    for (int w = 0; w < 8; ++w) out.mask[(size_t)vx_i * 8 + w] = mk[w];
    out.mass[vx_i] = m;
#pragma unroll
    for (int k = 0; k < 6; ++k) out.moment[(size_t)vx_i * 6 + k] = M[k];
    uint16_t occ;
    uint8_t pj[3];
    mask_counts(mk, occ, pj);
    out.occ[vx_i] = occ;
    out.occ_proj[(size_t)vx_i * 3 + 0] = pj[0];
    out.occ_proj[(size_t)vx_i * 3 + 1] = pj[1];
    out.occ_proj[(size_t)vx_i * 3 + 2] = pj[2];
    write_lobe(m, M, out.lobes + (size_t)vx_i * 7, out.compact + (size_t)vx_i * 6, out.lobe_count + vx_i);
}

}  // namespace

extern "C" vx_status vx_voxelize_sampled(vx_context* ctx, const vx_primitives* prims, const vx_grid* grid,
                                         int samples_per_segment, void* stream, vx_level* out0) {
    if (!ctx || !prims || !grid || !out0) return VX_ERR_INVALID_ARG;
    memset(out0, 0, sizeof(*out0));
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    const uint32_t R = grid->resolution;
    if (R == 0 || (R & (R - 1)) != 0) return VX_ERR_INVALID_ARG;
    if (prims->kind != VX_FIBERS || R > 1024 || grid->sub_res != 8) return VX_ERR_UNSUPPORTED;
    if (!(grid->voxel_size > 0.0f) || !isfinite(grid->voxel_size) || samples_per_segment < 1)
        return VX_ERR_INVALID_ARG;
    const int S = samples_per_segment;
    if (prims->num_prims < 0 || (uint64_t)prims->num_prims * (uint64_t)S >= 0x7fffffffull) return VX_ERR_CAPACITY;
    const uint32_t np = (uint32_t)prims->num_prims;
    int bits_R = 0;
    while ((1u << bits_R) < R) ++bits_R;
    if (np == 0) return vx_level_alloc(ctx, out0, 0, 1, 0, (int)R, s);
    if (!prims->ctrl || !prims->fiber_offsets || prims->num_fibers <= 0 || prims->num_fibers > 0x7fffffff)
        return VX_ERR_INVALID_ARG;
    if (((uintptr_t)prims->ctrl & 15) != 0) return VX_ERR_INVALID_ARG;
    GridDev g;
    g.o[0] = grid->origin[0]; g.o[1] = grid->origin[1]; g.o[2] = grid->origin[2];
    g.s = 1.0f / grid->voxel_size;
    g.R = (int)R;

    // ---- prep: grid-unit segment records (as vx_voxelize) ------------------------------
    VX_TRY(vx_ws_ensure(ctx, WS_REC_A, (size_t)np * 16, s));
    VX_TRY(vx_ws_ensure(ctx, WS_REC_B, (size_t)np * 16, s));
    VX_TRY(vx_ws_ensure(ctx, WS_MISC, 256, s));
    uint32_t* misc = (uint32_t*)ctx->ws[WS_MISC].p;   // [0] err, [2] runs, [4] segment total
    VX_CUDA_TRY(cudaMemsetAsync(misc, 0, 64, s));
    float4* ra = (float4*)ctx->ws[WS_REC_A].p;
    float4* rb = (float4*)ctx->ws[WS_REC_B].p;
    const int64_t F = prims->num_fibers;
    VX_TRY(vx_ws_ensure(ctx, WS_FIBER_START, (size_t)F * 4 + 256, s));
    uint32_t* fs = (uint32_t*)ctx->ws[WS_FIBER_START].p;
    VX_LAUNCH(ctx, ST_PREP, s, k_fiber_seg_counts<<<grid_for((size_t)F, 256), 256, 0, s>>>(prims->fiber_offsets, F, fs));
    VX_TRY(vx_scan_u32(ctx, fs, fs, (uint32_t)F, misc + 4, s));
    VX_LAUNCH(ctx, ST_PREP, s, k_prep_fibers<<<grid_for(np, 256), 256, 0, s>>>((const float4*)prims->ctrl,
                                                     prims->fiber_offsets, fs, F, misc + 4, prims->weights, np, g,
                                                     ra, rb, misc));
    VX_CUDA_TRY(cudaGetLastError());

    // ---- samples keyed by voxel, sorted (stable: sample order within a voxel) ----------
    const uint32_t n = np * (uint32_t)S;
    const int kbits = 3 * bits_R;
    VX_TRY(vx_ws_ensure(ctx, WS_KEYS0, (size_t)n * 4, s));
    VX_TRY(vx_ws_ensure(ctx, WS_VALS0, (size_t)n * 4, s));
    VX_TRY(vx_ws_ensure(ctx, WS_KEYS1, (size_t)n * 4, s));
    VX_TRY(vx_ws_ensure(ctx, WS_VALS1, (size_t)n * 4, s));
    uint32_t* k0 = (uint32_t*)ctx->ws[WS_KEYS0].p;
    uint32_t* v0 = (uint32_t*)ctx->ws[WS_VALS0].p;
    uint32_t* k1 = (uint32_t*)ctx->ws[WS_KEYS1].p;
    uint32_t* v1 = (uint32_t*)ctx->ws[WS_VALS1].p;
    VX_LAUNCH(ctx, ST_EMIT, s, k_sample_keys<<<grid_for(n, 256), 256, 0, s>>>(ra, rb, n, S, (int)R, kbits, k0, v0));
    VX_CUDA_TRY(cudaGetLastError());
    VX_TRY(vx_radix_sort_u32(ctx, &k0, &v0, &k1, &v1, n, kbits + 1, s));
    VX_TRY(vx_ws_ensure(ctx, WS_STARTS, (size_t)n * 4 + 8, s));
    uint32_t* starts = (uint32_t*)ctx->ws[WS_STARTS].p;
    VX_TRY(vx_segment_starts(ctx, k0, n, misc + 2, starts, s));
    VX_CUDA_TRY(cudaMemcpyAsync(ctx->host_pin, misc, 16, cudaMemcpyDeviceToHost, s));
    VX_CUDA_TRY(cudaMemcpyAsync((uint32_t*)ctx->host_pin + 4, k0 + (n - 1), 4, cudaMemcpyDeviceToHost, s));
    VX_CUDA_TRY(cudaStreamSynchronize(s));
    const uint32_t* hp = (const uint32_t*)ctx->host_pin;
    if (hp[0]) return VX_ERR_INVALID_ARG;
    // the run of samples outside the grid (key 1 << kbits) sorts last and is not a voxel
    const uint32_t nvox = hp[2] - (hp[4] == (1u << kbits) ? 1u : 0u);
    VX_TRY(vx_level_alloc(ctx, out0, nvox, 1, 0, (int)R, s));
    if (nvox > 0)
        VX_LAUNCH(ctx, ST_FINALIZE, s, k_sample_reduce<<<grid_for(nvox, 128), 128, 0, s>>>(k0, v0, starts, nvox, ra, rb,
                                                                                           S, *out0));
    VX_CUDA_TRY(cudaGetLastError());
    return VX_OK;
}
