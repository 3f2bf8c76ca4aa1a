// vx_sample.cu -- sample-based voxelization: the paper's vertex-map sampling (Sec. 3.2-3.3:
// samples generated from kernel indices, gathered per voxel) as a second workload, to compare
// occupancy and mass with the exact path of vx_voxelize.
//
// Fibers: segment p (grid units A, B, radius r, weight w) gives S samples on its axis at
// t_j = (j + 1/2) / S, each carrying c = (w pi r^2 |B - A|) / S.
// Triangles: triangle p (U0, U1, U2, weight w, area a) gives M_p = max(1, ceil(S a / a_max))
// samples (a_max the largest area: counts follow the area relative to the biggest triangle).
// Sample j takes the lattice point (x, y) = ((j + 1/2) / M_p, frac((j + 1/2) g)),
// g = 0.6180339887, through the square-to-triangle map of Heitz (2019): y > x gives
// b0 = x / 2, b1 = y - b0, else b1 = y / 2, b0 = x - b1; the point is
// (b0 U0 + b1 U1) + (1 - b0 - b1) U2, carrying c = (w a) / M_p.
// A sample at u marks the sub-cell floor(8 (u - floor(u))) of voxel floor(u) (dropped outside
// [0, R)^3) and adds c and c T(d) (d the unit tangent or normal) to that voxel; a voxel's
// sums run in sample order (p, then j), FP32 in the order written here.
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

// ---- triangles -------------------------------------------------------------------------
__device__ __forceinline__ void tri_frame(const float4& a, const float4& b, const float4& c, float* t, float& area) {
    const float f0[3] = {b.x - a.x, b.y - a.y, b.z - a.z};
    const float f1[3] = {c.x - b.x, c.y - b.y, c.z - b.z};
    const float n0 = f0[1] * f1[2] - f0[2] * f1[1];
    const float n1 = f0[2] * f1[0] - f0[0] * f1[2];
    const float n2 = f0[0] * f1[1] - f0[1] * f1[0];
    const float nn = sqrtf((n0 * n0 + n1 * n1) + n2 * n2);
    t[0] = t[1] = t[2] = 0.0f;
    if (nn > 0.0f) { t[0] = n0 / nn; t[1] = n1 / nn; t[2] = n2 / nn; }
    area = 0.5f * nn;
}

__global__ void k_tri_area_max(const float4* __restrict__ r0, const float4* __restrict__ r1,
                               const float4* __restrict__ r2, uint32_t np, uint32_t* __restrict__ amax_bits) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    float t[3], a;
    tri_frame(r0[p], r1[p], r2[p], t, a);
    atomicMax(amax_bits, __float_as_uint(a));   // areas are >= 0: ordered as unsigned
}

__device__ __forceinline__ uint32_t tri_sample_count(float a, float amax, int S) {
    if (!(amax > 0.0f)) return 1u;
    const float x = (float)S * (a / amax);
    const uint32_t m = (uint32_t)ceilf(x);
    return m < 1u ? 1u : (m > (uint32_t)S ? (uint32_t)S : m);
}

__global__ void k_tri_sample_counts(const float4* __restrict__ r0, const float4* __restrict__ r1,
                                    const float4* __restrict__ r2, uint32_t np, int S,
                                    const uint32_t* __restrict__ amax_bits, uint32_t* __restrict__ cnt) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    float t[3], a;
    tri_frame(r0[p], r1[p], r2[p], t, a);
    cnt[p] = tri_sample_count(a, __uint_as_float(*amax_bits), S);
}

__device__ __forceinline__ void tri_sample_point(const float4& a, const float4& b, const float4& c, uint32_t j,
                                                 uint32_t m, float* u) {
    const float x = ((float)j + 0.5f) / (float)m;
    const float yy = ((float)j + 0.5f) * 0.6180339887f;
    const float y = yy - floorf(yy);
    float b0, b1;
    if (y > x) { b0 = x * 0.5f; b1 = y - b0; } else { b1 = y * 0.5f; b0 = x - b1; }
    const float b2 = (1.0f - b0) - b1;
    u[0] = (b0 * a.x + b1 * b.x) + b2 * c.x;
    u[1] = (b0 * a.y + b1 * b.y) + b2 * c.y;
    u[2] = (b0 * a.z + b1 * b.z) + b2 * c.z;
}

// thread per triangle: its samples' keys at offs[p] + j, values p S + j
__global__ void k_tri_sample_keys(const float4* __restrict__ r0, const float4* __restrict__ r1,
                                  const float4* __restrict__ r2, uint32_t np, int S, int R, int kbits,
                                  const uint32_t* __restrict__ cnt, const uint32_t* __restrict__ offs,
                                  uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const float4 a = r0[p], b = r1[p], c = r2[p];
    const uint32_t m = cnt[p], o = offs[p];
    for (uint32_t j = 0; j < m; ++j) {
        float u[3];
        tri_sample_point(a, b, c, j, m, u);
        bool inside = true;
        uint32_t v[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (!(u[i] >= 0.0f) || !(u[i] < (float)R)) inside = false;
            v[i] = inside ? (uint32_t)floorf(u[i]) : 0u;
        }
        keys[o + j] = inside ? vx_morton3(v[0], v[1], v[2]) : (1u << kbits);
        vals[o + j] = p * (uint32_t)S + j;
    }
}

__global__ void k_tri_sample_reduce(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                                    const uint32_t* __restrict__ starts, uint32_t nvox, const float4* __restrict__ r0,
                                    const float4* __restrict__ r1, const float4* __restrict__ r2,
                                    const uint32_t* __restrict__ cnt, int S, vx_level out) {
    const uint32_t vi = blockIdx.x * blockDim.x + threadIdx.x;
    if (vi >= nvox) return;
    const uint32_t beg = starts[vi], end = starts[vi + 1];
    uint64_t mk[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    float m = 0.0f;
    float M[6] = {0, 0, 0, 0, 0, 0};
    for (uint32_t i = beg; i < end; ++i) {
        const uint32_t q = vals[i];
        const uint32_t p = q / (uint32_t)S;
        const uint32_t j = q - p * (uint32_t)S;
        const float4 a = r0[p], b = r1[p], c = r2[p];
        float u[3], t[3], area;
        const uint32_t mp = cnt[p];
        tri_sample_point(a, b, c, j, mp, u);
        tri_frame(a, b, c, t, area);
        int sc[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int s8 = (int)((u[k] - floorf(u[k])) * 8.0f);
            sc[k] = s8 > 7 ? 7 : s8;
        }
        mk[sc[2]] |= 1ull << (sc[0] + 8 * sc[1]);
        const float cc = (a.w * area) / (float)mp;
        m = m + cc;
        M[0] = M[0] + cc * (t[0] * t[0]);
        M[1] = M[1] + cc * (t[1] * t[1]);
        M[2] = M[2] + cc * (t[2] * t[2]);
        M[3] = M[3] + cc * (t[0] * t[1]);
        M[4] = M[4] + cc * (t[0] * t[2]);
        M[5] = M[5] + cc * (t[1] * t[2]);
    }
    out.keys[vi] = (uint64_t)keys[beg];
#pragma unroll
    for (int w = 0; w < 8; ++w) out.mask[(size_t)vi * 8 + w] = mk[w];
    out.mass[vi] = m;
#pragma unroll
    for (int k = 0; k < 6; ++k) out.moment[(size_t)vi * 6 + k] = M[k];
    uint16_t occ;
    uint8_t pj[3];
    mask_counts(mk, occ, pj);
    out.occ[vi] = occ;
    out.occ_proj[(size_t)vi * 3 + 0] = pj[0];
    out.occ_proj[(size_t)vi * 3 + 1] = pj[1];
    out.occ_proj[(size_t)vi * 3 + 2] = pj[2];
    write_lobe(m, M, out.lobes + (size_t)vi * 7, out.compact + (size_t)vi * 6, out.lobe_count + vi);
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
    const bool fiber = prims->kind == VX_FIBERS;
    if (!fiber && prims->kind != VX_TRIANGLES) return VX_ERR_INVALID_ARG;
    if (R > 1024 || grid->sub_res != 8) return VX_ERR_UNSUPPORTED;
    if (!(grid->voxel_size > 0.0f) || !isfinite(grid->voxel_size) || samples_per_segment < 1)
        return VX_ERR_INVALID_ARG;
    const int S = samples_per_segment;
    if (prims->num_prims < 0 || (uint64_t)prims->num_prims * (uint64_t)S >= 0x7fffffffull) return VX_ERR_CAPACITY;
    const uint32_t np = (uint32_t)prims->num_prims;
    int bits_R = 0;
    while ((1u << bits_R) < R) ++bits_R;
    if (np == 0) return vx_level_alloc(ctx, out0, 0, 1, 0, (int)R, s);
    if (fiber) {
        if (!prims->ctrl || !prims->fiber_offsets || prims->num_fibers <= 0 || prims->num_fibers > 0x7fffffff)
            return VX_ERR_INVALID_ARG;
        if (((uintptr_t)prims->ctrl & 15) != 0) return VX_ERR_INVALID_ARG;
    } else {
        if (!prims->tri_verts || ((uintptr_t)prims->tri_verts & 15) != 0) return VX_ERR_INVALID_ARG;
    }
    GridDev g;
    g.o[0] = grid->origin[0]; g.o[1] = grid->origin[1]; g.o[2] = grid->origin[2];
    g.s = 1.0f / grid->voxel_size;
    g.R = (int)R;

    // ---- prep: grid-unit records (as vx_voxelize) ----------------------------------------
    VX_TRY(vx_ws_ensure(ctx, WS_REC_A, (size_t)np * 16, s));
    VX_TRY(vx_ws_ensure(ctx, WS_REC_B, (size_t)np * 16, s));
    if (!fiber) VX_TRY(vx_ws_ensure(ctx, WS_REC_C, (size_t)np * 16, s));
    VX_TRY(vx_ws_ensure(ctx, WS_MISC, 256, s));
    uint32_t* misc = (uint32_t*)ctx->ws[WS_MISC].p;   // [0] err, [1] samples, [2] runs, [3] area max, [4] segments
    VX_CUDA_TRY(cudaMemsetAsync(misc, 0, 64, s));
    float4* r0 = (float4*)ctx->ws[WS_REC_A].p;
    float4* r1 = (float4*)ctx->ws[WS_REC_B].p;
    float4* r2 = fiber ? nullptr : (float4*)ctx->ws[WS_REC_C].p;
    uint32_t* cnt = nullptr;
    uint32_t n = 0;
    if (fiber) {
        const int64_t F = prims->num_fibers;
        VX_TRY(vx_ws_ensure(ctx, WS_FIBER_START, (size_t)F * 4 + 256, s));
        uint32_t* fs = (uint32_t*)ctx->ws[WS_FIBER_START].p;
        VX_LAUNCH(ctx, ST_PREP, s, k_fiber_seg_counts<<<grid_for((size_t)F, 256), 256, 0, s>>>(prims->fiber_offsets, F,
                                                                                              prims->num_ctrl, fs, misc));
        VX_TRY(vx_scan_u32(ctx, fs, fs, (uint32_t)F, misc + 4, s));
        VX_LAUNCH(ctx, ST_PREP, s, k_prep_fibers<<<grid_for(np, 256), 256, 0, s>>>((const float4*)prims->ctrl, prims->num_ctrl,
                                                         prims->fiber_offsets, fs, F, misc + 4, prims->weights, np, g,
                                                         r0, r1, misc));
        n = np * (uint32_t)S;
    } else {
        VX_LAUNCH(ctx, ST_PREP, s, k_prep_tris<<<grid_for(np, 256), 256, 0, s>>>((const float4*)prims->tri_verts,
                                                       prims->weights, np, g, r0, r1, r2, misc));
        VX_TRY(vx_ws_ensure(ctx, WS_COUNT, (size_t)np * 4, s));
        VX_TRY(vx_ws_ensure(ctx, WS_OFFS, (size_t)np * 4, s));
        cnt = (uint32_t*)ctx->ws[WS_COUNT].p;
        uint32_t* offs = (uint32_t*)ctx->ws[WS_OFFS].p;
        VX_LAUNCH(ctx, ST_PREP, s, k_tri_area_max<<<grid_for(np, 256), 256, 0, s>>>(r0, r1, r2, np, misc + 3));
        VX_LAUNCH(ctx, ST_PREP, s, k_tri_sample_counts<<<grid_for(np, 256), 256, 0, s>>>(r0, r1, r2, np, S, misc + 3,
                                                                                         cnt));
        VX_TRY(vx_scan_u32(ctx, cnt, offs, np, misc + 1, s));
        VX_TRY(vx_readback_async(ctx, 0, misc, 8, s));
        VX_CUDA_TRY(cudaStreamSynchronize(s));
        if (((const uint32_t*)ctx->host_pin)[0]) return VX_ERR_INVALID_ARG;
        n = ((const uint32_t*)ctx->host_pin)[1];
        if (n == 0) return vx_level_alloc(ctx, out0, 0, 1, 0, (int)R, s);   // no sample lands anywhere
    }
    VX_CUDA_TRY(cudaGetLastError());

    // ---- samples keyed by voxel, sorted (stable: sample order within a voxel) ----------
    const int kbits = 3 * bits_R;
    VX_TRY(vx_ws_ensure(ctx, WS_KEYS0, (size_t)n * 4, s));
    VX_TRY(vx_ws_ensure(ctx, WS_VALS0, (size_t)n * 4, s));
    VX_TRY(vx_ws_ensure(ctx, WS_KEYS1, (size_t)n * 4, s));
    VX_TRY(vx_ws_ensure(ctx, WS_VALS1, (size_t)n * 4, s));
    uint32_t* k0 = (uint32_t*)ctx->ws[WS_KEYS0].p;
    uint32_t* v0 = (uint32_t*)ctx->ws[WS_VALS0].p;
    uint32_t* k1 = (uint32_t*)ctx->ws[WS_KEYS1].p;
    uint32_t* v1 = (uint32_t*)ctx->ws[WS_VALS1].p;
    if (fiber)
        VX_LAUNCH(ctx, ST_EMIT, s, k_sample_keys<<<grid_for(n, 256), 256, 0, s>>>(r0, r1, n, S, (int)R, kbits, k0, v0));
    else
        VX_LAUNCH(ctx, ST_EMIT, s, k_tri_sample_keys<<<grid_for(np, 256), 256, 0, s>>>(
                                       r0, r1, r2, np, S, (int)R, kbits, cnt, (const uint32_t*)ctx->ws[WS_OFFS].p, k0,
                                       v0));
    VX_CUDA_TRY(cudaGetLastError());
    VX_TRY(vx_radix_sort_u32(ctx, &k0, &v0, &k1, &v1, n, kbits + 1, s, misc));
    VX_TRY(vx_ws_ensure(ctx, WS_STARTS, (size_t)n * 4 + 8, s));
    uint32_t* starts = (uint32_t*)ctx->ws[WS_STARTS].p;
    VX_TRY(vx_segment_starts(ctx, k0, n, misc + 2, starts, s));
    VX_TRY(vx_readback_async(ctx, 0, misc, 16, s));
    VX_TRY(vx_readback_async(ctx, 16, k0 + (n - 1), 4, s));
    VX_CUDA_TRY(cudaStreamSynchronize(s));
    const uint32_t* hp = (const uint32_t*)ctx->host_pin;
    if (hp[0] & 4u) return VX_ERR_TIMEOUT;   // a bounded wait of the sort gave up
    if (hp[0]) return VX_ERR_INVALID_ARG;
    // the run of samples outside the grid (key 1 << kbits) sorts last and is not a voxel
    const uint32_t nvox = hp[2] - (hp[4] == (1u << kbits) ? 1u : 0u);
    VX_TRY(vx_level_alloc(ctx, out0, nvox, 1, 0, (int)R, s));
    if (nvox > 0 && fiber)
        VX_LAUNCH(ctx, ST_FINALIZE, s, k_sample_reduce<<<grid_for(nvox, 128), 128, 0, s>>>(k0, v0, starts, nvox, r0, r1,
                                                                                           S, *out0));
    if (nvox > 0 && !fiber)
        VX_LAUNCH(ctx, ST_FINALIZE, s, k_tri_sample_reduce<<<grid_for(nvox, 128), 128, 0, s>>>(
                                           k0, v0, starts, nvox, r0, r1, r2, cnt, S, *out0));
    VX_CUDA_TRY(cudaGetLastError());
    return VX_OK;
}
