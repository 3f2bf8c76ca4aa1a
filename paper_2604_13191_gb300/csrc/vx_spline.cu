// vx_spline.cu -- Catmull-Rom spline fibers tessellated into capsule control points
// (Sec. 3.2: the spline through its stored nodes, sampled at equally spaced t), so that
// spline collections enter the capsule path of vx_voxelize as fibers.
//
// Spline f has nodes offsets[f] .. offsets[f+1]-1.  Span i joins nodes i and i+1 and uses
// P0..P3 = nodes i-1, i, i+1, i+2; past either end the missing node is the end node
// reflected through its neighbour (2 P_0 - P_1, 2 P_n-1 - P_n-2), so nodes on a line give
// points on it.  A span gives S points at t = j / S, j = 0..S-1, from the uniform form
//     C(t) = 0.5 (2 P1 + t (a + t (b + t c))),  a = P2 - P0,
//     b = ((2 P0 - 5 P1) + 4 P2) - P3,  c = ((3 P1 - P0) - 3 P2) + P3,
// and the radius linearly, r1 + t (r2 - r1); the spline's last node closes it.  FP32 in
// this order (the library is built without contraction).
#include "vx_internal.cuh"

namespace {

// Output offsets; the node offsets must run from 0 to num_nodes and increase strictly
// (every spline has a node), else the error flag is set and no node is read.
__global__ void k_spline_offsets(const int64_t* __restrict__ off, int64_t F, int64_t num_nodes, int S,
                                 int64_t* __restrict__ out_off, uint32_t* __restrict__ err) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f > F) return;
    out_off[f] = (off[f] - f) * S + f;
    if (f < F && off[f + 1] <= off[f]) atomicOr(err, 1u);
    if ((f == 0 && off[0] != 0) || (f == F && off[F] != num_nodes)) atomicOr(err, 1u);
}

__global__ void k_spline_points(const float4* __restrict__ nodes, const int64_t* __restrict__ off,
                                const int64_t* __restrict__ out_off, int64_t F, int S, int64_t total,
                                float4* __restrict__ out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= total) return;
    // spline of output point k: the last f with out_off[f] <= k
    int64_t lo = 0, hi = F;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (out_off[mid] <= k) lo = mid; else hi = mid;
    }
    const int64_t f = lo;
    const int64_t b = off[f], n = off[f + 1] - b;
    const int64_t l = k - out_off[f];
    const int64_t i = l / S;
    const int j = (int)(l - i * S);
    if (i >= n - 1) {                       // the closing node
        out[k] = nodes[b + n - 1];
        return;
    }
    const float4 P1 = nodes[b + i], P2 = nodes[b + i + 1];
    float4 P0, P3;
    if (i > 0) {
        P0 = nodes[b + i - 1];
    } else {
        P0 = make_float4(2.0f * P1.x - P2.x, 2.0f * P1.y - P2.y, 2.0f * P1.z - P2.z, 0.0f);
    }
    if (i + 2 < n) {
        P3 = nodes[b + i + 2];
    } else {
        P3 = make_float4(2.0f * P2.x - P1.x, 2.0f * P2.y - P1.y, 2.0f * P2.z - P1.z, 0.0f);
    }
    const float t = (float)j / (float)S;
    const float p0[3] = {P0.x, P0.y, P0.z}, p1[3] = {P1.x, P1.y, P1.z}, p2[3] = {P2.x, P2.y, P2.z},
                p3[3] = {P3.x, P3.y, P3.z};
    float q[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float a = p2[c] - p0[c];
        const float bb = ((2.0f * p0[c] - 5.0f * p1[c]) + 4.0f * p2[c]) - p3[c];
        const float cc = ((3.0f * p1[c] - p0[c]) - 3.0f * p2[c]) + p3[c];
        q[c] = 0.5f * (2.0f * p1[c] + t * (a + t * (bb + t * cc)));
    }
    out[k] = make_float4(q[0], q[1], q[2], P1.w + t * (P2.w - P1.w));
}

}  // namespace

vx_status vx_tessellate_catmull_rom(vx_context* ctx, const float* nodes, const int64_t* offsets, int64_t num_splines,
                                    int64_t num_nodes, int subdiv, float* out_ctrl, int64_t* out_offsets,
                                    void* stream) {
    if (!ctx || num_splines < 0 || num_nodes < 0 || subdiv < 1) return VX_ERR_INVALID_ARG;
    if (!offsets || !out_offsets) return VX_ERR_INVALID_ARG;
    if (num_splines > num_nodes) return VX_ERR_INVALID_ARG;   // every spline needs a node
    if (num_nodes > 0 && (!nodes || !out_ctrl)) return VX_ERR_INVALID_ARG;
    if (((uintptr_t)nodes | (uintptr_t)out_ctrl) & 15u) return VX_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    VX_TRY(vx_ws_ensure(ctx, WS_MISC, 256, s));
    uint32_t* err = (uint32_t*)ctx->ws[WS_MISC].p;
    VX_CUDA_TRY(cudaMemsetAsync(err, 0, 4, s));
    const int64_t F = num_splines;
    k_spline_offsets<<<(unsigned)((F + 1 + 255) / 256), 256, 0, s>>>(offsets, F, num_nodes, subdiv, out_offsets, err);
    VX_CUDA_TRY(cudaGetLastError());
    VX_TRY(vx_readback_async(ctx, 0, err, 4, s));
    VX_CUDA_TRY(cudaStreamSynchronize(s));
    if (((uint32_t*)ctx->host_pin)[0]) return VX_ERR_INVALID_ARG;
    const int64_t total = (num_nodes - F) * (int64_t)subdiv + F;
    if (total > 0)
        k_spline_points<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
            (const float4*)nodes, offsets, out_offsets, F, subdiv, total, (float4*)out_ctrl);
    VX_CUDA_TRY(cudaGetLastError());
    return VX_OK;
}
