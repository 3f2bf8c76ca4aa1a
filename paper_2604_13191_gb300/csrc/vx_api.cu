// vx_api.cu -- context, allocator plumbing and status strings of the C ABI.
#include <stdio.h>
#include <stdlib.h>

#include <new>

#include "vx_internal.cuh"

const char* const kStageNames[ST_NSTAGES] = {
    "prep", "candidates_count", "candidates_emit", "scan", "sort_hist", "sort_scatter", "segment_heads",
    "reduce_fibers", "reduce_tris", "finalize", "lod_counts", "lod_heads", "lod_reduce", "sggx_cluster",
    "batched_graph", "readback"};

namespace {
__global__ void k_readback(const uint32_t* __restrict__ src, uint32_t n, uint32_t* dst) {
    const uint32_t i = threadIdx.x;
    if (i < n) dst[i] = src[i];
}
}  // namespace

vx_status vx_readback_async(vx_context* ctx, size_t off, const void* src, size_t bytes, cudaStream_t s) {
    if ((bytes & 3) || (off & 3) || off + bytes > 64 * sizeof(uint64_t) || ((uintptr_t)src & 3) || !src)
        return VX_ERR_INVALID_ARG;
    const uint32_t n = (uint32_t)(bytes / 4);
    if (n == 0) return VX_OK;
    VX_LAUNCH(ctx, ST_READBACK, s,
              k_readback<<<1, 128, 0, s>>>((const uint32_t*)src, n,
                                           (uint32_t*)((char*)ctx->host_pin_dev + off)));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        vx_record_cuda_error(ctx, e, "k_readback");
        return VX_ERR_CUDA;
    }
    return VX_OK;
}

static void vx_prof_drain(vx_context* ctx) {
    for (int i = 0; i < ctx->nev; ++i) {
        float ms = 0.0f;
        if (cudaEventSynchronize(ctx->ev[i].b) == cudaSuccess &&
            cudaEventElapsedTime(&ms, ctx->ev[i].a, ctx->ev[i].b) == cudaSuccess)
            ctx->stage_ms[ctx->ev[i].stage] += ms;
    }
    ctx->nev = 0;
}

void vx_stage_begin(vx_context* ctx, int stage, cudaStream_t s) {
    ctx->launches[stage] += 1;
    if (!ctx->prof || !ctx->ev) return;
    if (ctx->nev == vx::kEventPool) vx_prof_drain(ctx);
    vx::EventRec& r = ctx->ev[ctx->nev];
    r.stage = stage;
    cudaEventRecord(r.a, s);
}

void vx_stage_end(vx_context* ctx, cudaStream_t s) {
    if (!ctx->prof || !ctx->ev) return;
    cudaEventRecord(ctx->ev[ctx->nev].b, s);
    ++ctx->nev;
}

void vx_record_cuda_error(vx_context* ctx, cudaError_t e, const char* what) {
    if (!ctx) return;
    snprintf(ctx->last_err, sizeof(ctx->last_err), "%s: %s", what, cudaGetErrorString(e));
}

void* vx_dev_alloc(vx_context* ctx, size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 256;
    if (ctx->own_alloc) {
        void* p = nullptr;
        cudaError_t e = cudaMallocAsync(&p, bytes, s);
        if (e != cudaSuccess) {
            vx_record_cuda_error(ctx, e, "cudaMallocAsync");
            return nullptr;
        }
        return p;
    }
    return ctx->alloc.alloc(ctx->alloc.ctx, bytes, (void*)s);
}

void vx_dev_free(vx_context* ctx, void* p, cudaStream_t s) {
    if (!p) return;
    if (ctx->own_alloc) {
        cudaFreeAsync(p, s);
        return;
    }
    ctx->alloc.free(ctx->alloc.ctx, p, (void*)s);
}

vx_status vx_ws_ensure(vx_context* ctx, int slot, size_t bytes, cudaStream_t s) {
    vx::Buf& b = ctx->ws[slot];
    if (b.cap >= bytes && b.p) return VX_OK;
    size_t want = bytes + bytes / 8 + 4096;   // a little headroom against regrowth
    void* p = vx_dev_alloc(ctx, want, s);
    if (!p) return VX_ERR_OUT_OF_MEMORY;
    if (b.p) vx_dev_free(ctx, b.p, s);
    b.p = p;
    b.cap = want;
    return VX_OK;
}

vx_status vx_level_alloc(vx_context* ctx, vx_level* L, int64_t n, int K, int level, int res,
                         cudaStream_t s) {
    memset(L, 0, sizeof(*L));
    LevelLayout lay = vx_level_layout(n, K);
    char* base = (char*)vx_dev_alloc(ctx, lay.total, s);
    if (!base) return VX_ERR_OUT_OF_MEMORY;
    L->level = level;
    L->resolution = res;
    L->num_voxels = n;
    L->K = K;
    L->block = base;
    L->keys = (uint64_t*)(base + lay.keys);
    L->mask = (uint64_t*)(base + lay.mask);
    L->mass = (float*)(base + lay.mass);
    L->moment = (float*)(base + lay.moment);
    L->occ = (uint16_t*)(base + lay.occ);
    L->occ_proj = (uint8_t*)(base + lay.proj);
    L->lobe_count = (uint8_t*)(base + lay.lobe_count);
    L->lobes = (float*)(base + lay.lobes);
    L->compact = (float*)(base + lay.compact);
    return VX_OK;
}

extern "C" {

vx_status vx_context_create(const vx_allocator* alloc, vx_context** out) {
    if (!out) return VX_ERR_INVALID_ARG;
    *out = nullptr;
    if (alloc && (!alloc->alloc || !alloc->free)) return VX_ERR_INVALID_ARG;
    vx_context* ctx = new (std::nothrow) vx_context();
    if (!ctx) return VX_ERR_OUT_OF_MEMORY;
    if (alloc) {
        ctx->alloc = *alloc;
        ctx->own_alloc = false;
    } else {
        memset(&ctx->alloc, 0, sizeof(ctx->alloc));
        ctx->own_alloc = true;
    }
    // the readback buffer is mapped: small results are stored into it by a kernel (see
    // vx_readback_async), not copied by a copy engine
    cudaError_t e = cudaHostAlloc((void**)&ctx->host_pin, 64 * sizeof(uint64_t), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&ctx->host_pin_dev, ctx->host_pin, 0);
    if (e != cudaSuccess) {
        vx_record_cuda_error(ctx, e, "cudaHostAlloc");
        if (ctx->host_pin) cudaFreeHost(ctx->host_pin);
        delete ctx;
        return VX_ERR_CUDA;
    }
    *out = ctx;
    return VX_OK;
}

void vx_context_destroy(vx_context* ctx) {
    if (!ctx) return;
    cudaStream_t s = ctx->last_stream;
    cudaStreamSynchronize(s);
    for (int i = 0; i < WS_NSLOTS; ++i) {
        if (ctx->ws[i].p) vx_dev_free(ctx, ctx->ws[i].p, s);
        ctx->ws[i].p = nullptr;
        ctx->ws[i].cap = 0;
    }
    cudaStreamSynchronize(s);
    if (ctx->host_pin) cudaFreeHost(ctx->host_pin);
    if (ctx->ev) {
        for (int i = 0; i < vx::kEventPool; ++i) {
            cudaEventDestroy(ctx->ev[i].a);
            cudaEventDestroy(ctx->ev[i].b);
        }
        delete[] ctx->ev;
    }
    if (ctx->dev_lobe_count) cudaFree(ctx->dev_lobe_count);
    delete ctx;
}

vx_status vx_set_max_pairs_per_pass(vx_context* ctx, int64_t max_pairs) {
    if (!ctx || max_pairs < 1) return VX_ERR_INVALID_ARG;
    ctx->max_pairs = max_pairs > 0x7fffffffll ? 0x7fffffffll : max_pairs;
    return VX_OK;
}

vx_status vx_profile_enable(vx_context* ctx, int enable) {
    if (!ctx) return VX_ERR_INVALID_ARG;
    if (enable && !ctx->ev) {
        ctx->ev = new (std::nothrow) vx::EventRec[vx::kEventPool];
        if (!ctx->ev) return VX_ERR_OUT_OF_MEMORY;
        for (int i = 0; i < vx::kEventPool; ++i) {
            cudaError_t e1 = cudaEventCreate(&ctx->ev[i].a);
            cudaError_t e2 = cudaEventCreate(&ctx->ev[i].b);
            if (e1 != cudaSuccess || e2 != cudaSuccess) {
                vx_record_cuda_error(ctx, e1 != cudaSuccess ? e1 : e2, "cudaEventCreate");
                return VX_ERR_CUDA;
            }
        }
    }
    if (enable && !ctx->dev_lobe_count) {
        cudaError_t e = cudaMalloc((void**)&ctx->dev_lobe_count, sizeof(unsigned long long));
        if (e != cudaSuccess) {
            vx_record_cuda_error(ctx, e, "cudaMalloc");
            return VX_ERR_CUDA;
        }
    }
    if (enable) {
        vx_prof_drain(ctx);
        for (int i = 0; i < ST_NSTAGES; ++i) { ctx->launches[i] = 0; ctx->stage_ms[i] = 0.0; ctx->units[i] = 0; }
        cudaMemset(ctx->dev_lobe_count, 0, sizeof(unsigned long long));
    }
    ctx->prof = enable != 0;
    return VX_OK;
}

vx_status vx_profile_read(vx_context* ctx, vx_stage_time* out, int max_stages, int* num_stages) {
    if (!ctx || !num_stages) return VX_ERR_INVALID_ARG;
    vx_prof_drain(ctx);
    *num_stages = ST_NSTAGES;
    if (ctx->dev_lobe_count) {
        unsigned long long n = 0;
        cudaDeviceSynchronize();
        if (cudaMemcpy(&n, ctx->dev_lobe_count, sizeof(n), cudaMemcpyDeviceToHost) == cudaSuccess)
            ctx->units[ST_SGGX_CLUSTER] = (int64_t)n;
    }
    if (out) {
        for (int i = 0; i < ST_NSTAGES && i < max_stages; ++i) {
            memset(out[i].name, 0, sizeof(out[i].name));
            strncpy(out[i].name, kStageNames[i], sizeof(out[i].name) - 1);
            out[i].launches = ctx->launches[i];
            out[i].total_ms = ctx->stage_ms[i];
            out[i].units = ctx->units[i];
        }
    }
    return VX_OK;
}

namespace {
// one byte of the compact export: round-half-even of x * scale + bias, clamped to [0, 255]
__device__ __forceinline__ uint8_t quantize8(float x, float scale, float bias) {
    const float q = rintf(x * scale + bias);
    return (uint8_t)fminf(fmaxf(q, 0.0f), 255.0f);
}

__global__ void k_export_compact8(const float* __restrict__ compact, const uint8_t* __restrict__ lobe_count,
                                  int64_t n, int K, uint8_t* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // (voxel, lobe)
    if (i >= n * K) return;
    const int64_t v = i / K;
    const int k = (int)(i - v * K);
    uint8_t q[6] = {0, 0, 0, 0, 0, 0};
    if (k < (int)lobe_count[v]) {
        const float* c = compact + (size_t)i * 6;
#pragma unroll
        for (int j = 0; j < 3; ++j) q[j] = quantize8(c[j], 255.0f, 0.0f);
#pragma unroll
        for (int j = 3; j < 6; ++j) q[j] = quantize8(c[j], 127.5f, 127.5f);
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) out[(size_t)i * 6 + j] = q[j];
}
}  // namespace

namespace {
// leaf (8^3 block) of each voxel: its Morton key >> 9
__global__ void k_leaf_ids(const uint64_t* __restrict__ keys, int64_t n, uint32_t* __restrict__ leaf) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) leaf[i] = (uint32_t)(keys[i] >> 9);
}

// thread per leaf: its key and the value mask of its voxels, in the leaf's x-major order
// (bit (x & 7) * 64 + (y & 7) * 8 + (z & 7))
__global__ void k_leaf_masks(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ first,
                             const uint32_t* __restrict__ nleaf_p, uint64_t* __restrict__ leaf_keys,
                             uint64_t* __restrict__ leaf_masks) {
    const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= *nleaf_p) return;
    uint64_t m[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const uint32_t b = first[l], e = first[l + 1];
    for (uint32_t i = b; i < e; ++i) {
        const uint32_t k = (uint32_t)(keys[i] & 511u);
        const uint32_t x = vx_compact1by2(k), y = vx_compact1by2(k >> 1), z = vx_compact1by2(k >> 2);
        const uint32_t bit = (x << 6) | (y << 3) | z;
        m[bit >> 6] |= 1ull << (bit & 63u);
    }
    leaf_keys[l] = keys[b] >> 9;
#pragma unroll
    for (int w = 0; w < 8; ++w) leaf_masks[(size_t)l * 8 + w] = m[w];
}
}  // namespace

vx_status vx_export_leaves(vx_context* ctx, const vx_level* level, uint64_t* leaf_keys, uint64_t* leaf_masks,
                           uint32_t* leaf_first, int64_t* num_leaves, void* stream) {
    if (!ctx || !level || !num_leaves) return VX_ERR_INVALID_ARG;
    *num_leaves = 0;
    const int64_t n = level->num_voxels;
    if (n < 0 || n > 0xfffffffell) return VX_ERR_INVALID_ARG;
    if (!leaf_first) return VX_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        VX_CUDA_TRY(cudaMemsetAsync(leaf_first, 0, 4, s));
        return VX_OK;
    }
    if (!level->keys || !leaf_keys || !leaf_masks) return VX_ERR_INVALID_ARG;
    if (level->resolution > 2048) return VX_ERR_UNSUPPORTED;
    VX_TRY(vx_ws_ensure(ctx, WS_LOD_IDX, (size_t)n * 4, s));
    VX_TRY(vx_ws_ensure(ctx, WS_MISC, 256, s));
    uint32_t* leaf = (uint32_t*)ctx->ws[WS_LOD_IDX].p;
    uint32_t* misc = (uint32_t*)ctx->ws[WS_MISC].p;
    k_leaf_ids<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(level->keys, n, leaf);
    VX_CUDA_TRY(cudaGetLastError());
    VX_TRY(vx_segment_starts(ctx, leaf, (uint32_t)n, misc + 10, leaf_first, s));
    k_leaf_masks<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(level->keys, leaf_first, misc + 10, leaf_keys,
                                                             leaf_masks);
    VX_CUDA_TRY(cudaGetLastError());
    VX_TRY(vx_readback_async(ctx, 0, misc + 10, 4, s));
    VX_CUDA_TRY(cudaStreamSynchronize(s));
    *num_leaves = ((const uint32_t*)ctx->host_pin)[0];
    return VX_OK;
}

vx_status vx_export_compact8(const vx_level* level, uint8_t* out, void* stream) {
    if (!level) return VX_ERR_INVALID_ARG;
    if (level->num_voxels == 0) return VX_OK;
    if (!out || level->num_voxels < 0 || level->K < 1 || level->K > vx::kMaxK || !level->compact || !level->lobe_count)
        return VX_ERR_INVALID_ARG;
    const int64_t items = level->num_voxels * level->K;
    const unsigned blocks = (unsigned)((items + 255) / 256);
    k_export_compact8<<<blocks, 256, 0, (cudaStream_t)stream>>>(level->compact, level->lobe_count, level->num_voxels,
                                                                level->K, out);
    return cudaGetLastError() == cudaSuccess ? VX_OK : VX_ERR_CUDA;
}

void vx_level_release(vx_context* ctx, vx_level* level, void* stream) {
    if (!ctx || !level) return;
    if (level->block) vx_dev_free(ctx, level->block, (cudaStream_t)stream);
    memset(level, 0, sizeof(*level));
}

const char* vx_status_string(vx_status s) {
    switch (s) {
        case VX_OK: return "ok";
        case VX_ERR_INVALID_ARG: return "invalid argument";
        case VX_ERR_OUT_OF_MEMORY: return "out of device memory (allocator returned NULL)";
        case VX_ERR_CAPACITY: return "capacity exceeded (more than 2^32-1 candidate pairs)";
        case VX_ERR_CUDA: return "CUDA runtime error";
        case VX_ERR_TIMEOUT: return "bounded wait timed out";
        case VX_ERR_UNSUPPORTED: return "unsupported parameter";
    }
    return "unknown status";
}

const char* vx_last_cuda_error(const vx_context* ctx) { return ctx ? ctx->last_err : ""; }

}  // extern "C"
