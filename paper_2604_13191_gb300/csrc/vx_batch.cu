// vx_batch.cu -- many instances (meshes and fiber patches of uneven size, each with its
// own grid) voxelized and reduced to all their pyramid levels by one captured CUDA graph.
//
// All instances of one primitive kind share one pipeline: the candidate pairs of every
// instance are emitted together (primitive-major, instances contiguous), sorted by Morton
// key and then, stably, by instance (a last radix pass whose digit is the instance of the
// pair's primitive), so each instance's voxels are contiguous and in key order.  Segment
// heads and LoD parents also split where the instance changes.  Counts stay on the
// device: buffers are sized by a planning run (synchronising, at creation) plus headroom,
// every later run clamps its counts to those capacities and raises an overflow flag.
// The run enqueues kernels only, so it is captured into a CUDA graph once and replayed.
// The per-instance kernels are persistent grid-stride kernels sized to the 152 SMs.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "vx_level0.cuh"

namespace {

constexpr int kMaxLevels = 11;

struct BInst {
    float o[3];
    float s;
    int R;
    int L;
    uint32_t prim_begin, num_prims;
};

__device__ __forceinline__ int find_inst(const BInst* __restrict__ inst, int ninst, uint32_t p) {
    int lo = 0, hi = ninst;   // last instance with prim_begin <= p
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (inst[mid].prim_begin <= p) lo = mid + 1; else hi = mid;
    }
    return lo - 1;
}

__global__ void k_bprep_fibers(const float4* __restrict__ ctrl, int64_t num_ctrl, const int64_t* __restrict__ off,
                               const uint32_t* __restrict__ seg_start, int64_t F, const float* __restrict__ weights,
                               uint32_t np, const BInst* __restrict__ inst, int ninst, float4* __restrict__ ra,
                               float4* __restrict__ rb, uint8_t* __restrict__ inst_of, uint32_t* __restrict__ err) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    int64_t lo = 0, hi = F;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (seg_start[mid] <= p) lo = mid + 1; else hi = mid;
    }
    const int64_t f = lo - 1;
    const int ii = find_inst(inst, ninst, p);
    if (f < 0 || ii < 0 || p >= inst[ii].prim_begin + inst[ii].num_prims) { atomicOr(err, 1u); return; }
    const int64_t o0 = off[f];
    const int64_t c = o0 + (int64_t)(p - seg_start[f]);
    if (o0 < 0 || c < 0 || c + 1 >= off[f + 1] || c + 1 >= num_ctrl) { atomicOr(err, 1u); return; }
    const BInst g = inst[ii];
    const float4 pa = ctrl[c], pb = ctrl[c + 1];
    float4 A, B;
    A.x = (pa.x - g.o[0]) * g.s; A.y = (pa.y - g.o[1]) * g.s; A.z = (pa.z - g.o[2]) * g.s;
    B.x = (pb.x - g.o[0]) * g.s; B.y = (pb.y - g.o[1]) * g.s; B.z = (pb.z - g.o[2]) * g.s;
    A.w = ((pa.w + pb.w) * 0.5f) * g.s;
    B.w = weights ? weights[p] : 1.0f;
    if (bad_record(A, B)) atomicOr(err, 1u);
    ra[p] = A;
    rb[p] = B;
    inst_of[p] = (uint8_t)ii;
}

__global__ void k_bprep_tris(const float4* __restrict__ tv, const float* __restrict__ weights, uint32_t np,
                             const BInst* __restrict__ inst, int ninst, float4* __restrict__ r0,
                             float4* __restrict__ r1, float4* __restrict__ r2, uint8_t* __restrict__ inst_of,
                             uint32_t* __restrict__ err) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int ii = find_inst(inst, ninst, p);
    if (ii < 0 || p >= inst[ii].prim_begin + inst[ii].num_prims) { atomicOr(err, 1u); return; }
    const BInst g = inst[ii];
    const float4 v0 = tv[3 * (size_t)p], v1 = tv[3 * (size_t)p + 1], v2 = tv[3 * (size_t)p + 2];
    float4 a, b, c;
    a.x = (v0.x - g.o[0]) * g.s; a.y = (v0.y - g.o[1]) * g.s; a.z = (v0.z - g.o[2]) * g.s;
    b.x = (v1.x - g.o[0]) * g.s; b.y = (v1.y - g.o[1]) * g.s; b.z = (v1.z - g.o[2]) * g.s;
    c.x = (v2.x - g.o[0]) * g.s; c.y = (v2.y - g.o[1]) * g.s; c.z = (v2.z - g.o[2]) * g.s;
    a.w = weights ? weights[p] : 1.0f;
    b.w = 0.0f;
    c.w = 0.0f;
    if (bad_record(a, b) || bad_record(c, c)) atomicOr(err, 1u);
    r0[p] = a; r1[p] = b; r2[p] = c;
    inst_of[p] = (uint8_t)ii;
}

// count / emit with the resolution of each primitive's instance; emission is clamped to
// the pair capacity (an overflow is reported by the count clamp)
template <bool FIBER, bool EMIT>
__global__ void __launch_bounds__(EMIT_WARPS * 32) k_bcandidates(const float4* __restrict__ r0,
                                                                 const float4* __restrict__ r1,
                                                                 const float4* __restrict__ r2, uint32_t np,
                                                                 const BInst* __restrict__ inst,
                                                                 const uint8_t* __restrict__ inst_of,
                                                                 uint32_t* __restrict__ counts,
                                                                 const uint32_t* __restrict__ offs, uint32_t cap,
                                                                 uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * EMIT_WARPS;
    for (uint32_t p = blockIdx.x * EMIT_WARPS + (threadIdx.x >> 5); p < np; p += warps) {
        const Window R = full_window(inst[inst_of[p]].R);
        float4 a = r0[p], b = r1[p], c;
        Range rg;
        if (FIBER) {
            rg = capsule_range(a, b, R);
        } else {
            c = r2[p];
            rg = tri_range(a, b, c, R);
        }
        uint32_t n = 0;
        const uint32_t base = EMIT ? offs[p] : 0u;
        const long long tot = rg.total;
        for (long long idx0 = 0; idx0 < tot; idx0 += 32) {
            const long long idx = idx0 + lane;
            bool hit = false;
            int vi = 0, vj = 0, vk = 0;
            if (idx < tot) {
                int ix, iy, iz;
                voxel_of(idx, tot, rg, ix, iy, iz);
                vi = rg.lo[0] + ix; vj = rg.lo[1] + iy; vk = rg.lo[2] + iz;
                hit = FIBER ? capsule_voxel_candidate(a, b, vi, vj, vk) : tri_voxel_candidate(a, b, c, vi, vj, vk);
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, hit);
            if (EMIT && hit) {
                const uint32_t pos = base + n + __popc(bal & ((1u << lane) - 1u));
                if (pos < cap) {
                    keys[pos] = vx_morton3((uint32_t)vi, (uint32_t)vj, (uint32_t)vk);
                    vals[pos] = p;
                }
            }
            n += __popc(bal);
        }
        if (!EMIT && lane == 0) counts[p] = n;
    }
}

__global__ void k_clamp(const uint32_t* __restrict__ total, uint32_t cap, uint32_t* __restrict__ n_out,
                        uint32_t* __restrict__ err) {
    const uint32_t t = *total;
    *n_out = t < cap ? t : cap;
    if (t > cap) atomicOr(err, 2u);
}

// padding behind the valid pairs: key and value 0xffffffff sort last
__global__ void k_pad(uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, const uint32_t* __restrict__ n_dev,
                      uint32_t cap) {
    const uint32_t n = *n_dev;
    for (uint32_t i = n + blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) {
        keys[i] = 0xffffffffu;
        vals[i] = 0xffffffffu;
    }
}

// zero a[i] for n <= i < cap (flags past a clamped count)
__global__ void k_zero_tail(uint32_t* __restrict__ a, const uint32_t* __restrict__ n_dev, uint32_t cap) {
    const uint32_t n = *n_dev;
    for (uint32_t i = n + blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) a[i] = 0u;
}

__global__ void k_bhead_flags(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                              const uint8_t* __restrict__ inst_of, const uint32_t* __restrict__ n_dev, uint32_t cap,
                              uint32_t* __restrict__ flags) {
    const uint32_t n = *n_dev;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x)
        flags[i] = (i < n && (i == 0 || keys[i] != keys[i - 1] || inst_of[vals[i]] != inst_of[vals[i - 1]])) ? 1u
                                                                                                           : 0u;
}

__global__ void k_bhead_starts(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                               const uint8_t* __restrict__ inst_of, const uint32_t* __restrict__ n_dev,
                               const uint32_t* __restrict__ idx, const uint32_t* __restrict__ total, uint32_t cap_seg,
                               uint32_t* __restrict__ starts) {
    const uint32_t n = *n_dev;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const bool head = i == 0 || keys[i] != keys[i - 1] || inst_of[vals[i]] != inst_of[vals[i - 1]];
        if (head && idx[i] <= cap_seg) starts[idx[i]] = i;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && *total <= cap_seg) starts[*total] = n;
}

// compaction into the level-0 block (guarded by its capacity) + instance id per voxel
__global__ void k_bfinalize(SegOut in, const uint32_t* __restrict__ nseg_p, const uint32_t* __restrict__ dst,
                            uint32_t cap_v, const uint32_t* __restrict__ starts, const uint32_t* __restrict__ vals,
                            const uint8_t* __restrict__ inst_of, vx_level L, uint16_t* __restrict__ inst_v) {
    const uint32_t nseg = *nseg_p;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += gridDim.x * blockDim.x) {
        if (!in.nonzero[s]) continue;
        const uint32_t o = dst[s];
        if (o >= cap_v) continue;
        L.keys[o] = (uint64_t)in.key[s];
        uint64_t m[8];
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            m[w] = in.mask[(size_t)s * 8 + w];
            L.mask[(size_t)o * 8 + w] = m[w];
        }
        const float mass = in.mass[s];
        float M[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            M[c] = in.moment[(size_t)s * 6 + c];
            L.moment[(size_t)o * 6 + c] = M[c];
        }
        L.mass[o] = mass;
        uint16_t occ;
        uint8_t pj[3];
        mask_counts(m, occ, pj);
        L.occ[o] = occ;
        L.occ_proj[(size_t)o * 3 + 0] = pj[0];
        L.occ_proj[(size_t)o * 3 + 1] = pj[1];
        L.occ_proj[(size_t)o * 3 + 2] = pj[2];
        write_lobe(mass, M, L.lobes + (size_t)o * 7, L.compact + (size_t)o * 6, L.lobe_count + o);
        inst_v[o] = inst_of[vals[starts[s]]];
    }
}

// first voxel of every instance in a level (lower bound on the instance ids) and the end
__global__ void k_inst_offsets(const uint16_t* __restrict__ inst_v, const uint32_t* __restrict__ n_dev, int ninst,
                               uint32_t* __restrict__ start) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > ninst) return;
    const uint32_t n = *n_dev;
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((int)inst_v[mid] < i) lo = mid + 1; else hi = mid;
    }
    start[i] = (i == ninst) ? n : lo;
}

__global__ void k_bparent_count_flags(const uint64_t* __restrict__ keys, const uint16_t* __restrict__ inst,
                                      const uint32_t* __restrict__ n_dev, uint32_t cap, uint32_t* __restrict__ flags) {
    const uint32_t n = *n_dev;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x)
        flags[i] = (i < n && (i == 0 || inst[i] != inst[i - 1] || (keys[i] >> 3) != (keys[i - 1] >> 3))) ? 1u : 0u;
}

inline unsigned gf(size_t n, int threads, size_t cap_blocks) {
    size_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return (unsigned)std::min(b, cap_blocks);
}

// counters of one sub-batch (device words)
enum {
    C_ERR = 0, C_SEGTOT, C_PAIRS_TOT, C_PAIRS, C_SEG_TOT, C_SEG, C_VOX_TOT, C_VOX,
    C_LVL = 8,  // C_LVL + l: parent count of level l (1..kMaxLevels); C_LVL + 16 + l: raw totals
    C_TAKE = 48, // work counter of the reduce kernel
    C_CLUSTER = 50  // [50] parents listed for clustering, [51] their take counter
};

struct SubBatch {
    bool fiber = false;
    int ninst = 0;
    uint32_t np = 0;
    int64_t F = 0;
    int Lmax = 0;
    int key_bits = 0;
    const float* tri = nullptr;
    const float* ctrl = nullptr;
    int64_t num_ctrl = 0;
    const int64_t* off = nullptr;
    const float* weights = nullptr;
    std::vector<BInst> hinst;
    BInst* dinst = nullptr;
    uint8_t* inst_of = nullptr;
    float4 *r0 = nullptr, *r1 = nullptr, *r2 = nullptr;
    uint32_t *cnt = nullptr, *offs = nullptr, *fs = nullptr;
    uint32_t *k0 = nullptr, *v0 = nullptr, *k1 = nullptr, *v1 = nullptr;
    uint32_t *hist = nullptr, *part = nullptr, *flags = nullptr, *idx = nullptr, *starts = nullptr;
    SegOut seg{};
    uint32_t* dst = nullptr;
    uint32_t* counters = nullptr;           // 64 words
    uint32_t* inst_start = nullptr;         // [(Lmax + 1)][ninst + 1]
    vx_level lv[kMaxLevels + 1];
    uint16_t* linst[kMaxLevels + 1];
    void* stats[kMaxLevels + 1] = {};      // K > 1: lobe statistics of each level (none for 0)
    uint32_t* work[kMaxLevels + 1] = {};   // K > 1: parents listed for clustering
    uint32_t cap_pairs = 0, cap_seg = 0, cap_v[kMaxLevels + 1];
};

}  // namespace

struct vx_batch {
    vx_context* ctx = nullptr;
    SubBatch sb[2];          // 0: triangles, 1: fibers
    std::vector<void*> allocs;
    float headroom = 0.125f;
    int K = 1;                              // lobes per voxel of the levels above 0
    int n_dirs = 0;
    int merge = 0;                          // SGGX-H merge rule (vx_lod_params.merge)
    float4* dirs4 = nullptr;                // direction table of the lobe histograms (K > 1)
    cudaStream_t cap_stream = nullptr;
    cudaStream_t cap_stream2 = nullptr;     // the triangle branch of the captured graph
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int num_instances = 0;
    std::vector<int> kind_of, local_of;   // instance -> (sub-batch, index in it)
    std::vector<uint32_t> host_counts[2];
    std::vector<uint32_t> host_starts[2];
    bool host_valid = false;
    int64_t launches_per_run = 0;
};

namespace {

vx_status balloc(vx_batch* b, void** p, size_t bytes, cudaStream_t s) {
    *p = vx_dev_alloc(b->ctx, bytes, s);
    if (!*p) return VX_ERR_OUT_OF_MEMORY;
    b->allocs.push_back(*p);
    return VX_OK;
}

uint32_t with_headroom(uint32_t n, float h) {
    double x = (double)n * (1.0 + (double)h) + 1024.0;
    return x > 4.0e9 ? 0xffffffffu : (uint32_t)x;
}

// Enqueue the pipeline of one sub-batch.  plan: synchronise after each counting stage,
// allocate the buffers it needs (capacity = measured count + headroom) and record them;
// otherwise only kernels are enqueued (capturable).  *nl counts the launches.
vx_status enqueue(vx_batch* b, SubBatch& S, cudaStream_t s, bool plan, int64_t* nl) {
    if (S.np == 0) return VX_OK;
    vx_context* ctx = b->ctx;
    uint32_t* C = S.counters;
    uint32_t* host = (uint32_t*)ctx->host_pin;
    const unsigned blk = vx::kSMs * 16;
    auto readback = [&](int word) -> uint32_t {
        if (cudaMemcpyAsync(host, C + word, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return 0xffffffffu;
        if (cudaStreamSynchronize(s) != cudaSuccess) return 0xffffffffu;
        return host[0];
    };
    if (cudaMemsetAsync(C, 0, 64 * 4, s) != cudaSuccess) return VX_ERR_CUDA;
    ++*nl;
    // ---- prep -------------------------------------------------------------------------
    if (S.fiber) {
        k_fiber_seg_counts<<<gf((size_t)S.F, 256, 1u << 30), 256, 0, s>>>(S.off, S.F, S.num_ctrl, S.fs, C + C_ERR);
        if (vx_scan_u32_scratch(S.fs, S.fs, (uint32_t)S.F, C + C_SEGTOT, S.part, s) != cudaSuccess) return VX_ERR_CUDA;
        k_bprep_fibers<<<gf(S.np, 256, 1u << 30), 256, 0, s>>>((const float4*)S.ctrl, S.num_ctrl, S.off, S.fs, S.F, S.weights,
                                                               S.np, S.dinst, S.ninst, S.r0, S.r1, S.inst_of,
                                                               C + C_ERR);
        *nl += 5;
    } else {
        k_bprep_tris<<<gf(S.np, 256, 1u << 30), 256, 0, s>>>((const float4*)S.tri, S.weights, S.np, S.dinst,
                                                             S.ninst, S.r0, S.r1, S.r2, S.inst_of, C + C_ERR);
        *nl += 1;
    }
    // ---- candidates ----------------------------------------------------------------------
    const unsigned cblocks = (unsigned)std::min<size_t>((S.np + EMIT_WARPS - 1) / EMIT_WARPS, (size_t)vx::kSMs * 64);
    if (S.fiber)
        k_bcandidates<true, false><<<cblocks, EMIT_WARPS * 32, 0, s>>>(S.r0, S.r1, S.r2, S.np, S.dinst, S.inst_of,
                                                                       S.cnt, nullptr, 0, nullptr, nullptr);
    else
        k_bcandidates<false, false><<<cblocks, EMIT_WARPS * 32, 0, s>>>(S.r0, S.r1, S.r2, S.np, S.dinst, S.inst_of,
                                                                        S.cnt, nullptr, 0, nullptr, nullptr);
    if (vx_scan_u32_scratch(S.cnt, S.offs, S.np, C + C_PAIRS_TOT, S.part, s) != cudaSuccess) return VX_ERR_CUDA;
    *nl += 4;
    if (plan) {
        const uint32_t err = readback(C_ERR);
        if (err) return VX_ERR_INVALID_ARG;
        const uint32_t np = readback(C_PAIRS_TOT);
        if (np >= 0x80000000u) return VX_ERR_CAPACITY;
        S.cap_pairs = with_headroom(np, b->headroom);
        const uint32_t nt = (S.cap_pairs + 4095) / 4096;
        const size_t hn = (size_t)256 * nt;
        VX_TRY(balloc(b, (void**)&S.k0, (size_t)S.cap_pairs * 4, s));
        VX_TRY(balloc(b, (void**)&S.v0, (size_t)S.cap_pairs * 4, s));
        VX_TRY(balloc(b, (void**)&S.k1, (size_t)S.cap_pairs * 4, s));
        VX_TRY(balloc(b, (void**)&S.v1, (size_t)S.cap_pairs * 4, s));
        VX_TRY(balloc(b, (void**)&S.hist, hn * 4, s));
        VX_TRY(balloc(b, (void**)&S.flags, (size_t)S.cap_pairs * 4, s));
        VX_TRY(balloc(b, (void**)&S.idx, (size_t)S.cap_pairs * 4, s));
        // scan partials: the largest scanned array is max(hist, pairs)
        const size_t mx = std::max<size_t>(hn, S.cap_pairs);
        VX_TRY(balloc(b, (void**)&S.part, (mx / 2048 + 64) * 4, s));
    }
    k_clamp<<<1, 1, 0, s>>>(C + C_PAIRS_TOT, S.cap_pairs, C + C_PAIRS, C + C_ERR);
    if (S.fiber)
        k_bcandidates<true, true><<<cblocks, EMIT_WARPS * 32, 0, s>>>(S.r0, S.r1, S.r2, S.np, S.dinst, S.inst_of,
                                                                      nullptr, S.offs, S.cap_pairs, S.k0, S.v0);
    else
        k_bcandidates<false, true><<<cblocks, EMIT_WARPS * 32, 0, s>>>(S.r0, S.r1, S.r2, S.np, S.dinst, S.inst_of,
                                                                       nullptr, S.offs, S.cap_pairs, S.k0, S.v0);
    k_pad<<<blk, 256, 0, s>>>(S.k0, S.v0, C + C_PAIRS, S.cap_pairs);
    *nl += 3;
    // ---- sort by (instance, key) ------------------------------------------------------------
    uint32_t *k0 = S.k0, *v0 = S.v0, *k1 = S.k1, *v1 = S.v1;
    if (vx_radix_sort_u32_scratch(&k0, &v0, &k1, &v1, S.cap_pairs, S.key_bits, S.inst_of, S.hist, S.part, s) !=
        cudaSuccess)
        return VX_ERR_CUDA;
    *nl += 5 * ((S.key_bits + 7) / 8 + 1);
    // ---- segments ---------------------------------------------------------------------------
    k_bhead_flags<<<gf(S.cap_pairs, 256, blk), 256, 0, s>>>(k0, v0, S.inst_of, C + C_PAIRS, S.cap_pairs, S.flags);
    if (vx_scan_u32_scratch(S.flags, S.idx, S.cap_pairs, C + C_SEG_TOT, S.part, s) != cudaSuccess) return VX_ERR_CUDA;
    *nl += 4;
    if (plan) {
        const uint32_t ns = readback(C_SEG_TOT);
        S.cap_seg = std::min(with_headroom(ns, b->headroom), S.cap_pairs);
        VX_TRY(balloc(b, (void**)&S.starts, ((size_t)S.cap_seg + 2) * 4, s));
        char* so = nullptr;
        VX_TRY(balloc(b, (void**)&so, (size_t)S.cap_seg * (64 + 4 + 24), s));
        S.seg.mask = (uint64_t*)so;
        S.seg.mass = (float*)(so + (size_t)S.cap_seg * 64);
        S.seg.moment = (float*)(so + (size_t)S.cap_seg * 68);
        VX_TRY(balloc(b, (void**)&S.seg.key, (size_t)S.cap_seg * 4, s));
        VX_TRY(balloc(b, (void**)&S.seg.nonzero, (size_t)S.cap_seg * 4, s));
        VX_TRY(balloc(b, (void**)&S.dst, (size_t)S.cap_seg * 4, s));
    }
    k_clamp<<<1, 1, 0, s>>>(C + C_SEG_TOT, S.cap_seg, C + C_SEG, C + C_ERR);
    k_bhead_starts<<<gf(S.cap_pairs, 256, blk), 256, 0, s>>>(k0, v0, S.inst_of, C + C_PAIRS, S.idx, C + C_SEG_TOT,
                                                             S.cap_seg, S.starts);
    // ---- per-voxel reduction ------------------------------------------------------------------
    // resident blocks taking voxels from a counter (zeroed by a node of the graph)
    if (cudaMemsetAsync(C + C_TAKE, 0, 4, s) != cudaSuccess) return VX_ERR_CUDA;
    if (S.fiber) {
        const unsigned rblocks = (unsigned)std::min<size_t>((S.cap_seg + RED_WARPS - 1) / RED_WARPS, (size_t)vx::kSMs * 7);
        k_reduce_fibers<<<rblocks, RED_WARPS * 32, 0, s>>>(k0, v0, S.starts, C + C_SEG, S.r0, S.r1, S.seg, 0, 0, 0,
                                                          C + C_TAKE);
    } else {
        const unsigned rblocks = (unsigned)std::min<size_t>((S.cap_seg + RED_WARPS - 1) / RED_WARPS, (size_t)vx::kSMs * 32);
        k_reduce_tris<<<rblocks, RED_WARPS * 32, 0, s>>>(k0, v0, S.starts, C + C_SEG, S.r0, S.r1, S.r2, S.seg, 0, 0,
                                                         0, C + C_TAKE);
    }
    // non-empty flags beyond the clamped segment count read as zero in the compaction scan
    k_zero_tail<<<blk, 256, 0, s>>>(S.seg.nonzero, C + C_SEG, S.cap_seg);
    if (vx_scan_u32_scratch(S.seg.nonzero, S.dst, S.cap_seg, C + C_VOX_TOT, S.part, s) != cudaSuccess)
        return VX_ERR_CUDA;
    *nl += 5;
    // ---- level 0 ------------------------------------------------------------------------------
    if (plan) {
        const uint32_t nv = readback(C_VOX_TOT);
        S.cap_v[0] = with_headroom(nv, b->headroom);
        VX_TRY(vx_level_alloc(ctx, &S.lv[0], S.cap_v[0], 1, 0, 0, s));
        b->allocs.push_back(S.lv[0].block);
        VX_TRY(balloc(b, (void**)&S.linst[0], (size_t)S.cap_v[0] * 2 + 16, s));
    }
    k_clamp<<<1, 1, 0, s>>>(C + C_VOX_TOT, S.cap_v[0], C + C_VOX, C + C_ERR);
    k_bfinalize<<<gf(S.cap_seg, 256, blk), 256, 0, s>>>(S.seg, C + C_SEG, S.dst, S.cap_v[0], S.starts, v0, S.inst_of,
                                                        S.lv[0], S.linst[0]);
    k_inst_offsets<<<(S.ninst + 1 + 127) / 128, 128, 0, s>>>(S.linst[0], C + C_VOX, S.ninst, S.inst_start);
    *nl += 3;
    // ---- coarser levels -------------------------------------------------------------------------
    for (int l = 1; l <= S.Lmax; ++l) {
        const uint32_t* nprev = (l == 1) ? C + C_VOX : C + C_LVL + (l - 1);
        if (plan) {
            // exact parent count of this level: run the flag scan once to measure it
            k_bparent_count_flags<<<gf(S.cap_v[l - 1], 256, blk), 256, 0, s>>>(S.lv[l - 1].keys, S.linst[l - 1], nprev,
                                                                               S.cap_v[l - 1], S.flags);
            if (vx_scan_u32_scratch(S.flags, S.idx, S.cap_v[l - 1], C + C_LVL + 16 + l, S.part, s) != cudaSuccess)
                return VX_ERR_CUDA;
            const uint32_t np = readback(C_LVL + 16 + l);
            S.cap_v[l] = with_headroom(np, b->headroom);
            VX_TRY(vx_level_alloc(ctx, &S.lv[l], S.cap_v[l], b->K, l, 0, s));
            b->allocs.push_back(S.lv[l].block);
            VX_TRY(balloc(b, (void**)&S.linst[l], (size_t)S.cap_v[l] * 2 + 16, s));
            if (b->K > 1) {
                VX_TRY(balloc(b, &S.stats[l], (size_t)S.cap_v[l] * b->K * kLobeStatsBytes, s));
                VX_TRY(balloc(b, (void**)&S.work[l], (size_t)S.cap_v[l] * 4 + 16, s));
            }
        }
        if (vx_lod_step_batched(&S.lv[l - 1], S.linst[l - 1], nprev, S.cap_v[l - 1], &S.lv[l], S.linst[l],
                                C + C_LVL + l, S.cap_v[l], S.flags, S.idx, S.starts, S.part, C + C_LVL + 16 + l,
                                C + C_ERR, b->dirs4, b->n_dirs, S.work[l], C + C_CLUSTER,
                                l > 1 ? S.stats[l - 1] : nullptr, S.stats[l], b->merge, s) != cudaSuccess)
            return VX_ERR_CUDA;
        k_inst_offsets<<<(S.ninst + 1 + 127) / 128, 128, 0, s>>>(S.linst[l], C + C_LVL + l, S.ninst,
                                                                 S.inst_start + (size_t)l * (S.ninst + 1));
        *nl += 9;
    }
    return VX_OK;
}

}  // namespace

// =====================================================================================
// C ABI
// =====================================================================================
extern "C" vx_status vx_batch_create(vx_context* ctx, const vx_primitives* tris, const vx_primitives* fibers,
                                     const vx_instance* instances, int num_instances, float headroom, void* stream,
                                     vx_batch** out) {
    return vx_batch_create_lod(ctx, tris, fibers, instances, num_instances, nullptr, headroom, stream, out);
}

extern "C" vx_status vx_batch_create_lod(vx_context* ctx, const vx_primitives* tris, const vx_primitives* fibers,
                                         const vx_instance* instances, int num_instances, const vx_lod_params* lod,
                                         float headroom, void* stream, vx_batch** out) {
    if (!ctx || !instances || num_instances <= 0 || !out || !(headroom >= 0.0f)) return VX_ERR_INVALID_ARG;
    *out = nullptr;
    const int K = lod ? lod->K : 1;
    if (K < 1 || K > vx::kMaxK) return VX_ERR_UNSUPPORTED;
    if (lod && lod->num_levels != 0) return VX_ERR_UNSUPPORTED;
    if (K > 1 && (!lod->dirs || lod->n_samples < 1 || lod->n_samples > 65536)) return VX_ERR_INVALID_ARG;
    if (lod && lod->merge != 0 && lod->merge != 1) return VX_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    vx_batch* b = new (std::nothrow) vx_batch();
    if (!b) return VX_ERR_OUT_OF_MEMORY;
    b->ctx = ctx;
    b->headroom = headroom;
    b->K = K;
    b->num_instances = num_instances;
    b->kind_of.resize(num_instances);
    b->local_of.resize(num_instances);
    vx_status st = VX_OK;
    auto fail = [&](vx_status e) {
        vx_batch_destroy(b);
        return e;
    };
    // instance tables per kind, checked on the host (ranges contiguous and in order)
    uint32_t next[2] = {0, 0};
    int64_t next_fiber = 0;
    for (int i = 0; i < num_instances; ++i) {
        const vx_instance& I = instances[i];
        const int k = I.kind == VX_FIBERS ? 1 : 0;
        if (I.kind != VX_FIBERS && I.kind != VX_TRIANGLES) return fail(VX_ERR_INVALID_ARG);
        const uint32_t R = I.grid.resolution;
        if (R == 0 || (R & (R - 1)) != 0 || !(I.grid.voxel_size > 0.0f)) return fail(VX_ERR_INVALID_ARG);
        if (R > 1024 || I.grid.sub_res != 8) return fail(VX_ERR_UNSUPPORTED);
        if (I.prim_begin != (int64_t)next[k] || I.num_prims < 0) return fail(VX_ERR_INVALID_ARG);
        if (k == 1 && (I.fiber_begin != next_fiber || I.num_fibers < 0)) return fail(VX_ERR_INVALID_ARG);
        SubBatch& S = b->sb[k];
        if (S.ninst >= 255) return fail(VX_ERR_UNSUPPORTED);
        BInst bi;
        bi.o[0] = I.grid.origin[0]; bi.o[1] = I.grid.origin[1]; bi.o[2] = I.grid.origin[2];
        bi.s = 1.0f / I.grid.voxel_size;
        bi.R = (int)R;
        int L = 0;
        while ((1u << L) < R) ++L;
        bi.L = L;
        bi.prim_begin = (uint32_t)I.prim_begin;
        bi.num_prims = (uint32_t)I.num_prims;
        S.hinst.push_back(bi);
        S.Lmax = std::max(S.Lmax, L);
        S.key_bits = std::max(S.key_bits, 3 * L);
        b->kind_of[i] = k;
        b->local_of[i] = S.ninst++;
        next[k] += (uint32_t)I.num_prims;
        if (k == 1) next_fiber += I.num_fibers;
    }
    if (next[0] && (!tris || tris->kind != VX_TRIANGLES || tris->num_prims != (int64_t)next[0] || !tris->tri_verts ||
                    ((uintptr_t)tris->tri_verts & 15)))
        return fail(VX_ERR_INVALID_ARG);
    if (next[1] && (!fibers || fibers->kind != VX_FIBERS || fibers->num_prims != (int64_t)next[1] || !fibers->ctrl ||
                    !fibers->fiber_offsets || fibers->num_fibers != next_fiber || ((uintptr_t)fibers->ctrl & 15)))
        return fail(VX_ERR_INVALID_ARG);
    if (K > 1) {
        // the direction table, copied once: runs use the directions given here
        b->n_dirs = lod->n_samples;
        b->merge = lod->merge;
        if ((st = balloc(b, (void**)&b->dirs4, (size_t)lod->n_samples * 16, s)) != VX_OK) return fail(st);
        if (vx_lod_batched_prepare(K, lod->dirs, lod->n_samples, b->dirs4, s) != cudaSuccess) return fail(VX_ERR_CUDA);
    }
    for (int k = 0; k < 2; ++k) {
        SubBatch& S = b->sb[k];
        S.fiber = k == 1;
        S.np = next[k];
        if (S.np == 0) continue;
        if (S.fiber) {
            S.ctrl = fibers->ctrl;
            S.num_ctrl = fibers->num_ctrl;
            S.off = fibers->fiber_offsets;
            S.F = fibers->num_fibers;
            S.weights = fibers->weights;
        } else {
            S.tri = tris->tri_verts;
            S.weights = tris->weights;
        }
        if ((st = balloc(b, (void**)&S.dinst, sizeof(BInst) * S.ninst, s)) != VX_OK) return fail(st);
        if (cudaMemcpyAsync(S.dinst, S.hinst.data(), sizeof(BInst) * S.ninst, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail(VX_ERR_CUDA);
        if ((st = balloc(b, (void**)&S.inst_of, (size_t)S.np + 16, s)) != VX_OK) return fail(st);
        if ((st = balloc(b, (void**)&S.r0, (size_t)S.np * 16, s)) != VX_OK) return fail(st);
        if ((st = balloc(b, (void**)&S.r1, (size_t)S.np * 16, s)) != VX_OK) return fail(st);
        if (!S.fiber && (st = balloc(b, (void**)&S.r2, (size_t)S.np * 16, s)) != VX_OK) return fail(st);
        if ((st = balloc(b, (void**)&S.cnt, (size_t)S.np * 4, s)) != VX_OK) return fail(st);
        if ((st = balloc(b, (void**)&S.offs, (size_t)S.np * 4, s)) != VX_OK) return fail(st);
        if ((st = balloc(b, (void**)&S.fs, (size_t)(S.fiber ? S.F : 1) * 4 + 16, s)) != VX_OK) return fail(st);
        if ((st = balloc(b, (void**)&S.counters, 64 * 4, s)) != VX_OK) return fail(st);
        if ((st = balloc(b, (void**)&S.inst_start, (size_t)(kMaxLevels + 1) * (S.ninst + 1) * 4, s)) != VX_OK)
            return fail(st);
        // partials for the scans before the pair buffers exist (largest: primitives or fibers)
        const size_t pre = std::max<size_t>(S.np, (size_t)(S.fiber ? S.F : 1));
        if ((st = balloc(b, (void**)&S.part, (pre / 2048 + 64) * 4, s)) != VX_OK) return fail(st);
        int64_t nl = 0;
        if ((st = enqueue(b, S, s, true, &nl)) != VX_OK) return fail(st);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(VX_ERR_CUDA);
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return fail(VX_ERR_CUDA);
    if (cudaStreamCreateWithFlags(&b->cap_stream2, cudaStreamNonBlocking) != cudaSuccess) return fail(VX_ERR_CUDA);
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) return fail(VX_ERR_CUDA);
    if (cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming) != cudaSuccess) return fail(VX_ERR_CUDA);
    *out = b;
    return VX_OK;
}

extern "C" vx_status vx_batch_run(vx_batch* b, void* stream) {
    if (!b) return VX_ERR_INVALID_ARG;
    vx_context* ctx = b->ctx;
    cudaStream_t s = (cudaStream_t)stream;
    if (!b->exec) {
        // capture the whole run once on a private stream, then replay it on any stream
        if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return VX_ERR_CUDA;
        // two branches: the triangle sub-batch forks onto a second stream and joins before
        // the end, so the graph runs the two pipelines (separate buffers) side by side
        int64_t nl = 0;
        vx_status st = VX_OK;
        if (cudaEventRecord(b->fork, b->cap_stream) != cudaSuccess ||
            cudaStreamWaitEvent(b->cap_stream2, b->fork, 0) != cudaSuccess)
            st = VX_ERR_CUDA;
        if (st == VX_OK) st = enqueue(b, b->sb[0], b->cap_stream2, false, &nl);
        if (st == VX_OK) st = enqueue(b, b->sb[1], b->cap_stream, false, &nl);
        if (cudaEventRecord(b->join, b->cap_stream2) != cudaSuccess ||
            cudaStreamWaitEvent(b->cap_stream, b->join, 0) != cudaSuccess)
            st = st == VX_OK ? VX_ERR_CUDA : st;
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
        if (st != VX_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess || !g) {
            vx_record_cuda_error(ctx, e, "cudaStreamEndCapture");
            return VX_ERR_CUDA;
        }
        if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
            cudaGraphDestroy(g);
            return VX_ERR_CUDA;
        }
        b->graph = g;
        // kernel launches per replay = kernel nodes of the captured graph
        size_t nn = 0;
        cudaGraphGetNodes(g, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
        int64_t kernels = 0;
        for (size_t i = 0; i < nn; ++i) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
        }
        b->launches_per_run = kernels;
        (void)nl;
    }
    vx_stage_begin(ctx, ST_BATCH, s);
    const cudaError_t e = cudaGraphLaunch(b->exec, s);
    vx_stage_end(ctx, s);
    ctx->launches[ST_BATCH] += b->launches_per_run - 1;
    if (e != cudaSuccess) {
        vx_record_cuda_error(ctx, e, "cudaGraphLaunch");
        return VX_ERR_CUDA;
    }
    b->host_valid = false;
    return VX_OK;
}

extern "C" vx_status vx_batch_level(vx_batch* b, int instance, int level, void* stream, vx_level* view) {
    if (!b || !view || instance < 0 || instance >= b->num_instances || level < 0) return VX_ERR_INVALID_ARG;
    memset(view, 0, sizeof(*view));
    const int k = b->kind_of[instance], li = b->local_of[instance];
    SubBatch& S = b->sb[k];
    const BInst& I = S.hinst[li];
    if (level > I.L) return VX_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (!b->host_valid) {
        for (int kk = 0; kk < 2; ++kk) {
            SubBatch& T = b->sb[kk];
            b->host_counts[kk].assign(64, 0);
            b->host_starts[kk].assign((size_t)(kMaxLevels + 1) * (T.ninst + 1), 0);
            if (T.np == 0) continue;
            if (cudaMemcpyAsync(b->host_counts[kk].data(), T.counters, 64 * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaMemcpyAsync(b->host_starts[kk].data(), T.inst_start, b->host_starts[kk].size() * 4,
                                cudaMemcpyDeviceToHost, s) != cudaSuccess)
                return VX_ERR_CUDA;
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) return VX_ERR_CUDA;
        b->host_valid = true;
    }
    const uint32_t err = b->host_counts[k][C_ERR];
    if (err & 2u) return VX_ERR_CAPACITY;
    if (err & 1u) return VX_ERR_INVALID_ARG;
    const uint32_t* st = b->host_starts[k].data() + (size_t)level * (S.ninst + 1);
    const uint32_t beg = st[li], end = st[li + 1];
    const vx_level& L = S.lv[level];
    view->level = level;
    view->resolution = I.R >> level;
    view->num_voxels = end - beg;
    view->K = L.K;
    view->block = nullptr;
    view->keys = L.keys + beg;
    view->mask = L.mask + (size_t)beg * 8;
    view->mass = L.mass + beg;
    view->moment = L.moment + (size_t)beg * 6;
    view->occ = L.occ + beg;
    view->occ_proj = L.occ_proj + (size_t)beg * 3;
    view->lobe_count = L.lobe_count + beg;
    view->lobes = L.lobes + (size_t)beg * L.K * 7;
    view->compact = L.compact + (size_t)beg * L.K * 6;
    return VX_OK;
}

extern "C" void vx_batch_destroy(vx_batch* b) {
    if (!b) return;
    cudaStream_t s = b->ctx->last_stream;
    cudaStreamSynchronize(s);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->cap_stream2) cudaStreamDestroy(b->cap_stream2);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    for (void* p : b->allocs) vx_dev_free(b->ctx, p, s);
    cudaStreamSynchronize(s);
    delete b;
}
