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
                                                                 uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                                 uint32_t* __restrict__ ballots) {
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
        // hit ballots stored by the count pass for the emit pass (as k_candidates)
        const bool stored = ballots != nullptr && tot <= 32ll * CAND_BALLOTS;
        uint32_t* const pb = stored ? ballots + (size_t)p * CAND_BALLOTS : nullptr;
        uint32_t words = 0;
        if (EMIT && stored && (long long)lane * 32 < tot) words = pb[lane];
        for (long long idx0 = 0; idx0 < tot; idx0 += 32) {
            const long long idx = idx0 + lane;
            bool hit = false;
            int vi = 0, vj = 0, vk = 0;
            uint32_t bal;
            if (EMIT && stored) {
                bal = __shfl_sync(0xffffffffu, words, (int)(idx0 >> 5));
                hit = (bal >> lane) & 1u;
                if (hit) {
                    int ix, iy, iz;
                    voxel_of(idx, tot, rg, ix, iy, iz);
                    vi = rg.lo[0] + ix; vj = rg.lo[1] + iy; vk = rg.lo[2] + iz;
                }
            } else {
                if (idx < tot) {
                    int ix, iy, iz;
                    voxel_of(idx, tot, rg, ix, iy, iz);
                    vi = rg.lo[0] + ix; vj = rg.lo[1] + iy; vk = rg.lo[2] + iz;
                    hit = FIBER ? capsule_voxel_candidate(a, b, vi, vj, vk) : tri_voxel_candidate(a, b, c, vi, vj, vk);
                }
                bal = __ballot_sync(0xffffffffu, hit);
                if (!EMIT && stored && lane == 0) pb[idx0 >> 5] = bal;
            }
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

// exact 64-bit candidate-pair total of every instance (block per instance)
__global__ void k_inst_pair_totals(const uint32_t* __restrict__ cnt, const BInst* __restrict__ inst,
                                   unsigned long long* __restrict__ out) {
    const BInst I = inst[blockIdx.x];
    unsigned long long acc = 0;
    for (uint32_t p = threadIdx.x; p < I.num_prims; p += blockDim.x) acc += cnt[I.prim_begin + p];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out + blockIdx.x, acc);
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

// Buffers of the pair stages (candidate pairs, sort, segments, per-voxel temporaries and
// the LoD scratch), shared by the groups of one primitive kind: the groups run one after
// the other on that kind's stream.  Grown while the groups are planned.
struct Pool {
    uint32_t *k0 = nullptr, *v0 = nullptr, *k1 = nullptr, *v1 = nullptr, *flags = nullptr, *idx = nullptr;
    uint32_t* hist = nullptr;
    char* so = nullptr;                                   // mask 64 + mass 4 + moment 24 per segment
    uint32_t *seg_key = nullptr, *seg_nonzero = nullptr, *dst = nullptr, *starts = nullptr;
    size_t pairs = 0, hist_words = 0, segs = 0;           // capacities
};

// One group of instances of one kind: planned, captured and replayed as one pipeline.
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
    std::vector<uint32_t> host_counts, host_starts;
    Pool* pool = nullptr;
    BInst* dinst = nullptr;
    uint8_t* inst_of = nullptr;
    float4 *r0 = nullptr, *r1 = nullptr, *r2 = nullptr;
    uint32_t *cnt = nullptr, *offs = nullptr, *fs = nullptr;
    uint32_t* ballots = nullptr;            // the count pass's hit ballots (NULL: emit tests again)
    uint32_t* part = nullptr;
    uint32_t* counters = nullptr;           // 64 words
    uint32_t* inst_start = nullptr;         // [(Lmax + 1)][ninst + 1]
    vx_level lv[kMaxLevels + 1];
    uint16_t* linst[kMaxLevels + 1];
    void* stats[kMaxLevels + 1] = {};      // K > 1: lobe statistics of each level (none for 0)
    uint32_t* work[kMaxLevels + 1] = {};   // K > 1: parents listed for clustering
    uint32_t cap_pairs = 0, cap_seg = 0, cap_v[kMaxLevels + 1];
    uint32_t plan_pairs = 0;                   // candidate pairs measured by the planning run
    // launch shapes picked by timing candidates on the planning run (autotuner)
    int red_bpsm = 0;                          // reduce kernel: resident blocks per SM
    int red_cand[5] = {};                      // the candidates timed, and their times
    float red_ms[5] = {};
    int tier[kMaxLevels + 1];                  // clustering tier per level (-1: by parent count)
    float tier_ms[kMaxLevels + 1][3] = {};
    SubBatch() {
        for (int& t : tier) t = -1;
    }
};

}  // namespace

struct vx_batch {
    vx_context* ctx = nullptr;
    std::vector<SubBatch> groups[2];   // per kind (0: triangles, 1: fibers), instances in order
    Pool pool[2];
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
    std::vector<int> kind_of, group_of, local_of;   // instance -> (kind, group, index in the group)
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

// Grows a pool buffer to at least `bytes` (its previous contents are not kept).
vx_status pool_grow(vx_batch* b, void** p, size_t bytes, cudaStream_t s) {
    if (*p) vx_dev_free(b->ctx, *p, s);
    *p = vx_dev_alloc(b->ctx, bytes, s);
    return *p ? VX_OK : VX_ERR_OUT_OF_MEMORY;
}

vx_status pool_pairs(vx_batch* b, Pool& P, size_t pairs, size_t hist_words, cudaStream_t s) {
    if (pairs > P.pairs) {
        for (uint32_t** q : {&P.k0, &P.v0, &P.k1, &P.v1, &P.flags, &P.idx})
            VX_TRY(pool_grow(b, (void**)q, pairs * 4, s));
        P.pairs = pairs;
    }
    if (hist_words > P.hist_words) {
        VX_TRY(pool_grow(b, (void**)&P.hist, hist_words * 4, s));
        P.hist_words = hist_words;
    }
    return VX_OK;
}

vx_status pool_segs(vx_batch* b, Pool& P, size_t segs, cudaStream_t s) {
    if (segs <= P.segs) return VX_OK;
    VX_TRY(pool_grow(b, (void**)&P.so, segs * (64 + 4 + 24), s));
    for (uint32_t** q : {&P.seg_key, &P.seg_nonzero, &P.dst}) VX_TRY(pool_grow(b, (void**)q, segs * 4, s));
    VX_TRY(pool_grow(b, (void**)&P.starts, (segs + 2) * 4, s));
    P.segs = segs;
    return VX_OK;
}

SegOut pool_segout(const Pool& P) {
    SegOut o;
    o.mask = (uint64_t*)P.so;
    o.moment = (float*)(P.so + P.segs * 64);
    o.mass = (float*)(P.so + P.segs * 88);
    o.key = P.seg_key;
    o.nonzero = P.seg_nonzero;
    return o;
}

uint32_t with_headroom(uint32_t n, float h) {
    double x = (double)n * (1.0 + (double)h) + 1024.0;
    return x > 4.0e9 ? 0xffffffffu : (uint32_t)x;
}

// Mean device time of `reps` runs of fn() on stream s (CUDA events; synchronises).
template <class F>
vx_status time_launches(cudaStream_t s, int reps, F fn, float* ms) {
    cudaEvent_t a = nullptr, e = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&e) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return VX_ERR_CUDA;
    }
    cudaError_t r = cudaEventRecord(a, s);
    for (int i = 0; i < reps && r == cudaSuccess; ++i) r = fn();
    if (r == cudaSuccess) r = cudaEventRecord(e, s);
    if (r == cudaSuccess) r = cudaEventSynchronize(e);
    if (r == cudaSuccess) r = cudaEventElapsedTime(ms, a, e);
    cudaEventDestroy(a);
    cudaEventDestroy(e);
    if (r != cudaSuccess) return VX_ERR_CUDA;
    *ms /= (float)reps;
    return VX_OK;
}

// Candidate pairs of every instance of one kind (prep and count over all of its primitives,
// in temporary buffers), for grouping the instances into passes.  Synchronises the stream.
vx_status instance_pairs(vx_batch* b, bool fiber, const vx_primitives* prims, const std::vector<BInst>& inst,
                         uint32_t np, int64_t F, cudaStream_t s, std::vector<uint64_t>* pairs) {
    vx_context* ctx = b->ctx;
    const int ninst = (int)inst.size();
    std::vector<void*> tmp;
    vx_status st = VX_OK;
    auto get = [&](size_t bytes) -> void* {
        void* p = vx_dev_alloc(ctx, bytes, s);
        if (p) tmp.push_back(p); else st = VX_ERR_OUT_OF_MEMORY;
        return p;
    };
    BInst* dinst = (BInst*)get(sizeof(BInst) * ninst);
    uint8_t* inst_of = (uint8_t*)get((size_t)np + 16);
    float4* r0 = (float4*)get((size_t)np * 16);
    float4* r1 = (float4*)get((size_t)np * 16);
    float4* r2 = fiber ? nullptr : (float4*)get((size_t)np * 16);
    uint32_t* cnt = (uint32_t*)get((size_t)np * 4);
    uint32_t* fs = (uint32_t*)get((size_t)(fiber ? F : 1) * 4 + 16);
    uint32_t* part = (uint32_t*)get((std::max<size_t>(np, (size_t)(fiber ? F : 1)) / 2048 + 64) * 4);
    uint32_t* C = (uint32_t*)get(64 * 4);
    unsigned long long* tot = (unsigned long long*)get((size_t)ninst * 8);
    cudaError_t e = cudaSuccess;
    if (st == VX_OK) {
        e = cudaMemcpyAsync(dinst, inst.data(), sizeof(BInst) * ninst, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(C, 0, 64 * 4, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(tot, 0, (size_t)ninst * 8, s);
        if (e == cudaSuccess && fiber) {
            k_fiber_seg_counts<<<gf((size_t)F, 256, 1u << 30), 256, 0, s>>>(prims->fiber_offsets, F, prims->num_ctrl, fs,
                                                                             C + C_ERR);
            e = vx_scan_u32_scratch(fs, fs, (uint32_t)F, C + C_SEGTOT, part, s);
            if (e == cudaSuccess)
                k_bprep_fibers<<<gf(np, 256, 1u << 30), 256, 0, s>>>((const float4*)prims->ctrl, prims->num_ctrl,
                                                                     prims->fiber_offsets, fs, F, prims->weights, np,
                                                                     dinst, ninst, r0, r1, inst_of, C + C_ERR);
        } else if (e == cudaSuccess) {
            k_bprep_tris<<<gf(np, 256, 1u << 30), 256, 0, s>>>((const float4*)prims->tri_verts, prims->weights, np,
                                                               dinst, ninst, r0, r1, r2, inst_of, C + C_ERR);
        }
        const unsigned cblocks = (unsigned)std::min<size_t>((np + EMIT_WARPS - 1) / EMIT_WARPS, (size_t)vx::kSMs * 64);
        if (e == cudaSuccess) {
            if (fiber)
                k_bcandidates<true, false><<<cblocks, EMIT_WARPS * 32, 0, s>>>(r0, r1, r2, np, dinst, inst_of, cnt,
                                                                               nullptr, 0, nullptr, nullptr, nullptr);
            else
                k_bcandidates<false, false><<<cblocks, EMIT_WARPS * 32, 0, s>>>(r0, r1, r2, np, dinst, inst_of, cnt,
                                                                                nullptr, 0, nullptr, nullptr, nullptr);
            k_inst_pair_totals<<<ninst, 256, 0, s>>>(cnt, dinst, tot);
            e = cudaGetLastError();
        }
        std::vector<unsigned long long> h(ninst);
        uint32_t err = 0, segtot = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), tot, (size_t)ninst * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&err, C + C_ERR, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&segtot, C + C_SEGTOT, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            vx_record_cuda_error(ctx, e, "instance pair counts");
            st = VX_ERR_CUDA;
        } else if (err || (fiber && segtot != np)) {
            st = VX_ERR_INVALID_ARG;
        } else {
            pairs->assign(h.begin(), h.end());
        }
    }
    for (void* p : tmp) vx_dev_free(ctx, p, s);
    return st;
}

// Enqueue the pipeline of one sub-batch.  plan: synchronise after each counting stage,
// allocate the buffers it needs (capacity = measured count + headroom) and record them;
// otherwise only kernels are enqueued (capturable).  *nl counts the launches.
vx_status enqueue(vx_batch* b, SubBatch& S, cudaStream_t s, bool plan, int64_t* nl) {
    if (S.np == 0) return VX_OK;
    vx_context* ctx = b->ctx;
    Pool& PL = *S.pool;
    uint32_t* C = S.counters;
    uint32_t* host = (uint32_t*)ctx->host_pin;
    const unsigned blk = vx::kSMs * 16;
    auto readback = [&](int word) -> uint32_t {
        if (vx_readback_async(ctx, 0, C + word, 4, s) != VX_OK) return 0xffffffffu;
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
        k_tangent_terms<<<gf(S.np, 256, 1u << 30), 256, 0, s>>>(S.r0, S.r1, S.np, S.r2);
        *nl += 6;
    } else {
        k_bprep_tris<<<gf(S.np, 256, 1u << 30), 256, 0, s>>>((const float4*)S.tri, S.weights, S.np, S.dinst,
                                                             S.ninst, S.r0, S.r1, S.r2, S.inst_of, C + C_ERR);
        *nl += 1;
    }
    // ---- candidates ----------------------------------------------------------------------
    const unsigned cblocks = (unsigned)std::min<size_t>((S.np + EMIT_WARPS - 1) / EMIT_WARPS, (size_t)vx::kSMs * 64);
    if (S.fiber)
        k_bcandidates<true, false><<<cblocks, EMIT_WARPS * 32, 0, s>>>(S.r0, S.r1, S.r2, S.np, S.dinst, S.inst_of,
                                                                       S.cnt, nullptr, 0, nullptr, nullptr, S.ballots);
    else
        k_bcandidates<false, false><<<cblocks, EMIT_WARPS * 32, 0, s>>>(S.r0, S.r1, S.r2, S.np, S.dinst, S.inst_of,
                                                                        S.cnt, nullptr, 0, nullptr, nullptr, S.ballots);
    if (vx_scan_u32_scratch(S.cnt, S.offs, S.np, C + C_PAIRS_TOT, S.part, s) != cudaSuccess) return VX_ERR_CUDA;
    *nl += 4;
    if (plan) {
        const uint32_t err = readback(C_ERR);
        if (err) return VX_ERR_INVALID_ARG;
        const uint32_t np = readback(C_PAIRS_TOT);
        if (np >= 0x80000000u) return VX_ERR_CAPACITY;
        S.plan_pairs = np;
        S.cap_pairs = with_headroom(np, b->headroom);
        const uint32_t nt = (S.cap_pairs + 4095) / 4096;
        const size_t hn = (size_t)256 * nt;
        VX_TRY(pool_pairs(b, PL, S.cap_pairs, hn, s));
        // scan partials: the largest scanned array is max(hist, pairs)
        const size_t mx = std::max<size_t>(hn, S.cap_pairs);
        VX_TRY(balloc(b, (void**)&S.part, (mx / 2048 + 64) * 4, s));
    }
    k_clamp<<<1, 1, 0, s>>>(C + C_PAIRS_TOT, S.cap_pairs, C + C_PAIRS, C + C_ERR);
    if (S.fiber)
        k_bcandidates<true, true><<<cblocks, EMIT_WARPS * 32, 0, s>>>(S.r0, S.r1, S.r2, S.np, S.dinst, S.inst_of,
                                                                      nullptr, S.offs, S.cap_pairs, PL.k0, PL.v0,
                                                                      S.ballots);
    else
        k_bcandidates<false, true><<<cblocks, EMIT_WARPS * 32, 0, s>>>(S.r0, S.r1, S.r2, S.np, S.dinst, S.inst_of,
                                                                       nullptr, S.offs, S.cap_pairs, PL.k0, PL.v0,
                                                                       S.ballots);
    k_pad<<<blk, 256, 0, s>>>(PL.k0, PL.v0, C + C_PAIRS, S.cap_pairs);
    *nl += 3;
    // ---- sort by (instance, key) ------------------------------------------------------------
    uint32_t *k0 = PL.k0, *v0 = PL.v0, *k1 = PL.k1, *v1 = PL.v1;
    if (vx_radix_sort_u32_scratch(&k0, &v0, &k1, &v1, S.cap_pairs, S.key_bits, S.inst_of, PL.hist, S.part, s) !=
        cudaSuccess)
        return VX_ERR_CUDA;
    *nl += 5 * ((S.key_bits + 7) / 8 + 1);
    // ---- segments ---------------------------------------------------------------------------
    k_bhead_flags<<<gf(S.cap_pairs, 256, blk), 256, 0, s>>>(k0, v0, S.inst_of, C + C_PAIRS, S.cap_pairs, PL.flags);
    if (vx_scan_u32_scratch(PL.flags, PL.idx, S.cap_pairs, C + C_SEG_TOT, S.part, s) != cudaSuccess) return VX_ERR_CUDA;
    *nl += 4;
    if (plan) {
        const uint32_t ns = readback(C_SEG_TOT);
        S.cap_seg = std::min(with_headroom(ns, b->headroom), S.cap_pairs);
        VX_TRY(pool_segs(b, PL, S.cap_seg, s));
    }
    const SegOut seg = pool_segout(PL);
    k_clamp<<<1, 1, 0, s>>>(C + C_SEG_TOT, S.cap_seg, C + C_SEG, C + C_ERR);
    k_bhead_starts<<<gf(S.cap_pairs, 256, blk), 256, 0, s>>>(k0, v0, S.inst_of, C + C_PAIRS, PL.idx, C + C_SEG_TOT,
                                                             S.cap_seg, PL.starts);
    // ---- per-voxel reduction ------------------------------------------------------------------
    // resident blocks taking voxels from a counter (zeroed by a node of the graph)
    auto launch_reduce = [&](int bpsm) -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(C + C_TAKE, 0, 4, s);
        if (e != cudaSuccess) return e;
        const unsigned rblocks =
            (unsigned)std::min<size_t>((S.cap_seg + RED_WARPS - 1) / RED_WARPS, (size_t)vx::kSMs * bpsm);
        if (S.fiber)
            k_reduce_fibers<<<std::max(rblocks, 1u), RED_WARPS * 32, 0, s>>>(k0, v0, PL.starts, C + C_SEG, S.r0, S.r1,
                                                                              S.r2, seg, 0, 0, 0, C + C_TAKE);
        else
            k_reduce_tris<<<std::max(rblocks, 1u), RED_WARPS * 32, 0, s>>>(k0, v0, PL.starts, C + C_SEG, S.r0, S.r1,
                                                                            S.r2, seg, 0, 0, 0, C + C_TAKE);
        return cudaGetLastError();
    };
    if (S.red_bpsm == 0) S.red_bpsm = S.fiber ? 7 : 32;
    if (launch_reduce(S.red_bpsm) != cudaSuccess) return VX_ERR_CUDA;
    if (plan) {
        // autotuner: time the reduce at each candidate grid on the planning run's pairs (every
        // grid gives the same outputs) and keep the fastest
        static const int fib_c[5] = {3, 4, 5, 6, 7}, tri_c[5] = {4, 8, 16, 24, 32};
        const int* cand = S.fiber ? fib_c : tri_c;
        float best = 0.0f;
        for (int c = 0; c < 5; ++c) {
            float ms = 0.0f;
            VX_TRY(time_launches(s, 2, [&]() { return launch_reduce(cand[c]); }, &ms));
            S.red_cand[c] = cand[c];
            S.red_ms[c] = ms;
            if (c == 0 || ms < best) {
                best = ms;
                S.red_bpsm = cand[c];
            }
        }
    }
    // non-empty flags beyond the clamped segment count read as zero in the compaction scan
    k_zero_tail<<<blk, 256, 0, s>>>(seg.nonzero, C + C_SEG, S.cap_seg);
    if (vx_scan_u32_scratch(seg.nonzero, PL.dst, S.cap_seg, C + C_VOX_TOT, S.part, s) != cudaSuccess)
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
    k_bfinalize<<<gf(S.cap_seg, 256, blk), 256, 0, s>>>(seg, C + C_SEG, PL.dst, S.cap_v[0], PL.starts, v0, S.inst_of,
                                                        S.lv[0], S.linst[0]);
    k_inst_offsets<<<(S.ninst + 1 + 127) / 128, 128, 0, s>>>(S.linst[0], C + C_VOX, S.ninst, S.inst_start);
    *nl += 3;
    // ---- coarser levels -------------------------------------------------------------------------
    for (int l = 1; l <= S.Lmax; ++l) {
        const uint32_t* nprev = (l == 1) ? C + C_VOX : C + C_LVL + (l - 1);
        if (plan) {
            // exact parent count of this level: run the flag scan once to measure it
            k_bparent_count_flags<<<gf(S.cap_v[l - 1], 256, blk), 256, 0, s>>>(S.lv[l - 1].keys, S.linst[l - 1], nprev,
                                                                               S.cap_v[l - 1], PL.flags);
            if (vx_scan_u32_scratch(PL.flags, PL.idx, S.cap_v[l - 1], C + C_LVL + 16 + l, S.part, s) != cudaSuccess)
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
                                C + C_LVL + l, S.cap_v[l], PL.flags, PL.idx, PL.starts, S.part, C + C_LVL + 16 + l,
                                C + C_ERR, b->dirs4, b->n_dirs, S.work[l], C + C_CLUSTER,
                                l > 1 ? S.stats[l - 1] : nullptr, S.stats[l], b->merge, S.tier[l], s) != cudaSuccess)
            return VX_ERR_CUDA;
        if (plan && b->K > 1) {
            // autotuner: time the three clustering tiers on this level's parents (same result)
            float best = 0.0f;
            for (int t = 0; t < 3; ++t) {
                float ms = 0.0f;
                VX_TRY(time_launches(s, 2, [&]() {
                    return vx_lod_cluster_batched(&S.lv[l - 1], &S.lv[l], PL.starts, S.work[l], C + C_CLUSTER,
                                                  b->dirs4, b->n_dirs, l > 1 ? S.stats[l - 1] : nullptr, S.stats[l],
                                                  S.cap_v[l], b->merge, t, s);
                }, &ms));
                S.tier_ms[l][t] = ms;
                if (t == 0 || ms < best) {
                    best = ms;
                    S.tier[l] = t;
                }
            }
        }
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
    b->group_of.resize(num_instances);
    b->local_of.resize(num_instances);
    vx_status st = VX_OK;
    auto fail = [&](vx_status e) {
        vx_batch_destroy(b);
        return e;
    };
    // instance tables per kind, checked on the host (ranges contiguous and in order)
    uint32_t next[2] = {0, 0};
    int64_t next_fiber = 0;
    std::vector<BInst> kinst[2];
    std::vector<int64_t> kfib[2];                 // fibers: first fiber of each instance
    std::vector<int> kidx[2];                     // batch index of each instance of a kind
    for (int i = 0; i < num_instances; ++i) {
        const vx_instance& I = instances[i];
        const int k = I.kind == VX_FIBERS ? 1 : 0;
        if (I.kind != VX_FIBERS && I.kind != VX_TRIANGLES) return fail(VX_ERR_INVALID_ARG);
        const uint32_t R = I.grid.resolution;
        if (R == 0 || (R & (R - 1)) != 0 || !(I.grid.voxel_size > 0.0f)) return fail(VX_ERR_INVALID_ARG);
        if (R > 1024 || I.grid.sub_res != 8) return fail(VX_ERR_UNSUPPORTED);
        if (I.prim_begin != (int64_t)next[k] || I.num_prims < 0) return fail(VX_ERR_INVALID_ARG);
        if ((int64_t)next[k] + I.num_prims > 0xffffffffll) return fail(VX_ERR_CAPACITY);
        if (k == 1 && (I.fiber_begin != next_fiber || I.num_fibers < 0)) return fail(VX_ERR_INVALID_ARG);
        if (kinst[k].size() >= 255) return fail(VX_ERR_UNSUPPORTED);
        BInst bi;
        bi.o[0] = I.grid.origin[0]; bi.o[1] = I.grid.origin[1]; bi.o[2] = I.grid.origin[2];
        bi.s = 1.0f / I.grid.voxel_size;
        bi.R = (int)R;
        int L = 0;
        while ((1u << L) < R) ++L;
        bi.L = L;
        bi.prim_begin = (uint32_t)I.prim_begin;
        bi.num_prims = (uint32_t)I.num_prims;
        kinst[k].push_back(bi);
        kfib[k].push_back(I.fiber_begin);
        kidx[k].push_back(i);
        b->kind_of[i] = k;
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
        if ((st = balloc(b, (void**)&b->dirs4, vx_dirs_bytes(lod->n_samples), s)) != VX_OK) return fail(st);
        if (vx_lod_batched_prepare(K, lod->dirs, lod->n_samples, b->dirs4, s) != cudaSuccess) return fail(VX_ERR_CUDA);
    }
    // Groups: consecutive instances of a kind whose candidate pairs fit one pass (with the
    // headroom), measured by counting every instance once.
    const uint64_t pass_limit = (uint64_t)std::min<int64_t>(ctx->max_pairs, 0x7fffffffll);
    const uint64_t group_limit =
        (uint64_t)std::max(0.0, ((double)pass_limit - 1024.0) / (1.0 + (double)headroom));
    for (int k = 0; k < 2; ++k) {
        const int ninst = (int)kinst[k].size();
        if (next[k] == 0 || ninst == 0) continue;
        std::vector<uint64_t> pairs;
        if ((st = instance_pairs(b, k == 1, k == 1 ? fibers : tris, kinst[k], next[k], k == 1 ? next_fiber : 0, s,
                                 &pairs)) != VX_OK)
            return fail(st);
        std::vector<std::pair<int, int>> ranges;   // [first, last) instance of each group
        int first = 0;
        uint64_t acc = 0;
        for (int i = 0; i < ninst; ++i) {
            if (pairs[i] > group_limit) return fail(VX_ERR_CAPACITY);   // one instance over one pass
            if (i > first && acc + pairs[i] > group_limit) {
                ranges.push_back({first, i});
                first = i;
                acc = 0;
            }
            acc += pairs[i];
        }
        ranges.push_back({first, ninst});
        b->groups[k].resize(ranges.size());
        for (size_t g = 0; g < ranges.size(); ++g) {
            SubBatch& S = b->groups[k][g];
            S.fiber = k == 1;
            S.pool = &b->pool[k];
            const int i0 = ranges[g].first, i1 = ranges[g].second;
            const uint32_t pbase = kinst[k][i0].prim_begin;
            for (int i = i0; i < i1; ++i) {
                BInst bi = kinst[k][i];
                bi.prim_begin -= pbase;
                S.hinst.push_back(bi);
                S.Lmax = std::max(S.Lmax, bi.L);
                S.key_bits = std::max(S.key_bits, 3 * bi.L);
                S.np += bi.num_prims;
                b->group_of[kidx[k][i]] = (int)g;
                b->local_of[kidx[k][i]] = S.ninst++;
            }
            if (S.fiber) {
                const int64_t f0 = kfib[k][i0];
                const int64_t f1 = (i1 < ninst) ? kfib[k][i1] : next_fiber;
                S.ctrl = fibers->ctrl;
                S.num_ctrl = fibers->num_ctrl;
                S.off = fibers->fiber_offsets + f0;
                S.F = f1 - f0;
                S.weights = fibers->weights ? fibers->weights + pbase : nullptr;
            } else {
                S.tri = tris->tri_verts + (size_t)pbase * 12;
                S.weights = tris->weights ? tris->weights + pbase : nullptr;
            }
        }
    }
    for (int k = 0; k < 2; ++k) {
        for (SubBatch& S : b->groups[k]) {
            if (S.np == 0) continue;
            if ((st = balloc(b, (void**)&S.dinst, sizeof(BInst) * S.ninst, s)) != VX_OK) return fail(st);
            if (cudaMemcpyAsync(S.dinst, S.hinst.data(), sizeof(BInst) * S.ninst, cudaMemcpyHostToDevice, s) !=
                cudaSuccess)
                return fail(VX_ERR_CUDA);
            if ((st = balloc(b, (void**)&S.inst_of, (size_t)S.np + 16, s)) != VX_OK) return fail(st);
            if ((st = balloc(b, (void**)&S.r0, (size_t)S.np * 16, s)) != VX_OK) return fail(st);
            if ((st = balloc(b, (void**)&S.r1, (size_t)S.np * 16, s)) != VX_OK) return fail(st);
            // triangles: the third vertex records; fibers: the tangent terms (two float4 each)
            if ((st = balloc(b, (void**)&S.r2, (size_t)S.np * (S.fiber ? 32 : 16), s)) != VX_OK) return fail(st);
            if ((st = balloc(b, (void**)&S.cnt, (size_t)S.np * 4, s)) != VX_OK) return fail(st);
            if ((st = balloc(b, (void**)&S.offs, (size_t)S.np * 4, s)) != VX_OK) return fail(st);
            // ballots for the emit pass, when they take at most 2 GB
            if ((size_t)S.np * CAND_BALLOTS * 4 <= ((size_t)2 << 30) &&
                (st = balloc(b, (void**)&S.ballots, (size_t)S.np * CAND_BALLOTS * 4, s)) != VX_OK)
                return fail(st);
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
        for (SubBatch& S : b->groups[0])
            if (st == VX_OK) st = enqueue(b, S, b->cap_stream2, false, &nl);
        for (SubBatch& S : b->groups[1])
            if (st == VX_OK) st = enqueue(b, S, b->cap_stream, false, &nl);
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
    SubBatch& S = b->groups[k][b->group_of[instance]];
    const BInst& I = S.hinst[li];
    if (level > I.L) return VX_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (!b->host_valid) {
        for (int kk = 0; kk < 2; ++kk) {
            for (SubBatch& T : b->groups[kk]) {
                T.host_counts.assign(64, 0);
                T.host_starts.assign((size_t)(kMaxLevels + 1) * (T.ninst + 1), 0);
                if (T.np == 0) continue;
                if (cudaMemcpyAsync(T.host_counts.data(), T.counters, 64 * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                    cudaMemcpyAsync(T.host_starts.data(), T.inst_start, T.host_starts.size() * 4,
                                    cudaMemcpyDeviceToHost, s) != cudaSuccess)
                    return VX_ERR_CUDA;
            }
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) return VX_ERR_CUDA;
        b->host_valid = true;
    }
    const uint32_t err = S.host_counts[C_ERR];
    if (err & 2u) return VX_ERR_CAPACITY;
    if (err & 1u) return VX_ERR_INVALID_ARG;
    const uint32_t* st = S.host_starts.data() + (size_t)level * (S.ninst + 1);
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

extern "C" vx_status vx_batch_query(const vx_batch* b, vx_batch_info* info) {
    if (!b || !info) return VX_ERR_INVALID_ARG;
    memset(info, 0, sizeof(*info));
    for (int k = 0; k < 2; ++k) {
        info->num_groups[k] = (int32_t)b->groups[k].size();
        for (int l = 0; l < 12; ++l) info->cluster_tier[k][l] = -1;
        const SubBatch* big = nullptr;
        for (const SubBatch& S : b->groups[k])
            if (!big || S.cap_pairs > big->cap_pairs) big = &S;
        if (!big) continue;
        info->max_group_pairs[k] = big->plan_pairs;
        info->reduce_blocks_per_sm[k] = big->red_bpsm;
        for (int c = 0; c < 5; ++c) {
            info->reduce_candidates[k][c] = big->red_cand[c];
            info->reduce_ms[k][c] = big->red_ms[c];
        }
        for (int l = 0; l <= kMaxLevels && l < 12; ++l) {
            info->cluster_tier[k][l] = big->tier[l];
            for (int t = 0; t < 3; ++t) info->cluster_ms[k][l][t] = big->tier_ms[l][t];
        }
    }
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
    for (Pool& P : b->pool)
        for (void* p : {(void*)P.k0, (void*)P.v0, (void*)P.k1, (void*)P.v1, (void*)P.flags, (void*)P.idx,
                        (void*)P.hist, (void*)P.so, (void*)P.seg_key, (void*)P.seg_nonzero, (void*)P.dst,
                        (void*)P.starts})
            if (p) vx_dev_free(b->ctx, p, s);
    cudaStreamSynchronize(s);
    delete b;
}
