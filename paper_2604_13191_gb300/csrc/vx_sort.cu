// vx_sort.cu -- device prefix sum and stable LSD radix sort of (uint32 key, uint32 value).
//
// The sort orders candidate (voxel key, primitive id) pairs by Morton key, keeping
// primitive-id order inside each key (stability), which is what makes the per-voxel
// reductions order-deterministic (the paper sorts samples by block id, Sec. 3.3).
#include <algorithm>

#include "vx_internal.cuh"

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

constexpr int SORT_THREADS = 256;
constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr int SORT_ITEMS = 16;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;
constexpr int RADIX = 256;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread (256 threads); returns the block total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* smem, uint32_t& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = warp_incl_scan(v);
    if (lane == 31) smem[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t x = (lane < SCAN_THREADS / 32) ? smem[lane] : 0u;
        uint32_t xi = warp_incl_scan(x);
        if (lane < SCAN_THREADS / 32) smem[lane] = xi - x;
        if (lane == SCAN_THREADS / 32 - 1) smem[SCAN_THREADS / 32] = xi;
    }
    __syncthreads();
    uint32_t r = smem[w] + inc - v;
    total = smem[SCAN_THREADS / 32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const uint32_t* __restrict__ in,
                                                              uint32_t n, uint32_t* __restrict__ part) {
    __shared__ uint32_t sm[SCAN_THREADS / 32 + 1];
    const size_t base = (size_t)blockIdx.x * SCAN_TILE;
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        size_t e = base + (size_t)j * SCAN_THREADS + threadIdx.x;
        if (e < n) s += in[e];
    }
    uint32_t tot;
    block_excl_scan(s, sm, tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// Single-block exclusive scan of the block partials (any length).
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_partials(uint32_t* part, uint32_t nb,
                                                                uint32_t* total) {
    __shared__ uint32_t sm[SCAN_THREADS / 32 + 1];
    uint32_t carry = 0;
    for (uint32_t b = 0; b < nb; b += SCAN_TILE) {
        uint32_t v[SCAN_ITEMS];
        uint32_t s = 0;
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; ++j) {
            uint32_t e = b + threadIdx.x * SCAN_ITEMS + j;
            v[j] = (e < nb) ? part[e] : 0u;
            s += v[j];
        }
        uint32_t tot;
        uint32_t off = block_excl_scan(s, sm, tot);
        uint32_t run = carry + off;
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; ++j) {
            uint32_t e = b + threadIdx.x * SCAN_ITEMS + j;
            if (e < nb) part[e] = run;
            run += v[j];
        }
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(const uint32_t* in, uint32_t* out, uint32_t n,
                                                            const uint32_t* __restrict__ part) {
    __shared__ uint32_t sm[SCAN_THREADS / 32 + 1];
    const size_t base = (size_t)blockIdx.x * SCAN_TILE;
    uint32_t v[SCAN_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        size_t e = base + (size_t)threadIdx.x * SCAN_ITEMS + j;
        v[j] = (e < n) ? in[e] : 0u;
        s += v[j];
    }
    uint32_t tot;
    uint32_t run = block_excl_scan(s, sm, tot) + part[blockIdx.x];
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        size_t e = base + (size_t)threadIdx.x * SCAN_ITEMS + j;
        if (e < n) out[e] = run;
        run += v[j];
    }
}

// Single-block exclusive scan of a short array (a few tiles): the tiles in order with a
// running carry, each thread on SCAN_ITEMS consecutive elements (in place allowed: a thread
// reads its elements before it writes them); *total (optional) receives the sum.
constexpr uint32_t SCAN_SMALL_TILES = 16;
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_small(const uint32_t* in, uint32_t* out, uint32_t n,
                                                             uint32_t* total) {
    __shared__ uint32_t sm[SCAN_THREADS / 32 + 1];
    uint32_t carry = 0;
    for (uint32_t b = 0; b < n; b += SCAN_TILE) {
        uint32_t v[SCAN_ITEMS];
        uint32_t s = 0;
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; ++j) {
            const uint32_t e = b + threadIdx.x * SCAN_ITEMS + j;
            v[j] = (e < n) ? in[e] : 0u;
            s += v[j];
        }
        uint32_t tot;
        uint32_t run = carry + block_excl_scan(s, sm, tot);
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; ++j) {
            const uint32_t e = b + threadIdx.x * SCAN_ITEMS + j;
            if (e < n) out[e] = run;
            run += v[j];
        }
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

// ---- segment starts ---------------------------------------------------------------
// Heads of the runs of equal keys in a sorted array: element e is a head when e == 0 or
// keys[e] != keys[e - 1].  A thread takes SCAN_ITEMS consecutive elements (as k_scan_down).
__device__ __forceinline__ uint32_t head_bits(const uint32_t* __restrict__ keys, uint32_t n, size_t e0) {
    static_assert(SCAN_ITEMS == 8, "two 16-byte loads per thread");
    uint32_t k[SCAN_ITEMS];
    if (e0 + SCAN_ITEMS <= n) {
        // e0 is a multiple of 8 and the key arrays are 256-byte aligned
        const uint4 x = __ldg(reinterpret_cast<const uint4*>(keys + e0));
        const uint4 y = __ldg(reinterpret_cast<const uint4*>(keys + e0) + 1);
        k[0] = x.x; k[1] = x.y; k[2] = x.z; k[3] = x.w;
        k[4] = y.x; k[5] = y.y; k[6] = y.z; k[7] = y.w;
    } else {
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; ++j) k[j] = e0 + j < n ? keys[e0 + j] : 0u;
    }
    uint32_t prev = e0 > 0 && e0 - 1 < n ? keys[e0 - 1] : 0u;
    uint32_t bits = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        const size_t e = e0 + j;
        if (e < n && (e == 0 || k[j] != prev)) bits |= 1u << j;
        prev = k[j];
    }
    return bits;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_seg_count(const uint32_t* __restrict__ keys, uint32_t n,
                                                            uint32_t* __restrict__ part) {
    __shared__ uint32_t sm[SCAN_THREADS / 32 + 1];
    const size_t e0 = (size_t)blockIdx.x * SCAN_TILE + (size_t)threadIdx.x * SCAN_ITEMS;
    uint32_t tot;
    block_excl_scan(__popc(head_bits(keys, n, e0)), sm, tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_seg_starts(const uint32_t* __restrict__ keys, uint32_t n,
                                                             const uint32_t* __restrict__ part,
                                                             const uint32_t* __restrict__ nseg,
                                                             uint32_t* __restrict__ starts) {
    __shared__ uint32_t sm[SCAN_THREADS / 32 + 1];
    const size_t e0 = (size_t)blockIdx.x * SCAN_TILE + (size_t)threadIdx.x * SCAN_ITEMS;
    uint32_t bits = head_bits(keys, n, e0);
    uint32_t tot;
    uint32_t idx = block_excl_scan(__popc(bits), sm, tot) + part[blockIdx.x];
    while (bits) {
        const int j = __ffs(bits) - 1;
        bits &= bits - 1;
        starts[idx++] = (uint32_t)(e0 + j);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) starts[*nseg] = n;
}

// ---- radix sort ----------------------------------------------------------------
// Digit of an element: bits [shift, shift + 8) of its key, or (LUT pass) a digit looked
// up from its value: lut[value], with 255 for the padding value 0xffffffff.
template <bool LUT>
__device__ __forceinline__ uint32_t radix_digit(uint32_t k, uint32_t v, int shift, uint32_t dmask,
                                                const uint8_t* __restrict__ lut) {
    if (LUT) return v == 0xffffffffu ? 255u : (uint32_t)lut[v];
    return (k >> shift) & dmask;
}

// RB buckets per pass (256: 8-bit digits; 512: 9-bit digits, three passes for a 27-bit key)
template <bool LUT, int RB>
__global__ void __launch_bounds__(SORT_THREADS) k_radix_hist(const uint32_t* __restrict__ keys,
                                                             const uint32_t* __restrict__ vals, uint32_t n,
                                                             int shift, uint32_t dmask, uint32_t nt,
                                                             const uint8_t* __restrict__ lut,
                                                             uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[RB];
    for (int d = threadIdx.x; d < RB; d += SORT_THREADS) h[d] = 0;
    __syncthreads();
    const size_t base = (size_t)blockIdx.x * SORT_TILE;
    if (!LUT && base + SORT_TILE <= n) {
        // a full tile: four consecutive keys per 16-byte load (the key arrays are 256-byte
        // aligned and a tile starts at a multiple of 4096 keys)
        const uint4* k4 = reinterpret_cast<const uint4*>(keys + base);
#pragma unroll
        for (int j = 0; j < SORT_ITEMS / 4; ++j) {
            const uint4 q = __ldg(k4 + (size_t)j * SORT_THREADS + threadIdx.x);
            atomicAdd(&h[(q.x >> shift) & dmask], 1u);
            atomicAdd(&h[(q.y >> shift) & dmask], 1u);
            atomicAdd(&h[(q.z >> shift) & dmask], 1u);
            atomicAdd(&h[(q.w >> shift) & dmask], 1u);
        }
    } else {
#pragma unroll 4
        for (int j = 0; j < SORT_ITEMS; ++j) {
            size_t e = base + (size_t)j * SORT_THREADS + threadIdx.x;
            if (e < n) atomicAdd(&h[radix_digit<LUT>(LUT ? 0u : keys[e], LUT ? vals[e] : 0u, shift, dmask, lut)], 1u);
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RB; d += SORT_THREADS) hist[(size_t)d * nt + blockIdx.x] = h[d];
}

// Stable scatter of one tile.  Each element's rank inside the tile (digit-major, original
// order within a digit) is found with per-warp running counters; the tile is then
// rearranged into that order in shared memory and written out with consecutive threads on
// consecutive elements, so that the writes of one digit's run are contiguous.
template <bool LUT, int RB>
__global__ void __launch_bounds__(SORT_THREADS, 3) k_radix_scatter(const uint32_t* __restrict__ keys,
                                                                const uint32_t* __restrict__ vals, uint32_t n,
                                                                int shift, uint32_t dmask, uint32_t nt,
                                                                const uint8_t* __restrict__ lut,
                                                                const uint32_t* __restrict__ hist,
                                                                uint32_t* __restrict__ okeys,
                                                                uint32_t* __restrict__ ovals) {
    static_assert(RB % SORT_THREADS == 0, "digits per thread");
    union Stage {
        uint32_t wcnt[SORT_WARPS][RB];           // ranking: per-warp counts, then warp offsets
        struct {
            uint32_t k[SORT_TILE], v[SORT_TILE];  // the tile in digit order
        } t;
    };
    __shared__ Stage st;
    __shared__ uint32_t gofs[RB];   // global start of the tile's run of each digit
    __shared__ uint32_t tofs[RB];   // start of each digit's run inside the tile
    __shared__ uint32_t scan_tmp[SORT_WARPS + 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < SORT_WARPS * RB; i += SORT_THREADS) (&st.wcnt[0][0])[i] = 0;
    for (int d = threadIdx.x; d < RB; d += SORT_THREADS) gofs[d] = hist[(size_t)d * nt + blockIdx.x];
    __syncthreads();
    const size_t tile0 = (size_t)blockIdx.x * SORT_TILE;
    const size_t base = tile0 + (size_t)w * (32 * SORT_ITEMS);
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t k[SORT_ITEMS], v[SORT_ITEMS], rk[SORT_ITEMS];
#pragma unroll
    for (int j = 0; j < SORT_ITEMS; ++j) {
        size_t e = base + (size_t)j * 32 + lane;
        bool valid = e < n;
        k[j] = valid ? keys[e] : 0u;
        v[j] = valid ? vals[e] : 0u;
        uint32_t d = valid ? radix_digit<LUT>(k[j], v[j], shift, dmask, lut) : (uint32_t)RB;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t r = 0;
        if (valid) r = st.wcnt[w][d] + __popc(peers & lt);
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) st.wcnt[w][d] += __popc(peers);
        __syncwarp();
        rk[j] = r;
    }
    __syncthreads();
    // warp offsets per digit (exclusive over warps) and the tile's count of each digit
    constexpr int DPT = RB / SORT_THREADS;
    uint32_t cnt[DPT];
#pragma unroll
    for (int i = 0; i < DPT; ++i) {
        const int d = threadIdx.x * DPT + i;
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < SORT_WARPS; ++ww) {
            const uint32_t t = st.wcnt[ww][d];
            st.wcnt[ww][d] = run;
            run += t;
        }
        cnt[i] = run;
    }
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < DPT; ++i) sum += cnt[i];
    uint32_t total;
    uint32_t ex = block_excl_scan(sum, scan_tmp, total);
#pragma unroll
    for (int i = 0; i < DPT; ++i) {
        tofs[threadIdx.x * DPT + i] = ex;
        ex += cnt[i];
    }
    __syncthreads();
    // tile-local positions (the counters are read before the tile overwrites them)
#pragma unroll
    for (int j = 0; j < SORT_ITEMS; ++j) {
        const size_t e = base + (size_t)j * 32 + lane;
        if (e < n) {
            const uint32_t d = radix_digit<LUT>(k[j], v[j], shift, dmask, lut);
            rk[j] += tofs[d] + st.wcnt[w][d];
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < SORT_ITEMS; ++j) {
        const size_t e = base + (size_t)j * 32 + lane;
        if (e < n) {
            st.t.k[rk[j]] = k[j];
            st.t.v[rk[j]] = v[j];
        }
    }
    __syncthreads();
    const uint32_t tn = (uint32_t)min((size_t)SORT_TILE, (size_t)n - tile0);
    for (uint32_t i = threadIdx.x; i < tn; i += SORT_THREADS) {
        const uint32_t kk = st.t.k[i], vv = st.t.v[i];
        const uint32_t d = radix_digit<LUT>(kk, vv, shift, dmask, lut);
        const uint32_t pos = gofs[d] + (i - tofs[d]);
        okeys[pos] = kk;
        ovals[pos] = vv;
    }
}

// ---- persistent scatter with double-buffered bulk copies ------------------------------
// A resident block takes tiles t, t + grid, ...; while it ranks and writes one tile, the next
// tile's keys and values stream into the other half of its shared memory through 1-D bulk
// async copies (cp.async.bulk, completion on an mbarrier).  Each wait is bounded: a wait that
// gives up sets bit 4 of *err, waits (bounded) for the block's own copies still in flight,
// and ends the block (the host then reports VX_ERR_TIMEOUT).
constexpr uint32_t PIPE_SPIN_LIMIT = 1u << 22;   // try_wait polls before a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// bounded wait for phase `parity` of the barrier; false when it gave up after `limit` polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit = PIPE_SPIN_LIMIT) {
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
// global -> shared bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

constexpr size_t pipe_smem(int rb) {
    return (size_t)2 * 2 * SORT_TILE * 4                 // two stages of keys + values
           + (size_t)SORT_WARPS * rb * 4                 // per-warp digit counters
           + (size_t)2 * rb * 4                          // gofs, tofs
           + 64;                                         // scan scratch, barriers
}

template <int RB>
__global__ void __launch_bounds__(SORT_THREADS, 2) k_radix_scatter_pipe(const uint32_t* __restrict__ keys,
                                                                      const uint32_t* __restrict__ vals, uint32_t n,
                                                                      int shift, uint32_t dmask, uint32_t nt,
                                                                      const uint32_t* __restrict__ hist,
                                                                      uint32_t* __restrict__ okeys,
                                                                      uint32_t* __restrict__ ovals,
                                                                      uint32_t* __restrict__ err) {
    static_assert(RB % SORT_THREADS == 0, "digits per thread");
    extern __shared__ __align__(128) unsigned char sm_raw[];
    // stage s: keys at sm + 2 s TILE, values right after them
    uint32_t* const stage0 = (uint32_t*)sm_raw;
    uint32_t (*wcnt)[RB] = reinterpret_cast<uint32_t (*)[RB]>((uint32_t*)sm_raw + 4 * SORT_TILE);
    uint32_t* gofs = (uint32_t*)sm_raw + 4 * SORT_TILE + SORT_WARPS * RB;
    uint32_t* tofs = gofs + RB;
    uint32_t* scan_tmp = tofs + RB;                       // SORT_WARPS + 1 words
    uint64_t* bar = reinterpret_cast<uint64_t*>(scan_tmp + 12);   // 8-byte aligned: two barriers
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    // a tile is loaded by bulk copies when it is whole (the last one may be short, and its
    // byte count a multiple of 4 only): else by the threads
    auto bulk_ok = [&](uint32_t t) { return (size_t)(t + 1) * SORT_TILE <= n; };
    auto issue = [&](uint32_t t, int st) {
        const size_t e0 = (size_t)t * SORT_TILE;
        uint32_t* sk = stage0 + (size_t)st * 2 * SORT_TILE;
        mbar_expect_tx(&bar[st], 2u * SORT_TILE * 4u);
        bulk_load(sk, keys + e0, SORT_TILE * 4u, &bar[st]);
        bulk_load(sk + SORT_TILE, vals + e0, SORT_TILE * 4u, &bar[st]);
    };
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0u, pending = 0u;   // bit s: the parity to wait for / a copy in flight, stage s
    if (threadIdx.x == 0 && blockIdx.x < nt && bulk_ok(blockIdx.x)) issue(blockIdx.x, 0);
    if (blockIdx.x < nt && bulk_ok(blockIdx.x)) pending |= 1u;
    bool lost = false;
    int st = 0;
    // this thread's digits' global offsets for the tile in hand, loaded one tile ahead (the
    // digit-major histogram puts a tile's offsets a stride nt apart)
    constexpr int DPG = RB / SORT_THREADS;
    uint32_t gcur[DPG];
#pragma unroll
    for (int i = 0; i < DPG; ++i)
        gcur[i] = blockIdx.x < nt ? hist[(size_t)(threadIdx.x + i * SORT_THREADS) * nt + blockIdx.x] : 0u;
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x, st ^= 1) {
        // the next tile streams into the other stage (its last reader finished: the loop ends
        // with a barrier); generic writes to that stage are ordered before the async copy
        const uint32_t tn = t + gridDim.x;
        if (tn < nt && bulk_ok(tn)) {
            if (threadIdx.x == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(tn, st ^ 1);
            }
            pending |= 1u << (st ^ 1);
        }
        uint32_t gnxt[DPG];
#pragma unroll
        for (int i = 0; i < DPG; ++i)
            gnxt[i] = tn < nt ? hist[(size_t)(threadIdx.x + i * SORT_THREADS) * nt + tn] : 0u;
        const size_t tile0 = (size_t)t * SORT_TILE;
        const uint32_t tn_items = (uint32_t)min((size_t)SORT_TILE, (size_t)n - tile0);
        uint32_t* const sk = stage0 + (size_t)st * 2 * SORT_TILE;
        uint32_t* const sv = sk + SORT_TILE;
        bool gave_up = false;
        if ((pending >> st) & 1u) {
            if (mbar_wait(&bar[st], (phase >> st) & 1u)) {
                phase ^= 1u << st;
                pending &= ~(1u << st);
            } else {
                gave_up = true;
            }
        } else {
            for (uint32_t i = threadIdx.x; i < tn_items; i += SORT_THREADS) {
                sk[i] = keys[tile0 + i];
                sv[i] = vals[tile0 + i];
            }
        }
        for (int i = threadIdx.x; i < SORT_WARPS * RB; i += SORT_THREADS) (&wcnt[0][0])[i] = 0;
#pragma unroll
        for (int i = 0; i < DPG; ++i) gofs[threadIdx.x + i * SORT_THREADS] = gcur[i];
        // the whole block leaves together when any thread's wait gave up
        if (__syncthreads_or(gave_up)) {
            lost = true;
            break;
        }
        // rank: per-warp running counters (stable within the tile)
        uint32_t k[SORT_ITEMS], v[SORT_ITEMS], rk[SORT_ITEMS];
        const uint32_t lb = (uint32_t)w * (32 * SORT_ITEMS);
#pragma unroll
        for (int j = 0; j < SORT_ITEMS; ++j) {
            const uint32_t e = lb + (uint32_t)j * 32 + lane;
            const bool valid = e < tn_items;
            k[j] = valid ? sk[e] : 0u;
            v[j] = valid ? sv[e] : 0u;
            const uint32_t d = valid ? ((k[j] >> shift) & dmask) : (uint32_t)RB;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            uint32_t r = 0;
            if (valid) r = wcnt[w][d] + __popc(peers & lt);
            __syncwarp();
            if (valid && lane == __ffs(peers) - 1) wcnt[w][d] += __popc(peers);
            __syncwarp();
            rk[j] = r;
        }
        __syncthreads();
        constexpr int DPT = RB / SORT_THREADS;
        uint32_t cnt[DPT];
#pragma unroll
        for (int i = 0; i < DPT; ++i) {
            const int d = threadIdx.x * DPT + i;
            uint32_t run = 0;
#pragma unroll
            for (int ww = 0; ww < SORT_WARPS; ++ww) {
                const uint32_t c = wcnt[ww][d];
                wcnt[ww][d] = run;
                run += c;
            }
            cnt[i] = run;
        }
        uint32_t sum = 0;
#pragma unroll
        for (int i = 0; i < DPT; ++i) sum += cnt[i];
        uint32_t total;
        uint32_t ex = block_excl_scan(sum, scan_tmp, total);
#pragma unroll
        for (int i = 0; i < DPT; ++i) {
            tofs[threadIdx.x * DPT + i] = ex;
            ex += cnt[i];
        }
        __syncthreads();
        // the tile in digit order, over the stage it was read from (every item is in registers)
#pragma unroll
        for (int j = 0; j < SORT_ITEMS; ++j) {
            const uint32_t e = lb + (uint32_t)j * 32 + lane;
            if (e < tn_items) {
                const uint32_t d = (k[j] >> shift) & dmask;
                const uint32_t pos = rk[j] + tofs[d] + wcnt[w][d];
                sk[pos] = k[j];
                sv[pos] = v[j];
            }
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < tn_items; i += SORT_THREADS) {
            const uint32_t kk = sk[i], vv = sv[i];
            const uint32_t d = (kk >> shift) & dmask;
            const uint32_t pos = gofs[d] + (i - tofs[d]);
            okeys[pos] = kk;
            ovals[pos] = vv;
        }
#pragma unroll
        for (int i = 0; i < DPG; ++i) gcur[i] = gnxt[i];
        __syncthreads();
    }
    if (lost) {
        if (threadIdx.x == 0) atomicOr(err, 4u);
        // the block's own copies still in flight land before it exits (bounded; a thread
        // whose wait succeeded has already cleared that stage's bit)
        for (int s2 = 0; s2 < 2; ++s2)
            if ((pending >> s2) & 1u) mbar_wait(&bar[s2], (phase >> s2) & 1u);
    }
}

// Self-test of the bounded wait: a barrier that expects bytes no copy will deliver, so the
// wait must give up after `limit` polls; *flag receives 4 (the sort's timeout bit) when it
// did, 1 when the barrier completed (which would be an error).  No copy is issued, so nothing
// is in flight when the kernel returns.
__global__ void k_selftest_wait(uint32_t limit, uint32_t* flag) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_expect_tx(&bar, 16u);
        *flag = mbar_wait(&bar, 0u, limit) ? 1u : 4u;
    }
}

}  // namespace

vx_status vx_scan_u32(vx_context* ctx, const uint32_t* in, uint32_t* out, uint32_t n,
                      uint32_t* total, cudaStream_t s) {
    uint32_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 0) nb = 1;
    VX_TRY(vx_ws_ensure(ctx, WS_SCAN_TMP, (size_t)nb * 4 + 256, s));
    uint32_t* part = (uint32_t*)ctx->ws[WS_SCAN_TMP].p;
    if (n == 0) {
        if (total) VX_CUDA_TRY(cudaMemsetAsync(total, 0, 4, s));
        return VX_OK;
    }
    if (nb <= SCAN_SMALL_TILES) {   // one launch for a short array
        VX_LAUNCH(ctx, ST_SCAN, s, k_scan_small<<<1, SCAN_THREADS, 0, s>>>(in, out, n, total));
        VX_CUDA_TRY(cudaGetLastError());
        return VX_OK;
    }
    VX_LAUNCH(ctx, ST_SCAN, s, k_scan_reduce<<<nb, SCAN_THREADS, 0, s>>>(in, n, part));
    VX_LAUNCH(ctx, ST_SCAN, s, k_scan_partials<<<1, SCAN_THREADS, 0, s>>>(part, nb, total));
    VX_LAUNCH(ctx, ST_SCAN, s, k_scan_down<<<nb, SCAN_THREADS, 0, s>>>(in, out, n, part));
    VX_CUDA_TRY(cudaGetLastError());
    return VX_OK;
}

vx_status vx_segment_starts(vx_context* ctx, const uint32_t* keys, uint32_t n, uint32_t* nseg, uint32_t* starts,
                            cudaStream_t s) {
    if (n == 0) {
        VX_CUDA_TRY(cudaMemsetAsync(nseg, 0, 4, s));
        VX_CUDA_TRY(cudaMemsetAsync(starts, 0, 4, s));
        return VX_OK;
    }
    const uint32_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    VX_TRY(vx_ws_ensure(ctx, WS_SCAN_TMP, (size_t)nb * 4 + 256, s));
    uint32_t* part = (uint32_t*)ctx->ws[WS_SCAN_TMP].p;
    VX_LAUNCH(ctx, ST_HEADS, s, k_seg_count<<<nb, SCAN_THREADS, 0, s>>>(keys, n, part));
    VX_LAUNCH(ctx, ST_HEADS, s, k_scan_partials<<<1, SCAN_THREADS, 0, s>>>(part, nb, nseg));
    VX_LAUNCH(ctx, ST_HEADS, s, k_seg_starts<<<nb, SCAN_THREADS, 0, s>>>(keys, n, part, nseg, starts));
    VX_CUDA_TRY(cudaGetLastError());
    return VX_OK;
}

// Digit widths of the passes of a `bits`-bit key: as few passes as 9-bit digits allow, digits
// as even as possible (27-bit keys: three passes of 9 instead of four of 8).  Returns the count.
static int digit_plan(int bits, int* widths) {
    const int passes = (bits + 8) / 9;
    const int width = (bits + passes - 1) / passes;
    int left = bits, n = 0;
    while (left > 0) {
        widths[n] = left < width ? left : width;
        left -= widths[n++];
    }
    return n;
}

template <int RB>
vx_status sort_pass(vx_context* ctx, uint32_t** keys, uint32_t** vals, uint32_t** keys_alt, uint32_t** vals_alt,
                    uint32_t n, int shift, uint32_t dmask, uint32_t nt, uint32_t* hist, cudaStream_t s,
                    uint32_t* err) {
    static bool attr_set = false;   // dynamic shared memory of the scatter, once per process
    if (!attr_set) {
        VX_CUDA_TRY(cudaFuncSetAttribute(k_radix_scatter_pipe<RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pipe_smem(RB)));
        attr_set = true;
    }
    const unsigned sblocks = (unsigned)std::min<uint32_t>(nt, (uint32_t)vx::kSMs * 2);
    VX_LAUNCH(ctx, ST_SORT_HIST, s, (k_radix_hist<false, RB><<<nt, SORT_THREADS, 0, s>>>(
                                        *keys, *vals, n, shift, dmask, nt, nullptr, hist)));
    VX_TRY(vx_scan_u32(ctx, hist, hist, (uint32_t)((size_t)RB * nt), nullptr, s));
    VX_LAUNCH(ctx, ST_SORT_SCATTER, s, (k_radix_scatter_pipe<RB><<<sblocks, SORT_THREADS, pipe_smem(RB), s>>>(
                                           *keys, *vals, n, shift, dmask, nt, hist, *keys_alt, *vals_alt, err)));
    VX_CUDA_TRY(cudaGetLastError());
    uint32_t* t = *keys; *keys = *keys_alt; *keys_alt = t;
    t = *vals; *vals = *vals_alt; *vals_alt = t;
    return VX_OK;
}

vx_status vx_radix_sort_u32(vx_context* ctx, uint32_t** keys, uint32_t** vals, uint32_t** keys_alt,
                            uint32_t** vals_alt, uint32_t n, int bits, cudaStream_t s, uint32_t* err) {
    if (n <= 1 || bits <= 0) return VX_OK;
    int widths[33];
    const int passes = digit_plan(bits, widths);
    int wmax = 0;
    for (int p = 0; p < passes; ++p) wmax = std::max(wmax, widths[p]);
    if (wmax > 10) return VX_ERR_CAPACITY;
    const uint32_t nt = (n + SORT_TILE - 1) / SORT_TILE;
    const size_t hn = ((size_t)1 << std::max(wmax, 8)) * nt;
    if (hn > 0xffffffffull) return VX_ERR_CAPACITY;
    VX_TRY(vx_ws_ensure(ctx, WS_SORT_HIST, hn * 4, s));
    uint32_t* hist = (uint32_t*)ctx->ws[WS_SORT_HIST].p;
    int shift = 0;
    for (int p = 0; p < passes; ++p) {
        const int w = widths[p];
        const uint32_t dmask = (1u << w) - 1u;
        if (w > 9)
            VX_TRY(sort_pass<1024>(ctx, keys, vals, keys_alt, vals_alt, n, shift, dmask, nt, hist, s, err));
        else if (w > 8)
            VX_TRY(sort_pass<512>(ctx, keys, vals, keys_alt, vals_alt, n, shift, dmask, nt, hist, s, err));
        else
            VX_TRY(sort_pass<256>(ctx, keys, vals, keys_alt, vals_alt, n, shift, dmask, nt, hist, s, err));
        shift += w;
    }
    return VX_OK;
}

// Exclusive prefix sum with caller-provided partials (at least ceil(n / 2048) words); for
// code that must not touch the context workspace.  Same kernels as vx_scan_u32.
cudaError_t vx_scan_u32_scratch(const uint32_t* in, uint32_t* out, uint32_t n, uint32_t* total,
                                uint32_t* partials, cudaStream_t s) {
    if (n == 0) return total ? cudaMemsetAsync(total, 0, 4, s) : cudaSuccess;
    const uint32_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb <= SCAN_SMALL_TILES) {   // one launch for a short array
        k_scan_small<<<1, SCAN_THREADS, 0, s>>>(in, out, n, total);
        return cudaGetLastError();
    }
    k_scan_reduce<<<nb, SCAN_THREADS, 0, s>>>(in, n, partials);
    k_scan_partials<<<1, SCAN_THREADS, 0, s>>>(partials, nb, total);
    k_scan_down<<<nb, SCAN_THREADS, 0, s>>>(in, out, n, partials);
    return cudaGetLastError();
}

// Stable LSD radix sort with caller-provided scratch (no context workspace): the `bits`
// low key bits, then, when lut != NULL, one more stable pass on the digit lut[value]
// (padding elements carry value 0xffffffff and go last).  hist needs 256 * ceil(n / 4096)
// words, partials ceil(256 * ceil(n / 4096) / 2048) words.  Enqueues only kernels, so it
// can be captured in a CUDA graph.  Leaves *keys / *vals pointing at the result.
cudaError_t vx_radix_sort_u32_scratch(uint32_t** keys, uint32_t** vals, uint32_t** keys_alt, uint32_t** vals_alt,
                                      uint32_t n, int bits, const uint8_t* lut, uint32_t* hist,
                                      uint32_t* partials, cudaStream_t s) {
    if (n <= 1) return cudaSuccess;
    const uint32_t nt = (n + SORT_TILE - 1) / SORT_TILE;
    const uint32_t hn = RADIX * nt;
    const int passes = (bits + 7) / 8 + (lut ? 1 : 0);
    for (int p = 0; p < passes; ++p) {
        const bool lutpass = lut && p == passes - 1;
        const int shift = 8 * p;
        const int nb = lutpass ? 8 : (bits - shift < 8 ? bits - shift : 8);
        const uint32_t dmask = (1u << nb) - 1u;
        if (lutpass)
            k_radix_hist<true, 256><<<nt, SORT_THREADS, 0, s>>>(*keys, *vals, n, 0, 0xffu, nt, lut, hist);
        else
            k_radix_hist<false, 256><<<nt, SORT_THREADS, 0, s>>>(*keys, *vals, n, shift, dmask, nt, nullptr, hist);
        cudaError_t e = vx_scan_u32_scratch(hist, hist, hn, nullptr, partials, s);
        if (e != cudaSuccess) return e;
        if (lutpass)
            k_radix_scatter<true, 256><<<nt, SORT_THREADS, 0, s>>>(*keys, *vals, n, 0, 0xffu, nt, lut, hist,
                                                                   *keys_alt, *vals_alt);
        else
            k_radix_scatter<false, 256><<<nt, SORT_THREADS, 0, s>>>(*keys, *vals, n, shift, dmask, nt, nullptr, hist,
                                                                    *keys_alt, *vals_alt);
        uint32_t* t = *keys; *keys = *keys_alt; *keys_alt = t;
        t = *vals; *vals = *vals_alt; *vals_alt = t;
    }
    return cudaGetLastError();
}

// Runs the bounded-wait self-test (k_selftest_wait) on `stream` and returns VX_ERR_TIMEOUT
// when the wait gave up as it must (see vx.h).
extern "C" vx_status vx_selftest_bounded_wait(vx_context* ctx, int polls, void* stream) {
    if (!ctx || polls < 1) return VX_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    VX_TRY(vx_ws_ensure(ctx, WS_MISC, 256, s));
    uint32_t* flag = (uint32_t*)ctx->ws[WS_MISC].p;
    VX_CUDA_TRY(cudaMemsetAsync(flag, 0, 4, s));
    k_selftest_wait<<<1, 32, 0, s>>>((uint32_t)polls, flag);
    VX_CUDA_TRY(cudaGetLastError());
    VX_TRY(vx_readback_async(ctx, 0, flag, 4, s));
    VX_CUDA_TRY(cudaStreamSynchronize(s));
    const uint32_t f = ((uint32_t*)ctx->host_pin)[0];
    return f == 4u ? VX_ERR_TIMEOUT : (f == 1u ? VX_OK : VX_ERR_CUDA);
}
