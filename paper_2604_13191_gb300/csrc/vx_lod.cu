// vx_lod.cu -- bottom-up LoD pyramid (Sec. 4.2-4.4): 2x2x2 aggregation of mass and
// second moments, OR-downsampled sub-cell masks, and SGGX-H lobe clustering.
//
// Per level l -> l+1 (children are contiguous in Morton order, the parent key is
// key >> 3, so no re-sort is needed):
//   heads     parent segment starts where key >> 3 changes
//   reduce    thread per parent: sums in child order, mask downsample, occupancy,
//             K = 1 lobe S = M / m, or the children's lobes when at most K of them
//   cluster   warp per parent with more than K candidate lobes: sampled histograms,
//             sliced Wasserstein-1 distances, agglomerative merges (Eq. similarity)
//
// SGGX-H arithmetic: every lobe S is sampled with the N given unit directions u_k as
// omega_k = normalize(S'^(1/2) u_k), S' = S + 1e-6 tr(S) I, S'^(1/2) by cyclic Jacobi
// (FP32, 6 sweeps); S'^(1/2) u_k is taken with fused multiply-adds.  Histograms are integer
// counts; the sample second moment sums the products omega_a omega_b, each rounded once to
// the 2^-20 grid, in integers.  Both are therefore independent of the order in which the
// warp visits the samples.
#include <math.h>

#include <algorithm>

#include "vx_internal.cuh"

namespace {

constexpr int CL_WARPS = 4;                 // warps per block in the cluster kernel

struct LevelIn {
    const uint64_t* keys;
    const uint64_t* mask;
    const float* mass;
    const float* moment;
    const uint8_t* lobe_count;
    const float* lobes;
    int K;
};

// Parents per level l = 1..L (L < 32): a key starts a parent of level l when its bits above
// 3 l differ from the previous key's.  Warps add their counts in shared memory, and each
// block adds its totals to counts[] once per level.
__global__ void k_level_counts(const uint64_t* __restrict__ keys, uint32_t n, int L, uint32_t* __restrict__ counts) {
    __shared__ uint32_t blk[32];
    const int lane = threadIdx.x & 31;
    for (int l = threadIdx.x; l < 32; l += blockDim.x) blk[l] = 0;
    __syncthreads();
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        uint32_t i = base + threadIdx.x;
        uint64_t k = (i < n) ? keys[i] : 0ull;
        uint64_t kp = (i < n && i > 0) ? keys[i - 1] : 0ull;
        for (int l = 1; l <= L; ++l) {
            bool head = (i < n) && (i == 0 || (k >> (3 * l)) != (kp >> (3 * l)));
            uint32_t b = __ballot_sync(0xffffffffu, head);
            if (lane == 0 && b) atomicAdd(&blk[l], (uint32_t)__popc(b));
        }
    }
    __syncthreads();
    for (int l = 1 + threadIdx.x; l <= L; l += blockDim.x)
        if (blk[l]) atomicAdd(&counts[l], blk[l]);
}

__global__ void k_parent_flags(const uint64_t* __restrict__ keys, uint32_t n, uint32_t* __restrict__ flags) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flags[i] = (i == 0 || (keys[i] >> 3) != (keys[i - 1] >> 3)) ? 1u : 0u;
}

__global__ void k_parent_starts(const uint64_t* __restrict__ keys, uint32_t n, const uint32_t* __restrict__ idx,
                                uint32_t np, uint32_t* __restrict__ starts) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && (i == 0 || (keys[i] >> 3) != (keys[i - 1] >> 3))) starts[idx[i]] = i;
    if (i == 0) starts[np] = n;
}

// 2x2x2 OR-downsample of two z-slabs a, b of a child mask (bit x + 8 y) into the parent word of
// its octant (ox, oy): the 4 x 4 result lands at bit 4 ox + qx + 8 (4 oy + qy).  The folds run on
// 32-bit halves (rows 0-3 low, 4-7 high): z, then the row pairs (2qy, 2qy + 1), then the x pairs;
// one byte permute gathers the even rows and two steps compact their even bits to nibbles.
__device__ __forceinline__ uint64_t downsample_word(uint64_t a, uint64_t b, int ox, int oy) {
    uint32_t lo = (uint32_t)a | (uint32_t)b;
    uint32_t hi = (uint32_t)(a >> 32) | (uint32_t)(b >> 32);
    lo |= lo >> 8;
    hi |= hi >> 8;
    lo |= lo >> 1;
    hi |= hi >> 1;
    uint32_t x = __byte_perm(lo, hi, 0x6420) & 0x55555555u;   // byte qy: rows 2qy | 2qy + 1
    x = (x | (x >> 1)) & 0x33333333u;
    x = (x | (x >> 2)) & 0x0f0f0f0fu;
    return (uint64_t)(x << (4 * ox)) << (32 * oy);
}

// the child's 2x2x2-downsampled mask ORed into octant (ox, oy, oz) of the parent mask pm
__device__ __forceinline__ void downsample_into(const uint64_t* cm, int oct, uint64_t* pm) {
    const int ox = oct & 1, oy = (oct >> 1) & 1, oz = (oct >> 2) & 1;
#pragma unroll
    for (int qz = 0; qz < 4; ++qz) {
        const uint64_t w = downsample_word(cm[2 * qz], cm[2 * qz + 1], ox, oy);
        // (constant indices: the parent mask stays in registers)
        pm[qz] |= oz ? 0ull : w;
        pm[4 + qz] |= oz ? w : 0ull;
    }
}

__device__ __forceinline__ void compact_params(const float* S, float* c) {
    c[0] = sqrtf(S[0]);
    c[1] = sqrtf(S[1]);
    c[2] = sqrtf(S[2]);
    float pxy = S[0] * S[1], pxz = S[0] * S[2], pyz = S[1] * S[2];
    c[3] = pxy > 0.0f ? S[3] / sqrtf(pxy) : 0.0f;
    c[4] = pxz > 0.0f ? S[4] / sqrtf(pxz) : 0.0f;
    c[5] = pyz > 0.0f ? S[5] / sqrtf(pyz) : 0.0f;
}

// Histogram counts and sample second moment of one lobe (Sec. 4.4), 48 bytes.  Kept per
// output lobe of a level so that the next level's clustering does not sample it again
// (the statistics are a deterministic function of the lobe's stored S); h[0] < 0 marks a
// lobe that was never sampled.
struct LobeStats {
    int32_t h[6];
    float Mh[6];
};
static_assert(sizeof(LobeStats) == kLobeStatsBytes, "lobe statistics record");

// One of the six moment components (or the mass, c = 6) picked by a lane index without a
// dynamically indexed array (which would go through local memory).
__device__ __forceinline__ float pick7(const float* M, float m, int c) {
    float r = m;
#pragma unroll
    for (int k = 0; k < 6; ++k) r = (c == k) ? M[k] : r;
    return r;
}
__device__ __forceinline__ uint64_t shfl_xor_u64(uint32_t m, uint64_t v, int o) {
    const uint32_t lo = __shfl_xor_sync(m, (uint32_t)v, o, 8);
    const uint32_t hi = __shfl_xor_sync(m, (uint32_t)(v >> 32), o, 8);
    return ((uint64_t)hi << 32) | lo;
}

// A group of 8 lanes reduces one parent p: its children are in[starts[p] .. starts[p+1]) in
// key order, at most 8 of them in a level of unique keys (one per octant), and lane j of the
// group reads children beg + j, beg + j + 8, ...  All children's records are read at once.
//   - mass and moment: the sequential FP32 chain in child order of the definition; the
//     children's values are broadcast in the group and every lane folds them in that order;
//   - mask: the OR of the children's 2x2x2-downsampled masks (exact in any order);
//   - lobes (Sec. 4.3-4.4): K = 1 gives S = M / m; K > 1 copies at most K candidate lobes by
//     weight, a lane per child; more candidates go to the SGGX-H work list.
// (np_dev, when given, overrides np with a device-side count.)
constexpr int LR_BLOCK = 256;

__global__ void __launch_bounds__(LR_BLOCK, 4) k_lod_reduce(LevelIn in, const uint32_t* __restrict__ starts, uint32_t np,
                                                         vx_level out, int K, uint32_t* __restrict__ work,
                                                         uint32_t* __restrict__ nwork,
                                                         const uint32_t* __restrict__ np_dev,
                                                         const LobeStats* __restrict__ cst,
                                                         LobeStats* __restrict__ pst) {
    if (np_dev) np = *np_dev;
    const int lane = threadIdx.x & 31;
    const int j = lane & 7;
    const uint32_t gm = 0xffu << (lane & 24);      // the lanes of this group
    const uint32_t groups = gridDim.x * (LR_BLOCK / 8);
    // the trip count is the same for the whole warp (full-warp ballot below); each iteration
    // loads the next one's child range while it works
    uint32_t base = (blockIdx.x * LR_BLOCK + (threadIdx.x & ~31u)) >> 3;
    uint32_t nbeg = 0, nend = 0;
    if (base + (uint32_t)(lane >> 3) < np) {
        nbeg = starts[base + (lane >> 3)];
        nend = starts[base + (lane >> 3) + 1];
    }
    for (; base < np; base += groups) {
        const uint32_t p = base + (uint32_t)(lane >> 3);
        const uint32_t beg = nbeg, end = nend;
        const uint32_t pn = p + groups;
        if (pn < np) {
            nbeg = starts[pn];
            nend = starts[pn + 1];
        }
        bool cluster = false;
        if (p < np) {
            float m = 0.0f;
            float M[6] = {0, 0, 0, 0, 0, 0};
            uint64_t pm[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            int ncand = 0;
            uint32_t lcj = 0;   // lobe count of this lane's child (last chunk read)
            for (uint32_t c0 = beg; c0 < end; c0 += 8) {
                const uint32_t c = c0 + (uint32_t)j;
                float cmass = 0.0f;
                float cmo[6] = {0, 0, 0, 0, 0, 0};
                if (c < end) {
                    cmass = in.mass[c];
                    // moments as 8-byte pairs (rows are 24 bytes, 8-byte aligned)
                    const float2* m2 = reinterpret_cast<const float2*>(in.moment + (size_t)c * 6);
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float2 q = m2[k];
                        cmo[2 * k] = q.x;
                        cmo[2 * k + 1] = q.y;
                    }
                    uint64_t cm[8];
                    const ulonglong2* cm2 = reinterpret_cast<const ulonglong2*>(in.mask + (size_t)c * 8);
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        const ulonglong2 x = cm2[w];
                        cm[2 * w] = x.x;
                        cm[2 * w + 1] = x.y;
                    }
                    downsample_into(cm, (int)(in.keys[c] & 7ull), pm);
                    lcj = in.lobe_count[c];
                    ncand += (int)lcj;
                }
                const int nc = (int)min(8u, end - c0);   // the same in the whole group
                for (int i = 0; i < nc; ++i) {
                    const float mi = __shfl_sync(gm, cmass, i, 8);
                    float Mi[6];
#pragma unroll
                    for (int k = 0; k < 6; ++k) Mi[k] = __shfl_sync(gm, cmo[k], i, 8);
                    m = m + mi;
#pragma unroll
                    for (int k = 0; k < 6; ++k) M[k] = M[k] + Mi[k];
                }
            }
            // a parent of at most 8 children, each with at most one lobe (every parent of level 1):
            // the lane's child's lobe row, read now so that it arrives during the mask reduction
            const bool one_chunk = end - beg <= 8u;
            const uint32_t cj = beg + (uint32_t)j;
            const bool has1 = K > 1 && one_chunk && cj < end && lcj == 1u;
            float row[7] = {0, 0, 0, 0, 0, 0, 0};
            if (has1) {
                const float* src = in.lobes + (size_t)cj * in.K * 7;
#pragma unroll
                for (int k = 0; k < 7; ++k) row[k] = src[k];
            }
            // the group's OR of the mask words, scattered so that lane j keeps word j: each step
            // keeps the half of the words its lane-index bit selects and ORs in the partner's copy
            uint64_t h4[4], h2[2];
            {
                const bool up = (j & 4) != 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint64_t keep = up ? pm[4 + q] : pm[q], give = up ? pm[q] : pm[4 + q];
                    h4[q] = keep | shfl_xor_u64(gm, give, 4);
                }
            }
            {
                const bool up = (j & 2) != 0;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const uint64_t keep = up ? h4[2 + q] : h4[q], give = up ? h4[q] : h4[2 + q];
                    h2[q] = keep | shfl_xor_u64(gm, give, 2);
                }
            }
            const bool up1 = (j & 1) != 0;
            const uint64_t word = (up1 ? h2[1] : h2[0]) | shfl_xor_u64(gm, up1 ? h2[0] : h2[1], 1);
            // occupancy counts of word j (the z-slab j), summed over the group
            int o = __popcll(word);
            uint64_t t = word | (word >> 4);
            t |= t >> 2;
            t |= t >> 1;
            int yz = __popcll(t & 0x0101010101010101ull);
            uint64_t rr = word | (word >> 32);
            rr |= rr >> 16;
            rr |= rr >> 8;
            int xz = __popc((uint32_t)(rr & 0xffu));
            uint64_t orz = word;
#pragma unroll
            for (int sh = 4; sh > 0; sh >>= 1) {
                o += __shfl_xor_sync(gm, o, sh, 8);
                yz += __shfl_xor_sync(gm, yz, sh, 8);
                xz += __shfl_xor_sync(gm, xz, sh, 8);
                orz |= shfl_xor_u64(gm, orz, sh);
                ncand += __shfl_xor_sync(gm, ncand, sh, 8);
            }
            const size_t pb = (size_t)p;
            out.mask[pb * 8 + j] = word;
            if (j < 6) out.moment[pb * 6 + j] = pick7(M, m, j);
            if (j == 0) {
                out.keys[pb] = in.keys[beg] >> 3;
                out.mass[pb] = m;
                out.occ[pb] = (uint16_t)o;
                out.occ_proj[pb * 3 + 0] = (uint8_t)yz;
                out.occ_proj[pb * 3 + 1] = (uint8_t)xz;
                out.occ_proj[pb * 3 + 2] = (uint8_t)__popcll(orz);
            }
            float* lo = out.lobes + pb * K * 7;
            float* co = out.compact + pb * K * 6;
            if (K == 1) {
                if (m > 0.0f) {
                    float S[6], cc[6];
#pragma unroll
                    for (int k = 0; k < 6; ++k) S[k] = M[k] / m;
                    compact_params(S, cc);
                    if (j < 7) lo[j] = pick7(S, m, j);
                    if (j < 6) co[j] = pick7(cc, 0.0f, j);
                    if (j == 0) out.lobe_count[pb] = 1;
                } else {
                    if (j < 7) lo[j] = 0.0f;
                    if (j < 6) co[j] = 0.0f;
                    if (j == 0) out.lobe_count[pb] = 0;
                }
            } else if (ncand <= K) {
                // the children's lobes ordered by weight (descending), ties by candidate order;
                // each lane places the lobes of its own children, the slots past ncand are zero
                for (int r = ncand + j; r < K; r += 8) {
                    for (int k = 0; k < 7; ++k) lo[r * 7 + k] = 0.0f;
                    for (int k = 0; k < 6; ++k) co[r * 6 + k] = 0.0f;
                }
                const bool fast = one_chunk && __all_sync(gm, !(cj < end && lcj > 1u));
                if (fast) {
                    // the ranks from the group's weights: candidate order is child order
                    const uint32_t hb = (__ballot_sync(gm, has1) >> (lane & 24)) & 0xffu;
                    const int idx = __popc(hb & ((1u << j) - 1u));
                    const float wx = row[6];
                    int rank = 0;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float wy = __shfl_sync(gm, wx, i, 8);
                        const int idy = __popc(hb & ((1u << i) - 1u));
                        if (((hb >> i) & 1u) && (wy > wx || (wy == wx && idy < idx))) ++rank;
                    }
                    if (has1) {
#pragma unroll
                        for (int k = 0; k < 7; ++k) lo[rank * 7 + k] = row[k];
                        compact_params(row, co + rank * 6);
                        if (pst) {
                            LobeStats st;
                            if (cst) {
                                st = cst[(size_t)cj * in.K];
                            } else {
#pragma unroll
                                for (int k = 0; k < 6; ++k) { st.h[k] = 0; st.Mh[k] = 0.0f; }
                                st.h[0] = -1;   // never sampled
                            }
                            pst[pb * K + rank] = st;
                        }
                    }
                } else
                for (uint32_t c = beg + (uint32_t)j; c < end; c += 8) {
                    int idx = 0;   // candidate index of the child's first lobe
                    for (uint32_t c2 = beg; c2 < c; ++c2) idx += in.lobe_count[c2];
                    const int nl = in.lobe_count[c];
                    for (int l = 0; l < nl; ++l, ++idx) {
                        const float* src = in.lobes + ((size_t)c * in.K + l) * 7;
                        const float wx = src[6];
                        int rank = 0, idy = 0;
                        for (uint32_t c2 = beg; c2 < end; ++c2)
                            for (int l2 = 0; l2 < in.lobe_count[c2]; ++l2, ++idy) {
                                const float wy = in.lobes[((size_t)c2 * in.K + l2) * 7 + 6];
                                if (wy > wx || (wy == wx && idy < idx)) ++rank;
                            }
                        for (int k = 0; k < 7; ++k) lo[rank * 7 + k] = src[k];
                        compact_params(src, co + rank * 6);
                        if (pst) {
                            LobeStats st;
                            if (cst) {
                                st = cst[(size_t)c * in.K + l];
                            } else {
#pragma unroll
                                for (int k = 0; k < 6; ++k) { st.h[k] = 0; st.Mh[k] = 0.0f; }
                                st.h[0] = -1;   // never sampled
                            }
                            pst[pb * K + rank] = st;
                        }
                    }
                }
                if (j == 0) out.lobe_count[pb] = (uint8_t)ncand;
            } else {
                if (j == 0) {
                    out.lobe_count[pb] = 0;
                    cluster = true;
                }
            }
        }
        // parents left for SGGX-H go to the work list with one atomic per warp (the list's
        // order does not change any output: each parent is clustered on its own)
        const uint32_t want = __ballot_sync(0xffffffffu, cluster);
        if (want) {
            uint32_t wbase = 0;
            if (lane == 0) wbase = atomicAdd(nwork, (uint32_t)__popc(want));
            wbase = __shfl_sync(0xffffffffu, wbase, 0);
            if (cluster) work[wbase + __popc(want & ((1u << lane) - 1u))] = p;
        }
    }
}

// grid of the LoD reduce: 8 lanes per parent, at most the 4 blocks per SM that are resident
inline unsigned lod_reduce_grid(size_t np) {
    return (unsigned)std::max<size_t>(1, std::min<size_t>((np * 8 + LR_BLOCK - 1) / LR_BLOCK, (size_t)vx::kSMs * 4));
}

// ------------------------------------------------------------------------------------
// SGGX-H
// ------------------------------------------------------------------------------------
// S'^(1/2) of a symmetric 3x3 matrix (packed xx,yy,zz,xy,xz,yz) by cyclic Jacobi (at most 6
// sweeps; a rotation is skipped when its off-diagonal is zero or negligible).  Returns
// true when the square root is well conditioned: smallest singular value above 1e-4 of the
// largest, and the largest above 1e-15.  S' = S + 1e-6 tr(S) I bounds the ratio below by
// ~1e-3 for any S with tr(S) > 0; the rounding of the FP32 Jacobi (orthogonality of the
// rotations, the product R u) is ~1e-6 of the largest value, so for every unit u the FP32
// v = R u then has |v| > 1e-4 sg_max (1 - 1e-2) and |v|^2 > 0.
__device__ bool sqrtm3(const float* S, float* Rm) {
    float a[3][3] = {{S[0], S[3], S[4]}, {S[3], S[1], S[5]}, {S[4], S[5], S[2]}};
    float V[3][3] = {{1.0f, 0.0f, 0.0f}, {0.0f, 1.0f, 0.0f}, {0.0f, 0.0f, 1.0f}};
    for (int sweep = 0; sweep < 6; ++sweep) {
        bool rotated = false;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int p = (r == 2) ? 1 : 0;
            const int q = (r == 0) ? 1 : 2;
            const int o = 3 - p - q;
            const float apq = a[p][q];
            if (apq == 0.0f) continue;
            const float app = a[p][p], aqq = a[q][q];
            // an off-diagonal negligible against both diagonals (adding 100 |apq| changes
            // neither in FP32) is set to zero instead of rotated
            const float g = 100.0f * fabsf(apq);
            if (fabsf(app) + g == fabsf(app) && fabsf(aqq) + g == fabsf(aqq)) {
                a[p][q] = 0.0f;
                a[q][p] = 0.0f;
                continue;
            }
            // tan of the rotation angle, sgn(d) 2 apq / (|d| + sqrt(d^2 + 4 apq^2)) with
            // d = aqq - app (the smaller root of t^2 + 2 t d / (2 apq) - 1 = 0)
            const float d = aqq - app, e = 2.0f * apq;
            float t = e / (fabsf(d) + sqrtf(d * d + e * e));
            if (d < 0.0f) t = -t;
            const float c = __frcp_rn(sqrtf(t * t + 1.0f));
            rotated = true;
            const float sn = t * c;
            a[p][p] = app - t * apq;
            a[q][q] = aqq + t * apq;
            a[p][q] = 0.0f;
            a[q][p] = 0.0f;
            const float arp = a[o][p], arq = a[o][q];
            const float nrp = c * arp - sn * arq;
            const float nrq = sn * arp + c * arq;
            a[o][p] = nrp; a[p][o] = nrp;
            a[o][q] = nrq; a[q][o] = nrq;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float vp = V[i][p], vq = V[i][q];
                V[i][p] = c * vp - sn * vq;
                V[i][q] = sn * vp + c * vq;
            }
        }
        if (!rotated) break;   // every off-diagonal is zero
    }
    float sg[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) sg[i] = sqrtf(a[i][i] > 0.0f ? a[i][i] : 0.0f);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            Rm[3 * i + j] = ((V[i][0] * sg[0]) * V[j][0] + (V[i][1] * sg[1]) * V[j][1]) + (V[i][2] * sg[2]) * V[j][2];
    const float smax = fmaxf(fmaxf(sg[0], sg[1]), sg[2]), smin = fminf(fminf(sg[0], sg[1]), sg[2]);
    return smax > 1e-15f && smin > 1e-4f * smax;
}

// a >= b as an integer mask (all ones or zero; zero when either is NaN)
__device__ __forceinline__ uint32_t ge_mask(float a, float b) {
    uint32_t m;
    asm("set.ge.u32.f32 %0, %1, %2;" : "=r"(m) : "f"(a), "f"(b));
    return m;
}

// Two FP32 values packed in a 64-bit register (low half first) and the packed FP32 operations
// on them; each half is rounded to nearest even, exactly as the scalar operation.
typedef unsigned long long f2;
__device__ __forceinline__ f2 f2_pack(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2 v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// One direction sample of a well-conditioned lobe (|v|^2 > 0): the six histogram masks and
// the six moment terms as raw FP32 bit patterns (x * 2^20 / |v|^2 + 1.5 * 2^23, rounded once).
struct SampleTerms {
    uint32_t m[6];
    uint32_t x[6];
};
__device__ __forceinline__ SampleTerms sample_terms(const float* Rm, float4 u4) {
    float v[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        v[i] = __fmaf_rn(Rm[3 * i + 2], u4.z, __fmaf_rn(Rm[3 * i + 1], u4.y, Rm[3 * i] * u4.x));
    const float c0 = v[0] * v[0], c1 = v[1] * v[1], c2 = v[2] * v[2];
    const float n2 = (c0 + c1) + c2;
    const float t6 = 0.36f * n2, t2 = 0.04f * n2;
    SampleTerms r;
    r.m[0] = ge_mask(c0, t6);
    r.m[1] = ge_mask(c1, t6);
    r.m[2] = ge_mask(c2, t6);
    r.m[3] = ge_mask(c0, t2);
    r.m[4] = ge_mask(c1, t2);
    r.m[5] = ge_mask(c2, t2);
    const float s20 = __frcp_rn(n2) * 1048576.0f;
    r.x[0] = __float_as_uint(__fmaf_rn(c0, s20, 12582912.0f));
    r.x[1] = __float_as_uint(__fmaf_rn(c1, s20, 12582912.0f));
    r.x[2] = __float_as_uint(__fmaf_rn(c2, s20, 12582912.0f));
    r.x[3] = __float_as_uint(__fmaf_rn(v[0] * v[1], s20, 12582912.0f));
    r.x[4] = __float_as_uint(__fmaf_rn(v[0] * v[2], s20, 12582912.0f));
    r.x[5] = __float_as_uint(__fmaf_rn(v[1] * v[2], s20, 12582912.0f));
    return r;
}


// round-half-even of the exact product x * s to an integer, for |x s| < 2^22: the fused
// x * s + 1.5 * 2^23 is rounded once, in a binade whose spacing is 1, so the integer lands
// in the low mantissa bits (1.5 * 2^23 is even, so ties go to the even integer)
__device__ __forceinline__ int rint_prod(float x, float s) {
    return __float_as_int(__fmaf_rn(x, s, 12582912.0f)) - 0x4B400000;
}

// Histogram and sample second moment of lobe S, computed cooperatively by G warps
// (G = 1: one warp; G > 1: the whole block, `red` is G * 13 words of shared memory).
// Every count and sum is an integer, so the result is independent of G and of the order
// in which the threads visit the samples.  Threads tid < 6 receive the result.
// The part of a lobe's statistics one thread keeps: component `tid` of the histogram and
// of M^ (threads tid < 6 of the group hold the six components).
struct LobeOwn {
    int32_t h;
    float mh;
};

template <int G>
__device__ LobeOwn sample_lobe(const float* S, const float4* __restrict__ dirs, int N, long long* red) {
    const float tr = (S[0] + S[1]) + S[2];
    const float eps = 1e-6f * tr;
    const float Sp[6] = {S[0] + eps, S[1] + eps, S[2] + eps, S[3], S[4], S[5]};
    float Rm[9];
    const bool wellcond = sqrtm3(Sp, Rm);
    int32_t h[6] = {0, 0, 0, 0, 0, 0};
    long long Q[6] = {0, 0, 0, 0, 0, 0};
    int cnt = 0;
    const int tid = (G == 1) ? (threadIdx.x & 31) : (int)threadIdx.x;
    constexpr int STRIDE = 32 * G;
    if (wellcond && N <= STRIDE * 1024) {
        // every sample has |v|^2 > 0: no sample is skipped.  Two samples (a whole pair of the
        // pair table) per step, their FP32 arithmetic as packed pairs: each half of a packed
        // operation rounds as the scalar one would, so the terms are those of sample_terms.
        // Histogram masks are -1 / 0; each moment term carries the constant 1.5 * 2^23, removed
        // at the end: the sums wrap modulo 2^32, and the true sum of at most 1025 terms of
        // magnitude <= 2^20 is recovered exactly.
        f2 R2[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) R2[i] = f2_pack(Rm[i], Rm[i]);
        const f2 k36 = f2_pack(0.36f, 0.36f), k04 = f2_pack(0.04f, 0.04f);
        const f2 k20 = f2_pack(1048576.0f, 1048576.0f), koff = f2_pack(12582912.0f, 12582912.0f);
        const int NP = N >> 1;
        const ulonglong2* __restrict__ pr = reinterpret_cast<const ulonglong2*>(dirs + N);
        uint32_t q[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll 1
        for (int j = tid; j < NP; j += STRIDE) {
            const ulonglong2 xy = __ldg(pr + 2 * j);
            const f2 z = __ldg(reinterpret_cast<const unsigned long long*>(pr + 2 * j + 1));
            f2 v[3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
                v[i] = f2_fma(R2[3 * i + 2], z, f2_fma(R2[3 * i + 1], xy.y, f2_mul(R2[3 * i], xy.x)));
            const f2 c0 = f2_mul(v[0], v[0]), c1 = f2_mul(v[1], v[1]), c2 = f2_mul(v[2], v[2]);
            const f2 n2 = f2_add(f2_add(c0, c1), c2);
            const f2 t6 = f2_mul(k36, n2), t2 = f2_mul(k04, n2);
            float a0, b0, a1, b1, a2, b2, a6, b6, a4, b4, an, bn;
            f2_unpack(c0, a0, b0);
            f2_unpack(c1, a1, b1);
            f2_unpack(c2, a2, b2);
            f2_unpack(t6, a6, b6);
            f2_unpack(t2, a4, b4);
            f2_unpack(n2, an, bn);
            h[0] = h[0] - (int32_t)ge_mask(a0, a6) - (int32_t)ge_mask(b0, b6);
            h[1] = h[1] - (int32_t)ge_mask(a1, a6) - (int32_t)ge_mask(b1, b6);
            h[2] = h[2] - (int32_t)ge_mask(a2, a6) - (int32_t)ge_mask(b2, b6);
            h[3] = h[3] - (int32_t)ge_mask(a0, a4) - (int32_t)ge_mask(b0, b4);
            h[4] = h[4] - (int32_t)ge_mask(a1, a4) - (int32_t)ge_mask(b1, b4);
            h[5] = h[5] - (int32_t)ge_mask(a2, a4) - (int32_t)ge_mask(b2, b4);
            const f2 s20 = f2_mul(f2_pack(__frcp_rn(an), __frcp_rn(bn)), k20);
            // each term is folded into its sum as soon as it is formed (short live ranges)
            f2 x = f2_fma(c0, s20, koff);
            q[0] = q[0] + (uint32_t)x + (uint32_t)(x >> 32);
            x = f2_fma(c1, s20, koff);
            q[1] = q[1] + (uint32_t)x + (uint32_t)(x >> 32);
            x = f2_fma(c2, s20, koff);
            q[2] = q[2] + (uint32_t)x + (uint32_t)(x >> 32);
            x = f2_fma(f2_mul(v[0], v[1]), s20, koff);
            q[3] = q[3] + (uint32_t)x + (uint32_t)(x >> 32);
            x = f2_fma(f2_mul(v[0], v[2]), s20, koff);
            q[4] = q[4] + (uint32_t)x + (uint32_t)(x >> 32);
            x = f2_fma(f2_mul(v[1], v[2]), s20, koff);
            q[5] = q[5] + (uint32_t)x + (uint32_t)(x >> 32);
        }
        // an odd N leaves one sample, taken by the thread next in line
        const bool last = (N & 1) && tid == NP % STRIDE;
        if (last) {
            const SampleTerms A = sample_terms(Rm, __ldg(dirs + N - 1));
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                h[c] = h[c] - (int32_t)A.m[c];
                q[c] = q[c] + A.x[c];
            }
        }
        const uint32_t ns = 2u * (tid < NP ? (uint32_t)((NP - 1 - tid) / STRIDE + 1) : 0u) + (last ? 1u : 0u);
        cnt = (int)ns;
#pragma unroll
        for (int c = 0; c < 6; ++c) Q[c] = (int32_t)(q[c] - ns * 0x4B400000u);
    } else
    // per-thread int32 partial sums (|term| <= 2^20), flushed to int64 every 1024 samples
    for (int k0 = tid; k0 < N; k0 += STRIDE * 1024) {
        int32_t q[6] = {0, 0, 0, 0, 0, 0};
        const int kend = min(N, k0 + STRIDE * 1024);
#pragma unroll 4
        for (int k = k0; k < kend; k += STRIDE) {
            const float4 u4 = __ldg(dirs + k);
            const float u0 = u4.x, u1 = u4.y, u2 = u4.z;
            float v[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) v[i] = __fmaf_rn(Rm[3 * i + 2], u2, __fmaf_rn(Rm[3 * i + 1], u1, Rm[3 * i] * u0));
            const float c0 = v[0] * v[0], c1 = v[1] * v[1], c2 = v[2] * v[2];
            const float n2 = (c0 + c1) + c2;
            if (!(n2 > 0.0f)) continue;
            ++cnt;
            const float t6 = 0.36f * n2, t2 = 0.04f * n2;
            h[0] += (c0 >= t6) ? 1 : 0;
            h[1] += (c1 >= t6) ? 1 : 0;
            h[2] += (c2 >= t6) ? 1 : 0;
            h[3] += (c0 >= t2) ? 1 : 0;
            h[4] += (c1 >= t2) ? 1 : 0;
            h[5] += (c2 >= t2) ? 1 : 0;
            const float inv = __frcp_rn(n2);
            const float s20 = inv * 1048576.0f;
            q[0] += rint_prod(c0, s20);
            q[1] += rint_prod(c1, s20);
            q[2] += rint_prod(c2, s20);
            q[3] += rint_prod(v[0] * v[1], s20);
            q[4] += rint_prod(v[0] * v[2], s20);
            q[5] += rint_prod(v[1] * v[2], s20);
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) Q[c] += q[c];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            h[c] += __shfl_xor_sync(0xffffffffu, h[c], o);
            Q[c] += __shfl_xor_sync(0xffffffffu, Q[c], o);
        }
    }
    if (G > 1) {
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        __syncthreads();
        if (lane == 0) {
            red[w * 13 + 0] = cnt;
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                red[w * 13 + 1 + c] = h[c];
                red[w * 13 + 7 + c] = Q[c];
            }
        }
        __syncthreads();
        // thread c < 6 keeps component c only (the result below reads nothing else)
        if (tid < 6) {
            long long tc = 0, th = 0, tq = 0;
            for (int ww = 0; ww < G; ++ww) {
                tc += red[ww * 13];
                th += red[ww * 13 + 1 + tid];
                tq += red[ww * 13 + 7 + tid];
            }
            cnt = (int)tc;
            h[0] = (int32_t)th;
            Q[0] = tq;
        }
        __syncthreads();
    }
    // component `tid` (tid < 6) of the histogram and of M^ (one FP64 division per thread)
    LobeOwn own;
    own.h = h[0];
    long long q = Q[0];
    if (G == 1) {
#pragma unroll
        for (int c = 1; c < 6; ++c) {
            if (tid == c) {
                own.h = h[c];
                q = Q[c];
            }
        }
    }
    own.mh = 0.0f;
    if (tid < 6 && cnt > 0) own.mh = (float)((double)q / ((double)cnt * 1048576.0));
    return own;
}

// Per-group shared state of SGGX-H, sized for `slots` lobes (candidates + merges, 2 * 8K):
// S [slots][6], w [slots], M^ [slots][6], histogram [slots][6], alive [slots].
struct ClusterView {
    float* S;
    float* w;
    float* Mh;
    int32_t* H;
    uint8_t* alive;
    uint8_t* list;    // the alive slots in increasing order (rebuilt before each merge)
};
__host__ __device__ inline size_t cluster_bytes(int slots) {
    return (((size_t)slots * 19 * 4 + (size_t)slots * 2) + 15) & ~size_t(15);
}
__device__ inline ClusterView cluster_view(unsigned char* base, int slots) {
    ClusterView v;
    v.S = (float*)base;
    v.w = v.S + (size_t)slots * 6;
    v.Mh = v.w + slots;
    v.H = (int32_t*)(v.Mh + (size_t)slots * 6);
    v.alive = (uint8_t*)(v.H + (size_t)slots * 6);
    v.list = v.alive + slots;
    return v;
}

// q -> (a, b), a > b, ordered by a then b, for the pairs of up to 64 alive lobes
struct PairTable {
    uint16_t ab[64 * 63 / 2];
};
constexpr PairTable make_pair_table() {
    PairTable t{};
    int q = 0;
    for (int a = 1; a < 64; ++a)
        for (int b = 0; b < a; ++b) t.ab[q++] = (uint16_t)((a << 8) | b);
    return t;
}
__device__ const PairTable kPairTable = make_pair_table();

// float3 direction table -> float4 (one 16-byte load per sample), followed by the table of
// whole pairs: directions 2j and 2j + 1 as {x0, x1, y0, y1} and {z0, z1, 0, 0}, so that each
// coordinate of the two loads as one packed FP32 pair
__global__ void k_pack_dirs(const float* __restrict__ d, int n, float4* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = make_float4(d[3 * k], d[3 * k + 1], d[3 * k + 2], 0.0f);
    if (k < n / 2) {
        float4* pr = out + n;
        const float* a = d + 6 * k;
        pr[2 * k] = make_float4(a[0], a[3], a[1], a[4]);
        pr[2 * k + 1] = make_float4(a[2], a[5], 0.0f, 0.0f);
    }
}

// One parent listed in `work` per group of G warps (G = 1: a warp per parent, for levels
// with many parents; G = CL_BLOCK_WARPS: a block per parent, for the few coarse parents
// whose long merge chains would otherwise run on a single warp).
constexpr int CL_BLOCK_WARPS = 8;
constexpr int CL_WIDE_WARPS = 16;   // levels with at most one parent per SM

template <int G>
__global__ void __launch_bounds__(G == 1 ? CL_WARPS * 32 : G * 32, G == 1 ? 7 : 0) k_sggx_cluster(
    LevelIn in, const uint32_t* __restrict__ starts, const uint32_t* __restrict__ work,
    const uint32_t* __restrict__ nwork_p, vx_level out, int K, const float4* __restrict__ dirs, int N,
    const LobeStats* __restrict__ cst, LobeStats* __restrict__ pst, unsigned long long* __restrict__ nsampled,
    int merge) {
    extern __shared__ unsigned char smem_raw[];
    constexpr int GROUPS = (G == 1) ? CL_WARPS : 1;
    const int group = (G == 1) ? (int)(threadIdx.x >> 5) : 0;
    const int slots = 16 * K;
    const ClusterView sm = cluster_view(smem_raw + cluster_bytes(slots) * group, slots);
    long long* red = (long long*)(smem_raw + cluster_bytes(slots) * GROUPS);
    __shared__ unsigned long long bestred[G];
    const int tid = (G == 1) ? (int)(threadIdx.x & 31) : (int)threadIdx.x;
    constexpr int NT = 32 * G;
    const int lane = threadIdx.x & 31;
    const uint32_t nwork = *nwork_p;
    auto gsync = [&]() {
        if (G == 1) __syncwarp(); else __syncthreads();
    };
    // parents are taken one at a time from a shared counter (nwork_p[1]), so that groups
    // that drew short merge chains take more parents
    __shared__ uint32_t take[GROUPS];
    for (;;) {
        uint32_t it;
        if (G == 1) {
            uint32_t v = 0;
            if (lane == 0) v = atomicAdd(const_cast<uint32_t*>(nwork_p) + 1, 1u);
            it = __shfl_sync(0xffffffffu, v, 0);
        } else {
            if (threadIdx.x == 0) take[0] = atomicAdd(const_cast<uint32_t*>(nwork_p) + 1, 1u);
            __syncthreads();
            it = take[0];
            __syncthreads();
        }
        if (it >= nwork) break;
        const uint32_t p = work[it];
        const uint32_t beg = starts[p], end = starts[p + 1];
        // gather candidates in (child, lobe) order, with their statistics where the child
        // level kept them (alive = 2: not sampled yet)
        int n = 0;
        for (uint32_t c = beg; c < end; ++c) {
            const int lc = in.lobe_count[c];
            for (int l = tid; l < lc * 7; l += NT) {
                const int li = l / 7, j = l % 7;
                const float x = in.lobes[((size_t)c * in.K + li) * 7 + j];
                if (j < 6) sm.S[(n + li) * 6 + j] = x; else sm.w[n + li] = x;
            }
            for (int l = tid; l < lc; l += NT) {
                bool have = false;
                if (cst) {
                    const LobeStats st = cst[(size_t)c * in.K + l];
                    if (st.h[0] >= 0) {
                        have = true;
#pragma unroll
                        for (int j = 0; j < 6; ++j) {
                            sm.H[(n + l) * 6 + j] = st.h[j];
                            sm.Mh[(n + l) * 6 + j] = st.Mh[j];
                        }
                    }
                }
                sm.alive[n + l] = have ? 1 : 2;
            }
            n += lc;
        }
        for (int l = n + tid; l < slots; l += NT) sm.alive[l] = 0;
        gsync();
        int sampled = 0;
        for (int l = 0; l < n; ++l) {
            if (sm.alive[l] != 2) continue;
            const LobeOwn st = sample_lobe<G>(sm.S + l * 6, dirs, N, red);
            if (tid < 6) {
                sm.H[l * 6 + tid] = st.h;
                sm.Mh[l * 6 + tid] = st.mh;
            }
            ++sampled;
        }
        gsync();
        for (int l = tid; l < n; l += NT) sm.alive[l] = 1;
        gsync();
        int count = n, next = n;
        while (count > K) {
            // the alive slots in increasing order (count <= 8K <= 64 of them)
            if (tid < 32) {
                int base = 0;
                for (int s0 = 0; s0 < next; s0 += 32) {
                    const int sl = s0 + tid;
                    const bool al = sl < next && sm.alive[sl];
                    const uint32_t m = __ballot_sync(0xffffffffu, al);
                    if (al) sm.list[base + __popc(m & ((1u << tid) - 1u))] = (uint8_t)sl;
                    base += __popc(m);
                }
            }
            gsync();
            // argmin over alive pairs (i > j) of (distance, i, j); the distance is a sum of
            // six histogram differences of at most N each, so it fits 32 bits
            unsigned long long best = ~0ull;
            const int npairs = count * (count - 1) / 2;
            for (int q = tid; q < npairs; q += NT) {
                const uint32_t ab = kPairTable.ab[q];
                const int i = sm.list[ab >> 8], j = sm.list[ab & 0xffu];
                uint32_t d = 0;
#pragma unroll
                for (int c = 0; c < 6; ++c) d = __sad(sm.H[i * 6 + c], sm.H[j * 6 + c], d);
                unsigned long long key = ((unsigned long long)d << 16) | ((unsigned long long)i << 8) | (unsigned long long)j;
                if (key < best) best = key;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
                if (other < best) best = other;
            }
            if (G > 1) {
                if (lane == 0) bestred[threadIdx.x >> 5] = best;
                __syncthreads();
                best = bestred[0];
                for (int ww = 1; ww < G; ++ww) best = bestred[ww] < best ? bestred[ww] : best;
                __syncthreads();
            }
            const int bi = (int)((best >> 8) & 0xffull), bj = (int)(best & 0xffull);
            // merge 0: pooled samples, (M^_i + M^_j) / 2; merge 1: mass-weighted moments
            if (tid < 6) {
                const float wi = sm.w[bi], wj = sm.w[bj], ws = wi + wj;
                sm.S[next * 6 + tid] = (merge == 1 && ws > 0.0f)
                                           ? (wi * sm.Mh[bi * 6 + tid] + wj * sm.Mh[bj * 6 + tid]) / ws
                                           : (sm.Mh[bi * 6 + tid] + sm.Mh[bj * 6 + tid]) * 0.5f;
            }
            if (tid == 0) {
                sm.w[next] = sm.w[bi] + sm.w[bj];
                sm.alive[bi] = 0;
                sm.alive[bj] = 0;
                sm.alive[next] = 1;
            }
            gsync();
            const LobeOwn st = sample_lobe<G>(sm.S + next * 6, dirs, N, red);
            if (tid < 6) {
                sm.H[next * 6 + tid] = st.h;
                sm.Mh[next * 6 + tid] = st.mh;
            }
            gsync();
            ++next;
            --count;
        }
        // output: alive lobes by weight (descending), ties by creation index
        float* lo = out.lobes + (size_t)p * K * 7;
        float* co = out.compact + (size_t)p * K * 6;
        for (int x = tid; x < next; x += NT) {
            if (!sm.alive[x]) continue;
            const float wx = sm.w[x];
            int rank = 0;
            for (int y = 0; y < next; ++y)
                if (sm.alive[y] && (sm.w[y] > wx || (sm.w[y] == wx && y < x))) ++rank;
            for (int j = 0; j < 6; ++j) lo[rank * 7 + j] = sm.S[x * 6 + j];
            lo[rank * 7 + 6] = wx;
            compact_params(sm.S + x * 6, co + rank * 6);
            if (pst) {
                LobeStats st;
#pragma unroll
                for (int j = 0; j < 6; ++j) {
                    st.h[j] = sm.H[x * 6 + j];
                    st.Mh[j] = sm.Mh[x * 6 + j];
                }
                pst[(size_t)p * K + rank] = st;
            }
        }
        if (tid == 0) {
            out.lobe_count[p] = (uint8_t)count;
            // lobe samplings: candidates without kept statistics + one per merge
            if (nsampled) atomicAdd(nsampled, (unsigned long long)(sampled + next - n));
        }
        gsync();
    }
}

// Dynamic shared memory of the three clustering tiers for K lobes.
inline size_t cluster_smem(int G, int K) {
    return G == 1 ? cluster_bytes(16 * K) * CL_WARPS : cluster_bytes(16 * K) + sizeof(long long) * 13 * G;
}

cudaError_t cluster_set_smem(int K) {
    cudaError_t e = cudaFuncSetAttribute(k_sggx_cluster<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)cluster_smem(1, K));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sggx_cluster<CL_BLOCK_WARPS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)cluster_smem(CL_BLOCK_WARPS, K));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sggx_cluster<CL_WIDE_WARPS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)cluster_smem(CL_WIDE_WARPS, K));
    return e;
}

// Clustering of one level.  tier: 0 a warp per parent (resident blocks of 4 warps), 1 a
// block of 8 warps, 2 a block of 16 warps per parent; -1 picks by n, the level's parent
// count (or an upper bound of it): warps on wide levels, blocks of 8 warps on narrow ones
// (on the 768k-capsule yarn the 8-warp blocks matched or beat the 16-warp ones on every
// level of at most 212 parents).  Every tier gives the same result.  wcnt[0] holds the number of listed parents and wcnt[1]
// (zero) the take counter.
void launch_cluster(const LevelIn& li, const uint32_t* starts, const uint32_t* work, const uint32_t* wcnt,
                    const vx_level& out, int K, const float4* dirs4, int N, const LobeStats* cst, LobeStats* pst,
                    unsigned long long* nsampled, uint32_t n, int merge, cudaStream_t s, int tier = -1) {
    if (tier < 0) tier = n > (uint32_t)(vx::kSMs * 16) ? 0 : 1;
    if (tier == 0) {
        const unsigned cb = (unsigned)std::min<size_t>((n + CL_WARPS - 1) / CL_WARPS, (size_t)vx::kSMs * 7);
        k_sggx_cluster<1><<<cb, CL_WARPS * 32, cluster_smem(1, K), s>>>(li, starts, work, wcnt, out, K, dirs4, N,
                                                                          cst, pst, nsampled, merge);
    } else if (tier == 1) {
        const unsigned cb = (unsigned)std::max<uint32_t>(1u, std::min<uint32_t>(n, vx::kSMs * 4));
        k_sggx_cluster<CL_BLOCK_WARPS><<<cb, CL_BLOCK_WARPS * 32, cluster_smem(CL_BLOCK_WARPS, K), s>>>(
            li, starts, work, wcnt, out, K, dirs4, N, cst, pst, nsampled, merge);
    } else {
        const unsigned cb = (unsigned)std::max<uint32_t>(1u, std::min<uint32_t>(n, vx::kSMs * 2));
        k_sggx_cluster<CL_WIDE_WARPS><<<cb, CL_WIDE_WARPS * 32, cluster_smem(CL_WIDE_WARPS, K), s>>>(
            li, starts, work, wcnt, out, K, dirs4, N, cst, pst, nsampled, merge);
    }
}

// ---- batched LoD step (several instances, counts on the device) -------------------------
__global__ void k_bparent_flags(const uint64_t* __restrict__ keys, const uint16_t* __restrict__ inst,
                                const uint32_t* __restrict__ n_dev, uint32_t cap, uint32_t* __restrict__ flags) {
    const uint32_t n = *n_dev;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x)
        flags[i] = (i < n && (i == 0 || inst[i] != inst[i - 1] || (keys[i] >> 3) != (keys[i - 1] >> 3))) ? 1u : 0u;
}

// clamp a device count to a capacity, raising the overflow flag
__global__ void k_clamp_count(const uint32_t* __restrict__ total, uint32_t cap, uint32_t* __restrict__ n_out,
                              uint32_t* __restrict__ err) {
    const uint32_t t = *total;
    *n_out = t < cap ? t : cap;
    if (t > cap) atomicOr(err, 2u);
}

__global__ void k_bparent_starts(const uint64_t* __restrict__ keys, const uint16_t* __restrict__ inst,
                                 const uint32_t* __restrict__ n_dev, const uint32_t* __restrict__ idx,
                                 const uint32_t* __restrict__ total, uint32_t cap_out, uint32_t* __restrict__ starts) {
    const uint32_t n = *n_dev;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const bool head = i == 0 || inst[i] != inst[i - 1] || (keys[i] >> 3) != (keys[i - 1] >> 3);
        if (head && idx[i] <= cap_out) starts[idx[i]] = i;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && *total <= cap_out) starts[*total] = n;
}

__global__ void k_bparent_inst(const uint16_t* __restrict__ inst_in, const uint32_t* __restrict__ starts,
                               const uint32_t* __restrict__ np_dev, uint16_t* __restrict__ inst_out) {
    const uint32_t np = *np_dev;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x)
        inst_out[p] = inst_in[starts[p]];
}

inline unsigned grid_for(size_t n, int threads) {
    size_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return (unsigned)std::min<size_t>(b, 0x7fffffff);
}

}  // namespace

namespace {
vx_status build_levels(vx_context* ctx, const vx_level* in, const vx_lod_params* params, cudaStream_t s,
                       vx_level* out, int L, const uint32_t* counts, uint32_t* misc, void* const* events, int nev);
vx_status build_lod(vx_context* ctx, const vx_level* in, const vx_lod_params* params, void* stream, vx_level* out,
                    void* const* events, int nev);
}  // namespace

extern "C" vx_status vx_build_lod(vx_context* ctx, const vx_level* in, const vx_lod_params* params, void* stream,
                                  vx_level* out) {
    return build_lod(ctx, in, params, stream, out, nullptr, 0);
}

extern "C" vx_status vx_build_lod_events(vx_context* ctx, const vx_level* in, const vx_lod_params* params,
                                         void* stream, vx_level* out, void* const* events, int num_events) {
    if (num_events < 0 || (num_events > 0 && !events)) return VX_ERR_INVALID_ARG;
    return build_lod(ctx, in, params, stream, out, events, num_events);
}

namespace {
vx_status build_lod(vx_context* ctx, const vx_level* in, const vx_lod_params* params, void* stream, vx_level* out,
                    void* const* events, int nev) {
    if (!ctx || !in || !params || !out) return VX_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    const int R = in->resolution;
    if (R <= 0 || (R & (R - 1)) != 0 || in->num_voxels < 0 || in->num_voxels > 0xffffffffll) return VX_ERR_INVALID_ARG;
    int maxL = 0;
    while ((1 << maxL) < R) ++maxL;
    const int L = params->num_levels == 0 ? maxL : params->num_levels;
    if (L < 0 || L > maxL) return VX_ERR_INVALID_ARG;
    const int K = params->K;
    if (K < 1 || K > vx::kMaxK) return VX_ERR_UNSUPPORTED;
    if (in->K < 1 || in->K > vx::kMaxK) return VX_ERR_INVALID_ARG;
    if (K > 1 && (!params->dirs || params->n_samples < 1 || params->n_samples > 65536)) return VX_ERR_INVALID_ARG;
    if (params->merge != 0 && params->merge != 1) return VX_ERR_INVALID_ARG;
    for (int l = 0; l < L; ++l) memset(&out[l], 0, sizeof(vx_level));
    if (L == 0) return VX_OK;
    const uint32_t n0 = (uint32_t)in->num_voxels;

    // ---- all level sizes in one pass + one readback ---------------------------------
    VX_TRY(vx_ws_ensure(ctx, WS_MISC, 256, s));
    uint32_t* misc = (uint32_t*)ctx->ws[WS_MISC].p;
    VX_CUDA_TRY(cudaMemsetAsync(misc, 0, 128, s));
    if (n0 > 0)
        VX_LAUNCH(ctx, ST_LOD_COUNTS, s, k_level_counts<<<(unsigned)std::min<size_t>(grid_for(n0, 256), (size_t)vx::kSMs * 16), 256, 0, s>>>(
            in->keys, n0, L, misc));
    VX_CUDA_TRY(cudaGetLastError());
    VX_TRY(vx_readback_async(ctx, 0, misc, 4 * (L + 1), s));
    VX_CUDA_TRY(cudaStreamSynchronize(s));
    uint32_t counts[32];
    memcpy(counts, ctx->host_pin, 4 * (L + 1));
    for (int l = 1; l <= L; ++l) {
        vx_status st = vx_level_alloc(ctx, &out[l - 1], counts[l], K, in->level + l, R >> l, s);
        if (st != VX_OK) {
            for (int j = 0; j < l - 1; ++j) vx_level_release(ctx, &out[j], s);
            return st;
        }
    }
    // an error past this point returns every level to the allocator (outputs unallocated)
    const vx_status st = build_levels(ctx, in, params, s, out, L, counts, misc, events, nev);
    if (st != VX_OK)
        for (int l = 0; l < L; ++l) vx_level_release(ctx, &out[l], s);
    return st;
}

vx_status build_levels(vx_context* ctx, const vx_level* in, const vx_lod_params* params, cudaStream_t s,
                       vx_level* out, int L, const uint32_t* counts, uint32_t* misc, void* const* events, int nev) {
    // the caller's event for out[l - 1], recorded once that level is complete
    auto level_done = [&](int l) -> cudaError_t {
        if (events && l - 1 < nev && events[l - 1]) return cudaEventRecord((cudaEvent_t)events[l - 1], s);
        return cudaSuccess;
    };
    const int K = params->K;
    const uint32_t n0 = (uint32_t)in->num_voxels;
    // ---- per level ------------------------------------------------------------------------
    VX_TRY(vx_ws_ensure(ctx, WS_LOD_FLAGS, (size_t)std::max<uint32_t>(n0, 1) * 4, s));
    VX_TRY(vx_ws_ensure(ctx, WS_LOD_STARTS, (size_t)std::max<uint32_t>(n0, 1) * 4 + 8, s));
    VX_TRY(vx_ws_ensure(ctx, WS_LOD_WORK, (size_t)std::max<uint32_t>(n0, 1) * 4, s));
    uint32_t* flags = (uint32_t*)ctx->ws[WS_LOD_FLAGS].p;
    uint32_t* starts = (uint32_t*)ctx->ws[WS_LOD_STARTS].p;
    uint32_t* work = (uint32_t*)ctx->ws[WS_LOD_WORK].p;
    // per-lobe statistics of the previous and the current level (K > 1), ping-pong
    LobeStats* stats[2] = {nullptr, nullptr};
    if (K > 1) {
        uint32_t vmax = 1;
        for (int l = 1; l <= L; ++l) vmax = std::max(vmax, counts[l]);
        VX_TRY(vx_ws_ensure(ctx, WS_LOD_STATS0, (size_t)vmax * K * sizeof(LobeStats), s));
        VX_TRY(vx_ws_ensure(ctx, WS_LOD_STATS1, (size_t)vmax * K * sizeof(LobeStats), s));
        stats[0] = (LobeStats*)ctx->ws[WS_LOD_STATS0].p;
        stats[1] = (LobeStats*)ctx->ws[WS_LOD_STATS1].p;
    }
    float4* dirs4 = nullptr;
    if (K > 1) {
        VX_TRY(vx_ws_ensure(ctx, WS_LOD_TMP, vx_dirs_bytes(params->n_samples), s));
        dirs4 = (float4*)ctx->ws[WS_LOD_TMP].p;
        VX_LAUNCH(ctx, ST_LOD_HEADS, s, k_pack_dirs<<<(params->n_samples + 255) / 256, 256, 0, s>>>(
                                            params->dirs, params->n_samples, dirs4));
        VX_CUDA_TRY(cluster_set_smem(K));
    }
    for (int l = 1; l <= L; ++l) {
        const vx_level* prev = (l == 1) ? in : &out[l - 2];
        const uint32_t nprev = (uint32_t)prev->num_voxels, ncur = counts[l];
        if (ncur == 0) {
            VX_CUDA_TRY(level_done(l));
            continue;
        }
        LevelIn li;
        li.keys = prev->keys; li.mask = prev->mask; li.mass = prev->mass; li.moment = prev->moment;
        li.lobe_count = prev->lobe_count; li.lobes = prev->lobes; li.K = prev->K;
        VX_LAUNCH(ctx, ST_LOD_HEADS, s, k_parent_flags<<<grid_for(nprev, 256), 256, 0, s>>>(prev->keys, nprev, flags));
        VX_TRY(vx_scan_u32(ctx, flags, flags, nprev, nullptr, s));
        VX_LAUNCH(ctx, ST_LOD_HEADS, s, k_parent_starts<<<grid_for(nprev, 256), 256, 0, s>>>(prev->keys, nprev, flags, ncur, starts));
        VX_CUDA_TRY(cudaMemsetAsync(misc + 40, 0, 8, s));   // [40] clustered parents, [41] taken
        vx_stage_units(ctx, ST_LOD_REDUCE, ncur);
        // statistics kept by the child level (none for the input level) and by this one
        const LobeStats* cst = (K > 1 && l > 1) ? stats[l & 1] : nullptr;
        LobeStats* pst = (K > 1) ? stats[(l + 1) & 1] : nullptr;
        VX_LAUNCH(ctx, ST_LOD_REDUCE, s, k_lod_reduce<<<lod_reduce_grid(ncur), LR_BLOCK, 0, s>>>(
            li, starts, ncur, out[l - 1], K, work, misc + 40, nullptr, cst, pst));
        VX_CUDA_TRY(cudaGetLastError());
        if (K > 1) {
            unsigned long long* cnt_dev = ctx->prof ? ctx->dev_lobe_count : nullptr;
            VX_LAUNCH(ctx, ST_SGGX_CLUSTER, s, launch_cluster(li, starts, work, misc + 40, out[l - 1], K, dirs4,
                                                              params->n_samples, cst, pst, cnt_dev, ncur,
                                                              params->merge, s));
            VX_CUDA_TRY(cudaGetLastError());
        }
        VX_CUDA_TRY(level_done(l));
    }
    return VX_OK;
}
}  // namespace

// Direction table and shared-memory limits of batched clustering with K lobes (host side,
// before any capture): dirs [n][3] -> the direction table (vx_dirs_bytes(n) bytes at dirs4).
cudaError_t vx_lod_batched_prepare(int K, const float* dirs, int n, float4* dirs4, cudaStream_t s) {
    if (K <= 1) return cudaSuccess;
    k_pack_dirs<<<(n + 255) / 256, 256, 0, s>>>(dirs, n, dirs4);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? cluster_set_smem(K) : e;
}

// One batched LoD step: the parents of `in` (n_dev voxels sorted by (instance, key),
// instance ids inst_in, capacity cap_in) into `out` (capacity cap_out, out->K lobes), their
// instance ids into inst_out and their count into np_dev; a parent count above cap_out sets
// bit 2 of err.  flags, idx: cap_in words; starts: cap_out + 1 words; partials:
// ceil(cap_in / 2048) words; tmp: one word.  With out->K > 1 the parents with more than K
// candidate lobes are clustered (SGGX-H): work holds cap_out words, wcnt two, cst / pst the
// lobe statistics of `in` (NULL for level 0) and of `out`.  Only enqueues work
// (graph-capturable).
cudaError_t vx_lod_step_batched(const vx_level* in, const uint16_t* inst_in, const uint32_t* n_dev, uint32_t cap_in,
                                vx_level* out, uint16_t* inst_out, uint32_t* np_dev, uint32_t cap_out,
                                uint32_t* flags, uint32_t* idx, uint32_t* starts, uint32_t* partials, uint32_t* tmp,
                                uint32_t* err, const float4* dirs4, int n_dirs, uint32_t* work, uint32_t* wcnt,
                                const void* cst, void* pst, int merge, int tier, cudaStream_t s) {
    const unsigned gb = (unsigned)std::min<size_t>(grid_for(cap_in, 256), (size_t)vx::kSMs * 16);
    k_bparent_flags<<<gb, 256, 0, s>>>(in->keys, inst_in, n_dev, cap_in, flags);
    cudaError_t e = vx_scan_u32_scratch(flags, idx, cap_in, tmp, partials, s);
    if (e != cudaSuccess) return e;
    k_clamp_count<<<1, 1, 0, s>>>(tmp, cap_out, np_dev, err);
    k_bparent_starts<<<gb, 256, 0, s>>>(in->keys, inst_in, n_dev, idx, tmp, cap_out, starts);
    LevelIn li;
    li.keys = in->keys; li.mask = in->mask; li.mass = in->mass; li.moment = in->moment;
    li.lobe_count = in->lobe_count; li.lobes = in->lobes; li.K = in->K;
    const unsigned rb = lod_reduce_grid(cap_out);
    const int K = out->K;
    if (K > 1) {
        cudaError_t e2 = cudaMemsetAsync(wcnt, 0, 8, s);
        if (e2 != cudaSuccess) return e2;
    }
    k_lod_reduce<<<rb, LR_BLOCK, 0, s>>>(li, starts, 0u, *out, K, K > 1 ? work : nullptr, K > 1 ? wcnt : nullptr, np_dev,
                                    (const LobeStats*)cst, (LobeStats*)pst);
    if (K > 1)
        launch_cluster(li, starts, work, wcnt, *out, K, dirs4, n_dirs, (const LobeStats*)cst, (LobeStats*)pst, nullptr,
                       cap_out, merge, s, tier);
    k_bparent_inst<<<gb, 256, 0, s>>>(inst_in, starts, np_dev, inst_out);
    return cudaGetLastError();
}

// The clustering of a batched LoD step run again on its own with the given tier (the
// step's parents, work list and statistics are still in place): for timing the tiers
// while a batch is planned.  The outputs are rewritten with the same values.
cudaError_t vx_lod_cluster_batched(const vx_level* in, const vx_level* out, const uint32_t* starts,
                                   const uint32_t* work, uint32_t* wcnt, const float4* dirs4, int n_dirs,
                                   const void* cst, void* pst, uint32_t cap_out, int merge, int tier,
                                   cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(wcnt + 1, 0, 4, s);
    if (e != cudaSuccess) return e;
    LevelIn li;
    li.keys = in->keys; li.mask = in->mask; li.mass = in->mass; li.moment = in->moment;
    li.lobe_count = in->lobe_count; li.lobes = in->lobes; li.K = in->K;
    launch_cluster(li, starts, work, wcnt, *out, out->K, dirs4, n_dirs, (const LobeStats*)cst, (LobeStats*)pst,
                   nullptr, cap_out, merge, s, tier);
    return cudaGetLastError();
}
