// vx_level0.cuh -- device code of the level-0 voxelization, shared by the single-problem
// path (vx_voxelize.cu) and the batched path (vx_batch.cu): the capsule and triangle
// sub-cell predicates and measures, the candidate, reduce and finalize kernels.
//
// Arithmetic: every FP32 quantity that decides a bit, and every per-voxel sum, is
// evaluated with the operation order written here and no contraction (the library is
// compiled with -fmad=false); per-voxel sums run sequentially in primitive order.
#pragma once

#include <math.h>

#include <algorithm>

#include "vx_internal.cuh"

namespace {

constexpr float kPi = 3.14159265358979f;
constexpr int RED_WARPS = 4;        // warps per block in the reduce kernels
constexpr int EMIT_WARPS = 8;

struct GridDev {
    float o[3];
    float s;      // 1 / voxel_size (FP32)
    int R;
};

// Per-segment temporary outputs (indexed by candidate-voxel segment id).
struct SegOut {
    uint32_t* key;
    uint64_t* mask;     // [n][8]
    float* mass;
    float* moment;      // [n][6]
    uint32_t* nonzero;
};

__device__ __forceinline__ float fmin2(float a, float b) { return (b < a) ? b : a; }
__device__ __forceinline__ float fmax2(float a, float b) { return (b > a) ? b : a; }

// ------------------------------------------------------------------------------------
// capsule vs closed box [lo, hi]: a, b local endpoints, rr = r^2
// ------------------------------------------------------------------------------------
__device__ __forceinline__ float sqdist_point_box(float px, float py, float pz, const float* lo,
                                                  const float* hi) {
    float p[3] = {px, py, pz};
    float e[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (p[i] < lo[i]) e[i] = lo[i] - p[i];
        else if (p[i] > hi[i]) e[i] = p[i] - hi[i];
        else e[i] = 0.0f;
    }
    return (e[0] * e[0] + e[1] * e[1]) + e[2] * e[2];
}

__device__ __forceinline__ float seg_g(const float* a, const float* d, float t, const float* lo,
                                       const float* hi) {
    if (!(t >= 0.0f)) t = 0.0f;
    else if (t > 1.0f) t = 1.0f;
    return sqdist_point_box(a[0] + t * d[0], a[1] + t * d[1], a[2] + t * d[2], lo, hi);
}

// Step 3 of the capsule test: min over t in [0,1] of the squared segment-box distance,
// taken at the stationary points of the quadratic pieces that can hold the minimum.
// (Scalar code with explicit selects: no dynamically indexed local arrays.)
__device__ __forceinline__ float sel3(int i, float x, float y, float z) { return i == 0 ? x : (i == 1 ? y : z); }

// Called out of line (it is the rare, long case) with scalar arguments, so that nothing of
// it goes through local memory: the box is [lo, lo + ext] (exact for the voxel [0, 1]^3 and
// for the sub-cells [k/8, (k+1)/8]).
__device__ __noinline__ float seg_box_min(float ax, float ay, float az, float dx, float dy, float dz, float lx,
                                          float ly, float lz, float ext) {
    const float a[3] = {ax, ay, az}, d[3] = {dx, dy, dz};
    const float lo[3] = {lx, ly, lz}, hi[3] = {lx + ext, ly + ext, lz + ext};
    float L = -INFINITY, U = INFINITY;
    int iL = -1, jU = -1, moving = 0;
    float plo0 = 0.0f, plo1 = 0.0f, plo2 = 0.0f, phi0 = 0.0f, phi1 = 0.0f, phi2 = 0.0f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (d[i] != 0.0f) {
            ++moving;
            const float pl = (d[i] > 0.0f) ? lo[i] : hi[i];
            const float ph = (d[i] > 0.0f) ? hi[i] : lo[i];
            if (i == 0) { plo0 = pl; phi0 = ph; } else if (i == 1) { plo1 = pl; phi1 = ph; } else { plo2 = pl; phi2 = ph; }
            const float jl = (pl - a[i]) / d[i];
            const float jh = (ph - a[i]) / d[i];
            if (jl > L) { L = jl; iL = i; }
            if (jh < U) { U = jh; jU = i; }
        }
    }
    if (moving == 0) return INFINITY;
    if (L <= U) {
        float t;
        if (U < 0.0f) t = 0.0f;
        else if (L > 1.0f) t = 1.0f;
        else t = fmax2(L, 0.0f);
        return seg_g(a, d, t, lo, hi);
    }
    // the axis giving L lies below its slab and the one giving U above it on [U, L]
    const int k = 3 - iL - jU;
    // beta per axis for the pair {iL, jU}: plo for iL, phi for jU
    const float b0 = (iL == 0) ? plo0 : phi0;
    const float b1 = (iL == 1) ? plo1 : phi1;
    const float b2 = (iL == 2) ? plo2 : phi2;
    const int p0 = iL < jU ? iL : jU, p1 = iL < jU ? jU : iL;
    const float a0 = sel3(p0, a[0], a[1], a[2]), a1 = sel3(p1, a[0], a[1], a[2]);
    const float d0 = sel3(p0, d[0], d[1], d[2]), d1 = sel3(p1, d[0], d[1], d[2]);
    const float e0 = sel3(p0, b0, b1, b2), e1 = sel3(p1, b0, b1, b2);
    float num = d0 * (e0 - a0);
    float den = d0 * d0;
    num = num + d1 * (e1 - a1);
    den = den + d1 * d1;
    float gmin = seg_g(a, d, num / den, lo, hi);
    const float dk = sel3(k, d[0], d[1], d[2]);
    if (dk != 0.0f) {
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            // beta: iL -> plo, jU -> phi, k -> plo (side 0) or phi (side 1)
            const float c0 = (k == 0) ? (side == 0 ? plo0 : phi0) : b0;
            const float c1 = (k == 1) ? (side == 0 ? plo1 : phi1) : b1;
            const float c2 = (k == 2) ? (side == 0 ? plo2 : phi2) : b2;
            float n3 = d[0] * (c0 - a[0]);
            float d3 = d[0] * d[0];
            n3 = n3 + d[1] * (c1 - a[1]);
            d3 = d3 + d[1] * d[1];
            n3 = n3 + d[2] * (c2 - a[2]);
            d3 = d3 + d[2] * d[2];
            const float gc = seg_g(a, d, n3 / d3, lo, hi);
            if (gc < gmin) gmin = gc;
        }
    }
    return gmin;
}

// Per-axis terms of steps 1 and 2 for the sub-cell interval [k/8, (k+1)/8] of one axis.
struct AxisTerms {
    float g2, ea2, eb2;
};
// The gap (lo > mx ? lo - mx : mn > hi ? mn - hi : 0) is written max(lo - mx, mn - hi, 0):
// at most one of the two differences is positive, and a difference is positive exactly when
// its comparison holds (FP subtraction of finite values), so the two forms round to the same
// value up to the sign of a zero, which the square removes.  Likewise the endpoint distances.
// max of three (one instruction on sm_100 and later; exact, like two two-input maxima)
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float gap3(float lo, float hi, float mn, float mx) {
    return fmax3(lo - mx, mn - hi, 0.0f);
}
__device__ __forceinline__ AxisTerms axis_terms(float a, float b, int k) {
    const float lo = (float)k * 0.125f, hi = (float)(k + 1) * 0.125f;
    const float mn = fminf(a, b), mx = fmaxf(a, b);
    const float g = gap3(lo, hi, mn, mx);
    const float ea = gap3(lo, hi, a, a);
    const float eb = gap3(lo, hi, b, b);
    AxisTerms t;
    t.g2 = g * g;
    t.ea2 = ea * ea;
    t.eb2 = eb * eb;
    return t;
}

// Per-axis bounds over a union of sub-cell intervals [lo, hi] on one axis:
//   gap  <= the step-1 gap of every sub-cell inside (FP subtraction is monotone)
//   farA >= the step-2 distance of endpoint a to every sub-cell inside, likewise farB.
struct AxisBound {
    float g2, fa2, fb2;
};
__device__ __forceinline__ AxisBound axis_bound(float a, float b, float lo, float hi) {
    const float mn = fminf(a, b), mx = fmaxf(a, b);
    const float g = gap3(lo, hi, mn, mx);
    const float fa = fmaxf(hi - a, a - lo);
    const float fb = fmaxf(hi - b, b - lo);
    AxisBound r;
    r.g2 = g * g;
    r.fa2 = fa * fa;
    r.fb2 = fb * fb;
    return r;
}

// Per-warp pool of step-3 work of one voxel: (capsule slot, sub-cell) tasks left undecided
// by steps 1-2 of the batch's capsules, those capsules, and the voxel's mask while the pool
// is evaluated.  Tasks of many capsules are evaluated 32 at a time, so that the exact
// minimum (the expensive case) runs with all lanes busy.
constexpr int CT_TASKS = 512;
// One capsule in voxel-local grid units: (a.xyz, r^2), (b.xyz, r + eta), (d = b - a, 1 / |d|^2)
// with eta the margin of capsule_cell_separated.
struct CapsuleLocal {
    float4 a_rr, b_reta, d_idd;
};
// The x-axis terms of steps 1-2 for the 8 sub-cell columns sx = 0..7 (the same for every
// lane): squared gap of the segment's extent, squared distances of the endpoints.
struct CapsuleX {
    float4 g2[2], ea2[2], eb2[2];
    float4 bx;                     // the voxel's x interval [0, 1]: gap^2, far_a^2, far_b^2
};
struct CapsuleTasks {
    uint16_t task[CT_TASKS];       // batch slot << 9 | sub-cell id
    uint32_t mask[16];             // 512-bit mask, word w = lanes 2w (low half) and 2w+1
    float q[32 * 7];               // w mu and w mu T(t) of up to 32 pairs (pair-major, stride 7)
    CapsuleLocal batch[32];        // the batch's capsules (by lane)
    CapsuleX xt[32];               // their x-axis terms
};

__device__ __forceinline__ CapsuleX capsule_x(float a, float b) {
    float g[8], ea[8], eb[8];
#pragma unroll
    for (int sx = 0; sx < 8; ++sx) {
        const AxisTerms t = axis_terms(a, b, sx);
        g[sx] = t.g2;
        ea[sx] = t.ea2;
        eb[sx] = t.eb2;
    }
    CapsuleX x;
    x.g2[0] = make_float4(g[0], g[1], g[2], g[3]);
    x.g2[1] = make_float4(g[4], g[5], g[6], g[7]);
    x.ea2[0] = make_float4(ea[0], ea[1], ea[2], ea[3]);
    x.ea2[1] = make_float4(ea[4], ea[5], ea[6], ea[7]);
    x.eb2[0] = make_float4(eb[0], eb[1], eb[2], eb[3]);
    x.eb2[1] = make_float4(eb[4], eb[5], eb[6], eb[7]);
    const AxisBound bx = axis_bound(a, b, 0.0f, 1.0f);
    x.bx = make_float4(bx.g2, bx.fa2, bx.fb2, 0.0f);
    return x;
}

// Steps 1-2 of the capsule test for the 16 sub-cells of one lane (sx = 0..7,
// sy = sy0 + (0|1), sz); bit b = sx + 8 (sy - sy0), so lane L holds bits 16L .. 16L+15 of
// the voxel's 512-bit mask (bit id sx + 8 sy + 64 sz).  Bits already set in `have` are
// skipped (OR is idempotent).  Returns `have` plus the bits step 1-2 decide set; `und`
// receives the sub-cells left for step 3.
// Both steps compare the x term with what r^2 leaves after the y and z terms:
//   step 1 fails  when  g_x^2 > r^2 - (g_y^2 + g_z^2),
//   step 2 passes when  e_x^2 <= r^2 - (e_y^2 + e_z^2)  for endpoint a or b,
// so a row's 8 sub-cells compare 8 x terms with one budget each.
// A group of sub-cells (the lane's 16, or one row of 8) is decided at once when its per-axis
// gap bounds fail step 1, or an endpoint's far bounds pass step 2: FP addition and
// subtraction are monotone, so every sub-cell inside then fails (passes) too, and the group
// result equals the per-sub-cell definition bit for bit.
__device__ __forceinline__ uint32_t capsule_steps12(const CapsuleLocal& c, const CapsuleX& X, int sy0, int sz,
                                                    uint32_t have, uint32_t& und) {
    uint32_t bits = have;
    und = 0;
    if (have == 0xffffu) return bits;
    const float a[3] = {c.a_rr.x, c.a_rr.y, c.a_rr.z}, b[3] = {c.b_reta.x, c.b_reta.y, c.b_reta.z};
    const float rr = c.a_rr.w;
    const float zlo = (float)sz * 0.125f, zhi = (float)(sz + 1) * 0.125f;
    const AxisBound bz = axis_bound(a[2], b[2], zlo, zhi);
    const float4 bxv = X.bx;
    const AxisBound bx = {bxv.x, bxv.y, bxv.z};
    const AxisBound bb = axis_bound(a[1], b[1], (float)sy0 * 0.125f, (float)(sy0 + 2) * 0.125f);
    if (bx.g2 > rr - (bb.g2 + bz.g2)) return bits;                       // all 16 fail step 1
    if (bx.fa2 <= rr - (bb.fa2 + bz.fa2) || bx.fb2 <= rr - (bb.fb2 + bz.fb2)) return 0xffffu;
    const AxisTerms tz = axis_terms(a[2], b[2], sz);
#pragma unroll
    for (int yi = 0; yi < 2; ++yi) {
        const uint32_t rowmask = 0xffu << (8 * yi);
        if ((bits & rowmask) == rowmask) continue;
        const float ylo = (float)(sy0 + yi) * 0.125f, yhi = (float)(sy0 + yi + 1) * 0.125f;
        const AxisBound by = axis_bound(a[1], b[1], ylo, yhi);
        if (bx.g2 > rr - (by.g2 + bz.g2)) continue;
        if (bx.fa2 <= rr - (by.fa2 + bz.fa2) || bx.fb2 <= rr - (by.fb2 + bz.fb2)) {
            bits |= rowmask;
            continue;
        }
        const AxisTerms ty = axis_terms(a[1], b[1], sy0 + yi);
        const float TG = rr - (ty.g2 + tz.g2);
        const float TA = rr - (ty.ea2 + tz.ea2);
        const float TB = rr - (ty.eb2 + tz.eb2);
        const float4 g0 = X.g2[0], g1 = X.g2[1], a0 = X.ea2[0], a1 = X.ea2[1], b0 = X.eb2[0], b1 = X.eb2[1];
        const float xg[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
        const float xa[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float xb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
        // per sub-cell: set when an endpoint passes step 2, open (step 3) when it passes
        // step 1 only.  e >= g on every axis (an endpoint is no closer to a sub-cell than the
        // segment's extent) and the operations are monotone, so a set sub-cell is open too;
        // bits set before are dropped from `und` at the end.
        uint32_t row_set = 0, row_open = 0;
#pragma unroll
        for (int sx = 0; sx < 8; ++sx) {
            row_set |= ((xa[sx] <= TA) || (xb[sx] <= TB) ? 1u : 0u) << sx;
            row_open |= (xg[sx] <= TG ? 1u : 0u) << sx;
        }
        bits |= row_set << (8 * yi);
        und |= row_open << (8 * yi);
    }
    und &= ~bits;
    return bits;
}

// Local capsule of endpoints a, b (voxel-local grid units) and radius r.  eta bounds, with
// a wide factor, the FP32 error of the separation test below plus that of step 3: both
// scale with the magnitude M of the local coordinates (and r), and sum to less than
// 3e-6 (M + r + 3).
__device__ __forceinline__ CapsuleLocal capsule_local(const float* a, const float* b, float r) {
    const float d[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    const float dd = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
    const float M = fmax3(fmax3(fabsf(a[0]), fabsf(a[1]), fabsf(a[2])), fmax3(fabsf(b[0]), fabsf(b[1]), fabsf(b[2])),
                          0.0f);
    const float eta = 2e-5f * ((M + r) + 3.0f);
    CapsuleLocal c;
    c.a_rr = make_float4(a[0], a[1], a[2], r * r);
    c.b_reta = make_float4(b[0], b[1], b[2], r + eta);
    c.d_idd = make_float4(d[0], d[1], d[2], dd > 0.0f ? 1.0f / dd : 0.0f);
    return c;
}

// True when segment a-b (a, b - a, 1/|b - a|^2) is farther than re from the cube of centre
// (cx, cy, cz) and half-size h.  For a unit n, the distance between two convex sets is at
// least their separation along n: here min(n.(a - c), n.(b - c)) - h |n|_1.  n is taken along
// v = p - c, p the point of the segment nearest to c (any v gives a bound; this one is
// nearly tight once the box is a few box sizes away).  The test s > re |v|, s the separation
// times |v|, is done in squares.
__device__ __forceinline__ bool segment_box_separated(float4 a, float4 b, float4 d_idd, float cx, float cy, float cz,
                                                      float h, float re) {
    const float Ax = a.x - cx, Ay = a.y - cy, Az = a.z - cz;
    const float Bx = b.x - cx, By = b.y - cy, Bz = b.z - cz;
    float tc = -((Ax * d_idd.x + Ay * d_idd.y) + Az * d_idd.z) * d_idd.w;
    tc = fminf(fmaxf(tc, 0.0f), 1.0f);
    const float vx = Ax + tc * d_idd.x, vy = Ay + tc * d_idd.y, vz = Az + tc * d_idd.z;
    const float sa = (vx * Ax + vy * Ay) + vz * Az;
    const float sb = (vx * Bx + vy * By) + vz * Bz;
    const float sep = fminf(sa, sb) - h * ((fabsf(vx) + fabsf(vy)) + fabsf(vz));
    const float vv = (vx * vx + vy * vy) + vz * vz;
    return sep > 0.0f && sep * sep > (re * re) * vv;
}

// True when the capsule provably misses sub-cell `id` by more than the rounding of the
// exact minimum: separated by more than r + eta, eta (per capsule) covering the FP32 errors
// of this bound and of step 3.  Step 3's FP32 value is the squared distance of a point
// within ~1e-6 (M + 1) of the segment, to relative 1e-6, so a sub-cell separated by more
// than r + eta has that value above r^2: the task can be dropped without changing the mask.
__device__ __forceinline__ bool capsule_cell_separated(const CapsuleLocal& c, int id) {
    return segment_box_separated(c.a_rr, c.b_reta, c.d_idd, (float)(id & 7) * 0.125f + 0.0625f,
                                 (float)((id >> 3) & 7) * 0.125f + 0.0625f, (float)(id >> 6) * 0.125f + 0.0625f,
                                 0.0625f, c.b_reta.w);
}

// Step 3 of every pooled task whose sub-cell is not set yet (warp-collective); returns the
// lane's 16 bits of the updated mask.  A task skipped because an earlier task of the same
// sub-cell set it would have returned a bit that is already 1, so the order of evaluation
// does not change the mask.  Tasks whose sub-cell is separated from the capsule are dropped
// first (compacting the rest in place), so that the exact minimum runs on full warps.
__device__ __forceinline__ uint32_t capsule_step3_pool(CapsuleTasks& ct, int ntask, uint32_t chunk) {
    const int lane = threadIdx.x & 31;
    const uint32_t lo16 = __shfl_sync(0xffffffffu, chunk, (2 * lane) & 31);
    const uint32_t hi16 = __shfl_sync(0xffffffffu, chunk, (2 * lane + 1) & 31);
    if (lane < 16) ct.mask[lane] = lo16 | (hi16 << 16);
    __syncwarp();
    int nkeep = 0;
    for (int t0 = 0; t0 < ntask; t0 += 32) {
        const int t = t0 + lane;
        uint32_t task = 0;
        bool keep = false;
        if (t < ntask) {
            task = ct.task[t];
            const int id = (int)(task & 511u);
            keep = !(ct.mask[id >> 5] & (1u << (id & 31))) && !capsule_cell_separated(ct.batch[task >> 9], id);
        }
        const uint32_t kept = __ballot_sync(0xffffffffu, keep);
        __syncwarp();   // the chunk is read before any lane writes (writes land at or below it)
        if (keep) ct.task[nkeep + __popc(kept & ((1u << lane) - 1u))] = (uint16_t)task;
        nkeep += __popc(kept);
    }
    __syncwarp();
    for (int t = lane; t < nkeep; t += 32) {
        const uint32_t task = ct.task[t];
        const int id = (int)(task & 511u);
        const uint32_t bit = 1u << (id & 31);
        if (ct.mask[id >> 5] & bit) continue;
        const CapsuleLocal& c = ct.batch[task >> 9];
        const int sx = id & 7, sy = (id >> 3) & 7, zz = id >> 6;
        if (seg_box_min(c.a_rr.x, c.a_rr.y, c.a_rr.z, c.d_idd.x, c.d_idd.y, c.d_idd.z, (float)sx * 0.125f,
                        (float)sy * 0.125f, (float)zz * 0.125f, 0.125f) <= c.a_rr.w)
            atomicOr(&ct.mask[id >> 5], bit);
    }
    __syncwarp();
    const uint32_t w = ct.mask[lane >> 1];
    __syncwarp();
    return (w >> (16 * (lane & 1))) & 0xffffu;
}

// pi r^2 * length of the axis a-b clipped to the closed voxel [0,1]^3 (Liang-Barsky)
__device__ __forceinline__ float capsule_measure(const float* a, const float* b, float rg) {
    float d[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    float t0 = 0.0f, t1 = 1.0f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (d[i] == 0.0f) {
            if (a[i] < 0.0f || a[i] > 1.0f) return 0.0f;
        } else {
            float ta = (0.0f - a[i]) / d[i];
            float tb = (1.0f - a[i]) / d[i];
            float tn = d[i] > 0.0f ? ta : tb;
            float tf = d[i] > 0.0f ? tb : ta;
            if (tn > t0) t0 = tn;
            if (tf < t1) t1 = tf;
        }
    }
    if (t1 <= t0) return 0.0f;
    float dn = sqrtf((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
    float len = (t1 - t0) * dn;
    float rr = rg * rg;
    return (kPi * rr) * len;
}

// ------------------------------------------------------------------------------------
// triangle vs closed box: separating axis test (13 axes)
// ------------------------------------------------------------------------------------
__device__ __forceinline__ bool sep3(float p0, float p1, float p2, float rad) {
    float mn = fmin2(fmin2(p0, p1), p2), mx = fmax2(fmax2(p0, p1), p2);
    return (mn > rad || mx < -rad);
}

// all 13 axes for a box (centre c, half extent e); v local vertices, f global edges
__device__ __forceinline__ bool tri_box(const float v[3][3], const float f[3][3], const float* c, float e) {
    float w[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) w[k][i] = v[k][i] - c[i];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        if (sep3(w[0][i], w[1][i], w[2][i], e)) return false;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float* q = f[j];
        if (sep3(q[1] * w[0][2] - q[2] * w[0][1], q[1] * w[1][2] - q[2] * w[1][1], q[1] * w[2][2] - q[2] * w[2][1],
                 e * (fabsf(q[1]) + fabsf(q[2]))))
            return false;
        if (sep3(q[2] * w[0][0] - q[0] * w[0][2], q[2] * w[1][0] - q[0] * w[1][2], q[2] * w[2][0] - q[0] * w[2][2],
                 e * (fabsf(q[0]) + fabsf(q[2]))))
            return false;
        if (sep3(q[0] * w[0][1] - q[1] * w[0][0], q[0] * w[1][1] - q[1] * w[1][0], q[0] * w[2][1] - q[1] * w[2][0],
                 e * (fabsf(q[0]) + fabsf(q[1]))))
            return false;
    }
    float n0 = f[0][1] * f[1][2] - f[0][2] * f[1][1];
    float n1 = f[0][2] * f[1][0] - f[0][0] * f[1][2];
    float n2 = f[0][0] * f[1][1] - f[0][1] * f[1][0];
    float p = (n0 * w[0][0] + n1 * w[0][1]) + n2 * w[0][2];
    float rad = e * ((fabsf(n0) + fabsf(n1)) + fabsf(n2));
    return !(p > rad || p < -rad);
}

// One edge-family test for the sub-cell pair index q (two sub-cell coordinates (i0,i1)
// along the axes (ax0, ax1) that the family's axis depends on).
// family 0: e_x x f (axes y,z), 1: e_y x f (axes x,z), 2: e_z x f (axes x,y)
__device__ __forceinline__ bool family_pass(int fam, const float v[3][3], const float f[3][3], int i0, int i1) {
    const float e = 0.0625f;
    const float c0 = (float)(2 * i0 + 1) * 0.0625f, c1 = (float)(2 * i1 + 1) * 0.0625f;
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float* q = f[j];
        float p[3];
        float rad;
        if (fam == 0) {          // w_y = v_y - c(i0), w_z = v_z - c(i1)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                float wy = v[k][1] - c0, wz = v[k][2] - c1;
                p[k] = q[1] * wz - q[2] * wy;
            }
            rad = e * (fabsf(q[1]) + fabsf(q[2]));
        } else if (fam == 1) {   // w_x = v_x - c(i0), w_z = v_z - c(i1)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                float wx = v[k][0] - c0, wz = v[k][2] - c1;
                p[k] = q[2] * wx - q[0] * wz;
            }
            rad = e * (fabsf(q[0]) + fabsf(q[2]));
        } else {                 // w_x = v_x - c(i0), w_y = v_y - c(i1)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                float wx = v[k][0] - c0, wy = v[k][1] - c1;
                p[k] = q[0] * wy - q[1] * wx;
            }
            rad = e * (fabsf(q[0]) + fabsf(q[1]));
        }
        ok = ok && !sep3(p[0], p[1], p[2], rad);
    }
    return ok;
}

// 16 sub-cell bits of one lane (sx 0..7, sy0+{0,1}, sz).  Warp-collective: every lane
// of the warp must call it with the same triangle.
__device__ __forceinline__ uint32_t tri_bits16(const float v[3][3], const float f[3][3], int sy0, int sz) {
    const int lane = threadIdx.x & 31;
    const float e = 0.0625f;
    // edge families over the 64 index pairs, two per lane, collected by ballot
    uint64_t fam[3];
#pragma unroll
    for (int fa = 0; fa < 3; ++fa) {
        bool p_lo = family_pass(fa, v, f, lane & 7, lane >> 3);
        bool p_hi = family_pass(fa, v, f, (lane + 32) & 7, (lane + 32) >> 3);
        uint32_t blo = __ballot_sync(0xffffffffu, p_lo);
        uint32_t bhi = __ballot_sync(0xffffffffu, p_hi);
        fam[fa] = (uint64_t)blo | ((uint64_t)bhi << 32);
    }
    // box normals
    uint32_t bx = 0, by = 0;
    bool bz;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        float c = (float)(2 * k + 1) * 0.0625f;
        if (!sep3(v[0][0] - c, v[1][0] - c, v[2][0] - c, e)) bx |= 1u << k;
    }
#pragma unroll
    for (int yi = 0; yi < 2; ++yi) {
        float c = (float)(2 * (sy0 + yi) + 1) * 0.0625f;
        if (!sep3(v[0][1] - c, v[1][1] - c, v[2][1] - c, e)) by |= 1u << yi;
    }
    {
        float c = (float)(2 * sz + 1) * 0.0625f;
        bz = !sep3(v[0][2] - c, v[1][2] - c, v[2][2] - c, e);
    }
    if (!bz || !by || !bx) return 0;
    // face normal plane
    float n0 = f[0][1] * f[1][2] - f[0][2] * f[1][1];
    float n1 = f[0][2] * f[1][0] - f[0][0] * f[1][2];
    float n2 = f[0][0] * f[1][1] - f[0][1] * f[1][0];
    float rad = e * ((fabsf(n0) + fabsf(n1)) + fabsf(n2));
    float cz = (float)(2 * sz + 1) * 0.0625f;
    float pz = n2 * (v[0][2] - cz);
    uint32_t bits = 0;
#pragma unroll
    for (int yi = 0; yi < 2; ++yi) {
        const int sy = sy0 + yi;
        if (!((by >> yi) & 1u)) continue;
        float cy = (float)(2 * sy + 1) * 0.0625f;
        float py = n1 * (v[0][1] - cy);
#pragma unroll
        for (int sx = 0; sx < 8; ++sx) {
            if (!((bx >> sx) & 1u)) continue;
            if (!((fam[0] >> (sy + 8 * sz)) & 1ull)) continue;
            if (!((fam[1] >> (sx + 8 * sz)) & 1ull)) continue;
            if (!((fam[2] >> (sx + 8 * sy)) & 1ull)) continue;
            float cx = (float)(2 * sx + 1) * 0.0625f;
            float p = (n0 * (v[0][0] - cx) + py) + pz;
            if (p > rad || p < -rad) continue;
            bits |= 1u << (sx + 8 * yi);
        }
    }
    return bits;
}

// Clipped-polygon buffers of the triangle measure: two polygons of up to 12 vertices per
// thread, in shared memory with the thread index fastest (element (poly, vertex, coord) of
// thread t at [((poly * 12 + vertex) * 3 + coord) * NT + t]), so the threads of a warp hit
// 32 different banks.  NT = threads per block.
template <int NT>
struct PolyBuf {
    float x[2 * 12 * 3 * NT];
};

// Sutherland-Hodgman clip of polygon `pi` (n vertices) against coord_axis >= c (ge) or
// <= c into polygon `po`; returns the new vertex count.
template <int NT>
__device__ __forceinline__ int clip_plane_s(float* __restrict__ buf, int pi, int po, int n, int axis, float c, bool ge) {
    const int t = threadIdx.x;
    auto at = [&](int poly, int v, int j) -> float& { return buf[((poly * 12 + v) * 3 + j) * NT + t]; };
    int m = 0;
    for (int k = 0; k < n; ++k) {
        const int kn = (k + 1) == n ? 0 : k + 1;
        const float Sa = at(pi, k, axis), Ea = at(pi, kn, axis);
        const bool sin_ = ge ? (Sa >= c) : (Sa <= c);
        const bool ein = ge ? (Ea >= c) : (Ea <= c);
        if (ein) {
            if (!sin_) {
                const float sv = (c - Sa) / (Ea - Sa);
                for (int j = 0; j < 3; ++j) {
                    const float Sj = at(pi, k, j), Ej = at(pi, kn, j);
                    at(po, m, j) = (j == axis) ? c : Sj + sv * (Ej - Sj);
                }
                ++m;
            }
            for (int j = 0; j < 3; ++j) at(po, m, j) = at(pi, kn, j);
            ++m;
        } else if (sin_) {
            const float sv = (c - Sa) / (Ea - Sa);
            for (int j = 0; j < 3; ++j) {
                const float Sj = at(pi, k, j), Ej = at(pi, kn, j);
                at(po, m, j) = (j == axis) ? c : Sj + sv * (Ej - Sj);
            }
            ++m;
        }
    }
    return m;
}

// area (voxel units^2) of the triangle clipped to the voxel [0,1]^3
template <int NT>
__device__ float tri_measure(const float v[3][3], PolyBuf<NT>& pb) {
    float* buf = pb.x;
    const int t = threadIdx.x;
    auto at = [&](int poly, int vv, int j) -> float& { return buf[((poly * 12 + vv) * 3 + j) * NT + t]; };
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) at(0, k, j) = v[k][j];
    int n = 3;
    for (int axis = 0; axis < 3 && n > 0; ++axis) {
        n = clip_plane_s<NT>(buf, 0, 1, n, axis, 0.0f, true);
        if (n == 0) break;
        n = clip_plane_s<NT>(buf, 1, 0, n, axis, 1.0f, false);
    }
    if (n < 3) return 0.0f;
    float cx = 0.0f, cy = 0.0f, cz = 0.0f;
    const float a0 = at(0, 0, 0), a1 = at(0, 0, 1), a2 = at(0, 0, 2);
    for (int k = 1; k + 1 < n; ++k) {
        const float e1[3] = {at(0, k, 0) - a0, at(0, k, 1) - a1, at(0, k, 2) - a2};
        const float e2[3] = {at(0, k + 1, 0) - a0, at(0, k + 1, 1) - a1, at(0, k + 1, 2) - a2};
        cx = cx + (e1[1] * e2[2] - e1[2] * e2[1]);
        cy = cy + (e1[2] * e2[0] - e1[0] * e2[2]);
        cz = cz + (e1[0] * e2[1] - e1[1] * e2[0]);
    }
    return 0.5f * sqrtf((cx * cx + cy * cy) + cz * cz);
}

// ------------------------------------------------------------------------------------
// prep kernels
// ------------------------------------------------------------------------------------
// Segments per fiber; offsets that are negative, decrease, or pass num_ctrl are flagged.
__global__ void k_fiber_seg_counts(const int64_t* __restrict__ off, int64_t F, int64_t num_ctrl,
                                   uint32_t* __restrict__ cnt, uint32_t* __restrict__ err) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f < F) {
        const int64_t a = off[f], b = off[f + 1];
        if (a < 0 || b < a || b > num_ctrl) atomicOr(err, 1u);
        int64_t c = b - a - 1;
        cnt[f] = (uint32_t)(c > 0 ? c : 0);
    }
}

// rec_a = (A.xyz, r_g), rec_b = (B.xyz, w) in grid coordinates
// a record the method cannot use: a non-finite coordinate, radius or weight, or a negative
// radius or weight
__device__ __forceinline__ bool bad_record(float4 a, float4 b) {
    const bool fin = isfinite(a.x) && isfinite(a.y) && isfinite(a.z) && isfinite(a.w) && isfinite(b.x) &&
                     isfinite(b.y) && isfinite(b.z) && isfinite(b.w);
    return !fin || a.w < 0.0f || b.w < 0.0f;
}

// A segment whose control points fall outside ctrl[0, num_ctrl) (malformed offsets: negative,
// past the end, or decreasing) is flagged and not read.
__global__ void k_prep_fibers(const float4* __restrict__ ctrl, int64_t num_ctrl, const int64_t* __restrict__ off,
                              const uint32_t* __restrict__ seg_start, int64_t F, const uint32_t* __restrict__ seg_total,
                              const float* __restrict__ weights, uint32_t np, GridDev g, float4* __restrict__ ra,
                              float4* __restrict__ rb, uint32_t* __restrict__ err) {
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0 && *seg_total != np) atomicOr(err, 1u);
    if (p >= np) return;
    // last fiber with seg_start <= p (fibers without segments share the next start)
    int64_t lo = 0, hi = F;   // upper_bound in [0, F)
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (seg_start[mid] <= p) lo = mid + 1; else hi = mid;
    }
    int64_t f = lo - 1;
    if (f < 0) { atomicOr(err, 1u); return; }
    const int64_t o0 = off[f];
    int64_t c = o0 + (int64_t)(p - seg_start[f]);
    if (o0 < 0 || c < 0 || c + 1 >= off[f + 1] || c + 1 >= num_ctrl) { atomicOr(err, 1u); return; }
    float4 pa = ctrl[c], pb = ctrl[c + 1];
    float4 A, B;
    A.x = (pa.x - g.o[0]) * g.s; A.y = (pa.y - g.o[1]) * g.s; A.z = (pa.z - g.o[2]) * g.s;
    B.x = (pb.x - g.o[0]) * g.s; B.y = (pb.y - g.o[1]) * g.s; B.z = (pb.z - g.o[2]) * g.s;
    A.w = ((pa.w + pb.w) * 0.5f) * g.s;
    B.w = weights ? weights[p] : 1.0f;
    if (bad_record(A, B)) atomicOr(err, 1u);
    ra[p] = A;
    rb[p] = B;
}

// The tangent terms of each capsule's moment, T = (t_x^2, t_y^2, t_z^2, t_x t_y, t_x t_z,
// t_y t_z) with t = (B - A) / |B - A| (zero for a degenerate segment), as two float4 per
// primitive (the last two lanes zero).  These are the operations the reduce applied to every
// candidate pair; they depend on the primitive only, so they run once per primitive.
__global__ void k_tangent_terms(const float4* __restrict__ ra, const float4* __restrict__ rb, uint32_t np,
                                float4* __restrict__ rt) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const float4 A = ra[p], B = rb[p];
    const float dg[3] = {B.x - A.x, B.y - A.y, B.z - A.z};
    const float dn = sqrtf((dg[0] * dg[0] + dg[1] * dg[1]) + dg[2] * dg[2]);
    float t[3] = {0.0f, 0.0f, 0.0f};
    if (dn > 0.0f) { t[0] = dg[0] / dn; t[1] = dg[1] / dn; t[2] = dg[2] / dn; }
    rt[2 * (size_t)p] = make_float4(t[0] * t[0], t[1] * t[1], t[2] * t[2], t[0] * t[1]);
    rt[2 * (size_t)p + 1] = make_float4(t[0] * t[2], t[1] * t[2], 0.0f, 0.0f);
}

// tri records: (U0, w), (U1, 0), (U2, 0)
__global__ void k_prep_tris(const float4* __restrict__ tv, const float* __restrict__ weights, uint32_t np, GridDev g,
                            float4* __restrict__ r0, float4* __restrict__ r1, float4* __restrict__ r2,
                            uint32_t* __restrict__ err) {
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    float4 v0 = tv[3 * (size_t)p], v1 = tv[3 * (size_t)p + 1], v2 = tv[3 * (size_t)p + 2];
    float4 a, b, c;
    a.x = (v0.x - g.o[0]) * g.s; a.y = (v0.y - g.o[1]) * g.s; a.z = (v0.z - g.o[2]) * g.s;
    b.x = (v1.x - g.o[0]) * g.s; b.y = (v1.y - g.o[1]) * g.s; b.z = (v1.z - g.o[2]) * g.s;
    c.x = (v2.x - g.o[0]) * g.s; c.y = (v2.y - g.o[1]) * g.s; c.z = (v2.z - g.o[2]) * g.s;
    a.w = weights ? weights[p] : 1.0f;
    b.w = 0.0f;
    c.w = 0.0f;
    if (bad_record(a, b) || bad_record(c, c)) atomicOr(err, 1u);
    r0[p] = a; r1[p] = b; r2[p] = c;
}

// voxel range of a primitive: [lo, hi] per axis, empty when lo > hi on an axis
struct Range {
    int lo[3], n[3];
    long long total;
};
// voxel window of one pass: indices [lo, hi] per axis (a tile of the grid, or all of it);
// candidate keys are Morton codes relative to lo
struct Window {
    int lo[3], hi[3];
};
__host__ __device__ inline Window full_window(int R) {
    Window w;
    for (int i = 0; i < 3; ++i) { w.lo[i] = 0; w.hi[i] = R - 1; }
    return w;
}
// (ix, iy, iz) of flat index idx < tot in a range (x fastest).  Ranges of at most 2^16
// voxels divide by the correctly rounded FP32 reciprocal: (i + 0.5) fl(1/n), rounded, is
// within i / n (1 + 2^-23) of the quotient plus 0.5 / n, so its integer part is floor(i / n)
// (checked for every n and i below 2^16; tests/test_host_arith.py keeps every n up to 4096).  Larger ranges use 32-bit division when they hold
// fewer than 2^32 voxels (always inside a 1024^3 window).
__device__ __forceinline__ void voxel_of(long long idx, long long tot, const Range& rg, int& ix, int& iy, int& iz) {
    if (tot <= 65536) {
        const float r0 = __frcp_rn((float)rg.n[0]), r1 = __frcp_rn((float)rg.n[1]);
        const int i = (int)idx;
        const int t = (int)(((float)i + 0.5f) * r0);
        ix = i - t * rg.n[0];
        iz = (int)(((float)t + 0.5f) * r1);
        iy = t - iz * rg.n[1];
    } else if (tot <= 0xffffffffll) {
        const uint32_t i = (uint32_t)idx, n0 = (uint32_t)rg.n[0], n1 = (uint32_t)rg.n[1];
        const uint32_t t = i / n0;
        ix = (int)(i - t * n0);
        iz = (int)(t / n1);
        iy = (int)(t - (uint32_t)iz * n1);
    } else {
        const long long t = idx / rg.n[0];
        ix = (int)(idx - t * rg.n[0]);
        iz = (int)(t / rg.n[1]);
        iy = (int)(t - (long long)iz * rg.n[1]);
    }
}

__device__ __forceinline__ Range make_range(const float* mn, const float* mx, const Window& w) {
    Range r;
    r.total = 1;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float fl = floorf(mn[i]), fh = floorf(mx[i]);
        const int lo = fl < (float)w.lo[i] ? w.lo[i] : (fl > (float)w.hi[i] ? w.hi[i] + 1 : (int)fl);
        const int hi = fh < (float)w.lo[i] ? w.lo[i] - 1 : (fh > (float)w.hi[i] ? w.hi[i] : (int)fh);
        r.lo[i] = lo;
        // a NaN bound (rejected input, flagged by the prep kernels) gives an empty range
        r.n[i] = (mn[i] <= mx[i] && hi >= lo) ? hi - lo + 1 : 0;
        r.total *= r.n[i];
    }
    return r;
}

// conservative voxel-level tests (never reject a voxel with a set sub-cell)
__device__ __forceinline__ float capsule_margin(float rg) { return 2e-3f * fmax2(1.0f, rg) + 1e-4f; }

__device__ __forceinline__ Range capsule_range(float4 A, float4 B, const Window& R) {
    const float rc = A.w + capsule_margin(A.w) + 0.01f;
    float mn[3] = {fmin2(A.x, B.x) - rc, fmin2(A.y, B.y) - rc, fmin2(A.z, B.z) - rc};
    float mx[3] = {fmax2(A.x, B.x) + rc, fmax2(A.y, B.y) + rc, fmax2(A.z, B.z) + rc};
    return make_range(mn, mx, R);
}

// The voxel is kept unless steps 1-2 reject it at the inflated radius, or it is separated
// from the segment by more than that radius plus the separation test's rounding margin.
__device__ __forceinline__ bool capsule_voxel_candidate(float4 A, float4 B, int vi, int vj, int vk) {
    const float a[3] = {A.x - (float)vi, A.y - (float)vj, A.z - (float)vk};
    const float b[3] = {B.x - (float)vi, B.y - (float)vj, B.z - (float)vk};
    const float r = A.w + capsule_margin(A.w);
    const float rr = r * r;
    const float lo[3] = {0.0f, 0.0f, 0.0f}, hi[3] = {1.0f, 1.0f, 1.0f};
    float g[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) g[i] = gap3(0.0f, 1.0f, fmin2(a[i], b[i]), fmax2(a[i], b[i]));
    if ((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2] > rr) return false;
    if (sqdist_point_box(a[0], a[1], a[2], lo, hi) <= rr) return true;
    if (sqdist_point_box(b[0], b[1], b[2], lo, hi) <= rr) return true;
    const CapsuleLocal c = capsule_local(a, b, r);
    return !segment_box_separated(c.a_rr, c.b_reta, c.d_idd, 0.5f, 0.5f, 0.5f, 0.5f, c.b_reta.w);
}

__device__ __forceinline__ Range tri_range(float4 a, float4 b, float4 c, const Window& R) {
    const float m = 0.01f;
    float mn[3] = {fmin2(fmin2(a.x, b.x), c.x) - m, fmin2(fmin2(a.y, b.y), c.y) - m, fmin2(fmin2(a.z, b.z), c.z) - m};
    float mx[3] = {fmax2(fmax2(a.x, b.x), c.x) + m, fmax2(fmax2(a.y, b.y), c.y) + m, fmax2(fmax2(a.z, b.z), c.z) + m};
    return make_range(mn, mx, R);
}

__device__ __forceinline__ void tri_local(float4 a, float4 b, float4 c, int vi, int vj, int vk, float v[3][3],
                                          float f[3][3]) {
    v[0][0] = a.x - (float)vi; v[0][1] = a.y - (float)vj; v[0][2] = a.z - (float)vk;
    v[1][0] = b.x - (float)vi; v[1][1] = b.y - (float)vj; v[1][2] = b.z - (float)vk;
    v[2][0] = c.x - (float)vi; v[2][1] = c.y - (float)vj; v[2][2] = c.z - (float)vk;
    f[0][0] = b.x - a.x; f[0][1] = b.y - a.y; f[0][2] = b.z - a.z;
    f[1][0] = c.x - b.x; f[1][1] = c.y - b.y; f[1][2] = c.z - b.z;
    f[2][0] = a.x - c.x; f[2][1] = a.y - c.y; f[2][2] = a.z - c.z;
}

__device__ __forceinline__ bool tri_voxel_candidate(float4 a, float4 b, float4 c, int vi, int vj, int vk) {
    float v[3][3], f[3][3];
    tri_local(a, b, c, vi, vj, vk, v, f);
    const float ctr[3] = {0.5f, 0.5f, 0.5f};
    return tri_box(v, f, ctr, 0.5f + 2e-3f);
}

// ------------------------------------------------------------------------------------
// count / emit: warp per primitive over its voxel range
// ------------------------------------------------------------------------------------
// With `ballots`, the count pass stores each primitive's hit ballots (one word per 32 voxels
// of its range, ranges of at most 32 * CAND_BALLOTS voxels) and the emit pass of the same
// window reads them instead of testing again; larger ranges are tested in both passes.
// The ballots are the same bits either way, so the emitted order does not change.
constexpr int CAND_BALLOTS = 8;

template <bool FIBER, bool EMIT>
__global__ void __launch_bounds__(EMIT_WARPS * 32) k_candidates(const float4* __restrict__ r0,
                                                                const float4* __restrict__ r1,
                                                                const float4* __restrict__ r2, uint32_t np, Window R,
                                                                uint32_t* __restrict__ counts,
                                                                const uint32_t* __restrict__ offs,
                                                                uint32_t* __restrict__ keys,
                                                                uint32_t* __restrict__ vals,
                                                                uint32_t* __restrict__ ballots = nullptr) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * EMIT_WARPS;
    for (uint32_t p = blockIdx.x * EMIT_WARPS + (threadIdx.x >> 5); p < np; p += warps) {
        float4 a = r0[p], b = r1[p], c;
        Range rg;
        if (FIBER) {
            rg = capsule_range(a, b, R);
        } else {
            c = r2[p];
            rg = tri_range(a, b, c, R);
        }
        uint32_t n = 0;
        uint32_t base = EMIT ? offs[p] : 0u;
        const long long tot = rg.total;
        const bool stored = ballots != nullptr && tot <= 32ll * CAND_BALLOTS;
        uint32_t* const pb = stored ? ballots + (size_t)p * CAND_BALLOTS : nullptr;
        // emit: the primitive's stored words, one per lane, broadcast per step below
        uint32_t words = 0;
        if (EMIT && stored && (long long)lane * 32 < tot) words = pb[lane];
        for (long long idx0 = 0; idx0 < tot; idx0 += 32) {
            long long idx = idx0 + lane;
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
                uint32_t pos = base + n + __popc(bal & ((1u << lane) - 1u));
                keys[pos] = vx_morton3((uint32_t)(vi - R.lo[0]), (uint32_t)(vj - R.lo[1]), (uint32_t)(vk - R.lo[2]));
                vals[pos] = p;
            }
            n += __popc(bal);
        }
        if (!EMIT && lane == 0) counts[p] = n;
    }
}

// ------------------------------------------------------------------------------------
// segments
// ------------------------------------------------------------------------------------
// ------------------------------------------------------------------------------------
// reduce: warp per candidate voxel
// lane l owns sub-cells sz = l >> 2, sy = 2 (l & 3) + {0,1}, sx = 0..7 (16 bits)
// ------------------------------------------------------------------------------------
// Writes one candidate voxel's outputs: its mask (lanes' 16-bit chunks gathered into the
// 8 words), key, non-empty flag and the sums spread over lanes 0..6 (lane c: component c).
__device__ __forceinline__ void write_seg7(SegOut out, uint32_t seg, uint32_t key, uint32_t chunk, float accc) {
    const int lane = threadIdx.x & 31;
    uint64_t w = (uint64_t)chunk << (16 * (lane & 3));
    w |= __shfl_down_sync(0xffffffffu, w, 1);
    w |= __shfl_down_sync(0xffffffffu, w, 2);
    const bool nz = __any_sync(0xffffffffu, chunk != 0);
    if ((lane & 3) == 0) out.mask[(size_t)seg * 8 + (lane >> 2)] = w;
    if (lane == 0) {
        out.key[seg] = key;
        out.mass[seg] = accc;
        out.nonzero[seg] = nz ? 1u : 0u;
    } else if (lane < 7) {
        out.moment[(size_t)seg * 6 + lane - 1] = accc;
    }
}

// Batch slot `lane` of a voxel at (fx, fy, fz): capsule p's local record, the x terms of its
// steps 1-2 and its w mu, w mu T(t) moment terms, in the warp's shared state.  Returns the
// key that orders the mask tests: capsules whose axis passes deepest into the voxel first
// (they set the most bits, so later capsules find more lanes already full).  The mask is an
// OR, so the order does not change it.
__device__ __forceinline__ uint32_t capsule_slot_setup(CapsuleTasks& ct, int lane, uint32_t p, float fx, float fy,
                                                       float fz, const float4* __restrict__ ra,
                                                       const float4* __restrict__ rb,
                                                       const float4* __restrict__ rt) {
    const float4 A = ra[p], B = rb[p];
    float a[3] = {A.x - fx, A.y - fy, A.z - fz};
    float b[3] = {B.x - fx, B.y - fy, B.z - fz};
    const CapsuleLocal cl = capsule_local(a, b, A.w);
    ct.batch[lane] = cl;
    ct.xt[lane] = capsule_x(a[0], b[0]);
    uint32_t okey;
    {
        // squared distance from the voxel centre to the axis, minus r^2 (an ordering key only:
        // any rounding of it leaves the outputs unchanged)
        const float e[3] = {cl.d_idd.x, cl.d_idd.y, cl.d_idd.z};
        const float w[3] = {0.5f - a[0], 0.5f - a[1], 0.5f - a[2]};
        float tt = ((w[0] * e[0] + w[1] * e[1]) + w[2] * e[2]) * cl.d_idd.w;
        tt = fminf(fmaxf(tt, 0.0f), 1.0f);
        const float dx = w[0] - tt * e[0], dy = w[1] - tt * e[1], dz = w[2] - tt * e[2];
        const float v = ((dx * dx + dy * dy) + dz * dz) - A.w * A.w;
        uint32_t bits = __float_as_uint(v);
        bits ^= (bits >> 31) ? 0xffffffffu : 0x80000000u;   // order-preserving as unsigned
        okey = (min(bits, 0xffffffbfu) & 0xffffffe0u) | (uint32_t)lane;   // below the empty lanes
    }
    const float mu = capsule_measure(a, b, A.w);
    // w mu and w mu T(t), T the primitive's tangent terms (k_tangent_terms)
    const float4 T0 = rt[2 * (size_t)p], T1 = rt[2 * (size_t)p + 1];
    const float c = B.w * mu;
    float* q = ct.q + lane * 7;
    q[0] = c;
    q[1] = c * T0.x;
    q[2] = c * T0.y;
    q[3] = c * T0.z;
    q[4] = c * T0.w;
    q[5] = c * T1.x;
    q[6] = c * T1.y;
    return okey;
}

// Steps 1-3 of the `cnt` capsules of one voxel whose ordering keys sit at lanes src0,
// src0 + dir, ... of `okey` (the batch slot is a key's low 5 bits), on top of the lane's
// 16-bit chunk of the mask.  The pooled step-3 tasks refer to this batch's slots, so they
// are evaluated before the function returns.
__device__ __forceinline__ uint32_t voxel_mask(CapsuleTasks& ct, uint32_t okey, uint32_t cnt, int src0, int dir,
                                               int sy0, int sz, uint32_t chunk, bool& full) {
    const int lane = threadIdx.x & 31;
    int ntask = 0;
    for (uint32_t j = 0; j < cnt; ++j) {
        if (full) break;
        const int slot = (int)(__shfl_sync(0xffffffffu, okey, src0 + dir * (int)j) & 31u);
        uint32_t und;
        chunk = capsule_steps12(ct.batch[slot], ct.xt[slot], sy0, sz, chunk, und);
        // pool the undecided sub-cells as step-3 tasks of this capsule
        if (__any_sync(0xffffffffu, und != 0u)) {
            const uint32_t n = __popc(und);
            uint32_t off = n;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, off, o);
                if (lane >= o) off += t;
            }
            const int total = (int)__shfl_sync(0xffffffffu, off, 31);
            if (ntask + total > CT_TASKS) {
                chunk = capsule_step3_pool(ct, ntask, chunk);
                ntask = 0;
            }
            uint32_t pos = (uint32_t)ntask + off - n;
            uint32_t u = und;
            while (u) {
                const int bpos = __ffs(u) - 1;
                u &= u - 1;
                ct.task[pos++] = (uint16_t)((slot << 9) | (16 * lane + bpos));
            }
            ntask += total;
            __syncwarp();
        }
        full = __all_sync(0xffffffffu, chunk == 0xffffu);
    }
    if (ntask > 0 && !full) chunk = capsule_step3_pool(ct, ntask, chunk);
    return chunk;
}

// Voxel origin (grid units) of a window-relative Morton key.
__device__ __forceinline__ void voxel_origin(uint32_t key, int bx, int by, int bz, float& fx, float& fy, float& fz) {
    fx = (float)((int)vx_compact1by2(key) + bx);
    fy = (float)((int)vx_compact1by2(key >> 1) + by);
    fz = (float)((int)vx_compact1by2(key >> 2) + bz);
}

// Warp per candidate voxel, four voxels per step.  The step's voxels form groups of
// consecutive voxels whose capsules fit one batch (at most 32 together), and one setup serves
// a group: lane l takes the group's l-th capsule (the capsules of consecutive voxels are
// consecutive in the sorted pairs), the sums of voxel u run on lanes 7u .. 7u+6, and one
// ordering sort with the voxel above the distance key leaves each voxel's capsules together,
// in voxel order; then the mask steps run voxel by voxel.  A voxel of more than 32 capsules
// is a group of its own and runs in batches of 32.  The setup, the mask steps and the output
// each have one call site, so that the kernel holds one copy of them.
__global__ void __launch_bounds__(RED_WARPS * 32, 7) k_reduce_fibers(const uint32_t* __restrict__ keys,
                                                                  const uint32_t* __restrict__ prims,
                                                                  const uint32_t* __restrict__ starts,
                                                                  const uint32_t* __restrict__ nseg_p,
                                                                  const float4* __restrict__ ra,
                                                                  const float4* __restrict__ rb,
                                                                  const float4* __restrict__ rt, SegOut out,
                                                                  int bx, int by, int bz,
                                                                  uint32_t* __restrict__ next) {
    constexpr uint32_t STEP = 4;   // voxels per warp step (a group's voxel index takes 2 bits)
    const int lane = threadIdx.x & 31;
    const uint32_t nseg = *nseg_p;
    const int sz = lane >> 2, sy0 = (lane & 3) * 2;
    const uint32_t warps = gridDim.x * RED_WARPS;
    __shared__ CapsuleTasks pool[RED_WARPS];
    CapsuleTasks& ct = pool[threadIdx.x >> 5];
    // voxels are taken STEP at a time from the counter `next` when it is given (a grid of
    // resident blocks), else in a fixed grid stride
    auto take = [&]() -> uint32_t {
        uint32_t v = 0;
        if (lane == 0) v = atomicAdd(next, STEP);
        return __shfl_sync(0xffffffffu, v, 0);
    };
    for (uint32_t s0 = next ? take() : STEP * (blockIdx.x * RED_WARPS + (threadIdx.x >> 5)); s0 < nseg;
         s0 = next ? take() : s0 + STEP * warps) {
        const uint32_t s_end = min(s0 + STEP, nseg);
        for (uint32_t g = s0; g < s_end;) {
            // the group [g, g + m): consecutive voxels of at most 32 capsules together, or one voxel
            const uint32_t gbeg = starts[g];
            uint32_t m = 1, gend = starts[g + 1];
            while (g + m < s_end) {
                const uint32_t nx = starts[g + m + 1];
                if (nx - gbeg > 32u) break;
                gend = nx;
                ++m;
            }
            uint32_t chunk = 0;
            bool full = false;
            float accc = 0.0f;   // lane 7u + c: component c of voxel u's sums
            for (uint32_t base = gbeg; base < gend; base += 32) {
                const uint32_t cnt = min(32u, gend - base);
                // the lane's voxel in the group, and its origin
                uint32_t v = 0;
                for (uint32_t t = 1; t < m; ++t) v += (base + (uint32_t)lane >= starts[g + t]) ? 1u : 0u;
                float fx, fy, fz;
                voxel_origin(keys[starts[g + v]], bx, by, bz, fx, fy, fz);
                __syncwarp();   // the previous batch's sums have read ct.q
                uint32_t okey = 0xffffffe0u | (uint32_t)lane;
                if ((uint32_t)lane < cnt) {
                    okey = capsule_slot_setup(ct, lane, prims[base + lane], fx, fy, fz, ra, rb, rt);
                    // the voxel above the distance key (still below the empty lanes' keys)
                    if (m > 1) okey = (v << 30) | ((okey >> 2) & 0x3fffffc0u) | (uint32_t)lane;
                }
                __syncwarp();
                // sums in primitive order, one component per lane (the same sequence of FP32
                // additions as a single running sum per component); all voxels at once
                if ((uint32_t)lane < 7u * m) {
                    const uint32_t u = (uint32_t)lane / 7u;
                    const uint32_t ub = m > 1 ? starts[g + u] - base : 0u;
                    const uint32_t un = m > 1 ? starts[g + u + 1] - starts[g + u] : cnt;
                    const float* q = ct.q + ub * 7 + ((uint32_t)lane - 7u * u);
                    for (uint32_t j = 0; j < un; ++j) accc = accc + q[j * 7];
                }
                // bitonic sort of the keys (unique: the lane is the low 5 bits); after the
                // stage of width k, lanes 0..k-1 hold their keys in ascending order, so the sort
                // stops once k covers the batch
#pragma unroll
                for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
                    for (int jj = k >> 1; jj > 0; jj >>= 1) {
                        const uint32_t other = __shfl_xor_sync(0xffffffffu, okey, jj);
                        const bool keep_min = ((lane & k) == 0) == ((lane & jj) == 0);
                        okey = keep_min ? min(okey, other) : max(okey, other);
                    }
                    if ((uint32_t)k >= cnt) break;
                }
                // the mask steps, voxel by voxel; a voxel's outputs once its last batch is in
                for (uint32_t u = 0; u < m; ++u) {
                    const uint32_t ub = m > 1 ? starts[g + u] - base : 0u;
                    const uint32_t un = m > 1 ? starts[g + u + 1] - starts[g + u] : cnt;
                    chunk = voxel_mask(ct, okey, un, (int)ub, 1, sy0, sz, chunk, full);
                    if (m > 1 || base + cnt >= gend) {
                        write_seg7(out, g + u, keys[starts[g + u]], chunk,
                                   __shfl_down_sync(0xffffffffu, accc, 7 * u));
                        chunk = 0;
                        full = false;
                    }
                }
            }
            g += m;
        }
    }
}

__global__ void __launch_bounds__(RED_WARPS * 32, 5) k_reduce_tris(const uint32_t* __restrict__ keys,
                                                                const uint32_t* __restrict__ prims,
                                                                const uint32_t* __restrict__ starts,
                                                                const uint32_t* __restrict__ nseg_p,
                                                                const float4* __restrict__ r0,
                                                                const float4* __restrict__ r1,
                                                                const float4* __restrict__ r2, SegOut out,
                                                                int bx, int by, int bz,
                                                                uint32_t* __restrict__ next) {
    const int lane = threadIdx.x & 31;
    const uint32_t nseg = *nseg_p;
    const int sz = lane >> 2, sy0 = (lane & 3) * 2;
    const uint32_t warps = gridDim.x * RED_WARPS;
    // voxels from the counter `next` when given (resident blocks), else a fixed grid stride
    auto take = [&]() -> uint32_t {
        uint32_t v = 0;
        if (lane == 0) v = atomicAdd(next, 1u);
        return __shfl_sync(0xffffffffu, v, 0);
    };
    __shared__ PolyBuf<RED_WARPS * 32> polys;
    __shared__ float qs[RED_WARPS][32 * 7];       // per-pair w mu, w mu T(n) (pair-major)
    float* const qw = qs[threadIdx.x >> 5];
    for (uint32_t seg = next ? take() : blockIdx.x * RED_WARPS + (threadIdx.x >> 5); seg < nseg;
         seg = next ? take() : seg + warps) {
        const uint32_t beg = starts[seg], end = starts[seg + 1];
        const uint32_t key = keys[beg];
        const uint32_t ix = vx_compact1by2(key) + bx, iy = vx_compact1by2(key >> 1) + by,
                       iz = vx_compact1by2(key >> 2) + bz;
        uint32_t chunk = 0;
        bool full = false;
        float accc = 0.0f;   // lane c < 7: component c of the mass / moment sums
        for (uint32_t base = beg; base < end; base += 32) {
            const uint32_t cnt = min(32u, end - base);
            float q[7] = {0, 0, 0, 0, 0, 0, 0};
            __syncwarp();   // the previous batch's sums have read qw
            if (lane < cnt) {
                const uint32_t p = prims[base + lane];
                const float4 a = r0[p], b = r1[p], c = r2[p];
                float v[3][3], f[3][3];
                tri_local(a, b, c, (int)ix, (int)iy, (int)iz, v, f);
                float mu = tri_measure<RED_WARPS * 32>(v, polys);
                float n0 = f[0][1] * f[1][2] - f[0][2] * f[1][1];
                float n1 = f[0][2] * f[1][0] - f[0][0] * f[1][2];
                float n2 = f[0][0] * f[1][1] - f[0][1] * f[1][0];
                float nn = sqrtf((n0 * n0 + n1 * n1) + n2 * n2);
                float t[3] = {0.0f, 0.0f, 0.0f};
                if (nn > 0.0f) { t[0] = n0 / nn; t[1] = n1 / nn; t[2] = n2 / nn; }
                float cc = a.w * mu;
                q[0] = cc;
                q[1] = cc * (t[0] * t[0]);
                q[2] = cc * (t[1] * t[1]);
                q[3] = cc * (t[2] * t[2]);
                q[4] = cc * (t[0] * t[1]);
                q[5] = cc * (t[0] * t[2]);
                q[6] = cc * (t[1] * t[2]);
#pragma unroll
                for (int c = 0; c < 7; ++c) qw[lane * 7 + c] = q[c];
            }
            __syncwarp();
            // sums in primitive order, one component per lane (one FP32 running sum each)
            if (lane < 7)
                for (uint32_t j = 0; j < cnt; ++j) accc = accc + qw[j * 7 + lane];
            for (uint32_t j = 0; j < cnt; ++j) {
                if (!full) {
                    const uint32_t p = prims[base + j];
                    const float4 a = r0[p], b = r1[p], c = r2[p];
                    float v[3][3], f[3][3];
                    tri_local(a, b, c, (int)ix, (int)iy, (int)iz, v, f);
                    chunk |= tri_bits16(v, f, sy0, sz);
                    full = __all_sync(0xffffffffu, chunk == 0xffffu);
                }
            }
        }
        write_seg7(out, seg, key, chunk, accc);
    }
}

// ------------------------------------------------------------------------------------
// finalize: compaction + occupancy + lobe
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void mask_counts(const uint64_t* m, uint16_t& occ, uint8_t* proj) {
    int o = 0, yz = 0, xz = 0;
    uint64_t orz = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        uint64_t x = m[w];
        o += __popcll(x);
        orz |= x;
        // along x: a row (byte) is occupied if any of its bits is
        uint64_t t = x | (x >> 4);
        t |= t >> 2;
        t |= t >> 1;
        yz += __popcll(t & 0x0101010101010101ull);
        // along y: OR of the 8 rows
        uint64_t r = x | (x >> 32);
        r |= r >> 16;
        r |= r >> 8;
        xz += __popc((uint32_t)(r & 0xffu));
    }
    occ = (uint16_t)o;
    proj[0] = (uint8_t)yz;
    proj[1] = (uint8_t)xz;
    proj[2] = (uint8_t)__popcll(orz);
}

__device__ __forceinline__ void write_lobe(float m, const float* M, float* lobe, float* comp, uint8_t* cnt) {
    if (m > 0.0f) {
        float S[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) S[c] = M[c] / m;
#pragma unroll
        for (int c = 0; c < 6; ++c) lobe[c] = S[c];
        lobe[6] = m;
        comp[0] = sqrtf(S[0]);
        comp[1] = sqrtf(S[1]);
        comp[2] = sqrtf(S[2]);
        float pxy = S[0] * S[1], pxz = S[0] * S[2], pyz = S[1] * S[2];
        comp[3] = pxy > 0.0f ? S[3] / sqrtf(pxy) : 0.0f;
        comp[4] = pxz > 0.0f ? S[4] / sqrtf(pxz) : 0.0f;
        comp[5] = pyz > 0.0f ? S[5] / sqrtf(pyz) : 0.0f;
        *cnt = 1;
    } else {
#pragma unroll
        for (int c = 0; c < 7; ++c) lobe[c] = 0.0f;
#pragma unroll
        for (int c = 0; c < 6; ++c) comp[c] = 0.0f;
        *cnt = 0;
    }
}

__global__ void k_finalize(SegOut in, const uint32_t* __restrict__ nseg_p, const uint32_t* __restrict__ dst,
                           vx_level L, uint64_t key_hi) {
    const uint32_t nseg = *nseg_p;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += gridDim.x * blockDim.x) {
        if (!in.nonzero[s]) continue;
        const uint32_t o = dst[s];
        L.keys[o] = key_hi | (uint64_t)in.key[s];
        // 16-byte mask and 8-byte moment accesses (mask rows are 64-byte aligned, moment
        // rows 8-byte aligned in both the temporaries and the level block)
        uint64_t m[8];
        const uint4* mi = reinterpret_cast<const uint4*>(in.mask + (size_t)s * 8);
        uint4* mo = reinterpret_cast<uint4*>(L.mask + (size_t)o * 8);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const uint4 q = mi[w];
            mo[w] = q;
            m[2 * w] = ((uint64_t)q.y << 32) | q.x;
            m[2 * w + 1] = ((uint64_t)q.w << 32) | q.z;
        }
        float mass = in.mass[s];
        float M[6];
        const float2* Mi = reinterpret_cast<const float2*>(in.moment + (size_t)s * 6);
        float2* Mo = reinterpret_cast<float2*>(L.moment + (size_t)o * 6);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 q = Mi[c];
            Mo[c] = q;
            M[2 * c] = q.x;
            M[2 * c + 1] = q.y;
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
    }
}

inline unsigned grid_for(size_t n, int threads) {
    size_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 0x7fffffff) b = 0x7fffffff;
    return (unsigned)b;
}

}  // namespace
