/*
 * vxoracle.c -- plain, slow CPU oracle for the voxelization + LoD + SGGX-H path of
 * "Fast Voxelization and Level of Detail for Microgeometry Rendering" (Fabre et al.).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's CPU
 * baseline leg may load this library.  It shares no code, header or table with the
 * CUDA library; both implement the same written definitions independently.
 *
 * What it computes (the plain definition, evaluated per primitive over its bounding
 * box, then grouped per voxel):
 *   - grid coordinates u = (p - origin) * (1/h)                     (Sec. 3.1, P_volume)
 *   - per voxel and per 8^3 sub-cell: closed-box overlap with each primitive
 *     (capsule = segment inflated by its radius; triangle = separating axes)
 *     -> 512-bit mask, occupancy O = popcount/512                     (Sec. 3.5, Eq. for O)
 *     -> projected occupancies along x, y, z                          (Sec. 3.5, projections)
 *   - per voxel mass m = sum_p w_p mu_p(v) and second moment M = sum_p w_p mu_p d_p d_p^T
 *     (mu = clipped length * pi r^2 for fibers, clipped area for triangles; d = tangent
 *     or face normal; symmetric sign-free second moment)              (Sec. 4.1, covariance)
 *   - SGGX S = M/m and its compact parameters                        (Sec. 4.1, Eq. compact-sggx)
 *   - LoD: 2x2x2 aggregation of m, M, OR-downsampled masks           (Sec. 4.2, 4.3)
 *   - SGGX-H: agglomerative merging of sampled-histogram lobes       (Sec. 4.4, Eq. similarity)
 *
 * Precision: every quantity that decides an integer result (sub-cell bits, histogram
 * bins, merge argmins) is evaluated in IEEE FP32 with the operation order written
 * here, no contraction (build with -ffp-contract=off), exactly as the kernels take
 * those decisions.  Mass and moment are also accumulated in FP64, as the reference
 * value for the attribute tolerances: the exact (FP64) measures of the geometry after
 * its FP32 normalisation to grid coordinates (the normalised positions are the
 * method's input, Sec. 3.1).
 *
 * Parity unpinned: none of the functions here; see tests/test_oracle_pins.py and
 * tests/test_oracle_adjoint_pins.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_API __attribute__((visibility("default")))
#define M_PI_D 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* small helpers                                                             */
/* ------------------------------------------------------------------------- */
static float fmin2(float a, float b) { return (b < a) ? b : a; }
static float fmax2(float a, float b) { return (b > a) ? b : a; }

/* Morton key: x bit in position 0, y in 1, z in 2 of each bit triple. */
ORC_API uint64_t vxo_morton(uint32_t x, uint32_t y, uint32_t z) {
    uint64_t k = 0;
    for (int b = 0; b < 21; ++b) {
        k |= (uint64_t)((x >> b) & 1u) << (3 * b);
        k |= (uint64_t)((y >> b) & 1u) << (3 * b + 1);
        k |= (uint64_t)((z >> b) & 1u) << (3 * b + 2);
    }
    return k;
}

ORC_API void vxo_demorton(uint64_t k, uint32_t* x, uint32_t* y, uint32_t* z) {
    uint32_t a = 0, b = 0, c = 0;
    for (int i = 0; i < 21; ++i) {
        a |= (uint32_t)((k >> (3 * i)) & 1u) << i;
        b |= (uint32_t)((k >> (3 * i + 1)) & 1u) << i;
        c |= (uint32_t)((k >> (3 * i + 2)) & 1u) << i;
    }
    *x = a; *y = b; *z = c;
}

/* sub-cell index inside a voxel: sx + 8*sy + 64*sz; word = sz, bit = sx + 8*sy */
static void mask_set(uint64_t* m, int sx, int sy, int sz) { m[sz] |= 1ull << (sx + 8 * sy); }
static int mask_get(const uint64_t* m, int sx, int sy, int sz) { return (int)((m[sz] >> (sx + 8 * sy)) & 1ull); }

static int popcount64(uint64_t v) { int c = 0; while (v) { v &= v - 1; ++c; } return c; }

/* ------------------------------------------------------------------------- */
/* Capsule (segment a-b inflated by radius r) vs closed box [lo,hi]           */
/* a, b in voxel-local grid coordinates; d = b - a; rr = r*r.                */
/* Three steps, each an exact geometric statement:                           */
/*   1. lower bound: squared gaps between the segment's extent and the box   */
/*   2. an endpoint within r of the box                                      */
/*   3. min over t in [0,1] of squared distance from a + t d to the box,     */
/*      evaluated at the stationary points of the active quadratic pieces.   */
/* Steps 1 and 2 compare the x term with what r^2 leaves after the y and z   */
/* terms, x^2 <= r^2 - (y^2 + z^2): the same inequality as the sum of the    */
/* three squares <= r^2, in the FP32 form in which the kernels evaluate it.  */
/* ------------------------------------------------------------------------- */
static float box_sqdist_point(const float* p, const float* lo, const float* hi) {
    float e[3];
    for (int i = 0; i < 3; ++i) {
        if (p[i] < lo[i]) e[i] = lo[i] - p[i];
        else if (p[i] > hi[i]) e[i] = p[i] - hi[i];
        else e[i] = 0.0f;
    }
    return (e[0] * e[0] + e[1] * e[1]) + e[2] * e[2];
}

static float seg_box_g(const float* a, const float* d, float t, const float* lo, const float* hi) {
    float p[3];
    if (!(t >= 0.0f)) t = 0.0f;      /* also maps a NaN (0/0 from underflow) to 0 */
    else if (t > 1.0f) t = 1.0f;
    for (int i = 0; i < 3; ++i) p[i] = a[i] + t * d[i];
    return box_sqdist_point(p, lo, hi);
}

/* squared distance from p to the box, compared with rr in the form x^2 <= rr - (y^2 + z^2) */
static int box_point_within(const float* p, const float* lo, const float* hi, float rr) {
    float e[3];
    for (int i = 0; i < 3; ++i) {
        if (p[i] < lo[i]) e[i] = lo[i] - p[i];
        else if (p[i] > hi[i]) e[i] = p[i] - hi[i];
        else e[i] = 0.0f;
    }
    return e[0] * e[0] <= rr - (e[1] * e[1] + e[2] * e[2]);
}

ORC_API int vxo_capsule_box(const float* a, const float* b, float rr, const float* lo, const float* hi) {
    float d[3];
    for (int i = 0; i < 3; ++i) d[i] = b[i] - a[i];
    /* step 1 */
    float g[3];
    for (int i = 0; i < 3; ++i) {
        float mn = fmin2(a[i], b[i]), mx = fmax2(a[i], b[i]);
        if (lo[i] > mx) g[i] = lo[i] - mx;
        else if (mn > hi[i]) g[i] = mn - hi[i];
        else g[i] = 0.0f;
    }
    if (g[0] * g[0] > rr - (g[1] * g[1] + g[2] * g[2])) return 0;
    /* step 2 */
    if (box_point_within(a, lo, hi, rr)) return 1;
    if (box_point_within(b, lo, hi, rr)) return 1;
    /* step 3 */
    float L = -INFINITY, U = INFINITY;
    int iL = -1, jU = -1, moving = 0;
    float plo[3], phi[3];       /* plane giving the lower / upper end of the t-interval */
    for (int i = 0; i < 3; ++i) {
        if (d[i] != 0.0f) {
            ++moving;
            plo[i] = (d[i] > 0.0f) ? lo[i] : hi[i];
            phi[i] = (d[i] > 0.0f) ? hi[i] : lo[i];
            float jl = (plo[i] - a[i]) / d[i];
            float jh = (phi[i] - a[i]) / d[i];
            if (jl > L) { L = jl; iL = i; }
            if (jh < U) { U = jh; jU = i; }
        }
    }
    if (moving == 0) return 0;
    float gmin;
    if (L <= U) {
        float t;
        if (U < 0.0f) t = 0.0f;
        else if (L > 1.0f) t = 1.0f;
        else t = fmax2(L, 0.0f);
        gmin = seg_box_g(a, d, t, lo, hi);
    } else {
        /* iL is below its slab, jU above it, on the whole bracket [U, L] */
        float beta[3];
        int use[3] = {0, 0, 0};
        beta[iL] = plo[iL]; use[iL] = 1;
        beta[jU] = phi[jU]; use[jU] = 1;
        float num = 0.0f, den = 0.0f;
        int first = 1;
        for (int i = 0; i < 3; ++i) {
            if (!use[i]) continue;
            float ti = d[i] * (beta[i] - a[i]);
            float di = d[i] * d[i];
            if (first) { num = ti; den = di; first = 0; }
            else { num = num + ti; den = den + di; }
        }
        gmin = seg_box_g(a, d, num / den, lo, hi);
        int k = 3 - iL - jU;
        if (d[k] != 0.0f) {
            for (int side = 0; side < 2; ++side) {
                beta[k] = side == 0 ? plo[k] : phi[k];
                float n3 = 0.0f, d3 = 0.0f;
                for (int i = 0; i < 3; ++i) {
                    float ti = d[i] * (beta[i] - a[i]);
                    float di = d[i] * d[i];
                    if (i == 0) { n3 = ti; d3 = di; }
                    else { n3 = n3 + ti; d3 = d3 + di; }
                }
                float gc = seg_box_g(a, d, n3 / d3, lo, hi);
                if (gc < gmin) gmin = gc;
            }
        }
    }
    return gmin <= rr ? 1 : 0;
}

/* 512-bit sub-cell mask of a capsule in voxel (vi,vj,vk); A,B grid coordinates. */
ORC_API int vxo_capsule_mask(const float* A, const float* B, float rg,
                             int vi, int vj, int vk, uint64_t* mask) {
    float a[3] = {A[0] - (float)vi, A[1] - (float)vj, A[2] - (float)vk};
    float b[3] = {B[0] - (float)vi, B[1] - (float)vj, B[2] - (float)vk};
    float rr = rg * rg;
    int any = 0;
    for (int w = 0; w < 8; ++w) mask[w] = 0;
    for (int sz = 0; sz < 8; ++sz)
        for (int sy = 0; sy < 8; ++sy)
            for (int sx = 0; sx < 8; ++sx) {
                float lo[3] = {(float)sx * 0.125f, (float)sy * 0.125f, (float)sz * 0.125f};
                float hi[3] = {(float)(sx + 1) * 0.125f, (float)(sy + 1) * 0.125f, (float)(sz + 1) * 0.125f};
                if (vxo_capsule_box(a, b, rr, lo, hi)) { mask_set(mask, sx, sy, sz); any = 1; }
            }
    return any;
}

/* Fiber measure in a voxel: pi r^2 * length of the axis clipped to the closed voxel. */
ORC_API float vxo_capsule_measure(const float* A, const float* B, float rg, int vi, int vj, int vk) {
    float a[3] = {A[0] - (float)vi, A[1] - (float)vj, A[2] - (float)vk};
    float b[3] = {B[0] - (float)vi, B[1] - (float)vj, B[2] - (float)vk};
    float d[3];
    for (int i = 0; i < 3; ++i) d[i] = b[i] - a[i];
    float t0 = 0.0f, t1 = 1.0f;
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
    return (3.14159265358979f * rr) * len;
}

static double capsule_measure64(const double* A, const double* B, double rg, int vi, int vj, int vk) {
    double a[3] = {A[0] - vi, A[1] - vj, A[2] - vk};
    double d[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    double t0 = 0.0, t1 = 1.0;
    for (int i = 0; i < 3; ++i) {
        if (d[i] == 0.0) {
            if (a[i] < 0.0 || a[i] > 1.0) return 0.0;
        } else {
            double ta = -a[i] / d[i], tb = (1.0 - a[i]) / d[i];
            double tn = d[i] > 0 ? ta : tb, tf = d[i] > 0 ? tb : ta;
            if (tn > t0) t0 = tn;
            if (tf < t1) t1 = tf;
        }
    }
    if (t1 <= t0) return 0.0;
    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    return 3.14159265358979323846 * rg * rg * (t1 - t0) * dn;
}

/* ------------------------------------------------------------------------- */
/* Triangle vs closed axis-aligned box: separating axis theorem with the 13   */
/* axes (3 box normals, 9 edge cross products, the face normal).             */
/* v: voxel-local vertices; f: the three edges f0=v1-v0, f1=v2-v1, f2=v0-v2; */
/* box given by centre c and half extent e.                                  */
/* ------------------------------------------------------------------------- */
static int tri_box(const float v[3][3], const float f[3][3], const float* c, float e) {
    float w[3][3];
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 3; ++i) w[k][i] = v[k][i] - c[i];
    /* box normals */
    for (int i = 0; i < 3; ++i) {
        float mn = fmin2(fmin2(w[0][i], w[1][i]), w[2][i]);
        float mx = fmax2(fmax2(w[0][i], w[1][i]), w[2][i]);
        if (mn > e || mx < -e) return 0;
    }
    /* e_x x f, e_y x f, e_z x f */
    for (int j = 0; j < 3; ++j) {
        const float* fj = f[j];
        float p[3], rad, mn, mx;
        for (int k = 0; k < 3; ++k) p[k] = fj[1] * w[k][2] - fj[2] * w[k][1];
        rad = e * (fabsf(fj[1]) + fabsf(fj[2]));
        mn = fmin2(fmin2(p[0], p[1]), p[2]); mx = fmax2(fmax2(p[0], p[1]), p[2]);
        if (mn > rad || mx < -rad) return 0;
        for (int k = 0; k < 3; ++k) p[k] = fj[2] * w[k][0] - fj[0] * w[k][2];
        rad = e * (fabsf(fj[0]) + fabsf(fj[2]));
        mn = fmin2(fmin2(p[0], p[1]), p[2]); mx = fmax2(fmax2(p[0], p[1]), p[2]);
        if (mn > rad || mx < -rad) return 0;
        for (int k = 0; k < 3; ++k) p[k] = fj[0] * w[k][1] - fj[1] * w[k][0];
        rad = e * (fabsf(fj[0]) + fabsf(fj[1]));
        mn = fmin2(fmin2(p[0], p[1]), p[2]); mx = fmax2(fmax2(p[0], p[1]), p[2]);
        if (mn > rad || mx < -rad) return 0;
    }
    /* face normal n = f0 x f1, plane through v0 */
    float n[3];
    n[0] = f[0][1] * f[1][2] - f[0][2] * f[1][1];
    n[1] = f[0][2] * f[1][0] - f[0][0] * f[1][2];
    n[2] = f[0][0] * f[1][1] - f[0][1] * f[1][0];
    float p = (n[0] * w[0][0] + n[1] * w[0][1]) + n[2] * w[0][2];
    float rad = e * ((fabsf(n[0]) + fabsf(n[1])) + fabsf(n[2]));
    if (p > rad || p < -rad) return 0;
    return 1;
}

static void tri_local(const float* U, int vi, int vj, int vk, float v[3][3], float f[3][3]) {
    /* U: 9 floats, grid coordinates of v0, v1, v2 */
    for (int k = 0; k < 3; ++k) {
        v[k][0] = U[3 * k + 0] - (float)vi;
        v[k][1] = U[3 * k + 1] - (float)vj;
        v[k][2] = U[3 * k + 2] - (float)vk;
    }
    for (int i = 0; i < 3; ++i) {
        f[0][i] = U[3 + i] - U[i];
        f[1][i] = U[6 + i] - U[3 + i];
        f[2][i] = U[i] - U[6 + i];
    }
}

ORC_API int vxo_tri_mask(const float* U, int vi, int vj, int vk, uint64_t* mask) {
    float v[3][3], f[3][3];
    tri_local(U, vi, vj, vk, v, f);
    int any = 0;
    for (int w = 0; w < 8; ++w) mask[w] = 0;
    for (int sz = 0; sz < 8; ++sz)
        for (int sy = 0; sy < 8; ++sy)
            for (int sx = 0; sx < 8; ++sx) {
                float c[3] = {(float)(2 * sx + 1) * 0.0625f, (float)(2 * sy + 1) * 0.0625f,
                              (float)(2 * sz + 1) * 0.0625f};
                if (tri_box((const float(*)[3])v, (const float(*)[3])f, c, 0.0625f)) {
                    mask_set(mask, sx, sy, sz);
                    any = 1;
                }
            }
    return any;
}

/* Sutherland-Hodgman clip of a polygon against the plane x_axis >= c (keep_ge=1) or <= c. */
static int clip_plane(const float in[][3], int n, float out[][3], int axis, float c, int keep_ge) {
    int m = 0;
    for (int k = 0; k < n; ++k) {
        const float* S = in[k];
        const float* E = in[(k + 1) % n];
        int sin_ = keep_ge ? (S[axis] >= c) : (S[axis] <= c);
        int ein = keep_ge ? (E[axis] >= c) : (E[axis] <= c);
        if (ein) {
            if (!sin_) {
                float s = (c - S[axis]) / (E[axis] - S[axis]);
                for (int j = 0; j < 3; ++j) out[m][j] = (j == axis) ? c : S[j] + s * (E[j] - S[j]);
                ++m;
            }
            for (int j = 0; j < 3; ++j) out[m][j] = E[j];
            ++m;
        } else if (sin_) {
            float s = (c - S[axis]) / (E[axis] - S[axis]);
            for (int j = 0; j < 3; ++j) out[m][j] = (j == axis) ? c : S[j] + s * (E[j] - S[j]);
            ++m;
        }
    }
    return m;
}

/* Triangle measure in a voxel: area (voxel units^2) of the triangle clipped to the voxel. */
ORC_API float vxo_tri_measure(const float* U, int vi, int vj, int vk) {
    float v[3][3], f[3][3];
    tri_local(U, vi, vj, vk, v, f);
    float A[16][3], B[16][3];
    int n = 3;
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j) A[k][j] = v[k][j];
    for (int axis = 0; axis < 3 && n > 0; ++axis) {
        n = clip_plane((const float(*)[3])A, n, B, axis, 0.0f, 1);
        if (n == 0) break;
        n = clip_plane((const float(*)[3])B, n, A, axis, 1.0f, 0);
    }
    if (n < 3) return 0.0f;
    float cx = 0.0f, cy = 0.0f, cz = 0.0f;
    for (int k = 1; k + 1 < n; ++k) {
        float e1[3], e2[3];
        for (int j = 0; j < 3; ++j) { e1[j] = A[k][j] - A[0][j]; e2[j] = A[k + 1][j] - A[0][j]; }
        cx = cx + (e1[1] * e2[2] - e1[2] * e2[1]);
        cy = cy + (e1[2] * e2[0] - e1[0] * e2[2]);
        cz = cz + (e1[0] * e2[1] - e1[1] * e2[0]);
    }
    return 0.5f * sqrtf((cx * cx + cy * cy) + cz * cz);
}

static int clip_plane64(const double in[][3], int n, double out[][3], int axis, double c, int keep_ge) {
    int m = 0;
    for (int k = 0; k < n; ++k) {
        const double* S = in[k];
        const double* E = in[(k + 1) % n];
        int sin_ = keep_ge ? (S[axis] >= c) : (S[axis] <= c);
        int ein = keep_ge ? (E[axis] >= c) : (E[axis] <= c);
        if (ein) {
            if (!sin_) {
                double s = (c - S[axis]) / (E[axis] - S[axis]);
                for (int j = 0; j < 3; ++j) out[m][j] = (j == axis) ? c : S[j] + s * (E[j] - S[j]);
                ++m;
            }
            for (int j = 0; j < 3; ++j) out[m][j] = E[j];
            ++m;
        } else if (sin_) {
            double s = (c - S[axis]) / (E[axis] - S[axis]);
            for (int j = 0; j < 3; ++j) out[m][j] = (j == axis) ? c : S[j] + s * (E[j] - S[j]);
            ++m;
        }
    }
    return m;
}

ORC_API double vxo_tri_measure64(const double* U, int vi, int vj, int vk) {
    double A[16][3], B[16][3];
    int n = 3;
    for (int k = 0; k < 3; ++k) {
        A[k][0] = U[3 * k] - vi; A[k][1] = U[3 * k + 1] - vj; A[k][2] = U[3 * k + 2] - vk;
    }
    for (int axis = 0; axis < 3 && n > 0; ++axis) {
        n = clip_plane64((const double(*)[3])A, n, B, axis, 0.0, 1);
        if (n == 0) break;
        n = clip_plane64((const double(*)[3])B, n, A, axis, 1.0, 0);
    }
    if (n < 3) return 0.0;
    double cx = 0, cy = 0, cz = 0;
    for (int k = 1; k + 1 < n; ++k) {
        double e1[3], e2[3];
        for (int j = 0; j < 3; ++j) { e1[j] = A[k][j] - A[0][j]; e2[j] = A[k + 1][j] - A[0][j]; }
        cx += e1[1] * e2[2] - e1[2] * e2[1];
        cy += e1[2] * e2[0] - e1[0] * e2[2];
        cz += e1[0] * e2[1] - e1[1] * e2[0];
    }
    return 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
}

/* ------------------------------------------------------------------------- */
/* Voxelization: per primitive, over its bounding box; then grouped per key   */
/* in primitive order.                                                        */
/* ------------------------------------------------------------------------- */
typedef struct {
    uint64_t key;
    int64_t prim;
    uint64_t mask[8];
    float c;          /* w * mu   (FP32) */
    float dir[3];     /* unit orientation (FP32) */
    double c64;       /* w * mu   (FP64) */
    double dir64[3];
} rec_t;

typedef struct {
    rec_t* r;
    int64_t n, cap;
} recs_t;

static void recs_push(recs_t* R, const rec_t* x) {
    if (R->n == R->cap) {
        R->cap = R->cap ? 2 * R->cap : 4096;
        R->r = (rec_t*)realloc(R->r, (size_t)R->cap * sizeof(rec_t));
    }
    R->r[R->n++] = *x;
}

static int rec_cmp(const void* pa, const void* pb) {
    const rec_t* a = (const rec_t*)pa;
    const rec_t* b = (const rec_t*)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->prim != b->prim) return a->prim < b->prim ? -1 : 1;
    return 0;
}

/* A level of the pyramid as the oracle returns it (arrays malloc'ed here). */
typedef struct {
    int64_t n;
    int32_t K;
    uint64_t* keys;
    uint64_t* mask;      /* [n][8] */
    float* mass;         /* [n] FP32 chain */
    float* moment;       /* [n][6] xx,yy,zz,xy,xz,yz */
    double* mass64;      /* [n] */
    double* moment64;    /* [n][6] */
    uint16_t* occ;       /* [n] */
    uint8_t* proj;       /* [n][3] yz (along x), xz (along y), xy (along z) */
    uint8_t* lobe_count; /* [n] */
    float* lobes;        /* [n][K][7] S6 + weight */
    float* compact;      /* [n][K][6] */
} vxo_level;

ORC_API void vxo_level_free(vxo_level* L) {
    free(L->keys); free(L->mask); free(L->mass); free(L->moment); free(L->mass64);
    free(L->moment64); free(L->occ); free(L->proj); free(L->lobe_count); free(L->lobes);
    free(L->compact);
    memset(L, 0, sizeof(*L));
}

static void level_alloc(vxo_level* L, int64_t n, int K) {
    memset(L, 0, sizeof(*L));
    L->n = n; L->K = K;
    size_t nn = (size_t)(n > 0 ? n : 1);
    L->keys = (uint64_t*)calloc(nn, 8);
    L->mask = (uint64_t*)calloc(nn * 8, 8);
    L->mass = (float*)calloc(nn, 4);
    L->moment = (float*)calloc(nn * 6, 4);
    L->mass64 = (double*)calloc(nn, 8);
    L->moment64 = (double*)calloc(nn * 6, 8);
    L->occ = (uint16_t*)calloc(nn, 2);
    L->proj = (uint8_t*)calloc(nn * 3, 1);
    L->lobe_count = (uint8_t*)calloc(nn, 1);
    L->lobes = (float*)calloc(nn * (size_t)K * 7, 4);
    L->compact = (float*)calloc(nn * (size_t)K * 6, 4);
}

/* occupancy O (as a count of hit sub-cells) and the three projected counts */
static void mask_stats(const uint64_t* m, uint16_t* occ, uint8_t* proj) {
    int o = 0;
    for (int w = 0; w < 8; ++w) o += popcount64(m[w]);
    int yz = 0, xz = 0, xy = 0;
    for (int sz = 0; sz < 8; ++sz)
        for (int sy = 0; sy < 8; ++sy) {
            int any = 0;
            for (int sx = 0; sx < 8; ++sx) any |= mask_get(m, sx, sy, sz);
            yz += any;
        }
    for (int sz = 0; sz < 8; ++sz)
        for (int sx = 0; sx < 8; ++sx) {
            int any = 0;
            for (int sy = 0; sy < 8; ++sy) any |= mask_get(m, sx, sy, sz);
            xz += any;
        }
    for (int sy = 0; sy < 8; ++sy)
        for (int sx = 0; sx < 8; ++sx) {
            int any = 0;
            for (int sz = 0; sz < 8; ++sz) any |= mask_get(m, sx, sy, sz);
            xy += any;
        }
    *occ = (uint16_t)o;
    proj[0] = (uint8_t)yz; proj[1] = (uint8_t)xz; proj[2] = (uint8_t)xy;
}

/* Compact SGGX parameters (Eq. compact-sggx): sigma = sqrt(S_ii), r_ij = S_ij / sqrt(S_ii S_jj). */
ORC_API void vxo_compact(const float* S, float* out) {
    out[0] = sqrtf(S[0]);
    out[1] = sqrtf(S[1]);
    out[2] = sqrtf(S[2]);
    float pxy = S[0] * S[1], pxz = S[0] * S[2], pyz = S[1] * S[2];
    out[3] = pxy > 0.0f ? S[3] / sqrtf(pxy) : 0.0f;
    out[4] = pxz > 0.0f ? S[4] / sqrtf(pxz) : 0.0f;
    out[5] = pyz > 0.0f ? S[5] / sqrtf(pyz) : 0.0f;
}

/* Catmull-Rom spline fibers (Sec. 3.2: the spline through its stored nodes, sampled at
 * equally spaced t).  Spline f has nodes off[f] .. off[f+1]-1 (at least one each).  Span i
 * joins nodes i and i+1 and uses P0..P3 = nodes i-1, i, i+1, i+2; past either end the
 * missing node is the end node reflected through its neighbour (2 P_0 - P_1, 2 P_n-1 -
 * P_n-2), so that nodes on a line give points on it.  It gives S points at t = j / S,
 * j = 0..S-1, from the uniform
 * Catmull-Rom form
 *     C(t) = 0.5 (2 P1 + t (a + t (b + t c))),  a = P2 - P0,
 *     b = ((2 P0 - 5 P1) + 4 P2) - P3,  c = ((3 P1 - P0) - 3 P2) + P3,
 * and the radius linearly, r1 + t (r2 - r1).  The spline's last node closes it.  Output
 * spline f: (n_f - 1) S + 1 points from (off[f] - f) S + f.  FP32, in this order. */
ORC_API void vxo_catmull_rom(const float* nodes, const int64_t* off, int64_t F, int S, float* out,
                             int64_t* out_off) {
    for (int64_t f = 0; f <= F; ++f) out_off[f] = (off[f] - f) * S + f;
    for (int64_t f = 0; f < F; ++f) {
        const int64_t b = off[f], n = off[f + 1] - off[f];
        float* o = out + out_off[f] * 4;
        for (int64_t i = 0; i + 1 < n; ++i) {
            const float* P1 = nodes + (b + i) * 4;
            const float* P2 = nodes + (b + i + 1) * 4;
            float P0[3], P3[3];
            for (int k = 0; k < 3; ++k) {
                P0[k] = i > 0 ? nodes[(b + i - 1) * 4 + k] : 2.0f * P1[k] - P2[k];
                P3[k] = i + 2 < n ? nodes[(b + i + 2) * 4 + k] : 2.0f * P2[k] - P1[k];
            }
            for (int j = 0; j < S; ++j) {
                const float t = (float)j / (float)S;
                float* q = o + (i * S + j) * 4;
                for (int k = 0; k < 3; ++k) {
                    const float a = P2[k] - P0[k];
                    const float bb = ((2.0f * P0[k] - 5.0f * P1[k]) + 4.0f * P2[k]) - P3[k];
                    const float c = ((3.0f * P1[k] - P0[k]) - 3.0f * P2[k]) + P3[k];
                    q[k] = 0.5f * (2.0f * P1[k] + t * (a + t * (bb + t * c)));
                }
                q[3] = P1[3] + t * (P2[3] - P1[3]);
            }
        }
        if (n > 0) {
            const float* L = nodes + (b + n - 1) * 4;
            float* q = o + (n - 1) * S * 4;
            for (int k = 0; k < 4; ++k) q[k] = L[k];
        }
    }
}

/* 8-bit compact SGGX (Sec. 4.3, Eq. compact-sggx, one byte per parameter): sigma in [0, 1]
 * -> round(255 sigma), r in [-1, 1] -> round(127.5 r + 127.5), FP32, ties to even, clamped
 * to [0, 255].  c: n parameter sextuples; out: n * 6 bytes. */
static uint8_t quant8(float x, float scale, float bias) {
    float q = rintf(x * scale + bias);
    if (q < 0.0f) q = 0.0f;
    if (q > 255.0f) q = 255.0f;
    return (uint8_t)q;
}
ORC_API void vxo_compact8(const float* c, int64_t n, uint8_t* out) {
    for (int64_t i = 0; i < n; ++i) {
        for (int j = 0; j < 3; ++j) out[i * 6 + j] = quant8(c[i * 6 + j], 255.0f, 0.0f);
        for (int j = 3; j < 6; ++j) out[i * 6 + j] = quant8(c[i * 6 + j], 127.5f, 127.5f);
    }
}

/* single normalised lobe from (m, M): S = M / m, weight m */
static void single_lobe(vxo_level* L, int64_t v) {
    float m = L->mass[v];
    if (m > 0.0f) {
        float* lo = L->lobes + (size_t)v * L->K * 7;
        for (int c = 0; c < 6; ++c) lo[c] = L->moment[6 * v + c] / m;
        lo[6] = m;
        vxo_compact(lo, L->compact + (size_t)v * L->K * 6);
        L->lobe_count[v] = 1;
    } else {
        L->lobe_count[v] = 0;
    }
}

static void reduce_records(recs_t* R, vxo_level* out, int K) {
    qsort(R->r, (size_t)R->n, sizeof(rec_t), rec_cmp);
    /* count keys with a non-zero mask */
    int64_t nv = 0;
    for (int64_t i = 0; i < R->n;) {
        int64_t j = i;
        uint64_t any = 0;
        while (j < R->n && R->r[j].key == R->r[i].key) {
            for (int w = 0; w < 8; ++w) any |= R->r[j].mask[w];
            ++j;
        }
        if (any) ++nv;
        i = j;
    }
    level_alloc(out, nv, K);
    int64_t v = 0;
    for (int64_t i = 0; i < R->n;) {
        int64_t j = i;
        uint64_t m8[8] = {0};
        float m = 0.0f, M[6] = {0, 0, 0, 0, 0, 0};
        double m64 = 0.0, M64[6] = {0, 0, 0, 0, 0, 0};
        while (j < R->n && R->r[j].key == R->r[i].key) {
            const rec_t* x = &R->r[j];
            for (int w = 0; w < 8; ++w) m8[w] |= x->mask[w];
            float c = x->c;
            const float* t = x->dir;
            m = m + c;
            M[0] = M[0] + c * (t[0] * t[0]);
            M[1] = M[1] + c * (t[1] * t[1]);
            M[2] = M[2] + c * (t[2] * t[2]);
            M[3] = M[3] + c * (t[0] * t[1]);
            M[4] = M[4] + c * (t[0] * t[2]);
            M[5] = M[5] + c * (t[1] * t[2]);
            const double* t6 = x->dir64;
            m64 += x->c64;
            M64[0] += x->c64 * t6[0] * t6[0];
            M64[1] += x->c64 * t6[1] * t6[1];
            M64[2] += x->c64 * t6[2] * t6[2];
            M64[3] += x->c64 * t6[0] * t6[1];
            M64[4] += x->c64 * t6[0] * t6[2];
            M64[5] += x->c64 * t6[1] * t6[2];
            ++j;
        }
        uint64_t any = 0;
        for (int w = 0; w < 8; ++w) any |= m8[w];
        if (any) {
            out->keys[v] = R->r[i].key;
            memcpy(out->mask + 8 * v, m8, sizeof(m8));
            out->mass[v] = m;
            memcpy(out->moment + 6 * v, M, sizeof(M));
            out->mass64[v] = m64;
            memcpy(out->moment64 + 6 * v, M64, sizeof(M64));
            mask_stats(m8, &out->occ[v], &out->proj[3 * v]);
            single_lobe(out, v);
            ++v;
        }
        i = j;
    }
}

typedef struct {
    float origin[3];
    float voxel_size;
    int32_t resolution;
} vxo_grid;

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Fibers: ctrl [P][4] (xyz, radius), offsets [F+1]; segment s of fiber f joins
 * ctrl[off[f]+s] and ctrl[off[f]+s+1]; primitive ids count segments fiber by fiber. */
ORC_API int vxo_voxelize_fibers(const float* ctrl, const int64_t* offsets, int64_t F,
                                const float* weights, const vxo_grid* g, int K, vxo_level* out) {
    const float s = 1.0f / g->voxel_size;
    const int R = g->resolution;
    recs_t recs = {0, 0, 0};
    int64_t prim = 0;
    for (int64_t f = 0; f < F; ++f) {
        for (int64_t c = offsets[f]; c + 1 < offsets[f + 1]; ++c, ++prim) {
            const float* pa = ctrl + 4 * c;
            const float* pb = ctrl + 4 * (c + 1);
            float A[3], B[3];
            double A64[3], B64[3];
            for (int i = 0; i < 3; ++i) {
                A[i] = (pa[i] - g->origin[i]) * s;
                B[i] = (pb[i] - g->origin[i]) * s;
                A64[i] = (double)A[i];
                B64[i] = (double)B[i];
            }
            float rg = ((pa[3] + pb[3]) * 0.5f) * s;
            double rg64 = (double)rg;
            float w = weights ? weights[prim] : 1.0f;
            float d[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
            float dn = sqrtf((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
            float t[3] = {0, 0, 0};
            if (dn > 0.0f) { t[0] = d[0] / dn; t[1] = d[1] / dn; t[2] = d[2] / dn; }
            double d64[3] = {B64[0] - A64[0], B64[1] - A64[1], B64[2] - A64[2]};
            double dn64 = sqrt(d64[0] * d64[0] + d64[1] * d64[1] + d64[2] * d64[2]);
            double t64[3] = {0, 0, 0};
            if (dn64 > 0) { t64[0] = d64[0] / dn64; t64[1] = d64[1] / dn64; t64[2] = d64[2] / dn64; }
            int lo[3], hi[3];
            for (int i = 0; i < 3; ++i) {
                double mn = fmin(A64[i], B64[i]) - rg64, mx = fmax(A64[i], B64[i]) + rg64;
                lo[i] = clampi((int)floor(mn) - 1, 0, R - 1);
                hi[i] = clampi((int)floor(mx) + 1, 0, R - 1);
                if (mx < -1.0 || mn > (double)R + 1.0) { lo[i] = 1; hi[i] = 0; }
            }
            for (int vk = lo[2]; vk <= hi[2]; ++vk)
                for (int vj = lo[1]; vj <= hi[1]; ++vj)
                    for (int vi = lo[0]; vi <= hi[0]; ++vi) {
                        rec_t x;
                        int any = vxo_capsule_mask(A, B, rg, vi, vj, vk, x.mask);
                        float mu = vxo_capsule_measure(A, B, rg, vi, vj, vk);
                        if (!any && mu == 0.0f) continue;
                        x.key = vxo_morton((uint32_t)vi, (uint32_t)vj, (uint32_t)vk);
                        x.prim = prim;
                        x.c = w * mu;
                        x.dir[0] = t[0]; x.dir[1] = t[1]; x.dir[2] = t[2];
                        x.c64 = (double)w * capsule_measure64(A64, B64, rg64, vi, vj, vk);
                        x.dir64[0] = t64[0]; x.dir64[1] = t64[1]; x.dir64[2] = t64[2];
                        recs_push(&recs, &x);
                    }
        }
    }
    reduce_records(&recs, out, K);
    free(recs.r);
    return 0;
}

/* Sample-based voxelization of fiber segments (the paper's vertex-map sampling, Sec. 3.2-3.3,
 * as a comparison workload): S samples per segment on its axis at t_j = (j + 1/2) / S, each
 * carrying 1/S of the segment's measure.  A sample at grid point u = A + t_j (B - A) marks
 * the sub-cell floor(8 (u - floor(u))) of voxel floor(u) (dropped outside [0, R)^3) and
 * adds c = (w pi r^2 |B - A|) / S and c T(t) to that voxel, summed in sample order
 * (segment-major).  FP32 in this order. */
ORC_API int vxo_voxelize_fibers_sampled(const float* ctrl, const int64_t* offsets, int64_t F,
                                        const float* weights, const vxo_grid* g, int S, vxo_level* out) {
    const float s = 1.0f / g->voxel_size;
    const int R = g->resolution;
    recs_t recs = {0, 0, 0};
    int64_t prim = 0;
    for (int64_t f = 0; f < F; ++f) {
        for (int64_t c = offsets[f]; c + 1 < offsets[f + 1]; ++c, ++prim) {
            const float* pa = ctrl + 4 * c;
            const float* pb = ctrl + 4 * (c + 1);
            float A[3], B[3];
            for (int i = 0; i < 3; ++i) {
                A[i] = (pa[i] - g->origin[i]) * s;
                B[i] = (pb[i] - g->origin[i]) * s;
            }
            const float rg = ((pa[3] + pb[3]) * 0.5f) * s;
            const float w = weights ? weights[prim] : 1.0f;
            const float d[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
            const float dn = sqrtf((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
            float t[3] = {0, 0, 0};
            if (dn > 0.0f) { t[0] = d[0] / dn; t[1] = d[1] / dn; t[2] = d[2] / dn; }
            const float mu = (3.14159265358979f * (rg * rg)) * dn;
            const float cs = (w * mu) / (float)S;
            const double cs64 = (double)w * (3.141592653589793 * (double)rg * (double)rg) *
                                sqrt((double)d[0] * d[0] + (double)d[1] * d[1] + (double)d[2] * d[2]) / S;
            for (int j = 0; j < S; ++j) {
                const float tj = ((float)j + 0.5f) / (float)S;
                float u[3];
                int v[3], sc[3], inside = 1;
                for (int i = 0; i < 3; ++i) {
                    u[i] = A[i] + tj * d[i];
                    const float fl = floorf(u[i]);
                    if (!(u[i] >= 0.0f) || !(u[i] < (float)R)) inside = 0;
                    v[i] = (int)fl;
                    int k = (int)((u[i] - fl) * 8.0f);
                    sc[i] = k > 7 ? 7 : k;
                }
                if (!inside) continue;
                rec_t x;
                memset(x.mask, 0, sizeof(x.mask));
                mask_set(x.mask, sc[0], sc[1], sc[2]);
                x.key = vxo_morton((uint32_t)v[0], (uint32_t)v[1], (uint32_t)v[2]);
                x.prim = prim * S + j;
                x.c = cs;
                x.dir[0] = t[0]; x.dir[1] = t[1]; x.dir[2] = t[2];
                x.c64 = cs64;
                x.dir64[0] = t[0]; x.dir64[1] = t[1]; x.dir64[2] = t[2];
                recs_push(&recs, &x);
            }
        }
    }
    reduce_records(&recs, out, 1);
    free(recs.r);
    return 0;
}

/* Sample-based voxelization of triangles (Sec. 3.2-3.3: sample counts by area relative to the
 * largest triangle, points from Heitz's square-to-triangle map): triangle p of area a gets
 * M_p = max(1, ceil(S a / a_max)) (at most S) samples; sample j is the lattice point
 * (x, y) = ((j + 1/2) / M_p, frac((j + 1/2) 0.6180339887)), mapped to barycentrics by
 * y > x: b0 = x/2, b1 = y - b0; else b1 = y/2, b0 = x - b1; the point is
 * (b0 U0 + b1 U1) + (1 - b0 - b1) U2, carrying (w a) / M_p and the normal's moment. */
ORC_API int vxo_voxelize_tris_sampled(const float* tri, int64_t T, const float* weights, const vxo_grid* g, int S,
                                      vxo_level* out) {
    const float s = 1.0f / g->voxel_size;
    const int R = g->resolution;
    float* U = (float*)malloc(sizeof(float) * 9 * (size_t)(T > 0 ? T : 1));
    float* area = (float*)malloc(sizeof(float) * (size_t)(T > 0 ? T : 1));
    float* nrm = (float*)malloc(sizeof(float) * 3 * (size_t)(T > 0 ? T : 1));
    float amax = 0.0f;
    for (int64_t p = 0; p < T; ++p) {
        for (int k = 0; k < 3; ++k)
            for (int i = 0; i < 3; ++i) U[9 * p + 3 * k + i] = (tri[12 * p + 4 * k + i] - g->origin[i]) * s;
        const float* u = U + 9 * p;
        float f0[3], f1[3];
        for (int i = 0; i < 3; ++i) { f0[i] = u[3 + i] - u[i]; f1[i] = u[6 + i] - u[3 + i]; }
        const float n0 = f0[1] * f1[2] - f0[2] * f1[1];
        const float n1 = f0[2] * f1[0] - f0[0] * f1[2];
        const float n2 = f0[0] * f1[1] - f0[1] * f1[0];
        const float nn = sqrtf((n0 * n0 + n1 * n1) + n2 * n2);
        nrm[3 * p] = nrm[3 * p + 1] = nrm[3 * p + 2] = 0.0f;
        if (nn > 0.0f) { nrm[3 * p] = n0 / nn; nrm[3 * p + 1] = n1 / nn; nrm[3 * p + 2] = n2 / nn; }
        area[p] = 0.5f * nn;
        if (area[p] > amax) amax = area[p];
    }
    recs_t recs = {0, 0, 0};
    for (int64_t p = 0; p < T; ++p) {
        const float* u = U + 9 * p;
        const float w = weights ? weights[p] : 1.0f;
        uint32_t m = 1;
        if (amax > 0.0f) {
            const float x = (float)S * (area[p] / amax);
            m = (uint32_t)ceilf(x);
            if (m < 1) m = 1;
            if (m > (uint32_t)S) m = (uint32_t)S;
        }
        const float cs = (w * area[p]) / (float)m;
        for (uint32_t j = 0; j < m; ++j) {
            const float x = ((float)j + 0.5f) / (float)m;
            const float yy = ((float)j + 0.5f) * 0.6180339887f;
            const float y = yy - floorf(yy);
            float b0, b1;
            if (y > x) { b0 = x * 0.5f; b1 = y - b0; } else { b1 = y * 0.5f; b0 = x - b1; }
            const float b2 = (1.0f - b0) - b1;
            float q[3];
            int v[3], sc[3], inside = 1;
            for (int i = 0; i < 3; ++i) {
                q[i] = (b0 * u[i] + b1 * u[3 + i]) + b2 * u[6 + i];
                const float fl = floorf(q[i]);
                if (!(q[i] >= 0.0f) || !(q[i] < (float)R)) inside = 0;
                v[i] = (int)fl;
                int k = (int)((q[i] - fl) * 8.0f);
                sc[i] = k > 7 ? 7 : k;
            }
            if (!inside) continue;
            rec_t x_;
            memset(x_.mask, 0, sizeof(x_.mask));
            mask_set(x_.mask, sc[0], sc[1], sc[2]);
            x_.key = vxo_morton((uint32_t)v[0], (uint32_t)v[1], (uint32_t)v[2]);
            x_.prim = p * S + (int64_t)j;
            x_.c = cs;
            for (int i = 0; i < 3; ++i) { x_.dir[i] = nrm[3 * p + i]; x_.dir64[i] = nrm[3 * p + i]; }
            x_.c64 = (double)cs;
            recs_push(&recs, &x_);
        }
    }
    reduce_records(&recs, out, 1);
    free(recs.r); free(U); free(area); free(nrm);
    return 0;
}

/* Triangles: tri [T][3][4] (xyz, w unused). */
ORC_API int vxo_voxelize_tris(const float* tri, int64_t T, const float* weights,
                              const vxo_grid* g, int K, vxo_level* out) {
    const float s = 1.0f / g->voxel_size;
    const int R = g->resolution;
    recs_t recs = {0, 0, 0};
    for (int64_t p = 0; p < T; ++p) {
        float U[9];
        double U64[9];
        for (int k = 0; k < 3; ++k)
            for (int i = 0; i < 3; ++i) {
                float x = tri[12 * p + 4 * k + i];
                U[3 * k + i] = (x - g->origin[i]) * s;
                U64[3 * k + i] = (double)U[3 * k + i];
            }
        float w = weights ? weights[p] : 1.0f;
        float f0[3], f1[3];
        for (int i = 0; i < 3; ++i) { f0[i] = U[3 + i] - U[i]; f1[i] = U[6 + i] - U[3 + i]; }
        float n[3];
        n[0] = f0[1] * f1[2] - f0[2] * f1[1];
        n[1] = f0[2] * f1[0] - f0[0] * f1[2];
        n[2] = f0[0] * f1[1] - f0[1] * f1[0];
        float nn = sqrtf((n[0] * n[0] + n[1] * n[1]) + n[2] * n[2]);
        float t[3] = {0, 0, 0};
        if (nn > 0.0f) { t[0] = n[0] / nn; t[1] = n[1] / nn; t[2] = n[2] / nn; }
        double e0[3], e1[3], n64[3], t64[3] = {0, 0, 0};
        for (int i = 0; i < 3; ++i) { e0[i] = U64[3 + i] - U64[i]; e1[i] = U64[6 + i] - U64[3 + i]; }
        n64[0] = e0[1] * e1[2] - e0[2] * e1[1];
        n64[1] = e0[2] * e1[0] - e0[0] * e1[2];
        n64[2] = e0[0] * e1[1] - e0[1] * e1[0];
        double nn64 = sqrt(n64[0] * n64[0] + n64[1] * n64[1] + n64[2] * n64[2]);
        if (nn64 > 0) { t64[0] = n64[0] / nn64; t64[1] = n64[1] / nn64; t64[2] = n64[2] / nn64; }
        int lo[3], hi[3];
        for (int i = 0; i < 3; ++i) {
            double mn = fmin(fmin(U64[i], U64[3 + i]), U64[6 + i]);
            double mx = fmax(fmax(U64[i], U64[3 + i]), U64[6 + i]);
            lo[i] = clampi((int)floor(mn) - 1, 0, R - 1);
            hi[i] = clampi((int)floor(mx) + 1, 0, R - 1);
            if (mx < -1.0 || mn > (double)R + 1.0) { lo[i] = 1; hi[i] = 0; }
        }
        for (int vk = lo[2]; vk <= hi[2]; ++vk)
            for (int vj = lo[1]; vj <= hi[1]; ++vj)
                for (int vi = lo[0]; vi <= hi[0]; ++vi) {
                    rec_t x;
                    int any = vxo_tri_mask(U, vi, vj, vk, x.mask);
                    float mu = vxo_tri_measure(U, vi, vj, vk);
                    if (!any && mu == 0.0f) continue;
                    x.key = vxo_morton((uint32_t)vi, (uint32_t)vj, (uint32_t)vk);
                    x.prim = p;
                    x.c = w * mu;
                    x.dir[0] = t[0]; x.dir[1] = t[1]; x.dir[2] = t[2];
                    x.c64 = (double)w * vxo_tri_measure64(U64, vi, vj, vk);
                    x.dir64[0] = t64[0]; x.dir64[1] = t64[1]; x.dir64[2] = t64[2];
                    recs_push(&recs, &x);
                }
    }
    reduce_records(&recs, out, K);
    free(recs.r);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* SGGX-H (Sec. 4.4)                                                          */
/* ------------------------------------------------------------------------- */

/* Symmetric square root of a 3x3 SPD matrix by cyclic Jacobi rotations (FP32,
 * at most 6 sweeps over the pairs (0,1),(0,2),(1,2); a rotation is skipped when its
 * off-diagonal is zero or negligible against both diagonals); S packed
 * xx,yy,zz,xy,xz,yz, R full row-major 3x3.  Sec. 4.4 samples a lobe through its square
 * root and fixes no method for computing it. */
ORC_API void vxo_sqrtm3(const float* S, float* Rm) {
    float a[3][3] = {{S[0], S[3], S[4]}, {S[3], S[1], S[5]}, {S[4], S[5], S[2]}};
    float V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    static const int PQ[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int sweep = 0; sweep < 6; ++sweep) {
        int rotated = 0;
        for (int r = 0; r < 3; ++r) {
            int p = PQ[r][0], q = PQ[r][1];
            float apq = a[p][q];
            if (apq == 0.0f) continue;
            float app = a[p][p], aqq = a[q][q];
            /* an off-diagonal negligible against both diagonals (adding 100 |apq|
             * changes neither in FP32) is set to zero instead of rotated */
            float g = 100.0f * fabsf(apq);
            if (fabsf(app) + g == fabsf(app) && fabsf(aqq) + g == fabsf(aqq)) {
                a[p][q] = 0.0f;
                a[q][p] = 0.0f;
                continue;
            }
            /* tan of the rotation angle: the smaller root of t^2 + 2 t d / (2 apq) - 1 = 0,
             * d = aqq - app, written sgn(d) 2 apq / (|d| + sqrt(d^2 + 4 apq^2)) */
            float d = aqq - app, e = 2.0f * apq;
            float t = e / (fabsf(d) + sqrtf(d * d + e * e));
            if (d < 0.0f) t = -t;
            float c = 1.0f / sqrtf(t * t + 1.0f);
            rotated = 1;
            float sn = t * c;
            a[p][p] = app - t * apq;
            a[q][q] = aqq + t * apq;
            a[p][q] = 0.0f;
            a[q][p] = 0.0f;
            int o = 3 - p - q;
            float arp = a[o][p], arq = a[o][q];
            float nrp = c * arp - sn * arq;
            float nrq = sn * arp + c * arq;
            a[o][p] = nrp; a[p][o] = nrp;
            a[o][q] = nrq; a[q][o] = nrq;
            for (int i = 0; i < 3; ++i) {
                float vp = V[i][p], vq = V[i][q];
                V[i][p] = c * vp - sn * vq;
                V[i][q] = sn * vp + c * vq;
            }
        }
        if (!rotated) break; /* every off-diagonal is zero */
    }
    float sg[3];
    for (int i = 0; i < 3; ++i) sg[i] = sqrtf(a[i][i] > 0.0f ? a[i][i] : 0.0f);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            Rm[3 * i + j] = ((V[i][0] * sg[0]) * V[j][0] + (V[i][1] * sg[1]) * V[j][1]) +
                            (V[i][2] * sg[2]) * V[j][2];
}

/* Histogram + empirical second moment of the N directions drawn from a lobe S.
 * omega_k = normalize(S'^(1/2) u_k), S' = S + 1e-6 tr(S) I, u_k the fixed direction set;
 * the product S'^(1/2) u_k row by row as fmaf(R2, u2, fmaf(R1, u1, R0 u0)).
 * Histogram (5 bins per axis over [-1,1], omega and -omega both counted): stored as
 * hist[a] = #(omega_a^2 >= 0.36 |v|^2), hist[3+a] = #(omega_a^2 >= 0.04 |v|^2).
 * Second moment: each product omega_a omega_b (= v_a v_b / |v|^2) rounded once to the
 * 2^-20 grid, summed exactly in integers, divided by N. */
ORC_API void vxo_sample_lobe(const float* S, const float* dirs, int N, int32_t* hist, float* Mhat) {
    float tr = (S[0] + S[1]) + S[2];
    float eps = 1e-6f * tr;
    float Sp[6] = {S[0] + eps, S[1] + eps, S[2] + eps, S[3], S[4], S[5]};
    float Rm[9];
    vxo_sqrtm3(Sp, Rm);
    int32_t h[6] = {0, 0, 0, 0, 0, 0};
    int64_t Q[6] = {0, 0, 0, 0, 0, 0};
    int64_t cnt = 0;
    for (int k = 0; k < N; ++k) {
        const float* u = dirs + 3 * k;
        float v[3];
        for (int i = 0; i < 3; ++i) v[i] = fmaf(Rm[3 * i + 2], u[2], fmaf(Rm[3 * i + 1], u[1], Rm[3 * i] * u[0]));
        float n2 = (v[0] * v[0] + v[1] * v[1]) + v[2] * v[2];
        if (!(n2 > 0.0f)) continue;
        ++cnt;
        float t6 = 0.36f * n2, t2 = 0.04f * n2;
        for (int a = 0; a < 3; ++a) {
            float c2 = v[a] * v[a];
            if (c2 >= t6) h[a] += 1;
            if (c2 >= t2) h[3 + a] += 1;
        }
        float inv = 1.0f / n2;
        float s20 = inv * 1048576.0f;
        static const int AB[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
        for (int c = 0; c < 6; ++c) {
            float p = v[AB[c][0]] * v[AB[c][1]];
            /* the product p * s20 is exact in FP64 (24 + 24 bits); rounded once, half to even */
            Q[c] += (int64_t)nearbyint((double)p * (double)s20);
        }
    }
    for (int c = 0; c < 6; ++c) hist[c] = h[c];
    for (int c = 0; c < 6; ++c)
        Mhat[c] = cnt > 0 ? (float)((double)Q[c] / ((double)cnt * 1048576.0)) : 0.0f;
}

/* integer sliced-Wasserstein distance between two lobe histograms (units of 0.4/N) */
ORC_API int64_t vxo_hist_dist(const int32_t* a, const int32_t* b) {
    int64_t d = 0;
    for (int c = 0; c < 6; ++c) d += llabs((long long)a[c] - (long long)b[c]);
    return d;
}

/* Agglomerative SGGX-H of n candidate lobes (S6 + weight each, in candidate order) to at
 * most K lobes.  Output lobes sorted by weight (descending), ties by creation index.
 * Returns the output count; merges_out (optional) receives (i, j) creation ids per merge.
 * merge 0: the merged lobe is the second moment of the two lobes' pooled samples,
 * (M^_i + M^_j) / 2; merge 1: the same moments weighted by the lobes' masses,
 * (w_i M^_i + w_j M^_j) / (w_i + w_j). */
ORC_API int vxo_sggx_h(const float* cand, int n, int K, const float* dirs, int N,
                       float* out, int32_t* merges_out, int merge) {
    int cap = 2 * n + 1;
    float* S = (float*)malloc(sizeof(float) * 6 * (size_t)cap);
    float* wgt = (float*)malloc(sizeof(float) * (size_t)cap);
    float* Mh = (float*)malloc(sizeof(float) * 6 * (size_t)cap);
    int32_t* H = (int32_t*)malloc(sizeof(int32_t) * 6 * (size_t)cap);
    int* alive = (int*)calloc((size_t)cap, sizeof(int));
    for (int i = 0; i < n; ++i) {
        memcpy(S + 6 * i, cand + 7 * i, 6 * sizeof(float));
        wgt[i] = cand[7 * i + 6];
        alive[i] = 1;
    }
    int count = n, next = n, nm = 0;
    if (n > K) {
        for (int i = 0; i < n; ++i) vxo_sample_lobe(S + 6 * i, dirs, N, H + 6 * i, Mh + 6 * i);
        while (count > K) {
            int bi = -1, bj = -1;
            int64_t best = 0;
            for (int i = 0; i < next; ++i) {
                if (!alive[i]) continue;
                for (int j = 0; j < i; ++j) {
                    if (!alive[j]) continue;
                    int64_t dd = vxo_hist_dist(H + 6 * i, H + 6 * j);
                    if (bi < 0 || dd < best) { best = dd; bi = i; bj = j; }
                }
            }
            const float wi = wgt[bi], wj = wgt[bj], ws = wgt[bi] + wgt[bj];
            for (int c = 0; c < 6; ++c) {
                if (merge == 1 && ws > 0.0f)
                    S[6 * next + c] = (wi * Mh[6 * bi + c] + wj * Mh[6 * bj + c]) / ws;
                else
                    S[6 * next + c] = (Mh[6 * bi + c] + Mh[6 * bj + c]) * 0.5f;
            }
            wgt[next] = wgt[bi] + wgt[bj];
            vxo_sample_lobe(S + 6 * next, dirs, N, H + 6 * next, Mh + 6 * next);
            alive[bi] = 0; alive[bj] = 0; alive[next] = 1;
            if (merges_out) { merges_out[2 * nm] = bi; merges_out[2 * nm + 1] = bj; }
            ++nm; ++next; --count;
        }
    }
    /* gather alive ids in creation order, then stable selection by weight desc */
    int ids[64 * 2 + 1];
    int na = 0;
    for (int i = 0; i < next; ++i) if (alive[i]) ids[na++] = i;
    for (int a = 1; a < na; ++a) {         /* insertion sort: stable */
        int x = ids[a], b = a - 1;
        while (b >= 0 && wgt[ids[b]] < wgt[x]) { ids[b + 1] = ids[b]; --b; }
        ids[b + 1] = x;
    }
    for (int a = 0; a < na; ++a) {
        memcpy(out + 7 * a, S + 6 * ids[a], 6 * sizeof(float));
        out[7 * a + 6] = wgt[ids[a]];
    }
    free(S); free(wgt); free(Mh); free(H); free(alive);
    return na;
}

/* ------------------------------------------------------------------------- */
/* LoD: level l -> l+1 (Sec. 4.2 density by projection, 4.3 2x2x2, 4.4 SGGX-H) */
/* ------------------------------------------------------------------------- */
ORC_API int vxo_lod_step(const vxo_level* in, int K, const float* dirs, int N, vxo_level* out, int merge) {
    int64_t np = 0;
    for (int64_t i = 0; i < in->n; ++i)
        if (i == 0 || (in->keys[i] >> 3) != (in->keys[i - 1] >> 3)) ++np;
    level_alloc(out, np, K);
    float cand[8 * 16 * 7];
    int64_t v = 0;
    for (int64_t i = 0; i < in->n;) {
        int64_t j = i;
        uint64_t pk = in->keys[i] >> 3;
        float m = 0.0f, M[6] = {0, 0, 0, 0, 0, 0};
        double m64 = 0.0, M64[6] = {0, 0, 0, 0, 0, 0};
        uint64_t pm[8] = {0};
        int nc = 0;
        while (j < in->n && (in->keys[j] >> 3) == pk) {
            int oct = (int)(in->keys[j] & 7ull);
            int ox = oct & 1, oy = (oct >> 1) & 1, oz = (oct >> 2) & 1;
            m = m + in->mass[j];
            m64 += in->mass64[j];
            for (int c = 0; c < 6; ++c) {
                M[c] = M[c] + in->moment[6 * j + c];
                M64[c] += in->moment64[6 * j + c];
            }
            const uint64_t* cm = in->mask + 8 * j;
            for (int pz = 4 * oz; pz < 4 * oz + 4; ++pz)
                for (int py = 4 * oy; py < 4 * oy + 4; ++py)
                    for (int px = 4 * ox; px < 4 * ox + 4; ++px) {
                        int bit = 0;
                        for (int dz = 0; dz < 2; ++dz)
                            for (int dy = 0; dy < 2; ++dy)
                                for (int dx = 0; dx < 2; ++dx)
                                    bit |= mask_get(cm, 2 * (px & 3) + dx, 2 * (py & 3) + dy, 2 * (pz & 3) + dz);
                        if (bit) mask_set(pm, px, py, pz);
                    }
            const float* cl = in->lobes + (size_t)j * in->K * 7;
            for (int l = 0; l < in->lobe_count[j]; ++l) {
                memcpy(cand + 7 * nc, cl + 7 * l, 7 * sizeof(float));
                ++nc;
            }
            ++j;
        }
        out->keys[v] = pk;
        memcpy(out->mask + 8 * v, pm, sizeof(pm));
        out->mass[v] = m;
        memcpy(out->moment + 6 * v, M, sizeof(M));
        out->mass64[v] = m64;
        memcpy(out->moment64 + 6 * v, M64, sizeof(M64));
        mask_stats(pm, &out->occ[v], &out->proj[3 * v]);
        if (K == 1) {
            single_lobe(out, v);
        } else {
            float res[16 * 7];
            int nl = vxo_sggx_h(cand, nc, K, dirs, N, res, NULL, merge);
            float* lo = out->lobes + (size_t)v * K * 7;
            memcpy(lo, res, (size_t)nl * 7 * sizeof(float));
            for (int l = 0; l < nl; ++l) vxo_compact(lo + 7 * l, out->compact + ((size_t)v * K + l) * 6);
            out->lobe_count[v] = (uint8_t)nl;
        }
        ++v;
        i = j;
    }
    return 0;
}

/* Attributes of a given list of voxels, computed from all fiber primitives by brute
 * force (used to check full-size runs on sampled voxels).  Outputs per key: mask[8],
 * mass, moment[6] (FP32 chain) and mass64, moment64[6]. */
ORC_API int vxo_fiber_voxels(const float* ctrl, const int64_t* offsets, int64_t F,
                             const float* weights, const vxo_grid* g,
                             const uint64_t* keys, int64_t nk,
                             uint64_t* mask, float* mass, float* moment,
                             double* mass64, double* moment64) {
    const float s = 1.0f / g->voxel_size;
    for (int64_t q = 0; q < nk; ++q) {
        uint32_t vi, vj, vk;
        vxo_demorton(keys[q], &vi, &vj, &vk);
        uint64_t m8[8] = {0};
        float m = 0.0f, M[6] = {0, 0, 0, 0, 0, 0};
        double m64 = 0.0, M64[6] = {0, 0, 0, 0, 0, 0};
        int64_t prim = 0;
        for (int64_t f = 0; f < F; ++f) {
            for (int64_t c = offsets[f]; c + 1 < offsets[f + 1]; ++c, ++prim) {
                const float* pa = ctrl + 4 * c;
                const float* pb = ctrl + 4 * (c + 1);
                float A[3], B[3];
                double A64[3], B64[3];
                for (int i = 0; i < 3; ++i) {
                    A[i] = (pa[i] - g->origin[i]) * s;
                    B[i] = (pb[i] - g->origin[i]) * s;
                    A64[i] = (double)A[i];
                    B64[i] = (double)B[i];
                }
                float rg = ((pa[3] + pb[3]) * 0.5f) * s;
                double rg64 = (double)rg;
                double vv[3] = {(double)vi, (double)vj, (double)vk};
                int skip = 0;
                for (int i = 0; i < 3; ++i) {
                    double mn = fmin(A64[i], B64[i]) - rg64 - 1.0, mx = fmax(A64[i], B64[i]) + rg64 + 1.0;
                    if (vv[i] + 1.0 < mn || vv[i] > mx) skip = 1;
                }
                if (skip) continue;
                uint64_t pm[8];
                vxo_capsule_mask(A, B, rg, (int)vi, (int)vj, (int)vk, pm);
                for (int w = 0; w < 8; ++w) m8[w] |= pm[w];
                float mu = vxo_capsule_measure(A, B, rg, (int)vi, (int)vj, (int)vk);
                if (mu == 0.0f) continue;
                float w = weights ? weights[prim] : 1.0f;
                float d[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
                float dn = sqrtf((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
                float t[3] = {d[0] / dn, d[1] / dn, d[2] / dn};
                float cc = w * mu;
                m = m + cc;
                M[0] = M[0] + cc * (t[0] * t[0]);
                M[1] = M[1] + cc * (t[1] * t[1]);
                M[2] = M[2] + cc * (t[2] * t[2]);
                M[3] = M[3] + cc * (t[0] * t[1]);
                M[4] = M[4] + cc * (t[0] * t[2]);
                M[5] = M[5] + cc * (t[1] * t[2]);
                double d64[3] = {B64[0] - A64[0], B64[1] - A64[1], B64[2] - A64[2]};
                double dn64 = sqrt(d64[0] * d64[0] + d64[1] * d64[1] + d64[2] * d64[2]);
                double t64[3] = {d64[0] / dn64, d64[1] / dn64, d64[2] / dn64};
                double c64 = (double)w * capsule_measure64(A64, B64, rg64, (int)vi, (int)vj, (int)vk);
                m64 += c64;
                M64[0] += c64 * t64[0] * t64[0];
                M64[1] += c64 * t64[1] * t64[1];
                M64[2] += c64 * t64[2] * t64[2];
                M64[3] += c64 * t64[0] * t64[1];
                M64[4] += c64 * t64[0] * t64[2];
                M64[5] += c64 * t64[1] * t64[2];
            }
        }
        memcpy(mask + 8 * q, m8, sizeof(m8));
        mass[q] = m;
        memcpy(moment + 6 * q, M, sizeof(M));
        mass64[q] = m64;
        memcpy(moment64 + 6 * q, M64, sizeof(M64));
    }
    return 0;
}

/* A level from per-voxel primaries (keys sorted, non-zero masks): recomputes occupancy,
 * projections and the single normalised lobe exactly as the voxelization does. */
ORC_API int vxo_level_from_voxels(const uint64_t* keys, const uint64_t* mask, const float* mass,
                                  const float* moment, const double* mass64, const double* moment64,
                                  int64_t n, vxo_level* out) {
    int64_t nv = 0;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t any = 0;
        for (int w = 0; w < 8; ++w) any |= mask[8 * i + w];
        if (any) ++nv;
    }
    level_alloc(out, nv, 1);
    int64_t v = 0;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t any = 0;
        for (int w = 0; w < 8; ++w) any |= mask[8 * i + w];
        if (!any) continue;
        out->keys[v] = keys[i];
        memcpy(out->mask + 8 * v, mask + 8 * i, 64);
        out->mass[v] = mass[i];
        memcpy(out->moment + 6 * v, moment + 6 * i, 24);
        out->mass64[v] = mass64[i];
        memcpy(out->moment64 + 6 * v, moment64 + 6 * i, 48);
        mask_stats(out->mask + 8 * v, &out->occ[v], &out->proj[3 * v]);
        single_lobe(out, v);
        ++v;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Adjoint of  loss = sum_v gm(v) m(v) + sum_v gM(v) . M(v)  over level-0 voxels      */
/* (coarser levels enter through gm, gM broadcast down: m and M of a parent are sums  */
/* of its children).  FP64, for fibers.                                               */
/* ------------------------------------------------------------------------- */

/* clipped parameter interval of segment a + t d (voxel-local) against [0,1]^3:
 * returns 0 if empty; t0, t1 and which axis/plane defines each end (-1 = endpoint). */
static int clip64(const double* a, const double* d, double* t0, double* t1, int* ax0, int* ax1) {
    double lo = 0.0, hi = 1.0;
    int alo = -1, ahi = -1;
    for (int i = 0; i < 3; ++i) {
        if (d[i] == 0.0) {
            if (a[i] < 0.0 || a[i] > 1.0) return 0;
        } else {
            double ta = -a[i] / d[i], tb = (1.0 - a[i]) / d[i];
            double tn = d[i] > 0 ? ta : tb, tf = d[i] > 0 ? tb : ta;
            if (tn > lo) { lo = tn; alo = i; }
            if (tf < hi) { hi = tf; ahi = i; }
        }
    }
    if (hi <= lo) return 0;
    *t0 = lo; *t1 = hi; *ax0 = alo; *ax1 = ahi;
    return 1;
}

/* gradient of f = w * pi r^2 len * (gm + gM . T(t)) for one (segment, voxel) pair.
 * A, B grid coordinates, r grid units; outputs d f / d(A, B, r, w) (grid units). */
ORC_API double vxo_pair_grad64(const double* A, const double* B, double r, double w, int vi, int vj, int vk,
                               double gm, const double* gM, double* dA, double* dB, double* dr, double* dw) {
    double a[3] = {A[0] - vi, A[1] - vj, A[2] - vk};
    double d[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    for (int i = 0; i < 3; ++i) { dA[i] = 0; dB[i] = 0; }
    *dr = 0; *dw = 0;
    double t0, t1;
    int ax0, ax1;
    if (!clip64(a, d, &t0, &t1, &ax0, &ax1)) return 0.0;
    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double t[3] = {d[0] / dn, d[1] / dn, d[2] / dn};
    double len = (t1 - t0) * dn;
    double mu = M_PI_D * r * r * len;
    double T[6] = {t[0] * t[0], t[1] * t[1], t[2] * t[2], t[0] * t[1], t[0] * t[2], t[1] * t[2]};
    double G = gm;
    for (int c = 0; c < 6; ++c) G += gM[c] * T[c];
    double f = w * mu * G;
    *dw = mu * G;
    *dr = w * (2.0 * mu / r) * G;
    /* d len: len = |Q1 - Q0|, Q = (1-t) A + t B; an end on plane i moves within that plane */
    double cA[3] = {0, 0, 0}, cB[3] = {0, 0, 0};
    for (int e = 0; e < 2; ++e) {
        double te = e == 0 ? t0 : t1;
        int ax = e == 0 ? ax0 : ax1;
        double sgn = e == 0 ? -1.0 : 1.0;     /* d len = t . (dQ1 - dQ0) */
        for (int k = 0; k < 3; ++k) {
            double gA = (1.0 - te) * t[k], gB = te * t[k];
            if (ax == k) { gA -= (1.0 - te) * dn / d[k]; gB -= te * dn / d[k]; }
            cA[k] += sgn * gA;
            cB[k] += sgn * gB;
        }
    }
    double kmu = w * M_PI_D * r * r * G;     /* d f / d len */
    /* d T / d d: dT = (I - t t^T)/|d| applied to grad_t (gM . T) */
    double gt[3];
    gt[0] = 2 * gM[0] * t[0] + gM[3] * t[1] + gM[4] * t[2];
    gt[1] = gM[3] * t[0] + 2 * gM[1] * t[1] + gM[5] * t[2];
    gt[2] = gM[4] * t[0] + gM[5] * t[1] + 2 * gM[2] * t[2];
    double tg = t[0] * gt[0] + t[1] * gt[1] + t[2] * gt[2];
    double wm = w * mu;
    for (int k = 0; k < 3; ++k) {
        double gd = wm * (gt[k] - t[k] * tg) / dn;   /* d f / d d_k through T */
        dA[k] = kmu * cA[k] - gd;
        dB[k] = kmu * cB[k] + gd;
    }
    return f;
}

static int64_t find_key(const uint64_t* keys, int64_t n, uint64_t k) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < k) lo = mid + 1; else hi = mid;
    }
    return (lo < n && keys[lo] == k) ? lo : -1;
}

/* Gradients of the loss w.r.t. ctrl [P][4] (xyz world, radius world) and weights [N],
 * given the broadcast level-0 adjoints gm0 [V], gM0 [V][6] on the sorted keys0.
 * Only the primitives listed in prims (or all when prims == NULL) are visited;
 * returns the loss contribution of the visited primitives.  d_abs (optional, [P][4])
 * receives the summed magnitudes of the per-pair terms of each control-point gradient. */
ORC_API double vxo_fiber_adjoint(const double* ctrl, const int64_t* offsets, int64_t F, const double* weights,
                                 const double* origin, double voxel_size, int R,
                                 const uint64_t* keys0, int64_t V, const double* gm0, const double* gM0,
                                 const int64_t* prims, int64_t nprims,
                                 double* d_ctrl, double* d_w, double* d_abs) {
    double s = 1.0 / voxel_size;
    double loss = 0.0;
    int64_t prim = 0;
    int64_t pi = 0;
    for (int64_t f = 0; f < F; ++f) {
        for (int64_t c = offsets[f]; c + 1 < offsets[f + 1]; ++c, ++prim) {
            if (prims) {
                while (pi < nprims && prims[pi] < prim) ++pi;
                if (pi >= nprims || prims[pi] != prim) continue;
            }
            const double* pa = ctrl + 4 * c;
            const double* pb = ctrl + 4 * (c + 1);
            double A[3], B[3];
            for (int i = 0; i < 3; ++i) { A[i] = (pa[i] - origin[i]) * s; B[i] = (pb[i] - origin[i]) * s; }
            double r = (pa[3] + pb[3]) * 0.5 * s;
            double w = weights ? weights[prim] : 1.0;
            int lo[3], hi[3];
            for (int i = 0; i < 3; ++i) {
                lo[i] = clampi((int)floor(fmin(A[i], B[i])) - 1, 0, R - 1);
                hi[i] = clampi((int)floor(fmax(A[i], B[i])) + 1, 0, R - 1);
            }
            double gA[3] = {0, 0, 0}, gB[3] = {0, 0, 0}, gr = 0, gw = 0;
            double aA[3] = {0, 0, 0}, aB[3] = {0, 0, 0}, ar = 0;   /* summed |per-pair terms| */
            for (int vk = lo[2]; vk <= hi[2]; ++vk)
                for (int vj = lo[1]; vj <= hi[1]; ++vj)
                    for (int vi = lo[0]; vi <= hi[0]; ++vi) {
                        int64_t v = find_key(keys0, V, vxo_morton((uint32_t)vi, (uint32_t)vj, (uint32_t)vk));
                        if (v < 0) continue;
                        double a3[3], b3[3], dr, dw;
                        loss += vxo_pair_grad64(A, B, r, w, vi, vj, vk, gm0[v], gM0 + 6 * v, a3, b3, &dr, &dw);
                        for (int i = 0; i < 3; ++i) {
                            gA[i] += a3[i]; gB[i] += b3[i];
                            aA[i] += fabs(a3[i]); aB[i] += fabs(b3[i]);
                        }
                        gr += dr;
                        ar += fabs(dr);
                        gw += dw;
                    }
            if (d_ctrl) {
                for (int i = 0; i < 3; ++i) { d_ctrl[4 * c + i] += gA[i] * s; d_ctrl[4 * (c + 1) + i] += gB[i] * s; }
                d_ctrl[4 * c + 3] += gr * 0.5 * s;
                d_ctrl[4 * (c + 1) + 3] += gr * 0.5 * s;
            }
            if (d_w) d_w[prim] += gw;
            if (d_abs) {
                for (int i = 0; i < 3; ++i) { d_abs[4 * c + i] += aA[i] * s; d_abs[4 * (c + 1) + i] += aB[i] * s; }
                d_abs[4 * c + 3] += ar * 0.5 * s;
                d_abs[4 * (c + 1) + 3] += ar * 0.5 * s;
            }
        }
    }
    return loss;
}

/* Active-set signature of the clipped pieces of the listed segments: a hash over every
 * (segment, voxel, entering plane, leaving plane) with a piece of positive length.  Equal
 * signatures at theta - h, theta, theta + h mean the loss is smooth on that stencil. */
ORC_API uint64_t vxo_clip_signature(const double* ctrl, const int64_t* offsets, int64_t F, const double* origin,
                                    double voxel_size, int R, const int64_t* prims, int64_t nprims) {
    double s = 1.0 / voxel_size;
    uint64_t h = 1469598103934665603ull;
    int64_t prim = 0, pi = 0;
    for (int64_t f = 0; f < F; ++f) {
        for (int64_t c = offsets[f]; c + 1 < offsets[f + 1]; ++c, ++prim) {
            while (pi < nprims && prims[pi] < prim) ++pi;
            if (pi >= nprims || prims[pi] != prim) continue;
            double A[3], B[3];
            for (int i = 0; i < 3; ++i) {
                A[i] = (ctrl[4 * c + i] - origin[i]) * s;
                B[i] = (ctrl[4 * (c + 1) + i] - origin[i]) * s;
            }
            double d[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
            int lo[3], hi[3];
            for (int i = 0; i < 3; ++i) {
                lo[i] = clampi((int)floor(fmin(A[i], B[i])) - 1, 0, R - 1);
                hi[i] = clampi((int)floor(fmax(A[i], B[i])) + 1, 0, R - 1);
            }
            for (int vk = lo[2]; vk <= hi[2]; ++vk)
                for (int vj = lo[1]; vj <= hi[1]; ++vj)
                    for (int vi = lo[0]; vi <= hi[0]; ++vi) {
                        double a[3] = {A[0] - vi, A[1] - vj, A[2] - vk};
                        double t0, t1;
                        int ax0, ax1;
                        if (!clip64(a, d, &t0, &t1, &ax0, &ax1)) continue;
                        uint64_t v = ((uint64_t)prim << 40) ^ (vxo_morton((uint32_t)vi, (uint32_t)vj, (uint32_t)vk) << 4) ^
                                     (uint64_t)((ax0 + 1) * 5 + (ax1 + 1));
                        for (int b = 0; b < 8; ++b) { h ^= (v >> (8 * b)) & 0xffu; h *= 1099511628211ull; }
                    }
        }
    }
    return h;
}

/* ------------------------------------------------------------------------- */
/* Triangle adjoint by complex-step differentiation                           */
/* ------------------------------------------------------------------------- */
/* The per-pair term of the loss is f = w * area(T ∩ voxel) * (gm + gM . T(n)), with
 * n the unit face normal (Sec. 4.1: the triangle's orientation is its normal) and
 * the area in grid units (Sec. 3.1 coordinates).  Each derivative d f / d U_jk is
 * Im f(U + i eps e_jk) / eps (complex step, Squire & Trapp 1998): the clip decisions
 * are taken on the real parts, every other operation (the Sutherland-Hodgman clip of
 * the triangle to the voxel, the polygon's cross-product sum, the square roots) is
 * analytic, so the result is the exact derivative of the active piece up to rounding,
 * with no subtractive cancellation.  This is deliberately a different method from the
 * analytic reference-domain formula the kernels use. */
#include <complex.h>
typedef double complex cplx;

static int clip_plane_c(const cplx in[][3], int n, cplx out[][3], int axis, double c, int keep_ge,
                        unsigned* inside_bits) {
    int m = 0;
    unsigned bits = 0;
    for (int k = 0; k < n; ++k) {
        const cplx* S = in[k];
        const cplx* E = in[(k + 1) % n];
        int sin_ = keep_ge ? (creal(S[axis]) >= c) : (creal(S[axis]) <= c);
        int ein = keep_ge ? (creal(E[axis]) >= c) : (creal(E[axis]) <= c);
        if (sin_) bits |= 1u << k;
        if (ein) {
            if (!sin_) {
                cplx s = (c - S[axis]) / (E[axis] - S[axis]);
                for (int j = 0; j < 3; ++j) out[m][j] = (j == axis) ? (cplx)c : S[j] + s * (E[j] - S[j]);
                ++m;
            }
            for (int j = 0; j < 3; ++j) out[m][j] = E[j];
            ++m;
        } else if (sin_) {
            cplx s = (c - S[axis]) / (E[axis] - S[axis]);
            for (int j = 0; j < 3; ++j) out[m][j] = (j == axis) ? (cplx)c : S[j] + s * (E[j] - S[j]);
            ++m;
        }
    }
    if (inside_bits) *inside_bits = bits;
    return m;
}

/* area of the triangle U (complex grid coordinates, [3][3]) clipped to voxel (vi,vj,vk);
 * sig (optional, [6]) receives (n << 16 | inside-bits) of each of the six clip stages. */
static cplx tri_area_c(const cplx U[3][3], int vi, int vj, int vk, uint32_t* sig) {
    cplx A[16][3], B[16][3];
    int n = 3;
    for (int k = 0; k < 3; ++k) {
        A[k][0] = U[k][0] - vi; A[k][1] = U[k][1] - vj; A[k][2] = U[k][2] - vk;
    }
    if (sig) for (int q = 0; q < 6; ++q) sig[q] = 0;
    for (int axis = 0; axis < 3 && n > 0; ++axis) {
        unsigned b0 = 0, b1 = 0;
        int n0 = n;
        n = clip_plane_c((const cplx(*)[3])A, n, B, axis, 0.0, 1, &b0);
        if (sig) sig[2 * axis] = ((uint32_t)n0 << 16) | b0;
        if (n == 0) break;
        int n1 = n;
        n = clip_plane_c((const cplx(*)[3])B, n, A, axis, 1.0, 0, &b1);
        if (sig) sig[2 * axis + 1] = ((uint32_t)n1 << 16) | b1;
    }
    if (n < 3) return 0.0;
    cplx cx = 0, cy = 0, cz = 0;
    for (int k = 1; k + 1 < n; ++k) {
        cplx e1[3], e2[3];
        for (int j = 0; j < 3; ++j) { e1[j] = A[k][j] - A[0][j]; e2[j] = A[k + 1][j] - A[0][j]; }
        cx += e1[1] * e2[2] - e1[2] * e2[1];
        cy += e1[2] * e2[0] - e1[0] * e2[2];
        cz += e1[0] * e2[1] - e1[1] * e2[0];
    }
    return 0.5 * csqrt(cx * cx + cy * cy + cz * cz);
}

/* area(T ∩ voxel) * (gm + gM . T(n)) with complex coordinates */
static cplx tri_pair_value_c(const cplx U[3][3], int vi, int vj, int vk, double gm, const double* gM) {
    cplx area = tri_area_c(U, vi, vj, vk, NULL);
    if (creal(area) == 0.0) return 0.0;
    cplx e0[3], e1[3], n[3];
    for (int i = 0; i < 3; ++i) { e0[i] = U[1][i] - U[0][i]; e1[i] = U[2][i] - U[1][i]; }
    n[0] = e0[1] * e1[2] - e0[2] * e1[1];
    n[1] = e0[2] * e1[0] - e0[0] * e1[2];
    n[2] = e0[0] * e1[1] - e0[1] * e1[0];
    cplx nn = csqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (creal(nn) == 0.0) return area * gm;
    cplx t[3] = {n[0] / nn, n[1] / nn, n[2] / nn};
    cplx G = gm + gM[0] * t[0] * t[0] + gM[1] * t[1] * t[1] + gM[2] * t[2] * t[2] + gM[3] * t[0] * t[1] +
             gM[4] * t[0] * t[2] + gM[5] * t[1] * t[2];
    return area * G;
}

static void tri_grid_coords(const double* tri, const double* origin, double s, double U[3][3]) {
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 3; ++i) U[k][i] = (tri[4 * k + i] - origin[i]) * s;
}

static void tri_voxel_range(const double U[3][3], int R, int lo[3], int hi[3]) {
    for (int i = 0; i < 3; ++i) {
        double mn = fmin(fmin(U[0][i], U[1][i]), U[2][i]);
        double mx = fmax(fmax(U[0][i], U[1][i]), U[2][i]);
        lo[i] = clampi((int)floor(mn) - 1, 0, R - 1);
        hi[i] = clampi((int)floor(mx) + 1, 0, R - 1);
        if (mx < -1.0 || mn > (double)R + 1.0) { lo[i] = 1; hi[i] = 0; }
    }
}

/* Gradients of the loss w.r.t. the triangle vertices tris [T][3][4] (xyz world; the
 * fourth component is ignored) and the per-triangle weights [T], given the broadcast
 * level-0 adjoints gm0 [V], gM0 [V][6] on the sorted keys0.  d_tris [T][3][3] (world
 * units), d_w [T]; d_abs (optional, [T][3][3]) receives the summed magnitudes of the
 * per-pair terms.  Only the listed prims (or all, when prims == NULL) are visited;
 * returns their loss contribution. */
ORC_API double vxo_tri_adjoint(const double* tris, int64_t T, const double* weights, const double* origin,
                               double voxel_size, int R, const uint64_t* keys0, int64_t V, const double* gm0,
                               const double* gM0, const int64_t* prims, int64_t nprims, double* d_tris,
                               double* d_w, double* d_abs) {
    const double s = 1.0 / voxel_size;
    const double eps = 1e-30;
    double loss = 0.0;
    int64_t pi = 0;
    for (int64_t p = 0; p < T; ++p) {
        if (prims) {
            while (pi < nprims && prims[pi] < p) ++pi;
            if (pi >= nprims || prims[pi] != p) continue;
        }
        double U[3][3];
        tri_grid_coords(tris + 12 * p, origin, s, U);
        const double w = weights ? weights[p] : 1.0;
        int lo[3], hi[3];
        tri_voxel_range(U, R, lo, hi);
        for (int vk = lo[2]; vk <= hi[2]; ++vk)
            for (int vj = lo[1]; vj <= hi[1]; ++vj)
                for (int vi = lo[0]; vi <= hi[0]; ++vi) {
                    int64_t v = find_key(keys0, V, vxo_morton((uint32_t)vi, (uint32_t)vj, (uint32_t)vk));
                    if (v < 0) continue;
                    cplx Uc[3][3];
                    for (int k = 0; k < 3; ++k)
                        for (int i = 0; i < 3; ++i) Uc[k][i] = U[k][i];
                    const double f0 = creal(tri_pair_value_c((const cplx(*)[3])Uc, vi, vj, vk, gm0[v], gM0 + 6 * v));
                    if (f0 == 0.0) continue;
                    loss += w * f0;
                    if (d_w) d_w[p] += f0;
                    for (int k = 0; k < 3; ++k)
                        for (int i = 0; i < 3; ++i) {
                            Uc[k][i] = U[k][i] + I * eps;
                            double g = cimag(tri_pair_value_c((const cplx(*)[3])Uc, vi, vj, vk, gm0[v], gM0 + 6 * v)) /
                                       eps;
                            Uc[k][i] = U[k][i];
                            if (d_tris) d_tris[9 * p + 3 * k + i] += w * g * s;
                            if (d_abs) d_abs[9 * p + 3 * k + i] += fabs(w * g * s);
                        }
                }
    }
    return loss;
}

/* Clip signature of the listed triangles: a hash over every (triangle, voxel) with a
 * clipped polygon of positive area and the vertex count and inside pattern of each of
 * its six clip stages.  Equal signatures at theta - h, theta, theta + h mean every
 * clipped polygon kept its combinatorial structure, so the loss is smooth there. */
ORC_API uint64_t vxo_tri_clip_signature(const double* tris, int64_t T, const double* origin, double voxel_size,
                                        int R, const int64_t* prims, int64_t nprims) {
    const double s = 1.0 / voxel_size;
    uint64_t h = 1469598103934665603ull;
    int64_t pi = 0;
    for (int64_t p = 0; p < T; ++p) {
        while (pi < nprims && prims[pi] < p) ++pi;
        if (pi >= nprims || prims[pi] != p) continue;
        double U[3][3];
        tri_grid_coords(tris + 12 * p, origin, s, U);
        int lo[3], hi[3];
        tri_voxel_range(U, R, lo, hi);
        cplx Uc[3][3];
        for (int k = 0; k < 3; ++k)
            for (int i = 0; i < 3; ++i) Uc[k][i] = U[k][i];
        for (int vk = lo[2]; vk <= hi[2]; ++vk)
            for (int vj = lo[1]; vj <= hi[1]; ++vj)
                for (int vi = lo[0]; vi <= hi[0]; ++vi) {
                    uint32_t sig[6];
                    if (creal(tri_area_c((const cplx(*)[3])Uc, vi, vj, vk, sig)) == 0.0) continue;
                    uint64_t key = ((uint64_t)p << 40) ^ vxo_morton((uint32_t)vi, (uint32_t)vj, (uint32_t)vk);
                    for (int b = 0; b < 8; ++b) { h ^= (key >> (8 * b)) & 0xffu; h *= 1099511628211ull; }
                    for (int q = 0; q < 6; ++q)
                        for (int b = 0; b < 4; ++b) { h ^= (sig[q] >> (8 * b)) & 0xffu; h *= 1099511628211ull; }
                }
    }
    return h;
}
