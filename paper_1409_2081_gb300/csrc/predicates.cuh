// Exact orientation signs and the segment-triangle test of the detection
// (Sec. 3: all edge-face intersections; front side = the side the normal
// (b - a) x (c - a) points to, Sec. 4).
//
// orient(a, b, c, x) = sign det[b - a, c - a, x - a].  Three stages:
//
// 1. float32 semi-static filter (float32 meshes).  det = u . (v x w) of the
//    rounded differences u, v, w is evaluated with explicit round-to-
//    nearest operations; every one of its six monomials passes through at
//    most 8 roundings (3 differences, 1 product, 1 subtraction, 1 product,
//    2 additions), so with unit roundoff e = 2^-24
//        |det_computed - det| <= 8e (1 + 16e) P + A,
//    P the permanent (the same expression with absolute values, computed
//    the same way) and A < 2^-108 the worst effect of underflow when every
//    coordinate is at most 2^38 in magnitude (each rounding in the
//    subnormal range adds at most 2^-150, amplified by at most |w| <= 2^39).
//    The sign is taken when |det_computed| > 2^-20 P + 2^-107 (twice the
//    relative bound, 4x the absolute one); otherwise the stage abstains.
// 2. float64 semi-static filter, same argument with e = 2^-53: the sign is
//    taken when |det| > 2^-49 P + 2^-1000.  With the validated input range
//    no intermediate underflows.  A computed permanent of exactly 0 means
//    every monomial has an exactly-zero factor, so det = 0.
// 3. exact fixed-point integers.  A float32 coordinate is an integer
//    multiple of 2^-149 and at most 2^38 in magnitude, so X = c * 2^149 is
//    an integer below 2^188 (6 x 32-bit limbs); a float64 coordinate in
//    [2^-200, 2^38] (or 0) is a multiple of 2^-252, X = c * 2^252 < 2^291
//    (10 limbs).  det is then the integer sum of six signed triple
//    products of integer differences, accumulated exactly in two's
//    complement; its sign is the sign of the original determinant.
//
// The test (strict crossing of the closed triangle):
//   orient(a,b,c,p) * orient(a,b,c,q) < 0 and orient(p,q,a,b),
//   orient(p,q,b,c), orient(p,q,c,a) all >= 0 or all <= 0.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace hfcr {

constexpr int SIGN_OPEN = 2;

struct f3 { float x, y, z; };
struct d3 { double x, y, z; };

__device__ __forceinline__ f3 fsub3(const f3 &a, const f3 &b) {
    return {__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y), __fsub_rn(a.z, b.z)};
}
__device__ __forceinline__ d3 dsub3(const d3 &a, const d3 &b) {
    return {__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y), __dsub_rn(a.z, b.z)};
}
__device__ __forceinline__ d3 widen(const f3 &a) { return {(double)a.x, (double)a.y, (double)a.z}; }

// cross = v x w with the permanent parts |v_j w_k| + |v_k w_j|
struct CrossF { f3 c, p; };
struct CrossD { d3 c, p; };

__device__ __forceinline__ CrossF fcross(const f3 &v, const f3 &w) {
    float a0 = __fmul_rn(v.y, w.z), b0 = __fmul_rn(v.z, w.y);
    float a1 = __fmul_rn(v.z, w.x), b1 = __fmul_rn(v.x, w.z);
    float a2 = __fmul_rn(v.x, w.y), b2 = __fmul_rn(v.y, w.x);
    CrossF r;
    r.c = {__fsub_rn(a0, b0), __fsub_rn(a1, b1), __fsub_rn(a2, b2)};
    r.p = {__fadd_rn(fabsf(a0), fabsf(b0)), __fadd_rn(fabsf(a1), fabsf(b1)),
           __fadd_rn(fabsf(a2), fabsf(b2))};
    return r;
}
__device__ __forceinline__ CrossD dcross(const d3 &v, const d3 &w) {
    double a0 = __dmul_rn(v.y, w.z), b0 = __dmul_rn(v.z, w.y);
    double a1 = __dmul_rn(v.z, w.x), b1 = __dmul_rn(v.x, w.z);
    double a2 = __dmul_rn(v.x, w.y), b2 = __dmul_rn(v.y, w.x);
    CrossD r;
    r.c = {__dsub_rn(a0, b0), __dsub_rn(a1, b1), __dsub_rn(a2, b2)};
    r.p = {__dadd_rn(fabs(a0), fabs(b0)), __dadd_rn(fabs(a1), fabs(b1)),
           __dadd_rn(fabs(a2), fabs(b2))};
    return r;
}

// sign of u . cr (= det[u, v, w] for cr = v x w) or SIGN_OPEN
__device__ __forceinline__ int fdot_sign(const f3 &u, const CrossF &cr) {
    float det = __fadd_rn(__fadd_rn(__fmul_rn(u.x, cr.c.x), __fmul_rn(u.y, cr.c.y)),
                          __fmul_rn(u.z, cr.c.z));
    float per = __fadd_rn(__fadd_rn(__fmul_rn(fabsf(u.x), cr.p.x), __fmul_rn(fabsf(u.y), cr.p.y)),
                          __fmul_rn(fabsf(u.z), cr.p.z));
    float eb = __fmaf_rn(per, 0x1p-20f, 0x1p-107f);
    if (det > eb) return 1;
    if (det < -eb) return -1;
    return SIGN_OPEN;
}
__device__ __forceinline__ int ddot_sign(const d3 &u, const CrossD &cr) {
    double det = __dadd_rn(__dadd_rn(__dmul_rn(u.x, cr.c.x), __dmul_rn(u.y, cr.c.y)),
                           __dmul_rn(u.z, cr.c.z));
    double per = __dadd_rn(__dadd_rn(__dmul_rn(fabs(u.x), cr.p.x), __dmul_rn(fabs(u.y), cr.p.y)),
                           __dmul_rn(fabs(u.z), cr.p.z));
    if (per == 0.0) return 0;
    double eb = __fma_rn(per, 0x1p-49, 0x1p-1000);
    if (det > eb) return 1;
    if (det < -eb) return -1;
    return SIGN_OPEN;
}

// ---------------------------------------------------------------------------
// exact fixed-point integer evaluation
// ---------------------------------------------------------------------------

// |c| * 2^149 as 6 limbs (float32 input, |c| <= 2^38)
__device__ __forceinline__ void fixed_of(float c, uint32_t *m, int &neg) {
    uint32_t bits = __float_as_uint(c);
    neg = (int)(bits >> 31);
    uint32_t E = (bits >> 23) & 0xffu, M = bits & 0x7fffffu;
    uint64_t mant = E ? (uint64_t)(M | 0x800000u) : (uint64_t)M;
    int shift = E ? (int)E - 1 : 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) m[i] = 0;
    if (mant == 0) { neg = 0; return; }
    int limb = shift >> 5, off = shift & 31;
    uint64_t v = mant << off;  // < 2^55
    if (limb < 6) m[limb] = (uint32_t)v;
    if (limb + 1 < 6) m[limb + 1] = (uint32_t)(v >> 32);
}
// |c| * 2^252 as 10 limbs (float64 input, c == 0 or 2^-200 <= |c| <= 2^38)
__device__ __forceinline__ void fixed_of(double c, uint32_t *m, int &neg) {
    uint64_t bits = (uint64_t)__double_as_longlong(c);
    neg = (int)(bits >> 63);
#pragma unroll
    for (int i = 0; i < 10; ++i) m[i] = 0;
    uint32_t E = (uint32_t)((bits >> 52) & 0x7ffu);
    uint64_t M = bits & 0xfffffffffffffull;
    if (E == 0) { neg = 0; return; }  // zero (subnormals are rejected at the boundary)
    uint64_t mant = M | (1ull << 52);
    int shift = (int)E - 823;  // value = mant * 2^(E - 1075), times 2^252
    if (shift < 0) shift = 0;  // unreachable for validated input
    int limb = shift >> 5, off = shift & 31;
    // mant << off spans up to 85 bits = three limbs
    uint64_t lo = mant << off;
    uint64_t hi = off ? (mant >> (64 - off)) : 0;
    if (limb < 10) m[limb] = (uint32_t)lo;
    if (limb + 1 < 10) m[limb + 1] = (uint32_t)(lo >> 32);
    if (limb + 2 < 10) m[limb + 2] = (uint32_t)hi;
}

template <int L>
__device__ __forceinline__ int mag_cmp(const uint32_t *a, const uint32_t *b) {
    for (int i = L - 1; i >= 0; --i)
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    return 0;
}

// (rn, r) = (an, a) - (bn, b) in sign-magnitude, L limbs; |a - b| < 2^(32L) holds
template <int L>
__device__ __forceinline__ void smag_sub(int an, const uint32_t *a, int bn, const uint32_t *b,
                                         int &rn, uint32_t *r) {
    if (an != bn) {  // magnitudes add
        uint64_t carry = 0;
        for (int i = 0; i < L; ++i) {
            uint64_t s = (uint64_t)a[i] + b[i] + carry;
            r[i] = (uint32_t)s;
            carry = s >> 32;
        }
        rn = an;
        return;
    }
    const uint32_t *x = a, *y = b;
    rn = an;
    if (mag_cmp<L>(a, b) < 0) { x = b; y = a; rn = !an; }
    int64_t borrow = 0;
    for (int i = 0; i < L; ++i) {
        int64_t s = (int64_t)x[i] - y[i] - borrow;
        borrow = s < 0;
        r[i] = (uint32_t)(s + (borrow << 32));
    }
}

// r[La + Lb] = a[La] * b[Lb]
template <int La, int Lb>
__device__ __forceinline__ void mag_mul(const uint32_t *a, const uint32_t *b, uint32_t *r) {
    for (int i = 0; i < La + Lb; ++i) r[i] = 0;
    for (int i = 0; i < La; ++i) {
        uint64_t carry = 0;
        for (int j = 0; j < Lb; ++j) {
            uint64_t t = (uint64_t)a[i] * b[j] + r[i + j] + carry;
            r[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
        r[i + Lb] = (uint32_t)carry;
    }
}

// exact sign of det[b - a, c - a, x - a]; T = float (6 limbs) or double (10)
template <typename T, int L>
__device__ __noinline__ int orient_exact(T ax, T ay, T az, T bx, T by, T bz, T cx, T cy, T cz,
                                         T xx, T xy, T xz) {
    uint32_t P[4][3][L];
    int Pn[4][3];
    const T pts[4][3] = {{ax, ay, az}, {bx, by, bz}, {cx, cy, cz}, {xx, xy, xz}};
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 3; ++k) fixed_of(pts[i][k], P[i][k], Pn[i][k]);
    // D[r][k]: row r (0: b - a, 1: c - a, 2: x - a), component k
    uint32_t D[3][3][L];
    int Dn[3][3];
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k)
            smag_sub<L>(Pn[r + 1][k], P[r + 1][k], Pn[0][k], P[0][k], Dn[r][k], D[r][k]);
    constexpr int NA = 3 * L + 1;
    uint32_t acc[NA];
    for (int i = 0; i < NA; ++i) acc[i] = 0;
    // det = sum over permutations (i, j, k) of sgn * D0_i D1_j D2_k
    const int perm[6][4] = {{0, 1, 2, 0}, {1, 2, 0, 0}, {2, 0, 1, 0},
                            {0, 2, 1, 1}, {2, 1, 0, 1}, {1, 0, 2, 1}};
    for (int t = 0; t < 6; ++t) {
        int i = perm[t][0], j = perm[t][1], k = perm[t][2];
        uint32_t m2[2 * L], m3[3 * L];
        mag_mul<L, L>(D[0][i], D[1][j], m2);
        mag_mul<2 * L, L>(m2, D[2][k], m3);
        int neg = perm[t][3] ^ Dn[0][i] ^ Dn[1][j] ^ Dn[2][k];
        // acc += (neg ? -m3 : m3), two's complement over NA limbs
        if (!neg) {
            uint64_t carry = 0;
            for (int q = 0; q < NA; ++q) {
                uint64_t s = (uint64_t)acc[q] + (q < 3 * L ? m3[q] : 0u) + carry;
                acc[q] = (uint32_t)s;
                carry = s >> 32;
            }
        } else {
            int64_t borrow = 0;
            for (int q = 0; q < NA; ++q) {
                int64_t s = (int64_t)acc[q] - (q < 3 * L ? (int64_t)m3[q] : 0) - borrow;
                borrow = s < 0;
                acc[q] = (uint32_t)(s + (borrow << 32));
            }
        }
    }
    if (acc[NA - 1] >> 31) return -1;
    for (int q = 0; q < NA; ++q)
        if (acc[q]) return 1;
    return 0;
}

// orientation from the float64 filter on, for float32 or float64 inputs
template <typename T>
__device__ __noinline__ int orient_slow(T ax, T ay, T az, T bx, T by, T bz, T cx, T cy, T cz,
                                        T xx, T xy, T xz, DevStats *st) {
    d3 a = {(double)ax, (double)ay, (double)az}, b = {(double)bx, (double)by, (double)bz},
       c = {(double)cx, (double)cy, (double)cz}, x = {(double)xx, (double)xy, (double)xz};
    d3 u = dsub3(b, a), v = dsub3(c, a), w = dsub3(x, a);
    // det[u, v, w] = w . (u x v)
    int s = ddot_sign(w, dcross(u, v));
    if (s != SIGN_OPEN) return s;
    if (st) atomicAdd(&st->exact_fallbacks, 1ull);
    constexpr int L = sizeof(T) == 4 ? 6 : 10;
    return orient_exact<T, L>(ax, ay, az, bx, by, bz, cx, cy, cz, xx, xy, xz);
}

// ---------------------------------------------------------------------------
// segment-triangle test
// ---------------------------------------------------------------------------

// float32 inputs with the float32 filter first.  Returns true on a strict
// crossing of the closed triangle; side_p = orient(a, b, c, p).
__device__ __forceinline__ bool segtri_f32(const f3 &p, const f3 &q, const f3 &a, const f3 &b,
                                           const f3 &c, int &side_p, DevStats *st) {
    f3 e1 = fsub3(b, a), e2 = fsub3(c, a);
    CrossF N = fcross(e1, e2);
    // det[e1, e2, w] = w . (e1 x e2)
    int sp = fdot_sign(fsub3(p, a), N);
    if (sp == SIGN_OPEN) {
        atomicAdd(&st->f64_fallbacks, 1ull);
        sp = orient_slow<float>(a.x, a.y, a.z, b.x, b.y, b.z, c.x, c.y, c.z, p.x, p.y, p.z, st);
    }
    if (sp == 0) return false;
    int sq = fdot_sign(fsub3(q, a), N);
    if (sq == SIGN_OPEN) {
        atomicAdd(&st->f64_fallbacks, 1ull);
        sq = orient_slow<float>(a.x, a.y, a.z, b.x, b.y, b.z, c.x, c.y, c.z, q.x, q.y, q.z, st);
    }
    if (sq != -sp) return false;
    // orient(p, q, u, v) = det[q - p, u - p, v - p] = (q - p) . ((u - p) x (v - p))
    f3 e = fsub3(q, p), wa = fsub3(a, p), wb = fsub3(b, p), wc = fsub3(c, p);
    int t1 = fdot_sign(e, fcross(wa, wb));
    if (t1 == SIGN_OPEN) {
        atomicAdd(&st->f64_fallbacks, 1ull);
        t1 = orient_slow<float>(p.x, p.y, p.z, q.x, q.y, q.z, a.x, a.y, a.z, b.x, b.y, b.z, st);
    }
    int t2 = fdot_sign(e, fcross(wb, wc));
    if (t2 == SIGN_OPEN) {
        atomicAdd(&st->f64_fallbacks, 1ull);
        t2 = orient_slow<float>(p.x, p.y, p.z, q.x, q.y, q.z, b.x, b.y, b.z, c.x, c.y, c.z, st);
    }
    if (t1 * t2 < 0) return false;
    int t3 = fdot_sign(e, fcross(wc, wa));
    if (t3 == SIGN_OPEN) {
        atomicAdd(&st->f64_fallbacks, 1ull);
        t3 = orient_slow<float>(p.x, p.y, p.z, q.x, q.y, q.z, c.x, c.y, c.z, a.x, a.y, a.z, st);
    }
    if (t1 * t3 < 0 || t2 * t3 < 0) return false;
    side_p = sp;
    return true;
}

// float64 filter first (float64 inputs, or float32 inputs with the float32
// filter switched off).
template <typename T>
__device__ __forceinline__ bool segtri_f64(const T *P, const T *Q, const T *A, const T *B,
                                           const T *C, int &side_p, DevStats *st) {
    d3 p = {(double)P[0], (double)P[1], (double)P[2]}, q = {(double)Q[0], (double)Q[1], (double)Q[2]};
    d3 a = {(double)A[0], (double)A[1], (double)A[2]}, b = {(double)B[0], (double)B[1], (double)B[2]};
    d3 c = {(double)C[0], (double)C[1], (double)C[2]};
    constexpr int L = sizeof(T) == 4 ? 6 : 10;
    d3 e1 = dsub3(b, a), e2 = dsub3(c, a);
    CrossD N = dcross(e1, e2);
    int sp = ddot_sign(dsub3(p, a), N);
    if (sp == SIGN_OPEN) {
        atomicAdd(&st->exact_fallbacks, 1ull);
        sp = orient_exact<T, L>(A[0], A[1], A[2], B[0], B[1], B[2], C[0], C[1], C[2], P[0], P[1], P[2]);
    }
    if (sp == 0) return false;
    int sq = ddot_sign(dsub3(q, a), N);
    if (sq == SIGN_OPEN) {
        atomicAdd(&st->exact_fallbacks, 1ull);
        sq = orient_exact<T, L>(A[0], A[1], A[2], B[0], B[1], B[2], C[0], C[1], C[2], Q[0], Q[1], Q[2]);
    }
    if (sq != -sp) return false;
    d3 e = dsub3(q, p), wa = dsub3(a, p), wb = dsub3(b, p), wc = dsub3(c, p);
    int t1 = ddot_sign(e, dcross(wa, wb));
    if (t1 == SIGN_OPEN) {
        atomicAdd(&st->exact_fallbacks, 1ull);
        t1 = orient_exact<T, L>(P[0], P[1], P[2], Q[0], Q[1], Q[2], A[0], A[1], A[2], B[0], B[1], B[2]);
    }
    int t2 = ddot_sign(e, dcross(wb, wc));
    if (t2 == SIGN_OPEN) {
        atomicAdd(&st->exact_fallbacks, 1ull);
        t2 = orient_exact<T, L>(P[0], P[1], P[2], Q[0], Q[1], Q[2], B[0], B[1], B[2], C[0], C[1], C[2]);
    }
    if (t1 * t2 < 0) return false;
    int t3 = ddot_sign(e, dcross(wc, wa));
    if (t3 == SIGN_OPEN) {
        atomicAdd(&st->exact_fallbacks, 1ull);
        t3 = orient_exact<T, L>(P[0], P[1], P[2], Q[0], Q[1], Q[2], C[0], C[1], C[2], A[0], A[1], A[2]);
    }
    if (t1 * t3 < 0 || t2 * t3 < 0) return false;
    side_p = sp;
    return true;
}

// orient(a, b, c, x) through all stages, for the stencil builder
template <typename T>
__device__ __forceinline__ int orient_full(const T *A, const T *B, const T *C, const T *X,
                                           int f32_filter, DevStats *st) {
    if (sizeof(T) == 4 && f32_filter) {
        f3 a = {(float)A[0], (float)A[1], (float)A[2]}, b = {(float)B[0], (float)B[1], (float)B[2]};
        f3 c = {(float)C[0], (float)C[1], (float)C[2]}, x = {(float)X[0], (float)X[1], (float)X[2]};
        int s = fdot_sign(fsub3(x, a), fcross(fsub3(b, a), fsub3(c, a)));
        if (s != SIGN_OPEN) return s;
        atomicAdd(&st->f64_fallbacks, 1ull);
    }
    return orient_slow<T>(A[0], A[1], A[2], B[0], B[1], B[2], C[0], C[1], C[2], X[0], X[1], X[2], st);
}

}  // namespace hfcr
