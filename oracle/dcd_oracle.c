/*
 * CPU oracle for exact discrete collision detection (DCD) of edge-face
 * intersections between two triangle meshes.  TEST INFRASTRUCTURE ONLY:
 * the tests, the smoke check and the benchmark's CPU-baseline leg are the
 * only callers; the product's CUDA path never links or calls this file, and
 * this file shares no code with it.
 *
 * What it computes (Sec. 3 and Sec. 4 of the paper): every pair (edge pq of
 * the edge mesh, face abc of the oriented mesh) such that the segment pq
 * properly crosses the triangle abc.  "Properly crosses" is read as
 *   - strict plane crossing: orient(a,b,c,p) * orient(a,b,c,q) < 0, and
 *   - closed triangle: orient(p,q,a,b), orient(p,q,b,c), orient(p,q,c,a) all
 *     >= 0 or all <= 0,
 * where orient(a,b,c,x) = sign det[b-a, c-a, x-a] is positive when x lies on
 * the side the normal (b-a) x (c-a) points to (the front side, Sec. 4).
 * An endpoint on the plane, a coplanar edge, a zero-area face or a
 * zero-length edge never yields a pair.
 *
 * Exactness: orient() evaluates the determinant exactly with big integers.
 * Every finite double is m * 2^e with an integer m (|m| < 2^53); scaling all
 * twelve coordinates by 2^-emin turns them into integers, the determinant
 * of integer differences is an integer, and its sign is the sign of the
 * original determinant (the scale is a positive power of two).  No floating
 * point rounding takes part in any decision.
 *
 * The search is brute force over all edges x faces, with an axis-aligned
 * box rejection that is exact (min/max of doubles are exact): a segment and
 * a triangle that share a point share it inside both boxes.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* 2^13 bits: enough for a product of three differences of any finite
 * doubles (exponent span < 2^11, mantissa 53 bits, three factors). */
#define MAXL 256

typedef struct {
    int n;            /* limbs in use (no leading zero limbs)            */
    int neg;          /* sign of the value when n > 0                    */
    uint32_t d[MAXL]; /* magnitude, little-endian base 2^32              */
} big;

static void big_zero(big *r) { r->n = 0; r->neg = 0; }

static void big_trim(big *r) {
    while (r->n > 0 && r->d[r->n - 1] == 0) r->n--;
    if (r->n == 0) r->neg = 0;
}

/* r = m * 2^shift, m a signed 64-bit integer with |m| < 2^63 */
static void big_from_shifted(big *r, int64_t m, int shift) {
    big_zero(r);
    if (m == 0) return;
    uint64_t a = (uint64_t)(m < 0 ? -m : m);
    int limb = shift / 32, bit = shift % 32;
    memset(r->d, 0, sizeof(uint32_t) * (size_t)(limb + 4));
    /* a << bit spans at most three limbs (64 + 31 bits) */
    uint64_t lo = a << bit;
    uint64_t hi = bit ? (a >> (64 - bit)) : 0;
    r->d[limb] = (uint32_t)lo;
    r->d[limb + 1] = (uint32_t)(lo >> 32);
    r->d[limb + 2] = (uint32_t)hi;
    r->n = limb + 3;
    r->neg = m < 0;
    big_trim(r);
}

static int mag_cmp(const big *a, const big *b) {
    if (a->n != b->n) return a->n < b->n ? -1 : 1;
    for (int i = a->n - 1; i >= 0; --i)
        if (a->d[i] != b->d[i]) return a->d[i] < b->d[i] ? -1 : 1;
    return 0;
}

/* |r| = |a| + |b| */
static void mag_add(big *r, const big *a, const big *b) {
    int n = a->n > b->n ? a->n : b->n;
    uint64_t carry = 0;
    for (int i = 0; i < n; ++i) {
        uint64_t s = carry;
        if (i < a->n) s += a->d[i];
        if (i < b->n) s += b->d[i];
        r->d[i] = (uint32_t)s;
        carry = s >> 32;
    }
    r->d[n] = (uint32_t)carry;
    r->n = n + 1;
}

/* |r| = |a| - |b|, requires |a| >= |b| */
static void mag_sub(big *r, const big *a, const big *b) {
    int64_t borrow = 0;
    for (int i = 0; i < a->n; ++i) {
        int64_t s = (int64_t)a->d[i] - borrow - (i < b->n ? (int64_t)b->d[i] : 0);
        borrow = s < 0;
        r->d[i] = (uint32_t)(s + (borrow << 32));
    }
    r->n = a->n;
}

/* r = a + (negate_b ? -b : b); r must not alias a or b */
static void big_addsub(big *r, const big *a, const big *b, int negate_b) {
    int bneg = b->n ? (b->neg ^ negate_b) : 0;
    if (a->n == 0) { *r = *b; r->neg = bneg; big_trim(r); return; }
    if (b->n == 0) { *r = *a; return; }
    if (a->neg == bneg) {
        mag_add(r, a, b);
        r->neg = a->neg;
    } else if (mag_cmp(a, b) >= 0) {
        mag_sub(r, a, b);
        r->neg = a->neg;
    } else {
        mag_sub(r, b, a);
        r->neg = bneg;
    }
    big_trim(r);
}

/* r = a * b; r must not alias a or b */
static void big_mul(big *r, const big *a, const big *b) {
    if (a->n == 0 || b->n == 0) { big_zero(r); return; }
    int n = a->n + b->n;
    memset(r->d, 0, sizeof(uint32_t) * (size_t)n);
    for (int i = 0; i < a->n; ++i) {
        uint64_t carry = 0;
        for (int j = 0; j < b->n; ++j) {
            uint64_t t = (uint64_t)a->d[i] * b->d[j] + r->d[i + j] + carry;
            r->d[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
        r->d[i + b->n] = (uint32_t)carry;
    }
    r->n = n;
    r->neg = a->neg ^ b->neg;
    big_trim(r);
}

static int big_sign(const big *a) { return a->n == 0 ? 0 : (a->neg ? -1 : 1); }

/* sign of det[b-a, c-a, x-a] for points given as 3 doubles each */
int oracle_orient(const double *a, const double *b, const double *c, const double *x) {
    const double *pts[4] = {a, b, c, x};
    int64_t m[4][3];
    int e[4][3];
    int emin = 1 << 30, any = 0;
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 3; ++k) {
            double v = pts[i][k];
            if (v == 0.0) { m[i][k] = 0; e[i][k] = 0; continue; }
            int ex;
            double f = frexp(v, &ex);               /* v = f * 2^ex, 0.5 <= |f| < 1 */
            m[i][k] = (int64_t)ldexp(f, 53);        /* exact: f has a 53-bit mantissa */
            e[i][k] = ex - 53;
            if (e[i][k] < emin) emin = e[i][k];
            any = 1;
        }
    if (!any) return 0;
    /* the big-integer work area lives on the heap: it is large */
    big *B = (big *)malloc(sizeof(big) * 24);
    big *P = B;        /* P[i*3+k] = coordinate k of point i, as an integer */
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 3; ++k)
            big_from_shifted(&P[i * 3 + k], m[i][k], m[i][k] ? e[i][k] - emin : 0);
    big *u = B + 12, *v = B + 15, *w = B + 18;
    for (int k = 0; k < 3; ++k) {
        big_addsub(&u[k], &P[3 + k], &P[k], 1);  /* b - a */
        big_addsub(&v[k], &P[6 + k], &P[k], 1);  /* c - a */
        big_addsub(&w[k], &P[9 + k], &P[k], 1);  /* x - a */
    }
    /* det = u0 (v1 w2 - v2 w1) - u1 (v0 w2 - v2 w0) + u2 (v0 w1 - v1 w0) */
    big *t1 = B + 21, *t2 = B + 22, *t3 = B + 23;
    big *acc = (big *)malloc(sizeof(big) * 3);
    big *minor = acc + 1, *term = acc + 2;
    big_zero(&acc[0]);
    const int idx[3][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}};
    /* cyclic form: det = sum_i u_i (v_j w_k - v_k w_j), (i,j,k) cyclic */
    for (int r = 0; r < 3; ++r) {
        int i = idx[r][0], j = idx[r][1], k = idx[r][2];
        big_mul(t1, &v[j], &w[k]);
        big_mul(t2, &v[k], &w[j]);
        big_addsub(minor, t1, t2, 1);
        big_mul(term, &u[i], minor);
        big_addsub(t3, &acc[0], term, 0);
        acc[0] = *t3;
    }
    int s = big_sign(&acc[0]);
    free(acc);
    free(B);
    return s;
}

/* Segment pq against triangle abc under the strict-crossing, closed-triangle
 * reading.  Returns 1 on intersection and stores orient(a,b,c,p) in *side_p
 * (always -1 or +1 when 1 is returned). */
int oracle_segtri(const double *p, const double *q, const double *a,
                  const double *b, const double *c, int *side_p) {
    int sp = oracle_orient(a, b, c, p);
    if (sp == 0) return 0;
    int sq = oracle_orient(a, b, c, q);
    if (sq == 0 || sq == sp) return 0;
    int t1 = oracle_orient(p, q, a, b);
    int t2 = oracle_orient(p, q, b, c);
    int t3 = oracle_orient(p, q, c, a);
    int ok = (t1 >= 0 && t2 >= 0 && t3 >= 0) || (t1 <= 0 && t2 <= 0 && t3 <= 0);
    if (ok && side_p) *side_p = sp;
    return ok;
}

typedef struct {
    int64_t n, cap;
    int32_t *rec; /* [cap][3]: edge index, face index, side of the edge's first vertex */
} hitbuf;

static void hit_push(hitbuf *h, int32_t e, int32_t f, int32_t s) {
    if (h->n == h->cap) {
        h->cap = h->cap ? 2 * h->cap : 1024;
        h->rec = (int32_t *)realloc(h->rec, sizeof(int32_t) * 3 * (size_t)h->cap);
    }
    h->rec[3 * h->n] = e;
    h->rec[3 * h->n + 1] = f;
    h->rec[3 * h->n + 2] = s;
    h->n++;
}

/*
 * Brute-force detection of every (edge, face) intersection.
 *   PE [nve][3]   positions of the edge mesh (doubles; float inputs widened)
 *   edges [n_edges][2] vertex ids of the edges, first id smaller
 *   PF [nvf][3]   positions of the face mesh
 *   tris [n_tris][3]
 *   out [cap][3]  (edge index, face index, orient(face, first vertex))
 * Returns the number of intersecting pairs (entries past cap are dropped;
 * call again with a larger buffer).  n_threads <= 0 uses every core.
 */
int64_t oracle_detect(const double *PE, const int32_t *edges, int64_t n_edges,
                      const double *PF, const int32_t *tris, int64_t n_tris,
                      int32_t *out, int64_t cap, int n_threads) {
    double *box = (double *)malloc(sizeof(double) * 6 * (size_t)(n_tris > 0 ? n_tris : 1));
    for (int64_t f = 0; f < n_tris; ++f)
        for (int k = 0; k < 3; ++k) {
            double v0 = PF[3 * tris[3 * f] + k], v1 = PF[3 * tris[3 * f + 1] + k],
                   v2 = PF[3 * tris[3 * f + 2] + k];
            double lo = v0 < v1 ? v0 : v1, hi = v0 < v1 ? v1 : v0;
            box[6 * f + k] = v2 < lo ? v2 : lo;
            box[6 * f + 3 + k] = v2 > hi ? v2 : hi;
        }
    int nt = 1;
#ifdef _OPENMP
    nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#endif
    hitbuf *bufs = (hitbuf *)calloc((size_t)nt, sizeof(hitbuf));
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
#endif
    for (int64_t e = 0; e < n_edges; ++e) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        const double *p = PE + 3 * edges[2 * e], *q = PE + 3 * edges[2 * e + 1];
        double elo[3], ehi[3];
        for (int k = 0; k < 3; ++k) {
            elo[k] = p[k] < q[k] ? p[k] : q[k];
            ehi[k] = p[k] < q[k] ? q[k] : p[k];
        }
        for (int64_t f = 0; f < n_tris; ++f) {
            const double *bx = box + 6 * f;
            if (elo[0] > bx[3] || bx[0] > ehi[0] || elo[1] > bx[4] || bx[1] > ehi[1] ||
                elo[2] > bx[5] || bx[2] > ehi[2])
                continue;
            const double *a = PF + 3 * tris[3 * f], *b = PF + 3 * tris[3 * f + 1],
                         *c = PF + 3 * tris[3 * f + 2];
            int side;
            if (oracle_segtri(p, q, a, b, c, &side)) hit_push(&bufs[tid], (int32_t)e, (int32_t)f, side);
        }
    }
    int64_t total = 0;
    for (int t = 0; t < nt; ++t) {
        for (int64_t i = 0; i < bufs[t].n; ++i, ++total)
            if (total < cap) memcpy(out + 3 * total, bufs[t].rec + 3 * i, sizeof(int32_t) * 3);
        free(bufs[t].rec);
    }
    free(bufs);
    free(box);
    return total;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
