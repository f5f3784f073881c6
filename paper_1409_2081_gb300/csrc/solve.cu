// Constraint assembly and the global displacement minimizer (Sec. 4).
//
// Stencil s = {x0; x1, x2, x3} gives the row of grad(D) (Eq. 2): +n^T at x0
// and -n^T/3 at x1, x2, x3, n the unit normal of the face on the
// pre-response positions; D = n . (x0 - (x1 + x2 + x3)/3) (Eq. 1) and the
// right-hand side of Eq. 8 is b = D - d.  The system
// grad(D) M^-1 grad(D)^T lambda = b (Eq. 7 / Eq. 8) is solved matrix-free:
//   u = M^-1 grad(D)^T p   (per touched vertex: a fixed-order sum over the
//                           vertex's stencil entries, a CSR built by a
//                           stable sort, hence deterministic)
//   q = grad(D) u          (per stencil: gather of four vertices).
// Displacement x' - x = -M^-1 grad(D)^T lambda (Eq. 5).
//
// The matrix is block-diagonal by impact zone (stencils that share a vertex:
// connected components by min-label hooking or a lock-free union-find, both
// giving each zone its smallest stencil as label); every zone is solved on
// its own.  The response setup (vertex CSR, zones, zone-ordered rows and
// CSR, preconditioner groups) runs in one cooperative launch (k_setup), or
// as a sequence of kernels.
// MIXED: per zone (a thread group sized to the zone: one warp up to 32
// stencils, a 256-thread half CTA up to 255, a 512-thread CTA up to 1,023,
// a 512-thread CTA with all of an SM's shared memory above, an 8-CTA
// cluster beyond that; staged in shared memory), conjugate gradients in float32 on
// float32 normals, preconditioned by the inverses of the blocks of rows that
// share x0, solve for a correction of lambda; the zone's residual
// b - A lambda is recomputed in float64 with the float64 normals after every
// run (iterative refinement), until |r_zone| <= rel_tol |b_zone|.
// FP64: conjugate gradients in float64 on the whole system.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cooperative_groups.h>

#include "internal.h"
#include "sortdev.cuh"

namespace hfcr {

namespace {

constexpr int CG_THREADS = 1024;
constexpr int BIG_ZONE_THREADS = 512;  // threads of the solver of the zones of ZONE_BIG rows or more

// Loads of data written earlier in the same launch: plain where only the
// loading CTA wrote it (PlainLd), through L2 where another CTA may have
// (L2Ld), never through a possibly stale L1 line.
struct PlainLd {
    static constexpr bool L2 = false;
    template <class T> __device__ static T ld(const T *p) { return *p; }
};
struct L2Ld {
    static constexpr bool L2 = true;
    template <class T> __device__ static T ld(const T *p) { return __ldcg(p); }
};

template <class G>
__device__ __forceinline__ double4_32a ld_n64(const double4_32a *p) {
    if (!G::L2) return *p;
    const double2 lo = __ldcg((const double2 *)p), hi = __ldcg((const double2 *)p + 1);
    double4_32a r;
    r.x = lo.x; r.y = lo.y; r.z = hi.x; r.w = hi.y;
    return r;
}

constexpr int RES_BLOCKS = 512;

__device__ __forceinline__ int chk(int i, int n, uint32_t *st) {
    if ((unsigned)i < (unsigned)n) return i;
    atomicOr(st, ST_BAD_INDEX);
    return 0;
}

template <typename T>
__device__ __forceinline__ double ldd(const void *p, int i) {
    return (double)((const T *)p)[i];
}

__device__ __forceinline__ void ld_pos(const hfcr_mesh &m, int i, double *o) {
    if (m.dtype == HFCR_F32) {
        o[0] = ldd<float>(m.x, i); o[1] = ldd<float>(m.y, i); o[2] = ldd<float>(m.z, i);
    } else {
        o[0] = ldd<double>(m.x, i); o[1] = ldd<double>(m.y, i); o[2] = ldd<double>(m.z, i);
    }
}

// the largest of a non-negative double over the warp into *dst: the bit
// patterns of non-negative doubles order like the unsigned integers
__device__ __forceinline__ void warp_max_to(double v, unsigned long long *dst) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v > 0.0) atomicMax(dst, (unsigned long long)__double_as_longlong(v));
}

// row s of the constraints (Eq. 1, Eq. 2) and its right-hand side (Eq. 8);
// returns |b_s|
__device__ __forceinline__ double assemble_row(const hfcr_mesh &A, const hfcr_mesh &B,
                                               const hfcr_stencil *st, int s, double d, int4 *ids,
                                               double4_32a *n64, float4 *n32, double *b,
                                               uint32_t *status) {
    hfcr_stencil S = st[s];
    const int nA = A.n_verts;
    const hfcr_mesh &E = S.dir ? B : A;  // mesh of x0
    const hfcr_mesh &F = S.dir ? A : B;  // mesh of the face
    if (S.dir > 1u) atomicOr(status, ST_BAD_INDEX);
    int x0 = chk((int)S.x0, E.n_verts, status);
    int f = chk((int)S.face, F.n_tris, status);
    int v1 = chk(F.tris[3 * f], F.n_verts, status), v2 = chk(F.tris[3 * f + 1], F.n_verts, status),
        v3 = chk(F.tris[3 * f + 2], F.n_verts, status);
    double p0[3], p1[3], p2[3], p3[3];
    ld_pos(E, x0, p0);
    ld_pos(F, v1, p1);
    ld_pos(F, v2, p2);
    ld_pos(F, v3, p3);
    double e1[3] = {p2[0] - p1[0], p2[1] - p1[1], p2[2] - p1[2]};
    double e2[3] = {p3[0] - p1[0], p3[1] - p1[1], p3[2] - p1[2]};
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                   e1[0] * e2[1] - e1[1] * e2[0]};
    double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    double D = 0.0;
    if (nn > 0.0) {
        n[0] /= nn; n[1] /= nn; n[2] /= nn;
        double c[3];
        for (int q = 0; q < 3; ++q) c[q] = p0[q] - (p1[q] + p2[q] + p3[q]) / 3.0;
        D = n[0] * c[0] + n[1] * c[1] + n[2] * c[2];
    } else {
        n[0] = n[1] = n[2] = 0.0;  // zero-area face: an empty row, b = 0 (only from caller input)
    }
    int o = S.dir ? 0 : nA;  // offset of the face mesh in the global numbering
    int g0 = S.dir ? nA + x0 : x0;
    ids[s] = make_int4(g0, o + v1, o + v2, o + v3);
    n64[s] = make_double4_32a(n[0], n[1], n[2], 0.0);
    n32[s] = make_float4((float)n[0], (float)n[1], (float)n[2], 0.f);
    const double bs = nn > 0.0 ? D - d : 0.0;
    b[s] = bs;
    return fabs(bs);
}

// the rows, and the largest |b| of the call into *max_rhs
__global__ void k_assemble(hfcr_mesh A, hfcr_mesh B, const hfcr_stencil *st, const int *d_k,
                           int cap, double d, int4 *ids, double4_32a *n64, float4 *n32, double *b,
                           unsigned long long *max_rhs, uint32_t *status) {
    HFCR_PDL_WAIT();
    const int k = min(*d_k, cap);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const double mb = s < k ? assemble_row(A, B, st, s, d, ids, n64, n32, b, status) : 0.0;
    warp_max_to(mb, max_rhs);
}

__global__ void k_csr_entries(const int4 *ids, const int *d_k, int cap, unsigned *key, int *val) {
    HFCR_PDL_WAIT();
    int k = min(*d_k, cap);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * k) return;
    int s = i >> 2, role = i & 3;
    key[i] = (unsigned)((const int *)ids)[4 * s + role];
    val[i] = i;  // s * 4 + role
}

__global__ void k_csr_flags(const unsigned *key, const int *d_k, int cap, unsigned *flag,
                            int *d_n4) {
    HFCR_PDL_WAIT();
    int n = 4 * min(*d_k, cap);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *d_n4 = n;
    if (i < n) flag[i] = (i == 0 || key[i] != key[i - 1]) ? 1u : 0u;
}

__global__ void k_csr_build(const unsigned *key, const int *val, const unsigned *excl,
                            const int *d_k, int cap, int nA, const float *wA, const float *wB,
                            int4 *vidx, int *seg, int *gvert, float *winv) {
    HFCR_PDL_WAIT();
    int n = 4 * min(*d_k, cap);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned f = (i == 0 || key[i] != key[i - 1]) ? 1u : 0u;
    int j = (int)(excl[i] + f) - 1;
    ((int *)vidx)[val[i]] = j;
    if (f) {
        int g = (int)key[i];
        seg[j] = i;
        gvert[j] = g;
        const float *w = g < nA ? wA : wB;
        int lv = g < nA ? g : g - nA;
        winv[j] = w ? w[lv] : 1.0f;
    }
    if (i == n - 1) seg[j + 1] = n;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        T x = lane < (int)(blockDim.x >> 5) ? sh[lane] : (T)0;
#pragma unroll
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sh[32] = x;
    }
    __syncthreads();
    return sh[32];
}

template <typename T>
struct NrmT;
template <>
struct NrmT<float> { typedef float4 type; };
template <>
struct NrmT<double> { typedef double4_32a type; };

// Conjugate gradients on A x = rhs, A = J M^-1 J^T, by one CTA.
// mode 0 (MIXED inner run): rhs = r64, skipped when ctl[0] (done) is set,
//   on exit lam += x.  mode 1 (FP64): rhs = b, on exit lam = x.
// ctl[0] done flag, ctl[1] total iterations, ctl[2] inner runs.
template <typename T>
__global__ void __launch_bounds__(CG_THREADS) k_cg(
    int mode, const int *d_k, const int *d_U, const int *seg, const int *cval, const float *winv,
    const typename NrmT<T>::type *nrm, const int4 *vidx, const double *rhs64, double *lam, T *x,
    T *r, T *p, T *q, T *u, int maxit, double tol, int *ctl) {
    HFCR_PDL_WAIT();
    __shared__ T sh[33];
    if (mode == 0 && ctl[0]) return;
    const int k = *d_k, U = *d_U, tid = threadIdx.x;
    T rr_loc = 0;
    for (int s = tid; s < k; s += CG_THREADS) {
        T v = (T)rhs64[s];
        r[s] = v;
        p[s] = v;
        x[s] = 0;
        rr_loc += v * v;
    }
    T rr = block_sum(rr_loc, sh);
    const T rr0 = rr;
    const T third = (T)1 / (T)3;
    const T stop = (T)(tol * tol) * rr0;
    int it = 0;
    while (it < maxit && rr > stop && rr > (T)0) {
        // u = M^-1 J^T p
        for (int j = tid; j < U; j += CG_THREADS) {
            T a0 = 0, a1 = 0, a2 = 0;
            for (int e = seg[j]; e < seg[j + 1]; ++e) {
                int v = cval[e];
                int s = v >> 2;
                T c = (v & 3) ? -third : (T)1;
                T ps = c * p[s];
                typename NrmT<T>::type n = nrm[s];
                a0 += ps * (T)n.x;
                a1 += ps * (T)n.y;
                a2 += ps * (T)n.z;
            }
            T w = (T)winv[j];
            u[3 * j] = w * a0;
            u[3 * j + 1] = w * a1;
            u[3 * j + 2] = w * a2;
        }
        __syncthreads();
        // q = J u, pq = p . q
        T pq_loc = 0;
        for (int s = tid; s < k; s += CG_THREADS) {
            int4 vi = vidx[s];
            typename NrmT<T>::type n = nrm[s];
            T d0 = u[3 * vi.x] - (u[3 * vi.y] + u[3 * vi.z] + u[3 * vi.w]) * third;
            T d1 = u[3 * vi.x + 1] - (u[3 * vi.y + 1] + u[3 * vi.z + 1] + u[3 * vi.w + 1]) * third;
            T d2 = u[3 * vi.x + 2] - (u[3 * vi.y + 2] + u[3 * vi.z + 2] + u[3 * vi.w + 2]) * third;
            T qs = (T)n.x * d0 + (T)n.y * d1 + (T)n.z * d2;
            q[s] = qs;
            pq_loc += p[s] * qs;
        }
        T pq = block_sum(pq_loc, sh);
        if (!(pq > (T)0)) break;  // breakdown: A is singular on p
        T alpha = rr / pq;
        T rn_loc = 0;
        for (int s = tid; s < k; s += CG_THREADS) {
            x[s] += alpha * p[s];
            T rs = r[s] - alpha * q[s];
            r[s] = rs;
            rn_loc += rs * rs;
        }
        T rn = block_sum(rn_loc, sh);
        T beta = rn / rr;
        rr = rn;
        for (int s = tid; s < k; s += CG_THREADS) p[s] = r[s] + beta * p[s];
        __syncthreads();
        ++it;
    }
    for (int s = tid; s < k; s += CG_THREADS) {
        if (mode == 0) lam[s] += (double)x[s];
        else lam[s] = (double)x[s];
    }
    if (tid == 0) {
        ctl[1] += it;
        ctl[2] += 1;
    }
}

// ---------------------------------------------------------------------------
// float32 CG of the mixed solver, one CTA, single reduction per iteration
// (Chronopoulos-Gear form: s = A p is carried by a recurrence, so each
// iteration needs one product w = A r and one fused reduction of (r, r) and
// (w, r)).  Everything the iteration touches is staged in shared memory
// when it fits (64 k + 20 U bytes, k stencils, U touched vertices);
// otherwise the same loop runs on global scratch.
// ---------------------------------------------------------------------------

constexpr int FAST_SMEM = 231424;  // 226 KB dynamic (+256 B static) under the 227 KB per-CTA limit
constexpr int ZONE_MID = 256;   // zones with at least this many stencils get all 512 threads
constexpr int ZONE_PAIR_SMEM = 112 * 1024;  // k_cg_zone_pair: 2 CTAs per SM, 56 KB per half
constexpr int ZONE_BIG = 1024;  // zones with at least this many stencils get a CTA of their own

// Index types of a view: the global-memory path reads the int arrays as
// they are; the zone staged in shared memory holds zone-local indices in
// 16 bits (a staged zone has fewer than 2^16 touched vertices and CSR
// entries, since shared memory holds at most 227 KB)
__device__ __forceinline__ int4 as_int4(const int4 &v) { return v; }
__device__ __forceinline__ int4 as_int4(const ushort4 &v) { return make_int4(v.x, v.y, v.z, v.w); }

template <typename VI, typename IX>
struct CgViewT {
    float *r, *p, *x, *sv, *w;   // [k]
    float *z;                    // [k] preconditioned residual P^-1 r
    const float4 *pinv;          // [k] row of its group's inverse block (up to 4 columns)
    const int *gst;              // [G + 1] first row of each group (row offsets relative to the zone)
    int G = 0;                   // groups in the zone
    int goff = 0;                // subtracted from gst values (global path)
    float4 *u;                   // [U] M^-1 J^T r per touched vertex (w unused)
    const float4 *n4;            // [k] unit normals (float32)
    const VI *vidx;              // [k]
    const IX *seg;               // [U + 1]
    const IX *cval;              // [4 k]
    const float *winv;           // [U]
    int voff = 0, coff = 0, eoff = 0;  // subtracted from vidx, cval and seg values (global path)
    // the large zones' preconditioner (null bperm: the groups' inverse rows):
    // blocks of rows sharing x0 or a face; place q of the block order holds
    // row bperm[q], its block starts at place binfo[q] >> 5 and has
    // binfo[q] & 31 rows, and binv + 16 q holds its row of the block's
    // inverse (columns in block order)
    const uint16_t *bperm = nullptr;
    const int *binfo = nullptr;
    const float *binv = nullptr;
    __device__ __forceinline__ float3 nrm(int s) const {
        float4 v = n4[s];
        return make_float3(v.x, v.y, v.z);
    }
};
typedef CgViewT<int4, int> CgView;                // global memory
typedef CgViewT<ushort4, uint16_t> CgViewS;       // staged in shared memory

// deterministic block reduction of three sums with a single barrier: warp
// partials go to red[3 * warp]; after the barrier every warp loads the
// partials lane-parallel, folds them with the same shuffle tree and takes
// lane 0's result (lanes of a butterfly may differ in the last bit; lane
// 0's value is the same in every warp), so all threads get identical sums
__device__ __forceinline__ void block_sum3(float a, float b, float c, float *red, float &sa,
                                           float &sb_, float &sc) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        red[3 * w] = a;
        red[3 * w + 1] = b;
        red[3 * w + 2] = c;
    }
    __syncthreads();
    const int nw = blockDim.x >> 5;
    float x = lane < nw ? red[3 * lane] : 0.f;
    float y = lane < nw ? red[3 * lane + 1] : 0.f;
    float q = lane < nw ? red[3 * lane + 2] : 0.f;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
        q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    sa = __shfl_sync(0xffffffffu, x, 0);
    sb_ = __shfl_sync(0xffffffffu, y, 0);
    sc = __shfl_sync(0xffffffffu, q, 0);
}

// sum over the block, identical in every thread: each warp folds its values
// with a butterfly and keeps lane 0's result, and every thread adds the warp
// results in warp order
__device__ __forceinline__ double block_sum_uniform(double x, double *redd) {
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    x = __shfl_sync(0xffffffffu, x, 0);
    if ((threadIdx.x & 31) == 0) redd[threadIdx.x >> 5] = x;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += redd[w];
    __syncthreads();
    return s;
}

// The thread group that solves one zone: a whole CTA (CtaGroup) or one
// warp (WarpGroup, for small zones; barriers are __syncwarp and every
// reduction stays in shuffles).  Sums are identical in every lane.
struct CtaGroup {
    __device__ static int rank() { return threadIdx.x; }
    __device__ static int size() { return blockDim.x; }
    __device__ static void sync() { __syncthreads(); }
    __device__ static void sum3(float a, float b, float c, float *red, float &sa, float &sb,
                                float &sc) {
        block_sum3(a, b, c, red, sa, sb, sc);
    }
    __device__ static double sum(double x, double *redd) { return block_sum_uniform(x, redd); }
};

struct WarpGroup {
    __device__ static int rank() { return threadIdx.x & 31; }
    __device__ static int size() { return 32; }
    __device__ static void sync() { __syncwarp(); }
    __device__ static void sum3(float a, float b, float c, float *, float &sa, float &sb, float &sc) {
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
        sa = __shfl_sync(0xffffffffu, a, 0);
        sb = __shfl_sync(0xffffffffu, b, 0);
        sc = __shfl_sync(0xffffffffu, c, 0);
    }
    __device__ static double sum(double x, double *) {
#pragma unroll
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        return __shfl_sync(0xffffffffu, x, 0);
    }
};

// One 256-thread half H of a 512-thread CTA (threads 256 H .. 256 H + 255)
// solving a zone of its own: its barrier is the named barrier 1 + H, its
// reductions run over its 8 warps through its own red / redd slices (24
// floats, 8 doubles; each slot is rewritten only after another of the
// half's barriers).  Sums are identical in every thread of the half.
template <int H>
struct HalfGroup {
    __device__ static int rank() { return threadIdx.x - 256 * H; }
    __device__ static int size() { return 256; }
    __device__ static void sync() { asm volatile("bar.sync %0, 256;" ::"n"(1 + H) : "memory"); }
    __device__ static void sum3(float a, float b, float c, float *red, float &sa, float &sb,
                                float &sc) {
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
        const int lane = threadIdx.x & 31, w = (threadIdx.x >> 5) & 7;
        if (lane == 0) {
            red[3 * w] = a;
            red[3 * w + 1] = b;
            red[3 * w + 2] = c;
        }
        sync();
        float x = lane < 8 ? red[3 * lane] : 0.f;
        float y = lane < 8 ? red[3 * lane + 1] : 0.f;
        float q = lane < 8 ? red[3 * lane + 2] : 0.f;
#pragma unroll
        for (int o = 4; o; o >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, o);
            y += __shfl_xor_sync(0xffffffffu, y, o);
            q += __shfl_xor_sync(0xffffffffu, q, o);
        }
        sa = __shfl_sync(0xffffffffu, x, 0);
        sb = __shfl_sync(0xffffffffu, y, 0);
        sc = __shfl_sync(0xffffffffu, q, 0);
    }
    __device__ static double sum(double x, double *redd) {
#pragma unroll
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        x = __shfl_sync(0xffffffffu, x, 0);
        if ((threadIdx.x & 31) == 0) redd[(threadIdx.x >> 5) & 7] = x;
        sync();
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += redd[w];
        sync();
        return s;
    }
};

// z = P^-1 r for the rows of one group (block-Jacobi over rows sharing x0)
template <class V>
__device__ __forceinline__ void cg_precond_group(const V &v, int g) {
    const int a = v.gst[g] - v.goff, b = v.gst[g + 1] - v.goff;
    float rr[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) rr[q] = a + q < b ? v.r[a + q] : 0.f;
    for (int t = a; t < b; ++t) {
        float4 m = v.pinv[t];
        v.z[t] = m.x * rr[0] + m.y * rr[1] + m.z * rr[2] + m.w * rr[3];
    }
}

// z = P^-1 r with P the blocks of rows sharing x0 or a face: one place of
// the block order per thread, its row of the block's inverse (four float4
// loads) against the block's residuals, summed in column order
constexpr int BLOCK_MAX = 16;

__host__ __device__ constexpr int tri(int i) { return i * (i + 1) / 2; }

template <class Gp, class V>
__device__ __forceinline__ void cg_precond_blocks(const V &v, int k) {
    for (int q = Gp::rank(); q < k; q += Gp::size()) {
        const int info = v.binfo[q];
        const int r0 = info >> 5, m = info & 31;
        const float4 *row = (const float4 *)(v.binv + 16 * (size_t)q);
        float c[BLOCK_MAX];
#pragma unroll
        for (int t = 0; t < BLOCK_MAX / 4; ++t) {
            const float4 x = t * 4 < m ? row[t] : make_float4(0.f, 0.f, 0.f, 0.f);
            c[4 * t] = x.x;
            c[4 * t + 1] = x.y;
            c[4 * t + 2] = x.z;
            c[4 * t + 3] = x.w;
        }
        float acc = 0.f;
#pragma unroll
        for (int t = 0; t < BLOCK_MAX; ++t)
            if (t < m) acc += c[t] * v.r[v.bperm[r0 + t]];
        v.z[v.bperm[q]] = acc;
    }
}

template <class Gp, class V>
__device__ __forceinline__ void cg_matvec_vertex(const V &v, int U) {
    const float third = 1.0f / 3.0f;
    for (int j = Gp::rank(); j < U; j += Gp::size()) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
        const int e1 = (int)v.seg[j + 1] - v.eoff;
        for (int e = (int)v.seg[j] - v.eoff; e < e1; ++e) {
            int c = (int)v.cval[e] - v.coff;
            int s = c >> 2;
            float ps = ((c & 3) ? -third : 1.0f) * v.z[s];
            float3 n = v.nrm(s);
            a0 += ps * n.x;
            a1 += ps * n.y;
            a2 += ps * n.z;
        }
        float w = v.winv[j];
        v.u[j] = make_float4(w * a0, w * a1, w * a2, 0.f);
    }
}

template <class V>
__device__ __forceinline__ float cg_matvec_stencil(const V &v, int s) {
    const float third = 1.0f / 3.0f;
    int4 g = as_int4(v.vidx[s]);
    g.x -= v.voff; g.y -= v.voff; g.z -= v.voff; g.w -= v.voff;
    float3 n = v.nrm(s);
    float4 u0 = v.u[g.x], u1 = v.u[g.y], u2 = v.u[g.z], u3 = v.u[g.w];
    float d0 = u0.x - (u1.x + u2.x + u3.x) * third;
    float d1 = u0.y - (u1.y + u2.y + u3.y) * third;
    float d2 = u0.z - (u1.z + u2.z + u3.z) * third;
    return n.x * d0 + n.y * d1 + n.z * d2;
}

// returns the iteration count; x holds the solution of A x = r0
// Preconditioned CG in the Chronopoulos-Gear form (one fused reduction per
// iteration): u = P^-1 r, w = A u, s = A p by recurrence.  P is the
// block-Jacobi preconditioner over the groups.  Stops when |r| <= tol |r0|.
// Returns the iteration count; x holds the solution of A x = r0.
template <class Gp, class V>
__device__ __forceinline__ int cg_cg_loop(const V &v, int k, int U, int maxit, float tol,
                                          float *red) {
    const int tid = Gp::rank(), nt = Gp::size();
    if (v.bperm) {
        cg_precond_blocks<Gp>(v, k);
    } else {
        for (int g = tid; g < v.G; g += nt) cg_precond_group(v, g);
    }
    Gp::sync();
    cg_matvec_vertex<Gp>(v, U);
    Gp::sync();
    float ga = 0.f, de = 0.f, rh = 0.f;
    for (int s = tid; s < k; s += nt) {
        float ws = cg_matvec_stencil(v, s);
        float rs = v.r[s], zs = v.z[s];
        v.w[s] = ws;
        ga += rs * zs;
        de += ws * zs;
        rh += rs * rs;
    }
    float gamma, delta, rho;
    Gp::sum3(ga, de, rh, red, gamma, delta, rho);
    const float stop = tol * tol * rho;
    float alpha = gamma / delta, beta = 0.f;
    int it = 0;
    while (it < maxit && rho > stop && rho > 0.f && alpha > 0.f && isfinite(alpha)) {
        if (v.bperm) {
            // the blocks span rows of other threads: the update, a barrier,
            // then the blocks
            for (int s = tid; s < k; s += nt) {
                const float ps = v.z[s] + beta * v.p[s];
                const float ss = v.w[s] + beta * v.sv[s];
                v.p[s] = ps;
                v.sv[s] = ss;
                v.x[s] += alpha * ps;
                v.r[s] -= alpha * ss;
            }
            Gp::sync();
            cg_precond_blocks<Gp>(v, k);
        } else {
            for (int g = tid; g < v.G; g += nt) {
                const int a = v.gst[g] - v.goff, b = v.gst[g + 1] - v.goff;
                for (int s = a; s < b; ++s) {
                    float ps = v.z[s] + beta * v.p[s];
                    float ss = v.w[s] + beta * v.sv[s];
                    v.p[s] = ps;
                    v.sv[s] = ss;
                    v.x[s] += alpha * ps;
                    v.r[s] -= alpha * ss;
                }
                cg_precond_group(v, g);
            }
        }
        Gp::sync();
        cg_matvec_vertex<Gp>(v, U);
        Gp::sync();
        ga = 0.f;
        de = 0.f;
        rh = 0.f;
        for (int s = tid; s < k; s += nt) {
            float ws = cg_matvec_stencil(v, s);
            float rs = v.r[s], zs = v.z[s];
            v.w[s] = ws;
            ga += rs * zs;
            de += ws * zs;
            rh += rs * rs;
        }
        float gn, dn, rn;
        Gp::sum3(ga, de, rh, red, gn, dn, rn);
        beta = gn / gamma;
        alpha = gn / (dn - beta * gn / alpha);
        gamma = gn;
        rho = rn;
        ++it;
    }
    return it;
}

// ---------------------------------------------------------------------------
// impact zones (Sec. 4: constraints with overlapping stencils form one
// zone, and each zone is one linear system).  Lock-free union-find over the
// stencils that share a vertex: a root is only ever hooked under a smaller
// root (atomicCAS), so each zone ends with its smallest stencil index as
// root; path halving only rewrites non-root entries with an ancestor.
// ---------------------------------------------------------------------------

__device__ __forceinline__ int uf_find(int *parent, int x) {
    while (true) {
        int p = __ldcg(parent + x);
        if (p == x) return x;
        int gp = __ldcg(parent + p);
        if (gp != p) parent[x] = gp;
        x = p;
    }
}

// Inputs of up to UF_SMALL stencils: one CTA runs the whole union-find in
// shared memory (the same hooking rule as below, so the same labels) and
// writes the zone keys; the global-memory kernels then return at once.
constexpr int UF_SMALL = 12288;  // 48 KB of parents

__device__ __forceinline__ int uf_find_s(volatile int *par, int x) {
    while (true) {
        const int p = par[x];
        if (p == x) return x;
        const int gp = par[p];
        if (gp != p) par[x] = gp;
        x = p;
    }
}

__global__ void __launch_bounds__(1024) k_uf_small(const int *d_k, const int *d_U, const int *seg,
                                                   const int *cval, unsigned *zlab, int *zsrc,
                                                   uint32_t *status) {
    HFCR_PDL_WAIT();
    __shared__ int par[UF_SMALL];
    const int k = *d_k;
    if (k > UF_SMALL) return;
    for (int i = threadIdx.x; i < k; i += blockDim.x) par[i] = i;
    __syncthreads();
    const int U = *d_U;
    for (int j = threadIdx.x; j < U; j += blockDim.x) {
        const int e0 = seg[j], e1 = seg[j + 1];
        const int s0 = cval[e0] >> 2;
        for (int e = e0 + 1; e < e1; ++e) {
            int a = s0, b = cval[e] >> 2;
            int guard = 0;
            while (true) {
                a = uf_find_s(par, a);
                b = uf_find_s(par, b);
                if (a == b) break;
                if (a < b) { int t = a; a = b; b = t; }
                const int old = atomicCAS(par + a, a, b);
                if (old == a) break;
                a = old;
                if (++guard > (1 << 24)) { atomicOr(status, ST_TIMEOUT); break; }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        zlab[i] = (unsigned)uf_find_s(par, i);
        zsrc[i] = i;
    }
}

__global__ void k_uf_init(const int *d_k, int *parent) {
    HFCR_PDL_WAIT();
    const int k = *d_k;
    if (k <= UF_SMALL) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x)
        parent[i] = i;
}

// unions the stencils of every touched vertex (CSR by vertex)
__global__ void k_uf_union(const int *d_k, const int *d_U, const int *seg, const int *cval,
                           int *parent, uint32_t *status) {
    HFCR_PDL_WAIT();
    if (*d_k <= UF_SMALL) return;
    const int U = *d_U;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < U; j += gridDim.x * blockDim.x) {
        const int e0 = seg[j], e1 = seg[j + 1];
        const int s0 = cval[e0] >> 2;
        for (int e = e0 + 1; e < e1; ++e) {
            int a = s0, b = cval[e] >> 2;
            // every failed exchange means another thread hooked that root:
            // the count of roots falls, so the loop ends; the bound is a guard
            int guard = 0;
            while (true) {
                a = uf_find(parent, a);
                b = uf_find(parent, b);
                if (a == b) break;
                if (a < b) { int t = a; a = b; b = t; }
                int old = atomicCAS(parent + a, a, b);
                if (old == a) break;
                a = old;
                if (++guard > (1 << 24)) { atomicOr(status, ST_TIMEOUT); break; }
            }
        }
    }
}

// zone label of every stencil (its root = the smallest stencil of its zone)
__global__ void k_zone_keys(const int *d_k, int *parent, unsigned *zlab, int *zsrc) {
    HFCR_PDL_WAIT();
    const int k = *d_k;
    if (k <= UF_SMALL) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
        zlab[i] = (unsigned)uf_find(parent, i);
        zsrc[i] = i;
    }
}

__global__ void k_zone_flags(const int *d_k, const unsigned *zlab, unsigned *flags) {
    HFCR_PDL_WAIT();
    const int k = *d_k;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < k; t += gridDim.x * blockDim.x)
        flags[t] = (t == 0 || zlab[t] != zlab[t - 1]) ? 1u : 0u;
}

// regroups the rows zone by zone (zones in the order of their smallest
// stencil, stencils ascending inside a zone: the label sort is stable)
__global__ void k_zone_gather(const int *d_k, const unsigned *zlab, const int *zsrc,
                              const unsigned *excl, const int4 *ids_raw,
                              const double4_32a *n64_raw, const float4 *n32_raw,
                              const double *b_raw, int4 *ids, double4_32a *n64, float4 *n32,
                              double *b, int *szone, int *zs, int *pos_of) {
    HFCR_PDL_WAIT();
    const int k = *d_k;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < k; t += gridDim.x * blockDim.x) {
        int src = zsrc[t];
        unsigned f = (t == 0 || zlab[t] != zlab[t - 1]) ? 1u : 0u;
        int z = (int)(excl[t] + f) - 1;
        szone[t] = z;
        pos_of[src] = t;
        if (f) zs[z] = t;
        if (t == k - 1) zs[z + 1] = k;
        ids[t] = ids_raw[src];
        n64[t] = n64_raw[src];
        n32[t] = n32_raw[src];
        b[t] = b_raw[src];
    }
}

// Zone-ordered CSR: the vertex-ordered entries (s * 4 + role) are re-sorted
// stably by the zone of their stencil, so vertices come out grouped by zone
// (vertex order kept inside a zone) and entries renumbered to zone order.
__global__ void k_csr2_entries(const int *cv1, const int *pos_of, const int *szone,
                               const int *d_k, int cap, unsigned *key, int *val) {
    HFCR_PDL_WAIT();
    int k = min(*d_k, cap);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * k) return;
    int e = cv1[i];
    int t = pos_of[e >> 2];
    key[i] = (unsigned)szone[t];
    val[i] = 4 * t + (e & 3);
}

__global__ void k_csr2_flags(const int *val, const int4 *ids, const int *d_k, int cap,
                             unsigned *flag) {
    HFCR_PDL_WAIT();
    int n = 4 * min(*d_k, cap);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        flag[i] = (i == 0 || ((const int *)ids)[val[i]] != ((const int *)ids)[val[i - 1]]) ? 1u : 0u;
}

__global__ void k_csr2_build(const unsigned *zkey, const int *val, const unsigned *excl,
                             const int4 *ids, const int *d_k, int cap, int nA, const float *wA,
                             const float *wB, int4 *vidx, int *seg, int *gvert, float *winv,
                             int *zv, const int *d_nz) {
    HFCR_PDL_WAIT();
    int n = 4 * min(*d_k, cap);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int g = ((const int *)ids)[val[i]];
    unsigned f = (i == 0 || g != ((const int *)ids)[val[i - 1]]) ? 1u : 0u;
    int j = (int)(excl[i] + f) - 1;
    ((int *)vidx)[val[i]] = j;
    if (f) {
        seg[j] = i;
        gvert[j] = g;
        const float *w = g < nA ? wA : wB;
        int lv = g < nA ? g : g - nA;
        winv[j] = w ? w[lv] : 1.0f;
        if (i == 0 || zkey[i] != zkey[i - 1]) zv[zkey[i]] = j;
    }
    if (i == n - 1) {
        seg[j + 1] = n;
        zv[*d_nz] = j + 1;
    }
}

// ---------------------------------------------------------------------------
// block-Jacobi preconditioner: rows whose stencils share x0 (an edge
// endpoint crossing several faces) are nearly dependent; they are
// contiguous inside a zone (stencils are sorted by (dir, x0, face)) and are
// grouped, at most GMAX rows per group.  Each group's block of A is inverted
// once per solve.
// ---------------------------------------------------------------------------
constexpr int GMAX = 4;

__device__ __forceinline__ bool group_start(const int4 *ids, const int *szone, const int *zs,
                                            int t) {
    const int zs0 = zs[szone[t]], x0 = ids[t].x;
    int rs = t;
    while (rs > zs0 && ids[rs - 1].x == x0) --rs;
    return ((t - rs) % GMAX) == 0;
}

__global__ void k_group_flags(const int *d_k, const int4 *ids, const int *szone, const int *zs,
                              unsigned *flags) {
    HFCR_PDL_WAIT();
    const int k = *d_k;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < k; t += gridDim.x * blockDim.x)
        flags[t] = group_start(ids, szone, zs, t) ? 1u : 0u;
}

__global__ void k_group_build(const int *d_k, const int4 *ids, const int *szone, const int *zs,
                              const unsigned *excl, const int *d_nz, int *gst, int *zg) {
    HFCR_PDL_WAIT();
    const int k = *d_k;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < k; t += gridDim.x * blockDim.x) {
        const bool st = group_start(ids, szone, zs, t);
        const int g = (int)excl[t];
        if (st) {
            gst[g] = t;
            const int z = szone[t];
            if (zs[z] == t) zg[z] = g;
        }
        if (t == k - 1) {
            const int ng = g + (st ? 1 : 0);
            gst[ng] = k;
            zg[*d_nz] = ng;
        }
    }
}

// inverse mass of global vertex g (1 where the mesh gives none)
__device__ __forceinline__ double inv_mass_of(int g, int nA, const float *wA, const float *wB) {
    const float *w = g < nA ? wA : wB;
    return w ? (double)w[g < nA ? g : g - nA] : 1.0;
}

// inverse of each group's block of A = J M^-1 J^T (float64, stored float32):
// A_ab = (n_a . n_b) (w(x0) + 1/9 sum of w over the face vertices shared by
// a and b); ids are the global vertex ids (x0, face) of the zone-ordered rows
__device__ __forceinline__ void store_inv_row(float4 *p, const double *row) {
    *p = make_float4((float)row[0], (float)row[1], (float)row[2], (float)row[3]);
}
__device__ __forceinline__ void store_inv_row(double4_32a *p, const double *row) {
    *p = make_double4_32a(row[0], row[1], row[2], row[3]);
}

// R: float4 rows for the mixed solver, double4_32a rows for the float64 one
template <class G, typename R>
__device__ __forceinline__ void group_inverse_one(int g, const int *gst, const int4 *ids,
                                                  const double4_32a *n64, int nA, const float *wA,
                                                  const float *wB, R *pinv) {
    {
        const int a0 = G::ld(gst + g), m = G::ld(gst + g + 1) - a0;
        double A[GMAX][2 * GMAX];
        for (int a = 0; a < m; ++a) {
            const int4 va = G::ld(ids + a0 + a);
            const double4_32a na = ld_n64<G>(n64 + a0 + a);
            for (int b = 0; b < m; ++b) {
                const int4 vb = G::ld(ids + a0 + b);
                const double4_32a nb = ld_n64<G>(n64 + a0 + b);
                double w = inv_mass_of(va.x, nA, wA, wB);
                const int fa[3] = {va.y, va.z, va.w}, fb[3] = {vb.y, vb.z, vb.w};
                for (int p = 0; p < 3; ++p)
                    for (int q = 0; q < 3; ++q)
                        if (fa[p] == fb[q]) w += inv_mass_of(fa[p], nA, wA, wB) / 9.0;
                A[a][b] = (na.x * nb.x + na.y * nb.y + na.z * nb.z) * w;
                A[a][GMAX + b] = a == b ? 1.0 : 0.0;
            }
        }
        // Gauss-Jordan with partial pivoting; a (near-)singular block falls
        // back to the inverse of its diagonal
        bool ok = true;
        double dmax = 0.0;
        for (int a = 0; a < m; ++a) dmax = fmax(dmax, fabs(A[a][a]));
        for (int c = 0; c < m && ok; ++c) {
            int piv = c;
            for (int r = c + 1; r < m; ++r)
                if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
            if (!(fabs(A[piv][c]) > 1e-12 * dmax)) { ok = false; break; }
            if (piv != c)
                for (int q = 0; q < 2 * GMAX; ++q) {
                    double tmp = A[c][q];
                    A[c][q] = A[piv][q];
                    A[piv][q] = tmp;
                }
            const double inv = 1.0 / A[c][c];
            for (int q = 0; q < 2 * GMAX; ++q) A[c][q] *= inv;
            for (int r = 0; r < m; ++r)
                if (r != c) {
                    const double f = A[r][c];
                    for (int q = 0; q < 2 * GMAX; ++q) A[r][q] -= f * A[c][q];
                }
        }
        for (int a = 0; a < m; ++a) {
            double row[GMAX] = {0.0, 0.0, 0.0, 0.0};
            if (ok) {
                for (int b = 0; b < m; ++b) row[b] = A[a][GMAX + b];
            } else {
                // diagonal fallback computed from the untouched inputs
                const int4 va = G::ld(ids + a0 + a);
                double w = inv_mass_of(va.x, nA, wA, wB) +
                           (inv_mass_of(va.y, nA, wA, wB) + inv_mass_of(va.z, nA, wA, wB) +
                            inv_mass_of(va.w, nA, wA, wB)) / 9.0;
                row[a] = w > 0.0 ? 1.0 / w : 0.0;
            }
            store_inv_row(pinv + a0 + a, row);
        }
    }
}

__global__ void k_group_inverse(const int *d_ng, const int *gst, const int4 *ids,
                                const double4_32a *n64, int nA, const float *wA, const float *wB,
                                float4 *pinv) {
    HFCR_PDL_WAIT();
    const int ng = *d_ng;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x)
        group_inverse_one<PlainLd>(g, gst, ids, n64, nA, wA, wB, pinv);
}

// float64 residual r = b - J M^-1 J^T lam of one zone (the float64 normals;
// Eq. 7), written to v.r in float32 as the next right-hand side.  The
// vertex half goes through u64 (global scratch, this zone's rows only).
// Returns |r|^2, identical in every thread.
template <class Gp, class V>
__device__ __forceinline__ double zone_residual(const V &v, int k, int U, int s0, int j0,
                                                const double4_32a *n64, const double *b64,
                                                const double *lam, double *u64, double *redd) {
    const int tid = Gp::rank(), nt = Gp::size();
    const double third = 1.0 / 3.0;
    for (int j = tid; j < U; j += nt) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        const int e1 = (int)v.seg[j + 1] - v.eoff;
        for (int e = (int)v.seg[j] - v.eoff; e < e1; ++e) {
            const int c = (int)v.cval[e] - v.coff;
            const int sl = c >> 2;
            const double ps = ((c & 3) ? -third : 1.0) * lam[s0 + sl];
            const double4_32a n = n64[s0 + sl];
            a0 += ps * n.x;
            a1 += ps * n.y;
            a2 += ps * n.z;
        }
        const double w = (double)v.winv[j];
        double *u = u64 + 3 * (size_t)(j0 + j);
        u[0] = w * a0;
        u[1] = w * a1;
        u[2] = w * a2;
    }
    Gp::sync();
    double rr = 0.0;
    for (int t = tid; t < k; t += nt) {
        const int4 g = as_int4(v.vidx[t]);
        const double *ux = u64 + 3 * (size_t)(j0 + g.x - v.voff);
        const double *ua = u64 + 3 * (size_t)(j0 + g.y - v.voff);
        const double *ub = u64 + 3 * (size_t)(j0 + g.z - v.voff);
        const double *uc = u64 + 3 * (size_t)(j0 + g.w - v.voff);
        const double4_32a n = n64[s0 + t];
        const double d0 = ux[0] - (ua[0] + ub[0] + uc[0]) * third;
        const double d1 = ux[1] - (ua[1] + ub[1] + uc[1]) * third;
        const double d2 = ux[2] - (ua[2] + ub[2] + uc[2]) * third;
        const double r = b64[s0 + t] - (n.x * d0 + n.y * d1 + n.z * d2);
        v.r[t] = (float)r;
        rr += r * r;
    }
    return Gp::sum(rr, redd);
}

// Arguments of the zone solvers (device pointers of the zone-ordered system).
struct ZoneArgs {
    const int *zs, *zv, *zg;       // zone starts of rows, touched vertices, groups
    const int *seg, *cval;         // vertex CSR (zone-contiguous)
    const float *winv;
    const float4 *n32, *pinv;
    const double4_32a *n64;
    const int4 *vidx;
    const int *gst;
    const double *b64;
    double *lam, *u64, *zres, *zbb;
    int maxit, max_refine;
    double tol, rel_tol;
    int *ctl;
    unsigned *ticket;  // [2] zone counters of the pair launch (zero before a solve)
    // float64 per-zone solve: rows' global vertex ids, inverse masses, and the
    // float64 inverse blocks it computes
    const int4 *ids;
    int nA;
    const float *wA, *wB;
    double4_32a *pinv64;  // [cap_k]
    float *binv;          // [16 cap_k] rows of the large zones' block inverses (mixed solver)
    int block_switch;     // iterations of a large zone's run before its blocks (-1: never)
};

// |b_zone|^2 with lam = 0 for the zone's rows
template <class Gp>
__device__ __forceinline__ double zone_start(const ZoneArgs &a, int s0, int k, double *redd) {
    double bb = 0.0;
    for (int t = Gp::rank(); t < k; t += Gp::size()) {
        const double bv = a.b64[s0 + t];
        bb += bv * bv;
        a.lam[s0 + t] = 0.0;
    }
    return Gp::sum(bb, redd);
}

// shared memory a zone needs for the staged solve: per row the float32
// normal, the preconditioner row, six CG vectors, four 16-bit CSR entries
// and 16-bit vertex ids (72 B); per touched vertex u, the inverse mass and
// a 16-bit CSR offset (22 B); per group its first row; alignment slack
__device__ __forceinline__ long long zone_smem_need(int k, int U, int G) {
    return 72ll * k + 22ll * U + 4ll * G + 48;
}

struct ZoneResult {
    double rr;   // final |r|^2 of the zone
    int its;     // CG iterations
    int rounds;  // float32 runs
};

// exclusive prefix sums of a[0 .. n) in place over the whole group (each
// thread a contiguous run, warp and group scans of the runs' totals);
// returns the total.  ws: 32 ints of scratch.
template <class Gp>
__device__ __forceinline__ int group_scan_excl(int *a, int n, int *ws) {
    const int tid = Gp::rank(), nt = Gp::size();
    const int lane = tid & 31, w = tid >> 5, nw = nt >> 5;
    const int per = (n + nt - 1) / nt, lo = tid * per, hi = lo + per < n ? lo + per : n;
    int sum = 0;
    for (int i = lo; i < hi; ++i) sum += a[i];
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    Gp::sync();
    if (w == 0) {
        int t = lane < nw ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) ws[lane] = t;
    }
    Gp::sync();
    int run = (w > 0 ? ws[w - 1] : 0) + x - sum;
    const int total = ws[nw - 1];
    for (int i = lo; i < hi; ++i) {
        const int t = a[i];
        a[i] = run;
        run += t;
    }
    Gp::sync();
    return total;
}

// one union of the shared-memory union-find: the larger root is hooked
// under the smaller (so every zone's blocks are the same whatever the
// order of the unions); a lost race retries, at most a bounded number of
// times (a skipped union leaves two blocks where one would do: still a
// valid block preconditioner)
__device__ __forceinline__ void uf_union_s(int *par, int a, int b) {
    volatile int *vp = par;
    for (int tries = 0; tries < 4096; ++tries) {
        a = uf_find_s(vp, a);
        b = uf_find_s(vp, b);
        if (a == b) return;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(par + b, b, a) == b) return;
    }
}

// The inverse of one block of m <= N rows (rows[0 .. m)), in float64 (a
// block of nearly dependent rows has a large condition number, and its
// float32 inverse can come out indefinite): the matrix from the float32
// normals (products exact in float64), factored L L^T (the diagonal kept as
// 1 / L_ii; a pivot below 1e-12 of its diagonal entry makes the block its
// diagonal), L^-1, then L^-T L^-1, symmetric by construction, rounded to
// float32; row i to out + 16 i.  N fixes the unrolled bounds (a block pays
// for the size class it falls in).
template <int N, class V>
__device__ __forceinline__ void block_inverse(const V &v, const uint16_t *rows, int m, float *out) {
    const double third = 1.0 / 3.0;
    double Lr[tri(N)];
    bool ok = true;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (i >= m) continue;
        const int si = rows[i];
        const ushort4 gi = v.vidx[si];
        const float3 ni = v.nrm(si);
        const int vi[4] = {gi.x, gi.y, gi.z, gi.w};
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            const int sj = rows[j];
            const ushort4 gj = v.vidx[sj];
            const float3 nj = v.nrm(sj);
            const int vj[4] = {gj.x, gj.y, gj.z, gj.w};
            double wsh = 0.0;
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (vi[p] == vj[q]) wsh += (p ? -third : 1.0) * (q ? -third : 1.0) * (double)v.winv[vi[p]];
            const double dot = (double)ni.x * nj.x + (double)ni.y * nj.y + (double)ni.z * nj.z;
            double a_ij = dot * wsh;
            const double a_ii = a_ij;
#pragma unroll
            for (int q = 0; q < j; ++q) a_ij -= Lr[tri(i) + q] * Lr[tri(j) + q];
            if (j < i) {
                Lr[tri(i) + j] = a_ij * Lr[tri(j) + j];
            } else if (ok && a_ij > 1e-12 * a_ii && isfinite(a_ij)) {
                Lr[tri(i) + i] = rsqrt(a_ij);
            } else {
                ok = false;
            }
        }
    }
    if (!ok) {
        // the block's diagonal alone
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (i >= m) continue;
            const int si = rows[i];
            const ushort4 gi = v.vidx[si];
            const float3 ni = v.nrm(si);
            const int vi[4] = {gi.x, gi.y, gi.z, gi.w};
            double wsh = 0.0;
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (vi[p] == vi[q]) wsh += (p ? -third : 1.0) * (q ? -third : 1.0) * (double)v.winv[vi[p]];
            const double d = ((double)ni.x * ni.x + (double)ni.y * ni.y + (double)ni.z * ni.z) * wsh;
#pragma unroll
            for (int q = 0; q < i; ++q) Lr[tri(i) + q] = 0.0;
            Lr[tri(i) + i] = d > 0.0 && isfinite(d) ? rsqrt(d) : 1.0;
        }
    }
    double Li[tri(N)];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        if (j >= m) continue;
        Li[tri(j) + j] = Lr[tri(j) + j];
#pragma unroll
        for (int i = j + 1; i < N; ++i) {
            if (i >= m) continue;
            double t = 0.0;
#pragma unroll
            for (int q = j; q < i; ++q) t += Lr[tri(i) + q] * Li[tri(q) + j];
            Li[tri(i) + j] = -t * Lr[tri(i) + i];
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (i >= m) continue;
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            double t = 0.0;
#pragma unroll
            for (int q = i; q < N; ++q)
                if (q < m) t += Li[tri(q) + i] * Li[tri(q) + j];
            out[16 * i + j] = (float)t;
            out[16 * j + i] = (float)t;
        }
    }
}

// The inverse of one block of 4 < m <= BLOCK_MAX rows by one warp, in
// float64: lane j < 16 holds column j of the block's matrix, lane 16 + j
// column j of the identity; Gauss-Jordan elimination without pivoting (the
// matrix is symmetric positive definite), the pivot column broadcast by
// shuffles at each step, turns the right half into the inverse, which is
// written rounded to float32 and made symmetric pairwise; a pivot that is
// not positive makes the block its diagonal.  Called by every lane.
template <class V>
__device__ __forceinline__ void block_inverse_warp(const V &v, const uint16_t *rows, int m, float *out) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, j = lane & 15;
    const double third = 1.0 / 3.0;
    double c[BLOCK_MAX];
#pragma unroll
    for (int i = 0; i < BLOCK_MAX; ++i) c[i] = 0.0;
    if (lane < 16 && j < m) {
        const int sj = rows[j];
        const ushort4 gj = v.vidx[sj];
        const float3 nj = v.nrm(sj);
        const int vj[4] = {gj.x, gj.y, gj.z, gj.w};
#pragma unroll
        for (int i = 0; i < BLOCK_MAX; ++i) {
            if (i >= m) continue;
            const int si = rows[i];
            const ushort4 gi = v.vidx[si];
            const float3 ni = v.nrm(si);
            const int vi[4] = {gi.x, gi.y, gi.z, gi.w};
            double wsh = 0.0;
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (vi[p] == vj[q]) wsh += (p ? -third : 1.0) * (q ? -third : 1.0) * (double)v.winv[vi[p]];
            c[i] = ((double)ni.x * nj.x + (double)ni.y * nj.y + (double)ni.z * nj.z) * wsh;
        }
    } else if (lane >= 16 && j < m) {
#pragma unroll
        for (int i = 0; i < BLOCK_MAX; ++i)
            if (i == j) c[i] = 1.0;
    }
    double dj = 0.0;  // the block's diagonal entry of lane j (< 16), for the fallback
#pragma unroll
    for (int i = 0; i < BLOCK_MAX; ++i)
        if (i == j) dj = c[i];
    bool ok = true;
#pragma unroll
    for (int kk = 0; kk < BLOCK_MAX; ++kk) {
        if (kk >= m) break;
        const double piv = __shfl_sync(full, c[kk], kk);
        const double d0 = __shfl_sync(full, dj, kk);
        ok = ok && piv > 1e-12 * d0 && isfinite(piv);
        c[kk] *= 1.0 / piv;
#pragma unroll
        for (int i = 0; i < BLOCK_MAX; ++i) {
            if (i >= m || i == kk) continue;
            const double f = __shfl_sync(full, c[i], kk);
            c[i] -= f * c[kk];
        }
    }
    if (ok) {
        if (lane >= 16 && j < m) {
#pragma unroll
            for (int i = 0; i < BLOCK_MAX; ++i)
                if (i < m) out[16 * i + j] = (float)c[i];
        }
        __syncwarp();
        // (i, u) and (u, i) to their mean, the pair handled by lane i > u
        if (lane < m) {
            for (int u = 0; u < lane; ++u) {
                const float x = 0.5f * (out[16 * lane + u] + out[16 * u + lane]);
                out[16 * lane + u] = x;
                out[16 * u + lane] = x;
            }
        }
    } else if (lane < 16 && j < m) {
        for (int i = 0; i < m; ++i) out[16 * i + j] = i == j ? (dj > 0.0 && isfinite(dj) ? (float)(1.0 / dj) : 1.f) : 0.f;
    }
    __syncwarp();
}

// The preconditioner blocks of a staged large zone (Sec. 4's rows of one
// impact zone): rows joined when they share x0 or the face (their nearly
// parallel rows make the zone's system ill-conditioned, and a block that
// holds them all captures that); a component of at most BLOCK_MAX rows is
// one block, a larger one is cut into runs of whole x0 groups of at most
// BLOCK_MAX rows, in row order.  Rows are ordered by block
// (ascending within a block), and every block's matrix, entry (s, t) =
// (n_s . n_t) sum over the vertices v the two rows share of c_s(v) c_t(v)
// w(v) (c = 1 at x0, -1/3 at a face vertex), is factored L L^T in float32
// (a pivot that is not positive makes the block its diagonal) and inverted
// as L^-T L^-1, which is symmetric by construction; place q of the block
// order gets its row bperm[q], its block's start and size binfo[q] and its
// row of the inverse at binv + 16 q.  Called between rounds; scratch: the
// CG vectors p, sv, w, z and x (dead between rounds), bst (k + 1 ints) and
// 96 ints at ws.  Returns the block count.  Not inlined: its register
// needs (the unrolled factorisations) stay out of the CG loop's allocation.
template <class Gp>
__device__ __noinline__ int zone_blocks(const CgViewS &v, int k, int U, const int *gst, int G,
                                           uint16_t *bperm, int *binfo, int *bst, float *binv,
                                           int *ws) {
    const int tid = Gp::rank(), nt = Gp::size();
    int *par = (int *)v.p;   // [k] union-find parents, then each row's block key
    int *cnt = (int *)v.sv;  // [k] component sizes, then block numbers of the keys
    int *hist = (int *)v.w;  // [k + 1] rows per key (w and z are contiguous)
    for (int t = tid; t < k; t += nt) {
        par[t] = t;
        cnt[t] = 0;
    }
    for (int t = tid; t <= k; t += nt) hist[t] = 0;
    Gp::sync();
    // rows with the same x0 are neighbours in the zone's order (dir, x0, face)
    for (int t = 1 + tid; t < k; t += nt)
        if (v.vidx[t].x == v.vidx[t - 1].x) uf_union_s(par, t, t - 1);
    // rows with the same face both list its first vertex in role 1
    for (int j = tid; j < U; j += nt) {
        const int e0 = v.seg[j], e1 = v.seg[j + 1];
        for (int e = e0; e < e1; ++e) {
            const int c = v.cval[e];
            if ((c & 3) != 1) continue;
            const ushort4 gs = v.vidx[c >> 2];
            for (int f = e + 1; f < e1; ++f) {
                const int c2 = v.cval[f];
                if ((c2 & 3) != 1) continue;
                const ushort4 gt = v.vidx[c2 >> 2];
                if (gs.z == gt.z && gs.w == gt.w) uf_union_s(par, c >> 2, c2 >> 2);
            }
        }
    }
    Gp::sync();
    for (int t = tid; t < k; t += nt) par[t] = uf_find_s((volatile int *)par, t);
    Gp::sync();
    for (int t = tid; t < k; t += nt) atomicAdd(&cnt[par[t]], 1);
    int *keys = (int *)v.x;  // the block key of each row (x is dead between rounds)
    int *nbig = ws + 32, *big = ws + 33;
    if (tid == 0) *nbig = 0;
    Gp::sync();
    // the components of more than BLOCK_MAX rows (up to 63 of them)
    for (int t = tid; t < k; t += nt)
        if (par[t] == t && cnt[t] > BLOCK_MAX) {
            const int i = atomicAdd(nbig, 1);
            if (i < 63) big[i] = t;
        }
    // block key of a row: its component's root; in a larger component the
    // first row of its x0 group, unless that component is split below
    for (int g = tid; g < G; g += nt)
        for (int t = gst[g]; t < gst[g + 1]; ++t) {
            const int r = par[t];
            keys[t] = cnt[r] <= BLOCK_MAX ? r : gst[g];
        }
    Gp::sync();
    // a listed large component in runs of whole x0 groups, in row order, of
    // at most BLOCK_MAX rows (one thread a component; the key of a run is
    // its first row)
    const int nb_list = *nbig < 63 ? *nbig : 63;
    for (int c = tid; c < nb_list; c += nt) {
        const int r = big[c];
        int acc = 0, key = -1;
        for (int g = 0; g < G; ++g) {
            const int t0 = gst[g];
            if (par[t0] != r) continue;
            const int sz = gst[g + 1] - t0;
            if (key < 0 || acc + sz > BLOCK_MAX) {
                key = t0;
                acc = 0;
            }
            acc += sz;
            for (int t = t0; t < t0 + sz; ++t) keys[t] = key;
        }
    }
    Gp::sync();
    for (int t = tid; t < k; t += nt) atomicAdd(&hist[keys[t]], 1);
    Gp::sync();
    group_scan_excl<Gp>(hist, k + 1, ws);  // hist[key]: first place of the key's rows
    for (int q = tid; q < k; q += nt) cnt[q] = hist[q + 1] > hist[q] ? 1 : 0;
    Gp::sync();
    const int NB = group_scan_excl<Gp>(cnt, k, ws);
    for (int q = tid; q < k; q += nt)
        if (hist[q + 1] > hist[q]) bst[cnt[q]] = hist[q];
    if (tid == 0) bst[NB] = k;
    Gp::sync();
    for (int t = tid; t < k; t += nt) bperm[atomicAdd(&hist[keys[t]], 1)] = (uint16_t)t;
    Gp::sync();
    // one thread per block: its rows in ascending order, then the inverse of
    // a block of at most 4 rows; the larger ones are listed for the warps
    int *wlist = cnt;  // the block numbers are no longer needed
    int *nwl = ws + 32;
    if (tid == 0) *nwl = 0;
    Gp::sync();
    for (int b = tid; b < NB; b += nt) {
        const int r0 = bst[b], m = bst[b + 1] - r0;
        for (int i = 1; i < m; ++i) {
            const uint16_t x = bperm[r0 + i];
            int j = i - 1;
            while (j >= 0 && bperm[r0 + j] > x) {
                bperm[r0 + j + 1] = bperm[r0 + j];
                --j;
            }
            bperm[r0 + j + 1] = x;
        }
        for (int i = 0; i < m; ++i) binfo[r0 + i] = (r0 << 5) | m;
        if (m <= 4)
            block_inverse<4>(v, bperm + r0, m, binv + 16 * (size_t)r0);
        else
            wlist[atomicAdd(nwl, 1)] = b;  // for a warp below
    }
    Gp::sync();
    // the larger blocks, one warp each
    {
        const int nwarps = nt >> 5, w = tid >> 5, nl = *nwl;
        for (int i = w; i < nl; i += nwarps) {
            const int b = wlist[i], r0 = bst[b];
            block_inverse_warp(v, bperm + r0, bst[b + 1] - r0, binv + 16 * (size_t)r0);
        }
    }
    Gp::sync();
    return NB;
}

// Rounds of iterative refinement of zone z, everything the float32 CG
// touches staged in shared memory at base (zone_smem_need bytes); BLK: the
// large zones' preconditioner blocks (zone_blocks) instead of the groups.
template <class Gp, bool BLK = false>
__device__ __forceinline__ ZoneResult solve_zone_smem(const ZoneArgs &a, int z, char *base, double bb,
                                                      float *red, double *redd) {
    const int tid = Gp::rank(), nt = Gp::size();
    const int s0 = a.zs[z], k = a.zs[z + 1] - s0;
    const int j0 = a.zv[z], U = a.zv[z + 1] - j0;
    const int g0 = a.zg[z], G = a.zg[z + 1] - g0;
    const int e0 = a.seg[j0];
    const double target = a.rel_tol * a.rel_tol * bb;
    CgViewS v;
    // layout: n4 | pinv | u | r p x sv w z | winv | gst | vidx (16-bit) | seg (16-bit) | cval (16-bit)
    float4 *n4 = (float4 *)base;
    float4 *pinv = n4 + k;
    v.u = pinv + k;
    float *f = (float *)(v.u + U);
    v.r = f; v.p = f + k; v.x = f + 2 * k; v.sv = f + 3 * k; v.w = f + 4 * k; v.z = f + 5 * k;
    float *winv = f + 6 * k;
    int *gst = (int *)(winv + U);
    ushort4 *vidx = (ushort4 *)(((uintptr_t)(gst + G + 1) + 7) & ~(uintptr_t)7);
    uint16_t *seg = (uint16_t *)(vidx + k);
    uint16_t *cval = seg + U + 1;
    for (int t = tid; t < k; t += nt) {
        const int4 g = a.vidx[s0 + t];
        vidx[t] = make_ushort4((unsigned short)(g.x - j0), (unsigned short)(g.y - j0),
                               (unsigned short)(g.z - j0), (unsigned short)(g.w - j0));
        n4[t] = a.n32[s0 + t];
        pinv[t] = a.pinv[s0 + t];
        v.r[t] = (float)a.b64[s0 + t];
    }
    for (int g = tid; g <= G; g += nt) gst[g] = a.gst[g0 + g] - s0;
    v.pinv = pinv; v.gst = gst; v.G = G; v.goff = 0;
    for (int j = tid; j <= U; j += nt) seg[j] = (uint16_t)(a.seg[j0 + j] - e0);
    for (int j = tid; j < U; j += nt) winv[j] = a.winv[j0 + j];
    for (int e = tid; e < 4 * k; e += nt) cval[e] = (uint16_t)(a.cval[e0 + e] - 4 * s0);
    v.n4 = n4;
    v.vidx = vidx; v.seg = seg; v.cval = cval; v.winv = winv;
    v.voff = 0; v.coff = 0; v.eoff = 0;
    double rr = bb;
    int its = 0, rounds = 0, extra = 0;
    // BLK: a run stops after block_switch iterations; a zone that needs
    // more (an ill-conditioned one) keeps that run's correction and
    // continues on the blocks (that run is not counted)
    bool blocks_on = false;
    const bool may_switch = BLK && a.block_switch > 0 && a.block_switch < a.maxit;
    while (rr > target && rounds < a.max_refine + extra) {
        for (int t = tid; t < k; t += nt) {
            v.p[t] = 0.f;
            v.sv[t] = 0.f;
            v.x[t] = 0.f;
        }
        Gp::sync();
        const int cap_it = may_switch && !blocks_on ? a.block_switch : a.maxit;
        const int n_it = cg_cg_loop<Gp>(v, k, U, cap_it, (float)a.tol, red);
        its += n_it;
        for (int t = tid; t < k; t += nt) a.lam[s0 + t] += (double)v.x[t];
        Gp::sync();
        const double rr_prev = rr;
        rr = zone_residual<Gp>(v, k, U, s0, j0, a.n64, a.b64, a.lam, a.u64, redd);
        ++rounds;
        if (!(rr < rr_prev)) {
            // the run did not reduce the float64 residual (a stagnating or
            // failing float32 run): its correction is taken back, the zone
            // keeps the best lambda found
            for (int t = tid; t < k; t += nt) a.lam[s0 + t] -= (double)v.x[t];
            rr = rr_prev;
            Gp::sync();
            break;
        }
        if (may_switch && !blocks_on && n_it >= cap_it && rr > target) {
            // the block order, the places' blocks and the block starts in
            // the groups' inverse rows' slot (16 B a row: 2 + 4 + 4)
            uint16_t *bperm = (uint16_t *)pinv;
            int *binfo = (int *)(bperm + ((k + 7) & ~7));
            int *bst = binfo + k;
            float *binv = a.binv + 16 * (size_t)s0;
            zone_blocks<Gp>(v, k, U, gst, G, bperm, binfo, bst, binv, (int *)red);
            v.bperm = bperm;
            v.binfo = binfo;
            v.binv = binv;
            blocks_on = true;
            extra = 1;
        }
    }
    ZoneResult res;
    res.rr = rr;
    res.its = its;
    res.rounds = rounds;
    return res;
}

__device__ __forceinline__ void zone_finish(const ZoneArgs &a, int z, double rr, double bb, int its,
                                            int rounds, bool in_smem) {
    a.zres[z] = rr;
    a.zbb[z] = bb;
    atomicAdd(&a.ctl[1], its);
    atomicAdd(&a.ctl[2], rounds);
    atomicMax(&a.ctl[3], rounds);
    atomicOr(&a.ctl[4], in_smem ? 1 : 2);
}

// One warp per zone of at most WARP_ZONE stencils (most zones of a batch of
// small mesh pairs): a 256-thread CTA runs eight of them side by side, each
// in its own WARP_ZONE_SMEM slice of shared memory.
constexpr int WARP_ZONE = 32;
constexpr int WARP_ZONE_SMEM = 6272;  // at least zone_smem_need(32, 128, 32), a multiple of 16 B
constexpr int WARP_ZONE_WARPS = 8;

__global__ void __launch_bounds__(256, 4) k_cg_zone_warp(const int *d_nz, ZoneArgs a) {
    HFCR_PDL_WAIT();
    extern __shared__ float4 smem4[];
    const int nz = *d_nz, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    char *base = (char *)smem4 + (size_t)w * WARP_ZONE_SMEM;
    const int nwarps = gridDim.x * WARP_ZONE_WARPS;
    for (int z = blockIdx.x * WARP_ZONE_WARPS + w; z < nz; z += nwarps) {
        const int s0 = a.zs[z], k = a.zs[z + 1] - s0;
        if (k > WARP_ZONE) continue;
        const double bb = zone_start<WarpGroup>(a, s0, k, nullptr);
        const ZoneResult r = solve_zone_smem<WarpGroup>(a, z, base, bb, nullptr, nullptr);
        if (lane == 0) zone_finish(a, z, r.rr, bb, r.its, r.rounds, true);
        __syncwarp();  // the slice is reused by the warp's next zone
    }
}

// Zone z solved by the thread group Gp: staged in shared memory at base
// when its data fit smem_bytes, else the same rounds on global scratch.
// The two paths are instantiated separately so that the shared-memory one
// sees pointers derived only from the shared array (LDS/STS, not generic
// loads).
struct ZoneScratch {
    float *x, *r, *p, *s, *w, *z, *u;
};

template <class Gp, bool BLK = false>
__device__ __forceinline__ void solve_zone(const ZoneArgs &a, int z, char *base, int smem_bytes,
                                           float *red, double *redd, const ZoneScratch &g) {
    const int tid = Gp::rank(), nt = Gp::size();
    const int s0 = a.zs[z], k = a.zs[z + 1] - s0;
    const int j0 = a.zv[z], U = a.zv[z + 1] - j0;
    const double bb = zone_start<Gp>(a, s0, k, redd);
    const int g0 = a.zg[z], G = a.zg[z + 1] - g0;
    const bool in_smem = zone_smem_need(k, U, G) <= smem_bytes;
    int its = 0, rounds = 0;
    double rr;
    if (in_smem) {
        const ZoneResult r = solve_zone_smem<Gp, BLK>(a, z, base, bb, red, redd);
        rr = r.rr;
        its = r.its;
        rounds = r.rounds;
    } else {
        const double target = a.rel_tol * a.rel_tol * bb;
        CgView v;
        v.r = g.r + s0; v.p = g.p + s0; v.x = g.x + s0; v.sv = g.s + s0; v.w = g.w + s0;
        v.z = g.z + s0;
        v.u = (float4 *)g.u + j0;
        v.n4 = a.n32 + s0;
        v.pinv = a.pinv + s0; v.gst = a.gst + g0; v.G = G; v.goff = s0;
        v.vidx = a.vidx + s0; v.seg = a.seg + j0; v.cval = a.cval; v.winv = a.winv + j0;
        v.voff = j0; v.coff = 4 * s0; v.eoff = 0;
        for (int t = tid; t < k; t += nt) v.r[t] = (float)a.b64[s0 + t];
        rr = bb;
        while (rr > target && rounds < a.max_refine) {
            for (int t = tid; t < k; t += nt) {
                v.p[t] = 0.f;
                v.sv[t] = 0.f;
                v.x[t] = 0.f;
            }
            Gp::sync();
            its += cg_cg_loop<Gp>(v, k, U, a.maxit, (float)a.tol, red);
            for (int t = tid; t < k; t += nt) a.lam[s0 + t] += (double)v.x[t];
            Gp::sync();
            const double rr_prev = rr;
            rr = zone_residual<Gp>(v, k, U, s0, j0, a.n64, a.b64, a.lam, a.u64, redd);
            ++rounds;
            if (!(rr < rr_prev)) {  // as in the staged path: the run is taken back
                for (int t = tid; t < k; t += nt) a.lam[s0 + t] -= (double)v.x[t];
                rr = rr_prev;
                Gp::sync();
                break;
            }
        }
    }
    if (tid == 0) zone_finish(a, z, rr, bb, its, rounds, in_smem);
    Gp::sync();  // shared memory is reused by the group's next zone
}

// The mixed solver's CTA launches (k_cg_zone_warp takes the zones of at
// most WARP_ZONE stencils).  k_cg_zone_pair: the zones of ZONE_MID to
// ZONE_BIG - 1 stencils one at a time on all 512 threads, then the smaller
// ones two at a time, one per 256-thread half (its own named barrier, half
// the shared memory), so that a zone gets about one to four rows per
// thread.  k_cg_zone<BIG_ZONE_THREADS>: the rest, one CTA with all of
// shared memory each (512 threads: measured a little faster than 1,024 on
// the frame sequence's large zones, 0.546 against 0.566 ms per frame, and
// cheaper barriers and reductions).  (solve_zone
// ends with its group's barrier, so the halves may reuse the shared memory
// of the CTA's last whole-CTA zone.)
// Zone assignment of the pair launch: a solver's first zone is fixed (so
// that while there are fewer zones than solvers each zone has an SM to
// itself), the following ones are taken from a counter in turn (zones
// differ widely in size; the counter balances them).  stride = the
// solvers; the counter counts the zones taken beyond the fixed ones.
// Returns the group's next zone, identical in every thread of the group
// (slot: the group's shared word).
template <class Gp>
__device__ __forceinline__ int next_zone(unsigned *counter, int stride, int *slot) {
    if (Gp::rank() == 0) *slot = stride + (int)atomicAdd(counter, 1u);
    Gp::sync();
    const int z = *slot;
    Gp::sync();  // the slot is rewritten by the next call
    return z;
}

// The zones of at least ZONE_MID stencils go to the large-zone launch, one
// CTA each, when at least one of them has ZONE_BIG stencils or more and
// there are at most ROUTE_MAX of them (and no more than its CTAs): a
// frame's large contact zone and the few medium ones beside it then run
// side by side instead of one launch after the other, and each may switch
// to its blocks.  Otherwise the pair launch takes those below ZONE_BIG:
// alone, a medium zone is faster there (measured: a 538-row zone of the
// two-tori scene, 0.26 against 0.37 ms; the large-zone CTA's shared memory
// leaves little L1 for the float64 rounds), and many of them (a batch)
// share its two CTAs per SM.  Both launches count the zones from the zone
// starts (one barrier per blockDim.x zones), so they take the same
// decision.  Returns how many zones have at least lo stencils, *n_big how
// many at least ZONE_BIG; *pick: the zone of rank `rank` among the first
// ones in zone order, -1 if none (all identical in every thread of the CTA).
constexpr int ROUTE_MAX = 8;

__device__ __forceinline__ int zones_at_least(const int *zs, int nz, int lo, int rank, int *pick,
                                              int *n_big) {
    __shared__ int wc[32];
    __shared__ int found;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) found = -1;
    int total = 0, big = 0;
    for (int base = 0; base < nz; base += blockDim.x) {
        const int z = base + threadIdx.x;
        const int kz = z < nz ? zs[z + 1] - zs[z] : 0;
        const bool pred = kz >= lo;
        big += __syncthreads_count(kz >= ZONE_BIG);
        const int c = __syncthreads_count(pred);
        if (rank >= total && rank < total + c) {  // the same in every thread
            const unsigned bal = __ballot_sync(0xffffffffu, pred);
            if (lane == 0) wc[w] = __popc(bal);
            __syncthreads();
            int before = total + __popc(bal & ((1u << lane) - 1u));
            for (int q = 0; q < w; ++q) before += wc[q];
            if (pred && before == rank) found = z;
        }
        total += c;
    }
    __syncthreads();
    *pick = found;
    *n_big = big;
    return total;
}

// the zones of small_lo < k < ZONE_MID stencils on half H (first fixed
// zone: blockIdx.x + H gridDim.x)
template <int H>
__device__ __forceinline__ void half_zones(const ZoneArgs &a, int nz, int small_lo, char *base,
                                           int bytes, float *red, double *redd,
                                           const ZoneScratch &g, int *slot) {
    const bool more = nz > 2 * (int)gridDim.x;  // zones beyond the fixed ones
    for (int z = blockIdx.x + H * gridDim.x; z < nz;
         z = more ? next_zone<HalfGroup<H>>(a.ticket + 1, 2 * gridDim.x, slot) : nz) {
        const int k = a.zs[z + 1] - a.zs[z];
        if (k <= small_lo || k >= ZONE_MID) continue;
        solve_zone<HalfGroup<H>>(a, z, base, bytes, red, redd, g);
    }
}

__global__ void __launch_bounds__(512, 2) k_cg_zone_pair(const int *d_nz, ZoneArgs a, int small_lo,
                                                         ZoneScratch g, int smem_bytes, int big_ctas) {
    HFCR_PDL_WAIT();
    extern __shared__ float4 smem4[];
    __shared__ float red[96];     // halves: 24 floats each; the whole CTA: 48
    __shared__ double redd[16];   // halves: 8 each; the whole CTA: 16
    __shared__ int slot[3];
    const int nz = *d_nz;
    // the larger zones first, on all 512 threads (unless the large-zone
    // launch takes them)
    __shared__ int first;
    {
        int unused, n_big;
        const int n_mid = zones_at_least(a.zs, nz, ZONE_MID, -1, &unused, &n_big);
        const bool to_big = n_big > 0 && n_mid <= ROUTE_MAX && n_mid <= big_ctas;
        if (threadIdx.x == 0) first = to_big ? nz : (int)blockIdx.x;
        __syncthreads();
    }
    const bool more = nz > (int)gridDim.x;  // zones beyond the fixed ones
    for (int z = first; z < nz; z = more ? next_zone<CtaGroup>(a.ticket, gridDim.x, slot + 2) : nz) {
        const int k = a.zs[z + 1] - a.zs[z];
        if (k < ZONE_MID || k >= ZONE_BIG) continue;
        solve_zone<CtaGroup>(a, z, (char *)smem4, smem_bytes, red, redd, g);
    }
    // then the smaller ones, two at a time (a whole-CTA zone ends with a
    // barrier of the whole CTA, so the halves may reuse the shared memory)
    const int half_bytes = (smem_bytes / 2) & ~15;
    if (threadIdx.x < 256)
        half_zones<0>(a, nz, small_lo, (char *)smem4, half_bytes, red, redd, g, slot);
    else
        half_zones<1>(a, nz, small_lo, (char *)smem4 + half_bytes, half_bytes, red + 24, redd + 8,
                      g, slot + 1);
}

// The zones of more than k_lo stencils, one CTA each; or, when the zones
// of at least mid_lo stencils come to this launch (zones_at_least), the
// zone of rank blockIdx.x among those.  leave_big: zones that do not
// fit smem_bytes are left to the cluster solver (k_cg_zone_cl) instead of
// the global-memory path.
template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1) k_cg_zone(const int *d_nz, ZoneArgs a, int k_lo,
                                                        int mid_lo, ZoneScratch g, int smem_bytes,
                                                        int leave_big) {
    HFCR_PDL_WAIT();
    extern __shared__ float4 smem4[];
    __shared__ float red[96];
    __shared__ double redd[THREADS / 32];
    const int nz = *d_nz;
    // the loop's first zone, its stride, and the zones' smallest size minus one
    __shared__ int sel[3];
    {
        int pick, n_big;
        const int n_mid = zones_at_least(a.zs, nz, mid_lo, blockIdx.x, &pick, &n_big);
        const bool ranked = n_big > 0 && n_mid <= ROUTE_MAX && n_mid <= (int)gridDim.x;
        if (threadIdx.x == 0) {
            sel[0] = ranked ? (pick >= 0 ? pick : nz) : (int)blockIdx.x;
            sel[1] = ranked ? nz : (int)gridDim.x;
            sel[2] = ranked ? mid_lo - 1 : k_lo;
        }
        __syncthreads();
    }
    for (int z = sel[0]; z < nz; z += sel[1]) {
        const int k = a.zs[z + 1] - a.zs[z];
        if (k <= sel[2]) continue;
        if (leave_big && zone_smem_need(k, a.zv[z + 1] - a.zv[z], a.zg[z + 1] - a.zg[z]) > smem_bytes)
            continue;
        solve_zone<CtaGroup, true>(a, z, (char *)smem4, smem_bytes, red, redd, g);
        if (threadIdx.x == 0) {  // rows and touched vertices of the zones of this launch
            atomicAdd(&a.ctl[5], k);
            atomicAdd(&a.ctl[6], a.zv[z + 1] - a.zv[z]);
        }
    }
}

// ---------------------------------------------------------------------------
// The plain float64 form's per-zone solve: the same impact zones,
// zone-ordered rows, vertex CSR and block-Jacobi groups as the mixed
// solver, each zone solved by one 256-thread CTA with preconditioned CG in
// the Chronopoulos-Gear form, in float64 on the float64 normals, on global
// (L2-resident) arrays, to |r_zone| <= rel_tol |b_zone| (no refinement: the
// arithmetic is already float64).
// ---------------------------------------------------------------------------

struct Zone64Scratch {
    double *r, *p, *s, *w, *z;  // [cap_k] each, zone-ordered rows
};

constexpr int ZONE64_THREADS = 256;

// three block sums with one barrier, identical in every thread (the
// float64 counterpart of block_sum3)
__device__ __forceinline__ void block_sum3d(double a, double b, double c, double *red, double &sa,
                                            double &sb_, double &sc) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();  // red is free of its previous use
    if (lane == 0) {
        red[3 * w] = a;
        red[3 * w + 1] = b;
        red[3 * w + 2] = c;
    }
    __syncthreads();
    const int nw = blockDim.x >> 5;
    double x = lane < nw ? red[3 * lane] : 0.0;
    double y = lane < nw ? red[3 * lane + 1] : 0.0;
    double q = lane < nw ? red[3 * lane + 2] : 0.0;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
        q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    sa = __shfl_sync(0xffffffffu, x, 0);
    sb_ = __shfl_sync(0xffffffffu, y, 0);
    sc = __shfl_sync(0xffffffffu, q, 0);
}

// out = J M^-1 J^T in over the zone's rows (u: the zone's touched
// vertices, 3 doubles each); returns nothing, the caller synchronises
__device__ __forceinline__ void zone64_vertex(const ZoneArgs &a, int s0, int j0, int U,
                                              const double *in, double *u) {
    const double third = 1.0 / 3.0;
    for (int j = threadIdx.x; j < U; j += blockDim.x) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int e = a.seg[j0 + j]; e < a.seg[j0 + j + 1]; ++e) {
            const int c = a.cval[e] - 4 * s0;
            const int sl = c >> 2;
            const double ps = ((c & 3) ? -third : 1.0) * in[sl];
            const double4_32a n = a.n64[s0 + sl];
            a0 += ps * n.x;
            a1 += ps * n.y;
            a2 += ps * n.z;
        }
        const double wv = (double)a.winv[j0 + j];
        u[3 * j] = wv * a0;
        u[3 * j + 1] = wv * a1;
        u[3 * j + 2] = wv * a2;
    }
}

__device__ __forceinline__ double zone64_stencil(const ZoneArgs &a, int s0, int j0, int t,
                                                 const double *u) {
    const double third = 1.0 / 3.0;
    const int4 g = a.vidx[s0 + t];
    const double *ux = u + 3 * (g.x - j0), *ua = u + 3 * (g.y - j0), *ub = u + 3 * (g.z - j0),
                 *uc = u + 3 * (g.w - j0);
    const double4_32a n = a.n64[s0 + t];
    return n.x * (ux[0] - (ua[0] + ub[0] + uc[0]) * third) +
           n.y * (ux[1] - (ua[1] + ub[1] + uc[1]) * third) +
           n.z * (ux[2] - (ua[2] + ub[2] + uc[2]) * third);
}

// z = P^-1 r over the zone's groups (the float64 inverse blocks)
__device__ __forceinline__ void zone64_precond(const ZoneArgs &a, int s0, int g0, int G,
                                               const double *r, double *zz) {
    for (int gi = threadIdx.x; gi < G; gi += blockDim.x) {
        const int lo = a.gst[g0 + gi] - s0, hi = a.gst[g0 + gi + 1] - s0;
        double rr[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) rr[q] = lo + q < hi ? r[lo + q] : 0.0;
        for (int t = lo; t < hi; ++t) {
            const double4_32a m = a.pinv64[s0 + t];
            zz[t] = m.x * rr[0] + m.y * rr[1] + m.z * rr[2] + m.w * rr[3];
        }
    }
}

// rescue: only the zones whose recorded |r|^2 (the mixed solver's) misses
// the target, solved again from lam = 0 (zones on which the float32 runs
// stopped reducing the float64 residual)
__global__ void __launch_bounds__(ZONE64_THREADS) k_cg_zone64(const int *d_nz, ZoneArgs a,
                                                              Zone64Scratch g, int maxit, int rescue) {
    HFCR_PDL_WAIT();
    __shared__ double red[3 * (ZONE64_THREADS / 32)];
    __shared__ double redd[ZONE64_THREADS / 32];
    const int nz = *d_nz;
    for (int z = blockIdx.x; z < nz; z += gridDim.x) {
        if (rescue && a.zres[z] <= a.rel_tol * a.rel_tol * a.zbb[z]) continue;
        const int s0 = a.zs[z], k = a.zs[z + 1] - s0;
        const int j0 = a.zv[z], U = a.zv[z + 1] - j0;
        const int g0 = a.zg[z], G = a.zg[z + 1] - g0;
        const double bb = zone_start<CtaGroup>(a, s0, k, redd);  // lam = 0 on the zone's rows
        // the zone's block-Jacobi inverses in float64 (a block of nearly
        // dependent rows has a large inverse that float32 would not hold)
        for (int gi = threadIdx.x; gi < G; gi += blockDim.x)
            group_inverse_one<PlainLd>(g0 + gi, a.gst, a.ids, a.n64, a.nA, a.wA, a.wB, a.pinv64);
        double *r = g.r + s0, *p = g.p + s0, *sv = g.s + s0, *w = g.w + s0, *zz = g.z + s0;
        double *x = a.lam + s0, *u = a.u64 + 3 * (size_t)j0;
        for (int t = threadIdx.x; t < k; t += blockDim.x) {
            r[t] = a.b64[s0 + t];
            p[t] = 0.0;
            sv[t] = 0.0;
        }
        __syncthreads();
        zone64_precond(a, s0, g0, G, r, zz);
        __syncthreads();
        zone64_vertex(a, s0, j0, U, zz, u);
        __syncthreads();
        double ga = 0.0, de = 0.0, rh = 0.0;
        for (int t = threadIdx.x; t < k; t += blockDim.x) {
            const double wt = zone64_stencil(a, s0, j0, t, u);
            w[t] = wt;
            ga += r[t] * zz[t];
            de += wt * zz[t];
            rh += r[t] * r[t];
        }
        double gamma, delta, rho;
        block_sum3d(ga, de, rh, red, gamma, delta, rho);
        const double stop = a.rel_tol * a.rel_tol * bb;
        double alpha = gamma / delta, beta = 0.0;
        int it = 0;
        while (it < maxit && rho > stop && alpha > 0.0 && isfinite(alpha)) {
            for (int t = threadIdx.x; t < k; t += blockDim.x) {
                const double pt = zz[t] + beta * p[t];
                const double st = w[t] + beta * sv[t];
                p[t] = pt;
                sv[t] = st;
                x[t] += alpha * pt;
                r[t] -= alpha * st;
            }
            __syncthreads();
            zone64_precond(a, s0, g0, G, r, zz);
            __syncthreads();
            zone64_vertex(a, s0, j0, U, zz, u);
            __syncthreads();
            ga = de = rh = 0.0;
            for (int t = threadIdx.x; t < k; t += blockDim.x) {
                const double wt = zone64_stencil(a, s0, j0, t, u);
                w[t] = wt;
                ga += r[t] * zz[t];
                de += wt * zz[t];
                rh += r[t] * r[t];
            }
            double gn, dn, rn;
            block_sum3d(ga, de, rh, red, gn, dn, rn);
            beta = gn / gamma;
            alpha = gn / (dn - beta * gn / alpha);
            gamma = gn;
            rho = rn;
            ++it;
        }
        // the zone's true residual b - A lam (not the recurrence's)
        __syncthreads();
        zone64_vertex(a, s0, j0, U, x, u);
        __syncthreads();
        double rr = 0.0;
        for (int t = threadIdx.x; t < k; t += blockDim.x) {
            const double rt = a.b64[s0 + t] - zone64_stencil(a, s0, j0, t, u);
            rr += rt * rt;
        }
        rr = block_sum_uniform(rr, redd);
        if (threadIdx.x == 0) {
            a.zres[z] = rr;
            a.zbb[z] = bb;
            atomicAdd(&a.ctl[1], it);
            atomicAdd(&a.ctl[2], 1);
            atomicMax(&a.ctl[3], 1);
            atomicOr(&a.ctl[4], 4);
        }
        __syncthreads();  // u and the scalars' shared words are reused by the next zone
    }
}

// ---------------------------------------------------------------------------
// Large impact zones on a thread-block cluster: the zone's rows and touched
// vertices are split over the CL CTAs of a cluster (CL SMs), each CTA
// stages its share in its own shared memory, and the products that cross
// shares read the other CTAs' shared memory directly (distributed shared
// memory) between hardware cluster barriers.  The arithmetic is that of the
// one-CTA staged solve (float32 Chronopoulos-Gear PCG on the float32
// normals, block-Jacobi groups, float64 residual rounds, the same stopping
// rules); zones too large for one SM's shared memory (which would
// otherwise iterate on global memory) stay in shared memory, up to CL times
// larger.  (Measured: a zone that fits one SM iterates no faster on a
// cluster: an iteration is a chain of barriers and dependent loads either
// way, so such zones stay on one CTA.)  Rows are split at group boundaries, so
// the preconditioner stays local to a CTA.  Every CTA uses one layout,
// sized for the largest share of the zone, so another CTA's array is this
// CTA's array mapped to that rank.  Reductions: each CTA writes its
// partial sums into every CTA's slot for it, and after the barrier each
// CTA adds the CL slots in rank order (identical sums everywhere).
// ---------------------------------------------------------------------------

constexpr int CL = 8;               // CTAs per cluster (portable cluster size)
constexpr int CL_THREADS = 512;
constexpr int CL_SMEM = 200 * 1024; // dynamic shared memory per CTA
constexpr int ZONE_CL_MIN = ZONE_BIG;  // zones of at least this many rows

namespace cgx = cooperative_groups;

struct ClLayout {
    int Kc, Uc, Ec, Gc;       // capacities: rows, vertices, CSR entries, groups per CTA
    int o_n4, o_pinv, o_vidx, o_u, o_f, o_winv, o_seg, o_ent, o_gst;
    int bytes;
};

__device__ __forceinline__ ClLayout cl_layout(int Kc, int Uc, int Ec, int Gc) {
    ClLayout L;
    L.Kc = Kc; L.Uc = Uc; L.Ec = Ec; L.Gc = Gc;
    int o = 0;
    L.o_n4 = o;   o += 16 * Kc;
    L.o_pinv = o; o += 16 * Kc;
    L.o_vidx = o; o += 16 * Kc;
    L.o_u = o;    o += 16 * Uc;
    L.o_f = o;    o += 4 * 6 * Kc;          // r p x sv w z
    L.o_winv = o; o += 4 * Uc;
    L.o_seg = o;  o += 4 * (Uc + 1);
    L.o_ent = o;  o += 4 * Ec;
    L.o_gst = o;  o += 4 * (Gc + 1);
    L.bytes = o;
    return L;
}

// the partial sums of this CTA (nv values, the same in every thread) into
// slot `rank` of every CTA's red, then after the barrier the sums over the
// CL slots in rank order
template <typename T, int NV>
__device__ __forceinline__ void cl_reduce(cgx::cluster_group &cl, const T *part, T *red, T *out) {
    if (threadIdx.x < CL * NV) {
        const int dst = threadIdx.x / NV, v = threadIdx.x % NV;
        T *r = cl.map_shared_rank(red, dst);
        r[cl.block_rank() * NV + v] = part[v];
    }
    cl.sync();
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        T t = 0;
        for (int c = 0; c < CL; ++c) t += red[c * NV + v];
        out[v] = t;
    }
}

// CTA-wide float sums of three values (identical in every thread)
__device__ __forceinline__ void cl_block3(float a, float b, float c, float *red, float *out) {
    float sa, sb, sc;
    block_sum3(a, b, c, red, sa, sb, sc);
    __syncthreads();  // red is rewritten by the next call
    out[0] = sa; out[1] = sb; out[2] = sc;
}

// one_cta_smem: the shared memory of the one-CTA solver (k_cg_zone): the
// zones that fit it are its, this kernel takes the larger ones
__global__ void __launch_bounds__(CL_THREADS, 1) k_cg_zone_cl(const int *d_nz, ZoneArgs a,
                                                              ZoneScratch gs, int one_cta_smem) {
    HFCR_PDL_WAIT();
    cgx::cluster_group cl = cgx::this_cluster();
    extern __shared__ float4 smem4[];
    char *base = (char *)smem4;
    __shared__ float redf[CL * 3];          // cluster partials (float)
    __shared__ double redd[CL * 2];         // cluster partials (double)
    __shared__ float bred[96];              // block reductions
    __shared__ double bredd[CL_THREADS / 32];
    __shared__ int rb[CL + 1], gb[CL + 1], vb[CL + 1], eb[CL + 1];
    const int rank = cl.block_rank();
    const int tid = threadIdx.x, nt = CL_THREADS;
    const int nz = *d_nz;
    const int ncl = gridDim.x / CL;
    const int ci = blockIdx.x / CL;
    for (int z = ci; z < nz; z += ncl) {
        const int s0 = a.zs[z], k = a.zs[z + 1] - s0;
        if (k < ZONE_CL_MIN) continue;
        const int j0 = a.zv[z], U = a.zv[z + 1] - j0;
        const int g0 = a.zg[z], G = a.zg[z + 1] - g0;
        if (zone_smem_need(k, U, G) <= one_cta_smem) continue;   // the one-CTA solver's
        const int e0 = a.seg[j0];
        // shares: rows split at group boundaries (CL nearly equal group
        // counts), vertex j in CTA j / Ucap; every CTA computes all
        // boundaries, so every CTA derives the same layout
        const int Ucap = (U + CL - 1) / CL;
        if (tid <= CL) {
            const int gc = (int)(((long long)G * tid) / CL);
            gb[tid] = gc;
            rb[tid] = tid == CL ? k : a.gst[g0 + gc] - s0;
            const int vc = min(U, tid * Ucap);
            vb[tid] = vc;
            eb[tid] = a.seg[j0 + vc] - e0;
        }
        __syncthreads();
        int Kc = 0, Ec = 0, Gc = 0;
        for (int c = 0; c < CL; ++c) {
            Kc = max(Kc, rb[c + 1] - rb[c]);
            Ec = max(Ec, eb[c + 1] - eb[c]);
            Gc = max(Gc, gb[c + 1] - gb[c]);
        }
        const ClLayout L = cl_layout(Kc, Ucap, Ec, Gc);
        const double bb = [&] {
            double t = 0.0;
            for (int q = tid; q < k; q += nt) {
                const double bv = a.b64[s0 + q];
                t += bv * bv;
            }
            return block_sum_uniform(t, bredd);
        }();
        if (L.bytes > CL_SMEM) {
            // too large for the cluster's shared memory: the first CTA solves
            // it on global memory (the one-CTA path), the others go on
            if (rank == 0) solve_zone<CtaGroup>(a, z, base, 0, bred, bredd, gs);
            continue;
        }
        const int r0 = rb[rank], kr = rb[rank + 1] - r0;            // own rows
        const int v0 = vb[rank], ur = vb[rank + 1] - v0;            // own vertices
        const int gg0 = gb[rank], gr = gb[rank + 1] - gg0;          // own groups
        const int ee0 = eb[rank], er = eb[rank + 1] - ee0;          // own CSR entries
        float4 *n4 = (float4 *)(base + L.o_n4);
        float4 *pinv = (float4 *)(base + L.o_pinv);
        int4 *vidx = (int4 *)(base + L.o_vidx);
        float4 *u = (float4 *)(base + L.o_u);
        float *f = (float *)(base + L.o_f);
        float *r = f, *p = f + Kc, *x = f + 2 * Kc, *sv = f + 3 * Kc, *w = f + 4 * Kc, *zz = f + 5 * Kc;
        float *winv = (float *)(base + L.o_winv);
        int *seg = (int *)(base + L.o_seg);
        int *ent = (int *)(base + L.o_ent);
        int *gst = (int *)(base + L.o_gst);
        // stage the own share
        for (int t = tid; t < kr; t += nt) {
            const int4 g = a.vidx[s0 + r0 + t];
            vidx[t] = make_int4(g.x - j0, g.y - j0, g.z - j0, g.w - j0);
            n4[t] = a.n32[s0 + r0 + t];
            pinv[t] = a.pinv[s0 + r0 + t];
            a.lam[s0 + r0 + t] = 0.0;
        }
        for (int q = tid; q <= gr; q += nt) gst[q] = a.gst[g0 + gg0 + q] - s0 - r0;
        for (int j = tid; j <= ur; j += nt) seg[j] = a.seg[j0 + v0 + j] - e0 - ee0;
        for (int j = tid; j < ur; j += nt) winv[j] = a.winv[j0 + v0 + j];
        for (int e = tid; e < er; e += nt) ent[e] = a.cval[e0 + ee0 + e] - 4 * s0;
        // the CTA that owns row s (rows split at rb)
        auto row_owner = [&](int sl) {
            int c = 0;
#pragma unroll
            for (int q = 1; q < CL; ++q) c += sl >= rb[q];
            return c;
        };
        const double target = a.rel_tol * a.rel_tol * bb;
        const float third = 1.0f / 3.0f;
        double rr = bb;
        int its = 0, rounds = 0;
        // the first round's right-hand side: b (lam = 0)
        for (int t = tid; t < kr; t += nt) r[t] = (float)a.b64[s0 + r0 + t];
        cl.sync();
        while (rr > target && rounds < a.max_refine) {
            for (int t = tid; t < kr; t += nt) { p[t] = 0.f; sv[t] = 0.f; x[t] = 0.f; }
            // ---- float32 PCG (Chronopoulos-Gear) on the float32 normals ----
            auto precond = [&]() {
                for (int g = tid; g < gr; g += nt) {
                    const int lo = gst[g], hi = gst[g + 1];
                    float rq[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) rq[q] = lo + q < hi ? r[lo + q] : 0.f;
                    for (int t = lo; t < hi; ++t) {
                        const float4 m = pinv[t];
                        zz[t] = m.x * rq[0] + m.y * rq[1] + m.z * rq[2] + m.w * rq[3];
                    }
                }
            };
            auto matvec_vertex = [&]() {   // u = M^-1 J^T z over the own vertices
                for (int j = tid; j < ur; j += nt) {
                    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
                    for (int e = seg[j]; e < seg[j + 1]; ++e) {
                        const int c = ent[e];
                        const int sl = c >> 2;
                        const int ow = row_owner(sl);
                        const int li = sl - rb[ow];
                        const float zs = *cl.map_shared_rank(zz + li, ow);
                        const float4 nn = *cl.map_shared_rank(n4 + li, ow);
                        const float ps = ((c & 3) ? -third : 1.0f) * zs;
                        a0 += ps * nn.x;
                        a1 += ps * nn.y;
                        a2 += ps * nn.z;
                    }
                    const float wv = winv[j];
                    u[j] = make_float4(wv * a0, wv * a1, wv * a2, 0.f);
                }
            };
            auto matvec_rows = [&](float *ga, float *de, float *rh) {   // w = J u, partial sums
                for (int t = tid; t < kr; t += nt) {
                    const int4 g = vidx[t];
                    const float4 u0 = *cl.map_shared_rank(u + g.x % Ucap, g.x / Ucap);
                    const float4 u1 = *cl.map_shared_rank(u + g.y % Ucap, g.y / Ucap);
                    const float4 u2 = *cl.map_shared_rank(u + g.z % Ucap, g.z / Ucap);
                    const float4 u3 = *cl.map_shared_rank(u + g.w % Ucap, g.w / Ucap);
                    const float4 nn = n4[t];
                    const float ws = nn.x * (u0.x - (u1.x + u2.x + u3.x) * third) +
                                     nn.y * (u0.y - (u1.y + u2.y + u3.y) * third) +
                                     nn.z * (u0.z - (u1.z + u2.z + u3.z) * third);
                    w[t] = ws;
                    *ga += r[t] * zz[t];
                    *de += ws * zz[t];
                    *rh += r[t] * r[t];
                }
            };
            precond();
            cl.sync();
            matvec_vertex();
            cl.sync();
            float ga = 0.f, de = 0.f, rh = 0.f;
            matvec_rows(&ga, &de, &rh);
            float part[3], sums[3];
            cl_block3(ga, de, rh, bred, part);
            cl_reduce<float, 3>(cl, part, redf, sums);
            float gamma = sums[0], delta = sums[1], rho = sums[2];
            const float stop = (float)a.tol * (float)a.tol * rho;
            float alpha = gamma / delta, beta = 0.f;
            int it = 0;
            while (it < a.maxit && rho > stop && rho > 0.f && alpha > 0.f && isfinite(alpha)) {
                for (int g = tid; g < gr; g += nt) {
                    const int lo = gst[g], hi = gst[g + 1];
                    for (int t = lo; t < hi; ++t) {
                        const float ps = zz[t] + beta * p[t];
                        const float ss = w[t] + beta * sv[t];
                        p[t] = ps;
                        sv[t] = ss;
                        x[t] += alpha * ps;
                        r[t] -= alpha * ss;
                    }
                }
                __syncthreads();
                precond();
                cl.sync();
                matvec_vertex();
                cl.sync();
                ga = de = rh = 0.f;
                matvec_rows(&ga, &de, &rh);
                cl_block3(ga, de, rh, bred, part);
                cl_reduce<float, 3>(cl, part, redf, sums);
                beta = sums[0] / gamma;
                alpha = sums[0] / (sums[1] - beta * sums[0] / alpha);
                gamma = sums[0];
                rho = sums[2];
                ++it;
            }
            its += it;
            // ---- lam += x, then the zone's float64 residual b - A lam ----
            for (int t = tid; t < kr; t += nt) a.lam[s0 + r0 + t] += (double)x[t];
            __threadfence();
            cl.sync();
            const double third64 = 1.0 / 3.0;
            for (int j = tid; j < ur; j += nt) {
                double a0 = 0.0, a1 = 0.0, a2 = 0.0;
                for (int e = seg[j]; e < seg[j + 1]; ++e) {
                    const int c = ent[e];
                    const int sl = c >> 2;
                    const double ps = ((c & 3) ? -third64 : 1.0) * __ldcg(a.lam + s0 + sl);
                    const double4_32a nn = a.n64[s0 + sl];
                    a0 += ps * nn.x;
                    a1 += ps * nn.y;
                    a2 += ps * nn.z;
                }
                const double wv = (double)winv[j];
                double *uo = a.u64 + 3 * (size_t)(j0 + v0 + j);
                uo[0] = wv * a0;
                uo[1] = wv * a1;
                uo[2] = wv * a2;
            }
            __threadfence();
            cl.sync();
            double rrl = 0.0;
            for (int t = tid; t < kr; t += nt) {
                const int4 g = vidx[t];
                const double *ux = a.u64 + 3 * (size_t)(j0 + g.x), *ua = a.u64 + 3 * (size_t)(j0 + g.y);
                const double *ub = a.u64 + 3 * (size_t)(j0 + g.z), *uc = a.u64 + 3 * (size_t)(j0 + g.w);
                double d[3];
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    d[c] = __ldcg(ux + c) - (__ldcg(ua + c) + __ldcg(ub + c) + __ldcg(uc + c)) * third64;
                const double4_32a nn = a.n64[s0 + r0 + t];
                const double rv = a.b64[s0 + r0 + t] - (nn.x * d[0] + nn.y * d[1] + nn.z * d[2]);
                r[t] = (float)rv;
                rrl += rv * rv;
            }
            double pd[2] = {block_sum_uniform(rrl, bredd), 0.0}, sd[2];
            cl_reduce<double, 2>(cl, pd, redd, sd);
            rr = sd[0];
            ++rounds;
        }
        if (rank == 0 && tid == 0) {
            zone_finish(a, z, rr, bb, its, rounds, true);
            atomicAdd(&a.ctl[5], k);
            atomicAdd(&a.ctl[6], U);
        }
        // the shares (shared memory) of this zone are read by other CTAs until
        // every CTA has passed this barrier
        cl.sync();
    }
    cl.sync();
}

// |r| / |b| of the whole system from the zones' |r|^2 and |b|^2 (fixed
// summation order) to dres[0], |b|^2 to dres[1]; ctl[0] = converged
__global__ void __launch_bounds__(256) k_zone_final(const int *d_nz, const double *zres,
                                                    const double *zbb, double rel_tol,
                                                    double *dres, int *ctl) {
    HFCR_PDL_WAIT();
    __shared__ double redd[8];
    const int nz = *d_nz;
    double R = 0.0, Bn = 0.0;
    for (int z = threadIdx.x; z < nz; z += blockDim.x) {
        R += zres[z];
        Bn += zbb[z];
    }
    R = block_sum_uniform(R, redd);
    Bn = block_sum_uniform(Bn, redd);
    if (threadIdx.x == 0) {
        const double rel = Bn > 0.0 ? sqrt(R / Bn) : (R > 0.0 ? INFINITY : 0.0);
        dres[0] = rel;
        dres[1] = Bn;
        ctl[0] = rel <= rel_tol;
    }
}

// float64 residual, vertex half: u = M^-1 J^T lam
__global__ void k_res_vertex(const int *d_U, const int *seg, const int *cval, const float *winv,
                             const double4_32a *n64, const double *lam, double *u, const int *ctl) {
    HFCR_PDL_WAIT();
    if (ctl[0]) return;
    const int U = *d_U;
    const double third = 1.0 / 3.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < U; j += gridDim.x * blockDim.x) {
        double a0 = 0, a1 = 0, a2 = 0;
        for (int e = seg[j]; e < seg[j + 1]; ++e) {
            int v = cval[e];
            int s = v >> 2;
            double ps = ((v & 3) ? -third : 1.0) * lam[s];
            double4_32a n = n64[s];
            a0 += ps * n.x;
            a1 += ps * n.y;
            a2 += ps * n.z;
        }
        double w = (double)winv[j];
        u[3 * j] = w * a0;
        u[3 * j + 1] = w * a1;
        u[3 * j + 2] = w * a2;
    }
}

// float64 residual, stencil half: r = b - J u; per-block partial sums of
// r^2 and b^2 to red[blk] and red[RES_BLOCKS + blk].  The last block to
// finish (ticket counter) adds the partials in block order, records
// |r| / |b| in dres[0] and |b|^2 in dres[1], and sets ctl[0] when the
// relative residual meets rel_tol.
__global__ void k_res_stencil(const int *d_k, const int4 *vidx, const double4_32a *n64,
                              const double *b, const double *u, double *r, double *red,
                              int *ctl, unsigned *ticket, double rel_tol, double *dres,
                              int count_round) {
    HFCR_PDL_WAIT();
    __shared__ double sh[33];
    __shared__ bool last;
    if (ctl[0]) return;
    const int k = *d_k;
    const double third = 1.0 / 3.0;
    double rr = 0, bb = 0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < k; s += gridDim.x * blockDim.x) {
        int4 vi = vidx[s];
        double4_32a n = n64[s];
        double d0 = u[3 * vi.x] - (u[3 * vi.y] + u[3 * vi.z] + u[3 * vi.w]) * third;
        double d1 = u[3 * vi.x + 1] - (u[3 * vi.y + 1] + u[3 * vi.z + 1] + u[3 * vi.w + 1]) * third;
        double d2 = u[3 * vi.x + 2] - (u[3 * vi.y + 2] + u[3 * vi.z + 2] + u[3 * vi.w + 2]) * third;
        double rs = b[s] - (n.x * d0 + n.y * d1 + n.z * d2);
        r[s] = rs;
        rr += rs * rs;
        bb += b[s] * b[s];
    }
    rr = block_sum(rr, sh);
    bb = block_sum(bb, sh);
    if (threadIdx.x == 0) {
        red[blockIdx.x] = rr;
        red[RES_BLOCKS + blockIdx.x] = bb;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double R = 0, Bn = 0;
    for (int i = 0; i < (int)gridDim.x; ++i) {
        R += __ldcg(red + i);
        Bn += __ldcg(red + RES_BLOCKS + i);
    }
    double rel = Bn > 0 ? sqrt(R / Bn) : 0.0;
    dres[0] = rel;
    dres[1] = Bn;
    if (rel <= rel_tol) ctl[0] = 1;
    if (count_round) ctl[3] += 1;
    *ticket = 0;
}

__global__ void k_init_lam(const int *d_k, const double *b, double *lam, double *r) {
    HFCR_PDL_WAIT();
    const int k = *d_k;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < k; s += gridDim.x * blockDim.x) {
        lam[s] = 0.0;
        r[s] = b[s];
    }
}

// displacement of the touched vertices: dx = -M^-1 J^T lam (float64).
// apply 1: added to the positions; 0: written to the caller's arrays (mesh
// dtype); 2: written to the float64 field dA0 (x, y, z per global vertex)
__global__ void k_displace(const int *d_U, const int *seg, const int *cval, const float *winv,
                           const double4_32a *n64, const double *lam, const int *gvert, hfcr_mesh A,
                           hfcr_mesh B, int apply, void *dA0, void *dA1, void *dA2, void *dB0,
                           void *dB1, void *dB2, unsigned long long *max_dx) {
    HFCR_PDL_WAIT();
    const int U = *d_U;
    const double third = 1.0 / 3.0;
    double biggest = 0.0;  // the largest displacement component of this thread's vertices
    const int j_end = (U + (int)(gridDim.x * blockDim.x) - 1) / (int)(gridDim.x * blockDim.x) *
                      (int)(gridDim.x * blockDim.x);  // every thread of a warp runs the same trips
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < j_end; j += gridDim.x * blockDim.x) {
        if (j >= U) continue;
        double a0 = 0, a1 = 0, a2 = 0;
        for (int e = seg[j]; e < seg[j + 1]; ++e) {
            int v = cval[e];
            int s = v >> 2;
            double ps = ((v & 3) ? -third : 1.0) * lam[s];
            double4_32a n = n64[s];
            a0 += ps * n.x;
            a1 += ps * n.y;
            a2 += ps * n.z;
        }
        double w = (double)winv[j];
        double dx[3] = {-w * a0, -w * a1, -w * a2};
        biggest = fmax(biggest, fmax(fabs(dx[0]), fmax(fabs(dx[1]), fabs(dx[2]))));
        int g = gvert[j];
        if (apply == 2) {  // into the float64 field of the diffusion (AoS, global ids)
            double *f = (double *)dA0 + 3 * (size_t)g;
            f[0] = dx[0];
            f[1] = dx[1];
            f[2] = dx[2];
            continue;
        }
        const bool inA = g < A.n_verts;
        const hfcr_mesh &m = inA ? A : B;
        int lv = inA ? g : g - A.n_verts;
        if (apply) {
            void *P[3] = {m.x, m.y, m.z};
            for (int c = 0; c < 3; ++c) {
                if (m.dtype == HFCR_F32) {
                    float *pp = (float *)P[c] + lv;
                    *pp = (float)((double)*pp + dx[c]);
                } else {
                    double *pp = (double *)P[c] + lv;
                    *pp = *pp + dx[c];
                }
            }
        } else {
            void *O[3] = {inA ? dA0 : dB0, inA ? dA1 : dB1, inA ? dA2 : dB2};
            for (int c = 0; c < 3; ++c) {
                if (m.dtype == HFCR_F32) ((float *)O[c])[lv] = (float)dx[c];
                else ((double *)O[c])[lv] = dx[c];
            }
        }
    }
    warp_max_to(biggest, max_dx);
}

// ---------------------------------------------------------------------------
// The response setup in one cooperative launch: vertex CSR of the stencil
// entries, impact zones, zone-ordered rows, zone-ordered CSR, the groups of
// rows sharing x0 and the inverses of their blocks.  It computes exactly
// what the multi-kernel sequence of build_vertex_csr computes (the same
// stable sorts, the same union-find roots, hence the same arrays), in one
// launch instead of about twenty-five.  The elementwise phases run on every
// CTA taking part, separated by bounded grid-wide barriers, and data
// written by another CTA is read through L2.  Up to SETUP_SMALL_K stencils
// few CTAs take part (one per 1,024 entries) and the first CTA alone runs
// the sorts, the union-find (in shared memory) and the scans between two
// barriers; above, every CTA takes part in those too (the multi-CTA sort,
// union-find in global memory, the two-level scan).
// ---------------------------------------------------------------------------
constexpr int SETUP_SMALL_K = 8192;  // 4k <= SMALL_N sort keys, 32 KB of parents
constexpr int SETUP_SCAN_CHUNK = 4096;
constexpr int SETUP_ENTRIES_PER_CTA = 1024;

struct SetupArgs {
    const int *d_k;
    int cap, vbits, nA;
    const float *wA, *wB;
    const int4 *ids_raw;
    const double4_32a *n64_raw;
    const float4 *n32_raw;
    const double *b_raw;
    unsigned *ckey, *ckey_alt, *cflag;
    int *cval, *cval_alt;
    unsigned *zlab, *zlab_alt;
    int *zsrc, *zsrc_alt;
    unsigned *k2, *k2_alt;
    int *v2, *v2_alt;
    int *parent;  // union-find forest above SETUP_SMALL_K, then the position of each stencil
    int4 *ids;
    double4_32a *n64;
    float4 *n32;
    double *b;
    int *szone, *zs, *zv, *gst, *zg, *seg, *gvert;
    int4 *vidx;
    float *winv;
    float4 *pinv;
    int *d_n4, *d_U, *d_nz, *d_ng;
    unsigned *hist, *tot, *bar;
    uint32_t *status;
};

// the CTAs taking part (blockIdx.x < parts) and their barrier
struct SetupSync {
    unsigned *bar;
    unsigned epoch;
    uint32_t *status;
    unsigned parts;
    __device__ bool sync() {
        if (parts == 1) {
            __syncthreads();
            return true;
        }
        return grid_barrier(bar, ++epoch, status, parts);
    }
};

__device__ __forceinline__ unsigned cta_sum_u(unsigned v) {
    __shared__ unsigned ws[TPB / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();  // ws is free of its previous use
    if (lane == 0) ws[w] = v;
    __syncthreads();
    unsigned t = 0;
#pragma unroll
    for (int q = 0; q < TPB / 32; ++q) t += ws[q];
    return t;
}

// exclusive scan of a[0..m) in place, the sum to *d_total; on return the
// scanned values and the sum are visible to every CTA taking part.  Small:
// the first CTA scans alone.  Otherwise chunks of SETUP_SCAN_CHUNK: chunk
// sums, a barrier, each chunk scanned from the sum of the chunks before it.
__device__ __forceinline__ bool setup_scan(SetupSync &g, bool small, unsigned *a, int m,
                                           unsigned *part, int *d_total, unsigned &total) {
    if (small) {
        if (blockIdx.x == 0) {
            const unsigned t = block_scan_excl<TPB, true>(a, m);
            if (threadIdx.x == 0) *d_total = (int)t;
        }
        if (!g.sync()) return false;
        total = (unsigned)__ldcg(d_total);
        return true;
    }
    const int nc = (m + SETUP_SCAN_CHUNK - 1) / SETUP_SCAN_CHUNK;
    for (int c = blockIdx.x; c < nc; c += g.parts) {
        const int base = c * SETUP_SCAN_CHUNK, end = min(m, base + SETUP_SCAN_CHUNK);
        unsigned x = 0;
        for (int i = base + threadIdx.x; i < end; i += TPB) x += __ldcg(a + i);
        x = cta_sum_u(x);
        if (threadIdx.x == 0) part[c] = x;
    }
    if (!g.sync()) return false;
    for (int c = blockIdx.x; c < nc; c += g.parts) {
        unsigned x = 0;
        for (int i = threadIdx.x; i < c; i += TPB) x += __ldcg(part + i);
        const unsigned off = cta_sum_u(x);
        const int base = c * SETUP_SCAN_CHUNK;
        block_scan_excl<TPB, true>(a + base, min(m - base, SETUP_SCAN_CHUNK), off);
    }
    unsigned x = 0;
    for (int i = threadIdx.x; i < nc; i += TPB) x += __ldcg(part + i);
    total = cta_sum_u(x);
    if (blockIdx.x == 0 && threadIdx.x == 0) *d_total = (int)total;
    return g.sync();
}

// stable sort of (key, val) pairs over `bits` bits (a multiple of 8); the
// result is in (k1, v1) after an odd number of passes.  One CTA taking
// part: the single-CTA sort; otherwise every CTA taking part (at most one
// tile each on small inputs: no scan phase).
__device__ __forceinline__ bool setup_sort(SetupSync &g, bool small, unsigned *k0, int *v0,
                                           unsigned *k1, int *v1, int n, int bits,
                                           const SetupArgs &a, SortSmem &sm) {
    if (small && g.parts == 1) {
        sort_small_body<unsigned, true, true>(k0, v0, k1, v1, n, bits, sm);
        return g.sync();
    }
    return sort_grid_body<unsigned, true>(k0, v0, k1, v1, n, bits, a.hist, a.tot, g.bar, g.epoch,
                                          g.status, sm, g.parts);
}

__device__ __forceinline__ int setup_bits(int n) {  // 8 x the passes for keys < n (n >= 1)
    int b = 1;
    while ((1 << b) < n) ++b;
    return 8 * ((b + 7) / 8);
}

__device__ __forceinline__ bool group_start_l2(const int4 *ids, const int *szone, const int *zs,
                                               int t) {
    const int zs0 = __ldcg(zs + __ldcg(szone + t)), x0 = __ldcg(&ids[t].x);
    int rs = t;
    while (rs > zs0 && __ldcg(&ids[rs - 1].x) == x0) --rs;
    return ((t - rs) % GMAX) == 0;
}

// unites the zones of stencils s0 and s1 (the smaller root becomes the
// root); SH: parents in shared memory
template <bool SH>
__device__ __forceinline__ void setup_unite(int *par, int s0, int s1, uint32_t *status) {
    int a = s0, b = s1, guard = 0;
    while (true) {
        if constexpr (SH) {
            a = uf_find_s(par, a);
            b = uf_find_s(par, b);
        } else {
            a = uf_find(par, a);
            b = uf_find(par, b);
        }
        if (a == b) break;
        if (a < b) { int t = a; a = b; b = t; }
        const int old = atomicCAS(par + a, a, b);
        if (old == a) break;
        a = old;
        if (++guard > (1 << 24)) { atomicOr(status, ST_TIMEOUT); break; }
    }
}

// Impact zones of up to SETUP_SMALL_K stencils by one CTA, in shared
// memory: connected components of the stencils, two stencils being
// adjacent when consecutive entries of the vertex-sorted list (ck1, cv1)
// share a vertex.  Min-label hooking with shortcutting (the FastSV scheme of
// Zhang, Azad and Hu, 2020): every sweep hooks the parent of each end of an
// edge, and each end itself, under the smaller of their grandparents
// (atomicMin), then every stencil jumps to its grandparent; labels only
// fall and stay inside their component, so at the first sweep that changes
// nothing every stencil points straight at the smallest stencil of its
// zone (the root the lock-free union-find gives too).  After SV_SWEEPS
// sweeps without convergence the forest (every parent smaller than its
// child, inside the same zone) is finished by the union-find.
constexpr int SV_SWEEPS = 64;

// edge[i] (i < n4): the stencils (u << 16 | v) of entries i and i - 1 of the
// vertex-sorted list when they share a vertex, NO_EDGE otherwise
constexpr unsigned NO_EDGE = 0xffffffffu;

__device__ void zones_min_label(int *f, int k, const unsigned *edge, int n4, uint32_t *status) {
    __shared__ int changed;
    for (int s = threadIdx.x; s < k; s += TPB) f[s] = s;
    if (threadIdx.x == 0) changed = 0;
    __syncthreads();
    int again = 1;
    for (int sweep = 0; sweep < SV_SWEEPS; ++sweep) {
        bool ch = false;
        for (int i = threadIdx.x + 1; i < n4; i += TPB) {
            const unsigned e = edge[i];
            if (e == NO_EDGE) continue;
            const int u = (int)(e >> 16), v = (int)(e & 0xffffu);
            const int fu = f[u], fv = f[v];
            const int m = min(f[fu], f[fv]);
            ch |= atomicMin(f + fu, m) > m;
            ch |= atomicMin(f + fv, m) > m;
            ch |= atomicMin(f + u, m) > m;
            ch |= atomicMin(f + v, m) > m;
        }
        __syncthreads();
        for (int s = threadIdx.x; s < k; s += TPB) {
            const int gp = f[f[s]];
            ch |= atomicMin(f + s, gp) > gp;
        }
        if (ch) changed = 1;
        __syncthreads();
        again = changed;
        __syncthreads();
        if (!again) break;
        if (threadIdx.x == 0) changed = 0;  // written again only after the next sweep's barrier
    }
    if (again) {
        for (int i = threadIdx.x + 1; i < n4; i += TPB) {
            const unsigned e = edge[i];
            if (e != NO_EDGE) setup_unite<true>(f, (int)(e >> 16), (int)(e & 0xffffu), status);
        }
        __syncthreads();
    }
}

// word of the barrier row raised when the groups are built (zeroed with
// the barrier counter before the launch)
constexpr int SETUP_READY = 1;

// the inverse blocks of CTAs first .. first + n - 1 (consecutive groups on
// different CTAs)
__device__ __forceinline__ void setup_inverses(const SetupArgs &a, int first, int n) {
    const int ng = __ldcg(a.d_ng);
    for (int gi = threadIdx.x * n + (blockIdx.x - first); gi < ng; gi += n * TPB)
        group_inverse_one<L2Ld>(gi, a.gst, a.ids, a.n64, a.nA, a.wA, a.wB, a.pinv);
}

// a CTA not taking part in the phases (first = the first such CTA): waits
// (bounded, like the barrier) for the groups, then computes its share of
// the inverse blocks
__device__ void setup_helper(const SetupArgs &a, int first) {
    __shared__ int go;
    if (threadIdx.x == 0) {
        go = 0;
        long long spins = 0;
        while (true) {
            unsigned seen;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(seen)
                         : "l"(a.bar + SETUP_READY) : "memory");
            if (seen) { go = 1; break; }
            if (*(volatile uint32_t *)a.status & ST_TIMEOUT) break;
            if (++spins > BARRIER_SPIN_LIMIT) {
                atomicOr(a.status, ST_TIMEOUT);
                break;
            }
            __nanosleep(100);
        }
    }
    __syncthreads();
    if (go) setup_inverses(a, first, (int)gridDim.x - first);
}

__device__ bool setup_phases(SetupSync &g, const SetupArgs &a, int k, SortSmem &sm, int *par_s) {
    const bool small = k <= SETUP_SMALL_K;
    const int tid = blockIdx.x * TPB + threadIdx.x, nt = (int)g.parts * TPB, n4 = 4 * k;
    if (tid == 0) *a.d_n4 = n4;
    if (k == 0) {
        if (tid == 0) { *a.d_U = 0; *a.d_nz = 0; *a.d_ng = 0; }
        return true;
    }
    // vertex CSR: entries (vertex, 4 s + role) sorted by vertex
    for (int i = tid; i < n4; i += nt) {
        a.ckey[i] = (unsigned)((const int *)a.ids_raw)[i];
        a.cval[i] = i;
    }
    if (!g.sync()) return false;
    const bool f1 = (a.vbits / 8) & 1;
    const unsigned *ck1 = f1 ? a.ckey_alt : a.ckey;
    const int *cv1 = f1 ? a.cval_alt : a.cval;
    // impact zones: stencils of consecutive entries on the same vertex are
    // united; every zone's root is its smallest stencil.  Then the rows
    // regrouped zone by zone (zones in the order of their root).
    const int zbits = setup_bits(k);
    const bool f2 = (zbits / 8) & 1;
    const unsigned *zl = f2 ? a.zlab_alt : a.zlab;
    const int *zr = f2 ? a.zsrc_alt : a.zsrc;
    if (small) {
        // the entries sorted by every CTA taking part (one CTA: by itself),
        // then the zones, the labels and their sort in the first CTA
        if (g.parts > 1 &&
            !sort_grid_body<unsigned, true>(a.ckey, a.cval, a.ckey_alt, a.cval_alt, n4, a.vbits,
                                            a.hist, a.tot, g.bar, g.epoch, g.status, sm, g.parts))
            return false;
        if (blockIdx.x == 0) {
            if (g.parts == 1)
                sort_small_body<unsigned, true, true>(a.ckey, a.cval, a.ckey_alt, a.cval_alt, n4,
                                                      a.vbits, sm);
            int *par = par_s;  // overlays the sort's shared memory (the sort is done)
            // the adjacent pairs of sorted entries, read once through L2
            // (other CTAs wrote them; eight entries' loads in flight per
            // thread) and packed into cflag (free here)
            for (int i0 = 0; i0 < n4; i0 += 8 * TPB) {
                unsigned kc[8], kb[8];
                int vc[8], vb[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int i = i0 + q * TPB + threadIdx.x;
                    const bool ok = i > 0 && i < n4;
                    kc[q] = ok ? __ldcg(ck1 + i) : 0u;
                    kb[q] = ok ? __ldcg(ck1 + i - 1) : 1u;
                    vc[q] = ok ? __ldcg(cv1 + i) : 0;
                    vb[q] = ok ? __ldcg(cv1 + i - 1) : 0;
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int i = i0 + q * TPB + threadIdx.x;
                    if (i < n4)
                        a.cflag[i] = kc[q] == kb[q]
                                         ? (unsigned)(vc[q] >> 2) << 16 | (unsigned)(vb[q] >> 2)
                                         : NO_EDGE;
                }
            }
            __syncthreads();
            zones_min_label(par, k, a.cflag, n4, a.status);
            for (int s = threadIdx.x; s < k; s += TPB) {
                a.zlab[s] = (unsigned)uf_find_s(par, s);
                a.zsrc[s] = s;
            }
            __syncthreads();
            sort_small_body<unsigned, true>(a.zlab, a.zsrc, a.zlab_alt, a.zsrc_alt, k, zbits, sm);
            for (int t = threadIdx.x; t < k; t += TPB)
                a.cflag[t] = (t == 0 || zl[t] != zl[t - 1]) ? 1u : 0u;
            __syncthreads();
        }
    } else {
        if (!setup_sort(g, false, a.ckey, a.cval, a.ckey_alt, a.cval_alt, n4, a.vbits, a, sm))
            return false;
        int *par = a.parent;
        for (int s = tid; s < k; s += nt) par[s] = s;
        if (!g.sync()) return false;
        for (int i = tid + 1; i < n4; i += nt)
            if (__ldcg(ck1 + i) == __ldcg(ck1 + i - 1))
                setup_unite<false>(par, __ldcg(cv1 + i) >> 2, __ldcg(cv1 + i - 1) >> 2, a.status);
        if (!g.sync()) return false;
        for (int s = tid; s < k; s += nt) {
            a.zlab[s] = (unsigned)uf_find(par, s);
            a.zsrc[s] = s;
        }
        if (!g.sync()) return false;
        if (!setup_sort(g, false, a.zlab, a.zsrc, a.zlab_alt, a.zsrc_alt, k, zbits, a, sm))
            return false;
        for (int t = tid; t < k; t += nt)
            a.cflag[t] = (t == 0 || __ldcg(zl + t) != __ldcg(zl + t - 1)) ? 1u : 0u;
        if (!g.sync()) return false;
    }
    unsigned nz;
    if (!setup_scan(g, small, a.cflag, k, a.hist, a.d_nz, nz)) return false;
    int *pos_of = a.parent;
    for (int t = tid; t < k; t += nt) {
        const int src = __ldcg(zr + t);
        const unsigned f = (t == 0 || __ldcg(zl + t) != __ldcg(zl + t - 1)) ? 1u : 0u;
        const int z = (int)(__ldcg(a.cflag + t) + f) - 1;
        a.szone[t] = z;
        pos_of[src] = t;
        if (f) a.zs[z] = t;
        if (t == k - 1) a.zs[z + 1] = k;
        a.ids[t] = a.ids_raw[src];
        a.n64[t] = a.n64_raw[src];
        a.n32[t] = a.n32_raw[src];
        a.b[t] = a.b_raw[src];
    }
    if (!g.sync()) return false;
    // groups of rows sharing x0 (at most GMAX rows each)
    for (int t = tid; t < k; t += nt)
        a.cflag[t] = group_start_l2(a.ids, a.szone, a.zs, t) ? 1u : 0u;
    if (!g.sync()) return false;
    unsigned ng;
    if (!setup_scan(g, small, a.cflag, k, a.hist, a.d_ng, ng)) return false;
    for (int t = tid; t < k; t += nt) {
        const bool st = group_start_l2(a.ids, a.szone, a.zs, t);
        const int gi = (int)__ldcg(a.cflag + t);
        if (st) {
            a.gst[gi] = t;
            const int z = __ldcg(a.szone + t);
            if (__ldcg(a.zs + z) == t) a.zg[z] = gi;
        }
        if (t == k - 1) {
            a.gst[ng] = k;
            a.zg[nz] = (int)ng;
        }
    }
    // the inverse blocks (float64) need only the groups, the zone-ordered
    // rows and the masses: the CTAs not taking part compute them while the
    // others build the zone-ordered CSR (they wait for this flag,
    // SETUP_READY); without such CTAs the others compute them at the end
    const bool helpers = g.parts < gridDim.x;
    if (helpers) {
        __threadfence();  // the groups are written before the flag below
        if (!g.sync()) return false;
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(a.bar + SETUP_READY, 1u);
    }
    // zone-ordered CSR: the vertex-ordered entries re-sorted stably by zone
    // (an odd pass count starts from the spare buffers, so that the sorted
    // entries end in v2, where the solver reads them)
    const int qbits = setup_bits((int)nz);
    const bool qodd = (qbits / 8) & 1;
    unsigned *k2in = qodd ? a.k2_alt : a.k2, *k2out = qodd ? a.k2 : a.k2_alt;
    int *v2in = qodd ? a.v2_alt : a.v2, *v2out = qodd ? a.v2 : a.v2_alt;
    for (int i = tid; i < n4; i += nt) {
        const int e = __ldcg(cv1 + i);
        const int t = __ldcg(pos_of + (e >> 2));
        k2in[i] = (unsigned)__ldcg(a.szone + t);
        v2in[i] = 4 * t + (e & 3);
    }
    if (!g.sync()) return false;
    if (!setup_sort(g, small, k2in, v2in, k2out, v2out, n4, qbits, a, sm)) return false;
    const unsigned *zk = a.k2;
    const int *val = a.v2;
    const int *idsi = (const int *)a.ids;
    for (int i = tid; i < n4; i += nt)
        a.cflag[i] = (i == 0 || __ldcg(idsi + __ldcg(val + i)) != __ldcg(idsi + __ldcg(val + i - 1)))
                         ? 1u : 0u;
    if (!g.sync()) return false;
    unsigned U;
    if (!setup_scan(g, small, a.cflag, n4, a.hist, a.d_U, U)) return false;
    for (int i = tid; i < n4; i += nt) {
        const int vi = __ldcg(val + i);
        const int gv = __ldcg(idsi + vi);
        const unsigned f = (i == 0 || gv != __ldcg(idsi + __ldcg(val + i - 1))) ? 1u : 0u;
        const int j = (int)(__ldcg(a.cflag + i) + f) - 1;
        ((int *)a.vidx)[vi] = j;
        if (f) {
            a.seg[j] = i;
            a.gvert[j] = gv;
            const float *w = gv < a.nA ? a.wA : a.wB;
            const int lv = gv < a.nA ? gv : gv - a.nA;
            a.winv[j] = w ? w[lv] : 1.0f;
            const unsigned zi = __ldcg(zk + i);
            if (i == 0 || zi != __ldcg(zk + i - 1)) a.zv[zi] = j;
        }
        if (i == n4 - 1) {
            a.seg[j + 1] = n4;
            a.zv[nz] = j + 1;
        }
    }
    if (!g.sync()) return false;
    if (!helpers) setup_inverses(a, 0, (int)g.parts);
    return true;
}

union SetupSmem {
    SortSmem sort;
    int par[SETUP_SMALL_K];
};

__global__ void __launch_bounds__(TPB) k_setup(SetupArgs a) {
    HFCR_PDL_WAIT();
    const int k = max(0, min(*a.d_k, a.cap));
    // CTAs taking part: every CTA on large inputs, one per 1,024 entries on
    // small ones (the others leave at once; every CTA reads the same count)
    unsigned parts = gridDim.x;
    if (k <= SETUP_SMALL_K) {
        const unsigned want = (unsigned)max(1, (4 * k + SETUP_ENTRIES_PER_CTA - 1) / SETUP_ENTRIES_PER_CTA);
        if (want < parts) parts = want;
    }
    if (blockIdx.x >= parts) {
        if (k > 0) setup_helper(a, (int)parts);
        return;
    }
    __shared__ SetupSmem sh;
    SetupSync g{a.bar, 0u, a.status, parts};
    setup_phases(g, a, k, sh.sort, sh.par);
}

}  // namespace

void assemble(const MeshPair &mp, const hfcr_stencil *st, const int *d_k, int cap, double d,
              SolveBuffers &sb, uint32_t *d_status, cudaStream_t s) {
    if (cap <= 0) return;
    // dwork[8] / dwork[9]: the largest |b| and |dx| of the call, as the
    // bits of non-negative doubles
    { launch_pdl(k_assemble, (cap + 255) / 256, 256, 0, s, mp.A, mp.B, st, d_k, cap, d, sb.ids_raw,
                 sb.n64_raw, sb.n32_raw, sb.b_raw, (unsigned long long *)(sb.dwork + 8),
                 d_status); note_launch(); }
}

// dynamic shared memory granted to the zone CG kernels (0: the global-memory
// path runs); set once per process, outside any stream capture
static int g_fast_smem = -1, g_zone_pair_smem = 0, g_warp_zone_smem = 0;
static bool g_cluster_ok = false;  // k_cg_zone_cl can be launched on this device

void solver_init() {
    if (g_fast_smem >= 0) return;
    g_fast_smem = cudaFuncSetAttribute(k_cg_zone<BIG_ZONE_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       FAST_SMEM) == cudaSuccess ? FAST_SMEM : 0;
    if (!g_fast_smem) cudaGetLastError();
    g_zone_pair_smem = cudaFuncSetAttribute(k_cg_zone_pair, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            ZONE_PAIR_SMEM) == cudaSuccess ? ZONE_PAIR_SMEM : 0;
    if (!g_zone_pair_smem) cudaGetLastError();
    const int wz = WARP_ZONE_WARPS * WARP_ZONE_SMEM;
    g_warp_zone_smem = cudaFuncSetAttribute(k_cg_zone_warp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            wz) == cudaSuccess ? wz : 0;
    if (!g_warp_zone_smem) cudaGetLastError();
    // the cluster solver of large zones: its shared memory, and whether a
    // cluster of CL such CTAs fits on this device at all
    g_cluster_ok = false;
    if (cudaFuncSetAttribute(k_cg_zone_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, CL_SMEM) ==
        cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(CL);
        cfg.blockDim = dim3(CL_THREADS);
        cfg.dynamicSmemBytes = CL_SMEM;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = CL;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int ncl = 0;
        g_cluster_ok = cudaOccupancyMaxActiveClusters(&ncl, (const void *)k_cg_zone_cl, &cfg) ==
                           cudaSuccess && ncl > 0;
    }
    cudaGetLastError();
}

// co-resident CTAs of k_setup on this device (0: cooperative launch unavailable)
static int setup_grid_max() {
    static int g[64] = {0};
    static bool done[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!done[dev]) {
        int per_sm = 0, sms = 0, coop = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_setup, TPB, 0) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop)
            // two CTAs per SM at most: the grid-wide phases are short and
            // every barrier costs one arrival per CTA
            g[dev] = (per_sm < 2 ? per_sm : 2) * sms;
        else
            cudaGetLastError();
        done[dev] = true;
    }
    return g[dev];
}

// the whole setup as one cooperative launch; false when it cannot be launched
static bool build_setup_fused(const MeshPair &mp, const int *d_k, int cap, SolveBuffers &sb,
                              SortTemp &t, int *d_n4, uint32_t *d_status, cudaStream_t s) {
    int grid = setup_grid_max();
    if (grid <= 0 || !d_status || t.max_blocks < 3) return false;
    const int tiles = (4 * cap + TILE - 1) / TILE;
    if (grid > tiles) grid = tiles > 0 ? tiles : 1;
    SetupArgs a;
    const int vb = bits_for((long long)mp.A.n_verts + mp.B.n_verts);
    a.d_k = d_k;
    a.cap = cap;
    a.vbits = 8 * ((vb + 7) / 8);
    a.nA = mp.A.n_verts;
    a.wA = mp.A.inv_mass;
    a.wB = mp.B.inv_mass;
    a.ids_raw = sb.ids_raw;
    a.n64_raw = sb.n64_raw;
    a.n32_raw = sb.n32_raw;
    a.b_raw = sb.b_raw;
    a.ckey = sb.ckey;
    a.ckey_alt = sb.ckey_alt;
    a.cflag = sb.cflag;
    a.cval = sb.cval;
    a.cval_alt = sb.cval_alt;
    a.zlab = (unsigned *)sb.zkey;
    a.zlab_alt = (unsigned *)sb.zkey_alt;
    a.zsrc = (int *)sb.zkey + cap;
    a.zsrc_alt = (int *)sb.zkey_alt + cap;
    a.k2 = (unsigned *)sb.ck64;
    a.k2_alt = (unsigned *)sb.ck64_alt;
    a.v2 = (int *)sb.ck64 + 4 * (size_t)cap;
    a.v2_alt = (int *)sb.ck64_alt + 4 * (size_t)cap;
    a.parent = sb.parent;
    a.ids = sb.ids;
    a.n64 = sb.n64;
    a.n32 = sb.n32;
    a.b = sb.b;
    a.szone = sb.szone;
    a.zs = sb.zs;
    a.zv = sb.zv;
    a.gst = sb.gst;
    a.zg = sb.zg;
    a.seg = sb.seg;
    a.gvert = sb.gvert;
    a.vidx = sb.vidx;
    a.winv = sb.winv;
    a.pinv = sb.pinv;
    a.d_n4 = d_n4;
    a.d_U = sb.d_U;
    a.d_nz = sb.d_nz;
    a.d_ng = sb.d_ng;
    a.hist = t.hist;
    a.tot = t.hist + 256 * (size_t)(t.max_blocks - 1);
    a.bar = t.hist + 256 * (size_t)(t.max_blocks - 2);
    a.status = d_status;
    cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), s);  // barrier counter, ready flag
    void *args[] = {&a};
    if (cudaLaunchCooperativeKernel((const void *)k_setup, grid, TPB, args, 0, s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    note_launch();
    sb.cval_s = a.v2;
    return true;
}

void build_vertex_csr(const MeshPair &mp, const int *d_k, int cap, SolveBuffers &sb, SortTemp &t,
                      int *d_n4, uint32_t *d_status, int path, cudaStream_t s) {
    if (cap <= 0) return;
    if (path == 0 && build_setup_fused(mp, d_k, cap, sb, t, d_n4, d_status, s)) return;
    // the same setup as a sequence of kernels
    int n4 = 4 * cap;
    int nb = (n4 + 255) / 256;
    int gb = (cap + 255) / 256;
    if (gb > 1024) gb = 1024;
    // vertex -> stencils of the rows as assembled (for the impact zones)
    { launch_pdl(k_csr_entries, nb, 256, 0, s, sb.ids_raw, d_k, cap, sb.ckey,
                 sb.cval); note_launch(); }
    { launch_pdl(k_csr_flags, 1, 1, 0, s, sb.ckey, d_k, cap, sb.cflag,
                 d_n4); note_launch(); }  // count only
    int vb = bits_for((long long)mp.A.n_verts + mp.B.n_verts);
    bool flip = radix_sort_u32_dev(sb.ckey, sb.cval, sb.ckey_alt, sb.cval_alt, d_n4, n4, vb, t, s);
    unsigned *ck1 = flip ? sb.ckey_alt : sb.ckey;
    int *cv1 = flip ? sb.cval_alt : sb.cval;
    { launch_pdl(k_csr_flags, nb, 256, 0, s, ck1, d_k, cap, sb.cflag, d_n4); note_launch(); }
    scan_flags_dev(sb.cflag, d_n4, n4, sb.d_U, t, s);
    { launch_pdl(k_csr_build, nb, 256, 0, s, ck1, cv1, sb.cflag, d_k, cap, mp.A.n_verts,
                 mp.A.inv_mass,
                                   mp.B.inv_mass, sb.vidx, sb.seg, sb.gvert, sb.winv); note_launch(); }
    // impact zones and the zone-ordered rows.  The 64-bit scratch arrays
    // are used as pairs of 32-bit arrays: (label, stencil) for the zone sort,
    // (zone, entry) for the zone-ordered CSR.
    int kb = bits_for((long long)cap + 1);
    unsigned *zlab = (unsigned *)sb.zkey, *zlab_alt = (unsigned *)sb.zkey_alt;
    int *zsrc = (int *)sb.zkey + cap, *zsrc_alt = (int *)sb.zkey_alt + cap;
    { launch_pdl(k_uf_small, 1, 1024, 0, s, d_k, sb.d_U, sb.seg, cv1, zlab, zsrc,
                 d_status); note_launch(); }
    if (cap > UF_SMALL) {
        { launch_pdl(k_uf_init, gb, 256, 0, s, d_k, sb.parent); note_launch(); }
        { launch_pdl(k_uf_union, nb < 1024 ? nb : 1024, 256, 0, s, d_k, sb.d_U, sb.seg, cv1,
                     sb.parent, d_status); note_launch(); }
        { launch_pdl(k_zone_keys, gb, 256, 0, s, d_k, sb.parent, zlab, zsrc); note_launch(); }
    }
    bool zflip = radix_sort_u32_dev(zlab, zsrc, zlab_alt, zsrc_alt, d_k, cap, kb, t, s);
    unsigned *zl = zflip ? zlab_alt : zlab;
    int *zr = zflip ? zsrc_alt : zsrc;
    { launch_pdl(k_zone_flags, gb, 256, 0, s, d_k, zl, sb.cflag); note_launch(); }
    scan_flags_dev(sb.cflag, d_k, cap, sb.d_nz, t, s);
    int *pos_of = sb.parent;  // the forest is no longer needed
    { launch_pdl(k_zone_gather, gb, 256, 0, s, d_k, zl, zr, sb.cflag, sb.ids_raw, sb.n64_raw,
                 sb.n32_raw,
                                     sb.b_raw, sb.ids, sb.n64, sb.n32, sb.b, sb.szone, sb.zs,
                                     pos_of); note_launch(); }
    // vertex-ordered entries re-sorted stably by zone: zone-contiguous numbering
    unsigned *k2 = (unsigned *)sb.ck64, *k2_alt = (unsigned *)sb.ck64_alt;
    int *v2 = (int *)sb.ck64 + n4, *v2_alt = (int *)sb.ck64_alt + n4;
    { launch_pdl(k_csr2_entries, nb, 256, 0, s, cv1, pos_of, sb.szone, d_k, cap, k2,
                 v2); note_launch(); }
    bool flip2 = radix_sort_u32_dev(k2, v2, k2_alt, v2_alt, d_n4, n4, kb, t, s);
    unsigned *zk2 = flip2 ? k2_alt : k2;
    sb.cval_s = flip2 ? v2_alt : v2;
    { launch_pdl(k_csr2_flags, nb, 256, 0, s, sb.cval_s, sb.ids, d_k, cap,
                 sb.cflag); note_launch(); }
    scan_flags_dev(sb.cflag, d_n4, n4, sb.d_U, t, s);
    { launch_pdl(k_csr2_build, nb, 256, 0, s, zk2, sb.cval_s, sb.cflag, sb.ids, d_k, cap,
                 mp.A.n_verts,
                                    mp.A.inv_mass, mp.B.inv_mass, sb.vidx, sb.seg, sb.gvert, sb.winv,
                                    sb.zv, sb.d_nz); note_launch(); }
    // groups of rows sharing x0 and the inverses of their blocks
    { launch_pdl(k_group_flags, gb, 256, 0, s, d_k, sb.ids, sb.szone, sb.zs,
                 sb.cflag); note_launch(); }
    scan_flags_dev(sb.cflag, d_k, cap, sb.d_ng, t, s);
    { launch_pdl(k_group_build, gb, 256, 0, s, d_k, sb.ids, sb.szone, sb.zs, sb.cflag, sb.d_nz,
                 sb.gst,
                                     sb.zg); note_launch(); }
    { launch_pdl(k_group_inverse, gb, 128, 0, s, sb.d_ng, sb.gst, sb.ids, sb.n64, mp.A.n_verts,
                 mp.A.inv_mass, mp.B.inv_mass, sb.pinv); note_launch(); }
}

void solve(const SolveParams &p, const MeshPair &mp, const int *d_k, int cap, SolveBuffers &sb,
           uint32_t *d_status, cudaStream_t s) {
    (void)d_status;
    if (cap <= 0) return;
    solver_init();
    const int fast_smem = g_fast_smem;
    int rb = (cap + 255) / 256;
    if (rb > RES_BLOCKS) rb = RES_BLOCKS;
    // sb.iwork and sb.dwork were zeroed with the call's other device words
    if (p.solver == HFCR_SOLVER_FP64) {
        // the plain float64 form: every impact zone by its own CTA, float64
        // CG with the whole iteration budget of the mixed solver
        ZoneArgs za;
        za.zs = sb.zs; za.zv = sb.zv; za.zg = sb.zg;
        za.seg = sb.seg; za.cval = sb.cval_s; za.winv = sb.winv;
        za.n32 = sb.n32; za.pinv = sb.pinv; za.n64 = sb.n64; za.vidx = sb.vidx; za.gst = sb.gst;
        za.b64 = sb.b; za.lam = sb.lam; za.u64 = sb.u64; za.zres = sb.r64; za.zbb = sb.q64;
        za.maxit = p.max_cg_iters; za.max_refine = p.max_refine;
        za.tol = p.inner_tol; za.rel_tol = p.rel_tol; za.ctl = sb.iwork;
        za.ticket = (unsigned *)(sb.iwork + 13);
        za.ids = sb.ids;
        za.nA = mp.A.n_verts;
        za.wA = mp.A.inv_mass;
        za.wB = mp.B.inv_mass;
        za.pinv64 = sb.pinv64;
        Zone64Scratch g64;
        g64.r = sb.cg64; g64.p = sb.cg64 + cap; g64.s = sb.cg64 + 2 * (size_t)cap;
        g64.w = sb.cg64 + 3 * (size_t)cap; g64.z = sb.cg64 + 4 * (size_t)cap;
        int zg = cap < 4 * 152 ? cap : 4 * 152;
        { launch_pdl(k_cg_zone64, zg, ZONE64_THREADS, 0, s, sb.d_nz, za, g64,
                     p.max_cg_iters * p.max_refine, 0); note_launch(); }
        { launch_pdl(k_zone_final, 1, 256, 0, s, sb.d_nz, sb.r64, sb.q64, p.rel_tol, sb.dwork,
                     sb.iwork); note_launch(); }
        return;
    }
    if (p.solver == HFCR_SOLVER_FP64_GLOBAL) {
        // one float64 run with the whole iteration budget of the mixed solver
        { launch_pdl(k_init_lam, rb, 256, 0, s, d_k, sb.b, sb.lam, sb.r64); note_launch(); }
        { launch_pdl(k_cg<double>, 1, CG_THREADS, 0, s, 1, d_k, sb.d_U, sb.seg, sb.cval_s,
                     sb.winv, sb.n64,
                                              sb.vidx, sb.b, sb.lam, sb.p64 + 0, sb.r64, sb.p64 + cap,
                                              sb.q64, sb.u64, p.max_cg_iters * p.max_refine,
                                              p.rel_tol, sb.iwork); note_launch(); }
        { launch_pdl(k_res_vertex, rb, 256, 0, s, sb.d_U, sb.seg, sb.cval_s, sb.winv, sb.n64,
                     sb.lam, sb.u64,
                                         sb.iwork); note_launch(); }
        { launch_pdl(k_res_stencil, rb, 256, 0, s, d_k, sb.vidx, sb.n64, sb.b, sb.u64, sb.r64,
                     sb.red,
                                          sb.iwork, (unsigned *)(sb.iwork + 12), p.rel_tol,
                                          sb.dwork, 0); note_launch(); }
        return;
    }
    // MIXED: float32 PCG with float64 refinement, each zone to convergence
    // in its own CTA.  r64 and q64 (float64 scratch of the FP64 solver) hold
    // the zones' final |r|^2 and |b|^2.
    ZoneArgs za;
    za.zs = sb.zs; za.zv = sb.zv; za.zg = sb.zg;
    za.seg = sb.seg; za.cval = sb.cval_s; za.winv = sb.winv;
    za.n32 = sb.n32; za.pinv = sb.pinv; za.n64 = sb.n64; za.vidx = sb.vidx; za.gst = sb.gst;
    za.b64 = sb.b; za.lam = sb.lam; za.u64 = sb.u64; za.zres = sb.r64; za.zbb = sb.q64;
    za.maxit = p.max_cg_iters; za.max_refine = p.max_refine;
    za.tol = p.inner_tol; za.rel_tol = p.rel_tol; za.ctl = sb.iwork;
    za.ticket = (unsigned *)(sb.iwork + 13);  // iwork is zeroed before every solve
    za.binv = sb.binv;
    za.block_switch = p.block_switch;
    const int warp_max = g_warp_zone_smem ? WARP_ZONE : 0;
    if (warp_max) {
        int zw = (cap + WARP_ZONE_WARPS - 1) / WARP_ZONE_WARPS;  // CTAs of the warp launch
        if (zw > 4 * 152) zw = 4 * 152;
        { launch_pdl(k_cg_zone_warp, zw, 32 * WARP_ZONE_WARPS, g_warp_zone_smem, s, sb.d_nz,
                     za); note_launch(); }
    }
    ZoneScratch gs;
    gs.x = sb.x32; gs.r = sb.r32; gs.p = sb.p32; gs.s = sb.q32; gs.w = sb.w32; gs.z = sb.z32;
    gs.u = sb.u32;
    // CTAs of the pair launch: two zones of more than warp_max stencils at
    // a time (at most 2 CTAs per SM); of the large-zone launch: one zone
    // of ZONE_BIG or more stencils each
    int zpair = (cap / (WARP_ZONE + 1) + 1) / 2 + 1;
    if (zpair > 2 * 152) zpair = 2 * 152;
    int zbig = (cap + ZONE_MID - 1) / ZONE_MID;
    if (zbig > 152) zbig = 152;
    { launch_pdl(k_cg_zone_pair, zpair, 512, g_zone_pair_smem, s, sb.d_nz, za, warp_max, gs,
                 g_zone_pair_smem, zbig); note_launch(); }
    // zones of ZONE_BIG rows or more: one CTA each when they fit its shared
    // memory; larger ones on a cluster of CL CTAs (or, without
    // clusters, on global memory)
    p.big_mark(1, s);
    { launch_pdl(k_cg_zone<BIG_ZONE_THREADS>, zbig, BIG_ZONE_THREADS, fast_smem, s, sb.d_nz, za, ZONE_BIG - 1,
                 ZONE_MID, gs, fast_smem, g_cluster_ok ? 1 : 0); note_launch(); }
    if (g_cluster_ok) {
        int ncl = (cap + ZONE_CL_MIN - 1) / ZONE_CL_MIN;
        if (ncl > 152 / CL) ncl = 152 / CL;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(ncl * CL);
        cfg.blockDim = dim3(CL_THREADS);
        cfg.dynamicSmemBytes = CL_SMEM;
        cfg.stream = s;
        cudaLaunchAttribute at[2];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = CL;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 2;
        cudaLaunchKernelEx(&cfg, k_cg_zone_cl, (const int *)sb.d_nz, za, gs, fast_smem);
        note_launch();
    }
    p.big_mark(0, s);
    // a zone whose float32 runs stopped reducing its float64 residual before
    // the target (the residual guard) is solved again by the float64 per-zone
    // CG; every other zone is skipped at once
    za.ids = sb.ids;
    za.nA = mp.A.n_verts;
    za.wA = mp.A.inv_mass;
    za.wB = mp.B.inv_mass;
    za.pinv64 = sb.pinv64;
    {
        Zone64Scratch g64;
        g64.r = sb.cg64; g64.p = sb.cg64 + cap; g64.s = sb.cg64 + 2 * (size_t)cap;
        g64.w = sb.cg64 + 3 * (size_t)cap; g64.z = sb.cg64 + 4 * (size_t)cap;
        int zr = cap < 152 ? cap : 152;
        { launch_pdl(k_cg_zone64, zr, ZONE64_THREADS, 0, s, sb.d_nz, za, g64,
                     p.max_cg_iters * p.max_refine, 1); note_launch(); }
    }
    { launch_pdl(k_zone_final, 1, 256, 0, s, sb.d_nz, sb.r64, sb.q64, p.rel_tol, sb.dwork,
                 sb.iwork); note_launch(); }
}

void displacement(const MeshPair &mp, int cap, SolveBuffers &sb, int apply, void *const *dxA,
                  void *const *dxB, cudaStream_t s) {
    if (cap <= 0) return;
    int nb = (4 * cap + 255) / 256;
    if (nb > 1024) nb = 1024;
    void *a0 = dxA ? dxA[0] : nullptr, *a1 = dxA ? dxA[1] : nullptr, *a2 = dxA ? dxA[2] : nullptr;
    void *b0 = dxB ? dxB[0] : nullptr, *b1 = dxB ? dxB[1] : nullptr, *b2 = dxB ? dxB[2] : nullptr;
    { launch_pdl(k_displace, nb, 256, 0, s, sb.d_U, sb.seg, sb.cval_s, sb.winv, sb.n64, sb.lam,
                 sb.gvert, mp.A, mp.B, apply, a0, a1, a2, b0, b1, b2,
                 (unsigned long long *)(sb.dwork + 9)); note_launch(); }
}

}  // namespace hfcr
