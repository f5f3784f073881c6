// Topology (edges), input validation and the linear BVH over the faces of
// an oriented mesh.
//
// The paper only says that detection uses tight bounding volumes (Sec. 1);
// the hierarchy here is a binary radix tree over 30-bit Morton codes of the
// face centroids (Karras 2012), refitted bottom-up with arrival counters.
// Boxes are float32 and conservative: for float32 coordinates min/max are
// exact, for float64 they are rounded outward, so box rejection never drops
// a true intersection.
#include <cuda_runtime.h>
#include <float.h>
#include <stdint.h>

#include "internal.h"

namespace hfcr {

namespace {

// segment table sanity: rows non-decreasing, first row 0, last row equal to
// the mesh sizes (the concatenated A and B)
__global__ void k_check_segs(const int *segs, int nseg, int nva, int nta, int nvb, int ntb,
                             uint32_t *st) {
    HFCR_PDL_WAIT();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > nseg) return;
    const int tot[4] = {nva, nta, nvb, ntb};
    for (int c = 0; c < 4; ++c) {
        int v = segs[4 * i + c];
        bool bad = (i == 0 && v != 0) || (i == nseg && v != tot[c]) ||
                   (i > 0 && v < segs[4 * (i - 1) + c]) || v < 0 || v > tot[c];
        if (bad) atomicOr(st, ST_BAD_INDEX);
    }
}

// index into [0, n): out-of-range ids read element 0 and raise ST_BAD_INDEX
__device__ __forceinline__ int chk(int i, int n, uint32_t *st) {
    if ((unsigned)i < (unsigned)n) return i;
    atomicOr(st, ST_BAD_INDEX);
    return 0;
}

template <typename T>
__global__ void k_validate(const T *x, const T *y, const T *z, int n, uint32_t *status) {
    HFCR_PDL_WAIT();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t bad = 0;
    if (i < n) {
        T c[3] = {x[i], y[i], z[i]};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            T v = c[k];
            if (!isfinite(v)) {
                bad |= ST_NONFINITE;
            } else {
                T a = fabs(v);
                if (a > (T)0x1p38) bad |= ST_RANGE;
                if (sizeof(T) == 8 && a != (T)0 && a < (T)0x1p-200) bad |= ST_RANGE;
            }
        }
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (bad && (threadIdx.x & 31) == 0) atomicOr(status, bad);
}

// both meshes of a pair in one launch: vertex i < nA of A, else i - nA of B
template <typename T>
__global__ void k_validate_pair(const T *ax, const T *ay, const T *az, int nA, const T *bx,
                                const T *by, const T *bz, int nB, uint32_t *status) {
    HFCR_PDL_WAIT();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t bad = 0;
    if (i < nA + nB) {
        const bool inA = i < nA;
        const int j = inA ? i : i - nA;
        T c[3] = {inA ? ax[j] : bx[j], inA ? ay[j] : by[j], inA ? az[j] : bz[j]};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            T v = c[k];
            if (!isfinite(v)) {
                bad |= ST_NONFINITE;
            } else {
                T a = fabs(v);
                if (a > (T)0x1p38) bad |= ST_RANGE;
                if (sizeof(T) == 8 && a != (T)0 && a < (T)0x1p-200) bad |= ST_RANGE;
            }
        }
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (bad && (threadIdx.x & 31) == 0) atomicOr(status, bad);
}

__global__ void k_edge_keys(const int *tris, int nt, int vb, unsigned long long *keys,
                            uint32_t *status, int nv) {
    HFCR_PDL_WAIT();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int v[3] = {tris[3 * t], tris[3 * t + 1], tris[3 * t + 2]};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int a = v[k], b = v[(k + 1) % 3];
        if ((unsigned)a >= (unsigned)nv || (unsigned)b >= (unsigned)nv) {
            atomicOr(status, ST_BAD_INDEX);
            a = b = 0;
        }
        unsigned long long lo = (unsigned)min(a, b), hi = (unsigned)max(a, b);
        keys[3 * t + k] = (lo << vb) | hi;
    }
}

__global__ void k_unique_flags(const unsigned long long *keys, int n, unsigned *flags) {
    HFCR_PDL_WAIT();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flags[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

__global__ void k_write_edges(const unsigned long long *keys, const unsigned *pos, int n, int vb,
                              int *edges) {
    HFCR_PDL_WAIT();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (i == 0 || keys[i] != keys[i - 1]) {
        unsigned long long k = keys[i];
        unsigned p = pos[i];
        edges[2 * p] = (int)(k >> vb);
        edges[2 * p + 1] = (int)(k & ((1ull << vb) - 1));
    }
}

template <typename T>
__device__ __forceinline__ void load3(const T *x, const T *y, const T *z, int i, T *o) {
    o[0] = x[i];
    o[1] = y[i];
    o[2] = z[i];
}

__device__ __forceinline__ float lo_f(float v) { return v; }
__device__ __forceinline__ float hi_f(float v) { return v; }
__device__ __forceinline__ float lo_f(double v) { return __double2float_rd(v); }
__device__ __forceinline__ float hi_f(double v) { return __double2float_ru(v); }

// per-block min/max of the vertex positions (coalesced; they contain every
// face centroid, and float32 approximations suffice: the codes only order
// the leaves)
template <typename T>
__global__ void k_vertex_bounds(const T *x, const T *y, const T *z, int nv, float *part) {
    HFCR_PDL_WAIT();
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
        const float c[3] = {(float)x[v], (float)y[v], (float)z[v]};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lo[k] = fminf(lo[k], c[k]);
            hi[k] = fmaxf(hi[k], c[k]);
        }
    }
    __shared__ float s[6][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        for (int o = 16; o; o >>= 1) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
        if (lane == 0) { s[k][w] = lo[k]; s[3 + k][w] = hi[k]; }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        int nw = blockDim.x >> 5;
        float v = s[threadIdx.x][0];
        for (int i = 1; i < nw; ++i)
            v = threadIdx.x < 3 ? fminf(v, s[threadIdx.x][i]) : fmaxf(v, s[threadIdx.x][i]);
        part[6 * blockIdx.x + threadIdx.x] = v;
    }
}

// the nb per-block partials folded by one CTA of 256 threads
__global__ void __launch_bounds__(256) k_bounds_final(const float *part, int nb, float *bounds) {
    HFCR_PDL_WAIT();
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lo[k] = fminf(lo[k], part[6 * i + k]);
            hi[k] = fmaxf(hi[k], part[6 * i + 3 + k]);
        }
    __shared__ float sh[6][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        for (int o = 16; o; o >>= 1) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
        if (lane == 0) { sh[k][w] = lo[k]; sh[3 + k][w] = hi[k]; }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int k = threadIdx.x;
        float v = sh[k][0];
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) v = k < 3 ? fminf(v, sh[k][q]) : fmaxf(v, sh[k][q]);
        bounds[k] = v;
    }
}

__device__ __forceinline__ unsigned spread10(unsigned v) {
    v = (v * 0x00010001u) & 0xFF0000FFu;
    v = (v * 0x00000101u) & 0x0F00F00Fu;
    v = (v * 0x00000011u) & 0xC30C30C3u;
    v = (v * 0x00000005u) & 0x49249249u;
    return v;
}

// Morton code of each face's centroid, quantised to `cells` per axis in the
// scene bounds (cells <= 1024), above it the face's segment
template <typename T>
__global__ void k_morton(const T *x, const T *y, const T *z, int nv, const int *tris, int nt,
                         const float *bounds, const int *segs, int col, int nseg, float cells,
                         unsigned long long *keys, int *vals, uint32_t *st) {
    HFCR_PDL_WAIT();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    T a[3], b[3], c[3];
    load3(x, y, z, chk(tris[3 * t], nv, st), a);
    load3(x, y, z, chk(tris[3 * t + 1], nv, st), b);
    load3(x, y, z, chk(tris[3 * t + 2], nv, st), c);
    unsigned q[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float m = (float)((a[k] + b[k] + c[k]) / (T)3);
        float ext = bounds[3 + k] - bounds[k];
        float u = ext > 0.f ? (m - bounds[k]) / ext : 0.f;
        u = fminf(fmaxf(u * cells, 0.f), cells - 1.f);
        q[k] = (unsigned)u;
    }
    const unsigned long long seg = (unsigned long long)seg_of(segs, col, nseg, t);
    keys[t] = (seg << 30) | (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
    vals[t] = t;
}

// sort key of an edge: (segment of its first vertex, Morton code of its
// midpoint); value = the edge's index
template <typename T>
__global__ void k_edge_order_keys(const int2 *edges, int ne, const T *x, const T *y, const T *z,
                                  int nv, const float *bounds, const int *segs, int col, int nseg,
                                  unsigned long long *keys, int *vals, uint32_t *st) {
    HFCR_PDL_WAIT();
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const int2 ed = edges[e];
    const int a = chk(ed.x, nv, st), b = chk(ed.y, nv, st);
    const T pa[3] = {x[a], y[a], z[a]}, pb[3] = {x[b], y[b], z[b]};
    unsigned q[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float m = (float)((pa[k] + pb[k]) / (T)2);
        const float ext = bounds[3 + k] - bounds[k];
        float u = ext > 0.f ? (m - bounds[k]) / ext : 0.f;
        u = fminf(fmaxf(u * 1024.f, 0.f), 1023.f);
        q[k] = (unsigned)u;
    }
    const unsigned long long seg = (unsigned long long)seg_of(segs, col, nseg, a);
    keys[e] = (seg << 30) | (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
    vals[e] = e;
}

// common-prefix length of the keys of leaves i and j of one segment (its
// sorted keys start at K); keys made unique by appending the local index
__device__ __forceinline__ int kdelta(const unsigned long long *K, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    unsigned long long ki = ((K[i] & 0x3fffffffull) << 32) | (unsigned)i;
    unsigned long long kj = ((K[j] & 0x3fffffffull) << 32) | (unsigned)j;
    return __clzll(ki ^ kj);
}

// Karras 2012, one tree per segment: internal node l of the segment whose
// faces start at t0 covers a key range found from the common-prefix lengths
// of its neighbours.  Segment-local node l is stored at t0 + l, leaf c at
// t0 + c (encoded ~(t0 + c)); each segment's root (l = 0) has parent -1.
__global__ void k_karras(const unsigned long long *keys, int n_total, const int *segs, int col,
                         int nseg, float4 *nodes, int *iparent, int *lparent) {
    HFCR_PDL_WAIT();
    int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= n_total) return;
    const int sgi = seg_of(segs, col, nseg, gi);
    int t0, n;
    seg_range(segs, col, sgi, n_total, t0, n);
    const int i = gi - t0;
    if (i < 0 || i >= n - 1) return;
    const unsigned long long *K = keys + t0;
    int d = (kdelta(K, n, i, i + 1) - kdelta(K, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = kdelta(K, n, i, i - d);
    int lmax = 2;
    while (kdelta(K, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (kdelta(K, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = kdelta(K, n, i, j);
    int s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (kdelta(K, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int gamma = i + s * d + min(d, 0);
    int left = (min(i, j) == gamma) ? ~(t0 + gamma) : t0 + gamma;
    int right = (max(i, j) == gamma + 1) ? ~(t0 + gamma + 1) : t0 + gamma + 1;
    // child ids, then the node's leaf range (first, last; one end is gi), which
    // the refit uses to keep a warp's own subtrees in shared memory
    nodes[4 * gi + 3] = make_float4(__int_as_float(left), __int_as_float(right),
                                    __int_as_float(t0 + min(i, j)), __int_as_float(t0 + max(i, j)));
    // parent links carry the child's slot: (parent << 1) | (1 for the right child)
    if (left < 0) lparent[~left] = gi << 1; else iparent[left] = gi << 1;
    if (right < 0) lparent[~right] = (gi << 1) | 1; else iparent[right] = (gi << 1) | 1;
    if (i == 0) iparent[gi] = -1;
}

template <typename T>
__device__ __forceinline__ void pack_leaf(void *leaf_tri, int j, const T *a, const T *b,
                                          const T *c, int f);
template <>
__device__ __forceinline__ void pack_leaf<float>(void *leaf_tri, int j, const float *a,
                                                 const float *b, const float *c, int f) {
    float4 *L = (float4 *)leaf_tri + 3 * j;
    L[0] = make_float4(a[0], a[1], a[2], b[0]);
    L[1] = make_float4(b[1], b[2], c[0], c[1]);
    L[2] = make_float4(c[2], __int_as_float(f), 0.f, 0.f);
}
template <>
__device__ __forceinline__ void pack_leaf<double>(void *leaf_tri, int j, const double *a,
                                                  const double *b, const double *c, int f) {
    double2 *L = (double2 *)leaf_tri + 5 * j;
    L[0] = make_double2(a[0], a[1]);
    L[1] = make_double2(a[2], b[0]);
    L[2] = make_double2(b[1], b[2]);
    L[3] = make_double2(c[0], c[1]);
    L[4] = make_double2(c[2], __longlong_as_double((long long)f));
}

// Bottom-up refit, one thread per leaf, warp by warp: warp w owns leaves
// [32 w, 32 w + 32).  A node whose leaf range lies in its warp's block (its
// whole subtree does) is met by two lanes of that warp: they hand over
// through shared memory (box slots and an arrival counter, block-scope
// fences), and the second writes both child boxes of the node.  Above the
// block, the second child to arrive at a node (an acquire-release atomic
// counter in global memory) merges the two boxes.  Min and max are exact,
// so the boxes do not depend on the arrival order.
constexpr int REFIT_WARPS = 8;

template <typename T>
__global__ void __launch_bounds__(32 * REFIT_WARPS) k_refit(
    const T *x, const T *y, const T *z, int nv, const int *tris, const int *leaf_face, int n,
    float4 *nodes, const int *iparent, const int *lparent, unsigned *flags, void *leaf_tri,
    uint32_t *st) {
    HFCR_PDL_WAIT();
    __shared__ unsigned cnt[REFIT_WARPS][32];
    __shared__ float sbox[REFIT_WARPS][32][12];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int base = (blockIdx.x * REFIT_WARPS + w) * 32;
    cnt[w][lane] = 0u;
    __syncwarp();
    const int j = base + lane;
    if (j >= n) return;
    int f = leaf_face[j];
    T a[3], b[3], c[3];
    load3(x, y, z, chk(tris[3 * f], nv, st), a);
    load3(x, y, z, chk(tris[3 * f + 1], nv, st), b);
    load3(x, y, z, chk(tris[3 * f + 2], nv, st), c);
    pack_leaf<T>(leaf_tri, j, a, b, c, f);
    float lo[3], hi[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        lo[k] = lo_f(fmin(fmin(a[k], b[k]), c[k]));
        hi[k] = hi_f(fmax(fmax(a[k], b[k]), c[k]));
    }
    int link = lparent[j];  // (parent << 1) | slot, -1 at a root
    // bounded by the tree depth (< 64 for unique 62-bit keys); the guard
    // only keeps a corrupted parent array from looping
    for (int guard = 0; guard < 128 && link >= 0; ++guard) {
        const int node = link >> 1;
        const int side = link & 1;
        const int up = iparent[node];  // read-only: load it before the handshake
        float *nf = (float *)(nodes + 4 * node);
        const float4 n3 = nodes[4 * node + 3];  // ids and leaf range: not written here
        const int first = __float_as_int(n3.z), last = __float_as_int(n3.w);
        // both children's lanes are in this warp when the range is: the
        // node's slot q (one end of its range is the node's own index)
        const int q = node - base;
        if (first >= base && last < base + 32 && q >= 0 && q < 32) {
            float *mine = sbox[w][q] + 6 * side;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                mine[k] = lo[k];
                mine[3 + k] = hi[k];
            }
            __threadfence_block();
            if (atomicAdd(&cnt[w][q], 1u) == 0u) return;
            __threadfence_block();
            const volatile float *sb = sbox[w][q];
            float bx[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) bx[k] = sb[k];
            float4 *nd = nodes + 4 * node;
            nd[0] = make_float4(bx[0], bx[1], bx[2], bx[3]);
            nd[1] = make_float4(bx[4], bx[5], bx[6], bx[7]);
            nd[2] = make_float4(bx[8], bx[9], bx[10], bx[11]);
            const int o = 6 * (1 - side);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                lo[k] = fminf(lo[k], bx[o + k]);
                hi[k] = fmaxf(hi[k], bx[o + 3 + k]);
            }
        } else {
            const int slot = 6 * side;
            nf[slot + 0] = lo[0];
            nf[slot + 1] = lo[1];
            nf[slot + 2] = lo[2];
            nf[slot + 3] = hi[0];
            nf[slot + 4] = hi[1];
            nf[slot + 5] = hi[2];
            // the first child to arrive leaves; the second (acquire) sees the
            // first one's box (release) and carries the union upwards
            unsigned old;
            asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;"
                         : "=r"(old) : "l"(flags + node) : "memory");
            if (old == 0) return;
            const int sib = 6 - slot;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                lo[k] = fminf(lo[k], __ldcg(nf + sib + k));
                hi[k] = fmaxf(hi[k], __ldcg(nf + sib + 3 + k));
            }
        }
        link = up;
    }
}

}  // namespace

void validate_positions(const hfcr_mesh &m, uint32_t *d_status, cudaStream_t s) {
    if (m.n_verts <= 0) return;
    int nb = (m.n_verts + 255) / 256;
    if (m.dtype == HFCR_F32)
        { launch_pdl(k_validate<float>, nb, 256, 0, s, (const float *)m.x, (const float *)m.y,
                                             (const float *)m.z, m.n_verts, d_status); note_launch(); }
    else
        { launch_pdl(k_validate<double>, nb, 256, 0, s, (const double *)m.x, (const double *)m.y,
                                              (const double *)m.z, m.n_verts, d_status); note_launch(); }
}

void validate_pair(const hfcr_mesh &A, const hfcr_mesh &B, uint32_t *d_status, cudaStream_t s) {
    if (A.dtype != B.dtype) {
        validate_positions(A, d_status, s);
        validate_positions(B, d_status, s);
        return;
    }
    const int nA = A.n_verts > 0 ? A.n_verts : 0, nB = B.n_verts > 0 ? B.n_verts : 0;
    if (nA + nB <= 0) return;
    const int nb = (nA + nB + 255) / 256;
    if (A.dtype == HFCR_F32)
        { launch_pdl(k_validate_pair<float>, nb, 256, 0, s, (const float *)A.x, (const float *)A.y,
                     (const float *)A.z, nA, (const float *)B.x, (const float *)B.y,
                     (const float *)B.z, nB, d_status); note_launch(); }
    else
        { launch_pdl(k_validate_pair<double>, nb, 256, 0, s, (const double *)A.x,
                     (const double *)A.y, (const double *)A.z, nA, (const double *)B.x,
                     (const double *)B.y, (const double *)B.z, nB, d_status); note_launch(); }
}

void build_edges(const int *tris, int n_tris, int n_verts, int *edges_out, int *d_count,
                 unsigned long long *keys, unsigned long long *keys_alt, unsigned *flags,
                 SortTemp &t, uint32_t *d_status, cudaStream_t s) {
    int n = 3 * n_tris;
    if (n == 0) {
        cudaMemsetAsync(d_count, 0, sizeof(int), s);
        return;
    }
    int vb = bits_for(n_verts > 1 ? n_verts : 2);
    { launch_pdl(k_edge_keys, (n_tris + 255) / 256, 256, 0, s, tris, n_tris, vb, keys, d_status,
                 n_verts); note_launch(); }
    bool flip = radix_sort_u64(keys, nullptr, keys_alt, nullptr, n, 2 * vb, t, s);
    unsigned long long *sorted = flip ? keys_alt : keys;
    { launch_pdl(k_unique_flags, (n + 255) / 256, 256, 0, s, sorted, n, flags); note_launch(); }
    scan_flags_dev(flags, nullptr, n, d_count, t, s);
    { launch_pdl(k_write_edges, (n + 255) / 256, 256, 0, s, sorted, flags, n, vb,
                 edges_out); note_launch(); }
}

void check_segments(const int *segs, int nseg, const hfcr_mesh &A, const hfcr_mesh &B,
                    uint32_t *d_status, cudaStream_t s) {
    { launch_pdl(k_check_segs, (nseg + 1 + 127) / 128, 128, 0, s, segs, nseg, A.n_verts, A.n_tris,
                 B.n_verts,
                                                        B.n_tris, d_status); note_launch(); }
}

void bvh_build(Bvh &b, const hfcr_mesh &m, const int *segs, int col, int nseg, SortTemp &t,
               uint32_t *d_status, cudaStream_t s) {
    int nv = m.n_verts;
    int n = m.n_tris;
    b.n = n;
    b.dtype = m.dtype;
    b.segs = segs;
    b.col = col;
    b.nseg = nseg;
    if (n <= 0) return;
    int nb = (n + 255) / 256;
    // one mesh: 8 bits per axis (24-bit codes, three radix passes; at the
    // face counts here a cell holds about one or two centroids, and equal
    // codes are ordered by face index); a batch: 10 bits per axis below the
    // segment number, each pair's faces sorted by their own CTA
    const bool single = nseg <= 1;
    const float cells = single ? 256.f : 1024.f;
    const int kbits = single ? 24 : 30 + bits_for(nseg + 1);
    // an odd pass count of the one-mesh sort starts from the spare buffers,
    // so that the sorted keys and faces end in the tree's own
    const bool odd = single && (((kbits + 7) / 8) & 1);
    unsigned long long *kin = odd ? b.keys_alt : b.keys, *kout = odd ? b.keys : b.keys_alt;
    int *vin = odd ? b.vals_alt : b.leaf_face, *vout = odd ? b.leaf_face : b.vals_alt;
    int vbk = (nv + 255) / 256;
    if (vbk > 1024) vbk = 1024;
    if (vbk < 1) vbk = 1;
    if (m.dtype == HFCR_F32) {
        const float *x = (const float *)m.x, *y = (const float *)m.y, *z = (const float *)m.z;
        { launch_pdl(k_vertex_bounds<float>, vbk, 256, 0, s, x, y, z, nv,
                     b.bounds_part); note_launch(); }
        { launch_pdl(k_bounds_final, 1, 256, 0, s, b.bounds_part, vbk, b.bounds); note_launch(); }
        { launch_pdl(k_morton<float>, nb, 256, 0, s, x, y, z, nv, m.tris, n, b.bounds, segs, col,
                     nseg, cells, kin, vin, d_status); note_launch(); }
    } else {
        const double *x = (const double *)m.x, *y = (const double *)m.y, *z = (const double *)m.z;
        { launch_pdl(k_vertex_bounds<double>, vbk, 256, 0, s, x, y, z, nv,
                     b.bounds_part); note_launch(); }
        { launch_pdl(k_bounds_final, 1, 256, 0, s, b.bounds_part, vbk, b.bounds); note_launch(); }
        { launch_pdl(k_morton<double>, nb, 256, 0, s, x, y, z, nv, m.tris, n, b.bounds, segs, col,
                     nseg, cells, kin, vin, d_status); note_launch(); }
    }
    // a batch sorts each pair's faces in its own CTA (the segment bits above
    // the 30 Morton bits are constant within a pair); one mesh globally
    bool flip = !single
                    ? radix_sort_u64v_segments(b.keys, b.leaf_face, b.keys_alt, b.vals_alt, n,
                                               kbits, segs, col, nseg, 30, b.d_rest, t, s)
                    : radix_sort_u64(kin, vin, kout, vout, n, kbits, t, s) != (kin == b.keys_alt);
    if (flip) {
        cudaMemcpyAsync(b.keys, b.keys_alt, sizeof(unsigned long long) * n, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(b.leaf_face, b.vals_alt, sizeof(int) * n, cudaMemcpyDeviceToDevice, s);
    }
    // leaves of one-face segments keep parent -1
    cudaMemsetAsync(b.parent + b.cap, 0xff, sizeof(int) * n, s);
    { launch_pdl(k_karras, nb, 256, 0, s, b.keys, n, segs, col, nseg, b.nodes, b.parent,
                 b.parent + b.cap); note_launch(); }
}

void edge_order(const int *edges, int ne, const hfcr_mesh &m, const int *segs, int col, int nseg,
                int *order, int *order_alt, unsigned long long *keys, unsigned long long *keys_alt,
                float *bounds_part, float *bounds, SortTemp &t, uint32_t *d_status, cudaStream_t s) {
    if (ne <= 0 || m.n_verts <= 0) return;
    const int nv = m.n_verts, nb = (ne + 255) / 256;
    int vbk = (nv + 255) / 256;
    if (vbk > 1024) vbk = 1024;
    if (m.dtype == HFCR_F32) {
        const float *x = (const float *)m.x, *y = (const float *)m.y, *z = (const float *)m.z;
        { launch_pdl(k_vertex_bounds<float>, vbk, 256, 0, s, x, y, z, nv,
                     bounds_part); note_launch(); }
        { launch_pdl(k_bounds_final, 1, 256, 0, s, bounds_part, vbk, bounds); note_launch(); }
        { launch_pdl(k_edge_order_keys<float>, nb, 256, 0, s, (const int2 *)edges, ne, x, y, z,
                     nv, bounds, segs,
                                                    col, nseg, keys, order, d_status); note_launch(); }
    } else {
        const double *x = (const double *)m.x, *y = (const double *)m.y, *z = (const double *)m.z;
        { launch_pdl(k_vertex_bounds<double>, vbk, 256, 0, s, x, y, z, nv,
                     bounds_part); note_launch(); }
        { launch_pdl(k_bounds_final, 1, 256, 0, s, bounds_part, vbk, bounds); note_launch(); }
        { launch_pdl(k_edge_order_keys<double>, nb, 256, 0, s, (const int2 *)edges, ne, x, y, z,
                     nv, bounds, segs,
                                                     col, nseg, keys, order, d_status); note_launch(); }
    }
    if (radix_sort_u64(keys, order, keys_alt, order_alt, ne, 30 + bits_for(nseg + 1), t, s))
        cudaMemcpyAsync(order, order_alt, sizeof(int) * (size_t)ne, cudaMemcpyDeviceToDevice, s);
}

void bvh_refit(Bvh &b, const hfcr_mesh &m, uint32_t *d_status, cudaStream_t s) {
    int n = b.n;
    if (n <= 0) return;
    cudaMemsetAsync(b.flags, 0, sizeof(unsigned) * n, s);
    int nb = (n + 32 * REFIT_WARPS - 1) / (32 * REFIT_WARPS);
    if (m.dtype == HFCR_F32)
        { launch_pdl(k_refit<float>, nb, 32 * REFIT_WARPS, 0, s, (const float *)m.x, (const float *)m.y,
                     (const float *)m.z,
                                          m.n_verts, m.tris, b.leaf_face, n, b.nodes, b.parent,
                                          b.parent + b.cap, b.flags, b.leaf_tri, d_status); note_launch(); }
    else
        { launch_pdl(k_refit<double>, nb, 32 * REFIT_WARPS, 0, s, (const double *)m.x, (const double *)m.y,
                                           (const double *)m.z, m.n_verts, m.tris, b.leaf_face, n,
                                           b.nodes, b.parent, b.parent + b.cap, b.flags, b.leaf_tri,
                                           d_status); note_launch(); }
}

}  // namespace hfcr
