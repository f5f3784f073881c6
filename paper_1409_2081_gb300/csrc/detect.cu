// Narrow and broad phase of the edge-face detection (Sec. 3) and the
// penetration stencils (Sec. 4, Fig. 3).
//
// One thread per edge of the edge mesh walks the BVH of the oriented mesh's
// faces with the edge's box, testing both children of a node with one
// 64-byte node load; at a leaf the exact segment-triangle test decides.
// Threads take the edges in the Morton order of their midpoints (a cached
// permutation), so that a warp walks one region of the tree; the packet
// variants walk a warp's edges together.
// Hits are appended (one atomic per hit) as 64-bit keys
// (dir | edge | face), which a radix sort turns into the lexicographic
// (dir, v0, v1, face) order because the edges are sorted by (v0, v1).
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "predicates.cuh"

namespace hfcr {

namespace {

constexpr int STACK = 64;

__device__ __forceinline__ int chk(int i, int n, uint32_t *st) {
    if ((unsigned)i < (unsigned)n) return i;
    atomicOr(st, ST_BAD_INDEX);
    return 0;
}

__device__ __forceinline__ bool overlap(const float *lo, const float *hi, float l0, float l1,
                                        float l2, float h0, float h1, float h2) {
    return lo[0] <= h0 && l0 <= hi[0] && lo[1] <= h1 && l1 <= hi[1] && lo[2] <= h2 && l2 <= hi[2];
}

__device__ __forceinline__ float lo_f(float v) { return v; }
__device__ __forceinline__ float hi_f(float v) { return v; }
__device__ __forceinline__ float lo_f(double v) { return __double2float_rd(v); }
__device__ __forceinline__ float hi_f(double v) { return __double2float_ru(v); }

template <typename T>
struct Leaf;
template <>
struct Leaf<float> {
    float a[3], b[3], c[3];
    int face;
    __device__ __forceinline__ void load(const void *base, int j) {
        const float4 *L = (const float4 *)base + 3 * j;
        float4 l0 = __ldg(L), l1 = __ldg(L + 1), l2 = __ldg(L + 2);
        a[0] = l0.x; a[1] = l0.y; a[2] = l0.z; b[0] = l0.w;
        b[1] = l1.x; b[2] = l1.y; c[0] = l1.z; c[1] = l1.w;
        c[2] = l2.x; face = __float_as_int(l2.y);
    }
};
template <>
struct Leaf<double> {
    double a[3], b[3], c[3];
    int face;
    __device__ __forceinline__ void load(const void *base, int j) {
        const double2 *L = (const double2 *)base + 5 * j;
        double2 l0 = __ldg(L), l1 = __ldg(L + 1), l2 = __ldg(L + 2), l3 = __ldg(L + 3),
                l4 = __ldg(L + 4);
        a[0] = l0.x; a[1] = l0.y; a[2] = l1.x; b[0] = l1.y;
        b[1] = l2.x; b[2] = l2.y; c[0] = l3.x; c[1] = l3.y;
        c[2] = l4.x; face = (int)__double_as_longlong(l4.y);
    }
};

template <typename T, bool F32F>
__device__ __forceinline__ bool leaf_test_body(const T *p, const T *q, const Leaf<T> &L, DevStats *st) {
    int side;
    if constexpr (F32F && sizeof(T) == 4) {
        f3 P = {(float)p[0], (float)p[1], (float)p[2]}, Q = {(float)q[0], (float)q[1], (float)q[2]};
        f3 A = {(float)L.a[0], (float)L.a[1], (float)L.a[2]};
        f3 B = {(float)L.b[0], (float)L.b[1], (float)L.b[2]};
        f3 C = {(float)L.c[0], (float)L.c[1], (float)L.c[2]};
        return segtri_f32(P, Q, A, B, C, side, st);
    } else {
        return segtri_f64<T>(p, q, L.a, L.b, L.c, side, st);
    }
}

// the exact narrow phase out of line: the traversal loop then needs far
// fewer registers (leaf tests are rare next to node visits)
template <typename T, bool F32F>
__device__ __noinline__ bool leaf_test_call(const T *p, const T *q, const Leaf<T> &L, DevStats *st) {
    return leaf_test_body<T, F32F>(p, q, L, st);
}

// Traversal variants (picked by hfcr_autotune): MINB = CTAs of 256 threads
// the compiler must fit per SM (register budget), NOINL = narrow phase out
// of line, PACKET = a warp whose edges all belong to one mesh pair walks
// that pair's tree together (one broadcast load per node, a node entered
// when any lane's box overlaps it, a shared stack per warp); each lane still
// tests exactly the leaves its own box overlaps, because every box of the
// tree contains its children's, so the tests and pairs are those of the
// per-thread walk.  Warps that span two pairs walk per thread.
template <typename T, bool F32F, int MINB, bool NOINL, bool PACKET>
__global__ void __launch_bounds__(256, MINB) k_traverse(
    const int2 *edges, const int *order, int ne, const T *ex, const T *ey, const T *ez, int nv,
    const float4 *nodes, const void *leaf_tri, int nfaces, const int *segs, int nseg, int ecol,
    int fcol, unsigned long long dirbit, int face_bits, unsigned long long *out, int *count, int cap,
    DevStats *st, uint32_t *status) {
    HFCR_PDL_WAIT();
    // thread t takes edge order[t] (a spatially coherent permutation of the
    // edges, when there is one): a warp then walks neighbouring parts of the
    // tree; the keys carry the edge's own index
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int e = t >= ne ? ne : (order ? order[t] : t);
    unsigned tests = 0;
    int2 ev = make_int2(0, 0);
    int pair = 0, t0 = 0, nleaf = 0;
    if (e < ne) {
        ev = edges[e];
        // the faces of this edge's own mesh pair form one tree
        pair = seg_of(segs, ecol, nseg, ev.x);
        seg_range(segs, fcol, pair, nfaces, t0, nleaf);
    }
    const bool active = e < ne && nleaf > 0;
    bool walked = false;  // by the warp's packet walk
    if constexpr (PACKET) {
        const unsigned full = 0xffffffffu;
        const unsigned act = __ballot_sync(full, active);
        const int leader = act ? __ffs(act) - 1 : 0;
        const int lt0 = __shfl_sync(full, t0, leader), lnl = __shfl_sync(full, nleaf, leader);
        if (act && __all_sync(full, !active || (t0 == lt0 && nleaf == lnl))) {
            walked = true;
            __shared__ int pstack[256 / 32][STACK];
            int *stk = pstack[threadIdx.x >> 5];
            const int lane = threadIdx.x & 31;
            T p[3] = {0, 0, 0}, q[3] = {0, 0, 0};
            float lo[3] = {1.f, 1.f, 1.f}, hi[3] = {0.f, 0.f, 0.f};  // empty for idle lanes
            if (active) {
                const int i0 = chk(ev.x, nv, status), i1 = chk(ev.y, nv, status);
                p[0] = ex[i0]; p[1] = ey[i0]; p[2] = ez[i0];
                q[0] = ex[i1]; q[1] = ey[i1]; q[2] = ez[i1];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    lo[k] = lo_f(p[k] < q[k] ? p[k] : q[k]);
                    hi[k] = hi_f(p[k] < q[k] ? q[k] : p[k]);
                }
            }
            const unsigned long long ebits = ((unsigned long long)e) << face_bits;
            int sp = 0;
            int node = lnl == 1 ? ~lt0 : lt0;
            int visits = 0;
            const int max_visits = 2 * lnl + 8;
            while (true) {
                if (++visits > max_visits) {
                    if (lane == 0) atomicOr(status, ST_BAD_INDEX);
                    break;
                }
                int leaf0 = -1, leaf1 = -1, next = -1, push = -1;
                bool m0 = false, m1 = false;
                if (node < 0) {
                    leaf0 = ~node;
                    m0 = active;
                } else {
                    const float4 *nd = nodes + 4 * node;
                    const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
                    const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
                    const bool h0 = active && overlap(lo, hi, n0.x, n0.y, n0.z, n0.w, n1.x, n1.y);
                    const bool h1 = active && overlap(lo, hi, n1.z, n1.w, n2.x, n2.y, n2.z, n2.w);
                    const bool a0 = __any_sync(full, h0), a1 = __any_sync(full, h1);
                    if (a0) {
                        if (c0 < 0) { leaf0 = ~c0; m0 = h0; } else next = c0;
                    }
                    if (a1) {
                        if (c1 < 0) { leaf1 = ~c1; m1 = h1; }
                        else if (next < 0) next = c1;
                        else push = c1;
                    }
                }
#pragma unroll
                for (int w = 0; w < 2; ++w) {
                    const int lf = w ? leaf1 : leaf0;
                    if (lf >= 0 && (w ? m1 : m0)) {
                        Leaf<T> L;
                        L.load(leaf_tri, lf);
                        ++tests;
                        bool hit;
                        if constexpr (NOINL) hit = leaf_test_call<T, F32F>(p, q, L, st);
                        else hit = leaf_test_body<T, F32F>(p, q, L, st);
                        if (hit) {
                            int pos = atomicAdd(count, 1);
                            if (pos < cap) out[pos] = dirbit | ebits | (unsigned)L.face;
                        }
                    }
                }
                __syncwarp();
                if (push >= 0) {
                    if (sp < STACK) {
                        if (lane == 0) stk[sp] = push;
                        ++sp;
                        __syncwarp();
                    } else if (lane == 0) {
                        atomicOr(status, ST_BAD_INDEX);  // unreachable: depth < 64
                    }
                }
                if (next >= 0) {
                    node = next;
                    continue;
                }
                if (sp == 0) break;
                node = stk[--sp];
            }
        }
    }
    if (active && !walked) {
        int i0 = chk(ev.x, nv, status), i1 = chk(ev.y, nv, status);
        T p[3] = {ex[i0], ey[i0], ez[i0]}, q[3] = {ex[i1], ey[i1], ez[i1]};
        float lo[3], hi[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lo[k] = lo_f(p[k] < q[k] ? p[k] : q[k]);
            hi[k] = hi_f(p[k] < q[k] ? q[k] : p[k]);
        }
        const unsigned long long ebits = ((unsigned long long)e) << face_bits;
        int stack[STACK];
        int sp = 0;
        int node = nleaf == 1 ? ~t0 : t0;
        // a tree of nleaf leaves has 2 nleaf - 1 nodes; each is visited at
        // most once per edge, so the bound only guards a corrupted tree
        int visits = 0;
        const int max_visits = 2 * nleaf + 8;
        while (true) {
            if (++visits > max_visits) {
                atomicOr(status, ST_BAD_INDEX);
                break;
            }
            int leaf0 = -1, leaf1 = -1;
            int next = -1, push = -1;
            if (node < 0) {
                leaf0 = ~node;
            } else {
                const float4 *nd = nodes + 4 * node;
                float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
                int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
                bool h0 = overlap(lo, hi, n0.x, n0.y, n0.z, n0.w, n1.x, n1.y);
                bool h1 = overlap(lo, hi, n1.z, n1.w, n2.x, n2.y, n2.z, n2.w);
                if (h0) { if (c0 < 0) leaf0 = ~c0; else next = c0; }
                if (h1) {
                    if (c1 < 0) leaf1 = ~c1;
                    else if (next < 0) next = c1;
                    else push = c1;
                }
            }
#pragma unroll
            for (int w = 0; w < 2; ++w) {
                int lf = w ? leaf1 : leaf0;
                if (lf >= 0) {
                    Leaf<T> L;
                    L.load(leaf_tri, lf);
                    ++tests;
                    bool hit;
                    if constexpr (NOINL) hit = leaf_test_call<T, F32F>(p, q, L, st);
                    else hit = leaf_test_body<T, F32F>(p, q, L, st);
                    if (hit) {
                        int pos = atomicAdd(count, 1);
                        if (pos < cap) out[pos] = dirbit | ebits | (unsigned)L.face;
                    }
                }
            }
            if (push >= 0) {
                if (sp < STACK) stack[sp++] = push;
                else atomicOr(status, ST_BAD_INDEX);  // unreachable: depth < 64
            }
            if (next >= 0) {
                node = next;
                continue;
            }
            if (sp == 0) break;
            node = stack[--sp];
        }
    }
    unsigned tot = __reduce_add_sync(0xffffffffu, tests);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(&st->narrow_tests, (unsigned long long)tot);
}

// ---------------------------------------------------------------------------
// Persistent traversal with a device work queue (variants 5 to 8): a grid
// of as many CTAs as fit on the GPU at once; every warp keeps its lanes
// busy by handing each lane whose walk has ended the next edge of the
// traversal order from one global counter (one atomic per refill, once at
// least FETCH lanes are idle).  Every lane then takes one node per step,
// so short walks (edges that leave at the root of their pair's tree) no
// longer idle their warp until its longest walk ends, and no CTA outlives
// the others with a few long walks.  Edges are handed out in the Morton
// order of their midpoints, so a warp still walks one region of a tree.
// The pairs and tests are exactly those of the per-edge walk.
// ---------------------------------------------------------------------------
template <typename T, bool F32F, int MINB, int FETCH>
__global__ void __launch_bounds__(256, MINB) k_traverse_q(
    const int2 *edges, const int *order, int ne, const T *ex, const T *ey, const T *ez, int nv,
    const float4 *nodes, const void *leaf_tri, int nfaces, const int *segs, int nseg, int ecol,
    int fcol, unsigned long long dirbit, int face_bits, unsigned long long *out, int *count, int cap,
    int *queue, DevStats *st, uint32_t *status) {
    HFCR_PDL_WAIT();
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    bool active = false, drained = false;
    int e = 0, node = 0, sp = 0, visits = 0, max_visits = 0;
    T p[3] = {0, 0, 0}, q[3] = {0, 0, 0};
    float lo[3] = {0.f, 0.f, 0.f}, hi[3] = {0.f, 0.f, 0.f};
    unsigned long long ebits = 0;
    int stack[STACK];
    unsigned tests = 0;
    while (true) {
        // refill the idle lanes from the queue (warp-uniform decision)
        const unsigned idle = __ballot_sync(full, !active);
        if (!drained && __popc(idle) >= (idle == full ? 1 : FETCH)) {
            const int leader = __ffs(idle) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(queue, __popc(idle));
            base = __shfl_sync(full, base, leader);
            if (base + __popc(idle) >= ne) drained = true;
            if (!active) {
                const int t = base + __popc(idle & below);
                if (t < ne) {
                    e = order ? order[t] : t;
                    const int2 ev = edges[e];
                    const int pair = seg_of(segs, ecol, nseg, ev.x);
                    int t0, nleaf;
                    seg_range(segs, fcol, pair, nfaces, t0, nleaf);
                    if (nleaf > 0) {
                        const int i0 = chk(ev.x, nv, status), i1 = chk(ev.y, nv, status);
                        p[0] = ex[i0]; p[1] = ey[i0]; p[2] = ez[i0];
                        q[0] = ex[i1]; q[1] = ey[i1]; q[2] = ez[i1];
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            lo[k] = lo_f(p[k] < q[k] ? p[k] : q[k]);
                            hi[k] = hi_f(p[k] < q[k] ? q[k] : p[k]);
                        }
                        ebits = ((unsigned long long)e) << face_bits;
                        node = nleaf == 1 ? ~t0 : t0;
                        sp = 0;
                        visits = 0;
                        // a tree of nleaf leaves has 2 nleaf - 1 nodes, each
                        // visited at most once per edge: the bound only guards
                        // a corrupted tree
                        max_visits = 2 * nleaf + 8;
                        active = true;
                    }
                }
            }
        }
        if (!__any_sync(full, active)) {
            if (drained) break;
            continue;  // every fetched edge had an empty pair; fetch again
        }
        if (!active) continue;
        // one step of this lane's walk
        if (++visits > max_visits) {
            atomicOr(status, ST_BAD_INDEX);
            active = false;
            continue;
        }
        int leaf0 = -1, leaf1 = -1, next = -1, push = -1;
        if (node < 0) {
            leaf0 = ~node;
        } else {
            const float4 *nd = nodes + 4 * node;
            const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
            const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
            const bool h0 = overlap(lo, hi, n0.x, n0.y, n0.z, n0.w, n1.x, n1.y);
            const bool h1 = overlap(lo, hi, n1.z, n1.w, n2.x, n2.y, n2.z, n2.w);
            if (h0) { if (c0 < 0) leaf0 = ~c0; else next = c0; }
            if (h1) {
                if (c1 < 0) leaf1 = ~c1;
                else if (next < 0) next = c1;
                else push = c1;
            }
        }
#pragma unroll
        for (int w = 0; w < 2; ++w) {
            const int lf = w ? leaf1 : leaf0;
            if (lf >= 0) {
                Leaf<T> L;
                L.load(leaf_tri, lf);
                ++tests;
                if (leaf_test_call<T, F32F>(p, q, L, st)) {
                    const int pos = atomicAdd(count, 1);
                    if (pos < cap) out[pos] = dirbit | ebits | (unsigned)L.face;
                }
            }
        }
        if (push >= 0) {
            if (sp < STACK) stack[sp++] = push;
            else atomicOr(status, ST_BAD_INDEX);  // unreachable: depth < 64
        }
        if (next >= 0) node = next;
        else if (sp > 0) node = stack[--sp];
        else active = false;
    }
    unsigned tot = __reduce_add_sync(full, tests);
    if (lane == 0 && tot) atomicAdd(&st->narrow_tests, (unsigned long long)tot);
}

__global__ void k_keys_to_pairs(const unsigned long long *keys, const int *d_n, int cap,
                                const int2 *edgesA, const int2 *edgesB, int edge_bits,
                                int face_bits, hfcr_pair *out) {
    HFCR_PDL_WAIT();
    int n = min(*d_n, cap);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long k = keys[i];
    unsigned dir = (unsigned)(k >> (edge_bits + face_bits));
    unsigned e = (unsigned)((k >> face_bits) & ((1ull << edge_bits) - 1));
    unsigned f = (unsigned)(k & ((1ull << face_bits) - 1));
    int2 ev = dir ? edgesB[e] : edgesA[e];
    out[i] = hfcr_pair{dir, (unsigned)ev.x, (unsigned)ev.y, f};
}

template <typename T>
__device__ __forceinline__ void ld3(const hfcr_mesh &m, int i, T *o) {
    o[0] = ((const T *)m.x)[i];
    o[1] = ((const T *)m.y)[i];
    o[2] = ((const T *)m.z)[i];
}

// x0 = the endpoint of the pair's edge on the back side of its face
// stencil key of the pair (dir, v0, v1, f): x0 = the endpoint of the edge on
// the back side of its face
template <typename T>
__device__ __forceinline__ unsigned long long stencil_key_of(const hfcr_mesh &A, const hfcr_mesh &B,
                                                             unsigned dir, unsigned pv0, unsigned pv1,
                                                             unsigned pf, int vert_bits, int face_bits,
                                                             int f32_filter, DevStats *st,
                                                             uint32_t *status) {
    const hfcr_mesh &E = dir ? B : A;
    const hfcr_mesh &F = dir ? A : B;
    int v0 = chk((int)pv0, E.n_verts, status), v1 = chk((int)pv1, E.n_verts, status);
    int f = chk((int)pf, F.n_tris, status);
    int ia = chk(F.tris[3 * f], F.n_verts, status), ib = chk(F.tris[3 * f + 1], F.n_verts, status),
        ic = chk(F.tris[3 * f + 2], F.n_verts, status);
    T a[3], b[3], c[3], p[3];
    ld3<T>(F, ia, a);
    ld3<T>(F, ib, b);
    ld3<T>(F, ic, c);
    ld3<T>(E, v0, p);
    int s = orient_full<T>(a, b, c, p, f32_filter, st);
    // a crossing pair has s != 0; a pair given by the caller with the first
    // endpoint on the plane keeps v1 (the crossing test would reject it)
    unsigned x0 = s < 0 ? (unsigned)v0 : (unsigned)v1;
    return ((unsigned long long)dir << (vert_bits + face_bits)) |
           ((unsigned long long)x0 << face_bits) | (unsigned long long)(unsigned)f;
}

template <typename T>
__global__ void k_stencil_keys(hfcr_mesh A, hfcr_mesh B, const hfcr_pair *pairs, const int *d_n,
                               int cap, int vert_bits, int face_bits, int f32_filter,
                               unsigned long long *keys, DevStats *st, uint32_t *status) {
    HFCR_PDL_WAIT();
    int n = min(*d_n, cap);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    hfcr_pair pr = pairs[i];
    unsigned dir = pr.dir ? 1u : 0u;
    if (pr.dir > 1u) atomicOr(status, ST_BAD_INDEX);
    keys[i] = stencil_key_of<T>(A, B, dir, pr.v0, pr.v1, pr.face, vert_bits, face_bits, f32_filter,
                                st, status);
}

// The same from the traversal's pair keys (dir | edge | face) as appended:
// the pair count is clamped here (more than cap: ST_CAPACITY and no pair;
// the clamped count to *d_eff for the kernels that follow)
template <typename T>
__global__ void k_stencil_keys_from_pair_keys(hfcr_mesh A, hfcr_mesh B,
                                              const unsigned long long *pkeys, const int *d_n,
                                              int cap, const int2 *edgesA, const int2 *edgesB,
                                              int edge_bits, int pface_bits, int vert_bits,
                                              int face_bits, int f32_filter,
                                              unsigned long long *keys, int *d_eff, DevStats *st,
                                              uint32_t *status) {
    HFCR_PDL_WAIT();
    int n = *d_n;
    if (n > cap) n = 0;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        if (*d_n > cap) atomicOr(status, ST_CAPACITY);
        *d_eff = n;
    }
    if (i >= n) return;
    const unsigned long long k = pkeys[i];
    const unsigned dir = (unsigned)(k >> (edge_bits + pface_bits));
    const int e = (int)((k >> pface_bits) & ((1ull << edge_bits) - 1));
    const unsigned f = (unsigned)(k & ((1ull << pface_bits) - 1));
    const int2 ev = dir ? edgesB[e] : edgesA[e];
    keys[i] = stencil_key_of<T>(A, B, dir, (unsigned)ev.x, (unsigned)ev.y, f, vert_bits, face_bits,
                                f32_filter, st, status);
}

__global__ void k_stencil_flags(const unsigned long long *keys, const int *d_n, int cap,
                                unsigned *flags) {
    HFCR_PDL_WAIT();
    int n = min(*d_n, cap);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flags[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

__global__ void k_stencil_write(const unsigned long long *keys, const unsigned *pos,
                                const int *d_n, int cap, int vert_bits, int face_bits,
                                hfcr_stencil *out) {
    HFCR_PDL_WAIT();
    int n = min(*d_n, cap);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (i == 0 || keys[i] != keys[i - 1]) {
        unsigned long long k = keys[i];
        hfcr_stencil s;
        s.dir = (unsigned)(k >> (vert_bits + face_bits));
        s.x0 = (unsigned)((k >> face_bits) & ((1ull << vert_bits) - 1));
        s.face = (unsigned)(k & ((1ull << face_bits) - 1));
        s.pad = 0;
        out[pos[i]] = s;
    }
}

// effective count = count when it fits the capacity, else 0 with
// ST_CAPACITY raised (so nothing downstream runs on a truncated set)
__device__ __forceinline__ int first_edge_from(const int2 *E, int ne, int v) {
    int lo = 0, hi = ne;  // first edge whose first vertex is >= v
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (E[mid].x < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void k_pair_products(const int2 *E, int ne, const int *segs, int nseg, int ecol, int fcol,
                                int nfaces, DevStats *st) {
    HFCR_PDL_WAIT();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (i < nseg) {
        int e0 = first_edge_from(E, ne, segs[4 * i + ecol]);
        int e1 = first_edge_from(E, ne, segs[4 * (i + 1) + ecol]);
        int f0, nf;
        seg_range(segs, fcol, i, nfaces, f0, nf);
        v = (unsigned long long)max(e1 - e0, 0) * (unsigned long long)nf;
    }
    v = __reduce_add_sync(0xffffffffu, (unsigned)(v & 0xffffffffu)) +
        ((unsigned long long)__reduce_add_sync(0xffffffffu, (unsigned)(v >> 32)) << 32);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&st->bf, v);
}

}  // namespace

void pair_products(const int *edges, int ne, const int *segs, int nseg, int ecol, int fcol,
                   int nfaces, DevStats *stats, cudaStream_t s) {
    if (ne <= 0 || nseg <= 0) return;
    { launch_pdl(k_pair_products, (nseg + 255) / 256, 256, 0, s, (const int2 *)edges, ne, segs,
                 nseg, ecol,
                                                        fcol, nfaces, stats); note_launch(); }
}

template <typename T, bool F32F, int MINB, bool NOINL, bool PACKET>
static void launch_traverse(const DetectArgs &a, const T *x, const T *y, const T *z, int nb,
                            unsigned long long dirbit, cudaStream_t s, uint32_t *d_status) {
    const hfcr_mesh &m = *a.edge_mesh;
    { launch_pdl(k_traverse<T, F32F, MINB, NOINL, PACKET>, nb, 256, 0, s, (const int2 *)a.edges,
                 a.order, a.n_edges, x, y, z, m.n_verts, a.bvh->nodes, a.bvh->leaf_tri,
          a.bvh->n, a.segs, a.nseg, a.ecol, a.fcol, dirbit, a.face_bits, a.keys, a.d_count, a.cap,
          a.stats, d_status); note_launch(); }
}

// resident CTAs of a persistent traversal kernel on this device (cached)
template <typename K>
static int resident_ctas(K kern) {
    static int dev_cache[64];
    static bool done[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 152;
    if (!done[dev]) {
        int sms = 0, per = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, 0);
        dev_cache[dev] = sms * (per > 0 ? per : 1);
        done[dev] = true;
    }
    return dev_cache[dev];
}

template <typename T, bool F32F, int MINB, int FETCH>
static void launch_queue(const DetectArgs &a, const T *x, const T *y, const T *z,
                         unsigned long long dirbit, cudaStream_t s, uint32_t *d_status) {
    const hfcr_mesh &m = *a.edge_mesh;
    auto kern = k_traverse_q<T, F32F, MINB, FETCH>;
    int grid = resident_ctas(kern);
    const int need = (a.n_edges + 255) / 256;
    if (grid > need) grid = need;
    cudaMemsetAsync(a.queue, 0, sizeof(int), s);
    { launch_pdl(kern, grid, 256, 0, s, (const int2 *)a.edges, a.order, a.n_edges, x, y, z,
                 m.n_verts, a.bvh->nodes, a.bvh->leaf_tri, a.bvh->n, a.segs, a.nseg, a.ecol, a.fcol,
                 dirbit, a.face_bits, a.keys, a.d_count, a.cap, a.queue, a.stats, d_status);
      note_launch(); }
}

template <typename T, bool F32F>
static void launch_variant(const DetectArgs &a, const T *x, const T *y, const T *z, int nb,
                           unsigned long long dirbit, cudaStream_t s, uint32_t *d_status) {
    switch (a.variant) {
        case 5: launch_queue<T, F32F, 3, 8>(a, x, y, z, dirbit, s, d_status); return;
        case 6: launch_queue<T, F32F, 4, 8>(a, x, y, z, dirbit, s, d_status); return;
        case 7: launch_queue<T, F32F, 3, 16>(a, x, y, z, dirbit, s, d_status); return;
        case 8: launch_queue<T, F32F, 4, 16>(a, x, y, z, dirbit, s, d_status); return;
        default: break;
    }
    switch (a.variant) {
        case 1: launch_traverse<T, F32F, 4, true, false>(a, x, y, z, nb, dirbit, s, d_status); break;
        case 2: launch_traverse<T, F32F, 3, true, false>(a, x, y, z, nb, dirbit, s, d_status); break;
        case 3: launch_traverse<T, F32F, 2, false, true>(a, x, y, z, nb, dirbit, s, d_status); break;
        case 4: launch_traverse<T, F32F, 4, true, true>(a, x, y, z, nb, dirbit, s, d_status); break;
        default: launch_traverse<T, F32F, 2, false, false>(a, x, y, z, nb, dirbit, s, d_status); break;
    }
}

void detect_launch(const DetectArgs &a, cudaStream_t s, uint32_t *d_status) {
    if (a.n_edges <= 0 || a.bvh->n <= 0) return;
    const hfcr_mesh &m = *a.edge_mesh;
    int nb = (a.n_edges + 255) / 256;
    unsigned long long dirbit = (unsigned long long)a.dir << (a.edge_bits + a.face_bits);
    if (m.dtype == HFCR_F32) {
        const float *x = (const float *)m.x, *y = (const float *)m.y, *z = (const float *)m.z;
        if (a.f32_filter) launch_variant<float, true>(a, x, y, z, nb, dirbit, s, d_status);
        else launch_variant<float, false>(a, x, y, z, nb, dirbit, s, d_status);
    } else {
        const double *x = (const double *)m.x, *y = (const double *)m.y, *z = (const double *)m.z;
        launch_variant<double, false>(a, x, y, z, nb, dirbit, s, d_status);
    }
}

void keys_to_pairs(const unsigned long long *keys, const int *d_n, int cap, const int *edgesA,
                   const int *edgesB, int edge_bits, int face_bits, hfcr_pair *out, cudaStream_t s) {
    if (cap <= 0) return;
    { launch_pdl(k_keys_to_pairs, (cap + 255) / 256, 256, 0, s, keys, d_n, cap,
                 (const int2 *)edgesA,
                                                      (const int2 *)edgesB, edge_bits, face_bits, out); note_launch(); }
}

void stencil_keys(const MeshPair &mp, const hfcr_pair *pairs, const int *d_n, int cap,
                  int vert_bits, int face_bits, int f32_filter, unsigned long long *keys,
                  DevStats *stats, uint32_t *d_status, cudaStream_t s) {
    if (cap <= 0) return;
    int nb = (cap + 255) / 256;
    if (mp.A.dtype == HFCR_F32)
        { launch_pdl(k_stencil_keys<float>, nb, 256, 0, s, mp.A, mp.B, pairs, d_n, cap, vert_bits,
                     face_bits,
                                                 f32_filter, keys, stats, d_status); note_launch(); }
    else
        { launch_pdl(k_stencil_keys<double>, nb, 256, 0, s, mp.A, mp.B, pairs, d_n, cap,
                     vert_bits, face_bits,
                                                  f32_filter, keys, stats, d_status); note_launch(); }
}

void stencil_keys_from_pair_keys(const MeshPair &mp, const unsigned long long *pkeys, const int *d_n,
                                 int cap, const int *edgesA, const int *edgesB, int edge_bits,
                                 int pface_bits, int vert_bits, int face_bits, int f32_filter,
                                 unsigned long long *keys, int *d_eff, DevStats *stats,
                                 uint32_t *d_status, cudaStream_t s) {
    if (cap <= 0) return;
    const int nb = (cap + 255) / 256;
    if (mp.A.dtype == HFCR_F32)
        launch_pdl(k_stencil_keys_from_pair_keys<float>, nb, 256, 0, s, mp.A, mp.B, pkeys, d_n, cap,
                   (const int2 *)edgesA, (const int2 *)edgesB, edge_bits, pface_bits, vert_bits,
                   face_bits, f32_filter, keys, d_eff, stats, d_status);
    else
        launch_pdl(k_stencil_keys_from_pair_keys<double>, nb, 256, 0, s, mp.A, mp.B, pkeys, d_n, cap,
                   (const int2 *)edgesA, (const int2 *)edgesB, edge_bits, pface_bits, vert_bits,
                   face_bits, f32_filter, keys, d_eff, stats, d_status);
    note_launch();
}

void stencil_unique(const unsigned long long *keys, const int *d_n, int cap, int vert_bits,
                    int face_bits, unsigned *flags, hfcr_stencil *out, int *d_k, SortTemp &t,
                    cudaStream_t s) {
    if (cap <= 0) return;
    int nb = (cap + 255) / 256;
    { launch_pdl(k_stencil_flags, nb, 256, 0, s, keys, d_n, cap, flags); note_launch(); }
    scan_flags_dev(flags, d_n, cap, d_k, t, s);
    { launch_pdl(k_stencil_write, nb, 256, 0, s, keys, flags, d_n, cap, vert_bits, face_bits,
                 out); note_launch(); }
}

}  // namespace hfcr
