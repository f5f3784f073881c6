// Diffusion of displacement vectors (Sec. 5): the correction the minimizer
// gives the stencil vertices is spread over their vicinity as a harmonic
// vector field, so that the mesh moves smoothly instead of only at the
// penetrating vertices.  The paper names constrained diffusion without
// equations; the reading implemented here, per mesh: vertices with a
// nonzero displacement keep it (Dirichlet values), vertices more than R
// edges away and kinematic vertices (inverse mass 0) keep zero, and every
// vertex in between (the band) is the mean of its neighbours, i.e. the
// band's graph Laplacian system
//     deg(v) u_v - sum of u_w over band neighbours w
//         = sum of the Dirichlet values of v's other neighbours
// is solved for each coordinate, by Jacobi-preconditioned conjugate
// gradients to a relative residual `tol` (k_band_cl on one thread-block
// cluster for bands of up to some 27,000 vertices, k_band_cg over the whole
// grid beyond).  The older fixed-sweep form (S Jacobi sweeps of
// the neighbour mean from zero, whose limit is that field) stays available
// as a named approximation.
//
// Layout: the field u is float64 AoS (x, y, z per vertex) over the global
// vertex numbering of the pair (A's vertices, then B's), so that a
// neighbour read is one 24-byte load.  Each mesh's vertex adjacency is a
// CSR with ascending neighbours, built from its sorted edge list.  The
// band's vertices are compacted into a list (a flag scan), and the CG state
// of band vertex i is one 96-byte record (r, w, s per coordinate, 1/deg and
// its range of neighbour slots) in one of two buffers that alternate by
// iteration.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cfloat>

#include <cooperative_groups.h>

#include "internal.h"
#include "sortdev.cuh"

namespace hfcr {

namespace {

__global__ void k_adj_count(const int2 *edges, int ne, int nv, int *deg, uint32_t *st) {
    HFCR_PDL_WAIT();
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const int2 ed = edges[e];
    if ((unsigned)ed.x >= (unsigned)nv || (unsigned)ed.y >= (unsigned)nv) {
        atomicOr(st, ST_BAD_INDEX);
        return;
    }
    atomicAdd(&deg[ed.x], 1);
    atomicAdd(&deg[ed.y], 1);
}

__global__ void k_adj_fill(const int2 *edges, int ne, int nv, const int *ptr, int *cur, int *nbr) {
    HFCR_PDL_WAIT();
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const int2 ed = edges[e];
    if ((unsigned)ed.x >= (unsigned)nv || (unsigned)ed.y >= (unsigned)nv) return;
    nbr[ptr[ed.x] + atomicAdd(&cur[ed.x], 1)] = ed.y;
    nbr[ptr[ed.y] + atomicAdd(&cur[ed.y], 1)] = ed.x;
}

// ascending order within each vertex's list (the fill order is arbitrary)
__global__ void k_adj_sort(const int *ptr, int nv, int *nbr) {
    HFCR_PDL_WAIT();
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const int a = ptr[v], b = ptr[v + 1];
    for (int i = a + 1; i < b; ++i) {
        const int x = nbr[i];
        int j = i - 1;
        while (j >= a && nbr[j] > x) {
            nbr[j + 1] = nbr[j];
            --j;
        }
        nbr[j + 1] = x;
    }
}

struct DMesh {
    const int *ptr = nullptr, *nbr = nullptr;
    const float *inv_mass = nullptr;
    const int *rank = nullptr;  // place of each vertex in the band list's order (null: identity)
    int n = 0, off = 0;
};
struct DPair {
    DMesh m[2];
    int ntot = 0;
    __device__ __forceinline__ const DMesh &of(int g) const { return g >= m[1].off ? m[1] : m[0]; }
};

__global__ void k_ring_init(DPair P, const double *u, int *ring, int far) {
    HFCR_PDL_WAIT();
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P.ntot) return;
    const double *x = u + 3 * (size_t)g;
    ring[g] = (x[0] != 0.0 || x[1] != 0.0 || x[2] != 0.0) ? 0 : far;
}

// breadth-first level r: every vertex at level r - 1 gives level r to its
// neighbours not reached yet (levels r - 1 and below no longer change; all
// writers of a vertex write the same r, and a vertex reached in this step is
// not read as a source of it)
__global__ void k_ring_step(DPair P, int *ring, int r, int far) {
    HFCR_PDL_WAIT();
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P.ntot || ring[g] != r - 1) return;
    const DMesh &M = P.of(g);
    const int v = g - M.off;
    for (int e = M.ptr[v]; e < M.ptr[v + 1]; ++e) {
        const int w = M.off + M.nbr[e];
        if (ring[w] == far) ring[w] = r;
    }
}

// one Jacobi sweep: band vertices (1 <= ring <= R, not kinematic) take the
// neighbour mean; every other vertex keeps its value
__global__ void k_sweep(DPair P, const int *ring, int R, const double *uin, double *uout) {
    HFCR_PDL_WAIT();
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P.ntot) return;
    const DMesh &M = P.of(g);
    const int v = g - M.off;
    const int rg = ring[g];
    const bool free = rg >= 1 && rg <= R && !(M.inv_mass && M.inv_mass[v] == 0.f);
    double a0, a1, a2;
    if (free) {
        a0 = a1 = a2 = 0.0;
        const int e0 = M.ptr[v], e1 = M.ptr[v + 1];
        for (int e = e0; e < e1; ++e) {
            const double *w = uin + 3 * (size_t)(M.off + M.nbr[e]);
            a0 += w[0];
            a1 += w[1];
            a2 += w[2];
        }
        const double deg = (double)(e1 - e0);
        a0 /= deg;
        a1 /= deg;
        a2 /= deg;
    } else {
        const double *w = uin + 3 * (size_t)g;
        a0 = w[0];
        a1 = w[1];
        a2 = w[2];
    }
    double *o = uout + 3 * (size_t)g;
    o[0] = a0;
    o[1] = a1;
    o[2] = a2;
}

template <typename T>
__device__ __forceinline__ void add_to(void *p, int i, double d) {
    T *q = (T *)p + i;
    *q = (T)((double)*q + d);
}

// x' = x + u on the vertices within R rings (u is zero elsewhere)
__global__ void k_apply_field(hfcr_mesh A, hfcr_mesh B, const int *ring, int R, const double *u,
                              int ntot) {
    HFCR_PDL_WAIT();
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ntot) return;
    const int rg = ring[g];
    if (rg < 0 || rg > R) return;
    const bool inA = g < A.n_verts;
    const hfcr_mesh &m = inA ? A : B;
    const int v = inA ? g : g - A.n_verts;
    const double *w = u + 3 * (size_t)g;
    if (m.dtype == HFCR_F32) {
        add_to<float>(m.x, v, w[0]);
        add_to<float>(m.y, v, w[1]);
        add_to<float>(m.z, v, w[2]);
    } else {
        add_to<double>(m.x, v, w[0]);
        add_to<double>(m.y, v, w[1]);
        add_to<double>(m.z, v, w[2]);
    }
}

__global__ void k_soa_to_aos(const double *x, const double *y, const double *z, int n, double *u) {
    HFCR_PDL_WAIT();
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    u[3 * (size_t)v] = x[v];
    u[3 * (size_t)v + 1] = y[v];
    u[3 * (size_t)v + 2] = z[v];
}

__global__ void k_aos_to_soa(const double *u, int n, double *x, double *y, double *z) {
    HFCR_PDL_WAIT();
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    x[v] = u[3 * (size_t)v];
    y[v] = u[3 * (size_t)v + 1];
    z[v] = u[3 * (size_t)v + 2];
}

// ---- the harmonic field: CG on the band's graph Laplacian ----

constexpr int BAND_TPB = 256;
constexpr int BAND_MIN_PER_CTA = 32;     // band vertices per CTA taking part, at least
constexpr int BAND_REC = 12;             // floats per record: r[3] w[3] s[3] 1/deg, first / end slot
constexpr float BAND_INNER_TOL = 1e-5f;  // residual reduction of one float32 round
constexpr int BAND_MAX_ROUNDS = 32;
constexpr long long BAND_SPIN_LIMIT = 1ll << 22;

__device__ __forceinline__ bool band_vertex(const DPair &P, const int *ring, int R, int g) {
    const int rg = ring[g];
    if (rg < 1 || rg > R) return false;
    const DMesh &M = P.of(g);
    return !(M.inv_mass && M.inv_mass[g - M.off] == 0.f);
}

// place of global vertex g in the band list's order: its mesh's offset
// plus its rank there (the Morton order of the positions, where given)
__device__ __forceinline__ int band_slot(const DPair &P, int g) {
    const DMesh &M = P.of(g);
    return M.rank ? M.off + M.rank[g - M.off] : g;
}

// flag of every vertex at its slot: 1 in the band (scanned in place into the
// compact index), then the list of band vertices and the vertex -> index map
__global__ void k_band_flags(DPair P, const int *ring, int R, unsigned *flags) {
    HFCR_PDL_WAIT();
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < P.ntot) flags[band_slot(P, g)] = band_vertex(P, ring, R, g) ? 1u : 0u;
}

__global__ void k_band_list(DPair P, const int *ring, int R, const unsigned *pos, int *cidx,
                            int *fv) {
    HFCR_PDL_WAIT();
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P.ntot) return;
    if (band_vertex(P, ring, R, g)) {
        const unsigned i = pos[band_slot(P, g)];
        cidx[g] = (int)i;
        fv[i] = g;
    } else {
        cidx[g] = -1;
    }
}

// ---- the Morton rank of a mesh's vertices (once per kept adjacency) ----

// float -> int with the same order (for atomicMin / atomicMax)
__device__ __forceinline__ int ordered_int(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ordered_float(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

template <typename T>
__global__ void k_rank_bounds(const T *x, const T *y, const T *z, int n, int *box) {
    HFCR_PDL_WAIT();
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const float c[3] = {(float)x[v], (float)y[v], (float)z[v]};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lo[k] = fminf(lo[k], c[k]);
            hi[k] = fmaxf(hi[k], c[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        for (int o = 16; o; o >>= 1) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            atomicMin(box + k, ordered_int(lo[k]));
            atomicMax(box + 3 + k, ordered_int(hi[k]));
        }
    }
}

__device__ __forceinline__ unsigned spread3(unsigned v) {  // 10 bits -> every third of 30
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

template <typename T>
__global__ void k_rank_keys(const T *x, const T *y, const T *z, int n, const int *box,
                            unsigned long long *keys, int *vals) {
    HFCR_PDL_WAIT();
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const float c[3] = {(float)x[v], (float)y[v], (float)z[v]};
    unsigned q[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float lo = ordered_float(box[k]), hi = ordered_float(box[3 + k]);
        const float ext = hi - lo;
        float t = ext > 0.f ? (c[k] - lo) / ext : 0.f;  // NaN coordinates fall to cell 0
        t = t > 0.f ? (t < 1.f ? t : 1.f) : 0.f;
        const unsigned cell = (unsigned)(t * 1023.f);
        q[k] = cell > 1023u ? 1023u : cell;
    }
    keys[v] = (unsigned long long)(spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2));
    vals[v] = v;
}

__global__ void k_rank_box_init(int *box) {
    HFCR_PDL_WAIT();
    if (threadIdx.x < 6) box[threadIdx.x] = threadIdx.x < 3 ? 0x7fffffff : (int)0x80000000;
}

__global__ void k_rank_scatter(const int *vals, int n, int *rank) {
    HFCR_PDL_WAIT();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) rank[vals[i]] = i;
}

struct BandArgs {
    DPair P;
    const int *cidx;     // [ntot] index of a band vertex in fv, -1 elsewhere
    const int *fv;       // [nfree] global id of each band vertex
    const int *d_nfree;
    double *u;           // field: Dirichlet values in; the band's solution written at the end
    double *b64;         // [cap][3] right-hand side (Dirichlet sums), float64
    double *u64;         // [2][cap][3] float64 solution, alternating by round
    float *x32, *p32;    // [cap][3] the float32 correction of the round and its search direction
    float *rec;          // [2][cap][BAND_REC] float32 CG records, alternating by iteration
    int *cnbr;           // band index of every adjacency slot (-1: Dirichlet), slots of
    int eoffB;           //   mesh B from eoffB on
    double *part;        // [2][grid][9] per-CTA partial sums (doubles, or floats in the same space)
    unsigned *bar;       // grid barrier counter, zeroed before the launch
    int *ctl;            // [0] CG iterations run, [1] set when a coordinate stopped unconverged
    uint32_t *status;
    double tol;
    int max_iters;
    int cap;
};

// Barrier of the `parts` CTAs taking part: an arrival counter, polled
// without sleeping first (these waits are microseconds), bounded all the
// same: after the spin limit the CTA records ST_TIMEOUT and every CTA
// that sees it leaves (the caller then reports HFCR_ERR_TIMEOUT).
__device__ __forceinline__ bool band_barrier(unsigned *bar, unsigned target, uint32_t *status) {
    __shared__ int failed;
    __syncthreads();
    if (threadIdx.x == 0) {
        failed = 0;
        // arrival: a release reduction (this CTA's writes, ordered before
        // the barrier by __syncthreads, become visible with it)
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
        long long spins = 0;
        while (true) {
            unsigned seen;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(seen) : "l"(bar) : "memory");
            if (seen >= target) break;
            if (++spins > BAND_SPIN_LIMIT) {
                atomicOr(status, ST_TIMEOUT);
                failed = 1;
                break;
            }
            if ((spins & 255) == 0) {
                if (*(volatile uint32_t *)status & ST_TIMEOUT) { failed = 1; break; }
                __nanosleep(64);
            }
        }
    }
    __syncthreads();
    return failed == 0;
}

// the nine sums of this CTA's threads to part[9 blockIdx.x ...], fixed
// order (T float in the inner iterations: float64 arithmetic is scarce on
// GB300; double for the float64 residual of a round)
template <typename T>
__device__ __forceinline__ void band_cta_partials(const T *v, T *part) {
    __shared__ T sh[BAND_TPB / 32][9];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        T t = v[k];
#pragma unroll
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sh[w][k] = t;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        T t = 0;
        for (int q = 0; q < BAND_TPB / 32; ++q) t += sh[q][threadIdx.x];
        part[9 * blockIdx.x + threadIdx.x] = t;
    }
}

// the grid's nine sums from the partials of the `parts` CTAs (written
// before the barrier): warp w folds sums w and w + 8, lanes striding over
// the CTAs; the fixed order makes the result identical in every CTA
template <typename T>
__device__ __forceinline__ void band_grid_sums(const T *part, int parts, T *out) {
    __shared__ T sh[9];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = w; k < 9; k += BAND_TPB / 32) {
        T t = 0;
        for (int c = lane; c < parts; c += 32) t += __ldcg(part + 9 * c + k);
#pragma unroll
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sh[k] = t;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 9; ++k) out[k] = sh[k];
    __syncthreads();
}

// one float32 record (48 B): r[3] w[3] s[3] 1/deg, then the first and end
// adjacency slot; read through L2 (written by another CTA before the last
// barrier; an L1 line of an earlier use of the buffer may be stale)
struct BandRec {
    float r[3], w[3], s[3], id;
    int e0, e1;
};
__device__ __forceinline__ BandRec band_load(const float *rec) {
    const float4 *q = (const float4 *)rec;
    const float4 a = __ldcg(q), b = __ldcg(q + 1), c = __ldcg(q + 2);
    BandRec t;
    t.r[0] = a.x; t.r[1] = a.y; t.r[2] = a.z; t.w[0] = a.w;
    t.w[1] = b.x; t.w[2] = b.y; t.s[0] = b.z; t.s[1] = b.w;
    t.s[2] = c.x; t.id = c.y; t.e0 = __float_as_int(c.z); t.e1 = __float_as_int(c.w);
    return t;
}
__device__ __forceinline__ void band_store(float *rec, const float *r, const float *w,
                                           const float *s, float id, int e0, int e1) {
    float4 *q = (float4 *)rec;
    q[0] = make_float4(r[0], r[1], r[2], w[0]);
    q[1] = make_float4(w[1], w[2], s[0], s[1]);
    q[2] = make_float4(s[2], id, __int_as_float(e0), __int_as_float(e1));
}

// The band's Laplacian system L u = b (three right-hand sides, the
// coordinates) by iterative refinement: each round solves L e = r for the
// float64 residual r = b - L u with Jacobi-preconditioned CG in float32
// (the Laplacian's entries, deg and -1, are exact in float32; the
// Chronopoulos-Gear form, one reduction per iteration) to a reduction of
// BAND_INNER_TOL, then u += e and the residual is recomputed in float64;
// until |r| <= tol |b| per coordinate.  GB300's float64 rate is a small
// fraction of its float32 rate, so only the residual runs in float64.
//
// Iteration i of a round reads the record (r_i, w_i = L z_i, s_{i-1}) of
// every band vertex from buffer i mod 2 and writes (r_{i+1}, w_{i+1}, s_i)
// of its own vertices to the other; the neighbours' z_{i+1} = (r_i -
// alpha (w_i + beta s_{i-1})) / deg that w_{i+1} needs are recomputed from
// their records, so an iteration has one grid-wide barrier (its
// reduction).  A round's end computes u_new = u + e of its own vertices
// and the float64 residual from the neighbours' u and e as they stand, so
// it needs no barrier of its own either.  Band vertex i belongs to CTA i
// mod parts, so the band spreads over every CTA taking part (the float64
// work included); the neighbours' band indices are resolved once (cnbr).
// sum over the band neighbours j (slots e0 .. e1) of f(record j), the
// records fetched eight at a time so that their loads are in flight
// together (the neighbour loop is otherwise a chain of dependent L2 loads)
template <class F>
__device__ __forceinline__ void band_neighbours(const float *recs, const int *cnbr, int e0, int e1,
                                                F f) {
    constexpr int B = 8;
    for (int base = e0; base < e1; base += B) {
        int js[B];
#pragma unroll
        for (int k = 0; k < B; ++k) js[k] = base + k < e1 ? cnbr[base + k] : -1;
        float4 q0[B], q1[B];
        float2 q2[B];
#pragma unroll
        for (int k = 0; k < B; ++k)
            if (js[k] >= 0) {
                const float *r = recs + (size_t)BAND_REC * js[k];
                q0[k] = __ldcg((const float4 *)r);
                q1[k] = __ldcg((const float4 *)r + 1);
                q2[k] = __ldcg((const float2 *)(r + 8));
            }
#pragma unroll
        for (int k = 0; k < B; ++k)
            if (js[k] >= 0) {
                BandRec t;
                t.r[0] = q0[k].x; t.r[1] = q0[k].y; t.r[2] = q0[k].z; t.w[0] = q0[k].w;
                t.w[1] = q1[k].x; t.w[2] = q1[k].y; t.s[0] = q1[k].z; t.s[1] = q1[k].w;
                t.s[2] = q2[k].x; t.id = q2[k].y; t.e0 = t.e1 = 0;
                f(t);
            }
    }
}

// The band's Laplacian system L u = b (three right-hand sides, the
// coordinates) by iterative refinement: each round solves L e = r for the
// float64 residual r = b - L u with Jacobi-preconditioned CG in float32
// (the Laplacian's entries, deg and -1, are exact in float32; the
// Chronopoulos-Gear form, one reduction per iteration) to a reduction of
// BAND_INNER_TOL, then u += e and the residual is recomputed in float64;
// until |r| <= tol |b| per coordinate.  GB300's float64 rate is a small
// fraction of its float32 rate, so only the residual (and its norm) runs
// in float64; the inner iterations reduce in float32.
//
// Iteration i of a round reads the record (r_i, w_i = L z_i, s_{i-1}) of
// every band vertex from buffer i mod 2 and writes (r_{i+1}, w_{i+1}, s_i)
// of its own vertices to the other; the neighbours' z_{i+1} = (r_i -
// alpha (w_i + beta s_{i-1})) / deg that w_{i+1} needs are recomputed from
// their records, so an iteration has one grid-wide barrier (its
// reduction).  A round's end computes u_new = u + e of its own vertices
// and the float64 residual from the neighbours' u and e as they stand, so
// it needs no barrier of its own either.  Band vertex i belongs to CTA i
// mod parts, so the band spreads over every CTA taking part; the
// neighbours' band indices are resolved once (cnbr).  All reductions run
// in a fixed order, so the result is deterministic.  This kernel takes the
// bands larger than the cluster kernel (k_band_cl) holds.
__global__ void __launch_bounds__(BAND_TPB) k_band_cg(BandArgs a, int limit) {
    HFCR_PDL_WAIT();
    const int n = *a.d_nfree;
    if (n <= limit) return;  // the cluster kernel's band
    int parts = (n + BAND_MIN_PER_CTA - 1) / BAND_MIN_PER_CTA;
    parts = parts < 1 ? 1 : (parts > (int)gridDim.x ? (int)gridDim.x : parts);
    if ((int)blockIdx.x >= parts) return;
    const int i0 = blockIdx.x + parts * threadIdx.x, stride = parts * BAND_TPB;
    unsigned epoch = 0;
    float *R0 = a.rec, *R1 = a.rec + (size_t)BAND_REC * a.cap;
    double *U0 = a.u64, *U1 = a.u64 + 3 * (size_t)a.cap;
    // partial sums: [2][grid][9] doubles, or as floats in the same space
    double *const pd0 = a.part, *const pd1 = a.part + (size_t)9 * gridDim.x;
    double dl[9], ds[9];
    float fl[9], fs[9];
    // the right-hand side (Dirichlet values of the neighbours outside the
    // band), the neighbours' band indices, the first round's records
    // (r = b, since u = 0), |b|^2
#pragma unroll
    for (int k = 0; k < 9; ++k) dl[k] = 0.0;
    for (int i = i0; i < n; i += stride) {
        const int g = a.fv[i];
        const bool inB = g >= a.P.m[1].off;
        const DMesh &M = inB ? a.P.m[1] : a.P.m[0];
        const int v = g - M.off;
        const int e0 = M.ptr[v], e1 = M.ptr[v + 1];
        const int s0 = (inB ? a.eoffB : 0) + e0;
        double b[3] = {0.0, 0.0, 0.0};
        for (int e = e0; e < e1; ++e) {
            const int w = M.off + M.nbr[e];
            const int j = a.cidx[w];
            a.cnbr[s0 + e - e0] = j;
            if (j < 0) {
                const double *uw = a.u + 3 * (size_t)w;
                b[0] += uw[0];
                b[1] += uw[1];
                b[2] += uw[2];
            }
        }
        const float rb[3] = {(float)b[0], (float)b[1], (float)b[2]}, z3[3] = {0.f, 0.f, 0.f};
        // a band vertex has a neighbour one ring closer, so e1 > e0
        band_store(R0 + (size_t)BAND_REC * i, rb, z3, z3, 1.0f / (float)(e1 - e0), s0,
                   s0 + e1 - e0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a.b64[3 * (size_t)i + c] = b[c];
            U0[3 * (size_t)i + c] = 0.0;
            a.x32[3 * (size_t)i + c] = 0.f;
            a.p32[3 * (size_t)i + c] = 0.f;
            dl[6 + c] += b[c] * b[c];
        }
    }
    int pb = 0;  // parity of the partials buffer
    band_cta_partials(dl, (pb ? pd1 : pd0));
    if (!band_barrier(a.bar, parts * ++epoch, a.status)) return;
    band_grid_sums((pb ? pd1 : pd0), parts, ds);
    pb ^= 1;
    double target[3];
    bool act[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        target[c] = a.tol * a.tol * ds[6 + c];
        act[c] = ds[6 + c] > 0.0;
    }
    int it = 0, rounds = 0;
    int ub = 0;  // U buffer holding the current float64 solution
    int rb = 0;  // record buffer of the current iteration
    bool fail = false;
    while (act[0] || act[1] || act[2]) {
        if (++rounds > BAND_MAX_ROUNDS) { fail = true; break; }
        // ---- a round: w_0 = L z_0 and the first sums ----
        const float *cur = rb ? R1 : R0;
#pragma unroll
        for (int k = 0; k < 9; ++k) fl[k] = 0.f;
        for (int i = i0; i < n; i += stride) {
            float *rec = (rb ? R1 : R0) + (size_t)BAND_REC * i;
            const BandRec me = band_load(rec);
            float w[3] = {me.r[0], me.r[1], me.r[2]};
            band_neighbours(cur, a.cnbr, me.e0, me.e1, [&](const BandRec &nb) {
#pragma unroll
                for (int c = 0; c < 3; ++c) w[c] -= nb.r[c] * nb.id;
            });
            // only w changes (the neighbours read r and 1/deg of this record)
            rec[3] = w[0];
            rec[4] = w[1];
            rec[5] = w[2];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                a.x32[3 * (size_t)i + c] = 0.f;
                a.p32[3 * (size_t)i + c] = 0.f;
                fl[c] += me.r[c] * me.r[c] * me.id;   // gamma = (r, z)
                fl[3 + c] += w[c] * me.r[c] * me.id;  // delta = (w, z)
                fl[6 + c] += me.r[c] * me.r[c];       // rho = |r|^2
            }
        }
        band_cta_partials(fl, (float *)(pb ? pd1 : pd0));
        if (!band_barrier(a.bar, parts * ++epoch, a.status)) return;
        band_grid_sums((float *)(pb ? pd1 : pd0), parts, fs);
        pb ^= 1;
        float gam[3], alp[3], bet[3], stop[3];
        bool in[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            gam[c] = fs[c];
            alp[c] = fs[c] / fs[3 + c];
            bet[c] = 0.f;
            stop[c] = BAND_INNER_TOL * BAND_INNER_TOL * fs[6 + c];
            in[c] = act[c] && fs[6 + c] > 0.f && alp[c] > 0.f && isfinite(alp[c]);
        }
        // ---- inner float32 iterations ----
        const int it_round = it;
        while ((in[0] || in[1] || in[2]) && it < a.max_iters) {
            const float *cr = rb ? R1 : R0;
            float *nx = rb ? R0 : R1;
#pragma unroll
            for (int k = 0; k < 9; ++k) fl[k] = 0.f;
            for (int i = i0; i < n; i += stride) {
                const BandRec me = band_load(cr + (size_t)BAND_REC * i);
                float rn[3], sn[3], wn[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (in[c]) {
                        const float pn = me.r[c] * me.id + bet[c] * a.p32[3 * (size_t)i + c];
                        sn[c] = me.w[c] + bet[c] * me.s[c];
                        a.p32[3 * (size_t)i + c] = pn;
                        a.x32[3 * (size_t)i + c] += alp[c] * pn;
                        rn[c] = me.r[c] - alp[c] * sn[c];
                        wn[c] = rn[c];  // deg_v z_{i+1, v}
                    } else {
                        sn[c] = me.s[c];
                        rn[c] = me.r[c];
                        wn[c] = me.w[c];
                    }
                }
                band_neighbours(cr, a.cnbr, me.e0, me.e1, [&](const BandRec &nb) {
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        if (in[c]) wn[c] -= (nb.r[c] - alp[c] * (nb.w[c] + bet[c] * nb.s[c])) * nb.id;
                });
                band_store(nx + (size_t)BAND_REC * i, rn, wn, sn, me.id, me.e0, me.e1);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    fl[c] += rn[c] * rn[c] * me.id;
                    fl[3 + c] += wn[c] * rn[c] * me.id;
                    fl[6 + c] += rn[c] * rn[c];
                }
            }
            rb ^= 1;
            ++it;
            band_cta_partials(fl, (float *)(pb ? pd1 : pd0));
            if (!band_barrier(a.bar, parts * ++epoch, a.status)) return;
            band_grid_sums((float *)(pb ? pd1 : pd0), parts, fs);
            pb ^= 1;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (!in[c]) continue;
                if (fs[6 + c] <= stop[c]) { in[c] = false; continue; }
                const float b = fs[c] / gam[c];
                const float al = fs[c] / (fs[3 + c] - b * fs[c] / alp[c]);
                if (!(al > 0.f && isfinite(al))) { in[c] = false; continue; }
                bet[c] = b;
                alp[c] = al;
                gam[c] = fs[c];
            }
        }
        // ---- the round's end: u += e, the float64 residual, the next
        // round's records (r = the residual, s = 0; w follows) ----
        const double *Uc = ub ? U1 : U0;
        double *Un = ub ? U0 : U1;
        const float *nr = rb ? R1 : R0;   // the records last written
#pragma unroll
        for (int k = 0; k < 9; ++k) dl[k] = 0.0;
        for (int i = i0; i < n; i += stride) {
            const BandRec me = band_load(nr + (size_t)BAND_REC * i);
            double un[3], r64[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                un[c] = __ldcg(Uc + 3 * (size_t)i + c) + (double)__ldcg(a.x32 + 3 * (size_t)i + c);
                r64[c] = a.b64[3 * (size_t)i + c] - (double)(me.e1 - me.e0) * un[c];
            }
            for (int e = me.e0; e < me.e1; ++e) {
                const int j = a.cnbr[e];
                if (j < 0) continue;
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    r64[c] += __ldcg(Uc + 3 * (size_t)j + c) + (double)__ldcg(a.x32 + 3 * (size_t)j + c);
            }
            float rf[3];
            const float z3[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                Un[3 * (size_t)i + c] = un[c];
                rf[c] = act[c] ? (float)r64[c] : 0.f;
                dl[6 + c] += r64[c] * r64[c];
            }
            // written to the buffer the last iteration read: every CTA has
            // passed the barrier after that read
            band_store((rb ? R0 : R1) + (size_t)BAND_REC * i, rf, z3, z3, me.id, me.e0, me.e1);
        }
        band_cta_partials(dl, (pb ? pd1 : pd0));
        if (!band_barrier(a.bar, parts * ++epoch, a.status)) return;
        band_grid_sums((pb ? pd1 : pd0), parts, ds);
        pb ^= 1;
        ub ^= 1;
        rb ^= 1;
        bool progress = false;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (!act[c]) continue;
            if (ds[6 + c] <= target[c]) { act[c] = false; continue; }
            progress = true;
        }
        if (progress && (it >= a.max_iters || it == it_round)) { fail = true; break; }
    }
    const double *Uf = ub ? U1 : U0;
    for (int i = i0; i < n; i += stride) {
        double *ug = a.u + 3 * (size_t)a.fv[i];
#pragma unroll
        for (int c = 0; c < 3; ++c) ug[c] = __ldcg(Uf + 3 * (size_t)i + c);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl[0] += it;
        if (fail) a.ctl[1] = 1;
    }
}

// ---- the band on one thread-block cluster ----
//
// The same refinement rounds and Chronopoulos-Gear iterations as k_band_cg
// on one cluster of BCL_THREADS-thread CTAs, for bands of up to `limit`
// vertices (the bands of a frame sequence are a few thousand to a few tens
// of thousands of vertices: one grid-wide barrier per iteration over every
// SM costs more than the iteration's work).  Band vertex i belongs to CTA
// i / chunk and keeps its CG state in that CTA's shared memory, one array
// per field so that a warp's own-vertex accesses are conflict-free: r with
// 1/deg, p, s, x, w, z (float4), its neighbour codes, the float64 u of the
// rounds.
// Each neighbour slot of cnbr holds -2 - (local index) for a neighbour of
// the same CTA (read from shared memory), the band index for one of
// another CTA, -1 for a Dirichlet neighbour.  Other CTAs' values are read
// from global copies (z as float4 in rec, u in u64) that every vertex
// writes beside its record, through L2: random reads of other SMs' shared
// memory serialise on the SM-to-SM network, L2 serves them in parallel.
// The preconditioner is local to each CTA: z_v = (r_v + theta sum r_u /
// deg_u) / deg_v over v's band neighbours u in the same CTA, that is
// D^-1 (I + theta N D^-1) with N the adjacency inside the CTAs' blocks: one
// Jacobi sweep on each CTA's block after the first, symmetric, and
// positive definite for theta < 1 (the eigenvalues of D^-1/2 N D^-1/2 lie
// in [-1, 1] since deg counts every neighbour).  It needs only this CTA's
// r, so it costs a CTA barrier, not a cluster barrier, and takes about a
// quarter fewer iterations than Jacobi on the bands of a frame sequence.
// An iteration has two cluster barriers (the neighbours' z, then the
// sums); every CTA stores its sums into every CTA's receive slots before
// the second, and each folds them in rank order after it, so every CTA
// takes the same decisions from the same values.  Hardware cluster
// barriers: nothing here spins.
namespace cgx = cooperative_groups;

constexpr int BCL_THREADS = 1024;
constexpr int BCL_MAX = 16;                  // CTAs per cluster at most
constexpr int BCL_SMEM = 220 * 1024;  // dynamic shared memory per CTA
constexpr int BCL_NB = 8;             // neighbour codes kept in shared memory per vertex
// r p s x w z (float4), the neighbour codes, the float64 u, slot range
constexpr int BCL_VBYTES = 6 * 16 + 4 * BCL_NB + 24 + 8;
constexpr int BCL_VCAP = BCL_SMEM / BCL_VBYTES;  // band vertices per CTA (1,408)
constexpr float BCL_THETA = 0.9f;            // weight of the preconditioner's local sweep


struct BclState {
    float recv[2][BCL_MAX][9];    // the CTAs' float sums, by parity and sender
    double recvd[2][BCL_MAX][3];  // their float64 sums
    float sums[9];
    double sumsd[3];
    // the CG scalars per coordinate (the same for every thread: kept here,
    // set by thread 0, rather than in every thread's registers)
    float gam[3], alp[3], bet[3], stop[3];
    double target[3];
    int in;  // coordinates whose float32 run goes on (bit c)
    float scr[32 * 9];
    double scrd[32 * 3];
    float *recv_of[BCL_MAX];
    double *recvd_of[BCL_MAX];
};

// K warp butterflies side by side (level by level, so the shuffles of the
// K values overlap); every lane ends with lane 0's sums
template <typename T, int K>
__device__ __forceinline__ void warp_sums(T (&t)[K]) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
#pragma unroll
        for (int k = 0; k < K; ++k) t[k] += __shfl_xor_sync(0xffffffffu, t[k], o);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) t[k] = __shfl_sync(0xffffffffu, t[k], 0);
}

// the K sums of v over the cluster into out (shared, identical in every
// CTA): warp sums, warp 0 folds the warps' values into this CTA's sums and
// stores them into every CTA's receive slots (recv[par][rank], remote
// stores: no round trip), a cluster barrier, then warp 0 folds the
// received sums in rank order (lane q holds CTA q's).  A parity's slots are
// rewritten two calls later, after every CTA has passed the barrier that
// follows its reads.
template <typename T, int K, bool SYNC_END = true>
__device__ __forceinline__ void bcl_sums(cgx::cluster_group &cl, const T (&v)[K], T *scr, T *recv,
                                         T *const *recv_of, int par, int rank, int ncta, T *out) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T t[K];
#pragma unroll
    for (int k = 0; k < K; ++k) t[k] = v[k];
    warp_sums<T, K>(t);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) scr[w * K + k] = t[k];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) t[k] = lane < BCL_THREADS / 32 ? scr[lane * K + k] : (T)0;
        warp_sums<T, K>(t);
        if (lane < ncta) {
            T *dst = recv_of[lane] + (par * BCL_MAX + rank) * K;
#pragma unroll
            for (int k = 0; k < K; ++k) dst[k] = t[k];
        }
    }
    cl.sync();  // every CTA's sums received
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) t[k] = lane < ncta ? recv[(par * BCL_MAX + lane) * K + k] : (T)0;
        warp_sums<T, K>(t);
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) out[k] = t[k];
        }
    }
    if (SYNC_END) __syncthreads();  // otherwise out[] is thread 0's until the caller's barrier
}

// the codes of neighbours base .. base + BCL_NB - 1 of a vertex (-1 past its
// degree): from shared memory when they all fit there, else from cnbr
__device__ __forceinline__ void bcl_codes(const int4 *cq, const int *cnbr, int li, int2 e, int base,
                                          int (&cd)[BCL_NB]) {
    if (e.y <= BCL_NB) {
        const int4 c0 = cq[2 * li], c1 = cq[2 * li + 1];
        cd[0] = c0.x; cd[1] = c0.y; cd[2] = c0.z; cd[3] = c0.w;
        cd[4] = c1.x; cd[5] = c1.y; cd[6] = c1.z; cd[7] = c1.w;
    } else {
#pragma unroll
        for (int k = 0; k < BCL_NB; ++k) cd[k] = base + k < e.y ? cnbr[e.x + base + k] : -1;
    }
}

__global__ void __launch_bounds__(BCL_THREADS, 1) k_band_cl(BandArgs a, int limit) {
    constexpr int vcap = BCL_VCAP;
    HFCR_PDL_WAIT();
    cgx::cluster_group cl = cgx::this_cluster();
    const int n = *a.d_nfree;
    if (n > limit) return;  // the grid kernel's band (the same n in every CTA)
    extern __shared__ float4 bsm[];
    __shared__ BclState st;
    const int ncta = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int chunk = n > 0 ? (n + ncta - 1) / ncta : 1;
    const int lo = rank * chunk;
    const int cnt = n - lo < chunk ? (n - lo > 0 ? n - lo : 0) : chunk;
    float4 *rq = bsm;  // r (x, y, z) and 1 / deg
    float4 *gz = (float4 *)a.rec;  // z of every band vertex, for the other CTAs
    double *gu = a.u64;            // u of every band vertex
    float4 *pq = rq + vcap, *sq = pq + vcap, *xq = sq + vcap, *wq = xq + vcap;
    float4 *zq = wq + vcap;
    int4 *cq = (int4 *)(zq + vcap);  // two int4 (BCL_NB codes) per vertex
    double *uq = (double *)(cq + 2 * (size_t)vcap);  // u (x, y, z) of the rounds
    int2 *ed = (int2 *)(uq + 3 * (size_t)vcap);
    if ((int)threadIdx.x < ncta) {
        st.recv_of[threadIdx.x] = cl.map_shared_rank(&st.recv[0][0][0], threadIdx.x);
        st.recvd_of[threadIdx.x] = cl.map_shared_rank(&st.recvd[0][0][0], threadIdx.x);
    }
    // the right-hand side (Dirichlet values of the neighbours outside the
    // band), the neighbours' record addresses, the first round's state
    // (r = b, u = 0)
    double dl[3] = {0.0, 0.0, 0.0};
    for (int li = threadIdx.x; li < cnt; li += BCL_THREADS) {
        const int i = lo + li;
        const int g = a.fv[i];
        const bool inB = g >= a.P.m[1].off;
        const DMesh &M = inB ? a.P.m[1] : a.P.m[0];
        const int v = g - M.off;
        const int e0 = M.ptr[v], e1 = M.ptr[v + 1];
        const int s0 = (inB ? a.eoffB : 0) + e0;
        double b[3] = {0.0, 0.0, 0.0};
        int cs[BCL_NB];
#pragma unroll
        for (int k = 0; k < BCL_NB; ++k) cs[k] = -1;
        for (int e = e0; e < e1; ++e) {
            const int w = M.off + M.nbr[e];
            const int j = a.cidx[w];
            int code = -1;
            if (j >= 0) {
                code = j / chunk == rank ? -2 - (j - lo) : j;
            } else {
                const double *uw = a.u + 3 * (size_t)w;
                b[0] += uw[0];
                b[1] += uw[1];
                b[2] += uw[2];
            }
            a.cnbr[s0 + e - e0] = code;
#pragma unroll
            for (int k = 0; k < BCL_NB; ++k)
                if (e - e0 == k) cs[k] = code;
        }
        cq[2 * li] = make_int4(cs[0], cs[1], cs[2], cs[3]);
        cq[2 * li + 1] = make_int4(cs[4], cs[5], cs[6], cs[7]);
        // a band vertex has a neighbour one ring closer, so e1 > e0
        ed[li] = make_int2(s0, e1 - e0);
        rq[li] = make_float4((float)b[0], (float)b[1], (float)b[2], 1.0f / (float)(e1 - e0));
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        pq[li] = z4;
        sq[li] = z4;
        xq[li] = z4;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a.b64[3 * (size_t)i + c] = b[c];
            uq[3 * li + c] = 0.0;
            gu[3 * (size_t)i + c] = 0.0;
            dl[c] += b[c] * b[c];
        }
    }
    int pf = 0, pd = 0;  // parities of the float and float64 receive slots
    bcl_sums<double, 3>(cl, dl, st.scrd, &st.recvd[0][0][0], st.recvd_of, pd, rank, ncta, st.sumsd);
    pd ^= 1;
    int act = 0;  // coordinates not yet converged (bit c), the same in every thread
#pragma unroll
    for (int c = 0; c < 3; ++c)
        if (st.sumsd[c] > 0.0) act |= 1 << c;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) st.target[c] = a.tol * a.tol * st.sumsd[c];
    }
    int it = 0, rounds = 0;
    bool fail = false;
    while (act) {
        if (++rounds > BAND_MAX_ROUNDS) { fail = true; break; }
        const int it_round = it;
        bool first = true;
        while (true) {
            __syncthreads();  // this CTA's r visible
            // z = M^-1 r from this CTA's r
            for (int li = threadIdx.x; li < cnt; li += BCL_THREADS) {
                const float4 me = rq[li];
                const int2 e = ed[li];
                float s0 = 0.f, s1 = 0.f, s2 = 0.f;
                for (int base = 0; base < e.y; base += BCL_NB) {
                    int cd[BCL_NB];
                    bcl_codes(cq, a.cnbr, li, e, base, cd);
                    float4 nb[BCL_NB];
#pragma unroll
                    for (int k = 0; k < BCL_NB; ++k)
                        nb[k] = cd[k] <= -2 ? rq[-2 - cd[k]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int k = 0; k < BCL_NB; ++k) {
                        s0 += nb[k].x * nb[k].w;
                        s1 += nb[k].y * nb[k].w;
                        s2 += nb[k].z * nb[k].w;
                    }
                }
                const float4 z4 = make_float4((me.x + BCL_THETA * s0) * me.w, (me.y + BCL_THETA * s1) * me.w,
                                              (me.z + BCL_THETA * s2) * me.w, 0.f);
                zq[li] = z4;
                gz[lo + li] = z4;
            }
            cl.sync();  // every band vertex's z visible
            // w = L z, and the sums (r, z), (w, z), |r|^2
            float fl[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) fl[k] = 0.f;
            for (int li = threadIdx.x; li < cnt; li += BCL_THREADS) {
                const float4 me = rq[li], zm = zq[li];
                const int2 e = ed[li];
                const float dg = (float)e.y;
                float w0 = dg * zm.x, w1 = dg * zm.y, w2 = dg * zm.z;
                for (int base = 0; base < e.y; base += BCL_NB) {
                    int cd[BCL_NB];
                    bcl_codes(cq, a.cnbr, li, e, base, cd);
#pragma unroll
                    for (int h = 0; h < BCL_NB; h += 4) {
                        float4 nb[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            nb[k] = cd[h + k] >= 0 ? __ldcg(gz + cd[h + k])
                                                   : (cd[h + k] <= -2 ? zq[-2 - cd[h + k]]
                                                                      : make_float4(0.f, 0.f, 0.f, 0.f));
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            w0 -= nb[k].x;
                            w1 -= nb[k].y;
                            w2 -= nb[k].z;
                        }
                    }
                }
                wq[li] = make_float4(w0, w1, w2, 0.f);
                fl[0] += me.x * zm.x; fl[1] += me.y * zm.y; fl[2] += me.z * zm.z;
                fl[3] += w0 * zm.x;   fl[4] += w1 * zm.y;   fl[5] += w2 * zm.z;
                fl[6] += me.x * me.x; fl[7] += me.y * me.y; fl[8] += me.z * me.z;
            }
            bcl_sums<float, 9, false>(cl, fl, st.scr, &st.recv[0][0][0], st.recv_of, pf, rank, ncta,
                                      st.sums);
            pf ^= 1;
            if (threadIdx.x == 0) {  // the scalars, from the sums thread 0 has just folded
                const float *fs = st.sums;
                int in = 0;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (first) {
                        const float al = __fdividef(fs[c], fs[3 + c]);
                        st.gam[c] = fs[c];
                        st.alp[c] = al;
                        st.bet[c] = 0.f;
                        st.stop[c] = BAND_INNER_TOL * BAND_INNER_TOL * fs[6 + c];
                        if ((act >> c & 1) && fs[6 + c] > 0.f && al > 0.f && isfinite(al)) in |= 1 << c;
                    } else {
                        const float b = __fdividef(fs[c], st.gam[c]);
                        const float al = __fdividef(fs[c], fs[3 + c] - b * __fdividef(fs[c], st.alp[c]));
                        if ((st.in >> c & 1) && fs[6 + c] > st.stop[c] && al > 0.f && isfinite(al)) {
                            st.bet[c] = b;
                            st.alp[c] = al;
                            st.gam[c] = fs[c];
                            in |= 1 << c;
                        }
                    }
                }
                st.in = in;
            }
            __syncthreads();
            first = false;
            const int in = st.in;
            if (!in || it >= a.max_iters) break;
            // p = z + beta p, s = w + beta s, x += alpha p, r -= alpha s
            const float al[3] = {st.alp[0], st.alp[1], st.alp[2]};
            const float be[3] = {st.bet[0], st.bet[1], st.bet[2]};
            for (int li = threadIdx.x; li < cnt; li += BCL_THREADS) {
                float4 r4 = rq[li], p4 = pq[li], s4 = sq[li], x4 = xq[li];
                const float4 w4 = wq[li], z4 = zq[li];
                float *r = &r4.x, *p = &p4.x, *sv = &s4.x, *x = &x4.x;
                const float *w = &w4.x, *zz = &z4.x;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (!(in >> c & 1)) continue;
                    p[c] = zz[c] + be[c] * p[c];
                    sv[c] = w[c] + be[c] * sv[c];
                    x[c] += al[c] * p[c];
                    r[c] -= al[c] * sv[c];
                }
                rq[li] = r4;
                pq[li] = p4;
                sq[li] = s4;
                xq[li] = x4;
            }
            ++it;
        }
        // the round's end: u += x, then the float64 residual b - L u from
        // the neighbours' u; the next round starts from it (x = p = s = 0)
        for (int li = threadIdx.x; li < cnt; li += BCL_THREADS) {
            const float4 x4 = xq[li];
            double *u = uq + 3 * li;
            u[0] += (double)x4.x;
            u[1] += (double)x4.y;
            u[2] += (double)x4.z;
#pragma unroll
            for (int c = 0; c < 3; ++c) gu[3 * (size_t)(lo + li) + c] = u[c];
        }
        cl.sync();  // every band vertex's u visible
#pragma unroll
        for (int c = 0; c < 3; ++c) dl[c] = 0.0;
        for (int li = threadIdx.x; li < cnt; li += BCL_THREADS) {
            const int i = lo + li;
            const int2 e = ed[li];
            const double *u = uq + 3 * li;
            double r64[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) r64[c] = a.b64[3 * (size_t)i + c] - (double)e.y * u[c];
            for (int k = 0; k < e.y; ++k) {
                const int cd = a.cnbr[e.x + k];
                if (cd == -1) continue;
                if (cd >= 0) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) r64[c] += __ldcg(gu + 3 * (size_t)cd + c);
                } else {
#pragma unroll
                    for (int c = 0; c < 3; ++c) r64[c] += uq[3 * (-2 - cd) + c];
                }
            }
            rq[li] = make_float4((act & 1) ? (float)r64[0] : 0.f, (act & 2) ? (float)r64[1] : 0.f,
                                 (act & 4) ? (float)r64[2] : 0.f, rq[li].w);
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            pq[li] = z4;
            sq[li] = z4;
            xq[li] = z4;
#pragma unroll
            for (int c = 0; c < 3; ++c) dl[c] += r64[c] * r64[c];
        }
        bcl_sums<double, 3>(cl, dl, st.scrd, &st.recvd[0][0][0], st.recvd_of, pd, rank, ncta, st.sumsd);
        pd ^= 1;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if ((act >> c & 1) && st.sumsd[c] <= st.target[c]) act &= ~(1 << c);
        if (act && (it >= a.max_iters || it == it_round)) { fail = true; break; }
    }
    for (int li = threadIdx.x; li < cnt; li += BCL_THREADS) {
        double *ug = a.u + 3 * (size_t)a.fv[lo + li];
#pragma unroll
        for (int c = 0; c < 3; ++c) ug[c] = uq[3 * li + c];
    }
    if (rank == 0 && threadIdx.x == 0) {
        a.ctl[0] += it;
        if (fail) a.ctl[1] = 1;
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
}

inline int blocks(int n) { return (n + 255) / 256; }

DPair make_pair(const DiffMeshArgs &a, const DiffMeshArgs &b) {
    DPair P;
    P.m[0].ptr = a.ptr; P.m[0].nbr = a.nbr; P.m[0].inv_mass = a.inv_mass; P.m[0].n = a.n; P.m[0].off = 0;
    P.m[1].ptr = b.ptr; P.m[1].nbr = b.nbr; P.m[1].inv_mass = b.inv_mass; P.m[1].n = b.n; P.m[1].off = a.n;
    P.m[0].rank = a.rank;
    P.m[1].rank = b.rank;
    P.ntot = a.n + b.n;
    return P;
}

}  // namespace

void build_adjacency(const int *edges, int ne, int nv, int *ptr, int *nbr, int *cur, SortTemp &t,
                     uint32_t *d_status, cudaStream_t s) {
    if (nv <= 0) return;
    cudaMemsetAsync(ptr, 0, sizeof(int) * (size_t)(nv + 1), s);
    cudaMemsetAsync(cur, 0, sizeof(int) * (size_t)nv, s);
    if (ne > 0) { launch_pdl(k_adj_count, blocks(ne), 256, 0, s, (const int2 *)edges, ne, nv, ptr,
                             d_status); note_launch(); }
    // degrees -> exclusive offsets in place, total (2 x valid edges) to ptr[nv]
    scan_flags_dev((unsigned *)ptr, nullptr, nv, ptr + nv, t, s);
    if (ne > 0) { launch_pdl(k_adj_fill, blocks(ne), 256, 0, s, (const int2 *)edges, ne, nv, ptr,
                             cur, nbr); note_launch(); }
    { launch_pdl(k_adj_sort, blocks(nv), 256, 0, s, ptr, nv, nbr); note_launch(); }
}

// co-resident CTAs of k_band_cg on this device (0: no cooperative launch)
static int band_grid_max() {
    static int cached[64];
    static bool done[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 0;
    if (!done[dev]) {
        int coop = 0, sms = 0, per = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_band_cg, BAND_TPB, 0);
        cached[dev] = coop ? sms * (per < 1 ? 0 : 1) : 0;  // one CTA per SM: cheaper barriers
        done[dev] = true;
    }
    return cached[dev];
}

// the cluster of k_band_cl on this device: the most CTAs (16, 8, 4, 2)
// whose cluster fits, and the band vertices one CTA holds
struct BclConfig {
    bool ok = false;
    int ncta = 0, vcap = 0;
};
static BclConfig band_cl_config() {
    static BclConfig cached[64];
    static bool done[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return BclConfig();
    if (!done[dev]) {
        BclConfig c;
        if (cudaFuncSetAttribute(k_band_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, BCL_SMEM) ==
                cudaSuccess &&
            cudaFuncSetAttribute(k_band_cl, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                cudaSuccess) {
            for (int n = BCL_MAX; n >= 2 && !c.ok; n /= 2) {
                cudaLaunchConfig_t lc = {};
                lc.gridDim = dim3(n);
                lc.blockDim = dim3(BCL_THREADS);
                lc.dynamicSmemBytes = BCL_SMEM;
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeClusterDimension;
                at[0].val.clusterDim.x = n;
                at[0].val.clusterDim.y = 1;
                at[0].val.clusterDim.z = 1;
                lc.attrs = at;
                lc.numAttrs = 1;
                int ncl = 0;
                if (cudaOccupancyMaxActiveClusters(&ncl, (const void *)k_band_cl, &lc) == cudaSuccess &&
                    ncl > 0) {
                    c.ok = true;
                    c.ncta = n;
                }
                cudaGetLastError();
            }
        }
        cudaGetLastError();
        c.vcap = BCL_VCAP;
        cached[dev] = c;
        done[dev] = true;
    }
    return cached[dev];
}

void vertex_rank(const hfcr_mesh &m, int *rank, const DiffScratch &ds, SortTemp &t, cudaStream_t s) {
    const int n = m.n_verts;
    if (n <= 0) return;
    // scratch: keys and values in the grid kernel's record buffer (48 floats
    // per vertex of capacity; the sort needs 24 bytes), the box in `part`
    unsigned long long *k0 = (unsigned long long *)ds.rec, *k1 = k0 + n;
    int *v0 = (int *)(k1 + n), *v1 = v0 + n;
    int *box = (int *)ds.part;
    { launch_pdl(k_rank_box_init, 1, 32, 0, s, box); note_launch(); }
    int nb = blocks(n);
    const int nbb = nb > 1024 ? 1024 : nb;
    if (m.dtype == HFCR_F32) {
        const float *x = (const float *)m.x, *y = (const float *)m.y, *z = (const float *)m.z;
        { launch_pdl(k_rank_bounds<float>, nbb, 256, 0, s, x, y, z, n, box); note_launch(); }
        { launch_pdl(k_rank_keys<float>, nb, 256, 0, s, x, y, z, n, (const int *)box, k0, v0); note_launch(); }
    } else {
        const double *x = (const double *)m.x, *y = (const double *)m.y, *z = (const double *)m.z;
        { launch_pdl(k_rank_bounds<double>, nbb, 256, 0, s, x, y, z, n, box); note_launch(); }
        { launch_pdl(k_rank_keys<double>, nb, 256, 0, s, x, y, z, n, (const int *)box, k0, v0); note_launch(); }
    }
    const bool flip = radix_sort_u64(k0, v0, k1, v1, n, 30, t, s);
    { launch_pdl(k_rank_scatter, nb, 256, 0, s, (const int *)(flip ? v1 : v0), n, rank); note_launch(); }
}

void diffusion_init() {
    (void)band_grid_max();
    (void)band_cl_config();
}

const double *diffuse_field(const DiffMeshArgs &a, const DiffMeshArgs &b, double *u, double *u_alt,
                            int *ring, int rings, int sweeps, double tol, int max_iters,
                            const DiffScratch &ds, SortTemp &t, uint32_t *d_status,
                            cudaStream_t s, const StageMark &mark) {
    DPair P = make_pair(a, b);
    if (P.ntot <= 0 || rings <= 0) return u;
    const int far = rings + 1, nb = blocks(P.ntot);
    { launch_pdl(k_ring_init, nb, 256, 0, s, P, u, ring, far); note_launch(); }
    for (int r = 1; r <= rings; ++r) { launch_pdl(k_ring_step, nb, 256, 0, s, P, ring, r,
                                                  far); note_launch(); }
    if (sweeps > 0) {
        // the named approximation: a fixed number of Jacobi sweeps from zero
        double *in = u, *out = u_alt;
        for (int q = 0; q < sweeps; ++q) {
            { launch_pdl(k_sweep, nb, 256, 0, s, P, ring, rings, in, out); note_launch(); }
            double *tmp = in; in = out; out = tmp;
        }
        return in;
    }
    // the harmonic field: the band compacted, then CG on its Laplacian
    { launch_pdl(k_band_flags, nb, 256, 0, s, P, ring, rings, ds.flags); note_launch(); }
    scan_flags_dev(ds.flags, nullptr, P.ntot, ds.d_nfree, t, s);
    { launch_pdl(k_band_list, nb, 256, 0, s, P, ring, rings, (const unsigned *)ds.flags, ds.cidx,
                 ds.fv); note_launch(); }
    int grid = band_grid_max();
    const int want = (P.ntot + 4 * BAND_TPB - 1) / (4 * BAND_TPB);
    if (grid > want) grid = want;
    if (grid < 1) {
        cudaMemsetAsync(ds.ctl + 1, 0xff, sizeof(int), s);  // reported as not converged
        return u;
    }
    BandArgs ba;
    ba.P = P;
    ba.cidx = ds.cidx;
    ba.fv = ds.fv;
    ba.d_nfree = ds.d_nfree;
    ba.u = u;
    ba.b64 = ds.b64;
    ba.u64 = ds.u64;
    ba.x32 = ds.x32;
    ba.p32 = ds.p32;
    ba.rec = ds.rec;
    ba.cnbr = ds.cnbr;
    ba.eoffB = ds.eoffB;
    ba.part = ds.part;
    ba.bar = ds.bar;
    ba.ctl = ds.ctl;
    ba.status = d_status;
    ba.tol = tol;
    ba.max_iters = max_iters;
    ba.cap = ds.cap;
    cudaMemsetAsync(ds.bar, 0, sizeof(unsigned), s);
    // bands of up to `limit` vertices on one cluster, larger ones on the
    // grid (each kernel returns at once when the band is the other's)
    const BclConfig bc = band_cl_config();
    int limit = bc.ok ? bc.ncta * bc.vcap : -1;
    mark(1, s);
    if (bc.ok) {
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3(bc.ncta);
        lc.blockDim = dim3(BCL_THREADS);
        lc.dynamicSmemBytes = BCL_SMEM;
        lc.stream = s;
        cudaLaunchAttribute at[2];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = bc.ncta;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[1].val.programmaticStreamSerializationAllowed = 1;
        lc.attrs = at;
        lc.numAttrs = 2;
        if (cudaLaunchKernelEx(&lc, k_band_cl, ba, limit) == cudaSuccess) {
            note_launch();
        } else {
            cudaGetLastError();
            limit = -1;
        }
    }
    void *args[] = {&ba, &limit};
    const cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_band_cg, grid, BAND_TPB, args, 0, s);
    mark(0, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaMemsetAsync(ds.ctl + 1, 0xff, sizeof(int), s);  // reported as not converged
        return u;
    }
    note_launch();
    return u;
}

void apply_field(const hfcr_mesh &A, const hfcr_mesh &B, const int *ring, int rings,
                 const double *u, cudaStream_t s) {
    const int ntot = A.n_verts + B.n_verts;
    if (ntot <= 0) return;
    { launch_pdl(k_apply_field, blocks(ntot), 256, 0, s, A, B, ring, rings, u,
                 ntot); note_launch(); }
}

void field_from_soa(const double *x, const double *y, const double *z, int n, double *u,
                    cudaStream_t s) {
    if (n > 0) { launch_pdl(k_soa_to_aos, blocks(n), 256, 0, s, x, y, z, n, u); note_launch(); }
}

void field_to_soa(const double *u, int n, double *x, double *y, double *z, cudaStream_t s) {
    if (n > 0) { launch_pdl(k_aos_to_soa, blocks(n), 256, 0, s, u, n, x, y, z); note_launch(); }
}

}  // namespace hfcr
