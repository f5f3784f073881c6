// Diffusion of displacement vectors (Sec. 5): the correction the minimizer
// gives the stencil vertices is spread over their vicinity as a harmonic
// vector field, so that the mesh moves smoothly instead of only at the
// penetrating vertices.  The paper names constrained diffusion without
// equations; the reading implemented here: vertices with a nonzero
// displacement keep it (Dirichlet values), vertices more than R edges away
// and kinematic vertices (inverse mass 0) keep zero, and every vertex in
// between takes the mean of its neighbours, S Jacobi sweeps from zero.
//
// Layout: the field u is float64 AoS (x, y, z per vertex) over the global
// vertex numbering of the pair (A's vertices, then B's), so that a
// neighbour read is one 24-byte load.  Each mesh's vertex adjacency is a
// CSR with ascending neighbours, built from its sorted edge list.  The
// neighbour sums run in that ascending order and divide by the degree, so
// the result is bit-identical to a sequential float64 evaluation.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

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

// breadth-first level r: a vertex not reached yet joins when a neighbour
// sits at level r - 1 (levels r - 1 and below no longer change)
__global__ void k_ring_step(DPair P, int *ring, int r, int far) {
    HFCR_PDL_WAIT();
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P.ntot || ring[g] != far) return;
    const DMesh &M = P.of(g);
    const int v = g - M.off;
    for (int e = M.ptr[v]; e < M.ptr[v + 1]; ++e)
        if (ring[M.off + M.nbr[e]] == r - 1) {
            ring[g] = r;
            return;
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

inline int blocks(int n) { return (n + 255) / 256; }

DPair make_pair(const DiffMeshArgs &a, const DiffMeshArgs &b) {
    DPair P;
    P.m[0].ptr = a.ptr; P.m[0].nbr = a.nbr; P.m[0].inv_mass = a.inv_mass; P.m[0].n = a.n; P.m[0].off = 0;
    P.m[1].ptr = b.ptr; P.m[1].nbr = b.nbr; P.m[1].inv_mass = b.inv_mass; P.m[1].n = b.n; P.m[1].off = a.n;
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

const double *diffuse_field(const DiffMeshArgs &a, const DiffMeshArgs &b, double *u, double *u_alt,
                            int *ring, int rings, int sweeps, cudaStream_t s) {
    DPair P = make_pair(a, b);
    if (P.ntot <= 0) return u;
    const int far = rings + 1, nb = blocks(P.ntot);
    { launch_pdl(k_ring_init, nb, 256, 0, s, P, u, ring, far); note_launch(); }
    for (int r = 1; r <= rings; ++r) { launch_pdl(k_ring_step, nb, 256, 0, s, P, ring, r,
                                                  far); note_launch(); }
    double *in = u, *out = u_alt;
    for (int q = 0; q < sweeps; ++q) {
        { launch_pdl(k_sweep, nb, 256, 0, s, P, ring, rings, in, out); note_launch(); }
        double *tmp = in; in = out; out = tmp;
    }
    return in;
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
