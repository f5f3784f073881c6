// Internal declarations shared by the translation units of libhfcr: the
// host-side wrappers of each translation unit's kernels, the launch helper
// and the few device helpers (segment lookup) more than one unit needs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <atomic>
#include <string>

#include "../../include/hfcr.h"

namespace hfcr {

// Process-wide count of kernel launches made by this library.
extern std::atomic<long long> g_launches;
inline void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Every kernel of the library starts with HFCR_PDL_WAIT.  Launched by
// launch_pdl, a kernel is the programmatic dependent of the previous kernel
// in its stream: it may be scheduled while that kernel still runs, and the
// wait holds each thread until that kernel has completed and its writes
// are visible (no kernel triggers its dependents early), so the order is
// that of a plain launch and only the launch latency overlaps.  Launched
// any other way, the wait returns at once.
#define HFCR_PDL_WAIT() asm volatile("griddepcontrol.wait;" ::: "memory")

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, static_cast<Args &&>(args)...);
}

// Device-side status bits (one 32-bit word per context, OR-ed by kernels).
enum : uint32_t {
    ST_NONFINITE = 1u << 0,
    ST_RANGE = 1u << 1,
    ST_CAPACITY = 1u << 2,
    ST_TIMEOUT = 1u << 3,
    ST_BAD_INDEX = 1u << 4,
};

#ifdef __CUDACC__
// Segment of element idx in a batch: the largest i < nseg with
// segs[4 i + col] <= idx.  Segment table rows hold the offsets of one mesh
// pair in the concatenated meshes: (A vertex, A face, B vertex, B face).
__device__ __forceinline__ int seg_of(const int *segs, int col, int nseg, int idx) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (segs[4 * mid + col] <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// [first, first + count) of segment i in column col, clamped into [0, total)
// (a malformed table is reported by check_segments; this keeps every index
// in range meanwhile)
__device__ __forceinline__ void seg_range(const int *segs, int col, int i, int total, int &first,
                                          int &count) {
    int a = min(max(segs[4 * i + col], 0), total);
    int b = min(max(segs[4 * (i + 1) + col], a), total);
    first = a;
    count = b - a;
}
#endif

// Counters a detection accumulates on the device.
struct DevStats {
    unsigned long long narrow_tests;
    unsigned long long f64_fallbacks;
    unsigned long long exact_fallbacks;
    unsigned long long bf;  // sum over mesh pairs of |edges| x |faces| tested
};

// A BVH over the faces of one mesh (Karras 2012 binary radix tree).
// A batch of independent mesh pairs builds one tree per pair (segment) in the
// same arrays: the internal nodes of the segment whose faces start at t0 are
// stored at t0 .. t0 + n_seg - 2, its leaves at t0 .. t0 + n_seg - 1.
// Internal node i is stored as 4 x 16 bytes:
//   [c0.lo.xyz, c0.hi.x] [c0.hi.yz, c1.lo.xy] [c1.lo.z, c1.hi.xyz] [child0, child1, -, -]
// child >= 0 is an internal node, child < 0 the leaf ~child.  Leaf j holds
// face leaf_face[j]; its triangle is packed (in leaf order) for the
// narrow phase: float32 meshes 3 x float4 (a.xyz b.x | b.yz c.xy | c.z face - -),
// float64 meshes 5 x double2 (a.xy | a.z b.x | b.yz | c.xy | c.z face).
struct Bvh {
    int n = 0;                  // leaves (faces)
    int cap = 0;
    float4 *nodes = nullptr;    // [4 * (cap - 1)]
    int *parent = nullptr;      // [2 * cap - 1]: parent of internal i at [i], of leaf j at [cap - 1 + j]
    unsigned *flags = nullptr;  // [cap - 1] arrival counters of the refit
    int *leaf_face = nullptr;   // [cap]
    void *leaf_tri = nullptr;   // [cap] packed triangles in leaf order
    unsigned long long *keys = nullptr;      // [cap] (segment, Morton code) sort keys
    unsigned long long *keys_alt = nullptr;
    int *vals_alt = nullptr;
    float *bounds = nullptr;    // [6] scene bounds of the centroids
    float *bounds_part = nullptr;  // per-block partial bounds
    int *d_rest = nullptr;      // [1] the segmented sort's request for the global sort
    int dtype = 0;
    // one tree per segment: segment i owns faces [segs[4 i + col], segs[4 (i + 1) + col])
    const int *segs = nullptr;
    int col = 0, nseg = 1;
};

struct SortTemp {
    unsigned *hist = nullptr;   // [256 * max_blocks]: tile histograms, then a row for the grid
                                // barrier of the cooperative sort and a row of digit totals
    int max_blocks = 0;         // tiles of the largest sort + 2
    uint32_t *status = nullptr; // device status word (ST_TIMEOUT of the cooperative sort)
};

// Radix sort (stable LSD, 8-bit digits) of keys with optional int values.
// Sorts bits [0, bits).  Ping-pongs between (k0, v0) and (k1, v1); returns
// true when the result ended in (k1, v1).  n is read from the host.
bool radix_sort_u32(unsigned *k0, int *v0, unsigned *k1, int *v1, int n, int bits,
                    SortTemp &t, cudaStream_t s);
bool radix_sort_u64(unsigned long long *k0, int *v0, unsigned long long *k1, int *v1, int n,
                    int bits, SortTemp &t, cudaStream_t s);
// Same with the element count read from a device word (launch sized by cap).
bool radix_sort_u64_dev(unsigned long long *k0, unsigned long long *k1, const int *d_n, int cap,
                        int bits, SortTemp &t, cudaStream_t s);
bool radix_sort_u32_dev(unsigned *k0, int *v0, unsigned *k1, int *v1, const int *d_n, int cap,
                        int bits, SortTemp &t, cudaStream_t s);
bool radix_sort_u64v_dev(unsigned long long *k0, int *v0, unsigned long long *k1, int *v1,
                         const int *d_n, int cap, int bits, SortTemp &t, cudaStream_t s);
// keys of a batch grouped by segment (segment number in the bits above
// seg_bits): one CTA sorts each segment over its low seg_bits bits; if a
// segment is longer than one CTA sorts, *d_rest (scratch) routes the whole
// input through the global sort over all `bits` bits.  Same result and
// buffer as radix_sort_u64 with values.
bool radix_sort_u64v_segments(unsigned long long *k0, int *v0, unsigned long long *k1, int *v1,
                              int n, int bits, const int *segs, int col, int nseg, int seg_bits,
                              int *d_rest, SortTemp &t, cudaStream_t s);
int sort_blocks_for(int n);

// Exclusive scan of n unsigned flags (in place), total written to *d_total.
// n read from a device word, cap bounds it.
void scan_flags_dev(unsigned *flags, const int *d_n, int cap, int *d_total, SortTemp &t,
                    cudaStream_t s);

// ---- topology ----
// Unique sorted edges of a triangle list.  Scratch: keys/keys_alt of
// 3 * n_tris u64 and flags of 3 * n_tris unsigned.
void build_edges(const int *tris, int n_tris, int n_verts, int *edges_out, int *d_count,
                 unsigned long long *keys, unsigned long long *keys_alt, unsigned *flags,
                 SortTemp &t, uint32_t *d_status, cudaStream_t s);

// ---- BVH ----
// segs: device [(nseg + 1)][4] rows (A vertex, A face, B vertex, B face)
// offsets; col selects the face column of the mesh the tree is built over
void bvh_build(Bvh &b, const hfcr_mesh &m, const int *segs, int col, int nseg, SortTemp &t,
               uint32_t *d_status, cudaStream_t s);
void check_segments(const int *segs, int nseg, const hfcr_mesh &A, const hfcr_mesh &B,
                    uint32_t *d_status, cudaStream_t s);
void bvh_refit(Bvh &b, const hfcr_mesh &m, uint32_t *d_status, cudaStream_t s);
// a traversal order of an edge list: the edges sorted by (segment, Morton
// code of the midpoint in the mesh's vertex bounds), stable; order [ne] gets
// the permutation (order_alt [ne] and the keys [ne] each are scratch)
void edge_order(const int *edges, int ne, const hfcr_mesh &m, const int *segs, int col, int nseg,
                int *order, int *order_alt, unsigned long long *keys, unsigned long long *keys_alt,
                float *bounds_part, float *bounds, SortTemp &t, uint32_t *d_status, cudaStream_t s);

// ---- validation ----
void validate_positions(const hfcr_mesh &m, uint32_t *d_status, cudaStream_t s);
// both meshes of a pair (one launch when they share a dtype)
void validate_pair(const hfcr_mesh &A, const hfcr_mesh &B, uint32_t *d_status, cudaStream_t s);

// ---- detection ----
struct DetectArgs {
    const int *segs;    // segment table of the batch (one row per mesh pair + a closing row)
    int nseg;
    int ecol, fcol;     // vertex column of the edge mesh, face column of the face mesh
    const hfcr_mesh *edge_mesh;
    const int *edges;   // [n_edges][2]
    const int *order = nullptr;  // traversal order of the edges (a permutation), or null
    int n_edges;
    const Bvh *bvh;     // over the faces of the other mesh
    int dir;
    int f32_filter;
    int edge_bits, face_bits;  // key layout
    unsigned long long *keys;  // output keys (dir | edge | face)
    int *d_count;
    int cap;
    DevStats *stats;
    int variant = 0;  // traversal variant (0 to 8; see detect.cu)
    int *queue = nullptr;  // work counter of the persistent variants (zeroed by the launch)
};
constexpr int N_TRAVERSE_VARIANTS = 9;
void detect_launch(const DetectArgs &a, cudaStream_t s, uint32_t *d_status);
// adds sum_i |edges of pair i| x |faces of pair i| to stats->bf (edges are
// sorted by first vertex, so each pair's edges are contiguous)
void pair_products(const int *edges, int ne, const int *segs, int nseg, int ecol, int fcol,
                   int nfaces, DevStats *stats, cudaStream_t s);
// keys (sorted) -> hfcr_pair records
void keys_to_pairs(const unsigned long long *keys, const int *d_n, int cap, const int *edgesA,
                   const int *edgesB, int edge_bits, int face_bits, hfcr_pair *out, cudaStream_t s);

// ---- stencils ----
struct MeshPair {
    hfcr_mesh A, B;
};
// one stencil key per pair of the traversal's pair keys (dir | edge | face,
// in append order); the pair count *d_n is clamped to cap into *d_eff (more
// than cap: ST_CAPACITY and none)
void stencil_keys_from_pair_keys(const MeshPair &mp, const unsigned long long *pkeys, const int *d_n,
                                 int cap, const int *edgesA, const int *edgesB, int edge_bits,
                                 int pface_bits, int vert_bits, int face_bits, int f32_filter,
                                 unsigned long long *keys, int *d_eff, DevStats *stats,
                                 uint32_t *d_status, cudaStream_t s);
// one stencil key per pair (dir | x0 | face); n pairs from host count
void stencil_keys(const MeshPair &mp, const hfcr_pair *pairs, const int *d_n, int cap,
                  int vert_bits, int face_bits, int f32_filter, unsigned long long *keys,
                  DevStats *stats, uint32_t *d_status, cudaStream_t s);
// sorted keys -> unique stencils, count to d_k
void stencil_unique(const unsigned long long *keys, const int *d_n, int cap, int vert_bits,
                    int face_bits, unsigned *flags, hfcr_stencil *out, int *d_k, SortTemp &t,
                    cudaStream_t s);

// ---- solver ----
struct SolveBuffers {
    int cap_k = 0;       // stencils
    // rows as assembled (stencil order) ...
    int4 *ids_raw = nullptr;
    double4_32a *n64_raw = nullptr;
    float4 *n32_raw = nullptr;
    double *b_raw = nullptr;
    // ... and regrouped by impact zone (the arrays below are zone-ordered)
    int *parent = nullptr;       // [cap_k] union-find forest over stencils
    unsigned long long *zkey = nullptr, *zkey_alt = nullptr;  // [cap_k] (zone label, stencil)
    int *szone = nullptr;        // [cap_k] zone of each zone-ordered stencil
    int *zs = nullptr;           // [cap_k + 1] first stencil of each zone
    int *zv = nullptr;           // [4 cap_k + 1] first touched vertex of each zone
    int *d_nz = nullptr;         // zone count (device)
    int *gst = nullptr;          // [cap_k + 1] first row of each preconditioner group
    int *zg = nullptr;           // [cap_k + 1] first group of each zone
    int *d_ng = nullptr;         // group count (device)
    float4 *pinv = nullptr;      // [cap_k] row of the group's inverse block
    float *z32 = nullptr;        // [cap_k] preconditioned residual (global-memory CG path)
    unsigned long long *ck64 = nullptr, *ck64_alt = nullptr;  // [4 cap_k] (zone, vertex) keys
    int4 *ids = nullptr;         // [cap_k] global vertex ids
    double4_32a *n64 = nullptr;      // [cap_k] unit normal (w unused)
    float4 *n32 = nullptr;       // [cap_k]
    double *b = nullptr;         // [cap_k] D - d
    double *lam = nullptr;       // [cap_k]
    double *r64 = nullptr;       // [cap_k]
    float *r32 = nullptr, *x32 = nullptr, *p32 = nullptr, *q32 = nullptr, *w32 = nullptr;  // [cap_k]
    double *p64 = nullptr, *q64 = nullptr;   // p64 [2 cap_k] (x and p), q64 [cap_k] (FP64 solver)
    double *cg64 = nullptr;      // [5 cap_k] r, p, s, w, z of the float64 per-zone CG
    double4_32a *pinv64 = nullptr;  // [cap_k] float64 inverse-block rows of that CG
    float *binv = nullptr;          // [16 cap_k] rows of the large zones' block inverses (mixed)
    int4 *vidx = nullptr;        // [cap_k] compact vertex index of each stencil role
    // vertex CSR over 4k entries
    unsigned *ckey = nullptr, *ckey_alt = nullptr;   // [4 cap_k]
    int *cval = nullptr, *cval_alt = nullptr;        // [4 cap_k]
    unsigned *ckey_s = nullptr;  // the sorted key buffer (ckey or ckey_alt)
    int *cval_s = nullptr;       // the sorted entry buffer (cval or cval_alt)
    unsigned *cflag = nullptr;                       // [4 cap_k]
    int *seg = nullptr;          // [4 cap_k + 1]
    int *gvert = nullptr;        // [4 cap_k]
    float *winv = nullptr;       // [4 cap_k]
    double *u64 = nullptr;       // [3 * 4 cap_k]
    float *u32 = nullptr;        // [4 * 4 cap_k] (float4 per touched vertex)
    double *red = nullptr;       // reduction partials [1024]
    int *d_U = nullptr;          // touched vertex count (device)
    int *iwork = nullptr;        // [16] solver control words (zeroed by the caller before a solve)
    double *dwork = nullptr;     // [16]
};

// StageMark brackets a launch for the caller's stage profiler (fn(arg, 1, s)
// before it, fn(arg, 0, s) after; no-op when fn is null).
struct StageMark {
    void (*fn)(void *arg, int begin, cudaStream_t s) = nullptr;
    void *arg = nullptr;
    void operator()(int begin, cudaStream_t s) const {
        if (fn) fn(arg, begin, s);
    }
};
struct SolveParams {
    int solver;
    int max_cg_iters;
    int max_refine;
    double rel_tol;
    double inner_tol;
    int block_switch = 48;  // iterations of a large zone's run before the blocks (-1: never)
    StageMark big_mark;  // brackets the launches of the zones of ZONE_BIG rows or more
};

void assemble(const MeshPair &mp, const hfcr_stencil *st, const int *d_k, int cap, double d,
              SolveBuffers &sb, uint32_t *d_status, cudaStream_t s);
// d_n4: device word receiving 4k (the CSR entry count)
// path 0: one cooperative launch (the multi-kernel sequence where that
// launch is refused); 1: the multi-kernel sequence
void build_vertex_csr(const MeshPair &mp, const int *d_k, int cap, SolveBuffers &sb, SortTemp &t,
                      int *d_n4, uint32_t *d_status, int path, cudaStream_t s);
// One-time kernel attributes (shared-memory opt-in); call outside stream capture.
void solver_init();
// Solves and leaves lambda in sb.lam; results (iters, residual) in sb.iwork / sb.dwork.
void solve(const SolveParams &p, const MeshPair &mp, const int *d_k, int cap, SolveBuffers &sb,
           uint32_t *d_status, cudaStream_t s);
// dx = -M^-1 J^T lambda for the touched vertices; apply to positions (apply=1)
// or write full dx arrays (zeroed first).
// apply 1: x += dx; 0: dx to dxA / dxB (three arrays each, mesh dtype);
// 2: dx to the float64 field dxA[0] (AoS over global vertex ids)
void displacement(const MeshPair &mp, int cap, SolveBuffers &sb, int apply, void *const *dxA,
                  void *const *dxB, cudaStream_t s);

int bits_for(long long n);  // smallest b with n <= 2^b (at least 1)

// diffusion of displacement vectors (diffuse.cu)
struct DiffMeshArgs {
    const int *ptr = nullptr, *nbr = nullptr;  // vertex adjacency CSR, ascending neighbours
    const float *inv_mass = nullptr;           // null: no kinematic vertices
    const int *rank = nullptr;                 // order of the band list (null: vertex order)
    int n = 0;                                 // vertices
};
// rank[v] = place of vertex v in the Morton order of the mesh's positions
// (30-bit codes in its bounding box, ties by index): the band list follows it,
// so that neighbouring band vertices sit close in the list.  Scratch: the
// diffusion's record buffer and partial-sum buffer (nothing kept there
// between calls).
void vertex_rank(const hfcr_mesh &m, int *rank, const struct DiffScratch &ds, SortTemp &t,
                 cudaStream_t s);
// CSR of an edge list: ptr [nv + 1], nbr [2 ne], cur [nv] scratch
void build_adjacency(const int *edges, int ne, int nv, int *ptr, int *nbr, int *cur, SortTemp &t,
                     uint32_t *d_status, cudaStream_t s);
// scratch of the harmonic diffusion (capacity cap = vertices of both meshes)
struct DiffScratch {
    int cap = 0;
    unsigned *flags = nullptr;  // [cap] band flags, scanned in place
    int *cidx = nullptr;        // [cap] band index of a vertex, -1 outside the band
    int *fv = nullptr;          // [cap] band vertices
    double *b64 = nullptr;      // [3 cap] right-hand side of the band system
    double *u64 = nullptr;      // [2 * 3 cap] float64 solution, alternating by round
    float *x32 = nullptr, *p32 = nullptr;  // [3 cap] float32 correction and search direction
    float *rec = nullptr;       // [2 * 12 cap] float32 CG records
    int *cnbr = nullptr;        // band index of every adjacency slot: A's slots, then B's from eoffB
    int eoffB = 0;
    double *part = nullptr;     // [2 * 9 * 1024] per-CTA partial sums
    unsigned *bar = nullptr;    // [1] grid barrier counter
    int *d_nfree = nullptr;     // band size (device)
    int *ctl = nullptr;         // [2] CG iterations (accumulated), unconverged flag
};
// Diffusion of the field u (AoS float64 over A's then B's vertices) over
// `rings` rings: the harmonic field (sweeps 0: conjugate gradients to the
// relative residual tol, at most max_iters iterations) or `sweeps` Jacobi
// sweeps.  Returns the buffer holding the result (u, or u_alt after an odd
// number of sweeps); ring [a.n + b.n] gets the ring distances (0: moved,
// rings + 1: beyond).

const double *diffuse_field(const DiffMeshArgs &a, const DiffMeshArgs &b, double *u, double *u_alt,
                            int *ring, int rings, int sweeps, double tol, int max_iters,
                            const DiffScratch &ds, SortTemp &t, uint32_t *d_status, cudaStream_t s,
                            const StageMark &mark = StageMark());
// one-time device query of the diffusion kernels; call outside stream capture
void diffusion_init();
void apply_field(const hfcr_mesh &A, const hfcr_mesh &B, const int *ring, int rings,
                 const double *u, cudaStream_t s);
void field_from_soa(const double *x, const double *y, const double *z, int n, double *u,
                    cudaStream_t s);
void field_to_soa(const double *u, int n, double *x, double *y, double *z, cudaStream_t s);

}  // namespace hfcr
