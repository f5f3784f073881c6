/*
 * hfcr.h - C ABI of the GB300 implementation of history-free collision
 * response between two triangle meshes (J. Ye, "History-free Collision
 * Response for Deformable Surfaces", arXiv 1409.2081).
 *
 * The library finds every edge-face (E-F) intersection between two meshes,
 * at least one of them oriented (Sec. 3), turns the crossings into
 * penetration stencils (Sec. 4, Fig. 3), and moves the stencil vertices by
 * the global displacement minimizer (Sec. 4, Eq. 3, solved through the
 * normal equations Eq. 7 / Eq. 8).  The repair loop repeats the three
 * steps until no intersection remains (Sec. 3).
 *
 * Conventions shared by every entry point:
 *  - All array pointers are DEVICE pointers unless a parameter says "host".
 *    The caller owns every input and output buffer; the library only reads
 *    inputs and writes outputs.  A context owns its scratch memory, which
 *    hfcr_reserve allocates; no other call allocates device memory.
 *  - Work is enqueued on the given CUDA stream (NULL = legacy default).
 *    Entry points that return a count (detect, build_stencils, resolve)
 *    synchronise that stream before returning; respond does not.
 *  - Positions are structure-of-arrays x[], y[], z[] of the mesh's dtype.
 *    float32 coordinates must be finite with magnitude at most 2^38;
 *    float64 coordinates must be finite and either 0 or of magnitude in
 *    [2^-200, 2^38].  Outside that range the exactness argument of the
 *    predicates does not hold and the call returns HFCR_ERR_RANGE (or
 *    HFCR_ERR_NONFINITE) without producing output.
 *  - Triangles are int32 [n_tris][3], counter-clockwise seen from the
 *    front side of an oriented mesh (the normal (b-a) x (c-a) points to
 *    the front).
 *  - Vertex and face ids in pairs and stencils are local to their mesh.
 *  - Errors are returned as hfcr_status; no C++ exception crosses the ABI.
 *    hfcr_last_error(ctx) gives a human-readable message.
 *  - A context keeps, between calls, data derived from the caller's
 *    buffers, keyed by their addresses and sizes: the traversal order and
 *    the vertex adjacency of a caller's edge list, and the hierarchy over a
 *    face mesh (refitted to the current positions on every call, rebuilt
 *    every bvh_rebuild_interval calls).  The positions may change freely.
 *    An edge list or a batch's segment table whose contents change while
 *    the same buffer is passed again must come with a new reservation
 *    (hfcr_reserve with larger sizes frees everything kept), or set
 *    bvh_rebuild_interval to 1 and pass the edges in a fresh buffer.
 *
 * Readings of the paper fixed by this interface:
 *  - An E-F intersection is a strict crossing of the face's plane by the
 *    edge inside the closed triangle: an endpoint on the plane, a coplanar
 *    edge, a zero-area face or a zero-length edge gives no pair; a crossing
 *    through a shared triangle edge or vertex is reported for every face
 *    containing that point.
 *  - Direction 0 pairs an edge of A with a face of B (needs B oriented);
 *    direction 1 an edge of B with a face of A (needs A oriented).
 *  - n is the unit face normal of the pre-response positions, alpha = 1/3
 *    (Eq. 1), x' = x - M^-1 grad(D)^T lambda with
 *    grad(D) M^-1 grad(D)^T lambda = grad(D) x - d (Eq. 8; d = 0 is Eq. 7).
 */
#ifndef HFCR_H
#define HFCR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HFCR_OK = 0,
    HFCR_ERR_ARG = 1,           /* invalid argument (NULL, negative size, no oriented mesh) */
    HFCR_ERR_CAPACITY = 2,      /* output or reserved scratch too small; *n_out holds the size needed */
    HFCR_ERR_CUDA = 3,          /* a CUDA call failed (see hfcr_last_error) */
    HFCR_ERR_NONFINITE = 4,     /* a position is NaN or infinite */
    HFCR_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
    HFCR_ERR_NOT_CONVERGED = 6, /* the solver or the repair loop stopped at its iteration limit */
    HFCR_ERR_UNSUPPORTED = 7,   /* option combination not implemented */
    HFCR_ERR_RANGE = 8          /* a coordinate is outside the range the exact predicates cover */
} hfcr_status;

typedef enum { HFCR_F32 = 0, HFCR_F64 = 1 } hfcr_dtype;

/* Solver of Eq. 7/8, one linear system per impact zone (Sec. 4).  MIXED:
 * conjugate gradients in float32 with float64 iterative refinement of the
 * residual against the float64 constraint gradients, each zone staged in
 * shared memory by a thread group sized to it; FP64: conjugate gradients
 * in float64 throughout, each zone by one CTA on global memory (with
 * float64 meshes and f32_filter 0 this is the plain float64 form);
 * FP64_GLOBAL: float64 conjugate gradients over the whole system in one
 * CTA (the same x', a different solver structure). */
typedef enum { HFCR_SOLVER_MIXED = 0, HFCR_SOLVER_FP64 = 1, HFCR_SOLVER_FP64_GLOBAL = 2 } hfcr_solver;

/* Role schedule of the repair loop when both meshes are oriented (Sec. 4:
 * "one is regarded as oriented and the other as un-oriented" in the
 * iterations).  ALTERNATE: iteration i tests direction i mod 2; BOTH: both
 * directions every iteration. */
typedef enum { HFCR_ROLES_ALTERNATE = 0, HFCR_ROLES_BOTH = 1 } hfcr_roles;

typedef struct {
    int32_t dtype;          /* hfcr_dtype of x, y, z */
    int32_t n_verts;
    void *x, *y, *z;        /* device [n_verts] each; resolve updates them in place */
    int32_t n_tris;
    const int32_t *tris;    /* device [n_tris][3] */
    int32_t n_edges;        /* 0 with edges == NULL: the library derives them */
    const int32_t *edges;   /* device [n_edges][2], unique, v0 < v1, lexicographic (see hfcr_build_edges) */
    int32_t oriented;       /* 1 = faces have a front side (closed outward surface) */
    const float *inv_mass;  /* device [n_verts] inverse masses M^-1, or NULL for all 1 (Sec. 4) */
} hfcr_mesh;

/* One E-F intersection: edge (v0 < v1) of the edge mesh crossing `face` of
 * the oriented mesh; dir 0 = edge of A / face of B, dir 1 = edge of B /
 * face of A. */
typedef struct { uint32_t dir, v0, v1, face; } hfcr_pair;

/* One penetration stencil {x0; face} (Sec. 4): x0 is the endpoint of a
 * crossing edge on the back side of `face`; mesh of x0 and of the face
 * follow `dir` as in hfcr_pair. */
typedef struct { uint32_t dir, x0, face, pad; } hfcr_stencil;

typedef struct {
    int32_t solver;         /* hfcr_solver (default MIXED) */
    int32_t f32_filter;     /* 1 (default): float32 meshes try the float32 filter first */
    int32_t roles;          /* hfcr_roles (default ALTERNATE) */
    int32_t max_cg_iters;   /* per float32 run of MIXED (default 500); FP64 runs once with max_cg_iters * max_refine */
    int32_t max_refine;     /* MIXED: float32 runs per impact zone, each followed by the zone's
                               float64 residual (default 6) */
    double rel_tol;         /* target |b - A lambda| / |b| (default 1e-12) */
    double inner_tol;       /* MIXED: residual reduction of one float32 run (default 1e-4) */
    int32_t graphs;         /* 1 (default): resolve replays each repair iteration as a captured
                               CUDA graph (re-captured when any argument changes); 0: plain launches.
                               Graphs are not used while the profiler is enabled. */
    int32_t diffuse_rings;  /* Sec. 5 diffusion in hfcr_resolve (see hfcr_diffuse): rings R of the
                               band; 0 (default): no diffusion, the minimizer's displacement is
                               applied as it is */
    int32_t diffuse_sweeps; /* 0 (default): the harmonic field (conjugate gradients to diffuse_tol);
                               S > 0: the fixed-sweep approximation, S Jacobi sweeps from zero */
    int32_t traverse_variant; /* traversal kernel variant 0..8 used until hfcr_autotune picks one
                                 (default 0; every variant finds the same pairs) */
    int32_t setup_path;     /* response setup (vertex CSR, impact zones, preconditioner groups):
                               0 (default) one cooperative launch, 1 a sequence of about 25
                               kernels; both build the same arrays, so the results are identical */
    int32_t diffuse_max_iters; /* harmonic diffusion: iteration limit (0: default 1000) */
    double diffuse_tol;     /* harmonic diffusion: stop at |r| <= diffuse_tol |b| per coordinate,
                               0 < tol < 1 (0: default 1e-10) */
    double amplification_limit; /* hfcr_resolve counts the responses whose max_dx / max_rhs
                                   exceeds it (0: default 1000) */
    int32_t bvh_rebuild_interval; /* a hierarchy built over the same face mesh (triangle buffer,
                                     counts, batch table) by an earlier call is refitted to the
                                     current positions (exact boxes) instead of rebuilt, up to this
                                     many calls in a row (0: default 8; 1: rebuild every call).
                                     Only the traversal's speed depends on it, never the pairs. */
    int32_t block_switch_iters; /* MIXED, impact zones of 1,024 rows or more: a float32 run that
                                   reaches this many iterations ends there, and the zone's later
                                   runs are preconditioned by blocks of up to 16 rows that share
                                   x0 or a face (ill-conditioned zones) instead of the groups of
                                   rows sharing x0 (0: default 48; -1: never) */
} hfcr_options;

typedef struct {
    int32_t cg_iters;        /* conjugate-gradient iterations, all runs */
    int32_t refine_rounds;   /* MIXED: the most float32 runs any impact zone needed */
    double rel_residual;     /* |b - A lambda| / |b| at exit, float64 (MIXED: every zone stops
                                at |r_zone| <= rel_tol |b_zone|, which bounds the whole) */
    int32_t converged;       /* rel_residual <= rel_tol */
    int32_t n_stencils;
    int32_t n_touched;       /* distinct vertices in the stencils */
    double max_rhs;          /* largest |D - d| of the stencils (Eq. 8) */
    double max_dx;           /* largest displacement component |dx|; max_dx / max_rhs is the
                                response's amplification: below ~10 for a well-posed system,
                                far above when Eq. 7 is nearly singular (e.g. a stencil whose
                                face is kinematic and whose x0 crosses near-parallel faces) */
} hfcr_solve_info;

typedef struct {
    int64_t narrow_tests;    /* segment-triangle tests run at BVH leaves */
    int64_t f64_fallbacks;   /* orientation signs the float32 filter left open */
    int64_t exact_fallbacks; /* signs the float64 filter left open (exact expansion arithmetic) */
    int64_t brute_force_equiv; /* |E| x |F| summed over the tested directions */
} hfcr_detect_stats;

typedef struct {
    int32_t iters;                 /* detections run */
    int32_t converged;             /* the last detections of every active direction found no pair */
    int64_t pairs_first;           /* pairs of the first detection */
    int64_t pairs_last;            /* pairs of the last detection */
    int64_t total_pairs;           /* pairs over all detections */
    int64_t total_stencils;
    int32_t cg_iters;              /* all solves */
    double worst_rel_residual;     /* largest solver residual over the iterations */
    hfcr_detect_stats stats;       /* summed over the detections */
    int32_t solver_path;           /* bit 0: the float32 CG ran in shared memory, bit 1: in global
                                      memory; bit 2: the float64 per-zone CG ran (the float64
                                      form, or in the mixed form for a zone whose float32 runs
                                      stopped reducing its residual before rel_tol) */
    int32_t diffuse_cg_iters;      /* harmonic diffusion: CG iterations over all iterations */
    int32_t diffuse_unconverged;   /* iterations whose harmonic diffusion stopped at diffuse_max_iters */
    double worst_amplification;    /* largest max_dx / max_rhs of a response (see hfcr_solve_info) */
    int32_t amplified_iters;       /* responses whose amplification exceeded the option
                                      amplification_limit: an ill-conditioned system moved
                                      vertices far more than the penetration depths */
    int64_t band_vertices;         /* harmonic diffusion: free band vertices (the unknowns of
                                      the band's Dirichlet problem), summed over the iterations */
    int64_t big_zone_rows;         /* MIXED: rows of the impact zones solved one CTA or one
                                      cluster per zone: those of 1,024 rows or more, and
                                      those of 256 or more when there are at most as many
                                      of them as the launch's CTAs; summed over the
                                      iterations */
    int64_t big_zone_vertices;     /* and the vertices those zones touch */
} hfcr_resolve_info;

/* Stages timed by the optional profiler (instrumentation; the paper has no
 * counterpart). */
typedef enum {
    HFCR_STAGE_VALIDATE = 0,  /* input range / finiteness checks */
    HFCR_STAGE_BVH = 1,       /* hierarchy build and refit */
    HFCR_STAGE_TRAVERSE = 2,  /* the traversal + exact narrow-phase kernel, one interval per launch */
    HFCR_STAGE_STENCILS = 3,  /* pair sort, pair records, stencil keys, sort, unique */
    HFCR_STAGE_ASSEMBLE = 4,  /* constraint rows and the vertex CSR */
    HFCR_STAGE_SOLVE = 5,     /* Eq. 7 / Eq. 8 solve */
    HFCR_STAGE_DISPLACE = 6,  /* x' - x and its application */
    HFCR_STAGE_DIFFUSE = 7,   /* diffusion of the displacement (Sec. 5) and its application */
    HFCR_STAGE_BAND_CG = 8,   /* the band CG kernels alone: their intervals lie inside DIFFUSE's,
                                 so they are not added to the other stages */
    HFCR_STAGE_ZONE_BIG = 9,  /* the solver launches of the impact zones of 1,024 rows or more
                                 (MIXED), inside SOLVE's intervals */
    HFCR_N_STAGES = 10
} hfcr_stage;

typedef struct {
    double ms[HFCR_N_STAGES];          /* summed CUDA-event time per stage */
    int64_t intervals[HFCR_N_STAGES];  /* timed intervals per stage */
} hfcr_profile;

typedef struct hfcr_ctx hfcr_ctx;

/* Create a context.  opt may be NULL (defaults above).  Allocates nothing
 * on the device.  Returns HFCR_ERR_ARG for a NULL ctx pointer. */
hfcr_status hfcr_create(hfcr_ctx **ctx, const hfcr_options *opt);

/* Destroy a context and free its scratch.  NULL is accepted. */
hfcr_status hfcr_destroy(hfcr_ctx *ctx);

/* Allocate the context's device scratch for meshes of up to max_verts
 * vertices and max_tris triangles each and up to max_pairs E-F pairs per
 * detection (stencils <= pairs).  May be called again to grow; calls that
 * exceed the reserved sizes return HFCR_ERR_CAPACITY.  Synchronous. */
hfcr_status hfcr_reserve(hfcr_ctx *ctx, int64_t max_verts, int64_t max_tris, int64_t max_pairs);

/* Unique undirected edges (v0 < v1, lexicographic) of a triangle list: the
 * primitives of the detection (every face-face contact decomposes into two
 * E-F contacts, Sec. 4).  out: device int32 [cap][2]; *n_out (host) gets
 * the edge count, HFCR_ERR_CAPACITY if it exceeds cap.  Synchronises. */
hfcr_status hfcr_build_edges(hfcr_ctx *ctx, const int32_t *tris, int32_t n_tris, int32_t n_verts,
                             int32_t *out, int64_t cap, int64_t *n_out, void *stream);

/* hfcr_build_edges for callers that cannot allocate device memory: the
 * same sorted unique edges, computed without a context and without any
 * cudaMalloc, cudaFree or other allocating call.  The paper has no
 * counterpart; this exists for code that may not allocate on the device
 * while it runs - for example a host application whose device memory is
 * owned by its own pool or budget, a plugin that is given device buffers
 * but no right to allocate, or a latency-critical loop that cannot afford
 * cudaMalloc's implicit synchronisation.
 *
 * Its scratch is one fixed device array inside the library (about 3.9 MB,
 * enough for n_tris <= 65,536), which every GPU that loads the library
 * holds until the process exits.  Larger inputs return HFCR_ERR_CAPACITY
 * (message in hfcr_last_error(NULL)), as does cap < 3 * n_tris: out must
 * have room for the largest possible edge count; a vertex index outside
 * [0, n_verts) returns HFCR_ERR_ARG.  The first call on a device looks up
 * that device's address of the array (cudaGetSymbolAddress) and keeps it
 * for the process; make that first call before any stream capture.  After
 * cudaDeviceReset the kept address is no longer valid: do not call this
 * entry point again in that process.  All calls share the one array:
 * calls that overlap on the GPU (different streams, or different host
 * threads) race and give undefined results; calls in sequence are fine,
 * since each call clears the words it needs cleared.
 * tris, out: device; *n_out (host) gets the edge count.  The call
 * synchronises `stream` before it returns (it reads the count back). */
hfcr_status hfcr_build_edges_noalloc(const int32_t *tris, int32_t n_tris, int32_t n_verts,
                                     int32_t *out, int64_t cap, int64_t *n_out, void *stream);

/* Exact discrete collision detection (Sec. 3): every E-F pair of the
 * active directions (0 when B is oriented, 1 when A is), sorted by
 * (dir, v0, v1, face).  out: device [cap]; *n_out (host) gets the pair
 * count (HFCR_ERR_CAPACITY when above cap, out then holds the first cap in
 * unspecified order).  stats may be NULL.  Synchronises. */
hfcr_status hfcr_detect(hfcr_ctx *ctx, const hfcr_mesh *A, const hfcr_mesh *B,
                        hfcr_pair *out, int64_t cap, int64_t *n_out,
                        hfcr_detect_stats *stats, void *stream);

/* hfcr_detect over a batch of independent mesh pairs (A_i, B_i), i <
 * n_pairs, in one set of launches: each edge of A_i is tested against the
 * faces of B_i only (and each edge of B_i against A_i's faces).  A and B
 * are the concatenations of the A_i and of the B_i: positions and faces
 * back to back, triangle vertex ids global within the concatenation.
 * segs: device int32 [(n_pairs + 1)][4], row i = first vertex of A_i, first
 * face of A_i, first vertex of B_i, first face of B_i; row n_pairs =
 * (A.n_verts, A.n_tris, B.n_verts, B.n_tris); rows non-decreasing (checked:
 * HFCR_ERR_ARG otherwise).  The oriented flags of A and B apply to every
 * pair.  Pairs are reported with global ids, sorted by (dir, v0, v1,
 * face); a pair's mesh index follows from the offsets.  Synchronises. */
hfcr_status hfcr_detect_batch(hfcr_ctx *ctx, const hfcr_mesh *A, const hfcr_mesh *B,
                              int32_t n_pairs, const int32_t *segs, hfcr_pair *out, int64_t cap,
                              int64_t *n_out, hfcr_detect_stats *stats, void *stream);

/* Penetration stencils from sorted pairs (Sec. 3 and Sec. 4, Fig. 3):
 * x0 = the endpoint on the back side of the face (exact sign), identical
 * (dir, x0, face) merged, sorted.  out: device [cap]; *n_out (host) gets
 * the count.  Synchronises. */
hfcr_status hfcr_build_stencils(hfcr_ctx *ctx, const hfcr_mesh *A, const hfcr_mesh *B,
                                const hfcr_pair *pairs, int64_t n_pairs,
                                hfcr_stencil *out, int64_t cap, int64_t *n_out, void *stream);

/* Global displacement minimizer (Sec. 4, Eq. 3 via Eq. 8): for k stencils
 * on the current positions, writes dxA [A.n_verts], dxB [B.n_verts]
 * (device SoA pairs of three arrays each, in the mesh's dtype: dx?[0]=x,
 * [1]=y, [2]=z) with x' = x + dx; untouched vertices get 0.  info (host,
 * may be NULL) is filled after the stream is synchronised when non-NULL. */
hfcr_status hfcr_respond(hfcr_ctx *ctx, const hfcr_mesh *A, const hfcr_mesh *B,
                         const hfcr_stencil *st, int64_t k, double d,
                         void *const *dxA, void *const *dxB, hfcr_solve_info *info, void *stream);

/* Diffusion of a displacement field over one mesh (Sec. 5: the
 * correction is propagated from the penetrating vertices to their vicinity
 * as a harmonic vector field; the paper gives no equations, this is the
 * reading implemented).  On the graph of M's edges (M.edges, or derived
 * from the triangles): vertices with a nonzero displacement keep it,
 * vertices more than `rings` edges from all of them, and kinematic
 * vertices (M.inv_mass 0), get 0 (Dirichlet values), and every vertex in
 * between (the band) gets the value that makes it the mean of its
 * neighbours.  sweeps == 0: that harmonic field, solved per coordinate by
 * Jacobi-preconditioned conjugate gradients on the band's graph Laplacian
 * to |r| <= diffuse_tol |b| (options), HFCR_ERR_NOT_CONVERGED when
 * diffuse_max_iters iterations do not reach it; sweeps > 0: the fixed-sweep
 * approximation instead, `sweeps` Jacobi sweeps of the neighbour mean
 * starting from 0 (each mean summed in ascending vertex order in float64).
 * dx, dy, dz: device float64 [M.n_verts], read and overwritten.  rings in
 * [0, 1024] (0 leaves the field as it is), sweeps in [0, 100000].
 * Synchronises. */
hfcr_status hfcr_diffuse(hfcr_ctx *ctx, const hfcr_mesh *M, double *dx, double *dy, double *dz,
                         int32_t rings, int32_t sweeps, void *stream);

/* The repair loop (Sec. 3): detect, build stencils, displace, repeated
 * until no E-F intersection remains or max_iters detections ran.  Updates
 * A and B's positions in place.  With option diffuse_rings > 0, each
 * iteration's displacement is first spread over both meshes as by
 * hfcr_diffuse (Sec. 5; the harmonic field unless diffuse_sweeps > 0), then
 * applied.  info (host) may be NULL.  Returns HFCR_ERR_NOT_CONVERGED when the loop stopped at
 * max_iters.  Synchronises. */
hfcr_status hfcr_resolve(hfcr_ctx *ctx, hfcr_mesh *A, hfcr_mesh *B, double d, int32_t max_iters,
                         hfcr_resolve_info *info, void *stream);

/* Autotuner of the traversal kernel (no counterpart in the paper): builds
 * the hierarchies for A and B (a batch laid out as in hfcr_detect_batch
 * when segs is given, one pair when segs is NULL and n_pairs is ignored),
 * times every traversal variant three times on this scene and makes the
 * fastest the context's choice for every later call.  The variants span:
 * the register budget (2, 3 or 4 CTAs of 256 threads per SM), the exact
 * narrow phase inline or out of line, one walk per edge or one per warp of
 * edges of the same mesh pair (0 to 4), and persistent walks fed by a
 * device work queue of edges, with 3 or 4 CTAs per SM and a warp refilling
 * its idle lanes once 8 or 16 are idle (5 to 8).  The stack depth is not
 * tuned: it is set by the deepest tree the build makes.  *chosen (host,
 * may be NULL) gets the chosen index; ms (host [n_ms], may be NULL) the
 * best time of each variant per traversal launch (one launch per direction
 * with edges, as a repair iteration of that direction runs it).
 * Synchronises. */
hfcr_status hfcr_autotune(hfcr_ctx *ctx, const hfcr_mesh *A, const hfcr_mesh *B, int32_t n_pairs,
                          const int32_t *segs, int32_t *chosen, double *ms, int32_t n_ms,
                          void *stream);

/* Profiler (instrumentation, no counterpart in the paper).  When enabled,
 * every later call records CUDA events on its stream around each stage;
 * enabling resets the sums.  hfcr_profile_read waits for the recorded
 * events and returns the sums. */
hfcr_status hfcr_profile_enable(hfcr_ctx *ctx, int32_t on);
hfcr_status hfcr_profile_read(hfcr_ctx *ctx, hfcr_profile *out);

/* Kernel launches made by this library in this process so far
 * (instrumentation, no counterpart in the paper). */
int64_t hfcr_launch_count(void);

/* hfcr_resolve over a batch of independent mesh pairs laid out as in
 * hfcr_detect_batch: one repair loop for all pairs (each iteration detects
 * every pair, and the minimizer's impact zones never span two pairs, so
 * the result equals resolving the pairs one by one with the same iteration
 * schedule); the loop ends when no pair has an intersection or after
 * max_iters detections.  Positions are updated in place.  Synchronises. */
hfcr_status hfcr_resolve_batch(hfcr_ctx *ctx, hfcr_mesh *A, hfcr_mesh *B, int32_t n_pairs,
                               const int32_t *segs, double d, int32_t max_iters,
                               hfcr_resolve_info *info, void *stream);

/* Message of the last failing call on this context ("" if none); with
 * ctx == NULL, of the last failing context-free call of this thread. */
const char *hfcr_last_error(const hfcr_ctx *ctx);

/* Static name of a status code. */
const char *hfcr_status_string(hfcr_status s);

#ifdef __cplusplus
}
#endif
#endif /* HFCR_H */
