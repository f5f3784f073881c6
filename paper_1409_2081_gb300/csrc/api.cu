// C ABI of libhfcr: context, scratch reservation and the entry points that
// chain the detection (Sec. 3), the stencils (Sec. 4) and the minimizer
// (Sec. 4, Eqs. 3-8) into the repair loop (Sec. 3).
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "internal.h"

using namespace hfcr;

std::atomic<long long> hfcr::g_launches{0};

namespace hfcr {
// message of the last failing context-free call of this thread
static thread_local std::string g_noctx_err;
void set_noctx_error(const std::string &msg) { g_noctx_err = msg; }
}  // namespace hfcr

struct ProfInterval {
    int stage;
    cudaEvent_t a, b;
    bool pooled = true;  // false: the events belong to a captured graph
};

// A captured repair iteration: the exact launch sequence of one set of
// arguments, replayed with cudaGraphLaunch.
struct GraphEntry {
    std::string key;
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;
    unsigned long long last_use = 0;
};

// The small device words of one call (status, statistics, counters, solver
// control words and scalars, the touched-vertex count): one allocation, so
// that a call clears them with one memset and reads them back with one
// copy into the pinned mirror of the same layout.
struct DevWords {
    uint32_t status;
    uint32_t pad0;
    DevStats stats;
    int cnt[16];
    int iwork[16];
    double dwork[16];
    int touched;
    int pad1[3];
};

struct hfcr_ctx {
    hfcr_options opt;
    std::string err;
    int64_t max_verts = 0, max_tris = 0, max_pairs = 0;
    int device = 0;
    DevWords *d_words = nullptr;  // the words below point into these two
    DevWords *h_words = nullptr;  // pinned mirror
    uint32_t *d_status = nullptr;
    DevStats *d_stats = nullptr;
    int *d_cnt = nullptr;         // [16] device counters
    uint32_t *h_status = nullptr;
    int *h_cnt = nullptr;         // [16]
    DevStats *h_stats = nullptr;
    double *h_dw = nullptr;       // solver scalars
    int trav_variant = 0;         // traversal variant (hfcr_autotune)
    int *d_segs = nullptr;        // [8] segment table of a single mesh pair
    int *h_segs = nullptr;        // pinned [8]
    int *h_iw = nullptr;          // solver control words
    SortTemp sort;
    Bvh bvh[2];                   // [0]: faces of B (direction 0), [1]: faces of A (direction 1)
    // what each hierarchy was last built over, and the calls since: a later
    // call over the same faces refits it (exact boxes) and rebuilds it only
    // every opt.bvh_rebuild_interval calls
    struct BvhKey {
        const void *tris = nullptr;
        const int *segs = nullptr;
        int n_tris = -1, n_verts = -1, nseg = -1, dtype = -1;
    } bvh_key[2];
    int bvh_age[2] = {0, 0};
    int *edges[2] = {nullptr, nullptr};
    // traversal order of each edge list (a permutation; it only steers
    // performance, so a stale one for a moved mesh is still correct)
    int *eorder[2] = {nullptr, nullptr};
    const int *eorder_src[2] = {nullptr, nullptr};
    int eorder_n[2] = {0, 0};
    unsigned long long *ekeys = nullptr, *ekeys_alt = nullptr;
    unsigned *eflags = nullptr;
    unsigned long long *pkeys = nullptr, *pkeys_alt = nullptr;
    unsigned long long *skeys = nullptr, *skeys_alt = nullptr;
    unsigned *sflags = nullptr;
    hfcr_stencil *stencils = nullptr;
    SolveBuffers sb;
    // diffusion (Sec. 5): vertex adjacency per mesh, float64 field ping-pong
    // over both meshes' vertices (AoS), ring distances
    int *adj_ptr[2] = {nullptr, nullptr}, *adj_nbr[2] = {nullptr, nullptr}, *adj_cur = nullptr;
    int *adj_rank[2] = {nullptr, nullptr};  // Morton rank of each vertex (cached adjacencies)
    bool adj_ranked[2] = {false, false};
    const int *adj_src[2] = {nullptr, nullptr};  // caller edge list behind adj_ptr / adj_nbr
    int adj_ne[2] = {0, 0}, adj_nv[2] = {0, 0};
    double *field = nullptr, *field_alt = nullptr;
    int *ring = nullptr;
    DiffScratch dscr;             // the harmonic diffusion's band and CG state
    // profiler
    bool prof_on = false;
    double prof_ms[HFCR_N_STAGES] = {0};
    long long prof_n[HFCR_N_STAGES] = {0};
    std::vector<ProfInterval> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    // graph replay
    std::vector<GraphEntry> graphs;
    unsigned long long graph_clock = 0;
    cudaStream_t own = nullptr;          // used when the caller passes the legacy default stream
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

// device counter slots
enum { C_PAIRS = 0, C_STENCILS = 1, C_EDGES_A = 2, C_EDGES_B = 3, C_N4 = 4, C_NPAIRS_IN = 5, C_PEFF = 6,
       C_DIFF_ITERS = 7, C_DIFF_FAIL = 8, C_NFREE = 9, C_QUEUE = 10 };

namespace {

hfcr_status fail(hfcr_ctx *c, hfcr_status s, const char *fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

#define CK(call)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(ctx, HFCR_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    return cudaMalloc((void **)p, sizeof(T) * n);
}

void free_all(hfcr_ctx *c) {
    void *ptrs[] = {c->d_words, c->sort.hist, c->edges[0], c->edges[1],
                    c->ekeys, c->ekeys_alt, c->eflags, c->pkeys, c->pkeys_alt,
                    c->skeys, c->skeys_alt, c->sflags, c->stencils,
                    c->sb.ids_raw, c->sb.n64_raw, c->sb.n32_raw, c->sb.b_raw, c->sb.parent,
                    c->sb.zkey, c->sb.zkey_alt, c->sb.szone, c->sb.zs, c->sb.zv, c->sb.d_nz,
                    c->sb.ck64, c->sb.ck64_alt, c->sb.gst, c->sb.zg, c->sb.d_ng, c->sb.pinv,
                    c->sb.z32,
                    c->sb.ids, c->sb.n64, c->sb.n32, c->sb.b, c->sb.lam, c->sb.r64, c->sb.r32,
                    c->sb.x32, c->sb.p32, c->sb.q32, c->sb.w32, c->sb.p64, c->sb.q64, c->sb.cg64, c->sb.pinv64, c->sb.binv, c->sb.vidx, c->sb.ckey,
                    c->sb.ckey_alt, c->sb.cval, c->sb.cval_alt, c->sb.cflag, c->sb.seg, c->sb.gvert,
                    c->sb.winv, c->sb.u64, c->sb.u32, c->sb.red};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    void *dp[] = {c->adj_ptr[0], c->adj_ptr[1], c->adj_nbr[0], c->adj_nbr[1], c->adj_cur,
                  c->adj_rank[0], c->adj_rank[1], c->field,
                  c->field_alt, c->ring, c->eorder[0], c->eorder[1], c->dscr.flags, c->dscr.cidx,
                  c->dscr.fv, c->dscr.b64, c->dscr.u64, c->dscr.x32, c->dscr.p32, c->dscr.rec,
                  c->dscr.cnbr, c->dscr.part, c->dscr.bar};
    for (void *p : dp)
        if (p) cudaFree(p);
    c->adj_ptr[0] = c->adj_ptr[1] = c->adj_nbr[0] = c->adj_nbr[1] = c->adj_cur = nullptr;
    c->adj_rank[0] = c->adj_rank[1] = nullptr;
    c->adj_ranked[0] = c->adj_ranked[1] = false;
    c->field = c->field_alt = nullptr;
    c->ring = nullptr;
    c->dscr = DiffScratch();
    for (int i = 0; i < 2; ++i) {
        c->bvh_key[i] = hfcr_ctx::BvhKey();
        c->bvh_age[i] = 0;
    }
    c->adj_src[0] = c->adj_src[1] = nullptr;
    c->eorder[0] = c->eorder[1] = nullptr;
    c->eorder_src[0] = c->eorder_src[1] = nullptr;
    c->eorder_n[0] = c->eorder_n[1] = 0;
    for (int i = 0; i < 2; ++i) {
        Bvh &b = c->bvh[i];
        void *bp[] = {b.nodes, b.parent, b.flags, b.leaf_face, b.leaf_tri, b.keys, b.keys_alt,
                      b.vals_alt, b.bounds, b.bounds_part, b.d_rest};
        for (void *p : bp)
            if (p) cudaFree(p);
        b = Bvh();
    }
    if (c->h_words) cudaFreeHost(c->h_words);
    if (c->h_segs) cudaFreeHost(c->h_segs);
    if (c->d_segs) cudaFree(c->d_segs);
    c->d_words = nullptr; c->h_words = nullptr;
    c->d_status = nullptr; c->d_stats = nullptr; c->d_cnt = nullptr; c->sort = SortTemp();
    c->edges[0] = c->edges[1] = nullptr;
    c->ekeys = c->ekeys_alt = nullptr; c->eflags = nullptr;
    c->pkeys = c->pkeys_alt = nullptr;
    c->skeys = c->skeys_alt = nullptr; c->sflags = nullptr; c->stencils = nullptr;
    c->sb = SolveBuffers();
    c->h_status = nullptr; c->h_cnt = nullptr; c->h_stats = nullptr; c->h_dw = nullptr; c->h_iw = nullptr;
    c->h_segs = nullptr; c->d_segs = nullptr;
    c->max_verts = c->max_tris = c->max_pairs = 0;
}

cudaEvent_t prof_event(hfcr_ctx *c) {
    cudaEvent_t e = nullptr;
    if (!c->prof_pool.empty()) {
        e = c->prof_pool.back();
        c->prof_pool.pop_back();
    } else {
        cudaEventCreate(&e);
    }
    return e;
}

void prof_begin(hfcr_ctx *c, int stage, cudaStream_t s) {
    if (!c->prof_on) return;
    ProfInterval iv{stage, prof_event(c), nullptr};
    cudaEventRecord(iv.a, s);
    c->prof_pending.push_back(iv);
}

void prof_end(hfcr_ctx *c, int stage, cudaStream_t s) {
    if (!c->prof_on) return;
    for (auto it = c->prof_pending.rbegin(); it != c->prof_pending.rend(); ++it)
        if (it->stage == stage && !it->b) {
            it->b = prof_event(c);
            cudaEventRecord(it->b, s);
            return;
        }
}

// the band CG's own interval, nested inside the diffusion stage's
void band_mark(void *c, int begin, cudaStream_t s) {
    if (begin)
        prof_begin((hfcr_ctx *)c, HFCR_STAGE_BAND_CG, s);
    else
        prof_end((hfcr_ctx *)c, HFCR_STAGE_BAND_CG, s);
}

// the large zones' solver launches, nested inside the solve stage
void zone_big_mark(void *c, int begin, cudaStream_t s) {
    if (begin)
        prof_begin((hfcr_ctx *)c, HFCR_STAGE_ZONE_BIG, s);
    else
        prof_end((hfcr_ctx *)c, HFCR_STAGE_ZONE_BIG, s);
}

// accumulates every closed interval (waits for its end event)
void prof_collect(hfcr_ctx *c) {
    std::vector<ProfInterval> keep;
    for (auto &iv : c->prof_pending) {
        if (!iv.b) { keep.push_back(iv); continue; }
        float ms = 0.f;
        cudaEventSynchronize(iv.b);
        if (cudaEventElapsedTime(&ms, iv.a, iv.b) == cudaSuccess) {
            c->prof_ms[iv.stage] += ms;
            c->prof_n[iv.stage] += 1;
        }
        if (iv.pooled) {
            c->prof_pool.push_back(iv.a);
            c->prof_pool.push_back(iv.b);
        }
    }
    c->prof_pending.swap(keep);
}

hfcr_status device_status(hfcr_ctx *ctx, uint32_t st) {
    if (st & ST_NONFINITE) return fail(ctx, HFCR_ERR_NONFINITE, "a position is NaN or infinite");
    if (st & ST_RANGE)
        return fail(ctx, HFCR_ERR_RANGE,
                    "a coordinate is outside the exact-predicate range (|c| <= 2^38; float64 "
                    "nonzero |c| >= 2^-200)");
    if (st & ST_BAD_INDEX) return fail(ctx, HFCR_ERR_ARG, "a vertex or face index is out of range");
    if (st & ST_TIMEOUT) return fail(ctx, HFCR_ERR_TIMEOUT, "a device-side wait gave up");
    return HFCR_OK;
}

hfcr_status check_mesh(hfcr_ctx *ctx, const hfcr_mesh *m, const char *name) {
    if (!m) return fail(ctx, HFCR_ERR_ARG, "mesh %s is NULL", name);
    if (m->dtype != HFCR_F32 && m->dtype != HFCR_F64)
        return fail(ctx, HFCR_ERR_ARG, "mesh %s: unknown dtype %d", name, m->dtype);
    if (m->n_verts < 0 || m->n_tris < 0 || m->n_edges < 0)
        return fail(ctx, HFCR_ERR_ARG, "mesh %s: negative size", name);
    if (m->n_verts > 0 && (!m->x || !m->y || !m->z))
        return fail(ctx, HFCR_ERR_ARG, "mesh %s: NULL positions", name);
    if (m->n_tris > 0 && !m->tris) return fail(ctx, HFCR_ERR_ARG, "mesh %s: NULL tris", name);
    if (m->n_edges > 0 && !m->edges) return fail(ctx, HFCR_ERR_ARG, "mesh %s: NULL edges", name);
    if (m->n_verts > ctx->max_verts || m->n_tris > ctx->max_tris)
        return fail(ctx, HFCR_ERR_CAPACITY,
                    "mesh %s (%d verts, %d tris) exceeds the reserved %lld verts / %lld tris", name,
                    m->n_verts, m->n_tris, (long long)ctx->max_verts, (long long)ctx->max_tris);
    if (m->n_edges > 3 * ctx->max_tris)
        return fail(ctx, HFCR_ERR_CAPACITY, "mesh %s: too many edges", name);
    return HFCR_OK;
}

hfcr_status check_pair(hfcr_ctx *ctx, const hfcr_mesh *A, const hfcr_mesh *B) {
    if (!ctx) return HFCR_ERR_ARG;
    if (ctx->max_tris == 0) return fail(ctx, HFCR_ERR_CAPACITY, "hfcr_reserve was not called");
    hfcr_status s = check_mesh(ctx, A, "A");
    if (s) return s;
    if ((s = check_mesh(ctx, B, "B"))) return s;
    if (A->dtype != B->dtype) return fail(ctx, HFCR_ERR_UNSUPPORTED, "A and B differ in dtype");
    if (!A->oriented && !B->oriented)
        return fail(ctx, HFCR_ERR_ARG, "at least one mesh must be oriented (Sec. 3)");
    return HFCR_OK;
}

// Edges of mesh `which` (0 = A, 1 = B): the caller's, or built into the
// context (synchronises to learn the count).
hfcr_status mesh_edges(hfcr_ctx *ctx, const hfcr_mesh *m, int which, const int **edges, int *ne,
                       cudaStream_t s) {
    if (m->edges) {
        *edges = m->edges;
        *ne = m->n_edges;
        return HFCR_OK;
    }
    int slot = which ? C_EDGES_B : C_EDGES_A;
    build_edges(m->tris, m->n_tris, m->n_verts, ctx->edges[which], ctx->d_cnt + slot, ctx->ekeys,
                ctx->ekeys_alt, ctx->eflags, ctx->sort, ctx->d_status, s);
    CK(cudaMemcpyAsync(ctx->h_cnt + slot, ctx->d_cnt + slot, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *edges = ctx->edges[which];
    *ne = ctx->h_cnt[slot];
    return HFCR_OK;
}

struct DetectPlan {
    const int *edges[2] = {nullptr, nullptr};  // edges of A, of B
    int ne[2] = {0, 0};
    int edge_bits = 1, face_bits = 1;
    const int *segs = nullptr;  // segment table (one row per mesh pair + a closing row)
    int nseg = 1;
};

hfcr_status plan_detect(hfcr_ctx *ctx, const hfcr_mesh *A, const hfcr_mesh *B, bool dir0, bool dir1,
                        DetectPlan &pl, cudaStream_t s, const int *segs = nullptr, int nseg = 1) {
    hfcr_status st;
    if (segs) {
        pl.segs = segs;
        pl.nseg = nseg;
    } else {
        // a single pair: one segment covering both meshes
        const int one[8] = {0, 0, 0, 0, A->n_verts, A->n_tris, B->n_verts, B->n_tris};
        memcpy(ctx->h_segs, one, sizeof one);
        CK(cudaMemcpyAsync(ctx->d_segs, ctx->h_segs, sizeof one, cudaMemcpyHostToDevice, s));
        pl.segs = ctx->d_segs;
        pl.nseg = 1;
    }
    if (dir0 && A->n_tris > 0 && (st = mesh_edges(ctx, A, 0, &pl.edges[0], &pl.ne[0], s))) return st;
    if (dir1 && B->n_tris > 0 && (st = mesh_edges(ctx, B, 1, &pl.edges[1], &pl.ne[1], s))) return st;
    for (int d = 0; d < 2; ++d) {
        if (!pl.edges[d] || pl.ne[d] <= 0) continue;
        if (ctx->eorder_src[d] == pl.edges[d] && ctx->eorder_n[d] == pl.ne[d]) continue;
        // first use of this edge list: its traversal order from the current
        // positions (kept for later calls)
        const hfcr_mesh &E = d == 0 ? *A : *B;
        edge_order(pl.edges[d], pl.ne[d], E, pl.segs, d == 0 ? 0 : 2, pl.nseg, ctx->eorder[d],
                   (int *)ctx->eflags, ctx->ekeys, ctx->ekeys_alt, ctx->bvh[d].bounds_part,
                   ctx->bvh[d].bounds, ctx->sort, ctx->d_status, s);
        CK(cudaGetLastError());
        ctx->eorder_src[d] = pl.edges[d];
        ctx->eorder_n[d] = pl.ne[d];
    }
    int maxe = pl.ne[0] > pl.ne[1] ? pl.ne[0] : pl.ne[1];
    int maxf = A->n_tris > B->n_tris ? A->n_tris : B->n_tris;
    pl.edge_bits = bits_for(maxe > 1 ? maxe : 2);
    pl.face_bits = bits_for(maxf > 1 ? maxf : 2);
    return HFCR_OK;
}

// Whether the hierarchy of direction d can be refitted instead of rebuilt
// for faces F: it was built over the same triangle buffer, counts and
// segment table, fewer than bvh_rebuild_interval calls ago.
bool bvh_reusable(const hfcr_ctx *ctx, int d, const hfcr_mesh &F, const DetectPlan &pl) {
    const hfcr_ctx::BvhKey &k = ctx->bvh_key[d];
    return ctx->opt.bvh_rebuild_interval > 1 && k.tris == F.tris && k.n_tris == F.n_tris &&
           k.n_verts == F.n_verts && k.segs == pl.segs && k.nseg == pl.nseg && k.dtype == F.dtype &&
           ctx->bvh_age[d] < ctx->opt.bvh_rebuild_interval - 1 && ctx->bvh[d].n == F.n_tris;
}

// The hierarchies a call may keep (built[d] true: refit only)
void bvh_start(const hfcr_ctx *ctx, const hfcr_mesh *A, const hfcr_mesh *B, const DetectPlan &pl,
               bool *built) {
    built[0] = bvh_reusable(ctx, 0, *B, pl);
    built[1] = bvh_reusable(ctx, 1, *A, pl);
}

void bvh_note(hfcr_ctx *ctx, int d, const hfcr_mesh &F, const DetectPlan &pl, bool rebuilt);

// After a call that started from kept[]: record the hierarchies it built
// and age the ones it kept
void bvh_finish(hfcr_ctx *ctx, const hfcr_mesh *A, const hfcr_mesh *B, const DetectPlan &pl,
                const bool *kept, const bool *built) {
    for (int d = 0; d < 2; ++d) {
        if (kept[d]) bvh_note(ctx, d, d == 0 ? *B : *A, pl, false);
        else if (built[d]) bvh_note(ctx, d, d == 0 ? *B : *A, pl, true);
    }
}

// After a call: record a fresh build of direction d, or age the kept one.
void bvh_note(hfcr_ctx *ctx, int d, const hfcr_mesh &F, const DetectPlan &pl, bool rebuilt) {
    if (rebuilt) {
        hfcr_ctx::BvhKey &k = ctx->bvh_key[d];
        k.tris = F.tris;
        k.n_tris = F.n_tris;
        k.n_verts = F.n_verts;
        k.segs = pl.segs;
        k.nseg = pl.nseg;
        k.dtype = F.dtype;
        ctx->bvh_age[d] = 0;
    } else {
        ++ctx->bvh_age[d];
    }
}

// Launches the traversal of the active directions; positions validated and
// the BVHs refitted (built first when `build`).  Pair keys -> ctx->pkeys.
void launch_detect(hfcr_ctx *ctx, const hfcr_mesh *A, const hfcr_mesh *B, bool dir0, bool dir1,
                   const DetectPlan &pl, bool *built, cudaStream_t s, bool traverse_only = false,
                   int variant = -1) {
    if (traverse_only) {
        // timing of the traversal alone (hierarchies already built and refitted)
        for (int d = 0; d < 2; ++d) {
            if (!(d == 0 ? dir0 : dir1)) continue;
            const hfcr_mesh &F = d == 0 ? *B : *A;
            const hfcr_mesh &E = d == 0 ? *A : *B;
            if (F.n_tris <= 0 || pl.ne[d] <= 0) continue;
            DetectArgs a;
            a.segs = pl.segs;
            a.nseg = pl.nseg;
            a.ecol = d == 0 ? 0 : 2;
            a.fcol = d == 0 ? 3 : 1;
            a.edge_mesh = &E;
            a.edges = pl.edges[d];
            a.order = (ctx->eorder_src[d] == pl.edges[d] && ctx->eorder_n[d] == pl.ne[d])
                          ? ctx->eorder[d]
                          : nullptr;
            a.n_edges = pl.ne[d];
            a.bvh = &ctx->bvh[d];
            a.dir = d;
            a.f32_filter = ctx->opt.f32_filter;
            a.edge_bits = pl.edge_bits;
            a.face_bits = pl.face_bits;
            a.keys = ctx->pkeys;
            a.d_count = ctx->d_cnt + C_PAIRS;
            a.cap = (int)ctx->max_pairs;
            a.stats = ctx->d_stats;
            a.variant = variant;
            a.queue = ctx->d_cnt + C_QUEUE;
            detect_launch(a, s, ctx->d_status);
        }
        return;
    }
    prof_begin(ctx, HFCR_STAGE_VALIDATE, s);
    validate_pair(*A, *B, ctx->d_status, s);
    check_segments(pl.segs, pl.nseg, *A, *B, ctx->d_status, s);
    prof_end(ctx, HFCR_STAGE_VALIDATE, s);
    for (int d = 0; d < 2; ++d) {
        if (!(d == 0 ? dir0 : dir1)) continue;
        const hfcr_mesh &F = d == 0 ? *B : *A;
        const hfcr_mesh &E = d == 0 ? *A : *B;
        if (F.n_tris <= 0 || pl.ne[d] <= 0) continue;
        Bvh &b = ctx->bvh[d];
        prof_begin(ctx, HFCR_STAGE_BVH, s);
        if (!built[d] || b.n != F.n_tris) {
            // direction 0 builds over B's faces (column 3), direction 1 over A's (column 1)
            bvh_build(b, F, pl.segs, d == 0 ? 3 : 1, pl.nseg, ctx->sort, ctx->d_status, s);
            built[d] = true;
        }
        bvh_refit(b, F, ctx->d_status, s);
        prof_end(ctx, HFCR_STAGE_BVH, s);
        DetectArgs a;
        a.segs = pl.segs;
        a.nseg = pl.nseg;
        a.ecol = d == 0 ? 0 : 2;  // edge mesh A (vertex column 0) or B (column 2)
        a.fcol = d == 0 ? 3 : 1;
        a.edge_mesh = &E;
        a.edges = pl.edges[d];
        a.order = (ctx->eorder_src[d] == pl.edges[d] && ctx->eorder_n[d] == pl.ne[d]) ? ctx->eorder[d]
                                                                                    : nullptr;
        a.n_edges = pl.ne[d];
        a.bvh = &b;
        a.dir = d;
        a.f32_filter = ctx->opt.f32_filter;
        a.edge_bits = pl.edge_bits;
        a.face_bits = pl.face_bits;
        a.keys = ctx->pkeys;
        a.d_count = ctx->d_cnt + C_PAIRS;
        a.cap = (int)ctx->max_pairs;
        a.stats = ctx->d_stats;
        a.variant = ctx->trav_variant;
        a.queue = ctx->d_cnt + C_QUEUE;
        prof_begin(ctx, HFCR_STAGE_TRAVERSE, s);
        detect_launch(a, s, ctx->d_status);
        prof_end(ctx, HFCR_STAGE_TRAVERSE, s);
        // a single pair's count is |edges| x |faces|, added on the host
        // (single_pair_bf); a batch counts per pair on the device
        if (pl.nseg > 1)
            pair_products(a.edges, a.n_edges, pl.segs, pl.nseg, a.ecol, a.fcol, F.n_tris,
                          ctx->d_stats, s);
    }
}

// brute-force-equivalent E-F tests of one detection of a single mesh pair
// (a batch counts its pairs on the device)
int64_t single_pair_bf(const DetectPlan &pl, bool d0, bool d1, const hfcr_mesh *A,
                       const hfcr_mesh *B) {
    if (pl.nseg > 1) return 0;
    return (d0 ? (int64_t)pl.ne[0] * B->n_tris : 0) + (d1 ? (int64_t)pl.ne[1] * A->n_tris : 0);
}

hfcr_status read_back(hfcr_ctx *ctx, cudaStream_t s) {
    CK(cudaMemcpyAsync(ctx->h_words, ctx->d_words, sizeof(DevWords), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    prof_collect(ctx);
    return device_status(ctx, *ctx->h_status);
}

void add_stats(hfcr_detect_stats *o, const DevStats &d) {
    o->narrow_tests += (int64_t)d.narrow_tests;
    o->f64_fallbacks += (int64_t)d.f64_fallbacks;
    o->exact_fallbacks += (int64_t)d.exact_fallbacks;
    o->brute_force_equiv += (int64_t)d.bf;
}

// sorted pair keys (count P on the host) -> hfcr_pair records in out
hfcr_status finish_pairs(hfcr_ctx *ctx, int P, const DetectPlan &pl, hfcr_pair *out,
                         cudaStream_t s) {
    if (P <= 0) return HFCR_OK;
    int bits = 1 + pl.edge_bits + pl.face_bits;
    prof_begin(ctx, HFCR_STAGE_STENCILS, s);
    bool flip = radix_sort_u64(ctx->pkeys, nullptr, ctx->pkeys_alt, nullptr, P, bits, ctx->sort, s);
    unsigned long long *sorted = flip ? ctx->pkeys_alt : ctx->pkeys;
    keys_to_pairs(sorted, ctx->d_cnt + C_PAIRS, P, pl.edges[0], pl.edges[1], pl.edge_bits,
                  pl.face_bits, out, s);
    prof_end(ctx, HFCR_STAGE_STENCILS, s);
    CK(cudaGetLastError());
    return HFCR_OK;
}

// pairs (count in d_cnt[slot]) -> unique stencils in out; returns k on the host
hfcr_status make_stencils(hfcr_ctx *ctx, const hfcr_mesh *A, const hfcr_mesh *B,
                          const hfcr_pair *pairs, int P, int slot, hfcr_stencil *out, int64_t *k,
                          cudaStream_t s) {
    *k = 0;
    if (P <= 0) return HFCR_OK;
    MeshPair mp{*A, *B};
    int maxv = A->n_verts > B->n_verts ? A->n_verts : B->n_verts;
    int maxf = A->n_tris > B->n_tris ? A->n_tris : B->n_tris;
    int vb = bits_for(maxv > 1 ? maxv : 2), fb = bits_for(maxf > 1 ? maxf : 2);
    prof_begin(ctx, HFCR_STAGE_STENCILS, s);
    stencil_keys(mp, pairs, ctx->d_cnt + slot, P, vb, fb, ctx->opt.f32_filter, ctx->skeys,
                 ctx->d_stats, ctx->d_status, s);
    bool flip = radix_sort_u64(ctx->skeys, nullptr, ctx->skeys_alt, nullptr, P, 1 + vb + fb,
                               ctx->sort, s);
    unsigned long long *sorted = flip ? ctx->skeys_alt : ctx->skeys;
    stencil_unique(sorted, ctx->d_cnt + slot, P, vb, fb, ctx->sflags, out, ctx->d_cnt + C_STENCILS,
                   ctx->sort, s);
    prof_end(ctx, HFCR_STAGE_STENCILS, s);
    hfcr_status st = read_back(ctx, s);
    if (st) return st;
    *k = ctx->h_cnt[C_STENCILS];
    return HFCR_OK;
}

SolveParams params_of(const hfcr_options &o) {
    SolveParams p;
    p.solver = o.solver;
    p.max_cg_iters = o.max_cg_iters;
    p.max_refine = o.max_refine;
    p.rel_tol = o.rel_tol;
    p.inner_tol = o.inner_tol;
    p.block_switch = o.block_switch_iters;
    return p;
}

// assemble, solve and displace k stencils (count in d_cnt[C_STENCILS])
hfcr_status run_response(hfcr_ctx *ctx, const hfcr_mesh *A, const hfcr_mesh *B,
                         const hfcr_stencil *st, int k, double d, int apply, void *const *dxA,
                         void *const *dxB, cudaStream_t s) {
    if (k <= 0) return HFCR_OK;
    MeshPair mp{*A, *B};
    prof_begin(ctx, HFCR_STAGE_ASSEMBLE, s);
    assemble(mp, st, ctx->d_cnt + C_STENCILS, k, d, ctx->sb, ctx->d_status, s);
    build_vertex_csr(mp, ctx->d_cnt + C_STENCILS, k, ctx->sb, ctx->sort, ctx->d_cnt + C_N4,
                     ctx->d_status, ctx->opt.setup_path, s);
    prof_end(ctx, HFCR_STAGE_ASSEMBLE, s);
    prof_begin(ctx, HFCR_STAGE_SOLVE, s);
    SolveParams sp = params_of(ctx->opt);
    if (ctx->prof_on) {
        sp.big_mark.fn = zone_big_mark;
        sp.big_mark.arg = ctx;
    }
    solve(sp, mp, ctx->d_cnt + C_STENCILS, k, ctx->sb, ctx->d_status, s);
    prof_end(ctx, HFCR_STAGE_SOLVE, s);
    prof_begin(ctx, HFCR_STAGE_DISPLACE, s);
    displacement(mp, k, ctx->sb, apply, dxA, dxB, s);
    prof_end(ctx, HFCR_STAGE_DISPLACE, s);
    CK(cudaGetLastError());
    return HFCR_OK;
}

bool diffusing(const hfcr_ctx *ctx) { return ctx->opt.diffuse_rings > 0; }

// vertex adjacency of both meshes for the diffusion, from their edge lists
// (the plan's, or derived from the triangles)
hfcr_status prepare_diffusion(hfcr_ctx *ctx, const hfcr_mesh *A, const hfcr_mesh *B,
                              DetectPlan &pl, cudaStream_t s) {
    const hfcr_mesh *M[2] = {A, B};
    for (int i = 0; i < 2; ++i) {
        if (M[i]->n_verts <= 0) continue;
        // a caller's edge list is taken to stay the same while its buffer
        // and counts do (as for the traversal order): its adjacency is kept
        if (M[i]->edges && ctx->adj_src[i] == M[i]->edges && ctx->adj_ne[i] == M[i]->n_edges &&
            ctx->adj_nv[i] == M[i]->n_verts)
            continue;
        const int *e = pl.edges[i];
        int ne = pl.ne[i];
        if (!e && M[i]->n_tris > 0) {
            hfcr_status st = mesh_edges(ctx, M[i], i, &e, &ne, s);
            if (st) return st;
        }
        build_adjacency(e, e ? ne : 0, M[i]->n_verts, ctx->adj_ptr[i], ctx->adj_nbr[i], ctx->adj_cur,
                        ctx->sort, ctx->d_status, s);
        // a kept adjacency also gets the Morton order of the band list (once)
        ctx->adj_ranked[i] = M[i]->edges != nullptr;
        if (ctx->adj_ranked[i]) vertex_rank(*M[i], ctx->adj_rank[i], ctx->dscr, ctx->sort, s);
        ctx->adj_src[i] = M[i]->edges;
        ctx->adj_ne[i] = M[i]->n_edges;
        ctx->adj_nv[i] = M[i]->n_verts;
    }
    CK(cudaGetLastError());
    return HFCR_OK;
}

// One repair iteration enqueued on device counts only: detection, clamped
// pair count, stencils, assembly, solve, applied displacement.  Grids are
// sized by the reserved capacity; kernels read the live counts.  Nothing is
// read back.  The pair keys stay in the order the traversal appended them:
// the stencils are sorted and deduplicated on their own keys, so their list
// does not depend on that order.
void enqueue_iteration(hfcr_ctx *ctx, const hfcr_mesh *A, const hfcr_mesh *B, bool d0, bool d1,
                       const DetectPlan &pl, bool *built, double d, cudaStream_t s) {
    const int cap = (int)ctx->max_pairs;
    launch_detect(ctx, A, B, d0, d1, pl, built, s);
    prof_begin(ctx, HFCR_STAGE_STENCILS, s);
    MeshPair mp{*A, *B};
    // stencil keys (dir, x0, face): x0 and face fields sized to the meshes
    // of the directions this iteration runs, the direction bit sorted only
    // when both run (otherwise it is the same in every key)
    int maxv = 0, maxf = 0;
    if (d0) { maxv = A->n_verts; maxf = B->n_tris; }
    if (d1) {
        if (B->n_verts > maxv) maxv = B->n_verts;
        if (A->n_tris > maxf) maxf = A->n_tris;
    }
    int vb = bits_for(maxv > 1 ? maxv : 2), fb = bits_for(maxf > 1 ? maxf : 2);
    // the pair keys as appended, decoded straight into stencil keys (the
    // clamped pair count to C_PEFF)
    stencil_keys_from_pair_keys(mp, ctx->pkeys, ctx->d_cnt + C_PAIRS, cap, pl.edges[0], pl.edges[1],
                                pl.edge_bits, pl.face_bits, vb, fb, ctx->opt.f32_filter,
                                ctx->skeys, ctx->d_cnt + C_PEFF, ctx->d_stats, ctx->d_status, s);
    const bool flip = radix_sort_u64_dev(ctx->skeys, ctx->skeys_alt, ctx->d_cnt + C_PEFF, cap,
                                         (d0 && d1 ? 1 : 0) + vb + fb, ctx->sort, s);
    stencil_unique(flip ? ctx->skeys_alt : ctx->skeys, ctx->d_cnt + C_PEFF, cap, vb, fb, ctx->sflags,
                   ctx->stencils, ctx->d_cnt + C_STENCILS, ctx->sort, s);
    prof_end(ctx, HFCR_STAGE_STENCILS, s);
    if (!diffusing(ctx)) {
        run_response(ctx, A, B, ctx->stencils, cap, d, 1, nullptr, nullptr, s);
        return;
    }
    // Sec. 5: the minimizer's displacement into the float64 field, spread
    // over each mesh, then applied
    const int ntot = A->n_verts + B->n_verts;
    cudaMemsetAsync(ctx->field, 0, sizeof(double) * 3 * (size_t)ntot, s);
    void *fld[3] = {ctx->field, nullptr, nullptr};
    run_response(ctx, A, B, ctx->stencils, cap, d, 2, fld, nullptr, s);
    prof_begin(ctx, HFCR_STAGE_DIFFUSE, s);
    DiffMeshArgs da, db;
    da.ptr = ctx->adj_ptr[0]; da.nbr = ctx->adj_nbr[0]; da.inv_mass = A->inv_mass; da.n = A->n_verts;
    db.ptr = ctx->adj_ptr[1]; db.nbr = ctx->adj_nbr[1]; db.inv_mass = B->inv_mass; db.n = B->n_verts;
    da.rank = ctx->adj_ranked[0] ? ctx->adj_rank[0] : nullptr;
    db.rank = ctx->adj_ranked[1] ? ctx->adj_rank[1] : nullptr;
    StageMark mark;
    if (ctx->prof_on) {
        mark.fn = band_mark;
        mark.arg = ctx;
    }
    const double *u = diffuse_field(da, db, ctx->field, ctx->field_alt, ctx->ring,
                                    ctx->opt.diffuse_rings, ctx->opt.diffuse_sweeps,
                                    ctx->opt.diffuse_tol, ctx->opt.diffuse_max_iters, ctx->dscr,
                                    ctx->sort, ctx->d_status, s, mark);
    apply_field(*A, *B, ctx->ring, ctx->opt.diffuse_rings, u, s);
    prof_end(ctx, HFCR_STAGE_DIFFUSE, s);
}

// Reads the counters, status, statistics and solver words of the last
// iteration (one copy) and synchronises.
hfcr_status read_iteration(hfcr_ctx *ctx, cudaStream_t s) { return read_back(ctx, s); }

hfcr_status reset_words(hfcr_ctx *ctx, cudaStream_t s);

void clear_graphs(hfcr_ctx *c) {
    for (auto &g : c->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
}

template <typename T>
void key_add(std::string &k, const T &v) {
    k.append(reinterpret_cast<const char *>(&v), sizeof(T));
}

// Resets the per-iteration words and enqueues one repair iteration,
// directly or through a cached CUDA graph of the same arguments.
hfcr_status run_iteration(hfcr_ctx *ctx, const hfcr_mesh *A, const hfcr_mesh *B, bool d0, bool d1,
                          const DetectPlan &pl, bool *built, double d, cudaStream_t s) {
    auto body = [&]() -> hfcr_status {
        hfcr_status st = reset_words(ctx, s);  // the solver words too
        if (st) return st;
        enqueue_iteration(ctx, A, B, d0, d1, pl, built, d, s);
        return HFCR_OK;
    };
    if (!ctx->opt.graphs || ctx->prof_on || !s) return body();
    std::string key;
    key_add(key, *A);
    key_add(key, *B);
    key_add(key, d);
    key_add(key, d0);
    key_add(key, d1);
    key_add(key, built[0]);
    key_add(key, built[1]);
    key_add(key, ctx->opt);
    key_add(key, ctx->max_pairs);
    key_add(key, pl.edges[0]);
    key_add(key, pl.edges[1]);
    key_add(key, pl.ne[0]);
    key_add(key, pl.ne[1]);
    key_add(key, s);
    key_add(key, pl.segs);
    key_add(key, pl.nseg);
    key_add(key, ctx->trav_variant);
    GraphEntry *g = nullptr;
    for (auto &e : ctx->graphs)
        if (e.key == key) g = &e;
    if (!g) {
        if (ctx->graphs.size() >= 8) {  // evict the least recently used
            size_t lru = 0;
            for (size_t i = 1; i < ctx->graphs.size(); ++i)
                if (ctx->graphs[i].last_use < ctx->graphs[lru].last_use) lru = i;
            cudaGraphExecDestroy(ctx->graphs[lru].exec);
            ctx->graphs.erase(ctx->graphs.begin() + lru);
        }
        long long l0 = g_launches.load();
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        hfcr_status st = body();
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(s, &graph);
        if (st) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess)
            return fail(ctx, HFCR_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
        GraphEntry ne;
        ne.key = key;
        e = cudaGraphInstantiate(&ne.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess)
            return fail(ctx, HFCR_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
        ne.launches = g_launches.load() - l0;
        g_launches.fetch_sub(ne.launches);  // counted when replayed
        ctx->graphs.push_back(ne);
        g = &ctx->graphs.back();
    } else {
        // the captured sequence builds exactly the hierarchies the body would
        for (int dd = 0; dd < 2; ++dd)
            if ((dd == 0 ? d0 : d1) && (dd == 0 ? B : A)->n_tris > 0 && pl.ne[dd] > 0)
                built[dd] = true;
    }
    g->last_use = ++ctx->graph_clock;
    CK(cudaGraphLaunch(g->exec, s));
    g_launches.fetch_add(g->launches);
    return HFCR_OK;
}

hfcr_status solve_info(hfcr_ctx *ctx, int k, hfcr_solve_info *info, cudaStream_t s) {
    if (k > 0)
        CK(cudaMemcpyAsync(ctx->h_words, ctx->d_words, sizeof(DevWords), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const DevWords &w = *ctx->h_words;
    info->cg_iters = k > 0 ? w.iwork[1] : 0;
    info->refine_rounds = k > 0 ? w.iwork[3] : 0;
    info->rel_residual = k > 0 ? w.dwork[0] : 0.0;
    info->converged = k == 0 || w.dwork[0] <= ctx->opt.rel_tol;
    info->n_stencils = k;
    info->n_touched = k > 0 ? w.touched : 0;
    info->max_rhs = k > 0 ? w.dwork[8] : 0.0;
    info->max_dx = k > 0 ? w.dwork[9] : 0.0;
    return HFCR_OK;
}

hfcr_status reset_words(hfcr_ctx *ctx, cudaStream_t s) {
    CK(cudaMemsetAsync(ctx->d_words, 0, sizeof(DevWords), s));
    return HFCR_OK;
}

}  // namespace

extern "C" {

hfcr_status hfcr_create(hfcr_ctx **out, const hfcr_options *opt) {
    if (!out) return HFCR_ERR_ARG;
    hfcr_ctx *c = new (std::nothrow) hfcr_ctx();
    if (!c) return HFCR_ERR_ARG;
    c->opt.solver = HFCR_SOLVER_MIXED;
    c->opt.f32_filter = 1;
    c->opt.roles = HFCR_ROLES_ALTERNATE;
    c->opt.max_cg_iters = 500;
    c->opt.max_refine = 6;
    c->opt.rel_tol = 1e-12;
    c->opt.inner_tol = 1e-4;
    c->opt.graphs = 1;
    c->opt.diffuse_rings = 0;
    c->opt.diffuse_sweeps = 0;
    c->opt.traverse_variant = 0;
    c->opt.setup_path = 0;
    c->opt.diffuse_max_iters = 1000;
    c->opt.diffuse_tol = 1e-10;
    c->opt.amplification_limit = 1000.0;
    c->opt.bvh_rebuild_interval = 8;
    c->opt.block_switch_iters = 48;
    if (opt) {
        c->opt = *opt;
        if (c->opt.max_cg_iters <= 0) c->opt.max_cg_iters = 500;
        if (c->opt.max_refine <= 0) c->opt.max_refine = 6;
        if (!(c->opt.rel_tol > 0)) c->opt.rel_tol = 1e-12;
        if (!(c->opt.inner_tol > 0)) c->opt.inner_tol = 1e-4;
        if (c->opt.solver != HFCR_SOLVER_FP64 && c->opt.solver != HFCR_SOLVER_FP64_GLOBAL)
            c->opt.solver = HFCR_SOLVER_MIXED;
        if (c->opt.roles != HFCR_ROLES_BOTH) c->opt.roles = HFCR_ROLES_ALTERNATE;
        if (c->opt.traverse_variant < 0 || c->opt.traverse_variant >= N_TRAVERSE_VARIANTS) {
            delete c;
            set_noctx_error("hfcr_create: traverse_variant out of range");
            return HFCR_ERR_ARG;
        }
        if (c->opt.setup_path != 0 && c->opt.setup_path != 1) {
            delete c;
            set_noctx_error("hfcr_create: setup_path must be 0 or 1");
            return HFCR_ERR_ARG;
        }
        if (c->opt.diffuse_max_iters == 0) c->opt.diffuse_max_iters = 1000;
        if (c->opt.diffuse_tol == 0.0) c->opt.diffuse_tol = 1e-10;
        if (!(c->opt.amplification_limit > 0.0)) c->opt.amplification_limit = 1000.0;
        if (c->opt.block_switch_iters == 0) c->opt.block_switch_iters = 48;
        if (c->opt.block_switch_iters < 0) c->opt.block_switch_iters = -1;
        if (c->opt.bvh_rebuild_interval <= 0) c->opt.bvh_rebuild_interval = 8;
        if (!(c->opt.diffuse_tol > 0.0 && c->opt.diffuse_tol < 1.0) || c->opt.diffuse_max_iters < 0 ||
            c->opt.diffuse_max_iters > 100000) {
            delete c;
            set_noctx_error("hfcr_create: diffuse_tol must be in (0, 1) and diffuse_max_iters in [0, 100000]");
            return HFCR_ERR_ARG;
        }
        if (c->opt.diffuse_rings < 0 || c->opt.diffuse_sweeps < 0 || c->opt.diffuse_rings > 1024 ||
            c->opt.diffuse_sweeps > 100000) {
            delete c;
            set_noctx_error("hfcr_create: diffuse_rings must be in [0, 1024] and diffuse_sweeps in [0, 100000]");
            return HFCR_ERR_ARG;
        }
    }
    c->trav_variant = c->opt.traverse_variant;
    cudaGetDevice(&c->device);
    *out = c;
    return HFCR_OK;
}

hfcr_status hfcr_destroy(hfcr_ctx *ctx) {
    if (!ctx) return HFCR_OK;
    prof_collect(ctx);
    for (auto &iv : ctx->prof_pending) {
        if (iv.a) cudaEventDestroy(iv.a);
        if (iv.b) cudaEventDestroy(iv.b);
    }
    for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
    clear_graphs(ctx);
    if (ctx->own) cudaStreamDestroy(ctx->own);
    if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
    if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
    free_all(ctx);
    delete ctx;
    return HFCR_OK;
}

hfcr_status hfcr_reserve(hfcr_ctx *ctx, int64_t max_verts, int64_t max_tris, int64_t max_pairs) {
    if (!ctx) return HFCR_ERR_ARG;
    if (max_verts < 0 || max_tris < 0 || max_pairs < 0 || max_verts > (1ll << 30) ||
        max_tris > (1ll << 29) || max_pairs > (1ll << 28))
        return fail(ctx, HFCR_ERR_ARG, "reserve sizes out of range");
    if (max_verts <= ctx->max_verts && max_tris <= ctx->max_tris && max_pairs <= ctx->max_pairs)
        return HFCR_OK;
    if (max_verts < ctx->max_verts) max_verts = ctx->max_verts;
    if (max_tris < ctx->max_tris) max_tris = ctx->max_tris;
    if (max_pairs < ctx->max_pairs) max_pairs = ctx->max_pairs;
    CK(cudaDeviceSynchronize());
    clear_graphs(ctx);
    free_all(ctx);
    solver_init();
    diffusion_init();
    if (max_tris < 1) max_tris = 1;
    if (max_pairs < 1) max_pairs = 1;
    const size_t T = (size_t)max_tris, P = (size_t)max_pairs, E3 = 3 * T;
    CK(dalloc(&ctx->d_words, 1));
    CK(cudaMemset(ctx->d_words, 0, sizeof(DevWords)));
    CK(cudaMallocHost((void **)&ctx->h_words, sizeof(DevWords)));
    memset(ctx->h_words, 0, sizeof(DevWords));
    ctx->d_status = &ctx->d_words->status;
    ctx->d_stats = &ctx->d_words->stats;
    ctx->d_cnt = ctx->d_words->cnt;
    ctx->h_status = &ctx->h_words->status;
    ctx->h_stats = &ctx->h_words->stats;
    ctx->h_cnt = ctx->h_words->cnt;
    ctx->h_dw = ctx->h_words->dwork;
    ctx->h_iw = ctx->h_words->iwork;
    CK(cudaMallocHost((void **)&ctx->h_segs, sizeof(int) * 8));
    CK(dalloc(&ctx->d_segs, 8));
    size_t maxn = E3 > 4 * P ? E3 : 4 * P;
    ctx->sort.max_blocks = sort_blocks_for((int)maxn) + 2;
    CK(dalloc(&ctx->sort.hist, 256 * (size_t)ctx->sort.max_blocks));
    ctx->sort.status = ctx->d_status;
    for (int i = 0; i < 2; ++i) {
        Bvh &b = ctx->bvh[i];
        b.cap = (int)T;
        CK(dalloc(&b.nodes, 4 * T));
        CK(dalloc(&b.parent, 2 * T));
        CK(dalloc(&b.flags, T));
        CK(dalloc(&b.leaf_face, T));
        CK(cudaMalloc(&b.leaf_tri, 80 * T));
        CK(dalloc(&b.keys, T));
        CK(dalloc(&b.keys_alt, T));
        CK(dalloc(&b.vals_alt, T));
        CK(dalloc(&b.bounds, 8));
        CK(dalloc(&b.bounds_part, 6 * 1024));
        CK(dalloc(&b.d_rest, 1));
        CK(dalloc(&ctx->edges[i], 2 * E3));
        CK(dalloc(&ctx->eorder[i], E3));
    }
    CK(dalloc(&ctx->ekeys, E3));
    CK(dalloc(&ctx->ekeys_alt, E3));
    CK(dalloc(&ctx->eflags, E3));
    CK(dalloc(&ctx->pkeys, P));
    CK(dalloc(&ctx->pkeys_alt, P));
    CK(dalloc(&ctx->skeys, P));
    CK(dalloc(&ctx->skeys_alt, P));
    CK(dalloc(&ctx->sflags, P));
    CK(dalloc(&ctx->stencils, P));
    {
        const size_t V = (size_t)max_verts;
        for (int i = 0; i < 2; ++i) {
            CK(dalloc(&ctx->adj_ptr[i], V + 1));
            CK(dalloc(&ctx->adj_nbr[i], 2 * E3));
            CK(dalloc(&ctx->adj_rank[i], V));
        }
        CK(dalloc(&ctx->adj_cur, V));
        CK(dalloc(&ctx->field, 6 * V));
        CK(dalloc(&ctx->field_alt, 6 * V));
        CK(dalloc(&ctx->ring, 2 * V));
        DiffScratch &ds = ctx->dscr;
        ds.cap = (int)(2 * V);
        CK(dalloc(&ds.flags, 2 * V));
        CK(dalloc(&ds.cidx, 2 * V));
        CK(dalloc(&ds.fv, 2 * V));
        CK(dalloc(&ds.b64, 6 * V));
        CK(dalloc(&ds.u64, 12 * V));
        CK(dalloc(&ds.x32, 6 * V));
        CK(dalloc(&ds.p32, 6 * V));
        CK(dalloc(&ds.rec, 48 * V));
        CK(dalloc(&ds.cnbr, 4 * E3));   // the capacity of both adjacency arrays
        ds.eoffB = (int)(2 * E3);
        CK(dalloc(&ds.part, 2 * 9 * 1024));
        CK(dalloc(&ds.bar, 1));
        ds.d_nfree = ctx->d_cnt + C_NFREE;
        ds.ctl = ctx->d_cnt + C_DIFF_ITERS;
    }
    SolveBuffers &sb = ctx->sb;
    sb.cap_k = (int)P;
    CK(dalloc(&sb.ids_raw, P));
    CK(dalloc(&sb.n64_raw, P));
    CK(dalloc(&sb.n32_raw, P));
    CK(dalloc(&sb.b_raw, P));
    CK(dalloc(&sb.parent, P));
    CK(dalloc(&sb.zkey, P));
    CK(dalloc(&sb.zkey_alt, P));
    CK(dalloc(&sb.szone, P));
    CK(dalloc(&sb.zs, P + 1));
    CK(dalloc(&sb.zv, 4 * P + 1));
    CK(dalloc(&sb.d_nz, 1));
    CK(dalloc(&sb.gst, P + 1));
    CK(dalloc(&sb.zg, P + 1));
    CK(dalloc(&sb.d_ng, 1));
    CK(dalloc(&sb.pinv, P));
    CK(dalloc(&sb.z32, P));
    CK(dalloc(&sb.ck64, 4 * P));
    CK(dalloc(&sb.ck64_alt, 4 * P));
    CK(dalloc(&sb.ids, P));
    CK(dalloc(&sb.n64, P));
    CK(dalloc(&sb.n32, P));
    CK(dalloc(&sb.b, P));
    CK(dalloc(&sb.lam, P));
    CK(dalloc(&sb.r64, P));
    CK(dalloc(&sb.r32, P));
    CK(dalloc(&sb.x32, P));
    CK(dalloc(&sb.p32, P));
    CK(dalloc(&sb.q32, P));
    CK(dalloc(&sb.w32, P));
    CK(dalloc(&sb.p64, 2 * P));
    CK(dalloc(&sb.cg64, 5 * P));
    CK(dalloc(&sb.pinv64, P));
    CK(dalloc(&sb.binv, 16 * P));
    CK(dalloc(&sb.q64, P));
    CK(dalloc(&sb.vidx, P));
    CK(dalloc(&sb.ckey, 4 * P));
    CK(dalloc(&sb.ckey_alt, 4 * P));
    CK(dalloc(&sb.cval, 4 * P));
    CK(dalloc(&sb.cval_alt, 4 * P));
    CK(dalloc(&sb.cflag, 4 * P));
    CK(dalloc(&sb.seg, 4 * P + 1));
    CK(dalloc(&sb.gvert, 4 * P));
    CK(dalloc(&sb.winv, 4 * P));
    CK(dalloc(&sb.u64, 12 * P));
    CK(dalloc(&sb.u32, 16 * P));
    CK(dalloc(&sb.red, 1024));
    sb.d_U = &ctx->d_words->touched;
    sb.iwork = ctx->d_words->iwork;
    sb.dwork = ctx->d_words->dwork;
    ctx->max_verts = max_verts;
    ctx->max_tris = max_tris;
    ctx->max_pairs = max_pairs;
    return HFCR_OK;
}

hfcr_status hfcr_build_edges(hfcr_ctx *ctx, const int32_t *tris, int32_t n_tris, int32_t n_verts,
                             int32_t *out, int64_t cap, int64_t *n_out, void *stream) {
    if (!ctx) return HFCR_ERR_ARG;
    if (n_tris < 0 || n_verts < 0 || !n_out || (n_tris > 0 && (!tris || !out)))
        return fail(ctx, HFCR_ERR_ARG, "hfcr_build_edges: bad arguments");
    if (n_tris > ctx->max_tris) return fail(ctx, HFCR_ERR_CAPACITY, "n_tris exceeds the reservation");
    cudaStream_t s = (cudaStream_t)stream;
    *n_out = 0;
    if (n_tris == 0) return HFCR_OK;
    hfcr_status st = reset_words(ctx, s);
    if (st) return st;
    build_edges(tris, n_tris, n_verts, ctx->edges[0], ctx->d_cnt + C_EDGES_A, ctx->ekeys,
                ctx->ekeys_alt, ctx->eflags, ctx->sort, ctx->d_status, s);
    if ((st = read_back(ctx, s))) return st;
    int ne = ctx->h_cnt[C_EDGES_A];
    *n_out = ne;
    if (ne > cap) return fail(ctx, HFCR_ERR_CAPACITY, "%d edges exceed cap %lld", ne, (long long)cap);
    CK(cudaMemcpyAsync(out, ctx->edges[0], sizeof(int) * 2 * (size_t)ne, cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    return HFCR_OK;
}

static hfcr_status detect_impl(hfcr_ctx *ctx, const hfcr_mesh *A, const hfcr_mesh *B,
                               const int *segs, int nseg, hfcr_pair *out, int64_t cap,
                               int64_t *n_out, hfcr_detect_stats *stats, void *stream) {
    hfcr_status st = check_pair(ctx, A, B);
    if (st) return st;
    if (!n_out || cap < 0 || (cap > 0 && !out)) return fail(ctx, HFCR_ERR_ARG, "hfcr_detect: bad output");
    cudaStream_t s = (cudaStream_t)stream;
    *n_out = 0;
    if (stats) memset(stats, 0, sizeof *stats);
    if ((st = reset_words(ctx, s))) return st;
    bool dir0 = B->oriented != 0, dir1 = A->oriented != 0;
    DetectPlan pl;
    if ((st = plan_detect(ctx, A, B, dir0, dir1, pl, s, segs, nseg))) return st;
    bool built[2];
    bvh_start(ctx, A, B, pl, built);
    const bool kept[2] = {built[0], built[1]};
    launch_detect(ctx, A, B, dir0, dir1, pl, built, s);
    bvh_finish(ctx, A, B, pl, kept, built);
    if ((st = read_back(ctx, s))) return st;
    int P = ctx->h_cnt[C_PAIRS];
    *n_out = P;
    if (stats) {
        add_stats(stats, *ctx->h_stats);
        stats->brute_force_equiv += single_pair_bf(pl, dir0, dir1, A, B);
    }
    if (P > ctx->max_pairs)
        return fail(ctx, HFCR_ERR_CAPACITY, "%d pairs exceed the reserved %lld", P,
                    (long long)ctx->max_pairs);
    if (P > cap) return fail(ctx, HFCR_ERR_CAPACITY, "%d pairs exceed cap %lld", P, (long long)cap);
    if ((st = finish_pairs(ctx, P, pl, out, s))) return st;
    CK(cudaStreamSynchronize(s));
    return HFCR_OK;
}

hfcr_status hfcr_detect(hfcr_ctx *ctx, const hfcr_mesh *A, const hfcr_mesh *B, hfcr_pair *out,
                        int64_t cap, int64_t *n_out, hfcr_detect_stats *stats, void *stream) {
    return detect_impl(ctx, A, B, nullptr, 1, out, cap, n_out, stats, stream);
}

hfcr_status hfcr_detect_batch(hfcr_ctx *ctx, const hfcr_mesh *A, const hfcr_mesh *B,
                              int32_t n_pairs, const int32_t *segs, hfcr_pair *out, int64_t cap,
                              int64_t *n_out, hfcr_detect_stats *stats, void *stream) {
    if (!ctx) return HFCR_ERR_ARG;
    if (n_pairs < 1 || !segs) return fail(ctx, HFCR_ERR_ARG, "hfcr_detect_batch: need n_pairs >= 1 and a segment table");
    return detect_impl(ctx, A, B, segs, n_pairs, out, cap, n_out, stats, stream);
}

hfcr_status hfcr_build_stencils(hfcr_ctx *ctx, const hfcr_mesh *A, const hfcr_mesh *B,
                                const hfcr_pair *pairs, int64_t n_pairs, hfcr_stencil *out,
                                int64_t cap, int64_t *n_out, void *stream) {
    hfcr_status st = check_pair(ctx, A, B);
    if (st) return st;
    if (!n_out || n_pairs < 0 || (n_pairs > 0 && !pairs) || cap < 0 || (cap > 0 && !out))
        return fail(ctx, HFCR_ERR_ARG, "hfcr_build_stencils: bad arguments");
    if (n_pairs > ctx->max_pairs)
        return fail(ctx, HFCR_ERR_CAPACITY, "%lld pairs exceed the reservation", (long long)n_pairs);
    cudaStream_t s = (cudaStream_t)stream;
    *n_out = 0;
    if (n_pairs == 0) return HFCR_OK;
    if ((st = reset_words(ctx, s))) return st;
    ctx->h_cnt[C_NPAIRS_IN] = (int)n_pairs;
    CK(cudaMemcpyAsync(ctx->d_cnt + C_NPAIRS_IN, ctx->h_cnt + C_NPAIRS_IN, sizeof(int),
                       cudaMemcpyHostToDevice, s));
    validate_pair(*A, *B, ctx->d_status, s);
    int64_t k = 0;
    if ((st = make_stencils(ctx, A, B, pairs, (int)n_pairs, C_NPAIRS_IN, ctx->stencils, &k, s)))
        return st;
    *n_out = k;
    if (k > cap) return fail(ctx, HFCR_ERR_CAPACITY, "%lld stencils exceed cap %lld", (long long)k, (long long)cap);
    if (k > 0)
        CK(cudaMemcpyAsync(out, ctx->stencils, sizeof(hfcr_stencil) * (size_t)k,
                           cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    return HFCR_OK;
}

hfcr_status hfcr_respond(hfcr_ctx *ctx, const hfcr_mesh *A, const hfcr_mesh *B,
                         const hfcr_stencil *st_in, int64_t k, double d, void *const *dxA,
                         void *const *dxB, hfcr_solve_info *info, void *stream) {
    hfcr_status st = check_pair(ctx, A, B);
    if (st) return st;
    if (k < 0 || (k > 0 && !st_in) || !dxA || !dxB || !(d == d))
        return fail(ctx, HFCR_ERR_ARG, "hfcr_respond: bad arguments");
    for (int c = 0; c < 3; ++c)
        if ((A->n_verts > 0 && !dxA[c]) || (B->n_verts > 0 && !dxB[c]))
            return fail(ctx, HFCR_ERR_ARG, "hfcr_respond: NULL displacement array");
    if (k > ctx->max_pairs)
        return fail(ctx, HFCR_ERR_CAPACITY, "%lld stencils exceed the reservation", (long long)k);
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = reset_words(ctx, s))) return st;
    size_t es = A->dtype == HFCR_F32 ? 4 : 8;
    for (int c = 0; c < 3; ++c) {
        if (A->n_verts > 0) CK(cudaMemsetAsync(dxA[c], 0, es * (size_t)A->n_verts, s));
        if (B->n_verts > 0) CK(cudaMemsetAsync(dxB[c], 0, es * (size_t)B->n_verts, s));
    }
    ctx->h_cnt[C_STENCILS] = (int)k;
    CK(cudaMemcpyAsync(ctx->d_cnt + C_STENCILS, ctx->h_cnt + C_STENCILS, sizeof(int),
                       cudaMemcpyHostToDevice, s));
    validate_pair(*A, *B, ctx->d_status, s);
    if ((st = run_response(ctx, A, B, st_in, (int)k, d, 0, dxA, dxB, s))) return st;
    if (info) {
        memset(info, 0, sizeof *info);
        if ((st = solve_info(ctx, (int)k, info, s))) return st;
        CK(cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if ((st = device_status(ctx, *ctx->h_status))) return st;
    }
    return HFCR_OK;
}

hfcr_status hfcr_diffuse(hfcr_ctx *ctx, const hfcr_mesh *M, double *dx, double *dy, double *dz,
                         int32_t rings, int32_t sweeps, void *stream) {
    if (!ctx) return HFCR_ERR_ARG;
    hfcr_status st = check_mesh(ctx, M, "M");
    if (st) return st;
    if (rings < 0 || sweeps < 0 || rings > 1024 || sweeps > 100000)
        return fail(ctx, HFCR_ERR_ARG, "hfcr_diffuse: rings must be in [0, 1024], sweeps in [0, 100000]");
    if (M->n_verts > 0 && (!dx || !dy || !dz))
        return fail(ctx, HFCR_ERR_ARG, "hfcr_diffuse: NULL displacement array");
    if (M->n_verts == 0 || rings == 0) return HFCR_OK;
    if (M->n_verts > ctx->dscr.cap)
        return fail(ctx, HFCR_ERR_CAPACITY, "hfcr_diffuse: mesh exceeds the reserved vertices");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = reset_words(ctx, s))) return st;
    const int *e = M->edges;
    int ne = M->n_edges;
    if (!e && M->n_tris > 0 && (st = mesh_edges(ctx, M, 0, &e, &ne, s))) return st;
    build_adjacency(e, e ? ne : 0, M->n_verts, ctx->adj_ptr[0], ctx->adj_nbr[0], ctx->adj_cur,
                    ctx->sort, ctx->d_status, s);
    ctx->adj_src[0] = nullptr;  // slot 0 no longer holds a resolve call's adjacency
    ctx->adj_ranked[0] = false;
    field_from_soa(dx, dy, dz, M->n_verts, ctx->field, s);
    DiffMeshArgs a, none;
    a.ptr = ctx->adj_ptr[0]; a.nbr = ctx->adj_nbr[0]; a.inv_mass = M->inv_mass; a.n = M->n_verts;
    const double *u = diffuse_field(a, none, ctx->field, ctx->field_alt, ctx->ring, rings, sweeps,
                                    ctx->opt.diffuse_tol, ctx->opt.diffuse_max_iters, ctx->dscr,
                                    ctx->sort, ctx->d_status, s);
    field_to_soa(u, M->n_verts, dx, dy, dz, s);
    CK(cudaGetLastError());
    if ((st = read_back(ctx, s))) return st;
    if (sweeps == 0 && ctx->h_cnt[C_DIFF_FAIL])
        return fail(ctx, HFCR_ERR_NOT_CONVERGED,
                    "hfcr_diffuse: the harmonic solve stopped after %d iterations above tol %g",
                    ctx->h_cnt[C_DIFF_ITERS], ctx->opt.diffuse_tol);
    return HFCR_OK;
}

static hfcr_status resolve_impl(hfcr_ctx *ctx, hfcr_mesh *A, hfcr_mesh *B, const int *segs,
                                int nseg, double d, int32_t max_iters, hfcr_resolve_info *info,
                                void *stream) {
    hfcr_status st = check_pair(ctx, A, B);
    if (st) return st;
    if (max_iters < 0 || !(d == d)) return fail(ctx, HFCR_ERR_ARG, "hfcr_resolve: bad arguments");
    cudaStream_t user = (cudaStream_t)stream, s = user;
    if (!user && ctx->opt.graphs && !ctx->prof_on) {
        // the legacy default stream cannot be captured: work on an own
        // stream ordered after everything the caller queued before
        if (!ctx->own) {
            CK(cudaStreamCreateWithFlags(&ctx->own, cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming));
        }
        CK(cudaEventRecord(ctx->ev_in, user));
        CK(cudaStreamWaitEvent(ctx->own, ctx->ev_in, 0));
        s = ctx->own;
    }
    hfcr_resolve_info loc;
    memset(&loc, 0, sizeof loc);
    const bool has0 = B->oriented != 0, has1 = A->oriented != 0;
    const int n_dirs = (int)has0 + (int)has1;
    const bool alternate = n_dirs == 2 && ctx->opt.roles == HFCR_ROLES_ALTERNATE;
    const int need_quiet = alternate ? 2 : 1;
    if ((st = reset_words(ctx, s))) return st;
    DetectPlan pl;
    if ((st = plan_detect(ctx, A, B, has0, has1, pl, s, segs, nseg))) return st;
    if (diffusing(ctx) && (st = prepare_diffusion(ctx, A, B, pl, s))) return st;
    bool built[2];
    bvh_start(ctx, A, B, pl, built);
    const bool kept[2] = {built[0], built[1]};
    int quiet = 0;
    for (int it = 0; it < max_iters; ++it) {
        bool d0 = has0, d1 = has1;
        if (alternate) { d0 = (it % 2) == 0; d1 = !d0; }
        if ((st = run_iteration(ctx, A, B, d0, d1, pl, built, d, s))) return st;
        CK(cudaGetLastError());
        st = read_iteration(ctx, s);
        int P = ctx->h_cnt[C_PAIRS];
        int64_t k = ctx->h_cnt[C_STENCILS];
        loc.iters = it + 1;
        if (st) {
            if (info) *info = loc;
            return st;
        }
        add_stats(&loc.stats, *ctx->h_stats);
        loc.stats.brute_force_equiv += single_pair_bf(pl, d0, d1, A, B);
        loc.diffuse_cg_iters += ctx->h_cnt[C_DIFF_ITERS];
        if (diffusing(ctx) && ctx->opt.diffuse_sweeps <= 0) loc.band_vertices += ctx->h_cnt[C_NFREE];
        if (P > 0) {
            loc.big_zone_rows += ctx->h_iw[5];
            loc.big_zone_vertices += ctx->h_iw[6];
        }
        if (ctx->h_cnt[C_DIFF_FAIL]) loc.diffuse_unconverged += 1;
        if (it == 0) loc.pairs_first = P;
        loc.pairs_last = P;
        loc.total_pairs += P;
        loc.total_stencils += k;
        if (P == 0) {
            if (++quiet >= need_quiet) { loc.converged = 1; break; }
            continue;
        }
        quiet = 0;
        loc.cg_iters += ctx->h_iw[1];
        loc.solver_path |= ctx->h_iw[4];
        if (ctx->h_dw[8] > 0.0) {
            // the minimizer's own displacement (before any diffusion) against
            // the largest penetration it answers
            const double amp = ctx->h_dw[9] / ctx->h_dw[8];
            if (amp > loc.worst_amplification) loc.worst_amplification = amp;
            if (amp > ctx->opt.amplification_limit) loc.amplified_iters += 1;
        }
        if (ctx->h_dw[0] > loc.worst_rel_residual) loc.worst_rel_residual = ctx->h_dw[0];
    }
    if (info) *info = loc;
    // the hierarchies built by this call, or kept, for the next call
    bvh_finish(ctx, A, B, pl, kept, built);
    CK(cudaStreamSynchronize(s));
    if (s != user) {
        CK(cudaEventRecord(ctx->ev_out, s));
        CK(cudaStreamWaitEvent(user, ctx->ev_out, 0));
    }
    if (!loc.converged) return fail(ctx, HFCR_ERR_NOT_CONVERGED, "repair loop stopped after %d detections", loc.iters);
    return HFCR_OK;
}

hfcr_status hfcr_resolve(hfcr_ctx *ctx, hfcr_mesh *A, hfcr_mesh *B, double d, int32_t max_iters,
                         hfcr_resolve_info *info, void *stream) {
    return resolve_impl(ctx, A, B, nullptr, 1, d, max_iters, info, stream);
}

hfcr_status hfcr_resolve_batch(hfcr_ctx *ctx, hfcr_mesh *A, hfcr_mesh *B, int32_t n_pairs,
                               const int32_t *segs, double d, int32_t max_iters,
                               hfcr_resolve_info *info, void *stream) {
    if (!ctx) return HFCR_ERR_ARG;
    if (n_pairs < 1 || !segs) return fail(ctx, HFCR_ERR_ARG, "hfcr_resolve_batch: need n_pairs >= 1 and a segment table");
    return resolve_impl(ctx, A, B, segs, n_pairs, d, max_iters, info, stream);
}

hfcr_status hfcr_autotune(hfcr_ctx *ctx, const hfcr_mesh *A, const hfcr_mesh *B, int32_t n_pairs,
                          const int32_t *segs, int32_t *chosen, double *ms, int32_t n_ms,
                          void *stream) {
    hfcr_status st = check_pair(ctx, A, B);
    if (st) return st;
    if (segs && n_pairs < 1) return fail(ctx, HFCR_ERR_ARG, "hfcr_autotune: n_pairs must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = reset_words(ctx, s))) return st;
    bool dir0 = B->oriented != 0, dir1 = A->oriented != 0;
    DetectPlan pl;
    if ((st = plan_detect(ctx, A, B, dir0, dir1, pl, s, segs, segs ? n_pairs : 1))) return st;
    bool built[2] = {false, false};
    launch_detect(ctx, A, B, dir0, dir1, pl, built, s);  // builds and refits the hierarchies
    const bool none[2] = {false, false};
    bvh_finish(ctx, A, B, pl, none, built);
    if ((st = read_back(ctx, s))) return st;
    // traversal launches per timed call (one per active direction with
    // work): the times below are per launch, as a repair iteration of one
    // direction runs it
    int nl = 0;
    if (dir0 && B->n_tris > 0 && pl.ne[0] > 0) ++nl;
    if (dir1 && A->n_tris > 0 && pl.ne[1] > 0) ++nl;
    if (nl == 0) nl = 1;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int best = 0;
    double best_ms = 1e300;
    for (int v = 0; v < N_TRAVERSE_VARIANTS; ++v) {
        double vbest = 1e300;
        for (int rep = 0; rep < 3; ++rep) {
            CK(cudaMemsetAsync(ctx->d_cnt + C_PAIRS, 0, sizeof(int), s));
            CK(cudaEventRecord(e0, s));
            launch_detect(ctx, A, B, dir0, dir1, pl, built, s, true, v);
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, e0, e1));
            if (t / nl < vbest) vbest = t / nl;
        }
        if (ms && v < n_ms) ms[v] = vbest;
        if (vbest < best_ms) {
            best_ms = vbest;
            best = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if ((st = read_back(ctx, s))) return st;
    ctx->trav_variant = best;
    if (chosen) *chosen = best;
    return HFCR_OK;
}

hfcr_status hfcr_profile_enable(hfcr_ctx *ctx, int32_t on) {
    if (!ctx) return HFCR_ERR_ARG;
    prof_collect(ctx);
    for (int i = 0; i < HFCR_N_STAGES; ++i) {
        ctx->prof_ms[i] = 0;
        ctx->prof_n[i] = 0;
    }
    ctx->prof_on = on != 0;
    return HFCR_OK;
}

hfcr_status hfcr_profile_read(hfcr_ctx *ctx, hfcr_profile *out) {
    if (!ctx || !out) return HFCR_ERR_ARG;
    prof_collect(ctx);
    for (int i = 0; i < HFCR_N_STAGES; ++i) {
        out->ms[i] = ctx->prof_ms[i];
        out->intervals[i] = ctx->prof_n[i];
    }
    return HFCR_OK;
}

int64_t hfcr_launch_count(void) { return (int64_t)g_launches.load(); }

const char *hfcr_last_error(const hfcr_ctx *ctx) {
    return ctx ? ctx->err.c_str() : hfcr::g_noctx_err.c_str();
}

const char *hfcr_status_string(hfcr_status s) {
    switch (s) {
        case HFCR_OK: return "HFCR_OK";
        case HFCR_ERR_ARG: return "HFCR_ERR_ARG";
        case HFCR_ERR_CAPACITY: return "HFCR_ERR_CAPACITY";
        case HFCR_ERR_CUDA: return "HFCR_ERR_CUDA";
        case HFCR_ERR_NONFINITE: return "HFCR_ERR_NONFINITE";
        case HFCR_ERR_TIMEOUT: return "HFCR_ERR_TIMEOUT";
        case HFCR_ERR_NOT_CONVERGED: return "HFCR_ERR_NOT_CONVERGED";
        case HFCR_ERR_UNSUPPORTED: return "HFCR_ERR_UNSUPPORTED";
        case HFCR_ERR_RANGE: return "HFCR_ERR_RANGE";
    }
    return "HFCR_UNKNOWN";
}

}  // extern "C"
