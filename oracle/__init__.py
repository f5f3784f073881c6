"""CPU oracle for the history-free collision response path.

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg import this package; the product path (the CUDA library
and its Python binding) never does, and the two share no code.  Inputs come
from the seeded generators in `meshgen`, which hold none of the method's
arithmetic.

It computes, plainly and slowly, what the paper's method computes:

* edges of a triangle mesh (sorted unique undirected vertex pairs);
* exact DCD: every (edge, face) pair where the edge properly crosses a face
  of an oriented mesh (Sec. 3; brute force in `dcd_oracle.c` with exact
  big-integer orientation signs);
* penetration stencils {x0; x1, x2, x3}: x0 the endpoint of the crossing
  edge on the back side of the oriented face, duplicates merged (Sec. 4,
  Fig. 3);
* the constraint D(x) = n . [x0 - (x1 + x2 + x3)/3] (Eq. 1) and its
  gradient (Eq. 2), stacked into a k x 3n matrix (Sec. 4);
* the global displacement minimizer (Eq. 3): lambda from the normal
  equations (Eq. 7, or Eq. 8 with post-response distance d), solved per
  impact zone, then x' = x - M^-1 grad(D)^T lambda (the first stationary
  equation, Eq. 5);
* the repair loop: detect, build stencils, displace, until no edge-face
  intersection remains (Sec. 3).

Readings of the paper used here (the paper is silent or ambiguous):
  - "intersection" is a strict plane crossing of a closed triangle; touching
    and coplanar contacts, zero-area faces and zero-length edges give no pair;
  - n is the unit normal (b - a) x (c - a) / |.| of the pre-response face;
  - detection of a pair of meshes reports every active direction (edges of
    A vs faces of B when B is oriented, edges of B vs faces of A when A is);
    in the repair loop, when both are oriented, the two roles alternate
    from one iteration to the next (Sec. 4: one is regarded as oriented and
    the other as un-oriented in turn), or optionally both run every time;
  - x' = x - M^-1 grad(D)^T lambda with grad(D) M^-1 grad(D)^T lambda =
    grad(D) x - d (the sign of lambda is immaterial to x');
  - unit masses unless inverse masses are given;
  - stencils are deduplicated by (direction, x0, face).

Parity status: every function here is pinned by tests that do not use it
(exact rational arithmetic, closed forms, library solvers, invariants of
closed meshes); see tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile dcd_oracle.c into liboracle.so beside it (gcc, OpenMP)."""
    src = os.path.join(_HERE, "dcd_oracle.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _LIB_PATH, src, "-lm"])
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        lib.oracle_orient.argtypes = [dp, dp, dp, dp]
        lib.oracle_orient.restype = ctypes.c_int
        lib.oracle_segtri.argtypes = [dp, dp, dp, dp, dp, ctypes.POINTER(ctypes.c_int)]
        lib.oracle_segtri.restype = ctypes.c_int
        lib.oracle_detect.argtypes = [dp, ip, ctypes.c_int64, dp, ip, ctypes.c_int64, ip,
                                      ctypes.c_int64, ctypes.c_int]
        lib.oracle_detect.restype = ctypes.c_int64
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


# ----------------------------------------------------------------------------
# exact predicates (Sec. 4: front side = side the face normal points to)
# ----------------------------------------------------------------------------

def orient(a, b, c, x) -> int:
    """Exact sign of det[b-a, c-a, x-a]; +1 when x is on the front side of
    the counter-clockwise triangle abc."""
    arr = [np.ascontiguousarray(np.asarray(v, dtype=np.float64)) for v in (a, b, c, x)]
    return int(_load().oracle_orient(*[_dptr(v) for v in arr]))


def segtri(p, q, a, b, c) -> Tuple[bool, int]:
    """Exact test of segment pq against triangle abc; returns (hit, side of
    p) with side = orient(a, b, c, p) when hit."""
    arr = [np.ascontiguousarray(np.asarray(v, dtype=np.float64)) for v in (p, q, a, b, c)]
    side = ctypes.c_int(0)
    hit = _load().oracle_segtri(*[_dptr(v) for v in arr], ctypes.byref(side))
    return bool(hit), int(side.value)


# ----------------------------------------------------------------------------
# topology
# ----------------------------------------------------------------------------

def edges(T: np.ndarray) -> np.ndarray:
    """Unique undirected edges (v0 < v1) of a triangle list, sorted
    lexicographically; int32 [E, 2].  Every face-face contact is a pair of
    edge-face contacts (Sec. 4), so edges are the primitives the detection
    runs over."""
    T = np.asarray(T, dtype=np.int64)
    if T.size == 0:
        return np.zeros((0, 2), np.int32)
    e = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]], 0)
    e = np.stack([e.min(1), e.max(1)], 1)
    e = np.unique(e, axis=0)           # lexicographic (v0, v1)
    return e.astype(np.int32)


# ----------------------------------------------------------------------------
# detection (Sec. 3: all E-F intersections, face from the oriented mesh)
# ----------------------------------------------------------------------------

def detect_one_direction(PE: np.ndarray, E: np.ndarray, PF: np.ndarray, TF: np.ndarray,
                         n_threads: int = 0) -> np.ndarray:
    """All (edge index, face, side of the edge's first vertex) with edge E[i]
    of the edge mesh crossing face TF[f] of the face mesh; int32 [P, 3],
    sorted by (edge index, face)."""
    PE = np.ascontiguousarray(PE, dtype=np.float64)
    PF = np.ascontiguousarray(PF, dtype=np.float64)
    if not (np.all(np.isfinite(PE)) and np.all(np.isfinite(PF))):
        raise ValueError("non-finite position")
    E = np.ascontiguousarray(E, dtype=np.int32)
    TF = np.ascontiguousarray(TF, dtype=np.int32)
    cap = max(1024, 4 * len(E) // 100)
    lib = _load()
    while True:
        out = np.zeros((cap, 3), np.int32)
        n = lib.oracle_detect(_dptr(PE), _iptr(E), len(E), _dptr(PF), _iptr(TF), len(TF),
                              _iptr(out), cap, int(n_threads))
        if n <= cap:
            out = out[:n]
            break
        cap = int(n)
    order = np.lexsort((out[:, 1], out[:, 0]))
    return out[order]


def directions(orientedA: bool, orientedB: bool) -> List[int]:
    """Active directions: 0 = edges of A against faces of B (needs B
    oriented), 1 = edges of B against faces of A (needs A oriented)."""
    d = []
    if orientedB:
        d.append(0)
    if orientedA:
        d.append(1)
    return d


@dataclass
class Pairs:
    """Sorted edge-face pairs: rows (dir, v0, v1, face) with v0 < v1 local
    ids of the edge mesh, and side = orient(face, v0) in {-1, +1}."""
    rec: np.ndarray   # uint32 [P, 4]
    side: np.ndarray  # int8 [P]

    def __len__(self):
        return int(self.rec.shape[0])


def detect(PA, TA, orientedA, PB, TB, orientedB, EA=None, EB=None, n_threads: int = 0) -> Pairs:
    """Exact DCD between meshes A and B (positions as float64 [n, 3])."""
    if not (orientedA or orientedB):
        raise ValueError("at least one mesh must be oriented")
    EA = edges(TA) if EA is None else EA
    EB = edges(TB) if EB is None else EB
    recs, sides = [], []
    for d in directions(orientedA, orientedB):
        PE, E, PF, TF = (PA, EA, PB, TB) if d == 0 else (PB, EB, PA, TA)
        hits = detect_one_direction(PE, E, PF, TF, n_threads)
        r = np.zeros((len(hits), 4), np.uint32)
        r[:, 0] = d
        r[:, 1] = E[hits[:, 0], 0]
        r[:, 2] = E[hits[:, 0], 1]
        r[:, 3] = hits[:, 1]
        recs.append(r)
        sides.append(hits[:, 2].astype(np.int8))
    rec = np.concatenate(recs, 0) if recs else np.zeros((0, 4), np.uint32)
    side = np.concatenate(sides, 0) if sides else np.zeros((0,), np.int8)
    order = np.lexsort((rec[:, 3], rec[:, 2], rec[:, 1], rec[:, 0]))
    return Pairs(rec[order], side[order])


# ----------------------------------------------------------------------------
# stencils (Sec. 4, Fig. 3)
# ----------------------------------------------------------------------------

def stencils(pairs: Pairs) -> np.ndarray:
    """Penetration stencils (dir, x0, face), sorted unique.  x0 is the
    endpoint of the crossing edge on the back side of the oriented face
    (the illegal vertex, Sec. 3); two pairs with the same illegal vertex and
    face give one stencil (Fig. 3a)."""
    if len(pairs) == 0:
        return np.zeros((0, 3), np.uint32)
    x0 = np.where(pairs.side < 0, pairs.rec[:, 1], pairs.rec[:, 2])
    st = np.stack([pairs.rec[:, 0], x0, pairs.rec[:, 3]], 1).astype(np.uint32)
    return np.unique(st, axis=0)


# ----------------------------------------------------------------------------
# constraints and the minimizer (Sec. 4, Eqs. 1-8)
# ----------------------------------------------------------------------------

@dataclass
class Assembly:
    """k stacked constraints: ids [k, 4] global vertex ids (x0, x1, x2, x3)
    with A's vertices first, then B's; n [k, 3] unit face normals; D [k]
    signed distances (Eq. 1) and rhs b = D - d (Eq. 8)."""
    ids: np.ndarray
    n: np.ndarray
    D: np.ndarray
    b: np.ndarray
    n_verts: int


def assemble(st: np.ndarray, PA, TA, PB, TB, d: float) -> Assembly:
    """Eq. 1 with alpha = 1/3 and unit n, on the pre-response positions."""
    PA = np.asarray(PA, np.float64)
    PB = np.asarray(PB, np.float64)
    nA = PA.shape[0]
    P = np.concatenate([PA, PB], 0)
    k = st.shape[0]
    ids = np.zeros((k, 4), np.int64)
    for i in range(k):
        dr, x0, f = int(st[i, 0]), int(st[i, 1]), int(st[i, 2])
        if dr == 0:   # edge of A (x0 in A), face of B
            ids[i] = [x0, nA + TB[f, 0], nA + TB[f, 1], nA + TB[f, 2]]
        else:         # edge of B (x0 in B), face of A
            ids[i] = [nA + x0, TA[f, 0], TA[f, 1], TA[f, 2]]
    x0, x1, x2, x3 = (P[ids[:, j]] for j in range(4))
    nrm = np.cross(x2 - x1, x3 - x1)
    nrm = nrm / np.linalg.norm(nrm, axis=1, keepdims=True) if k else nrm
    D = np.einsum("ij,ij->i", nrm, x0 - (x1 + x2 + x3) / 3.0)
    return Assembly(ids, nrm, D, D - d, P.shape[0])


def gradient_matrix(asm: Assembly):
    """grad(D) as a sparse k x 3n matrix (Eq. 2 rows: n^T at x0, -n^T/3 at
    x1, x2, x3, assembled like a finite-element stiffness matrix)."""
    import scipy.sparse as sp
    k = asm.ids.shape[0]
    rows, cols, vals = [], [], []
    coef = [1.0, -1.0 / 3.0, -1.0 / 3.0, -1.0 / 3.0]
    for j in range(4):
        for c in range(3):
            rows.append(np.arange(k))
            cols.append(3 * asm.ids[:, j] + c)
            vals.append(coef[j] * asm.n[:, c])
    if k == 0:
        return sp.csr_matrix((0, 3 * asm.n_verts))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(k, 3 * asm.n_verts))


def impact_zones(ids: np.ndarray) -> np.ndarray:
    """Impact zones (Sec. 4): constraints connected through shared stencil
    vertices, found with union-find; returns a zone label per constraint
    (labels are the smallest constraint index of the zone)."""
    k = ids.shape[0]
    parent = list(range(k))

    def find(i):
        while parent[i] != i:
            parent[i] = parent[parent[i]]
            i = parent[i]
        return i

    owner = {}
    for i in range(k):
        for v in ids[i]:
            v = int(v)
            if v in owner:
                ri, rj = find(i), find(owner[v])
                if ri != rj:
                    parent[max(ri, rj)] = min(ri, rj)
            else:
                owner[v] = i
    return np.array([find(i) for i in range(k)], np.int64)


def _cg(apply_A, b, tol, max_iter):
    """Textbook conjugate gradients on an SPD operator (float64)."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    bn = float(np.sqrt(b @ b))
    it = 0
    while np.sqrt(rr) > tol * bn and it < max_iter:
        Ap = apply_A(p)
        alpha = rr / float(p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it


@dataclass
class Solution:
    dx: np.ndarray          # [n_verts, 3] displacement x' - x
    lam: np.ndarray         # [k] multipliers (not unique when rows repeat)
    zones: np.ndarray       # [k] impact-zone labels
    n_zones: int
    cg_iters: int = 0
    info: dict = field(default_factory=dict)


def solve(asm: Assembly, inv_mass: Optional[np.ndarray] = None, dense_max: int = 2048,
          cg_tol: float = 1e-14) -> Solution:
    """Eq. 3 through Eq. 7/8, one linear system per impact zone:
    (grad(D) M^-1 grad(D)^T) lambda = grad(D) x - d, then
    x' - x = -M^-1 grad(D)^T lambda.  Zones up to `dense_max` constraints
    use a dense Cholesky factorisation; larger ones conjugate gradients to
    a relative residual of `cg_tol`.  A Cholesky pivot below 1e-12 times the
    largest diagonal entry (dependent rows) falls back to the minimum-norm
    least-squares solution of that zone."""
    k = asm.ids.shape[0]
    nv = asm.n_verts
    w = np.ones(nv) if inv_mass is None else np.asarray(inv_mass, np.float64)
    if k == 0:
        return Solution(np.zeros((nv, 3)), np.zeros(0), np.zeros(0, np.int64), 0)
    J = gradient_matrix(asm)
    Minv3 = np.repeat(w, 3)
    A = (J.multiply(Minv3[None, :]) @ J.T).tocsr()
    zones = impact_zones(asm.ids)
    lam = np.zeros(k)
    labels, inverse = np.unique(zones, return_inverse=True)
    members = [[] for _ in labels]
    for i, z in enumerate(inverse):
        members[z].append(i)
    cg_total = 0
    for mem in members:
        mem = np.asarray(mem)
        Az = A[mem][:, mem]
        bz = asm.b[mem]
        if len(mem) <= dense_max:
            Ad = Az.toarray()
            dmax = np.max(np.diag(Ad))
            try:
                L = np.linalg.cholesky(Ad)
                ok = np.min(np.diag(L)) ** 2 > 1e-12 * dmax
            except np.linalg.LinAlgError:
                ok = False
            if ok:
                y = np.linalg.solve(L, bz)
                lam[mem] = np.linalg.solve(L.T, y)
            else:
                lam[mem] = np.linalg.lstsq(Ad, bz, rcond=None)[0]
        else:
            x, it = _cg(lambda v: Az @ v, bz, cg_tol, 20 * len(mem))
            lam[mem] = x
            cg_total += it
    dx = -(Minv3 * (J.T @ lam)).reshape(nv, 3)
    return Solution(dx, lam, zones, len(labels), cg_total)


def respond(st: np.ndarray, PA, TA, PB, TB, d: float, inv_mass=None):
    """Displacements (dxA, dxB) for a stencil set on given positions."""
    asm = assemble(st, PA, TA, PB, TB, d)
    sol = solve(asm, inv_mass)
    nA = np.asarray(PA).shape[0]
    return sol.dx[:nA], sol.dx[nA:], asm, sol


# ----------------------------------------------------------------------------
# diffusion of displacement vectors (Sec. 5)
# ----------------------------------------------------------------------------

def vertex_adjacency(E: np.ndarray, n_verts: int):
    """Neighbours of every vertex over the mesh edges, as CSR (indptr,
    indices), indices ascending within a vertex."""
    E = np.asarray(E, np.int64)
    src = np.concatenate([E[:, 0], E[:, 1]])
    dst = np.concatenate([E[:, 1], E[:, 0]])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    indptr = np.zeros(n_verts + 1, np.int64)
    np.add.at(indptr, src + 1, 1)
    return np.cumsum(indptr), dst


def ring_distance(moved: np.ndarray, indptr, nbr, rings: int) -> np.ndarray:
    """Edge-count distance of every vertex to the nearest moved vertex,
    found breadth-first over `rings` levels; vertices farther away get
    rings + 1."""
    n = len(moved)
    dist = np.full(n, rings + 1, np.int64)
    dist[moved] = 0
    frontier = np.nonzero(moved)[0]
    for r in range(1, rings + 1):
        nxt = []
        for v in frontier:
            for w in nbr[indptr[v]:indptr[v + 1]]:
                if dist[w] > r:
                    dist[w] = r
                    nxt.append(w)
        frontier = np.array(sorted(set(nxt)), np.int64)
    return dist


def diffuse(dx: np.ndarray, E: np.ndarray, rings: int, sweeps: int = 0,
            fixed: Optional[np.ndarray] = None) -> np.ndarray:
    """Spreads the displacement of the vertices the minimizer moved over
    their vicinity as a harmonic vector field (Sec. 5 names constrained
    diffusion to a harmonic field and gives no equations; this is the
    reading used here).  On the mesh graph (vertices, edges E):

      * the moved vertices (nonzero dx) keep their displacement: Dirichlet
        values;
      * the band = the vertices 1 .. `rings` edges from the nearest moved
        vertex, except `fixed` (kinematic) ones: the unknowns;
      * every other vertex is held at zero: Dirichlet values too.

    sweeps == 0: the harmonic field itself, i.e. each band vertex equals
    the mean of its neighbours: deg(v) u_v - sum of u_w over the band
    neighbours w = sum of the Dirichlet values of its other neighbours,
    one sparse linear system per coordinate (the graph Laplacian of the
    band), solved directly.  Every band vertex is joined to a Dirichlet
    vertex by a path of band vertices (its ring number falls along a
    shortest path to the moved set), so the system is positive definite.

    sweeps > 0: the named approximation instead: `sweeps` Jacobi sweeps of
    the neighbour mean over the band, starting from zero (the harmonic
    field is their limit).  dx: [n, 3]."""
    n = dx.shape[0]
    C = np.any(dx != 0.0, axis=1)
    if rings <= 0 or not C.any():
        return dx.copy()
    indptr, nbr = vertex_adjacency(E, n)
    deg = np.diff(indptr)
    dist = ring_distance(C, indptr, nbr, rings)
    free = (dist >= 1) & (dist <= rings)
    if fixed is not None:
        free &= ~np.asarray(fixed, bool)
    u = np.where(C[:, None], dx, 0.0)
    fv = np.nonzero(free)[0]
    if sweeps > 0:
        for _ in range(sweeps):
            new = u.copy()
            for v in fv:
                acc = np.zeros(3)
                for w in nbr[indptr[v]:indptr[v + 1]]:
                    acc += u[w]
                new[v] = acc / deg[v]
            u = new
        return u
    if len(fv) == 0:
        return u
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla
    col = np.full(n, -1, np.int64)
    col[fv] = np.arange(len(fv))
    rows, cols, vals = [], [], []
    rhs = np.zeros((len(fv), 3))
    for i, v in enumerate(fv):
        rows.append(i)
        cols.append(i)
        vals.append(float(deg[v]))
        for w in nbr[indptr[v]:indptr[v + 1]]:
            if free[w]:
                rows.append(i)
                cols.append(col[w])
                vals.append(-1.0)
            else:
                rhs[i] += u[w]       # Dirichlet neighbour (moved: dx, else 0)
    L = sp.csc_matrix((vals, (rows, cols)), shape=(len(fv), len(fv)))
    for c in range(3):
        u[fv, c] = sla.spsolve(L, rhs[:, c])
    return u


@dataclass
class ResolveResult:
    PA: np.ndarray
    PB: np.ndarray
    iters: int                 # detections run
    pair_counts: List[int]     # pairs found by each detection
    stencil_counts: List[int]  # stencils of each response
    dirs: List[List[int]]      # directions tested by each detection
    converged: bool


def role_schedule(orientedA: bool, orientedB: bool, it: int, mode: str) -> List[int]:
    """Directions tested in iteration `it`.  When both meshes are oriented,
    Sec. 4 regards one as oriented and the other as un-oriented in turn:
    mode 'alternate' tests edges of A against faces of B in even iterations
    and edges of B against faces of A in odd ones; mode 'both' tests both
    directions in every iteration."""
    act = directions(orientedA, orientedB)
    if len(act) == 2 and mode == "alternate":
        return [it % 2]
    return act


def resolve(PA, TA, orientedA, PB, TB, orientedB, d: float = 1e-4, max_iters: int = 64,
            store_dtype=np.float64, inv_mass=None, n_threads: int = 0,
            mode: str = "alternate", diffuse_rings: int = 0,
            diffuse_sweeps: int = 0) -> ResolveResult:
    """The repair loop of Sec. 3: detect, build stencils, displace by the
    minimizer, repeated until no edge-face intersection remains.  It stops
    when the most recent detections covering every active direction found
    no pair, or after `max_iters` detections.  Positions are rounded to
    `store_dtype` after each displacement (the storage type of the scene).
    With diffuse_rings > 0, each mesh's displacement is spread by `diffuse`
    (Sec. 5) before it is applied: the harmonic field when diffuse_sweeps is
    0, else that many Jacobi sweeps; vertices of inverse mass 0 are held
    fixed."""
    if mode not in ("alternate", "both"):
        raise ValueError(mode)
    PA = np.asarray(PA, np.float64).astype(store_dtype).astype(np.float64)
    PB = np.asarray(PB, np.float64).astype(store_dtype).astype(np.float64)
    EA, EB = edges(TA), edges(TB)
    n_dirs = len(directions(orientedA, orientedB))
    need_quiet = n_dirs if mode == "alternate" else 1
    pc, sc, dl = [], [], []
    quiet = 0
    for it in range(max_iters):
        dirs = role_schedule(orientedA, orientedB, it, mode)
        oa, ob = (1 in dirs), (0 in dirs)
        pr = detect(PA, TA, oa, PB, TB, ob, EA, EB, n_threads)
        pc.append(len(pr))
        dl.append(dirs)
        if len(pr) == 0:
            quiet += 1
            if quiet >= need_quiet:
                return ResolveResult(PA, PB, it + 1, pc, sc, dl, True)
            continue
        quiet = 0
        st = stencils(pr)
        sc.append(len(st))
        dA, dB, _, _ = respond(st, PA, TA, PB, TB, d, inv_mass)
        if diffuse_rings > 0:
            nA = PA.shape[0]
            fx = None if inv_mass is None else np.asarray(inv_mass) == 0.0
            dA = diffuse(dA, EA, diffuse_rings, diffuse_sweeps, None if fx is None else fx[:nA])
            dB = diffuse(dB, EB, diffuse_rings, diffuse_sweeps, None if fx is None else fx[nA:])
        PA = (PA + dA).astype(store_dtype).astype(np.float64)
        PB = (PB + dB).astype(store_dtype).astype(np.float64)
    return ResolveResult(PA, PB, max_iters, pc, sc, dl, False)
