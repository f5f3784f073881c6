"""Pins for the oracle's brute-force edge-face detection on whole meshes.

* Closed-mesh parity: for an edge pq and a closed surface B in general
  position, the number of B's faces the edge crosses is odd exactly when
  one endpoint is inside B and the other outside.  "Inside" comes from the
  generalized winding number (sum of solid angles, Van Oosterom-Strackee),
  computed in float64 here, independently of the oracle.  A missed or a
  spurious pair on any edge flips that parity.
* Independent float64 decisions: on every box-overlapping candidate whose
  five determinants are far from zero, a plain float64 evaluation must
  agree with the oracle.
* Exact soundness: every reported pair re-verified with rational
  arithmetic.
"""
import numpy as np
import pytest

import meshgen
import oracle
from test_oracle_predicates import frac_segtri


def winding_number(P, V, T):
    """Generalized winding number of closed mesh (V, T) at points P."""
    w = np.zeros(len(P))
    chunk = max(1, min(256, (1 << 22) // max(1, len(T))))   # bounded temporaries
    for i in range(0, len(P), chunk):
        Q = P[i:i + chunk, None, :]
        a, b, c = V[T[:, 0]][None] - Q, V[T[:, 1]][None] - Q, V[T[:, 2]][None] - Q
        la, lb, lc = (np.linalg.norm(x, axis=2) for x in (a, b, c))
        num = np.einsum("pfk,pfk->pf", a, np.cross(b, c))
        den = (la * lb * lc + np.einsum("pfk,pfk->pf", a, b) * lc
               + np.einsum("pfk,pfk->pf", a, c) * lb + np.einsum("pfk,pfk->pf", b, c) * la)
        w[i:i + chunk] = 2.0 * np.arctan2(num, den).sum(1) / (4.0 * np.pi)
    return w


def _scenes():
    out = [("c1", meshgen.scene_c1())]
    for seed, kind in [(11, "spheres"), (12, "torus_sphere"), (13, "spheres")]:
        out.append((f"{kind}{seed}", meshgen.scene_random_small(seed, kind)))
    return out


@pytest.mark.parametrize("name,scene", _scenes(), ids=lambda x: x if isinstance(x, str) else "")
def test_closed_mesh_crossing_parity(name, scene):
    PA, PB = scene.positions("A"), scene.positions("B")
    pr = oracle.detect(PA, scene.A.T, True, PB, scene.B.T, True)
    assert len(pr) > 0
    for d, (PE, TE, PF, TF) in enumerate([(PA, scene.A.T, PB, scene.B.T),
                                          (PB, scene.B.T, PA, scene.A.T)]):
        E = oracle.edges(TE)
        w = winding_number(PE, PF, TF)
        assert np.all(np.abs(w - np.round(w)) < 1e-3)   # general position
        inside = np.round(w).astype(int) != 0
        sel = pr.rec[pr.rec[:, 0] == d]
        key = sel[:, 1].astype(np.int64) * (len(PE) + 1) + sel[:, 2]
        ekey = E[:, 0].astype(np.int64) * (len(PE) + 1) + E[:, 1]
        cnt = np.zeros(len(E), np.int64)
        idx = np.searchsorted(ekey, key)
        np.add.at(cnt, idx, 1)
        assert np.array_equal(cnt % 2, (inside[E[:, 0]] ^ inside[E[:, 1]]).astype(np.int64))


def _f64_orient(a, b, c, x):
    u, v, w = b - a, c - a, x - a
    det = np.einsum("ij,ij->i", u, np.cross(v, w))
    scale = (np.linalg.norm(u, axis=1) * np.linalg.norm(v, axis=1) * np.linalg.norm(w, axis=1))
    return det, scale


def test_float64_agrees_where_well_conditioned():
    sc = meshgen.scene_c1()
    PA, PB = sc.positions("A"), sc.positions("B")
    for d, (PE, TE, PF, TF) in enumerate([(PA, sc.A.T, PB, sc.B.T), (PB, sc.B.T, PA, sc.A.T)]):
        E = oracle.edges(TE)
        p, q = PE[E[:, 0]], PE[E[:, 1]]
        a, b, c = PF[TF[:, 0]], PF[TF[:, 1]], PF[TF[:, 2]]
        elo, ehi = np.minimum(p, q), np.maximum(p, q)
        flo, fhi = np.minimum(np.minimum(a, b), c), np.maximum(np.maximum(a, b), c)
        ov = np.all((elo[:, None] <= fhi[None]) & (flo[None] <= ehi[:, None]), axis=2)
        ei, fi = np.nonzero(ov)
        P, Q, A_, B_, C_ = p[ei], q[ei], a[fi], b[fi], c[fi]
        dets = [_f64_orient(A_, B_, C_, P), _f64_orient(A_, B_, C_, Q), _f64_orient(P, Q, A_, B_),
                _f64_orient(P, Q, B_, C_), _f64_orient(P, Q, C_, A_)]
        good = np.all([np.abs(dt) > 1e-9 * sc_ for dt, sc_ in dets], axis=0)
        s = [np.sign(dt) for dt, _ in dets]
        hit = (s[0] * s[1] < 0) & (((s[2] >= 0) & (s[3] >= 0) & (s[4] >= 0)) | ((s[2] <= 0) & (s[3] <= 0) & (s[4] <= 0)))
        pr = oracle.detect(PA, sc.A.T, d == 1, PB, sc.B.T, d == 0)
        got = set(map(tuple, pr.rec[:, [1, 2, 3]].tolist()))
        n_checked = 0
        for k in np.nonzero(good)[0]:
            key = (int(E[ei[k], 0]), int(E[ei[k], 1]), int(fi[k]))
            assert (key in got) == bool(hit[k])
            n_checked += 1
        assert n_checked > 200 and good.mean() > 0.99


def test_exact_soundness_and_subset():
    sc = meshgen.scene_c1()
    PA, PB = sc.positions("A"), sc.positions("B")
    pr = oracle.detect(PA, sc.A.T, True, PB, sc.B.T, True)
    for (d, v0, v1, f), s in zip(pr.rec.tolist(), pr.side.tolist()):
        PE, PF, TF = (PA, PB, sc.B.T) if d == 0 else (PB, PA, sc.A.T)
        ok, side = frac_segtri(PE[v0], PE[v1], *PF[TF[f]])
        assert ok and side == s
    # detection restricted to a subset of edges = full result on that subset
    E = oracle.edges(sc.A.T)
    sub = np.arange(3, len(E), 7)
    hits = oracle.detect_one_direction(PA, E[sub], PB, sc.B.T)
    full = oracle.detect_one_direction(PA, E, PB, sc.B.T)
    keep = np.isin(full[:, 0], sub)
    mapped = np.c_[sub[hits[:, 0]], hits[:, 1:]]
    assert np.array_equal(mapped, full[keep])
    # single-threaded run gives the identical set
    assert np.array_equal(oracle.detect_one_direction(PA, E, PB, sc.B.T, n_threads=1), full)


# ---------------------------------------------------------------------------
# Triangle-pair accounting (Sec. 4: a face-face contact is two edge-face
# contacts).  In general position two triangles of closed meshes A and B
# intersect in a segment whose two ends are edge-face crossings, and every
# crossing of an edge of A (B) through a face of B (A) is an end of the
# segments of both triangles that share the edge; so the number of
# intersecting triangle pairs equals #crossings(edges of A, faces of B) +
# #crossings(edges of B, faces of A).  The triangle-triangle test below is
# the interval test on the line where the two planes meet, in float64,
# written here independently of the oracle; scenes are in general position
# (every determinant it uses is far from zero, checked).
# ---------------------------------------------------------------------------

def _tri_tri_pairs(PA, TA, PB, TB):
    a0, a1, a2 = PA[TA[:, 0]], PA[TA[:, 1]], PA[TA[:, 2]]
    b0, b1, b2 = PB[TB[:, 0]], PB[TB[:, 1]], PB[TB[:, 2]]
    alo, ahi = np.minimum(np.minimum(a0, a1), a2), np.maximum(np.maximum(a0, a1), a2)
    blo, bhi = np.minimum(np.minimum(b0, b1), b2), np.maximum(np.maximum(b0, b1), b2)
    cand = []
    for i in range(0, len(TA), 512):
        ov = np.all((alo[i:i + 512, None] <= bhi[None]) & (blo[None] <= ahi[i:i + 512, None]), axis=2)
        ii, jj = np.nonzero(ov)
        cand.append(np.stack([ii + i, jj], 1))
    cand = np.concatenate(cand)
    P = np.stack([a0[cand[:, 0]], a1[cand[:, 0]], a2[cand[:, 0]]], 1)   # [m, 3, 3]
    Q = np.stack([b0[cand[:, 1]], b1[cand[:, 1]], b2[cand[:, 1]]], 1)
    n1 = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    n2 = np.cross(Q[:, 1] - Q[:, 0], Q[:, 2] - Q[:, 0])
    dP = np.einsum("mk,mvk->mv", n2, P - Q[:, :1])      # P's vertices against Q's plane
    dQ = np.einsum("mk,mvk->mv", n1, Q - P[:, :1])
    # a signed distance (times the normal's length) below 1e-10 of the
    # coordinate scale would make a float64 sign doubtful
    L = max(np.abs(PA).max(), np.abs(PB).max())
    tiny = (np.abs(dP).min(1) < 1e-10 * np.linalg.norm(n2, axis=1) * L) | \
           (np.abs(dQ).min(1) < 1e-10 * np.linalg.norm(n1, axis=1) * L)
    straddle = ~(np.all(dP > 0, 1) | np.all(dP < 0, 1) | np.all(dQ > 0, 1) | np.all(dQ < 0, 1))
    D = np.cross(n1, n2)

    def interval(V, d, D):
        # the lone vertex (sign differs from the other two) and the two
        # edges from it crossing the other plane
        s = np.sign(d)
        lone = np.where(s[:, 0] == s[:, 1], 2, np.where(s[:, 0] == s[:, 2], 1, 0))
        o1, o2 = (lone + 1) % 3, (lone + 2) % 3
        r = np.arange(len(V))
        proj = np.einsum("mk,mvk->mv", D, V)
        t = []
        for o in (o1, o2):
            f = d[r, lone] / (d[r, lone] - d[r, o])
            t.append(proj[r, lone] + (proj[r, o] - proj[r, lone]) * f)
        return np.minimum(t[0], t[1]), np.maximum(t[0], t[1])

    m = straddle
    lo1, hi1 = interval(P[m], dP[m], D[m])
    lo2, hi2 = interval(Q[m], dQ[m], D[m])
    hit = np.zeros(len(cand), bool)
    hit[np.nonzero(m)[0]] = (lo1 < hi2) & (lo2 < hi1)
    return int(hit.sum()), int(tiny.sum())


def _accounting_scenes():
    out = [("c1", meshgen.scene_c1())]
    for i, sc in enumerate(meshgen.scene_c4(n_pairs=6, lmax=3, seed=meshgen.BASE_SEED + 44)):
        # no jitter in these pairs: keep those in general position (checked)
        out.append((f"c4pair{i}", sc))
    return out


@pytest.mark.parametrize("name,scene", _accounting_scenes(), ids=lambda x: x if isinstance(x, str) else "")
def test_triangle_pair_accounting(name, scene):
    PA, PB = scene.positions("A"), scene.positions("B")
    n_tt, degenerate = _tri_tri_pairs(PA, scene.A.T, PB, scene.B.T)
    if degenerate:
        pytest.skip("not in general position")
    pr = oracle.detect(PA, scene.A.T, True, PB, scene.B.T, True)
    n0 = int((pr.rec[:, 0] == 0).sum())
    n1 = int((pr.rec[:, 0] == 1).sum())
    assert n_tt == n0 + n1, (n_tt, n0, n1)
    if name == "c1":
        assert n_tt > 50


# ---------------------------------------------------------------------------
# Closed-mesh crossing parity on the large scenes: the two tori (262,144
# faces each) and sampled pairs of the 1,024-pair batch.  Inside/outside
# comes from the analytic shape (torus: distance from the core circle
# below r; sphere: distance from the centre below its radius) wherever the
# point is farther from that surface than the mesh can deviate from it,
# and from the winding number against the mesh near the surface.
# ---------------------------------------------------------------------------

def _inside(P, analytic_dist, r_surface, V, T, margin):
    d = analytic_dist(P)
    inside = d < r_surface
    near = np.abs(d - r_surface) <= margin
    if near.any():
        w = winding_number(P[near], V, T)
        assert np.all(np.abs(w - np.round(w)) < 1e-3)
        inside[near] = np.round(w).astype(int) != 0
    return inside


def _parity_check(PE, E, pairs_dir, inside):
    key = pairs_dir[:, 1].astype(np.int64) * (len(PE) + 1) + pairs_dir[:, 2]
    ekey = E[:, 0].astype(np.int64) * (len(PE) + 1) + E[:, 1]
    cnt = np.zeros(len(E), np.int64)
    np.add.at(cnt, np.searchsorted(ekey, key), 1)
    assert np.array_equal(cnt % 2, (inside[E[:, 0]] ^ inside[E[:, 1]]).astype(np.int64))


def test_closed_mesh_crossing_parity_two_tori():
    # The oracle runs on the edges that can reach the other torus: the
    # distance to the analytic surface is 1-Lipschitz, so an edge whose two
    # endpoints lie on the same side of it, each farther than the edge's
    # length plus the mesh's deviation from it, meets no face (and has no
    # crossing to count).  Every other edge goes through the brute-force
    # detection (the result on a subset of edges equals the full result on
    # that subset, pinned above).
    sc = meshgen.scene_c3()
    PA, PB = sc.positions("A"), sc.positions("B")
    R, r = sc.meta["R"], sc.meta["r"]
    Rm, centre = sc.meta["frame_B"]
    margin = 1e-3     # the polygonal tori lie within ~1.3e-4 of the analytic ones

    def dist_A(P):    # A sits at the origin around z
        return np.hypot(np.hypot(P[:, 0], P[:, 1]) - R, P[:, 2])

    def dist_B(P):
        q = (P - centre) @ Rm
        return np.hypot(np.hypot(q[:, 0], q[:, 1]) - R, q[:, 2])

    total = 0
    for PE, TE, PF, TF, dist in ((PA, sc.A.T, PB, sc.B.T, dist_B), (PB, sc.B.T, PA, sc.A.T, dist_A)):
        E = oracle.edges(TE)
        s = dist(PE) - r
        length = np.linalg.norm(PE[E[:, 0]] - PE[E[:, 1]], axis=1)
        far = (np.sign(s[E[:, 0]]) == np.sign(s[E[:, 1]])) & \
              (np.minimum(np.abs(s[E[:, 0]]), np.abs(s[E[:, 1]])) > length + margin)
        sub = np.nonzero(~far)[0]
        hits = oracle.detect_one_direction(PE, E[sub], PF, TF)
        cnt = np.zeros(len(E), np.int64)
        np.add.at(cnt, sub[hits[:, 0]], 1)
        inside = _inside(PE, dist, r, PF, TF, margin)
        assert np.array_equal(cnt % 2, (inside[E[:, 0]] ^ inside[E[:, 1]]).astype(np.int64))
        total += len(hits)
        assert len(sub) < len(E) // 5
    assert total > 500


def test_closed_mesh_crossing_parity_batch_pairs():
    scenes = meshgen.scene_c4()
    rng = np.random.default_rng(3)
    picked = 0
    for i in rng.permutation(len(scenes)):
        sc = scenes[i]
        if sc.A.n_tris > 5120 or sc.B.n_tris > 5120:
            continue
        PA, PB = sc.positions("A"), sc.positions("B")
        cB = sc.B.V.mean(axis=0)      # B = a unit icosphere rotated about its centre and moved
        pr = oracle.detect(PA, sc.A.T, True, PB, sc.B.T, True)
        # an icosphere's faces lie between radius cos(largest face angle)
        # and 1: the winding number decides within that shell
        inB = _inside(PA, lambda P: np.linalg.norm(P - cB, axis=1), 1.0, PB, sc.B.T, 0.25)
        inA = _inside(PB, lambda P: np.linalg.norm(P, axis=1), 1.0, PA, sc.A.T, 0.25)
        _parity_check(PA, oracle.edges(sc.A.T), pr.rec[pr.rec[:, 0] == 0], inB)
        _parity_check(PB, oracle.edges(sc.B.T), pr.rec[pr.rec[:, 0] == 1], inA)
        picked += len(pr) > 0
        if picked >= 8:
            break
    assert picked >= 8
