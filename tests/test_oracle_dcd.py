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
    for i in range(0, len(P), 256):
        Q = P[i:i + 256, None, :]
        a, b, c = V[T[:, 0]][None] - Q, V[T[:, 1]][None] - Q, V[T[:, 2]][None] - Q
        la, lb, lc = (np.linalg.norm(x, axis=2) for x in (a, b, c))
        num = np.einsum("pfk,pfk->pf", a, np.cross(b, c))
        den = (la * lb * lc + np.einsum("pfk,pfk->pf", a, b) * lc
               + np.einsum("pfk,pfk->pf", a, c) * lb + np.einsum("pfk,pfk->pf", b, c) * la)
        w[i:i + 256] = 2.0 * np.arctan2(num, den).sum(1) / (4.0 * np.pi)
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
