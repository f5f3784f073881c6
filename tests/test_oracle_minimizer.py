"""Pins for the oracle's constraint assembly and displacement minimizer
(Sec. 4, Eqs. 1-8) and for its repair loop (Sec. 3).

* Single constraint, closed form (Sec. 4, k = 1, equal masses, alpha = 1/3):
  with D = -h and target d, lambda solves (4/3) lambda = -h - d, so x0
  moves by +3/4 (h + d) n, each face vertex by -1/4 (h + d) n, the face
  normal is unchanged and the new signed distance is exactly d.
* Eq. 3 as a constrained least-squares problem solved through its KKT
  system with numpy's lstsq (a different route from the normal equations).
* Per-zone solves equal one global dense solve (the zones only split a
  block-diagonal system).
* scipy.sparse.linalg.spsolve on the full first-iteration system of the
  cloth-vs-torus scene; the conjugate-gradient branch against the dense one.
* Impact zones equal scipy's connected components of the stencil graph.
* Termination: after the loop the exact detection finds no pair.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg
import scipy.sparse.linalg as spla

import meshgen
import oracle


def _single(h, d, tilt=0.0):
    # oriented face B in the plane z=0 (normal +z), A: an edge from x0 below
    # the face to a vertex above it
    B = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0]])
    A = np.array([[0.3, 0.3, -h], [0.3 + tilt, 0.3, 1.0], [2.0, 2.0, 1.0]])
    return A, np.array([[0, 1, 2]], np.int32), B, np.array([[0, 1, 2]], np.int32)


@pytest.mark.parametrize("h,d", [(0.1, 0.0), (0.25, 1e-4), (1e-3, 0.05)])
def test_single_constraint_closed_form(h, d):
    PA, TA, PB, TB = _single(h, d)
    pr = oracle.detect(PA, TA, False, PB, TB, True)
    st = oracle.stencils(pr)
    assert st.tolist() == [[0, 0, 0]]
    dA, dB, asm, sol = oracle.respond(st, PA, TA, PB, TB, d)
    n = np.array([0, 0, 1.0])
    assert asm.D[0] == pytest.approx(-h, abs=1e-15)
    assert np.allclose(dA[0], 0.75 * (h + d) * n, atol=1e-15)
    assert np.allclose(dA[1:], 0, atol=0)
    for v in range(3):
        assert np.allclose(dB[v], -0.25 * (h + d) * n, atol=1e-15)
    nA, nB = PA + dA, PB + dB
    new_n = np.cross(nB[1] - nB[0], nB[2] - nB[0])
    assert np.allclose(new_n / np.linalg.norm(new_n), n, atol=1e-15)
    D_new = np.dot(new_n / np.linalg.norm(new_n), nA[0] - nB.mean(0))
    assert D_new == pytest.approx(d, abs=1e-14)


def _random_problem(rng, nA=40, nB_tris=12, k=15, inv_mass=False):
    VB = rng.uniform(-1, 1, (3 * nB_tris, 3))
    TB = np.arange(3 * nB_tris, dtype=np.int32).reshape(-1, 3)
    VA = rng.uniform(-1, 1, (nA, 3))
    TA = np.array([[0, 1, 2]], np.int32)
    x0 = rng.choice(nA, k, replace=False)
    f = rng.integers(0, nB_tris, k)
    st = np.unique(np.stack([np.zeros(k, np.uint32), x0, f], 1).astype(np.uint32), axis=0)
    w = rng.uniform(0.5, 2.0, nA + 3 * nB_tris) if inv_mass else None
    return VA, TA, VB, TB, st, w


@pytest.mark.parametrize("seed,inv_mass", [(0, False), (1, False), (2, True), (3, True)])
def test_minimizer_matches_kkt_lstsq(seed, inv_mass):
    """Eq. 3: min |x' - x|_M^2 s.t. grad(D) x' = d, solved as the KKT system
    [[M, J^T], [J, 0]] [x'; mu] = [M x; d]."""
    rng = np.random.default_rng(seed)
    VA, TA, VB, TB, st, w = _random_problem(rng, inv_mass=inv_mass)
    d = 0.01
    dA, dB, asm, sol = oracle.respond(st, VA, TA, VB, TB, d, w)
    J = oracle.gradient_matrix(asm).toarray()
    x = np.concatenate([VA, VB]).ravel()
    wv = np.ones(asm.n_verts) if w is None else w
    M = np.diag(np.repeat(1.0 / wv, 3))
    k, n3 = J.shape
    K = np.block([[M, J.T], [J, np.zeros((k, k))]])
    rhs = np.concatenate([M @ x, np.full(k, d)])
    sol_kkt = np.linalg.lstsq(K, rhs, rcond=None)[0]
    xp = sol_kkt[:n3]
    got = x + np.concatenate([dA, dB]).ravel()
    assert np.allclose(got, xp, atol=1e-12)
    # identities: grad(D) x = D (Sec. 4), grad(D) x' = d (Eq. 8)
    assert np.allclose(J @ x, asm.D, atol=1e-13)
    assert np.allclose(J @ got, d, atol=1e-12)
    # first stationary equation: M (x' - x) lies in the range of grad(D)^T
    mdx = M @ (got - x)
    coef = np.linalg.lstsq(J.T, mdx, rcond=None)[0]
    assert np.allclose(J.T @ coef, mdx, atol=1e-12)


def test_zones_equal_global_solve_and_connected_components():
    rng = np.random.default_rng(7)
    VA, TA, VB, TB, st, _ = _random_problem(rng, nA=200, nB_tris=60, k=50)
    asm = oracle.assemble(st, VA, TA, VB, TB, 0.0)
    sol = oracle.solve(asm)
    assert sol.n_zones > 1
    J = oracle.gradient_matrix(asm).toarray()
    A = J @ J.T
    lam = np.linalg.solve(A, asm.b)
    assert np.allclose(sol.dx.ravel(), -(J.T @ lam), atol=1e-12)
    # zones = connected components of the constraint-vertex incidence graph
    k = asm.ids.shape[0]
    rows = np.repeat(np.arange(k), 4)
    G = sp.csr_matrix((np.ones(4 * k), (rows, asm.ids.ravel() + k)), shape=(k + asm.n_verts,) * 2)
    ncomp, lab = csg.connected_components(G, directed=False)
    lab = lab[:k]
    for i in range(k):
        for j in range(k):
            assert (sol.zones[i] == sol.zones[j]) == (lab[i] == lab[j])


def test_spsolve_and_cg_branch_on_cloth_torus():
    sc = meshgen.scene_c2()
    PA, PB = sc.positions("A"), sc.positions("B")
    pr = oracle.detect(PA, sc.A.T, False, PB, sc.B.T, True)
    assert 2000 <= len(pr) <= 5000
    st = oracle.stencils(pr)
    asm = oracle.assemble(st, PA, sc.A.T, PB, sc.B.T, 1e-4)
    sol = oracle.solve(asm)
    J = oracle.gradient_matrix(asm).tocsc()
    A = (J @ J.T).tocsc()
    lam = spla.spsolve(A, asm.b)
    dx = -(J.T @ lam).reshape(-1, 3)
    scale = np.abs(dx).max()
    assert np.abs(sol.dx - dx).max() <= 1e-10 * scale
    x = np.concatenate([PA, PB]).ravel()
    assert np.abs(J @ (x + sol.dx.ravel()) - 1e-4).max() < 1e-12
    sol_cg = oracle.solve(asm, dense_max=0)
    assert sol_cg.cg_iters > 0
    assert np.abs(sol_cg.dx - sol.dx).max() <= 1e-10 * scale


def test_resolve_terminates_with_no_pairs():
    sc = meshgen.scene_c1()
    PA, PB = sc.positions("A"), sc.positions("B")
    r = oracle.resolve(PA, sc.A.T, True, PB, sc.B.T, True, 1e-4, 64)
    assert r.converged and r.pair_counts[0] > 0 and r.pair_counts[-1] == 0
    assert oracle.detect(r.PA, sc.A.T, True, r.PB, sc.B.T, True).rec.shape[0] == 0
    # alternate roles: even iterations edges of A vs faces of B, odd the reverse
    assert [dl for dl in r.dirs[:4]] == [[0], [1], [0], [1]]
    for seed in (21, 24):
        s = meshgen.scene_random_small(seed, "spheres")
        r = oracle.resolve(s.positions("A"), s.A.T, True, s.positions("B"), s.B.T, True,
                           1e-4, 64, store_dtype=np.float32)
        assert r.converged, r.pair_counts
        assert len(oracle.detect(r.PA, s.A.T, True, r.PB, s.B.T, True)) == 0


def test_resolve_reports_non_convergence():
    """Without the diffusion step of Sec. 5 the loop does not always reach a
    penetration-free state (a cloth patch sunk into a sphere keeps being
    peeled ring by ring while the sphere dents); the loop must then stop at
    max_iters and say so."""
    s = meshgen.scene_random_small(23, "cloth_sphere")
    r = oracle.resolve(s.positions("A"), s.A.T, False, s.positions("B"), s.B.T, True,
                       1e-4, 6, store_dtype=np.float32)
    assert not r.converged and r.iters == 6 and len(r.pair_counts) == 6
    assert all(c > 0 for c in r.pair_counts)


def test_resolve_both_directions_mode():
    sc = meshgen.scene_c1(offset=1.8)
    r = oracle.resolve(sc.positions("A"), sc.A.T, True, sc.positions("B"), sc.B.T, True,
                       1e-4, 64, mode="both")
    assert r.converged and all(dl == [0, 1] for dl in r.dirs)
    assert len(oracle.detect(r.PA, sc.A.T, True, r.PB, sc.B.T, True)) == 0
