"""Pins of the oracle's diffusion of displacement vectors (Sec. 5: the
correction is spread from the penetrating vertices to their vicinity as a
harmonic vector field).  The reading: moved vertices are Dirichlet values,
vertices more than `rings` edges away and kinematic vertices are zero, the
band in between takes `sweeps` Jacobi sweeps of the neighbour mean from zero.

Each pin comes from outside the oracle's code: closed forms on a path graph,
the exact discrete Dirichlet problem solved by scipy (the limit the sweeps
approach), unweighted graph distances from scipy.sparse.csgraph, and the
maximum principle."""
import numpy as np
import pytest

import meshgen
import oracle


def path_edges(n):
    return np.array([[i, i + 1] for i in range(n - 1)], np.int32)


def test_disabled_is_identity():
    E = path_edges(6)
    dx = np.zeros((6, 3))
    dx[0] = (1.0, -2.0, 0.5)
    for R, S in ((0, 5), (3, 0)):
        assert np.array_equal(oracle.diffuse(dx, E, R, S), dx)


def test_path_first_sweeps_closed_form():
    # path 0-1-2-...; vertex 0 moved by 1: one sweep gives u1 = 1/2 (its
    # neighbours 0 and 2 hold 1 and 0), two sweeps u1 = 1/2, u2 = 1/4,
    # three sweeps u1 = (1 + 1/4)/2, u2 = 1/4, u3 = 1/8
    E = path_edges(10)
    dx = np.zeros((10, 3))
    dx[0, 0] = 1.0
    u1 = oracle.diffuse(dx, E, 5, 1)[:, 0]
    assert np.array_equal(u1[:4], [1.0, 0.5, 0.0, 0.0])
    u2 = oracle.diffuse(dx, E, 5, 2)[:, 0]
    assert np.array_equal(u2[:4], [1.0, 0.5, 0.25, 0.0])
    u3 = oracle.diffuse(dx, E, 5, 3)[:, 0]
    assert np.array_equal(u3[:5], [1.0, 0.625, 0.25, 0.125, 0.0])


def test_path_limit_is_linear_interpolation():
    # the harmonic field on a path with u0 = 1 and u_{R+1} = 0 is linear
    R, n = 5, 12
    E = path_edges(n)
    dx = np.zeros((n, 3))
    dx[0] = (1.0, 2.0, -3.0)
    u = oracle.diffuse(dx, E, R, 4000)
    i = np.arange(n)
    lin = np.where(i <= R + 1, 1.0 - i / (R + 1), 0.0)
    assert np.allclose(u, lin[:, None] * dx[0][None, :], rtol=0, atol=1e-12)


def _grid(n):
    V, T = meshgen.cloth(n, 1.0)
    return V, T, oracle.edges(T)


def test_ring_distance_matches_graph_distance():
    scipy = pytest.importorskip("scipy.sparse.csgraph")
    import scipy.sparse as sp
    V, T, E = _grid(12)
    n = len(V)
    rng = np.random.default_rng(5)
    dx = np.zeros((n, 3))
    moved = rng.choice(n, 4, replace=False)
    dx[moved] = rng.normal(size=(4, 3))
    R = 3
    u = oracle.diffuse(dx, E, R, 1)
    A = sp.coo_matrix((np.ones(len(E)), (E[:, 0], E[:, 1])), shape=(n, n))
    dist = scipy.shortest_path(A, directed=False, unweighted=True, indices=moved).min(axis=0)
    # after one sweep exactly the vertices at distance 1 have nonzero values
    nz = np.any(u != 0, axis=1)
    assert np.array_equal(nz, dist <= 1)
    # a vertex farther than R never moves, however many sweeps
    u = oracle.diffuse(dx, E, R, 50)
    assert np.all(u[dist > R] == 0) and np.all(np.any(u[(dist >= 1) & (dist <= R)] != 0, axis=1))


def test_sweep_limit_is_the_dirichlet_solution():
    # the discrete Dirichlet problem (graph Laplacian on the band, moved
    # vertices and the outer boundary fixed), solved directly by scipy
    pytest.importorskip("scipy.sparse.linalg")
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla
    import scipy.sparse.csgraph as cg
    V, T, E = _grid(10)
    n = len(V)
    rng = np.random.default_rng(7)
    dx = np.zeros((n, 3))
    moved = np.array([33, 34, 45, 46])
    dx[moved] = rng.normal(size=(4, 3)) * 0.01
    R = 3
    A = sp.coo_matrix((np.ones(len(E)), (E[:, 0], E[:, 1])), shape=(n, n)).tocsr()
    A = A + A.T
    dist = cg.shortest_path(A, directed=False, unweighted=True, indices=moved).min(axis=0)
    free = (dist >= 1) & (dist <= R)
    fi = np.nonzero(free)[0]
    deg = np.asarray(A.sum(axis=1)).ravel()
    L = sp.diags(deg[fi]) - A[fi][:, fi]
    rhs = A[fi][:, moved] @ dx[moved]
    exact = np.zeros_like(dx)
    exact[moved] = dx[moved]
    for c in range(3):
        exact[fi, c] = sla.spsolve(L.tocsc(), rhs[:, c])
    u = oracle.diffuse(dx, E, R, 3000)
    assert np.max(np.abs(u - exact)) <= 1e-13


def test_maximum_principle_and_fixed_vertices():
    V, T, E = _grid(14)
    n = len(V)
    rng = np.random.default_rng(11)
    dx = np.zeros((n, 3))
    moved = rng.choice(n, 6, replace=False)
    dx[moved] = rng.normal(size=(6, 3))
    fixed = np.zeros(n, bool)
    fixed[rng.choice(np.setdiff1d(np.arange(n), moved), 20, replace=False)] = True
    u = oracle.diffuse(dx, E, 4, 25, fixed)
    assert np.array_equal(u[moved], dx[moved])
    assert np.all(u[fixed] == 0)
    for c in range(3):
        lo, hi = min(0.0, dx[moved, c].min()), max(0.0, dx[moved, c].max())
        assert np.all(u[:, c] >= lo - 1e-15) and np.all(u[:, c] <= hi + 1e-15)
