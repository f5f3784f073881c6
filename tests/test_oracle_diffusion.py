"""Pins of the oracle's diffusion of displacement vectors (Sec. 5: the
correction is spread from the penetrating vertices to their vicinity as a
harmonic vector field).  The reading: moved vertices are Dirichlet values,
vertices more than `rings` edges away and kinematic vertices are zero, and
every vertex of the band in between is the mean of its neighbours (the
harmonic field, `sweeps` = 0); with `sweeps` > 0 the named approximation,
that many Jacobi sweeps of the neighbour mean from zero, instead.

Each pin comes from outside the oracle's code: closed forms of the harmonic
field on a path and on a torus band (where symmetry makes it linear in the
ring index), closed forms of the first Jacobi sweeps, unweighted graph
distances from scipy.sparse.csgraph, the maximum principle, and the mean
value property checked with neighbour lists built from the triangles."""
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
    for S in (0, 5):
        assert np.array_equal(oracle.diffuse(dx, E, 0, S), dx)
    # nothing moved: nothing to spread
    z = np.zeros((6, 3))
    assert np.array_equal(oracle.diffuse(z, E, 3), z)


def test_path_harmonic_is_linear_interpolation():
    # on a path, u0 = c and u_{R+1} = 0 with u_i the mean of u_{i-1} and
    # u_{i+1} in between: u_i = c (R + 1 - i) / (R + 1), zero beyond
    for R in (1, 2, 5):
        n = R + 6
        E = path_edges(n)
        dx = np.zeros((n, 3))
        dx[0] = (1.0, 2.0, -3.0)
        u = oracle.diffuse(dx, E, R)
        i = np.arange(n)
        lin = np.where(i <= R + 1, (R + 1 - i) / (R + 1), 0.0)
        assert np.allclose(u, lin[:, None] * dx[0][None, :], rtol=0, atol=1e-14), R


def test_path_between_two_moved_vertices():
    # both ends moved (u0 = a, u6 = b), the band is the five vertices in
    # between: the harmonic field interpolates linearly from a to b
    E = path_edges(7)
    dx = np.zeros((7, 3))
    a, b = np.array([1.0, -1.0, 0.25]), np.array([-2.0, 0.5, 4.0])
    dx[0], dx[6] = a, b
    u = oracle.diffuse(dx, E, 3)
    t = np.arange(7)[:, None] / 6.0
    assert np.allclose(u, (1 - t) * a + t * b, rtol=0, atol=1e-14)


def test_torus_band_closed_form():
    # every vertex of one meridian circle (index i = 0 of a torus grid)
    # moved by the same vector c.  The triangulation's diagonal joins (i, j)
    # to (i + 1, j + 1), so each vertex has two neighbours with index i - 1,
    # two with i and two with i + 1: by symmetry in j the harmonic field
    # depends on i alone and is linear in |i| on the band, reaching zero
    # at ring R + 1: u = c (R + 1 - |i|) / (R + 1)
    nu, nv, R = 24, 10, 4
    V, T = meshgen.torus(nu, nv, 1.0, 0.3)
    E = oracle.edges(T)
    dx = np.zeros((nu * nv, 3))
    c = np.array([0.003, -0.0015, 0.0007])
    dx[0:nv] = c                      # vertex id = i * nv + j
    u = oracle.diffuse(dx, E, R)
    i = np.arange(nu * nv) // nv
    ring = np.minimum(i, nu - i)      # distance around the torus to i = 0
    want = np.where(ring <= R + 1, (R + 1 - ring) / (R + 1), 0.0)[:, None] * c[None, :]
    assert np.allclose(u, want, rtol=0, atol=1e-15)
    # the fixed-sweep approximation lags behind the harmonic field inside
    # the band and approaches it with more sweeps
    u8 = oracle.diffuse(dx, E, R, 8)
    u400 = oracle.diffuse(dx, E, R, 400)
    band = (ring >= 1) & (ring <= R)
    assert np.all(np.abs(u8[band, 0]) < np.abs(want[band, 0]))
    assert np.abs(u400 - want).max() < 1e-12 < np.abs(u8 - want).max()


def test_path_first_sweeps_closed_form():
    # the fixed-sweep approximation: path 0-1-2-...; vertex 0 moved by 1:
    # one sweep gives u1 = 1/2 (its neighbours 0 and 2 hold 1 and 0), two
    # sweeps u1 = 1/2, u2 = 1/4, three sweeps u1 = (1 + 1/4)/2, u2 = 1/4,
    # u3 = 1/8
    E = path_edges(10)
    dx = np.zeros((10, 3))
    dx[0, 0] = 1.0
    u1 = oracle.diffuse(dx, E, 5, 1)[:, 0]
    assert np.array_equal(u1[:4], [1.0, 0.5, 0.0, 0.0])
    u2 = oracle.diffuse(dx, E, 5, 2)[:, 0]
    assert np.array_equal(u2[:4], [1.0, 0.5, 0.25, 0.0])
    u3 = oracle.diffuse(dx, E, 5, 3)[:, 0]
    assert np.array_equal(u3[:5], [1.0, 0.625, 0.25, 0.125, 0.0])


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
    A = sp.coo_matrix((np.ones(len(E)), (E[:, 0], E[:, 1])), shape=(n, n))
    dist = scipy.shortest_path(A, directed=False, unweighted=True, indices=moved).min(axis=0)
    # after one sweep exactly the vertices at distance 1 have nonzero values
    u = oracle.diffuse(dx, E, R, 1)
    assert np.array_equal(np.any(u != 0, axis=1), dist <= 1)
    # the harmonic field is nonzero exactly within R rings (the grid is
    # connected and the moved values are generic)
    u = oracle.diffuse(dx, E, R)
    assert np.all(u[dist > R] == 0) and np.all(np.any(u[dist <= R] != 0, axis=1))


def _neighbours_from_triangles(T, n):
    nb = [set() for _ in range(n)]
    for a, b, c in np.asarray(T):
        for p, q in ((a, b), (b, c), (c, a)):
            nb[p].add(int(q))
            nb[q].add(int(p))
    return nb


@pytest.mark.parametrize("kind", ["cloth", "sphere"])
def test_mean_value_property_on_the_band(kind):
    # every band vertex equals the mean of its neighbours (degrees 4..8 on
    # the cloth grid with its borders, 5 and 6 on the icosphere); moved
    # vertices keep their values, vertices beyond the band stay zero
    if kind == "cloth":
        V, T, E = _grid(15)
    else:
        V, T = meshgen.icosphere(3, 1.0)
        E = oracle.edges(T)
    n = len(V)
    rng = np.random.default_rng(13)
    dx = np.zeros((n, 3))
    moved = rng.choice(n, 7, replace=False)
    dx[moved] = rng.normal(size=(7, 3)) * 1e-3
    R = 3
    u = oracle.diffuse(dx, E, R)
    nb = _neighbours_from_triangles(T, n)
    # ring distances by breadth-first search over the triangle neighbours
    dist = np.full(n, 10 ** 9)
    dist[moved] = 0
    front = list(moved)
    while front:
        nxt = []
        for v in front:
            for w in nb[v]:
                if dist[w] > dist[v] + 1:
                    dist[w] = dist[v] + 1
                    nxt.append(w)
        front = nxt
    assert np.array_equal(u[moved], dx[moved])
    assert np.all(u[dist > R] == 0)
    scale = np.abs(dx).max()
    for v in np.nonzero((dist >= 1) & (dist <= R))[0]:
        mean = np.mean([u[w] for w in nb[v]], axis=0)
        assert np.abs(u[v] - mean).max() <= 1e-12 * scale, v


def test_maximum_principle_and_fixed_vertices():
    V, T, E = _grid(14)
    n = len(V)
    rng = np.random.default_rng(11)
    dx = np.zeros((n, 3))
    moved = rng.choice(n, 6, replace=False)
    dx[moved] = rng.normal(size=(6, 3))
    fixed = np.zeros(n, bool)
    fixed[rng.choice(np.setdiff1d(np.arange(n), moved), 20, replace=False)] = True
    for S in (0, 25):
        u = oracle.diffuse(dx, E, 4, S, fixed)
        assert np.array_equal(u[moved], dx[moved])
        assert np.all(u[fixed] == 0)
        for c in range(3):
            lo, hi = min(0.0, dx[moved, c].min()), max(0.0, dx[moved, c].max())
            assert np.all(u[:, c] >= lo - 1e-15) and np.all(u[:, c] <= hi + 1e-15)
