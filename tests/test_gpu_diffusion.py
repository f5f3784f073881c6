"""Diffusion of displacement vectors (Sec. 5) on the GPU against the oracle.

The harmonic field (hfcr_diffuse with sweeps = 0, the default inside
hfcr_resolve): conjugate gradients on the band's graph Laplacian to a
relative residual of 1e-10 against the oracle's direct sparse solve of the
same Dirichlet problem.  The error of a CG iterate is at most the condition
number of the band Laplacian (below 10^3 for bands of up to 8 rings) times
its relative residual, so the bar is 1e-7 of the largest displacement.
The fixed-sweep approximation (sweeps > 0) runs the same sweeps as the
oracle's in the same float64 summation order: bit-identical.

Inside hfcr_resolve the field comes from the GPU's own minimizer; there the
check is the oracle's response + diffusion on the GPU's positions before the
iteration, within the solver tolerance, and exact detection on the positions
after it."""
import numpy as np
import pytest

import meshgen
import oracle
from gpu_util import dev_mesh, detect, positions

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-7   # of max |dx|, harmonic field at diffuse_tol 1e-10


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_2081_gb300 import api as a
    a.lib()
    return a


def _field(n, moved, rng, scale=1e-3):
    dx = np.zeros((n, 3))
    dx[moved] = rng.normal(size=(len(moved), 3)) * scale
    return dx


def _gpu_diffuse(api, ctx, M, dx, R, S=0):
    import torch
    t = [torch.tensor(np.ascontiguousarray(dx[:, c]), dtype=torch.float64, device="cuda:0")
         for c in range(3)]
    ctx.hfcr_diffuse(M, t, R, S)
    return np.stack([x.cpu().numpy() for x in t], 1)


def _mesh_of(kind):
    if kind == "cloth":
        return meshgen.cloth(97, 2.0)           # 9,409 vertices: a ragged tail of every grid
    if kind == "sphere":
        return meshgen.icosphere(4, 1.0)
    return meshgen.torus(61, 29, 1.0, 0.3)


@pytest.mark.parametrize("kind", ["cloth", "sphere", "torus"])
def test_diffuse_harmonic_matches_direct_solve(api, kind):
    rng = np.random.default_rng({"cloth": 1, "sphere": 2, "torus": 3}[kind])
    V, T = _mesh_of(kind)
    n = len(V)
    ctx = api.Context()
    ctx.hfcr_reserve(n, len(T), 16)
    for edges in (False, True):                 # the caller's edge list, or derived from the faces
        M, _ = dev_mesh(api, V, T, False, np.float32, edges=edges)
        for R in (1, 4, 8):
            dx = _field(n, rng.choice(n, 40, replace=False), rng)
            got = _gpu_diffuse(api, ctx, M, dx, R)
            ref = oracle.diffuse(dx, oracle.edges(T), R)
            err = np.abs(got - ref).max() / np.abs(dx).max()
            assert err <= FIELD_TOL, (kind, edges, R, err)
            # moved vertices keep their values exactly, far ones stay zero
            moved = np.any(dx != 0, axis=1)
            assert np.array_equal(got[moved], dx[moved])
            assert np.array_equal(got[np.all(ref == 0, axis=1)], ref[np.all(ref == 0, axis=1)])


def test_diffuse_harmonic_full_size_cloth_field(api):
    # the cloth's displacement of the first response of the 200 x 200
    # cloth / 256 x 128 torus scene (the oracle's), spread over R = 4 rings:
    # a band of about 8,600 vertices in several pieces
    sc = meshgen.scene_c2()
    PA, PB = sc.positions("A"), sc.positions("B")
    st = oracle.stencils(oracle.detect(PA, sc.A.T, False, PB, sc.B.T, True))
    dA, dB, _, _ = oracle.respond(st, PA, sc.A.T, PB, sc.B.T, 1e-4)
    ctx = api.Context()
    ctx.hfcr_reserve(sc.A.n_verts, sc.A.n_tris, 16)
    for dx, m in ((dA, sc.A), (dB, sc.B)):
        M, _ = dev_mesh(api, m.V, m.T, False, np.float32)
        got = _gpu_diffuse(api, ctx, M, dx, 4)
        ref = oracle.diffuse(dx, oracle.edges(m.T), 4)
        err = np.abs(got - ref).max() / np.abs(dx).max()
        assert err <= FIELD_TOL, err


def test_diffuse_harmonic_band_beyond_one_cluster(api):
    # 600 scattered moved vertices of a 400 x 400 cloth over R = 8 rings: a
    # band of tens of thousands of vertices, more than one thread-block
    # cluster holds, so the grid-wide kernel solves it
    rng = np.random.default_rng(12)
    V, T = meshgen.cloth(400, 2.0)
    n = len(V)
    ctx = api.Context()
    ctx.hfcr_reserve(n, len(T), 16)
    M, _ = dev_mesh(api, V, T, False, np.float32)
    dx = _field(n, rng.choice(n, 600, replace=False), rng)
    got = _gpu_diffuse(api, ctx, M, dx, 8)
    ref = oracle.diffuse(dx, oracle.edges(T), 8)
    band = int(np.count_nonzero(np.any(ref != 0, axis=1) & ~np.any(dx != 0, axis=1)))
    assert band > 40000, band
    err = np.abs(got - ref).max() / np.abs(dx).max()
    assert err <= FIELD_TOL, err


@pytest.mark.parametrize("kind", ["cloth", "sphere", "torus"])
def test_diffuse_jacobi_sweeps_bit_exact(api, kind):
    # the fixed-sweep approximation
    rng = np.random.default_rng({"cloth": 4, "sphere": 5, "torus": 6}[kind])
    V, T = _mesh_of(kind)
    n = len(V)
    ctx = api.Context()
    ctx.hfcr_reserve(n, len(T), 16)
    for edges in (False, True):
        M, _ = dev_mesh(api, V, T, False, np.float32, edges=edges)
        for R, S in ((1, 1), (4, 8), (7, 33)):
            dx = _field(n, rng.choice(n, 40, replace=False), rng)
            got = _gpu_diffuse(api, ctx, M, dx, R, S)
            ref = oracle.diffuse(dx, oracle.edges(T), R, S)
            assert np.array_equal(got, ref), (kind, edges, R, S)


def test_diffuse_kinematic_vertices_and_disabled(api):
    rng = np.random.default_rng(9)
    V, T = meshgen.cloth(40, 1.0)
    n = len(V)
    moved = rng.choice(n, 12, replace=False)
    w = np.ones(n, np.float32)
    fixed = rng.choice(np.setdiff1d(np.arange(n), moved), 150, replace=False)
    w[fixed] = 0.0
    ctx = api.Context()
    ctx.hfcr_reserve(n, len(T), 16)
    M, _ = dev_mesh(api, V, T, False, np.float32, inv_mass=w)
    dx = _field(n, moved, rng)
    got = _gpu_diffuse(api, ctx, M, dx, 5, 12)
    ref = oracle.diffuse(dx, oracle.edges(T), 5, 12, w == 0)
    assert np.array_equal(got, ref) and np.all(got[fixed] == 0)
    got = _gpu_diffuse(api, ctx, M, dx, 5)
    ref = oracle.diffuse(dx, oracle.edges(T), 5, 0, w == 0)
    assert np.abs(got - ref).max() <= FIELD_TOL * np.abs(dx).max() and np.all(got[fixed] == 0)
    # rings 0 leaves the field as it is; an all-zero field stays zero
    assert np.array_equal(_gpu_diffuse(api, ctx, M, dx, 0, 5), dx)
    assert np.array_equal(_gpu_diffuse(api, ctx, M, dx, 0), dx)
    assert np.all(_gpu_diffuse(api, ctx, M, np.zeros((n, 3)), 3) == 0)
    with pytest.raises(api.HfcrError):
        _gpu_diffuse(api, ctx, M, dx, -1, 3)


def test_diffuse_empty_band_and_iteration_limit(api):
    V, T = meshgen.cloth(30, 1.0)
    n = len(V)
    E = oracle.edges(T)
    ctx = api.Context()
    ctx.hfcr_reserve(n, len(T), 16)
    # every neighbour of the one moved vertex is kinematic: the band beyond
    # them sees only zero Dirichlet values, so the field stays as it is
    v = 15 * 30 + 15
    w = np.ones(n, np.float32)
    w[E[E[:, 0] == v, 1]] = 0.0
    w[E[E[:, 1] == v, 0]] = 0.0
    M, _ = dev_mesh(api, V, T, False, np.float32, inv_mass=w)
    dx = np.zeros((n, 3))
    dx[v] = (1e-3, -2e-3, 5e-4)
    assert np.array_equal(_gpu_diffuse(api, ctx, M, dx, 4), dx)
    # every vertex moved: the band is empty
    full = np.random.default_rng(3).normal(size=(n, 3)) * 1e-3
    M1, _ = dev_mesh(api, V, T, False, np.float32)
    assert np.array_equal(_gpu_diffuse(api, ctx, M1, full, 4), full)
    # two iterations cannot reach 1e-10 on a band of 4 rings: the call says so
    ctx2 = api.Context(diffuse_max_iters=2)
    ctx2.hfcr_reserve(n, len(T), 16)
    M2, _ = dev_mesh(api, V, T, False, np.float32)
    with pytest.raises(api.HfcrError) as e:
        _gpu_diffuse(api, ctx2, M2, dx, 4)
    assert e.value.status == api.HFCR_ERR_NOT_CONVERGED


def _resolve_step_parity(api, sc, R, S, iters, d=1e-4):
    """One repair iteration at a time with diffusion: the GPU's pairs equal
    the oracle's on the GPU positions (exact), and the GPU's new positions
    equal the oracle's response + diffusion from the same positions within
    the solver tolerance (a few float32 ulps)."""
    A, _ = dev_mesh(api, sc.A.V, sc.A.T, sc.A.oriented, np.float32)
    B, _ = dev_mesh(api, sc.B.V, sc.B.T, sc.B.oriented, np.float32)
    ctx = api.Context(diffuse_rings=R, diffuse_sweeps=S)
    ctx.hfcr_reserve(max(sc.A.n_verts, sc.B.n_verts), max(sc.A.n_tris, sc.B.n_tris), 1 << 16)
    EA, EB = oracle.edges(sc.A.T), oracle.edges(sc.B.T)
    converged = False
    for it in range(iters):
        PA, PB = positions(A), positions(B)
        _, n, got, _ = detect(ctx, A, B)
        ref = oracle.detect(PA, sc.A.T, sc.A.oriented, PB, sc.B.T, sc.B.oriented)
        assert np.array_equal(got, ref.rec), f"iteration {it}"
        if n == 0:
            converged = True
            break
        st = oracle.stencils(ref)
        dA, dB, _, _ = oracle.respond(st, PA, sc.A.T, PB, sc.B.T, d)
        eA = (PA + oracle.diffuse(dA, EA, R, S)).astype(np.float32).astype(np.float64)
        eB = (PB + oracle.diffuse(dB, EB, R, S)).astype(np.float32).astype(np.float64)
        info = ctx.hfcr_resolve(A, B, d, 1)
        assert info.pairs_first == n
        assert S > 0 or (info.diffuse_cg_iters > 0 and info.diffuse_unconverged == 0)
        gA, gB = positions(A), positions(B)
        scale = max(np.abs(dA).max(), np.abs(dB).max())
        tol = 1e-6 * scale + 4 * np.spacing(np.float32(max(np.abs(PA).max(), np.abs(PB).max())))
        assert np.abs(gA - eA).max() <= tol and np.abs(gB - eB).max() <= tol, f"iteration {it}"
        # diffusion moved vertices beyond the stencils
        moved = np.any(gA != PA, axis=1)
        assert moved.sum() > len(np.unique(np.concatenate([st[:, 1][st[:, 0] == 0]])))
    return converged


@pytest.mark.parametrize("S", [0, 8])
def test_resolve_with_diffusion_step_parity(api, S):
    sc = meshgen.scene_random_small(23, "cloth_sphere")
    _resolve_step_parity(api, sc, 4, S, 6)


def test_resolve_with_diffusion_converges(api):
    # the small cloth/sphere scene: the literal loop (no diffusion) does not
    # converge in 40 iterations, the loop with the harmonic diffusion does;
    # the final positions have no E-F intersection under the oracle's exact
    # detection
    sc = meshgen.scene_random_small(23, "cloth_sphere")
    res = {}
    for R in (0, 4):
        A, _ = dev_mesh(api, sc.A.V, sc.A.T, sc.A.oriented, np.float32)
        B, _ = dev_mesh(api, sc.B.V, sc.B.T, sc.B.oriented, np.float32)
        ctx = api.Context(diffuse_rings=R)
        ctx.hfcr_reserve(max(sc.A.n_verts, sc.B.n_verts), max(sc.A.n_tris, sc.B.n_tris), 1 << 17)
        info = ctx.hfcr_resolve(A, B, 1e-4, 40)
        res[R] = info
        if info.converged:
            left = oracle.detect(positions(A), sc.A.T, sc.A.oriented, positions(B), sc.B.T, sc.B.oriented)
            assert len(left) == 0
    assert res[4].converged and not res[0].converged
