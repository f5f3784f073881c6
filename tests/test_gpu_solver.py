"""The minimizer (Eq. 7 / Eq. 8) on every path of the zone solver against the
float64 oracle: one stencil system whose impact zones (Sec. 4) have every
size class the solver distinguishes, in one hfcr_respond call.

The face mesh B is a set of disjoint quad strips; stencil j of a strip
pairs face j with its own edge-mesh vertex x0, so a strip's stencils share
face vertices with their neighbours (one zone per strip) and no vertex
with another strip.  Every row has its own x0, so the system is positive
definite.  Zone sizes: 20 stencils (one warp), 100 (a 256-thread half
CTA), 600 (a whole 512-thread CTA), 1,500 (a 1,024-thread CTA), 3,000 (too
large for one CTA's shared memory: a cluster of CTAs sharing theirs), and
700 zones of 40 stencils (more zones than the half-CTA solvers, so they
are handed out by the counter).  The same system through the float64 per-zone
solver of the plain float64 form (one CTA per zone, every size) and the
one-CTA global float64 CG, on float64 positions."""
import numpy as np
import pytest

import oracle
from gpu_util import dev_mesh, rel_err, respond

pytestmark = pytest.mark.gpu

TOL_DX = 1e-6


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_2081_gb300 import api as a
    a.lib()
    return a


def strips(sizes, rng):
    """Disjoint strips of faces (sizes[i] faces each, an even count), seeded
    jitter; returns vertices, counter-clockwise triangles and the first face
    of every strip."""
    V, T, first = [], [], []
    for s, nf in enumerate(sizes):
        L = nf // 2
        base = len(V)
        y0 = 0.5 * s
        for i in range(L + 1):
            V.append((0.1 * i, y0, 0.0))
            V.append((0.1 * i, y0 + 0.1, 0.0))
        first.append(len(T))
        for i in range(L):
            a, b, c, d = base + 2 * i, base + 2 * i + 1, base + 2 * i + 2, base + 2 * i + 3
            T.append((a, c, b))
            T.append((b, c, d))
    V = np.array(V) + rng.uniform(-0.01, 0.01, (len(V), 3))
    return V, np.array(T, np.int32), first


@pytest.mark.parametrize("solver,dtype,tol", [(0, np.float32, TOL_DX), (1, np.float64, 1e-9),
                                              (2, np.float64, 1e-9)],
                         ids=["mixed", "fp64_per_zone", "fp64_global"])
def test_zone_size_classes_against_oracle(api, solver, dtype, tol):
    import torch
    rng = np.random.default_rng(1409)
    sizes = [20, 20, 20, 100, 100, 100, 600, 600, 1500, 3000] + [40] * 700
    VB, TB, _ = strips(sizes, rng)
    k = sum(sizes)
    assert len(TB) == k
    # one edge-mesh vertex per stencil, just below its face's centroid
    cen = VB[TB].mean(axis=1)
    VA = cen + np.array([0.0, 0.0, -0.02]) + rng.uniform(-0.005, 0.005, (k, 3))
    TA = np.array([[0, 1, 2]], np.int32)
    A, PA = dev_mesh(api, VA, TA, False, dtype)
    B, PB = dev_mesh(api, VB, TB, True, dtype)
    st = np.zeros((k, 4), np.int32)
    st[:, 1] = np.arange(k)      # x0 (dir 0: a vertex of A)
    st[:, 2] = np.arange(k)      # its face of B
    ctx = api.Context(solver=solver)
    ctx.hfcr_reserve(max(len(VA), len(VB)), max(len(TA), len(TB)), 1 << 16)
    st_t = torch.tensor(st, device="cuda:0")
    g, info = respond(ctx, A, B, st_t, k, 1e-4, len(VA), len(VB), dtype)
    assert info.converged and info.n_stencils == k and info.rel_residual <= 1e-12
    rA, rB, _, sol = oracle.respond(st[:, :3].astype(np.uint32), PA, TA, PB, TB, 1e-4)
    assert rel_err(g, np.concatenate([rA, rB])) <= tol
    # every zone of the system is one strip (the oracle's union-find)
    assert sol.n_zones == len(sizes)
