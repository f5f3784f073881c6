"""The response setup (vertex CSR of the stencil entries, impact zones,
zone-ordered rows, groups of rows sharing x0 and their inverse blocks) as
one cooperative launch (setup_path 0, the default) against the same setup
as a sequence of kernels (setup_path 1).  Both take the same stable sorts
and the same union-find roots, so they build the same arrays and the
displacements are bit-identical.  One CTA runs the launch up to 8,192
stencils and the whole grid above; both sides of that boundary are
covered, with the float64 oracle minimizer (Eq. 7 / Eq. 8) as the reference
of the displacements."""
import numpy as np
import pytest

import meshgen
import oracle
from gpu_util import dev_mesh, detect, positions, rel_err, respond, stencils

pytestmark = pytest.mark.gpu

TOL_DX = 1e-6
SINGLE_CTA_MAX = 8192


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_2081_gb300 import api as a
    a.lib()
    return a


@pytest.fixture(scope="module")
def batch(api):
    """The 1,024-pair icosphere batch (levels 1..5) and its stencils
    (tens of thousands), on the concatenated meshes."""
    import torch
    scenes = meshgen.scene_c4()
    VA, TA, VB, TB, segs = meshgen.concat_batch(scenes)
    A, PA = dev_mesh(api, VA, TA, True, np.float32)
    B, PB = dev_mesh(api, VB, TB, True, np.float32)
    dsegs = torch.tensor(segs, device="cuda:0")
    ctx = api.Context()
    cap = 1 << 18
    ctx.hfcr_reserve(max(len(PA), len(PB)), max(len(TA), len(TB)), cap)
    out = torch.zeros((cap, 4), dtype=torch.int32, device="cuda:0")
    n = ctx.hfcr_detect_batch(A, B, dsegs, out)
    st_t, k, st = stencils(ctx, A, B, out, n, cap)
    assert k > 4 * SINGLE_CTA_MAX
    return dict(VA=VA, TA=TA, VB=VB, TB=TB, PA=PA, PB=PB, A=A, B=B, st_t=st_t, st=st, k=k,
                dsegs=dsegs, cap=cap)


def _respond_path(api, b, k, path):
    ctx = api.Context(setup_path=path)
    ctx.hfcr_reserve(max(len(b["PA"]), len(b["PB"])), max(len(b["TA"]), len(b["TB"])), b["cap"])
    g, info = respond(ctx, b["A"], b["B"], b["st_t"], k, 1e-4, len(b["PA"]), len(b["PB"]),
                      np.float32)
    ctx.close()
    return g, info


def test_paths_identical_cloth_torus(api):
    """The cloth/torus frame (about 1,600 stencils: the single-CTA form)."""
    sc = meshgen.scene_c2()
    A, PA = dev_mesh(api, sc.A.V, sc.A.T, False, np.float32)
    B, PB = dev_mesh(api, sc.B.V, sc.B.T, True, np.float32)
    res = []
    for path in (0, 1):
        ctx = api.Context(setup_path=path)
        ctx.hfcr_reserve(sc.A.n_verts, sc.A.n_tris, 1 << 16)
        out, n, _, _ = detect(ctx, A, B)
        st_t, k, st = stencils(ctx, A, B, out, n)
        g, info = respond(ctx, A, B, st_t, k, 1e-4, sc.A.n_verts, sc.B.n_verts, np.float32)
        res.append((g, info.cg_iters, info.n_touched, info.converged, st))
        ctx.close()
    assert np.array_equal(res[0][0], res[1][0]) and res[0][1:4] == res[1][1:4]
    assert 0 < len(res[0][4]) <= SINGLE_CTA_MAX
    rA, rB, _, _ = oracle.respond(res[0][4], PA, sc.A.T, PB, sc.B.T, 1e-4)
    assert rel_err(res[0][0], np.concatenate([rA, rB])) <= TOL_DX


@pytest.mark.parametrize("k", [1, 2, SINGLE_CTA_MAX - 1, SINGLE_CTA_MAX, SINGLE_CTA_MAX + 1, 30000])
def test_paths_identical_around_the_single_cta_limit(api, batch, k):
    """Prefixes of the batch's sorted stencil list (any subset of stencils
    is a valid system): one stencil, the last single-CTA size, the first
    grid-wide size and a larger one."""
    g0, i0 = _respond_path(api, batch, k, 0)
    g1, i1 = _respond_path(api, batch, k, 1)
    assert np.array_equal(g0, g1), k
    assert (i0.cg_iters, i0.n_touched, i0.converged) == (i1.cg_iters, i1.n_touched, i1.converged)
    assert i0.n_stencils == k and i0.converged
    if k in (SINGLE_CTA_MAX, SINGLE_CTA_MAX + 1):
        st = batch["st"][:k]
        rA, rB, _, _ = oracle.respond(st, batch["PA"], batch["TA"], batch["PB"], batch["TB"], 1e-4)
        assert rel_err(g0, np.concatenate([rA, rB])) <= TOL_DX


def test_batch_resolve_paths_identical(api, batch):
    """One batched repair iteration of all 1,024 pairs (the grid-wide form)
    through hfcr_resolve_batch: identical positions either way."""
    import torch
    res = []
    for path in (0, 1):
        A, _ = dev_mesh(api, batch["VA"], batch["TA"], True, np.float32)
        B, _ = dev_mesh(api, batch["VB"], batch["TB"], True, np.float32)
        ctx = api.Context(setup_path=path)
        ctx.hfcr_reserve(max(len(batch["PA"]), len(batch["PB"])),
                         max(len(batch["TA"]), len(batch["TB"])), batch["cap"])
        info = ctx.hfcr_resolve_batch(A, B, batch["dsegs"], 1e-4, 1)
        torch.cuda.synchronize()
        res.append((positions(A), positions(B), info.total_stencils, info.cg_iters))
        ctx.close()
    assert res[0][2] > SINGLE_CTA_MAX
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert res[0][2:] == res[1][2:]


def test_setup_path_validated(api):
    with pytest.raises(api.HfcrError) as e:
        api.Context(setup_path=2)
    assert e.value.status == api.HFCR_ERR_ARG
