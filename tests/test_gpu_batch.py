"""Batches of independent mesh pairs in one launch sequence
(hfcr_detect_batch / hfcr_resolve_batch) against the oracle run pair by
pair: the batched pair set is the union of the per-pair exact pair sets
(global ids), the displacements match the float64 minimizer, and the
batched repair loop leaves no intersection in any pair."""
import numpy as np
import pytest

import meshgen
import oracle
from gpu_util import dev_mesh, detect, positions, rel_err, respond, stencils

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_2081_gb300 import api as a
    a.lib()
    return a


def _batch(api, scenes):
    import torch
    VA, TA, VB, TB, segs = meshgen.concat_batch(scenes)
    A, PA = dev_mesh(api, VA, TA, True, np.float32)
    B, PB = dev_mesh(api, VB, TB, True, np.float32)
    return A, PA, TA, B, PB, TB, segs, torch.tensor(segs, device="cuda:0")


def _oracle_union(scenes, segs, PA, PB, dirs=(0, 1)):
    recs = []
    for i, sc in enumerate(scenes):
        a0, b0 = segs[i, 0], segs[i, 2]
        pA = PA[a0:segs[i + 1, 0]]
        pB = PB[b0:segs[i + 1, 2]]
        pr = oracle.detect(pA, sc.A.T, 1 in dirs, pB, sc.B.T, 0 in dirs)
        r = pr.rec.astype(np.int64)
        for d, ev, ef in ((0, a0, segs[i, 3]), (1, b0, segs[i, 1])):
            m = r[:, 0] == d
            r[m, 1] += ev
            r[m, 2] += ev
            r[m, 3] += ef
        recs.append(r)
    rec = np.concatenate(recs)
    return rec[np.lexsort((rec[:, 3], rec[:, 2], rec[:, 1], rec[:, 0]))].astype(np.uint32)


def test_batch_pairs_equal_per_pair_oracle(api):
    import torch
    scenes = meshgen.scene_c4(n_pairs=24, lmax=3)
    A, PA, TA, B, PB, TB, segs, dsegs = _batch(api, scenes)
    ctx = api.Context()
    ctx.hfcr_reserve(max(len(PA), len(PB)), max(len(TA), len(TB)), 1 << 17)
    out = torch.zeros((1 << 17, 4), dtype=torch.int32, device="cuda:0")
    n, st = ctx.hfcr_detect_batch(A, B, dsegs, out, stats=True)
    got = out[:n].cpu().numpy().astype(np.uint32)
    ref = _oracle_union(scenes, segs, PA, PB)
    assert n == len(ref) and np.array_equal(got, ref)
    # brute-force equivalent counts pair by pair, not across pairs
    bf = sum(2 * 1.5 * sc.A.n_tris * sc.B.n_tris for sc in scenes)
    assert st.brute_force_equiv == bf
    # the same stencils and displacements as the float64 minimizer on the concatenation
    st_t, k, stc = stencils(ctx, A, B, out, n, 1 << 17)
    assert np.array_equal(stc, oracle.stencils(oracle.Pairs(ref, _sides(ref, PA, TA, PB, TB))))
    assert k > 0
    g, info = respond(ctx, A, B, st_t, k, 1e-4, len(PA), len(PB), np.float32)
    rA, rB, _, _ = oracle.respond(stc, PA, TA, PB, TB, 1e-4)
    assert rel_err(g, np.concatenate([rA, rB])) <= 1e-6
    # every traversal variant, the per-warp packet walks included (warps of
    # these small pairs often span two pairs and fall back to per-edge walks)
    # and the persistent walks fed by a work queue (lanes of one warp walk
    # edges of different pairs)
    for v in range(1, api.N_TRAVERSE_VARIANTS):
        cv = api.Context(traverse_variant=v)
        cv.hfcr_reserve(max(len(PA), len(PB)), max(len(TA), len(TB)), 1 << 17)
        nv = cv.hfcr_detect_batch(A, B, dsegs, out)
        assert nv == n and np.array_equal(out[:nv].cpu().numpy().astype(np.uint32), ref), v
        cv.close()


def _sides(rec, PA, TA, PB, TB):
    side = np.zeros(len(rec), np.int8)
    for i, (d, v0, v1, f) in enumerate(rec.tolist()):
        PE, PF, TF = (PA, PB, TB) if d == 0 else (PB, PA, TA)
        side[i] = oracle.orient(*PF[TF[f]], PE[v0])
    return side


def test_single_segment_batch_equals_detect(api):
    import torch
    sc = meshgen.scene_random_small(71, "torus_sphere")
    A, PA = dev_mesh(api, sc.A.V, sc.A.T, True, np.float32)
    B, PB = dev_mesh(api, sc.B.V, sc.B.T, True, np.float32)
    ctx = api.Context()
    ctx.hfcr_reserve(4096, 4096, 1 << 14)
    segs = torch.tensor([[0, 0, 0, 0], [sc.A.n_verts, sc.A.n_tris, sc.B.n_verts, sc.B.n_tris]],
                        dtype=torch.int32, device="cuda:0")
    out = torch.zeros((1 << 14, 4), dtype=torch.int32, device="cuda:0")
    n = ctx.hfcr_detect_batch(A, B, segs, out)
    _, n1, got1, _ = detect(ctx, A, B, 1 << 14)
    assert n == n1 and np.array_equal(out[:n].cpu().numpy().astype(np.uint32), got1)
    bad = segs.clone()
    bad[1, 1] = sc.A.n_tris + 3
    with pytest.raises(api.HfcrError) as e:
        ctx.hfcr_detect_batch(A, B, bad, out)
    assert e.value.status == api.HFCR_ERR_ARG


def test_batch_resolve_leaves_no_pair(api):
    # moderate overlaps (centre distance 1.6..1.9 radii): deeper ones make the
    # literal repair loop diverge, pair or batch alike
    scenes = meshgen.scene_c4(n_pairs=16, lmax=3, seed=meshgen.BASE_SEED + 33, rho_lo=1.6, rho_hi=1.9)
    A, PA, TA, B, PB, TB, segs, dsegs = _batch(api, scenes)
    ctx = api.Context()
    ctx.hfcr_reserve(max(len(PA), len(PB)), max(len(TA), len(TB)), 1 << 17)
    info = ctx.hfcr_resolve_batch(A, B, dsegs, 1e-4, 64)
    assert info.pairs_first > 0
    assert info.converged, (info.iters, info.pairs_last)
    fA, fB = positions(A), positions(B)
    assert len(_oracle_union(scenes, segs, fA, fB)) == 0


def test_batch_resolve_with_diffusion_deep_overlaps(api):
    # deeper overlaps (centre distance 1.35..1.6 radii): the harmonic diffusion
    # of Sec. 5 spreads each pair's displacement over its own mesh only (the
    # concatenated meshes have no edge between pairs), and the batched loop
    # ends with no pair left
    scenes = meshgen.scene_c4(n_pairs=12, lmax=3, seed=meshgen.BASE_SEED + 34, rho_lo=1.35, rho_hi=1.6)
    A, PA, TA, B, PB, TB, segs, dsegs = _batch(api, scenes)
    ctx = api.Context(diffuse_rings=4)
    ctx.hfcr_reserve(max(len(PA), len(PB)), max(len(TA), len(TB)), 1 << 17)
    info = ctx.hfcr_resolve_batch(A, B, dsegs, 1e-4, 64)
    assert info.diffuse_unconverged == 0
    assert info.pairs_first > 0
    assert info.converged, (info.iters, info.pairs_last)
    fA, fB = positions(A), positions(B)
    assert len(_oracle_union(scenes, segs, fA, fB)) == 0
    # every vertex stayed within its own pair's displacement field: the
    # vertices of a pair without any intersection did not move
    for i, sc in enumerate(scenes):
        a0, a1, b0, b1 = segs[i, 0], segs[i + 1, 0], segs[i, 2], segs[i + 1, 2]
        hit = len(oracle.detect(PA[a0:a1], sc.A.T, True, PB[b0:b1], sc.B.T, True)) > 0
        if not hit:
            assert np.array_equal(fA[a0:a1], PA[a0:a1]) and np.array_equal(fB[b0:b1], PB[b0:b1])


def test_batch_with_a_long_pair_takes_the_global_sort(api):
    # a pair whose mesh has more faces than one CTA sorts (36,000 > 32,768):
    # the per-pair BVH sort hands the whole batch to the global sort, and
    # the pairs still equal the per-pair oracle's
    import torch
    rng = np.random.default_rng(41)
    VT, TT = meshgen.torus(200, 90, 1.0, 0.3)
    VS, TS = meshgen.icosphere(2, 0.5)
    scenes = []
    for k in range(3):
        VA = VS + np.array([1.0, 0.0, 0.25]) + rng.uniform(-0.05, 0.05, 3)
        VB, TB = (VT, TT) if k == 1 else meshgen.icosphere(2, 0.6)
        scenes.append(meshgen.Scene(meshgen.Mesh(VA, TS, True), meshgen.Mesh(VB, TB, True), np.float32))
    A, PA, TA, B, PB, TB, segs, dsegs = _batch(api, scenes)
    assert segs[2, 3] - segs[1, 3] > 32768
    ctx = api.Context()
    ctx.hfcr_reserve(max(len(PA), len(PB)), max(len(TA), len(TB)), 1 << 17)
    out = torch.zeros((1 << 17, 4), dtype=torch.int32, device="cuda:0")
    n = ctx.hfcr_detect_batch(A, B, dsegs, out)
    got = out[:n].cpu().numpy().astype(np.uint32)
    ref = _oracle_union(scenes, segs, PA, PB)
    assert n > 0 and n == len(ref) and np.array_equal(got, ref)


def test_full_batch_sampled(api):
    """1,024 pairs, levels 1..5 (the batched workload): every reported pair
    of a sample re-checked exactly, and 12 sampled pairs compared in full."""
    import torch
    scenes = meshgen.scene_c4()
    A, PA, TA, B, PB, TB, segs, dsegs = _batch(api, scenes)
    ctx = api.Context()
    ctx.hfcr_reserve(max(len(PA), len(PB)), max(len(TA), len(TB)), 1 << 22)
    out = torch.zeros((1 << 22, 4), dtype=torch.int32, device="cuda:0")
    n = ctx.hfcr_detect_batch(A, B, dsegs, out)
    got = out[:n].cpu().numpy().astype(np.int64)
    assert n > 10000
    rng = np.random.default_rng(5)
    for d, v0, v1, f in got[rng.choice(n, 500, replace=False)].tolist():
        PE, PF, TF = (PA, PB, TB) if d == 0 else (PB, PA, TA)
        assert oracle.segtri(PE[v0], PE[v1], *PF[TF[f]])[0]
    for i in rng.choice(len(scenes), 12, replace=False):
        sub = [scenes[i]]
        ref = _oracle_union(sub, np.array([[0, 0, 0, 0], [scenes[i].A.n_verts, scenes[i].A.n_tris,
                                                          scenes[i].B.n_verts, scenes[i].B.n_tris]]),
                            PA[segs[i, 0]:segs[i + 1, 0]], PB[segs[i, 2]:segs[i + 1, 2]]).astype(np.int64)
        m0 = (got[:, 0] == 0) & (got[:, 1] >= segs[i, 0]) & (got[:, 1] < segs[i + 1, 0])
        m1 = (got[:, 0] == 1) & (got[:, 1] >= segs[i, 2]) & (got[:, 1] < segs[i + 1, 2])
        mine = got[m0 | m1].copy()
        mine[mine[:, 0] == 0, 1:3] -= segs[i, 0]
        mine[mine[:, 0] == 0, 3] -= segs[i, 3]
        mine[mine[:, 0] == 1, 1:3] -= segs[i, 2]
        mine[mine[:, 0] == 1, 3] -= segs[i, 1]
        assert np.array_equal(mine, ref), i
