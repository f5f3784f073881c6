"""Parity of the CUDA path (called through the C ABI) with the CPU oracle.

* Pair sets and stencil sets: bit-exact (they are exact combinatorial
  results, Sec. 3 and Sec. 4).
* Displacements: |dx_gpu - dx_oracle|_inf <= 1e-6 |dx_oracle|_inf on the
  same stencils and positions (the float64 oracle solves Eq. 8 directly).
* Repair loop: every iteration's detection equals the oracle's detection on
  the GPU's own positions; after convergence the oracle finds no pair.
"""
import json
import os

import numpy as np
import pytest

import meshgen
import oracle
from gpu_util import dev_mesh, detect, positions, rel_err, respond, stencils

pytestmark = pytest.mark.gpu

TOL_DX = 1e-6
GOLD = os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_2081_gb300 import api as a
    a.lib()
    return a


def make_ctx(api, nv, nt, pairs=1 << 16, **kw):
    ctx = api.Context(**kw)
    ctx.hfcr_reserve(nv, nt, pairs)
    return ctx


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("case", json.load(open(GOLD))["cases"], ids=lambda c: c["name"])
def test_hand_cases(api, case, dtype):
    A, _ = dev_mesh(api, case["A"]["V"], case["A"]["T"], case["A"]["oriented"], dtype)
    B, _ = dev_mesh(api, case["B"]["V"], case["B"]["T"], case["B"]["oriented"], dtype)
    ctx = make_ctx(api, 16, 16, 64)
    out, n, got, _ = detect(ctx, A, B, 64)
    assert got.tolist() == case["pairs"]
    _, k, st = stencils(ctx, A, B, out, n, 64)
    assert st.tolist() == case["stencils"]


def _scene_parity(api, sc, solver, f32_filter, d=1e-4):
    dt = sc.dtype
    A, PA = dev_mesh(api, sc.A.V, sc.A.T, sc.A.oriented, dt)
    B, PB = dev_mesh(api, sc.B.V, sc.B.T, sc.B.oriented, dt)
    ctx = make_ctx(api, max(sc.A.n_verts, sc.B.n_verts), max(sc.A.n_tris, sc.B.n_tris), 1 << 16,
                   solver=solver, f32_filter=f32_filter)
    out, n, got, stats = detect(ctx, A, B)
    ref = oracle.detect(PA, sc.A.T, sc.A.oriented, PB, sc.B.T, sc.B.oriented)
    assert n == len(ref) and np.array_equal(got, ref.rec)
    st_t, k, st = stencils(ctx, A, B, out, n)
    ref_st = oracle.stencils(ref)
    assert np.array_equal(st, ref_st)
    g, info = respond(ctx, A, B, st_t, k, d, sc.A.n_verts, sc.B.n_verts, dt)
    rA, rB, _, _ = oracle.respond(ref_st, PA, sc.A.T, PB, sc.B.T, d)
    r = np.concatenate([rA, rB])
    err = rel_err(g, r)
    assert err <= TOL_DX, f"dx relative error {err:.3e}"
    assert info.converged and info.rel_residual <= 1e-12
    assert stats.narrow_tests > 0
    return n, k, err, stats


@pytest.mark.parametrize("solver", [0, 1, 2], ids=["mixed", "fp64", "fp64_global"])
@pytest.mark.parametrize("seed,kind", [(31, "spheres"), (32, "torus_sphere"), (33, "cloth_sphere"),
                                       (34, "spheres")])
def test_small_scenes(api, seed, kind, solver):
    _scene_parity(api, meshgen.scene_random_small(seed, kind), solver, True)


@pytest.mark.parametrize("seed,kind", [(35, "torus_sphere"), (36, "cloth_sphere")])
def test_small_scenes_without_f32_filter(api, seed, kind):
    _scene_parity(api, meshgen.scene_random_small(seed, kind), 0, False)


@pytest.mark.parametrize("solver", [0, 1, 2], ids=["mixed", "fp64", "fp64_global"])
def test_two_icospheres_fp64(api, solver):
    """Two jittered level-3 icospheres offset by 1.5, float64 positions."""
    n, k, err, st = _scene_parity(api, meshgen.scene_c1(), solver, True)
    assert n > 100 and k > 50


def test_cloth_torus_full_size(api):
    """The cloth (200 x 200) over the torus (65,536 faces), float32: the
    full pair set against the brute-force oracle, and the displacements of
    the full stencil set."""
    n, k, err, st = _scene_parity(api, meshgen.scene_c2(), 0, True)
    assert 2000 <= n <= 5000
    assert st.narrow_tests < st.brute_force_equiv / 1000


def _loop_with_oracle(api, sc, max_iters, d=1e-4, roles="alternate"):
    """Drives detect -> stencils -> respond -> x += dx through the ABI and
    checks every detection against the oracle on the GPU's own positions."""
    import torch
    dt = sc.dtype
    A, _ = dev_mesh(api, sc.A.V, sc.A.T, sc.A.oriented, dt)
    B, _ = dev_mesh(api, sc.B.V, sc.B.T, sc.B.oriented, dt)
    ctx = make_ctx(api, max(sc.A.n_verts, sc.B.n_verts), max(sc.A.n_tris, sc.B.n_tris))
    counts, quiet = [], 0
    n_dirs = len(oracle.directions(sc.A.oriented, sc.B.oriented))
    need = n_dirs if roles == "alternate" else 1
    for it in range(max_iters):
        dirs = oracle.role_schedule(sc.A.oriented, sc.B.oriented, it, roles)
        A.c.oriented, B.c.oriented = int(1 in dirs), int(0 in dirs)
        out, n, got, _ = detect(ctx, A, B)
        PA, PB = positions(A), positions(B)
        ref = oracle.detect(PA, sc.A.T, bool(A.c.oriented), PB, sc.B.T, bool(B.c.oriented))
        assert np.array_equal(got, ref.rec), f"iteration {it}"
        counts.append(n)
        if n == 0:
            quiet += 1
            if quiet >= need:
                return counts, True, A, B
            continue
        quiet = 0
        st_t, k, st = stencils(ctx, A, B, out, n)
        assert np.array_equal(st, oracle.stencils(ref))
        g, _ = respond(ctx, A, B, st_t, k, d, sc.A.n_verts, sc.B.n_verts, dt)
        rA, rB, _, _ = oracle.respond(st, PA, sc.A.T, PB, sc.B.T, d)
        assert rel_err(g, np.concatenate([rA, rB])) <= TOL_DX
        nA = sc.A.n_verts
        for m, lo, hi in ((A, 0, nA), (B, nA, nA + sc.B.n_verts)):
            for c, t in enumerate((m.x, m.y, m.z)):
                t += torch.tensor(g[lo:hi, c], dtype=t.dtype, device=t.device)
    return counts, False, A, B


def test_repair_loop_per_iteration(api):
    sc = meshgen.scene_c1()
    counts, conv, A, B = _loop_with_oracle(api, sc, 64)
    assert conv and counts[0] > 0
    assert len(oracle.detect(positions(A), sc.A.T, True, positions(B), sc.B.T, True)) == 0


@pytest.mark.parametrize("seed", [41, 42])
def test_resolve_api_converges(api, seed):
    for sc in (meshgen.scene_c1(), meshgen.scene_random_small(seed, "spheres")):
        A, _ = dev_mesh(api, sc.A.V, sc.A.T, True, sc.dtype)
        B, _ = dev_mesh(api, sc.B.V, sc.B.T, True, sc.dtype)
        ctx = make_ctx(api, max(sc.A.n_verts, sc.B.n_verts), max(sc.A.n_tris, sc.B.n_tris))
        info = ctx.hfcr_resolve(A, B, 1e-4, 64)
        assert info.converged and info.pairs_first > 0 and info.pairs_last == 0
        assert info.worst_rel_residual <= 1e-12
        assert len(oracle.detect(positions(A), sc.A.T, True, positions(B), sc.B.T, True)) == 0


def test_resolve_api_matches_oracle_loop_counts(api):
    """Same role schedule and stopping rule as the oracle's loop: the
    detection counts agree while both runs see the same positions up to
    rounding; at least the first detection is identical."""
    sc = meshgen.scene_c1()
    A, PA = dev_mesh(api, sc.A.V, sc.A.T, True, sc.dtype)
    B, PB = dev_mesh(api, sc.B.V, sc.B.T, True, sc.dtype)
    ctx = make_ctx(api, sc.A.n_verts, sc.A.n_tris)
    info = ctx.hfcr_resolve(A, B, 1e-4, 64)
    r = oracle.resolve(PA, sc.A.T, True, PB, sc.B.T, True, 1e-4, 64)
    assert info.pairs_first == r.pair_counts[0]
    assert info.converged == r.converged


def test_resolve_reports_non_convergence(api):
    sc = meshgen.scene_random_small(23, "cloth_sphere")
    A, _ = dev_mesh(api, sc.A.V, sc.A.T, False, sc.dtype)
    B, _ = dev_mesh(api, sc.B.V, sc.B.T, True, sc.dtype)
    ctx = make_ctx(api, max(sc.A.n_verts, sc.B.n_verts), max(sc.A.n_tris, sc.B.n_tris))
    info = ctx.hfcr_resolve(A, B, 1e-4, 6)
    assert info.converged == 0 and info.iters == 6 and info.pairs_last > 0
    with pytest.raises(api.HfcrError) as e:
        ctx.hfcr_resolve(A, B, 1e-4, 2, raise_not_converged=True)
    assert e.value.status == api.HFCR_ERR_NOT_CONVERGED


def test_resolve_both_roles(api):
    sc = meshgen.scene_c1(offset=1.8)
    A, _ = dev_mesh(api, sc.A.V, sc.A.T, True, sc.dtype)
    B, _ = dev_mesh(api, sc.B.V, sc.B.T, True, sc.dtype)
    ctx = make_ctx(api, sc.A.n_verts, sc.A.n_tris, roles=api.HFCR_ROLES_BOTH)
    info = ctx.hfcr_resolve(A, B, 1e-4, 64)
    assert info.converged
    assert len(oracle.detect(positions(A), sc.A.T, True, positions(B), sc.B.T, True)) == 0


def test_near_degenerate_fallbacks(api):
    """Cloth vertices placed exactly on, or one ulp off, the planes of an
    oriented surface: the float32 filter must abstain and the float64 and
    exact stages decide; the pair set stays exact."""
    rng = np.random.default_rng(9)
    VB, TB = meshgen.cloth(9, 2.0)          # oriented sheet in z = 0
    VA, TA = meshgen.cloth(23, 1.7)
    VA[:, :2] += rng.uniform(-0.01, 0.01, (len(VA), 2))
    VA = VA.astype(np.float32)
    z = np.zeros(len(VA), np.float32)
    pick = rng.integers(0, 3, len(VA))
    z[pick == 1] = np.float32(1e-30)
    z[pick == 2] = -np.float32(1e-30)
    z += rng.choice(np.array([0, 1], np.float32), len(VA)) * np.float32(0.05) * rng.choice([-1, 1], len(VA)).astype(np.float32)
    VA[:, 2] = z
    sc = meshgen.Scene(meshgen.Mesh(VA.astype(np.float64), TA, False),
                       meshgen.Mesh(VB, TB, True), np.float32)
    n, k, err, st = _scene_parity(api, sc, 0, True)
    assert n > 0
    assert st.f64_fallbacks > 0


def test_edge_cases(api):
    import torch
    sc = meshgen.scene_random_small(51, "spheres")
    A, _ = dev_mesh(api, sc.A.V, sc.A.T, True, np.float32)
    B, _ = dev_mesh(api, sc.B.V, sc.B.T, True, np.float32)
    ctx = make_ctx(api, 1000, 1000, 4096)
    # capacity: the count is reported, the status says so
    out = torch.zeros((3, 4), dtype=torch.int32, device="cuda:0")
    with pytest.raises(api.HfcrError) as e:
        ctx.hfcr_detect(A, B, out)
    assert e.value.status == api.HFCR_ERR_CAPACITY
    # far apart: no pair, empty stencil set, respond with k = 0
    Bf, _ = dev_mesh(api, sc.B.V + 10.0, sc.B.T, True, np.float32)
    o2, n, got, _ = detect(ctx, A, Bf, 64)
    assert n == 0
    _, k, _ = stencils(ctx, A, Bf, o2, 0, 64)
    assert k == 0
    # empty face mesh
    E, _ = dev_mesh(api, sc.B.V, np.zeros((0, 3), np.int32), True, np.float32)
    assert detect(ctx, A, E, 64)[1] >= 0
    # no oriented mesh
    Au, _ = dev_mesh(api, sc.A.V, sc.A.T, False, np.float32)
    Bu, _ = dev_mesh(api, sc.B.V, sc.B.T, False, np.float32)
    with pytest.raises(api.HfcrError) as e:
        detect(ctx, Au, Bu, 64)
    assert e.value.status == api.HFCR_ERR_ARG
    # non-finite and out-of-range positions are refused
    V = sc.A.V.copy()
    V[5, 1] = np.nan
    An, _ = dev_mesh(api, V, sc.A.T, True, np.float32)
    with pytest.raises(api.HfcrError) as e:
        detect(ctx, An, B, 64)
    assert e.value.status == api.HFCR_ERR_NONFINITE
    V = sc.A.V.copy()
    V[7, 0] = 2.0 ** 40
    Ar, _ = dev_mesh(api, V, sc.A.T, True, np.float32)
    with pytest.raises(api.HfcrError) as e:
        detect(ctx, Ar, B, 64)
    assert e.value.status == api.HFCR_ERR_RANGE
    # a triangle index past the vertex count
    T = sc.A.T.copy()
    T[3, 2] = sc.A.n_verts + 5
    Ai, _ = dev_mesh(api, sc.A.V, T, True, np.float32)
    with pytest.raises(api.HfcrError) as e:
        detect(ctx, Ai, B, 64)
    assert e.value.status == api.HFCR_ERR_ARG
    # the context still works afterwards
    assert detect(ctx, A, B, 4096)[1] > 0
    # sizes above the reservation
    small = make_ctx(api, 10, 10, 10)
    with pytest.raises(api.HfcrError) as e:
        detect(small, A, B, 64)
    assert e.value.status == api.HFCR_ERR_CAPACITY


def test_caller_edges_and_build_edges(api):
    import torch
    sc = meshgen.scene_random_small(52, "torus_sphere")
    ctx = make_ctx(api, 4096, 4096)
    tris = torch.tensor(sc.A.T, device="cuda:0")
    out = torch.zeros((3 * sc.A.n_tris, 2), dtype=torch.int32, device="cuda:0")
    ne = ctx.hfcr_build_edges(tris, sc.A.n_verts, out)
    assert np.array_equal(out[:ne].cpu().numpy(), oracle.edges(sc.A.T))
    A, PA = dev_mesh(api, sc.A.V, sc.A.T, True, np.float32, edges=True)
    B, PB = dev_mesh(api, sc.B.V, sc.B.T, True, np.float32, edges=True)
    _, n, got, _ = detect(ctx, A, B)
    assert np.array_equal(got, oracle.detect(PA, sc.A.T, True, PB, sc.B.T, True).rec)


def test_inverse_masses(api):
    """Non-unit masses enter Eq. 7 as M^-1 (Sec. 4)."""
    sc = meshgen.scene_random_small(53, "spheres")
    rng = np.random.default_rng(53)
    wA = rng.uniform(0.5, 2.0, sc.A.n_verts)
    wB = rng.uniform(0.5, 2.0, sc.B.n_verts)
    A, PA = dev_mesh(api, sc.A.V, sc.A.T, True, np.float32, inv_mass=wA)
    B, PB = dev_mesh(api, sc.B.V, sc.B.T, True, np.float32, inv_mass=wB)
    ctx = make_ctx(api, 1000, 1000)
    out, n, got, _ = detect(ctx, A, B)
    st_t, k, st = stencils(ctx, A, B, out, n)
    g, info = respond(ctx, A, B, st_t, k, 1e-3, sc.A.n_verts, sc.B.n_verts, np.float32)
    w = np.concatenate([wA, wB]).astype(np.float32).astype(np.float64)
    rA, rB, _, _ = oracle.respond(st, PA, sc.A.T, PB, sc.B.T, 1e-3, inv_mass=w)
    assert rel_err(g, np.concatenate([rA, rB])) <= TOL_DX


def test_two_tori_sampled_full_size(api):
    """Two 262,144-face tori (float32): every GPU pair re-checked exactly,
    and completeness on a seeded sample of edges brute-forced by the
    oracle against all faces."""
    sc = meshgen.scene_c3()
    A, PA = dev_mesh(api, sc.A.V, sc.A.T, True, np.float32)
    B, PB = dev_mesh(api, sc.B.V, sc.B.T, True, np.float32)
    ctx = make_ctx(api, sc.A.n_verts, sc.A.n_tris, 1 << 20)
    out, n, got, st = detect(ctx, A, B, 1 << 20)
    assert n > 0
    for (d, v0, v1, f) in got[:: max(1, n // 2000)].tolist():
        PE, PF, TF = (PA, PB, sc.B.T) if d == 0 else (PB, PA, sc.A.T)
        ok, _ = oracle.segtri(PE[v0], PE[v1], *PF[TF[f]])
        assert ok
    rng = np.random.default_rng(3)
    for d, (PE, TE, PF, TF) in enumerate([(PA, sc.A.T, PB, sc.B.T), (PB, sc.B.T, PA, sc.A.T)]):
        E = oracle.edges(TE)
        # half the sample from edges that have pairs, half uniform
        have = np.unique(np.searchsorted(E[:, 0].astype(np.int64) * (1 << 32) + E[:, 1],
                                         got[got[:, 0] == d][:, 1].astype(np.int64) * (1 << 32)
                                         + got[got[:, 0] == d][:, 2]))
        sub = np.unique(np.concatenate([rng.choice(have, min(len(have), 500), replace=False)
                                        if len(have) else np.zeros(0, np.int64),
                                        rng.choice(len(E), 1500, replace=False)]))
        hits = oracle.detect_one_direction(PE, E[sub], PF, TF)
        ref = set((int(E[sub[h[0]], 0]), int(E[sub[h[0]], 1]), int(h[1])) for h in hits)
        subset = set(map(tuple, E[sub].tolist()))
        mine = set((v0, v1, f) for (dd, v0, v1, f) in got.tolist() if dd == d and (v0, v1) in subset)
        assert mine == ref


def test_two_tori_full_size_response(api):
    """The precision form on the two 262,144-face tori: every GPU pair is
    re-verified exactly (which also gives the side of v0), the stencils
    follow from those pairs as in the oracle, and the float32 CG with
    float64 refinement matches the float64 oracle minimizer on the full
    stencil set."""
    sc = meshgen.scene_c3()
    A, PA = dev_mesh(api, sc.A.V, sc.A.T, True, np.float32)
    B, PB = dev_mesh(api, sc.B.V, sc.B.T, True, np.float32)
    ctx = make_ctx(api, sc.A.n_verts, sc.A.n_tris, 1 << 20)
    out, n, got, _ = detect(ctx, A, B, 1 << 20)
    assert n > 0
    side = np.zeros(n, np.int8)
    for i, (d, v0, v1, f) in enumerate(got.tolist()):
        PE, PF, TF = (PA, PB, sc.B.T) if d == 0 else (PB, PA, sc.A.T)
        ok, sd = oracle.segtri(PE[v0], PE[v1], *PF[TF[f]])
        assert ok
        side[i] = sd
    ref_st = oracle.stencils(oracle.Pairs(got, side))
    st_t, k, st = stencils(ctx, A, B, out, n, 1 << 20)
    assert np.array_equal(st, ref_st)
    g, info = respond(ctx, A, B, st_t, k, 1e-4, sc.A.n_verts, sc.B.n_verts, np.float32)
    rA, rB, _, _ = oracle.respond(st, PA, sc.A.T, PB, sc.B.T, 1e-4)
    err = rel_err(g, np.concatenate([rA, rB]))
    assert err <= TOL_DX and info.converged


def test_graph_replay_matches_plain_launches(api):
    """Repair iterations replayed from captured CUDA graphs give bit-identical
    positions to plain launches, on the default and on a created stream, and
    a changed argument (d) is re-captured rather than replayed stale."""
    import torch
    sc = meshgen.scene_random_small(61, "spheres")
    results = []
    for graphs, use_stream in ((False, False), (True, False), (True, True)):
        A, _ = dev_mesh(api, sc.A.V, sc.A.T, True, np.float32)
        B, _ = dev_mesh(api, sc.B.V, sc.B.T, True, np.float32)
        ctx = make_ctx(api, 1000, 1000, graphs=graphs)
        st = torch.cuda.Stream() if use_stream else torch.cuda.current_stream()
        with torch.cuda.stream(st):
            for d in (1e-4, 1e-4, 3e-4):
                info = ctx.hfcr_resolve(A, B, d, 3)
        torch.cuda.synchronize()
        results.append((positions(A), positions(B), info.pairs_first, info.cg_iters))
    for r in results[1:]:
        assert np.array_equal(r[0], results[0][0]) and np.array_equal(r[1], results[0][1])
        assert r[2:] == results[0][2:]


def test_autotuned_variants_give_identical_pairs(api):
    """Every traversal variant (per-edge walks, per-warp packet walks, the
    persistent walks fed by a work queue) finds the same exact pair set,
    and the autotuner picks one of them."""
    sc = meshgen.scene_c2()
    A, PA = dev_mesh(api, sc.A.V, sc.A.T, False, np.float32)
    B, PB = dev_mesh(api, sc.B.V, sc.B.T, True, np.float32)
    ref = oracle.detect(PA, sc.A.T, False, PB, sc.B.T, True)
    nvar = api.N_TRAVERSE_VARIANTS
    for v in range(nvar):
        ctx = make_ctx(api, sc.A.n_verts, sc.A.n_tris, traverse_variant=v)
        _, n, got, st = detect(ctx, A, B)
        assert np.array_equal(got, ref.rec), v
        # the same narrow-phase tests as the per-edge walk
        if v == 0:
            tests0 = st.narrow_tests
        elif v not in (3, 4):   # the packet walks test the same leaves too
            assert st.narrow_tests == tests0, v
        ctx.close()
    ctx = make_ctx(api, sc.A.n_verts, sc.A.n_tris)
    chosen, ms = ctx.hfcr_autotune(A, B)
    assert 0 <= chosen < nvar and len(ms) == nvar and all(t > 0 for t in ms)
    _, n, got, _ = detect(ctx, A, B)
    assert np.array_equal(got, ref.rec)
    with pytest.raises(api.HfcrError):
        api.Context(traverse_variant=nvar)


def test_kinematic_body_respond(api):
    """Inverse mass 0 for half of the oriented body's vertices (Sec. 4: M^-1
    in Eq. 7; kinematic vertices): the displacement against the oracle's,
    the kinematic vertices' exactly zero, and the response's amplification
    (largest |dx| over largest |D - d|) as the oracle's.  (With the whole
    body kinematic this scene's Eq. 7 is singular and inconsistent: an x0
    with five stencils on immovable faces is over-determined, and Eq. 3 has
    no exact solution.)"""
    sc = meshgen.scene_random_small(23, "cloth_sphere")
    nA, nB = sc.A.n_verts, sc.B.n_verts
    wB = (np.random.default_rng(23).random(nB) >= 0.5).astype(np.float64)
    w = np.r_[np.ones(nA), wB]
    A, PA = dev_mesh(api, sc.A.V, sc.A.T, False, np.float32)
    B, PB = dev_mesh(api, sc.B.V, sc.B.T, True, np.float32, inv_mass=wB)
    ctx = make_ctx(api, max(nA, nB), max(sc.A.n_tris, sc.B.n_tris))
    out, n, got, _ = detect(ctx, A, B)
    ref = oracle.detect(PA, sc.A.T, False, PB, sc.B.T, True)
    assert np.array_equal(got, ref.rec)
    st_t, k, st = stencils(ctx, A, B, out, n)
    g, info = respond(ctx, A, B, st_t, k, 1e-4, nA, nB, np.float32)
    rA, rB, asm, _ = oracle.respond(st, PA, sc.A.T, PB, sc.B.T, 1e-4, w)
    r = np.concatenate([rA, rB])
    assert info.converged and rel_err(g, r) <= TOL_DX
    fixed = nA + np.nonzero(wB == 0)[0]
    assert np.all(g[fixed] == 0) and np.all(r[fixed] == 0)
    assert np.any(np.abs(r[nA:]).max(axis=1) > 0)      # the other half moved
    assert abs(info.max_rhs - np.abs(asm.b).max()) <= 1e-12 * np.abs(asm.b).max()
    amp_ref = np.abs(r).max() / np.abs(asm.b).max()
    assert abs(info.max_dx / info.max_rhs - amp_ref) <= 1e-5 * amp_ref


def _stacked_faces(s=5e-5):
    # two nearly parallel kinematic faces 0.02 apart (the second tilted by
    # about s), both crossed by the edges of one vertex x0 below them: the
    # planes offset by d meet about 0.02 / s away, so Eq. 7 moves x0 there
    VB = np.array([[-1, -1, 0], [1, -1, 0], [0, 1, 0], [-1, -1, 0.02], [1, -1, 0.02],
                   [0, 1, 0.02 + 2 * s]], float)
    TB = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    VA = np.array([[0, 0, -0.1], [0, 0.1, 0.2], [0.3, 0, 0.2]], float)
    TA = np.array([[0, 1, 2]], np.int32)
    return VA, TA, VB, TB


@pytest.mark.parametrize("solver", [1, 0], ids=["fp64", "mixed"])
def test_ill_conditioned_response_is_reported(api, solver):
    # condition number ~1e9 with kinematic faces: the float64 per-zone
    # solver meets the 1e-6 bar on x' (its residual cannot reach 1e-12: in
    # float64, b - A lambda itself is only good to ~1e-9 relative with
    # |lambda| ~ 1e6); the mixed solver's float32 normals cannot
    # tell the two planes apart (1 - n1.n2 ~ 1e-9 is below float32's
    # epsilon), so it must either meet the bar or report non-convergence
    VA, TA, VB, TB = _stacked_faces()
    d = 1e-4
    for kinematic in (True, False):
        wB = np.zeros(len(VB)) if kinematic else None
        A, PA = dev_mesh(api, VA, TA, False, np.float64)
        B, PB = dev_mesh(api, VB, TB, True, np.float64, inv_mass=wB)
        ctx = make_ctx(api, 8, 8, solver=solver)
        out, n, got, _ = detect(ctx, A, B)
        st_t, k, st = stencils(ctx, A, B, out, n)
        assert k == 2
        g, info = respond(ctx, A, B, st_t, k, d, len(VA), len(VB), np.float64)
        w = None if wB is None else np.r_[np.ones(len(VA)), wB]
        rA, rB, asm, _ = oracle.respond(st, PA, TA, PB, TB, d, w)
        r = np.concatenate([rA, rB])
        amp_ref = np.abs(r).max() / np.abs(asm.b).max()
        if solver == 1 or info.converged:
            # float64: b - A lambda cancels to ~cond(A) eps |b| (~1e-7 here,
            # above the 1e-12 target), while x' meets the 1e-6 bar
            assert info.rel_residual <= 1e-6 and rel_err(g, r) <= TOL_DX
            amp = info.max_dx / info.max_rhs
            assert abs(amp - amp_ref) <= 1e-5 * amp_ref
        if kinematic:
            assert amp_ref > 1000    # x0 flung about 400 units for penetrations of 0.1
        else:
            assert amp_ref < 10      # unit masses: the faces absorb a share of the motion
        if solver == 1:
            for limit, flagged in ((1000.0, kinematic), (1e9, False)):
                A2, _ = dev_mesh(api, VA, TA, False, np.float64)
                B2, _ = dev_mesh(api, VB, TB, True, np.float64, inv_mass=wB)
                ctx2 = make_ctx(api, 8, 8, solver=solver, amplification_limit=limit)
                inf = ctx2.hfcr_resolve(A2, B2, d, 1)
                assert inf.amplified_iters == int(flagged)
                assert abs(inf.worst_amplification - amp_ref) <= 1e-5 * amp_ref
