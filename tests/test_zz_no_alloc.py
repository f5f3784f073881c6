"""The allocation-free edge extraction (hfcr_build_edges_noalloc), called
through the C ABI, against the context-based hfcr_build_edges on the same
triangles, two calls in a row (the fixed scratch is reused between calls).

Some callers may not allocate device memory while they run (their memory
belongs to their own pool or budget, or they cannot pay for cudaMalloc's
synchronisation); this entry point serves them with scratch that lives in
the library itself.
"""
import numpy as np
import pytest

import meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_2081_gb300 import api as a
    a.lib()
    return a


def _edges_with_context(api, T, nv):
    import torch
    ctx = api.Context()
    ctx.hfcr_reserve(nv, len(T), 16)
    tris = torch.tensor(T, device="cuda:0")
    out = torch.zeros((3 * len(T), 2), dtype=torch.int32, device="cuda:0")
    n = ctx.hfcr_build_edges(tris, nv, out)
    ctx.close()
    return out[:n].cpu().numpy()


def test_noalloc_edges_match_the_context_entry_point(api):
    import torch
    meshes = [meshgen.torus(128, 64, 1.0, 0.3),    # 16,384 faces: the multi-CTA sort path
              meshgen.icosphere(3, 1.0),           # 1,280 faces: the single-CTA sort path
              meshgen.torus(256, 128, 1.0, 0.3)]   # 65,536 faces: exactly the scratch limit
    for V, T in meshes + meshes[:1]:              # calls in a row, then the first again
        nv = len(V)
        tris = torch.tensor(T, device="cuda:0")
        out = torch.full((3 * len(T), 2), -7, dtype=torch.int32, device="cuda:0")
        n = api.hfcr_build_edges_noalloc(tris, nv, out)
        got = out[:n].cpu().numpy()
        ref = _edges_with_context(api, T, nv)
        assert n == len(ref) and np.array_equal(got, ref)


def test_noalloc_rejects_sizes_beyond_its_scratch(api):
    import torch
    tris = torch.zeros((65537, 3), dtype=torch.int32, device="cuda:0")
    out = torch.zeros((3 * 65537, 2), dtype=torch.int32, device="cuda:0")
    with pytest.raises(api.HfcrError) as e:
        api.hfcr_build_edges_noalloc(tris, 3, out)
    assert e.value.status == api.HFCR_ERR_CAPACITY and "65536" in str(e.value)
    small = torch.zeros((2, 2), dtype=torch.int32, device="cuda:0")
    with pytest.raises(api.HfcrError) as e:
        api.hfcr_build_edges_noalloc(tris[:10], 3, small)
    assert e.value.status == api.HFCR_ERR_CAPACITY


def test_noalloc_allocates_nothing_and_checks_indices(api):
    import torch
    V, T = meshgen.torus(64, 32, 1.0, 0.3)
    tris = torch.tensor(T, device="cuda:0")
    out = torch.zeros((3 * len(T), 2), dtype=torch.int32, device="cuda:0")
    api.hfcr_build_edges_noalloc(tris, len(V), out)          # warm: the device address is looked up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    n = api.hfcr_build_edges_noalloc(tris, len(V), out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert n == 3 * 64 * 32 and free1 == free0
    # a vertex index beyond n_verts is an argument error, not a fault
    bad = tris.clone()
    bad[5, 1] = len(V)
    with pytest.raises(api.HfcrError) as e:
        api.hfcr_build_edges_noalloc(bad, len(V), out)
    assert e.value.status == api.HFCR_ERR_ARG
    # and the next call is served normally
    assert api.hfcr_build_edges_noalloc(tris, len(V), out) == n
