"""The frame sequence (cloth falling onto an oriented body, one repair loop
per frame) at reduced size: every frame's detection is compared bit for bit
with the oracle's on the GPU's own positions, and every frame whose loop
converged leaves no edge-face intersection (Sec. 3: repeat until no E-F
intersection remains)."""
import numpy as np
import pytest

import meshgen
import oracle
from gpu_util import dev_mesh, detect, positions

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_2081_gb300 import api as a
    a.lib()
    return a


def test_frame_sequence_reduced(api):
    import torch
    sc = meshgen.scene_c5(n=96, body_level=4)
    mot = sc.meta["motion"]
    A, _ = dev_mesh(api, sc.A.V, sc.A.T, False, np.float32, edges=True)
    B, _ = dev_mesh(api, sc.B.V, sc.B.T, True, np.float32)
    ctx = api.Context()
    ctx.hfcr_reserve(max(sc.A.n_verts, sc.B.n_verts), max(sc.A.n_tris, sc.B.n_tris), 1 << 17)
    contact = converged_with_contact = 0
    # the first contact is near frame 42; without the diffusion of Sec. 5 the
    # kinematic cloth tangles after a few dozen contact frames
    for f in range(56):
        PA = positions(A)
        PA = (PA + mot.velocity(PA, f)).astype(np.float32)
        for c, t in enumerate((A.x, A.y, A.z)):
            t.copy_(torch.tensor(np.ascontiguousarray(PA[:, c]), device=t.device))
        PA, PB = positions(A), positions(B)
        _, n, got, _ = detect(ctx, A, B, 1 << 17)
        ref = oracle.detect(PA, sc.A.T, False, PB, sc.B.T, True)
        assert np.array_equal(got, ref.rec), f"frame {f}"
        info = ctx.hfcr_resolve(A, B, 1e-4, 8)
        assert info.pairs_first == n
        if n:
            contact += 1
        if info.converged:
            left = oracle.detect(positions(A), sc.A.T, False, positions(B), sc.B.T, True)
            assert len(left) == 0, f"frame {f}"
            converged_with_contact += n > 0
    assert contact >= 8 and converged_with_contact >= 4
