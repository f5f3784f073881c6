"""Helpers of the GPU tests: scenes onto the device through the C ABI
binding, results back to numpy."""
import numpy as np

import oracle


def torch_dev():
    import torch
    return torch.device("cuda:0")


def dev_mesh(api, V, T, oriented, dtype, edges=False, inv_mass=None):
    """(api.Mesh, float64 copy of the stored positions)."""
    import torch
    dev = torch_dev()
    P = np.ascontiguousarray(np.asarray(V, np.float64).astype(dtype))
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    xyz = [torch.tensor(np.ascontiguousarray(P[:, c]), dtype=tdt, device=dev) for c in range(3)]
    tris = torch.tensor(np.ascontiguousarray(T, dtype=np.int32), device=dev)
    e = torch.tensor(oracle.edges(T), device=dev) if edges else None
    w = None if inv_mass is None else torch.tensor(np.asarray(inv_mass, np.float32), device=dev)
    return api.Mesh(*xyz, tris, oriented, edges=e, inv_mass=w), P.astype(np.float64)


def positions(m):
    return np.stack([t.detach().cpu().numpy() for t in (m.x, m.y, m.z)], 1).astype(np.float64)


def detect(ctx, A, B, cap=1 << 16):
    import torch
    out = torch.zeros((cap, 4), dtype=torch.int32, device=torch_dev())
    n, st = ctx.hfcr_detect(A, B, out, stats=True)
    return out, n, out[:n].cpu().numpy().astype(np.uint32), st


def stencils(ctx, A, B, pairs, n, cap=1 << 16):
    import torch
    out = torch.zeros((cap, 4), dtype=torch.int32, device=torch_dev())
    k = ctx.hfcr_build_stencils(A, B, pairs, n, out)
    return out, k, out[:k, :3].cpu().numpy().astype(np.uint32)


def respond(ctx, A, B, st, k, d, nA, nB, dtype):
    import torch
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    dxA = [torch.zeros(nA, dtype=tdt, device=torch_dev()) for _ in range(3)]
    dxB = [torch.zeros(nB, dtype=tdt, device=torch_dev()) for _ in range(3)]
    info = ctx.hfcr_respond(A, B, st, k, d, dxA, dxB)
    g = np.concatenate([torch.stack(dxA, 1).cpu().numpy(), torch.stack(dxB, 1).cpu().numpy()])
    return g.astype(np.float64), info


def rel_err(g, r):
    s = np.abs(r).max()
    return float(np.abs(g - r).max() / s) if s > 0 else float(np.abs(g).max())
