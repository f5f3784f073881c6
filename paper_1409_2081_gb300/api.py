"""ctypes binding of libhfcr (include/hfcr.h), argument marshalling only.

Every computation runs in the CUDA library; this module converts torch CUDA
tensors into the C structs and pointers the ABI takes.  Loading fails
loudly when the library is missing or no CUDA device is present: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhfcr.so")

HFCR_OK = 0
HFCR_ERR_ARG = 1
HFCR_ERR_CAPACITY = 2
HFCR_ERR_CUDA = 3
HFCR_ERR_NONFINITE = 4
HFCR_ERR_TIMEOUT = 5
HFCR_ERR_NOT_CONVERGED = 6
HFCR_ERR_UNSUPPORTED = 7
HFCR_ERR_RANGE = 8

HFCR_F32 = 0
HFCR_F64 = 1
HFCR_SOLVER_MIXED = 0
HFCR_SOLVER_FP64 = 1
HFCR_SOLVER_FP64_GLOBAL = 2
N_TRAVERSE_VARIANTS = 9
HFCR_ROLES_ALTERNATE = 0
HFCR_ROLES_BOTH = 1


class hfcr_mesh(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("n_verts", ctypes.c_int32),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("n_tris", ctypes.c_int32), ("tris", ctypes.c_void_p),
                ("n_edges", ctypes.c_int32), ("edges", ctypes.c_void_p),
                ("oriented", ctypes.c_int32), ("inv_mass", ctypes.c_void_p)]


class hfcr_pair(ctypes.Structure):
    _fields_ = [("dir", ctypes.c_uint32), ("v0", ctypes.c_uint32), ("v1", ctypes.c_uint32),
                ("face", ctypes.c_uint32)]


class hfcr_stencil(ctypes.Structure):
    _fields_ = [("dir", ctypes.c_uint32), ("x0", ctypes.c_uint32), ("face", ctypes.c_uint32),
                ("pad", ctypes.c_uint32)]


class hfcr_options(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int32), ("f32_filter", ctypes.c_int32),
                ("roles", ctypes.c_int32), ("max_cg_iters", ctypes.c_int32),
                ("max_refine", ctypes.c_int32), ("rel_tol", ctypes.c_double),
                ("inner_tol", ctypes.c_double), ("graphs", ctypes.c_int32),
                ("diffuse_rings", ctypes.c_int32), ("diffuse_sweeps", ctypes.c_int32),
                ("traverse_variant", ctypes.c_int32), ("setup_path", ctypes.c_int32),
                ("diffuse_max_iters", ctypes.c_int32), ("diffuse_tol", ctypes.c_double),
                ("amplification_limit", ctypes.c_double), ("bvh_rebuild_interval", ctypes.c_int32),
                ("block_switch_iters", ctypes.c_int32)]


class hfcr_solve_info(ctypes.Structure):
    _fields_ = [("cg_iters", ctypes.c_int32), ("refine_rounds", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("converged", ctypes.c_int32),
                ("n_stencils", ctypes.c_int32), ("n_touched", ctypes.c_int32),
                ("max_rhs", ctypes.c_double), ("max_dx", ctypes.c_double)]


class hfcr_detect_stats(ctypes.Structure):
    _fields_ = [("narrow_tests", ctypes.c_int64), ("f64_fallbacks", ctypes.c_int64),
                ("exact_fallbacks", ctypes.c_int64), ("brute_force_equiv", ctypes.c_int64)]


class hfcr_resolve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("pairs_first", ctypes.c_int64), ("pairs_last", ctypes.c_int64),
                ("total_pairs", ctypes.c_int64), ("total_stencils", ctypes.c_int64),
                ("cg_iters", ctypes.c_int32), ("worst_rel_residual", ctypes.c_double),
                ("stats", hfcr_detect_stats), ("solver_path", ctypes.c_int32),
                ("diffuse_cg_iters", ctypes.c_int32), ("diffuse_unconverged", ctypes.c_int32),
                ("worst_amplification", ctypes.c_double), ("amplified_iters", ctypes.c_int32),
                ("band_vertices", ctypes.c_int64), ("big_zone_rows", ctypes.c_int64),
                ("big_zone_vertices", ctypes.c_int64)]


HFCR_N_STAGES = 10
STAGES = ("validate", "bvh", "traverse", "stencils", "assemble", "solve", "displace", "diffuse",
          "band_cg", "zone_big")


class hfcr_profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * HFCR_N_STAGES), ("intervals", ctypes.c_int64 * HFCR_N_STAGES)]


_lib = None

_SIGS = {
    "hfcr_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(hfcr_options)], ctypes.c_int),
    "hfcr_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "hfcr_reserve": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64], ctypes.c_int),
    "hfcr_build_edges": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                          ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                          ctypes.c_void_p], ctypes.c_int),
    "hfcr_build_edges_noalloc": ([ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                  ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p],
                                 ctypes.c_int),
    "hfcr_detect": ([ctypes.c_void_p, ctypes.POINTER(hfcr_mesh), ctypes.POINTER(hfcr_mesh),
                     ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                     ctypes.POINTER(hfcr_detect_stats), ctypes.c_void_p], ctypes.c_int),
    "hfcr_detect_batch": ([ctypes.c_void_p, ctypes.POINTER(hfcr_mesh), ctypes.POINTER(hfcr_mesh),
                           ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                           ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(hfcr_detect_stats),
                           ctypes.c_void_p], ctypes.c_int),
    "hfcr_resolve_batch": ([ctypes.c_void_p, ctypes.POINTER(hfcr_mesh), ctypes.POINTER(hfcr_mesh),
                            ctypes.c_int32, ctypes.c_void_p, ctypes.c_double, ctypes.c_int32,
                            ctypes.POINTER(hfcr_resolve_info), ctypes.c_void_p], ctypes.c_int),
    "hfcr_build_stencils": ([ctypes.c_void_p, ctypes.POINTER(hfcr_mesh), ctypes.POINTER(hfcr_mesh),
                             ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                             ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p], ctypes.c_int),
    "hfcr_respond": ([ctypes.c_void_p, ctypes.POINTER(hfcr_mesh), ctypes.POINTER(hfcr_mesh),
                      ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                      ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                      ctypes.POINTER(hfcr_solve_info), ctypes.c_void_p], ctypes.c_int),
    "hfcr_diffuse": ([ctypes.c_void_p, ctypes.POINTER(hfcr_mesh), ctypes.c_void_p, ctypes.c_void_p,
                      ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p], ctypes.c_int),
    "hfcr_resolve": ([ctypes.c_void_p, ctypes.POINTER(hfcr_mesh), ctypes.POINTER(hfcr_mesh),
                      ctypes.c_double, ctypes.c_int32, ctypes.POINTER(hfcr_resolve_info),
                      ctypes.c_void_p], ctypes.c_int),
    "hfcr_autotune": ([ctypes.c_void_p, ctypes.POINTER(hfcr_mesh), ctypes.POINTER(hfcr_mesh),
                       ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                       ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_void_p], ctypes.c_int),
    "hfcr_profile_enable": ([ctypes.c_void_p, ctypes.c_int32], ctypes.c_int),
    "hfcr_profile_read": ([ctypes.c_void_p, ctypes.POINTER(hfcr_profile)], ctypes.c_int),
    "hfcr_launch_count": ([], ctypes.c_int64),
    "hfcr_last_error": ([ctypes.c_void_p], ctypes.c_char_p),
    "hfcr_status_string": ([ctypes.c_int], ctypes.c_char_p),
}

EXPORTS = tuple(_SIGS)


def lib():
    """Load libhfcr.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_1409_2081_gb300.build.build() (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


class HfcrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


def hfcr_launch_count() -> int:
    return int(lib().hfcr_launch_count())


def hfcr_build_edges_noalloc(tris, n_verts: int, out, stream=None) -> int:
    """hfcr_build_edges without a context or any device allocation (fixed
    scratch inside the library, n_tris <= 65,536; out must hold 3 * n_tris
    edges)."""
    n = ctypes.c_int64()
    st = lib().hfcr_build_edges_noalloc(_ptr(tris), int(tris.shape[0]), n_verts, _ptr(out),
                                        int(out.shape[0]), ctypes.byref(n), _stream_ptr(stream))
    if st != HFCR_OK:
        raise HfcrError(st, (lib().hfcr_last_error(None) or b"").decode())
    return int(n.value)


def status_string(s: int) -> str:
    return lib().hfcr_status_string(int(s)).decode()


def _stream_ptr(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) or None


def _ptr(t) -> Optional[int]:
    return None if t is None else int(t.data_ptr())


class Context:
    """Owns an hfcr_ctx (device scratch reserved up front)."""

    def __init__(self, solver: int = HFCR_SOLVER_MIXED, f32_filter: bool = True,
                 roles: int = HFCR_ROLES_ALTERNATE, max_cg_iters: int = 500, max_refine: int = 6,
                 rel_tol: float = 1e-12, inner_tol: float = 1e-4, graphs: bool = True,
                 diffuse_rings: int = 0, diffuse_sweeps: int = 0, traverse_variant: int = 0,
                 setup_path: int = 0, diffuse_max_iters: int = 1000, diffuse_tol: float = 1e-10,
                 amplification_limit: float = 1000.0, bvh_rebuild_interval: int = 8,
                 block_switch_iters: int = 48):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("hfcr needs a CUDA device")
        opt = hfcr_options(solver, int(f32_filter), roles, max_cg_iters, max_refine, rel_tol, inner_tol,
                           int(graphs), diffuse_rings, diffuse_sweeps, traverse_variant, setup_path,
                           diffuse_max_iters, diffuse_tol, amplification_limit, bvh_rebuild_interval,
                           block_switch_iters)
        h = ctypes.c_void_p()
        self.handle = None
        # a refused create has no context: its message is the thread's
        # context-free one (hfcr_last_error(NULL))
        self._check(lib().hfcr_create(ctypes.byref(h), ctypes.byref(opt)))
        self.handle = h

    def _check(self, status: int, h=None, allow=()):
        if status != HFCR_OK and status not in allow:
            msg = lib().hfcr_last_error(h if h is not None else self.handle) or b""
            raise HfcrError(status, msg.decode())
        return status

    def close(self):
        if getattr(self, "handle", None):
            lib().hfcr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def hfcr_autotune(self, A: "Mesh", B: "Mesh", segs=None, stream=None):
        """Times the traversal variants on this scene (a batch when segs is
        given) and keeps the fastest; returns (chosen index, [ms per variant])."""
        chosen = ctypes.c_int32()
        ms = (ctypes.c_double * N_TRAVERSE_VARIANTS)()
        n_pairs = 0 if segs is None else int(segs.shape[0]) - 1
        self._check(lib().hfcr_autotune(self.handle, ctypes.byref(A.c), ctypes.byref(B.c), n_pairs,
                                        _ptr(segs), ctypes.byref(chosen), ms, N_TRAVERSE_VARIANTS,
                                        _stream_ptr(stream)))
        return int(chosen.value), [round(ms[i], 5) for i in range(N_TRAVERSE_VARIANTS)]

    def hfcr_profile_enable(self, on: bool = True):
        self._check(lib().hfcr_profile_enable(self.handle, int(on)))

    def hfcr_profile_read(self) -> dict:
        p = hfcr_profile()
        self._check(lib().hfcr_profile_read(self.handle, ctypes.byref(p)))
        return {n: (p.ms[i], int(p.intervals[i])) for i, n in enumerate(STAGES)}

    def hfcr_reserve(self, max_verts: int, max_tris: int, max_pairs: int):
        self._check(lib().hfcr_reserve(self.handle, max_verts, max_tris, max_pairs))

    def hfcr_build_edges(self, tris, n_verts: int, out, stream=None) -> int:
        n = ctypes.c_int64()
        self._check(lib().hfcr_build_edges(self.handle, _ptr(tris), int(tris.shape[0]), n_verts,
                                           _ptr(out), int(out.shape[0]), ctypes.byref(n),
                                           _stream_ptr(stream)))
        return int(n.value)

    def hfcr_detect(self, A: "Mesh", B: "Mesh", out, stream=None, stats: bool = False):
        n = ctypes.c_int64()
        st = hfcr_detect_stats()
        self._check(lib().hfcr_detect(self.handle, ctypes.byref(A.c), ctypes.byref(B.c), _ptr(out),
                                      int(out.shape[0]), ctypes.byref(n), ctypes.byref(st),
                                      _stream_ptr(stream)))
        return (int(n.value), st) if stats else int(n.value)

    def hfcr_detect_batch(self, A: "Mesh", B: "Mesh", segs, out, stream=None, stats: bool = False):
        """segs: int32 CUDA tensor [n_pairs + 1, 4] (see include/hfcr.h)."""
        n = ctypes.c_int64()
        st = hfcr_detect_stats()
        self._check(lib().hfcr_detect_batch(self.handle, ctypes.byref(A.c), ctypes.byref(B.c),
                                            int(segs.shape[0]) - 1, _ptr(segs), _ptr(out),
                                            int(out.shape[0]), ctypes.byref(n), ctypes.byref(st),
                                            _stream_ptr(stream)))
        return (int(n.value), st) if stats else int(n.value)

    def hfcr_resolve_batch(self, A: "Mesh", B: "Mesh", segs, d: float, max_iters: int, stream=None,
                           raise_not_converged: bool = False):
        info = hfcr_resolve_info()
        allow = () if raise_not_converged else (HFCR_ERR_NOT_CONVERGED,)
        self._check(lib().hfcr_resolve_batch(self.handle, ctypes.byref(A.c), ctypes.byref(B.c),
                                             int(segs.shape[0]) - 1, _ptr(segs), d, max_iters,
                                             ctypes.byref(info), _stream_ptr(stream)), allow=allow)
        return info

    def hfcr_build_stencils(self, A: "Mesh", B: "Mesh", pairs, n_pairs: int, out, stream=None) -> int:
        n = ctypes.c_int64()
        self._check(lib().hfcr_build_stencils(self.handle, ctypes.byref(A.c), ctypes.byref(B.c),
                                              _ptr(pairs), n_pairs, _ptr(out), int(out.shape[0]),
                                              ctypes.byref(n), _stream_ptr(stream)))
        return int(n.value)

    def hfcr_respond(self, A: "Mesh", B: "Mesh", stencils, k: int, d: float,
                     dxA: Sequence, dxB: Sequence, stream=None, info: bool = True):
        pa = (ctypes.c_void_p * 3)(*[_ptr(t) for t in dxA])
        pb = (ctypes.c_void_p * 3)(*[_ptr(t) for t in dxB])
        si = hfcr_solve_info()
        self._check(lib().hfcr_respond(self.handle, ctypes.byref(A.c), ctypes.byref(B.c),
                                       _ptr(stencils), k, d, pa, pb,
                                       ctypes.byref(si) if info else None, _stream_ptr(stream)))
        return si

    def hfcr_diffuse(self, M: "Mesh", dx, rings: int, sweeps: int = 0, stream=None):
        """dx: three float64 CUDA tensors [n] (x, y, z), overwritten; sweeps
        0: the harmonic field, > 0: that many Jacobi sweeps."""
        self._check(lib().hfcr_diffuse(self.handle, ctypes.byref(M.c), _ptr(dx[0]), _ptr(dx[1]),
                                       _ptr(dx[2]), rings, sweeps, _stream_ptr(stream)))

    def hfcr_resolve(self, A: "Mesh", B: "Mesh", d: float, max_iters: int, stream=None,
                     raise_not_converged: bool = False):
        info = hfcr_resolve_info()
        allow = () if raise_not_converged else (HFCR_ERR_NOT_CONVERGED,)
        self._check(lib().hfcr_resolve(self.handle, ctypes.byref(A.c), ctypes.byref(B.c), d,
                                       max_iters, ctypes.byref(info), _stream_ptr(stream)),
                    allow=allow)
        return info


class Mesh:
    """A mesh view over torch CUDA tensors: x, y, z (float32 or float64,
    [n]), tris int32 [m, 3], optional edges int32 [E, 2] and inverse masses
    float32 [n].  Keeps the tensors alive while the C struct points at
    them."""

    def __init__(self, x, y, z, tris, oriented: bool, edges=None, inv_mass=None):
        import torch
        for t in (x, y, z, tris):
            if not t.is_cuda or not t.is_contiguous():
                raise ValueError("mesh tensors must be contiguous CUDA tensors")
        if x.dtype not in (torch.float32, torch.float64) or y.dtype != x.dtype or z.dtype != x.dtype:
            raise ValueError("positions must share dtype float32 or float64")
        if tris.dtype != torch.int32:
            raise ValueError("tris must be int32")
        self.x, self.y, self.z, self.tris, self.edges, self.inv_mass = x, y, z, tris, edges, inv_mass
        self.c = hfcr_mesh(HFCR_F32 if x.dtype == torch.float32 else HFCR_F64, int(x.shape[0]),
                           _ptr(x), _ptr(y), _ptr(z), int(tris.shape[0]), _ptr(tris),
                           int(edges.shape[0]) if edges is not None else 0, _ptr(edges),
                           int(bool(oriented)), _ptr(inv_mass))
