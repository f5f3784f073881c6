"""Seeded synthetic triangle meshes for the collision-response workloads.

This module only builds inputs: vertex positions and triangle lists of
closed (outward, counter-clockwise) or open surfaces, rigid transforms and
the scene layouts of the five benchmark workloads.  It contains none of the
collision method's arithmetic (no orientation predicates, no intersection
tests, no constraint assembly, no solves); both the CPU oracle and the CUDA
path read the arrays produced here.

The paper's own scenes (a spike through an 18,896-vertex sheet, two
576-vertex tori, a dressed dummy; Sec. 6) are not available, so every
workload is a seeded stand-in with the sizes and structure the paper's
scenes have: an oriented closed body (sphere, torus, star-shaped blob)
against a cloth grid or a second closed body.

Every generator is deterministic given its seed (numpy PCG64).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

BASE_SEED = 14092081


@dataclass
class Mesh:
    """A triangle mesh: V float64 [n,3], T int32 [m,3] (counter-clockwise
    seen from the front side), and whether the mesh is oriented (its faces
    have a front and a back side, Sec. 1 and Sec. 4 of the paper)."""
    V: np.ndarray
    T: np.ndarray
    oriented: bool
    name: str = ""

    @property
    def n_verts(self) -> int:
        return int(self.V.shape[0])

    @property
    def n_tris(self) -> int:
        return int(self.T.shape[0])

    def copy(self) -> "Mesh":
        return Mesh(self.V.copy(), self.T.copy(), self.oriented, self.name)


# ----------------------------------------------------------------------------
# primitive surfaces
# ----------------------------------------------------------------------------

def icosahedron() -> Tuple[np.ndarray, np.ndarray]:
    """Regular icosahedron on the unit sphere, faces counter-clockwise seen
    from outside."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    V = np.array([
        [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
        [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
        [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
    ], dtype=np.float64)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    T = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ], dtype=np.int32)
    return V, T


def icosphere(level: int, radius: float = 1.0) -> Tuple[np.ndarray, np.ndarray]:
    """Icosahedron subdivided `level` times (each triangle into four) and
    projected onto the sphere: V = 10*4^L + 2, F = 20*4^L, E = 30*4^L."""
    V, T = icosahedron()
    for _ in range(level):
        nv = V.shape[0]
        a, b, c = T[:, 0].astype(np.int64), T[:, 1].astype(np.int64), T[:, 2].astype(np.int64)
        # one midpoint per undirected edge, numbered after the old vertices
        e = np.stack([np.stack([a, b], 1), np.stack([b, c], 1), np.stack([c, a], 1)], 0)
        lo, hi = np.minimum(e[..., 0], e[..., 1]), np.maximum(e[..., 0], e[..., 1])
        key = lo * nv + hi
        uk, inv = np.unique(key.ravel(), return_inverse=True)
        mid_lo, mid_hi = uk // nv, uk % nv
        M = 0.5 * (V[mid_lo] + V[mid_hi])
        M /= np.linalg.norm(M, axis=1, keepdims=True)
        inv = inv.reshape(3, -1) + nv
        ab, bc, ca = inv[0], inv[1], inv[2]
        T = np.concatenate([
            np.stack([a, ab, ca], 1), np.stack([b, bc, ab], 1),
            np.stack([c, ca, bc], 1), np.stack([ab, bc, ca], 1)], 0).astype(np.int32)
        V = np.concatenate([V, M], 0)
    return V * radius, T


def torus(nu: int, nv: int, R: float, r: float) -> Tuple[np.ndarray, np.ndarray]:
    """Torus around the z axis (core radius R, tube radius r), nu segments
    around the axis and nv around the tube: V = nu*nv, F = 2*nu*nv,
    E = 3*nu*nv.  Faces counter-clockwise seen from outside."""
    i = np.arange(nu)[:, None]
    j = np.arange(nv)[None, :]
    u = 2.0 * np.pi * i / nu
    v = 2.0 * np.pi * j / nv
    rho = R + r * np.cos(v)
    X = np.broadcast_to(rho * np.cos(u), (nu, nv))
    Y = np.broadcast_to(rho * np.sin(u), (nu, nv))
    Z = np.broadcast_to(r * np.sin(v), (nu, nv))
    V = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1).astype(np.float64)
    ii, jj = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    v00 = ii * nv + jj
    v10 = ((ii + 1) % nu) * nv + jj
    v11 = ((ii + 1) % nu) * nv + (jj + 1) % nv
    v01 = ii * nv + (jj + 1) % nv
    T = np.concatenate([
        np.stack([v00.ravel(), v10.ravel(), v11.ravel()], 1),
        np.stack([v00.ravel(), v11.ravel(), v01.ravel()], 1)], 0).astype(np.int32)
    return V, T


def cloth(n: int, side: float) -> Tuple[np.ndarray, np.ndarray]:
    """n x n regular grid in the z=0 plane centred on the z axis, vertex
    (i, j) = i*n + j, split along the diagonal (i,j)-(i+1,j+1):
    V = n^2, F = 2(n-1)^2, E = 2n(n-1) + (n-1)^2."""
    s = np.linspace(-side / 2.0, side / 2.0, n)
    Y, X = np.meshgrid(s, s, indexing="ij")
    V = np.stack([X.ravel(), Y.ravel(), np.zeros(n * n)], 1)
    ii, jj = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="ij")
    v00 = (ii * n + jj).ravel()
    v01 = v00 + 1
    v10 = v00 + n
    v11 = v00 + n + 1
    T = np.concatenate([np.stack([v00, v01, v11], 1),
                        np.stack([v00, v11, v10], 1)], 0).astype(np.int32)
    return V, T


def signed_volume(V: np.ndarray, T: np.ndarray) -> float:
    """Enclosed volume of a closed mesh (positive when faces wind
    counter-clockwise seen from outside); used only to validate generators."""
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    return float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0)


def undirected_edge_count(T: np.ndarray) -> int:
    """Number of distinct undirected edges of a triangle list (generator
    validation only)."""
    e = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]], 0).astype(np.int64)
    lo, hi = e.min(1), e.max(1)
    return int(np.unique(lo * (int(T.max()) + 1) + hi).size)


# ----------------------------------------------------------------------------
# transforms and fields
# ----------------------------------------------------------------------------

def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform rotation in SO(3) from a normalised Gaussian quaternion."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def random_unit(rng: np.random.Generator) -> np.ndarray:
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)


def axis_angle(axis: np.ndarray, angle: float) -> np.ndarray:
    """Rotation matrix about a unit axis (Rodrigues)."""
    k = axis / np.linalg.norm(axis)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * (K @ K)


def sinusoid_field_2d(rng: np.random.Generator, n_modes: int = 8):
    """Seeded sum of plane sinusoids s(x, y); returns a callable."""
    ang = rng.uniform(0.0, 2.0 * np.pi, n_modes)
    mag = rng.uniform(8.0, 24.0, n_modes)
    amp = rng.uniform(0.5, 1.0, n_modes)
    ph = rng.uniform(0.0, 2.0 * np.pi, n_modes)
    wx, wy = mag * np.cos(ang), mag * np.sin(ang)

    def s(x, y):
        return (amp[None, :] * np.sin(np.outer(x, wx) + np.outer(y, wy) + ph[None, :])).sum(1)
    return s


def _assoc_legendre(lmax: int, x: np.ndarray) -> dict:
    """P_l^m(x) for 0 <= m <= l <= lmax by the standard three-term
    recurrences (Condon-Shortley phase omitted; only a seeded smooth field
    is needed)."""
    P = {}
    sx = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    P[(0, 0)] = np.ones_like(x)
    for m in range(1, lmax + 1):
        P[(m, m)] = (2 * m - 1) * sx * P[(m - 1, m - 1)]
    for m in range(0, lmax):
        P[(m + 1, m)] = (2 * m + 1) * x * P[(m, m)]
    for m in range(0, lmax + 1):
        for l in range(m + 2, lmax + 1):
            P[(l, m)] = ((2 * l - 1) * x * P[(l - 1, m)] - (l + m - 1) * P[(l - 2, m)]) / (l - m)
    return P


def sh_field(rng: np.random.Generator, lmax: int, dirs: np.ndarray) -> np.ndarray:
    """f = sum_{l=1..lmax} sum_m c_lm Y_lm at unit directions, c_lm ~ N(0,1),
    real orthonormal spherical harmonics."""
    ct = np.clip(dirs[:, 2], -1.0, 1.0)
    phi = np.arctan2(dirs[:, 1], dirs[:, 0])
    P = _assoc_legendre(lmax, ct)
    f = np.zeros(dirs.shape[0])
    for l in range(1, lmax + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            norm = math.sqrt((2 * l + 1) / (4 * math.pi)
                             * math.factorial(l - am) / math.factorial(l + am))
            if m == 0:
                y = norm * P[(l, 0)]
            elif m > 0:
                y = math.sqrt(2.0) * norm * P[(l, am)] * np.cos(am * phi)
            else:
                y = math.sqrt(2.0) * norm * P[(l, am)] * np.sin(am * phi)
            f += rng.standard_normal() * y
    return f


# ----------------------------------------------------------------------------
# scenes
# ----------------------------------------------------------------------------

@dataclass
class Scene:
    """Two meshes A and B, their working precision and the response
    parameters.  `dtype` is the position storage type (float32 / float64)."""
    A: Mesh
    B: Mesh
    dtype: type
    d: float = 1e-4
    name: str = ""
    meta: dict = field(default_factory=dict)

    def positions(self, which: str) -> np.ndarray:
        """Positions cast to the scene's storage type, widened back to
        float64 (the exact values both sides compute on)."""
        m = self.A if which == "A" else self.B
        return m.V.astype(self.dtype).astype(np.float64)


def scene_c1(seed: int = BASE_SEED + 0, level: int = 3, jitter: float = 0.01,
             offset: float = 1.5) -> Scene:
    """Two closed oriented icospheres (level 3: 642 vertices, 1,280
    triangles, radius 1), B offset by +1.5 on x, every vertex jittered
    uniformly in [-0.01, 0.01]^3, float64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    VA, TA = icosphere(level, 1.0)
    VB, TB = icosphere(level, 1.0)
    VA = VA + rng.uniform(-jitter, jitter, VA.shape)
    VB = VB + rng.uniform(-jitter, jitter, VB.shape) + np.array([offset, 0.0, 0.0])
    return Scene(Mesh(VA, TA, True, "sphereA"), Mesh(VB, TB, True, "sphereB"),
                 np.float64, name=f"icosphere L{level} x2, offset {offset}, jitter {jitter}, fp64")


# z0 of the cloth in the cloth-vs-torus scene; fixed once so that the
# initial frame has between 2,000 and 5,000 edge-face intersections.
C2_Z0 = 0.4


def scene_c2(seed: int = BASE_SEED + 1, n: int = 200, side: float = 2.0,
             nu: int = 256, nv: int = 128, R: float = 1.0, r: float = 0.4,
             z0: Optional[float] = None, amp: float = 0.3) -> Scene:
    """Un-oriented cloth grid (200 x 200, side 2.0, centred on the z axis)
    with seeded sinusoidal height noise of amplitude 0.3 around z0, over an
    oriented closed torus (R 1.0, r 0.4, 256 x 128 quads) at the origin;
    float32 positions.  Only cloth edges against torus faces are tested."""
    rng = np.random.Generator(np.random.PCG64(seed))
    VC, TC = cloth(n, side)
    s = sinusoid_field_2d(rng)(VC[:, 0], VC[:, 1])
    s /= np.abs(s).max()
    VC[:, 2] = (C2_Z0 if z0 is None else z0) + amp * s
    VT, TT = torus(nu, nv, R, r)
    return Scene(Mesh(VC, TC, False, "cloth"), Mesh(VT, TT, True, "torus"),
                 np.float32, name=f"cloth {n}x{n} vs torus {nu}x{nv}, fp32")


def scene_c3(seed: int = BASE_SEED + 2, nu: int = 512, nv: int = 256,
             R: float = 1.0, r: float = 0.35) -> Scene:
    """Two oriented tori (512 x 256 quads each, R 1.0, r 0.35), float32.
    A sits at the origin around z.  B touches A locally: a seeded point P1
    on A's core circle and a seeded unit u1 normal to A's core tangent there
    give B's core point P2 = P1 + (2r - delta) u1, delta ~ U(0, 0.2 r); B's
    axis is u1 (its core circle lies in the plane normal to u1 through P2)
    and its rotation about u1 is seeded."""
    rng = np.random.Generator(np.random.PCG64(seed))
    VA, TA = torus(nu, nv, R, r)
    VB, TB = torus(nu, nv, R, r)
    phi1 = rng.uniform(0, 2 * np.pi)
    P1 = R * np.array([math.cos(phi1), math.sin(phi1), 0.0])
    t1 = np.array([-math.sin(phi1), math.cos(phi1), 0.0])
    radial = np.array([math.cos(phi1), math.sin(phi1), 0.0])
    beta = rng.uniform(0, 2 * np.pi)
    u1 = math.cos(beta) * radial + math.sin(beta) * np.array([0.0, 0.0, 1.0])
    delta = rng.uniform(0.0, 0.2 * r)
    P2 = P1 + (2 * r - delta) * u1
    # B's frame: local z -> u1; its radial direction at P2 (n2, normal to
    # u1) is set by a seeded angle about u1; centre = P2 - R n2.
    e1 = t1 - np.dot(t1, u1) * u1
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(u1, e1)
    gamma = rng.uniform(0, 2 * np.pi)
    n2 = math.cos(gamma) * e1 + math.sin(gamma) * e2
    centre = P2 - R * n2
    # rotation taking the torus's own frame (x, y, z) to (n2, u1 x n2, u1),
    # so the generator's vertex at angle u = 0 lands at P2's side.
    Rm = np.stack([n2, np.cross(u1, n2), u1], 1)
    VB = VB @ Rm.T + centre
    return Scene(Mesh(VA, TA, True, "torusA"), Mesh(VB, TB, True, "torusB"),
                 np.float32, name=f"two tori {nu}x{nv}, r {r}, delta {delta:.4f}, fp32",
                 meta={"delta": float(delta), "R": R, "r": r,
                       "frame_B": (Rm, centre)})    # world = local @ Rm.T + centre


def scene_c4(seed: int = BASE_SEED + 3, n_pairs: int = 1024, lmin: int = 1,
             lmax: int = 5, rho_lo: float = 0.5, rho_hi: float = 1.8) -> List[Scene]:
    """Batch of independent pairs of oriented icospheres (radius 1), each
    level uniform in {1..5} (80 to 20,480 triangles per mesh), B under a
    uniform random rotation and offset rho*u, rho ~ U(0.5, 1.8), u uniform
    on the sphere; float32, no jitter."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cache = {}
    out = []
    for p in range(n_pairs):
        la, lb = int(rng.integers(lmin, lmax + 1)), int(rng.integers(lmin, lmax + 1))
        for L in (la, lb):
            if L not in cache:
                cache[L] = icosphere(L, 1.0)
        Rm = random_rotation(rng)
        rho = rng.uniform(rho_lo, rho_hi)
        off = rho * random_unit(rng)
        VA, TA = cache[la]
        VB, TB = cache[lb]
        out.append(Scene(Mesh(VA.copy(), TA, True, f"ico{la}"),
                         Mesh(VB @ Rm.T + off, TB, True, f"ico{lb}"),
                         np.float32, name=f"pair {p}: L{la} vs L{lb}, rho {rho:.3f}"))
    return out


def body_c5(seed: int = BASE_SEED + 4, level: int = 7, amp: float = 0.1,
            lmax: int = 8) -> Mesh:
    """Closed star-shaped oriented body: icosphere (level 7: 163,842
    vertices, 327,680 triangles) with radius 1 + amp * f / max|f|, f a
    seeded real spherical-harmonic series of degrees 1..8."""
    rng = np.random.Generator(np.random.PCG64(seed))
    V, T = icosphere(level, 1.0)
    f = sh_field(rng, lmax, V)
    V = V * (1.0 + amp * f / np.abs(f).max())[:, None]
    return Mesh(V, T, True, "body")


class ClothMotion:
    """Seeded smooth velocity field for the frame sequence: a downward
    drift of v0 per frame plus 8 sinusoidal modes of amplitude 0.5*v0."""

    def __init__(self, seed: int, v0: float = 0.004, n_modes: int = 8):
        rng = np.random.Generator(np.random.PCG64(seed))
        self.v0 = v0
        self.k = rng.standard_normal((n_modes, 3)) * 2.0
        self.w = rng.uniform(0.01, 0.05, n_modes)
        self.ph = rng.uniform(0, 2 * np.pi, n_modes)
        d = rng.standard_normal((n_modes, 3))
        self.dir = d / np.linalg.norm(d, axis=1, keepdims=True)
        a = rng.uniform(0.5, 1.0, n_modes)
        self.amp = a / a.sum()

    def velocity(self, X: np.ndarray, frame: int) -> np.ndarray:
        ang = X @ self.k.T + self.w[None, :] * frame + self.ph[None, :]
        v = (np.sin(ang) * self.amp[None, :]) @ self.dir * (0.5 * self.v0)
        v[:, 2] -= self.v0
        return v

    def device_params(self, torch, dev):
        """The field's parameters as float32 tensors on `dev` (for advance)."""
        f32 = torch.float32
        return (torch.tensor(self.k.T, dtype=f32, device=dev),
                torch.tensor(self.w, dtype=f32, device=dev),
                torch.tensor(self.ph, dtype=f32, device=dev),
                torch.tensor((self.amp[:, None] * self.dir) * (0.5 * self.v0), dtype=f32, device=dev))

    def advance(self, torch, params, x, y, z, frame: int):
        """Moves the cloth by one frame in place: x, y, z are float32 device
        tensors, params from device_params (the same field as velocity,
        evaluated in float32 on the device)."""
        K, W, PH, AD = params
        X = torch.stack([x, y, z], 1)
        V = torch.sin(X @ K + W * frame + PH) @ AD
        V[:, 2] -= self.v0
        X += V
        x.copy_(X[:, 0])
        y.copy_(X[:, 1])
        z.copy_(X[:, 2])


def scene_c5(seed: int = BASE_SEED + 4, n: int = 512, side: float = 3.0,
             z_start: float = 1.15, body_level: int = 7) -> Scene:
    """Frame-sequence scene at frame 0: un-oriented cloth grid (512 x 512,
    side 3.0) at z = 1.15 above the oriented spherical-harmonic body;
    float32.  `meta['motion']` moves the cloth between frames."""
    body = body_c5(seed, body_level)
    VC, TC = cloth(n, side)
    VC[:, 2] = z_start
    return Scene(Mesh(VC, TC, False, "cloth"), body, np.float32,
                 name=f"cloth {n}x{n} over SH body L{body_level}, fp32",
                 meta={"motion": ClothMotion(seed + 1000)})


def scene_random_small(seed: int, kind: str = "spheres") -> Scene:
    """Small ragged scenes for parity tests (sizes not multiples of any
    tile): jittered icospheres of different levels, a torus against a
    sphere, or a cloth patch against a sphere."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "spheres":
        VA, TA = icosphere(2, 1.0)
        VB, TB = icosphere(1, 0.8)
        VA = VA + rng.uniform(-0.02, 0.02, VA.shape)
        VB = (VB + rng.uniform(-0.02, 0.02, VB.shape)) @ random_rotation(rng).T + np.array([1.1, 0.2, -0.1])
        return Scene(Mesh(VA, TA, True), Mesh(VB, TB, True), np.float32, name=f"small spheres {seed}")
    if kind == "torus_sphere":
        VA, TA = torus(37, 23, 1.0, 0.3)
        VB, TB = icosphere(2, 0.5)
        VB = VB @ random_rotation(rng).T + np.array([1.0, 0.0, 0.25]) + rng.uniform(-0.05, 0.05, 3)
        return Scene(Mesh(VA, TA, True), Mesh(VB, TB, True), np.float32, name=f"small torus/sphere {seed}")
    if kind == "cloth_sphere":
        VA, TA = cloth(41, 2.0)
        VA[:, 2] = 0.85 + 0.1 * rng.uniform(-1, 1, VA.shape[0])
        VB, TB = icosphere(3, 1.0)
        return Scene(Mesh(VA, TA, False), Mesh(VB, TB, True), np.float32, name=f"small cloth/sphere {seed}")
    raise ValueError(kind)


def soa(V: np.ndarray, dtype) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Structure-of-arrays copy of positions in the storage type."""
    W = np.ascontiguousarray(V.astype(dtype))
    return (np.ascontiguousarray(W[:, 0]), np.ascontiguousarray(W[:, 1]),
            np.ascontiguousarray(W[:, 2]))


def concat_batch(scenes: List[Scene]):
    """Lays a batch of independent mesh pairs out as two concatenated meshes
    and a segment table: returns (VA, TA, VB, TB, segs) with triangle ids
    global within each concatenation and segs int32 [(n + 1), 4], row i =
    (first vertex of A_i, first face of A_i, first vertex of B_i, first face
    of B_i), last row the totals."""
    VA, TA, VB, TB = [], [], [], []
    segs = np.zeros((len(scenes) + 1, 4), np.int64)
    va = ta = vb = tb = 0
    for i, sc in enumerate(scenes):
        segs[i] = [va, ta, vb, tb]
        VA.append(sc.A.V)
        TA.append(sc.A.T.astype(np.int64) + va)
        VB.append(sc.B.V)
        TB.append(sc.B.T.astype(np.int64) + vb)
        va += sc.A.n_verts
        ta += sc.A.n_tris
        vb += sc.B.n_verts
        tb += sc.B.n_tris
    segs[-1] = [va, ta, vb, tb]
    return (np.concatenate(VA), np.concatenate(TA).astype(np.int32), np.concatenate(VB),
            np.concatenate(TB).astype(np.int32), segs.astype(np.int32))
