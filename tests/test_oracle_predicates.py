"""Pins for the oracle's exact predicates and its brute-force detection on
hand-built cases.

The oracle decides signs with its own big-integer determinant.  These tests
check it against exact rational arithmetic (Python's `fractions`, a
different algorithm: the Leibniz expansion of the 4x4 determinant with a
column of ones, which equals minus the 3x3 determinant of differences), on
random, near-degenerate (points snapped onto a plane then moved by a few
ulps) and exactly degenerate inputs, and check detection against answers
derived by hand (tests/golden/hand_cases.json).
"""
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")


def _perm_parity(p):
    inv = sum(1 for i in range(len(p)) for j in range(i + 1, len(p)) if p[i] > p[j])
    return -1 if inv % 2 else 1


_PERMS4 = [(p, _perm_parity(p)) for p in itertools.permutations(range(4))]


def frac_orient(a, b, c, x):
    """sign det[b-a, c-a, x-a] = -sign det[[a,1],[b,1],[c,1],[x,1]] (Leibniz
    formula over exact rationals; floats convert to Fractions exactly)."""
    M = [[Fraction(float(v)) for v in p] + [Fraction(1)] for p in (a, b, c, x)]
    det = Fraction(0)
    for p, s in _PERMS4:
        t = Fraction(s)
        for r in range(4):
            t *= M[r][p[r]]
        det += t
    return -((det > 0) - (det < 0))


def frac_segtri(p, q, a, b, c):
    sp, sq = frac_orient(a, b, c, p), frac_orient(a, b, c, q)
    if sp * sq >= 0:
        return False, 0
    t = [frac_orient(p, q, a, b), frac_orient(p, q, b, c), frac_orient(p, q, c, a)]
    hit = all(v >= 0 for v in t) or all(v <= 0 for v in t)
    return hit, (sp if hit else 0)


def test_orient_sign_convention():
    # Sec. 4: the face normal designates the front side; a point the
    # counter-clockwise normal (0,0,1) points to is in front (+1).
    a, b, c = [0, 0, 0], [1, 0, 0], [0, 1, 0]
    assert oracle.orient(a, b, c, [0, 0, 1]) == 1
    assert oracle.orient(a, b, c, [0.3, 0.3, -1e-300]) == -1
    assert oracle.orient(a, b, c, [5, -7, 0]) == 0
    assert oracle.orient(a, c, b, [0, 0, 1]) == -1


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_orient_random_vs_fraction(dtype):
    rng = np.random.default_rng(1)
    for _ in range(300):
        P = rng.uniform(-3, 3, (4, 3)).astype(dtype).astype(np.float64)
        assert oracle.orient(*P) == frac_orient(*P)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_orient_near_degenerate_vs_fraction(dtype):
    """Points computed on the plane in floating point (so near but usually
    not on it), then moved by -4..4 ulps in one coordinate."""
    rng = np.random.default_rng(2)
    n_zero = n_pos = n_neg = 0
    for _ in range(150):
        a, b, c = rng.uniform(-2, 2, (3, 3)).astype(dtype)
        s, t = rng.uniform(-0.5, 1.5, 2).astype(dtype)
        x0 = (a + s * (b - a) + t * (c - a)).astype(dtype)
        for k in range(-4, 5):
            x = x0.copy()
            ax = int(rng.integers(0, 3))
            for _ in range(abs(k)):
                x[ax] = np.nextafter(x[ax], dtype(np.inf) if k > 0 else dtype(-np.inf))
            pts = [np.asarray(v, np.float64) for v in (a, b, c, x)]
            ref = frac_orient(*pts)
            assert oracle.orient(*pts) == ref
            n_zero += ref == 0
            n_pos += ref > 0
            n_neg += ref < 0
    assert n_pos > 50 and n_neg > 50


def test_orient_exact_zero_and_huge_range():
    # integer points on the plane z = 2x - 3y + 1: exactly coplanar
    rng = np.random.default_rng(3)
    for _ in range(100):
        xy = rng.integers(-1000, 1000, (4, 2)).astype(np.float64)
        P = np.c_[xy, 2 * xy[:, 0] - 3 * xy[:, 1] + 1]
        assert oracle.orient(*P) == 0 == frac_orient(*P)
        P[3, 2] = np.nextafter(P[3, 2], np.inf)
        assert oracle.orient(*P) == frac_orient(*P) == (1 if oracle.orient(P[0], P[1], P[2], P[3] + [0, 0, 1]) > 0 else -1)
    # widely spread exponents, including subnormals
    cases = [
        ([1e-300, 0, 0], [0, 1e-300, 0], [0, 0, 1e-300], [1e-310, 1e-310, 1e-310]),
        ([1e30, 0, 0], [0, 1e30, 0], [0, 0, 1e30], [1e-30, 1e-30, 1e-30]),
        ([5e-324, 0, 0], [0, 5e-324, 0], [0, 0, 0], [0, 0, 5e-324]),
        ([1.0, 2.0, 3.0], [1.0 + 2 ** -52, 2.0, 3.0], [1.0, 2.0 + 2 ** -51, 3.0], [1.0, 2.0, 3.0 - 2 ** -52]),
    ]
    for P in cases:
        assert oracle.orient(*P) == frac_orient(*P)


def test_segtri_near_degenerate_vs_fraction():
    """Segments aimed at triangle corners and edges (where the closed-
    triangle reading matters) and at the plane (endpoint nearly on it)."""
    rng = np.random.default_rng(4)
    hits = 0
    for _ in range(200):
        a, b, c = rng.uniform(-1, 1, (3, 3)).astype(np.float32).astype(np.float64)
        w = rng.choice([0.0, 0.5, 1.0], 3)
        if w.sum() == 0:
            w[0] = 1
        w = w / w.sum()
        target = w[0] * a + w[1] * b + w[2] * c
        nrm = np.cross(b - a, c - a)
        d = nrm / np.linalg.norm(nrm) + rng.normal(0, 0.3, 3)
        p = (target + rng.uniform(0.01, 1.0) * d).astype(np.float32).astype(np.float64)
        q = (target - rng.uniform(0.0, 1.0) * d).astype(np.float32).astype(np.float64)
        ref = frac_segtri(p, q, a, b, c)
        got = oracle.segtri(p, q, a, b, c)
        assert got == ref
        hits += ref[0]
    assert hits > 20


def _case_meshes(case):
    A, B = case["A"], case["B"]
    return (np.asarray(A["V"], np.float64), np.asarray(A["T"], np.int32), A["oriented"],
            np.asarray(B["V"], np.float64), np.asarray(B["T"], np.int32), B["oriented"])


@pytest.mark.parametrize("case", json.load(open(GOLD))["cases"], ids=lambda c: c["name"])
def test_hand_cases(case):
    PA, TA, oA, PB, TB, oB = _case_meshes(case)
    pr = oracle.detect(PA, TA, oA, PB, TB, oB)
    assert pr.rec.tolist() == case["pairs"]
    assert oracle.stencils(pr).tolist() == case["stencils"]
    # every reported pair re-checked by exact rationals, and its side
    for (d, v0, v1, f), s in zip(pr.rec.tolist(), pr.side.tolist()):
        PE, PF, TF = (PA, PB, TB) if d == 0 else (PB, PA, TA)
        ok, side = frac_segtri(PE[v0], PE[v1], *PF[TF[f]])
        assert ok and side == s


def test_edges_counts():
    import meshgen
    for L in range(4):
        V, T = meshgen.icosphere(L)
        E = oracle.edges(T)
        assert len(E) == 30 * 4 ** L
        assert np.all(E[:, 0] < E[:, 1])
        assert np.all(np.diff(E[:, 0].astype(np.int64) * 10 ** 6 + E[:, 1]) > 0)
    V, T = meshgen.cloth(17, 1.0)
    assert len(oracle.edges(T)) == 2 * 17 * 16 + 16 * 16
    V, T = meshgen.torus(13, 7, 1.0, 0.3)
    assert len(oracle.edges(T)) == 3 * 13 * 7
    assert len(oracle.edges(np.zeros((0, 3), np.int32))) == 0
