#!/usr/bin/env python
"""DCD + response ms/frame and E-F tests/s on one GB300.

Workload (default): un-oriented cloth, 200 x 200 vertices (119,201 edges,
79,202 faces, side 2.0, seeded sinusoidal heights of amplitude 0.3) draped
into an oriented torus (256 x 128 quads = 65,536 faces, R 1.0, r 0.4),
float32 positions, about 2,200 E-F intersections.  One frame = one pass of
the whole path: exact E-F detection (BVH build, refit, traversal, exact
narrow phase), pair sort, stencils, constraint assembly, the Eq. 8 solve and
the displacement of the stencil vertices, starting from the same initial
positions every frame (restored inside the timed region).

Printed: one JSON line (rank 0).  `value` is ms per frame (lower is
better); E-F tests/s is reported beside it, brute-force equivalent
(|E| x |F| per frame over the frame time) and executed narrow-phase tests.
`--impl reference` times the CPU oracle on the same frame instead.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DCD+response ms/frame and E-F tests/s on 1 GB300 vs plain FP64 GPU form"
D_POST = 1e-4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-form", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 1,024-pair batched workload")
    ap.add_argument("--no-c3", action="store_true",
                    help="skip the two-spheres and two-tori sections (precision form, d-sweep)")
    ap.add_argument("--frames", type=int, default=300,
                    help="frames of the cloth-over-body sequence (0 to skip)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock and throttle samples while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = list(csv.reader(open(self.path)))
        os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [c.strip() for c in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCES = {"k_traverse": ("detect.cu", "predicates.cuh"), "k_cg_zone_pair": ("solve.cu",)}
PROFILES = {"k_traverse": "k_traverse_cloth_torus.md", "k_cg_zone_pair": "k_cg_zone_pair_cloth_torus.md"}


def kernel_source_hash(kernel: str = "k_traverse") -> str:
    """First 16 hex digits of the SHA-256 of the kernel's source files, code
    lines only (lines that are blank or hold only a // comment are left out,
    so a comment edit keeps a profile valid)."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        for line in open(os.path.join(ROOT, "paper_1409_2081_gb300", "csrc", f), "rb"):
            t = line.strip()
            if t and not t.startswith(b"//"):
                h.update(t + b"\n")
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str = "k_traverse"):
    """DRAM bytes per launch of `kernel` from its committed ncu summary, if
    the summary was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", PROFILES[kernel])
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and line.strip().startswith(("traffic_bytes_per_launch", "source_sha")):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_sha") != kernel_source_hash(kernel):
        return None
    try:
        return int(float(vals["traffic_bytes_per_launch"]))
    except (KeyError, ValueError):
        return None


def whole_job(local_total_ms: float, steps: int, dist=None, device=None):
    """Replicas only: every rank runs the same workload on its own GPU; the
    job's time is the slowest rank's, and the whole-job ms per frame is
    that time over all frames of all ranks.  Returns (max total ms, ms per
    frame)."""
    ws = 1
    t = local_total_ms
    if dist is not None and dist.is_initialized():
        import torch
        ws = dist.get_world_size()
        x = torch.tensor([local_total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return t, t / (steps * ws)


def packed(torch, xs):
    """One buffer holding the coordinate arrays xs back to back, views into
    it (in order) and a copy of its initial state: a step restores, uploads
    or downloads every array of both meshes with one copy."""
    pos = torch.cat([t.reshape(-1) for t in xs])
    views, o = [], 0
    for t in xs:
        views.append(pos[o:o + t.numel()])
        o += t.numel()
    return pos, pos.clone(), views


def scene():
    import meshgen
    return meshgen.scene_c2()


def cpu_oracle_frame(sc, edge_fraction=1.0):
    """One frame on the CPU oracle (detection over a fraction of the cloth
    edges, then stencils and the float64 solve of what was found); returns
    (seconds, cores, scaled seconds per full frame)."""
    import numpy as np
    import oracle
    PA, PB = sc.positions("A"), sc.positions("B")
    E = oracle.edges(sc.A.T)
    m = max(1, int(round(len(E) * edge_fraction)))
    sub = E if m >= len(E) else E[np.linspace(0, len(E) - 1, m).astype(np.int64)]
    t0 = time.perf_counter()
    hits = oracle.detect_one_direction(PA, sub, PB, sc.B.T)
    t1 = time.perf_counter()
    rec = np.zeros((len(hits), 4), np.uint32)
    rec[:, 1] = sub[hits[:, 0], 0]
    rec[:, 2] = sub[hits[:, 0], 1]
    rec[:, 3] = hits[:, 1]
    st = oracle.stencils(oracle.Pairs(rec, hits[:, 2].astype(np.int8)))
    oracle.respond(st, PA, sc.A.T, PB, sc.B.T, D_POST)
    t2 = time.perf_counter()
    frac = len(sub) / len(E)
    return (t2 - t0), oracle.num_threads(), (t1 - t0) / frac + (t2 - t1)


def frame_sequence(api, torch, dev, n_frames, max_iters=1, rings=4, sweeps=16, body_inv_mass=1.0,
                   time_budget_s=45.0):
    """Cloth 512 x 512 (side 3.0, float32, un-oriented) falling onto an
    oriented body (icosphere level 7 with spherical-harmonic radius noise of
    amplitude 0.1): each frame moves the cloth by the seeded velocity field
    (torch ops on the device, outside the timed region), then resolve is
    timed: max_iters repair iterations (default one DCD response per frame,
    the paper's use in its animation, Sec. 6), graph-replayed, with the
    diffusion of Sec. 5 over `rings` rings and `sweeps` sweeps.  The
    prescribed drift pushes the resting cloth into the body every frame, so
    contact frames keep a few thousand fresh pairs for the next response; a
    run whose frames blow up stops at `time_budget_s` and reports the frames
    it completed."""
    import time
    import numpy as np
    import meshgen
    sc = meshgen.scene_c5()
    mot = sc.meta["motion"]
    ctx = api.Context(diffuse_rings=rings, diffuse_sweeps=sweeps)
    cap = 1 << 18
    ctx.hfcr_reserve(max(sc.A.n_verts, sc.B.n_verts), max(sc.A.n_tris, sc.B.n_tris), cap)

    def dev_xyz(V):
        P = V.astype(np.float32)
        return [torch.tensor(np.ascontiguousarray(P[:, c]), device=dev) for c in range(3)]

    xa, xb = dev_xyz(sc.A.V), dev_xyz(sc.B.V)
    ta, tb = torch.tensor(sc.A.T, device=dev), torch.tensor(sc.B.T, device=dev)
    ea = torch.zeros((3 * sc.A.n_tris, 2), dtype=torch.int32, device=dev)
    ea = ea[:ctx.hfcr_build_edges(ta, sc.A.n_verts, ea)].contiguous()
    A = api.Mesh(*xa, ta, False, edges=ea)
    wb = None if body_inv_mass == 1.0 else torch.full((sc.B.n_verts,), body_inv_mass,
                                                      dtype=torch.float32, device=dev)
    B = api.Mesh(*xb, tb, True, inv_mass=wb)
    K = torch.tensor(mot.k.T, dtype=torch.float32, device=dev)
    W = torch.tensor(mot.w, dtype=torch.float32, device=dev)
    PH = torch.tensor(mot.ph, dtype=torch.float32, device=dev)
    AD = torch.tensor((mot.amp[:, None] * mot.dir) * (0.5 * mot.v0), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    ms, pairs, iters = [], [], []
    stop, t_start = "all frames", time.time()
    for f in range(n_frames):
        X = torch.stack([A.x, A.y, A.z], 1)
        V = torch.sin(X @ K + W * f + PH) @ AD
        V[:, 2] -= mot.v0
        X += V
        A.x.copy_(X[:, 0]); A.y.copy_(X[:, 1]); A.z.copy_(X[:, 2])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        try:
            info = ctx.hfcr_resolve(A, B, D_POST, max_iters)
        except api.HfcrError as e:
            stop = f"frame {f}: {e}"[:120]
            break
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        pairs.append(int(info.pairs_first))
        iters.append(int(info.iters))
        if time.time() - t_start > time_budget_s:
            stop = f"time budget {time_budget_s:.0f} s after frame {f}"
            break
    ctx.close()
    contact = [i for i, p in enumerate(pairs) if p > 0]
    srt = sorted(ms)
    cms = sorted(ms[i] for i in contact)
    return {"workload": "cloth 512x512 (784,385 edges) falling on SH body (icosphere L7, 327,680 faces), "
                        "float32, one resolve (<= %d iterations, diffusion R=%d S=%d, body inverse "
                        "mass %g) per frame" % (max_iters, rings, sweeps, body_inv_mass),
            "frames_requested": n_frames, "frames_completed": len(ms), "stopped": stop,
            "ms_p50": round(statistics.median(ms), 4) if ms else None,
            "ms_p99": round(srt[min(len(srt) - 1, int(0.99 * len(srt)))], 4) if ms else None,
            "first_contact_frame": contact[0] if contact else None,
            "contact_frames": len(contact),
            "contact_ms_p50": round(statistics.median(cms), 4) if cms else None,
            "contact_ms_p99": round(cms[min(len(cms) - 1, int(0.99 * len(cms)))], 4) if cms else None,
            "pairs_last_frame": pairs[-1] if pairs else 0,
            "max_pairs": max(pairs) if pairs else 0,
            "mean_iters": round(statistics.mean(iters), 2) if iters else None}


def batched(api, torch, dev, steps, warmup, timed_fn):
    """1,024 independent pairs of oriented icospheres (levels 1..5, 80 to
    20,480 faces each, random rotation, centre distance U(0.5, 1.8) radii),
    float32, concatenated into two meshes with a segment table.  A step is
    one repair iteration of every pair from the initial state
    (hfcr_resolve_batch, max_iters 1: detection of A-edges vs B-faces of
    all pairs, stencils, zones, solve, displacement)."""
    import numpy as np
    import meshgen
    VA, TA, VB, TB, segs = meshgen.concat_batch(meshgen.scene_c4())
    ctx = api.Context()
    ctx.hfcr_reserve(max(len(VA), len(VB)), max(len(TA), len(TB)), 1 << 21)

    def xyz(V):
        P = V.astype(np.float32)
        return [torch.tensor(np.ascontiguousarray(P[:, c]), device=dev) for c in range(3)]

    xa, xb = xyz(VA), xyz(VB)
    ta, tb = torch.tensor(TA, device=dev), torch.tensor(TB, device=dev)
    ea = torch.zeros((3 * len(TA), 2), dtype=torch.int32, device=dev)
    ea = ea[:ctx.hfcr_build_edges(ta, len(VA), ea)].contiguous()
    eb = torch.zeros((3 * len(TB), 2), dtype=torch.int32, device=dev)
    eb = eb[:ctx.hfcr_build_edges(tb, len(VB), eb)].contiguous()
    pos, pos0, v = packed(torch, xa + xb)
    A = api.Mesh(*v[:3], ta, True, edges=ea)
    B = api.Mesh(*v[3:], tb, True, edges=eb)
    dsegs = torch.tensor(segs, device=dev)

    def step():
        pos.copy_(pos0, non_blocking=True)
        return ctx.hfcr_resolve_batch(A, B, dsegs, D_POST, 1)

    variant, variant_ms = ctx.hfcr_autotune(A, B, dsegs)
    for _ in range(warmup):
        step()
    ctx.hfcr_profile_enable(True)
    timed_fn(step, max(3, steps // 4), 1)
    prof = ctx.hfcr_profile_read()
    ctx.hfcr_profile_enable(False)
    ms, infos = timed_fn(step, steps, 1)
    info = infos[-1]
    trav_ms, trav_n = prof["traverse"]
    P = int(info.pairs_first)
    alg = len(VA) * 12 + len(ea) * 8 + len(VB) * 12 + len(TB) * 12 + P * 8
    peak, kind = measured_peak_hbm()
    ach = alg / (trav_ms / max(1, trav_n) * 1e-3) / 1e9
    ctx.close()
    n_frames = max(1, prof["traverse"][1])
    return {"workload": "1,024 pairs of icospheres L1..5 (A: %d faces, B: %d faces), float32, "
                        "one batched repair iteration" % (len(TA), len(TB)),
            "ms_per_step": round(statistics.mean(ms), 4), "ms_p50": round(statistics.median(ms), 4),
            "pairs": P, "stencils": int(info.total_stencils),
            "ef_tests_per_s_bruteforce": round(info.stats.brute_force_equiv / (statistics.mean(ms) / 1e3), 1),
            "stage_ms_per_step": {k: round(v[0] / n_frames, 4) for k, v in prof.items()},
            "roofline": {"kernel": "k_traverse", "bound": "hbm", "achieved": round(ach, 2),
                         "peak": peak, "peak_kind": kind, "unit": "GB/s", "frac": round(ach / peak, 5),
                         "alg_bytes_per_launch": alg,
                         "avg_launch_ms": round(trav_ms / max(1, trav_n), 5),
                         "traverse_variant": variant, "variant_ms": variant_ms}}


def small_form(api, torch, dev, steps, timed_fn):
    """Two jittered level-3 icospheres offset by 1.5 (642 vertices, 1,280
    faces each), float64: one repair iteration from the initial state in
    the plain float64 form and the mixed form, and the whole repair loop
    (alternating roles) to convergence.  This size is bound by launch
    latency, so it is reported in microseconds."""
    import numpy as np
    import meshgen
    sc = meshgen.scene_c1()

    def mesh(ctx, m):
        xyz = [torch.tensor(np.ascontiguousarray(m.V[:, c]), dtype=torch.float64, device=dev) for c in range(3)]
        tris = torch.tensor(m.T, device=dev)
        # topology preparation (once per mesh, outside the timed region)
        e = torch.zeros((3 * m.n_tris, 2), dtype=torch.int32, device=dev)
        e = e[:ctx.hfcr_build_edges(tris, m.n_verts, e)].contiguous()
        return tris, e, xyz

    out = {"workload": "two icospheres L3 (1,280 faces each), offset 1.5, jitter 0.01, float64"}
    for name, solver, f32f, graphs in (("fp64_form", api.HFCR_SOLVER_FP64, False, False),
                                       ("mixed_form", api.HFCR_SOLVER_MIXED, True, True)):
        ctx = api.Context(solver=solver, f32_filter=f32f, graphs=graphs)
        ctx.hfcr_reserve(sc.A.n_verts, sc.A.n_tris, 1 << 14)
        (ta, ea, a0), (tb, eb, b0) = mesh(ctx, sc.A), mesh(ctx, sc.B)
        pos, pos0, v = packed(torch, a0 + b0)
        A = api.Mesh(*v[:3], ta, True, edges=ea)
        B = api.Mesh(*v[3:], tb, True, edges=eb)

        def step():
            pos.copy_(pos0, non_blocking=True)
            return ctx.hfcr_resolve(A, B, D_POST, 1)

        ms, infos = timed_fn(step, steps, 3)
        out[name] = {"us_per_iteration": round(1e3 * statistics.median(ms), 1),
                     "pairs": int(infos[-1].pairs_first)}
        if solver == api.HFCR_SOLVER_MIXED:
            def loop():
                pos.copy_(pos0, non_blocking=True)
                return ctx.hfcr_resolve(A, B, D_POST, 64)
            lms, linfo = timed_fn(loop, max(3, steps // 10), 1)
            out["repair_loop"] = {"ms": round(statistics.median(lms), 3),
                                  "detections": int(linfo[-1].iters),
                                  "converged": bool(linfo[-1].converged)}
        ctx.close()
    return out


def precision_form(api, torch, dev, steps, timed_fn, d_values=(1e-4, 1e-3, 1e-2), rings=4,
                   sweeps=16, max_iters=32):
    """Two 262,144-face tori, float32, a seeded local overlap: one repair
    iteration (float32 filter -> float64 -> exact; float32 CG + float64
    refinement) timed from the initial state; the float32 solver's
    displacement error against the float64 GPU solver on the same stencils;
    and the d-sweep (each d resolved with diffusion, at most max_iters
    detections: detections run, and the signed distance D' of every
    first-iteration stencil's x0 from its face at the final positions,
    relative to d)."""
    import numpy as np
    import meshgen
    sc = meshgen.scene_c3()

    def fresh():
        # the six coordinate arrays are views of one buffer (one restore copy);
        # init = (buffer, its initial copy, the six initial arrays)
        xyz = [torch.tensor(np.ascontiguousarray(m.V[:, c].astype(np.float32)), device=dev)
               for m in (sc.A, sc.B) for c in range(3)]
        pos, pos0, views = packed(torch, xyz)
        A = api.Mesh(*views[:3], torch.tensor(sc.A.T, device=dev), True)
        B = api.Mesh(*views[3:], torch.tensor(sc.B.T, device=dev), True)
        return A, B, (pos, pos0, xyz)

    def restore(A, B, init):
        init[0].copy_(init[1], non_blocking=True)  # all six coordinate arrays

    cap = 1 << 20
    ctx = api.Context()
    ctx.hfcr_reserve(sc.A.n_verts, sc.A.n_tris, cap)
    A, B, init = fresh()
    variant, _ = ctx.hfcr_autotune(A, B)

    def step():
        restore(A, B, init)
        return ctx.hfcr_resolve(A, B, D_POST, 1)

    ms, infos = timed_fn(step, steps, 3)
    info = infos[-1]
    # float32 CG + float64 refinement vs the float64 CG on the same stencils
    restore(A, B, init)
    pairs = torch.zeros((cap, 4), dtype=torch.int32, device=dev)
    n = ctx.hfcr_detect(A, B, pairs)
    st = torch.zeros((cap, 4), dtype=torch.int32, device=dev)
    k = ctx.hfcr_build_stencils(A, B, pairs, n, st)
    ctx64 = api.Context(solver=api.HFCR_SOLVER_FP64)
    ctx64.hfcr_reserve(sc.A.n_verts, sc.A.n_tris, cap)
    A64 = api.Mesh(*[t.double() for t in init[2][:3]], A.tris, True)
    B64 = api.Mesh(*[t.double() for t in init[2][3:]], B.tris, True)
    dx = {}
    for name, c, MA, MB in (("mixed", ctx, A64, B64), ("fp64", ctx64, A64, B64)):
        da = [torch.zeros(sc.A.n_verts, dtype=torch.float64, device=dev) for _ in range(3)]
        db = [torch.zeros(sc.B.n_verts, dtype=torch.float64, device=dev) for _ in range(3)]
        si = c.hfcr_respond(MA, MB, st, k, D_POST, da, db)
        dx[name] = (torch.cat([torch.stack(da, 1), torch.stack(db, 1)]), si)
    err = float((dx["mixed"][0] - dx["fp64"][0]).abs().max() / dx["fp64"][0].abs().max())
    ctx64.close()
    ctx.close()
    # d-sweep: repair to convergence from the initial state (the overlap is
    # several edge lengths deep: the loop uses the diffusion of Sec. 5)
    ctx = api.Context(diffuse_rings=rings, diffuse_sweeps=sweeps)
    ctx.hfcr_reserve(sc.A.n_verts, sc.A.n_tris, cap)
    stn = st[:k, :3].cpu().numpy().astype(np.int64)
    sweep = []
    for d in d_values:
        restore(A, B, init)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = ctx.hfcr_resolve(A, B, d, max_iters)
        e1.record()
        e1.synchronize()
        PA = torch.stack([A.x, A.y, A.z], 1).double().cpu().numpy()
        PB = torch.stack([B.x, B.y, B.z], 1).double().cpu().numpy()
        # D' of x0 against its face at the final positions (Eq. 1); dir 0:
        # x0 in A, face in B; dir 1: the reverse
        m0 = stn[:, 0] == 0
        x0 = np.empty((len(stn), 3))
        tri = np.empty((len(stn), 3, 3))
        x0[m0], tri[m0] = PA[stn[m0, 1]], PB[sc.B.T[stn[m0, 2]]]
        x0[~m0], tri[~m0] = PB[stn[~m0, 1]], PA[sc.A.T[stn[~m0, 2]]]
        nrm = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
        ln = np.linalg.norm(nrm, axis=1)
        ok = ln > 0
        Dp = np.einsum("ij,ij->i", nrm[ok] / ln[ok, None], x0[ok] - tri[ok].mean(axis=1))
        sweep.append({"d": d, "converged": bool(r.converged), "detections": int(r.iters),
                      "pairs_first": int(r.pairs_first), "ms": round(e0.elapsed_time(e1), 3),
                      "gap_over_d_min": round(float(Dp.min() / d), 4),
                      "gap_over_d_median": round(float(np.median(Dp) / d), 4)})
    ctx.close()
    return {"workload": "two tori 512x256 quads (262,144 faces each), float32, local overlap "
                        "depth U(0, 0.2 r); one repair iteration from the initial state",
            "ms_p50": round(statistics.median(ms), 4), "ms_mean": round(statistics.mean(ms), 4),
            "pairs": int(info.pairs_first), "stencils": int(k),
            "filter": {"narrow_tests": int(info.stats.narrow_tests),
                       "f64_fallbacks": int(info.stats.f64_fallbacks),
                       "exact_fallbacks": int(info.stats.exact_fallbacks)},
            "dx_rel_err_vs_fp64_solver": err,
            "mixed_solver": {"cg_iters": int(dx["mixed"][1].cg_iters),
                             "rel_residual": dx["mixed"][1].rel_residual},
            "traverse_variant": variant,
            "d_sweep": {"diffusion": {"rings": rings, "sweeps": sweeps}, "max_iters": max_iters,
                        "runs": sweep}}


def run_reference(args, ws, rank):
    """The CPU oracle as the reference arm (rank 0 only)."""
    if rank != 0:
        return
    sc = scene()
    # size each step so that warmup + steps finish within a few minutes
    t_full, cores, _ = cpu_oracle_frame(sc, 1.0)
    budget = 150.0
    frac = min(1.0, budget / max(1e-9, t_full * (args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_oracle_frame(sc, frac)
    times = []
    for _ in range(args.steps):
        _, _, scaled = cpu_oracle_frame(sc, frac)
        times.append(scaled * 1e3)
    ms = statistics.mean(times)
    bf = 119201 * 65536
    sample = (f"{frac:.3f} of the cloth edges per step against all 65,536 torus faces, "
              f"stencils and float64 solve of the found pairs; scaled to a full frame")
    line = {"metric": METRIC, "value": round(ms, 3), "unit": "ms/frame", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "cloth 200x200 vs torus 256x128 (65,536 faces), one frame",
                       "l2": "n/a (CPU)"},
            "ef_tests_per_s_bruteforce": bf / (ms / 1e3),
            "cpu_baseline": {"value": round(ms, 3), "unit": "ms/frame", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(ms, 3), "unit": "ms/frame", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import numpy as np
    import torch
    from paper_1409_2081_gb300 import api

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    # a dedicated stream (the legacy default stream cannot be graph-captured)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)

    sc = scene()

    def dev_mesh(m, dtype):
        # the float64 form computes on the exact widening of the same float32 data
        P = np.ascontiguousarray(m.V.astype(np.float32).astype(dtype))
        tdt = torch.float32 if dtype == np.float32 else torch.float64
        xyz = [torch.tensor(np.ascontiguousarray(P[:, c]), dtype=tdt, device=dev) for c in range(3)]
        return xyz, torch.tensor(m.T, device=dev)

    def build(dtype, solver, f32_filter, graphs=True):
        ctx = api.Context(solver=solver, f32_filter=f32_filter, graphs=graphs)
        ctx.hfcr_reserve(max(sc.A.n_verts, sc.B.n_verts), max(sc.A.n_tris, sc.B.n_tris), 1 << 16)
        (xa, ta), (xb, tb) = dev_mesh(sc.A, dtype), dev_mesh(sc.B, dtype)
        # topology preparation (once per mesh, outside every timed region)
        ea = torch.zeros((3 * sc.A.n_tris, 2), dtype=torch.int32, device=dev)
        ne = ctx.hfcr_build_edges(ta, sc.A.n_verts, ea)
        ea = ea[:ne].contiguous()
        # the six coordinate arrays are views of one buffer, so that a frame
        # restores (or uploads, or downloads) the positions in one copy
        pos, pos0, views = packed(torch, xa + xb)
        A = api.Mesh(*views[:3], ta, False, edges=ea)
        B = api.Mesh(*views[3:], tb, True)
        return ctx, A, B, (pos, pos0), ne

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def restore(A, B, init):
        init[0].copy_(init[1], non_blocking=True)  # all six coordinate arrays

    def frame(ctx, A, B, init):
        restore(A, B, init)
        return ctx.hfcr_resolve(A, B, D_POST, 1)

    def timed(fn, K, W):
        for _ in range(W):
            fn()
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(K)]
        infos = []
        for i in range(K):
            flush.fill_(float(i))          # L2 flush between steps (not timed)
            evs[i][0].record(stream)
            infos.append(fn())
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        ms = [a.elapsed_time(b) for a, b in evs]
        return ms, infos

    # ---- optimized form: float32 filter, mixed-precision solver ----
    ctx, A, B, init, ne = build(np.float32, api.HFCR_SOLVER_MIXED, True)
    # traversal variant chosen by the library's autotuner on this scene
    variant, variant_ms = ctx.hfcr_autotune(A, B)
    for _ in range(args.warmup):
        frame(ctx, A, B, init)
    # profiled pass: CUDA events around every stage on the launching stream
    # (the library launches the stages directly while profiling)
    k_prof = max(5, min(args.steps, 50))
    ctx.hfcr_profile_enable(True)
    prof_ms, _ = timed(lambda: frame(ctx, A, B, init), k_prof, 2)
    prof = ctx.hfcr_profile_read()
    ctx.hfcr_profile_enable(False)
    # headline pass: each repair iteration replayed as a CUDA graph
    launches0 = api.hfcr_launch_count()
    sampler = ClockSampler(local)
    sampler.start()
    ms, infos = timed(lambda: frame(ctx, A, B, init), args.steps, 2)
    clocks = sampler.stop()
    launches = api.hfcr_launch_count() - launches0
    total_ms, per_frame = whole_job(sum(ms), args.steps, pg, dev)
    info = infos[-1]
    bf = int(info.stats.brute_force_equiv)
    narrow = int(info.stats.narrow_tests)

    P = int(info.pairs_first)
    peak, peak_kind = measured_peak_hbm()
    n_prof_frames = max(1, prof["traverse"][1])
    stage_ms = {k: round(v[0] / n_prof_frames, 4) for k, v in prof.items()}
    dominant = max(stage_ms, key=stage_ms.get)
    # rooflines of the two kernels that own a stage each: the traversal +
    # exact narrow phase, and the per-zone solver (the solve stage is
    # k_cg_zone_pair, which solves this frame's ten zones, the
    # one-warp-per-zone and 1024-thread launches, both nearly empty here,
    # and the one-CTA k_zone_final); algorithmic bytes = compulsory reads +
    # writes
    trav_ms, trav_n = prof["traverse"]
    trav_avg_ms = trav_ms / max(1, trav_n)
    alg_trav = (sc.A.n_verts * 12 + ne * 8 + sc.B.n_verts * 12 + sc.B.n_tris * 12 + P * 8)
    ach_trav = alg_trav / (trav_avg_ms * 1e-3) / 1e9
    solve_ms, solve_n = prof["solve"]
    solve_avg_ms = solve_ms / max(1, solve_n)
    # stencil count and touched vertices of this frame's system (outside the
    # timed regions)
    restore(A, B, init)
    pbuf = torch.zeros((1 << 16, 4), dtype=torch.int32, device=dev)
    n_p = ctx.hfcr_detect(A, B, pbuf)
    sbuf = torch.zeros((1 << 16, 4), dtype=torch.int32, device=dev)
    k_st = ctx.hfcr_build_stencils(A, B, pbuf, n_p, sbuf)
    dxa = [torch.zeros(sc.A.n_verts, device=dev) for _ in range(3)]
    dxb = [torch.zeros(sc.B.n_verts, device=dev) for _ in range(3)]
    si = ctx.hfcr_respond(A, B, sbuf, k_st, D_POST, dxa, dxb)
    # per stencil: ids 16 + float32 normal 16 + preconditioner row 16 + b 8
    # + float64 normal 32 + lam 8 (written) + 4 vertex-CSR entries 16 + group
    # start 4; per touched vertex: CSR offset 4 + inverse mass 4
    alg_cg = 116 * k_st + 8 * int(si.n_touched)
    ach_cg = alg_cg / (solve_avg_ms * 1e-3) / 1e9
    roof = {
        "k_traverse": {"kernel": "k_traverse (BVH traversal + exact narrow phase)", "bound": "hbm",
                       "achieved": round(ach_trav, 2), "peak": peak, "peak_kind": peak_kind,
                       "unit": "GB/s", "frac": round(ach_trav / peak, 5),
                       "traffic": profiled_traffic("k_traverse"), "alg_bytes_per_launch": alg_trav,
                       "avg_launch_ms": round(trav_avg_ms, 5), "launches_timed": trav_n,
                       "traverse_variant": variant, "variant_ms": variant_ms},
        "k_cg_zone_pair": {"kernel": "k_cg_zone_pair (float32 PCG per impact zone, float64 "
                                     "refinement in the kernel)", "bound": "hbm",
                      "achieved": round(ach_cg, 3), "peak": peak, "peak_kind": peak_kind,
                      "unit": "GB/s", "frac": round(ach_cg / peak, 6),
                      "traffic": profiled_traffic("k_cg_zone_pair"), "alg_bytes_per_launch": alg_cg,
                      "avg_launch_ms": round(solve_avg_ms, 5), "launches_timed": solve_n,
                      "stencils": k_st, "touched_vertices": int(si.n_touched)},
    }
    dom_kernel = "k_cg_zone_pair" if stage_ms["solve"] >= stage_ms["traverse"] else "k_traverse"
    roofline = dict(roof[dom_kernel], dominant_stage=dominant,
                    chosen_by="the larger of the solve and traverse stages in the profiled pass")

    # ---- end to end through the C ABI with host buffers ----
    # both meshes' coordinates, one pinned host buffer each way
    host_in = init[1].detach().cpu().pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()

    def e2e_frame():
        init[0].copy_(host_in, non_blocking=True)
        info = ctx.hfcr_resolve(A, B, D_POST, 1)
        host_out.copy_(init[0], non_blocking=True)
        return info

    e2e_ms, _ = timed(e2e_frame, args.steps, 2)
    e2e_total, _ = whole_job(sum(e2e_ms), args.steps, pg, dev)
    io_bytes = host_in.numel() * host_in.element_size()

    # ---- the plain float64 GPU form on the same frame ----
    fp64 = None
    if not args.no_fp64_form:
        # the plain float64 form: float64 positions, float64 filter -> exact,
        # float64 CG, plain launches (no graphs)
        ctx64, A64, B64, init64, _ = build(np.float64, api.HFCR_SOLVER_FP64, False, graphs=False)
        k64 = max(3, args.steps // 3)
        ms64, inf64 = timed(lambda: frame(ctx64, A64, B64, init64), k64, 2)
        fp64 = {"ms_per_frame": round(statistics.mean(ms64), 4), "steps": k64,
                "pairs": int(inf64[-1].pairs_first),
                "speedup_of_f32_form": round(statistics.mean(ms64) / statistics.mean(ms), 2)}
        ctx64.close()

    frames = frame_sequence(api, torch, dev, args.frames) if args.frames > 0 else None
    c3 = None if args.no_c3 else precision_form(api, torch, dev, max(5, args.steps // 5), timed)
    c1 = None if args.no_c3 else small_form(api, torch, dev, max(10, args.steps // 2), timed)
    batch = None if args.no_batch else batched(api, torch, dev, max(5, args.steps // 10), 2, timed)

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            sec, cores, scaled = cpu_oracle_frame(sc, 1.0)
            cpu = {"value": round(scaled * 1e3, 2), "unit": "ms/frame", "cores": cores, "kind": "oracle",
                   "sample": "one full frame: brute-force exact detection of all 119,201 cloth edges "
                             "against all 65,536 torus faces, stencils, float64 per-zone solve"}
        line = {
            "metric": METRIC, "value": round(per_frame, 4), "unit": "ms/frame",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "cloth 200x200 (119,201 edges) vs torus 256x128 (65,536 faces), "
                                   "float32, one DCD+response frame from the initial state",
                       "pairs": P, "stencils": int(info.total_stencils),
                       "predicates": "float32 semi-static filter -> float64 filter -> exact integers",
                       "solver": "float32 CG + float64 iterative refinement to 1e-12",
                       "l2": "flushed between steps (256 MB write)",
                       "parallelism": f"replicas x{ws}"},
            "ms_p50": round(statistics.median(ms), 4),
            "ms_p99": round(sorted(ms)[min(len(ms) - 1, int(0.99 * len(ms)))], 4),
            "ef_tests_per_s_bruteforce": round(bf / (per_frame / 1e3), 1),
            "ef_tests_per_s_executed": round(narrow / (per_frame / 1e3), 1),
            "filter": {"narrow_tests": narrow, "f64_fallbacks": int(info.stats.f64_fallbacks),
                       "exact_fallbacks": int(info.stats.exact_fallbacks)},
            "solver": {"cg_iters": int(info.cg_iters), "rel_residual": info.worst_rel_residual,
                       "float32_cg_in_shared_memory": bool(info.solver_path & 1)},
            "stage_ms_per_frame": stage_ms,
            "profiled_ms_per_frame": round(statistics.mean(prof_ms), 4),
            "graphs": True,
            "roofline": roofline,
            "rooflines": roof,
            "e2e": {"value": round(e2e_total / (args.steps * ws), 4), "unit": "ms/frame",
                    "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes},
            "fp64_form": fp64,
            "small_form": c1,
            "precision_form": c3,
            "frame_sequence": frames,
            "batch": batch,
            "gpu_launches": launches,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if pg:
        pg.barrier()
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
