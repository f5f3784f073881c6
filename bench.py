#!/usr/bin/env python
"""DCD + response ms/frame and E-F tests/s on one GB300.

Workload (default): the frame sequence.  An un-oriented float32 cloth of
512 x 512 vertices (784,385 edges, side 3.0) falls onto an oriented closed
body: an icosphere of level 7 (327,680 faces) whose radius carries
seeded spherical-harmonic noise.  Every frame, a seeded smooth velocity
field moves the cloth; then one DCD response runs: one repair iteration of
exact E-F detection (BVH build and refit, traversal, exact narrow phase),
stencils, constraint assembly, the Eq. 8 solve, and the harmonic diffusion
of the displacement (Sec. 5), replayed as a CUDA graph.  This is one DCD
response per output frame, the paper's own use (Sec. 6, third experiment).
A step is the whole 300-frame sequence from the initial state.

Printed: one JSON line (rank 0).  `value` is ms per frame over all timed
frames (lower is better), with p50 / p99 beside it.  E-F tests/s is
reported both as brute-force equivalent (|E| x |F| per frame over the
frame time) and as executed narrow-phase tests.  The other configurations
are extra keys: the cloth / torus frame, the two tori (precision form and
d-sweep), the two small spheres, and the 1,024-pair batch.
`--impl reference` times the CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
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
RINGS = 4          # diffusion band of the frame sequence (Sec. 5)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20, help="timed 300-frame sequences")
    ap.add_argument("--warmup", type=int, default=5, help="untimed 300-frame sequences")
    ap.add_argument("--frames", type=int, default=300, help="frames per sequence")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--ref-budget", type=float, default=150.0,
                    help="reference arm: seconds of oracle work for warmup + steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the lockstep pass of the float64 and graph-less forms")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the cloth/torus, two-tori, two-spheres and batch sections")
    ap.add_argument("--frame-log", default=None, help="write a per-frame CSV of the last timed sequence")
    ap.add_argument("--profile", default=None, metavar="CASE",
                    help="profiling run instead of the bench: 'frame:N' (the frame sequence up to "
                         "frame N), 'cloth_torus' or 'batch' (one iteration after three); the "
                         "profiled call runs inside the NVTX range 'profile'")
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
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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


# kernel -> (source files whose code lines it depends on, its ncu summary)
KERNELS = {
    "k_traverse": (("detect.cu", "predicates.cuh"), "k_traverse_frame_sequence.md"),
    "k_traverse_batch": (("detect.cu", "predicates.cuh"), "k_traverse_batch.md"),
    "k_band_cl": (("diffuse.cu",), "k_band_cl_frame_sequence.md"),
    "k_cg_zone_pair": (("solve.cu",), "k_cg_zone_pair_cloth_torus.md"),
    "k_refit": (("bvh.cu",), "k_refit_frame_sequence.md"),
    "k_cg_zone_big": (("solve.cu",), "k_cg_zone_big_frame_sequence.md"),
}


def kernel_source_hash(kernel: str = "k_traverse") -> str:
    """First 16 hex digits of the SHA-256 of the kernel's source files, code
    lines only (lines that are blank or hold only a // comment are left out,
    so a comment edit keeps a profile valid)."""
    h = hashlib.sha256()
    for f in KERNELS[kernel][0]:
        for line in open(os.path.join(ROOT, "paper_1409_2081_gb300", "csrc", f), "rb"):
            t = line.strip()
            if t and not t.startswith(b"//"):
                h.update(t + b"\n")
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from its committed ncu summary, if
    the summary was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", KERNELS[kernel][1])
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
    job's time is the slowest rank's, and the whole-job ms per unit (frame)
    is that time over all units of all ranks.  Returns (max total ms, ms
    per unit)."""
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


def pct(xs, q):
    s = sorted(xs)
    return s[min(len(s) - 1, int(q * len(s)))] if s else None


# ---------------------------------------------------------------------------
# the frame sequence (headline workload)
# ---------------------------------------------------------------------------

class Sequence:
    """The cloth-over-body frame sequence on the device: both meshes'
    coordinates in one packed buffer (restore / upload / download in one
    copy), the cloth's edge list built once, a context with the harmonic
    diffusion of Sec. 5 over RINGS rings."""

    def __init__(self, api, torch, dev, sc, dtype, **ctx_kw):
        import numpy as np
        self.api, self.torch, self.sc = api, torch, sc
        tdt = torch.float32 if dtype == np.float32 else torch.float64
        xyz = [torch.tensor(np.ascontiguousarray(m.V.astype(np.float32).astype(dtype)[:, c]), dtype=tdt,
                            device=dev) for m in (sc.A, sc.B) for c in range(3)]
        self.pos, self.pos0, v = packed(torch, xyz)
        self.ctx = api.Context(diffuse_rings=RINGS, **ctx_kw)
        self.ctx.hfcr_reserve(max(sc.A.n_verts, sc.B.n_verts), max(sc.A.n_tris, sc.B.n_tris), 1 << 18)
        ta, tb = torch.tensor(sc.A.T, device=dev), torch.tensor(sc.B.T, device=dev)
        # topology preparation (once per mesh): both edge lists, so that the
        # diffusion's vertex adjacency is built once and kept
        ea = torch.zeros((3 * sc.A.n_tris, 2), dtype=torch.int32, device=dev)
        ea = ea[:self.ctx.hfcr_build_edges(ta, sc.A.n_verts, ea)].contiguous()
        eb = torch.zeros((3 * sc.B.n_tris, 2), dtype=torch.int32, device=dev)
        eb = eb[:self.ctx.hfcr_build_edges(tb, sc.B.n_verts, eb)].contiguous()
        self.A = api.Mesh(*v[:3], ta, False, edges=ea)
        self.B = api.Mesh(*v[3:], tb, True, edges=eb)
        self.ne = int(ea.shape[0])
        self.ne_b = int(eb.shape[0])
        self.motion = sc.meta["motion"]
        self.params = self.motion.device_params(torch, dev)

    def restore(self):
        self.pos.copy_(self.pos0, non_blocking=True)

    def advance(self, f):
        self.motion.advance(self.torch, self.params, self.A.x, self.A.y, self.A.z, f)

    def load_from(self, other):
        self.pos.copy_(other.pos, non_blocking=True)   # widened when self is float64

    def resolve(self):
        return self.ctx.hfcr_resolve(self.A, self.B, D_POST, 1)

    def positions(self):
        import numpy as np
        P = self.pos.double().cpu().numpy()
        nA, nB = self.sc.A.n_verts, self.sc.B.n_verts
        return (np.stack([P[0:nA], P[nA:2 * nA], P[2 * nA:3 * nA]], 1),
                np.stack([P[3 * nA + i * nB:3 * nA + (i + 1) * nB] for i in range(3)], 1))

    def close(self):
        self.ctx.close()


def run_sequences(seq, torch, stream, flush, n_seq, n_frames, keep=None, on_frame=None):
    """n_seq passes of the whole sequence from the initial state; each
    frame's response timed with CUDA events on the launching stream, the L2
    flushed (256 MB write) before it, outside the timed interval.  Returns
    (per-frame ms of all passes, infos of the last pass)."""
    ms, infos = [], []
    for k in range(n_seq):
        seq.restore()
        evs = []
        last = []
        for f in range(n_frames):
            seq.advance(f)
            if keep is not None and k == n_seq - 1 and f in keep:
                keep[f] = seq.positions()
            flush.fill_(float(f))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = seq.resolve()
            e1.record(stream)
            evs.append((e0, e1))
            last.append(info)
            if on_frame is not None:
                on_frame(f)
        torch.cuda.synchronize()
        ms.extend(a.elapsed_time(b) for a, b in evs)
        infos = last
    return ms, infos


def frame_stats(infos):
    import numpy as np
    pairs = np.array([int(i.pairs_first) for i in infos])
    contact = np.nonzero(pairs > 0)[0]
    return {"first_contact_frame": int(contact[0]) if len(contact) else None,
            "contact_frames": int(len(contact)),
            "pairs_last_frame": int(pairs[-1]) if len(pairs) else 0,
            "max_pairs": int(pairs.max()) if len(pairs) else 0,
            "mean_pairs_contact_frames": round(float(pairs[contact].mean()), 1) if len(contact) else 0.0}


def lockstep_forms(api, torch, dev, sc, stream, flush, n_frames, drv):
    """The same frames through four forms: each frame the driver (mixed
    precision, graphs) moves the cloth; the float32 form without graphs,
    the plain float64 form (float64 positions = exact widening, float64
    filter -> exact, float64 CG per impact zone, plain launches) and the
    float64 form with one CTA's global CG load the driver's positions and
    run their response (timed, result discarded); then the driver runs its
    own (timed).  Splits the mixed form's gain into precision, solver
    structure and graph replay."""
    import numpy as np
    forms = {
        "mixed_no_graphs": Sequence(api, torch, dev, sc, np.float32, graphs=False),
        "fp64_per_zone": Sequence(api, torch, dev, sc, np.float64, solver=api.HFCR_SOLVER_FP64,
                                  f32_filter=False, graphs=False),
        "fp64_global_cg": Sequence(api, torch, dev, sc, np.float64,
                                   solver=api.HFCR_SOLVER_FP64_GLOBAL, f32_filter=False, graphs=False),
    }
    times = {k: [] for k in forms}
    times["mixed_graphs"] = []
    agree = {k: 0 for k in forms}
    drv.restore()
    for f in range(n_frames):
        drv.advance(f)
        for name, s in forms.items():
            s.load_from(drv)
            flush.fill_(float(f))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            inf = s.resolve()
            e1.record(stream)
            e1.synchronize()
            times[name].append(e0.elapsed_time(e1))
            agree[name] += int(inf.pairs_first)
        flush.fill_(float(f))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        inf = drv.resolve()
        e1.record(stream)
        e1.synchronize()
        times["mixed_graphs"].append(e0.elapsed_time(e1))
        for name in forms:
            agree[name] -= int(inf.pairs_first)
    for s in forms.values():
        s.close()
    mean = {k: statistics.mean(v) for k, v in times.items()}
    out = {k: {"ms_per_frame": round(mean[k], 4), "ms_p50": round(pct(times[k], 0.5), 4),
               "ms_p99": round(pct(times[k], 0.99), 4)} for k in times}
    out["fp64_per_zone"]["solver"] = "float64 CG per impact zone (one thread group per zone), float64 filter -> exact"
    out["fp64_global_cg"]["solver"] = "float64 CG of the whole system in one 1,024-thread CTA"
    out["pair_counts_identical"] = all(v == 0 for v in agree.values())
    out["factors"] = {
        "precision (fp64_per_zone / mixed_no_graphs)": round(mean["fp64_per_zone"] / mean["mixed_no_graphs"], 3),
        "solver structure (fp64_global_cg / fp64_per_zone)": round(mean["fp64_global_cg"] / mean["fp64_per_zone"], 3),
        "graph replay (mixed_no_graphs / mixed_graphs)": round(mean["mixed_no_graphs"] / mean["mixed_graphs"], 3),
        "plain fp64 form / headline (fp64_per_zone / mixed_graphs)": round(mean["fp64_per_zone"] / mean["mixed_graphs"], 3),
    }
    return out


def e2e_sequences(seq, torch, stream, n_seq, n_frames):
    """End to end through the C ABI with host buffers: every frame the
    cloth moves on the device (the simulator's state, untimed) and is read
    into a pinned host buffer; then, timed: the host -> device copy of both
    meshes' coordinates, the response, and the device -> host copy of the
    result."""
    host_in = torch.empty_like(seq.pos, device="cpu").pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    ms = []
    for _ in range(n_seq):
        seq.restore()
        for f in range(n_frames):
            seq.advance(f)
            host_in.copy_(seq.pos)           # synchronous: the state is on the host
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            seq.pos.copy_(host_in, non_blocking=True)
            seq.resolve()
            host_out.copy_(seq.pos, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
    return ms, host_in.numel() * host_in.element_size()


def oracle_frame(PA, TA, PB, TB, E, frac, offset=0):
    """The oracle on one frame of the cloth / body: brute-force exact
    detection of a stride sample of the cloth's edges against every body
    face, then stencils and the float64 response of what was found; both
    times scaled by 1 / frac to the whole edge list.  Returns (scaled
    seconds, seconds spent)."""
    import numpy as np
    import oracle
    step = max(1, int(round(1.0 / frac)))
    idx = np.arange(offset % step, len(E), step)
    sub = E[idx]
    t0 = time.perf_counter()
    hits = oracle.detect_one_direction(PA, sub, PB, TB)
    t1 = time.perf_counter()
    if len(hits):
        rec = np.zeros((len(hits), 4), np.uint32)
        rec[:, 1] = sub[hits[:, 0], 0]
        rec[:, 2] = sub[hits[:, 0], 1]
        rec[:, 3] = hits[:, 1]
        st = oracle.stencils(oracle.Pairs(rec, hits[:, 2].astype(np.int8)))
        dA, dB, _, _ = oracle.respond(st, PA, TA, PB, TB, D_POST)
        oracle.diffuse(dA, E, RINGS)
    t2 = time.perf_counter()
    f = len(idx) / len(E)
    return (t2 - t0) / f, t2 - t0


# ---------------------------------------------------------------------------
# the other configurations (extra keys)
# ---------------------------------------------------------------------------

def cloth_torus(api, torch, dev, stream, flush, steps, warmup, timed, cpu=True):
    """Cloth 200 x 200 (119,201 edges) draped into an oriented torus
    (65,536 faces), float32: one frame = one repair iteration from the
    initial positions (restored inside the timed region), graph-replayed;
    its stage profile, the rooflines of the traversal and of the per-zone
    solver, and the oracle on the same frame."""
    import numpy as np
    import meshgen
    sc = meshgen.scene_c2()
    xyz = [torch.tensor(np.ascontiguousarray(m.V.astype(np.float32)[:, c]), device=dev)
           for m in (sc.A, sc.B) for c in range(3)]
    pos, pos0, v = packed(torch, xyz)
    ctx = api.Context()
    ctx.hfcr_reserve(max(sc.A.n_verts, sc.B.n_verts), max(sc.A.n_tris, sc.B.n_tris), 1 << 16)
    ta, tb = torch.tensor(sc.A.T, device=dev), torch.tensor(sc.B.T, device=dev)
    ea = torch.zeros((3 * sc.A.n_tris, 2), dtype=torch.int32, device=dev)
    ne = ctx.hfcr_build_edges(ta, sc.A.n_verts, ea)
    ea = ea[:ne].contiguous()
    A = api.Mesh(*v[:3], ta, False, edges=ea)
    B = api.Mesh(*v[3:], tb, True)

    def frame():
        pos.copy_(pos0, non_blocking=True)
        return ctx.hfcr_resolve(A, B, D_POST, 1)

    variant, variant_ms = ctx.hfcr_autotune(A, B)
    ctx.hfcr_profile_enable(True)
    timed(frame, max(5, steps), 2)
    prof = ctx.hfcr_profile_read()
    ctx.hfcr_profile_enable(False)
    ms, infos = timed(frame, steps, warmup)
    info = infos[-1]
    n_prof = max(1, prof["traverse"][1])
    stage_ms = {k: round(val[0] / n_prof, 4) for k, val in prof.items()}
    P = int(info.pairs_first)
    peak, kind = measured_peak_hbm()
    trav_ms = prof["traverse"][0] / max(1, prof["traverse"][1])
    alg_trav = sc.A.n_verts * 12 + ne * 8 + sc.B.n_verts * 12 + sc.B.n_tris * 12 + P * 8
    # stencils and touched vertices of this frame's system (outside the timed regions)
    pos.copy_(pos0)
    cap = max(1 << 10, 2 * P)
    pbuf = torch.zeros((cap, 4), dtype=torch.int32, device=dev)
    n_p = ctx.hfcr_detect(A, B, pbuf)
    sbuf = torch.zeros((cap, 4), dtype=torch.int32, device=dev)
    k_st = ctx.hfcr_build_stencils(A, B, pbuf, n_p, sbuf)
    dxa = [torch.zeros(sc.A.n_verts, device=dev) for _ in range(3)]
    dxb = [torch.zeros(sc.B.n_verts, device=dev) for _ in range(3)]
    si = ctx.hfcr_respond(A, B, sbuf, k_st, D_POST, dxa, dxb)
    solve_ms = prof["solve"][0] / max(1, prof["solve"][1])
    # per stencil: ids 16 + float32 normal 16 + preconditioner row 16 + b 8 + float64
    # normal 32 + lam 8 (written) + 4 vertex-CSR entries 16 + group start 4; per
    # touched vertex: CSR offset 4 + inverse mass 4
    alg_cg = 116 * k_st + 8 * int(si.n_touched)
    out = {"workload": "cloth 200x200 (119,201 edges) vs torus 256x128 (65,536 faces), float32, one "
                       "repair iteration from the initial positions (restored inside the timed region)",
           "ms_per_frame": round(statistics.mean(ms), 4), "ms_p50": round(pct(ms, 0.5), 4),
           "ms_p99": round(pct(ms, 0.99), 4), "pairs": P, "stencils": int(info.total_stencils),
           "ef_tests_per_s_bruteforce": round(info.stats.brute_force_equiv / (statistics.mean(ms) / 1e3), 1),
           "stage_ms_per_frame": stage_ms, "traverse_variant": variant, "variant_ms": variant_ms,
           "rooflines": {
               "k_traverse": {"bound": "hbm", "achieved": round(alg_trav / (trav_ms * 1e-3) / 1e9, 2),
                              "peak": peak, "peak_kind": kind, "unit": "GB/s",
                              "frac": round(alg_trav / (trav_ms * 1e-3) / 1e9 / peak, 6),
                              "alg_bytes_per_launch": alg_trav, "avg_launch_ms": round(trav_ms, 5)},
               "k_cg_zone_pair": {"bound": "hbm", "achieved": round(alg_cg / (solve_ms * 1e-3) / 1e9, 3),
                                  "peak": peak, "peak_kind": kind, "unit": "GB/s",
                                  "frac": round(alg_cg / (solve_ms * 1e-3) / 1e9 / peak, 7),
                                  "traffic": profiled_traffic("k_cg_zone_pair"),
                                  "alg_bytes_per_launch": alg_cg, "avg_launch_ms": round(solve_ms, 5),
                                  "stencils": k_st, "touched_vertices": int(si.n_touched)}}}
    ctx.close()
    if cpu:
        import oracle
        PA, PB = sc.positions("A"), sc.positions("B")
        scaled, _ = oracle_frame_generic(PA, sc.A.T, PB, sc.B.T, oracle.edges(sc.A.T), 1.0)
        out["cpu_baseline"] = {"value": round(scaled * 1e3, 2), "unit": "ms/frame",
                               "cores": oracle.num_threads(), "kind": "oracle",
                               "sample": "one whole frame: brute-force exact detection of all 119,201 "
                                         "cloth edges against all 65,536 torus faces, stencils, float64 "
                                         "per-zone solve"}
    return out


def oracle_frame_generic(PA, TA, PB, TB, E, frac):
    import numpy as np
    import oracle
    step = max(1, int(round(1.0 / frac)))
    sub = E[::step]
    t0 = time.perf_counter()
    hits = oracle.detect_one_direction(PA, sub, PB, TB)
    t1 = time.perf_counter()
    rec = np.zeros((len(hits), 4), np.uint32)
    rec[:, 1] = sub[hits[:, 0], 0]
    rec[:, 2] = sub[hits[:, 0], 1]
    rec[:, 3] = hits[:, 1]
    st = oracle.stencils(oracle.Pairs(rec, hits[:, 2].astype(np.int8)))
    oracle.respond(st, PA, TA, PB, TB, D_POST)
    t2 = time.perf_counter()
    f = len(sub) / len(E)
    return (t1 - t0) / f + (t2 - t1), t2 - t0


def batched(api, torch, dev, steps, warmup, timed, cpu=True):
    """1,024 independent pairs of oriented icospheres (levels 1..5, 80 to
    20,480 faces each, random rotation, centre distance U(0.5, 1.8) radii),
    float32, concatenated into two meshes with a segment table.  A step is
    one repair iteration of every pair from the initial state
    (hfcr_resolve_batch, max_iters 1: detection of A-edges vs B-faces of
    all pairs, stencils, zones, solve, displacement)."""
    import numpy as np
    import meshgen
    scenes = meshgen.scene_c4()
    VA, TA, VB, TB, segs = meshgen.concat_batch(scenes)
    ctx = api.Context()
    ctx.hfcr_reserve(max(len(VA), len(VB)), max(len(TA), len(TB)), 1 << 21)
    xyz = [torch.tensor(np.ascontiguousarray(V.astype(np.float32)[:, c]), device=dev)
           for V in (VA, VB) for c in range(3)]
    ta, tb = torch.tensor(TA, device=dev), torch.tensor(TB, device=dev)
    ea = torch.zeros((3 * len(TA), 2), dtype=torch.int32, device=dev)
    ea = ea[:ctx.hfcr_build_edges(ta, len(VA), ea)].contiguous()
    eb = torch.zeros((3 * len(TB), 2), dtype=torch.int32, device=dev)
    eb = eb[:ctx.hfcr_build_edges(tb, len(VB), eb)].contiguous()
    pos, pos0, v = packed(torch, xyz)
    A = api.Mesh(*v[:3], ta, True, edges=ea)
    B = api.Mesh(*v[3:], tb, True, edges=eb)
    dsegs = torch.tensor(segs, device=dev)

    def step():
        pos.copy_(pos0, non_blocking=True)
        return ctx.hfcr_resolve_batch(A, B, dsegs, D_POST, 1)

    variant, variant_ms = ctx.hfcr_autotune(A, B, dsegs)
    ctx.hfcr_profile_enable(True)
    timed(step, max(3, steps // 2), 1)
    prof = ctx.hfcr_profile_read()
    ctx.hfcr_profile_enable(False)
    ms, infos = timed(step, steps, warmup)
    info = infos[-1]
    trav_ms, trav_n = prof["traverse"]
    P = int(info.pairs_first)
    alg = len(VA) * 12 + len(ea) * 8 + len(VB) * 12 + len(TB) * 12 + P * 8
    peak, kind = measured_peak_hbm()
    ach = alg / (trav_ms / max(1, trav_n) * 1e-3) / 1e9
    ctx.close()
    n_it = max(1, prof["traverse"][1])
    out = {"workload": "1,024 pairs of icospheres L1..5 (A: %d faces, B: %d faces), float32, "
                       "one batched repair iteration" % (len(TA), len(TB)),
           "ms_per_step": round(statistics.mean(ms), 4), "ms_p50": round(pct(ms, 0.5), 4),
           "pairs": P, "stencils": int(info.total_stencils),
           "ef_tests_per_s_bruteforce": round(info.stats.brute_force_equiv / (statistics.mean(ms) / 1e3), 1),
           "stage_ms_per_step": {k: round(val[0] / n_it, 4) for k, val in prof.items()},
           "roofline": {"kernel": "k_traverse", "bound": "hbm", "achieved": round(ach, 2),
                        "peak": peak, "peak_kind": kind, "unit": "GB/s", "frac": round(ach / peak, 5),
                        "traffic": profiled_traffic("k_traverse_batch"),
                        "alg_bytes_per_launch": alg, "avg_launch_ms": round(trav_ms / max(1, trav_n), 5),
                        "traverse_variant": variant, "variant_ms": variant_ms}}
    if cpu:
        # the oracle once per pair on a seeded sample of 24 pairs (direction 0,
        # as in the timed iteration), scaled by the brute-force candidates
        import oracle
        rng = np.random.default_rng(7)
        pick = rng.choice(len(scenes), 24, replace=False)
        bf_all = sum(len(oracle.edges(s.A.T)) * s.B.n_tris for s in scenes)
        bf_s, t_s = 0, 0.0
        for i in pick:
            s = scenes[i]
            PA = s.A.V.astype(np.float32).astype(np.float64)
            PB = s.B.V.astype(np.float32).astype(np.float64)
            t0 = time.perf_counter()
            pr = oracle.detect(PA, s.A.T, False, PB, s.B.T, True)
            st = oracle.stencils(pr)
            if len(st):
                oracle.respond(st, PA, s.A.T, PB, s.B.T, D_POST)
            t_s += time.perf_counter() - t0
            bf_s += len(oracle.edges(s.A.T)) * s.B.n_tris
        out["cpu_baseline"] = {"value": round(t_s * bf_all / bf_s * 1e3, 1), "unit": "ms/step",
                               "cores": oracle.num_threads(), "kind": "oracle",
                               "sample": "24 seeded pairs of the 1,024 (direction 0: detection, "
                                         "stencils, float64 response), scaled by |E| x |F| of all "
                                         "pairs over that of the sample"}
    return out


def small_form(api, torch, dev, steps, timed):
    """Two jittered level-3 icospheres offset by 1.5 (642 vertices, 1,280
    faces each), float64: one repair iteration from the initial state in
    the plain float64 form and the mixed form, and the whole repair loop
    (alternating roles) to convergence.  This size is bound by launch
    latency, so it is reported in microseconds."""
    import numpy as np
    import meshgen
    sc = meshgen.scene_c1()
    out = {"workload": "two icospheres L3 (1,280 faces each), offset 1.5, jitter 0.01, float64"}
    for name, solver, f32f, graphs in (("fp64_form", api.HFCR_SOLVER_FP64, False, False),
                                       ("mixed_form", api.HFCR_SOLVER_MIXED, True, True)):
        ctx = api.Context(solver=solver, f32_filter=f32f, graphs=graphs)
        ctx.hfcr_reserve(sc.A.n_verts, sc.A.n_tris, 1 << 14)
        xyz = [torch.tensor(np.ascontiguousarray(m.V[:, c]), dtype=torch.float64, device=dev)
               for m in (sc.A, sc.B) for c in range(3)]
        pos, pos0, v = packed(torch, xyz)
        A = api.Mesh(*v[:3], torch.tensor(sc.A.T, device=dev), True)
        B = api.Mesh(*v[3:], torch.tensor(sc.B.T, device=dev), True)

        def step():
            pos.copy_(pos0, non_blocking=True)
            return ctx.hfcr_resolve(A, B, D_POST, 1)

        ms, infos = timed(step, steps, 3)
        out[name] = {"us_per_iteration": round(1e3 * statistics.median(ms), 1),
                     "pairs": int(infos[-1].pairs_first)}
        if solver == api.HFCR_SOLVER_MIXED:
            def loop():
                pos.copy_(pos0, non_blocking=True)
                return ctx.hfcr_resolve(A, B, D_POST, 64)
            lms, linfo = timed(loop, max(3, steps // 10), 1)
            out["repair_loop"] = {"ms": round(statistics.median(lms), 3),
                                  "detections": int(linfo[-1].iters),
                                  "converged": bool(linfo[-1].converged)}
        ctx.close()
    return out


def precision_form(api, torch, dev, steps, timed, d_values=(1e-4, 3e-4, 1e-3, 3e-3, 1e-2),
                   max_iters=32):
    """Two 262,144-face tori, float32, a seeded local overlap: one repair
    iteration (float32 filter -> float64 -> exact; float32 CG + float64
    refinement) timed from the initial state; the float32 solver's
    displacement error against the float64 GPU solver on the same
    stencils; and the d-sweep (Eq. 8: each d resolved with the harmonic
    diffusion, at most max_iters detections).  For each d, the signed
    distance D' of every first-response stencil's x0 from its face (Eq. 1)
    right after the first response, where Eq. 8 makes it d up to the
    linearisation of the normals, and again at the end of the loop."""
    import numpy as np
    import meshgen
    sc = meshgen.scene_c3()
    xyz = [torch.tensor(np.ascontiguousarray(m.V[:, c].astype(np.float32)), device=dev)
           for m in (sc.A, sc.B) for c in range(3)]
    pos, pos0, v = packed(torch, xyz)
    A = api.Mesh(*v[:3], torch.tensor(sc.A.T, device=dev), True)
    B = api.Mesh(*v[3:], torch.tensor(sc.B.T, device=dev), True)
    cap = 1 << 20
    ctx = api.Context()
    ctx.hfcr_reserve(sc.A.n_verts, sc.A.n_tris, cap)
    variant, _ = ctx.hfcr_autotune(A, B)

    def step():
        pos.copy_(pos0, non_blocking=True)
        return ctx.hfcr_resolve(A, B, D_POST, 1)

    ms, infos = timed(step, steps, 3)
    info = infos[-1]
    pos.copy_(pos0)
    pairs = torch.zeros((cap, 4), dtype=torch.int32, device=dev)
    n = ctx.hfcr_detect(A, B, pairs)
    st = torch.zeros((cap, 4), dtype=torch.int32, device=dev)
    k = ctx.hfcr_build_stencils(A, B, pairs, n, st)
    ctx64 = api.Context(solver=api.HFCR_SOLVER_FP64)
    ctx64.hfcr_reserve(sc.A.n_verts, sc.A.n_tris, cap)
    A64 = api.Mesh(*[t.double() for t in xyz[:3]], A.tris, True)
    B64 = api.Mesh(*[t.double() for t in xyz[3:]], B.tris, True)
    dx = {}
    for name, c in (("mixed", ctx), ("fp64", ctx64)):
        da = [torch.zeros(sc.A.n_verts, dtype=torch.float64, device=dev) for _ in range(3)]
        db = [torch.zeros(sc.B.n_verts, dtype=torch.float64, device=dev) for _ in range(3)]
        si = c.hfcr_respond(A64, B64, st, k, D_POST, da, db)
        dx[name] = (torch.cat([torch.stack(da, 1), torch.stack(db, 1)]), si)
    err = float((dx["mixed"][0] - dx["fp64"][0]).abs().max() / dx["fp64"][0].abs().max())
    ctx64.close()
    ctx.close()
    stn = st[:k, :3].cpu().numpy().astype(np.int64)

    def gaps(d, dirs=(0, 1)):
        PA = torch.stack([A.x, A.y, A.z], 1).double().cpu().numpy()
        PB = torch.stack([B.x, B.y, B.z], 1).double().cpu().numpy()
        sel = stn[np.isin(stn[:, 0], dirs)]
        m0 = sel[:, 0] == 0
        x0 = np.empty((len(sel), 3))
        tri = np.empty((len(sel), 3, 3))
        x0[m0], tri[m0] = PA[sel[m0, 1]], PB[sc.B.T[sel[m0, 2]]]
        x0[~m0], tri[~m0] = PB[sel[~m0, 1]], PA[sc.A.T[sel[~m0, 2]]]
        nrm = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
        ln = np.linalg.norm(nrm, axis=1)
        ok = ln > 0
        Dp = np.einsum("ij,ij->i", nrm[ok] / ln[ok, None], x0[ok] - tri[ok].mean(axis=1)) / d
        return {"min": round(float(Dp.min()), 4), "p05": round(float(np.percentile(Dp, 5)), 4),
                "median": round(float(np.median(Dp)), 4), "p95": round(float(np.percentile(Dp, 95)), 4),
                "max": round(float(Dp.max()), 4)}

    sweep = []
    for d in d_values:
        # the first response alone, without diffusion (Eq. 8 on the stencils
        # of the initial positions; roles alternate, so the first iteration
        # responds to the direction-0 stencils)
        c1 = api.Context()
        c1.hfcr_reserve(sc.A.n_verts, sc.A.n_tris, cap)
        pos.copy_(pos0)
        c1.hfcr_resolve(A, B, d, 1)
        first = gaps(d, (0,))
        c1.close()
        c2 = api.Context(diffuse_rings=RINGS)
        c2.hfcr_reserve(sc.A.n_verts, sc.A.n_tris, cap)
        pos.copy_(pos0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = c2.hfcr_resolve(A, B, d, max_iters)
        e1.record()
        e1.synchronize()
        sweep.append({"d": d, "converged": bool(r.converged), "detections": int(r.iters),
                      "pairs_first": int(r.pairs_first), "ms": round(e0.elapsed_time(e1), 3),
                      "gap_over_d_after_first_response": first,
                      "gap_over_d_after_loop": gaps(d)})
        c2.close()
    return {"workload": "two tori 512x256 quads (262,144 faces each), float32, local overlap "
                        "depth U(0, 0.2 r); one repair iteration from the initial state",
            "ms_p50": round(pct(ms, 0.5), 4), "ms_mean": round(statistics.mean(ms), 4),
            "pairs": int(info.pairs_first), "stencils": int(k),
            "filter": {"narrow_tests": int(info.stats.narrow_tests),
                       "f64_fallbacks": int(info.stats.f64_fallbacks),
                       "exact_fallbacks": int(info.stats.exact_fallbacks)},
            "dx_rel_err_vs_fp64_solver": err,
            "mixed_solver": {"cg_iters": int(dx["mixed"][1].cg_iters),
                             "rel_residual": dx["mixed"][1].rel_residual},
            "traverse_variant": variant,
            "d_sweep": {"diffusion": {"rings": RINGS, "field": "harmonic"}, "max_iters": max_iters,
                        "stencils": "after the first response: its direction-0 stencils; after "
                                    "the loop: the stencils of both directions at the initial "
                                    "positions", "runs": sweep}}


# ---------------------------------------------------------------------------
# the reference arm: the CPU oracle
# ---------------------------------------------------------------------------

def run_reference(args, ws, rank):
    """The CPU oracle as the reference arm (rank 0 only), on the headline
    workload: frame 0 of the sequence (the cloth moved once by the motion
    field; before the first contact, so the frame is the detection alone).
    Each step is a stride sample of the cloth edges sized so that warmup +
    steps take about --ref-budget seconds, scaled to the whole frame."""
    if rank != 0:
        return
    import numpy as np
    import meshgen
    import oracle
    sc = meshgen.scene_c5()
    mot = sc.meta["motion"]
    PA = sc.A.V.astype(np.float32)
    PA = (PA + mot.velocity(PA.astype(np.float64), 0).astype(np.float32)).astype(np.float64)
    PB = sc.B.V.astype(np.float32).astype(np.float64)
    E = oracle.edges(sc.A.T)
    # calibration on 1/500 of the edges
    cal, spent = oracle_frame(PA, sc.A.T, PB, sc.B.T, E, 1 / 500)
    n = max(1, args.steps + args.warmup)
    frac = min(1.0, max(1 / 2000, args.ref_budget / n / max(1e-9, cal)))
    for w in range(args.warmup):
        oracle_frame(PA, sc.A.T, PB, sc.B.T, E, frac, w)
    times = []
    for s in range(args.steps):
        scaled, _ = oracle_frame(PA, sc.A.T, PB, sc.B.T, E, frac, s)
        times.append(scaled * 1e3)
    ms = statistics.mean(times)
    bf = len(E) * sc.B.n_tris
    step = max(1, int(round(1.0 / frac)))
    which = "all" if step == 1 else f"one in {step} of the"
    sample = (f"frame 0 of the 512x512 cloth / level-7 body sequence (before the first contact): "
              f"brute-force exact detection of {which} cloth edges against all 327,680 body "
              f"faces per step, scaled to all 784,385 edges")
    line = {"metric": METRIC, "value": round(ms, 3), "unit": "ms/frame", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "cloth 512x512 (784,385 edges) over SH body (icosphere L7, "
                                   "327,680 faces), float32 positions, one DCD response per frame",
                       "l2": "n/a (CPU)"},
            "ef_tests_per_s_bruteforce": bf / (ms / 1e3),
            "cpu_baseline": {"value": round(ms, 3), "unit": "ms/frame", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(ms, 3), "unit": "ms/frame", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# profiling runs (for ncu: --nvtx --nvtx-include "profile/")
# ---------------------------------------------------------------------------

def run_profile(case, api, torch, dev, stream):
    """One call of a bench workload inside the NVTX range 'profile', after
    the same warm-up the bench gives it (autotuner, earlier frames); prints
    one JSON line describing the profiled call."""
    import numpy as np
    import meshgen
    out = {"profile": case}
    if case.startswith("frame:"):
        target = int(case.split(":", 1)[1])
        sc = meshgen.scene_c5()
        seq = Sequence(api, torch, dev, sc, np.float32)
        out["traverse_variant"], _ = seq.ctx.hfcr_autotune(seq.A, seq.B)
        seq.restore()
        for f in range(target + 1):
            seq.advance(f)
            if f == target:
                torch.cuda.synchronize()
                torch.cuda.nvtx.range_push("profile")
            info = seq.resolve()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        seq.close()
    elif case in ("cloth_torus", "batch"):
        if case == "cloth_torus":
            sc = meshgen.scene_c2()
            VA, TA, VB, TB, segs = sc.A.V, sc.A.T, sc.B.V, sc.B.T, None
            oriented_a = False
        else:
            VA, TA, VB, TB, segs = meshgen.concat_batch(meshgen.scene_c4())
            oriented_a = True
        ctx = api.Context()
        ctx.hfcr_reserve(max(len(VA), len(VB)), max(len(TA), len(TB)), 1 << (21 if segs is not None else 16))
        xyz = [torch.tensor(np.ascontiguousarray(V.astype(np.float32)[:, c]), device=dev)
               for V in (VA, VB) for c in range(3)]
        ta, tb = torch.tensor(TA, device=dev), torch.tensor(TB, device=dev)
        ea = torch.zeros((3 * len(TA), 2), dtype=torch.int32, device=dev)
        ea = ea[:ctx.hfcr_build_edges(ta, len(VA), ea)].contiguous()
        pos, pos0, v = packed(torch, xyz)
        A = api.Mesh(*v[:3], ta, oriented_a, edges=ea)
        if segs is not None:
            eb = torch.zeros((3 * len(TB), 2), dtype=torch.int32, device=dev)
            eb = eb[:ctx.hfcr_build_edges(tb, len(VB), eb)].contiguous()
            B = api.Mesh(*v[3:], tb, True, edges=eb)
            dsegs = torch.tensor(segs, device=dev)
            out["traverse_variant"], _ = ctx.hfcr_autotune(A, B, dsegs)
            call = lambda: ctx.hfcr_resolve_batch(A, B, dsegs, D_POST, 1)
        else:
            B = api.Mesh(*v[3:], tb, True)
            out["traverse_variant"], _ = ctx.hfcr_autotune(A, B)
            call = lambda: ctx.hfcr_resolve(A, B, D_POST, 1)
        for _ in range(3):
            pos.copy_(pos0, non_blocking=True)
            call()
        pos.copy_(pos0, non_blocking=True)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("profile")
        info = call()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        ctx.close()
    else:
        raise SystemExit(f"unknown profile case {case!r}")
    out.update(pairs=int(info.pairs_first), stencils=int(info.total_stencils),
               cg_iters=int(info.cg_iters), solver_path=int(info.solver_path),
               diffuse_cg_iters=int(info.diffuse_cg_iters))
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------

def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import numpy as np
    import torch
    import meshgen
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
    if args.profile:
        run_profile(args.profile, api, torch, dev, stream)
        return
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    F = args.frames

    def timed(fn, K, W):
        for _ in range(W):
            fn()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(K)]
        infos = []
        for i in range(K):
            flush.fill_(float(i))          # L2 flush between steps (not timed)
            evs[i][0].record(stream)
            infos.append(fn())
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs], infos

    # ---- headline: the frame sequence, mixed form, graphs ----
    sc = meshgen.scene_c5()
    seq = Sequence(api, torch, dev, sc, np.float32)
    variant, variant_ms = seq.ctx.hfcr_autotune(seq.A, seq.B)
    keep = {0: None, F // 2 - 1: None, F - 1: None}
    run_sequences(seq, torch, stream, flush, max(1, args.warmup), F, keep=keep)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    launches0 = api.hfcr_launch_count()
    sampler = ClockSampler(local)
    sampler.start()
    t_wall = time.perf_counter()
    ms, infos = run_sequences(seq, torch, stream, flush, args.steps, F)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    launches = api.hfcr_launch_count() - launches0
    if pg:
        pg.barrier()
    total_ms, per_frame = whole_job(sum(ms), args.steps * F, pg, dev)
    fstats = frame_stats(infos)
    bf_frame = seq.ne * sc.B.n_tris
    narrow = statistics.mean(int(i.stats.narrow_tests) for i in infos)
    # per-frame record of the last timed sequence: the slowest frames and why
    last = ms[-F:]
    order = sorted(range(F), key=lambda f: -last[f])
    slow = [{"frame": f, "ms": round(last[f], 4), "pairs": int(infos[f].pairs_first),
             "stencils": int(infos[f].total_stencils), "cg_iters": int(infos[f].cg_iters),
             "solver_path": int(infos[f].solver_path),
             "diffuse_cg_iters": int(infos[f].diffuse_cg_iters),
             "band_vertices": int(infos[f].band_vertices)} for f in order[:6]]
    if args.frame_log:
        with open(args.frame_log, "w") as fh:
            fh.write("frame,ms,pairs,stencils,cg_iters,solver_path,diffuse_cg_iters,band_vertices\n")
            for f in range(F):
                i = infos[f]
                fh.write(f"{f},{last[f]:.5f},{i.pairs_first},{i.total_stencils},{i.cg_iters},"
                         f"{i.solver_path},{i.diffuse_cg_iters},{i.band_vertices}\n")

    # profiled pass: CUDA events around every stage (plain launches)
    seq.ctx.hfcr_profile_enable(True)
    pms, _ = run_sequences(seq, torch, stream, flush, 1, F)
    prof = seq.ctx.hfcr_profile_read()
    seq.ctx.hfcr_profile_enable(False)
    stage_ms = {k: round(v[0] / F, 4) for k, v in prof.items()}
    peak, peak_kind = measured_peak_hbm()
    # rooflines: the traversal (one launch per frame) and the harmonic
    # diffusion's band CG; algorithmic bytes = compulsory reads + writes
    trav_ms = prof["traverse"][0] / max(1, prof["traverse"][1])
    P_mean = statistics.mean(int(i.pairs_first) for i in infos)
    alg_trav = int(sc.A.n_verts * 12 + seq.ne * 8 + sc.B.n_verts * 12 + sc.B.n_tris * 12 + P_mean * 8)
    ach_trav = alg_trav / (trav_ms * 1e-3) / 1e9
    frame_bytes = (sc.A.n_verts + sc.B.n_verts) * 12 * 2 + seq.ne * 8 + sc.B.n_tris * 12
    # the band CG (one cluster launch per frame): compulsory bytes per free band
    # vertex = its index 4 + CSR offsets 8 + neighbour ids 4 x degree + the
    # field read 24 and written 24 (float64 xyz); the iterations' records
    # stay on chip / in L2 and are not compulsory
    band_ms = prof["band_cg"][0] / max(1, prof["band_cg"][1])
    nb_mean = statistics.mean(int(i.band_vertices) for i in infos)
    deg = 2.0 * (seq.ne + seq.ne_b) / (sc.A.n_verts + sc.B.n_verts)
    alg_band = int(nb_mean * (60 + 4 * deg))
    band_iters = statistics.mean(int(i.diffuse_cg_iters) for i in infos)
    ach_band = alg_band / (band_ms * 1e-3) / 1e9
    # the solver launches of the large impact zones (1,024 rows or more: the
    # frame's big contact zone, and the few medium zones beside it): per row
    # 116 B (ids, float32 and float64 normals, block-Jacobi row, b, lambda
    # written, four CSR entries, group start), per touched vertex 8 B
    zb_ms = prof["zone_big"][0] / max(1, prof["zone_big"][1])
    zb_rows = statistics.mean(int(i.big_zone_rows) for i in infos)
    zb_verts = statistics.mean(int(i.big_zone_vertices) for i in infos)
    alg_zb = int(116 * zb_rows + 8 * zb_verts)
    ach_zb = alg_zb / (zb_ms * 1e-3) / 1e9
    roof = {
        "k_traverse": {"kernel": "k_traverse (BVH traversal + exact narrow phase)", "bound": "hbm",
                       "achieved": round(ach_trav, 2), "peak": peak, "peak_kind": peak_kind,
                       "unit": "GB/s", "frac": round(ach_trav / peak, 5),
                       "traffic": profiled_traffic("k_traverse"), "alg_bytes_per_launch": alg_trav,
                       "avg_launch_ms": round(trav_ms, 5), "launches_timed": prof["traverse"][1]},
        "k_band_cl": {"kernel": "k_band_cl (harmonic diffusion: CG on the band Laplacian on one "
                                "thread-block cluster; k_band_cg, the grid-wide form, takes bands "
                                "beyond the cluster's capacity)", "bound": "hbm",
                      "achieved": round(ach_band, 3), "peak": peak, "peak_kind": peak_kind,
                      "unit": "GB/s", "frac": round(ach_band / peak, 7),
                      "traffic": profiled_traffic("k_band_cl"), "alg_bytes_per_launch": alg_band,
                      "avg_launch_ms": round(band_ms, 5), "launches_timed": prof["band_cg"][1],
                      "band_vertices_mean": round(nb_mean, 1), "cg_iters_mean": round(band_iters, 2),
                      "us_per_cg_iter": round(1e3 * band_ms / band_iters, 3) if band_iters else None},
        "k_cg_zone_big": {"kernel": "k_cg_zone<512> (+ k_cg_zone_cl): float32 PCG with float64 "
                                    "refinement of the impact zones of 1,024 rows or more (and of at "
                                    "most eight medium zones beside them), one CTA (or cluster) "
                                    "per zone", "bound": "hbm",
                          "achieved": round(ach_zb, 3), "peak": peak, "peak_kind": peak_kind,
                          "unit": "GB/s", "frac": round(ach_zb / peak, 7),
                          "traffic": profiled_traffic("k_cg_zone_big"), "alg_bytes_per_launch": alg_zb,
                          "avg_launch_ms": round(zb_ms, 5), "launches_timed": prof["zone_big"][1],
                          "rows_mean": round(zb_rows, 1), "vertices_mean": round(zb_verts, 1)},
        "whole_frame": {"bound": "hbm", "alg_bytes_per_frame": frame_bytes,
                        "achieved": round(frame_bytes / (per_frame * 1e-3) / 1e9, 2), "peak": peak,
                        "unit": "GB/s", "frac": round(frame_bytes / (per_frame * 1e-3) / 1e9 / peak, 5),
                        "note": "positions of both meshes read and written, cloth edges, body faces"},
    }
    # the headline roofline: the single kernel with the most time per frame
    # in the profiled pass (the traversal, the band CG, the large-zone solver)
    kernel_ms = {"k_traverse": prof["traverse"][0] / F, "k_band_cl": prof["band_cg"][0] / F,
                 "k_cg_zone_big": prof["zone_big"][0] / F}
    top = max(kernel_ms, key=kernel_ms.get)
    roofline = dict(roof[top], ms_per_frame=round(kernel_ms[top], 4),
                    chosen_by="the kernel with the most time per frame of %s (profiled pass, "
                              "ms/frame %s)" % (sorted(kernel_ms),
                                                {k: round(v, 4) for k, v in kernel_ms.items()}))

    # ---- the same frames through the other forms ----
    forms = None if args.no_forms else lockstep_forms(api, torch, dev, sc, stream, flush, F, seq)

    # ---- end to end through the C ABI with host buffers ----
    n_e2e = max(2, args.steps // 4)
    e2e_ms, io_bytes = e2e_sequences(seq, torch, stream, n_e2e, F)
    e2e_total, e2e_per_frame = whole_job(sum(e2e_ms), n_e2e * F, pg, dev)
    seq.close()

    extra = {}
    if not args.no_extra:
        extra["cloth_torus"] = cloth_torus(api, torch, dev, stream, flush, 20, 5, timed,
                                           cpu=rank == 0 and not args.no_cpu_baseline)
        extra["precision_form"] = precision_form(api, torch, dev, 5, timed)
        extra["small_form"] = small_form(api, torch, dev, 10, timed)
        extra["batch"] = batched(api, torch, dev, 5, 2, timed,
                                 cpu=rank == 0 and not args.no_cpu_baseline)

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            import oracle
            E = oracle.edges(sc.A.T)
            vals, spent = [], 0.0
            for i, f in enumerate(sorted(keep)):
                PA, PB = keep[f]
                scaled, s_ = oracle_frame(PA, sc.A.T, PB, sc.B.T, E, 1 / 3, i)
                vals.append(scaled)
                spent += s_
            cpu = {"value": round(1e3 * statistics.mean(vals), 1), "unit": "ms/frame",
                   "cores": oracle.num_threads(), "kind": "oracle",
                   "sample": "frames %s of the sequence (the GPU's positions before each frame's "
                             "response): brute-force exact detection of every third cloth edge "
                             "against all 327,680 body faces, stencils, float64 response and "
                             "harmonic diffusion of what was found, scaled by 3; %.1f s of CPU "
                             "work" % (sorted(keep), spent),
                   "per_frame_ms": [round(1e3 * v, 1) for v in vals]}
        line = {
            "metric": METRIC, "value": round(per_frame, 4), "unit": "ms/frame",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "frame sequence: cloth 512x512 (784,385 edges, float32, "
                                   "un-oriented) over an oriented SH body (icosphere L7, 327,680 "
                                   "faces); %d frames per step, one DCD response per frame "
                                   "(detection, stencils, Eq. 8 solve, harmonic diffusion R=%d), "
                                   "CUDA-graph replay" % (F, RINGS),
                       "frames_per_step": F,
                       "predicates": "float32 semi-static filter -> float64 filter -> exact integers",
                       "solver": "float32 CG + float64 iterative refinement to 1e-12 per impact zone",
                       "diffusion": "harmonic field: float64 CG on the band Laplacian to 1e-10",
                       "l2": "flushed before every frame (256 MB write, outside the timed interval)",
                       "parallelism": f"replicas x{ws}"},
            "ms_p50": round(pct(ms, 0.5), 4), "ms_p99": round(pct(ms, 0.99), 4),
            "frames": fstats,
            "slowest_frames": slow,
            "ef_tests_per_s_bruteforce": round(bf_frame / (per_frame / 1e3), 1),
            "ef_tests_per_s_executed": round(narrow / (per_frame / 1e3), 1),
            "stage_ms_per_frame": stage_ms,
            "profiled_ms_per_frame": round(statistics.mean(pms), 4),
            "traverse_variant": variant, "variant_ms": variant_ms,
            "graphs": True,
            "roofline": roofline,
            "rooflines": roof,
            "e2e": {"value": round(e2e_per_frame, 4), "unit": "ms/frame",
                    "h2d_bytes_per_step": io_bytes * F, "d2h_bytes_per_step": io_bytes * F,
                    "h2d_bytes_per_frame": io_bytes, "d2h_bytes_per_frame": io_bytes,
                    "steps": n_e2e},
            "forms_same_frames": forms,
            "gpu_launches": launches,
            "timed_wall_s": round(t_wall, 2),
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
