#!/usr/bin/env python3
"""Benchmark of one dynamic frame of the voxel ray-tracing path.

Workload (default): tractography-like bundles -- 100k streamlines x 100
vertices (9.9M segments) in 30 bundles inside an ellipsoid, 256^3 grid, tube
radius 0.35 voxel, 1920x1080 perspective camera, opacity 0.3 with full ordered
compositing, culling on; each frame 5% of the streamlines are replaced
(interactive filtering). A step = update of the replaced vertices + ingest +
voxelize pass 1 + mips + cull marks + scan + pass 2 + trace (+ repair rounds).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload bundles|walks|abc]

Prints ONE JSON line (rank 0). Under torchrun each rank renders its own replica
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms/frame (voxelize+cull+trace) at 1080p, 10M segs; p50/p99 served-frame latency"
FALLBACK_HBM_GBS = 6800.0


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------- workloads
def orbit(cam, deg):
    """cam turned by deg about the vertical axis through its target."""
    a = np.deg2rad(deg)
    e = np.array(cam.eye, np.float64) - np.array(cam.target, np.float64)
    e = np.array([e[0] * np.cos(a) - e[1] * np.sin(a), e[0] * np.sin(a) + e[1] * np.cos(a), e[2]])
    return dataclasses.replace(cam, eye=tuple(float(v) for v in np.array(cam.target) + e))


def make_workload(name, scale=1.0):
    from gen import linesets as G
    if name == "bundles":
        bs = G.bundles(n_lines=int(round(100_000 * scale)))
        cam = G.bundles_camera()
        upd = lambda f: G.bundles_update(bs, f)  # noqa: E731
        return dict(ls=bs.lineset, cam=cam, update=upd, alpha=0.3, ao=0, cull=1,
                    desc=("tractography-like bundles: 100k streamlines x 100 vertices "
                          "(9.9M segments), 30 bundles, grid 256^3, r 0.35, 1920x1080 "
                          "perspective, alpha 0.3 ordered compositing, culling on, 5% of "
                          "streamlines replaced per frame"))
    if name == "walks":
        ls = G.tiny_walks()
        cam = G.tiny_walks_camera()
        rng = np.random.default_rng(7)

        def upd(f):
            k = ls.n_vertices // 20
            first = (f * k) % (ls.n_vertices - k)
            return first, (ls.xyz[first:first + k] + rng.normal(0, 0.05, (k, 3))).astype(np.float32)
        return dict(ls=ls, cam=cam, update=upd, alpha=1.0, ao=0, cull=0,
                    desc="random walks: 2000 x 50 vertices, grid 64^3, r 0.4, 256x256 ortho, opaque")
    if name == "abc":
        npart = int(round(1_000_000 * scale))
        ls = G.abc_pathlines(n_particles=npart, frame=0)
        cam = G.abc_camera(frame=0)

        def upd(f):
            nl = G.abc_pathlines(n_particles=npart, frame=f + 1)
            return 0, nl.xyz
        return dict(ls=ls, cam=cam, update=upd, alpha=1.0, ao=6, cull=1,
                    desc=("ABC-flow lines: 1M x 32 vertices (31M segments), grid 512^3, r 0.25, "
                          "1920x1080 perspective from the centre, opaque, 6-cone AO, culling on, "
                          "every vertex moves per frame"))
    if name == "sparse":
        # the serving mix's heaviest request: its largest set (random walks of
        # 20-200 vertices, 512^3) seen at 4K and opacity 0.2
        rng = np.random.default_rng(20251013)
        sizes = np.exp(rng.uniform(np.log(1e4), np.log(5e6), 64)).astype(np.int64)
        k = int(np.argmax(sizes))
        ls = G.walk_set(int(round(int(sizes[k]) * scale)), 512, radius=0.4, seed=20251100 + 7 * k)
        c = 256.0
        cam = G.Camera(width=3840, height=2160, ortho=0, eye=(c + 1.7 * 512, c, c + 0.5 * 512),
                       target=(c, c, c), up=(0.0, 0.0, 1.0), fovy_deg=45.0)
        rng2 = np.random.default_rng(11)

        def upd(f):
            cnt = ls.n_vertices // 50
            first = (f * cnt) % (ls.n_vertices - cnt)
            return first, np.clip(ls.xyz[first:first + cnt] + rng2.normal(0, 0.05, (cnt, 3)), 1.0,
                                  511.0).astype(np.float32)
        return dict(ls=ls, cam=cam, update=upd, alpha=0.2, ao=0, cull=2,
                    desc=("sparse random walks: the serving mix's largest set (%d segments, "
                          "20-200 vertices per walk), grid 512^3, r 0.4, 3840x2160 perspective, "
                          "alpha 0.2 ordered compositing, automatic culling, 2%% of vertices "
                          "moved per frame" % ls.n_segments))
    raise SystemExit(f"unknown workload {name}")


# ------------------------------------------------------------------ clocks
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        self.f.flush()
        try:
            rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        except Exception:
            rows = []
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- roofline
def stage_bytes(stage, n, V, st, px, tw=None, mips=False):
    """Algorithmic (compulsory) DRAM bytes of one frame's stage: what the method
    must move, not what the kernels happen to move. V vertices, n^3 voxels,
    F_vis listed fragments, px pixels; the trace's share counts the distinct
    list entries (4 B), vertices (16 B) and voxel words (8 B: packed word and
    list end) its rays read, measured by the instrumented trace (tw)."""
    N3 = n ** 3
    Fv = st["fragments_listed"]
    tw = tw or {}
    return {
        "ingest": 0,                                     # folded into pass 1's vertex read
        "pass1": 16 * V + 8 * N3,                        # float4 vertices in; grid cleared + written back
        "mips": (4 * N3 + 4 * N3 // 7) if mips else 0,   # level 0 in, levels >= 1 out
        "cull": 4 * N3 + N3 // 7,                        # words in (with erosion halo), marks + OR pyramid out
        "scan": 4 * N3 + 4 * N3,                         # counts in, offsets out
        "pass2": 16 * V + 4 * Fv + 4 * N3,               # vertices in, list entries + cursors out
        "trace": (24 * px + 4 * tw.get("unique_entries", 0) + 16 * tw.get("unique_vertices", 0)
                  + 8 * tw.get("unique_voxels", 0)),     # outputs + what the rays read
        "repair": 0,
        "shade": 4 * N3 + N3 // 8 + N3 // 8,             # words + marks read, field mask written
    }[stage]


# The trace kernel is bound by instruction issue and latency, not by DRAM: its
# roofline counts the method's FP32 work, one ray-capsule entry test per list
# entry a ray examines, against the FP32 rate of the SMs.
SHADING_LIGHT = (0.4, 0.5, 0.77)  # direction toward the light for --shading voxel
TRACE_FLOPS_PER_ENTRY = 82        # FP32 operations of one capsule entry test
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
TRACE_SOURCES = ("paper_2510_09081_gb300/csrc/trace.cu", "paper_2510_09081_gb300/csrc/vrt_internal.cuh",
                 "paper_2510_09081_gb300/csrc/launch.h", "paper_2510_09081_gb300/csrc/pyramid.cuh")
TRACE_PROFILE = os.path.join(ROOT, "profiles", "k_trace_tile_bundles_traffic.md")


def trace_source_hash():
    h = hashlib.sha256()
    for f in TRACE_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def trace_traffic():
    """DRAM bytes per launch of the trace kernel from the committed ncu summary,
    or None when the kernel's sources changed since it was captured."""
    try:
        fields = {}
        for line in open(TRACE_PROFILE):
            if ":" in line and line.startswith("- "):
                k, v = line[2:].split(":", 1)
                fields[k.strip()] = v.strip().strip("`")
        if fields.get("source_hash") != trace_source_hash():
            return None
        return int(fields["traffic_bytes_per_launch"])
    except Exception:
        return None


def hbm_peak():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------ cpu baseline
def cpu_baseline(wl, budget_s=20.0):
    """The CPU oracle, as it stands, on a bounded sample of the same workload:
    lists for a 1% sample of the polylines (scaled x100) plus the render of every
    64th pixel of that sampled scene (scaled x64)."""
    import oracle
    from gen.linesets import LineSet
    ls = wl["ls"]
    P = ls.n_polylines
    step = 100 if P >= 1000 else 1
    keep = np.arange(0, P, step)
    lens = np.diff(ls.offsets)[keep]
    starts = ls.offsets[keep]
    xyz = np.concatenate([ls.xyz[s:s + l] for s, l in zip(starts, lens)], 0)
    sub = LineSet(xyz=xyz, offsets=np.concatenate([[0], np.cumsum(lens)]), n=ls.n, radius=ls.radius)
    cores = os.cpu_count() or 1
    o = oracle.Oracle.from_lineset(sub, nthreads=cores)
    t0 = time.perf_counter()
    o.build_lists()
    t_lists = time.perf_counter() - t0
    cam = wl["cam"]
    npx = cam.width * cam.height
    pstep = 64
    t0 = time.perf_counter()
    done = 0
    # render whole rows, every 64th row, to keep the sample spatially spread
    for row in range(0, cam.height, pstep):
        o.render(cam, alpha=wl["alpha"], ao_cones=wl["ao"], pix_begin=row * cam.width,
                 pix_end=(row + 1) * cam.width)
        done += cam.width
        if time.perf_counter() - t0 > budget_s:
            break
    t_render = time.perf_counter() - t0
    ms = 1e3 * (t_lists * step + t_render * npx / max(done, 1))
    out = {"value": ms, "unit": "ms/frame", "cores": cores, "kind": "oracle",
           "sample": (f"extrapolated from a bounded sample: the list build of every {step}th "
                      f"polyline ({sub.n_segments} segments, timed, x{step}) plus the render of "
                      f"{done} pixels (every {pstep}th row) of that sampled scene (timed, "
                      f"x{npx / max(done, 1):.0f}); the sampled scene is sparser than the full "
                      "one, so the render part is a lower bound")}
    out["random_walks_full_frame"] = walks_full_frame(cores)
    return out


def walks_full_frame(cores):
    """One whole frame of the random-walk workload (2000 x 50 vertices, 98k
    segments, 64^3, 256x256 orthographic, opaque) on the oracle, measured end to
    end: the list build from the raw vertices plus the render of every pixel."""
    import oracle
    from gen.linesets import tiny_walks, tiny_walks_camera
    ls, cam = tiny_walks(), tiny_walks_camera()
    t0 = time.perf_counter()
    o = oracle.Oracle.from_lineset(ls, nthreads=cores)
    o.build_lists()
    o.render(cam, alpha=1.0)
    ms = 1e3 * (time.perf_counter() - t0)
    o.close()
    return {"value": round(ms, 2), "unit": "ms/frame", "cores": cores, "segments": ls.n_segments,
            "pixels": cam.width * cam.height, "measured": "one full frame, not extrapolated"}


# ---------------------------------------------------------------- our arm
def max_over_ranks(values, world, device):
    """Each rank's timings -> their maximum over the ranks (every rank gets it)."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t]


def job_ms_per_frame(slowest_ms, world):
    """Whole-job time per frame: `world` replicas each finish a frame every
    `slowest_ms` (the slowest rank's mean), so the job renders one per
    slowest_ms / world."""
    return slowest_ms / world


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2510_09081_gb300 as vrt

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    t0 = time.time()
    wl = make_workload(args.workload, args.scale)
    ls, cam = wl["ls"], wl["cam"]
    log(f"[bench] workload ready in {time.time() - t0:.1f}s: V={ls.n_vertices} S={ls.n_segments}")
    n_upd = max(1, min(args.steps + args.warmup, 4))
    upd_host, upd_dev = [], []
    for f in range(n_upd):
        first, blk = wl["update"](f)
        h = torch.from_numpy(np.ascontiguousarray(blk, np.float32)).pin_memory()
        upd_host.append((first, h))
        upd_dev.append((first, h.to(dev)))
    r = vrt.Renderer(ls.n, ls.radius, stream=stream)
    xyz_dev = torch.from_numpy(ls.xyz).to(dev)
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        r.upload(xyz_dev, ls.offsets)
    vrt.set_option(r.h, vrt.OPT_STAGE_TIMING, 1)
    vrt.set_option(r.h, vrt.OPT_MIPS_FORMAT, {"fp32": vrt.MIPS_F32, "fp16": vrt.MIPS_F16,
                                              "bf16": vrt.MIPS_BF16}[args.mips])
    c = vrt.camera_c(cam)
    p = vrt.params_c(alpha=wl["alpha"], ao_cones=wl["ao"], cull=wl["cull"],
                     voxel_shading=1 if args.shading == "voxel" else 0, light=SHADING_LIGHT)
    rgba = torch.empty((cam.height, cam.width, 4), dtype=torch.float32, device=dev)
    fid = torch.empty((cam.height, cam.width), dtype=torch.int32, device=dev)
    ft = torch.empty((cam.height, cam.width), dtype=torch.float32, device=dev)
    rgba_host = torch.empty_like(rgba, device="cpu").pin_memory()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)

    vrt.set_option(r.h, vrt.OPT_GRAPH, 0 if args.no_graph else 1)
    hit_key = vrt.HIT_KEY_16_16 if args.hit_key == "16+16" else vrt.HIT_KEY_DEPTH_ID
    vrt.set_option(r.h, vrt.OPT_HIT_KEY, hit_key)
    static_cams = None
    if args.static:
        # lists (and the pyramid) built once, for every occupied voxel; each
        # frame traces from a camera turned one more degree about the target
        p.cull = 0
        with torch.cuda.stream(stream):
            vrt.frame(r.h, c, p, rgba, fid, ft)
        static_cams = [vrt.camera_c(orbit(cam, d)) for d in range(360)]

    def frame(f, host=False):
        if static_cams is not None:
            vrt.trace(r.h, static_cams[f % 360], p, rgba, fid, ft)
            return
        # one call per frame: update, voxelize, pyramid (AO only), cull, trace;
        # replayed as a CUDA graph unless --no-graph
        first, blk = (upd_host if host else upd_dev)[f % n_upd]
        vrt.frame(r.h, c, p, rgba, fid, ft, first_vertex=first, update=blk)

    with torch.cuda.stream(stream):
        for f in range(args.warmup):
            frame(f)
        vrt.sync(r.h)
    st0 = vrt.get_stats(r.h)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # ---- device-timed region
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stage_ms = {k: [] for k in vrt.STAGES}
    barrier()
    wall0 = time.perf_counter()
    with ClockSampler(local_rank) as clk, torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(i & 0xff)            # evict L2 between frames (outside the events)
            ev[i][0].record(stream)
            frame(args.warmup + i)
            ev[i][1].record(stream)
            for k, v in vrt.get_stage_ms(r.h).items():   # waits for the frame
                stage_ms[k].append(v)
        vrt.sync(r.h)
    barrier()
    wall = time.perf_counter() - wall0
    clocks = clk.summary()
    st = vrt.get_stats(r.h)
    frame_ms = [a.elapsed_time(b) for a, b in ev]
    mean_ms = statistics.mean(frame_ms)
    launches = (st["kernel_launches"] - st0["kernel_launches"])

    # ---- end-to-end through the C ABI with host buffers (warmed up like the
    # device frames: the first copy out of each pinned buffer maps it)
    e2e_ms = []
    with torch.cuda.stream(stream):
        for f in range(max(args.warmup, n_upd)):
            frame(f, host=True)
        vrt.sync(r.h)
        for i in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            frame(args.warmup + i, host=True)
            rgba_host.copy_(rgba, non_blocking=True)
            b.record(stream)
            b.synchronize()
            e2e_ms.append(a.elapsed_time(b))
        vrt.sync(r.h)
    h2d = 0 if args.static else int(upd_host[0][1].numel() * 4)
    d2h = int(rgba.numel() * 4)

    # ---- two frames in flight (dynamic workloads): a second grid holding the
    # same set on its own stream takes every other frame; each grid applies
    # the update blocks of the frames it skipped. Whole-run time / frames.
    pipe_ms = None
    if not args.static and not args.no_pipeline:
        s2 = torch.cuda.Stream(device=dev)
        r2 = vrt.Renderer(ls.n, ls.radius, stream=s2)
        with torch.cuda.stream(s2):
            r2.upload(xyz_dev, ls.offsets)
        vrt.set_option(r2.h, vrt.OPT_GRAPH, 0 if args.no_graph else 1)
        vrt.set_option(r2.h, vrt.OPT_HIT_KEY, hit_key)
        vrt.set_option(r2.h, vrt.OPT_MIPS_FORMAT, {"fp32": vrt.MIPS_F32, "fp16": vrt.MIPS_F16,
                                                   "bf16": vrt.MIPS_BF16}[args.mips])
        outs2 = (torch.empty_like(rgba), torch.empty_like(fid), torch.empty_like(ft))
        slots = [(stream, r, (rgba, fid, ft)), (s2, r2, outs2)]

        def pipe(n0, n):
            for f in range(n0, n0 + n):
                st_, g_, b_ = slots[f % 2]
                with torch.cuda.stream(st_):
                    if f > n0:
                        first, blk = upd_dev[(f - 1) % n_upd]
                        vrt.update_vertices(g_.h, first, blk)
                    first, blk = upd_dev[f % n_upd]
                    vrt.frame(g_.h, c, p, *b_, first_vertex=first, update=blk)

        pipe(0, max(args.warmup, 4))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        pipe(0, args.steps)
        torch.cuda.synchronize(dev)
        pipe_ms = (time.perf_counter() - t0) * 1e3 / args.steps
        vrt.sync(r2.h)
        r2.close()
        vrt.sync(r.h)

    # ---- one instrumented frame (not timed): list entries the rays examine
    vrt.set_option(r.h, vrt.OPT_TRACE_COUNTERS, 1)
    with torch.cuda.stream(stream):
        frame(args.warmup)
        vrt.sync(r.h)
    stc = vrt.get_stats(r.h)
    entries = stc["trace_entries"]
    cyc = stc["trace_cycles"]
    trace_work = {"entries": entries, "capsule_tests": stc["trace_capsule_tests"],
                  "unique_entries": stc["trace_unique_entries"],
                  "unique_vertices": stc["trace_unique_vertices"],
                  "unique_voxels": stc["trace_unique_voxels"],
                  "voxel_lists": stc["trace_voxels"], "dda_steps": stc["trace_steps"],
                  "hits_found": stc["trace_hits"],
                  "wholewarp_voxel_lists": stc["trace_wholewarp_voxels"],
                  "wholewarp_entries": stc["trace_wholewarp_entries"],
                  "cycle_share": {k: round(v / max(1, sum(cyc[:3])), 4) for k, v in
                                  zip(("dda", "shared_entry", "whole_warp",
                                       "capsule_tests_in_shared_entry"), cyc)}}
    vrt.set_option(r.h, vrt.OPT_TRACE_COUNTERS, 0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    # ---- max over ranks
    mean_ms, e2e_mean = max_over_ranks([mean_ms, statistics.mean(e2e_ms)], world, dev)

    if rank != 0:
        r.close()
        return None
    stages = {k: statistics.mean(v) for k, v in stage_ms.items() if v}
    if args.static:  # a static frame runs the trace alone (the field is reused)
        stages = {k: v for k, v in stages.items() if k == "trace"}
    hbm, hbm_src = hbm_peak()
    px = cam.width * cam.height
    frame_B = sum(stage_bytes(k, ls.n, ls.n_vertices, st, px, trace_work, mips=wl["ao"] > 0)
                  for k in stages)
    trace_B = stage_bytes("trace", ls.n, ls.n_vertices, st, px, trace_work)
    # dominant kernel: the trace (one launch per frame, timed by the library's
    # events on the grid's stream)
    alu_peak = sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    achieved = entries * TRACE_FLOPS_PER_ENTRY / (stages["trace"] * 1e-3) / 1e12
    srt = sorted(frame_ms)
    out = {
        "metric": METRIC,
        "value": round(job_ms_per_frame(mean_ms, world), 4),
        "unit": "ms/frame",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(mean_ms, 4),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "impl": "ours",
        "config": {"workload": wl["desc"] + (f" [scaled to {args.scale} of the lines]" if args.scale != 1.0 else "")
                   + (f" [occupancy pyramid in {args.mips}]" if args.mips != "fp32" else "")
                   + (" [hits ordered by the 16+16-bit per-voxel key]" if args.hit_key == "16+16" else "")
                   + (f" [voxel-space shading: AO x shadow toward {SHADING_LIGHT}]"
                      if args.shading == "voxel" else "")
                   + (" [static scene: lists built once for every occupied voxel; each frame "
                      "traces only, the camera turned 1 degree per frame]" if args.static else ""),
                   "l2": "flushed between frames (512 MB write)",
                   "cuda_graph": not args.no_graph,
                   "segments": ls.n_segments, "grid": ls.n, "pixels": px,
                   "p50_ms": round(srt[len(srt) // 2], 4),
                   "p99_ms": round(srt[min(len(srt) - 1, int(0.99 * len(srt)))], 4),
                   "wall_s": round(wall, 3),
                   "value_definition": "mean device time per frame (max over ranks) / ranks"},
        "throughput": {"segments_per_s": round(ls.n_segments * world / (mean_ms * 1e-3), 1),
                       "pixels_per_s": round(px * world / (mean_ms * 1e-3), 1)},
        "stages_ms": {k: round(v, 4) for k, v in stages.items()},
        "counters": {k: st[k] for k in ("fragments", "fragments_listed", "occupied_voxels",
                                        "visible_voxels", "repaired_voxels", "retraced_pixels",
                                        "exact_decisions", "max_count")},
        "trace_work": trace_work,
        "roofline": {"bound": "alu", "kernel": "k_trace_tile (trace stage)",
                     "achieved": round(achieved, 3), "peak": round(alu_peak, 2), "unit": "TFLOP/s",
                     "frac": round(achieved / alu_peak, 4),
                     "peak_source": (f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                                     f"{SM_MAX_MHZ:.0f} MHz"),
                     "work": (f"{entries} list entries examined x {TRACE_FLOPS_PER_ENTRY} FP32 ops "
                              "(one ray-capsule entry test each)"),
                     "traffic": trace_traffic(),
                     "trace_algorithmic_bytes": trace_B,
                     "trace_hbm_gbs": round(trace_B / (stages["trace"] * 1e-3) / 1e9, 1),
                     "trace_hbm_frac": round(trace_B / (stages["trace"] * 1e-3) / 1e9 / hbm, 4),
                     "frame_algorithmic_bytes": frame_B,
                     "frame_bytes_formula": ("16V + 8N^3 (pass 1) + [AO] 4N^3 + 4N^3/7 (pyramid) + "
                                             "4N^3 + N^3/7 (cull) + 8N^3 (scan) + 16V + 4F_vis + 4N^3 "
                                             "(pass 2) + 24 px + 4 F_t + 16 V_t + 8 N_t (trace: "
                                             "distinct entries, vertices, voxels the rays read)"),
                     "frame_hbm_gbs": round(frame_B / (mean_ms * 1e-3) / 1e9, 1),
                     "frame_hbm_frac": round(frame_B / (mean_ms * 1e-3) / 1e9 / hbm, 4),
                     "hbm_peak": hbm,
                     "hbm_peak_source": (f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)"
                                         if hbm_src == "measured" else hbm_src)},
        "pipelined": None if pipe_ms is None else {
            "frames_in_flight": 2, "ms_per_frame": round(pipe_ms, 4),
            "definition": "host wall time of back-to-back frames on two grids (two streams) "
                          "holding the same set, per frame; no L2 flush between frames"},
        "e2e": {"value": round(e2e_mean, 4), "unit": "ms/frame", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    r.close()
    if args.workload == "bundles" and not args.no_serving and args.scale == 1.0 and not args.static:
        # the metric's second half: served-frame latency over resident sets
        del xyz_dev, flush
        torch.cuda.empty_cache()
        n_req = 40
        sets, reqs, arrivals, total = serve_mix(n_req)
        arms = serve_arms(sets, reqs, arrivals, local_rank)
        out["serving"] = {
            "workload": ("64 resident random-walk line sets, log-uniform 10k..5M segments (total "
                         f"{total}), grids 128^3..512^3, outputs 720p..4K, alpha U[0.2, 1], 2% of "
                         "vertices updated per request, automatic culling"),
            "requests": n_req,
            "served_frames_per_s": arms["served_capacity"]["frames_per_s"],
            "plain_frames_per_s": arms["plain_capacity"]["frames_per_s"],
            "p50_ms": arms["served_poisson"]["p50_ms"], "p99_ms": arms["served_poisson"]["p99_ms"],
            "plain_p50_ms": arms["plain_poisson"]["p50_ms"],
            "plain_p99_ms": arms["plain_poisson"]["p99_ms"],
            "arms": arms,
            "small_sets_batched_frames_per_s": arms["small_sets_batched"]["frames_per_s"],
            "small_sets_unbatched_frames_per_s": arms["small_sets_unbatched"]["frames_per_s"],
            "definition": ("served: 4 stream slots (frames of different sets overlap); plain: 1 "
                           "slot; batched: frames of sets under 100k segments issued in batches of "
                           "up to 16 (one graph launch each); frames/s with every request "
                           "queued at once; latency submit -> frame finished seen by the host, "
                           "Poisson arrivals at 200 requests/s; small_sets: 8 frames (720p, no "
                           "update) of every set under 100k segments, queued at once")}
    if not args.no_cpu_baseline:
        try:
            out["cpu_baseline"] = cpu_baseline(wl)
        except Exception as e:  # the baseline is reported, never required
            out["cpu_baseline"] = {"value": None, "error": str(e)}
    return out


# ------------------------------------------------------------ serving (C4)
SERVE_METRIC = "served frames/s over 64 resident line sets (Poisson 200 req/s); p50/p99 latency"


def serve_mix(n_req):
    """The serving workload: 64 resident random-walk line sets of log-uniform
    size (10k..5M segments; grid 128^3 / 256^3 / 512^3 by size) and n_req frame
    requests, each a camera (720p..4K), an opacity in [0.2, 1] and an update of
    2% of the set's vertices, arriving as a Poisson stream at 200 requests/s."""
    from gen import linesets as G
    import paper_2510_09081_gb300 as vrt
    from gen import linesets as G
    rng = np.random.default_rng(20251013)
    n_sets = 64
    sizes = np.exp(rng.uniform(np.log(1e4), np.log(5e6), n_sets)).astype(np.int64)
    t0 = time.time()
    sets = []
    for k, S in enumerate(sizes):
        n = 128 if S < 200_000 else (256 if S < 1_500_000 else 512)
        sets.append(G.walk_set(int(S), n, radius=0.4, seed=20251100 + 7 * k))
    log(f"[bench] {n_sets} sets, {int(sizes.sum())} segments, ready in {time.time() - t0:.1f}s")
    res_choices = [(1280, 720), (1920, 1080), (2560, 1440), (3840, 2160)]
    arrivals = np.cumsum(rng.exponential(1.0 / 200.0, n_req))
    reqs = []
    for i in range(n_req):
        k = int(rng.integers(n_sets))
        ls = sets[k]
        w, h = res_choices[int(rng.integers(len(res_choices)))]
        th = rng.uniform(0, 2 * np.pi)
        c = ls.n / 2.0
        cam = G.Camera(width=w, height=h, ortho=0,
                       eye=(c + 1.7 * ls.n * np.cos(th), c + 1.7 * ls.n * np.sin(th), c + 0.5 * ls.n),
                       target=(c, c, c), up=(0.0, 0.0, 1.0), fovy_deg=45.0)
        cnt = max(1, ls.n_vertices // 50)
        first = int(rng.integers(0, ls.n_vertices - cnt + 1))
        upd = np.clip(ls.xyz[first:first + cnt] + rng.normal(0, 0.05, (cnt, 3)), 1.0,
                      ls.n - 1.0).astype(np.float32)
        reqs.append((k, cam, float(rng.uniform(0.2, 1.0)), first, upd))
    return sets, reqs, arrivals, int(sizes.sum())


def serve_arms(sets, reqs, arrivals, device=0):
    """Run the requests through the library's server: a Poisson stream at 200
    requests/s (latency) and every request queued at once (capacity), each with
    4 stream slots (served: frames of different sets overlap) and with 1 (the
    plain one-frame-at-a-time path)."""
    import torch
    import paper_2510_09081_gb300 as vrt
    n_sets = len(sets)
    dev = torch.device("cuda", device)
    bufs = [torch.empty((2160, 3840, 4), dtype=torch.float32, device=dev) for _ in range(n_sets)]

    def arm(slots, paced, small_segments=0, only=None):
        srv = vrt.Server(max_inflight=slots, small_segments=small_segments)
        ids = [srv.add_set(ls.xyz, ls.offsets, ls.n, ls.radius) for ls in sets]
        # warm-up (not timed): one frame of every set makes it resident
        for k in range(n_sets):
            srv.submit(ids[k], reqs[0][1], bufs[k], alpha=0.5)
        srv.poll(wait=True)
        t_start = time.perf_counter()
        for i, (k, cam, alpha, first, upd) in enumerate(reqs if only is None else only):
            if paced:
                delay = t_start + arrivals[i] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            srv.submit(ids[k], cam, bufs[k], alpha=alpha, cull_on=2, first_vertex=first, update=upd)
        res = srv.poll(wait=True)
        wall = time.perf_counter() - t_start
        st = srv.stats()
        srv.close()
        lat = np.array([r["latency_ms"] for r in res])
        bad = sum(r["status"] != 0 for r in res)
        return dict(frames_per_s=round(len(res) / wall, 2), p50_ms=round(float(np.percentile(lat, 50)), 3),
                    p99_ms=round(float(np.percentile(lat, 99)), 3), failed=int(bad),
                    resident_sets=st["resident_sets"], evictions=st["evictions"],
                    batches=st["batches"], batched_frames=st["batched_frames"])

    # small sets alone (fewer than 100k segments, 720p): batched vs one frame at a time
    rng = np.random.default_rng(5)
    small = [k for k, ls in enumerate(sets) if ls.n_segments < 100_000]
    small_reqs = []
    for i in range(8 * len(small)):
        k = small[i % len(small)]
        ls = sets[k]
        c = ls.n / 2.0
        th = rng.uniform(0, 2 * np.pi)
        from gen import linesets as G
        cam = G.Camera(width=1280, height=720, ortho=0,
                       eye=(c + 1.7 * ls.n * np.cos(th), c + 1.7 * ls.n * np.sin(th), c + 0.5 * ls.n),
                       target=(c, c, c), up=(0.0, 0.0, 1.0), fovy_deg=45.0)
        small_reqs.append((k, cam, float(rng.uniform(0.2, 1.0)), 0, None))
    out = {"served_poisson": arm(4, True), "plain_poisson": arm(1, True),
           "served_capacity": arm(4, False), "plain_capacity": arm(1, False),
           "served_capacity_batched": arm(4, False, small_segments=100_000),
           "small_sets_batched": arm(4, False, small_segments=100_000, only=small_reqs),
           "small_sets_unbatched": arm(4, False, only=small_reqs)}
    del bufs
    torch.cuda.empty_cache()
    return out


def run_serve(args, rank):
    """Serving (C4) as the benchmark's main line: frames/s with every request
    queued at once, 4 stream slots; the other arms beside it."""
    if rank != 0:
        return None
    n_req = max(args.steps, 40)
    sets, reqs, arrivals, total = serve_mix(n_req)
    out = serve_arms(sets, reqs, arrivals)
    sizes_sum = total
    sp = out["served_capacity"]["frames_per_s"]
    return {"metric": SERVE_METRIC, "value": sp, "unit": "frames/s", "n_gpus": 1, "steps": n_req,
            "warmup": n_sets, "ms_per_step": round(1000.0 / sp, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "impl": "ours",
            "config": {"workload": ("serving: 64 resident random-walk line sets, log-uniform "
                                    "10k..5M segments (total %d), grids 128^3..512^3, outputs "
                                    "720p..4K, alpha U[0.2, 1], 2%% of vertices updated per "
                                    "request, automatic culling" % sizes_sum),
                       "value_definition": "frames/s with every request queued at once, 4 stream slots",
                       **out}}


# ----------------------------------------------------------- reference arm
def run_reference(args, rank):
    """The oracle, as it stands, on the host cores; each step is a bounded
    sample of the workload scaled to ms/frame."""
    if rank != 0:
        return None
    wl = make_workload(args.workload, args.scale)
    vals, walls = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(wl, budget_s=4.0)
        if i >= args.warmup:
            vals.append(cb["value"])
            walls.append(time.perf_counter() - t0)
    v = statistics.mean(vals)
    return {"metric": METRIC, "value": round(v, 3), "unit": "ms/frame", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v, 3),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": wl["desc"]},
            "cpu_baseline": {"value": round(v, 3), "unit": "ms/frame", "cores": cb["cores"],
                             "kind": "oracle", "sample": cb["sample"],
                             "sample_wall_s_per_step": round(statistics.mean(walls), 2),
                             "note": ("each step times a bounded sample of the frame on the "
                                      "oracle and scales it to a whole frame, so the value "
                                      "exceeds the step's wall time")},
            "e2e": {"value": round(v, 3), "unit": "ms/frame", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bundles", choices=["bundles", "walks", "abc", "sparse", "serve"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--hit-key", choices=("depth-id", "16+16"), default="depth-id",
                    help="order of a ray's hits within a voxel (16+16: the paper's 32-bit key)")
    ap.add_argument("--no-serving", action="store_true",
                    help="leave the serving leg out of the bundles line")
    ap.add_argument("--no-graph", action="store_true",
                    help="issue the frame's launches one by one instead of replaying a CUDA graph")
    ap.add_argument("--mips", choices=("fp32", "fp16", "bf16"), default="fp32",
                    help="storage of the occupancy pyramid (AO workloads)")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="skip the two-frames-in-flight throughput measurement")
    ap.add_argument("--static", action="store_true",
                    help="static scene: build the lists once, then time trace-only frames")
    ap.add_argument("--shading", choices=("hit", "voxel"), default="hit",
                    help="hit: the workload's per-hit shading; voxel: voxel-space shading field "
                         "(AO when the workload has it, and a directional shadow)")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="fraction of the bundle streamlines (small cases for profiler captures)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if world > 1 and args.impl == "ours":
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    if args.impl == "reference":
        out = run_reference(args, rank)
    elif args.workload == "serve":
        out = run_serve(args, rank)
    else:
        out = run_ours(args, rank, world, local_rank)
    if out is not None:
        print(json.dumps(out), flush=True)
    if world > 1 and args.impl == "ours":
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
