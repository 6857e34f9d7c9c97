#!/usr/bin/env python
"""Benchmark of the render-and-compare step (fwd+bwd Mpixels/s) on GB300.

One step = render the reference under a fresh batch of random views, render
the candidate, antialias, take the tone-mapped L1 loss, backpropagate to
positions and the three texture maps, and apply Adam (with the Laplacian
term and schedules). Workload: 200k-tri procedural reference with 2048^2
maps, 5,120-tri candidate with 1024^2 maps and full mip chains, 8 views at
512x512, one point + one directional light.

Prints one JSON line. --impl reference times the CPU oracle instead.
"""

from __future__ import annotations

import argparse
import ctypes as C
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

VIEWS, RES = 8, 512
METRIC = "fwd+bwd Mpixels/s on 1 GB300 (fused vs plain, grads ≤1e-3 rel); p99 step ms"
WORKLOAD = ("reference 200k-tri fBm icosphere with 2048^2 procedural maps; candidate 5,120 tris with 1024^2 "
            "maps + mips; 8 random views at 512x512; point + directional light; log-L1 loss")
WORKLOAD_AGG = ("aggregate geometry (Sec. 6): reference canopy of 600k opaque leaf quads (1.2M tris) with 2048^2 "
                "procedural maps; candidate 5,500 billboard quads (11k tris) with a 2048^2 base colour + opacity "
                "atlas and 1024^2 (gamma, r, m) and normal maps, all optimized; 8 depth-peeling layers blended back "
                "to front (Sec. 5.2); 8 random views at 512x512; point + directional light; squared-L2 loss")

# DRAM bytes per launch of the dominant kernel from an ncu capture, valid only
# for the source it was measured on (sha256 of the listed files).
TRAFFIC = {
    "shade_bwd": {"bytes_per_launch": 151613440 + 28056576, "warp_instructions_per_launch": 119476965,
                  "files": ["paper_2104_03989_gb300/csrc/shade.cu", "paper_2104_03989_gb300/csrc/pixel.cuh",
                            "paper_2104_03989_gb300/csrc/common.cuh", "paper_2104_03989_gb300/csrc/kernels.cuh"],
                  "sha": "fd068b253bfdce39",
                  "capture": "profiles/shade_bwd_plain_workload.md"},
}

def _rank_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


# ----------------------------------------------------------------------------- replicas
# "Replicas only": each rank runs the whole step on its own GPU with its own
# views; nothing is exchanged but the timing, and the job's throughput is the
# sum over ranks of pixels over the slowest rank's time.
def replica_seed(rank):
    """Seed of a rank's camera/light stream (disjoint streams per rank)."""
    return rank * 100003 + 7


def max_over_ranks(x, world, device):
    """The maximum of a per-rank scalar over all ranks (every rank gets it)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t)


def whole_job_mpix(world, px_step, steps, seconds):
    """Whole-job Mpixels/s: every rank processed px_step pixels per step."""
    return world * px_step * steps / seconds / 1e6


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for k in ("hbm_gbs", "hbm_GBs", "hbm_gb_s"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- algorithmic bytes model
def algorithmic_bytes(stage, w):
    """Compulsory DRAM bytes of one step's launches of `stage` (the algorithmic bytes model).

    w: dict with P (pixels/step; samples/step under MSAA), C (covered candidate
    pixels or samples, summed over depth-peeling layers), Cr (covered reference
    pixels or samples), Ppix (pixels per step), S (samples per pixel side), L
    (depth-peeling layers, 0: opaque), texel counts and triangle/vertex counts."""
    P = w["P"]
    texel = 1.33 * 16               # unique texels per covered pixel per map x 16 B
    maps = w.get("tex_maps", 3)     # maps larger than one texel
    tex_px = texel * maps
    ref_px = texel * w.get("ref_maps", 3)
    views = w.get("views", VIEWS)
    L = w.get("L", 0)
    if L:
        # per layer and pixel: key, colour + opacity, the composite behind, its
        # gradient; the opaque reference as in the plain step
        if stage == "shade_bwd":
            return (8 + 16 + 16 + 16 + 16) * L * P + (tex_px * 3) * w["C"]
        if stage == "shade":
            return 24 * L * P + 24 * P + tex_px * w["C"] + ref_px * w["Cr"]
        if stage == "aa_loss":
            return (8 + 16 + 16 + 16) * L * P + 12 * P + (8 + 16 + 12) * P
        if stage == "raster":
            return (8 + 8) * L * P + 8 * P + 96 * views * (L * w["F"] + w["Fr"])
    if stage == "shade_bwd":
        # the survey's model: key 8 + dL/dx 12 per pixel; per covered pixel the texels
        # read again plus the read-modify-write of the optimized maps' texel gradients
        return 20 * P + texel * (maps + 2 * w.get("grad_maps", 3)) * w["C"]
    if stage == "shade_bwd_extended":
        # this kernel's own layout: dL/dx travels as a 16-byte record with the pair
        # blend bits in its fourth word (key 8 + 16 per pixel instead of 8 + 12)
        return 24 * P + texel * (maps + 2 * w.get("grad_maps", 3)) * w["C"]
    rc = 1 + w.get("recompute", 0)    # the backward recomputes raster, shading and AA once more
    if stage == "shade":
        return (24 * P + tex_px * w["C"]) * rc               # key read, colour write; texels of covered pixels
    if stage == "aa_loss" and w.get("S", 1) > 1:
        # per sample: AA reads key + pre and writes its colour, the resolve reads it
        # back (and writes g' for the candidate); per pixel: reference in, image out
        return (8 + 16 + 16) * 2 * P + (16 + 16) * P + 16 * P + (12 + 12) * w["Ppix"]
    if stage == "aa_loss":
        return (8 + 16 + 12 + 16) * P * rc                 # key, colour, reference in; dL/dx out
    if stage == "raster":
        return (8 * P + 96 * views * w["F"]) * rc
    if stage == "adam":
        return 32 * (w["texel_floats"] + 3 * w["V"])
    if stage == "mip_build":
        return int(16 * w["texels"] * (5 / 12))
    return None


def _sha(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


# ----------------------------------------------------------------------------- oracle timing
class OracleStep:
    """The CPU oracle's step (candidate fwd/bwd/Adam on pre-rendered references).

    Topology tables are built once, outside the timed calls."""

    def __init__(self, scene_cfg, msaa=1, layers=0):
        from oracle import step as S

        self.S = S
        self.msaa = msaa
        self.ref = S.OracleJob(scene_cfg["ref"], loss="l1")
        self.cand = S.OracleJob(scene_cfg["cand"], loss=scene_cfg["loss"], msaa=msaa, layers=layers)

    def seconds(self, n_views, res, seed=123):
        """Seconds of the candidate's step (forward + loss, backward, Adam) on the
        views' reference images, rendered first and not timed (the metric's step),
        and the threads used."""
        import torch

        import synth

        views = synth.sample_views(seed, 0, n_views, res, res)
        with torch.no_grad():
            ref = self.S.render(self.ref, self.ref.params, views, res, res, ssaa=self.msaa)["img"]
        t0 = time.perf_counter()
        self.S.step(self.cand, views, ref.numpy(), res, res)
        return time.perf_counter() - t0, torch.get_num_threads()


def run_reference_arm(args):
    rank, world, _ = _rank_env()
    if rank != 0:
        return
    import synth
    from oracle import _build

    _build.build()
    cfg = synth.config_plain()
    n_views = 1
    # bounded sample per step: one view of the batch, at 512^2 for short runs and
    # at 256^2 (a quarter of its pixels) when many steps are asked for
    res = RES if args.steps + args.warmup <= 40 else RES // 2
    orc = OracleStep(cfg)
    for _ in range(args.warmup):
        orc.seconds(n_views, res)
    times = []
    cores = None
    for k in range(args.steps):
        dt, cores = orc.seconds(n_views, res, seed=1000 + k)
        times.append(dt)
    px = n_views * res * res
    value = px * len(times) / sum(times) / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mpixels/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": f"{n_views} view of 8 at {res}^2 per step"},
        "cpu_baseline": {"value": value, "unit": "Mpixels/s", "cores": cores, "kind": "oracle",
                         "sample": f"{n_views} of 8 views at {res}^2 per step: the oracle's candidate step "
                                   "(fwd/loss, bwd, Adam) on its reference images, rendered untimed"},
        "e2e": {"value": value, "unit": "Mpixels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm
WORKLOADS = {
    # name: (views per step, resolution, backward recomputes the raster, description)
    "plain": (VIEWS, RES, 0, WORKLOAD),
    "aggregate": (VIEWS, RES, 0, WORKLOAD_AGG),
    "tess": (16, 1024, 1, "differentiation at scale (Sec. 5.1, Eq. 3): reference 1,003,520-tri fBm icosphere; "
                          "candidate 980-tri base mesh tessellated 3 times (62,720 tris) with a 1024^2 scalar "
                          "displacement map and a 2048^2 normal map, constant diffuse-dominated base colour and "
                          "(gamma, r, m); 16 random views at 1024x1024; point + directional light; log-L1 loss; "
                          "raster buffers recomputed in the backward"),
    "small": (1, 256, 0, "plain method, one step: reference 20,480-tri icosphere displaced by 8 sinusoids, albedo "
                         "0.7, roughness 0.5; candidate 320-tri icosphere with 256^2 base-colour and normal noise maps; "
                         "one fixed camera at distance 3, 256x256, one directional light; L1 loss (latency-bound)"),
}


def _config(wk):
    import synth

    return {"aggregate": synth.config_aggregate, "tess": synth.config_tess, "small": synth.config_small}.get(
        wk, synth.config_plain)()


def run_native(args):
    import torch

    rank, world, local = _rank_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    import synth
    from paper_2104_03989_gb300 import binding as B
    from paper_2104_03989_gb300.engine import Context

    L = B.lib()
    dev = torch.device("cuda", torch.cuda.current_device())
    wk = args.workload
    agg = wk == "aggregate"
    NV, RS, RECOMPUTE, wdesc = WORKLOADS[wk]
    cfg = _config(wk)
    LY = cfg["layers"] if agg else 0
    loss = cfg["loss"]
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = Context(stream=stream)
    MS = max(int(args.msaa), 1)
    # under MSAA the references are supersampled renders (every sample shaded)
    # the foliage reference is a dense cloud of small leaf triangles: rasterize those
    # of up to 256 samples directly instead of binning them, reading each sample's key
    # before its test (~160 fragments per sample)
    ref_job = ctx.create_job(cfg["ref"], frozen=True, samples=MS, shade_samples=True,
                             raster_direct_px=256 if agg else 0, raster_depth_filter=agg)
    pl = bool(args.per_level_textures)
    # the tessellated candidate's ~17-pixel triangles rasterize faster directly than
    # binned (the keys do not depend on the threshold), with plain atomicMin (about two
    # fragments per sample: the key read costs more); step ms for thresholds 64 / 128 /
    # 256 / 512 / 1024 / 2048 samples: 6.36 / 6.15 / 5.96 / 5.87 / 5.93 / 5.98
    cdirect = 512 if wk == "tess" else 0
    cand = ctx.create_job(cfg["cand"], loss=loss, lr0=0.01, per_level_textures=pl, samples=MS, layers=LY,
                          raster_direct_px=cdirect)
    plain = ctx.create_job(cfg["cand"], loss=loss, lr0=0.01, batch_views=NV, per_level_textures=pl, samples=MS,
                           layers=LY, raster_direct_px=cdirect)
    n_steps = args.warmup + args.steps
    if wk == "small":   # one fixed camera
        host_views = [synth.fixed_view(RS, RS) for _ in range(n_steps)]
    else:
        host_views = [synth.sample_views(replica_seed(rank), i, NV, RS, RS) for i in range(n_steps)]
    view_np = np.stack([v.view(np.uint8) for v in host_views])                  # (steps, NV*112)
    SKB = int(args.skinning)
    if SKB:
        # both meshes skinned by the same bones (Eq. 2); a new pose each step rides in
        # the step's input record after the views
        ctx.skinning(ref_job, synth.bone_weights(cfg["ref"].mesh.pos, SKB, seed=5), lr_scale=0.0)
        wc = synth.bone_weights(cfg["cand"].mesh.pos, SKB, seed=5)
        ctx.skinning(cand, wc, lr_scale=1.0 / SKB)   # weights of a vertex move together: keep the blend in step
        ctx.skinning(plain, wc, lr_scale=1.0 / SKB)
        pose_np = np.stack([synth.bone_pose(SKB, 5 + replica_seed(rank), i).reshape(-1).view(np.uint8)
                            for i in range(n_steps)])
        view_np = np.ascontiguousarray(np.concatenate([view_np, pose_np], axis=1))
    dev_views = torch.from_numpy(view_np).to(dev)
    staging = torch.empty(view_np.shape[1], dtype=torch.uint8, device=dev)       # graph's fixed input buffer
    ref_buf = torch.empty((NV, RS, RS, 3), dtype=torch.float32, device=dev)
    loss_buf = torch.zeros(n_steps + 1, dtype=torch.float32, device=dev)
    graph_loss = torch.zeros(1, dtype=torch.float32, device=dev)
    cptr = ctx.ctx
    if args.pipeline:
        # each step's texture Adam runs beside the next step's frame and raster
        B.adms_ctx_set_pipelining(cptr, True)
    i32 = C.c_int32
    jobs_c = (i32 * 1)(cand)
    plain_c = (i32 * 1)(plain)
    vpjN = (i32 * 1)(NV)
    vpj1 = (i32 * 1)(1)
    hw = (i32 * 2)(RS, RS)
    refsN = (C.c_void_p * 1)(ref_buf.data_ptr())
    refs1 = [(C.c_void_p * 1)(ref_buf[v:v + 1].data_ptr()) for v in range(NV)]
    view_bytes = 112

    def ck(st):
        if st != 0:
            raise B.AdmsError(st, L.adms_last_error(cptr).decode())

    def set_pose(vp, jobs):
        if SKB:
            for jb in jobs:
                ck(L.adms_job_set_bones(cptr, jb, vp + NV * 112))

    # the reference render runs on a stream of its own, alongside the candidate's
    # frame, raster and shading; the loss waits for it (adms_ctx_set_ref_event)
    ref_stream = torch.cuda.Stream()
    fork_ev, ref_ev = torch.cuda.Event(), torch.cuda.Event()

    def cand_step(vp, refs_c, loss_ptr):
        set_pose(vp, (cand,))
        ck(L.adms_forward_loss(cptr, jobs_c, 1, vp, vpjN, hw, refs_c, loss_ptr, None))
        B.adms_ctx_set_ref_event(cptr, None)
        ck(L.adms_backward(cptr, jobs_c, 1, RECOMPUTE))
        ck(L.adms_optimizer_step(cptr, jobs_c, 1))

    def step_at(vp, loss_ptr, overlap=True):
        """The step with its reference render (on a second stream when overlap)."""
        if overlap:
            fork_ev.record(stream)
            ref_stream.wait_event(fork_ev)
            B.adms_ctx_set_stream(cptr, ref_stream)
        B.adms_ctx_set_ref_event(cptr, None)
        set_pose(vp, (ref_job,))
        ck(L.adms_render_reference(cptr, ref_job, vp, NV, RS, RS, ref_buf.data_ptr()))
        if overlap:
            ref_ev.record(ref_stream)
            B.adms_ctx_set_stream(cptr, stream)
            B.adms_ctx_set_ref_event(cptr, ref_ev)
        cand_step(vp, refsN, loss_ptr)

    def step(i):
        step_at(dev_views[i].data_ptr(), loss_buf.data_ptr() + 4 * i)

    def plain_step(i):
        vp = dev_views[i].data_ptr()
        set_pose(vp, (ref_job, plain))
        for v in range(NV):
            one = vp + v * view_bytes
            ck(L.adms_render_reference(cptr, ref_job, one, 1, RS, RS, ref_buf[v:v + 1].data_ptr()))
            ck(L.adms_forward_loss(cptr, plain_c, 1, one, vpj1, hw, refs1[v], loss_buf.data_ptr() + 4 * i, None))
            ck(L.adms_backward(cptr, plain_c, 1, RECOMPUTE))
        ck(L.adms_optimizer_step(cptr, plain_c, 1))

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    def timed_region(fn, k0, k, name="region"):
        # an NVTX range per region, so that a profiler can keep one region's launches
        # (e.g. ncu --nvtx --nvtx-include "metric_step/")
        barrier()
        torch.cuda.nvtx.range_push(name)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(k + 1)]
        evs[0].record(stream)
        for s in range(k):
            fn(k0 + s)
            evs[s + 1].record(stream)
        barrier()
        torch.cuda.nvtx.range_pop()
        per = [evs[s].elapsed_time(evs[s + 1]) for s in range(k)]
        return max_over_ranks(evs[0].elapsed_time(evs[-1]), world, dev), per

    # warm-up (also sizes all scratch), then record the step with its reference render
    # as a CUDA graph
    for i in range(args.warmup):
        step(i)
        plain_step(i)
    staging.copy_(dev_views[0])
    torch.cuda.synchronize()
    B.adms_graph_begin(cptr)
    step_at(staging.data_ptr(), graph_loss.data_ptr())
    graph = B.adms_graph_end(cptr)

    def graph_step(i):
        staging.copy_(dev_views[i], non_blocking=True)
        B.adms_graph_launch(cptr, graph)

    # The metric's step (forward+loss, backward, Adam) with the reference images of its
    # views already rendered: a ring of R (views, references) slots rendered before the
    # timed region, one graph per slot, step i on slot i mod R
    R = min(args.steps, 16 if NV * RS * RS <= 8 * 512 * 512 else 4)
    ring_views = [dev_views[args.warmup + r].clone() for r in range(R)]
    ring_refs = [torch.empty((NV, RS, RS, 3), dtype=torch.float32, device=dev) for _ in range(R)]
    for r in range(R):
        set_pose(ring_views[r].data_ptr(), (ref_job,))
        ck(L.adms_render_reference(cptr, ref_job, ring_views[r].data_ptr(), NV, RS, RS, ring_refs[r].data_ptr()))
    ring_refs_c = [(C.c_void_p * 1)(t.data_ptr()) for t in ring_refs]
    torch.cuda.synchronize()
    ring_graphs = []
    for r in range(R):
        B.adms_graph_begin(cptr)
        cand_step(ring_views[r].data_ptr(), ring_refs_c[r], graph_loss.data_ptr())
        ring_graphs.append(B.adms_graph_end(cptr))

    def cand_graph_step(i):
        B.adms_graph_launch(cptr, ring_graphs[(i - args.warmup) % R])

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    launches0 = B.adms_launch_count()
    for i in range(args.warmup):
        cand_graph_step(args.warmup + i)
    launches0 = B.adms_launch_count()
    fused_ms_nograph, _ = timed_region(lambda i: cand_step(ring_views[(i - args.warmup) % R].data_ptr(),
                                                           ring_refs_c[(i - args.warmup) % R],
                                                           loss_buf.data_ptr() + 4 * i), args.warmup, args.steps)
    launches = (B.adms_launch_count() - launches0) / args.steps
    total_ms, per = timed_region(cand_graph_step, args.warmup, args.steps, "metric_step")
    with_ref_ms, per_ref = timed_region(graph_step, args.warmup, args.steps, "with_reference")
    plain_ms, _ = timed_region(plain_step, args.warmup, args.steps, "plain_loop")
    # per-stage profile of the metric's step (events between stages; not the headline)
    B.adms_ctx_profile(cptr, True)
    B.adms_ctx_stage_times(cptr)
    timed_region(lambda i: cand_step(ring_views[(i - args.warmup) % R].data_ptr(), ring_refs_c[(i - args.warmup) % R],
                                     loss_buf.data_ptr() + 4 * i), args.warmup, args.steps)
    stages = B.adms_ctx_stage_times(cptr)
    B.adms_ctx_profile(cptr, False)
    # end to end through the C ABI with host buffers, every step: the views from (pinned)
    # host memory passed to adms_forward_loss as is, the reference images copied in
    # from pinned host memory, the loss read back; no graph. As a training loop would,
    # the next step's references are copied on a copy stream while the current step
    # runs (two device buffers); forward_loss waits for them (adms_ctx_set_ref_event)
    # right before the first kernel that reads them.
    host_refs = [t.cpu().pin_memory() for t in ring_refs]
    pinned_views = torch.from_numpy(view_np).pin_memory()
    e2e_loss = torch.zeros(1, dtype=torch.float32, device=dev)
    ebufs = [torch.empty((NV, RS, RS, 3), dtype=torch.float32, device=dev) for _ in range(2)]
    ebufs_c = [(C.c_void_p * 1)(t.data_ptr()) for t in ebufs]
    copy_stream = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    step_done = [torch.cuda.Event() for _ in range(2)]
    loss_ready = [torch.cuda.Event() for _ in range(2)]
    loss_host = torch.zeros(2, dtype=torch.float32).pin_memory()
    e2e_losses = []
    h2d = view_np.shape[1] + host_refs[0].numel() * 4
    d2h = 4

    def fetch(s):
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(step_done[s % 2])  # step s - 2, the buffer's last reader, is done
            ebufs[s % 2].copy_(host_refs[s % R], non_blocking=True)
            copied[s % 2].record(copy_stream)

    def read_loss(s):
        loss_ready[s % 2].synchronize()
        e2e_losses.append(float(loss_host[s % 2]))

    barrier()
    t0 = time.perf_counter()
    fetch(0)
    for s in range(args.steps):
        r = s % R
        if s + 1 < args.steps:
            fetch(s + 1)
        B.adms_ctx_set_ref_event(cptr, copied[s % 2])
        cand_step(pinned_views[args.warmup + r].data_ptr(), ebufs_c[s % 2], e2e_loss.data_ptr())
        step_done[s % 2].record(stream)
        loss_host[s % 2:s % 2 + 1].copy_(e2e_loss, non_blocking=True)
        loss_ready[s % 2].record(stream)
        if s > 0:
            read_loss(s - 1)   # the previous step's loss, read while this step runs
    read_loss(args.steps - 1)
    assert len(e2e_losses) == args.steps and all(np.isfinite(e2e_losses))
    barrier()
    e2e_s = time.perf_counter() - t0
    clocks = sampler.stop()
    clocks["window"] = "graph, fused, with-reference, plain, profiled and end-to-end timed regions"
    e2e_s = max_over_ranks(e2e_s, world, dev)

    # workload facts for the bytes model
    keys = ctx.keys(cand, (max(LY, 1), NV, RS * MS, RS * MS))
    covered = int((keys != -1).sum())
    pv = ctx.params(cand)
    texels = sum(pv[n].shape[0] * pv[n].shape[1] for n in ("kd", "orm", "nrm"))
    # latent texels Adam updates: level 0, or every level of each chain with per-level latents
    opt_maps = [n for n in ("kd", "orm", "nrm") if pv.get("g_" + n) is not None]
    latent_texels = (sum(pv[n + "_chain"].shape[0] for n in opt_maps) if pl
                     else sum(pv[n].shape[0] * pv[n].shape[1] for n in opt_maps))
    tex_maps = sum(1 for n in ("kd", "orm", "nrm") if pv[n].shape[0] * pv[n].shape[1] > 1)
    ctx.render_reference(ref_job, host_views[-1], RS, RS, out=ref_buf)
    rkeys = ctx.keys(ref_job, (NV, RS * MS, RS * MS))
    covered_ref = int((rkeys != -1).sum())
    ref_maps = sum(1 for t in (cfg["ref"].kd, cfg["ref"].orm, cfg["ref"].nrm) if t.shape[0] * t.shape[1] > 1)
    disp_floats = cfg["cand"].disp.size if cfg["cand"].disp is not None else 0
    V_lat = cfg["cand"].mesh.n_verts
    F_cand = B.adms_job_params(cptr, cand).n_tris_render   # the tessellated mesh for tess
    wl = dict(P=NV * RS * RS * MS * MS, C=covered, Cr=covered_ref, texels=texels,
              texel_floats=4 * latent_texels + disp_floats, V=V_lat, F=F_cand, Fr=cfg["ref"].mesh.n_tris,
              Ppix=NV * RS * RS, S=MS, L=LY, views=NV, tex_maps=tex_maps, grad_maps=len(opt_maps),
              ref_maps=ref_maps, recompute=RECOMPUTE)

    px_step = NV * RS * RS
    value = whole_job_mpix(world, px_step, args.steps, total_ms / 1e3)
    nograph_value = whole_job_mpix(world, px_step, args.steps, fused_ms_nograph / 1e3)
    with_ref_value = whole_job_mpix(world, px_step, args.steps, with_ref_ms / 1e3)
    plain_value = whole_job_mpix(world, px_step, args.steps, plain_ms / 1e3)
    e2e_value = whole_job_mpix(world, px_step, args.steps, e2e_s)
    per_sorted = sorted(per)

    # roofline of the dominant kernel stage
    stage_rows = {}
    for name, (ms, n) in stages.items():
        if n == 0:
            continue
        ab = algorithmic_bytes(name, wl)
        row = {"ms_per_step": ms / args.steps, "launches_per_step": n / args.steps, "algorithmic_bytes_per_step": ab,
               "gbs": (ab / (ms / 1e3 / args.steps) / 1e9) if ab else None}
        if name == "shade_bwd" and not LY and MS == 1:
            ext = algorithmic_bytes("shade_bwd_extended", wl)
            row["extended_model"] = {"algorithmic_bytes_per_step": ext, "gbs": ext / (ms / 1e3 / args.steps) / 1e9}
        stage_rows[name] = row
    # the slowest stage with a bytes model (the multi-kernel raster setup has none)
    modelled = [k for k in stage_rows if stage_rows[k]["algorithmic_bytes_per_step"]]
    dominant = max(modelled or stage_rows, key=lambda k: stage_rows[k]["ms_per_step"])
    peak, peak_kind = _peaks()
    d = stage_rows[dominant]
    launches_per_step = max(d["launches_per_step"], 1e-9)
    achieved = d["gbs"]
    # the committed DRAM counters and instruction counts are the plain workload's
    tr = TRAFFIC.get(dominant) if (wk == "plain" and not (pl or SKB or MS > 1)) else None
    traffic = None
    if tr and _sha(tr["files"]) == tr["sha"]:
        traffic = tr["bytes_per_launch"]
    # the same kernel against the instruction-issue rate (one warp instruction per
    # scheduler per cycle: SMs x 4 x SM clock), with ncu's instruction count per launch
    issue = None
    if tr and _sha(tr["files"]) == tr["sha"] and tr.get("warp_instructions_per_launch") and clocks.get("sm_mhz"):
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        ach = tr["warp_instructions_per_launch"] / (d["ms_per_step"] / launches_per_step / 1e3) / 1e9
        pk = sms * 4 * clocks["sm_mhz"] / 1e3
        issue = {"bound": "issue", "achieved": ach, "peak": pk, "unit": "G warp instructions/s", "frac": ach / pk,
                 "instructions_per_launch": tr["warp_instructions_per_launch"], "sms": sms}
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "peak_source": peak_kind,
                "traffic": traffic,
                "algorithmic_bytes_per_launch": (d["algorithmic_bytes_per_step"] / launches_per_step)
                if d["algorithmic_bytes_per_step"] else None,
                "ms_per_launch": d["ms_per_step"] / launches_per_step, "issue_roofline": issue}
    if "extended_model" in d:
        roofline["frac_extended_model"] = d["extended_model"]["gbs"] / peak

    cpu = cpu1 = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import torch as _t

        cres = min(RS // MS, 512)    # the same samples per view as the plain sample (capped for the big views)
        orc = OracleStep(cfg, msaa=MS, layers=LY)
        dt, cores = orc.seconds(1, cres)
        sample = (f"1 of {NV} views at {cres}^2" + (f" with {MS}x{MS} MSAA" if MS > 1 else "")
                  + (f" with {LY} peeling layers" if LY else "")
                  + ": the oracle's candidate step (fwd/loss, bwd, Adam) on its reference images, rendered untimed")
        cpu = {"value": cres * cres / dt / 1e6, "unit": "Mpixels/s", "cores": cores, "kind": "oracle",
               "sample": sample}
        nthr = _t.get_num_threads()
        _t.set_num_threads(1)
        try:
            c1 = min(cres, 256)
            dt1, _ = orc.seconds(1, c1)
            cpu1 = {"value": c1 * c1 / dt1 / 1e6, "unit": "Mpixels/s", "cores": 1, "kind": "oracle",
                    "sample": sample.replace(f"{cres}^2", f"{c1}^2") + ", one thread"}
        finally:
            _t.set_num_threads(nthr)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Mpixels/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wdesc
                       + ("; every mip level of each texture its own latent (Sec. 6)" if pl else "")
                       + (f"; both meshes skinned by {SKB} bones (Eq. 2), dense weights optimized (learning rate / {SKB}), "
                          "a new pose per step"
                          if SKB else "")
                       + (f"; {MS}x{MS} multisampling (Sec. 5.2): visibility, shading and antialiasing on the "
                          f"{RS * MS}^2 sample grid, each sample shaded at its pixel centre, loss on the resolved "
                          f"pixels; references supersampled {MS}x{MS}" if MS > 1 else ""),
                       "global_batch": NV * world, "seq_len": None,
                       "parallelism": f"replicas x{world}" if world > 1 else "single",
                       "launch": "one CUDA graph per step: forward+loss, backward"
                                 + (" (raster recomputed)" if RECOMPUTE else "") + ", Adam; the step's reference "
                                 f"images rendered before the timed region (a ring of {R} view batches)"
                                 + ("; pipelined steps: each step's texture Adam runs beside the next step's frame "
                                    "and raster (every timed step runs one, the first the step's before the region)"
                                    if args.pipeline else ""),
                       "l2": "working set > 126 MB L2 (textures, moments, buffers); no flush",
                       "pipelined": bool(args.pipeline)},
            "p50_step_ms": per_sorted[len(per) // 2], "p99_step_ms": per_sorted[min(len(per) - 1, int(0.99 * len(per)))],
            "with_reference_render": {"value": with_ref_value, "unit": "Mpixels/s",
                                      "ms_per_step": with_ref_ms / args.steps,
                                      "p99_step_ms": sorted(per_ref)[min(len(per_ref) - 1, int(0.99 * len(per_ref)))],
                                      "launch": "one CUDA graph per step, reference render on a second stream"},
            "fused_without_graph": {"value": nograph_value, "unit": "Mpixels/s",
                                    "ms_per_step": fused_ms_nograph / args.steps},
            "plain_per_view_loop": {"value": plain_value, "unit": "Mpixels/s", "ms_per_step": plain_ms / args.steps,
                                    "note": "one view per call, each with its reference render"},
            "fused_over_plain": with_ref_value / plain_value,
            "gpu_launches": int(round(launches * args.steps)), "gpu_launches_per_step": launches,
            "e2e": {"value": e2e_value, "unit": "Mpixels/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "path": "adms_forward_loss with the views in pinned host memory, reference images copied from "
                            "pinned host memory (the next step's on a copy stream during the current step), "
                            "adms_backward, adms_optimizer_step, every step's loss copied to pinned host memory and "
                            "read by the host while the next step runs; no graph"},
            "roofline": roofline, "stages": stage_rows, "clocks": clocks, "cpu_baseline": cpu,
            "cpu_baseline_single_thread": cpu1,
            "coverage": covered / (px_step * MS * MS),
        }
        print(json.dumps(line), flush=True)
    B.adms_graph_destroy(graph)
    for g in ring_graphs:
        B.adms_graph_destroy(g)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


# ----------------------------------------------------------------------------- uneven jobs
def run_batched(args):
    """Uneven jobs: every job's step (reference render, forward+loss, backward,
    Adam) for all jobs, as one CUDA graph whose pixel stages are one launch
    each over all jobs' tiles (persistent or one block per tile, as the
    autotuner chose), against the per-job loop (each job through the
    single-job launches, one after another)."""
    import torch

    import synth
    from paper_2104_03989_gb300 import binding as B
    from paper_2104_03989_gb300.engine import Context

    L = B.lib()
    dev = torch.device("cuda", torch.cuda.current_device())
    recipes = synth.job_mix(args.jobs, seed=0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = Context(stream=stream)
    cptr = ctx.ctx
    refs_j, cands = [], []
    for r in recipes:
        cand, ref = synth.job_scenes(r)
        refs_j.append(ctx.create_job(ref, frozen=True, seed=r["seed"]))
        cands.append(ctx.create_job(cand, loss="logl1", lr0=0.01, seed=r["seed"]))
    n = len(recipes)
    nv = [r["n_views"] for r in recipes]
    res = [r["res"] for r in recipes]
    offs = np.concatenate([[0], np.cumsum(nv)]).astype(int)
    n_steps = args.warmup + args.steps
    view_np = np.stack([np.concatenate([synth.sample_views(7919 * r["seed"] + 11, i, r["n_views"], r["res"], r["res"])
                                        for r in recipes]).view(np.uint8) for i in range(n_steps)])
    dev_views = torch.from_numpy(view_np).to(dev)
    staging = torch.empty(view_np.shape[1], dtype=torch.uint8, device=dev)
    ref_bufs = [torch.empty((nv[k], res[k], res[k], 3), dtype=torch.float32, device=dev) for k in range(n)]
    loss = torch.zeros(n, dtype=torch.float32, device=dev)
    i32 = C.c_int32
    jobs_c = (i32 * n)(*cands)
    vpj = (i32 * n)(*nv)
    hw = (i32 * (2 * n))(*[x for k in range(n) for x in (res[k], res[k])])
    refs_c = (C.c_void_p * n)(*[b.data_ptr() for b in ref_bufs])
    one = [((i32 * 1)(cands[k]), (i32 * 1)(nv[k]), (i32 * 2)(res[k], res[k]), (C.c_void_p * 1)(ref_bufs[k].data_ptr()))
           for k in range(n)]

    def ck(st):
        if st != 0:
            raise B.AdmsError(st, L.adms_last_error(cptr).decode())

    # the references render on four side streams (round robin over the jobs), beside
    # each other and beside the candidates' forward, whose loss waits for all of them
    sides = [torch.cuda.Stream() for _ in range(4)]
    fork_ev, ref_ev = torch.cuda.Event(), torch.cuda.Event()
    side_evs = [torch.cuda.Event() for _ in sides]

    def references(vb):
        fork_ev.record(stream)
        for sd in sides:
            sd.wait_event(fork_ev)
        for k in range(n):
            B.adms_ctx_set_stream(cptr, sides[k % len(sides)])
            ck(L.adms_render_reference(cptr, refs_j[k], vb + 112 * int(offs[k]), nv[k], res[k], res[k],
                                       ref_bufs[k].data_ptr()))
        for sd, ev in zip(sides[1:], side_evs[1:]):
            ev.record(sd)
            sides[0].wait_event(ev)
        ref_ev.record(sides[0])
        B.adms_ctx_set_stream(cptr, stream)
        B.adms_ctx_set_ref_event(cptr, ref_ev)

    def batched_at(vb):
        references(vb)
        ck(L.adms_forward_loss(cptr, jobs_c, n, vb, vpj, hw, refs_c, loss.data_ptr(), None))
        B.adms_ctx_set_ref_event(cptr, None)
        ck(L.adms_backward(cptr, jobs_c, n, 0))
        ck(L.adms_optimizer_step(cptr, jobs_c, n))

    def per_job_at(vb):
        references(vb)
        for k in range(n):
            j1, v1, hw1, r1 = one[k]
            ck(L.adms_forward_loss(cptr, j1, 1, vb + 112 * int(offs[k]), v1, hw1, r1, loss.data_ptr() + 4 * k, None))
            ck(L.adms_backward(cptr, j1, 1, 0))
            ck(L.adms_optimizer_step(cptr, j1, 1))
        B.adms_ctx_set_ref_event(cptr, None)

    def timed(fn, k0, k):
        torch.cuda.synchronize()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(k + 1)]
        evs[0].record(stream)
        for s in range(k):
            fn(k0 + s)
            evs[s + 1].record(stream)
        torch.cuda.synchronize()
        return evs[0].elapsed_time(evs[-1]), sorted(evs[s].elapsed_time(evs[s + 1]) for s in range(k))

    references(dev_views[0].data_ptr())
    B.adms_ctx_set_ref_event(cptr, None)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B.adms_autotune(cptr, cands, view_np[0].view(synth.VIEW_DTYPE), nv, [(x, x) for x in res], ref_bufs)
    tune_s = time.perf_counter() - t0
    tune = B.adms_ctx_tuning(cptr)
    for i in range(args.warmup):
        batched_at(dev_views[i].data_ptr())
        per_job_at(dev_views[i].data_ptr())
    staging.copy_(dev_views[0])
    torch.cuda.synchronize()
    B.adms_graph_begin(cptr)
    batched_at(staging.data_ptr())
    graph = B.adms_graph_end(cptr)

    def graph_step(i):
        staging.copy_(dev_views[i], non_blocking=True)
        B.adms_graph_launch(cptr, graph)

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    l0 = B.adms_launch_count()
    nog_ms, _ = timed(lambda i: batched_at(dev_views[i].data_ptr()), args.warmup, args.steps)
    launches = (B.adms_launch_count() - l0) / args.steps
    g_ms, per = timed(graph_step, args.warmup, args.steps)
    pj_ms, _ = timed(lambda i: per_job_at(dev_views[i].data_ptr()), args.warmup, args.steps)
    clocks = sampler.stop()
    px = sum(nv[k] * res[k] * res[k] for k in range(n))
    mp = lambda ms: px * args.steps / (ms / 1e3) / 1e6  # noqa: E731
    line = {
        "metric": "fwd+bwd Mpixels/s, uneven jobs in one graph-captured launch per pixel stage",
        "value": mp(g_ms), "unit": "Mpixels/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": g_ms / args.steps, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{n} uneven jobs (synth.job_mix seed 0): candidates "
                               f"{min(r['cand_freq'] for r in recipes) ** 2 * 20}-{max(r['cand_freq'] for r in recipes) ** 2 * 20}"
                               " tris, references ~10x, textures 256^2-2048^2, 4-16 views at 256^2-1024^2",
                   "pixels_per_step": px, "views_per_step": int(offs[-1]),
                   "l2": "working set far above L2; no flush"},
        "p50_step_ms": per[len(per) // 2], "p99_step_ms": per[min(len(per) - 1, int(0.99 * len(per)))],
        "batched_without_graph": {"value": mp(nog_ms), "ms_per_step": nog_ms / args.steps},
        "per_job_loop": {"value": mp(pj_ms), "ms_per_step": pj_ms / args.steps},
        "batched_over_per_job": pj_ms / g_ms,
        "autotune": {"tile_w": tune["tile_w"], "blocks_per_sm": tune["blocks_per_sm"], "seconds": tune_s},
        "gpu_launches_per_step": launches, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    B.adms_graph_destroy(graph)
    ctx.close()


def run_serving(args):
    """Continuous batching: Poisson arrivals of uneven jobs admitted by an HBM
    budget, every live job stepped together each iteration, against the
    per-job loop measured on the same jobs."""
    import torch

    import synth
    from paper_2104_03989_gb300.serving import Request, SimplificationServer, poisson_arrivals

    recipes = synth.job_mix(args.jobs, seed=1)
    arrivals = poisson_arrivals(len(recipes), args.rate, seed=2)
    reqs = []
    for r, t in zip(recipes, arrivals):
        cand, ref = synth.job_scenes(r)
        reqs.append(Request(rid=r["job"], cand=cand, ref=ref, n_views=r["n_views"], res=r["res"],
                            iterations=args.iterations, seed=r["seed"], arrival=float(t)))
    budget = int(args.budget_gb * 1e9)
    srv = SimplificationServer(hbm_budget_bytes=budget)
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    rep = srv.run(reqs)
    clocks = sampler.stop()
    srv.close()
    # the per-job loop on the same jobs and the same work: each job alone, from its
    # submission (job creation, reference job) through all its iterations, timed per
    # job; its aggregate is pixels over the summed time
    pj_iters = args.per_job_iterations or args.iterations
    pj_px, pj_s = 0, 0.0
    for q in reqs:
        q1 = Request(**{**q.__dict__, "iterations": pj_iters, "arrival": 0.0})
        s1 = SimplificationServer()
        s1.start()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s1.submit(q1)
        while s1.queue or s1.live:
            s1.admit()
            if s1.live:
                s1.iterate()
        torch.cuda.synchronize()
        pj_s += time.perf_counter() - t0
        pj_px += pj_iters * q.n_views * q.res * q.res
        s1.close()
    comp = sorted(rep["job_completion_s"])
    line = {
        "metric": "served fwd+bwd Mpixels/s and per-iteration latency (continuous batching)",
        "value": rep["aggregate_mpixels_per_s"], "unit": "Mpixels/s", "n_gpus": 1, "higher_is_better": True,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{len(reqs)} uneven jobs (synth.job_mix seed 1), Poisson arrivals at {args.rate}/s, "
                               f"{args.iterations} iterations each, HBM budget {args.budget_gb} GB"},
        "p50_iteration_ms": rep["p50_iteration_ms"], "p99_iteration_ms": rep["p99_iteration_ms"],
        "job_completion_s": {"p50": comp[len(comp) // 2] if comp else None, "max": comp[-1] if comp else None},
        "iterations": rep["iterations"], "done": rep["done"], "quarantined": rep["quarantined"],
        "rejected": rep["rejected"], "max_live": rep["max_live"], "wall_s": rep["wall_s"],
        "per_job_loop": {"value": pj_px / pj_s / 1e6, "unit": "Mpixels/s",
                         "sample": f"each job alone from submission through {pj_iters} iterations "
                                   "(the served jobs' work, job creation included on both sides)"},
        "served_over_per_job": rep["aggregate_mpixels_per_s"] / (pj_px / pj_s / 1e6),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="plain", choices=["plain", "tess", "small", "aggregate", "batched",
                                                            "serving"],
                    help="plain: the headline single-job step (8 views at 512^2); tess: tessellation + displacement "
                         "at scale (16 views at 1024^2, raster recomputed in the backward); small: the one-step "
                         "workload (one 256^2 view, latency-bound); aggregate: billboard quads with opacity under "
                         "depth peeling (Sec. 6 aggregate geometry); batched: uneven jobs in one launch per stage; "
                         "serving: continuous batching of Poisson arrivals")
    ap.add_argument("--jobs", type=int, default=64, help="jobs of the batched and serving workloads")
    ap.add_argument("--rate", type=float, default=20.0, help="serving: mean arrivals per second")
    ap.add_argument("--iterations", type=int, default=200, help="serving: iterations per job")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="serving: HBM budget")
    ap.add_argument("--per-job-iterations", type=int, default=0,
                    help="serving: iterations of each job in the per-job loop (0: --iterations, the same work)")
    ap.add_argument("--skinning", type=int, default=0, metavar="BONES",
                    help="plain workload with both meshes skinned by BONES bones and a new pose per step (Eq. 2)")
    ap.add_argument("--msaa", type=int, default=1, metavar="S",
                    help="plain workload rendered with S x S samples per pixel (MSAA, Sec. 5.2), references "
                         "supersampled; the metric counts pixels")
    ap.add_argument("--pipeline", type=int, default=1, choices=[0, 1],
                    help="plain-family workloads: defer each step's texture Adam to the next step's forward, "
                         "beside its frame and raster (adms_ctx_set_pipelining; results unchanged); 0: sequential")
    ap.add_argument("--per-level-textures", action="store_true",
                    help="plain workload with every mip level of each texture an independent latent (Sec. 6)")
    args = ap.parse_args()
    if args.workload in ("aggregate", "tess", "small") and (args.msaa > 1 or args.skinning or args.per_level_textures):
        ap.error("the aggregate, tess and small workloads run without --msaa, --skinning and --per-level-textures")
    if args.impl == "reference":
        run_reference_arm(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
