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

# DRAM bytes per launch of the dominant kernel from an ncu capture, valid only
# for the source it was measured on (sha256 of the listed files).
TRAFFIC = {}


def _rank_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


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
    """Compulsory DRAM bytes of one step's launches of `stage` (bytes model).

    w: dict with P (pixels/step), C (covered candidate pixels), Cr (covered
    reference pixels), texel counts and triangle/vertex counts."""
    P = w["P"]
    tex_px = 1.33 * 16 * 3          # unique texels per covered pixel per map x 16 B x 3 maps
    if stage == "shade_bwd":
        return 40 * P + (tex_px * 3) * w["C"]          # key+g'+pre per pixel; texel read + grad RMW
    if stage == "shade":
        return 2 * 24 * P + tex_px * (w["C"] + w["Cr"])  # candidate + reference launches
    if stage == "aa_loss":
        return (8 + 16 + 12 + 16) * P + (8 + 16 + 12) * P  # candidate (loss, g') + reference (image)
    if stage == "raster":
        return 2 * 8 * P + 96 * VIEWS * (w["F"] + w["Fr"])
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
    """The CPU oracle's full step (reference render + candidate fwd/bwd/Adam).

    Topology tables are built once, outside the timed calls."""

    def __init__(self, scene_cfg):
        from oracle import step as S

        self.S = S
        self.ref = S.OracleJob(scene_cfg["ref"], loss="l1")
        self.cand = S.OracleJob(scene_cfg["cand"], loss="logl1")

    def seconds(self, n_views, res, seed=123):
        import torch

        import synth

        views = synth.sample_views(seed, 0, n_views, res, res)
        t0 = time.perf_counter()
        with torch.no_grad():
            ref = self.S.render(self.ref, self.ref.params, views, res, res)["img"]
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
                         "sample": f"{n_views} of 8 views at {res}^2 per step, full oracle step "
                                   "(reference render + candidate fwd/bwd/Adam)"},
        "e2e": {"value": value, "unit": "Mpixels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm
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
    cfg = synth.config_plain()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = Context(stream=stream)
    ref_job = ctx.create_job(cfg["ref"], frozen=True)
    cand = ctx.create_job(cfg["cand"], loss="logl1", lr0=0.01)
    plain = ctx.create_job(cfg["cand"], loss="logl1", lr0=0.01, batch_views=VIEWS)
    n_steps = args.warmup + args.steps
    host_views = [synth.sample_views(rank * 100003 + 7, i, VIEWS, RES, RES) for i in range(n_steps)]
    view_np = np.stack([v.view(np.uint8) for v in host_views])                  # (steps, 8*112)
    dev_views = torch.from_numpy(view_np).to(dev)
    pinned_views = torch.from_numpy(view_np).pin_memory()
    staging = torch.empty(VIEWS * 112, dtype=torch.uint8, device=dev)            # graph's fixed view buffer
    ref_buf = torch.empty((VIEWS, RES, RES, 3), dtype=torch.float32, device=dev)
    loss_buf = torch.zeros(n_steps + 1, dtype=torch.float32, device=dev)
    graph_loss = torch.zeros(1, dtype=torch.float32, device=dev)
    cptr = ctx.ctx
    i32 = C.c_int32
    jobs_c = (i32 * 1)(cand)
    plain_c = (i32 * 1)(plain)
    vpj8 = (i32 * 1)(VIEWS)
    vpj1 = (i32 * 1)(1)
    hw = (i32 * 2)(RES, RES)
    refs8 = (C.c_void_p * 1)(ref_buf.data_ptr())
    refs1 = [(C.c_void_p * 1)(ref_buf[v:v + 1].data_ptr()) for v in range(VIEWS)]
    view_bytes = 112

    def ck(st):
        if st != 0:
            raise B.AdmsError(st, L.adms_last_error(cptr).decode())

    def step_at(vp, loss_ptr):
        ck(L.adms_render_reference(cptr, ref_job, vp, VIEWS, RES, RES, ref_buf.data_ptr()))
        ck(L.adms_forward_loss(cptr, jobs_c, 1, vp, vpj8, hw, refs8, loss_ptr, None))
        ck(L.adms_backward(cptr, jobs_c, 1, 0))
        ck(L.adms_optimizer_step(cptr, jobs_c, 1))

    def step(i):
        step_at(dev_views[i].data_ptr(), loss_buf.data_ptr() + 4 * i)

    def plain_step(i):
        vp = dev_views[i].data_ptr()
        for v in range(VIEWS):
            one = vp + v * view_bytes
            ck(L.adms_render_reference(cptr, ref_job, one, 1, RES, RES, ref_buf[v:v + 1].data_ptr()))
            ck(L.adms_forward_loss(cptr, plain_c, 1, one, vpj1, hw, refs1[v], loss_buf.data_ptr() + 4 * i, None))
            ck(L.adms_backward(cptr, plain_c, 1, 0))
        ck(L.adms_optimizer_step(cptr, plain_c, 1))

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    def timed_region(fn, k0, k):
        barrier()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(k + 1)]
        evs[0].record(stream)
        for s in range(k):
            fn(k0 + s)
            evs[s + 1].record(stream)
        barrier()
        per = [evs[s].elapsed_time(evs[s + 1]) for s in range(k)]
        total = evs[0].elapsed_time(evs[-1])
        if world > 1:
            t = torch.tensor([total], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            total = float(t)
        return total, per

    # warm-up (also sizes all scratch), then record one step as a CUDA graph
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

    # headline: the graph-captured fused step, inputs resident in HBM
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    launches0 = B.adms_launch_count()
    fused_ms_nograph, _ = timed_region(step, args.warmup, args.steps)
    launches = (B.adms_launch_count() - launches0) / args.steps
    total_ms, per = timed_region(graph_step, args.warmup, args.steps)
    plain_ms, _ = timed_region(plain_step, args.warmup, args.steps)
    # per-stage profile of the fused step (events between stages; not the headline)
    B.adms_ctx_profile(cptr, True)
    B.adms_ctx_stage_times(cptr)
    timed_region(step, args.warmup, args.steps)
    stages = B.adms_ctx_stage_times(cptr)
    B.adms_ctx_profile(cptr, False)
    # end to end through the C ABI: host views in (pinned), graph step, loss read back, every step
    h2d = VIEWS * view_bytes
    d2h = 4
    barrier()
    t0 = time.perf_counter()
    for s in range(args.steps):
        staging.copy_(pinned_views[args.warmup + s], non_blocking=True)
        B.adms_graph_launch(cptr, graph)
        float(graph_loss.item())
    barrier()
    e2e_s = time.perf_counter() - t0
    clocks = sampler.stop()
    clocks["window"] = "graph, fused, plain, profiled and end-to-end timed regions"
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t)

    # workload facts for the bytes model
    keys = ctx.keys(cand, (VIEWS, RES, RES))
    covered = int((keys != -1).sum())
    pv = ctx.params(cand)
    texels = sum(pv[n].shape[0] * pv[n].shape[1] for n in ("kd", "orm", "nrm"))
    ctx.render_reference(ref_job, host_views[-1], RES, RES, out=ref_buf)
    rkeys = ctx.keys(ref_job, (VIEWS, RES, RES))
    covered_ref = int((rkeys != -1).sum())
    wl = dict(P=VIEWS * RES * RES, C=covered, Cr=covered_ref, texels=texels, texel_floats=4 * texels,
              V=cfg["cand"].mesh.n_verts, F=cfg["cand"].mesh.n_tris, Fr=cfg["ref"].mesh.n_tris)

    px_step = VIEWS * RES * RES
    value = world * px_step * args.steps / (total_ms / 1e3) / 1e6
    nograph_value = world * px_step * args.steps / (fused_ms_nograph / 1e3) / 1e6
    plain_value = world * px_step * args.steps / (plain_ms / 1e3) / 1e6
    e2e_value = world * px_step * args.steps / e2e_s / 1e6
    per_sorted = sorted(per)

    # roofline of the dominant kernel stage
    stage_rows = {}
    for name, (ms, n) in stages.items():
        if n == 0:
            continue
        ab = algorithmic_bytes(name, wl)
        stage_rows[name] = {"ms_per_step": ms / args.steps, "launches_per_step": n / args.steps,
                            "algorithmic_bytes_per_step": ab,
                            "gbs": (ab / (ms / 1e3 / args.steps) / 1e9) if ab else None}
    dominant = max(stage_rows, key=lambda k: stage_rows[k]["ms_per_step"])
    peak, peak_kind = _peaks()
    d = stage_rows[dominant]
    launches_per_step = max(d["launches_per_step"], 1e-9)
    achieved = d["gbs"]
    tr = TRAFFIC.get(dominant)
    traffic = None
    if tr and _sha(tr["files"]) == tr["sha"]:
        traffic = tr["bytes_per_launch"]
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "peak_source": peak_kind,
                "traffic": traffic,
                "algorithmic_bytes_per_launch": (d["algorithmic_bytes_per_step"] / launches_per_step)
                if d["algorithmic_bytes_per_step"] else None,
                "ms_per_launch": d["ms_per_step"] / launches_per_step}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, cores = OracleStep(cfg).seconds(1, RES)
        cpu = {"value": RES * RES / dt / 1e6, "unit": "Mpixels/s", "cores": cores, "kind": "oracle",
               "sample": f"1 of 8 views at {RES}^2: full oracle step (reference render + fwd/bwd/Adam)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Mpixels/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "global_batch": VIEWS * world, "seq_len": None,
                       "parallelism": f"replicas x{world}" if world > 1 else "single",
                       "launch": "one CUDA graph per step (reference render, forward+loss, backward, Adam)",
                       "l2": "working set > 126 MB L2 (textures, moments, buffers); no flush"},
            "p50_step_ms": per_sorted[len(per) // 2], "p99_step_ms": per_sorted[min(len(per) - 1, int(0.99 * len(per)))],
            "fused_without_graph": {"value": nograph_value, "unit": "Mpixels/s",
                                    "ms_per_step": fused_ms_nograph / args.steps},
            "plain_per_view_loop": {"value": plain_value, "unit": "Mpixels/s", "ms_per_step": plain_ms / args.steps},
            "fused_over_plain": value / plain_value,
            "gpu_launches": int(round(launches * args.steps)), "gpu_launches_per_step": launches,
            "e2e": {"value": e2e_value, "unit": "Mpixels/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "roofline": roofline, "stages": stage_rows, "clocks": clocks, "cpu_baseline": cpu,
            "coverage": covered / px_step,
        }
        print(json.dumps(line), flush=True)
    B.adms_graph_destroy(graph)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference_arm(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
