"""Benchmark: ray samples/s of the cube ray-casting path on B300.

Default workload ("dvr1024"): a 1024^3 float32 cube (N(0,1) noise + 2000
Gaussian sources, seed 2; 256^3 bricks), one step = fused statistics with a
4096-bin histogram + front-to-back DVR of a 32-view orbit at 1920x1080,
step 0.5 voxel, trilinear sampling, 256-entry transfer function, early
termination at alpha 0.99, all 32 views in one persistent launch.  Inputs are
seeded and synthetic (the paper's spectral cubes are not available).

Prints one JSON line.  `--impl reference` times the CPU oracle on the same
workload instead (bounded pixel sample per step).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6400.0
SM_COUNT = 148
FP32_LANES_PER_SM = 128

# Algorithmic work per DVR sample (trilinear + transfer function + over):
# trilinear 7 lerps (2 flops each) = 14, TF index 3 + lerp 4x2 = 11, over 8,
# position 6, t_k 3  -> 42 flops; 8 voxel reads + 2 TF reads.
DVR_FLOPS_PER_SAMPLE = 42
MIP_TRI_FLOPS_PER_SAMPLE = 14 + 6 + 3 + 1


def workload(name: str) -> dict:
    if name == "dvr1024":
        return dict(name="dvr1024", dims=(1024, 1024, 1024), n_sources=2000, seed=2, brick=256, views=32,
                    W=1920, H=1080, step=0.5, tf="sparse", term=0.99, nbins=4096, storage="f32")
    if name == "small128":
        return dict(name="small128", dims=(128, 128, 128), n_sources=8, seed=1, brick=128, views=1,
                    W=256, H=256, step=1.0, tf="sparse", term=0.99, nbins=256, storage="f32", ortho=True)
    raise SystemExit(f"unknown workload {name}")


def workload_config(w: dict, views: int) -> dict:
    """Workload identity shared by both arms of the benchmark."""
    return {"workload": w["name"], "dims": list(w["dims"]), "sources": w["n_sources"], "seed": w["seed"],
            "brick": w["brick"], "storage": w["storage"], "views": views, "image": [w["W"], w["H"]],
            "step": w["step"], "sampling": "trilinear", "tf": w["tf"], "term_alpha": w["term"],
            "hist_bins": w["nbins"]}


RENDER_SOURCES = ("paper_1111_6661_b300/csrc/render.cu", "paper_1111_6661_b300/csrc/ray.cuh")
TRAFFIC_PROFILE = "profiles/k_render_fused_dvr768_traffic.md"


def render_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in RENDER_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


BINDING_PROFILE = "profiles/k_render_fused_dvr768_1view.md"


def profile_values(path: str):
    """`- key: value` lines of a committed ncu summary, or None if the render
    kernel's sources changed since it was taken."""
    try:
        with open(os.path.join(ROOT, path)) as f:
            text = f.read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    return vals if vals.get("source_sha256") == render_source_hash() else None


def render_traffic():
    """DRAM bytes per launch of the render kernel (one-pass ncu count)."""
    vals = profile_values(TRAFFIC_PROFILE)
    try:
        return float(vals["dram_bytes_per_launch"]) if vals else None
    except (KeyError, ValueError):
        return None


def render_binding():
    """The unit that binds the render kernel, from its full ncu capture."""
    vals = profile_values(BINDING_PROFILE)
    if not vals:
        return None
    try:
        return {"unit": vals["binding_unit"], "busy_pct": float(vals["binding_unit_busy_pct"]),
                "issue_active_pct": float(vals["issue_active_pct"]), "source": BINDING_PROFILE}
    except (KeyError, ValueError):
        return None


def peaks():
    try:
        with open(PEAKS) as f:
            p = json.load(f)
        return p, "measured"
    except OSError:
        return {"hbm_gbs": FALLBACK_HBM_GBS, "sm_max_mhz": 2032.0}, "fallback"


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait(timeout=5)
        self.t.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank, local


def barrier_max(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def make_inputs(w: dict):
    import cubegen
    v = cubegen.generate(w["dims"], w["n_sources"], w["seed"])
    if w.get("ortho"):
        cams = [cubegen.ortho_z_camera(w["dims"])]
    else:
        cams = cubegen.orbit_cameras(w["dims"], w["views"])
    tf = cubegen.tf_sparse() if w["tf"] == "sparse" else cubegen.tf_dense()
    return v, cams, tf


# ---------------------------------------------------------------- CPU oracle
def oracle_rate(v, cams, tf, w, vmin, vmax, budget_s: float, seed: int = 0):
    """Time the CPU oracle (as it stands) on random pixels of the views until
    about budget_s seconds of wall time; returns samples/s and the sample."""
    import oracle
    rng = np.random.default_rng(seed)
    npix_total = w["W"] * w["H"]
    done_samples = 0
    done_pix = 0
    t0 = time.perf_counter()
    batch = 256
    views_used = set()
    while True:
        vi = int(rng.integers(0, len(cams)))
        pix = rng.choice(npix_total, size=batch, replace=False)
        r = oracle.render(v, cams[vi], w["W"], w["H"], w["step"], "trilinear", "dvr", tf=tf, vmin=vmin, vmax=vmax,
                          term=w["term"], pixels=pix)
        done_samples += int(r["nsamp"].sum())
        done_pix += batch
        views_used.add(vi)
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
        batch = min(batch * 2, 8192)
    return done_samples / el, done_pix, done_samples, el, len(views_used)


def run_reference(args, w):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle
    v, cams, tf = make_inputs(w)
    ref = oracle.stats(v) if v.size <= 2 ** 27 else None
    vmin = float(v.min()) if ref is None else ref["min"]
    vmax = float(v.max()) if ref is None else ref["max"]
    cores = os.cpu_count()
    budget = float(os.environ.get("VRC_REF_STEP_S", "8"))
    for _ in range(args.warmup):
        oracle_rate(v, cams, tf, w, vmin, vmax, 0.5)
    rates, pix_total = [], 0
    t_all = time.perf_counter()
    for s in range(args.steps):
        rate, npix, nsamp, el, nv = oracle_rate(v, cams, tf, w, vmin, vmax, budget, seed=s + 1)
        rates.append(rate)
        pix_total += npix
    elapsed = time.perf_counter() - t_all
    value = float(np.mean(rates))
    line = {"metric": "ray samples/s (DVR, trilinear)", "value": value, "unit": "samples/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": dict(workload_config(w, len(cams)), parallelism="rank0 only (CPU oracle)"),
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": cores, "kind": "oracle",
                             "sample": f"{pix_total} random pixels over {args.steps} steps, ~{budget:.0f} s each"},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def run_gpu(args, w):
    import torch

    import paper_1111_6661_b300 as vrc
    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    v, cams, tf = make_inputs(w)
    ctx = vrc.Context(local)
    st = torch.cuda.current_stream()
    cid = ctx.cube_upload(v, w["storage"], brick=w["brick"])
    info = ctx.cube_info(cid)
    rc = vrc.raycfg(w["W"], w["H"], w["step"], "trilinear", path=args.path)
    out = torch.empty((len(cams), w["H"], w["W"], 4), dtype=torch.float32, device=dev)
    dstats = torch.empty(8, dtype=torch.float64, device=dev)
    dhist = torch.empty(w["nbins"], dtype=torch.int64, device=dev)

    def step():
        ctx.cube_stats_async(cid, w["nbins"], dstats, dhist)
        ctx.render_dvr(cid, cams, rc, tf, w["term"], out=out)

    # warm-up (also fixes the sample count of one step: it is deterministic)
    for _ in range(max(args.warmup, 3) if args.warmup >= 3 else args.warmup):
        step()
    torch.cuda.synchronize()
    samples_per_step = ctx.last_render_samples()
    render_path = ctx.last_render_path()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clk = Clocks(local)
    launches0 = ctx.launch_count()
    barrier(ws)
    torch.cuda.synchronize()
    clk.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(st)
    for i in range(args.steps):
        ev[i][0].record(st)
        ctx.cube_stats_async(cid, w["nbins"], dstats, dhist)
        ev[i][1].record(st)
        ctx.render_dvr(cid, cams, rc, tf, w["term"], out=out)
        ev[i][2].record(st)
    t_end.record(st)
    torch.cuda.synchronize()
    clocks = clk.stop()
    barrier(ws)
    launches = ctx.launch_count() - launches0
    ms = t_start.elapsed_time(t_end)
    ms = barrier_max(ms, ws)
    stats_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    render_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in ev]))
    value = ws * samples_per_step * args.steps / (ms / 1e3)

    pk, pk_kind = peaks()
    sm_max = pk.get("sm_max_mhz", 2032.0)
    fp32_peak_tflops = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved_tflops = samples_per_step * DVR_FLOPS_PER_SAMPLE / (render_ms / 1e3) / 1e12
    stats_bytes = info["dims"][0] * info["dims"][1] * info["dims"][2] * {"f32": 4, "bf16": 2, "fp8": 1}[w["storage"]]
    stats_gbs = stats_bytes / (stats_ms / 1e3) / 1e9

    # exact median of the same cube (radix selection bracketed by a sampled first digit: one pass
    # over the cube keeps the keys of the bounded bins, the digits come from those; not part of the step)
    ctx.cube_median(cid)
    t_med = time.perf_counter()
    for _ in range(3):
        ctx.cube_median(cid)
    median_ms = (time.perf_counter() - t_med) * 1e3 / 3

    # the same step with empty-space skipping (identical image): frames/s, and
    # how many of the lattice samples were actually fetched
    skip = None
    if not args.no_skip_variant:
        rc_s = vrc.raycfg(w["W"], w["H"], w["step"], "trilinear", skip_empty=True)
        ctx.render_dvr(cid, cams, rc_s, tf, w["term"], out=out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            ctx.render_dvr(cid, cams, rc_s, tf, w["term"], out=out)
        e1.record(st)
        torch.cuda.synchronize()
        sk_ms = e0.elapsed_time(e1) / args.steps
        lat, ev = ctx.last_render_samples(evaluated=True)
        skip = {"render_ms": sk_ms, "frames_per_s": len(cams) / (sk_ms / 1e3), "lattice_samples": lat,
                "evaluated_samples": ev, "evaluated_samples_per_s": ev / (sk_ms / 1e3),
                "note": "skip_empty=1: samples whose 8^3 macro-cell is transparent under the TF are not fetched; "
                        "the image is bit-identical"}

    # axis-aligned nearest MIP at native resolution (an orthographic view along
    # z, NX x NY pixels, step 1: one sample per voxel, each voxel read once):
    # the ray-casting case that HBM bounds; algorithmic bytes = the stored
    # bytes of the samples
    mip_native = None
    if not args.no_mip_native:
        import cubegen
        NX, NY, NZ = w["dims"]
        cam_n = [cubegen.ortho_z_camera(w["dims"])]
        rc_n = vrc.raycfg(NX, NY, 1.0, "nearest")
        img_n = torch.empty((1, NY, NX), dtype=torch.float32, device=dev)
        ctx.render_mip(cid, cam_n, rc_n, out=img_n)
        torch.cuda.synchronize()
        reps = 10
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            ctx.render_mip(cid, cam_n, rc_n, out=img_n)
        e1.record(st)
        torch.cuda.synchronize()
        n_ms = e0.elapsed_time(e1) / reps
        n_samp = ctx.last_render_samples()
        n_path = ctx.last_render_path()
        n_bytes = n_samp * {"f32": 4, "bf16": 2, "fp8": 1}[w["storage"]]
        n_gbs = n_bytes / (n_ms / 1e3) / 1e9
        mip_native = {"ms": n_ms, "samples": n_samp, "samples_per_s": n_samp / (n_ms / 1e3), "hbm_gbs": n_gbs,
                      "hbm_frac": n_gbs / pk["hbm_gbs"], "hbm_peak_kind": pk_kind, "render_path": n_path,
                      "note": "orthographic MIP along z at native resolution (%dx%d pixels, step 1, nearest): one "
                              "sample per voxel, each voxel read once; algorithmic bytes = stored bytes of the "
                              "samples; cube larger than L2" % (NX, NY)}

    # latency of one view alone: each orbit view rendered by its own call
    # (n_views = 1), CUDA events around each call, three rounds over the orbit
    view_ms = []
    if not args.no_view_latency:
        ctx.render_dvr(cid, cams[:1], rc, tf, w["term"], out=out[:1])
        for _ in range(3):
            for i, cam in enumerate(cams):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                ctx.render_dvr(cid, [cam], rc, tf, w["term"], out=out[i:i + 1])
                e1.record(st)
                e1.synchronize()
                view_ms.append(e0.elapsed_time(e1))
    view_latency = None
    if view_ms:
        view_latency = {"p50_ms": float(np.percentile(view_ms, 50)), "p99_ms": float(np.percentile(view_ms, 99)),
                        "max_ms": float(np.max(view_ms)), "renders": len(view_ms),
                        "note": "one 1920x1080 view per render call (the orbit's views, 3 rounds), CUDA events; "
                                "the batched step renders all views in one launch"}

    # end to end through the public API with host buffers.  Every step uploads
    # its cube from pinned host memory, computes the statistics, renders the
    # views and copies images and statistics back to pinned host memory.  The
    # steps are pipelined on three streams: step i+1's upload (its host-to-
    # device copy) overlaps step i's render, and step i's images are copied
    # back while step i+1 renders (double-buffered images).  The cubes are
    # freed after the timed region.
    e2e = None
    if not args.no_e2e:
        vt = torch.from_numpy(v).pin_memory()
        outs = [out, torch.empty_like(out)]
        host_img = [torch.empty(out.shape, dtype=torch.float32, pin_memory=True) for _ in range(2)]
        dst = [dstats, torch.empty_like(dstats)]
        dhi = [dhist, torch.empty_like(dhist)]
        host_stats = torch.empty(8, dtype=torch.float64, pin_memory=True)
        host_hist = torch.empty(w["nbins"], dtype=torch.int64, pin_memory=True)
        s_up, s_rd, s_dn = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        rendered = [torch.cuda.Event(), torch.cuda.Event()]
        # at least 32 steps: the first upload and the last image copy (pipeline
        # fill and drain) stay inside the timed region but do not dominate it
        e2e_steps = max(32, args.steps)
        arrived = [torch.cuda.Event(enable_timing=True) for _ in range(e2e_steps)]
        ctx.cube_free(cid)
        cid = None
        torch.cuda.synchronize()
        def issue_step(i, cube):
            b = i % 2
            if i >= 2:
                s_rd.wait_event(copied[b])          # images and statistics of step i-2 are back on the host
            ctx.cube_stats_async(cube, w["nbins"], dst[b], dhi[b], stream=s_rd)
            ctx.render_dvr(cube, cams, rc, tf, w["term"], out=outs[b], stream=s_rd)
            rendered[b].record(s_rd)

        # Order of host calls: step i+1 is issued before step i's images are
        # copied back.  A render's small input tables are read from host memory
        # by the device; such reads wait behind an image download in flight to
        # host memory, so they go first.
        t0 = time.perf_counter()
        cubes = [ctx.cube_upload(vt, w["storage"], brick=w["brick"], stream=s_up)]
        issue_step(0, cubes[0])
        if e2e_steps > 1:
            cubes.append(ctx.cube_upload(vt, w["storage"], brick=w["brick"], stream=s_up))
        for i in range(e2e_steps):
            b = i % 2
            if i + 1 < e2e_steps:
                issue_step(i + 1, cubes[i + 1])
            s_dn.wait_event(rendered[b])
            with torch.cuda.stream(s_dn):
                host_img[b].copy_(outs[b], non_blocking=True)
                host_stats.copy_(dst[b], non_blocking=True)
                host_hist.copy_(dhi[b], non_blocking=True)
            copied[b].record(s_dn)
            arrived[i].record(s_dn)
            # every read of cube i is ordered before the copies on s_dn: release
            # it there, so a later upload reuses its memory without a device wait
            ctx.cube_free_async(cubes[i], stream=s_dn)
            if i + 2 < e2e_steps:
                # its host-to-device copy overlaps the render of step i+1
                cubes.append(ctx.cube_upload(vt, w["storage"], brick=w["brick"], stream=s_up))
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        e2e_s = barrier_max(e2e_s, ws)
        period = [arrived[i - 1].elapsed_time(arrived[i]) for i in range(1, e2e_steps)]
        e2e = {"value": ws * samples_per_step / e2e_s, "unit": "samples/s",
               "h2d_bytes_per_step": int(v.nbytes + 4096 + 48 * len(cams)),
               "d2h_bytes_per_step": int(host_img[0].numel() * 4 + 8 * w["nbins"] + 64),
               "ms_per_step": 1e3 * e2e_s, "steps": e2e_steps,
               "steady_ms_per_step": float(np.median(period)),
               "pipeline": "upload of step i+2 overlaps the render of step i+1; images of step i copied back "
                           "while step i+1 renders; each cube released in stream order after its images "
                           "(vrc_cube_free_async), so uploads reuse its memory; timed from the first upload to "
                           "the last image on the host (fill and drain included); steady_ms_per_step = median interval "
                           "between consecutive steps' images arriving on the host"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, npix, nsamp, el, nv = oracle_rate(v, cams, tf, w, info["vmin"], info["vmax"], args.cpu_seconds)
        cpu = {"value": rate, "unit": "samples/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{npix} random pixels of {nv} views ({nsamp} samples, {el:.1f} s), FP64 oracle, OpenMP"}

    # precision forms: the same step with the cube stored as bf16 and fp8
    precision = None
    if not args.no_precision and w["storage"] == "f32":
        fp32_row = {"step_samples_per_s": samples_per_step / ((render_ms + stats_ms) / 1e3),
                    "samples_per_s": samples_per_step / (render_ms / 1e3), "render_ms": render_ms,
                    "stats_ms": stats_ms, "view_latency": view_latency, "render_path": render_path}
        precision = precision_forms(ctx, v, cams, tf, w, rc, out, args, fp32_row)
    if cid is not None:
        ctx.cube_free(cid)
    ctx.close()   # the serving contexts below need the device memory this one caches
    serving = serving_forms(args) if (not args.no_serving and rank == 0) else None
    serving_budget = (serving_budget_forms(args) if (not args.no_serving and not args.no_serving_budget and rank == 0)
                      else None)

    # the committed captures are of the default step (fp32 cube, fused path, 32 views)
    profiled = w["name"] == "dvr1024" and w["storage"] == "f32" and args.path == "fused" and len(cams) == 32
    if rank == 0:
        line = {"metric": "ray samples/s (DVR, trilinear)", "value": value, "unit": "samples/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": w["storage"],
                "data": "synthetic",
                "config": dict(workload_config(w, len(cams)),
                               **{"samples_per_step": samples_per_step, "parallelism": f"replicas{ws}",
                                  "render_copy_bytes": info["render_copy_bytes"],
                                  "l2": "inputs larger than L2 (cube bricks %.1f GB > 126 MB)" % (info["bytes"] / 1e9)}),
                "roofline": {"bound": "alu", "kernel": "k_render_fused (DVR)", "achieved": achieved_tflops,
                             "peak": fp32_peak_tflops, "unit": "TFLOP/s", "frac": achieved_tflops / fp32_peak_tflops,
                             "traffic": render_traffic() if profiled else None,
                             "flops_per_sample": DVR_FLOPS_PER_SAMPLE,
                             "peak_kind": "derived: 148 SM x 128 FP32 lanes x 2 x sm_max_mhz",
                             "binding": render_binding() if profiled else None},
                "frames_per_s": len(cams) / (render_ms / 1e3), "render_path": render_path,
                "precision_forms": precision, "serving_forms": serving, "serving_budget_forms": serving_budget,
                "skip_empty_variant": skip,
                "view_latency": view_latency, "mip_native": mip_native,
                "kernels": {"render_ms": render_ms, "stats_ms": stats_ms, "median_ms": median_ms,
                            "stats_hbm_gbs": stats_gbs, "stats_hbm_frac": stats_gbs / pk["hbm_gbs"],
                            "hbm_peak_gbs": pk["hbm_gbs"], "hbm_peak_kind": pk_kind},
                "clocks": clocks, "gpu_launches": launches, "e2e": e2e, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)


# ------------------------------------------------- precision and serving forms
# Stated error bounds of the precision forms: largest difference, per RGBA
# channel, between a DVR pixel of the stored cube and the FP64 oracle on the
# original fp32 cube (the error a user sees: storage rounding plus kernel
# error).  The bound is one spacing of the storage format at 1.0 (the images'
# channels lie in [0, 1]): 2^-7 for bf16 (7 stored mantissa bits), 2^-3 for
# fp8 e4m3 (3 stored mantissa bits, per-brick scale).
ERROR_BOUNDS = {"bf16": 2.0 ** -7, "fp8": 2.0 ** -3}


def view_latency_ms(ctx, cid, cams, rc, tf, term, out, rounds=2):
    import torch
    st = torch.cuda.current_stream()
    ms = []
    ctx.render_dvr(cid, cams[:1], rc, tf, term, out=out[:1])
    for _ in range(rounds):
        for i, cam in enumerate(cams):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            ctx.render_dvr(cid, [cam], rc, tf, term, out=out[i:i + 1])
            e1.record(st)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
    return {"p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)), "renders": len(ms)}


def precision_forms(ctx, v, cams, tf, w, rc, out, args, fp32_row):
    """The step of the default workload on the cube stored as bf16 and as fp8
    e4m3 (per-brick scale): samples/s, one-view latency, and the error of
    sampled DVR pixels against the FP64 oracle on the original fp32 cube and
    on the stored cube."""
    import torch

    import oracle
    rows = {"f32": fp32_row}
    rng = np.random.default_rng(7)
    npix = w["W"] * w["H"]
    pix = rng.choice(npix, size=args.error_pixels, replace=False)
    err_views = [0, len(cams) // 2]
    dstats = torch.empty(8, dtype=torch.float64, device="cuda")
    dhist = torch.empty(w["nbins"], dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream()
    for dt in ("bf16", "fp8"):
        cid = ctx.cube_upload(v, dt, brick=w["brick"])
        info = ctx.cube_info(cid)
        for _ in range(max(args.warmup, 1)):
            ctx.cube_stats_async(cid, w["nbins"], dstats, dhist)
            ctx.render_dvr(cid, cams, rc, tf, w["term"], out=out)
        torch.cuda.synchronize()
        samples = ctx.last_render_samples()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(st)
        for _ in range(args.steps):
            ctx.cube_stats_async(cid, w["nbins"], dstats, dhist)
        e[1].record(st)
        for _ in range(args.steps):
            ctx.render_dvr(cid, cams, rc, tf, w["term"], out=out)
        e[2].record(st)
        torch.cuda.synchronize()
        stats_ms = e[0].elapsed_time(e[1]) / args.steps
        render_ms = e[1].elapsed_time(e[2]) / args.steps
        path = ctx.last_render_path()
        lat = view_latency_ms(ctx, cid, cams, rc, tf, w["term"], out)
        ctx.render_dvr(cid, cams, rc, tf, w["term"], out=out)
        torch.cuda.synchronize()
        err32, errs, fragile = 0.0, 0.0, 0
        for vi in err_views:
            got = out[vi].reshape(-1, 4).cpu().numpy().astype(np.float64)[pix]
            kw = dict(tf=tf, vmin=info["vmin"], vmax=info["vmax"], term=w["term"], pixels=pix)
            r32 = oracle.render(v, cams[vi], w["W"], w["H"], w["step"], "trilinear", "dvr", **kw)
            rst = oracle.render(v, cams[vi], w["W"], w["H"], w["step"], "trilinear", "dvr", dtype=dt,
                                brick=w["brick"], **kw)
            err32 = max(err32, float(np.abs(got - r32["out"]).max()))
            d = np.abs(got - rst["out"]).max(axis=1)
            ok = (d <= 1e-4) | (rst["fragile"] & np.all((got >= rst["lo"] - 1e-4) & (got <= rst["hi"] + 1e-4), axis=1))
            errs = max(errs, float(d[~rst["fragile"]].max()) if (~rst["fragile"]).any() else 0.0)
            fragile += int(rst["fragile"].sum())
            assert ok.all(), (dt, vi)
        rows[dt] = {"samples_per_s": samples / (render_ms / 1e3),
                    "step_samples_per_s": samples / ((render_ms + stats_ms) / 1e3), "render_ms": render_ms,
                    "stats_ms": stats_ms, "stored_bytes": info["bytes"], "render_copy_bytes": info["render_copy_bytes"],
                    "render_path": path, "view_latency": lat,
                    "dvr_max_abs_err_vs_fp32_oracle": err32, "dvr_max_abs_err_vs_stored_oracle": errs,
                    "error_bound_vs_fp32_oracle": ERROR_BOUNDS[dt], "fragile_pixels": fragile,
                    "error_sample": f"{len(pix)} random pixels of views {err_views}"}
        rows[dt]["meets_error_bound"] = err32 <= ERROR_BOUNDS[dt]
        rows[dt]["beats_fp32_samples_per_s"] = rows[dt]["step_samples_per_s"] > fp32_row["step_samples_per_s"]
        rows[dt]["beats_fp32_view_p99"] = lat["p99_ms"] < fp32_row["view_latency"]["p99_ms"]
        ctx.cube_free(cid)
    return rows


def serving_forms(args):
    """cfg4 serving, bounded: the Poisson stream (200 requests/s) over 64 cubes
    of 256^3-1024^3 (one generated volume per side) as a resident set, served
    for a few seconds with every cube stored as fp32, bf16 and fp8 in turn."""
    import torch

    import cubegen
    import paper_1111_6661_b300 as vrc
    wl = cubegen.serving_stream(seed=5, rate_hz=200.0, duration_s=args.serving_seconds, n_cubes=64)
    out = {}
    vols = {}
    for dt in ("f32", "bf16", "fp8"):
        for c in wl["cubes"]:
            c["dtype"] = dt
        ctx = vrc.Context(0, hbm_budget_bytes=220 * 2 ** 30, n_streams=4, max_inflight=32)
        ids = []
        t0 = time.perf_counter()
        for c in wl["cubes"]:
            if c["dims"] not in vols:
                vols[c["dims"]] = cubegen.generate(c["dims"], c["n_sources"], c["seed"])
            ids.append(ctx.cube_upload(vols[c["dims"]], dt, brick=128 if c["dims"][0] <= 512 else 256))
        setup = time.perf_counter() - t0
        r = serving_run(ctx, wl, ids)
        r["setup_s"] = setup
        r["resident_bytes"] = ctx.memory()[0]
        out[dt] = r
        ctx.close()
        torch.cuda.empty_cache()
    for dt in ("bf16", "fp8"):
        out[dt]["beats_fp32_p99"] = out[dt]["p99_ms"] < out["f32"]["p99_ms"]
        out[dt]["beats_fp32_p50"] = out[dt]["p50_ms"] < out["f32"]["p50_ms"]
    out["workload"] = ("Poisson 200 requests/s for %.0f s (%d requests), 64 cubes 256^3-1024^3 (one generated volume "
                       "per side), resident set, 50%% DVR / 30%% MIP / 20%% statistics, 512^2-1920x1080"
                       % (args.serving_seconds, len(wl["requests"])))
    return out


def serving_budget_forms(args):
    """cfg4 serving under the HBM budget: the same stream over the 64 cubes
    registered (kept on the host, made resident on demand, least recently used
    evicted) under 32 GiB, every cube stored as fp32, bf16 and fp8 in turn.
    The budget holds a few of the cubes, so most requests wait for an upload:
    bf16 / fp8 cubes load from their packed host copies (half / a quarter of
    the bytes) and more of them fit."""
    import torch

    import cubegen
    import paper_1111_6661_b300 as vrc
    wl = cubegen.serving_stream(seed=5, rate_hz=200.0, duration_s=args.serving_budget_seconds, n_cubes=64)
    out, vols = {}, {}
    for dt in ("f32", "bf16", "fp8"):
        for c in wl["cubes"]:
            c["dtype"] = dt
        ctx = vrc.Context(0, hbm_budget_bytes=32 * 2 ** 30, n_streams=4, max_inflight=32)
        ids = []
        t0 = time.perf_counter()
        for c in wl["cubes"]:
            if c["dims"] not in vols:
                vols[c["dims"]] = cubegen.generate(c["dims"], c["n_sources"], c["seed"])
            ids.append(ctx.cube_register(vols[c["dims"]], dt, brick=128 if c["dims"][0] <= 512 else 256))
        setup = time.perf_counter() - t0
        r = serving_run(ctx, wl, ids)
        r["setup_s"] = setup
        r["residency_counts"] = ctx.residency()
        out[dt] = r
        for i in ids:
            ctx.cube_free(i)
        ctx.close()
        torch.cuda.empty_cache()
    for dt in ("bf16", "fp8"):
        out[dt]["beats_fp32_p99"] = out[dt]["p99_ms"] < out["f32"]["p99_ms"]
        out[dt]["beats_fp32_samples_per_s"] = out[dt]["samples_per_s"] > out["f32"]["samples_per_s"]
    out["workload"] = ("Poisson 200 requests/s for %.0f s (%d requests), 64 registered cubes 256^3-1024^3 (one "
                       "generated volume per side) under a 32 GiB HBM budget, 50%% DVR / 30%% MIP / 20%% statistics, "
                       "512^2-1920x1080" % (args.serving_budget_seconds, len(wl["requests"])))
    return out


# ------------------------------------------------- axis-aligned native MIP
def run_mip_native(args):
    """Orthographic nearest MIP along z at native resolution (one sample per
    voxel, each voxel read once) on the 1024^3 bench cube (or --dims): the
    ray-casting case that HBM bounds.  Samples/s and GB/s of stored bytes."""
    import torch

    import cubegen
    import paper_1111_6661_b300 as vrc
    w = workload("dvr1024")
    if args.dims:
        w["dims"] = tuple(args.dims)
    v = cubegen.generate(w["dims"], w["n_sources"], w["seed"])
    storage = args.storage or "f32"
    ctx = vrc.Context(0)
    cid = ctx.cube_upload(v, storage, brick=w["brick"])
    NX, NY, NZ = w["dims"]
    cam = [cubegen.ortho_z_camera(w["dims"])]
    rc = vrc.raycfg(NX, NY, 1.0, "nearest")
    img = torch.empty((1, NY, NX), dtype=torch.float32, device="cuda")
    for _ in range(max(args.warmup, 1)):
        ctx.render_mip(cid, cam, rc, out=img)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        ctx.render_mip(cid, cam, rc, out=img)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    n = ctx.last_render_samples()
    pk, pk_kind = peaks()
    gbs = n * {"f32": 4, "bf16": 2, "fp8": 1}[storage] / (ms / 1e3) / 1e9
    print(json.dumps({"metric": "ray samples/s (MIP, nearest, axis-aligned native resolution)",
                      "value": n / (ms / 1e3), "unit": "samples/s", "ms_per_step": ms, "steps": args.steps,
                      "warmup": args.warmup, "dtype": storage, "data": "synthetic",
                      "config": {"workload": "mip_native", "dims": list(w["dims"]), "image": [NX, NY], "step": 1.0,
                                 "sampling": "nearest", "storage": storage},
                      "hbm_gbs": gbs, "hbm_frac": gbs / pk["hbm_gbs"], "hbm_peak_kind": pk_kind,
                      "render_path": ctx.last_render_path()}), flush=True)
    ctx.cube_free(cid)
    ctx.close()


# ---------------------------------------------------------------- precision form
def run_precision(args):
    """BF16 / FP8 storage against fp32 on the 2048x2048x4096 cube: samples/s
    per dtype and the error of every image and statistic against the FP64
    oracle, both on the original fp32 cube and on the stored (dequantised) cube."""
    import torch

    import cubegen
    import oracle
    import paper_1111_6661_b300 as vrc
    dims = tuple(args.dims) if args.dims else (2048, 2048, 4096)
    nsrc = int(16000 * (dims[0] * dims[1] * dims[2]) / 2 ** 34) or 8
    t0 = time.perf_counter()
    v = cubegen.generate(dims, nsrc, 3)
    gen_s = time.perf_counter() - t0
    views = args.views or 16
    cams = cubegen.orbit_cameras(dims, views)
    W, H = 1920, 1080
    tf = cubegen.tf_dense()
    rng = np.random.default_rng(0)
    pix = rng.choice(W * H, size=args.error_pixels, replace=False)
    ref_views = list(range(0, views, max(1, views // 2)))[:2]
    st_ref = oracle.stats(v)
    out = {}
    pk, pk_kind = peaks()
    nvox = dims[0] * dims[1] * dims[2]
    for dt in ("f32", "bf16", "fp8"):
        # a context per storage type: the previous one's cached device memory
        # (bricks, render copies, the upload's staging) goes back to the device
        ctx = vrc.Context(0)
        torch.cuda.synchronize()
        t_up = time.perf_counter()
        cid = ctx.cube_upload(v, dt, brick=256)
        upload_s = time.perf_counter() - t_up
        info = ctx.cube_info(cid)
        s, h = ctx.cube_stats(cid, 4096)
        row = {"stats": {k: s[k] for k in ("min", "max", "mean", "std")}, "upload_s": upload_s}
        # the statistics pass alone (4096 bins), CUDA events over 5 calls
        dstats = torch.empty(8, dtype=torch.float64, device="cuda")
        dhist = torch.empty(4096, dtype=torch.int64, device="cuda")
        ctx.cube_stats_async(cid, 4096, dstats, dhist)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            ctx.cube_stats_async(cid, 4096, dstats, dhist)
        e1.record()
        torch.cuda.synchronize()
        st_ms = e0.elapsed_time(e1) / 5
        st_gbs = nvox * {"f32": 4, "bf16": 2, "fp8": 1}[dt] / (st_ms / 1e3) / 1e9
        row["stats_pass"] = {"ms": st_ms, "voxels_per_s": nvox / (st_ms / 1e3), "stored_hbm_gbs": st_gbs,
                             "hbm_frac": st_gbs / pk["hbm_gbs"], "hbm_peak_kind": pk_kind}
        row["stats_rel_err_vs_fp32_oracle"] = {k: abs(s[k] - st_ref[k]) / max(abs(st_ref[k]), st_ref["std"])
                                               for k in ("min", "max", "mean", "std")}
        if dt != "f32":
            dq = oracle.dequantize(v, dt, 256)
            sq = oracle.stats(dq)
            row["stats_rel_err_vs_stored_oracle"] = {k: abs(s[k] - sq[k]) / max(abs(sq[k]), sq["std"])
                                                     for k in ("min", "max", "mean", "std")}
            del dq
        for mode in ("mip", "dvr"):
            rc = vrc.raycfg(W, H, 0.5, "trilinear")
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            img = ctx.render_mip(cid, cams, rc) if mode == "mip" else ctx.render_dvr(cid, cams, rc, tf, 0.99)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            nsamp = ctx.last_render_samples()
            errs = {"vs_fp32_oracle": [], "vs_stored_oracle": []}
            for vi in ref_views:
                got = img[vi].reshape(-1, 1 if mode == "mip" else 4).cpu().numpy().astype(np.float64)[pix]
                kw = dict(pixels=pix, tf=tf, vmin=info["vmin"], vmax=info["vmax"])
                r32 = oracle.render(v, cams[vi], W, H, 0.5, "trilinear", mode, **kw)
                rs = r32 if dt == "f32" else oracle.render(v, cams[vi], W, H, 0.5, "trilinear", mode, dtype=dt,
                                                           brick=256, **kw)
                ref32 = r32["out"].reshape(got.shape)
                refs = rs["out"].reshape(got.shape)
                hit = (r32["nsamp"] > 0)
                errs["vs_fp32_oracle"].append(float(np.abs(got - ref32)[hit].max()) if hit.any() else 0.0)
                errs["vs_stored_oracle"].append(float(np.abs(got - refs)[hit].max()) if hit.any() else 0.0)
            row[mode] = {"ms": ms, "samples": nsamp, "samples_per_s": nsamp / (ms / 1e3),
                         "max_abs_err_vs_fp32_oracle": max(errs["vs_fp32_oracle"]),
                         "max_abs_err_vs_stored_oracle": max(errs["vs_stored_oracle"])}
            del img
        row["stored_bytes"] = info["bytes"]
        row["render_copy_bytes"] = info["render_copy_bytes"]
        out[dt] = row
        ctx.cube_free(cid)
        ctx.close()
        torch.cuda.empty_cache()
    line = {"metric": "precision form: samples/s and error vs FP64 oracle per storage type", "workload":
            f"precision{dims[0]}x{dims[1]}x{dims[2]}", "views": views, "image": [W, H], "step": 0.5,
            "error_sample": f"{args.error_pixels} random pixels of views {ref_views}; stats over all voxels",
            "generate_s": gen_s, "results": out}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- out-of-core form
def host_mem_available() -> int:
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def link_probe_gbs() -> float:
    """Host-to-device link: pinned copies of a 1 GiB buffer (CUDA events)."""
    import torch
    hb = torch.empty(1 << 30, dtype=torch.uint8).pin_memory()
    db = torch.empty(hb.shape, dtype=torch.uint8, device="cuda")
    for _ in range(2):
        db.copy_(hb, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(8):
        db.copy_(hb, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    gbs = 8 * hb.numel() / (e0.elapsed_time(e1) / 1e3) / 1e9
    del db, hb
    return gbs


def ooc_window_parity(ctx, cid, dims, nsrc, seed, info, tf, x0=1536, y0=1024, win=64, dtype="f32"):
    """Orthographic view along z of a win x win window at native resolution,
    rendered from the out-of-core cube, against the oracle on a generated
    sub-box holding the window's columns (plus a two-voxel margin) over the
    full depth: rays along z keep x and y exact, so translating the camera by
    the sub-box origin gives the same samples."""
    import torch

    import cubegen
    import oracle
    import paper_1111_6661_b300 as vrc
    cx, cy, nz = x0 + win // 2, y0 + win // 2, dims[2]
    cam = cubegen.camera("ortho", (cx, cy, -1.0), (cx, cy, float(nz)), (0, 1, 0), ortho_height=float(win))
    rc = vrc.raycfg(win, win, 0.5, "trilinear")
    out = {}
    sub = cubegen.generate(dims, nsrc, seed, box=(x0 - 2, y0 - 2, 0, win + 4, win + 4, nz))
    cam_s = cubegen.camera("ortho", (cx - (x0 - 2), cy - (y0 - 2), -1.0), (cx - (x0 - 2), cy - (y0 - 2), float(nz)),
                           (0, 1, 0), ortho_height=float(win))
    for mode in ("mip", "dvr"):
        img = ctx.render_mip(cid, [cam], rc) if mode == "mip" else ctx.render_dvr(cid, [cam], rc, tf, 0.99)
        torch.cuda.synchronize()
        got = img.cpu().numpy().reshape(win * win, -1).astype(np.float64)
        # (bf16 rounding acts voxel by voxel, so the sub-box stored as bf16 holds the cube's values)
        r = oracle.render(sub, cam_s, win, win, 0.5, "trilinear", mode, tf=tf, vmin=info["vmin"], vmax=info["vmax"],
                          dtype=dtype)
        ref = r["out"].reshape(got.shape)
        if mode == "mip":
            err = float((np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)).max())
            out[mode] = {"max_rel_err": err, "ok": err <= 1e-5}
        else:
            d = np.abs(got - ref).max(axis=1)
            inside = np.all((got >= r["lo"] - 1e-4) & (got <= r["hi"] + 1e-4), axis=1)
            ok = (d <= 1e-4) | (r["fragile"] & inside)
            out[mode] = {"max_abs_err": float(d.max()), "fragile_pixels": int(r["fragile"].sum()),
                         "ok": bool(ok.all())}
    out["pixels"] = win * win
    out["window"] = [x0, y0, win]
    return out


def run_ooc(args):
    """4096x4096x3072 fp32 cube in 256^3 bricks (+halo), out of core.  Default:
    the bricks come from the seeded generator's C brick provider through a
    pinned host cache as large as host memory allows (the cube itself, 216 GB
    with halos, does not fit this machine's host memory); --aliased instead fills a
    pinned pool of --host-bricks distinct bricks that logical bricks alias."""
    import torch

    import cubegen
    import paper_1111_6661_b300 as vrc
    dims = tuple(args.dims) if args.dims else (4096, 4096, 3072)
    B = 256
    nb = [(d + B - 1) // B for d in dims]
    total = nb[0] * nb[1] * nb[2]
    nsrc = max(8, int(96000 * (dims[0] * dims[1] * dims[2]) / (4096 * 4096 * 3072)))
    seed = 4
    storage = args.storage or "f32"
    if args.aliased and storage != "f32":
        raise SystemExit("--aliased fills float32 host slots; --storage applies to the provider cube")
    es = {"f32": 4, "bf16": 2, "fp8": 1}[storage]
    brick_bytes = (B + 2 * (16 // es)) * (B + 2) * (B + 2) * es     # out-of-core rows: 16-byte aligned interiors
    avail = host_mem_available()
    ctx = vrc.Context(0)
    src = None
    t0 = time.perf_counter()
    if args.aliased:
        K = min(total, args.host_bricks)
        cid = ctx.cube_create_streamed(dims, B, K, args.ring)
        for slot in range(K):
            b = slot
            bx, by, bz = b % nb[0], (b // nb[0]) % nb[1], b // (nb[0] * nb[1])
            lo = [bx * B - 1, by * B - 1, bz * B - 1]
            box = [max(0, lo[a]) for a in range(3)]
            hi = [min(dims[a], lo[a] + B + 2) for a in range(3)]
            sub = cubegen.generate(dims, nsrc, seed, box=(box[0], box[1], box[2], hi[0] - box[0], hi[1] - box[1],
                                                          hi[2] - box[2]))
            pad = [(box[a] - lo[a], lo[a] + B + 2 - hi[a]) for a in (2, 1, 0)]
            ctx.cube_put_brick(cid, slot, np.pad(sub, pad, mode="edge"))
    else:
        # host cache: every brick if it fits, else what 70% of the available
        # host memory holds (the rest is regenerated on demand)
        K = total if total * brick_bytes <= 0.7 * avail else max(2, int(0.7 * avail) // brick_bytes)
        K = min(K, args.host_bricks) if args.host_bricks > 0 else K
        src = cubegen.BrickSource(dims, nsrc, seed, B)
        cid = ctx.cube_upload_streamed(dims, B, (src.fn, src.user), K, args.ring, storage=storage)
    create_s = time.perf_counter() - t0
    scan_calls = src.calls if src else 0
    link_gbs = link_probe_gbs()
    cams = cubegen.orbit_cameras(dims, 1)
    rc = vrc.raycfg(1920, 1080, 0.5, "trilinear")
    tf = cubegen.tf_sparse()
    out = torch.empty((1, 1080, 1920, 4), device="cuda")
    frames = []
    for f in range(max(1, args.steps)):
        c0 = src.calls if src else 0
        w0 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.render_dvr(cid, cams, rc, tf, 0.99, out=out)
        e1.record()
        torch.cuda.synchronize()
        frames.append({"frame_ms": e0.elapsed_time(e1), "wall_ms": 1e3 * (time.perf_counter() - w0),
                       "provider_calls": (src.calls - c0) if src else 0})
    nsamp = ctx.last_render_samples()
    traversed, culled = ctx.last_render_bricks()
    info = ctx.cube_info(cid)
    streamed = traversed * brick_bytes
    frame_ms = frames[-1]["frame_ms"]
    parity = None
    if not args.aliased and not args.no_parity and storage != "fp8":
        parity = ooc_window_parity(ctx, cid, dims, nsrc, seed, info, tf,
                                   x0=min(1536, dims[0] - 68), y0=min(1024, dims[1] - 68), dtype=storage)
    elif storage == "fp8":
        parity = {"skipped": "fp8 codes depend on the scale of each whole brick, which a generated sub-box of "
                             "the window does not reproduce; the fp8 out-of-core cube equals the resident fp8 cube "
                             "brick for brick (tests/test_gpu_streaming.py)"}
    overlap = None
    if not args.aliased and K == total and dims[0] * dims[1] * dims[2] * 4 <= 0.25 * avail:
        # copy/compute overlap of the streamed frame: the same view rendered by
        # the same brick kernels (sort-last, global loads) from resident bricks
        # gives the compute time; the pinned-copy probe gives the copy time
        rid = ctx.cube_upload(cubegen.generate(dims, nsrc, seed), storage, brick=B, render_copy="none")
        rs = vrc.raycfg(1920, 1080, 0.5, "trilinear", path="sortlast")
        ref = out.clone()
        ct = []
        for _ in range(3):
            e0.record()
            ctx.render_dvr(rid, cams, rs, tf, 0.99, out=out)
            e1.record()
            torch.cuda.synchronize()
            ct.append(e0.elapsed_time(e1))
        comp_ms = float(np.median(ct))
        copy_ms = streamed / (link_gbs * 1e9) * 1e3
        hidden = copy_ms + comp_ms - frame_ms
        overlap = {"compute_ms_resident": comp_ms, "copy_ms_at_probe": copy_ms, "frame_ms": frame_ms,
                   "overlap_pct": max(0.0, min(100.0, 100.0 * hidden / min(copy_ms, comp_ms))),
                   "max_abs_diff_vs_streamed": float((ref - out).abs().max()),
                   "note": "share of the shorter of copy and compute hidden under the other: "
                           "(copy + compute - frame) / min(copy, compute); compute = the same sort-last "
                           "render from resident bricks, copy = streamed bytes at the pinned-copy probe"}
        ctx.cube_free(rid)
        out.copy_(ref)
    zc = None
    if args.zerocopy_frames > 0 and (args.aliased or K == total):
        # zero-copy variant: the brick kernels read the mapped pinned slots in place
        ref = out.clone()
        rz = vrc.raycfg(1920, 1080, 0.5, "trilinear", path="zerocopy")
        zt = []
        for _ in range(args.zerocopy_frames):
            e0.record()
            ctx.render_dvr(cid, cams, rz, tf, 0.99, out=out)
            e1.record()
            torch.cuda.synchronize()
            zt.append(e0.elapsed_time(e1))
        zms = float(np.median(zt))
        zc = {"frame_ms": zms, "frames": len(zt), "max_abs_diff_vs_streamed": float((ref - out).abs().max()),
              "brick_bytes_per_s": streamed / (zms / 1e3),
              "note": "bricks read in place from mapped pinned host memory; no device ring, no copies"}
    line = {"metric": "out-of-core DVR frame time", "value": frame_ms, "unit": "ms", "higher_is_better": False,
            "workload": f"ooc{dims[0]}x{dims[1]}x{dims[2]}", "storage": storage, "bricks": total, "host_slots": K,
            "host_mem_available_bytes": avail, "host_pinned_bytes": K * brick_bytes,
            "mode": "aliased pool" if args.aliased else "brick provider (seeded generator) + host cache",
            "create_s": create_s, "scan_provider_calls": scan_calls, "frames": frames,
            "ring_bricks": args.ring, "brick_bytes": brick_bytes, "bricks_traversed": traversed,
            "bricks_culled": culled, "bytes_streamed_per_frame": streamed,
            "achieved_link_gbs": streamed / (frame_ms / 1e3) / 1e9, "pinned_h2d_probe_gbs": link_gbs,
            "link_bound_frame_ms": streamed / (link_gbs * 1e9) * 1e3, "samples": nsamp,
            "samples_per_s": nsamp / (frame_ms / 1e3), "parity_window": parity, "copy_compute_overlap": overlap,
            "note": ("bricks missing from the host cache are generated on the rendering thread before their "
                     "copies (provider-bound frames)") if not args.aliased else
                    "logical brick b reads pinned host slot b % host_slots",
            "zero_copy_variant": zc}
    ctx.cube_free(cid)
    ctx.close()
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- serving form
def serving_run(ctx, wl, cube_ids, duration_s=None, seed_outs=8):
    """Submit the request stream in real time (Poisson arrivals) and poll every
    ticket; latency per request, samples/s and memory waits."""
    import torch

    import cubegen
    import paper_1111_6661_b300 as vrc
    outs = {}
    for (w, h) in [(512, 512), (1024, 1024), (1920, 1080)]:
        outs[(w, h)] = [torch.empty(w * h * 4, device="cuda") for _ in range(seed_outs)]
    hists = [torch.empty(4096, dtype=torch.int64, device="cuda") for _ in range(seed_outs)]
    reqs = [r for r in wl["requests"] if duration_s is None or r["t"] < duration_s]
    tickets = []
    start = time.perf_counter()
    for i, r in enumerate(reqs):
        now = time.perf_counter() - start
        if r["t"] > now:
            time.sleep(r["t"] - now)
        cid = cube_ids[r["cube"]]
        dims = wl["cubes"][r["cube"]]["dims"]
        if r["kind"] == "stats":
            t = ctx.submit("stats", cid, nbins=4096, out=hists[i % seed_outs])
        else:
            cam = cubegen.random_cameras(dims, 1, r["view_seed"])[0]
            rc = vrc.raycfg(r["width"], r["height"], 0.5, "trilinear")
            tf = cubegen.tf_random(r["tf_seed"] % 1000)
            t = ctx.submit(r["kind"], cid, cam=cam, rc=rc, tf=tf, out=outs[(r["width"], r["height"])][i % seed_outs])
        tickets.append((t, r["kind"]))
    res = [(ctx.poll(t, -1), k) for t, k in tickets]
    wall = time.perf_counter() - start
    lat = np.array([r["latency_ms"] for r, _ in res])
    waits = np.array([r["memory_wait_ms"] for r, _ in res])
    samples = sum(r["samples"] for r, _ in res)
    bykind = {}
    for kind in ("dvr", "mip", "stats"):
        l = np.array([r["latency_ms"] for r, k in res if k == kind])
        if l.size:
            bykind[kind] = {"n": int(l.size), "p50_ms": float(np.percentile(l, 50)), "p99_ms": float(np.percentile(l, 99))}
    paths = {}
    for r, k in res:
        if k != "stats":
            paths[r["path"]] = paths.get(r["path"], 0) + 1
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "samples_per_s": samples / wall, "requests": len(res),
            "errors": int(sum(1 for r, _ in res if r["status"] != 0)), "wall_s": wall, "by_kind": bykind,
            "queue_ms_p99": float(np.percentile([r["queue_ms"] for r, _ in res], 99)),
            "memory_waits": {"requests_waited": int((waits > 0).sum()),
                             "p50_ms_of_waited": float(np.percentile(waits[waits > 0], 50)) if (waits > 0).any() else 0.0,
                             "p99_ms": float(np.percentile(waits, 99)),
                             "uploads_triggered": int(sum(1 for r, _ in res if r["cube_loaded"]))},
            "render_paths": paths}


def make_serving_cubes(ctx, wl, registered: bool, shared_volumes: bool):
    """Cubes of the serving workload: uploaded (resident set) or registered
    (made resident on demand under the budget).  shared_volumes: one generated
    volume per cube side, shared by every cube of that side (bounds the host
    generation time; every cube is still uploaded, cached and evicted on its own)."""
    import cubegen
    vols, ids = {}, []
    t0 = time.perf_counter()
    for c in wl["cubes"]:
        key = c["dims"] if shared_volumes else (c["dims"], c["seed"])
        if key not in vols:
            vols[key] = cubegen.generate(c["dims"], c["n_sources"], c["seed"])
        brick = 128 if c["dims"][0] <= 512 else 256
        if registered:
            ids.append(ctx.cube_register(vols[key], c["dtype"], brick=brick))
        else:
            ids.append(ctx.cube_upload(vols[key], c["dtype"], brick=brick))
    return ids, vols, time.perf_counter() - t0


def run_serving(args):
    import paper_1111_6661_b300 as vrc
    import cubegen
    wl = cubegen.serving_stream(seed=5, rate_hz=args.rate, duration_s=args.duration, n_cubes=args.n_cubes)
    if args.serving_dtype != "mix":
        for c in wl["cubes"]:
            c["dtype"] = args.serving_dtype
    registered = args.residency == "registered"
    budget = args.budget_gib if args.budget_gib > 0 else (32.0 if registered else 200.0)
    ctx = vrc.Context(0, hbm_budget_bytes=int(budget * 2 ** 30), n_streams=4, max_inflight=32)
    ids, vols, load_s = make_serving_cubes(ctx, wl, registered, args.shared_volumes)
    used, bud = ctx.memory()
    line = {"metric": "serving p50/p99 latency and samples/s", "rate_hz": args.rate, "duration_s": args.duration,
            "cubes": len(ids), "cube_dtype": args.serving_dtype,
            "residency": "registered (uploaded on demand, LRU eviction under the budget)" if registered else
                         "resident set (all cubes uploaded before the stream)",
            "distinct_volumes": len(vols), "host_cube_bytes": int(sum(v.nbytes for v in vols.values())),
            "resident_bytes_at_start": used, "budget_bytes": bud, "setup_s": load_s}
    line.update(serving_run(ctx, wl, ids))
    line["residency_counts"] = ctx.residency()
    line["resident_bytes_at_end"] = ctx.memory()[0]
    ctx.close()
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dvr1024")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-skip-variant", action="store_true")
    ap.add_argument("--no-view-latency", action="store_true")
    ap.add_argument("--no-mip-native", action="store_true")
    ap.add_argument("--storage", default=None, choices=["f32", "bf16", "fp8"],
                    help="storage type of the cube (default workload, mip_native, ooc provider cube: fp32)")
    ap.add_argument("--path", default="fused", choices=["fused", "slab", "sortlast"],
                    help="render path of the timed step")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-precision", action="store_true", help="skip the bf16/fp8 forms of the default step")
    ap.add_argument("--no-serving", action="store_true", help="skip the bounded serving run per storage type")
    ap.add_argument("--serving-seconds", type=float, default=8.0)
    ap.add_argument("--no-serving-budget", action="store_true",
                    help="skip the serving run of registered cubes under the 32 GiB budget")
    ap.add_argument("--serving-budget-seconds", type=float, default=6.0)
    ap.add_argument("--views", type=int, default=0, help="override the workload's view count (profiling)")
    ap.add_argument("--dims", type=int, nargs=3, default=None, help="precision/ooc: cube dims")
    ap.add_argument("--error-pixels", type=int, default=4096)
    ap.add_argument("--host-bricks", type=int, default=0,
                    help="ooc: host slots (aliased pool: default 512; provider cache: 0 = as many as fit)")
    ap.add_argument("--aliased", action="store_true", help="ooc: caller-filled aliased pool instead of the provider")
    ap.add_argument("--no-parity", action="store_true", help="ooc: skip the oracle check of a window")
    ap.add_argument("--ring", type=int, default=8)
    ap.add_argument("--zerocopy-frames", type=int, default=1,
                    help="ooc workload: frames timed with the zero-copy path (0 = skip)")
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--duration", type=float, default=20.0)
    ap.add_argument("--n-cubes", type=int, default=64)
    ap.add_argument("--budget-gib", type=float, default=0.0,
                    help="serving: HBM budget (0 = 32 GiB for registered cubes, 200 GiB for a resident set)")
    ap.add_argument("--serving-dtype", default="mix", choices=["mix", "f32", "bf16", "fp8"])
    ap.add_argument("--residency", default="registered", choices=["registered", "resident"],
                    help="serving: cubes registered (uploaded on demand under the budget) or all uploaded first")
    ap.add_argument("--shared-volumes", action="store_true",
                    help="serving: one generated volume per cube side, shared by the cubes of that side")
    args = ap.parse_args()
    if args.workload == "precision":
        return run_precision(args)
    if args.workload == "mip_native":
        return run_mip_native(args)
    if args.workload == "ooc":
        if args.aliased and args.host_bricks <= 0:
            args.host_bricks = 512
        return run_ooc(args)
    if args.workload == "serving":
        return run_serving(args)
    w = workload(args.workload)
    if args.views:
        w["views"] = args.views
    if args.storage:
        w["storage"] = args.storage
    if args.dims:   # profiling: a smaller cube of the same recipe (sources scaled with the volume)
        scale = args.dims[0] * args.dims[1] * args.dims[2] / float(np.prod(w["dims"]))
        w["dims"] = tuple(args.dims)
        w["n_sources"] = max(1, int(round(w["n_sources"] * scale)))
        w["name"] = w["name"] + "-dims%dx%dx%d" % tuple(args.dims)
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_gpu(args, w)


if __name__ == "__main__":
    main()
