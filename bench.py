#!/usr/bin/env python
"""Benchmark of the Top-K feature render training step on B300.

    python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]
                    [--workload frame] [--no-graph] [--no-cpu-baseline] [--no-e2e]

A step is one pass of the whole hot path over one synthetic batch: EWA projection,
tile binning + radix sort, the Top-K walk, the gather-blend (forward), the training loss
(1 - cosine on features, L1 on colour and depth) and the full adjoint down to every
per-Gaussian gradient.  The default workload is 200k Gaussians (80% on 5 planes, 20%
clutter), 640x480, D=512, K=8, float32 ('frame').  Inputs are resident in HBM; the
step's working set (410 MB of feature rows, 629 MB of F, 629 MB of target features) is
larger than the 126 MB L2, so nothing is flushed between steps.  The step is replayed
as one CUDA graph (--no-graph: direct launches).

Prints ONE JSON line (rank 0).  With N>1 (torchrun) every rank renders its own
replica of the workload (replicas only: the path has no exchange step) and the line
reports total pixels over the max per-rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TopK feature render fwd+bwd Mpix/s (D=512,K=8), BF16-batched vs FP32; %HBM peak"
UNIT = "Mpix/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
            # the sampler is live (first row in) before the timed region starts
            t0 = time.time()
            while not self.rows and time.time() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [r for r in self.rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ----------------------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------------------
class Step:
    """All buffers of one training step, resident on the device."""

    def __init__(self, workload, seed=0, tile=None, scene=None, max_instances=0, topk_layout=0, depth_cut=True):
        import torch
        import gs_scenes as S
        from paper_2602_06991_b300.renderer import TopKRenderer
        sc, cams, K, tile0, fdt = scene if scene is not None else S.make_config(workload, seed)
        tile = tuple(tile) if tile is not None else tile0
        self.scene, self.cams, self.K, self.tile, self.fdt = sc, cams, K, tile, fdt
        self.r = TopKRenderer(cams, K=K, D=sc.d, tile=tile, feat_dtype=fdt, check_overflow=True,
                              max_instances=max_instances, topk_layout=topk_layout, depth_cut=depth_cut)
        self.layout = topk_layout
        dev = self.r.device
        tdt = self.r.feat_torch_dtype
        t = lambda a, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(a)).to(dev).to(dt).contiguous()
        self.inp = [t(sc.mean3d), t(sc.cov3d), t(sc.opacity), t(sc.rgb), t(sc.feats, tdt)]
        # loss targets: 12 Voronoi cells per view, expanded on the device from labels
        lab, fv, cv, dv = S.voronoi_sites(seed + 100, cams, sc.d)
        lab = torch.from_numpy(lab).to(dev).long()
        self.tgt = [t(fv, tdt)[lab].contiguous(), t(cv)[lab].contiguous(), t(dv)[lab].contiguous()]
        del lab
        self.N, self.P, self.D = sc.n, self.r.P, sc.d
        # the first forward and backward check the instance and partial-row capacities
        # once (host syncs, growing them if needed), then steps run free
        self.out = self.r.forward(*self.inp)
        self.lo = self.r.alloc_loss()
        self.r.blend_loss(self.inp[4], self.tgt[0], self.tgt[1], self.tgt[2], lo=self.lo)
        self.grads = self.r.alloc_grads(self.N)
        self.r.backward(self.lo["dL_dF"], self.lo["dL_dC"], self.lo["dL_dD"], grads=self.grads)
        self.r.check_overflow = False
        torch.cuda.synchronize()

    def run(self, events=None):
        """preprocess, bin_sort, topk_select | fused blend + loss | backward"""
        r, o = self.r, self.out
        if events: events[0].record()
        r._select_into(self.N, *self.inp[:4], o)
        if events: events[1].record()
        r.blend_loss(self.inp[4], self.tgt[0], self.tgt[1], self.tgt[2], lo=self.lo)
        if events: events[2].record()
        r.backward(self.lo["dL_dF"], self.lo["dL_dC"], self.lo["dL_dD"], grads=self.grads, h_from_loss=True)
        if events: events[3].record()

    def run_blend_only(self):
        import ctypes
        from paper_2602_06991_b300.renderer import _p
        o = self.out
        self.r.lib.gs_feature_blend(ctypes.byref(self.r.cfg), self.P, self.N, _p(o["topk_idx"]), _p(o["topk_w"]),
                                    _p(self.inp[4]), _p(o["F"]), self.r._stream())


def run_bf16_batched(args, hbm, sm_mhz=None):
    """The BF16 multi-keyframe form: 1M Gaussians, BF16 rows, 8 orbit keyframes of mixed
    resolution rendered and back-propagated as one step (one launch per stage over all
    views, the whole step one CUDA graph), tile shape picked by the autotuner."""
    import torch
    import gs_scenes as S
    from paper_2602_06991_b300 import autotune
    scene = S.make_config("batched", 0)
    sc, cams, K0, tile0, fdt = scene
    sweep = []
    main_launches = None
    for K in (4, 8, 16):
        # K is the model's parameter (it changes the render); the tile shape is tuned per K
        scene_k = (sc, cams, K, tile0, fdt)
        tuned = autotune.tune(cams, sc.n, K, sc.d, fdt,
                              lambda tile, lay: Step("batched", tile=tile, scene=scene_k, topk_layout=lay).run)
        torch.cuda.empty_cache()
        step = Step("batched", tile=tuned["tile"], scene=scene_k, topk_layout=autotune.KBUF_LAYOUTS[tuned["layout"]])
        ms = autotune.time_step(lambda: step.run, reps=max(5, min(args.steps, 20)), warmup=args.warmup)
        st = status_of(step)
        sweep.append({"K": K, "tile": list(tuned["tile"]), "kbuf_layout": tuned["layout"], "ms_per_step": round(ms, 4),
                      "value": round(step.P / (ms * 1e-3) / 1e6, 3), "autotune_ms": tuned["ms"], "status": st})
        if K == K0:
            main_roof = stage_rooflines(step, hbm)
            main_kernels = kernel_rooflines(step, hbm, sm_mhz)
            main_launches = None if args.no_launch_count else count_launches(step)
        P, N, D = step.P, step.N, step.D
        del step
        torch.cuda.empty_cache()
    main = next(r for r in sweep if r["K"] == K0)
    launches = main_launches if main_launches else 70
    node_ms = graph_node_cost(launches)
    out = {"value": main["value"], "unit": UNIT, "ms_per_step": main["ms_per_step"], "pixels_per_step": P,
           "graph": {"launches_per_step": launches, "graph_of_as_many_empty_nodes_ms": round(node_ms, 4),
                     "share_of_step": round(node_ms / main["ms_per_step"], 4),
                     "note": "bound on what one persistent launch of the same stages could save over the graph"},
           "gaussians": N, "views": len(cams), "D": D, "K": K0, "dtype": "bf16", "tile": main["tile"],
           "kbuf_layout": main["kbuf_layout"],
           "status": main["status"], "roofline": main_roof["blend_loss"], "backward_roofline": main_roof["backward"],
           "kernels": main_kernels,
           "autotune_ms": main["autotune_ms"], "k_sweep": [{k: v for k, v in r.items() if k != "autotune_ms"}
                                                            for r in sweep],
           "workload": "batched: " + S.CONFIGS["batched"]}
    if any(r["status"] != "ok" for r in sweep):
        out["rejected"] = "a workspace status after timed steps was not ok"
    return out


MAPPING_INSTANCES = 1_150_000_000


def run_mapping(args, hbm, iters=100, sm_mhz=None):
    """The mapping-iteration workload: 3M Gaussians (70% on 20 planes and boxes, 30%
    clutter), 8 keyframes of 1200x680, D=768 BF16 rows, K=16.  One iteration renders and
    back-propagates all 8 views (a1-a3, the fused a4 + loss, a5 with every per-Gaussian
    feature and geometry gradient) and takes the fused Adam step over every parameter:
    float32 master weights, the bf16 feature rows the renderer reads refreshed by the same
    launch.  `iters` iterations are captured into one CUDA graph (each with its own Adam
    step count) and replayed; timed by CUDA events on the launching stream."""
    import torch
    import gs_scenes as S
    from paper_2602_06991_b300.hybrid import AdamState, adam_step
    scene = S.make_config("mapping", 0)
    sc, cams, K, tile, fdt = scene
    step = Step("mapping", scene=scene, max_instances=MAPPING_INSTANCES)
    feat32 = torch.from_numpy(sc.feats).cuda()
    del scene, sc
    params = {"mean3d": step.inp[0], "cov3d": step.inp[1], "opacity": step.inp[2], "rgb": step.inp[3],
              "feat": feat32}
    grads = {k: step.grads[k] for k in ("mean3d", "cov3d", "opacity", "rgb", "feat")}
    lr = {"mean3d": 1e-5, "cov3d": 1e-7, "opacity": 1e-4, "rgb": 1e-4, "feat": 1e-4}
    state = AdamState(params)
    copies = {"feat": step.inp[4]}

    def iteration():
        step.run()
        adam_step(params, grads, state, lr, bf16_copies=copies)

    for _ in range(2):
        iteration()
    torch.cuda.synchronize()
    n_inst, n_rows = step.r.counts()
    # stage times of one iteration (direct launches, events on the launching stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    step.run(ev[:4])
    adam_step(params, grads, state, lr, bf16_copies=copies)
    ev[4].record()
    torch.cuda.synchronize()
    stages = {"select_ms": ev[0].elapsed_time(ev[1]), "blend_loss_ms": ev[1].elapsed_time(ev[2]),
              "backward_ms": ev[2].elapsed_time(ev[3]), "adam_ms": ev[3].elapsed_time(ev[4])}
    stream = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        iteration()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(iters):
            iteration()
    g.replay()                                   # warm-up replay
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    g.replay()
    t1.record()
    torch.cuda.synchronize()
    status = status_of(step)
    ms = t0.elapsed_time(t1) / iters
    sr = stage_rooflines(step, hbm, reps=3)
    kr = kernel_rooflines(step, hbm, sm_mhz, reps=2)
    out = {"value": round(step.P / (ms * 1e-3) / 1e6, 3), "unit": UNIT, "ms_per_iteration": round(ms, 3),
           "iterations": iters, "captured": "one CUDA graph of all iterations, replayed once after a warm-up replay",
           "pixels_per_iteration": step.P, "gaussians": step.N, "views": len(cams), "D": step.D, "K": step.K,
           "dtype": "bf16", "instances": n_inst, "instance_capacity": MAPPING_INSTANCES, "feature_rows": n_rows,
           "status": status, "stages": {k: round(v, 3) for k, v in stages.items()},
           "roofline": sr["blend_loss"], "backward_roofline": sr["backward"], "kernels": kr,
           "workload": "mapping: " + S.CONFIGS["mapping"]}
    if status != "ok":
        out["rejected"] = f"workspace status after the timed iterations: {status}"
    del g, step, params, grads, state, feat32
    torch.cuda.empty_cache()
    return out


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.txt")


def source_digest(rel):
    """Short digest of a kernel source file: an ncu traffic figure is reported only while
    the kernel's source is the one it was measured on."""
    import hashlib
    with open(os.path.join(ROOT, rel), "rb") as fh:
        return hashlib.sha1(fh.read()).hexdigest()[:12]


def measured_traffic(kernel, rel_src):
    """DRAM bytes (read + write) per launch of `kernel` on the 'frame' workload from the
    committed ncu summary, or None when absent or measured on other source."""
    try:
        with open(TRAFFIC_FILE) as fh:
            for line in fh:
                f = line.split()
                if len(f) >= 3 and not line.startswith("#") and f[0] == kernel:
                    return int(f[2]) if f[1] == source_digest(rel_src) else None
    except OSError:
        return None
    return None


def blend_loss_algorithmic_bytes(step):
    """Bytes the fused gather-blend + loss must move: F written, F_gt read and dL/dF
    written (3 P D s), the Top-K record read (P K 8), colour/depth and their targets read
    and their gradients written (P (3 + 3 + 1 + 1 + 3 + 1) 4), the re-walk's per-slot
    terms h written (P K 4), each distinct row once."""
    idx = step.out["topk_idx"]
    uniq = int(np.unique(idx.cpu().numpy()[idx.cpu().numpy() >= 0]).size)
    s = 2 if step.fdt == "bf16" else 4
    return (3 * step.P * step.D * s + step.P * step.K * 8 + step.P * 12 * 4 + step.P * step.K * 4 +
            uniq * step.D * s)


def blend_algorithmic_bytes(step):
    """Bytes the gather-blend must move: F written (P D s), the Top-K record read
    (P K (4 + 4)), and each distinct selected feature row read once (U D s)."""
    idx = step.out["topk_idx"]
    uniq = int(np.unique(idx.cpu().numpy()[idx.cpu().numpy() >= 0]).size)
    s = 2 if step.fdt == "bf16" else 4
    return step.P * step.D * s + step.P * step.K * 8 + uniq * step.D * s, uniq


def count_launches(step):
    """Kernels of this library launched by one step, counted with the torch profiler
    (CUPTI) on one extra untimed step."""
    import torch
    try:
        from torch.profiler import ProfilerActivity, profile
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            step.run()
            torch.cuda.synchronize()
        n = 0
        for ev in prof.events():
            if getattr(ev, "device_type", None) is not None and "CUDA" in str(ev.device_type):
                nm = ev.name
                if nm.startswith("void gs::") or nm.startswith("gs::") or "gs::k_" in nm:
                    n += 1
        return n if n > 0 else None
    except Exception:
        return None


def aggregate_ranks(ms: float, pixels: int, world: int, device=None):
    """Whole-job timing of N replicas: the slowest rank's ms per step and the pixels all
    ranks processed per step (barrier, then all-reduce MAX and SUM).  Every rank gets
    the same pair.  No data-path collective: only these two scalars are exchanged."""
    if world <= 1:
        return ms, pixels
    import torch
    import torch.distributed as dist
    dist.barrier()
    t_ms = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    t_px = torch.tensor([float(pixels)], dtype=torch.float64, device=device)
    dist.all_reduce(t_ms, op=dist.ReduceOp.MAX)
    dist.all_reduce(t_px, op=dist.ReduceOp.SUM)
    return float(t_ms.item()), int(round(t_px.item()))


def workload_config(workload, world, N, P, D, K, tile):
    """The `config` object of the JSON line; both arms print the same one."""
    import gs_scenes as S
    return {"workload": f"{workload}: {S.CONFIGS[workload]}", "gaussians": N, "pixels_per_step": P, "D": D, "K": K,
            "tile": list(tile), "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{world}"}


def blend_loss_bytes(P, D, K, s, uniq):
    """Bytes the fused gather-blend + loss must move: F written, F_gt read and dL/dF
    written (3 P D s), the Top-K record read (P K 8), colour/depth and their targets read
    and their gradients written (P (3 + 3 + 1 + 1 + 3 + 1) 4), the re-walk's per-slot
    terms h written (P K 4), each distinct selected row once (U D s)."""
    return 3 * P * D * s + P * K * 8 + P * 12 * 4 + P * K * 4 + uniq * D * s


def backward_bytes(P, D, K, s, N, NE):
    """Bytes the adjoint must move: dL/dF read (P D s), the Top-K record and the per-slot
    h read (P K 12), dL/dC, dL/dD, C and D read (P 8 4), the projected records read
    (NE 64), the feature gradient written (N D 4) and the geometry gradients written
    (N 13 4)."""
    return P * D * s + P * K * 12 + P * 32 + NE * 64 + N * D * 4 + N * 52


def unique_rows(step):
    idx = step.out["topk_idx"]
    v = idx[idx >= 0]
    import torch
    return int(torch.unique(v).numel())


def graph_stage_ms(fn, reps):
    """fn captured alone as one CUDA graph and replayed `reps` times (CUDA events on the
    replaying stream): its device time as it runs inside the graph-replayed step, with no
    host launch latency between its kernels and its streams ordered as the step orders them."""
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn()                                        # warm inside the side stream before capture
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    g.replay()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def stage_rooflines(step, hbm, reps=10):
    """The step's two HBM-bound stages timed alone with CUDA events on the launching
    stream (averaged over reps): the fused gather-blend + loss (one kernel and two small
    fixed-order sums) and the whole adjoint (gs_backward_ex), against their algorithmic
    bytes.  The adjoint is timed twice: by direct launches, and captured alone as a graph
    the way the step runs it (stage_ms_graph, frac_graph)."""
    import torch
    s = 2 if step.fdt == "bf16" else 4
    uniq = unique_rows(step)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    for _ in range(reps):
        step.r.blend_loss(step.inp[4], step.tgt[0], step.tgt[1], step.tgt[2], lo=step.lo)
    ev[1].record()
    for _ in range(reps):
        step.r.backward(step.lo["dL_dF"], step.lo["dL_dC"], step.lo["dL_dD"], grads=step.grads, h_from_loss=True)
    ev[2].record()
    torch.cuda.synchronize()
    bl_ms, bw_ms = ev[0].elapsed_time(ev[1]) / reps, ev[1].elapsed_time(ev[2]) / reps
    bw_graph_ms = graph_stage_ms(lambda: step.r.backward(step.lo["dL_dF"], step.lo["dL_dC"], step.lo["dL_dD"],
                                                         grads=step.grads, h_from_loss=True), reps)
    blb = blend_loss_bytes(step.P, step.D, step.K, s, uniq)
    bwb = backward_bytes(step.P, step.D, step.K, s, step.N, step.N * len(step.cams))
    kname = ("gs_feature_blend_loss (k_blend_mma: tensor-core, bf16 rows)" if step.fdt == "bf16"
             else "gs_feature_blend_loss (k_blend_loss_group: pixel groups, float32 rows)")
    out = {"blend_loss": {"kernel": kname, "bound": "hbm",
                          "achieved": round(blb / (bl_ms * 1e-3) / 1e9, 1), "peak": hbm, "unit": "GB/s",
                          "frac": round(blb / (bl_ms * 1e-3) / 1e9 / hbm, 4), "algorithmic_bytes": blb,
                          "unique_rows": uniq, "kernel_ms": round(bl_ms, 4)},
           "backward": {"stage": "gs_backward_ex (feature gradient, re-walk, projection adjoint)", "bound": "hbm",
                        "achieved": round(bwb / (bw_ms * 1e-3) / 1e9, 1), "peak": hbm, "unit": "GB/s",
                        "frac": round(bwb / (bw_ms * 1e-3) / 1e9 / hbm, 4), "algorithmic_bytes": bwb,
                        "stage_ms": round(bw_ms, 4), "stage_ms_graph": round(bw_graph_ms, 4),
                        "frac_graph": round(bwb / (bw_graph_ms * 1e-3) / 1e9 / hbm, 4)}}
    return out


# FP32-pipe operations per accepted (pixel, contributor) in the re-walk (k_walk_bwd), one
# per lane-instruction (an FMA counts once): the offset and quadratic form 9, the cut-off
# tests 4, alpha and transmittance 7, the weight 1, the colour/depth/feature term g_i 5,
# the prefix and the alpha adjoint 6, the colour/depth partials 4, the opacity, conic and
# mean partials 16.  Integer work (the Top-K slot match) and the two MUFU operations are
# not counted; nor are candidates the walk rejects.
REWALK_FP32_OPS = 52


def kernel_times(step, reps=5):
    """Device times of the timed stages from the library's kernel timers (a CUDA event
    pair recorded around each timed launch on the stream it runs on), averaged over
    `reps` steps of direct launches."""
    import torch
    from paper_2602_06991_b300 import _abi as A
    names = {"binning": A.GS_TIMER_BINNING, "tile_sort": A.GS_TIMER_TILE_SORT, "walk_fwd": A.GS_TIMER_WALK_FWD,
             "block_grad": A.GS_TIMER_BLOCK_GRAD, "walk_bwd": A.GS_TIMER_WALK_BWD, "complete": A.GS_TIMER_COMPLETE}
    acc = {k: [] for k in names}
    torch.cuda.synchronize()
    A.timer_enable(True)
    try:
        for _ in range(reps):
            step.run()
            for k, t in names.items():
                ms = A.timer_read(t)
                if ms is not None:
                    acc[k].append(ms)
    finally:
        A.timer_enable(False)
    return {k: float(np.mean(v)) for k, v in acc.items() if v}


def kernel_rooflines(step, hbm, sm_mhz, reps=5):
    """The re-walk against the FP32 ALU peak, the per-block feature-gradient kernel
    against HBM, and the binning and tile-sort times, all from kernel timers."""
    import torch
    kt = kernel_times(step, reps)
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    mhz = sm_mhz or 2032.0
    peak_ops = props.multi_processor_count * 128 * mhz * 1e6 / 1e12      # FP32 lanes x clock
    contrib = int(step.out["n_contrib"].sum().item())
    n_inst, n_rows = step.r.counts()
    out = {"timer_reps": reps}
    if "walk_bwd" in kt:
        ach = REWALK_FP32_OPS * contrib / (kt["walk_bwd"] * 1e-3) / 1e12
        out["rewalk"] = {"kernel": "k_walk_bwd (re-walk adjoint)", "bound": "alu", "achieved": round(ach, 3),
                         "peak": round(peak_ops, 2), "unit": "Tops/s (FP32 lane operations)",
                         "frac": round(ach / peak_ops, 4), "ops_per_contributor": REWALK_FP32_OPS,
                         "contributors": contrib, "kernel_ms": round(kt["walk_bwd"], 4),
                         "peak_derivation": f"{props.multi_processor_count} SMs x 128 FP32 lanes x {mhz:.0f} MHz"}
    if "block_grad" in kt:
        s = 2 if step.fdt == "bf16" else 4
        # dL/dF read, one 8-byte slot record read per Top-K slot, the partial rows written
        # (float32) with their (Gaussian, row) pair
        b = step.P * step.D * s + step.P * step.K * 8 + n_rows * (step.D * 4 + 8)
        kname = "k_block_mma (tensor-core, bf16)" if (step.fdt == "bf16" and step.D % 64 == 0) else "k_block_accum (TMA pipeline)"
        out["block_grad"] = {"kernel": kname, "bound": "hbm",
                             "achieved": round(b / (kt["block_grad"] * 1e-3) / 1e9, 1), "peak": hbm, "unit": "GB/s",
                             "frac": round(b / (kt["block_grad"] * 1e-3) / 1e9 / hbm, 4), "algorithmic_bytes": b,
                             "partial_rows": n_rows, "kernel_ms": round(kt["block_grad"], 4)}
    if "binning" in kt and "tile_sort" in kt:
        bs = step.r.binning_stats()
        out["binning"] = {"count_scan_emit_ms": round(kt["binning"], 4), "tile_sort_ms": round(kt["tile_sort"], 4),
                          "completion_ms": round(kt.get("complete", 0.0), 4),
                          "total_ms": round(kt["binning"] + kt["tile_sort"] + kt.get("complete", 0.0), 4),
                          "instances": bs["instances"], "sorted_first": bs["sorted_first"],
                          "sorted_second": bs["sorted_second"], "tiles_completed": bs["tiles_completed"],
                          "depth_cut": bool(step.r.cfg.depth_cut)}
    if "walk_fwd" in kt:
        out["walk_fwd_ms"] = round(kt["walk_fwd"], 4)
    return out


def graph_node_cost(n_nodes, reps=50):
    """Milliseconds that a CUDA graph of n_nodes trivial kernels takes per replay: the
    launch cost a step of that many graph nodes pays beyond its kernels' work, i.e. the
    most a single persistent launch of the same stages could save."""
    import torch
    x = torch.zeros(1, device="cuda")
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        x.add_(1)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        for _ in range(n_nodes):
            x.add_(1)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def status_of(step):
    """The workspace status after timed work: anything but ok rejects the timing (a
    bounded wait that ran out, or a capacity overflow, skips work)."""
    from paper_2602_06991_b300 import _abi as A
    code, _ = step.r.sync_status()
    return A.status_string(code)


def run_ours(args, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    from paper_2602_06991_b300 import build
    build()
    scene = None
    if args.views:
        import gs_scenes as S
        sc, cams, K, tile, fdt = S.make_config(args.workload, rank)
        scene = (sc, [cams[int(i)] for i in args.views.split(",")], K, tile, fdt)
    step = Step(args.workload, seed=rank, scene=scene, max_instances=args.max_instances,
                depth_cut=not args.no_depth_cut)
    stream = torch.cuda.current_stream()
    launches_per_step = None if args.no_launch_count else count_launches(step)
    graph = None
    if not args.no_graph:
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(stream)
        with torch.cuda.stream(s):
            step.run()                      # warm inside the side stream before capture
        stream.wait_stream(s)
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            step.run()
        graph = g
    fn = graph.replay if graph is not None else step.run
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    # stage breakdown (untimed pass, direct launches, events on the launching stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    step.run(events=ev)
    torch.cuda.synchronize()
    stages = {"select_ms": ev[0].elapsed_time(ev[1]), "blend_loss_ms": ev[1].elapsed_time(ev[2]),
              "backward_ms": ev[2].elapsed_time(ev[3])}
    # the same three stages, each captured alone as a graph and replayed (as the step runs them)
    stages_graph = None
    if graph is not None:
        r, o = step.r, step.out
        stages_graph = {
            "select_ms": graph_stage_ms(lambda: r._select_into(step.N, *step.inp[:4], o), 20),
            "blend_loss_ms": graph_stage_ms(lambda: r.blend_loss(step.inp[4], step.tgt[0], step.tgt[1], step.tgt[2],
                                                                 lo=step.lo), 20),
            "backward_ms": graph_stage_ms(lambda: r.backward(step.lo["dL_dF"], step.lo["dL_dC"], step.lo["dL_dD"],
                                                             grads=step.grads, h_from_loss=True), 20)}
    # blend kernel alone, averaged, for the roofline
    nb = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(nb):
        step.run_blend_only()
    e1.record()
    torch.cuda.synchronize()
    blend_ms = e0.elapsed_time(e1) / nb
    # the step's fused gather-blend + loss alone (its kernel and two small sums)
    e0.record()
    for _ in range(nb):
        step.r.blend_loss(step.inp[4], step.tgt[0], step.tgt[1], step.tgt[2], lo=step.lo)
    e1.record()
    torch.cuda.synchronize()
    blend_loss_ms = e0.elapsed_time(e1) / nb

    clocks = ClockSampler(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        fn()
    t1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    status = status_of(step)
    ms = t0.elapsed_time(t1) / args.steps
    ms, total_pixels = aggregate_ranks(ms, step.P, world, device="cuda")
    value = total_pixels / (ms * 1e-3) / 1e6

    hbm, peak_kind = peaks()
    ab, uniq = blend_algorithmic_bytes(step)
    achieved = ab / (blend_ms * 1e-3) / 1e9
    abl = blend_loss_algorithmic_bytes(step)
    achieved_bl = abl / (blend_loss_ms * 1e-3) / 1e9
    sr = stage_rooflines(step, hbm)
    res = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if step.fdt == "f32" else "bf16", "data": "synthetic",
        "config": dict(workload_config(args.workload, world, step.N, step.P, step.D, step.K, step.tile),
                       **({"views": args.views} if args.views else {}),
                       **({"depth_cut": False} if args.no_depth_cut else {})),
        "graph": graph is not None, "status": status,
        "stages": {k: round(v, 4) for k, v in stages.items()},
        "stages_graph": {k: round(v, 4) for k, v in stages_graph.items()} if stages_graph else None,
        "backward_roofline": sr["backward"],
        "roofline": {"kernel": ("gs_feature_blend_loss (k_blend_loss_group): the step's a4 stage" if step.fdt == "f32"
                                else "gs_feature_blend_loss (k_blend_mma: tensor-core, bf16 rows): the step's a4 stage"),
                     "bound": "hbm",
                     "achieved": round(achieved_bl, 1), "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": round(achieved_bl / hbm, 4),
                     # the committed DRAM capture is of the 'frame' workload's kernel
                     "traffic": (measured_traffic("k_blend_loss_group", "paper_2602_06991_b300/csrc/gs_blend.cu")
                                 if args.workload == "frame" and not args.views else None),
                     "algorithmic_bytes": abl, "unique_rows": uniq, "kernel_ms": round(blend_loss_ms, 4)},
        "rooflines_other": [
            {"kernel": "gs_feature_blend (k_blend_group): a4 alone", "bound": "hbm", "achieved": round(achieved, 1),
             "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
             "traffic": (measured_traffic("k_blend_group", "paper_2602_06991_b300/csrc/gs_blend.cu")
                         if args.workload == "frame" and not args.views else None),
             "algorithmic_bytes": ab, "kernel_ms": round(blend_ms, 4)}],
        "clocks": clk,
        "gpu_launches": (launches_per_step * args.steps) if launches_per_step else None,
        "launches_per_step": launches_per_step,
    }
    res["kernels"] = kernel_rooflines(step, hbm, clk.get("sm_mhz"))
    if rank == 0:
        res["hybrid"] = run_hybrid(step, ms)
        res["prune"] = run_prune(step)
        res["vanilla"] = run_vanilla(step)
    if rank == 0 and not args.no_e2e:
        res["e2e"] = run_e2e(step, args)
    if status != "ok":
        res["rejected"] = f"workspace status after the timed steps: {status}"
    if rank == 0 and not args.no_batched:
        del step
        torch.cuda.empty_cache()
        res["bf16_batched"] = run_bf16_batched(args, hbm, clk.get("sm_mhz"))
        res["bf16_batched"]["speedup_vs_f32_frame"] = round(res["bf16_batched"]["value"] / res["value"], 3)
    if rank == 0 and not args.no_mapping:
        torch.cuda.empty_cache()
        res["mapping"] = run_mapping(args, hbm, sm_mhz=clk.get("sm_mhz"))
    if rank == 0 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(args.workload, budget_s=args.cpu_seconds)
        # the same leg checks the BF16-row form against the oracle on sampled pixels
        try:
            res["cpu_baseline"]["bf16_form_parity"] = bf16_form_parity()
        except Exception as e:
            res["cpu_baseline"]["bf16_form_parity"] = {"unavailable": f"{type(e).__name__}: {e}"}
    return res


def run_hybrid(step, full_ms, semantic_every=4):
    """Hybrid field optimisation (Sec. 3.4): the geometry-only iteration (a1-a3, colour/
    depth loss, adjoint without its feature part) replayed as a graph, the schedule's
    mean step time with semantics every `semantic_every` iterations, and the fused Adam
    step over every parameter tensor of the workload."""
    import torch
    from paper_2602_06991_b300 import autotune
    from paper_2602_06991_b300.hybrid import AdamState, adam_step
    r = step.r
    lo = r.loss_geo(step.out["rgb"], step.tgt[1], step.out["depth"], step.tgt[2])

    def geo():
        r._select_into(step.N, *step.inp[:4], step.out)
        r.loss_geo(step.out["rgb"], step.tgt[1], step.out["depth"], step.tgt[2], out=lo)
        r.backward(None, lo["dL_dC"], lo["dL_dD"], grads=step.grads)

    geo_ms = autotune.time_step(lambda: geo, reps=20)
    avg = ((semantic_every - 1) * geo_ms + full_ms) / semantic_every
    params = {"mean3d": step.inp[0], "cov3d": step.inp[1], "opacity": step.inp[2], "rgb": step.inp[3]}
    if step.fdt == "f32":
        params["feat"] = step.inp[4]
    st = AdamState(params)
    grads = {"mean3d": step.grads["mean3d"], "cov3d": step.grads["cov3d"], "opacity": step.grads["opacity"],
             "rgb": step.grads["rgb"], "feat": step.grads["feat"]}
    lr = {k: 0.0 for k in params}                     # timing only: parameters unchanged
    adam_step(params, grads, st, lr)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        adam_step(params, grads, st, lr)
    e1.record()
    torch.cuda.synchronize()
    adam_ms = e0.elapsed_time(e1) / 20
    n_el = sum(v.numel() for v in params.values())
    return {"geometry_step_ms": round(geo_ms, 4), "full_step_ms": round(full_ms, 4), "semantic_every": semantic_every,
            "schedule_mean_step_ms": round(avg, 4), "schedule_Mpix_s": round(step.P / (avg * 1e-3) / 1e6, 3),
            "adam_ms": round(adam_ms, 4), "adam_elements": n_el,
            "adam_GBps": round(n_el * 4 * 7 / (adam_ms * 1e-3) / 1e9, 1)}


def run_vanilla(step, reps=5):
    """The full alpha-blending feature render (Tab. 4 'vanilla') of the step's view against
    the Top-K forward (a1-a3 + a4) on the same inputs, both timed with CUDA events."""
    import torch

    def timed(fn, n):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(n):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    F = torch.empty_like(step.out["F"])

    def topk_forward():
        step.r._select_into(step.N, *step.inp[:4], step.out)
        step.run_blend_only()

    topk_ms = timed(topk_forward, 10)
    van_ms = timed(lambda: step.r.forward_vanilla(step.inp[4], F), reps) + timed(
        lambda: step.r._select_into(step.N, *step.inp[:4], step.out), 10)
    return {"forward_ms": round(van_ms, 3), "topk_forward_ms": round(topk_ms, 3),
            "slowdown_vs_topk": round(van_ms / topk_ms, 2),
            "note": "vanilla = a1-a3 + full alpha-blended D-wide feature over every contributor; "
                    "topk = a1-a3 + Top-K gather-blend"}


def run_prune(step, reps=20):
    """Consistency-pruning statistics of the step's view (Sec. 3.3, Eq. 8: Top-K count and
    S = max w, one re-walk) and the survival selection over all Gaussians (Eq. 9), each
    timed with CUDA events on the launching stream."""
    import torch
    from paper_2602_06991_b300.renderer import prune_select
    acc = step.r.alloc_prune_stats(step.N)
    for _ in range(3):
        step.r.prune_stats(acc)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        step.r.prune_stats(acc)
    e1.record()
    torch.cuda.synchronize()
    stats_ms = e0.elapsed_time(e1) / reps
    acc = step.r.prune_stats(step.r.alloc_prune_stats(step.N))
    expo = torch.empty(step.N, device="cuda").exponential_()
    for _ in range(3):
        prune_select(acc["count"], acc["S"], 1, 0.5, expo)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        keep = prune_select(acc["count"], acc["S"], 1, 0.5, expo)
    e1.record()
    torch.cuda.synchronize()
    sel_ms = e0.elapsed_time(e1) / reps
    return {"stats_ms": round(stats_ms, 4), "select_ms": round(sel_ms, 4),
            "candidates": int((acc["count"] < 1).sum().item()), "kept": int(keep.sum().item()),
            "note": "per view: Top-K count + S = max w re-walk; selection: tau = 1, ratio 0.5, over all Gaussians"}


def run_e2e(step, args):
    """Same metric through the C ABI with host buffers: every step copies its inputs
    (Gaussian parameters and target maps) from pinned host memory, runs the step, and
    reads the loss and every per-Gaussian gradient back.  Steps are pipelined over two
    buffer sets (a second Step with its own renderer): step i+1's inputs go up on one
    copy stream and step i-1's results come down on another while step i computes."""
    import torch
    sets = [step, Step(args.workload, seed=0, tile=step.tile)]
    dev_in = [s.inp + s.tgt for s in sets]
    dev_out = [list(s.grads.values()) + [s.lo["loss"]] for s in sets]
    host_in = [[t.cpu().pin_memory() for t in d] for d in dev_in]
    host_out = [[t.cpu().pin_memory() for t in d] for d in dev_out]
    bi = sum(t.numel() * t.element_size() for t in host_in[0])
    bo = sum(t.numel() * t.element_size() for t in host_out[0])
    comp = torch.cuda.current_stream()
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    ev = lambda: torch.cuda.Event()

    def run(n):
        computed = [None, None]              # per set: its last compute, then its last download
        downloaded = [None, None]
        for i in range(n):
            k = i & 1
            if computed[k] is not None:
                up.wait_event(computed[k])   # the set's inputs are free once its last step ran
            with torch.cuda.stream(up):
                for h, d in zip(host_in[k], dev_in[k]):
                    d.copy_(h, non_blocking=True)
                uploaded = ev()
                uploaded.record(up)
            comp.wait_event(uploaded)
            if downloaded[k] is not None:
                comp.wait_event(downloaded[k])   # its previous results have been read back
            sets[k].run()
            computed[k] = ev()
            computed[k].record(comp)
            down.wait_event(computed[k])
            with torch.cuda.stream(down):
                for h, d in zip(host_out[k], dev_out[k]):
                    h.copy_(d, non_blocking=True)
                downloaded[k] = ev()
                downloaded[k].record(down)
        comp.wait_stream(up)
        comp.wait_stream(down)

    run(2)
    torch.cuda.synchronize()
    n = max(4, min(args.steps, 10))
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(comp)
    up.wait_event(t0)                        # the first upload starts inside the timed region
    run(n)
    t1.record(comp)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / n
    del sets[1]
    torch.cuda.empty_cache()
    return {"value": round(step.P / (ms * 1e-3) / 1e6, 3), "unit": UNIT, "h2d_bytes_per_step": bi,
            "d2h_bytes_per_step": bo, "ms_per_step": round(ms, 3), "steps": n,
            "pipelined": "2 buffer sets; uploads, compute and downloads of neighbouring steps overlap"}


# ----------------------------------------------------------------------------------------
# CPU baseline / reference arm: the FP64 oracle, as it stands, on a bounded pixel sample
# ----------------------------------------------------------------------------------------
def _cpu_pixels(workload, budget_s, seed=0, pixel_seed=0):
    """Oracle forward + loss + backward on random pixels of the workload until budget_s
    has passed (projection included); returns (pixels done, seconds)."""
    import gs_scenes as S
    import oracle
    sc, cams, K, tile, fdt = S.make_config(workload, seed)
    cam = cams[0]
    Fgt, Cgt, Dgt = S.voronoi_targets(seed + 100, [cam], sc.d)
    rng = np.random.default_rng(pixel_seed)
    t_start = time.perf_counter()
    proj = oracle.project(sc, cam)
    done = 0
    batch = 8
    while time.perf_counter() - t_start < budget_s:
        pix = rng.choice(cam.n_pix, batch, replace=False)
        r = oracle.render(sc, cam, K, pixels=pix, proj=proj)
        # the loss and its gradient at those pixels (their share of the frame's mean), then
        # the oracle adjoint
        _, dF, dC, dD = oracle.loss_cos_l1(r["F"], Fgt[pix], r["C"], Cgt[pix], r["D"], Dgt[pix],
                                           n_total=cam.n_pix)
        oracle.backward(sc, cam, K, dF, dC, dD, pixels=pix, proj=proj)
        done += batch
    return done, time.perf_counter() - t_start


def _cpu_worker(a):
    return _cpu_pixels(*a)


def _rel_l2(a, b):
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def bf16_form_parity(n_pix=64, seed=0):
    """Precision of the BF16-row form against the FP64 oracle on sampled pixels of the
    'frame_1m_bf16' workload (1M Gaussians, 640x480, D=512 bf16 rows, K=8): per-pixel
    cosine of F against the oracle fed the bf16 rows and against the oracle fed the
    original float32 rows, the largest element error of F, the relative L2 error of each
    gradient group (upstream gradients seeded at the sampled unflagged pixels only), and
    the pixels the oracle flags as near a threshold (excluded) or near a Top-K tie."""
    import torch
    import gs_scenes as S
    import oracle
    from paper_2602_06991_b300.renderer import TopKRenderer
    sc, cams, K, tile, fdt = S.make_config("frame_1m_bf16", seed)
    cam = cams[0]
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    feats = t(sc.feats).float().to(torch.bfloat16).contiguous()
    r = TopKRenderer(cams, K=K, D=sc.d, tile=tile, feat_dtype="bf16")
    ins = [t(sc.mean3d), t(sc.cov3d), t(sc.opacity), t(sc.rgb)]
    out = r.forward(*ins, feats)
    torch.cuda.synchronize()
    rng = np.random.default_rng(seed + 7)
    pix = np.sort(rng.choice(cam.n_pix, n_pix, replace=False))
    feats64 = feats.float().cpu().numpy().astype(np.float64)
    proj = oracle.project(sc, cam)
    o = oracle.render(sc, cam, K, pixels=pix, proj=proj, feats=feats64)
    o32 = oracle.render(sc, cam, K, pixels=pix, proj=proj, feats=sc.feats)
    fragile = (o["flags"] & oracle.F_SET_FRAGILE) != 0
    near_tie = (o["flags"] & oracle.F_NEAR_TIE) != 0
    ok = ~fragile
    gF = out["F"][torch.from_numpy(pix).to(dev)].float().cpu().numpy().astype(np.float64)

    def cos_min(a, b):
        nz = np.linalg.norm(b, axis=1) > 0
        c = (a[nz] * b[nz]).sum(1) / (np.linalg.norm(a[nz], axis=1) * np.linalg.norm(b[nz], axis=1) + 1e-300)
        return float(c.min()) if c.size else 1.0

    res = {"workload": "frame_1m_bf16: " + S.CONFIGS["frame_1m_bf16"], "pixels": int(n_pix),
           "flagged_near_threshold": int(fragile.sum()), "flagged_near_tie": int(near_tie.sum()),
           "F_cos_min_vs_bf16_rows": round(cos_min(gF[ok], o["F"][ok]), 7),
           "F_cos_min_vs_f32_rows": round(cos_min(gF[ok], o32["F"][ok]), 7),
           "F_max_abs_err_vs_bf16_rows": float(np.abs(gF[ok] - o["F"][ok]).max()) if ok.any() else 0.0}
    keep = (o["flags"] & (oracle.F_SET_FRAGILE | oracle.F_NEAR_TIE | oracle.F_NEAR_CLAMP)) == 0
    dF, dC, dD = S.upstream_grads(seed + 9, len(pix), sc.d)
    dF = np.where(keep[:, None], dF, 0.0).astype(np.float32)
    dC = np.where(keep[:, None], dC, 0.0).astype(np.float32)
    dD = np.where(keep, dD, 0.0).astype(np.float32)
    P = r.P
    dF_t = torch.zeros(P, sc.d, dtype=torch.bfloat16, device=dev)
    dC_t = torch.zeros(P, 3, device=dev)
    dD_t = torch.zeros(P, device=dev)
    sel = torch.from_numpy(pix).to(dev)
    dF_t[sel] = t(dF).to(torch.bfloat16)
    dC_t[sel] = t(dC)
    dD_t[sel] = t(dD)
    dF_exact = dF_t[sel].float().cpu().numpy().astype(np.float64)
    g = r.backward(dF_t, dC_t, dD_t)
    torch.cuda.synchronize()
    og = oracle.backward(sc, cam, K, dF_exact, dC.astype(np.float64), dD.astype(np.float64), pixels=pix,
                         proj=proj, feats=feats64)
    res["grad_rel_l2"] = {gk: round(_rel_l2(g[gk].cpu().numpy(), og[ok_]), 9) for gk, ok_ in
                          (("feat", "feat"), ("opacity", "opac"), ("rgb", "rgb"), ("mean3d", "mean3d"),
                           ("cov3d", "cov3d"))}
    res["bars"] = "cosine >= 0.999 against both; gradients relative L2 <= 1e-4 (the GPU tests assert these)"
    del r, out, g, feats, ins
    torch.cuda.empty_cache()
    return res


def cpu_baseline(workload, budget_s=15.0, seed=0, all_cores=True):
    """The oracle as it stands on the host cores: one process (the reported value), and,
    beside it, one process per core (capped at 16: each holds its own copy of the scene)
    on disjoint random pixel draws, started by spawn."""
    done, el = _cpu_pixels(workload, budget_s, seed, seed)
    cpu_model = "unknown"
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.startswith("model name"):
                    cpu_model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    out = {"value": round(done / el / 1e6, 9), "unit": UNIT, "cores": 1, "kind": "oracle", "cpu_model": cpu_model,
           "host_cores": os.cpu_count(),
           "sample": f"{done} random pixels of the '{workload}' workload, forward + loss + backward, "
                     f"FP64 single-threaded C, {el:.1f} s (projection included)"}
    if all_cores:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        n = max(1, min(os.cpu_count() or 1, 16))
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ.setdefault(v, "1")
        try:
            with ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn")) as ex:
                res = list(ex.map(_cpu_worker, [(workload, budget_s, seed, 1000 + i) for i in range(n)]))
            tot = sum(r[0] for r in res)
            wall = max(r[1] for r in res)
            out["all_cores"] = {"value": round(tot / wall / 1e6, 9), "unit": UNIT, "cores": n,
                                "host_cores": os.cpu_count(),
                                "sample": f"{n} processes x {budget_s:.0f} s, {tot} random pixels in all"}
        except Exception as e:      # the single-process figure stands on its own
            out["all_cores"] = {"unavailable": f"{type(e).__name__}: {e}"}
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return None
    cb = cpu_baseline(args.workload, budget_s=max(5.0, min(60.0, 3.0 * args.steps)), all_cores=False)
    import gs_scenes as S
    sc, cams, K, tile, _ = S.make_config(args.workload, 0)
    P = sum(c.width * c.height for c in cams)
    return {"metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(args.workload, world, sc.n, P, sc.d, K, tile),
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="frame")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-launch-count", action="store_true", help="skip the CUPTI launch count (for ncu runs)")
    ap.add_argument("--no-batched", action="store_true", help="skip the BF16 multi-keyframe measurement")
    ap.add_argument("--no-mapping", action="store_true", help="skip the mapping-iteration measurement")
    ap.add_argument("--views", default="", help="comma-separated view indices of the workload to render "
                    "(reduced cases for profiling captures; default: all)")
    ap.add_argument("--max-instances", type=int, default=0, help="instance capacity (0: the library default)")
    ap.add_argument("--no-depth-cut", action="store_true", help="sort every instance on every render")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            torch.cuda.set_device(local_rank)
            torch.distributed.init_process_group("nccl")
        res = run_ours(args, rank, world, local_rank)
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
