#!/usr/bin/env python
"""Benchmark of the splatting hot path on one GB300 (or N replicas).

One step = one mapping iteration (Eq. (2) of RT-GuIDE: render 4 keyframes of a
500,000-Gaussian room map at 640x480, L1 colour + 0.1 L1 depth loss, hand-written
adjoint, Adam update; captured once in a CUDA graph and replayed) followed by one
batched information-gain pass (Eq. (nbv):
256 candidate views, one third each at 80x60 / 160x120 / 320x240, over a
1,000,000-Gaussian room map).  Inputs are seeded synthetic scenes shaped like the
paper's onboard maps (the paper's iTHOR / MP3D scenes are not available).

Printed: ONE JSON line.  `value` is candidate views/s of the batched pass
(256 / device time of the pass); `fwd_bwd` carries mapping iterations/s of the
500k-Gaussian step.  Both are measured with CUDA events on the launching stream
over exactly --steps steps after --warmup untimed steps; an L2 flush (a 256 MB
write) separates every timed part and is not timed.  `e2e` repeats the loop
through the public API with the inputs copied each step from pinned host
memory and the results read back.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (candidates 0 and 1 per step, 80x60 and 160x120,
scaled to the 256-view resolution mix by pixel count).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "candidate views/sec (batched info-gain) and fwd+bwd iters/sec at 500k Gaussians"
WORKLOAD = ("ig: 1,000,000 room Gaussians, 256 candidates (80x60/160x120/320x240 thirds); "
            "map: 500,000 room Gaussians, 4 keyframes 640x480, fwd+bwd+Adam")
L2_FLUSH_BYTES = 256 << 20
IG_INSTR_PER_EVAL = 12.0    # FP32 lane-instructions per contributing evaluation of the U-only compositing

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one full-size k_ig_items launch,
# from one-pass ncu captures of
#   python bench.py --part ig --ig-tiles <tiles> --ig-batch <batch> --steps 1 --warmup 1 --no-e2e
#       --no-cpu-baseline --graph 0
# for the tile and chunk-depth choices the autotuner makes; each holds while the choices match and
# the sources that shape the kernel are unchanged (the tile lists themselves are fixed by the
# bit-exact binning).
IG_TRAFFIC_SHA1 = "23aba96b5c3e3fadfbdbb983f5c76f56bbb47afe"
IG_TRAFFIC = [
    {"tiles": {"80x60": "8x8", "160x120": "16x16", "320x240": "32x16"}, "batch": 8, "bytes": 5.1101e9 + 4.18e6},
    {"tiles": {"80x60": "8x8", "160x120": "16x8", "320x240": "32x16"}, "batch": 8, "bytes": 5.0264e9 + 4.10e6},
]
IG_TRAFFIC_HEADERS = ("render_common.cuh", "gs_common.cuh")


def ig_sources_sha1() -> str:
    """SHA-1 of what shapes k_ig_items: its source text in render.cu (with the chunk compositing
    it calls) and the two headers it uses."""
    import hashlib
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2409_18122_gb300", "csrc")
    with open(os.path.join(csrc, "render.cu")) as f:
        src = f.read()
    a = src.find("void composite_chunks(")
    a = src.rfind("\n", 0, a)
    b = src.find("\n}\n", src.find("k_ig_items(", a))
    h.update(src[a:b].encode() if a >= 0 and b > a else src.encode())
    for name in IG_TRAFFIC_HEADERS:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cfg4", action="store_true", help="skip the 3M-Gaussian exploration-map loop")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--graph", type=int, default=1, help="capture the information-gain pass in a CUDA graph")
    # options for profiling runs (defaults give the benchmark)
    ap.add_argument("--part", choices=["both", "ig", "map"], default="both", help="which part of the step to run")
    ap.add_argument("--ig-tiles", default="auto",
                    help="'auto' (autotuner) or fixed tiles per resolution, e.g. 80x60=8x8,160x120=16x16")
    ap.add_argument("--ig-views", type=int, default=0, help="score only the first N candidates (0: all 256)")
    ap.add_argument("--no-unbatched", action="store_true", help="skip the one-view-per-call comparison")
    ap.add_argument("--ig-batch", type=int, default=None,
                    help="chunk depth of the information-gain compositing (4, 8, 16; default: autotuned "
                         "with --ig-tiles auto, else 8)")
    ap.add_argument("--no-map-tune", action="store_true",
                    help="mapping step at the default tile and depth instead of the autotuner's")
    return ap.parse_args()


def parse_tiles(spec: str):
    """'80x60=8x8,160x120=16x16' -> {(80, 60): (8, 8), (160, 120): (16, 16)}; 'auto' -> None."""
    if spec == "auto":
        return None
    out = {}
    for item in spec.split(","):
        res, tile = item.split("=")
        w, h = (int(x) for x in res.split("x"))
        tw, th = (int(x) for x in tile.split("x"))
        out[(w, h)] = (tw, th)
    return out


# ----------------------------------------------------------------------------- helpers
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms while running."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """The largest x over all ranks (the job's time is its slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, seconds_per_rank: float, world: int) -> float:
    """Whole-job rate of N replicas: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / max_over_ranks(seconds_per_rank, world)


# ----------------------------------------------------------------------------- workloads
class MapStep:
    """One mapping iteration on the 500k-Gaussian, 4-keyframe map: render, the loss and its
    image gradient (gs_image_loss; by default mean L1 over RGB + 0.1 x mean L1 depth, or the
    paper's Eq. 3 weights with SSIM), gs_render_bwd, Adam (gs_adam_step).  With graph=True
    the whole iteration (forward, loss, backward, Adam) is captured once in a CUDA graph and
    replayed; eager() runs it op by op (used for the per-stage breakdown)."""

    def __init__(self, gs, scenes, weights=None, graph=True, scene=None, tune=True, render_params=None):
        import torch
        self.torch = torch
        self.gs = gs
        sc = scenes.config2() if scene is None else scene
        self.scene = sc
        gm = gs.GaussianMapTensors.from_numpy(sc.gmap)
        # keyframe tile and forward chunk depth picked by the autotuner (timed fwd + bwd passes)
        if render_params is not None:
            self.render_params, self.tune_timings = render_params, {}
        else:
            self.render_params, self.tune_timings = (gs.autotune_mapping(gm, sc.cams) if tune
                                                     else (gs.RenderParams(), {}))
        self.frame = gs.Frame(gm.n, sc.cams, self.render_params, with_pair_tiles=False)
        tgt = gs.GaussianMapTensors.from_numpy(scenes.perturbed(sc.gmap, seed=2002))
        while True:
            self.frame.reset_status()
            img = self.frame.forward(tgt)
            torch.cuda.synchronize()
            if not self.frame.grow_if_needed():
                break
        self.frame.check_status()
        self.tgt_rgb = img["rgb"].clone()
        self.tgt_depth = img["depth"].clone()
        self.params = [t.clone().requires_grad_(True) for t in (gm.mo, gm.su, gm.q, gm.rgb)]
        self.host = [t.detach().cpu().pin_memory() for t in self.params]
        self.host_tgt = [self.tgt_rgb.cpu().pin_memory(), self.tgt_depth.cpu().pin_memory()]
        self.opt = gs.Adam(self.params, lr=1e-4)   # gs_adam_step: one kernel, device step count
        self.loss_host = torch.zeros(1, dtype=torch.float32).pin_memory()
        self.loss_fn = gs.ImageLoss.for_cameras(sc.cams, gs.L1_WEIGHTS if weights is None else weights)
        self.graph = None
        self.kernels_per_replay = 0   # library kernels in one replay (0: eager, counted as launched)
        if graph:
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                for _ in range(3):
                    self.eager()
            torch.cuda.current_stream().wait_stream(side)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            k0 = gs.L.lib().gs_kernel_launches()
            with torch.cuda.graph(g):
                self.graph_loss = self.eager()
            self.kernels_per_replay = int(gs.L.lib().gs_kernel_launches() - k0)
            torch.cuda.synchronize()
            self.graph = g

    def eager(self):
        gs, torch = self.gs, self.torch
        self.opt.zero_grad(set_to_none=True)
        rgb, depth, _ = gs.render(*self.params, self.frame)
        loss, d_rgb, d_depth = self.loss_fn(rgb.detach(), depth.detach(), self.tgt_rgb, self.tgt_depth)
        torch.autograd.backward((rgb, depth), (d_rgb, d_depth))
        self.opt.step()
        return loss[:1]

    def __call__(self):
        if self.graph is not None:
            self.graph.replay()
            return self.graph_loss
        return self.eager()

    def upload(self):
        """This step's inputs from pinned host memory (on the current stream)."""
        with self.torch.no_grad():
            for d, h in zip(self.params, self.host):
                d.copy_(h, non_blocking=True)
            self.tgt_rgb.copy_(self.host_tgt[0], non_blocking=True)
            self.tgt_depth.copy_(self.host_tgt[1], non_blocking=True)

    def e2e(self):
        """Host inputs -> device, step, loss -> host (all enqueued on the current stream)."""
        self.upload()
        loss = self()
        self.loss_host.copy_(loss.detach().reshape(1), non_blocking=True)

    def h2d_bytes(self):
        return sum(h.numel() * h.element_size() for h in self.host + self.host_tgt)


class IGStep:
    """The batched information-gain pass over 256 candidate views of a 1M-Gaussian map.

    project -> bin_sort -> composite (the three stages of gs_info_gain_batch) on
    colour-free records, captured in one CUDA graph; the tile size of each
    resolution class is picked by the autotuner at set-up.  Events recorded inside
    the graph bracket the compositing kernel (the step's dominant kernel).
    """

    def __init__(self, gs, scenes, graph: bool, tiles=None, n_views: int = 0, scene=None, cams=None,
                 record_capacity=None, pair_capacity: int = 300_000_000, batch=None):
        import torch
        self.torch = torch
        self.gs = gs
        sc = scenes.config3() if scene is None else scene
        self.scene = sc
        self.gm = gs.GaussianMapTensors.from_numpy(sc.gmap)
        cams = sc.cams if cams is None else cams
        cams = cams[:n_views] if n_views > 0 else cams
        if tiles is None:
            self.tile_choice, self.tile_timings = gs.autotune_tiles(self.gm, cams, pair_capacity=400_000_000)
            torch.cuda.empty_cache()
        else:
            self.tile_choice = dict(tiles)
        cams = gs.with_tiles(cams, self.tile_choice)
        self.cams = cams
        # chunk depth of the compositing: autotuned with the tiles, or given
        if batch is None and tiles is None:
            batch, self.batch_timings = gs.autotune_ig_batch(self.gm, cams, pair_capacity=400_000_000)
        else:
            self.batch_timings = {}
        self.params = gs.RenderParams(ig_batch=int(batch or 0))
        self.frame = gs.Frame(self.gm.n, cams, self.params, pair_capacity=pair_capacity, with_color=False,
                              with_pair_tiles=False, record_capacity=record_capacity, with_gid=False,
                              with_view=False, with_item_order=False)
        while True:
            self.frame.reset_status()
            self.frame.project(self.gm)
            self.frame.bin_sort()
            torch.cuda.synchronize()
            if not self.frame.grow_if_needed():
                break
        self.frame.check_status()
        self.out = torch.zeros(len(cams), dtype=torch.float32, device="cuda")
        self.frame.info_gain(self.out)
        torch.cuda.synchronize()
        self.host = [t.cpu().pin_memory() for t in (self.gm.mo, self.gm.su, self.gm.q, self.gm.rgb)]
        self.host_cams = self.frame.cams_dev.cpu().pin_memory()
        self.out_host = torch.zeros(len(cams), dtype=torch.float32).pin_memory()
        # a second device copy of the map: the end-to-end loop uploads the next step's map into
        # one buffer while the current step runs from the other
        self.gms = [self.gm, gs.GaussianMapTensors(*(t.clone() for t in (self.gm.mo, self.gm.su, self.gm.q,
                                                                          self.gm.rgb)))]
        self.graph = None
        self.graphs = []
        self.kernels_per_replay = 0
        try:
            self.ev = (torch.cuda.Event(enable_timing=True, external=True),
                       torch.cuda.Event(enable_timing=True, external=True))
            # recorded after each buffer's projection, the last stage that reads the map
            self.ev_proj = [torch.cuda.Event(external=True), torch.cuda.Event(external=True)]
        except TypeError:
            self.ev = None
        if graph and self.ev is not None:
            for b in (0, 1):
                s = torch.cuda.Stream()
                s.wait_stream(torch.cuda.current_stream())
                with torch.cuda.stream(s):
                    self._run(b)
                torch.cuda.current_stream().wait_stream(s)
                torch.cuda.synchronize()
                g = torch.cuda.CUDAGraph()
                k0 = gs.L.lib().gs_kernel_launches()
                with torch.cuda.graph(g):
                    self._run(b)
                self.kernels_per_replay = int(gs.L.lib().gs_kernel_launches() - k0)
                self.graphs.append(g)
            self.graph = self.graphs[0]
        if self.ev is None:
            self.ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            self.ev_proj = [torch.cuda.Event(), torch.cuda.Event()]

    def _run(self, b=0):
        self.frame.project(self.gms[b])
        self.ev_proj[b].record()
        self.frame.bin_sort()
        self.ev[0].record()
        self.frame.info_gain(self.out)
        self.ev[1].record()

    @property
    def n_views(self):
        return len(self.cams)

    def __call__(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self._run()
        return self.out

    def composite_ms(self, reps: int, flush):
        """Device time of the compositing stage, from the events around it (mean of `reps` passes)."""
        t = []
        for _ in range(reps):
            flush()
            self()
            self.torch.cuda.synchronize()
            t.append(self.ev[0].elapsed_time(self.ev[1]))
        return statistics.mean(t)

    def contributing(self):
        """Contributing (pixel, Gaussian) evaluations of one pass, counted with the forward kernel."""
        torch, gs = self.torch, self.gs
        fr = gs.Frame(self.gm.n, self.cams, pair_capacity=self.frame.pair_capacity)
        img = fr.new_images(with_rgb=False, with_depth=False, with_unc=False, with_counts=True)
        fr.forward(self.gm, img)
        torch.cuda.synchronize()
        c = int(img["n_contrib"].to(torch.int64).sum().item())
        e = int(img["last"].to(torch.int64).sum().item())
        del fr, img
        torch.cuda.empty_cache()
        return c, e

    def upload_map(self, b):
        """This step's map from pinned host memory into buffer b (on the current stream)."""
        with self.torch.no_grad():
            g = self.gms[b]
            for d, h in zip((g.mo, g.su, g.q, g.rgb), self.host):
                d.copy_(h, non_blocking=True)

    def run_buffer(self, b):
        """One pass projecting the map in buffer b, its cameras uploaded first (current stream)."""
        with self.torch.no_grad():
            self.frame.cams_dev.copy_(self.host_cams, non_blocking=True)
        if self.graphs:
            self.graphs[b].replay()
        else:
            self._run(b)
        return self.out

    def e2e(self):
        self.upload_map(0)
        self.run_buffer(0)
        self.out_host.copy_(self.out, non_blocking=True)

    def h2d_bytes(self):
        return sum(h.numel() * h.element_size() for h in self.host) + self.host_cams.numel()


class Unbatched:
    """The same candidates scored one view at a time (gs_info_gain_batch with one camera per call)."""

    def __init__(self, gs, istep):
        import torch
        self.torch = torch
        self.istep = istep
        self.cams_all = istep.frame.cams_dev.view(len(istep.cams), -1)   # the batch's 80-byte camera records
        self.per_class = {}
        for v, c in enumerate(istep.cams):
            key = (c.width, c.height, c.tile_w, c.tile_h)
            if key not in self.per_class:
                self.per_class[key] = gs.InfoGain(istep.gm.n, [c], pair_capacity=1 << 24)
        self.keys = [(c.width, c.height, c.tile_w, c.tile_h) for c in istep.cams]
        self.out = torch.zeros(len(istep.cams), dtype=torch.float32, device="cuda")
        self()
        torch.cuda.synchronize()
        for ig in self.per_class.values():
            while ig.grow_if_needed():
                self()
                torch.cuda.synchronize()

    def __call__(self):
        for v, key in enumerate(self.keys):
            ig = self.per_class[key]
            ig.cams_dev.view(1, -1).copy_(self.cams_all[v:v + 1], non_blocking=True)
            ig(self.istep.gm, out=self.out[v:v + 1])
        return self.out


# ----------------------------------------------------------------------------- end-to-end loops
def pipelined_e2e_ms(torch, steps, upload, run, readback, last_reader, flush):
    """Device time of `steps` end-to-end steps, each uploading its inputs from pinned host
    memory into one of two input buffers (b = step mod 2), running from that buffer and
    reading its result back to the host.  The uploads go on a copy stream: step k+1's upload
    starts as soon as the last reader of its buffer (in step k-1) is done, so it overlaps
    step k.  upload(b) / run(b) / readback(b) enqueue on the current stream; last_reader(b)
    is an event recorded by run(b) after the last read of buffer b.  The L2 flush before
    every step is not counted."""
    main = torch.cuda.current_stream()
    cs = torch.cuda.Stream()
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fl = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    start.record(main)
    cs.wait_stream(main)
    with torch.cuda.stream(cs):
        upload(0)
        copied[0].record(cs)
    for k in range(steps):
        b = k & 1
        if k + 1 < steps:
            nb = b ^ 1
            with torch.cuda.stream(cs):
                if k >= 1:
                    cs.wait_event(last_reader(nb))
                upload(nb)
                copied[nb].record(cs)
        fl[k][0].record(main)
        flush()
        fl[k][1].record(main)
        main.wait_event(copied[b])
        run(b)
        readback(b)
    end.record(main)
    torch.cuda.synchronize()
    return start.elapsed_time(end) - sum(a.elapsed_time(c) for a, c in fl)


def map_e2e_ms(torch, pair, steps, flush):
    """pipelined_e2e_ms for the mapping step: two MapSteps (their own parameters, targets,
    frame and graph) take the steps in turn."""
    done = [torch.cuda.Event(), torch.cuda.Event()]

    def run(b):
        pair[b].last_loss = pair[b]()
        done[b].record()

    def readback(b):
        pair[b].loss_host.copy_(pair[b].last_loss.detach().reshape(1), non_blocking=True)

    return pipelined_e2e_ms(torch, steps, lambda b: pair[b].upload(), run, readback, lambda b: done[b], flush)


def ig_e2e_ms(torch, istep, steps, flush):
    """pipelined_e2e_ms for the information-gain pass: the two map buffers of one IGStep."""
    return pipelined_e2e_ms(torch, steps, istep.upload_map, istep.run_buffer,
                            lambda b: istep.out_host.copy_(istep.out, non_blocking=True),
                            lambda b: istep.ev_proj[b], flush)


# ----------------------------------------------------------------------------- timing loops
def timed_loop(torch, steps, parts, flush):
    """Per part: list of per-step device milliseconds (events on the current stream)."""
    ev = {name: [] for name, _ in parts}
    st = torch.cuda.current_stream()
    for _ in range(steps):
        for name, fn in parts:
            flush()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            ev[name].append((e0, e1))
    torch.cuda.synchronize()
    return {name: [a.elapsed_time(b) for a, b in lst] for name, lst in ev.items()}


def work_stats(torch, gs, mstep):
    """Pairs, records and evaluated / contributing (pixel, Gaussian) counts of one mapping forward."""
    fr = mstep.frame
    gm = gs.GaussianMapTensors(*(p.detach() for p in mstep.params))
    img = fr.new_images(with_counts=True)
    fr.forward(gm, img)
    torch.cuda.synchronize()
    return dict(pairs=int(fr.pair_count.item()) & 0xFFFFFFFF, records=int(fr.rec_count.item()),
                evaluated=int(img["last"].to(torch.int64).sum().item()),
                contributing=int(img["n_contrib"].to(torch.int64).sum().item()),
                pixels=fr.n_pixels, tiles=fr.n_tiles)


def pipeline_roofline(istep, contributing, t_pass, hbm_gbs, issue_tps):
    """Roofline of the whole information-gain pass: per stage the larger of algorithmic
    bytes / HBM bandwidth and algorithmic FP32 instructions / issue peak, summed, over
    the measured pass time.  Units: (Gaussian, view) pairs and visible records for the
    projection (~25 instructions per culled pair, ~110 per visible one; 64 B read per
    Gaussian, 48 B written per scoring record), (tile, record) pairs for binning (44 B
    per pair: emit, one permutation, ranges), contributing (pixel, Gaussian) evaluations
    for compositing (~12 instructions each)."""
    fr = istep.frame
    n, v = istep.gm.n, istep.n_views
    recs = int(fr.rec_count.item())
    pairs = int(fr.pair_count.item()) & 0xFFFFFFFF
    st = {
        "project": (64.0 * n + 48.0 * recs, 25.0 * n * v + 110.0 * recs),
        "bin_sort": (44.0 * pairs, 0.0),
        "composite": (0.0, 12.0 * contributing),
    }
    out = {}
    total = 0.0
    for k, (b, ins) in st.items():
        t = max(b / (hbm_gbs * 1e9), ins / (issue_tps * 1e12))
        out[k + "_roof_ms"] = t * 1e3
        total += t
    out.update(records=recs, pairs=pairs, pair_views=n * v, contributing=contributing,
               roof_ms=total * 1e3, measured_ms=t_pass * 1e3, frac=total / t_pass)
    return out


def compositing_rate(contributing, launch_s):
    """Achieved rate of the information-gain compositing kernel in T lane-instructions/s:
    IG_INSTR_PER_EVAL per contributing (pixel, Gaussian) evaluation over one launch's duration."""
    return IG_INSTR_PER_EVAL * contributing / launch_s / 1e12


def at_load_clock(rooflines, sms, load_mhz):
    """Adds to each FP32-issue roofline the issue peak at the median SM clock sampled under
    load (SMs x 128 lanes x MHz) and the fraction of it achieved; no-op without a sample."""
    if not load_mhz:
        return rooflines
    for r in rooflines:
        if r.get("bound") == "alu":
            r["peak_at_load_clock"] = sms * 128 * float(load_mhz) * 1e6 / 1e12
            r["frac_at_load_clock"] = r["achieved"] / r["peak_at_load_clock"]
    return rooflines


def stage_roofline(pipe, stage_ms, hbm_gbs, issue_tps):
    """Per stage of the information-gain pass: achieved algorithmic rate over the stage's
    eager event-timed duration, against the roofline that bounds it (units as in
    pipeline_roofline: the projection and compositing by FP32 issue, the binning by HBM)."""
    n_pairs, recs, contrib = pipe["pairs"], pipe["records"], pipe["contributing"]
    n_pv = pipe["pair_views"]
    rows = {
        "gs_project": ("alu", 25.0 * n_pv + 110.0 * recs, issue_tps * 1e12, "T lane-instr/s"),
        "gs_bin_sort": ("hbm", 44.0 * n_pairs, hbm_gbs * 1e9, "GB/s"),
        "gs_info_gain_composite": ("alu", 12.0 * contrib, issue_tps * 1e12, "T lane-instr/s"),
    }
    out = {}
    for k, (bound, work, peak, unit) in rows.items():
        ms = stage_ms.get(k)
        if not ms:
            continue
        rate = work / (ms / 1e3)
        scale = 1e12 if bound == "alu" else 1e9
        out[k] = {"bound": bound, "ms": ms, "achieved": rate / scale, "peak": peak / scale, "unit": unit,
                  "frac": rate / peak}
    return out


def map_stage_roofline(ws, n, n_views, stage_ms, hbm_gbs, issue_tps):
    """Per stage of the mapping step: projection (25 instructions per (Gaussian, view), 110 per
    visible record), binning (44 B per pair), forward compositing (10 instructions per
    evaluated, 6 more per contributing (pixel, Gaussian)), backward (10 per evaluated, 38 per
    contributing, plus the projection adjoint), loss (mean L1: 12 B per pixel and channel of
    colour and depth: two reads, one gradient write), Adam (28 B per parameter)."""
    rows = {
        "gs_project": ("alu", 25.0 * n * n_views + 110.0 * ws["records"]),
        "gs_bin_sort": ("hbm", 44.0 * ws["pairs"]),
        "gs_render_fwd": ("alu", 10.0 * ws["evaluated"] + 6.0 * ws["contributing"]),
        "gs_render_bwd": ("alu", 10.0 * ws["evaluated"] + 38.0 * ws["contributing"]),
        "gs_image_loss": ("hbm", 12.0 * 4 * ws["pixels"]),
        "gs_adam_step": ("hbm", 28.0 * 16 * n),   # p, g, m, v read, p, m, v written; 16 floats per Gaussian
    }
    out = {}
    for k, (bound, work) in rows.items():
        ms = stage_ms.get(k)
        if not ms:
            continue
        rate = work / (ms / 1e3)
        peak, scale, unit = (issue_tps * 1e12, 1e12, "T lane-instr/s") if bound == "alu" else (hbm_gbs * 1e9, 1e9, "GB/s")
        out[k] = {"bound": bound, "ms": ms, "achieved": rate / scale, "peak": peak / scale, "unit": unit,
                  "frac": rate / peak}
    return out


def cfg0_latency_us(torch, gs, scenes, reps=30, scene=None):
    """Device time of one forward render of config 0 (project, bin, composite), launched
    call by call and replayed from a CUDA graph (median microseconds); `scene` renders
    another single-view config the same way."""
    sc = scenes.config0() if scene is None else scene
    gm = gs.GaussianMapTensors.from_numpy(sc.gmap)
    fr = gs.Frame(gm.n, sc.cams)
    img = fr.new_images()
    while True:
        fr.reset_status()
        fr.forward(gm, img)
        torch.cuda.synchronize()
        if not fr.grow_if_needed():
            break
        img = fr.new_images()
    fr.check_status()
    for _ in range(3):
        fr.forward(gm, img)
    torch.cuda.synchronize()

    def median_us(fn):
        t = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            t.append(e0.elapsed_time(e1) * 1e3)
        return statistics.median(t)

    eager = median_us(lambda: fr.forward(gm, img))
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fr.forward(gm, img)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fr.forward(gm, img)
    g.replay()
    torch.cuda.synchronize()
    out = {"eager": eager, "graph": median_us(g.replay), "unit": "us"}
    # the same render in one launch (gs_render_small), when the map is small enough for it
    if gm.n <= gs.L.GS_SMALL_MAX_GAUSSIANS:
        simg = {k: torch.empty_like(v) for k, v in img.items() if v is not None}
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        gs.render_small(gm, sc.cams, images=simg, status=st)
        torch.cuda.synchronize()
        ok = int(st.item()) & gs.L.GS_FLAG_ERROR_MASK == 0
        same = ok and all(torch.equal(simg[k], img[k]) for k in simg)
        out["one_launch"] = {"eager": median_us(lambda: gs.render_small(gm, sc.cams, images=simg, status=st)),
                             "identical_to_tiled": bool(same), "unit": "us"}
        cams_dev = gs.cameras_to_device(sc.cams)
        with torch.cuda.stream(side):
            gs.render_small(gm, cams_dev, images=simg, status=st)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g2 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g2):
            gs.render_small(gm, cams_dev, images=simg, status=st)
        g2.replay()
        torch.cuda.synchronize()
        out["one_launch"]["graph"] = median_us(g2.replay)
    return out


def render_free_xi(torch, gs, istep, flush, reps=10):
    """The paper's render-free scoring (Eq. view_util) of the same candidates over the
    same map: thresholds + batched xi, device time per pass."""
    vu = gs.ViewUtility(istep.scene.cams)
    for _ in range(3):
        vu.thresholds(istep.gm)
        vu(istep.gm, gs.L.GS_XI)
    torch.cuda.synchronize()
    t = []
    for _ in range(reps):
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        vu.thresholds(istep.gm)
        vu(istep.gm, gs.L.GS_XI)
        e1.record()
        torch.cuda.synchronize()
        t.append(e0.elapsed_time(e1))
    ms = statistics.mean(t)
    return {"value": vu.V / (ms / 1e3), "unit": "views/s", "ms": ms, "views": vu.V,
            "paper_context": "0.013 s per planning step for RTGuIDE's render-free score on an RTX A4000 "
                             "(number of candidate views per step not stated)"}


def eq3_map_step(torch, gs, scenes, flush, steps=10):
    """The mapping step with the paper's full loss (Eq. 3: depth L1 + 0.4 colour L1 + 0.1 (1 - SSIM))
    on the same 500k-Gaussian, 4 x 640x480 workload; iterations/s and the loss kernels' share."""
    m = MapStep(gs, scenes, weights=gs.EQ3_WEIGHTS)
    for _ in range(3):
        m()
    torch.cuda.synchronize()
    t = timed_loop(torch, steps, [("m", m)], flush)["m"]
    gs.TIMER = gs.StageTimer()
    timed_loop(torch, 3, [("m", m.eager)], flush)
    loss_ms = statistics.mean(gs.TIMER.durations_ms("gs_image_loss"))
    gs.TIMER = None
    ms = statistics.mean(t)
    out = {"value": 1e3 / ms, "unit": "iters/s", "ms": ms, "gs_image_loss_ms": loss_ms,
           "loss": float(m.loss_fn.loss[0].item()), "ssim": float(m.loss_fn.loss[3].item())}
    del m
    torch.cuda.empty_cache()
    return out


def config4_loop(torch, gs, scenes, tiles, flush, steps=5, batch=None):
    """The large exploration map (3M Gaussians, 40x40 m): one mapping iteration over 8
    keyframes at 1280x720 (loss as in the 500k step) and one information-gain pass over
    1,024 candidates (160x120 / 320x240 halves, the tiles the autotuner picked for those
    classes), captured together in one CUDA graph and replayed; events inside the graph
    split the two parts."""
    sc, cands = scenes.config4()
    m = MapStep(gs, scenes, graph=False, scene=sc)
    ig = IGStep(gs, scenes, graph=False, tiles=tiles, scene=sc, cams=cands, record_capacity=400_000_000,
                pair_capacity=1_500_000_000, batch=batch)
    try:
        ev = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(3)]
    except TypeError:
        return {"unavailable": "events inside a captured graph need torch.cuda.Event(external=True)"}
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):
            m.eager()
            ig._run()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ev[0].record()
        m.eager()
        ev[1].record()
        ig._run()
        ev[2].record()
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    t_map, t_ig = [], []
    for _ in range(steps):
        flush()
        g.replay()
        torch.cuda.synchronize()
        t_map.append(ev[0].elapsed_time(ev[1]))
        t_ig.append(ev[1].elapsed_time(ev[2]))
    ms_map, ms_ig = statistics.mean(t_map), statistics.mean(t_ig)
    fr = ig.frame
    out = {"gaussians": sc.gmap.n, "keyframes": len(sc.cams), "keyframe_px": "1280x720",
           "candidates": len(cands), "steps": steps, "ms_per_step": ms_map + ms_ig,
           "fwd_bwd": {"value": 1e3 / ms_map, "unit": "iters/s", "ms": ms_map},
           "ig": {"value": len(cands) / (ms_ig / 1e3), "unit": "views/s", "ms": ms_ig},
           "ig_records": int(fr.rec_count.item()), "ig_pairs": int(fr.pair_count.item()) & 0xFFFFFFFF,
           "map_pairs": int(m.frame.pair_count.item()) & 0xFFFFFFFF,
           "ig_tiles": {"%dx%d" % k: "%dx%d" % v for k, v in ig.tile_choice.items()},
           "ig_batch": ig.params.ig_batch, "map_tile": "%dx%d" % (m.render_params.tile_w, m.render_params.tile_h),
           "map_fwd_batch": m.render_params.fwd_batch}
    del g, m, ig, fr
    torch.cuda.empty_cache()
    return out


COLLISION_POINTS = 129    # test points of one planning call (Fig. planning_time, Sec. V-B)


def collision_timing(torch, gs, scenes, reps=20):
    """Collision check of 129 test points (one motion-primitive tree layer) against every
    Gaussian of the 3M-Gaussian, 40x40 m map, r_robot 0.3 m, lambda_g 3 (Sec. IV-B)."""
    import numpy as np
    sc, _ = scenes.config4()
    gm = gs.GaussianMapTensors.from_numpy(sc.gmap)
    rng = np.random.default_rng(129)
    pts = np.zeros((COLLISION_POINTS, 4), np.float32)
    pts[:, :3] = rng.uniform([0.5, 0.5, 0.3], [39.5, 39.5, 1.0], (COLLISION_POINTS, 3))
    p = torch.from_numpy(pts).cuda()
    for _ in range(3):
        gs.collision_check(gm, p, 0.3, gs.LAMBDA_G)
    torch.cuda.synchronize()
    t = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        gs.collision_check(gm, p, 0.3, gs.LAMBDA_G)
        e1.record()
        torch.cuda.synchronize()
        t.append(e0.elapsed_time(e1))
    ms = statistics.median(t)
    del gm
    torch.cuda.empty_cache()
    return {"ms": ms, "points": COLLISION_POINTS, "gaussians": sc.gmap.n,
            "pair_tests_per_s": COLLISION_POINTS * sc.gmap.n / (ms / 1e3),
            "paper_context": "0.62 s for planning a 5 m trajectory with 129 collision points at 3e6 "
                             "Gaussians (GPU collision checks, tree search included, hardware not stated)"}


def mix_pixels_per_view(cams):
    return sum(c.width * c.height for c in cams) / len(cams)


def oracle_sample(sc3):
    """IG of candidates 0 (80x60) and 1 (160x120) by the oracle; returns (seconds, pixels)."""
    from oracle import oracle as O
    cams = [sc3.cams[0], sc3.cams[1]]
    t0 = time.perf_counter()
    O.info_gain(sc3.gmap, cams)
    return time.perf_counter() - t0, sum(c.width * c.height for c in cams)


def cpu_baseline(sc3):
    """The FP64 oracle, as it stands, on the host cores (bounded sample, scaled per pixel)."""
    from oracle import oracle as O
    import time
    from paper_2409_18122_gb300 import scenes
    t, px = oracle_sample(sc3)
    value = px / t / mix_pixels_per_view(sc3.cams)
    sc0 = scenes.config0()
    t0 = time.perf_counter()
    O.render_images(sc0.gmap, sc0.cams)
    t_cfg0 = time.perf_counter() - t0
    return {"value": value, "unit": "views/s", "cores": O.num_threads(), "kind": "oracle",
            "cfg0_full_render_s": t_cfg0,
            "sample": "FP64 brute-force information gain of candidates 0 (80x60) and 1 (160x120) over the full "
                      "1M-Gaussian map (%.1f s for %d pixels), scaled to the 256-view mix by pixel count "
                      "(%.0f pixels per view)" % (t, px, mix_pixels_per_view(sc3.cams))}


# ----------------------------------------------------------------------------- arms
def run_ours(args):
    import torch
    from paper_2409_18122_gb300 import build as B
    B.build()
    from paper_2409_18122_gb300 import gs, scenes

    rank, world, local = dist_setup()
    torch.backends.cuda.matmul.allow_tf32 = False
    mstep = MapStep(gs, scenes, tune=not args.no_map_tune) if args.part in ("both", "map") else None
    istep = (IGStep(gs, scenes, graph=bool(args.graph), tiles=parse_tiles(args.ig_tiles), n_views=args.ig_views,
                    batch=args.ig_batch) if args.part in ("both", "ig") else None)
    flush_buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    flush = lambda: flush_buf.fill_(1.0)
    parts = [(n, f) for n, f in (("map", mstep), ("ig", istep)) if f is not None]

    for _ in range(args.warmup):
        for _, fn in parts:
            fn()
    torch.cuda.synchronize()

    barrier(world)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    k0 = gs.L.lib().gs_kernel_launches()
    # an NVTX range around the timed steps: a profiler can keep exactly their kernels
    # (ncu --nvtx --nvtx-include "timed_steps/")
    torch.cuda.nvtx.range_push("timed_steps")
    times = timed_loop(torch, args.steps, parts, flush)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    launches = (int(gs.L.lib().gs_kernel_launches() - k0) + (args.steps * istep.kernels_per_replay if istep else 0)
                + (args.steps * mstep.kernels_per_replay if mstep else 0))
    barrier(world)
    clocks = sampler.stop()
    # per-stage breakdown (entry points of the C ABI) from eager iterations outside the
    # timed region (the timed iterations replay CUDA graphs)
    def stages(fn):
        gs.TIMER = gs.StageTimer()
        timed_loop(torch, max(3, min(args.steps, 10)), [("part", fn)], flush)
        out = {k: statistics.mean(gs.TIMER.durations_ms(k)) for k in list(gs.TIMER.events)}
        gs.TIMER = None
        return out

    map_stage_ms = stages(mstep.eager) if mstep is not None else {}
    ig_stage_ms = stages(istep._run) if istep is not None else {}
    stage_ms = map_stage_ms if mstep is not None else ig_stage_ms

    t_map = sum(times.get("map", [0.0])) / 1e3
    t_ig = sum(times.get("ig", [0.0])) / 1e3
    t_map_all = max_over_ranks(t_map, world)
    t_ig_all = max_over_ranks(t_ig, world)
    value = job_throughput(istep.n_views * args.steps, t_ig, world) if istep else None
    fwd_bwd = job_throughput(args.steps, t_map, world) if mstep else None
    ms_per_step = (max_over_ranks(t_map + t_ig, world) / args.steps) * 1e3

    e2e = None
    if not args.no_e2e and mstep is not None and istep is not None:
        # end to end through the same public calls: every step uploads its inputs from pinned
        # host memory and reads its result back; uploads overlap the previous step (two input
        # buffers, a copy stream)
        mstep_b = MapStep(gs, scenes, render_params=mstep.render_params)
        pair = (mstep, mstep_b)
        ig_e2e_ms(torch, istep, 2, flush)
        map_e2e_ms(torch, pair, 2, flush)
        e_ig = max_over_ranks(ig_e2e_ms(torch, istep, args.steps, flush) / 1e3, world)
        e_map = max_over_ranks(map_e2e_ms(torch, pair, args.steps, flush) / 1e3, world)
        del mstep_b, pair
        e2e = {"value": istep.n_views * args.steps * world / e_ig, "unit": "views/s",
               "fwd_bwd_iters_per_s": args.steps * world / e_map,
               "h2d_bytes_per_step": mstep.h2d_bytes() + istep.h2d_bytes(),
               "d2h_bytes_per_step": 4 + 4 * istep.n_views,
               "pipelined": "each step's uploads overlap the previous step (double-buffered inputs, copy stream)"}

    if istep is None or mstep is None:
        # a profiling run of one part: a short line, no roofline bookkeeping
        if rank == 0:
            print(json.dumps({"part": args.part, "steps": args.steps, "ms_per_step": ms_per_step,
                              "value": value, "fwd_bwd": fwd_bwd, "stages_ms": stage_ms, "clocks": clocks,
                              "ig_tiles": ({"%dx%d" % k: "%dx%d" % v for k, v in istep.tile_choice.items()}
                                           if istep else None),
                              "ig_batch": istep.params.ig_batch if istep else None,
                              "ig_batch_ms": ({str(k): v for k, v in istep.batch_timings.items()} if istep else None),
                              "map_params": ({"tile": "%dx%d" % (mstep.render_params.tile_w,
                                                                         mstep.render_params.tile_h),
                                              "fwd_batch": mstep.render_params.fwd_batch,
                                              "timings_ms": {"%dx%d/%d" % k: v for k, v in mstep.tune_timings.items()}}
                                             if mstep else None)}))
        return

    ws = work_stats(torch, gs, mstep)
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = sms * 128 * sm_max * 1e6 / 1e12
    peak_src = "derived: %d SMs x 128 FP32 lanes x %.0f MHz (max SM clock); no FP32 peak is measured" % (sms, sm_max)
    # dominant kernel of the step: the information-gain compositing (gs_info_gain_composite);
    # algorithmic work = 12 FP32 lane-instructions per contributing (pixel, Gaussian) evaluation
    # of the U-only compositing (the unit count of the scope's measurement plan): the pixel
    # offset (2 sub), the quadratic form with the opacity in the exponent (3 fma/mul), ex2,
    # the clamp, the skip test, w = alpha T, T - w, the stop test and the U accumulation;
    # contributing evaluations are counted by the forward kernel at the same tiles (its
    # per-pixel count equals the oracle's in the GPU parity tests)
    t_comp = istep.composite_ms(max(3, args.steps), flush) / 1e3
    ig_contrib, ig_walked = istep.contributing()
    hbm = float(peaks.get("hbm_gbs", 6673.5))
    pipe = pipeline_roofline(istep, ig_contrib, t_ig_all / args.steps, hbm, peak)
    lat0 = cfg0_latency_us(torch, gs, scenes)
    lat1 = cfg0_latency_us(torch, gs, scenes, reps=20, scene=scenes.config1())
    xi_free = render_free_xi(torch, gs, istep, flush)
    collide = collision_timing(torch, gs, scenes)
    eq3 = eq3_map_step(torch, gs, scenes, flush)
    cfg4 = None if args.no_cfg4 else config4_loop(torch, gs, scenes, istep.tile_choice, flush,
                                                  batch=istep.params.ig_batch)
    achieved = compositing_rate(ig_contrib, t_comp)
    tiles_now = {"%dx%d" % k: "%dx%d" % v for k, v in istep.tile_choice.items()}
    traffic_src = None
    if IG_TRAFFIC_SHA1 == ig_sources_sha1():
        traffic_src = next((t for t in IG_TRAFFIC if t["tiles"] == tiles_now
                            and t["batch"] == (istep.params.ig_batch or 8)), None)
    traffic = traffic_src["bytes"] if traffic_src else None
    roofline = {"bound": "alu", "kernel": "k_ig_items (gs_info_gain_composite)", "achieved": achieved,
                "peak": peak, "unit": "T lane-instr/s", "frac": achieved / peak, "traffic": traffic,
                "peak_source": peak_src, "launch_ms": t_comp * 1e3, "contributing_evals": ig_contrib,
                "instr_per_eval": IG_INSTR_PER_EVAL, "list_entries_to_last_contributor": ig_walked,
                "traffic_note": "dram read + write bytes per launch from a one-pass ncu capture at full size with "
                                "the same tiles; null when no capture matches the tiles or the kernel sources",
                "dram_gbs_at_traffic": (traffic / t_comp / 1e9 if traffic else None)}
    # the mapping step's backward kernel, for reference: 10 per evaluated + 38 per contributing evaluation
    t_bwd = stage_ms.get("gs_render_bwd", float("nan")) / 1e3
    bwd_ach = (10.0 * ws["evaluated"] + 38.0 * ws["contributing"]) / t_bwd / 1e12
    rooflines = [roofline, {"bound": "alu", "kernel": "gs_render_bwd (k_render_bwd + k_proj_adjoint)",
                            "achieved": bwd_ach, "peak": peak, "unit": "T lane-instr/s", "frac": bwd_ach / peak,
                            "launch_ms": t_bwd * 1e3}]
    at_load_clock(rooflines, sms, (clocks or {}).get("sm_mhz"))

    # the batched pass against the same candidates one view per call, at identical outputs
    unbatched = None
    if not args.no_unbatched:
        unb = Unbatched(gs, istep)
        ref = istep().clone()
        got = unb().clone()
        torch.cuda.synchronize()
        t_unb = statistics.mean(timed_loop(torch, 3, [("u", unb)], flush)["u"]) / 1e3
        unbatched = {"value": istep.n_views / t_unb, "unit": "views/s", "ms": t_unb * 1e3,
                     "batch_speedup": value * t_unb / istep.n_views,
                     "identical_outputs": bool(torch.equal(ref, got)),
                     "max_abs_diff": float((ref - got).abs().max().item())}
        del unb
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(istep.scene)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "views/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "views_per_step": istep.n_views, "gaussians_ig": istep.gm.n,
                       "gaussians_map": mstep.frame.n, "keyframes": len(mstep.scene.cams),
                       "l2": "flushed (256 MB write) before every timed part", "parallelism": "replicas" if world > 1
                       else "single GPU", "ig_cuda_graph": istep.graph is not None,
                       "map_cuda_graph": mstep.graph is not None,
                       "ig_tiles": {"%dx%d" % k: "%dx%d" % v for k, v in istep.tile_choice.items()},
                       "ig_batch": istep.params.ig_batch,
                       "map_tile": "%dx%d" % (mstep.render_params.tile_w, mstep.render_params.tile_h),
                       "map_fwd_batch": mstep.render_params.fwd_batch},
            "autotune": {"ig_tile_ms": {"%dx%d" % res: {"%dx%d" % t: ms for t, ms in tt.items()}
                                        for res, tt in getattr(istep, "tile_timings", {}).items()},
                         "ig_batch_ms": {str(k): v for k, v in istep.batch_timings.items()},
                         "map_ms": {"%dx%d/%d" % k: v for k, v in mstep.tune_timings.items()}},
            "fwd_bwd": {"value": fwd_bwd, "unit": "iters/s", "ms": t_map_all / args.steps * 1e3},
            "ig_ms": t_ig_all / args.steps * 1e3,
            "ig_unbatched": unbatched,
            "stages_ms": stage_ms,
            "ig_stages_ms_eager": ig_stage_ms,
            "ig_stage_roofline": stage_roofline(pipe, ig_stage_ms, hbm, peak),
            "map_stage_roofline": map_stage_roofline(ws, mstep.frame.n, len(mstep.scene.cams), map_stage_ms, hbm,
                                                     peak),
            "work": ws,
            "ig_pipeline_roofline": pipe,
            "cfg0_forward_latency_us": lat0,
            "cfg1_forward_latency_us": lat1,
            "render_free_xi": xi_free,
            "collision_check": collide,
            "fwd_bwd_eq3_ssim": eq3,
            "config4_loop": cfg4,
            "e2e": e2e,
            "roofline": roofline,
            "rooflines": rooflines,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": launches,
            "gpu": props.name,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(args):
    """The oracle on the host cores, on the same workload: 2 candidates per step, scaled per pixel."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2409_18122_gb300 import scenes
    sc = scenes.config3()
    for _ in range(args.warmup):
        O.info_gain(sc.gmap, [sc.cams[0]])
    t, px = 0.0, 0
    for _ in range(args.steps):
        dt, p = oracle_sample(sc)
        t += dt
        px += p
    value = px / t / mix_pixels_per_view(sc.cams)
    sample = ("FP64 brute-force information gain of candidates 0 (80x60) and 1 (160x120) of the 256 over the "
              "1M-Gaussian map per step, scaled to the 256-view mix by pixel count")
    line = {"metric": METRIC, "value": value, "unit": "views/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD}, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "views/s", "cores": O.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "views/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
