#!/usr/bin/env python
"""Benchmark of the ray-traced Gaussian rendering path (RaySplats, arXiv 2501.19196) on GB300.

One step = one training pass of the whole path over one batch: LBVH rebuild + forward render
+ adjoint for every camera of the workload.  Default workload: 1,000,000 Gaussians (clustered
scene with a background shell) seen by 16 ring cameras of mixed resolution
(8 x 1280x832, 4 x 960x640, 4 x 640x416 = 12,042,240 rays); headline path: one persistent
launch per pass, captured with the rebuild in a CUDA graph.

Prints ONE JSON line (rank 0).  `value` is the device-timed fwd+bwd throughput (Mrays/s) of
the batched path; the line also carries the plain (one launch per camera) numbers, fwd-only
numbers, an end-to-end number through host buffers, the roofline of the dominant kernel, the
SM clocks seen during the timed region and the oracle timed on the host cores.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mrays/s fwd and fwd+bwd at 1M Gaussians, batched vs plain, at oracle tolerance"
L2_FLUSH_BYTES = 256 << 20

# ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of the forward and of the
# hit-list replay on two 640x416 cameras of the same scene (532,480 rays), scaled to a launch of
# the 16-camera workload by its rays (x 22.615; profiles/k_render_fwd_k_replay_list_dram_traffic_
# 1m_gaussians_2x640x416.md).  Reported only while the kernel sources are unchanged (hash).
KERNEL_SOURCES = ("trace.cuh", "render_fwd.cu", "render_bwd.cuh", "render_bwd.cu", "render_bwd_depth.cu",
                  "rs_internal.cuh")
TRAFFIC = {"kernels": "09612d7246d67739", "fwd_bytes": 6.014e9, "bwd_bytes": 6.447e9}
# from the small-case --set full profiles of the same sources, per kernel (forward, list replay):
# the fraction of cycles with an instruction issued (smsp__issue_active), the L2 hit rate
# (lts__t_sector_hit_rate) and the active lanes per warp instruction over 32
# (smsp__thread_inst_executed_per_inst_executed / 32, the warp execution efficiency)
ISSUE_ACTIVE = {"kernels": "09612d7246d67739", "fwd": 0.6482, "bwd": 0.6819}
L2_HIT = {"kernels": "09612d7246d67739", "fwd": 0.8433, "bwd": 0.7610}
WARP_EFF = {"kernels": "09612d7246d67739", "fwd": 23.85 / 32, "bwd": 27.07 / 32}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", type=int, default=4, help="1..4 (see workloads.scenes.workload)")
    p.add_argument("--case", choices=["full", "small"], default="full",
                   help="small: 1M Gaussians, two 640x416 cameras (for ncu captures)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-train", action="store_true", help="skip the full training-step measurement")
    p.add_argument("--no-mirror", action="store_true", help="skip the mirror / shadow scene measurement")
    p.add_argument("--mirror-only", action="store_true", help="only the mirror / shadow scene measurement")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--kbuf", type=int, default=None)
    p.add_argument("--leaf", type=int, default=None)
    p.add_argument("--tile-w", type=int, default=None)
    p.add_argument("--morton-bits", type=int, default=None)
    p.add_argument("--block-warps", type=int, default=None)
    p.add_argument("--traversal", type=int, default=None)
    p.add_argument("--hit-list", type=int, default=None, help="per-ray hit-list capacity (0: adjoint re-traverses)")
    p.add_argument("--smem-nodes", type=int, default=None)
    p.add_argument("--no-autotune", action="store_true", help="default tunables instead of the autotuner's pick")
    p.add_argument("--no-parity", action="store_true", help="skip the oracle check of the bench's own outputs")
    p.add_argument("--profile", action="store_true",
                   help="ncu mode: `warmup` eager batched steps, then one more step, then exit (no JSON)")
    return p.parse_args()


def max_over_ranks(ms, world, device="cpu"):
    """The job's time per step: the slowest rank's (every rank times the same steps between two
    barriers).  One rank: the time itself."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mrays_s(rays_per_rank, ms, world):
    """Whole-job throughput: the rays all ranks processed per step over the job's time per step."""
    return rays_per_rank * world / ms / 1e3


def src_hash(names=KERNEL_SOURCES):
    """Hash of the kernel sources' code: comments and blank lines are left out, so that a change
    of wording does not retire the profile figures, while any change of code does."""
    import re
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2501_19196_gb300", "csrc", name)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        code = "\n".join(line.rstrip() for line in text.splitlines() if line.strip())
        h.update(code.encode())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], parts[5:9]):
                if v.lower() in ("active", "1", "0x1"):
                    reasons.add(nm)
        loaded = [s for s in sm if s > 0.5 * (max(smax) if smax else 1)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------
# workload
# ------------------------------------------------------------------------------------------
def make_workload(args):
    from workloads import scenes
    wl = scenes.workload(args.workload)
    if args.case == "small":
        cams = scenes.concat_cameras([scenes.look_at_camera((12.0, 2.0, 0.0), (0, 0, 0), 640, 416, 60.0),
                                      scenes.look_at_camera((0.0, 2.0, 12.0), (0, 0, 0), 640, 416, 60.0)])
        wl = scenes.Workload(wl.name + "_small2cams", wl.scene, cams, wl.Q, wl.eps1, wl.k_max, wl.background, True)
    return wl


def bench_config(wl, world=1):
    """The workload description both arms print (identical, so the two lines compare)."""
    return {"workload": wl.name, "gaussians": int(wl.scene.n), "cameras": int(wl.cams.count),
            "rays_per_step": int(wl.cams.total_rays()),
            "step": "LBVH rebuild + forward render + adjoint, all cameras",
            "l2": "flushed between timed steps (256 MiB write, untimed)", "parallelism": f"replicas x{world}"}


def step_stats(ms_list):
    """Mean (the contract's time per step), median, min and max of the timed steps (ms)."""
    return {"mean": sum(ms_list) / len(ms_list), "median": statistics.median(ms_list), "min": min(ms_list),
            "max": max(ms_list)}


def parity_pixels(cams, target=1000):
    """A fixed stratified sample of about `target` distinct pixels: every s-th pixel in x and y
    of every camera."""
    import numpy as np
    from workloads import scenes
    s = max(1, int(round((cams.total_rays() / target) ** 0.5)))
    cam, px, py = scenes.pixel_grid(cams, stride=s)
    base = np.concatenate([[0], np.cumsum(cams.n_pixels())[:-1]])
    idx = base[cam] + py.astype(np.int64) * cams.width[cam].astype(np.int64) + px
    return cam, px, py, idx, s


def bench_parity(wl, prm, replay, outs, grads, d_rgb, d_alpha, target=1000, seed=11):
    """The oracle against the benchmark's own outputs: the captured step (`replay`) runs once
    more with an upstream gradient on a stratified pixel sample only (zero elsewhere, and zero
    on rays whose discrete decisions FP32 may take differently), then its image at those pixels
    and its gradients are compared with the FP64 oracle's."""
    import numpy as np
    import torch
    import oracle
    cam, px, py, idx, stride = parity_pixels(wl.cams, target)
    sc = wl.scene
    ora0 = oracle.render(sc, wl.cams, cam, px, py, prm.Q, prm.eps1, prm.k_max, prm.background)
    bad = (ora0["mask"] & oracle.AMB_DECISION) != 0
    rng = np.random.default_rng(seed)
    gc = rng.standard_normal((len(cam), 3))
    ga = rng.standard_normal(len(cam))
    gc[bad] = 0.0
    ga[bad] = 0.0
    ora = oracle.render(sc, wl.cams, cam, px, py, prm.Q, prm.eps1, prm.k_max, prm.background, dl_rgb=gc, dl_alpha=ga)
    keep = (d_rgb.clone(), d_alpha.clone())
    ti = torch.from_numpy(idx).to(d_rgb.device)
    d_rgb.zero_()
    d_alpha.zero_()
    d_rgb[ti] = torch.from_numpy(gc.astype(np.float32)).to(d_rgb.device)
    d_alpha[ti] = torch.from_numpy(ga.astype(np.float32)).to(d_rgb.device)
    replay()
    torch.cuda.synchronize()
    rgb = outs[0][ti].cpu().numpy().astype(np.float64)
    alpha = outs[1][ti].cpu().numpy().astype(np.float64)
    depth = outs[2][ti].cpu().numpy().astype(np.float64)
    got = {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}
    d_rgb.copy_(keep[0])
    d_alpha.copy_(keep[1])
    ok = (ora["mask"] & oracle.AMB_IMPACT) == 0
    e_rgb = float(np.abs(rgb[ok] - ora["rgb"][ok]).max(initial=0.0))
    e_a = float(np.abs(alpha[ok] - ora["alpha"][ok]).max(initial=0.0))
    e_d = float((np.abs(depth[ok] - ora["depth"][ok]) / np.maximum(1.0, ora["depth"][ok])).max(initial=0.0))
    rel = {}
    for k in ("means", "quats", "scales", "opacities", "rgb"):
        ref = ora["grads"][k]
        rel[k] = float(np.linalg.norm(got[k].reshape(ref.shape) - ref) / max(np.linalg.norm(ref), 1e-30))
    ok_all = e_rgb <= 2e-4 and e_a <= 2e-4 and max(rel.values()) <= 1e-3
    return {"pixels": int(len(cam)), "sample": f"every {stride}th pixel in x and y of every camera",
            "masked_frac": float(1.0 - ok.mean()), "decision_flagged_frac": float(bad.mean()),
            "max_abs_rgb": e_rgb, "max_abs_alpha": e_a, "max_rel_depth": e_d, "grad_rel_l2": rel,
            "tolerance": {"rgb_alpha_abs": 2e-4, "grad_rel_l2": 1e-3}, "pass": bool(ok_all),
            "path": "the timed CUDA graph, replayed with the sampled upstream gradient"}


def bench_candidates(native, base):
    """The autotuner's candidates for the benchmark: the default and three neighbours."""
    d = base.as_dict()
    out = [native.default_tune(**d)]
    for kw in (dict(tile_w=4, tile_h=8), dict(leaf_size=24), dict(morton_bits=20)):
        out.append(native.default_tune(**dict(d, **kw)))
    return out


def _timed_events(fn, steps, warmup, flush, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(steps):
        flush.fill_(1.0)  # L2 flush (untimed)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    return total / steps, None


def run_mirror(args, dev, timed=None, stream=None):
    """Gaussians with a mirror sphere and a diffuse floor lit through them (rs_render_scene):
    forward and forward + adjoint rays per second, one 1280 x 832 camera, up to two bounces
    and one shadow ray per floor hit."""
    import numpy as np
    import torch
    from paper_2501_19196_gb300 import RenderParams, native
    from paper_2501_19196_gb300.scene import SceneRenderer
    from workloads import scenes
    sc, mesh, cams = scenes.workload_mirror()
    params = [torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev)
              for a in (sc.means, sc.quats, sc.scales, sc.opacities, sc.rgb)]
    P = int(cams.total_rays())
    prm = RenderParams(Q=scenes.default_Q(), eps1=1e-4, background=(0.0, 0.0, 0.0))
    sr = SceneRenderer(mesh, tune=native.default_tune(), Q_box=scenes.default_Q(), list_cap=1024, shadow_cap=1024)
    outs = (torch.empty((P, 3), device=dev), torch.empty(P, device=dev), torch.empty(P, device=dev))
    g_rgb, g_alpha = scenes.upstream_grad(P)
    d_rgb, d_alpha = torch.from_numpy(g_rgb).to(dev), torch.from_numpy(g_alpha).to(dev)
    n = params[0].shape[0]
    grads = {"means": torch.zeros((n, 3), device=dev), "quats": torch.zeros((n, 4), device=dev),
             "scales": torch.zeros((n, 3), device=dev), "opacities": torch.zeros(n, device=dev),
             "rgb": torch.zeros((n, 3), device=dev)}

    def step(backward):
        sr.build(*params)
        sr.render(cams, prm, out=outs)
        if backward:
            for t in grads.values():
                t.zero_()
            sr.backward(d_rgb, d_alpha, grads=grads)

    if timed is None:
        stream = torch.cuda.current_stream()
        flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)
        timed = lambda fn, k, w: _timed_events(fn, k, w, flush, stream)  # noqa: E731
    step(True)
    sr.check_device()
    ms_f, _ = timed(lambda: step(False), max(1, min(3, args.steps)), 1)
    ms_fb, _ = timed(lambda: step(True), max(1, min(3, args.steps)), 1)
    sr.check_device()
    sr.close()
    return {"workload": "2m_gaussians_mirror_sphere_50k_tris_floor_1280x832", "gaussians": n,
            "triangles": int(len(mesh["mat"])), "rays": P, "max_bounces": mesh["max_bounces"],
            "fwd_mrays_s": P / ms_f / 1e3, "fwd_bwd_mrays_s": P / ms_fb / 1e3, "ms_fwd": ms_f, "ms_fwd_bwd": ms_fb,
            "step": "LBVH rebuild + scene render (mirror bounces, shadow rays) [+ adjoint]"}


def oracle_sample_pixels(wl, n_rays, seed=5):
    """Stratified pixel sample over all cameras (proportional to each camera's pixel count)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    npx = wl.cams.n_pixels()
    cam = rng.choice(wl.cams.count, size=n_rays, p=npx / npx.sum()).astype(np.int32)
    px = (rng.random(n_rays) * wl.cams.width[cam]).astype(np.int32)
    py = (rng.random(n_rays) * wl.cams.height[cam]).astype(np.int32)
    return cam, px, py


def cpu_oracle_rate(wl, seconds, threads=None):
    """Oracle (fwd + gradient) on a bounded ray sample of the workload: Mrays/s on the host."""
    import numpy as np
    import oracle
    threads = threads or oracle.default_threads()
    n = 64
    while True:
        cam, px, py = oracle_sample_pixels(wl, n)
        rng = np.random.default_rng(1)
        gc, ga = rng.standard_normal((n, 3)), rng.standard_normal(n)
        t0 = time.perf_counter()
        oracle.render(wl.scene, wl.cams, cam, px, py, wl.Q, wl.eps1, wl.k_max, wl.background, dl_rgb=gc,
                      dl_alpha=ga, threads=threads)
        dt = time.perf_counter() - t0
        if dt >= 0.5 * seconds or n >= 1 << 20:
            return n / dt / 1e6, n, dt, threads
        n = int(min(n * max(2.0, 0.8 * seconds / max(dt, 1e-3)), 1 << 20))


# ------------------------------------------------------------------------------------------
# reference arm: the oracle, as it stands, on the host cores
# ------------------------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = make_workload(args)
    import oracle
    threads = oracle.default_threads()
    rate, n, dt, _ = cpu_oracle_rate(wl, seconds=min(args.cpu_seconds, 8.0), threads=threads)
    import numpy as np
    times = []
    for s in range(args.warmup + args.steps):
        cam, px, py = oracle_sample_pixels(wl, n, seed=100 + s)
        rng = np.random.default_rng(s)
        t0 = time.perf_counter()
        oracle.render(wl.scene, wl.cams, cam, px, py, wl.Q, wl.eps1, wl.k_max, wl.background,
                      dl_rgb=rng.standard_normal((n, 3)), dl_alpha=rng.standard_normal(n), threads=threads)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    mean = sum(times) / len(times)
    value = n / mean / 1e6
    sample = f"{n} rays per step, stratified over the {wl.cams.count} cameras, fwd + gradient, brute force"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(wl, 1), "path": "FP64 CPU oracle (brute force)",
        "cpu_baseline": {"value": value, "unit": "Mrays/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2501_19196_gb300 import Renderer, RenderParams, native
    from workloads import scenes

    native.load()
    dev = torch.device("cuda", local)
    if args.mirror_only:
        m = run_mirror(args, dev)
        if rank == 0:
            print(json.dumps({"metric": "Mrays/s of the mirror / shadow scene render", "value": m["fwd_bwd_mrays_s"],
                              "unit": "Mrays/s", "higher_is_better": True, "mirror_scene": m}), flush=True)
        return
    wl = make_workload(args)
    host = [np.ascontiguousarray(a, np.float32) for a in (wl.scene.means, wl.scene.quats, wl.scene.scales,
                                                         wl.scene.opacities, wl.scene.rgb)]
    params = [torch.from_numpy(a).to(dev) for a in host]
    P = int(wl.cams.total_rays())
    g_rgb_h, g_alpha_h = scenes.upstream_grad(P, seed=1)
    d_rgb = torch.from_numpy(g_rgb_h).to(dev)
    d_alpha = torch.from_numpy(g_alpha_h).to(dev)
    prm = RenderParams(Q=wl.Q, eps1=wl.eps1, background=wl.background, k_max=wl.k_max)
    overrides = {}
    if args.kbuf:
        overrides["kbuf"] = args.kbuf
    if args.leaf:
        overrides["leaf_size"] = args.leaf
    if args.tile_w:
        overrides["tile_w"] = args.tile_w
    if args.morton_bits:
        overrides["morton_bits"] = args.morton_bits
    if args.block_warps:
        overrides["block_warps"] = args.block_warps
    if args.traversal is not None:
        overrides["traversal"] = args.traversal
    if args.smem_nodes is not None:
        overrides["smem_nodes"] = args.smem_nodes
    if args.hit_list is not None:
        overrides["hit_list"] = args.hit_list
    tune_default = native.default_tune(persistent=1, **overrides)
    autotune = None
    tune_b = tune_default
    if not overrides and not args.no_autotune and not args.profile:
        # the batched arm runs the autotuner's pick (cached per GPU / scene size / rays / cameras)
        from paper_2501_19196_gb300 import tune as tuner
        cands = bench_candidates(native, tune_default)
        t0 = time.perf_counter()
        tune_b, table = tuner.autotune(params, wl.cams, prm, d_rgb=d_rgb, d_alpha=d_alpha, cands=cands, reps=3)
        autotune = {"chosen": tune_b.as_dict(), "candidates": len(cands), "seconds": time.perf_counter() - t0,
                    "ms_per_candidate": {json.dumps(c.as_dict(), sort_keys=True): table.get(
                        json.dumps(c.as_dict(), sort_keys=True)) for c in cands},
                    "default_ms": table.get(json.dumps(tune_default.as_dict(), sort_keys=True)),
                    "timing": "rs_tune: eager LBVH rebuild + forward + adjoint, CUDA events, 3 repetitions"}
    tune_p = native.default_tune(**dict(tune_b.as_dict(), persistent=0))
    n = wl.scene.n
    outs = (torch.empty((P, 3), device=dev), torch.empty(P, device=dev), torch.empty(P, device=dev))
    grads = {"means": torch.zeros((n, 3), device=dev), "quats": torch.zeros((n, 4), device=dev),
             "scales": torch.zeros((n, 3), device=dev), "opacities": torch.zeros(n, device=dev),
             "rgb": torch.zeros((n, 3), device=dev)}
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)
    stream = torch.cuda.current_stream()

    rb = Renderer(tune=tune_b, Q_box=wl.Q)
    rp = Renderer(tune=tune_p, Q_box=wl.Q)
    rb.set_cameras(wl.cams)
    rp.set_cameras(wl.cams)

    def step(r, backward=True):
        r.build(*params)
        r.render(None, prm, out=outs)
        if backward:
            for t in grads.values():
                t.zero_()
            r.backward(d_rgb, d_alpha, grads=grads)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    step_ms = {}

    def timed(fn, steps, warmup, sampler=None, name=None):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        barrier()
        if sampler:
            sampler.start()
        evs = []
        for _ in range(steps):
            flush.fill_(1.0)  # L2 flush (untimed)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        barrier()
        clocks = sampler.stop() if sampler else None
        each = [a.elapsed_time(b) for a, b in evs]
        if name:
            step_ms[name] = step_stats(each)
        ms = max_over_ranks(sum(each) / steps, world, dev)
        return ms, clocks

    if args.profile:
        for _ in range(args.warmup + 1):
            step(rb)
        torch.cuda.synchronize()
        rb.check_device()
        rb.close()
        rp.close()
        return

    # --- warm up both renderers eagerly (allocations happen here) ---
    step(rb)
    step(rp)
    rb.check_device()
    rp.check_device()

    # --- CUDA graphs: rebuild + fwd + bwd, and rebuild + fwd ---
    def capture(fn):
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            fn()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            fn()
        torch.cuda.synchronize()
        return g

    g_fb = capture(lambda: step(rb, True))
    g_f = capture(lambda: step(rb, False))

    sampler = ClockSampler(local)
    ms_fb, clocks = timed(g_fb.replay, args.steps, args.warmup, sampler, name="fwd_bwd")
    ms_f, _ = timed(g_f.replay, args.steps, args.warmup, name="fwd")
    rb.check_device()
    # the oracle against this run's own outputs (the same graph, replayed once more)
    parity = None
    if rank == 0 and not args.no_parity:
        t0 = time.perf_counter()
        parity = bench_parity(wl, prm, g_fb.replay, outs, grads, d_rgb, d_alpha)
        parity["seconds"] = time.perf_counter() - t0
        rb.check_device()
    ms_fb_nograph, _ = timed(lambda: step(rb, True), max(3, args.steps // 2), 1)
    # the adjoint without hit lists (every ray re-traverses the BVH), same graph-captured step
    replay = None
    if tune_b.hit_list > 0 and not args.no_plain:
        rr = Renderer(tune=native.default_tune(**dict(tune_b.as_dict(), hit_list=0)), Q_box=wl.Q)
        rr.set_cameras(wl.cams)
        step(rr)
        g_rr = capture(lambda: step(rr, True))
        ms_rr, _ = timed(g_rr.replay, max(3, args.steps // 2), args.warmup)
        rr.check_device()
        del g_rr
        rr.close()
        replay = {"fwd_bwd_mrays_s": P / ms_rr / 1e3 * world, "ms_per_step_fwd_bwd": ms_rr,
                  "adjoint": "re-traversal of every ray (hit_list 0)"}
    # the paper's adjoint variants on the same step (eager launches, the batched renderer):
    # hits ordered by the maximum-response parameter t_m, the depth gradient, and the eps2
    # estimator for the last meaningful Gaussian
    variants = None
    if not args.no_plain:
        variants = {}
        d_depth = torch.from_numpy(scenes.upstream_grad(P, seed=3)[1]).to(dev)

        def vstep(p, depth_grad=False):
            rb.build(*params)
            rb.render(None, p, out=outs)
            for t in grads.values():
                t.zero_()
            rb.backward(d_rgb, d_alpha, grads=grads, d_depth=d_depth if depth_grad else None)

        for name, p, dg in (("sort_key_tm", RenderParams(Q=wl.Q, eps1=wl.eps1, background=wl.background,
                                                         k_max=wl.k_max, sort_key=1), False),
                            ("depth_gradient", prm, True),
                            ("eps2_estimator", RenderParams(Q=wl.Q, eps1=wl.eps1, background=wl.background,
                                                            k_max=wl.k_max, eps2=0.01), False)):
            ms_v, _ = timed(lambda: vstep(p, dg), max(3, args.steps // 3), 1)
            variants[name] = {"fwd_bwd_mrays_s": P / ms_v / 1e3 * world, "ms_per_step_fwd_bwd": ms_v}
        rb.check_device()
        variants["launches"] = "eager (no graph), batched persistent path, hit lists"
        variants["eps2"] = 0.01
    plain = {}
    if not args.no_plain:
        ms_p_fb, _ = timed(lambda: step(rp, True), max(3, args.steps // 2), 1)
        ms_p_f, _ = timed(lambda: step(rp, False), max(3, args.steps // 2), 1)
        rp.check_device()
        plain = {"fwd_bwd_mrays_s": P / ms_p_fb / 1e3 * world, "fwd_mrays_s": P / ms_p_f / 1e3 * world,
                 "ms_per_step_fwd_bwd": ms_p_fb, "ms_per_step_fwd": ms_p_f,
                 "launches_per_step": "one forward and one hit-list replay launch per camera, one "
                                      "re-traversal launch over the overflow tiles"}

    # --- per-kernel durations (events on the launching stream), batched path ---
    kt = {"build": [], "fwd": [], "bwd": []}
    for _ in range(max(3, args.steps // 2)):
        flush.fill_(1.0)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        rb.build(*params)
        ev[1].record(stream)
        rb.render(None, prm, out=outs)
        ev[2].record(stream)
        for t in grads.values():
            t.zero_()
        rb.backward(d_rgb, d_alpha, grads=grads)
        ev[3].record(stream)
        torch.cuda.synchronize()
        kt["build"].append(ev[0].elapsed_time(ev[1]))
        kt["fwd"].append(ev[1].elapsed_time(ev[2]))
        kt["bwd"].append(ev[2].elapsed_time(ev[3]))
    kms = {k: sum(v) / len(v) for k, v in kt.items()}

    # --- traversal counters (instrumented kernels, same inputs) ---
    stats_f = torch.zeros(10, dtype=torch.int64, device=dev)
    stats_b = torch.zeros(10, dtype=torch.int64, device=dev)
    rb.build(*params)
    rb.render(None, prm, out=outs, stats=stats_f)
    for t in grads.values():
        t.zero_()
    rb.backward(d_rgb, d_alpha, grads=grads, stats=stats_b)
    torch.cuda.synchronize()
    rb.check_device()
    sf = dict(zip(native.STATS_FIELDS, stats_f.cpu().tolist()))
    sb = dict(zip(native.STATS_FIELDS, stats_b.cpu().tolist()))
    # algorithmic bytes per launch: node 64 B, test record 48 B, shade 16 B, outputs + state
    # 36 B per ray, 4 B per hit-list id written; backward: replayed hit 64 B record + 64 B
    # atomics, 4 B per id read from a hit list, 32 B per ray.  A re-traversed ray had more hits
    # than the list holds, so the forward wrote a full list for it.
    ids_written = sb["hits_listed"] + tune_b.hit_list * sb["rays_retraced"] if tune_b.hit_list > 0 else 0
    fwd_bytes = (64 * sf["nodes_visited"] + 48 * sf["gaussians_tested"] + 16 * sf["hits_composited"] +
                 36 * sf["rays"] + 4 * ids_written)
    bwd_bytes = (64 * sb["nodes_visited"] + 48 * sb["gaussians_tested"] + 128 * sb["hits_composited"] +
                 4 * sb["hits_listed"] + 32 * sb["rays"])
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    dom = "bwd" if kms["bwd"] >= kms["fwd"] else "fwd"
    dom_bytes = bwd_bytes if dom == "bwd" else fwd_bytes
    achieved = dom_bytes / (kms[dom] * 1e-3) / 1e9
    traffic = None
    if TRAFFIC.get("kernels") == src_hash():
        traffic = TRAFFIC["bwd_bytes" if dom == "bwd" else "fwd_bytes"]
    # The dominant kernel is bound by instruction issue and latency (small-case --set full
    # profile: issue slots busy ISSUE_ACTIVE of the time, DRAM nearly idle), not by HBM: `frac`
    # is the touched-bytes fraction (node, record and output bytes the method must read, mostly
    # L1/L2 hits) against the HBM copy peak, and `dram_frac` the measured DRAM traffic's.
    roofline = {"bound": "issue/latency", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "frac_kind": "touched (algorithmic) bytes over the HBM copy peak",
                "traffic": traffic,
                "dram_frac": (traffic / (kms[dom] * 1e-3) / 1e9 / hbm) if traffic else None,
                "issue_active": ISSUE_ACTIVE.get(dom) if ISSUE_ACTIVE.get("kernels") == src_hash() else None,
                "l2_hit_rate": L2_HIT.get(dom) if L2_HIT.get("kernels") == src_hash() else None,
                "warp_exec_efficiency": WARP_EFF.get(dom) if WARP_EFF.get("kernels") == src_hash() else None,
                "kernel": "adjoint: k_replay_list + k_render_bwd + k_finalize" if dom == "bwd"
                else "k_render_fwd (persistent)", "peak_source": f"{peak_kind} hbm_gbs",
                "algorithmic_bytes_per_launch": dom_bytes, "kernel_ms": kms[dom],
                "counts_fwd": sf, "counts_bwd": sb,
                "min_bytes_fraction": (64 * sf["hits_composited"] + 36 * sf["rays"]) / (kms["fwd"] * 1e-3) / 1e9 / hbm}

    # --- end to end through host buffers (pinned) ---
    e2e = None
    if not args.no_e2e:
        pinned_in = [torch.from_numpy(a).pin_memory() for a in host] + \
                    [torch.from_numpy(g_rgb_h).pin_memory(), torch.from_numpy(g_alpha_h).pin_memory()]
        pinned_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in grads.items()}
        h2d = sum(t.numel() * t.element_size() for t in pinned_in)
        d2h = sum(t.numel() * t.element_size() for t in pinned_out.values())

        # A pipelined loop, as a training loop would run it: two sets of device buffers (inputs,
        # gradients) with their own graphs (rebuild + render, adjoint); step i's inputs cross on
        # a copy stream and its gradients return on another while the steps before and after it
        # compute.  Every step still copies all of its inputs in and its gradients out.

        def adjoint_on(dr, da, gr):
            def fn():
                for t in gr.values():
                    t.zero_()
                rb.backward(dr, da, grads=gr)
            return fn

        sets = [(params, d_rgb, d_alpha, grads, g_f, capture(adjoint_on(d_rgb, d_alpha, grads)), pinned_out)]
        p1 = [t.clone() for t in params]
        dr1, da1 = d_rgb.clone(), d_alpha.clone()
        gr1 = {k: torch.zeros_like(v) for k, v in grads.items()}
        gf1 = capture(lambda: (rb.build(*p1), rb.render(None, prm, out=outs)))
        sets.append((p1, dr1, da1, gr1, gf1, capture(adjoint_on(dr1, da1, gr1)),
                     {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in grads.items()}))
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

        def e2e_run(k):
            main = torch.cuda.current_stream()
            free = [None, None]  # set j may be overwritten once this event fires
            for i in range(k):
                pj, drj, daj, grj, gfj, gbj, poj = sets[i % 2]
                with torch.cuda.stream(s_in):
                    if free[i % 2] is not None:
                        s_in.wait_event(free[i % 2])
                    for h, d in zip(pinned_in, pj + [drj, daj]):
                        d.copy_(h, non_blocking=True)
                    ev_in = torch.cuda.Event()
                    ev_in.record(s_in)
                main.wait_event(ev_in)
                gfj.replay()
                gbj.replay()
                ev_done = torch.cuda.Event()
                ev_done.record(main)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ev_done)
                    for kk, v in grj.items():
                        poj[kk].copy_(v, non_blocking=True)
                    free[i % 2] = torch.cuda.Event()
                    free[i % 2].record(s_out)
            torch.cuda.synchronize()

        e2e_run(2)
        barrier()
        t0 = time.perf_counter()
        e2e_run(args.steps)
        barrier()
        ms_e2e = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps, world, dev)
        e2e = {"value": job_mrays_s(P, ms_e2e, world), "unit": "Mrays/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e,
               "path": "every step: pinned host params + dL -> device on a copy stream, rebuild + render "
                       "and adjoint graphs, gradients -> pinned host on a second copy stream; two buffer "
                       "sets, so a step's copies overlap its neighbours' compute"}
        del sets, gf1
        # the graphs above leave the renderer's scene pointers at the second set: point them back
        rb.build(*params)

    # --- full training step: activations, rebuild, render, L2 + D-SSIM loss, adjoint, Adam ---
    train = None
    if not args.no_train:
        from paper_2501_19196_gb300 import TrainStep
        del g_fb, g_f
        target = outs[0].clone()  # the images of the scene; training starts from perturbed colours
        gen = torch.Generator(device="cpu").manual_seed(11)
        rgb0 = (params[4] + 0.2 * torch.randn(params[4].shape, generator=gen).to(dev)).clamp(0, 1)
        logit = lambda x: torch.log(x / (1 - x))  # noqa: E731
        ts = TrainStep(params[0], params[1], logit(params[2]), logit(params[3]), rgb0, params=prm, tune=tune_b,
                       Q_box=wl.Q)
        ts.renderer.set_cameras(wl.cams)
        ms_train, _ = timed(lambda: ts.step(target), max(3, args.steps // 2), 2)
        l0 = float(ts.step(target).item())
        lt = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            rgb_out = ts.renderer.render(None, prm)[0]
            e0.record(stream)
            ts.loss_fn(rgb_out, target, ts.renderer._cams)
            e1.record(stream)
            torch.cuda.synchronize()
            lt.append(e0.elapsed_time(e1))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        from paper_2501_19196_gb300 import adam_step
        adam_step(ts.flat, ts.grad, ts.m, ts.v, 1, 0.0)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.close()
        train = {"mrays_s": P / ms_train / 1e3 * world, "ms_per_step": ms_train, "loss_ms": sum(lt) / len(lt),
                 "adam_ms": e0.elapsed_time(e1), "loss_after_warmup": l0, "lambda": 0.2,
                 "step": "sigmoid activations + LBVH rebuild + render + L2/D-SSIM loss and gradient + adjoint + "
                         "sigmoid adjoints + Adam (eager launches)"}

    # --- secondary rays: 2M Gaussians, a 50,000-triangle mirror sphere, a lit floor ---
    mirror = None
    if not args.no_mirror and args.case == "full":
        mirror = run_mirror(args, dev, timed, stream)

    # --- CPU oracle baseline (rank 0) ---
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, nr, dt, thr = cpu_oracle_rate(wl, args.cpu_seconds)
        cpu = {"value": rate, "unit": "Mrays/s", "cores": thr, "kind": "oracle",
               "sample": f"{nr} stratified rays of the same workload, fwd + gradient, FP64 brute force, {dt:.1f} s"}

    # the LBVH rebuild, reported apart: algorithmic bytes per Gaussian (bounds 12; Morton codes
    # 12 read + 12 written; 8 radix passes of 8 B histogram reads and 24 B scatter traffic;
    # records 56 read + 88 written; Karras and refit about 160 per node) over its event time
    build_bytes = n * (12 + 24 + 8 * 32 + 144 + 160)
    build = {"ms": kms["build"], "algorithmic_bytes": build_bytes,
             "achieved_gbs": build_bytes / (kms["build"] * 1e-3) / 1e9,
             "frac_of_hbm": build_bytes / (kms["build"] * 1e-3) / 1e9 / hbm,
             "launches": 3 + 3 * (4 if tune_b.morton_bits == 10 else 8) + 3 + (1 if tune_b.smem_nodes > 0 else 0),
             "bound": "launch and latency (31 short launches, 1M-element kernels)"}
    # bounds init, bounds, morton, 3 per sort pass, records, karras, refit, top-node staging
    launches_build = 3 + 3 * (4 if tune_b.morton_bits == 10 else 8) + 3 + (1 if tune_b.smem_nodes > 0 else 0)
    # forward; adjoint: list replay + re-traversal of the overflow tiles (or one re-traversal
    # launch without hit lists) + finalize
    gpu_launches = args.steps * (launches_build + 1 + (3 if tune_b.hit_list > 0 else 2))
    # ALU side of the forward (secondary): the FP32 lane operations the traversal must execute
    # per launch (a model: 30 per node visit for its two slab tests, 55 per full Gaussian test
    # for the stable solve with its division, 60 per composited hit for the solve again, exp
    # and the blend; an FMA counts once), against the FP32 lane rate at the sampled SM clock
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    fp32_ops = 30 * sf["nodes_visited"] + 55 * sf["gaussians_tested"] + 60 * sf["hits_composited"]
    alu_peak = sms * 128 * mhz * 1e6 / 1e12
    roofline["alu_secondary"] = {
        "fp32_ops_per_launch": fp32_ops, "achieved": fp32_ops / (kms["fwd"] * 1e-3) / 1e12, "peak": alu_peak,
        "unit": "T FP32 lane ops/s", "frac": fp32_ops / (kms["fwd"] * 1e-3) / 1e12 / alu_peak,
        "peak_source": f"{sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz (sampled)",
        "kernel": "k_render_fwd (persistent)"}
    value = job_mrays_s(P, ms_fb, world)
    line = {
        "metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_fb, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(wl, world),
        "path": "batched: one persistent forward launch; adjoint: one persistent hit-list replay "
                "launch and one persistent re-traversal launch over the overflow tiles; CUDA graph",
        "tune": tune_b.as_dict(), "autotune": autotune, "step_ms": step_ms, "parity": parity,
        "fwd_mrays_s": P / ms_f / 1e3 * world, "ms_per_step_fwd": ms_f,
        "render_only_mrays_s": P / kms["fwd"] / 1e3 * world,
        "fwd_bwd_mrays_s_no_graph": P / ms_fb_nograph / 1e3 * world,
        "plain": plain,
        "batched_over_plain_fwd_bwd": (plain["ms_per_step_fwd_bwd"] / ms_fb) if plain else None,
        "kernel_ms": kms,
        "adjoint_without_hit_lists": replay, "adjoint_variants": variants, "training_step": train,
        "mirror_scene": mirror,
        "roofline": roofline, "build": build, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line))
    rb.close()
    rp.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
