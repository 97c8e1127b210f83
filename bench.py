"""Benchmark of the NGP-RT render path on GB300: 1080p frames/s and Grays/s.

``python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]``

One step = one 1920x1080 frame of the hd workload (unbounded 360-style scene, L=16
levels 16..4096, T=2^19, 128^3 occupancy + distance grid, MLP 23->64->64->3), plain
FP32 tables and MLP: the march kernel (occupancy-distance marching, coarse fetch,
16-level gathers, attention, compositing) then the deferred-MLP kernel.  Inputs are
resident in HBM; L2 is flushed (a 256 MiB write) between timed frames, outside the
timed events.  Under torchrun every rank renders its own view (weak scaling,
replicas: no data-path collective); rank 0 prints one JSON line.

``--impl reference`` times the CPU oracle (the only other program of the same
computation) on a bounded pixel sample of the same frame, on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2407_10482_gb300 import scenes as S  # noqa: E402

METRIC = "1080p frames/s & Grays/s, plain FP32 vs FP16+proposal at ≤0.1 dB PSNR loss"
# DRAM bytes (read + write) of one march_kernel<16,F32> launch on this frame, from the
# ncu capture summarised in profiles/march_kernel_hd_1080p_fp32.md; None while the
# kernel has changed since the counters were taken
MARCH_DRAM_BYTES = 2.545277e9  # 2.187119 GB read + 0.358158 GB written
# l1tex__data_pipe_lsu_wavefronts.avg.pct_of_peak_sustained_elapsed of the same capture
L1_LSU_PCT = 80.34
WORKLOAD = "hd 1920x1080 unbounded-360 synthetic scene, L=16 (16..4096), T=2^19, 128^3 occupancy+G, MLP 23-64-64-3"


def _peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return dict(hbm_gbs=d.get("hbm_gbs"), bf16_tflops=d.get("bf16_tflops"), source="measured")
    return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, source="fallback")


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"ngprt_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_views(rank: int, views_per_rank: int = 1, step_deg: float = 45.0) -> list:
    """Azimuths (degrees) of the views rank `rank` renders: ranks are independent
    replicas, each with its own views of the orbit, so there is no data-path
    collective; the whole-job rate is the views of all ranks over the slowest rank."""
    return [step_deg * (rank * views_per_rank + k) for k in range(views_per_rank)]


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Largest value over the ranks (the timing of the slowest rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(cfg, scene, cams, opts, sample_stride: int = 16) -> dict:
    """The oracle on a stratified pixel sample (every sample_stride-th pixel) of the
    frame, on all host cores; rays/s scaled to frames/s of the full frame."""
    from oracle import oracle as O
    orc = O.oracle_for_scene(scene)
    n = cfg.W * cfg.H
    pix = np.arange(0, n, sample_stride, dtype=np.int32)
    t0 = time.perf_counter()
    orc.render(opts, cams=cams, pix=pix)
    dt = time.perf_counter() - t0
    rays_s = len(pix) / dt
    return {"value": rays_s / n, "unit": "frames/s", "rays_per_s": rays_s, "cores": O.max_threads(),
            "kind": "oracle", "seconds": dt,
            "sample": f"{len(pix)} pixels (every {sample_stride}th pixel of the 1920x1080 frame), FP64 oracle, OpenMP"}


def run_reference(args):
    world, rank, _ = _dist_setup()
    if rank != 0:
        return
    cfg = S.hd_config()
    scene = S.make_scene(cfg)
    cams = S.orbit_cameras(cfg, 1)
    opts = S.default_options(cfg)
    from oracle import oracle as O
    orc = O.oracle_for_scene(scene)
    stride = args.ref_stride
    n = cfg.W * cfg.H
    steps = []
    for k in range(args.warmup + args.steps):
        pix = np.arange(k % stride, n, stride, dtype=np.int32)
        t0 = time.perf_counter()
        orc.render(opts, cams=cams, pix=pix)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            steps.append(dt * stride)  # seconds per full frame
    ms = 1000.0 * statistics.mean(steps)
    value = 1000.0 / ms
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"1/{stride} of the pixels per step, extrapolated"},
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": O.max_threads(), "kind": "oracle",
                             "sample": f"every {stride}th pixel of the frame per step (offset by step)"},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _timed(fn, stream, flush, reps, warmup):
    """Mean CUDA-event time (ms) of fn() on `stream`, L2 flushed before each call."""
    import torch
    for _ in range(warmup):
        fn()
    out = []
    for k in range(reps):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return statistics.mean(out)


def other_forms(args, cfg, scene, ds, docc, cams, opts, dev, stream, flush, plain_rgb):
    """The FP16 + proposal form, 8-view batches, the training step and the gather
    ceiling, on the same GPU (reported beside the plain FP32 frame)."""
    import torch
    from paper_2407_10482_gb300 import ngprt as ng
    from paper_2407_10482_gb300 import proposal as P
    n = cfg.W * cfg.H
    res = {}
    reps, warm = max(3, args.steps // 2), args.warmup
    rend32 = ng.Renderer(ds, docc, device=dev)
    plain = rend32.render(opts, cams=cams, W=cfg.W, H=cfg.H, stats=True)
    plain_rgb = plain["rgb"].clone()
    plain_st = plain["stats"].float().mean(0)
    # learned proposal: trained on the plain renderer's weights over 64 orbit views
    # that differ from the test views, every step in the library's kernels
    t0 = time.perf_counter()
    train_cams = S.orbit_cameras(cfg, 64, azimuth0=2.8125, step_deg=5.625)
    pix = torch.as_tensor(S.random_pixels(1 << 20, 64, cfg.W, cfg.H, 4)).to(dev)
    targets = P.make_targets(rend32, opts, train_cams, cfg.W, cfg.H, pix)
    pc = P.ProposalConfig()
    w, hist = P.train(train_cams, cfg.W, cfg.H, pix, targets, pc, log_every=500)
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0
    # FP16 tables, FP16 tensor-core MLP, proposal + fallback
    ds16 = ng.DeviceScene(cfg, scene.tables, scene.coarse, scene.mlp_w, table_dtype=1, mlp_dtype=1, device=dev)
    fr = P.FastRenderer(ds16, docc, w, pc, device=dev)
    rgb = torch.empty(n, 3, device=dev)
    fr.render(opts, cams, cfg.W, cfg.H, rgb, stats=True)
    torch.cuda.synchronize(dev)
    fast_st = fr.stats.float().mean(0)
    fast_psnr = P.psnr(rgb, plain_rgb)
    ms_fast = _timed(lambda: fr.render(opts, cams, cfg.W, cfg.H, rgb, stream=stream), stream, flush, reps, warm)
    # a 4x finer-step render of the same model approximates its continuous volume
    # rendering: the PSNR loss of the fast form is measured against it as well
    opts_fine = S.default_options(cfg, step_gamma=0.25, max_march=4096, max_samples=4096)
    ref = rend32.render(opts_fine, cams=cams, W=cfg.W, H=cfg.H)["rgb"].clone()
    psnr_plain_ref = P.psnr(plain_rgb, ref)
    psnr_fast_ref = P.psnr(rgb, ref)
    # FP16 tables + tensor-core MLP without the proposal (precision form alone)
    r16 = ng.Renderer(ds16, docc, device=dev)
    o16 = r16.render(opts, cams=cams, W=cfg.W, H=cfg.H)
    p16 = P.psnr(o16["rgb"], plain_rgb)
    ms_16 = _timed(lambda: r16.render(opts, cams=cams, W=cfg.W, H=cfg.H, out=o16), stream, flush, reps, warm)
    res["forms"] = {
        "fp16_tables_tc_mlp": {"ms_per_frame": ms_16, "frames_per_s": 1000.0 / ms_16, "psnr_vs_plain_db": p16},
        "fp16_tc_mlp_proposal": {
            "ms_per_frame": ms_fast, "frames_per_s": 1000.0 / ms_fast, "grays_per_s": n / ms_fast / 1e6,
            "psnr_vs_plain_db": fast_psnr, "loss_0p1dB_threshold_db": 41.9,
            "psnr_vs_fine_ref_db": psnr_fast_ref, "plain_psnr_vs_fine_ref_db": psnr_plain_ref,
            "psnr_loss_vs_fine_ref_db": psnr_plain_ref - psnr_fast_ref,
            "marching_per_ray": float(fast_st[0]), "samples_per_ray": float(fast_st[1]),
            "plain_marching_per_ray": float(plain_st[0]), "plain_samples_per_ray": float(plain_st[1]),
            "fallback_rays": float(((fr.a_hat - fr.state[:, 7]) > pc.fallback).float().mean()),
            "proposal_train_s": train_s, "proposal_loss": hist,
            "training": "2^20 rays of 64 orbit views (azimuth 2.8125 + 5.625 k deg), 6000 Adam steps of 2^15"}}
    # batches of 8 views (azimuth 45 k deg): plain FP32 and the fast form
    cams8 = S.orbit_cameras(cfg, 8)
    n8 = 8 * n
    out8 = {"rgb": torch.empty(n8, 3, device=dev), "depth": torch.empty(n8, device=dev),
            "opacity": torch.empty(n8, device=dev)}
    ms8 = _timed(lambda: rend32.render(opts, cams=cams8, W=cfg.W, H=cfg.H, out=out8), stream, flush, 3, 2)
    rgb8 = torch.empty(n8, 3, device=dev)
    fr8 = P.FastRenderer(ds16, docc, w, pc, device=dev)
    ms8f = _timed(lambda: fr8.render(opts, cams8, cfg.W, cfg.H, rgb8, stream=stream), stream, flush, 3, 2)
    psnr8 = [P.psnr(rgb8[k * n:(k + 1) * n], out8["rgb"][k * n:(k + 1) * n]) for k in range(8)]
    res["batch8"] = {"plain_fp32_frames_per_s": 8000.0 / ms8, "fast_frames_per_s": 8000.0 / ms8f,
                     "fast_psnr_vs_plain_db_per_view": psnr8}
    del out8, rgb8, fr8
    # one training step: 2^18 random rays of 8 views, L2 loss against the plain
    # render of a perturbed scene, reverse pass, Adam over all parameters
    tgt = rend32.render(opts, cams=cams8, W=cfg.W, H=cfg.H)["rgb"]
    student_t = ds.tables + 0.02 * torch.randn_like(ds.tables)
    dss = ng.DeviceScene(cfg, student_t.cpu().numpy(), scene.coarse, scene.mlp_w, device=dev)
    from paper_2407_10482_gb300 import train_step as TS
    pix8 = torch.as_tensor(S.random_pixels(1 << 18, 8, cfg.W, cfg.H, 3)).to(dev)
    tg = tgt[pix8.long()].contiguous()
    train_step, _ = TS.make_step(cfg, dss, docc, cams8, tg, pix8, stream=stream)
    ms_train = _timed(train_step, stream, flush, 5, 3)
    res["train_step"] = {"rays": 1 << 18, "ms": ms_train, "rays_per_s": (1 << 18) / ms_train * 1e3,
                         "parts": "render (with state, rays in pixel-tile order) + L2 loss + reverse pass (rays in drawn "
                                  "order) + Adam on 50.5M table, grid and MLP parameters"}
    del dss
    # gather ceiling: random whole-entry gathers at three footprints, FP32 with and
    # without L1 allocation (the march reads its large levels without it)
    sink = torch.zeros(1, device=dev)
    gcl = {}
    for name, dt, rows, flags in (("l1_resident_f32", 0, 1 << 11, 0), ("l1_resident_f16", 1, 1 << 12, 0),
                                  ("l2_resident_f32", 0, 1 << 20, 0), ("l2_resident_f32_noalloc", 0, 1 << 20, 1),
                                  ("l2_resident_f16", 1, 1 << 21, 0),
                                  ("hd_footprint_f32", 0, 1 << 23, 0), ("hd_footprint_f32_noalloc", 0, 1 << 23, 1)):
        tab = torch.rand(rows, 8, device=dev, dtype=torch.float32 if dt == 0 else torch.float16)
        nthr, per = 152 * 2048, 256

        def g():
            ng.ngprt_gather_bench(tab, dt, rows, nthr, per, 7, sink, stream=stream, flags=flags)
        ms_g = _timed(g, stream, flush, 5, 2)
        gcl[name + "_GBps"] = nthr * per * (32 if dt == 0 else 16) / (ms_g * 1e-3) / 1e9
        del tab
    res["gather_ceiling"] = gcl
    if not args.no_paper_shape:
        res["paper_shape"] = paper_shape(args, dev, stream, flush)
        res["aggregation_ablation"] = aggregation_ablation(args, dev, stream, flush)
    return res


AGG_NAMES = {0: "Separate-Att (V)", 1: "Shared-Att (V)", 2: "Separate-Att (Inv)", 3: "Shared-Att (Inv)", 4: "SUM",
             5: "MLP"}


def aggregation_ablation(args, dev, stream, flush):
    """Table 3's aggregation methods on the paper-shaped L = 4 scene (T = 2^22, 512^3
    coarse grid in each method's own layout), 1080p FP32 frames; per method the frame
    time, samples per ray and the multiply-adds that fuse the levels per sample.  The
    paper's times (RTX 3090, L = 4): MLP 68.02, SUM 14.94, Shared-Att (Inv) 15.18,
    Separate-Att (Inv) 15.13, Shared-Att (V) 16.04, Separate-Att (V) 16.17 ms."""
    import torch
    from paper_2407_10482_gb300 import ngprt as ng
    out = {}
    L = 4
    occ = None
    for agg in (0, 1, 2, 3, 4, 5):
        cfg = S.paper_config(L, aggregation=agg)
        sc = S.make_scene_torch(cfg, device=dev)
        if occ is None:
            occ = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels, device=dev, dist_level=cfg.dist_level)
        ds = ng.DeviceScene(cfg, sc.tables, sc.coarse, sc.mlp_w, device=dev, attn_inv=sc.attn_inv, agg_mlp=sc.agg_mlp)
        rend = ng.Renderer(ds, occ, device=dev)
        opts = S.default_options(cfg)
        cams = S.orbit_cameras(cfg, 1)
        o = rend.render(opts, cams=cams, W=cfg.W, H=cfg.H, stats=True)
        st = o["stats"].float().mean(0)
        ms = _timed(lambda: rend.render(opts, cams=cams, W=cfg.W, H=cfg.H, out=o), stream, flush, 5, 3)
        macs = {5: S.AGG_HIDDEN * 8 * L + 8 * S.AGG_HIDDEN, 4: 0}.get(agg, 8 * L)
        out[AGG_NAMES[agg]] = {"ms_per_frame": ms, "frames_per_s": 1000.0 / ms, "samples_per_ray": float(st[1]),
                               "marching_per_ray": float(st[0]), "fusion_macs_per_sample": macs,
                               "coarse_channels": S.coarse_channels(cfg)}
        del sc, ds, rend, o
        torch.cuda.empty_cache()
    out["config"] = "paper shape L = 4 (N_l = 1024 * 2^l, T = 2^22, R_C = 512, R_O = 512, G at 256^3), FP32, 1080p, hd scene"
    return out


def paper_shape(args, dev, stream, flush):
    """The paper's render-time shape (L = 2, 3, 4 fine levels at 1024 * 2^l, T = 2^22,
    512^3 coarse grid, 512^3 occupancy with 5 levels; Tables 2 and 4) on the hd scene:
    1080p frames/s in FP32 and FP16, and marching / occupied points per ray with and
    without G.  The paper's numbers (RTX 3090, Mip-NeRF 360): 108 / 79.7 / 61.8 fps."""
    import torch
    from paper_2407_10482_gb300 import ngprt as ng
    out = {}
    for L in (2, 3, 4):
        cfg = S.paper_config(L)
        sc = S.make_scene_torch(cfg, device=dev)
        docc = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels, device=dev, dist_level=cfg.dist_level)
        opts = S.default_options(cfg)
        cams = S.orbit_cameras(cfg, 1)
        n = cfg.W * cfg.H
        row = {}
        for dt in (0, 1):
            ds = ng.DeviceScene(cfg, sc.tables, sc.coarse, sc.mlp_w, table_dtype=dt, mlp_dtype=dt, device=dev)
            rend = ng.Renderer(ds, docc, device=dev)
            o = rend.render(opts, cams=cams, W=cfg.W, H=cfg.H, stats=True)
            ms = _timed(lambda: rend.render(opts, cams=cams, W=cfg.W, H=cfg.H, out=o), stream, flush, 5, 3)
            key = "fp32" if dt == 0 else "fp16_tc"
            row[key] = {"ms_per_frame": ms, "frames_per_s": 1000.0 / ms}
            ref_rgb = o["rgb"].clone()
            # the same frame through the block-sparse coarse grid (identical pixels)
            ds.sparsify_coarse(docc)
            o_s = rend.render(opts, cams=cams, W=cfg.W, H=cfg.H)
            ms_s = _timed(lambda: rend.render(opts, cams=cams, W=cfg.W, H=cfg.H, out=o_s), stream, flush, 5, 3)
            row[key + "_sparse_coarse"] = {"ms_per_frame": ms_s, "frames_per_s": 1000.0 / ms_s,
                                           "blocks": ds.coarse_blocks,
                                           "grid_bytes": ds.coarse.numel() * ds.coarse.element_size(),
                                           "identical_to_dense": bool(torch.equal(o_s["rgb"], ref_rgb))}
            del o_s, ref_rgb
            if dt == 0:
                st = o["stats"].float().mean(0)
                st0 = rend.render(opts, cams=cams, W=cfg.W, H=cfg.H, stats=True, use_dist=False)["stats"].float().mean(0)
                row["marching_per_ray"] = {"with_G": float(st[0]), "without_G": float(st0[0])}
                row["occupied_per_ray"] = {"with_G": float(st[1]), "without_G": float(st0[1])}
            del ds, rend, o
        out[f"L{L}"] = row
        del sc, docc
        torch.cuda.empty_cache()
    out["config"] = ("N_l = 1024 * 2^l, T = 2^22, R_C = 512 dense (8 + 2L channels; *_sparse_coarse: 8^3-cell "
                     "blocks of 9^3 vertices reached by the occupancy), R_O = 512 (5 levels), G at 256^3")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-stride", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--table-dtype", type=int, default=0, help="0 F32, 1 F16, 2 BF16 (plain form: 0)")
    ap.add_argument("--mlp-dtype", type=int, default=0, help="0 F32 (CUDA cores), 1 F16 (tensor cores)")
    ap.add_argument("--engine", default="fused", choices=["wavefront", "fused"])
    ap.add_argument("--plain-only", action="store_true", help="time only the plain FP32 frame")
    ap.add_argument("--no-paper-shape", action="store_true", help="skip the paper-shaped L = 2, 3, 4 frames")
    ap.add_argument("--workload", default="hd", choices=["hd", "paper2", "paper3", "paper4"],
                    help="the timed frame: the hd scene, or the paper-shaped scene with L = 2, 3 or 4 "
                         "(those run the plain frame only, without the CPU baseline)")
    ap.add_argument("--coarse-res", type=int, default=512, help="coarse-grid resolution of the paper-shaped scenes")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist
    from paper_2407_10482_gb300 import ngprt as ng

    world, rank, local = _dist_setup()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ng.lib()

    if args.workload == "hd":
        cfg = S.hd_config()
        scene = S.make_scene(cfg)
    else:
        # the paper-shaped scenes are drawn on the GPU (their grids are too large for numpy)
        cfg = S.paper_config(int(args.workload[-1]), R_C=args.coarse_res)
        scene = S.make_scene_torch(cfg, device=dev)
    cams = S.orbit_cameras(cfg, 1, azimuth0=rank_views(rank)[0])
    opts = S.default_options(cfg)
    ds = ng.DeviceScene(cfg, scene.tables, scene.coarse, scene.mlp_w, table_dtype=args.table_dtype, device=dev,
                        mlp_dtype=args.mlp_dtype)
    docc = ng.DeviceOcc(scene.occ, cfg.R_O, cfg.n_occ_levels, device=dev, dist_level=cfg.dist_level)
    rend = ng.Renderer(ds, docc, device=dev)
    n = cfg.W * cfg.H
    cam_arr, n_cams = ng.cameras_struct(cams, cfg.W, cfg.H)
    ro = ng.render_opts(opts)
    state = torch.empty(n, ng.STATE_FLOATS, device=dev)
    rgb = torch.empty(n, 3, device=dev)
    depth = torch.empty(n, device=dev)
    opac = torch.empty(n, device=dev)
    stream = torch.cuda.current_stream(dev)

    ws = torch.empty(ng.ngprt_wavefront_workspace_bytes(ds.struct, n), dtype=torch.uint8, device=dev)

    main_ws = ws if args.engine == "wavefront" else None

    def march(workspace=main_ws):
        # wavefront engine (advance / gather rounds) when given the workspace
        ng.ngprt_render(ds.struct, docc.struct, cam_arr, n_cams, None, None, None, n, None, ro, None,
                        ray_state=state, workspace=workspace, stream=stream)

    def shade():
        ng.ngprt_shade(ds.struct, state, n, opts.bg, rgb, depth, opac, stream=stream)

    # unit counts (samples, marching points) of this frame, with and without G
    st = rend.render(opts, cams=cams, W=cfg.W, H=cfg.H, stats=True)["stats"].float()
    samples = float(st[:, 1].sum())
    marching = float(st[:, 0].sum())
    st_nog = rend.render(opts, cams=cams, W=cfg.W, H=cfg.H, stats=True, use_dist=False)["stats"].float()
    optsmax = S.default_options(cfg, dist_rule=1)
    st_max = rend.render(optsmax, cams=cams, W=cfg.W, H=cfg.H, stats=True)["stats"].float()
    march_stats = {
        "marching_per_ray": marching / n, "samples_per_ray": samples / n,
        "without_G": {"marching_per_ray": float(st_nog[:, 0].sum()) / n,
                      "samples_per_ray": float(st_nog[:, 1].sum()) / n},
        "G_max_rule": {"marching_per_ray": float(st_max[:, 0].sum()) / n,
                       "samples_per_ray": float(st_max[:, 1].sum()) / n}}

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        march()
        shade()
    torch.cuda.synchronize(dev)

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        march()
        ev[k][1].record(stream)
        shade()
        ev[k][2].record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    t_march = [ev[k][0].elapsed_time(ev[k][1]) for k in range(args.steps)]
    t_shade = [ev[k][1].elapsed_time(ev[k][2]) for k in range(args.steps)]
    ms = statistics.mean(a + b for a, b in zip(t_march, t_shade))
    ms_max = max_over_ranks(ms, world, dev)
    fps = world * 1000.0 / ms_max

    # the single fused march kernel on the same frame, for comparison
    fused = []
    for k in range(args.warmup + 5):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        march(None)
        e1.record(stream)
        e1.synchronize()
        if k >= args.warmup:
            fused.append(e0.elapsed_time(e1))

    # end to end through the public call with host buffers: camera in, image out
    host = {"rgb": torch.empty(n, 3, pin_memory=True), "depth": torch.empty(n, pin_memory=True),
            "opacity": torch.empty(n, pin_memory=True)}
    d2h = n * 5 * 4
    h2d = 72 * n_cams
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cam_arr_k, _ = ng.cameras_struct(cams, cfg.W, cfg.H)
        ng.ngprt_render(ds.struct, docc.struct, cam_arr_k, n_cams, None, None, None, n, None, ro, rgb, depth, opac,
                        None, state, main_ws, stream=stream)
        host["rgb"].copy_(rgb, non_blocking=True)
        host["depth"].copy_(depth, non_blocking=True)
        host["opacity"].copy_(opac, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if k >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_fps = world * 1000.0 / max_over_ranks(statistics.mean(e2e_ms), world, dev)

    # ---------------------------------------------------------------- other forms
    extra = {}
    hd = args.workload == "hd"
    if not args.plain_only and hd:
        extra = other_forms(args, cfg, scene, ds, docc, cams, opts, dev, stream, flush, rgb)
    workload = WORKLOAD if hd else (f"paper-shaped 1920x1080 scene, L={cfg.L} (N_l = 1024*2^l), T=2^22, "
                                    f"{cfg.R_C}^3 dense coarse grid, 512^3 occupancy (5 levels), G at 256^3, "
                                    f"MLP 23-64-64-3")
    measured_here = hd and args.table_dtype == 0 and args.engine == "fused"

    peaks = _peaks()
    L = cfg.L
    entry_b = 32 if args.table_dtype == 0 else 16
    ch_b = 4 if args.table_dtype == 0 else 2
    bytes_per_sample = L * 8 * entry_b + 8 * S.coarse_channels(cfg) * ch_b
    alg_bytes = samples * bytes_per_sample + marching * 2 + n * ng.STATE_FLOATS * 4
    t_march_avg = statistics.mean(t_march)
    achieved = alg_bytes / (t_march_avg * 1e-3) / 1e9

    line = {
        "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {0: "f32", 1: "f16", 2: "bf16"}[args.table_dtype], "data": "synthetic",
        "config": {"workload": workload, "views_per_step": 1, "rays_per_step": n, "l2_flush": True,
                   "parallelism": f"replicas x{world}", "table_dtype": args.table_dtype},
        "grays_per_s": fps * n / 1e9,
        "kernels_ms": {"march": t_march_avg, "shade_mlp": statistics.mean(t_shade),
                       "march_fused_engine": statistics.mean(fused), "engine": args.engine},
        "march_stats": march_stats,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"],
                     "traffic": MARCH_DRAM_BYTES if measured_here else None,
                     "traffic_unit": "bytes per launch (ncu dram__bytes_read + write)",
                     "kernel": f"march_kernel<{L},{['F32', 'F16', 'BF16'][args.table_dtype]}> (fused march: occupancy, "
                               f"coarse fetch, {L}-level gathers, attention, compositing)",
                     "peak_source": peaks["source"],
                     "bytes_per_sample": bytes_per_sample,
                     "note": "algorithmic gather bytes (L*8 entries + 8 coarse vertices per sample, 2 B per "
                             "marching point, 48 B state per ray) over the march kernel's event time; they are "
                             "served by L1/L2 (DRAM traffic is the 'traffic' figure), and lanes of a pixel tile "
                             "share the coarse levels' entries, so they also exceed the per-lane random-gather "
                             "microbenchmark; the bound is the L1 load pipe (l1_lsu_pct_ncu)",
                     "l1_lsu_pct_ncu": L1_LSU_PCT if measured_here else None},
        "e2e": {"value": e2e_fps, "unit": "frames/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": (2 if args.engine == "fused" else 2 * 8 + 3) * args.steps,
        "clocks": clk,
        "wall_s": wall,
    }
    line.update(extra)
    if "gather_ceiling" in extra:
        gc = extra["gather_ceiling"]
        # the best random-gather rate the microbenchmark reaches in any of the access
        # modes the march uses (L1-resident with allocation, L2-resident without)
        if args.table_dtype == 0:
            ceil = max(gc["l1_resident_f32_GBps"], gc["l2_resident_f32_noalloc_GBps"])
        else:
            ceil = max(gc["l1_resident_f16_GBps"], gc["l2_resident_f16_GBps"])
        line["roofline"]["gather_ceiling_GBps"] = ceil
        line["roofline"]["gather_frac"] = achieved / ceil
    if rank == 0 and world == 1 and not args.no_cpu_baseline and hd:
        line["cpu_baseline"] = cpu_baseline(cfg, scene, cams, opts)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
