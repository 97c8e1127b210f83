"""Benchmark of the NGP-RT render path on GB300: 1080p frames/s and Grays/s.

``python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]``

Headline workload: the hd model (L=16 levels 16..4096, T=2^19, 16^3 coarse grid of
40 channels, 128^3 occupancy + distance grid G, MLP 23->64->64->3) fitted in this
run to ground-truth images of its synthetic unbounded 360-style scene
(``hdfit.fit_hd_scene``: 48 training views, Huber loss + distortion regulariser,
visibility-culled occupancy), rendered at 1920x1080 from a held-out orbit view.
One step = one frame of the plain FP32 renderer: the fused march kernel
(occupancy-distance marching, coarse fetch, 16-level gathers, attention,
compositing) and the deferred-MLP kernel.  Inputs are resident in HBM; L2 is
flushed (a 256 MiB write) between timed frames, outside the timed events.  Under
torchrun every rank fits its own replica and renders its own view (weak scaling,
no data-path collective); rank 0 prints one JSON line.

Beside it: the FP16 + tensor-core MLP + learned-proposal form with the PSNR of both
forms against the held-out targets (the <= 0.1 dB criterion), batches of 8 views,
one training step, the random-weight hd scene, the paper-shaped scenes (Tables 2-4),
the L1-pipe roofline of the march kernel, and the CPU oracle's rate.

``--impl reference`` times the CPU oracle (the plain FP64 program of the same
computation) on a bounded pixel sample per step, on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2407_10482_gb300 import scenes as S  # noqa: E402

METRIC = "1080p frames/s & Grays/s, plain FP32 vs FP16+proposal at ≤0.1 dB PSNR loss"
WORKLOAD = ("hd fitted scene 1920x1080 (unbounded 360-style, L=16 levels 16..4096, T=2^19, 16^3x40 coarse, "
            "128^3 occupancy+G, MLP 23-64-64-3), fitted in-run to 48 analytic views, held-out view")
RANDOM_WORKLOAD = ("hd random-weight scene 1920x1080 (same model shape, tables N(0, 0.1), coarse density offset "
                   "3.2), orbit view at azimuth 0")
COUNTERS = os.path.join(ROOT, "profiles", "march_kernel_counters.json")
# sources the march kernel is compiled from: counters taken on other sources are stale
KERNEL_SOURCES = ("paper_2407_10482_gb300/csrc/common.cuh", "paper_2407_10482_gb300/csrc/march.cuh",
                  "paper_2407_10482_gb300/csrc/render.cu")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def load_counters(key: str):
    """The committed ncu counters of the march kernel for workload `key`, or None
    when they are missing or were taken on other kernel sources."""
    try:
        with open(COUNTERS) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(key)
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return e


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


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    """The CPU oracle on the random-weight hd scene (the fitted model's shape; the
    oracle takes only seeded generator inputs), every step a 1/ref_stride pixel
    sample of one frame on all host cores; value = frames/s of that rate."""
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
            steps.append(dt)
    ms = 1000.0 * statistics.mean(steps)                 # one step = 1/stride of a frame
    value = 1000.0 / (ms * stride)                       # frames/s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": RANDOM_WORKLOAD, "step": f"1/{stride} of the frame's pixels (every "
                       f"{stride}th pixel, offset by the step index)", "rays_per_step": n // stride},
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": O.max_threads(), "kind": "oracle",
                             "sample": f"every {stride}th pixel of the frame per step"},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- helpers

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


def _psnr(a, b) -> float:
    mse = float(((a.double() - b.double()) ** 2).mean())
    return float("inf") if mse == 0 else -10.0 * math.log10(mse)


def _views(render_one, cams, W, H, dev):
    """rgb [V*H*W, 3] of render_one(cams[v:v+1], out) over the views."""
    import torch
    n = W * H
    out = torch.empty(len(cams) * n, 3, device=dev)
    for v in range(len(cams)):
        render_one(cams[v:v + 1], out[v * n:(v + 1) * n])
    return out


# ------------------------------------------------------------- fitted forms

def fitted_forms(args, fs, opts, dev, stream, flush):
    """On the fitted scene: the plain FP32 renderer, FP16 tables + tensor-core MLP,
    and that form with the learned proposal; PSNR of each against the held-out
    targets (8 views) and the loss of the fast form; batches of 8 views; one
    training step against the analytic targets."""
    import torch
    from paper_2407_10482_gb300 import ngprt as ng
    from paper_2407_10482_gb300 import proposal as P
    cfg = fs.cfg
    W, H = cfg.W, cfg.H
    n = W * H
    reps, warm = max(3, args.steps // 2), args.warmup
    res = {}
    ds = fs.scene
    rend = ng.Renderer(ds, fs.occ, device=dev)

    def plain_one(c, out):
        out.copy_(rend.render(opts, cams=c, W=W, H=H)["rgb"])
    rgb_plain = _views(plain_one, fs.cams_test, W, H, dev)
    # FP16 tables, FP16 tensor-core MLP
    ds16 = ng.DeviceScene(cfg, ds.tables, ds.coarse, ds.mlp_w, table_dtype=ng.F16, mlp_dtype=ng.F16, device=dev)
    r16 = ng.Renderer(ds16, fs.occ, device=dev)

    def f16_one(c, out):
        out.copy_(r16.render(opts, cams=c, W=W, H=H)["rgb"])
    rgb16 = _views(f16_one, fs.cams_test, W, H, dev)
    # BF16 tables with the same tensor-core MLP
    dsb = ng.DeviceScene(cfg, ds.tables, ds.coarse, ds.mlp_w, table_dtype=ng.BF16, mlp_dtype=ng.F16, device=dev)
    rb = ng.Renderer(dsb, fs.occ, device=dev)
    rgbb = _views(lambda c, out: out.copy_(rb.render(opts, cams=c, W=W, H=H)["rgb"]), fs.cams_test, W, H, dev)
    ob = rb.render(opts, cams=fs.cams_test[:1], W=W, H=H)
    ms_b = _timed(lambda: rb.render(opts, cams=fs.cams_test[:1], W=W, H=H, out=ob), stream, flush, reps, warm)
    del rb, ob
    c1 = fs.cams_test[:1]
    o16 = r16.render(opts, cams=c1, W=W, H=H, stats=True)
    samples16 = float(o16["stats"][:, 1].float().sum())
    ms_16 = _timed(lambda: r16.render(opts, cams=c1, W=W, H=H, out=o16), stream, flush, reps, warm)
    # the FP16 march kernel alone: bound by the L1 data pipe (one wavefront per SM
    # cycle), with instruction issue (4 warp instructions per SM cycle) the next
    # limit; wavefronts and warp instructions per occupied sample from the committed
    # ncu counters of this kernel source on this workload
    cam1, nc1 = ng.cameras_struct(c1, W, H)
    st16 = torch.empty(n, ng.STATE_FLOATS, device=dev)
    ws16 = torch.empty(ng.ngprt_render_workspace_bytes(ds16.struct, n), dtype=torch.uint8, device=dev)
    ro = ng.render_opts(opts)
    ms_m16 = _timed(lambda: ng.ngprt_render(ds16.struct, fs.occ.struct, cam1, nc1, None, None, None, n, None, ro, None,
                                            ray_state=st16, workspace=ws16, stream=stream), stream, flush, reps, warm)
    cnt16 = load_counters("hd_fit_1080p_fp16")
    roof16 = {"bound": "l1", "unit": "Gwavefronts/s", "kernel": "march_kernel<16,F16>",
              "march_ms": ms_m16, "source_hash": kernel_source_hash()}
    if cnt16:
        ach = cnt16["l1_wavefronts_per_sample"] * samples16 / (ms_m16 * 1e-3) / 1e9
        pk = cnt16["l1_wavefronts_peak_per_cycle_per_sm"] * cnt16["sms"] * args.clock_hz / 1e9
        iss = cnt16["warp_instructions_per_sample"] * samples16 / (ms_m16 * 1e-3) / 1e9
        roof16.update(achieved=ach, peak=pk, frac=ach / pk,
                      issue={"achieved_G_warp_inst_per_s": iss, "peak": 4 * 152 * args.clock_hz / 1e9,
                             "frac": iss / (4 * 152 * args.clock_hz / 1e9)},
                      traffic=cnt16["dram_bytes_per_sample"] * samples16)
    else:
        roof16.update(achieved=None, peak=None, frac=None, note="no ncu counters for this kernel source")
    # learned proposal: trained on the plain renderer's weights over 64 orbit views
    # between the held-out ones, every step in the library's kernels
    t0 = time.perf_counter()
    train_cams = S.orbit_cameras(cfg, 64, azimuth0=2.8125, step_deg=5.625)
    pix = torch.as_tensor(S.random_pixels(1 << 20, 64, W, H, 4)).to(dev)
    targets = P.make_targets(rend, opts, train_cams, W, H, pix)
    pc = P.ProposalConfig()
    w, hist = P.train(train_cams, W, H, pix, targets, pc, log_every=2000)
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0
    fr = P.FastRenderer(ds16, fs.occ, w, pc, device=dev)
    stats_fast, stats_plain = [], []

    def fast_one(c, out):
        fr.render(opts, c, W, H, out, stats=True)
        stats_fast.append(fr.stats.float().mean(0))
    rgb_fast = _views(fast_one, fs.cams_test, W, H, dev)
    for v in range(len(fs.cams_test)):
        stats_plain.append(rend.render(opts, cams=fs.cams_test[v:v + 1], W=W, H=H, stats=True)["stats"].float()
                           .mean(0))
    sf, sp = torch.stack(stats_fast).mean(0), torch.stack(stats_plain).mean(0)
    ob = torch.empty(n, 3, device=dev)
    ms_fast = _timed(lambda: fr.render(opts, c1, W, H, ob, stream=stream), stream, flush, reps, warm)
    tg = fs.targets_test
    p_plain, p16, p_fast = _psnr(rgb_plain, tg), _psnr(rgb16, tg), _psnr(rgb_fast, tg)

    def per_view(rgb):
        return [_psnr(rgb[k * n:(k + 1) * n], tg[k * n:(k + 1) * n]) for k in range(len(fs.cams_test))]
    loss = p_plain - p_fast
    vs_plain = _psnr(rgb_fast, rgb_plain)
    res["forms"] = {
        "held_out_views": "8 views, orbit radius 3, elevation 20 deg, azimuths 22.5 + 45 k (not trained on)",
        "plain_fp32": {"psnr_vs_targets_db": p_plain, "psnr_vs_targets_db_per_view": per_view(rgb_plain),
                       "marching_per_ray": float(sp[0]), "samples_per_ray": float(sp[1])},
        "fp16_tables_tc_mlp": {"ms_per_frame": ms_16, "frames_per_s": 1000.0 / ms_16,
                               "psnr_vs_targets_db": p16, "psnr_loss_vs_targets_db": p_plain - p16,
                               "psnr_vs_plain_db": _psnr(rgb16, rgb_plain), "roofline_march": roof16},
        "bf16_tables_tc_mlp": {"ms_per_frame": ms_b, "frames_per_s": 1000.0 / ms_b,
                               "psnr_vs_targets_db": _psnr(rgbb, tg), "psnr_loss_vs_targets_db": p_plain - _psnr(rgbb, tg),
                               "psnr_vs_plain_db": _psnr(rgbb, rgb_plain)},
        "fp16_tc_mlp_proposal": {
            "ms_per_frame": ms_fast, "frames_per_s": 1000.0 / ms_fast, "grays_per_s": n / ms_fast / 1e6,
            "psnr_vs_targets_db": p_fast, "psnr_vs_targets_db_per_view": per_view(rgb_fast),
            "psnr_loss_vs_targets_db": loss, "loss_criterion_db": 0.1, "meets_0p1dB_vs_targets": bool(loss <= 0.1),
            "psnr_vs_plain_db": vs_plain, "vs_plain_threshold_db": 41.9,
            "meets_41p9dB_vs_plain": bool(vs_plain >= 41.9),
            "marching_per_ray": float(sf[0]), "samples_per_ray": float(sf[1]),
            "fallback_rays": float(((fr.a_hat - fr.state[:, 7]) > pc.fallback).float().mean()),
            "margin_near": pc.margin_near, "margin_far": pc.margin_far,
            "proposal_train_s": train_s, "proposal_loss": hist,
            "training": "2^20 rays of 64 orbit views (azimuth 2.8125 + 5.625 k deg), 6000 Adam steps of 2^15"}}
    # batches of the 8 held-out views: plain FP32 and the fast form
    cams8 = fs.cams_test
    n8 = len(cams8) * n
    out8 = {"rgb": torch.empty(n8, 3, device=dev), "depth": torch.empty(n8, device=dev),
            "opacity": torch.empty(n8, device=dev)}
    rend8 = ng.Renderer(ds, fs.occ, device=dev)
    ms8 = _timed(lambda: rend8.render(opts, cams=cams8, W=W, H=H, out=out8), stream, flush, 3, 2)
    rgb8 = torch.empty(n8, 3, device=dev)
    fr8 = P.FastRenderer(ds16, fs.occ, w, pc, device=dev)
    ms8f = _timed(lambda: fr8.render(opts, cams8, W, H, rgb8, stream=stream), stream, flush, 3, 2)
    res["batch8"] = {"plain_fp32_frames_per_s": 8000.0 / ms8, "fast_frames_per_s": 8000.0 / ms8f}
    del out8, rgb8, fr8, rend8, ds16, r16, o16
    # one training step (2^18 random rays of the 8 held-out 1080p analytic targets,
    # L2 loss, reverse pass, Adam over every parameter) on a copy of the fitted scene
    from paper_2407_10482_gb300 import train_step as TS
    dss = ng.DeviceScene(cfg, ds.tables.clone(), ds.coarse.clone(), ds.mlp_w.clone(), device=dev)
    pix8 = torch.as_tensor(S.random_pixels(1 << 18, len(cams8), W, H, 3)).to(dev)
    tg8 = tg[pix8.long()].contiguous()
    train_step, _ = TS.make_step(cfg, dss, fs.occ, cams8, tg8, pix8, stream=stream)
    ms_train = _timed(train_step, stream, flush, 5, 3)
    res["train_step"] = {"rays": 1 << 18, "ms": ms_train, "rays_per_s": (1 << 18) / ms_train * 1e3,
                         "targets": "analytic ground truth of the 8 held-out 1080p views",
                         "parts": "render (with state, rays in pixel-tile order) + L2 loss + reverse pass (rays in "
                                  "drawn order) + Adam on 50.5M table, grid and MLP parameters"}
    del dss
    torch.cuda.empty_cache()
    return res


# ------------------------------------------------------- random-weight scene

def random_scene(args, dev, stream, flush):
    """The random-weight hd scene (the model's stress case, no fit): plain FP32 and
    FP16 + tensor-core MLP frames, and Table 4's counts with and without G."""
    import torch
    from paper_2407_10482_gb300 import ngprt as ng
    cfg = S.hd_config()
    sc = S.make_scene(cfg)
    cams = S.orbit_cameras(cfg, 1)
    opts = S.default_options(cfg)
    docc = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels, device=dev)
    out = {"workload": RANDOM_WORKLOAD}
    for dt, key in ((ng.F32, "fp32"), (ng.F16, "fp16_tc"), (ng.BF16, "bf16_tc")):
        ds = ng.DeviceScene(cfg, sc.tables, sc.coarse, sc.mlp_w, table_dtype=dt,
                            mlp_dtype=ng.F32 if dt == ng.F32 else ng.F16, device=dev)
        rend = ng.Renderer(ds, docc, device=dev)
        o = rend.render(opts, cams=cams, W=cfg.W, H=cfg.H)
        ms = _timed(lambda: rend.render(opts, cams=cams, W=cfg.W, H=cfg.H, out=o), stream, flush, 5, 3)
        out[key] = {"ms_per_frame": ms, "frames_per_s": 1000.0 / ms}
        if dt == ng.F32:
            n = cfg.W * cfg.H
            st = {}
            for name, kw in (("with_G", {}), ("without_G", {"use_dist": False}), ("G_eq9_literal", {"dist_rule": 0})):
                s = rend.render(S.default_options(cfg, **kw), cams=cams, W=cfg.W, H=cfg.H, stats=True,
                                use_dist=kw.get("use_dist", True))["stats"].float()
                st[name] = {"marching_per_ray": float(s[:, 0].sum()) / n, "samples_per_ray": float(s[:, 1].sum()) / n}
            out["march_stats"] = st
        del ds, rend, o
    torch.cuda.empty_cache()
    return out


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
                st = {}
                for name, kw in (("with_G", {}), ("without_G", {"use_dist": False}),
                                 ("G_eq9_literal", {"dist_rule": 0})):
                    s = rend.render(S.default_options(cfg, **kw), cams=cams, W=cfg.W, H=cfg.H, stats=True,
                                    use_dist=kw.get("use_dist", True))["stats"].float().mean(0)
                    st[name] = {"marching_per_ray": float(s[0]), "occupied_per_ray": float(s[1])}
                row["march_stats"] = st
            del ds, rend, o
        out[f"L{L}"] = row
        del sc, docc
        torch.cuda.empty_cache()
    out["config"] = ("N_l = 1024 * 2^l, T = 2^22, R_C = 512 dense (8 + 2L channels; *_sparse_coarse: 8^3-cell "
                     "blocks of 9^3 vertices reached by the occupancy), R_O = 512 (5 levels), G at 256^3")
    return out


# --------------------------------------------------------------- CPU oracle leg

def cpu_leg(dev, sample_stride: int = 16, one_core_stride: int = 512, n_precision_pixels: int = 2000):
    """The FP64 oracle on the host cores (the timed CPU baseline) and, from the same
    oracle, the error of each precision form against it (8 orbit views of the
    random-weight hd scene, azimuths 45 k).  The oracle sees only the seeded
    generator's inputs."""
    import torch
    from oracle import oracle as O
    from paper_2407_10482_gb300 import ngprt as ng
    cfg = S.hd_config()
    sc = S.make_scene(cfg)
    opts = S.default_options(cfg)
    orc = O.oracle_for_scene(sc)
    n = cfg.W * cfg.H
    cams1 = S.orbit_cameras(cfg, 1)
    pix = np.arange(0, n, sample_stride, dtype=np.int32)
    t0 = time.perf_counter()
    orc.render(opts, cams=cams1, pix=pix)
    dt_all = time.perf_counter() - t0
    threads = O.max_threads()
    O.set_threads(1)
    pix1 = np.arange(0, n, one_core_stride, dtype=np.int32)
    t0 = time.perf_counter()
    orc.render(opts, cams=cams1, pix=pix1)
    dt_one = time.perf_counter() - t0
    O.set_threads(threads)
    base = {"value": len(pix) / dt_all / n, "unit": "frames/s", "rays_per_s": len(pix) / dt_all, "cores": threads,
            "kind": "oracle", "seconds": dt_all,
            "sample": f"{len(pix)} pixels (every {sample_stride}th) of one 1920x1080 frame of the random-weight hd "
                      f"scene, FP64 oracle, OpenMP",
            "one_core": {"rays_per_s": len(pix1) / dt_one, "frames_per_s": len(pix1) / dt_one / n,
                         "sample": f"{len(pix1)} pixels (every {one_core_stride}th), 1 thread"}}
    # precision forms against the oracle, per view: on the FP32 master and on the
    # 16-bit values the kernel reads
    cams8 = S.orbit_cameras(cfg, 8)
    docc = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels, device=dev)
    rng = np.random.default_rng(19)
    prec = {"views": "8 orbit views, azimuth 45 k deg, 1920x1080; random-weight hd scene",
            "pixels_per_view": n_precision_pixels,
            "excluded": "rays the FP64 oracle flags as decidable either way in FP32 (its march decisions)"}
    master = {}
    for v in range(8):
        pv = rng.choice(n, n_precision_pixels, replace=False).astype(np.int32)
        r = orc.render(opts, cams=cams8[v:v + 1], pix=pv)
        ok = ~r["ambiguous"]          # rays whose march FP32 may decide otherwise
        master[v] = (pv[ok], r["rgb"][ok])
    for name, tdt in (("fp16", ng.F16), ("bf16", ng.BF16)):
        ds = ng.DeviceScene(cfg, sc.tables, sc.coarse, sc.mlp_w, table_dtype=tdt, mlp_dtype=ng.F16, device=dev)
        rend = ng.Renderer(ds, docc, device=dev)
        orq = O.Oracle(cfg, ds.tables.float().cpu().numpy(), ds.coarse.float().cpu().numpy(),
                       ds.mlp_w.float().cpu().numpy(), O.build_pyramid(sc.occ, cfg.R_O, cfg.n_occ_levels),
                       O.occ_dist(sc.occ, cfg.R_O))
        rows = []
        for v in range(8):
            pv, ref_m = master[v]
            rgb = rend.render(opts, cams=cams8[v:v + 1], W=cfg.W, H=cfg.H)["rgb"][torch.as_tensor(pv).long().to(dev)]
            g = rgb.double().cpu().numpy()
            ref_r = orq.render(opts, cams=cams8[v:v + 1], pix=pv)["rgb"]
            e_m, e_r = np.abs(g - ref_m), np.abs(g - ref_r)
            rows.append({"max_abs_master": float(e_m.max()), "psnr_master_db": float(-10 * np.log10((e_m ** 2).mean())),
                         "max_abs_rounded": float(e_r.max()),
                         "psnr_rounded_db": float(-10 * np.log10((e_r ** 2).mean()))})
        prec[f"{name}_tables_fp16_tc_mlp"] = rows
        del ds, rend
    return base, prec


# ---------------------------------------------------------------------- main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-stride", type=int, default=64)
    ap.add_argument("--fit-steps", type=int, default=800, help="Adam steps of the in-run fit of the hd scene")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-only", action="store_true", help="time only the plain FP32 frame of the fitted scene")
    ap.add_argument("--no-paper-shape", action="store_true", help="skip the paper-shaped L = 2, 3, 4 frames")
    ap.add_argument("--save-scene", default="", help="write the fitted scene (tables, grid, MLP, occupancy) here")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist
    from paper_2407_10482_gb300 import hdfit as HF
    from paper_2407_10482_gb300 import ngprt as ng

    world, rank, local = _dist_setup()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ng.lib()
    stream = torch.cuda.current_stream(dev)

    # the headline scene: fitted in this run, in bounded time
    fs = HF.fit_hd_scene(S.hd_fit_config(), HF.HdFitConfig(steps=args.fit_steps), device=dev)
    if args.save_scene:
        from paper_2407_10482_gb300 import checkpoint as CK
        CK.save_scene(args.save_scene, S.Scene(cfg=fs.cfg, tables=fs.scene.tables, coarse=fs.scene.coarse,
                                                mlp_w=fs.scene.mlp_w, occ=fs.occ.occ))
    cfg = fs.cfg
    ds, docc = fs.scene, fs.occ
    opts = S.default_options(cfg)
    view = rank % len(fs.cams_test)
    cams = fs.cams_test[view:view + 1]
    n = cfg.W * cfg.H
    cam_arr, n_cams = ng.cameras_struct(cams, cfg.W, cfg.H)
    ro = ng.render_opts(opts)
    state = torch.empty(n, ng.STATE_FLOATS, device=dev)
    ws = torch.empty(ng.ngprt_render_workspace_bytes(ds.struct, n), dtype=torch.uint8, device=dev)
    rgb = torch.empty(n, 3, device=dev)
    depth = torch.empty(n, device=dev)
    opac = torch.empty(n, device=dev)

    def march():
        ng.ngprt_render(ds.struct, docc.struct, cam_arr, n_cams, None, None, None, n, None, ro, None,
                        ray_state=state, workspace=ws, stream=stream)

    def shade():
        ng.ngprt_shade(ds.struct, state, n, opts.bg, rgb, depth, opac, stream=stream)

    rend = ng.Renderer(ds, docc, device=dev)
    st = rend.render(opts, cams=cams, W=cfg.W, H=cfg.H, stats=True)["stats"].float()
    samples, marching = float(st[:, 1].sum()), float(st[:, 0].sum())
    march_stats = {"marching_per_ray": marching / n, "samples_per_ray": samples / n,
                   "marching_p99": float(st[:, 0].quantile(0.99)), "marching_max": float(st[:, 0].max())}
    for name, kw in (("without_G", {"use_dist": False}), ("G_eq9_literal", {"dist_rule": 0})):
        s = rend.render(S.default_options(cfg, **kw), cams=cams, W=cfg.W, H=cfg.H, stats=True,
                        use_dist=kw.get("use_dist", True))["stats"].float()
        march_stats[name] = {"marching_per_ray": float(s[:, 0].sum()) / n, "samples_per_ray": float(s[:, 1].sum()) / n}
    del rend

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
                        None, state, ws, stream=stream)
        host["rgb"].copy_(rgb, non_blocking=True)
        host["depth"].copy_(depth, non_blocking=True)
        host["opacity"].copy_(opac, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if k >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_fps = world * 1000.0 / max_over_ranks(statistics.mean(e2e_ms), world, dev)

    args.clock_hz = clock_hz = (clk.get("sm_mhz") or 2070.0) * 1e6
    # roofline of the march kernel: the L1 load pipe it runs at.  Wavefronts per
    # occupied sample come from the committed ncu counters of this kernel source on
    # this workload; times this frame's samples, over the kernel's event time,
    # against 152 SMs x the pipe's wavefronts per cycle x the sampled SM clock.  The
    # DRAM traffic of the same capture is reported against HBM beside it.
    peaks = _peaks()
    t_march_avg = statistics.mean(t_march)
    cnt = load_counters("hd_fit_1080p_fp32")
    roof = {"bound": "l1", "unit": "Gwavefronts/s",
            "kernel": "march_kernel<16,F32> (fused march: occupancy, coarse fetch, 16-level gathers, attention, "
                      "compositing)",
            "counters": os.path.relpath(COUNTERS, ROOT), "source_hash": kernel_source_hash()}
    if cnt:
        wf = cnt["l1_wavefronts_per_sample"] * samples
        peak = cnt["l1_wavefronts_peak_per_cycle_per_sm"] * cnt["sms"] * clock_hz / 1e9
        achieved = wf / (t_march_avg * 1e-3) / 1e9
        roof.update(achieved=achieved, peak=peak, frac=achieved / peak,
                    traffic=cnt["dram_bytes_per_sample"] * samples,
                    hbm={"achieved_GBps": cnt["dram_bytes_per_sample"] * samples / (t_march_avg * 1e-3) / 1e9,
                         "peak_GBps": peaks["hbm_gbs"], "peak_source": peaks["source"]},
                    note="L1 wavefronts per occupied sample (ncu, this kernel source, this workload) x this frame's "
                         "samples / the kernel's event time, against the L1 data pipe's peak wavefront rate at the "
                         "sampled SM clock; traffic = ncu DRAM bytes per sample x samples")
    else:
        roof.update(achieved=None, peak=None, frac=None, traffic=None,
                    note="no ncu counters for this kernel source and workload")

    line = {
        "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded analytic scene; model fitted in-run)",
        "config": {"workload": WORKLOAD, "views_per_step": 1, "rays_per_step": n, "l2_flush": True,
                   "parallelism": f"replicas x{world}", "fit": {k: v for k, v in fs.info.items() if k != "loss"},
                   "fit_loss": fs.info.get("loss")},
        "grays_per_s": fps * n / 1e9,
        "kernels_ms": {"march": t_march_avg, "shade_mlp": statistics.mean(t_shade)},
        "march_stats": march_stats,
        "roofline": roof,
        "e2e": {"value": e2e_fps, "unit": "frames/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": 2 * args.steps,
        "clocks": clk,
        "wall_s": wall,
    }
    if not args.plain_only:
        line.update(fitted_forms(args, fs, opts, dev, stream, flush))
        line["random_scene"] = random_scene(args, dev, stream, flush)
        if not args.no_paper_shape:
            line["paper_shape"] = paper_shape(args, dev, stream, flush)
            line["aggregation_ablation"] = aggregation_ablation(args, dev, stream, flush)
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"], line["precision_8view"] = cpu_leg(dev)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
