"""Render frames of a saved scene file through the library (and time them).

    python -m paper_2407_10482_gb300.render_scene SCENE_FILE [--frames 3] [--dtype f32|f16|bf16] [--view 0]

Loads a scene written by ``checkpoint.save_scene`` (for instance the fitted hd
scene of ``bench.py --save-scene``), builds its occupancy pyramid and distance grid,
and renders 1920x1080 frames of one held-out orbit view (``hdfit.test_cameras``):
the fused march kernel, then the deferred-MLP kernel (FP32 on CUDA cores, or FP16
or BF16 tables with the FP16 tensor-core MLP).  Prints the mean CUDA-event time per frame
and the marching points and samples per ray.  Used to profile a fitted scene's
frames on their own.
"""
from __future__ import annotations

import argparse
import statistics

import torch

from . import checkpoint as CK
from . import hdfit as HF
from . import ngprt as ng
from . import scenes as S


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("scene")
    ap.add_argument("--frames", type=int, default=3)
    ap.add_argument("--dtype", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--view", type=int, default=0)
    args = ap.parse_args()
    ng.lib()
    sc = CK.load_scene(args.scene)
    cfg = sc.cfg
    dt = {"f32": ng.F32, "f16": ng.F16, "bf16": ng.BF16}[args.dtype]
    ds = ng.DeviceScene(cfg, sc.tables, sc.coarse, sc.mlp_w, table_dtype=dt, mlp_dtype=ng.F32 if dt == ng.F32 else ng.F16)
    docc = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels)
    cams = HF.test_cameras(cfg)[args.view:args.view + 1]
    opts = S.default_options(cfg)
    rend = ng.Renderer(ds, docc)
    st = rend.render(opts, cams=cams, W=cfg.W, H=cfg.H, stats=True)["stats"].float().mean(0)
    out = rend.render(opts, cams=cams, W=cfg.W, H=cfg.H)
    times = []
    for _ in range(args.frames):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rend.render(opts, cams=cams, W=cfg.W, H=cfg.H, out=out)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    print(f"{args.dtype} view {args.view}: {statistics.mean(times):.3f} ms per frame, "
          f"{float(st[0]):.2f} marching points and {float(st[1]):.2f} samples per ray")


if __name__ == "__main__":
    main()
