"""One training step of the render path, timed: render a minibatch of random pixels
of 8 orbit views (rays in pixel-tile order, keeping the per-ray state), photometric
L2 loss, reverse pass (rays in the drawn order), Adam on the tables, coarse grid
and MLP.  Render, loss, reverse pass and Adam run in the library's kernels; torch
permutes the rays between the two orders.

    python -m paper_2407_10482_gb300.train_step --rays 65536 --steps 5 [--scene FILE]

Without --scene: the random-weight hd scene and 8 orbit views; with it, a scene
written by ``checkpoint.save_scene`` (for instance the fitted hd scene of
``bench.py --save-scene``) and its 8 held-out views.  Targets are uniform random
colours (the work of a step does not depend on them).
"""
from __future__ import annotations

import argparse
import statistics

import numpy as np
import torch

from . import fit as F
from . import ngprt as ng
from . import scenes as S


def make_step(cfg, ds: ng.DeviceScene, docc: ng.DeviceOcc, cams: np.ndarray, targets: torch.Tensor,
              pixel_ids: torch.Tensor, lr: float = 1e-3, stream=None):
    """A closure running one step on `pixel_ids` (rays of `cams`) against `targets`
    [n, 3] (one colour per ray); returns it with its loss buffer."""
    dev = ds.tables.device
    B = pixel_ids.numel()
    rend = ng.Renderer(ds, docc, device=dev)
    opts = S.default_options(cfg)
    params = [ds.tables, ds.coarse, ds.mlp_w]
    grads = [torch.zeros_like(t) for t in params]
    moms = [(torch.zeros_like(t), torch.zeros_like(t)) for t in params]
    loss = torch.zeros(1, device=dev)
    d_rgb = torch.empty(B, 3, device=dev)
    step_no = [0]

    def step():
        # the ray order is part of the step (a new minibatch would need it again)
        perm, inv = F.tile_order(pixel_ids, cfg.W, cfg.H)
        pix_f = pixel_ids[perm].contiguous()
        tg_f = targets[perm].contiguous()
        o = rend.render(opts, cams=cams, W=cfg.W, H=cfg.H, pixel_ids=pix_f, state=True)
        ng.ngprt_l2_loss(o["rgb"], tg_f, 3 * B, 1.0 / (3 * B), loss, d_rgb, stream=stream)
        rend.backward(opts, o["state"][inv].contiguous(), d_rgb[inv].contiguous(), None, None, grads[0], grads[1],
                      grads[2], cams=cams, W=cfg.W, H=cfg.H, pixel_ids=pixel_ids)
        step_no[0] += 1
        for t, g, (m, v) in zip(params, grads, moms):
            ng.ngprt_adam_step(t, g, m, v, lr, 0.9, 0.99, 1e-8, step_no[0], True, stream=stream)
    return step, loss


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rays", type=int, default=1 << 18)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--scene", default="", help="a saved scene (checkpoint.save_scene) instead of the random hd scene")
    args = ap.parse_args()
    ng.lib()
    if args.scene:
        from . import checkpoint as CK
        from . import hdfit as HF
        sc = CK.load_scene(args.scene)
        cfg = sc.cfg
        cams = HF.test_cameras(cfg, 8)
    else:
        cfg = S.hd_config()
        sc = S.make_scene(cfg)
        cams = S.orbit_cameras(cfg, 8)
    ds = ng.DeviceScene(cfg, sc.tables, sc.coarse, sc.mlp_w)
    docc = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels)
    pix = torch.as_tensor(S.random_pixels(args.rays, 8, cfg.W, cfg.H, 3)).cuda()
    targets = torch.rand(args.rays, 3, generator=torch.Generator().manual_seed(3)).cuda()
    step, loss = make_step(cfg, ds, docc, cams, targets, pix)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ts = []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    print(f"training step, {args.rays} rays: {statistics.mean(ts):.3f} ms "
          f"({args.rays / statistics.mean(ts) * 1e3:.3e} rays/s)")


if __name__ == "__main__":
    main()
