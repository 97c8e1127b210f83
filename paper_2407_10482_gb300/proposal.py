"""Learned per-ray proposal: training on the GPU and the fast render path.

The proposal network (6 -> 32 -> 32 -> 3 on (o / in_scale, d)) predicts the interval
[t_near, t_far] holding a ray's significant weights and its opacity.  It learns
from the plain renderer: ``ngprt_proposal_targets`` reads the weight distribution
of a plain render, ``ngprt_propose_backward`` gives the loss gradient and
``ngprt_adam_step`` updates the weights; every step runs in the library's kernels
(torch only holds the buffers and draws the minibatch indices).  The fast render
then marches each ray only inside its predicted interval and re-marches, in a
fallback pass, the rays whose interval missed more than 1% of the predicted
opacity.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from . import ngprt as ng


@dataclass
class ProposalConfig:
    in_scale: float = 3.0      # origins are divided by this (the orbit radius)
    t_scale: float = 16.0      # t_near, t_far = t_scale * sigmoid(.)
    # world units the march starts before t_near.  The rays the proposal gets wrong
    # are opaque ones started behind their surface, which the opacity fallback cannot
    # see.  On the fitted hd scene (8 held-out views) 1.0 keeps the PSNR loss against
    # the ground truth at 0.06 dB; 0.5 and 0.25 lose 0.3 and 0.8 dB for 1.5% and 3.6%
    # less frame time
    margin_near: float = 1.0
    # after t_far (inf: no far clip, termination ends the ray); a clip at 2.0 or 0.5
    # measured 11-19% slower there, with no PSNR gain
    margin_far: float = float("inf")
    a_min: float = 0.01        # predicted opacity below which nothing is marched
    fallback: float = 0.01     # re-march when a_hat - A(interval) exceeds this
    steps: int = 6000
    batch: int = 1 << 15
    lr: float = 1e-2
    seed: int = 4


def init_weights(seed: int, device="cuda") -> torch.Tensor:
    n = ng.ngprt_proposal_param_count()
    rng = np.random.default_rng(seed)
    w = np.zeros(n, np.float32)
    W = 32
    o = 0
    for fan_in, fan_out in ((6, W), (W, W), (W, 3)):
        w[o:o + fan_out * fan_in] = rng.normal(0, 1.0 / math.sqrt(fan_in), fan_out * fan_in)
        o += fan_out * fan_in + fan_out  # weights then zero biases
    return torch.as_tensor(w).to(device)


def make_targets(renderer: ng.Renderer, opts, cams: np.ndarray, W: int, H: int, pixel_ids: torch.Tensor):
    """Plain render of the training rays and the weight-interval targets [n][3]."""
    out = renderer.render(opts, cams=cams, W=W, H=H, pixel_ids=pixel_ids, state=True)
    cam_arr, n_cams = ng.cameras_struct(cams, W, H)
    n = pixel_ids.numel()
    targets = torch.empty(n, 3, device=pixel_ids.device)
    ng.ngprt_proposal_targets(renderer.scene.struct, renderer.occ.struct, cam_arr, n_cams, pixel_ids, None, None, n,
                              ng.render_opts(opts), out["state"], targets)
    return targets


def train(cams: np.ndarray, W: int, H: int, pixel_ids: torch.Tensor, targets: torch.Tensor,
          cfg: ProposalConfig = ProposalConfig(), log_every: int = 0):
    """Adam on minibatches of the training rays; returns (weights, loss history)."""
    dev = pixel_ids.device
    w = init_weights(cfg.seed, dev)
    g = torch.zeros_like(w)
    m = torch.zeros_like(w)
    v = torch.zeros_like(w)
    loss = torch.zeros(1, device=dev)
    cam_arr, n_cams = ng.cameras_struct(cams, W, H)
    gen = torch.Generator(device=dev)
    gen.manual_seed(cfg.seed)
    hist = []
    n = pixel_ids.numel()
    for step in range(1, cfg.steps + 1):
        idx = torch.randint(0, n, (cfg.batch,), device=dev, generator=gen)
        pix = pixel_ids[idx].contiguous()
        tg = targets[idx].contiguous()
        if log_every and step % log_every == 0:
            loss.zero_()
        ng.ngprt_propose_backward(w, cam_arr, n_cams, pix, None, None, cfg.batch, cfg.in_scale, cfg.t_scale, tg, g,
                                  loss if (log_every and step % log_every == 0) else None)
        lr = cfg.lr * min(1.0, step / 100.0)
        ng.ngprt_adam_step(w, g, m, v, lr, 0.9, 0.99, 1e-8, step, True)
        if log_every and step % log_every == 0:
            hist.append((step, float(loss.item())))
    return w, hist


class FastRenderer:
    """FP16 tables + tensor-core FP16 MLP + learned proposal (FP16 weights) with
    fallback.

    ``render`` writes rgb/depth/opacity for one batch of camera rays; all buffers
    are allocated once per ray count."""

    def __init__(self, scene: ng.DeviceScene, occ: ng.DeviceOcc, prop_w: torch.Tensor,
                 cfg: ProposalConfig = ProposalConfig(), device="cuda"):
        self.scene, self.occ, self.cfg, self.device = scene, occ, cfg, device
        self.w = prop_w.to(torch.float16).contiguous()  # FP16 copy of the trained FP32 master
        self._n = -1

    def _buffers(self, n: int):
        if n != self._n:
            d = self.device
            self.interval = torch.empty(n, 2, device=d)
            self.a_hat = torch.empty(n, device=d)
            self.state = torch.empty(n, ng.STATE_FLOATS, device=d)
            self.stats = torch.empty(n, 2, dtype=torch.int32, device=d)
            # the render's workspace (the march's tile counter past the state's bytes)
            self.ws = torch.empty(ng.ngprt_render_workspace_bytes(self.scene.struct, n), dtype=torch.uint8, device=d)
            self._n = n

    def render(self, opts, cams: np.ndarray, W: int, H: int, rgb, depth=None, opacity=None, stats=False,
               stream=None):
        cam_arr, n_cams = ng.cameras_struct(cams, W, H)
        n = n_cams * W * H
        self._buffers(n)
        ro = ng.render_opts(opts)
        c = self.cfg
        st = self.stats if stats else None
        ng.ngprt_propose(self.w, cam_arr, n_cams, None, None, None, n, c.in_scale, c.t_scale, c.margin_near,
                         c.margin_far, c.a_min, self.interval, self.a_hat, stream=stream)
        ng.ngprt_render(self.scene.struct, self.occ.struct, cam_arr, n_cams, None, None, None, n, self.interval, ro,
                        None, ray_stats=st, ray_state=self.state, workspace=self.ws, stream=stream)
        ng.ngprt_render_fallback(self.scene.struct, self.occ.struct, cam_arr, n_cams, None, None, None, n,
                                 self.interval, self.a_hat, c.fallback, ro, self.state, st, stream=stream)
        ng.ngprt_shade(self.scene.struct, self.state, n, opts.bg, rgb, depth, opacity, stream=stream)


def psnr(a: torch.Tensor, b: torch.Tensor) -> float:
    """PSNR with peak 1 over all pixels and channels (no clamping)."""
    mse = float(((a.double() - b.double()) ** 2).mean())
    return float("inf") if mse == 0 else 10.0 * math.log10(1.0 / mse)
