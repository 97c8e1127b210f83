"""Fitting an NGP-RT scene to images with the library's own kernels.

A fitted model is what the render path is meant to draw: the PSNR loss of a faster
form only means something against the images the model was fitted to (Sec. 4).
``fit`` runs the training loop of Sec. S2.1 on the render path of this library:
each step renders a random minibatch of pixels with ``ngprt_render`` (keeping the
per-ray state), takes the colour loss and its gradient (L2, or the Huber loss of
Sec. S2.4 with ``huber_delta`` > 0), runs ``ngprt_render_backward`` into the table,
coarse-grid and MLP gradients, adds eta times the distortion regulariser of Eq. S2
(``ngprt_distortion_loss`` / ``ngprt_distortion_backward``) when eta > 0, and applies
``ngprt_adam_step`` to each parameter array.  With ``autotune`` the step scaler gamma
follows Eq. S3 from the batch's mean sample count.  torch holds the buffers, draws
the minibatch indices and permutes the rays between pixel-tile and drawn order.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import ngprt as ng
from . import scenes as S


@dataclass
class FitConfig:
    steps: int = 1500
    batch: int = 1 << 18
    lr: float = 1e-2           # tables and coarse grid
    lr_mlp: float = 3e-3
    beta1: float = 0.9
    beta2: float = 0.99
    eps: float = 1e-15
    warmup: int = 50           # linear learning-rate warm-up, steps
    decay_from: float = 0.6    # cosine decay to lr / 10 over the last 40% of steps
    table_std: float = 1e-4    # initial tables and coarse grid ~ N(0, table_std)
    density_init: float = 0.0  # initial coarse density logit (sigma = exp(density_init))
    huber_delta: float = 0.0   # > 0: Huber colour loss with this delta (Sec. S2.4); 0: L2
    eta: float = 0.0           # weight of the distortion regulariser (Eq. S2; 0.01 in Sec. S2.4)
    autotune: bool = False     # step scaler gamma by Eq. S3
    n_min: float = 3.0
    kappa: float = 1e-3
    gamma_min: float = 0.2217
    seed: int = 3


def initial_scene(cfg: S.SceneConfig, fc: FitConfig, device="cuda"):
    """(tables, coarse, mlp_w) device tensors to start a fit from: small Gaussian
    grids with the coarse density logit at ``density_init`` and an MLP ~ N(0, 1/fan_in)."""
    g = torch.Generator(device=device)
    g.manual_seed(fc.seed)
    tables = torch.randn(S.table_entries(cfg), S.N_FEAT, generator=g, device=device) * fc.table_std
    coarse = torch.randn(cfg.R_C ** 3, S.coarse_channels(cfg), generator=g, device=device) * fc.table_std
    coarse[:, 0] += fc.density_init
    rng = np.random.default_rng(fc.seed)
    ws = []
    for k, (o, i) in enumerate(S.mlp_shapes(cfg)):
        real_in = 23 if k == 0 else i
        w = rng.normal(0.0, 1.0 / math.sqrt(real_in), (o, i)).astype(np.float32)
        if k == 0:
            w[:, 23:] = 0.0
        ws.append(w.reshape(-1))
    mlp_w = torch.as_tensor(np.concatenate(ws)).to(device)
    return tables, coarse, mlp_w


def initial_agg_mlp(cfg: S.SceneConfig, fc: FitConfig, device="cuda"):
    """Weights of the tiny-MLP aggregation (W1 [64][8L] ~ N(0, 1/(8L)), W2 [8][64] ~
    N(0, 1/64), no biases) for the MLP form; None for the other forms."""
    if cfg.aggregation != 5:
        return None
    rng = np.random.default_rng(fc.seed + 2)
    nx = S.N_FEAT * cfg.L
    w1 = rng.normal(0.0, 1.0 / math.sqrt(nx), (64, nx))
    w2 = rng.normal(0.0, 1.0 / math.sqrt(64), (S.N_FEAT, 64))
    return torch.as_tensor(np.concatenate([w1.reshape(-1), w2.reshape(-1)]).astype(np.float32)).to(device)


def initial_attn_inv(cfg: S.SceneConfig, fc: FitConfig, device="cuda"):
    """The constant gate logits of the spatially invariant forms (2L for separate
    gates, L for shared ones), drawn like the coarse grid's spatial logits; None for
    the other forms."""
    agg = cfg.aggregation
    if agg not in (2, 3):
        return None
    g = torch.Generator(device=device)
    g.manual_seed(fc.seed + 1)
    return torch.randn((2 if agg == 2 else 1) * cfg.L, generator=g, device=device) * fc.table_std


def tile_order(pixel_ids: torch.Tensor, W: int, H: int, tile: int = 32):
    """(perm, inv): the permutation that groups a minibatch's pixel ids by view and
    tile x tile image tile (row-major inside a tile), and its inverse.  The render
    runs fastest on rays in this order (neighbouring lanes sample neighbouring
    points); the reverse pass runs fastest in the drawn random order (neighbouring
    lanes then rarely add gradients to the same entries), so the state moves back
    through inv between the two."""
    p = pixel_ids.long()
    v, rem = p // (W * H), p % (W * H)
    row, col = rem // W, rem % W
    key = (v << 40) | ((row // tile) << 28) | ((col // tile) << 16) | ((row % tile) << 8) | (col % tile)
    perm = torch.argsort(key)
    inv = torch.empty_like(perm)
    inv[perm] = torch.arange(len(perm), device=perm.device)
    return perm, inv


def _lr_factor(step: int, fc: FitConfig) -> float:
    f = min(1.0, step / max(1, fc.warmup))
    s0 = fc.decay_from * fc.steps
    if step > s0:
        x = (step - s0) / max(1.0, fc.steps - s0)
        f *= 0.1 + 0.45 * (1.0 + math.cos(math.pi * x))
    return f


def fit(scene: ng.DeviceScene, occ: ng.DeviceOcc, opts, cams: np.ndarray, W: int, H: int,
        targets: torch.Tensor, fc: FitConfig = FitConfig(), log_every: int = 0, stream=None,
        refine_at=(), refine=None):
    """Fit ``scene`` (FP32 tables, coarse grid, MLP and the aggregation form's own
    parameters: constant gate logits or the tiny MLP's weights; updated in place) to
    the images ``targets`` [n_views * H * W, 3] of the cameras ``cams``.
    After each step in ``refine_at`` the occupancy becomes ``refine(step, occ)`` (a
    DeviceOcc built from the model so far).
    Returns the loss history [(step, loss)] and the wall time in seconds; with
    ``autotune`` the final gamma is left in ``fit.last_gamma``, and the occupancy the
    fit ended with in ``fit.last_occ``."""
    from dataclasses import replace
    dev = scene.tables.device
    rend = ng.Renderer(scene, occ, device=dev)
    params = [scene.tables, scene.coarse, scene.mlp_w]
    lrs = [fc.lr, fc.lr, fc.lr_mlp]
    extra = {}                           # the aggregation's own parameters, by backward keyword
    if scene.attn_inv is not None and scene.cfg.aggregation in (2, 3):       # constant gate logits
        extra["g_attn_inv"] = len(params)
        params.append(scene.attn_inv)
        lrs.append(fc.lr)
    if scene.agg_mlp is not None and scene.cfg.aggregation == 5:             # tiny-MLP weights
        extra["g_agg_mlp"] = len(params)
        params.append(scene.agg_mlp)
        lrs.append(fc.lr_mlp)
    grads = [torch.zeros_like(p) for p in params]
    moms = [(torch.zeros_like(p), torch.zeros_like(p)) for p in params]
    n_pix = len(cams) * W * H
    gen = torch.Generator(device=dev)
    gen.manual_seed(fc.seed)
    B = fc.batch
    loss = torch.zeros(1, device=dev)
    d_rgb = torch.empty(B, 3, device=dev)
    out = dict(rgb=torch.empty(B, 3, device=dev), depth=torch.empty(B, device=dev),
               opacity=torch.empty(B, device=dev), state=torch.empty(B, ng.STATE_FLOATS, device=dev))
    if fc.autotune:
        out["stats"] = torch.empty(B, 2, dtype=torch.int32, device=dev)
        n_mean = torch.empty(1, device=dev)
    dist_state = torch.empty(B, 4, device=dev) if fc.eta > 0 else None
    dist_ws = None
    cam_arr, n_cams = ng.cameras_struct(cams, W, H)
    gamma = opts.step_gamma
    hist = []
    t0 = time.perf_counter()
    for step in range(1, fc.steps + 1):
        idx = torch.randint(0, n_pix, (B,), device=dev, generator=gen)
        pix = idx.to(torch.int32)
        perm, back = tile_order(pix, W, H)
        pix_f = pix[perm].contiguous()
        tg = targets[idx[perm]].contiguous()
        logging = bool(log_every) and (step % log_every == 0 or step == fc.steps)
        if logging:
            loss.zero_()
        o_step = replace(opts, step_gamma=gamma) if fc.autotune else opts
        rend.render(o_step, cams=cams, W=W, H=H, pixel_ids=pix_f, state=True, out=out)
        if fc.huber_delta > 0:
            ng.ngprt_huber_loss(out["rgb"], tg, 3 * B, fc.huber_delta, 1.0 / (3 * B), loss if logging else None,
                                d_rgb, stream=stream)
        else:
            ng.ngprt_l2_loss(out["rgb"], tg, 3 * B, 1.0 / (3 * B), loss if logging else None, d_rgb, stream=stream)
        rend.backward(o_step, out["state"][back].contiguous(), d_rgb[back].contiguous(), None, None, grads[0],
                      grads[1], grads[2], cams=cams, W=W, H=H, pixel_ids=pix,
                      **{k: grads[i] for k, i in extra.items()})
        if fc.eta > 0:
            ro = ng.render_opts(o_step)
            ng.ngprt_distortion_loss(scene.struct, occ.struct, cam_arr, n_cams, pix, None, None, B, ro, fc.eta / B,
                                     dist_state, loss if logging else None, stream=stream)
            need = ng.ngprt_distortion_backward_workspace_bytes(scene.struct, ro, B)
            if need and (dist_ws is None or dist_ws.numel() < need):
                dist_ws = torch.empty(need, dtype=torch.uint8, device=dev)
            ng.ngprt_distortion_backward(scene.struct, occ.struct, cam_arr, n_cams, pix, None, None, B, ro,
                                         dist_state, fc.eta / B, grads[0], grads[1], stream=stream,
                                         workspace=dist_ws if need else None,
                                         **{k: grads[i] for k, i in extra.items()})
        if fc.autotune:
            ng.ngprt_mean_samples(out["stats"], B, n_mean, stream=stream)
            gamma = ng.ngprt_step_autotune(gamma, float(n_mean.item()), fc.n_min, fc.kappa, fc.gamma_min)
        f = _lr_factor(step, fc)
        for p, g, (m, v), lr in zip(params, grads, moms, lrs):
            ng.ngprt_adam_step(p, g, m, v, lr * f, fc.beta1, fc.beta2, fc.eps, step, True, stream=stream)
        if logging:
            hist.append((step, float(loss.item())))
        if refine is not None and step in refine_at:
            occ = refine(step, occ)
            rend = ng.Renderer(scene, occ, device=dev)
    torch.cuda.synchronize(dev)
    fit.last_gamma = gamma
    fit.last_occ = occ
    return hist, time.perf_counter() - t0
