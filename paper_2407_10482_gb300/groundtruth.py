"""Ground-truth images of the analytic synthetic scene.

These images stand in for the captured photographs of Mip-NeRF 360 that the paper
fits and evaluates on (Sec. 4): they are the targets the NGP-RT model is fitted to
and the ground truth its PSNR is measured against.  They are not produced by the
rendering method.  The scene's true field is analytic: Gaussian blobs

    sigma_k(x) = p_k exp(-|x - mu_k|^2 / (2 s_k^2)),  colour c_k (constant per blob),

plus, for the unbounded scene, a shell of density 20 between world radii 8 and 10
whose colour is a smooth function of the direction x / |x| (``shell_color``).

Along a straight ray x(t) = o + t d (|d| = 1) the optical depth of blob k over
[t0, t1] has the closed form

    a_k s_k sqrt(pi/2) (erf((t1 - t_k) / (sqrt(2) s_k)) - erf((t0 - t_k) / (sqrt(2) s_k))),

with t_k = (mu_k - o).d and a_k = p_k exp(-b_k^2 / (2 s_k^2)), b_k the ray's distance
from mu_k.  The image is the emission-absorption integral over fine steps: each step
takes its exact optical depth tau = sum_k tau_k, its opacity 1 - exp(-tau), and the
colour mix sum_k tau_k c_k / tau (exact when the blob ratio is constant within the
step, and converging with the step count).  Only the ``top_k`` blobs with the
largest a_k s_k on each ray are integrated; the others add less than that share.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import scenes as S

SHELL_SIGMA = 20.0
SHELL_R0, SHELL_R1 = 8.0, 10.0


def shell_color(u: torch.Tensor) -> torch.Tensor:
    """Colour of the background shell for unit directions u [..., 3] (values in [0, 1])."""
    x, y, z = u[..., 0], u[..., 1], u[..., 2]
    return torch.stack([0.5 + 0.5 * torch.sin(3.0 * x + 2.0 * y + 1.0),
                        0.5 + 0.5 * torch.sin(4.0 * y - 3.0 * z + 2.0),
                        0.5 + 0.5 * torch.sin(5.0 * z + 2.0 * x + 3.0)], -1)


def camera_rays(cams: np.ndarray, W: int, H: int, pixel_ids: torch.Tensor, dtype=torch.float64):
    """World origins and unit directions of pixel-centre rays (OpenCV pinhole axes);
    pixel id = view * W * H + row * W + col."""
    dev = pixel_ids.device
    c = torch.as_tensor(np.asarray(cams, np.float64).reshape(-1, S.CAM_FLOATS), device=dev, dtype=dtype)
    pid = pixel_ids.long()
    v = pid // (W * H)
    rem = pid % (W * H)
    row, col = rem // W, rem % W
    cv = c[v]
    m = cv[:, :12].reshape(-1, 3, 4)
    fx, fy, cx, cy = cv[:, 12], cv[:, 13], cv[:, 14], cv[:, 15]
    dc = torch.stack([(col.to(dtype) + 0.5 - cx) / fx, (row.to(dtype) + 0.5 - cy) / fy,
                      torch.ones_like(fx)], -1)
    d = torch.einsum("nij,nj->ni", m[:, :, :3], dc)
    d = d / torch.linalg.norm(d, dim=1, keepdim=True)
    return m[:, :, 3].clone(), d


def _sphere_interval(o, d, r):
    """t range of |o + t d| <= r (|d| = 1); empty rows get t0 >= t1."""
    b = (o * d).sum(1)
    c = (o * o).sum(1) - r * r
    disc = b * b - c
    sq = torch.sqrt(torch.clamp(disc, min=0.0))
    t0 = torch.where(disc > 0, -b - sq, torch.zeros_like(b))
    t1 = torch.where(disc > 0, -b + sq, torch.zeros_like(b))
    return t0, t1


def _box_interval(o, d):
    """t range of o + t d inside [-1, 1]^3; empty rows get t0 >= t1."""
    inv = 1.0 / torch.where(d == 0, torch.full_like(d, 1e-300), d)
    a = (-1.0 - o) * inv
    b = (1.0 - o) * inv
    return torch.minimum(a, b).amax(1), torch.maximum(a, b).amin(1)


def render_rays(blobs: dict, o: torch.Tensor, d: torch.Tensor, shell: bool, bg=(0.0, 0.0, 0.0),
                t_min: float = 0.0, n_steps: int = 1024, n_shell_steps: int = 64, top_k: int = 16,
                bounded: bool = False):
    """RGB [n, 3] and opacity [n] of the analytic scene along rays (o, unit d); a
    bounded scene holds only the field inside [-1, 1]^3."""
    dt = o.dtype
    dev = o.device
    mu = torch.as_tensor(blobs["mu"], device=dev, dtype=dt)
    s = torch.as_tensor(blobs["std"], device=dev, dtype=dt)
    p = torch.as_tensor(blobs["peak"], device=dev, dtype=dt)
    col = torch.as_tensor(blobs["rgb"], device=dev, dtype=dt)
    n = o.shape[0]
    rel = mu.unsqueeze(0) - o.unsqueeze(1)                   # [n, B, 3]
    tk = (rel * d.unsqueeze(1)).sum(-1)                      # [n, B]
    b2 = torch.clamp((rel * rel).sum(-1) - tk * tk, min=0.0)
    amp = p * torch.exp(-b2 / (2.0 * s * s)) * s * math.sqrt(math.pi / 2.0)  # tau of the whole blob / 2
    k = min(top_k, mu.shape[0])
    amp_k, idx = torch.topk(amp, k, dim=1)
    tk_k = torch.gather(tk, 1, idx)
    s_k = s[idx]
    inv_k = 1.0 / (math.sqrt(2.0) * s_k)
    col_k = col[idx]                                         # [n, k, 3]
    # blob segment: from 6 standard deviations before the first blob the ray meets to
    # 6 after the last (the optical depth beyond is below 1e-8 of a blob's); rays that
    # meet no blob skip the quadrature
    sig = amp_k > 1e-9
    ta = torch.where(sig, tk_k - 6.0 * s_k, torch.full_like(tk_k, float("inf"))).amin(1)
    tb = torch.where(sig, tk_k + 6.0 * s_k, torch.full_like(tk_k, float("-inf"))).amax(1)
    if bounded:
        ba, bb = _box_interval(o, d)
        ta, tb = torch.maximum(ta, ba), torch.minimum(tb, bb)
    ta = torch.clamp(ta, min=t_min)
    T = torch.ones(n, device=dev, dtype=dt)
    C = torch.zeros(n, 3, device=dev, dtype=dt)
    act = torch.nonzero(tb > ta).squeeze(1)
    if act.numel():
        ta_a, tb_a = ta[act], tb[act]
        tk_a, inv_a, amp_a, col_a = tk_k[act], inv_k[act], amp_k[act], col_k[act]
        T_a = torch.ones(len(act), device=dev, dtype=dt)
        C_a = torch.zeros(len(act), 3, device=dev, dtype=dt)
        e_prev = torch.erf((ta_a.unsqueeze(1) - tk_a) * inv_a)
        for i in range(1, n_steps + 1):
            t = ta_a + (tb_a - ta_a) * (i / n_steps)
            e = torch.erf((t.unsqueeze(1) - tk_a) * inv_a)
            tau_k = amp_a * (e - e_prev)
            e_prev = e
            tau = tau_k.sum(1)
            w = T_a * (1.0 - torch.exp(-tau))
            num = torch.bmm(tau_k.unsqueeze(1), col_a).squeeze(1)
            C_a += torch.where((tau > 0).unsqueeze(-1),
                               w.unsqueeze(-1) * num / torch.where(tau > 0, tau, 1.0).unsqueeze(-1), 0.0)
            T_a = T_a * torch.exp(-tau)
        T[act] = T_a
        C[act] = C_a
    if shell:
        _, t8 = _sphere_interval(o, d, SHELL_R0)
        _, t10 = _sphere_interval(o, d, SHELL_R1)
        t8 = torch.clamp(t8, min=t_min)
        # density 20 over a layer 2 units thick (optical depth 40): 64 sub-steps over the
        # first unit carry all but e^-20 of the light; the rest of the layer takes it
        t_end = torch.minimum(t8 + 1.0, t10)
        t_prev = t8
        for i in range(1, n_shell_steps + 1):
            t = t8 + (t_end - t8) * (i / n_shell_steps)
            tau = SHELL_SIGMA * (t - t_prev)
            w = T * (1.0 - torch.exp(-tau))
            x = o + (0.5 * (t + t_prev)).unsqueeze(1) * d
            C += w.unsqueeze(-1) * shell_color(x / torch.linalg.norm(x, dim=1, keepdim=True))
            T = T * torch.exp(-tau)
            t_prev = t
        tau = SHELL_SIGMA * (t10 - t_end)
        w = T * (1.0 - torch.exp(-tau))
        x = o + t_end.unsqueeze(1) * d
        C += w.unsqueeze(-1) * shell_color(x / torch.linalg.norm(x, dim=1, keepdim=True))
        T = T * torch.exp(-tau)
    bgt = torch.as_tensor(bg, device=dev, dtype=dt)
    return C + T.unsqueeze(-1) * bgt, 1.0 - T


def render_views(cfg: S.SceneConfig, blobs: dict, cams: np.ndarray, device="cuda", dtype=torch.float32,
                 chunk: int = 1 << 20, **kw) -> torch.Tensor:
    """Ground-truth RGB [n_views * H * W, 3] (float32) of the orbit views ``cams``."""
    n = len(cams) * cfg.W * cfg.H
    out = torch.empty(n, 3, device=device, dtype=torch.float32)
    for s0 in range(0, n, chunk):
        pid = torch.arange(s0, min(n, s0 + chunk), device=device, dtype=torch.int64)
        o, d = camera_rays(cams, cfg.W, cfg.H, pid, dtype=dtype)
        rgb, _ = render_rays(blobs, o, d, cfg.shell, t_min=cfg.t_min, bounded=cfg.bounded, **kw)
        out[s0:s0 + len(pid)] = rgb.float()
    return out
