"""The ground-truth images of the analytic scene (the fitting targets) against
closed forms and brute-force quadrature of the analytic field (CPU, FP64)."""
import math

import numpy as np
import pytest
import torch

from paper_2407_10482_gb300 import groundtruth as GT
from paper_2407_10482_gb300 import scenes as S


def _one_blob(p=30.0, s=0.1, mu=(0.2, -0.1, 0.05), rgb=(0.9, 0.2, 0.4)):
    return dict(mu=np.array([mu]), std=np.array([s]), peak=np.array([p]), rgb=np.array([rgb]))


def test_single_blob_through_centre_closed_form():
    # a ray through the centre crosses the whole Gaussian: tau = p s sqrt(2 pi)
    b = _one_blob()
    mu = torch.tensor(b["mu"], dtype=torch.float64)
    o = mu - torch.tensor([[3.0, 0.0, 0.0]], dtype=torch.float64)
    d = torch.tensor([[1.0, 0.0, 0.0]], dtype=torch.float64)
    rgb, a = GT.render_rays(b, o, d, shell=False, n_steps=64)
    tau = 30.0 * 0.1 * math.sqrt(2.0 * math.pi)
    # the integration segment ends 6 standard deviations out: erfc(6 / sqrt 2) ~ 2e-9
    assert abs(float(a[0]) - (1.0 - math.exp(-tau))) < 1e-9
    # one blob: the colour is its own, scaled by the opacity (black background)
    assert np.allclose(rgb[0].numpy(), (1.0 - math.exp(-tau)) * np.array(b["rgb"][0]), atol=1e-9)


def test_offset_ray_closed_form():
    # at distance b from the centre the whole-ray depth is p exp(-b^2 / 2 s^2) s sqrt(2 pi)
    b = _one_blob(p=40.0, s=0.12)
    off = 0.15
    o = torch.tensor([[0.2 - 3.0, -0.1 + off, 0.05]], dtype=torch.float64)
    d = torch.tensor([[1.0, 0.0, 0.0]], dtype=torch.float64)
    _, a = GT.render_rays(b, o, d, shell=False, n_steps=16)
    tau = 40.0 * math.exp(-off ** 2 / (2 * 0.12 ** 2)) * 0.12 * math.sqrt(2.0 * math.pi)
    assert abs(float(a[0]) - (1.0 - math.exp(-tau))) < 1e-9


def _brute(blobs, o, d, shell, t0, t1, n=400000):
    """Midpoint quadrature of the emission-absorption integral with the analytic
    density and density-weighted colour evaluated point by point."""
    t = t0 + (np.arange(n) + 0.5) * (t1 - t0) / n
    dt = (t1 - t0) / n
    x = o[None, :] + t[:, None] * d[None, :]
    sig = S.blob_density(blobs, x, False)
    col = S.blob_color(blobs, x)
    if shell:
        r = np.linalg.norm(x, axis=1)
        m = (r >= 8.0) & (r <= 10.0)
        sh = GT.shell_color(torch.as_tensor(x / r[:, None])).numpy()
        col = np.where(m[:, None], (sig[:, None] * col + 20.0 * sh) / (sig[:, None] + 20.0), col)
        sig = np.where(m, sig + 20.0, sig)
    alpha = 1.0 - np.exp(-sig * dt)
    T = np.concatenate([[1.0], np.cumprod(1.0 - alpha)[:-1]])
    w = T * alpha
    return (w[:, None] * col).sum(0), w.sum()


@pytest.mark.parametrize("seed", [0, 1])
def test_blob_field_matches_brute_force(seed):
    cfg = S.small_config(seed=seed)
    rng = np.random.default_rng(seed)
    blobs = S._blobs(cfg, rng)
    o_np, d_np = S.random_rays(6, seed + 10, True)
    d_np = d_np / np.linalg.norm(d_np, axis=1, keepdims=True)
    o = torch.as_tensor(o_np, dtype=torch.float64)
    d = torch.as_tensor(d_np, dtype=torch.float64)
    rgb, a = GT.render_rays(blobs, o, d, shell=False, n_steps=2048, top_k=8)
    for i in range(6):
        c_ref, a_ref = _brute(blobs, o_np[i].astype(np.float64), d_np[i].astype(np.float64), False, 0.0, 7.0)
        assert abs(float(a[i]) - a_ref) < 2e-4, (i, float(a[i]), a_ref)
        assert np.abs(rgb[i].numpy() - c_ref).max() < 2e-3, (i, rgb[i], c_ref)


def test_shell_and_blobs_match_brute_force():
    cfg = S.hd_config()
    blobs = S._blobs(cfg, np.random.default_rng(cfg.seed))
    cams = S.orbit_cameras(cfg, 1)
    pid = torch.tensor([540 * 1920 + 960, 300 * 1920 + 700], dtype=torch.int64)
    o, d = GT.camera_rays(cams, cfg.W, cfg.H, pid)
    rgb, a = GT.render_rays(blobs, o, d, shell=True, t_min=cfg.t_min, n_steps=2048, n_shell_steps=256, top_k=64)
    for i in range(len(pid)):
        c_ref, a_ref = _brute(blobs, o[i].numpy(), d[i].numpy(), True, cfg.t_min, 14.0, n=500000)
        assert abs(float(a[i]) - a_ref) < 1e-6
        assert np.abs(rgb[i].numpy() - c_ref).max() < 3e-3, (i, rgb[i], c_ref)


def test_camera_rays_are_pixel_centres():
    cfg = S.small_config()
    cams = S.orbit_cameras(cfg, 2)
    pid = torch.tensor([0, 63, 64 * 64 + 64 * 10 + 5], dtype=torch.int64)
    o, d = GT.camera_rays(cams, cfg.W, cfg.H, pid)
    for k, (v, row, col) in enumerate(((0, 0, 0), (0, 0, 63), (1, 10, 5))):
        c = cams[v].astype(np.float64)
        m = c[:12].reshape(3, 4)
        assert np.allclose(o[k].numpy(), m[:, 3])
        dc = np.linalg.solve(m[:, :3], d[k].numpy())   # camera-frame direction
        u = c[12] * dc[0] / dc[2] + c[14]
        vv = c[13] * dc[1] / dc[2] + c[15]
        assert abs(u - (col + 0.5)) < 1e-9 and abs(vv - (row + 0.5)) < 1e-9


def test_occupancy_torch_matches_numpy():
    cfg = S.hd_config(R_O=32)
    blobs = S._blobs(cfg, np.random.default_rng(cfg.seed))
    a = S._occupancy(cfg, blobs)
    b = S.occupancy_torch(cfg, blobs, device="cpu", chunk=5000).numpy()
    assert a.sum() > 0 and np.array_equal(a, b)


def test_bounded_field_is_clipped_to_the_box():
    # a blob centred on the box face: a ray along the face normal through the centre
    # sees only the inner half, tau = p s sqrt(2 pi) / 2
    b = _one_blob(p=20.0, s=0.1, mu=(1.0, 0.0, 0.0))
    o = torch.tensor([[-3.0, 0.0, 0.0]], dtype=torch.float64)
    d = torch.tensor([[1.0, 0.0, 0.0]], dtype=torch.float64)
    _, a = GT.render_rays(b, o, d, shell=False, n_steps=32, bounded=True)
    tau = 20.0 * 0.1 * math.sqrt(2.0 * math.pi) / 2.0
    assert abs(float(a[0]) - (1.0 - math.exp(-tau))) < 1e-9


def test_tile_order_is_a_grouping_permutation():
    from paper_2407_10482_gb300 import fit as F
    W, H = 100, 70
    pix = torch.as_tensor(S.random_pixels(5000, 3, W, H, 1))
    perm, inv = F.tile_order(pix, W, H, tile=32)
    assert torch.equal(torch.sort(perm).values, torch.arange(5000))
    assert torch.equal(perm[inv], torch.arange(5000))
    q = pix[perm].long()
    v, rem = q // (W * H), q % (W * H)
    key = v * 1000 + (rem // W // 32) * 10 + (rem % W) // 32
    assert torch.all(key[1:] >= key[:-1])          # views, then tile rows, then tile columns
