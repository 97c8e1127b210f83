"""Fitting the small scene's model to ground-truth images of its analytic field with
the library's forward, reverse pass and Adam kernels: the photometric error must
fall by a wide margin, on the training views and on a view between them."""
import numpy as np
import pytest
import torch

from paper_2407_10482_gb300 import fit as F
from paper_2407_10482_gb300 import groundtruth as GT
from paper_2407_10482_gb300 import proposal as P
from paper_2407_10482_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ng():
    from paper_2407_10482_gb300 import ngprt
    ngprt.lib()
    return ngprt


def test_fit_small_scene(ng):
    cfg = S.small_config()
    blobs = S._blobs(cfg, np.random.default_rng(cfg.seed))
    occ = S._occupancy(cfg, blobs)
    cams = S.orbit_cameras(cfg, 32, step_deg=360.0 / 32)
    targets = GT.render_views(cfg, blobs, cams, device="cuda", n_steps=512)
    held = S.orbit_cameras(cfg, 1, azimuth0=360.0 / 64)
    held_t = GT.render_views(cfg, blobs, held, device="cuda", n_steps=512)
    fc = F.FitConfig(steps=400, batch=1 << 14, seed=5)
    tables, coarse, mlp = F.initial_scene(cfg, fc, "cuda")
    ds = ng.DeviceScene(cfg, tables, coarse, mlp)
    docc = ng.DeviceOcc(occ, cfg.R_O, cfg.n_occ_levels)
    opts = S.default_options(cfg)
    r = ng.Renderer(ds, docc)
    before = P.psnr(r.render(opts, cams=cams, W=cfg.W, H=cfg.H)["rgb"], targets)
    before_h = P.psnr(r.render(opts, cams=held, W=cfg.W, H=cfg.H)["rgb"], held_t)
    hist, _ = F.fit(ds, docc, opts, cams, cfg.W, cfg.H, targets, fc, log_every=100)
    after = P.psnr(r.render(opts, cams=cams, W=cfg.W, H=cfg.H)["rgb"], targets)
    after_h = P.psnr(r.render(opts, cams=held, W=cfg.W, H=cfg.H)["rgb"], held_t)
    print(f"fit: train {before:.2f} -> {after:.2f} dB, held-out {before_h:.2f} -> {after_h:.2f} dB, loss {hist}")
    assert all(np.isfinite(l) for _, l in hist)
    assert hist[-1][1] < 0.2 * hist[0][1]
    assert after > before + 8.0 and after > 22.0
    assert after_h > before_h + 6.0
