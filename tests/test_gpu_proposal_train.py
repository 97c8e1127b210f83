"""The learned proposal trained on the GPU by the library's own kernels, then used to
render: the loss falls, the fast render stays close to the plain render, and the
proposal saves marching points and samples (what the network gains over the
method without it)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2407_10482_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def test_trained_proposal_gains_over_plain_marching():
    from paper_2407_10482_gb300 import ngprt as ng
    from paper_2407_10482_gb300 import proposal as P
    ng.lib()
    cfg = S.small_config(bounded=False, R_O=64, n_occ_levels=4, t_min=0.05, r_far=16.0, shell=True, mlp_layers=3,
                         mlp_width=64, step_base=2 * 3 ** 0.5 / 256, blob_std=(0.05, 0.15), density_bias=3.2,
                         n_blobs=24, blob_box=1.0, W=160, H=120, seed=5)
    sc = S.make_scene(cfg)
    ds = ng.DeviceScene(cfg, sc.tables, sc.coarse, sc.mlp_w)
    docc = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels)
    rend = ng.Renderer(ds, docc)
    opts = S.default_options(cfg)
    train_cams = S.orbit_cameras(cfg, 64, azimuth0=2.8125, step_deg=5.625)
    pix = torch.as_tensor(S.random_pixels(1 << 17, 64, cfg.W, cfg.H, 4)).cuda()
    targets = P.make_targets(rend, opts, train_cams, cfg.W, cfg.H, pix)
    pc = P.ProposalConfig(steps=1000, batch=1 << 14)
    w, hist = P.train(train_cams, cfg.W, cfg.H, pix, targets, pc, log_every=100)
    assert hist[-1][1] < 0.5 * hist[0][1], hist
    cams = S.orbit_cameras(cfg, 1, azimuth0=45.0)
    plain = rend.render(opts, cams=cams, W=cfg.W, H=cfg.H, stats=True)
    fr = P.FastRenderer(ds, docc, w, pc)
    n = cfg.W * cfg.H
    rgb = torch.empty(n, 3, device="cuda")
    fr.render(opts, cams, cfg.W, cfg.H, rgb, stats=True)
    torch.cuda.synchronize()
    psnr = P.psnr(rgb, plain["rgb"])
    st_fast = fr.stats.float().mean(0)
    st_plain = plain["stats"].float().mean(0)
    assert psnr > 30.0, psnr
    # counts of the fast path include the fallback pass's second march
    assert st_fast[0] < st_plain[0], (st_fast, st_plain)   # fewer marching points
    assert st_fast[1] <= st_plain[1] * 1.05, (st_fast, st_plain)
