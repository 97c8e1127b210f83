"""The learned proposal trained on the GPU by the library's own kernels, then used to
render a fitted scene: the loss falls, the fast render's PSNR against the held-out
ground truth stays within 0.1 dB of the plain render's, and the proposal saves
marching points without adding samples (what the network gains over the method
without it)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2407_10482_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def test_trained_proposal_keeps_the_fitted_scene_within_0p1_db():
    from paper_2407_10482_gb300 import hdfit as HF
    from paper_2407_10482_gb300 import ngprt as ng
    from paper_2407_10482_gb300 import proposal as P
    ng.lib()
    # a reduced fitted workload: the hd scene's field and orbit, 8 levels up to 512,
    # T = 2^16, 64^3 occupancy, 320x180 held-out views, 48 training views at 160x90
    cfg = S.hd_fit_config(L=8, N=S.level_resolutions(16, 512, 8), T_log2=16, R_O=64, n_occ_levels=4, W=320, H=180)
    hc = HF.HdFitConfig(steps=300, batch=1 << 16, refine_at=(80, 180), train_res=(160, 90))
    fs = HF.fit_hd_scene(cfg, hc, log_every=100)
    opts = S.default_options(cfg)
    rend = ng.Renderer(fs.scene, fs.occ)
    train_cams = S.orbit_cameras(cfg, 64, azimuth0=2.8125, step_deg=5.625)
    pix = torch.as_tensor(S.random_pixels(1 << 17, 64, cfg.W, cfg.H, 4)).cuda()
    targets = P.make_targets(rend, opts, train_cams, cfg.W, cfg.H, pix)
    pc = P.ProposalConfig(steps=1500, batch=1 << 14)
    w, hist = P.train(train_cams, cfg.W, cfg.H, pix, targets, pc, log_every=100)
    assert hist[-1][1] < 0.5 * hist[0][1], hist
    ds16 = ng.DeviceScene(cfg, fs.scene.tables, fs.scene.coarse, fs.scene.mlp_w, table_dtype=ng.F16,
                          mlp_dtype=ng.F16)
    fr = P.FastRenderer(ds16, fs.occ, w, pc)
    n = cfg.W * cfg.H
    rgb_plain = torch.empty(len(fs.cams_test) * n, 3, device="cuda")
    rgb_fast = torch.empty_like(rgb_plain)
    st_plain, st_fast = [], []
    for v in range(len(fs.cams_test)):
        c = fs.cams_test[v:v + 1]
        o = rend.render(opts, cams=c, W=cfg.W, H=cfg.H, stats=True)
        rgb_plain[v * n:(v + 1) * n] = o["rgb"]
        st_plain.append(o["stats"].float().mean(0))
        fr.render(opts, c, cfg.W, cfg.H, rgb_fast[v * n:(v + 1) * n], stats=True)
        st_fast.append(fr.stats.float().mean(0))
    torch.cuda.synchronize()
    p_plain = HF.psnr(rgb_plain, fs.targets_test)
    p_fast = HF.psnr(rgb_fast, fs.targets_test)
    sp, sf = torch.stack(st_plain).mean(0), torch.stack(st_fast).mean(0)
    print(f"proposal: held-out PSNR plain {p_plain:.3f} dB, fast {p_fast:.3f} dB (loss {p_plain - p_fast:.3f}); "
          f"marching {float(sp[0]):.1f} -> {float(sf[0]):.1f}, samples {float(sp[1]):.1f} -> {float(sf[1]):.1f}")
    assert p_plain > 15.0, p_plain                   # the fit reached a usable model
    assert p_plain - p_fast <= 0.1, (p_plain, p_fast)
    # counts of the fast path include the fallback pass's second march
    assert sf[0] < sp[0], (sf, sp)                   # fewer marching points
    assert sf[1] <= sp[1] * 1.05, (sf, sp)
