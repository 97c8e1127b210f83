"""GPU parity of the occupancy pipeline (Sec. S2.5) against the oracle, through the C
ABI: density occupancy and visibility marks (integer grids; voxels whose deciding
value lies within rounding of the threshold are left out and must be rare), box
dilation bit for bit, and the pipeline end to end on the hd scene."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2407_10482_gb300 import proposal as P
from paper_2407_10482_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ng():
    from paper_2407_10482_gb300 import ngprt
    ngprt.lib()
    return ngprt


def _device_scene(ng, sc):
    return ng.DeviceScene(sc.cfg, sc.tables, sc.coarse, sc.mlp_w, attn_inv=sc.attn_inv, agg_mlp=sc.agg_mlp)


@pytest.mark.parametrize("cfg_name,R", [("small", 32), ("small", 64), ("hd", 64)])
def test_density_occupancy_matches_oracle(ng, cfg_name, R):
    cfg = S.small_config() if cfg_name == "small" else S.hd_config()
    sc = S.make_scene(cfg)
    ds = _device_scene(ng, sc)
    opts = S.default_options(cfg)
    orc = O.oracle_for_scene(sc)
    occ_ref, sig_ref = orc.occupancy_density(opts, R, 1.0)
    thr = float(np.median(sig_ref))        # about half the voxels on each side
    occ_ref = (sig_ref > thr).astype(np.uint8)
    occ = torch.empty(R ** 3, dtype=torch.uint8, device="cuda")
    sig = torch.empty(R ** 3, device="cuda")
    ng.ngprt_occupancy_from_density(ds.struct, ng.render_opts(opts), R, thr, occ, sig)
    torch.cuda.synchronize()
    sig_g = sig.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(sig_g, sig_ref, rtol=2e-5)
    sure = np.abs(sig_ref - thr) > 5e-5 * thr
    assert (~sure).sum() <= max(2, R ** 3 // 500)
    assert np.array_equal(occ.cpu().numpy()[sure], occ_ref[sure])


@pytest.mark.parametrize("agg", [1, 2, 3, 4, 5])
def test_density_occupancy_of_the_aggregation_forms(ng, agg):
    """Table 3's other forms: each feeds its own density into the occupancy."""
    cfg = S.small_config(aggregation=agg)
    sc = S.make_scene(cfg)
    ds = _device_scene(ng, sc)
    opts = S.default_options(cfg)
    R = 32
    _, sig_ref = O.oracle_for_scene(sc).occupancy_density(opts, R, 1.0)
    thr = float(np.median(sig_ref))
    occ = torch.empty(R ** 3, dtype=torch.uint8, device="cuda")
    sig = torch.empty(R ** 3, device="cuda")
    ng.ngprt_occupancy_from_density(ds.struct, ng.render_opts(opts), R, thr, occ, sig)
    torch.cuda.synchronize()
    np.testing.assert_allclose(sig.cpu().numpy().astype(np.float64), sig_ref, rtol=2e-5)
    sure = np.abs(sig_ref - thr) > 5e-5 * thr
    assert (~sure).sum() <= max(2, R ** 3 // 500)
    assert np.array_equal(occ.cpu().numpy()[sure], (sig_ref > thr).astype(np.uint8)[sure])


@pytest.mark.parametrize("agg", [0, 1, 3, 5])
def test_visibility_marks_match_oracle(ng, agg):
    cfg = S.small_config(aggregation=agg)
    sc = S.make_scene(cfg)
    ds = _device_scene(ng, sc)
    docc = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels)
    opts = S.default_options(cfg)
    orc = O.oracle_for_scene(sc)
    cams = S.orbit_cameras(cfg, 3, azimuth0=10.0, step_deg=120.0)
    R, thr = 32, 0.01
    vis_ref, wmax = orc.occupancy_visibility(opts, R, thr, cams=cams)
    cam_arr, nc = ng.cameras_struct(cams, cfg.W, cfg.H)
    vis = torch.zeros(R ** 3, dtype=torch.uint8, device="cuda")
    ng.ngprt_occupancy_visibility(ds.struct, docc.struct, cam_arr, nc, None, None, None, nc * cfg.W * cfg.H,
                                  ng.render_opts(opts), thr, R, vis)
    torch.cuda.synchronize()
    sure = np.abs(wmax - thr) > 1e-5
    assert vis_ref.sum() > 50
    assert np.array_equal(vis.cpu().numpy()[sure], vis_ref[sure])


@pytest.mark.parametrize("R,r,frac,seed", [(32, 0, 0.02, 0), (32, 1, 0.01, 1), (32, 3, 0.003, 2), (64, 2, 0.001, 3),
                                           (5, 4, 0.1, 4)])
def test_dilate_bit_exact(ng, R, r, frac, seed):
    rng = np.random.default_rng(seed)
    occ = (rng.uniform(size=R ** 3) < frac).astype(np.uint8)
    mask = (rng.uniform(size=R ** 3) < 0.7).astype(np.uint8)
    d_in = torch.as_tensor(occ).cuda()
    out = torch.empty_like(d_in)
    ws = torch.empty(ng.ngprt_dilate_workspace_bytes(R), dtype=torch.uint8, device="cuda")
    ng.ngprt_dilate(d_in, R, r, out, ws)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), O.dilate(occ, R, r))
    ng.ngprt_dilate(d_in, R, r, out, ws, mask=torch.as_tensor(mask).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), O.dilate(occ, R, r, mask))


def test_visibility_culled_occupancy_keeps_orbit_views(ng):
    """MERF-style render occupancy for the hd scene: the voxels of the samples that 16
    orbit views composite (weight > w_thr), dilated by one voxel within the full
    (training-stage) occupancy.  Orbit views rendered with it (one of the 16 and one
    between them) stay within 50 dB (w_thr = 0) or 45 dB (w_thr = 0.005) of the
    renders with the full occupancy, with at most 80% of its voxels."""
    cfg = S.hd_config(W=480, H=270)
    sc = S.make_scene(cfg)
    ds = _device_scene(ng, sc)
    full = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels)
    opts = S.default_options(cfg)
    R = cfg.R_O
    train = S.orbit_cameras(cfg, 16, step_deg=22.5)
    cam_arr, nc = ng.cameras_struct(train, cfg.W, cfg.H)
    n_full = int(full.occ.sum())
    ws = torch.empty(ng.ngprt_dilate_workspace_bytes(R), dtype=torch.uint8, device="cuda")
    for w_thr in (0.0, 0.005):
        vis = torch.zeros(R ** 3, dtype=torch.uint8, device="cuda")
        ng.ngprt_occupancy_visibility(ds.struct, full.struct, cam_arr, nc, None, None, None, nc * cfg.W * cfg.H,
                                      ng.render_opts(opts), w_thr, R, vis)
        dil = torch.empty_like(vis)
        ng.ngprt_dilate(vis, R, 1, dil, ws, mask=full.occ)
        culled = ng.DeviceOcc(dil, R, cfg.n_occ_levels)
        n_cull = int(dil.sum())
        assert 0 < n_cull < 0.8 * n_full, (n_cull, n_full)
        for az in (0.0, 11.25):
            cams = S.orbit_cameras(cfg, 1, azimuth0=az)
            a = ng.Renderer(ds, full).render(opts, cams=cams, W=cfg.W, H=cfg.H, stats=True)
            b = ng.Renderer(ds, culled).render(opts, cams=cams, W=cfg.W, H=cfg.H, stats=True)
            torch.cuda.synchronize()
            psnr = P.psnr(b["rgb"], a["rgb"])
            print(f"w_thr {w_thr} azimuth {az}: {n_cull}/{n_full} voxels, PSNR {psnr:.2f} dB, marching "
                  f"{a['stats'][:, 0].float().mean():.1f} -> {b['stats'][:, 0].float().mean():.1f}, samples "
                  f"{a['stats'][:, 1].float().mean():.2f} -> {b['stats'][:, 1].float().mean():.2f}")
            assert psnr > (50.0 if w_thr == 0.0 else 45.0)
