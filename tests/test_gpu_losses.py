"""GPU parity of the training losses and controls (Sec. S2.4, Eq. S2, Eq. S3) with
the oracle, through the C ABI: Huber loss and gradient, the per-ray distortion
regulariser and its reverse pass, the sample-count mean of the step auto-tune."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2407_10482_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ng():
    from paper_2407_10482_gb300 import ngprt
    ngprt.lib()
    return ngprt


@pytest.mark.parametrize("n", [1, 777, 3 * 262144])
def test_huber_loss(ng, n):
    rng = np.random.default_rng(n)
    a = rng.uniform(0, 1, n).astype(np.float32)
    b = rng.uniform(0, 1, n).astype(np.float32)
    loss = torch.zeros(1, device="cuda")
    d = torch.empty(n, device="cuda")
    scale = 1.0 / n
    ng.ngprt_huber_loss(torch.as_tensor(a).cuda(), torch.as_tensor(b).cuda(), n, 0.1, scale, loss, d)
    torch.cuda.synchronize()
    L, dref = O.huber_loss(a, b, np.float32(0.1))
    assert abs(loss.item() - scale * L) <= 1e-5 * max(1e-6, scale * L)
    np.testing.assert_allclose(d.cpu().numpy(), scale * dref, rtol=1e-6, atol=1e-12)


def test_mean_samples(ng):
    st = np.random.default_rng(3).integers(0, 300, (100003, 2)).astype(np.int32)
    out = torch.empty(1, device="cuda")
    ng.ngprt_mean_samples(torch.as_tensor(st).cuda(), len(st), out)
    torch.cuda.synchronize()
    assert abs(out.item() - st[:, 1].mean()) < 1e-4 * st[:, 1].mean()


def _scene(ng, cfg):
    sc = S.make_scene(cfg)
    sc.coarse[:, 8:] *= 10.0
    ds = ng.DeviceScene(cfg, sc.tables, sc.coarse, sc.mlp_w)
    docc = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels)
    orc = O.Oracle(cfg, sc.tables, sc.coarse, sc.mlp_w, O.build_pyramid(sc.occ, cfg.R_O, cfg.n_occ_levels),
                   O.occ_dist(sc.occ, cfg.R_O))
    return sc, ds, docc, orc


@pytest.mark.parametrize("cfg_name", ["small", "hd"])
def test_distortion_loss_per_ray(ng, cfg_name):
    cfg = S.small_config(blob_std=(0.05, 0.15)) if cfg_name == "small" else S.hd_config()
    sc, ds, docc, orc = _scene(ng, cfg)
    opts = S.default_options(cfg, t_term=0.0) if cfg_name == "small" else S.default_options(cfg)
    cams = S.orbit_cameras(cfg, 1, azimuth0=30.0)
    cam_arr, nc = ng.cameras_struct(cams, cfg.W, cfg.H)
    if cfg_name == "small":
        pix = np.arange(cfg.W * cfg.H, dtype=np.int32)
    else:
        pix = np.random.default_rng(1).choice(cfg.W * cfg.H, 1500, replace=False).astype(np.int32)
    n = len(pix)
    out = torch.empty(n, 4, device="cuda")
    loss = torch.zeros(1, device="cuda")
    ng.ngprt_distortion_loss(ds.struct, docc.struct, cam_arr, nc, torch.as_tensor(pix).cuda(), None, None, n,
                             ng.render_opts(opts), 0.5, out, loss)
    torch.cuda.synchronize()
    ref = orc.distortion(opts, cams=cams, pix=pix)
    amb = orc.render(opts, cams=cams, pix=pix)["ambiguous"]
    # rays whose march FP32 may decide otherwise (flagged by the FP64 oracle) are
    # compared by neither side
    assert amb.mean() <= 0.02, amb.mean()
    g = out.cpu().numpy().astype(np.float64)
    ok = ~amb
    tol = 1e-4 * max(1.0, np.abs(ref[:, 0]).max())
    assert np.abs(g[ok, 0] - ref[ok, 0]).max() <= tol
    assert np.abs(g[ok, 1] - ref[ok, 1]).max() <= 1e-4
    assert np.abs(g[ok, 2] - ref[ok, 2]).max() <= 1e-4 * max(1.0, np.abs(ref[:, 2]).max())
    assert abs(loss.item() - 0.5 * g[:, 0].sum()) <= 1e-4 * max(1.0, 0.5 * g[:, 0].sum())
    assert (ref[:, 0] > 0).sum() > n // 10


@pytest.mark.parametrize("attn_mode,L", [(0, 4), (1, 4), (2, 4), (0, 3), (0, 8)])
def test_distortion_backward(ng, attn_mode, L):
    N = {3: [16, 40, 100], 4: [16, 32, 64, 128], 8: [16 + 12 * l for l in range(8)]}[L]
    cfg = S.small_config(blob_std=(0.05, 0.15), L=L, N=N)
    sc, ds, docc, orc = _scene(ng, cfg)
    opts = S.default_options(cfg, t_term=0.0, attn_mode=attn_mode)
    o, d = S.random_rays(4096, 21, True)
    ot, dt = torch.as_tensor(o).cuda(), torch.as_tensor(d).cuda()
    ro = ng.render_opts(opts)
    n = len(o)
    state = torch.empty(n, 4, device="cuda")
    ng.ngprt_distortion_loss(ds.struct, docc.struct, None, 0, None, ot, dt, n, ro, 1.0, state)
    g_t = torch.zeros_like(ds.tables)
    g_c = torch.zeros_like(ds.coarse)
    scale = 1.0 / n
    ng.ngprt_distortion_backward(ds.struct, docc.struct, None, 0, None, ot, dt, n, ro, state, scale, g_t, g_c)
    torch.cuda.synchronize()
    rt, rc = orc.distortion_backward(opts, scale, rays_o=o, rays_d=d)
    for got, ref in ((g_t.cpu().numpy(), rt), (g_c.cpu().numpy(), rc)):
        err = np.abs(got.astype(np.float64) - ref).max()
        assert err <= 2e-4 * np.abs(ref).max() + 1e-9, (err, np.abs(ref).max())
    assert np.abs(rt).max() > 0


@pytest.mark.parametrize("agg", [1, 2, 3, 4, 5])
def test_distortion_loss_and_backward_of_the_aggregation_forms(ng, agg):
    """Eq. S2 through Table 3's other forms: per-ray values and the density path's
    gradients (logits, constant logits, the tiny MLP's weights) against the oracle."""
    cfg = S.small_config(blob_std=(0.05, 0.15), aggregation=agg)
    sc = S.make_scene(cfg)
    if sc.coarse.shape[1] > 8:
        sc.coarse[:, 8:] *= 10.0
    if sc.attn_inv is not None:
        sc.attn_inv = sc.attn_inv * 20.0
    ds = ng.DeviceScene(cfg, sc.tables, sc.coarse, sc.mlp_w, attn_inv=sc.attn_inv, agg_mlp=sc.agg_mlp)
    docc = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels)
    orc = O.oracle_for_scene(sc)
    opts = S.default_options(cfg, t_term=0.0)
    o, d = S.random_rays(3000, 23, True)
    if agg == 5:     # the MLP form's ReLU decisions (see the render's reverse-pass parity)
        kink = orc.render_backward(opts, d_rgb=np.ones((len(o), 3)), rays_o=o, rays_d=d)["kink"].astype(bool)
        o, d = np.ascontiguousarray(o[~kink]), np.ascontiguousarray(d[~kink])
    n = len(o)
    ot, dt = torch.as_tensor(o).cuda(), torch.as_tensor(d).cuda()
    ro = ng.render_opts(opts)
    state = torch.empty(n, 4, device="cuda")
    ng.ngprt_distortion_loss(ds.struct, docc.struct, None, 0, None, ot, dt, n, ro, 1.0, state)
    torch.cuda.synchronize()
    ref_fwd = orc.distortion(opts, rays_o=o, rays_d=d)
    g_fwd = state.cpu().numpy().astype(np.float64)
    assert np.abs(g_fwd[:, 0] - ref_fwd[:, 0]).max() <= 1e-4 * max(1.0, np.abs(ref_fwd[:, 0]).max())
    g_t = torch.zeros_like(ds.tables)
    g_c = torch.zeros_like(ds.coarse)
    g_i = torch.zeros_like(ds.attn_inv) if ds.attn_inv is not None else None
    g_a = torch.zeros_like(ds.agg_mlp) if ds.agg_mlp is not None else None
    need = ng.ngprt_distortion_backward_workspace_bytes(ds.struct, ro, n)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda") if need else None
    scale = 1.0 / n
    ng.ngprt_distortion_backward(ds.struct, docc.struct, None, 0, None, ot, dt, n, ro, state, scale, g_t, g_c,
                                 g_attn_inv=g_i, g_agg_mlp=g_a, workspace=ws)
    torch.cuda.synchronize()
    ref = orc.distortion_backward(opts, scale, rays_o=o, rays_d=d, full=True)
    pairs = [(g_t, ref["tables"]), (g_c, ref["coarse"])]
    pairs += [(g, ref[k]) for g, k in ((g_i, "attn_inv"), (g_a, "agg_mlp")) if g is not None]
    for got, r in pairs:
        err = np.abs(got.cpu().numpy().astype(np.float64) - r).max()
        assert err <= 2e-4 * np.abs(r).max() + 1e-9, (err, np.abs(r).max())
        assert np.abs(r).max() > 0
