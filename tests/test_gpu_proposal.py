"""GPU proposal kernels against the oracle: the MLP forward, its loss and gradient,
the weight-interval targets of a plain render, and the fallback pass."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2407_10482_gb300 import scenes as S

pytestmark = pytest.mark.gpu
IN_SCALE, T_SCALE = 3.0, 12.0


@pytest.fixture(scope="module")
def ng():
    from paper_2407_10482_gb300 import ngprt
    ngprt.lib()
    return ngprt


def _w(seed, std=0.4):
    return np.random.default_rng(seed).normal(0, std, O.prop_param_count(32)).astype(np.float32)


@pytest.mark.parametrize("half", [False, True])
def test_propose_forward(ng, half):
    """FP32 weights, and FP16 copies (the oracle takes the same rounded values)."""
    w = _w(0)
    if half:
        w = w.astype(np.float16).astype(np.float32)
    wt = torch.as_tensor(w).cuda()
    o, d = S.random_rays(5000, 1, False)
    iv = torch.empty(5000, 2, device="cuda")
    ah = torch.empty(5000, device="cuda")
    ng.ngprt_propose(wt.half() if half else wt, None, 0, None, torch.as_tensor(o).cuda(), torch.as_tensor(d).cuda(),
                     5000, IN_SCALE, T_SCALE, 0.0, 0.0, 0.0, iv, ah)
    torch.cuda.synchronize()
    ref = O.prop_forward(w, o, d, IN_SCALE, T_SCALE)
    ivn = iv.cpu().numpy()
    ok = ref[:, 1] > ref[:, 0]
    np.testing.assert_allclose(ah.cpu().numpy(), ref[:, 2], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(ivn[ok, 0], ref[ok, 0], rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(ivn[ok, 1], ref[ok, 1], rtol=1e-5, atol=1e-5)
    assert np.all(np.isinf(ivn[~ok]))


def test_propose_loss_and_gradient(ng):
    w = _w(2)
    o, d = S.random_rays(3000, 3, False)
    rng = np.random.default_rng(4)
    tg = np.stack([rng.uniform(1, 3, 3000), rng.uniform(3, 6, 3000), rng.uniform(0, 1, 3000)], 1).astype(np.float32)
    g = torch.zeros(len(w), device="cuda")
    loss = torch.zeros(1, device="cuda")
    ng.ngprt_propose_backward(torch.as_tensor(w).cuda(), None, 0, None, torch.as_tensor(o).cuda(),
                              torch.as_tensor(d).cuda(), 3000, IN_SCALE, T_SCALE, torch.as_tensor(tg).cuda(), g, loss)
    torch.cuda.synchronize()
    L, gr = O.prop_loss_grad(w, o, d, tg, IN_SCALE, T_SCALE)
    assert abs(loss.item() - L) <= 1e-4 * abs(L)
    gn = g.cpu().numpy()
    assert np.abs(gn - gr).max() <= 1e-4 * np.abs(gr).max()


def _scene(ng, cfg):
    sc = S.make_scene(cfg)
    ds = ng.DeviceScene(cfg, sc.tables, sc.coarse, sc.mlp_w)
    docc = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels)
    return sc, ng.Renderer(ds, docc), O.oracle_for_scene(sc)


def test_targets_match_oracle(ng):
    cfg = S.small_config(bounded=False, R_O=32, n_occ_levels=4, t_min=0.05, r_far=16.0, shell=True, mlp_layers=3,
                         mlp_width=64, step_base=2 * 3 ** 0.5 / 256, blob_std=(0.05, 0.15), density_bias=3.0)
    sc, rend, orc = _scene(ng, cfg)
    opts = S.default_options(cfg)
    o, d = S.random_rays(4000, 5, False)
    rays = dict(rays_o=torch.as_tensor(o).cuda(), rays_d=torch.as_tensor(d).cuda())
    out = rend.render(opts, state=True, **rays)
    tg = torch.empty(4000, 3, device="cuda")
    ng.ngprt_proposal_targets(rend.scene.struct, rend.occ.struct, None, 0, None, rays["rays_o"], rays["rays_d"],
                              4000, ng.render_opts(opts), out["state"], tg)
    torch.cuda.synchronize()
    ref = orc.prop_targets(opts, rays_o=o, rays_d=d)
    amb = orc.render(opts, rays_o=o, rays_d=d)["ambiguous"]
    t = tg.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(t[~amb, 2], ref[~amb, 2], atol=1e-4)
    # the crossing sample is an FP decision (FP32 on the GPU, FP64 in the oracle):
    # nearly all rays agree exactly; the rest differ by one sample step
    same = (np.abs(t[:, 0] - ref[:, 0]) < 1e-5) & (np.abs(t[:, 1] - ref[:, 1]) < 1e-5)
    assert same[~amb].mean() > 0.99


def test_interval_then_fallback_matches_oracle(ng):
    cfg = S.small_config(blob_std=(0.05, 0.15), density_bias=2.0)
    sc, rend, orc = _scene(ng, cfg)
    opts = S.default_options(cfg)
    o, d = S.random_rays(3000, 6, True)
    rng = np.random.default_rng(7)
    iv = np.stack([rng.uniform(1.5, 3.0, 3000), rng.uniform(2.5, 4.5, 3000)], 1).astype(np.float32)
    iv[:100] = [-np.inf, np.inf]
    a_hat = rng.uniform(0, 1, 3000).astype(np.float32)
    rays = dict(rays_o=torch.as_tensor(o).cuda(), rays_d=torch.as_tensor(d).cuda())
    ivt, aht = torch.as_tensor(iv).cuda(), torch.as_tensor(a_hat).cuda()
    n = 3000
    state = torch.empty(n, ng.STATE_FLOATS, device="cuda")
    stats = torch.empty(n, 2, dtype=torch.int32, device="cuda")
    ro = ng.render_opts(opts)
    ng.ngprt_render(rend.scene.struct, rend.occ.struct, None, 0, None, rays["rays_o"], rays["rays_d"], n, ivt, ro,
                    None, ray_stats=stats, ray_state=state)
    ng.ngprt_render_fallback(rend.scene.struct, rend.occ.struct, None, 0, None, rays["rays_o"], rays["rays_d"], n,
                             ivt, aht, 0.01, ro, state, stats)
    rgb = torch.empty(n, 3, device="cuda")
    ng.ngprt_shade(rend.scene.struct, state, n, opts.bg, rgb)
    torch.cuda.synchronize()
    ref_iv = orc.render(opts, rays_o=o, rays_d=d, interval=iv)
    full = orc.render(opts, rays_o=o, rays_d=d)
    redo = (a_hat - ref_iv["opacity"] > 0.01) & ~np.all(np.isinf(iv), 1)
    want = np.where(redo[:, None], full["rgb"], ref_iv["rgb"])
    amb = ref_iv["ambiguous"] | full["ambiguous"] | (np.abs(a_hat - ref_iv["opacity"] - 0.01) < 1e-5)
    assert redo.sum() > 100
    err = np.abs(rgb.cpu().numpy()[~amb] - want[~amb]).max()
    assert err <= 1e-4
