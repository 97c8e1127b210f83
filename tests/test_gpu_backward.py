"""GPU reverse pass against the oracle's reverse pass (itself pinned by central
finite differences), through the C ABI and through torch.autograd.

FP32 atomics against FP64: per tensor, |g_gpu - g_oracle| <= 1e-3 |g_oracle| +
3e-5 max|g_oracle|.  Termination is kept away from the threshold (t_term = 0) so
that both sides sum the same samples."""
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


def _close(name, g, ref):
    g = np.asarray(g, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    scale = np.abs(ref).max()
    assert scale > 0, name
    bad = np.abs(g - ref) > 1e-3 * np.abs(ref) + 3e-5 * scale
    assert not bad.any(), f"{name}: {bad.sum()} of {bad.size} differ, worst {np.abs(g - ref).max():.3g} / {scale:.3g}"


def _run(ng, cfg, opts, n_rays=2000, seed=3, sc=None):
    sc = sc or S.make_scene(cfg)
    sc.coarse[:, 8:] *= 10.0
    ds = ng.DeviceScene(cfg, sc.tables, sc.coarse, sc.mlp_w)
    docc = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels)
    rend = ng.Renderer(ds, docc)
    o, d = S.random_rays(n_rays, seed, cfg.bounded)
    rng = np.random.default_rng(seed + 1)
    d_rgb = rng.normal(size=(n_rays, 3)).astype(np.float32)
    d_dep = (0.3 * rng.normal(size=n_rays)).astype(np.float32)
    d_op = rng.normal(size=n_rays).astype(np.float32)
    rays = dict(rays_o=torch.as_tensor(o).cuda(), rays_d=torch.as_tensor(d).cuda())
    out = rend.render(opts, state=True, **rays)
    g_t = torch.zeros_like(ds.tables)
    g_c = torch.zeros_like(ds.coarse)
    g_m = torch.zeros_like(ds.mlp_w)
    rend.backward(opts, out["state"], torch.as_tensor(d_rgb).cuda(), torch.as_tensor(d_dep).cuda(),
                  torch.as_tensor(d_op).cuda(), g_t, g_c, g_m, **rays)
    torch.cuda.synchronize()
    orc = O.oracle_for_scene(sc)
    ref = orc.render_backward(opts, d_rgb=d_rgb, d_depth=d_dep, d_opacity=d_op, rays_o=o, rays_d=d)
    _close("tables", g_t.cpu().numpy(), ref["tables"])
    _close("coarse", g_c.cpu().numpy(), ref["coarse"])
    _close("mlp_w", g_m.cpu().numpy(), ref["mlp_w"])
    return ds, rend, rays, (d_rgb, d_dep, d_op), (g_t, g_c, g_m)


@pytest.mark.parametrize("attn_mode", [0, 1, 2])
def test_backward_small_bounded(ng, attn_mode):
    cfg = S.small_config(blob_std=(0.05, 0.15))
    _run(ng, cfg, S.default_options(cfg, t_term=0.0, attn_mode=attn_mode))


@pytest.mark.parametrize("L,N", [(3, [16, 40, 100]), (8, [16 + 12 * l for l in range(8)])])
def test_backward_three_and_eight_levels(ng, L, N):
    """The paper's L = 3 shape and an 8-level stack (dense and hashed levels mixed)."""
    cfg = S.small_config(L=L, N=N, blob_std=(0.05, 0.15))
    _run(ng, cfg, S.default_options(cfg, t_term=0.0))


def test_backward_unbounded_wide_mlp(ng):
    cfg = S.small_config(bounded=False, R_O=32, n_occ_levels=4, t_min=0.05, r_far=16.0, shell=True, mlp_layers=3,
                         mlp_width=64, step_base=2 * 3 ** 0.5 / 256, blob_std=(0.05, 0.15))
    _run(ng, cfg, S.default_options(cfg, t_term=0.0), n_rays=1500)


def test_backward_hd_levels(ng):
    """The hd workload's 16 levels (5 dense, 11 hashed, T = 2^19), 3-layer MLP."""
    cfg = S.hd_config(density_bias=0.5)
    _run(ng, cfg, S.default_options(cfg, t_term=0.0, max_samples=64), n_rays=512)


def test_autograd_function_matches_direct_call(ng):
    cfg = S.small_config(blob_std=(0.05, 0.15))
    opts = S.default_options(cfg, t_term=0.0)
    ds, rend, rays, cot, grads = _run(ng, cfg, opts)
    t = ds.tables.requires_grad_(True)
    c = ds.coarse.requires_grad_(True)
    m = ds.mlp_w.requires_grad_(True)
    rgb, dep, opa = ng.RenderFunction.apply(t, c, m, rend, opts, rays)
    loss = (rgb * torch.as_tensor(cot[0]).cuda()).sum() + (dep * torch.as_tensor(cot[1]).cuda()).sum() + \
        (opa * torch.as_tensor(cot[2]).cuda()).sum()
    loss.backward()
    for a, b in zip((t.grad, c.grad, m.grad), grads):
        np.testing.assert_allclose(a.cpu().numpy(), b.cpu().numpy(), rtol=1e-4, atol=1e-6)


def agg_kinks_excluded(cfg):
    return cfg.aggregation == 5


def lattice_rays(n, seed):
    """Axis-aligned rays (+-x, +-y, +-z) from distance 3 through points on a 2^-7
    lattice: with lattice_snap and a power-of-two step every sample position is
    exact in FP32 and FP64 alike, so the kernels and the oracle evaluate the
    features at the same points."""
    rng = np.random.default_rng(seed)
    ax = rng.integers(0, 3, n)
    sgn = rng.choice([-1.0, 1.0], n)
    other = rng.integers(-120, 121, (n, 2)) / 128.0
    o = np.zeros((n, 3), np.float32)
    d = np.zeros((n, 3), np.float32)
    for i in range(n):
        rest = [a for a in range(3) if a != ax[i]]
        o[i, ax[i]] = -3.0 * sgn[i]
        d[i, ax[i]] = sgn[i]
        o[i, rest] = other[i]
    return o, d


def _run_agg(ng, cfg, opts, n_rays, seed=5):
    sc = S.make_scene(cfg)
    if sc.coarse.shape[1] > 8:
        sc.coarse[:, 8:] *= 10.0
    if sc.attn_inv is not None:
        sc.attn_inv = sc.attn_inv * 20.0
    ds = ng.DeviceScene(cfg, sc.tables, sc.coarse, sc.mlp_w, attn_inv=sc.attn_inv, agg_mlp=sc.agg_mlp)
    docc = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels)
    rend = ng.Renderer(ds, docc)
    exact = agg_kinks_excluded(cfg)
    o, d = lattice_rays(n_rays, seed) if exact else S.random_rays(n_rays, seed, cfg.bounded)
    rng = np.random.default_rng(seed + 1)
    d_rgb = rng.normal(size=(n_rays, 3)).astype(np.float32)
    d_dep = (0.3 * rng.normal(size=n_rays)).astype(np.float32)
    d_op = rng.normal(size=n_rays).astype(np.float32)
    orc = O.oracle_for_scene(sc)
    if agg_kinks_excluded(cfg):
        # the MLP form's ReLU decisions: on exact sample positions only FP32's own
        # rounding of a hidden pre-activation can put it on the other side of its
        # kink; rays with a unit that close are compared by neither side
        O.set_kink_position_error(0.0)
        kink = orc.render_backward(opts, d_rgb=d_rgb, rays_o=o, rays_d=d)["kink"].astype(bool)
        print(f"tiny-MLP form: {kink.mean():.2%} of {len(kink)} rays at a kink")
        assert kink.mean() < 0.1, kink.mean()
        o, d, d_rgb, d_dep, d_op = (np.ascontiguousarray(a[~kink]) for a in (o, d, d_rgb, d_dep, d_op))
    rays = dict(rays_o=torch.as_tensor(o).cuda(), rays_d=torch.as_tensor(d).cuda())
    out = rend.render(opts, state=True, **rays)
    g_t = torch.zeros_like(ds.tables)
    g_c = torch.zeros_like(ds.coarse)
    g_m = torch.zeros_like(ds.mlp_w)
    g_i = torch.zeros_like(ds.attn_inv) if ds.attn_inv is not None else None
    g_a = torch.zeros_like(ds.agg_mlp) if ds.agg_mlp is not None else None
    rend.backward(opts, out["state"], torch.as_tensor(d_rgb).cuda(), torch.as_tensor(d_dep).cuda(),
                  torch.as_tensor(d_op).cuda(), g_t, g_c, g_m, g_attn_inv=g_i, g_agg_mlp=g_a, **rays)
    torch.cuda.synchronize()
    ref = orc.render_backward(opts, d_rgb=d_rgb, d_depth=d_dep, d_opacity=d_op, rays_o=o, rays_d=d)
    if agg_kinks_excluded(cfg):
        assert not ref["kink"].any()
        O.set_kink_position_error(O.DEFAULT_POSITION_ERROR)
    _close("tables", g_t.cpu().numpy(), ref["tables"])
    _close("coarse", g_c.cpu().numpy(), ref["coarse"])
    _close("mlp_w", g_m.cpu().numpy(), ref["mlp_w"])
    if g_i is not None:
        _close("attn_inv", g_i.cpu().numpy(), ref["attn_inv"])
    if g_a is not None:
        _close("agg_mlp", g_a.cpu().numpy(), ref["agg_mlp"])
    return g_c


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("agg", [1, 2, 3, 4, 5])
def test_backward_aggregation_variants(ng, agg, L):
    """Table 3's forms in their own layouts (one spatial logit per level, constant
    logits, no logits, the tiny MLP with its weight gradient); 2500 rays span 20
    blocks and a ragged last one."""
    cfg = S.small_config(L=L, N=[16, 32, 64, 128][:L] if L == 4 else [24, 96], blob_std=(0.05, 0.15),
                         aggregation=agg)
    g_c = _run_agg(ng, cfg, _agg_opts(cfg), n_rays=2500)
    assert g_c.shape[1] == S.coarse_channels(cfg)


@pytest.mark.parametrize("agg", [1, 3, 5])
def test_backward_aggregation_variants_hd_levels(ng, agg):
    """16 levels (the hd workload's, T = 2^19): 24 coarse channels (SHARED_V), the 16
    shared constant logits summed over the block, and the tiny MLP's 128 inputs (on
    the bounded scene with the hd levels, where its rays have exact positions)."""
    if agg == 5:
        cfg = S.small_config(L=16, N=S.level_resolutions(16, 4096, 16), T_log2=19, blob_std=(0.05, 0.15),
                             aggregation=agg)
        _run_agg(ng, cfg, _agg_opts(cfg, max_samples=24), n_rays=1024)
    else:
        cfg = S.hd_config(density_bias=0.5, aggregation=agg)
        _run_agg(ng, cfg, S.default_options(cfg, t_term=0.0, max_samples=64), n_rays=384)


def _agg_opts(cfg, **kw):
    """Options of the aggregation tests; the tiny-MLP form marches its exact-position
    rays on a 2^-5 lattice."""
    if agg_kinks_excluded(cfg):
        return S.default_options(cfg, t_term=0.0, lattice_snap=True, step_base=2.0 ** -5, t_min=0.0, **kw)
    return S.default_options(cfg, t_term=0.0, **kw)


def test_autograd_function_returns_the_invariant_logits_gradient(ng):
    cfg = S.small_config(blob_std=(0.05, 0.15), aggregation=2)
    sc = S.make_scene(cfg)
    ds = ng.DeviceScene(cfg, sc.tables, sc.coarse, sc.mlp_w, attn_inv=sc.attn_inv)
    docc = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels)
    rend = ng.Renderer(ds, docc)
    o, d = S.random_rays(300, 2, cfg.bounded)
    rays = dict(rays_o=torch.as_tensor(o).cuda(), rays_d=torch.as_tensor(d).cuda())
    opts = S.default_options(cfg, t_term=0.0)
    params = [ds.tables.requires_grad_(), ds.coarse.requires_grad_(), ds.mlp_w.requires_grad_(),
              ds.attn_inv.requires_grad_()]
    rgb, dep, opa = ng.RenderFunction.apply(params[0], params[1], params[2], rend, opts, rays, params[3])
    (rgb.sum() + 0.1 * opa.sum()).backward()
    cot = dict(d_rgb=np.ones((300, 3)), d_depth=np.zeros(300), d_opacity=np.full(300, 0.1))
    ref = O.oracle_for_scene(sc).render_backward(opts, rays_o=o, rays_d=d, **cot)
    _close("attn_inv", ds.attn_inv.grad.cpu().numpy(), ref["attn_inv"])
    _close("coarse", ds.coarse.grad.cpu().numpy(), ref["coarse"])
