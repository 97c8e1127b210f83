"""The block-indexed sparse coarse grid on the GPU: the kept-block mask, the index
and the blocks match the oracle's byte for byte, and renders through the sparse grid
equal renders through the dense one bit for bit (both march engines, FP32 and FP16,
Eq. 8 and a Table 3 layout), hence the oracle within the render tolerance."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from parity import compare_rays
from paper_2407_10482_gb300 import scenes as S

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def ng():
    from paper_2407_10482_gb300 import ngprt
    ngprt.lib()
    return ngprt


BOUNDED = dict(blob_std=(0.05, 0.15), R_C=65)
UNBOUNDED = dict(blob_std=(0.05, 0.15), bounded=False, R_O=64, n_occ_levels=4, t_min=0.05, r_far=16.0, shell=True,
                 R_C=41, step_base=2 * 3 ** 0.5 / 256)


@pytest.mark.parametrize("kw", [BOUNDED, UNBOUNDED, dict(BOUNDED, R_C=9), dict(BOUNDED, R_C=120, R_O=16)])
def test_mask_index_and_blocks_bit_exact(ng, kw):
    cfg = S.small_config(**kw)
    sc = S.make_scene(cfg)
    docc = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels)
    nb = ng.coarse_blocks_per_axis(cfg.R_C)
    mask = torch.empty(nb ** 3, dtype=torch.uint8, device="cuda")
    ng.ngprt_coarse_block_mask(docc.struct, cfg.R_C, mask)
    ref_mask = O.coarse_block_mask(sc.occ, cfg.R_O, cfg.R_C)
    assert np.array_equal(mask.cpu().numpy(), ref_mask)
    assert ref_mask.any()
    if cfg.bounded and cfg.R_C > 9:       # the unbounded scenes' shell reaches every block
        assert not ref_mask.all()
    ds = ng.DeviceScene(cfg, sc.tables, sc.coarse, sc.mlp_w)
    ds.sparsify_coarse(docc)
    torch.cuda.synchronize()
    ref_index, ref_blocks = O.sparse_coarse(sc.coarse, cfg.R_C, ref_mask)
    assert np.array_equal(ds.coarse_index.cpu().numpy(), ref_index)
    assert ds.coarse_blocks == len(ref_blocks)
    assert np.array_equal(ds.coarse.cpu().numpy().view(np.uint32), ref_blocks.view(np.uint32))


def _compare(r_gpu, r_or):
    compare_rays(r_gpu, r_or, TOL)


@pytest.mark.parametrize("kw,table_dtype,agg", [(BOUNDED, 0, 0), (UNBOUNDED, 0, 0), (BOUNDED, 1, 0),
                                                (UNBOUNDED, 2, 0), (BOUNDED, 0, 1), (UNBOUNDED, 0, 3)])
def test_sparse_render_equals_dense_and_the_oracle(ng, kw, table_dtype, agg):
    cfg = S.small_config(**dict(kw, aggregation=agg, W=97, H=61))
    sc = S.make_scene(cfg)
    docc = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels)
    scenes = []
    for sparse in (False, True):
        ds = ng.DeviceScene(cfg, sc.tables, sc.coarse, sc.mlp_w, table_dtype=table_dtype, attn_inv=sc.attn_inv)
        if sparse:
            ds.sparsify_coarse(docc)
        scenes.append(ds)
    assert scenes[1].coarse.numel() < scenes[0].coarse.numel() or cfg.R_C < 50
    n = cfg.W * cfg.H
    cams = S.orbit_cameras(cfg, 2, azimuth0=17.0)
    for opts in (S.default_options(cfg), S.default_options(cfg, use_dist=0, max_samples=9)):
        if True:
            outs = []
            for ds in scenes:
                cam_arr, nc = ng.cameras_struct(cams, cfg.W, cfg.H)
                o = dict(rgb=torch.empty(2 * n, 3, device="cuda"), depth=torch.empty(2 * n, device="cuda"),
                         opacity=torch.empty(2 * n, device="cuda"),
                         stats=torch.empty(2 * n, 2, dtype=torch.int32, device="cuda"))
                ws_bytes = ng.ngprt_render_workspace_bytes(ds.struct, 2 * n)
                ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
                ng.ngprt_render(ds.struct, docc.struct, cam_arr, nc, None, None, None, 2 * n, None,
                                ng.render_opts(opts), o["rgb"], o["depth"], o["opacity"], o["stats"], None, ws)
                outs.append(o)
            torch.cuda.synchronize()
            for k in ("rgb", "depth", "opacity", "stats"):
                assert torch.equal(outs[0][k], outs[1][k]), k
    if table_dtype == 0:
        orc = O.oracle_for_scene(sc)
        pix = np.random.default_rng(3).choice(2 * n, 1500, replace=False).astype(np.int32)
        r_or = orc.render(S.default_options(cfg), cams=cams, pix=pix)
        _compare(_render_pix(ng, scenes[1], docc, S.default_options(cfg), cams, cfg, pix), r_or)


def _render_pix(ng, ds, docc, opts, cams, cfg, pix):
    rend = ng.Renderer(ds, docc)
    return rend.render(opts, cams=cams, W=cfg.W, H=cfg.H, pixel_ids=torch.as_tensor(pix).cuda(), stats=True)


def test_sparse_paper_grid_renders_like_the_dense_one(ng):
    """The paper's 512^3 coarse grid (L = 2: 12 channels, 6.4 GB dense FP32) against its
    sparse form on the 512^3 occupancy: a 1080p frame identical bit for bit, the grid
    a few percent of the dense one."""
    cfg = S.paper_config(2)
    sc = S.make_scene_torch(cfg, device="cuda")
    docc = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels, dist_level=cfg.dist_level)
    dense = ng.DeviceScene(cfg, sc.tables, sc.coarse, sc.mlp_w)
    opts = S.default_options(cfg)
    cams = S.orbit_cameras(cfg, 1)
    ref = ng.Renderer(dense, docc).render(opts, cams=cams, W=cfg.W, H=cfg.H, stats=True)
    ref = {k: v.clone() for k, v in ref.items()}
    sparse = ng.DeviceScene(cfg, sc.tables, sc.coarse, sc.mlp_w)
    del sc
    sparse.sparsify_coarse(docc)
    del dense
    frac = sparse.coarse.numel() / (cfg.R_C ** 3 * S.coarse_channels(cfg))
    print(f"\nsparse coarse grid: {sparse.coarse_blocks} blocks, {frac:.2%} of the dense grid")
    assert frac < 0.5
    out = ng.Renderer(sparse, docc).render(opts, cams=cams, W=cfg.W, H=cfg.H, stats=True)
    torch.cuda.synchronize()
    for k in ("rgb", "depth", "opacity", "stats"):
        assert torch.equal(out[k], ref[k]), k


def test_reverse_pass_refuses_the_sparse_grid(ng):
    cfg = S.small_config(**BOUNDED)
    sc = S.make_scene(cfg)
    docc = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels)
    ds = ng.DeviceScene(cfg, sc.tables, sc.coarse, sc.mlp_w)
    ds.sparsify_coarse(docc)
    rend = ng.Renderer(ds, docc)
    o, d = S.random_rays(64, 1, True)
    rays = dict(rays_o=torch.as_tensor(o).cuda(), rays_d=torch.as_tensor(d).cuda())
    out = rend.render(S.default_options(cfg), state=True, **rays)
    with pytest.raises(RuntimeError, match="dense coarse grid"):
        rend.backward(S.default_options(cfg), out["state"], torch.zeros(64, 3, device="cuda"), None, None,
                      torch.zeros(S.table_entries(cfg), 8, device="cuda"),
                      torch.zeros(cfg.R_C ** 3, S.coarse_channels(cfg), device="cuda"),
                      torch.zeros_like(ds.mlp_w), **rays)
