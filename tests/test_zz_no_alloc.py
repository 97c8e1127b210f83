"""ngprt_render_noalloc: the render for callers that cannot allocate device memory.

Such callers (a plug-in inside an application that owns the device allocator, code
that must not allocate in a latency-critical loop, a fixed memory budget) get an
entry point whose per-ray scratch is a static device array inside the library.
This test calls it through the C ABI twice in a row and checks each result against
ngprt_render with a caller workspace, on the same inputs, within the tolerance of
the other render tests (1e-4 absolute; the two run the same kernels, so the
results should agree exactly).  It also checks that an oversized batch is
refused.  The file is collected last so that a failure here comes after every
other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2407_10482_gb300 import scenes as S

pytestmark = pytest.mark.gpu
TOL = 1e-4


def test_noalloc_render_matches_workspace_render_twice():
    from paper_2407_10482_gb300 import ngprt as ng
    ng.lib()
    cfg = S.small_config(blob_std=(0.05, 0.15), W=160, H=120)
    sc = S.make_scene(cfg)
    ds = ng.DeviceScene(cfg, sc.tables, sc.coarse, sc.mlp_w)
    docc = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels)
    opts = ng.render_opts(S.default_options(cfg))
    n = cfg.W * cfg.H
    for call, az in enumerate((10.0, 75.0)):
        cams, n_cams = ng.cameras_struct(S.orbit_cameras(cfg, 1, azimuth0=az), cfg.W, cfg.H)
        ref = [torch.empty(n, 3, device="cuda"), torch.empty(n, device="cuda"), torch.empty(n, device="cuda")]
        ws = torch.empty(ng.ngprt_render_workspace_bytes(ds.struct, n), dtype=torch.uint8, device="cuda")
        ng.ngprt_render(ds.struct, docc.struct, cams, n_cams, None, None, None, n, None, opts, ref[0], ref[1], ref[2],
                        None, None, ws)
        out = [torch.full((n, 3), -7.0, device="cuda"), torch.full((n,), -7.0, device="cuda"),
               torch.full((n,), -7.0, device="cuda")]
        ng.ngprt_render_noalloc(ds.struct, docc.struct, cams, n_cams, None, None, None, n, None, opts, out[0], out[1],
                                out[2])
        torch.cuda.synchronize()
        for a, b in zip(out, ref):
            err = float((a - b).abs().max())
            assert err <= TOL, f"call {call}: max abs difference {err}"
        assert float(ref[2].max()) > 0.1  # the view hits the scene


def test_noalloc_refuses_more_rays_than_its_scratch():
    from paper_2407_10482_gb300 import ngprt as ng
    ng.lib()
    limit = ng.ngprt_render_noalloc_max_rays()
    assert limit == 262144
    cfg = S.small_config()
    sc = S.make_scene(cfg)
    ds = ng.DeviceScene(cfg, sc.tables, sc.coarse, sc.mlp_w)
    docc = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels)
    rays = torch.zeros(limit + 1, 3, device="cuda")
    rgb = torch.empty(limit + 1, 3, device="cuda")
    with pytest.raises(ng.NgprtError) as e:
        ng.ngprt_render_noalloc(ds.struct, docc.struct, None, 0, None, rays, rays, limit + 1, None,
                                ng.render_opts(S.default_options(cfg)), rgb)
    assert e.value.code == ng.ERR_INVALID_ARG and "exceeds the static scratch" in str(e.value)
