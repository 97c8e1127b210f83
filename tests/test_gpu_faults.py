"""Failure handling on the GPU without faulting it: NaN and Inf injected into the
scene's tables (the render completes, the affected rays are flagged by the
non-finite count, a clean scene renders as before) and a bounded wait that runs out
(reported by ngprt_sync_status as a timeout, with the context still usable)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2407_10482_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ng():
    from paper_2407_10482_gb300 import ngprt
    ngprt.lib()
    return ngprt


def _render(ng, cfg, tables, coarse, sc, docc):
    ds = ng.DeviceScene(cfg, tables, coarse, sc.mlp_w)
    r = ng.Renderer(ds, docc).render(S.default_options(cfg), cams=S.orbit_cameras(cfg, 1), W=cfg.W, H=cfg.H,
                                     stats=True)
    ng.ngprt_sync_status()
    return r


@pytest.mark.parametrize("what", ["nan_table", "inf_coarse"])
def test_nonfinite_scene_values_are_flagged_not_fatal(ng, what):
    cfg = S.small_config(blob_std=(0.05, 0.15))
    sc = S.make_scene(cfg)
    docc = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels)
    clean = _render(ng, cfg, sc.tables, sc.coarse, sc, docc)
    t, c = sc.tables.copy(), sc.coarse.copy()
    if what == "nan_table":
        t[4096 + 2000:4096 + 4000, 0] = np.nan          # density of part of level 1
    else:
        c[1000:1400, 1] = np.inf                           # one colour channel of some vertices
    bad = _render(ng, cfg, t, c, sc, docc)
    n = cfg.W * cfg.H
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    ng.ngprt_count_nonfinite(bad["rgb"], 3 * n, cnt)
    torch.cuda.synchronize()
    k = int(cnt.item())
    assert 0 < k < 3 * n, k
    # every ray still ended within its caps
    st = bad["stats"].cpu().numpy()
    assert st[:, 0].max() <= cfg.max_march and st[:, 1].max() <= cfg.max_samples
    # the context is healthy: the clean scene renders exactly as before
    again = _render(ng, cfg, sc.tables, sc.coarse, sc, docc)
    assert torch.equal(again["rgb"], clean["rgb"])
    ng.ngprt_count_nonfinite(again["rgb"], 3 * n, cnt)
    torch.cuda.synchronize()
    assert int(cnt.item()) == 0


def test_bounded_wait_timeout_is_reported(ng):
    ng.ngprt_sync_status()                                   # nothing pending
    ng.ngprt_test_bounded_wait(256)
    with pytest.raises(ng.NgprtError) as e:
        ng.ngprt_sync_status()
    assert e.value.code == ng.ERR_TIMEOUT
    ng.ngprt_sync_status()                                   # reported once, then clear
    # the GPU keeps working, including the tensor-core MLP that shares the flag
    cfg = S.small_config(mlp_layers=2, mlp_width=16)
    sc = S.make_scene(cfg)
    ds = ng.DeviceScene(cfg, sc.tables, sc.coarse, sc.mlp_w, mlp_dtype=1)
    docc = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels)
    ng.Renderer(ds, docc).render(S.default_options(cfg), cams=S.orbit_cameras(cfg, 1), W=cfg.W, H=cfg.H)
    ng.ngprt_sync_status()
    assert ng.lib().ngprt_tensor_core_error() == 0
