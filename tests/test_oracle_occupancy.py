"""Pins of the oracle's occupancy pipeline (Sec. S2.5): box dilation against scipy's
maximum filter, density occupancy against the closed form of an affine density
logit, visibility marks against the per-sample dump of the march."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2407_10482_gb300 import scenes as S

ndimage = pytest.importorskip("scipy.ndimage")


@pytest.mark.parametrize("R,r,frac,seed", [(12, 1, 0.02, 0), (12, 2, 0.01, 1), (9, 3, 0.05, 2), (16, 0, 0.1, 3)])
def test_dilate_equals_maximum_filter(R, r, frac, seed):
    occ = (np.random.default_rng(seed).uniform(size=R ** 3) < frac).astype(np.uint8)
    want = ndimage.maximum_filter(occ.reshape(R, R, R), size=2 * r + 1, mode="constant", cval=0).reshape(-1)
    assert np.array_equal(O.dilate(occ, R, r), want)


def test_dilate_mask_clears_outside():
    R = 12
    rng = np.random.default_rng(4)
    occ = (rng.uniform(size=R ** 3) < 0.02).astype(np.uint8)
    mask = (rng.uniform(size=R ** 3) < 0.5).astype(np.uint8)
    assert np.array_equal(O.dilate(occ, R, 1, mask), O.dilate(occ, R, 1) & mask)


def test_dilate_single_voxel_is_a_clipped_box():
    R = 10
    occ = np.zeros(R ** 3, np.uint8)
    occ[1 + R * (8 + R * 5)] = 1           # x = 1, y = 8, z = 5
    out = O.dilate(occ, R, 2).reshape(R, R, R)   # [z][y][x]
    zz, yy, xx = np.nonzero(out)
    assert (xx.min(), xx.max(), yy.min(), yy.max(), zz.min(), zz.max()) == (0, 3, 6, 9, 3, 7)
    assert out.sum() == 4 * 4 * 5


def _affine_density_scene(cfg, coef):
    sc = S.make_scene(cfg)
    sc.tables[:] = 0.0
    sc.coarse[:] = 0.0
    R = cfg.R_C
    g = np.arange(R, dtype=np.float64) / (R - 1)   # vertex positions in the unit cube
    zz, yy, xx = np.meshgrid(g, g, g, indexing="ij")
    sc.coarse[:, 0] = (coef[0] + coef[1] * xx + coef[2] * yy + coef[3] * zz).reshape(-1)
    return sc


def test_density_occupancy_of_an_affine_logit():
    cfg = S.small_config()
    coef = (-1.0, 2.0, -0.5, 1.25)
    sc = _affine_density_scene(cfg, coef)
    orc = O.oracle_for_scene(sc)
    R, thr = 16, 1.3
    occ, sig = orc.occupancy_density(S.default_options(cfg), R, thr)
    c = (np.arange(R) + 0.5) / R
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    want = np.exp(coef[0] + coef[1] * xx + coef[2] * yy + coef[3] * zz).reshape(-1)
    # the coarse grid stores the affine values in FP32
    np.testing.assert_allclose(sig, want, rtol=1e-6)
    sure = np.abs(want - thr) > 1e-5 * thr
    assert np.array_equal(occ[sure], (want > thr)[sure])
    assert 0 < occ.sum() < R ** 3


def test_visibility_marks_the_voxels_of_heavy_samples():
    cfg = S.small_config()
    sc = S.make_scene(cfg)
    orc = O.oracle_for_scene(sc)
    opts = S.default_options(cfg)
    o, d = S.random_rays(24, 6, True)
    R, thr = 32, 0.01
    vis, wmax = orc.occupancy_visibility(opts, R, thr, rays_o=o, rays_d=d)
    want = np.zeros(R ** 3, np.uint8)
    wm = np.zeros(R ** 3)
    n_heavy = 0
    for i in range(len(o)):
        smp = orc.ray_samples(opts, o[i], d[i])
        for t, delta, u0, u1, u2, sigma, w in smp:
            ix = [min(max(math.floor(np.float32(u) * np.float32(R)), 0), R - 1) for u in (u0, u1, u2)]
            v = ix[0] + R * (ix[1] + R * ix[2])
            wm[v] = max(wm[v], w)
            if w > thr:
                want[v] = 1
                n_heavy += 1
    assert n_heavy > 20
    assert np.array_equal(vis, want)
    np.testing.assert_allclose(wmax, wm, rtol=0, atol=0)
