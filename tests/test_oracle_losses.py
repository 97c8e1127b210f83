"""Pins of the oracle's training losses and controls (Sec. S2.4, Eq. S2, Eq. S3):
the Huber loss by its closed form, the step auto-tune by the geometric sequence it
produces, the distortion regulariser by the closed-form weights of a homogeneous
slab and by the exponential distribution's mean absolute difference, and its
reverse pass by central differences of the oracle's own forward."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2407_10482_gb300 import scenes as S

H = 1e-3


def test_huber_closed_form():
    x = np.array([0.0, 0.05, -0.05, 0.1, -0.3, 2.0])
    y = np.zeros_like(x)
    L, d = O.huber_loss(x, y, 0.1)
    want = 0.5 * 0.05 ** 2 * 2 + 0.5 * 0.1 ** 2 + 0.1 * (0.3 - 0.05) + 0.1 * (2.0 - 0.05)
    assert abs(L - want) < 1e-15
    np.testing.assert_array_equal(d, [0.0, 0.05, -0.05, 0.1, -0.1, 0.1])
    # quadratic region: half the squared error; the derivative by central differences
    r = np.random.default_rng(1).uniform(-0.5, 0.5, 50)
    z = np.zeros(50)
    for i in range(5):
        e = np.zeros(50)
        e[i] = 1e-6
        fd = (O.huber_loss(r + e, z, 0.2)[0] - O.huber_loss(r - e, z, 0.2)[0]) / 2e-6
        assert abs(fd - O.huber_loss(r, z, 0.2)[1][i]) < 1e-6
    small = r[np.abs(r) <= 0.2]
    assert abs(O.huber_loss(small, np.zeros_like(small), 0.2)[0] - 0.5 * (small ** 2).sum()) < 1e-15


def test_step_autotune_sequences():
    g = 1.0
    for k in range(1, 2001):
        g = O.step_autotune(g, 2.0)             # below N_min = 3: shrink
        assert abs(g - max(0.2217, 0.999 ** k)) < 1e-12
    assert g == 0.2217                          # the floor holds (0.999^2000 = 0.135)
    for k in range(1, 10):
        g = O.step_autotune(g, 3.0)             # at N_min: grow
    assert abs(g - 0.2217 * 1.001 ** 9) < 1e-12
    assert O.step_autotune(0.9995, 5.0) == 1.0  # capped at 1


def _slab(sigma_table, coarse_sigma, attn_logit=0.0):
    cfg = S.small_config()
    sc = S.make_scene(cfg)
    sc.tables[:] = 0.0
    sc.tables[:, 0] = sigma_table
    sc.coarse[:] = attn_logit
    sc.coarse[:, 0] = coarse_sigma
    sc.occ[:] = 1
    return cfg, sc


def test_distortion_of_a_homogeneous_slab():
    # ray along +x through the box: 128 samples of step 1/64 at t = 2 + i/64, constant
    # sigma, no termination.  Closed-form weights w_i = q^i (1 - q), q = exp(-sigma/64).
    L = 4
    s = np.float32(0.05)
    cfg, sc = _slab(s, s, attn_logit=60.0)   # gates = 1: sigma_raw = 5 s
    orc = O.oracle_for_scene(sc)
    opts = S.default_options(cfg, step_base=1.0 / 64.0, max_samples=1000, t_term=0.0)
    o = np.array([[-3.0, 0.1, 0.2]], np.float32)
    d = np.array([[1.0, 0.0, 0.0]], np.float32)
    out = orc.distortion(opts, rays_o=o, rays_d=d)[0]
    sigma = math.exp(float(s) * (1 + L))
    q = math.exp(-sigma / 64.0)
    w = np.array([q ** i * (1 - q) for i in range(128)])
    m = (np.arange(128) + 0.5) / 64.0
    pair = sum(w[i] * w[j] * abs(m[i] - m[j]) for i in range(128) for j in range(128))
    self_ = (w ** 2).sum() / 64.0 / 3.0
    assert abs(out[0] - (pair + self_)) < 1e-12
    assert abs(out[1] - w.sum()) < 1e-12
    assert abs(out[2] - (w * (2.0 + m)).sum()) < 1e-12


def test_distortion_tends_to_the_exponential_mean_difference():
    # an opaque slab with fine steps: the weights approach sigma e^{-sigma t}, whose
    # mean absolute difference between two independent draws is 1 / sigma
    s = np.float32(1.5)
    cfg, sc = _slab(np.float32(0.0), s, attn_logit=0.0)
    orc = O.oracle_for_scene(sc)
    opts = S.default_options(cfg, step_base=1.0 / 2048.0, max_samples=10000, max_march=10000, t_term=0.0)
    out = orc.distortion(opts, rays_o=np.array([[-3.0, 0.1, 0.2]], np.float32),
                         rays_d=np.array([[1.0, 0.0, 0.0]], np.float32))[0]
    sigma = math.exp(float(s))
    assert out[1] > 0.9998                                 # opaque over the 2 units
    assert abs(out[0] - 1.0 / sigma) < 0.01 / sigma


@pytest.mark.parametrize("attn_mode", [0, 2])
def test_distortion_gradient_matches_central_differences(attn_mode):
    cfg = S.small_config(blob_std=(0.05, 0.15))
    sc = S.make_scene(cfg)
    sc.coarse[:, 8:] *= 10.0
    orc = O.oracle_for_scene(sc)
    opts = S.default_options(cfg, t_term=0.0, attn_mode=attn_mode)
    o, d = S.random_rays(10, 13, True)
    scale = 0.7

    def loss():
        return scale * orc.distortion(opts, rays_o=o, rays_d=d)[:, 0].sum()
    g_t, g_c = orc.distortion_backward(opts, scale, rays_o=o, rays_d=d)
    rng = np.random.default_rng(2)
    checked = 0
    for arr, g, chans in ((orc.tables, g_t, [0]), (orc.coarse, g_c, [0, 8, 10])):
        flat = arr.reshape(-1)
        nz = [i for i in np.flatnonzero(np.abs(g.reshape(-1)) > 1e-6) if i % arr.shape[1] in chans]
        for i in rng.choice(nz, min(12, len(nz)), replace=False):
            keep = flat[i]
            flat[i] = keep + H
            fp = loss()
            flat[i] = keep - H
            fm = loss()
            flat[i] = keep
            fd = (fp - fm) / (2 * H)
            assert abs(fd - g.reshape(-1)[i]) < 1e-5 + 1e-4 * abs(fd), (i, fd, g.reshape(-1)[i])
            checked += 1
    assert checked >= 20
    # colour channels get no distortion gradient
    assert np.all(g_t[:, 1:] == 0) and np.all(g_c[:, 1:8] == 0)


@pytest.mark.parametrize("agg", [1, 2, 3, 4, 5])
def test_distortion_gradient_of_the_aggregation_forms(agg):
    """Eq. S2's gradient through Table 3's other forms (the density path of each: its
    gate logits, constant logits or the tiny MLP), by central differences along random
    directions and on single coordinates."""
    cfg = S.small_config(blob_std=(0.05, 0.15), aggregation=agg)
    sc = S.make_scene(cfg)
    if sc.coarse.shape[1] > 8:
        sc.coarse[:, 8:] *= 10.0
    if sc.attn_inv is not None:
        sc.attn_inv = sc.attn_inv * 20.0
    orc = O.oracle_for_scene(sc)
    opts = S.default_options(cfg, t_term=0.0)
    o, d = S.random_rays(10, 13, True)
    scale = 0.7
    h = 1e-5 if agg == 5 else H     # the MLP's ReLU kinks: a step shorter than the distance to them

    def loss():
        return scale * orc.distortion(opts, rays_o=o, rays_d=d)[:, 0].sum()
    g = orc.distortion_backward(opts, scale, rays_o=o, rays_d=d, full=True)
    rng = np.random.default_rng(agg)
    names = [("tables", orc.tables), ("coarse", orc.coarse)]
    names += [(k, getattr(orc, k)) for k in ("attn_inv", "agg_mlp") if getattr(orc, k) is not None]
    for name, arr in names:
        flat = arr.reshape(-1)
        gr = g[name].reshape(-1)
        nz = np.flatnonzero(np.abs(gr) > 1e-7)
        assert len(nz) > 0, name
        for i in rng.choice(nz, min(8, len(nz)), replace=False):
            keep = flat[i]
            flat[i] = keep + h
            fp = loss()
            flat[i] = keep - h
            fm = loss()
            flat[i] = keep
            fd = (fp - fm) / (2 * h)
            assert abs(fd - gr[i]) < 1e-5 + 1e-4 * abs(fd), (name, i, fd, gr[i])
        v = rng.normal(size=flat.size)
        v /= np.linalg.norm(v)
        keep = flat.copy()
        flat[:] = keep + h * v
        fp = loss()
        flat[:] = keep - h * v
        fm = loss()
        flat[:] = keep
        an = float(gr @ v)
        assert abs((fp - fm) / (2 * h) - an) < 1e-5 + 1e-4 * abs(an), (name, an)
    if agg != 5:       # only the density channels carry the regulariser's gradient
        assert np.all(g["tables"][:, 1:] == 0) and np.all(g["coarse"][:, 1:8] == 0)
