"""Pins of the learned-proposal oracle: central differences of its loss, the
output ranges, and the weight-interval targets against a homogeneous slab whose
weights are a geometric sequence (closed form)."""
import math

import numpy as np

from oracle import oracle as O
from paper_2407_10482_gb300 import scenes as S


def _rays(n, seed):
    o, d = S.random_rays(n, seed, False)
    return o, d


def test_proposal_loss_gradient_central_differences():
    rng = np.random.default_rng(0)
    w = rng.normal(0, 0.5, O.prop_param_count(32))
    o, d = _rays(40, 1)
    tg = np.stack([rng.uniform(1, 3, 40), rng.uniform(3, 6, 40), rng.uniform(0, 1, 40)], 1)
    L, g = O.prop_loss_grad(w, o, d, tg, 3.0, 12.0)
    h = 1e-6
    for k in rng.choice(len(w), 40, replace=False):
        wp = w.copy(); wp[k] += h
        wm = w.copy(); wm[k] -= h
        fd = (O.prop_loss_grad(wp, o, d, tg, 3.0, 12.0)[0] - O.prop_loss_grad(wm, o, d, tg, 3.0, 12.0)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 + 1e-4 * abs(g[k])


def test_proposal_outputs_in_range():
    rng = np.random.default_rng(2)
    w = rng.normal(0, 0.5, O.prop_param_count(32))
    o, d = _rays(200, 3)
    out = O.prop_forward(w, o, d, 3.0, 12.0)
    assert np.all((out[:, :2] > 0) & (out[:, :2] < 12.0)) and np.all((out[:, 2] > 0) & (out[:, 2] < 1))


def test_targets_of_a_homogeneous_slab():
    """Constant density over [2, 4] along +x, step 1/64: sample k has weight
    q^k (1-q) with q = exp(-sigma dt), so the 0.5% / 99.5% crossings are at known k."""
    cfg = S.small_config()
    sc = S.make_scene(cfg)
    sc.tables[:] = 0.0
    sc.coarse[:] = 0.0
    sc.coarse[:, 0] = 1.2   # sigma = e^1.2 with all gates at 1/2 and zero fine tables
    sc.occ[:] = 1
    orc = O.oracle_for_scene(sc)
    dt = 1.0 / 64.0
    opts = S.default_options(cfg, step_base=dt, max_samples=1000, t_term=0.0)
    o = np.array([[-3.0, 0.1, 0.2]], np.float32)
    d = np.array([[1.0, 0.0, 0.0]], np.float32)
    t = orc.prop_targets(opts, rays_o=o, rays_d=d)[0]
    sigma = math.exp(float(np.float32(1.2)))  # the table holds the FP32 value
    q = math.exp(-sigma * dt)
    n = 128
    A = 1 - q ** n
    cum = np.cumsum([(1 - q) * q ** k for k in range(n)])
    kn = int(np.argmax(cum > 0.005 * A))
    kf = int(np.argmax(cum >= 0.995 * A))
    assert abs(t[0] - (2.0 + kn * dt)) < 1e-12
    assert abs(t[1] - (2.0 + (kf + 1) * dt)) < 1e-12
    assert abs(t[2] - A) < 1e-12
