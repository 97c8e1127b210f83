"""Pins of the oracle's reverse pass: central finite differences of its own FP64
forward (h = 1e-3), per coordinate and along random directions.  Termination is
switched off (t_term = 0) so the sample set cannot change under perturbation, and
densities stay below the exp truncation (sigma_raw < 15)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2407_10482_gb300 import scenes as S

H = 1e-3


def _setup(attn_mode=0, bounded=True):
    if bounded:
        cfg = S.small_config(blob_std=(0.05, 0.15))
        o, d = S.random_rays(12, 11, True)
        kw = {}
    else:
        cfg = S.small_config(blob_std=(0.05, 0.15), bounded=False, R_O=32, n_occ_levels=3,
                             t_min=0.05, r_far=16.0, shell=True, mlp_layers=3, mlp_width=16)
        o, d = S.random_rays(12, 12, False)
        kw = {}
    sc = S.make_scene(cfg)
    sc.coarse[:, 8:] *= 10.0   # spread the attention gates away from 1/2
    orc = O.oracle_for_scene(sc)
    opts = S.default_options(cfg, t_term=0.0, attn_mode=attn_mode, **kw)
    rng = np.random.default_rng(5)
    cot = dict(d_rgb=rng.normal(size=(len(o), 3)), d_depth=rng.normal(size=len(o)) * 0.3,
               d_opacity=rng.normal(size=len(o)))
    return sc, orc, opts, o, d, cot


def _fd(orc, opts, o, d, cot, arr, flat_idx, direction=None, H=H):
    base = arr.reshape(-1)
    keep = base.copy()
    if direction is None:
        base[flat_idx] = keep[flat_idx] + H
        fp = orc.render_dot(opts, rays_o=o, rays_d=d, **cot)
        base[flat_idx] = keep[flat_idx] - H
        fm = orc.render_dot(opts, rays_o=o, rays_d=d, **cot)
    else:
        base[:] = keep + H * direction
        fp = orc.render_dot(opts, rays_o=o, rays_d=d, **cot)
        base[:] = keep - H * direction
        fm = orc.render_dot(opts, rays_o=o, rays_d=d, **cot)
    base[:] = keep
    return (fp - fm) / (2 * H)


@pytest.mark.parametrize("attn_mode,bounded", [(0, True), (2, True), (0, False)])
def test_reverse_pass_matches_central_differences(attn_mode, bounded):
    sc, orc, opts, o, d, cot = _setup(attn_mode, bounded)
    g = orc.render_backward(opts, rays_o=o, rays_d=d, **cot)
    rng = np.random.default_rng(9)
    checked = 0
    for name, arr in (("tables", orc.tables), ("coarse", orc.coarse), ("mlp_w", orc.mlp_w)):
        gr = g[name].reshape(-1)
        nz = np.nonzero(np.abs(gr) > 1e-8)[0]
        assert len(nz) > 0, name
        for k in rng.choice(nz, min(24, len(nz)), replace=False):
            fd = _fd(orc, opts, o, d, cot, arr, k)
            assert abs(fd - gr[k]) <= 1e-6 + 1e-4 * abs(gr[k]), (name, k, fd, gr[k])
            checked += 1
        for _ in range(2):
            v = rng.normal(size=arr.size)
            v /= np.linalg.norm(v)
            fd = _fd(orc, opts, o, d, cot, arr, None, v)
            an = float(gr @ v)
            assert abs(fd - an) <= 1e-6 + 1e-4 * abs(an), (name, fd, an)
    assert checked > 40


def test_loss_uses_each_cotangent_on_its_own_output():
    """render_dot must equal <d_rgb, rgb> + <d_depth, depth> + <d_opacity, A> formed
    from render()'s outputs: catches cotangents handed to the wrong output."""
    sc, orc, opts, o, d, cot = _setup(0, True)
    r = orc.render(opts, rays_o=o, rays_d=d)
    want = (cot["d_rgb"] * r["rgb"]).sum() + (cot["d_depth"] * r["depth"]).sum() + \
        (cot["d_opacity"] * r["opacity"]).sum()
    assert abs(orc.render_dot(opts, rays_o=o, rays_d=d, **cot) - want) < 1e-12 * max(1.0, abs(want))


@pytest.mark.parametrize("which", ["d_rgb", "d_depth", "d_opacity"])
def test_reverse_pass_per_output(which):
    """Central differences with one output's cotangent at a time."""
    sc, orc, opts, o, d, cot = _setup(0, True)
    one = {k: (v if k == which else np.zeros_like(v)) for k, v in cot.items()}
    g = orc.render_backward(opts, rays_o=o, rays_d=d, **one)
    rng = np.random.default_rng(13)
    for name, arr in (("tables", orc.tables), ("coarse", orc.coarse)):
        gr = g[name].reshape(-1)
        v = rng.normal(size=arr.size)
        v /= np.linalg.norm(v)
        fd = _fd(orc, opts, o, d, one, arr, None, v)
        an = float(gr @ v)
        assert abs(fd - an) <= 1e-7 + 1e-4 * abs(an), (which, name, fd, an)
        # density channel alone (the output-specific part of the reverse pass)
        v0 = np.zeros(arr.size)
        v0.reshape(arr.shape)[:, 0] = rng.normal(size=arr.shape[0])
        v0 /= np.linalg.norm(v0)
        fd = _fd(orc, opts, o, d, one, arr, None, v0)
        an = float(gr @ v0)
        assert abs(fd - an) <= 1e-7 + 1e-4 * abs(an), (which, name, "sigma", fd, an)


@pytest.mark.parametrize("agg", [1, 2, 3, 4, 5])
def test_reverse_pass_of_aggregation_variants(agg):
    """Table 3's forms: a per-level logit in the coarse grid (Shared (V)), constant
    logits (both Inv forms, gradient into attn_inv), the plain sum (no logits) and the
    tiny MLP (gradient into its weights W1, W2 and, through them, every level)."""
    cfg = S.small_config(blob_std=(0.05, 0.15), aggregation=agg)
    sc = S.make_scene(cfg)
    if sc.coarse.shape[1] > 8:
        sc.coarse[:, 8:] *= 10.0
    if sc.attn_inv is not None:
        sc.attn_inv = sc.attn_inv * 20.0
    orc = O.oracle_for_scene(sc)
    opts = S.default_options(cfg, t_term=0.0)
    o, d = S.random_rays(12, 11, True)
    rng = np.random.default_rng(21)
    cot = dict(d_rgb=rng.normal(size=(len(o), 3)), d_depth=rng.normal(size=len(o)) * 0.3,
               d_opacity=rng.normal(size=len(o)))
    g = orc.render_backward(opts, rays_o=o, rays_d=d, **cot)
    # the MLP's reverse pass does not depend on the gate form (pinned above); only the
    # parameters that feed the gated features are checked here
    names = [("tables", orc.tables), ("coarse", orc.coarse)]
    if orc.attn_inv is not None:
        names.append(("attn_inv", orc.attn_inv))
    else:
        assert g["attn_inv"] is None
    if orc.agg_mlp is not None:
        names.append(("agg_mlp", orc.agg_mlp))
    for name, arr in names:
        gr = g[name].reshape(-1)
        nz = np.nonzero(np.abs(gr) > 1e-8)[0]
        assert len(nz) > 0, name
        # the MLP form's ReLUs put kinks within 1e-3 of some weights: a step shorter
        # than the distance to them
        h = 1e-5 if agg == 5 else H
        for k in rng.choice(nz, min(12, len(nz)), replace=False):
            fd = _fd(orc, opts, o, d, cot, arr, k, H=h)
            assert abs(fd - gr[k]) <= 1e-6 + 1e-4 * abs(gr[k]), (name, k, fd, gr[k])
        v = rng.normal(size=arr.size)
        v /= np.linalg.norm(v)
        fd = _fd(orc, opts, o, d, cot, arr, None, v, H=h)
        an = float(gr @ v)
        assert abs(fd - an) <= 1e-6 + 1e-4 * abs(an), (name, fd, an)
    if agg == 1:
        # one logit per level: the channels past 8 + L do not exist, and every level's
        # logit receives gradient somewhere
        assert g["coarse"].shape[1] == 8 + cfg.L
        assert np.all(np.abs(g["coarse"][:, 8:]).sum(0) > 0)
    if agg == 4:
        assert g["coarse"].shape[1] == 8


def test_mlp_form_flags_rays_at_a_relu_kink():
    """A hidden unit whose W1 row is zero sits exactly at its kink for every sample:
    every ray with samples is flagged; with the generated weights and exact positions
    most rays are not, and allowing for a position error only adds flagged rays."""
    cfg = S.small_config(blob_std=(0.05, 0.15), aggregation=5)
    sc = S.make_scene(cfg)
    o, d = S.random_rays(200, 3, True)
    opts = S.default_options(cfg, t_term=0.0)
    cot = dict(d_rgb=np.ones((len(o), 3)))
    orc = O.oracle_for_scene(sc)
    try:
        O.set_kink_position_error(0.0)
        k_gen = orc.render_backward(opts, rays_o=o, rays_d=d, **cot)["kink"].astype(bool)
        stats = orc.render(opts, rays_o=o, rays_d=d)["stats"]
        assert k_gen.mean() < 0.2
        O.set_kink_position_error(O.DEFAULT_POSITION_ERROR)
        k_pos = orc.render_backward(opts, rays_o=o, rays_d=d, **cot)["kink"].astype(bool)
        assert np.all(k_pos[k_gen]) and k_pos.sum() > k_gen.sum()
        O.set_kink_position_error(0.0)
        nx = 8 * cfg.L
        orc.agg_mlp[5 * nx:6 * nx] = 0.0             # hidden unit 5: h = 0 at every sample
        k_zero = orc.render_backward(opts, rays_o=o, rays_d=d, **cot)["kink"]
        assert np.array_equal(k_zero.astype(bool), stats[:, 1] > 0)
    finally:
        O.set_kink_position_error(O.DEFAULT_POSITION_ERROR)
