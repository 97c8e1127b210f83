"""Pins of the oracle's aggregation variants (Table 3) against forms already pinned:
each variant is written as an Eq. 8 scene whose logits make the two identical, so a
wrong channel index, a transposed MLP weight or a missing ReLU fails here."""
from dataclasses import replace

import numpy as np

from oracle import oracle as O
from paper_2407_10482_gb300 import scenes as S


def _pixels(cfg, n=400, seed=9):
    rng = np.random.default_rng(seed)
    return rng.choice(cfg.W * cfg.H, n, replace=False).astype(np.int32)


def _render(scene, opts, pix):
    orc = O.oracle_for_scene(scene)
    return orc.render(opts, cams=S.orbit_cameras(scene.cfg, 1), pix=pix)


def _variant(base: S.Scene, agg: int, coarse, attn_inv=None, agg_mlp=None) -> S.Scene:
    return S.Scene(cfg=replace(base.cfg, aggregation=agg), tables=base.tables, coarse=coarse, mlp_w=base.mlp_w,
                   occ=base.occ, blobs=base.blobs, attn_inv=attn_inv, agg_mlp=agg_mlp)


def _same(a, b, tol=1e-12):
    np.testing.assert_allclose(a["rgb"], b["rgb"], atol=tol)
    np.testing.assert_allclose(a["depth"], b["depth"], atol=tol * 10)
    assert np.array_equal(a["stats"], b["stats"])


def test_sum_variant_equals_gates_fixed_at_one():
    cfg = S.small_config()
    sc = S.make_scene(cfg)
    pix = _pixels(cfg)
    a = _render(sc, S.default_options(cfg, attn_mode=1), pix)
    b = _render(_variant(sc, 4, np.ascontiguousarray(sc.coarse[:, :8])), S.default_options(cfg), pix)
    _same(a, b)


def test_shared_variable_gate_reads_its_own_channel():
    # one logit per level at channel 8 + l equals Eq. 8's shared mode reading omega^l
    cfg = S.small_config()
    sc = S.make_scene(cfg)
    L = cfg.L
    rng = np.random.default_rng(3)
    shared = rng.normal(0.0, 1.0, (sc.coarse.shape[0], L)).astype(np.float32)
    eq8 = sc.coarse.copy()
    eq8[:, 8::2] = shared                 # omega^l
    eq8[:, 9::2] = rng.normal(0.0, 1.0, (sc.coarse.shape[0], L))  # beta^l, unused by mode 2
    a = _render(_variant(sc, 0, eq8), S.default_options(cfg, attn_mode=2), _pixels(cfg))
    b = _render(_variant(sc, 1, np.ascontiguousarray(np.concatenate([sc.coarse[:, :8], shared], 1))),
                S.default_options(cfg), _pixels(cfg))
    _same(a, b)


def test_invariant_gates_equal_a_constant_logit_grid():
    cfg = S.small_config()
    sc = S.make_scene(cfg)
    L = cfg.L
    inv = np.array([0.7, -1.3, 0.2, 2.1, -0.4, 0.9, 1.5, -2.2][:2 * L], np.float64)
    eq8 = sc.coarse.copy()
    eq8[:, 8:] = inv                      # omega^1, beta^1, ... the same at every vertex
    pix = _pixels(cfg)
    a = _render(_variant(sc, 0, eq8), S.default_options(cfg), pix)
    b = _render(_variant(sc, 2, np.ascontiguousarray(sc.coarse[:, :8]), attn_inv=inv), S.default_options(cfg), pix)
    _same(a, b, tol=1e-10)  # trilinear weights of a constant sum to 1 up to rounding
    # the shared invariant form takes omega^l for both modalities
    eq8s = sc.coarse.copy()
    eq8s[:, 8::2] = inv[:L]
    c = _render(_variant(sc, 0, eq8s), S.default_options(cfg, attn_mode=2), pix)
    d = _render(_variant(sc, 3, np.ascontiguousarray(sc.coarse[:, :8]), attn_inv=inv[:L]), S.default_options(cfg),
                pix)
    _same(c, d, tol=1e-10)


def test_mlp_aggregation_reproduces_the_sum():
    # W1 rows j < 8 sum channel j over the levels, rows 8..15 its negative; W2 takes
    # relu(h_j) - relu(-h_j) = h_j: the MLP then equals SUM exactly (up to rounding).
    cfg = S.small_config()
    sc = S.make_scene(cfg)
    L, H = cfg.L, S.AGG_HIDDEN
    w1 = np.zeros((H, 8 * L))
    for l in range(L):
        for k in range(8):
            w1[k, 8 * l + k] = 1.0
            w1[8 + k, 8 * l + k] = -1.0
    w1[16:, :] = np.random.default_rng(5).normal(0.0, 1.0, (H - 16, 8 * L))  # hidden units W2 ignores
    w2 = np.zeros((8, H))
    for k in range(8):
        w2[k, k], w2[k, 8 + k] = 1.0, -1.0
    c8 = np.ascontiguousarray(sc.coarse[:, :8])
    pix = _pixels(cfg)
    a = _render(_variant(sc, 4, c8), S.default_options(cfg), pix)
    b = _render(_variant(sc, 5, c8, agg_mlp=np.concatenate([w1.reshape(-1), w2.reshape(-1)])), S.default_options(cfg),
                pix)
    _same(a, b, tol=1e-12)
    # a transposed level order changes the result (the pin sees the layout)
    w1p = np.zeros_like(w1)
    for l in range(L):
        w1p[:, 8 * l:8 * l + 8] = w1[:, 8 * (L - 1 - l):8 * (L - 1 - l) + 8] * (1.0 + l)
    c = _render(_variant(sc, 5, c8, agg_mlp=np.concatenate([w1p.reshape(-1), w2.reshape(-1)])), S.default_options(cfg),
                pix)
    assert np.abs(c["rgb"] - a["rgb"]).max() > 1e-4


def test_variant_scenes_draw_their_own_layouts():
    for agg, n in ((0, 16), (1, 12), (2, 8), (3, 8), (4, 8), (5, 8)):
        sc = S.make_scene(S.small_config(aggregation=agg))
        assert sc.coarse.shape == (16 ** 3, n)
        assert (sc.attn_inv is not None) == (agg in (2, 3))
        assert (sc.agg_mlp is not None) == (agg == 5)
    # Eq. 8 scenes are unchanged by the variants' extra draws
    a, b = S.make_scene(S.small_config()), S.make_scene(S.small_config(aggregation=0))
    assert np.array_equal(a.tables, b.tables) and np.array_equal(a.coarse, b.coarse)
