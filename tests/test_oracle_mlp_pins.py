"""Pins of the oracle's two MLPs by weights that make them exact linear maps: hidden
unit pairs carry +x_k and -x_k, so relu(x_k) - relu(-x_k) = x_k.  With a random
readout matrix a, the deferred MLP_psi (Eq. 5; [out][in] layouts, ReLU on the
hidden layers only, 23 real inputs of 32) must equal a x, and the proposal MLP
(with biases) must equal sigmoid(a e + b).  A transposed matrix, a misplaced or
missing ReLU, a wrong input slot or a dropped bias fails these."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2407_10482_gb300 import scenes as S


def _pair_rows(n_in, width):
    """W0 [width][32] whose rows 2k, 2k+1 pick +x_k, -x_k for k < n_in."""
    w0 = np.zeros((width, S.MLP_IN_PAD))
    for k in range(n_in):
        w0[2 * k, k], w0[2 * k + 1, k] = 1.0, -1.0
    return w0


@pytest.mark.parametrize("layers,width,n_in", [(3, 64, 23), (2, 16, 8)])
def test_deferred_mlp_is_an_exact_linear_map(layers, width, n_in):
    cfg = S.small_config(mlp_layers=layers, mlp_width=width)
    sc = S.make_scene(cfg)
    rng = np.random.default_rng(3)
    a = rng.normal(0, 1, (3, n_in)).astype(np.float32).astype(np.float64)  # exactly as stored
    w0 = _pair_rows(n_in, width)
    read = np.zeros((3, width))
    for k in range(n_in):
        read[:, 2 * k], read[:, 2 * k + 1] = a[:, k], -a[:, k]
    mats = [w0] + ([np.eye(width)] if layers == 3 else []) + [read]   # identity keeps h >= 0 unchanged
    sc.mlp_w = np.concatenate([m.reshape(-1) for m in mats]).astype(np.float32)
    orc = O.oracle_for_scene(sc)
    x = np.zeros((50, S.MLP_IN_PAD))
    x[:, :n_in] = rng.normal(0, 1, (50, n_in))
    np.testing.assert_allclose(orc.mlp(x), x[:, :n_in] @ a.T, atol=1e-12)
    # the readout sees relu'd hidden units: dropping the -x_k rows halves nothing but
    # leaves only the positive parts
    mats[0] = np.where(mats[0] > 0, mats[0], 0.0)
    sc.mlp_w = np.concatenate([m.reshape(-1) for m in mats]).astype(np.float32)
    y = O.oracle_for_scene(sc).mlp(x)
    np.testing.assert_allclose(y, np.maximum(x[:, :n_in], 0) @ a.T, atol=1e-12)


def test_proposal_mlp_is_sigmoid_of_a_linear_map():
    W = 32
    rng = np.random.default_rng(5)
    a = rng.normal(0, 0.7, (3, 6))
    b2 = rng.normal(0, 0.5, 3)
    w0 = np.zeros((W, 6))
    for k in range(6):
        w0[2 * k, k], w0[2 * k + 1, k] = 1.0, -1.0
    w1 = np.eye(W)
    w2 = np.zeros((3, W))
    for k in range(6):
        w2[:, 2 * k], w2[:, 2 * k + 1] = a[:, k], -a[:, k]
    w = np.concatenate([w0.reshape(-1), np.zeros(W), w1.reshape(-1), np.zeros(W), w2.reshape(-1), b2])
    assert len(w) == O.prop_param_count(W)
    o, d = S.random_rays(40, 8, False)
    in_scale, t_scale = 3.0, 12.0
    out = O.prop_forward(w, o, d, in_scale, t_scale)
    o64, d64 = o.astype(np.float64), d.astype(np.float64)
    e = np.concatenate([o64 / in_scale, d64 / np.linalg.norm(d64, axis=1, keepdims=True)], 1)
    z = e @ a.T + b2
    sig = 1.0 / (1.0 + np.exp(-z))
    np.testing.assert_allclose(out[:, 0], t_scale * sig[:, 0], rtol=1e-6)
    np.testing.assert_allclose(out[:, 1], t_scale * sig[:, 1], rtol=1e-6)
    np.testing.assert_allclose(out[:, 2], sig[:, 2], rtol=1e-6)
    # a first-layer bias enters before the ReLU: with b0[0] = 10 unit 0 is e_0 + 10
    # (always positive) while unit 1 stays relu(-e_0), so the readout of that pair
    # moves from e_0 to e_0 + 10 - relu(-e_0), i.e. by 10 + min(e_0, 0)
    w_b = w.copy()
    w_b[W * 6] = 10.0
    out_b = O.prop_forward(w_b, o, d, in_scale, t_scale)
    z_b = z + np.outer(10.0 + np.minimum(e[:, 0], 0.0), a[:, 0])
    np.testing.assert_allclose(out_b[:, 2], 1.0 / (1.0 + np.exp(-z_b[:, 2])), rtol=1e-6)
    assert math.isfinite(float(out_b.sum()))
