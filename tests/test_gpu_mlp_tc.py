"""The deferred MLP in FP16 on the tensor cores (tcgen05) against the oracle.

The oracle evaluates MLP_psi in FP64 on the FP16-rounded weights; the kernel also
rounds its input row and hidden activations to FP16 (accumulating in FP32), so the
bound is the FP16 rounding of activations, 3e-3 on the final colour.  The FP32
CUDA-core MLP is checked alongside at the 1e-4 bound of the plain path."""
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


def _states(n, seed):
    rng = np.random.default_rng(seed)
    st = np.zeros((n, 12), np.float32)
    st[:, 0:7] = rng.normal(0, 0.7, (n, 7))
    st[:, 7] = rng.uniform(0, 1, n)
    st[:, 8] = rng.uniform(0, 5, n)
    d = rng.normal(size=(n, 3))
    st[:, 9:12] = d / np.linalg.norm(d, axis=1, keepdims=True)
    return st


@pytest.mark.parametrize("width,layers", [(16, 2), (64, 3), (32, 3), (64, 2)])
@pytest.mark.parametrize("n", [128, 1000, 70001])
def test_tensor_core_mlp_matches_oracle(ng, width, layers, n):
    cfg = S.small_config(mlp_width=width, mlp_layers=layers)
    sc = S.make_scene(cfg)
    w16 = sc.mlp_w.astype(np.float16).astype(np.float32)
    st = _states(n, width * 7 + layers + n)
    bg = (0.1, 0.3, 0.6)
    out = {}
    for dt, w in ((1, w16), (0, sc.mlp_w)):
        ds = ng.DeviceScene(cfg, sc.tables, sc.coarse, w, mlp_dtype=dt)
        rgb = torch.empty(n, 3, device="cuda")
        dep = torch.empty(n, device="cuda")
        opa = torch.empty(n, device="cuda")
        ng.ngprt_shade(ds.struct, torch.as_tensor(st).cuda(), n, bg, rgb, dep, opa)
        torch.cuda.synchronize()
        out[dt] = rgb.cpu().numpy().astype(np.float64)
        np.testing.assert_array_equal(opa.cpu().numpy(), st[:, 7])
        np.testing.assert_array_equal(dep.cpu().numpy(), st[:, 8])
    assert ng.lib().ngprt_tensor_core_error() == 0
    x = np.zeros((n, 32))
    x[:, :7] = st[:, :7]
    x[:, 7:23] = O.sh16(st[:, 9:12].astype(np.float64))
    for dt, w in ((1, w16), (0, sc.mlp_w)):
        orc = O.Oracle(cfg, sc.tables, sc.coarse, w, np.zeros(1, np.uint32))
        y = orc.mlp(x)
        z = st[:, :3].astype(np.float64) + y
        A = st[:, 7:8].astype(np.float64)
        want = A / (1 + np.exp(-z)) + (1 - A) * np.array(bg)
        err = np.abs(out[dt] - want).max()
        assert err <= (3e-3 if dt == 1 else 1e-4), (dt, err)
