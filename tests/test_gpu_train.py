"""GPU loss and Adam kernels against the oracle (FP32 vs FP64)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ng():
    from paper_2407_10482_gb300 import ngprt
    ngprt.lib()
    return ngprt


@pytest.mark.parametrize("n", [1, 1000, 3 * 262144 + 5])
def test_l2_loss(ng, n):
    rng = np.random.default_rng(n)
    x = rng.uniform(size=n).astype(np.float32)
    t = rng.uniform(size=n).astype(np.float32)
    loss = torch.zeros(1, device="cuda")
    d = torch.empty(n, device="cuda")
    ng.ngprt_l2_loss(torch.as_tensor(x).cuda(), torch.as_tensor(t).cuda(), n, 1.0 / n, loss, d)
    torch.cuda.synchronize()
    L, dr = O.l2_loss(x, t, 1.0 / n)
    assert abs(loss.item() - L) <= 1e-5 * abs(L) + 1e-7
    np.testing.assert_allclose(d.cpu().numpy(), dr, rtol=1e-5, atol=1e-9)


@pytest.mark.parametrize("n", [7, 4096, 1000003])
def test_adam_three_steps(ng, n):
    rng = np.random.default_rng(n)
    p = rng.normal(size=n)
    pt = torch.as_tensor(p.astype(np.float32)).cuda()
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    pr, mr, vr = p.astype(np.float32).astype(np.float64), np.zeros(n), np.zeros(n)
    for s in range(1, 4):
        g = rng.normal(size=n).astype(np.float32)
        gt = torch.as_tensor(g).cuda()
        ng.ngprt_adam_step(pt, gt, m, v, 1e-2, 0.9, 0.99, 1e-8, s, True)
        O.adam_step(pr, g, mr, vr, 1e-2, 0.9, 0.99, 1e-8, s)
        torch.cuda.synchronize()
        assert float(gt.abs().max()) == 0.0
    np.testing.assert_allclose(pt.cpu().numpy(), pr, rtol=0, atol=2e-6)
