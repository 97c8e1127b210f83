"""Per-ray parity of a GPU render against the FP64 oracle.

The kernels take the march's voxel decisions on FP32 positions; the oracle takes
them in FP64 and flags every ray on which FP32 rounding could decide otherwise (a
deciding voxel face within the FP32 position error, a termination test within
3e-5 of t_term, the domain's end within 1e-6).  The rule, for rays i:

* counts: marching points and samples must be equal on every unflagged ray;
* values: |rgb - rgb_ref|, |opacity - opacity_ref| <= tol and |depth - depth_ref|
  <= tol max(1, |depth|) on every unflagged ray, except for at most
  max(1, 5e-4 n) rays within 10 tol: a sample position the FP32 march carries
  to ~1e-6 of the unit cube moves a high-frequency table's features (white-noise
  tables at 4096^3) by up to ~1e-3 of their range;
* the rays on which the two differ at all (counts or values beyond tol) stay
  below 0.1% of the rays (at least 2 allowed), and the flagged fraction below
  max_flagged.
"""
import numpy as np


def compare_rays(r_gpu, r_or, tol=1e-4, check_stats=True, max_flagged=0.02, name=""):
    amb = np.asarray(r_or["ambiguous"], bool)
    n = len(amb)
    rgb = r_gpu["rgb"].cpu().numpy().astype(np.float64).reshape(n, 3)
    opa = r_gpu["opacity"].cpu().numpy().astype(np.float64).reshape(n)
    dep = r_gpu["depth"].cpu().numpy().astype(np.float64).reshape(n)
    dscale = max(1.0, float(np.abs(r_or["depth"]).max())) if n else 1.0
    err = np.maximum(np.abs(rgb - r_or["rgb"]).max(1) if n else np.zeros(0),
                     np.maximum(np.abs(opa - r_or["opacity"]), np.abs(dep - r_or["depth"]) / dscale))
    bad_val = err > tol
    bad_cnt = np.zeros(n, bool)
    if check_stats:
        bad_cnt = np.any(r_gpu["stats"].cpu().numpy().reshape(n, 2) != r_or["stats"], axis=1)
    differ = bad_val | bad_cnt
    print(f"parity {name}: {n} rays, flagged {amb.mean() if n else 0:.4%}, differing {differ.mean() if n else 0:.4%}, "
          f"max err on unflagged {err[~amb].max() if (~amb).any() else 0.0:.3g}")
    assert not np.any(bad_cnt & ~amb), f"{name}: counts differ on {int(np.sum(bad_cnt & ~amb))} unflagged rays"
    loose = bad_val & ~amb
    assert loose.sum() <= max(1, int(5e-4 * n)), f"{name}: {int(loose.sum())} unflagged rays beyond {tol}"
    assert not np.any(err[loose] > 10 * tol), f"{name}: unflagged error {err[loose].max()}"
    assert differ.sum() <= max(2, int(1e-3 * n)), f"{name}: {int(differ.sum())} of {n} rays differ"
    assert amb.mean() <= max_flagged if n else True, f"{name}: {amb.mean():.3%} of rays flagged"
    return float(err[~amb].max()) if (~amb).any() else 0.0
