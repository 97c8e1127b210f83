"""Error of every precision form against the FP64 oracle, stated as max abs and PSNR
(the table is printed; run with -s): FP32 tables, FP16 and BF16 tables (16-bit
copies of the FP32 master), the FP16 deferred MLP on tensor cores, and FP16 tables
with it.  Each form is compared with the oracle on the FP32 master (the error a user
sees) and on the same rounded values (the kernel's own arithmetic error)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2407_10482_gb300 import scenes as S

pytestmark = pytest.mark.gpu

FORMS = [("fp32", 0, 0), ("fp16 tables", 1, 0), ("bf16 tables", 2, 0), ("fp16 mlp (tcgen05)", 0, 1),
         ("fp16 tables + fp16 mlp", 1, 1)]
# bounds on (max abs against the master, PSNR against the master)
BOUND = {"fp32": (1e-4, 100.0), "fp16 tables": (5e-3, 75.0), "bf16 tables": (1e-2, 70.0),
         "fp16 mlp (tcgen05)": (1e-3, 85.0), "fp16 tables + fp16 mlp": (5e-3, 75.0)}


@pytest.fixture(scope="module")
def ng():
    from paper_2407_10482_gb300 import ngprt
    ngprt.lib()
    return ngprt


def _psnr(err):
    mse = float((err ** 2).mean())
    return 10 * np.log10(1.0 / max(mse, 1e-30))


@pytest.mark.parametrize("cfg_name", ["small", "hd"])
def test_precision_forms_against_oracle(ng, cfg_name):
    if cfg_name == "small":
        cfg = S.small_config(blob_std=(0.05, 0.15))
        pix = None
    else:
        cfg = S.hd_config()
        pix = np.random.default_rng(8).choice(cfg.W * cfg.H, 3000, replace=False).astype(np.int32)
    sc = S.make_scene(cfg)
    opts = S.default_options(cfg)
    cams = S.orbit_cameras(cfg, 1, azimuth0=15.0)
    bits = O.build_pyramid(sc.occ, cfg.R_O, cfg.n_occ_levels)
    dist = O.occ_dist(sc.occ, cfg.R_O)
    master = O.Oracle(cfg, sc.tables, sc.coarse, sc.mlp_w, bits, dist).render(opts, cams=cams, pix=pix)
    docc = ng.DeviceOcc(sc.occ, cfg.R_O, cfg.n_occ_levels)
    lines = []
    for name, tdt, mdt in FORMS:
        ds = ng.DeviceScene(cfg, sc.tables, sc.coarse, sc.mlp_w, table_dtype=tdt, mlp_dtype=mdt)
        kw = dict(pixel_ids=torch.as_tensor(pix).cuda()) if pix is not None else {}
        r = ng.Renderer(ds, docc).render(opts, cams=cams, W=cfg.W, H=cfg.H, **kw)
        torch.cuda.synchronize()
        rgb = r["rgb"].cpu().numpy().astype(np.float64)
        ok = ~master["ambiguous"]        # rays the FP32 march may decide otherwise
        rgb = rgb[ok]
        e_master = np.abs(rgb - master["rgb"][ok])
        rounded = O.Oracle(cfg, ds.tables.float().cpu().numpy(), ds.coarse.float().cpu().numpy(),
                           ds.mlp_w.float().cpu().numpy(), bits, dist).render(opts, cams=cams, pix=pix)
        e_round = np.abs(rgb - rounded["rgb"][ok])
        lines.append(f"| {cfg_name} | {name} | {e_master.max():.2e} | {_psnr(e_master):.1f} | "
                     f"{e_round.max():.2e} | {_psnr(e_round):.1f} |")
        bmax, bpsnr = BOUND[name]
        assert e_master.max() <= bmax and _psnr(e_master) >= bpsnr, lines[-1]
        if name == "fp32":
            assert e_master.max() <= 1e-4
    print("\n| workload | form | max abs (master) | PSNR dB (master) | max abs (rounded) | PSNR dB (rounded) |")
    print("|---|---|---|---|---|---|")
    print("\n".join(lines))
