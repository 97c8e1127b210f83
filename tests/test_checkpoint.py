"""Scene files round-trip: configuration and every array bit for bit, and the oracle
renders the reloaded scene exactly as the original."""
import numpy as np

from oracle import oracle as O
from paper_2407_10482_gb300 import checkpoint as CK
from paper_2407_10482_gb300 import scenes as S


def test_scene_file_round_trip(tmp_path):
    for cfg in (S.small_config(), S.small_config(aggregation=5, L=2, N=[16, 32]), S.small_config(aggregation=2)):
        sc = S.make_scene(cfg)
        path = str(tmp_path / f"scene_{cfg.aggregation}.ngprt")
        CK.save_scene(path, sc)
        back = CK.load_scene(path)
        assert back.cfg == sc.cfg
        for name in ("tables", "coarse", "mlp_w", "occ", "attn_inv", "agg_mlp"):
            a, b = getattr(sc, name), getattr(back, name)
            assert (a is None) == (b is None)
            if a is not None:
                assert a.dtype == b.dtype and np.array_equal(a, b), name
        for k in sc.blobs:
            assert np.array_equal(sc.blobs[k], back.blobs[k])
        opts = S.default_options(cfg)
        cams = S.orbit_cameras(cfg, 1)
        pix = np.arange(0, cfg.W * cfg.H, 7, dtype=np.int32)
        a = O.oracle_for_scene(sc).render(opts, cams=cams, pix=pix)
        b = O.oracle_for_scene(back).render(opts, cams=cams, pix=pix)
        assert np.array_equal(a["rgb"], b["rgb"])


def test_scene_file_keeps_16_bit_tables(tmp_path):
    torch = __import__("torch")
    sc = S.make_scene(S.small_config())
    sc.tables = torch.as_tensor(sc.tables).to(torch.bfloat16)
    path = str(tmp_path / "bf16.ngprt")
    CK.save_scene(path, sc)
    back = CK.load_scene(path)
    want = sc.tables.view(torch.int16).numpy().view(np.uint16)
    assert back.tables.dtype == np.uint16 and np.array_equal(back.tables, want)
