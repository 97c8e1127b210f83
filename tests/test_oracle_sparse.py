"""Pins of the oracle's sparse coarse grid (the block-indexed storage of the baked
coarse grid, Sec. 3.1, Eq. S1): the kept blocks cover every cell a sample in an
occupied voxel can land in (brute force over float32 points, faces included), they
are no wider than one cell around those cells, and every corner of every kept cell
reads back the dense grid's vertex through the block layout."""
import numpy as np
import pytest

from oracle import oracle as O


def _occ(R, p, seed):
    rng = np.random.default_rng(seed)
    return (rng.random(R ** 3) < p).astype(np.uint8)


def _cells_hit(occ, R_O, R_C, per_axis=7):
    """Coarse cells (x, y, z) of float32 points spread over each occupied voxel,
    its faces included: cell = clamp(floor(u (R_C - 1)), 0, R_C - 2)."""
    g = occ.reshape(R_O, R_O, R_O)
    z, y, x = np.nonzero(g)
    f = np.linspace(0.0, 1.0, per_axis)
    cells = set()
    for v in zip(x, y, z):
        us = [((np.float32(v[a]) + f.astype(np.float32)) / np.float32(R_O)).astype(np.float32) for a in range(3)]
        cs = [np.clip(np.floor(u * np.float32(R_C - 1)), 0, R_C - 2).astype(int) for u in us]
        for cx in set(cs[0]):
            for cy in set(cs[1]):
                for cz in set(cs[2]):
                    cells.add((cx, cy, cz))
    return cells


@pytest.mark.parametrize("R_O,R_C,p", [(8, 17, 0.05), (16, 33, 0.01), (16, 40, 0.02), (8, 9, 0.1), (32, 20, 0.002)])
def test_mask_covers_every_reachable_cell_and_little_more(R_O, R_C, p):
    occ = _occ(R_O, p, R_O + R_C)
    assert occ.any()
    mask = O.coarse_block_mask(occ, R_O, R_C)
    nb = (R_C - 1 + 7) // 8
    assert mask.shape == (nb ** 3,)
    hit = _cells_hit(occ, R_O, R_C)
    for cx, cy, cz in hit:
        assert mask[cx // 8 + nb * (cy // 8 + nb * (cz // 8))] == 1, (cx, cy, cz)
    # no wider than one cell around the reachable cells
    near = set()
    for cx, cy, cz in hit:
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    x, y, z = cx + dx, cy + dy, cz + dz
                    if 0 <= min(x, y, z) and max(x, y, z) <= R_C - 2:
                        near.add((x // 8) + nb * ((y // 8) + nb * (z // 8)))
    assert set(np.nonzero(mask)[0]) <= near


def test_mask_special_cases():
    assert not O.coarse_block_mask(np.zeros(8 ** 3, np.uint8), 8, 33).any()
    assert O.coarse_block_mask(np.ones(8 ** 3, np.uint8), 8, 33).all()
    # one voxel in the corner: only the first block
    occ = np.zeros(16 ** 3, np.uint8)
    occ[0] = 1
    m = O.coarse_block_mask(occ, 16, 65)
    assert np.nonzero(m)[0].tolist() == [0]


@pytest.mark.parametrize("R_C,nch", [(17, 12), (20, 10), (33, 8)])
def test_blocks_read_back_the_dense_grid(R_C, nch):
    rng = np.random.default_rng(R_C)
    dense = rng.normal(size=(R_C ** 3, nch)).astype(np.float32)
    nb = (R_C - 1 + 7) // 8
    mask = (rng.random(nb ** 3) < 0.5).astype(np.uint8)
    mask[0] = 1
    index, blocks = O.sparse_coarse(dense, R_C, mask)
    assert blocks.shape == (1 + mask.sum(), 729, nch) and not blocks[0].any()
    assert sorted(index[mask == 1].tolist()) == list(range(1, mask.sum() + 1))
    assert not index[mask == 0].any()
    d = dense.reshape(R_C, R_C, R_C, nch)
    for b in np.nonzero(mask)[0]:
        bx, by, bz = b % nb, (b // nb) % nb, b // (nb * nb)
        s = index[b]
        # every corner of every cell of the block, addressed from the cell's base
        for cz in range(8 * bz, min(8 * bz + 8, R_C - 1)):
            for cy in range(8 * by, min(8 * by + 8, R_C - 1)):
                for cx in range(8 * bx, min(8 * bx + 8, R_C - 1)):
                    base = s * 729 + (cx & 7) + 9 * ((cy & 7) + 9 * (cz & 7))
                    for c in range(8):
                        dx, dy, dz = c & 1, (c >> 1) & 1, (c >> 2) & 1
                        row = base + dx + 9 * dy + 81 * dz
                        assert np.array_equal(blocks.reshape(-1, nch)[row], d[cz + dz, cy + dy, cx + dx])


@pytest.mark.parametrize("bounded", [True, False])
def test_vertices_outside_the_kept_blocks_never_reach_a_render(bounded):
    """The claim the sparse grid rests on, in the oracle: zeroing every coarse vertex
    that no kept block stores leaves renders (values and counts) unchanged bit for bit."""
    from paper_2407_10482_gb300 import scenes as S
    kw = dict(blob_std=(0.05, 0.15), R_C=41)
    if not bounded:
        kw.update(bounded=False, R_O=64, n_occ_levels=4, t_min=0.05, r_far=16.0, shell=True,
                  step_base=2 * 3 ** 0.5 / 256)
    cfg = S.small_config(**kw)
    sc = S.make_scene(cfg)
    mask = O.coarse_block_mask(sc.occ, cfg.R_O, cfg.R_C)
    nb = (cfg.R_C - 1 + 7) // 8
    kept = np.zeros((cfg.R_C,) * 3, bool)                      # [z][y][x] vertices some kept block stores
    for b in np.flatnonzero(mask):
        bx, by, bz = b % nb, (b // nb) % nb, b // (nb * nb)
        kept[8 * bz:8 * bz + 9, 8 * by:8 * by + 9, 8 * bx:8 * bx + 9] = True
    if bounded:
        assert not kept.all()
    masked = sc.coarse.copy()
    masked[~kept.reshape(-1)] = 0.0
    opts = S.default_options(cfg)
    cams = S.orbit_cameras(cfg, 1, azimuth0=25.0)
    a = O.oracle_for_scene(sc).render(opts, cams=cams)
    b = O.oracle_for_scene(sc, coarse=masked).render(opts, cams=cams)
    for k in ("rgb", "depth", "opacity", "stats"):
        assert np.array_equal(a[k], b[k]), k
    if bounded:
        # a planted mistake: one kept block fewer must show in the image
        worst = 0.0
        for b_drop in np.flatnonzero(mask)[:6]:
            bx, by, bz = b_drop % nb, (b_drop // nb) % nb, b_drop // (nb * nb)
            short = masked.reshape(cfg.R_C, cfg.R_C, cfg.R_C, -1).copy()
            short[8 * bz:8 * bz + 9, 8 * by:8 * by + 9, 8 * bx:8 * bx + 9] = 0.0
            c = O.oracle_for_scene(sc, coarse=short.reshape(masked.shape)).render(opts, cams=cams)
            worst = max(worst, float(np.abs(c["rgb"] - a["rgb"]).max()))
        assert worst > 1e-4
