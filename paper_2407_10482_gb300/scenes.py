"""Seeded synthetic inputs for the NGP-RT render path.

This module draws the inputs that both the CUDA path and the CPU oracle consume:
feature tables, the coarse feature/attention grid, deferred-MLP weights, an
occupancy grid thresholded from an analytic density made of Gaussian blobs,
pinhole cameras on an orbit, and explicit ray batches.  It implements no step of
the rendering method (no marching, hashing, interpolation, attention or
compositing): every value it returns is an input.

Workloads (the synthetic stand-ins for the Mip-NeRF 360 scenes the paper
evaluates on, §4 and Table 1):

* ``small``  : bounded [-1,1]^3 scene, 8 blobs, one 64x64 view, L=4 fine levels
  at 16/32/64/128, T=2^12, 32^3 occupancy, <=128 samples per ray, MLP 23->16->3.
* ``hd``     : unbounded 360-style scene (64 blobs inside [-1,1]^3 plus a dense
  shell at world radius 8..10) under the mip-NeRF-360 contraction, 1920x1080,
  L=16 levels from 16 to 4096, T=2^19, 128^3 occupancy, <=1024 marching points,
  MLP 23->64->64->3, camera orbit radius 3, elevation 20 degrees.  Its coarse
  density channel carries an offset of 3.2 (sigma ~ 25) so that rays stop about
  18 samples into occupied space, the shape of Table 4's "# Occupied" (17-18);
  ``density_bias=0`` gives the stress case without early termination.
* ``hd_fit`` : the hd model (same levels, grids, MLP, occupancy resolution,
  orbit and step rule) fitted to ground-truth images of its analytic field: the
  same law of 64 Gaussian blobs and the shell, with peak densities raised to
  U[100, 1000] so that the blobs are opaque as the surfaces of a captured scene
  are.  ``hdfit.fit_hd_scene`` fits it; it is the workload whose PSNR against its
  targets judges the fast render forms.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

N_FEAT = 8          # deferred feature per entry: [sigma, c_d(3), v_s(4)] (§3.1, Sec. S2.1)
MLP_IN_PAD = 32     # deferred-MLP input: C_d(3) + F(4) + SH16(d), zero padded to 32


@dataclass
class SceneConfig:
    name: str
    L: int
    N: list
    T_log2: int
    R_C: int
    bounded: bool
    mlp_layers: int
    mlp_width: int
    R_O: int
    n_occ_levels: int
    step_base: float
    t_min: float
    r_far: float
    max_march: int
    max_samples: int
    n_blobs: int
    blob_box: float
    shell: bool
    W: int
    H: int
    fov_y_deg: float
    orbit_radius: float
    elevation_deg: float
    init_std: float = 0.1
    density_bias: float = 0.0
    seed: int = 0
    occ_threshold: float = 0.01
    blob_std: tuple = (0.08, 0.25)
    blob_peak: tuple = (5.0, 50.0)
    aggregation: int = 0    # level fusion (Eq. 8 = 0; the Table 3 variants 1..5, see coarse_channels)
    dist_level: int = 0     # G on occupancy pyramid level k (resolution R_O >> k)


def level_resolutions(n_min: int, n_max: int, L: int) -> list:
    """Per-level vertex resolution, growing geometrically from n_min to n_max.

    The growth factor b = exp(ln(n_max/n_min)/(L-1)); N_l = floor(n_min * b^l + 1e-9)
    in FP64 on the host, so that the last level is exactly n_max.  The integers are
    handed to both the kernels and the oracle.
    """
    if L == 1:
        return [n_min]
    b = math.exp(math.log(n_max / n_min) / (L - 1))
    return [int(math.floor(n_min * b ** l + 1e-9)) for l in range(L)]


def small_config(**kw) -> SceneConfig:
    c = SceneConfig(
        name="small", L=4, N=[16, 32, 64, 128], T_log2=12, R_C=16, bounded=True,
        mlp_layers=2, mlp_width=16, R_O=32, n_occ_levels=3,
        step_base=2.0 * math.sqrt(3.0) / 128.0, t_min=0.0, r_far=0.0,
        max_march=1024, max_samples=128, n_blobs=8, blob_box=0.8, shell=False,
        W=64, H=64, fov_y_deg=50.0, orbit_radius=3.0, elevation_deg=20.0, seed=0)
    return replace(c, **kw)


def hd_config(**kw) -> SceneConfig:
    c = SceneConfig(
        name="hd", L=16, N=level_resolutions(16, 4096, 16), T_log2=19, R_C=16, bounded=False,
        mlp_layers=3, mlp_width=64, R_O=128, n_occ_levels=5,
        step_base=2.0 * math.sqrt(3.0) / 512.0, t_min=0.05, r_far=16.0,
        max_march=1024, max_samples=1024, n_blobs=64, blob_box=1.0, shell=True,
        W=1920, H=1080, fov_y_deg=50.0, orbit_radius=3.0, elevation_deg=20.0, seed=1,
        blob_std=(0.05, 0.15), density_bias=3.2)
    return replace(c, **kw)


def hd_fit_config(**kw) -> SceneConfig:
    """The fitted hd workload: hd's model shape, opaque blobs (peaks U[100, 1000]),
    no density offset (the fit starts from its own initial grids)."""
    c = hd_config(name="hd_fit", blob_peak=(100.0, 1000.0), density_bias=0.0)
    return replace(c, **kw)


def table_entries(cfg: SceneConfig) -> int:
    """Number of 8-channel entries across all levels (a level holds min(N^3, T))."""
    T = 1 << cfg.T_log2
    return int(sum(min(n ** 3, T) for n in cfg.N))


@dataclass
class Scene:
    cfg: SceneConfig
    tables: np.ndarray        # float32 [n_entries, 8]
    coarse: np.ndarray        # float32 [R_C^3, 8 + 2L]
    mlp_w: np.ndarray         # float32 flat, layer matrices [out][in] concatenated
    occ: np.ndarray           # uint8 [R_O^3], x fastest
    blobs: dict = field(default_factory=dict)
    attn_inv: np.ndarray = None  # float32 constant attention logits (aggregations 2, 3)
    agg_mlp: np.ndarray = None   # float32 W1 [64][8L] then W2 [8][64] (aggregation 5)


AGG_HIDDEN = 64  # hidden units of the tiny-MLP aggregation


def coarse_channels(cfg: SceneConfig) -> int:
    """Channels per coarse-grid vertex: the deferred feature (8), plus omega and beta per
    level for Eq. 8 (aggregation 0) or one logit per level (1, shared gates); the
    spatially invariant gates (2, 3), the plain sum (4) and the tiny MLP (5) keep 8."""
    return {0: N_FEAT + 2 * cfg.L, 1: N_FEAT + cfg.L}.get(int(cfg.aggregation), N_FEAT)


def _aggregation_params(cfg: SceneConfig, rng: np.random.Generator):
    """(attn_inv, agg_mlp) of the aggregation variants, drawn after everything else so
    that the Eq. 8 scenes do not change: invariant logits ~ N(0, init_std) (gates near
    1/2, as the variant grids' logits), MLP weights ~ N(0, 1/fan_in)."""
    agg = int(cfg.aggregation)
    attn_inv = agg_mlp = None
    if agg in (2, 3):
        attn_inv = rng.normal(0.0, cfg.init_std, (2 if agg == 2 else 1) * cfg.L).astype(np.float32)
    if agg == 5:
        w1 = rng.normal(0.0, 1.0 / math.sqrt(N_FEAT * cfg.L), (AGG_HIDDEN, N_FEAT * cfg.L))
        w2 = rng.normal(0.0, 1.0 / math.sqrt(AGG_HIDDEN), (N_FEAT, AGG_HIDDEN))
        agg_mlp = np.concatenate([w1.reshape(-1), w2.reshape(-1)]).astype(np.float32)
    return attn_inv, agg_mlp


def mlp_shapes(cfg: SceneConfig) -> list:
    """(out, in) of each deferred-MLP layer; hidden width cfg.mlp_width, 3 outputs."""
    shapes = []
    fan_in = MLP_IN_PAD
    for k in range(cfg.mlp_layers):
        out = 3 if k == cfg.mlp_layers - 1 else cfg.mlp_width
        shapes.append((out, fan_in))
        fan_in = out
    return shapes


def mlp_param_count(cfg: SceneConfig) -> int:
    return int(sum(o * i for o, i in mlp_shapes(cfg)))


def _blobs(cfg: SceneConfig, rng: np.random.Generator) -> dict:
    n = cfg.n_blobs
    return dict(
        mu=rng.uniform(-cfg.blob_box, cfg.blob_box, (n, 3)),
        std=rng.uniform(cfg.blob_std[0], cfg.blob_std[1], n),
        peak=rng.uniform(cfg.blob_peak[0], cfg.blob_peak[1], n),
        rgb=rng.uniform(0.0, 1.0, (n, 3)),
    )


def blob_density(blobs: dict, x: np.ndarray, shell: bool) -> np.ndarray:
    """Analytic ground-truth density of the synthetic scene at world points x [..., 3]."""
    x = np.asarray(x, dtype=np.float64)
    sig = np.zeros(x.shape[:-1])
    for k in range(len(blobs["std"])):
        d2 = np.sum((x - blobs["mu"][k]) ** 2, axis=-1)
        sig += blobs["peak"][k] * np.exp(-d2 / (2.0 * blobs["std"][k] ** 2))
    if shell:
        r = np.linalg.norm(x, axis=-1)
        sig = np.where((r >= 8.0) & (r <= 10.0), sig + 20.0, sig)
    return sig


def blob_color(blobs: dict, x: np.ndarray) -> np.ndarray:
    """Density-weighted blob colour at world points x [..., 3] (RGB in [0, 1])."""
    x = np.asarray(x, dtype=np.float64)
    num = np.zeros(x.shape[:-1] + (3,))
    den = np.zeros(x.shape[:-1]) + 1e-12
    for k in range(len(blobs["std"])):
        d2 = np.sum((x - blobs["mu"][k]) ** 2, axis=-1)
        s = blobs["peak"][k] * np.exp(-d2 / (2.0 * blobs["std"][k] ** 2))
        num += s[..., None] * blobs["rgb"][k]
        den += s
    return num / den[..., None]


def _occupancy(cfg: SceneConfig, blobs: dict) -> np.ndarray:
    R = cfg.R_O
    idx = (np.arange(R, dtype=np.float64) + 0.5) / R
    zz, yy, xx = np.meshgrid(idx, idx, idx, indexing="ij")
    if cfg.bounded:
        pts = np.stack([xx, yy, zz], -1) * 2.0 - 1.0
        occ = blob_density(blobs, pts, False) > cfg.occ_threshold
    else:
        # Voxel centres of the contracted cube [-2,2]^3, mapped back to world space
        # by inverting the radial mip-NeRF-360 map ||y|| = 2 - 1/||x|| (||x|| > 1).
        y = np.stack([xx, yy, zz], -1) * 4.0 - 2.0
        ry = np.linalg.norm(y, axis=-1)
        inside = ry < 2.0 - 1e-9
        rx = np.where(ry <= 1.0, ry, 1.0 / np.maximum(2.0 - ry, 1e-9))
        scale = np.where(ry > 0, rx / np.maximum(ry, 1e-30), 1.0)
        pts = y * scale[..., None]
        occ = (blob_density(blobs, pts, False) > cfg.occ_threshold) & inside
        if cfg.shell:
            # The shell (world radius 8..10, contracted 1.875..1.9) is thinner than a
            # voxel: mark every voxel whose box meets it.
            h = 2.0 / R
            lo = np.abs(y) - h
            rmin = np.linalg.norm(np.maximum(lo, 0.0), axis=-1)
            rmax = np.linalg.norm(np.abs(y) + h, axis=-1)
            occ |= (rmin <= 1.9) & (rmax >= 1.875)
    return occ.astype(np.uint8).reshape(-1)


def make_scene(cfg: SceneConfig) -> Scene:
    """Draw a seeded scene: tables ~N(0, init_std), coarse grid ~N(0, init_std) with the
    density channel offset by ``density_bias``, MLP weights ~N(0, 1/fan_in) and the
    thresholded blob occupancy."""
    rng = np.random.default_rng(cfg.seed)
    blobs = _blobs(cfg, rng)
    n_ent = table_entries(cfg)
    tables = rng.normal(0.0, cfg.init_std, (n_ent, N_FEAT)).astype(np.float32)
    n_ch = coarse_channels(cfg)
    coarse = rng.normal(0.0, cfg.init_std, (cfg.R_C ** 3, n_ch)).astype(np.float32)
    coarse[:, 0] += np.float32(cfg.density_bias)
    ws = []
    for k, (o, i) in enumerate(mlp_shapes(cfg)):
        real_in = 23 if k == 0 else i
        w = rng.normal(0.0, 1.0 / math.sqrt(real_in), (o, i)).astype(np.float32)
        if k == 0:
            w[:, 23:] = 0.0
        ws.append(w.reshape(-1))
    mlp_w = np.concatenate(ws).astype(np.float32)
    occ = _occupancy(cfg, blobs)
    attn_inv, agg_mlp = _aggregation_params(cfg, rng)
    return Scene(cfg=cfg, tables=tables, coarse=coarse, mlp_w=mlp_w, occ=occ, blobs=blobs, attn_inv=attn_inv,
                 agg_mlp=agg_mlp)


# --------------------------------------------------------------------------- cameras

CAM_FLOATS = 16  # c2w (3x4 row-major) + fx, fy, cx, cy


def orbit_camera(W: int, H: int, fov_y_deg: float, radius: float, azimuth_deg: float,
                 elevation_deg: float) -> np.ndarray:
    """Pinhole camera on an orbit looking at the origin, z up.

    OpenCV axes: camera x right, y down, z forward.  Returns float32 [16]:
    c2w rows (3x4, columns = right, down, forward, position) then fx, fy, cx, cy.
    """
    az, el = math.radians(azimuth_deg), math.radians(elevation_deg)
    pos = np.array([radius * math.cos(el) * math.cos(az),
                    radius * math.cos(el) * math.sin(az),
                    radius * math.sin(el)])
    fwd = -pos / np.linalg.norm(pos)
    right = np.cross(fwd, [0.0, 0.0, 1.0])
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    c2w = np.stack([right, down, fwd, pos], axis=1)  # 3x4
    f = 0.5 * H / math.tan(math.radians(fov_y_deg) * 0.5)
    return np.concatenate([c2w.reshape(-1), [f, f, 0.5 * W, 0.5 * H]]).astype(np.float32)


def orbit_cameras(cfg: SceneConfig, n_views: int, azimuth0: float = 0.0,
                  step_deg: float = 45.0) -> np.ndarray:
    return np.stack([orbit_camera(cfg.W, cfg.H, cfg.fov_y_deg, cfg.orbit_radius,
                                  azimuth0 + step_deg * k, cfg.elevation_deg)
                     for k in range(n_views)])


def random_rays(n: int, seed: int, bounded: bool) -> tuple:
    """Random rays aimed through the scene: origins on a sphere of radius 3, directions
    towards uniform points of [-0.9, 0.9]^3 (not normalised; the renderer normalises)."""
    rng = np.random.default_rng(seed)
    o = rng.normal(size=(n, 3))
    o = 3.0 * o / np.linalg.norm(o, axis=1, keepdims=True)
    tgt = rng.uniform(-0.9, 0.9, (n, 3))
    d = tgt - o
    return o.astype(np.float32), d.astype(np.float32)


def random_pixels(n: int, n_views: int, W: int, H: int, seed: int) -> np.ndarray:
    """Uniform random (view, pixel) ids for a training batch: id = view*W*H + row*W + col."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, n_views * W * H, n, dtype=np.int64).astype(np.int32)


# --------------------------------------------------------------------------- options

@dataclass
class RenderOptions:
    """Knobs of one render call (plain values; each side builds its own struct)."""
    step_base: float
    step_gamma: float = 1.0
    t_min: float = 0.0
    r_far: float = 0.0
    t_term: float = 2e-3
    bg: tuple = (0.0, 0.0, 0.0)
    max_march: int = 1024
    max_samples: int = 1024
    use_dist: bool = True
    lattice_snap: bool = False
    attn_mode: int = 0      # 0 separate attention (omega, beta), 1 SUM, 2 shared
    dist_rule: int = 1      # 1 max(v G, s_O) (default), 0 Eq. 9 as printed (v G alone)


def default_options(cfg: SceneConfig, **kw) -> RenderOptions:
    o = RenderOptions(step_base=cfg.step_base, t_min=cfg.t_min, r_far=cfg.r_far,
                      max_march=cfg.max_march, max_samples=cfg.max_samples)
    return replace(o, **kw)


# ------------------------------------------------------------- paper-shaped scenes

def paper_config(L: int = 2, **kw) -> SceneConfig:
    """The paper's render-time shape (Sec. S2.1, S2.5; Tables 2 and 4): L fine levels
    at 1024 * 2^l with T = 2^22, a 512^3 coarse grid (8 + 2L channels; drawn dense,
    DeviceScene.sparsify_coarse stores it block-sparse as the paper does), a 512^3
    occupancy grid with 5 levels down to 32^3 and the
    distance grid G at 256^3 (Sec. 3.3); hd's unbounded blob scene and orbit."""
    c = hd_config(name=f"paper_L{L}", L=L, N=[1024 * 2 ** l for l in range(L)], T_log2=22, R_C=512, R_O=512,
                  n_occ_levels=5, seed=7, dist_level=1)
    return replace(c, **kw)


def make_scene_torch(cfg: SceneConfig, device="cuda", occ_chunk: int = 1 << 22) -> Scene:
    """make_scene for grids too large for numpy: the same recipe drawn with a seeded
    torch generator on `device` (tables and coarse grid ~N(0, init_std), density
    offset on the coarse density channel, blob occupancy evaluated in chunks of voxel
    centres).  Arrays stay on the device (torch tensors); the MLP is drawn as in
    make_scene."""
    import torch
    rng = np.random.default_rng(cfg.seed)
    blobs = _blobs(cfg, rng)
    ws = []
    for k, (o, i) in enumerate(mlp_shapes(cfg)):
        real_in = 23 if k == 0 else i
        w = rng.normal(0.0, 1.0 / math.sqrt(real_in), (o, i)).astype(np.float32)
        if k == 0:
            w[:, 23:] = 0.0
        ws.append(w.reshape(-1))
    mlp_w = np.concatenate(ws).astype(np.float32)
    g = torch.Generator(device=device)
    g.manual_seed(cfg.seed)
    tables = torch.randn(table_entries(cfg), N_FEAT, generator=g, device=device) * cfg.init_std
    coarse = torch.randn(cfg.R_C ** 3, coarse_channels(cfg), generator=g, device=device) * cfg.init_std
    coarse[:, 0] += cfg.density_bias
    occ = occupancy_torch(cfg, blobs, device, occ_chunk)
    attn_inv, agg_mlp = _aggregation_params(cfg, rng)
    return Scene(cfg=cfg, tables=tables, coarse=coarse, mlp_w=mlp_w, occ=occ, blobs=blobs, attn_inv=attn_inv,
                 agg_mlp=agg_mlp)


def occupancy_torch(cfg: SceneConfig, blobs: dict, device="cuda", chunk: int = 1 << 22):
    """The unbounded scene's occupancy grid (as ``_occupancy``) evaluated with torch on
    ``device`` in chunks of voxel centres: blob density above ``occ_threshold`` at
    the voxel centre mapped back to world space, plus every voxel whose box meets the
    shell.  uint8 [R_O^3], x fastest."""
    import torch
    assert not cfg.bounded
    R = cfg.R_O
    mu = torch.as_tensor(blobs["mu"], device=device, dtype=torch.float64)
    std = torch.as_tensor(blobs["std"], device=device, dtype=torch.float64)
    peak = torch.as_tensor(blobs["peak"], device=device, dtype=torch.float64)
    occ = torch.empty(R ** 3, dtype=torch.uint8, device=device)
    for s0 in range(0, R ** 3, chunk):
        idx = torch.arange(s0, min(s0 + chunk, R ** 3), device=device, dtype=torch.int64)
        vx, vy, vz = idx % R, (idx // R) % R, idx // (R * R)
        y = (torch.stack([vx, vy, vz], 1).double() + 0.5) / R * 4.0 - 2.0
        ry = torch.linalg.norm(y, dim=1)
        rx = torch.where(ry <= 1.0, ry, 1.0 / torch.clamp(2.0 - ry, min=1e-9))
        pts = y * (rx / torch.clamp(ry, min=1e-30)).unsqueeze(1)
        d2 = ((pts.unsqueeze(1) - mu.unsqueeze(0)) ** 2).sum(-1)
        sig = (peak * torch.exp(-d2 / (2.0 * std ** 2))).sum(1)
        o = (sig > cfg.occ_threshold) & (ry < 2.0 - 1e-9)
        if cfg.shell:
            h = 2.0 / R
            rmin = torch.linalg.norm(torch.clamp(y.abs() - h, min=0.0), dim=1)
            rmax = torch.linalg.norm(y.abs() + h, dim=1)
            o |= (rmin <= 1.9) & (rmax >= 1.875)
        occ[s0:s0 + len(idx)] = o.to(torch.uint8)
    return occ
