"""Python bindings of the CPU oracle of the NGP-RT render path.

TEST INFRASTRUCTURE ONLY: the test-suite, the package smoke check and the
benchmark's CPU-baseline / reference arm call it; the CUDA library never does.
The arithmetic lives in ``ngprt_oracle.c`` (FP64 throughout, the march included);
this module only builds that file with gcc, marshals numpy arrays and converts
every table to FP64 before the call.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ngprt_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "libngprt_oracle.so")
MAXL = 32


def build(force: bool = False, defines: tuple = ()) -> str:
    """Compile the oracle with gcc (FP contraction off, OpenMP over rays).  `defines`
    (macro names) build a variant library beside it: the pins use one with a planted
    mistake to show that they catch it."""
    lib_path = _LIB if not defines else os.path.join(_LIBDIR, "libngprt_oracle_" + "_".join(defines) + ".so")
    if not force and os.path.exists(lib_path) and os.path.getmtime(lib_path) >= os.path.getmtime(_SRC):
        return lib_path
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = lib_path + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC"] + [f"-D{m}" for m in defines] + ["-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, lib_path)
    return lib_path


class OrScene(C.Structure):
    _fields_ = [("L", C.c_int), ("T_log2", C.c_int), ("N", C.c_int * MAXL),
                ("tables", C.c_void_p), ("R_C", C.c_int), ("coarse", C.c_void_p),
                ("mlp_layers", C.c_int), ("mlp_width", C.c_int), ("mlp_w", C.c_void_p),
                ("bounded", C.c_int), ("aggregation", C.c_int), ("attn_inv", C.c_void_p),
                ("agg_mlp", C.c_void_p)]


class OrOcc(C.Structure):
    _fields_ = [("R_O", C.c_int), ("n_levels", C.c_int), ("bits", C.c_void_p), ("dist", C.c_void_p),
                ("R_G", C.c_int)]


class OrOpts(C.Structure):
    _fields_ = [("step_base", C.c_float), ("step_gamma", C.c_float), ("t_min", C.c_float),
                ("r_far", C.c_float), ("t_term", C.c_float), ("bg", C.c_double * 3),
                ("max_march", C.c_int), ("max_samples", C.c_int), ("use_dist", C.c_int),
                ("lattice_snap", C.c_int), ("attn_mode", C.c_int), ("dist_rule", C.c_int)]


_lib_handle = None


def lib():
    global _lib_handle
    if _lib_handle is None:
        _lib_handle = C.CDLL(build())
        _lib_handle.or_hash.restype = C.c_uint32
        _lib_handle.or_hash.argtypes = [C.c_uint32] * 4
        _lib_handle.or_pyramid_words.restype = C.c_size_t
        _lib_handle.or_pyramid_words.argtypes = [C.c_int, C.c_int]
        _lib_handle.or_level_offset.restype = C.c_uint64
        _lib_handle.or_render_dot.restype = C.c_double
        _lib_handle.or_ray_samples.restype = C.c_int
        _lib_handle.or_max_threads.restype = C.c_int
    return _lib_handle


def _p(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def max_threads() -> int:
    return int(lib().or_max_threads())


DEFAULT_POSITION_ERROR = 8e-7   # the oracle's OR_AMB_U


def set_kink_position_error(e: float) -> None:
    """Unit-cube position error the tiny-MLP form's kink flag allows for (default: the
    FP32 march's; 0 for rays whose sample positions are exact in FP32)."""
    lib().or_set_kink_position_error(C.c_double(e))


# ----------------------------------------------------------------- primitives

def hash3(xyz: np.ndarray, T: int) -> np.ndarray:
    xyz = _c(xyz, np.uint32).reshape(-1, 3)
    out = np.empty(len(xyz), np.uint32)
    lib().or_hash_batch(_p(xyz), C.c_int(len(xyz)), C.c_uint32(T), _p(out))
    return out


def level_offset(N, T_log2: int, l: int) -> int:
    arr = (C.c_int * MAXL)(*N)
    return int(lib().or_level_offset(arr, C.c_int(len(N)), C.c_int(T_log2), C.c_int(l)))


def grid_indices(N, T_log2: int, u: np.ndarray):
    """Corner entry rows [n, L, 8] (uint64) and FP64 weights [n, L, 3] of positions u."""
    u = _c(u, np.float32).reshape(-1, 3)
    L = len(N)
    idx = np.empty((len(u), L, 8), np.uint64)
    w = np.empty((len(u), L, 3), np.float64)
    arr = (C.c_int * MAXL)(*N)
    lib().or_grid_indices(arr, C.c_int(L), C.c_int(T_log2), _p(u), C.c_int(len(u)), _p(idx), _p(w))
    return idx, w


def pyramid_words(R: int, n_levels: int) -> int:
    return int(lib().or_pyramid_words(R, n_levels))


def build_pyramid(occ: np.ndarray, R: int, n_levels: int) -> np.ndarray:
    occ = _c(occ, np.uint8).reshape(-1)
    out = np.empty(pyramid_words(R, n_levels), np.uint32)
    lib().or_build_pyramid(_p(occ), C.c_int(R), C.c_int(n_levels), _p(out))
    return out


def dilate(occ: np.ndarray, R: int, r: int, mask=None) -> np.ndarray:
    """Box dilation of an R^3 uint8 grid by radius r (faces clip the box), cleared
    where mask (optional) is 0."""
    occ = _c(occ, np.uint8).reshape(-1)
    mask = _c(mask, np.uint8)
    out = np.empty(R ** 3, np.uint8)
    lib().or_dilate(_p(occ), C.c_int(R), C.c_int(r), _p(mask), _p(out))
    return out


def occ_dist_brute(occ: np.ndarray, R: int) -> np.ndarray:
    occ = _c(occ, np.uint8).reshape(-1)
    out = np.empty(R ** 3, np.uint8)
    lib().or_occ_dist_brute(_p(occ), C.c_int(R), _p(out))
    return out


def occ_dist(occ: np.ndarray, R: int) -> np.ndarray:
    occ = _c(occ, np.uint8).reshape(-1)
    out = np.empty(R ** 3, np.uint8)
    lib().or_occ_dist(_p(occ), C.c_int(R), _p(out))
    return out


def sh16(d: np.ndarray) -> np.ndarray:
    d = _c(d, np.float64).reshape(-1, 3)
    out = np.empty((len(d), 16), np.float64)
    lib().or_sh16_batch(_p(d), C.c_int(len(d)), _p(out))
    return out


def camera_rays(cams: np.ndarray, W: int, H: int, pix=None, n=None):
    """FP64 origins and (unnormalised) directions of pixel-centre rays."""
    cams = _c(cams, np.float32).reshape(-1, 16)
    pix = _c(pix, np.int32)
    if n is None:
        n = len(pix) if pix is not None else len(cams) * W * H
    o = np.empty((n, 3), np.float64)
    d = np.empty((n, 3), np.float64)
    lib().or_camera_rays(_p(cams), C.c_int(len(cams)), C.c_int(W), C.c_int(H), _p(pix), C.c_int(n),
                         _p(o), _p(d))
    return o, d


# ----------------------------------------------------------------- the oracle

class Oracle:
    """FP64 renderer over one scene.  ``tables``/``coarse``/``mlp_w`` may be FP32 or
    FP16/BF16-rounded copies (pass them as float arrays); they are widened to FP64."""

    def __init__(self, cfg, tables, coarse, mlp_w, occ_bits, dist=None, attn_inv=None, agg_mlp=None, R_G=0):
        self.cfg = cfg
        self.tables = _c(np.asarray(tables, np.float64), np.float64)
        self.coarse = _c(np.asarray(coarse, np.float64), np.float64)
        self.mlp_w = _c(np.asarray(mlp_w, np.float64), np.float64)
        agg = int(getattr(cfg, "aggregation", 0))
        assert self.coarse.size == (cfg.R_C ** 3) * coarse_channels(cfg.L, agg), "coarse grid layout"
        self.attn_inv = None if attn_inv is None else _c(np.asarray(attn_inv, np.float64), np.float64)
        self.agg_mlp = None if agg_mlp is None else _c(np.asarray(agg_mlp, np.float64), np.float64)
        if agg in (2, 3):
            assert self.attn_inv is not None and self.attn_inv.size == (2 if agg == 2 else 1) * cfg.L
        if agg == 5:
            assert self.agg_mlp is not None and self.agg_mlp.size == AGG_HIDDEN * 8 * cfg.L + 8 * AGG_HIDDEN
        self.bits = _c(occ_bits, np.uint32)
        self.dist = _c(dist, np.uint8)
        s = OrScene()
        s.L = cfg.L
        s.T_log2 = cfg.T_log2
        for i, n in enumerate(cfg.N):
            s.N[i] = int(n)
        s.tables = self.tables.ctypes.data
        s.R_C = cfg.R_C
        s.coarse = self.coarse.ctypes.data
        s.mlp_layers = cfg.mlp_layers
        s.mlp_width = cfg.mlp_width
        s.mlp_w = self.mlp_w.ctypes.data
        s.bounded = 1 if cfg.bounded else 0
        s.aggregation = agg
        s.attn_inv = self.attn_inv.ctypes.data if self.attn_inv is not None else None
        s.agg_mlp = self.agg_mlp.ctypes.data if self.agg_mlp is not None else None
        self._s = s
        o = OrOcc()
        o.R_O = cfg.R_O
        o.n_levels = cfg.n_occ_levels
        o.bits = self.bits.ctypes.data
        o.dist = self.dist.ctypes.data if self.dist is not None else None
        o.R_G = int(R_G)
        if self.dist is not None:
            assert self.dist.size == (R_G or cfg.R_O) ** 3, "distance grid size"
        self._o = o

    @staticmethod
    def _opts(opts) -> OrOpts:
        p = OrOpts()
        p.step_base = opts.step_base
        p.step_gamma = opts.step_gamma
        p.t_min = opts.t_min
        p.r_far = opts.r_far
        p.t_term = opts.t_term
        for k in range(3):
            p.bg[k] = float(opts.bg[k])
        p.max_march = int(opts.max_march)
        p.max_samples = int(opts.max_samples)
        p.use_dist = 1 if opts.use_dist else 0
        p.lattice_snap = 1 if opts.lattice_snap else 0
        p.attn_mode = int(opts.attn_mode)
        p.dist_rule = int(opts.dist_rule)
        return p

    def _rays(self, cams, pix, rays_o, rays_d):
        cams = _c(cams, np.float32)
        pix = _c(pix, np.int32)
        ro = _c(rays_o, np.float32)
        rd = _c(rays_d, np.float32)
        if cams is not None:
            cams = cams.reshape(-1, 16)
            n = len(pix) if pix is not None else len(cams) * self.cfg.W * self.cfg.H
        else:
            n = len(ro.reshape(-1, 3))
        return cams, pix, ro, rd, n

    def render(self, opts, cams=None, pix=None, rays_o=None, rays_d=None, interval=None,
               W=None, H=None):
        W = W or self.cfg.W
        H = H or self.cfg.H
        cams, pix, ro, rd, n = self._rays(cams, pix, rays_o, rays_d)
        iv = _c(interval, np.float32)
        rgb = np.empty((n, 3), np.float64)
        depth = np.empty(n, np.float64)
        opac = np.empty(n, np.float64)
        stats = np.empty((n, 2), np.int32)
        amb = np.empty(n, np.int32)
        state = np.empty((n, 9), np.float64)
        op = self._opts(opts)
        lib().or_render(C.byref(self._s), C.byref(self._o), C.byref(op), _p(cams),
                        C.c_int(0 if cams is None else len(cams)), C.c_int(W), C.c_int(H), _p(pix),
                        _p(ro), _p(rd), C.c_int(n), _p(iv), _p(rgb), _p(depth), _p(opac), _p(stats),
                        _p(amb), _p(state))
        return dict(rgb=rgb, depth=depth, opacity=opac, stats=stats, ambiguous=amb.astype(bool),
                    state=state)

    def occupancy_density(self, opts, R: int, sigma_thr: float):
        """Occupancy from the model's density at the centres of an R^3 grid (Sec. S2.5):
        (uint8 occ [R^3], sigma [R^3])."""
        occ = np.empty(R ** 3, np.uint8)
        sig = np.empty(R ** 3, np.float64)
        op = self._opts(opts)
        lib().or_occupancy_density(C.byref(self._s), C.byref(op), C.c_int(R), C.c_double(sigma_thr), _p(occ),
                                   _p(sig))
        return occ, sig

    def occupancy_visibility(self, opts, R: int, w_thr: float, cams=None, pix=None, rays_o=None, rays_d=None,
                             W=None, H=None):
        """Voxels of an R^3 grid holding a sample of weight > w_thr on the given rays:
        (uint8 vis [R^3], largest weight per voxel [R^3])."""
        W = W or self.cfg.W
        H = H or self.cfg.H
        cams, pix, ro, rd, n = self._rays(cams, pix, rays_o, rays_d)
        vis = np.zeros(R ** 3, np.uint8)
        wmax = np.zeros(R ** 3, np.float64)
        op = self._opts(opts)
        lib().or_occupancy_visibility(C.byref(self._s), C.byref(self._o), C.byref(op), _p(cams),
                                      C.c_int(0 if cams is None else len(cams)), C.c_int(W), C.c_int(H), _p(pix),
                                      _p(ro), _p(rd), C.c_int(n), C.c_int(R), C.c_double(w_thr), _p(vis), _p(wmax))
        return vis, wmax

    def distortion(self, opts, cams=None, pix=None, rays_o=None, rays_d=None, W=None, H=None):
        """Per-ray distortion regulariser (Eq. S2): [n][4] = (L_dist, sum w, sum w m, 0)."""
        W = W or self.cfg.W
        H = H or self.cfg.H
        cams, pix, ro, rd, n = self._rays(cams, pix, rays_o, rays_d)
        out = np.empty((n, 4), np.float64)
        op = self._opts(opts)
        lib().or_distortion(C.byref(self._s), C.byref(self._o), C.byref(op), _p(cams),
                            C.c_int(0 if cams is None else len(cams)), C.c_int(W), C.c_int(H), _p(pix), _p(ro),
                            _p(rd), C.c_int(n), _p(out))
        return out

    def distortion_backward(self, opts, scale=1.0, cams=None, pix=None, rays_o=None, rays_d=None, W=None, H=None,
                            full=False):
        """Gradients of scale * sum over rays of L_dist: (g_tables, g_coarse), or with
        full=True a dict that adds the constant logits' and the tiny MLP's gradients."""
        W = W or self.cfg.W
        H = H or self.cfg.H
        cams, pix, ro, rd, n = self._rays(cams, pix, rays_o, rays_d)
        g_t = np.zeros_like(self.tables)
        g_c = np.zeros_like(self.coarse)
        g_i = np.zeros_like(self.attn_inv) if self.attn_inv is not None else None
        g_a = np.zeros_like(self.agg_mlp) if self.agg_mlp is not None else None
        op = self._opts(opts)
        lib().or_distortion_backward(C.byref(self._s), C.byref(self._o), C.byref(op), _p(cams),
                                     C.c_int(0 if cams is None else len(cams)), C.c_int(W), C.c_int(H), _p(pix),
                                     _p(ro), _p(rd), C.c_int(n), C.c_double(scale), _p(g_t), _p(g_c), _p(g_i),
                                     _p(g_a))
        if full:
            return dict(tables=g_t, coarse=g_c, attn_inv=g_i, agg_mlp=g_a)
        return g_t, g_c

    def render_backward(self, opts, d_rgb=None, d_depth=None, d_opacity=None, cams=None, pix=None,
                        rays_o=None, rays_d=None, W=None, H=None):
        """Gradients (+ for the MLP form, "kink": per ray 1 when a hidden unit of one
        of its samples lies within 1e-5 relative of its ReLU kink, where FP32 may take
        the other side)."""
        W = W or self.cfg.W
        H = H or self.cfg.H
        cams, pix, ro, rd, n = self._rays(cams, pix, rays_o, rays_d)
        g_t = np.zeros_like(self.tables)
        g_c = np.zeros_like(self.coarse)
        g_m = np.zeros_like(self.mlp_w)
        g_i = np.zeros_like(self.attn_inv) if self.attn_inv is not None else None
        g_a = np.zeros_like(self.agg_mlp) if self.agg_mlp is not None else None
        kink = np.zeros(n, np.int32)
        op = self._opts(opts)
        # hold the converted cotangents in locals: a temporary freed before the call
        # would hand the C code a dangling pointer
        cr, cd, co = _c(d_rgb, np.float64), _c(d_depth, np.float64), _c(d_opacity, np.float64)
        lib().or_render_backward(C.byref(self._s), C.byref(self._o), C.byref(op), _p(cams),
                                 C.c_int(0 if cams is None else len(cams)), C.c_int(W), C.c_int(H),
                                 _p(pix), _p(ro), _p(rd), C.c_int(n), _p(cr), _p(cd), _p(co),
                                 _p(g_t), _p(g_c), _p(g_m), _p(g_i), _p(g_a), _p(kink))
        return dict(tables=g_t, coarse=g_c, mlp_w=g_m, attn_inv=g_i, agg_mlp=g_a, kink=kink)

    def render_dot(self, opts, d_rgb=None, d_depth=None, d_opacity=None, cams=None, pix=None,
                   rays_o=None, rays_d=None, W=None, H=None) -> float:
        W = W or self.cfg.W
        H = H or self.cfg.H
        cams, pix, ro, rd, n = self._rays(cams, pix, rays_o, rays_d)
        op = self._opts(opts)
        cr, cd, co = _c(d_rgb, np.float64), _c(d_depth, np.float64), _c(d_opacity, np.float64)
        return float(lib().or_render_dot(
            C.byref(self._s), C.byref(self._o), C.byref(op), _p(cams),
            C.c_int(0 if cams is None else len(cams)), C.c_int(W), C.c_int(H), _p(pix), _p(ro), _p(rd),
            C.c_int(n), _p(cr), _p(cd), _p(co)))

    def ray_samples(self, opts, o, d, cap=4096) -> np.ndarray:
        """Per-sample records [n, 7] = t, delta, u(3), sigma, weight of one ray."""
        o = _c(o, np.float32).reshape(3)
        d = _c(d, np.float32).reshape(3)
        out = np.empty((cap, 7), np.float64)
        op = self._opts(opts)
        n = lib().or_ray_samples(C.byref(self._s), C.byref(self._o), C.byref(op), _p(o), _p(d),
                                 C.c_int(cap), _p(out))
        return out[:min(n, cap)]

    def mlp(self, x: np.ndarray) -> np.ndarray:
        x = _c(x, np.float64).reshape(-1, 32)
        y = np.empty((len(x), 3), np.float64)
        lib().or_mlp_batch(C.byref(self._s), _p(x), C.c_int(len(x)), _p(y))
        return y


def downsample_occ(occ: np.ndarray, R: int, k: int) -> np.ndarray:
    """Occupancy of pyramid level k as one byte per voxel: a voxel of R >> k is
    occupied when any of its 2^k x 2^k x 2^k finest voxels is (x fastest)."""
    g = np.asarray(occ, np.uint8).reshape(R, R, R)
    if k == 0:
        return np.ascontiguousarray(g.reshape(-1))
    f = 1 << k
    r = R >> k
    return np.ascontiguousarray(g.reshape(r, f, r, f, r, f).max(axis=(1, 3, 5)).reshape(-1))


COARSE_BLOCK = 8


def coarse_block_mask(occ: np.ndarray, R_O: int, R_C: int) -> np.ndarray:
    """Blocks of the sparse coarse grid a render can reach (the baked grid is stored
    sparse, Sec. 3.1 and Eq. S1; which vertices to keep is this build's reading):
    occupied finest voxel x covers u in [x / R_O, (x + 1) / R_O], so the cells
    floor(x (R_C - 1) / R_O) ... floor((x + 1) (R_C - 1) / R_O) per axis, widened by one
    cell and clamped to [0, R_C - 2]; a block of 8^3 cells is kept when it holds one
    of them.  uint8 [NB^3], NB = ceil((R_C - 1) / 8), entry bx + NB (by + NB bz)."""
    nb = (R_C - 1 + COARSE_BLOCK - 1) // COARSE_BLOCK
    g = np.asarray(occ, np.uint8).reshape(R_O, R_O, R_O)       # [z][y][x]
    z, y, x = np.nonzero(g)
    mask = np.zeros((nb, nb, nb), np.uint8)                     # [bz][by][bx]
    ranges = []
    for v in (x, y, z):
        v = v.astype(np.int64)
        lo = np.maximum(v * (R_C - 1) // R_O - 1, 0) // COARSE_BLOCK
        hi = np.minimum((v + 1) * (R_C - 1) // R_O + 1, R_C - 2) // COARSE_BLOCK
        ranges.append((lo, hi))
    for i in range(len(x)):
        (x0, x1), (y0, y1), (z0, z1) = [(lo[i], hi[i]) for lo, hi in ranges]
        mask[z0:z1 + 1, y0:y1 + 1, x0:x1 + 1] = 1
    return mask.reshape(-1)


def sparse_coarse(dense: np.ndarray, R_C: int, mask: np.ndarray):
    """(index, blocks) of the sparse coarse grid: marked blocks numbered 1, 2, ... in
    index order (0 = the all-zero slot 0); block s holds the 9^3 vertices
    (8 bx + i, 8 by + j, 8 bz + k), row i + 9 j + 81 k, zero past vertex R_C - 1."""
    nb = (R_C - 1 + COARSE_BLOCK - 1) // COARSE_BLOCK
    mask = np.asarray(mask, np.uint8).reshape(-1)
    nch = dense.shape[-1]
    d = np.asarray(dense).reshape(R_C, R_C, R_C, nch)          # [z][y][x][ch]
    index = np.zeros(nb ** 3, np.int32)
    marked = np.nonzero(mask)[0]
    index[marked] = np.arange(1, len(marked) + 1, dtype=np.int32)
    blocks = np.zeros((1 + len(marked), 9, 9, 9, nch), d.dtype)  # [s][k][j][i][ch]
    for s, e in enumerate(marked, start=1):
        bx, by, bz = e % nb, (e // nb) % nb, e // (nb * nb)
        x0, y0, z0 = COARSE_BLOCK * bx, COARSE_BLOCK * by, COARSE_BLOCK * bz
        part = d[z0:z0 + 9, y0:y0 + 9, x0:x0 + 9]
        blocks[s, :part.shape[0], :part.shape[1], :part.shape[2]] = part
    return index, blocks.reshape(1 + len(marked), 729, nch)


def oracle_for_scene(scene, tables=None, coarse=None, use_dist=True, dist_level=0) -> Oracle:
    """Oracle over a generated scene: builds the pyramid and distance grid itself (G
    on pyramid level dist_level)."""
    cfg = scene.cfg
    bits = build_pyramid(scene.occ, cfg.R_O, cfg.n_occ_levels)
    RG = cfg.R_O >> dist_level
    dist = occ_dist(downsample_occ(scene.occ, cfg.R_O, dist_level), RG) if use_dist else None
    return Oracle(cfg, scene.tables if tables is None else tables,
                  scene.coarse if coarse is None else coarse, scene.mlp_w, bits, dist,
                  attn_inv=getattr(scene, "attn_inv", None), agg_mlp=getattr(scene, "agg_mlp", None),
                  R_G=RG if dist_level else 0)


def contract(x: np.ndarray, bounded: bool = False):
    """FP64 contraction y and unit-cube position u of world points x [n, 3]."""
    x = _c(x, np.float64).reshape(-1, 3)
    y = np.empty_like(x)
    u = np.empty_like(x)
    lib().or_contract_batch(C.c_int(1 if bounded else 0), _p(x), C.c_int(len(x)), _p(y), _p(u))
    return y, u


AGG_HIDDEN = 64  # hidden units of the tiny-MLP aggregation


def coarse_channels(L: int, aggregation: int = 0) -> int:
    """Channels per coarse-grid vertex: deferred feature (8) plus omega, beta per level
    (Eq. 8), one logit per level (shared gates), or nothing (the other aggregations)."""
    return {0: 8 + 2 * L, 1: 8 + L}.get(int(aggregation), 8)


def huber_loss(rgb, target, delta):
    """Sum of the Huber loss h(rgb - target) and its derivative per value (Sec. S2.4)."""
    rgb = _c(rgb, np.float64).reshape(-1)
    target = _c(target, np.float64).reshape(-1)
    d = np.empty_like(rgb)
    f = lib().or_huber_loss
    f.restype = C.c_double
    L = f(_p(rgb), _p(target), C.c_long(len(rgb)), C.c_double(delta), _p(d))
    return float(L), d


def step_autotune(gamma, n_mean, n_min=3.0, kappa=1e-3, gamma_min=0.2217):
    """Eq. S3: the next step scaler."""
    f = lib().or_step_autotune
    f.restype = C.c_double
    return float(f(C.c_double(gamma), C.c_double(n_mean), C.c_double(n_min), C.c_double(kappa),
                   C.c_double(gamma_min)))


def l2_loss(rgb, target, scale=1.0):
    rgb = _c(rgb, np.float64).reshape(-1)
    target = _c(target, np.float64).reshape(-1)
    d = np.empty_like(rgb)
    f = lib().or_l2_loss
    f.restype = C.c_double
    L = f(_p(rgb), _p(target), C.c_int64(len(rgb)), C.c_double(scale), _p(d))
    return float(L), d


def adam_step(p, g, m, v, lr, b1, b2, eps, step):
    """In-place FP64 Adam step on numpy arrays p, m, v with gradient g."""
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _c(g, np.float64)
    lib().or_adam_step(_p(p), _p(g), _p(m), _p(v), C.c_int64(p.size), C.c_double(lr), C.c_double(b1),
                       C.c_double(b2), C.c_double(eps), C.c_int(step))


def prop_param_count(W: int = 32) -> int:
    """Flat proposal-MLP parameters: W0 [W][6], b0 [W], W1 [W][W], b1 [W], W2 [3][W], b2 [3]."""
    return W * 6 + W + W * W + W + 3 * W + 3


def prop_forward(w, rays_o, rays_d, in_scale, t_scale, W=32):
    w = _c(w, np.float64)
    o = _c(rays_o, np.float32).reshape(-1, 3)
    d = _c(rays_d, np.float32).reshape(-1, 3)
    out = np.empty((len(o), 3), np.float64)
    lib().or_prop_forward(_p(w), C.c_int(W), _p(o), _p(d), C.c_int(len(o)), C.c_double(in_scale),
                          C.c_double(t_scale), _p(out))
    return out


def prop_loss_grad(w, rays_o, rays_d, targets, in_scale, t_scale, W=32):
    w = _c(w, np.float64)
    o = _c(rays_o, np.float32).reshape(-1, 3)
    d = _c(rays_d, np.float32).reshape(-1, 3)
    tg = _c(targets, np.float64).reshape(-1, 3)
    g = np.zeros_like(w)
    f = lib().or_prop_loss_grad
    f.restype = C.c_double
    L = f(_p(w), C.c_int(W), _p(o), _p(d), C.c_int(len(o)), C.c_double(in_scale), C.c_double(t_scale), _p(tg), _p(g))
    return float(L), g


def _prop_targets(self, opts, cams=None, pix=None, rays_o=None, rays_d=None, W=None, H=None):
    W = W or self.cfg.W
    H = H or self.cfg.H
    cams, pix, ro, rd, n = self._rays(cams, pix, rays_o, rays_d)
    out = np.empty((n, 3), np.float64)
    op = self._opts(opts)
    lib().or_prop_targets(C.byref(self._s), C.byref(self._o), C.byref(op), _p(cams),
                          C.c_int(0 if cams is None else len(cams)), C.c_int(W), C.c_int(H), _p(pix), _p(ro), _p(rd),
                          C.c_int(n), _p(out))
    return out


Oracle.prop_targets = _prop_targets


def dist_step(x, d, rho, bounded=False):
    """World length of the distance step (Eq. 9) from points x along unit d for
    contracted radii rho (FP64)."""
    x = _c(x, np.float64).reshape(-1, 3)
    d = _c(d, np.float64).reshape(-1, 3)
    rho = _c(rho, np.float64).reshape(-1)
    out = np.empty(len(x), np.float64)
    lib().or_dist_step_batch(C.c_int(1 if bounded else 0), _p(x), _p(d), _p(rho), C.c_int(len(x)), _p(out))
    return out


def empty_step(x, d, Rk, R_O=None, bounded=False, handle=None):
    """s_O (Sec. 3.3) of world points x along unit d, each in its own voxel of a grid
    of Rk voxels per axis over the (contracted) domain, with the guard of the finest
    resolution R_O (default Rk) (FP64).  `handle`: another build of the oracle."""
    x = _c(x, np.float64).reshape(-1, 3)
    d = _c(d, np.float64).reshape(-1, 3)
    out = np.empty(len(x), np.float64)
    (handle or lib()).or_empty_step_batch(C.c_int(1 if bounded else 0), _p(x), _p(d), C.c_int(Rk), C.c_int(R_O or Rk),
                              C.c_int(len(x)), _p(out))
    return out
