"""Python binding of libngprt.so (the C ABI of ``include/ngprt.h``).

Argument marshalling only: every step of the render path runs in the library's
CUDA kernels.  Functions carry the C names and take torch CUDA tensors (device
memory), numpy arrays for host-side camera lists, and the current torch stream.
There is no fallback: if the library is missing or fails to load, ``lib()``
raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

ABI_VERSION = 201  # NGPRT_ABI_VERSION of include/ngprt.h that these structs and signatures follow
MAX_LEVELS = 32
MAX_CAMERAS = 64
STATE_FLOATS = 12
COARSE_BLOCK = 8  # cells per axis of a sparse coarse-grid block
COARSE_BLOCK_ROWS = 729  # its 9^3 stored vertices
F32, F16, BF16 = 0, 1, 2
_TORCH_DT = {F32: torch.float32, F16: torch.float16, BF16: torch.bfloat16}

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_CUDA, ERR_WORKSPACE, ERR_TIMEOUT = 0, -1, -2, -3, -4, -5


class NgprtError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__(f"{fn} failed ({code}): {msg}")
        self.code = code


class ngprt_scene(C.Structure):
    _fields_ = [("L", C.c_int32), ("T_log2", C.c_int32), ("N", C.c_int32 * MAX_LEVELS),
                ("table_dtype", C.c_int32), ("R_C", C.c_int32), ("mlp_layers", C.c_int32),
                ("mlp_width", C.c_int32), ("mlp_dtype", C.c_int32), ("bounded", C.c_int32),
                ("tables", C.c_void_p), ("coarse", C.c_void_p), ("mlp_w", C.c_void_p),
                ("aggregation", C.c_int32), ("attn_inv", C.c_void_p), ("agg_mlp", C.c_void_p),
                ("coarse_index", C.c_void_p), ("coarse_blocks", C.c_int64)]


class ngprt_occ(C.Structure):
    _fields_ = [("R_O", C.c_int32), ("n_levels", C.c_int32), ("bits", C.c_void_p), ("dist", C.c_void_p),
                ("R_G", C.c_int32)]


class ngprt_camera(C.Structure):
    _fields_ = [("c2w", C.c_float * 12), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("W", C.c_int32), ("H", C.c_int32)]


class ngprt_render_opts(C.Structure):
    _fields_ = [("step_base", C.c_float), ("step_gamma", C.c_float), ("t_min", C.c_float),
                ("r_far", C.c_float), ("t_term", C.c_float), ("bg", C.c_float * 3),
                ("max_march", C.c_int32), ("max_samples", C.c_int32), ("use_dist", C.c_int32),
                ("lattice_snap", C.c_int32), ("attn_mode", C.c_int32), ("dist_rule", C.c_int32)]


_P = C.c_void_p
_SIGS = {
    "ngprt_occ_bits_words": (C.c_size_t, [C.c_int32, C.c_int32]),
    "ngprt_build_occ_dist_workspace_bytes": (C.c_size_t, [C.c_int32]),
    "ngprt_build_occ_dist": (C.c_int32, [_P, C.c_int32, C.c_int32, C.c_int32, _P, _P, _P, C.c_size_t, _P]),
    "ngprt_table_entries": (C.c_int64, [_P]),
    "ngprt_coarse_channels": (C.c_int32, [C.c_int32, C.c_int32]),
    "ngprt_occupancy_from_density": (C.c_int32, [_P, _P, C.c_int32, C.c_float, _P, _P, _P]),
    "ngprt_occupancy_visibility": (C.c_int32, [_P, _P, _P, C.c_int32, _P, _P, _P, C.c_int64, _P, C.c_float,
                                               C.c_int32, _P, _P]),
    "ngprt_huber_loss": (C.c_int32, [_P, _P, C.c_int64, C.c_float, C.c_float, _P, _P, _P]),
    "ngprt_distortion_loss": (C.c_int32, [_P, _P, _P, C.c_int32, _P, _P, _P, C.c_int64, _P, C.c_float, _P, _P,
                                          _P]),
    "ngprt_distortion_backward": (C.c_int32, [_P, _P, _P, C.c_int32, _P, _P, _P, C.c_int64, _P, _P, C.c_float,
                                              _P, _P, _P, _P, _P, C.c_size_t, _P]),
    "ngprt_distortion_backward_workspace_bytes": (C.c_size_t, [_P, _P, C.c_int64]),
    "ngprt_mean_samples": (C.c_int32, [_P, C.c_int64, _P, _P]),
    "ngprt_step_autotune": (C.c_float, [C.c_float, C.c_float, C.c_float, C.c_float, C.c_float]),
    "ngprt_dilate_workspace_bytes": (C.c_size_t, [C.c_int32]),
    "ngprt_dilate": (C.c_int32, [_P, C.c_int32, C.c_int32, _P, _P, _P, C.c_size_t, _P]),
    "ngprt_render_workspace_bytes": (C.c_size_t, [_P, C.c_int64]),
    "ngprt_coarse_block_mask": (C.c_int32, [_P, C.c_int32, _P, _P]),
    "ngprt_coarse_sparsify_workspace_bytes": (C.c_size_t, [C.c_int32]),
    "ngprt_coarse_sparsify": (C.c_int32, [_P, C.c_int32, C.c_int32, _P, _P, _P, C.c_int64, _P, _P, C.c_size_t,
                                          _P]),
    "ngprt_render": (C.c_int32, [_P, _P, _P, C.c_int32, _P, _P, _P, C.c_int64, _P, _P, _P, _P, _P, _P, _P,
                                 _P, C.c_size_t, _P]),
    "ngprt_render_backward": (C.c_int32, [_P, _P, _P, C.c_int32, _P, _P, _P, C.c_int64, _P, _P, _P, _P, _P,
                                          _P, _P, _P, _P, _P, _P, C.c_size_t, _P]),
    "ngprt_render_backward_workspace_bytes": (C.c_size_t, [_P, _P, C.c_int64]),
    "ngprt_grid_indices": (C.c_int32, [_P, _P, C.c_int64, _P, _P]),
    "ngprt_shade": (C.c_int32, [_P, _P, C.c_int64, _P, _P, _P, _P, _P]),
    "ngprt_l2_loss": (C.c_int32, [_P, _P, C.c_int64, C.c_float, _P, _P, _P]),
    "ngprt_adam_step": (C.c_int32, [_P, _P, _P, _P, C.c_int64, C.c_float, C.c_float, C.c_float, C.c_float,
                                    C.c_int32, C.c_int32, _P]),
    "ngprt_proposal_param_count": (C.c_int32, []),
    "ngprt_propose": (C.c_int32, [_P, C.c_int32, _P, C.c_int32, _P, _P, _P, C.c_int64, C.c_float, C.c_float,
                                  C.c_float, C.c_float, C.c_float, _P, _P, _P]),
    "ngprt_propose_backward": (C.c_int32, [_P, _P, C.c_int32, _P, _P, _P, C.c_int64, C.c_float, C.c_float, _P, _P,
                                           _P, _P]),
    "ngprt_proposal_targets": (C.c_int32, [_P, _P, _P, C.c_int32, _P, _P, _P, C.c_int64, _P, _P, _P, _P]),
    "ngprt_render_fallback": (C.c_int32, [_P, _P, _P, C.c_int32, _P, _P, _P, C.c_int64, _P, _P, C.c_float, _P, _P,
                                          _P, _P]),
    "ngprt_render_noalloc_max_rays": (C.c_int64, []),
    "ngprt_render_noalloc": (C.c_int32, [_P, _P, _P, C.c_int32, _P, _P, _P, C.c_int64, _P, _P, _P, _P, _P, _P,
                                         _P]),
    "ngprt_tensor_core_error": (C.c_int32, []),
    "ngprt_sync_status": (C.c_int32, [_P]),
    "ngprt_test_bounded_wait": (C.c_int32, [C.c_int32, _P]),
    "ngprt_count_nonfinite": (C.c_int32, [_P, C.c_int64, _P, _P]),
    "ngprt_last_error": (C.c_char_p, []),
    "ngprt_version": (C.c_int32, []),
}

_lib = None


def lib_path() -> str:
    """The in-tree build, or the file named by NGPRT_LIB (for comparing builds)."""
    return os.environ.get("NGPRT_LIB", _build.LIB)


def lib(build_if_missing: bool = False):
    """Load libngprt.so (raises if it is absent; never falls back to anything)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            if not build_if_missing or path != _build.LIB:
                raise RuntimeError(f"{path} is missing: build it with `python -m paper_2407_10482_gb300.build`")
            _build.build()
        h = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(h, name)
            f.restype = res
            f.argtypes = args
        if h.ngprt_version() != ABI_VERSION:
            raise RuntimeError(f"{path} has ABI version {h.ngprt_version()}, this binding {ABI_VERSION}: rebuild it")
        _lib = h
    return _lib


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
        return t.data_ptr()
    return int(t)


def _stream(stream=None) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _check(fn: str, rc: int) -> None:
    if rc != OK:
        raise NgprtError(fn, rc, lib().ngprt_last_error().decode())


# ---------------------------------------------------------------- raw C calls

def ngprt_occ_bits_words(R: int, n_levels: int) -> int:
    return int(lib().ngprt_occ_bits_words(R, n_levels))


def ngprt_build_occ_dist_workspace_bytes(R: int) -> int:
    return int(lib().ngprt_build_occ_dist_workspace_bytes(R))


def ngprt_build_occ_dist(occ, R, n_levels, occ_bits_out, dist_out, workspace, stream=None, dist_level=0) -> None:
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check("ngprt_build_occ_dist", lib().ngprt_build_occ_dist(
        _ptr(occ), R, n_levels, dist_level, _ptr(occ_bits_out), _ptr(dist_out), _ptr(workspace), ws_bytes,
        _stream(stream)))


def ngprt_table_entries(scene: ngprt_scene) -> int:
    return int(lib().ngprt_table_entries(C.byref(scene)))


def ngprt_coarse_channels(L: int, aggregation: int) -> int:
    return int(lib().ngprt_coarse_channels(L, aggregation))


def ngprt_occupancy_from_density(scene, opts, R, sigma_thr, occ_out, sigma_out=None, stream=None) -> None:
    _check("ngprt_occupancy_from_density", lib().ngprt_occupancy_from_density(
        C.byref(scene), C.byref(opts), R, sigma_thr, _ptr(occ_out), _ptr(sigma_out), _stream(stream)))


def ngprt_occupancy_visibility(scene, occ, cams, n_cams, pixel_ids, rays_o, rays_d, n_rays, opts, w_thr, R, vis,
                               stream=None) -> None:
    _check("ngprt_occupancy_visibility", lib().ngprt_occupancy_visibility(
        C.byref(scene), C.byref(occ), cams, n_cams, _ptr(pixel_ids), _ptr(rays_o), _ptr(rays_d), n_rays,
        C.byref(opts), w_thr, R, _ptr(vis), _stream(stream)))


def ngprt_huber_loss(rgb, target, n, delta, scale, loss=None, d_rgb=None, stream=None) -> None:
    _check("ngprt_huber_loss", lib().ngprt_huber_loss(_ptr(rgb), _ptr(target), n, delta, scale, _ptr(loss),
                                                      _ptr(d_rgb), _stream(stream)))


def ngprt_distortion_loss(scene, occ, cams, n_cams, pixel_ids, rays_o, rays_d, n_rays, opts, scale, dist_state,
                          loss=None, stream=None) -> None:
    _check("ngprt_distortion_loss", lib().ngprt_distortion_loss(
        C.byref(scene), C.byref(occ), cams, n_cams, _ptr(pixel_ids), _ptr(rays_o), _ptr(rays_d), n_rays,
        C.byref(opts), scale, _ptr(dist_state), _ptr(loss), _stream(stream)))


def ngprt_distortion_backward(scene, occ, cams, n_cams, pixel_ids, rays_o, rays_d, n_rays, opts, dist_state, scale,
                              g_tables, g_coarse, stream=None, g_attn_inv=None, g_agg_mlp=None,
                              workspace=None) -> None:
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check("ngprt_distortion_backward", lib().ngprt_distortion_backward(
        C.byref(scene), C.byref(occ), cams, n_cams, _ptr(pixel_ids), _ptr(rays_o), _ptr(rays_d), n_rays,
        C.byref(opts), _ptr(dist_state), scale, _ptr(g_tables), _ptr(g_coarse), _ptr(g_attn_inv), _ptr(g_agg_mlp),
        _ptr(workspace), ws_bytes, _stream(stream)))


def ngprt_distortion_backward_workspace_bytes(scene, opts, n_rays) -> int:
    return int(lib().ngprt_distortion_backward_workspace_bytes(C.byref(scene), C.byref(opts), n_rays))


def ngprt_mean_samples(ray_stats, n_rays, out, stream=None) -> None:
    _check("ngprt_mean_samples", lib().ngprt_mean_samples(_ptr(ray_stats), n_rays, _ptr(out), _stream(stream)))


def ngprt_step_autotune(gamma, n_mean, n_min=3.0, kappa=1e-3, gamma_min=0.2217) -> float:
    return float(lib().ngprt_step_autotune(gamma, n_mean, n_min, kappa, gamma_min))


def ngprt_sync_status(stream=None) -> None:
    """Raises NgprtError (code ERR_TIMEOUT or ERR_CUDA) for a device-side failure."""
    _check("ngprt_sync_status", lib().ngprt_sync_status(_stream(stream)))


def ngprt_test_bounded_wait(limit, stream=None) -> None:
    _check("ngprt_test_bounded_wait", lib().ngprt_test_bounded_wait(limit, _stream(stream)))


def ngprt_count_nonfinite(x, n, count, stream=None) -> None:
    _check("ngprt_count_nonfinite", lib().ngprt_count_nonfinite(_ptr(x), n, _ptr(count), _stream(stream)))


def ngprt_dilate_workspace_bytes(R: int) -> int:
    return int(lib().ngprt_dilate_workspace_bytes(R))


def ngprt_dilate(occ, R, radius, out, workspace, mask=None, stream=None) -> None:
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check("ngprt_dilate", lib().ngprt_dilate(_ptr(occ), R, radius, _ptr(mask), _ptr(out), _ptr(workspace), ws_bytes,
                                              _stream(stream)))


def ngprt_render_workspace_bytes(scene: ngprt_scene, n_rays: int) -> int:
    return int(lib().ngprt_render_workspace_bytes(C.byref(scene), n_rays))


def cameras_struct(cams: np.ndarray, W: int, H: int):
    """Host array of ngprt_camera from float [V][16] (c2w 3x4, fx, fy, cx, cy)."""
    cams = np.asarray(cams, np.float32).reshape(-1, 16)
    arr = (ngprt_camera * len(cams))()
    for i, c in enumerate(cams):
        for k in range(12):
            arr[i].c2w[k] = float(c[k])
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = (float(v) for v in c[12:16])
        arr[i].W, arr[i].H = W, H
    return arr, len(cams)


def ngprt_render(scene, occ, cams, n_cams, pixel_ids, rays_o, rays_d, n_rays, t_interval, opts, rgb,
                 depth=None, opacity=None, ray_stats=None, ray_state=None, workspace=None, stream=None) -> None:
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check("ngprt_render", lib().ngprt_render(
        C.byref(scene), C.byref(occ), cams, n_cams, _ptr(pixel_ids), _ptr(rays_o), _ptr(rays_d), n_rays,
        _ptr(t_interval), C.byref(opts), _ptr(rgb), _ptr(depth), _ptr(opacity), _ptr(ray_stats), _ptr(ray_state),
        _ptr(workspace), ws_bytes, _stream(stream)))


def ngprt_render_backward(scene, occ, cams, n_cams, pixel_ids, rays_o, rays_d, n_rays, opts, ray_state, d_rgb,
                          d_depth, d_opacity, g_tables, g_coarse, g_mlp, workspace=None, stream=None,
                          g_attn_inv=None, g_agg_mlp=None) -> None:
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check("ngprt_render_backward", lib().ngprt_render_backward(
        C.byref(scene), C.byref(occ), cams, n_cams, _ptr(pixel_ids), _ptr(rays_o), _ptr(rays_d), n_rays,
        C.byref(opts), _ptr(ray_state), _ptr(d_rgb), _ptr(d_depth), _ptr(d_opacity), _ptr(g_tables),
        _ptr(g_coarse), _ptr(g_mlp), _ptr(g_attn_inv), _ptr(g_agg_mlp), _ptr(workspace), ws_bytes,
        _stream(stream)))


def ngprt_render_backward_workspace_bytes(scene, opts, n_rays) -> int:
    return int(lib().ngprt_render_backward_workspace_bytes(C.byref(scene), C.byref(opts), n_rays))


def coarse_blocks_per_axis(R_C: int) -> int:
    return (R_C - 1 + COARSE_BLOCK - 1) // COARSE_BLOCK


def ngprt_coarse_block_mask(occ, R_C, block_mask, stream=None) -> None:
    _check("ngprt_coarse_block_mask", lib().ngprt_coarse_block_mask(C.byref(occ), R_C, _ptr(block_mask),
                                                                    _stream(stream)))


def ngprt_coarse_sparsify_workspace_bytes(R_C) -> int:
    return int(lib().ngprt_coarse_sparsify_workspace_bytes(R_C))


def ngprt_coarse_sparsify(dense, R_C, row_bytes, block_mask, index, blocks, max_blocks, workspace,
                          stream=None) -> int:
    """Index (and, with `blocks`, the blocks) of the sparse coarse grid; returns the
    stored block count (slot 0 = zeros included)."""
    n = C.c_int64(0)
    ws_bytes = workspace.numel() * workspace.element_size()
    _check("ngprt_coarse_sparsify", lib().ngprt_coarse_sparsify(
        _ptr(dense), R_C, row_bytes, _ptr(block_mask), _ptr(index), _ptr(blocks), max_blocks, C.byref(n),
        _ptr(workspace), ws_bytes, _stream(stream)))
    return int(n.value)


def ngprt_shade(scene, ray_state, n_rays, bg, rgb, depth=None, opacity=None, stream=None) -> None:
    bgv = (C.c_float * 3)(*[float(b) for b in bg])
    _check("ngprt_shade", lib().ngprt_shade(C.byref(scene), _ptr(ray_state), n_rays, bgv, _ptr(rgb), _ptr(depth),
                                            _ptr(opacity), _stream(stream)))


def ngprt_l2_loss(rgb, target, n, scale, loss=None, d_rgb=None, stream=None) -> None:
    _check("ngprt_l2_loss", lib().ngprt_l2_loss(_ptr(rgb), _ptr(target), n, scale, _ptr(loss), _ptr(d_rgb),
                                                _stream(stream)))


def ngprt_adam_step(param, grad, m, v, lr, beta1=0.9, beta2=0.99, eps=1e-8, step=1, zero_grad=True,
                    stream=None) -> None:
    _check("ngprt_adam_step", lib().ngprt_adam_step(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(), lr,
                                                    beta1, beta2, eps, step, int(zero_grad), _stream(stream)))


def ngprt_proposal_param_count() -> int:
    return int(lib().ngprt_proposal_param_count())


def ngprt_propose(prop_w, cams, n_cams, pixel_ids, rays_o, rays_d, n_rays, in_scale, t_scale, margin_near,
                  margin_far, a_min, t_interval_out, a_hat_out=None, stream=None) -> None:
    """prop_w: float32 or float16 device tensor (the dtype is passed on)."""
    dt = F16 if prop_w.dtype == torch.float16 else F32
    _check("ngprt_propose", lib().ngprt_propose(
        _ptr(prop_w), dt, cams, n_cams, _ptr(pixel_ids), _ptr(rays_o), _ptr(rays_d), n_rays, in_scale, t_scale,
        margin_near, margin_far, a_min, _ptr(t_interval_out), _ptr(a_hat_out), _stream(stream)))


def ngprt_propose_backward(prop_w, cams, n_cams, pixel_ids, rays_o, rays_d, n_rays, in_scale, t_scale, targets,
                           g_prop_w, loss=None, stream=None) -> None:
    _check("ngprt_propose_backward", lib().ngprt_propose_backward(
        _ptr(prop_w), cams, n_cams, _ptr(pixel_ids), _ptr(rays_o), _ptr(rays_d), n_rays, in_scale, t_scale,
        _ptr(targets), _ptr(g_prop_w), _ptr(loss), _stream(stream)))


def ngprt_proposal_targets(scene, occ, cams, n_cams, pixel_ids, rays_o, rays_d, n_rays, opts, ray_state, targets,
                           stream=None) -> None:
    _check("ngprt_proposal_targets", lib().ngprt_proposal_targets(
        C.byref(scene), C.byref(occ), cams, n_cams, _ptr(pixel_ids), _ptr(rays_o), _ptr(rays_d), n_rays,
        C.byref(opts), _ptr(ray_state), _ptr(targets), _stream(stream)))


def ngprt_render_fallback(scene, occ, cams, n_cams, pixel_ids, rays_o, rays_d, n_rays, t_interval, a_hat, threshold,
                          opts, ray_state, ray_stats=None, stream=None) -> None:
    _check("ngprt_render_fallback", lib().ngprt_render_fallback(
        C.byref(scene), C.byref(occ), cams, n_cams, _ptr(pixel_ids), _ptr(rays_o), _ptr(rays_d), n_rays,
        _ptr(t_interval), _ptr(a_hat), threshold, C.byref(opts), _ptr(ray_state), _ptr(ray_stats), _stream(stream)))


def ngprt_render_noalloc_max_rays() -> int:
    return int(lib().ngprt_render_noalloc_max_rays())


def ngprt_render_noalloc(scene, occ, cams, n_cams, pixel_ids, rays_o, rays_d, n_rays, t_interval, opts, rgb,
                         depth=None, opacity=None, ray_stats=None, stream=None) -> None:
    """ngprt_render with its scratch in the library's static device array (no
    allocation anywhere); at most ngprt_render_noalloc_max_rays() rays per call."""
    _check("ngprt_render_noalloc", lib().ngprt_render_noalloc(
        C.byref(scene), C.byref(occ), cams, n_cams, _ptr(pixel_ids), _ptr(rays_o), _ptr(rays_d), n_rays,
        _ptr(t_interval), C.byref(opts), _ptr(rgb), _ptr(depth), _ptr(opacity), _ptr(ray_stats), _stream(stream)))


def ngprt_grid_indices(scene, u, n, idx_out, stream=None) -> None:
    _check("ngprt_grid_indices", lib().ngprt_grid_indices(C.byref(scene), _ptr(u), n, _ptr(idx_out),
                                                           _stream(stream)))


# ------------------------------------------------------- device-side objects

def render_opts(o) -> ngprt_render_opts:
    """ngprt_render_opts from any object with the RenderOptions fields."""
    p = ngprt_render_opts()
    p.step_base, p.step_gamma, p.t_min, p.r_far, p.t_term = (
        o.step_base, o.step_gamma, o.t_min, o.r_far, o.t_term)
    for k in range(3):
        p.bg[k] = float(o.bg[k])
    p.max_march, p.max_samples = int(o.max_march), int(o.max_samples)
    p.use_dist, p.lattice_snap = int(bool(o.use_dist)), int(bool(o.lattice_snap))
    p.attn_mode, p.dist_rule = int(o.attn_mode), int(o.dist_rule)
    return p


def _device_array(a, dtype, device):
    """A contiguous device tensor of `dtype` from a numpy array or a tensor."""
    if isinstance(a, torch.Tensor):
        return a.to(device=device, dtype=dtype).contiguous()
    return torch.as_tensor(np.asarray(a, np.float32)).to(device=device, dtype=dtype).contiguous()


class DeviceScene:
    """Scene arrays resident on the GPU plus the ngprt_scene struct pointing at them.

    ``tables``/``coarse`` are uploaded in ``table_dtype`` (F32, F16 or BF16; the
    16-bit forms round to nearest even from the FP32 master)."""

    def __init__(self, cfg, tables, coarse, mlp_w, table_dtype: int = F32, device="cuda", mlp_dtype: int = F32,
                 attn_inv=None, agg_mlp=None):
        dt = _TORCH_DT[table_dtype]
        self.cfg = cfg
        self.table_dtype = table_dtype
        self.mlp_dtype = mlp_dtype
        self.aggregation = int(getattr(cfg, "aggregation", 0))
        self.tables = _device_array(tables, dt, device)
        self.coarse = _device_array(coarse, dt, device)
        self.mlp_w = _device_array(mlp_w, _TORCH_DT[mlp_dtype], device)
        self.attn_inv = None if attn_inv is None else _device_array(attn_inv, torch.float32, device)
        self.agg_mlp = None if agg_mlp is None else _device_array(agg_mlp, torch.float32, device)
        self.coarse_index = None
        self.coarse_blocks = 0
        self.refresh()

    def sparsify_coarse(self, occ: "DeviceOcc") -> None:
        """Replace the dense coarse grid by its block-indexed sparse form: the 8^3-cell
        blocks that the occupied voxels of ``occ`` reach (ngprt_coarse_block_mask), each
        stored as its 9^3 vertices.  Renders are unchanged; the reverse passes then
        refuse the scene."""
        assert self.coarse_index is None, "already sparse"
        R_C = self.cfg.R_C
        nb = coarse_blocks_per_axis(R_C)
        dev = self.coarse.device
        mask = torch.empty(nb ** 3, dtype=torch.uint8, device=dev)
        ngprt_coarse_block_mask(occ.struct, R_C, mask)
        index = torch.empty(nb ** 3, dtype=torch.int32, device=dev)
        ws = torch.empty(ngprt_coarse_sparsify_workspace_bytes(R_C), dtype=torch.uint8, device=dev)
        nch = self.coarse.shape[1]
        row_bytes = nch * self.coarse.element_size()
        n = ngprt_coarse_sparsify(self.coarse, R_C, row_bytes, mask, index, None, 0, ws)
        blocks = torch.empty(n, COARSE_BLOCK_ROWS, nch, dtype=self.coarse.dtype, device=dev)
        ngprt_coarse_sparsify(self.coarse, R_C, row_bytes, mask, index, blocks, n, ws)
        self.coarse, self.coarse_index, self.coarse_blocks = blocks, index, n
        self.refresh()

    def refresh(self) -> None:
        s = ngprt_scene()
        c = self.cfg
        s.L, s.T_log2 = c.L, c.T_log2
        for i, n in enumerate(c.N):
            s.N[i] = int(n)
        s.table_dtype, s.R_C = self.table_dtype, c.R_C
        s.mlp_layers, s.mlp_width, s.mlp_dtype = c.mlp_layers, c.mlp_width, self.mlp_dtype
        s.bounded = 1 if c.bounded else 0
        s.tables, s.coarse, s.mlp_w = _ptr(self.tables), _ptr(self.coarse), _ptr(self.mlp_w)
        s.aggregation = self.aggregation
        s.attn_inv, s.agg_mlp = _ptr(self.attn_inv), _ptr(self.agg_mlp)
        s.coarse_index, s.coarse_blocks = _ptr(self.coarse_index), self.coarse_blocks
        self.struct = s


class DeviceOcc:
    """Occupancy pyramid and distance grid built on the GPU by ngprt_build_occ_dist."""

    def __init__(self, occ: np.ndarray, R: int, n_levels: int, with_dist: bool = True, device="cuda",
                 dist_level: int = 0):
        self.R, self.n_levels = R, n_levels
        self.R_G = R >> dist_level
        self.occ = (occ.to(device=device, dtype=torch.uint8) if isinstance(occ, torch.Tensor)
                    else torch.as_tensor(np.asarray(occ, np.uint8)).to(device)).contiguous()
        self.bits = torch.empty(ngprt_occ_bits_words(R, n_levels), dtype=torch.int32, device=device)
        self.dist = torch.empty(self.R_G ** 3, dtype=torch.uint8, device=device) if with_dist else None
        ws = torch.empty(ngprt_build_occ_dist_workspace_bytes(R), dtype=torch.uint8, device=device)
        ngprt_build_occ_dist(self.occ, R, n_levels, self.bits, self.dist, ws, dist_level=dist_level)
        self.struct = ngprt_occ(R, n_levels, _ptr(self.bits), _ptr(self.dist), self.R_G)
        self.struct_nodist = ngprt_occ(R, n_levels, _ptr(self.bits), None, self.R_G)


class Renderer:
    """Owns output and workspace tensors for repeated renders of one ray count."""

    def __init__(self, scene: DeviceScene, occ: DeviceOcc, device="cuda"):
        self.scene, self.occ, self.device = scene, occ, device
        self._ws = None
        self._bws = None  # the reverse pass's workspace

    def workspace(self, n_rays: int):
        need = ngprt_render_workspace_bytes(self.scene.struct, n_rays)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        return self._ws

    def render(self, opts, cams=None, W=None, H=None, pixel_ids=None, rays_o=None, rays_d=None,
               t_interval=None, stats=False, state=False, use_dist=True, out=None):
        if cams is not None:
            cam_arr, n_cams = cameras_struct(cams, W, H)
            n = len(pixel_ids) if pixel_ids is not None else n_cams * W * H
        else:
            cam_arr, n_cams = None, 0
            n = rays_o.shape[0]
        dev = self.device
        if out is None:
            out = dict(rgb=torch.empty(n, 3, device=dev), depth=torch.empty(n, device=dev),
                       opacity=torch.empty(n, device=dev))
            if stats:
                out["stats"] = torch.empty(n, 2, dtype=torch.int32, device=dev)
            if state:
                out["state"] = torch.empty(n, STATE_FLOATS, device=dev)
        occ = self.occ.struct if use_dist else self.occ.struct_nodist
        ngprt_render(self.scene.struct, occ, cam_arr, n_cams, pixel_ids, rays_o, rays_d, n, t_interval,
                     render_opts(opts), out["rgb"], out.get("depth"), out.get("opacity"), out.get("stats"),
                     out.get("state"), self.workspace(n))
        return out


class RenderFunction(torch.autograd.Function):
    """Differentiable render: (tables, coarse, mlp_w[, attn_inv]) -> (rgb, depth, opacity)
    through ngprt_render and ngprt_render_backward (gradients accumulate with atomics).
    attn_inv is the scene's constant gate logits (the spatially invariant gate forms)."""

    @staticmethod
    def forward(ctx, tables, coarse, mlp_w, renderer, opts, rays, attn_inv=None, agg_mlp=None):
        scene = renderer.scene
        assert tables.data_ptr() == scene.tables.data_ptr() and coarse.data_ptr() == scene.coarse.data_ptr()
        assert mlp_w.data_ptr() == scene.mlp_w.data_ptr()
        assert attn_inv is None or attn_inv.data_ptr() == scene.attn_inv.data_ptr()
        assert agg_mlp is None or agg_mlp.data_ptr() == scene.agg_mlp.data_ptr()
        out = renderer.render(opts, state=True, **rays)
        ctx.renderer, ctx.opts, ctx.rays = renderer, opts, rays
        ctx.save_for_backward(out["state"])
        return out["rgb"], out["depth"], out["opacity"]

    @staticmethod
    def backward(ctx, d_rgb, d_depth, d_opacity):
        (state,) = ctx.saved_tensors
        r = ctx.renderer
        s = r.scene
        g_t = torch.zeros_like(s.tables)
        g_c = torch.zeros_like(s.coarse)
        g_m = torch.zeros_like(s.mlp_w)
        g_i = torch.zeros_like(s.attn_inv) if s.attn_inv is not None else None
        g_a = torch.zeros_like(s.agg_mlp) if s.agg_mlp is not None else None
        r.backward(ctx.opts, state, d_rgb.contiguous(), None if d_depth is None else d_depth.contiguous(),
                   None if d_opacity is None else d_opacity.contiguous(), g_t, g_c, g_m, g_attn_inv=g_i,
                   g_agg_mlp=g_a, **ctx.rays)
        return g_t, g_c, g_m, None, None, None, g_i, g_a


def _renderer_backward(self, opts, state, d_rgb, d_depth, d_opacity, g_tables, g_coarse, g_mlp, cams=None, W=None,
                       H=None, pixel_ids=None, rays_o=None, rays_d=None, t_interval=None, g_attn_inv=None,
                       g_agg_mlp=None):
    if cams is not None:
        cam_arr, n_cams = cameras_struct(cams, W, H)
        n = len(pixel_ids) if pixel_ids is not None else n_cams * W * H
    else:
        cam_arr, n_cams = None, 0
        n = rays_o.shape[0]
    ro = render_opts(opts)
    need = ngprt_render_backward_workspace_bytes(self.scene.struct, ro, n)
    if self._bws is None or self._bws.numel() < need:
        self._bws = torch.empty(need, dtype=torch.uint8, device=self.device)
    ngprt_render_backward(self.scene.struct, self.occ.struct, cam_arr, n_cams, pixel_ids, rays_o, rays_d, n,
                          ro, state, d_rgb, d_depth, d_opacity, g_tables, g_coarse, g_mlp, self._bws,
                          g_attn_inv=g_attn_inv, g_agg_mlp=g_agg_mlp)


Renderer.backward = _renderer_backward
