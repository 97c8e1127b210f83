"""Host-side checks of the C ABI, no GPU needed: libngprt.so builds and loads, it
exports every function include/ngprt.h declares, size queries match the layout
rules, and argument errors return status codes before anything is launched."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2407_10482_gb300 import build as B
from paper_2407_10482_gb300 import scenes as S

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ngprt.h")


@pytest.fixture(scope="module")
def ng():
    B.build()
    from paper_2407_10482_gb300 import ngprt
    ngprt.lib()
    return ngprt


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ngprt_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(ng):
    names = declared_functions()
    assert len(names) >= 15
    h = C.CDLL(ng.lib_path())
    missing = [n for n in names if not hasattr(h, n)]
    assert not missing, missing
    assert set(names) <= set(ng._SIGS), "binding lacks a signature"


def test_size_queries(ng):
    assert ng.ngprt_occ_bits_words(128, 5) == (128 ** 3 + 64 ** 3 + 32 ** 3 + 16 ** 3 + 8 ** 3) // 32
    assert ng.ngprt_occ_bits_words(2, 2) == 2  # 8 bits -> 1 word, 1 bit -> 1 word
    cfg = S.hd_config()
    s = ng.ngprt_scene()
    s.L, s.T_log2 = cfg.L, cfg.T_log2
    for i, n in enumerate(cfg.N):
        s.N[i] = n
    assert ng.ngprt_table_entries(s) == S.table_entries(cfg) == 6272960
    assert ng.ngprt_render_workspace_bytes(s, 1000) >= 1000 * ng.STATE_FLOATS * 4
    assert ng.ngprt_proposal_param_count() == 1379
    assert ng.lib().ngprt_version() == ng.ABI_VERSION == 201


def test_argument_errors_are_reported_without_a_launch(ng):
    lib = ng.lib()
    rc = lib.ngprt_render(None, None, None, 0, None, None, None, 10, None, None, None, None, None, None, None,
                          None, 0, None)
    assert rc == ng.ERR_INVALID_ARG
    assert b"scene is NULL" in lib.ngprt_last_error()
    # R not a power of two
    rc = lib.ngprt_build_occ_dist(C.c_void_p(256), 12, 2, 0, C.c_void_p(256), None, None, 0, None)
    assert rc == ng.ERR_INVALID_ARG and b"power of two" in lib.ngprt_last_error()
    # an L without a kernel
    cfg = S.small_config()
    s = ng.ngprt_scene()
    s.L, s.T_log2, s.R_C, s.mlp_layers, s.mlp_width = 5, 12, 16, 2, 16
    for i in range(5):
        s.N[i] = 16
    s.tables = s.coarse = s.mlp_w = 256
    o = ng.ngprt_occ(32, 3, 256, None)
    opts = ng.render_opts(S.default_options(cfg))
    rc = lib.ngprt_render(C.byref(s), C.byref(o), None, 0, None, C.c_void_p(256), C.c_void_p(256), 4, None,
                          C.byref(opts), C.c_void_p(256), None, None, None, None, None, 0, None)
    assert rc == ng.ERR_INVALID_ARG and b"L=5" in lib.ngprt_last_error()
    # misaligned F32 tables
    s.L = 4
    s.tables = 256 + 16
    rc = lib.ngprt_render(C.byref(s), C.byref(o), None, 0, None, C.c_void_p(256), C.c_void_p(256), 4, None,
                          C.byref(opts), C.c_void_p(256), None, None, None, None, None, 0, None)
    assert rc == ng.ERR_INVALID_ARG and b"aligned" in lib.ngprt_last_error()
    # bad options
    s.tables = 256
    opts.attn_mode = 7
    rc = lib.ngprt_render(C.byref(s), C.byref(o), None, 0, None, C.c_void_p(256), C.c_void_p(256), 4, None,
                          C.byref(opts), C.c_void_p(256), None, None, None, None, None, 0, None)
    assert rc == ng.ERR_INVALID_ARG and b"attn_mode" in lib.ngprt_last_error()


def test_aggregation_layouts_and_validation(ng):
    """Coarse-grid channel counts of the Table 3 aggregations and the host-side checks
    (no device work: every call below returns before any launch)."""
    from oracle import oracle as O
    lib = ng.lib()
    for L in (2, 4, 16):
        for agg in range(6):
            n = ng.ngprt_coarse_channels(L, agg)
            assert n == O.coarse_channels(L, agg) == S.coarse_channels(S.small_config(L=L, aggregation=agg))
    assert ng.ngprt_coarse_channels(4, 6) == 0 and ng.ngprt_coarse_channels(0, 0) == 0
    cfg = S.small_config()
    s = ng.ngprt_scene()
    s.L, s.T_log2, s.R_C, s.mlp_layers, s.mlp_width = 4, 12, 16, 2, 16
    for i in range(4):
        s.N[i] = 16 << i
    s.tables = s.coarse = s.mlp_w = 256
    o = ng.ngprt_occ(32, 3, 256, None)
    opts = ng.render_opts(S.default_options(cfg))

    def render():
        return lib.ngprt_render(C.byref(s), C.byref(o), None, 0, None, C.c_void_p(256), C.c_void_p(256), 4, None,
                                C.byref(opts), C.c_void_p(256), None, None, None, None, None, 0, None)
    s.aggregation = 9
    assert render() == ng.ERR_INVALID_ARG and b"aggregation" in lib.ngprt_last_error()
    s.aggregation = 2                       # invariant gates without their logits
    assert render() == ng.ERR_INVALID_ARG and b"attn_inv" in lib.ngprt_last_error()
    s.aggregation = 5                       # MLP aggregation, misaligned weights
    s.agg_mlp = 256 + 4
    assert render() == ng.ERR_INVALID_ARG and b"agg_mlp" in lib.ngprt_last_error()
    s.aggregation, s.agg_mlp = 4, None
    opts.attn_mode = 1                      # attn_mode belongs to the Eq. 8 layout
    assert render() == ng.ERR_INVALID_ARG and b"attn_mode" in lib.ngprt_last_error()
    opts.attn_mode = 0
    s.L = 3                                 # no variant kernel for L = 3
    assert render() == ng.ERR_UNSUPPORTED and b"L=3" in lib.ngprt_last_error()
    s.L = 4

    def backward(g_inv=None):
        return lib.ngprt_render_backward(C.byref(s), C.byref(o), None, 0, None, C.c_void_p(256), C.c_void_p(256),
                                         4, C.byref(opts), C.c_void_p(256), C.c_void_p(256), None, None,
                                         C.c_void_p(256), C.c_void_p(256), C.c_void_p(256), g_inv, None, None, 0,
                                         None)
    s.aggregation, s.agg_mlp = 5, 256  # the MLP form needs its weight gradient buffer
    assert backward() == ng.ERR_INVALID_ARG and b"g_agg_mlp" in lib.ngprt_last_error()
    s.aggregation, s.agg_mlp, s.attn_inv = 2, None, 256
    assert backward() == ng.ERR_INVALID_ARG and b"g_attn_inv" in lib.ngprt_last_error()
    s.L = 3                                 # no variant reverse pass for L = 3
    assert backward(C.c_void_p(256)) == ng.ERR_UNSUPPORTED and b"L=3" in lib.ngprt_last_error()


def test_step_autotune_matches_oracle(ng):
    """Eq. S3's controller runs on the host: the library's FP32 result equals the
    oracle's FP64 one rounded, on both branches and both clamps."""
    from oracle import oracle as O
    rng = np.random.default_rng(0)
    for _ in range(200):
        g = float(np.float32(rng.uniform(0.2, 1.0)))
        n_mean = float(np.float32(rng.uniform(0.0, 6.0)))
        want = O.step_autotune(g, n_mean, 3.0, 1e-3, float(np.float32(0.2217)))
        got = ng.ngprt_step_autotune(g, n_mean, 3.0, 1e-3, 0.2217)
        assert abs(got - want) <= 1e-6 * want


def test_sparse_coarse_grid_validation(ng):
    """The sparse coarse grid's fields are checked before any launch."""
    lib = ng.lib()
    s = ng.ngprt_scene()
    s.L, s.T_log2, s.R_C, s.mlp_layers, s.mlp_width = 4, 12, 16, 2, 16
    for i in range(4):
        s.N[i] = 16 << i
    s.tables = s.coarse = s.mlp_w = 256
    o = ng.ngprt_occ(32, 3, 256, None)
    opts = ng.render_opts(S.default_options(S.small_config()))

    def render():
        return lib.ngprt_render(C.byref(s), C.byref(o), None, 0, None, C.c_void_p(256), C.c_void_p(256), 4, None,
                                C.byref(opts), C.c_void_p(256), None, None, None, None, None, 0, None)
    s.coarse_index, s.coarse_blocks = 256, 0
    assert render() == ng.ERR_INVALID_ARG and b"coarse_blocks" in lib.ngprt_last_error()
    s.coarse_index, s.coarse_blocks = 258, 3
    assert render() == ng.ERR_INVALID_ARG and b"coarse_index" in lib.ngprt_last_error()
    s.coarse_index = 256
    rc = lib.ngprt_render_backward(C.byref(s), C.byref(o), None, 0, None, C.c_void_p(256), C.c_void_p(256), 4,
                                   C.byref(opts), C.c_void_p(256), C.c_void_p(256), None, None, C.c_void_p(256),
                                   C.c_void_p(256), C.c_void_p(256), None, None, None, 0, None)
    assert rc == ng.ERR_INVALID_ARG and b"dense coarse grid" in lib.ngprt_last_error()
    assert ng.ngprt_coarse_sparsify_workspace_bytes(512) >= 16 + 2 * 4 * 256
    assert ng.ngprt_coarse_sparsify_workspace_bytes(1) == 0
    n = C.c_int64(0)
    rc = lib.ngprt_coarse_sparsify(None, 512, 6, C.c_void_p(256), C.c_void_p(256), None, 0, C.byref(n),
                                   C.c_void_p(256), 1 << 20, None)
    assert rc == ng.ERR_INVALID_ARG and b"row_bytes" in lib.ngprt_last_error()
    rc = lib.ngprt_coarse_sparsify(None, 512, 48, C.c_void_p(256), C.c_void_p(256), None, 0, C.byref(n),
                                   C.c_void_p(256), 8, None)
    assert rc == ng.ERR_WORKSPACE


def test_reverse_pass_workspace_sizes(ng):
    """The reverse passes' workspace: per-ray cotangents for every form, plus one
    (f^1..f^L, g_f) record per possible sample for the tiny-MLP form."""
    lib = ng.lib()
    s = ng.ngprt_scene()
    s.L, s.T_log2, s.R_C = 4, 12, 16
    opts = ng.render_opts(S.default_options(S.small_config(), max_samples=100))
    n = 1000
    cot = (n * 12 * 4 + 255) // 256 * 256 + 256
    for agg in range(5):
        s.aggregation = agg
        assert ng.ngprt_render_backward_workspace_bytes(s, opts, n) == cot
        assert ng.ngprt_distortion_backward_workspace_bytes(s, opts, n) == 0
    s.aggregation = 5
    rec = 256 + n * 100 * (8 * 4 + 8) * 4
    assert ng.ngprt_render_backward_workspace_bytes(s, opts, n) == cot + rec
    assert ng.ngprt_distortion_backward_workspace_bytes(s, opts, n) == rec
    assert lib.ngprt_render_backward_workspace_bytes(None, C.byref(opts), n) == 0
    assert ng.ngprt_render_backward_workspace_bytes(s, opts, -1) == 0


def test_distortion_reverse_pass_argument_checks(ng):
    """The regulariser's reverse pass asks each form for its own outputs before any
    launch: the constant logits' gradient, the tiny MLP's and its record workspace."""
    lib = ng.lib()
    s = ng.ngprt_scene()
    s.L, s.T_log2, s.R_C, s.mlp_layers, s.mlp_width = 4, 12, 16, 2, 16
    for i in range(4):
        s.N[i] = 16 << i
    s.tables = s.coarse = s.mlp_w = 256
    o = ng.ngprt_occ(32, 3, 256, None)
    opts = ng.render_opts(S.default_options(S.small_config()))
    P = C.c_void_p(256)

    def dist_bwd(g_inv=None, g_mlp=None, ws=None, ws_bytes=0):
        return lib.ngprt_distortion_backward(C.byref(s), C.byref(o), None, 0, None, P, P, 4, C.byref(opts), P,
                                             C.c_float(1.0), P, P, g_inv, g_mlp, ws, ws_bytes, None)
    s.aggregation, s.attn_inv = 2, 256
    assert dist_bwd() == ng.ERR_INVALID_ARG and b"g_attn_inv" in lib.ngprt_last_error()
    s.aggregation, s.attn_inv, s.agg_mlp = 5, None, 256
    assert dist_bwd() == ng.ERR_INVALID_ARG and b"g_agg_mlp" in lib.ngprt_last_error()
    assert dist_bwd(g_mlp=P) == ng.ERR_WORKSPACE
    s.L = 3                                 # the other forms are built for L = 2, 4, 16
    assert dist_bwd(g_mlp=P) == ng.ERR_UNSUPPORTED
