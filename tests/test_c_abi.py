"""The boundary as a C program sees it: include/ngprt.h compiles as strict C99, a
C program links against libngprt.so and calls the host-side entries (no GPU needed),
and every struct of the header has the layout the Python binding declares (size
and the offset of each field), so the two cannot drift apart."""
import json
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")

STRUCTS = ("ngprt_scene", "ngprt_occ", "ngprt_camera", "ngprt_render_opts")

PROGRAM = r"""
#include <stddef.h>
#include <stdio.h>
#include <string.h>
#include "ngprt.h"

#define FIELD(S, F) printf("%s\"%s\": %zu", first ? "" : ", ", #F, offsetof(S, F)); first = 0
#define OPEN(S) printf("%s\"%s\": {\"size\": %zu, \"fields\": {", nstruct++ ? ", " : "", #S, sizeof(S)); first = 1
#define CLOSE() printf("}}")

int main(void) {
    int first = 1, nstruct = 0;
    printf("{");
    OPEN(ngprt_scene);
    FIELD(ngprt_scene, L); FIELD(ngprt_scene, T_log2); FIELD(ngprt_scene, N); FIELD(ngprt_scene, table_dtype);
    FIELD(ngprt_scene, R_C); FIELD(ngprt_scene, mlp_layers); FIELD(ngprt_scene, mlp_width);
    FIELD(ngprt_scene, mlp_dtype); FIELD(ngprt_scene, bounded); FIELD(ngprt_scene, tables);
    FIELD(ngprt_scene, coarse); FIELD(ngprt_scene, mlp_w); FIELD(ngprt_scene, aggregation);
    FIELD(ngprt_scene, attn_inv); FIELD(ngprt_scene, agg_mlp); FIELD(ngprt_scene, coarse_index);
    FIELD(ngprt_scene, coarse_blocks);
    CLOSE();
    OPEN(ngprt_occ);
    FIELD(ngprt_occ, R_O); FIELD(ngprt_occ, n_levels); FIELD(ngprt_occ, bits); FIELD(ngprt_occ, dist);
    FIELD(ngprt_occ, R_G);
    CLOSE();
    OPEN(ngprt_camera);
    FIELD(ngprt_camera, c2w); FIELD(ngprt_camera, fx); FIELD(ngprt_camera, fy); FIELD(ngprt_camera, cx);
    FIELD(ngprt_camera, cy); FIELD(ngprt_camera, W); FIELD(ngprt_camera, H);
    CLOSE();
    OPEN(ngprt_render_opts);
    FIELD(ngprt_render_opts, step_base); FIELD(ngprt_render_opts, step_gamma); FIELD(ngprt_render_opts, t_min);
    FIELD(ngprt_render_opts, r_far); FIELD(ngprt_render_opts, t_term); FIELD(ngprt_render_opts, bg);
    FIELD(ngprt_render_opts, max_march); FIELD(ngprt_render_opts, max_samples); FIELD(ngprt_render_opts, use_dist);
    FIELD(ngprt_render_opts, lattice_snap); FIELD(ngprt_render_opts, attn_mode); FIELD(ngprt_render_opts, dist_rule);
    CLOSE();
    /* host-side calls: sizes, the step controller, and an argument error */
    ngprt_scene s;
    memset(&s, 0, sizeof s);
    s.L = 2; s.T_log2 = 12; s.N[0] = 8; s.N[1] = 64; s.R_C = 16;
    printf(", \"version\": %d, \"channels\": %d, \"entries\": %lld", ngprt_version(),
           ngprt_coarse_channels(4, NGPRT_AGG_SEPARATE_V), (long long)ngprt_table_entries(&s));
    printf(", \"gamma\": [%.9g, %.9g]", (double)ngprt_step_autotune(1.0f, 10.0f, 20.0f, 0.01f, 0.5f),
           (double)ngprt_step_autotune(0.8f, 30.0f, 20.0f, 0.01f, 0.5f));
    int32_t rc = ngprt_render(&s, NULL, NULL, 0, NULL, NULL, NULL, 1, NULL, NULL, NULL, NULL, NULL, NULL, NULL,
                              NULL, 0, NULL);
    printf(", \"rc\": %d, \"err_nonempty\": %d}\n", rc, ngprt_last_error()[0] != 0);
    return 0;
}
"""


@pytest.fixture(scope="module")
def c_run(tmp_path_factory):
    from paper_2407_10482_gb300 import build
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    lib = build.build()
    d = tmp_path_factory.mktemp("c_abi")
    src = d / "abi.c"
    src.write_text(PROGRAM)
    exe = d / "abi"
    libdir = os.path.dirname(lib)
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", INCLUDE, str(src),
                    "-L", libdir, "-lngprt", f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return json.loads(out)


def test_struct_layouts_match_the_binding(c_run):
    import ctypes
    from paper_2407_10482_gb300 import ngprt as ng
    for name in STRUCTS:
        cls = getattr(ng, name)
        c = c_run[name]
        assert ctypes.sizeof(cls) == c["size"], name
        py_fields = [f[0] for f in cls._fields_]
        assert py_fields == list(c["fields"]), name
        for f in py_fields:
            assert getattr(cls, f).offset == c["fields"][f], (name, f)


def test_header_compiles_as_cpp(tmp_path):
    """The same header from C++ (extern "C" linkage, no C-only constructs)."""
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "abi.cpp"
    src.write_text('#include "ngprt.h"\nint main() { ngprt_scene s{}; return (int)sizeof(s) > 0 ? 0 : 1; }\n')
    subprocess.run([gxx, "-std=c++17", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", INCLUDE, "-c", str(src),
                    "-o", str(tmp_path / "abi.o")], check=True)


def test_host_entries_from_c(c_run):
    from paper_2407_10482_gb300 import ngprt as ng
    assert c_run["version"] == 201
    assert c_run["channels"] == 16
    assert c_run["entries"] == 8 ** 3 + 4096
    # Eq. S3: too few samples shrink gamma by (1 - kappa), enough grow it by (1 + kappa)
    assert abs(c_run["gamma"][0] - 0.99) < 1e-7 and abs(c_run["gamma"][1] - 0.808) < 1e-7
    assert c_run["rc"] == ng.ERR_INVALID_ARG and c_run["err_nonempty"] == 1
