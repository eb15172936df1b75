"""The C ABI library builds, loads and exports what include/okron.h declares
(CPU only: no CUDA call is made here)."""
from __future__ import annotations

import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "okron.h")


@pytest.fixture(scope="module")
def built():
    from paper_2510_19608_gb300 import build
    return build.build()


def declared_functions() -> list[str]:
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(okr_[a-z_]+)\s*\(", text)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("okr_create", "okr_destroy", "okr_reduce", "okr_reduce_device", "okr_reduce_ops",
                 "okr_power_flow", "okr_get_summary", "okr_get_decisions", "okr_get_assignment",
                 "okr_get_voltages", "okr_get_recorded", "okr_status_str", "okr_last_error",
                 "okr_default_params"):
        assert must in names


def test_library_exports_every_declared_symbol(built):
    lib = C.CDLL(built)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(built):
    from paper_2510_19608_gb300 import _binding
    assert set(_binding.EXPORTS) <= set(declared_functions())
    assert set(declared_functions()) <= set(_binding.EXPORTS)


def test_struct_layouts_match_c(built, tmp_path):
    """sizeof/offsetof of the ABI structs as seen by a C compiler equal the ctypes view."""
    from paper_2510_19608_gb300 import _binding as B
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "okron.h"\n'
        "int main(void){\n"
        ' printf("%zu %zu %zu\\n", sizeof(okr_feeder), offsetof(okr_feeder, s_load), offsetof(okr_feeder, v_slack));\n'
        ' printf("%zu %zu %zu\\n", sizeof(okr_params), offsetof(okr_params, objective), offsetof(okr_params, max_spins));\n'
        ' printf("%zu %zu %zu\\n", sizeof(okr_summary), offsetof(okr_summary, candidates), offsetof(okr_summary, max_error));\n'
        ' printf("%zu %zu %zu\\n", sizeof(okr_summary), offsetof(okr_summary, terms), offsetof(okr_summary, inc_records));\n'
        ' printf("%zu %zu %zu\\n", sizeof(okr_inc_shape), offsetof(okr_inc_shape, eval_warps), offsetof(okr_inc_shape, records));\n'
        " return 0; }\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = [list(map(int, l.split())) for l in out if l.strip()]
    assert got[0] == [C.sizeof(B.Feeder), B.Feeder.s_load.offset, B.Feeder.v_slack.offset]
    assert got[1] == [C.sizeof(B.Params), B.Params.objective.offset, B.Params.max_spins.offset]
    assert got[2] == [C.sizeof(B.Summary), B.Summary.candidates.offset, B.Summary.max_error.offset]
    assert got[3] == [C.sizeof(B.Summary), B.Summary.terms.offset, B.Summary.inc_records.offset]
    assert got[4] == [C.sizeof(B.IncShape), B.IncShape.eval_warps.offset, B.IncShape.records.offset]


def test_default_params_from_the_library(built):
    from paper_2510_19608_gb300 import default_params
    p = default_params()
    assert p.margin == 0.005 and p.target_reduction == 1.0 and p.tie_tol == 1e-9
    assert p.objective == 0 and p.precision == 0 and p.max_merges == -1 and p.profile == 0
    q = default_params(margin=0.01, record_iters=3)
    assert q.margin == 0.01 and q.record_iters == 3


def header_define(name: str) -> int:
    m = re.search(rf"#define\s+{name}\s+(\d+)", open(HEADER).read())
    assert m, name
    return int(m.group(1))


def test_binding_constants_match_header():
    from paper_2510_19608_gb300 import _binding as B
    assert B.SCORER_FEATURES == header_define("OKR_SCORER_FEATURES")
    assert B.STATIC_MAX_BUS == header_define("OKR_STATIC_MAX_BUS")


@pytest.mark.gpu
def test_recorded_features_rows_have_the_declared_width(built):
    """okr_get_recorded_features writes rows of OKR_SCORER_FEATURES floats, as
    the header declares: a C caller that sizes its buffer by the header's
    constant gets every row filled and nothing written past cap rows."""
    import numpy as np
    import feedergen as fg
    import paper_2510_19608_gb300 as K
    from paper_2510_19608_gb300 import _binding as B
    width = header_define("OKR_SCORER_FEATURES")
    f, run = fg.preset("feeder40")
    with K.Context(0) as ctx:
        ctx.reduce(f, K.default_params(margin=run["margin"], record_iters=2, precision=0, engine=1))
        lib = B.lib()
        cnt = C.c_int32()
        assert lib.okr_get_recorded_features(ctx._h, 0, 0, None, C.byref(cnt)) == B.OK
        count = int(cnt.value)
        assert count > 4
        cap = count - 3                                   # fewer rows than candidates: the copy must stop at cap
        guard = 4 * width
        sentinel = np.float32(-1234.5)
        buf = np.full(cap * width + guard, sentinel, np.float32)
        assert lib.okr_get_recorded_features(ctx._h, 0, cap, buf.ctypes.data_as(C.c_void_p), C.byref(cnt)) == B.OK
        assert int(cnt.value) == count
        assert np.all(buf[cap * width:] == sentinel)      # nothing past cap rows of the declared width
        assert np.all(np.isfinite(buf[:cap * width]))
        assert not np.all(buf[(cap - 1) * width:cap * width] == sentinel)   # the last row was written
