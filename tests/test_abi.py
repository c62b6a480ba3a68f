"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/cddt.h declares.  Host-side argument checks answer without a GPU
(no compute call is made here)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1705_01167_gb300 import cddt
    return cddt.load(build_if_missing=True)


def _declared():
    src = open(os.path.join(ROOT, "include", "cddt.h")).read()
    return sorted(set(re.findall(r"^CDDT_API[^(]*?\b(cddt_\w+)\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("cddt_build", "cddt_prune", "cddt_update_cells", "cddt_calc_range_many",
                     "cddt_sensor_weights", "cddt_sensor_weights_backward", "cddt_destroy",
                     "cddt_export", "cddt_get_stats", "cddt_plan_create", "cddt_plan_run"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1705_01167_gb300 import cddt
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) == set(cddt.EXPORTED)
    assert lib.cddt_version() == 1


def test_status_strings(lib):
    from paper_1705_01167_gb300 import cddt
    for s in range(8):
        assert len(cddt.status_string(s)) > 0
        assert "unknown" not in cddt.status_string(s), s
    assert "unknown" in cddt.status_string(99)


def test_host_side_argument_errors(lib):
    """Invalid arguments are rejected on the host before any device call."""
    from paper_1705_01167_gb300 import cddt
    h = C.c_void_p()
    fake = C.c_void_p(0x1000)
    ARG = cddt.CDDT_ERR_ARG
    assert lib.cddt_build(fake, 0, 10, 8, 10.0, 0, None, C.byref(h)) == ARG
    assert lib.cddt_build(fake, 10, 10, 7, 10.0, 0, None, C.byref(h)) == ARG
    assert lib.cddt_build(fake, 10, 10, 8, -1.0, 0, None, C.byref(h)) == ARG
    assert lib.cddt_build(fake, 10, 10, 8, 10.0, 8, None, C.byref(h)) == ARG
    assert lib.cddt_build(None, 10, 10, 8, 10.0, 0, None, C.byref(h)) == ARG
    assert lib.cddt_build(fake, 40000, 10, 8, 10.0, 0, None, C.byref(h)) == ARG
    assert lib.cddt_build(fake, 10, 10, 8, 10.0, 0, None, None) == ARG
    assert lib.cddt_destroy(None) == cddt.CDDT_OK
    assert lib.cddt_prune(None, None) == ARG
    assert lib.cddt_calc_range_many(None, fake, fake, 1, 0, None) == ARG
    assert lib.cddt_set_search(None, 0) == ARG
    assert lib.cddt_plan_create(None, 0, None, C.byref(h)) == ARG
    assert lib.cddt_plan_destroy(None) == cddt.CDDT_OK
    bs = (C.c_int64 * 3)(0, 2, 4)
    zp = (C.c_float * 4)(0.0, 1.0, 2.0, 3.0)
    assert lib.cddt_import(fake, 10, 10, 8, 10.0, 0, 0, 2, None, zp, None, C.byref(h)) == ARG
    assert lib.cddt_import(fake, 10, 10, 8, 10.0, 0, 0, 2, bs, None, None, C.byref(h)) == ARG
    assert lib.cddt_import(fake, 10, 10, 8, 10.0, 0, 0, -1, bs, zp, None, C.byref(h)) == ARG
    assert lib.cddt_import(fake, 10, 10, 7, 10.0, 0, 0, 2, bs, zp, None, C.byref(h)) == ARG
    assert lib.cddt_import(None, 10, 10, 8, 10.0, 0, 0, 2, bs, zp, None, C.byref(h)) == ARG
    assert lib.cddt_import(fake, 10, 10, 8, 10.0, 0, 0, 2, bs, zp, None, None) == ARG
    # the comparison casters and the filter step
    assert lib.cddt_cast_bresenham(None, fake, fake, 1, None) == ARG
    assert lib.cddt_lut_build(None, None, C.byref(h)) == ARG
    assert lib.cddt_lut_info(None, None, None) == ARG
    assert lib.cddt_lut_calc_range_many(None, fake, fake, 1, None) == ARG
    assert lib.cddt_lut_destroy(None) == cddt.CDDT_OK
    assert lib.cddt_rm_build(None, None, C.byref(h)) == ARG
    assert lib.cddt_rm_build(fake, None, None) == ARG
    assert lib.cddt_rm_distances(None, None, None) == ARG
    assert lib.cddt_rm_calc_range_many(None, fake, fake, None, 1, None) == ARG
    assert lib.cddt_rm_destroy(None) == cddt.CDDT_OK
    assert lib.cddt_motion(fake, -1, fake, 1, fake, fake, None) == ARG
    assert lib.cddt_motion(fake, 1, fake, 0, fake, fake, None) == ARG
    assert lib.cddt_resample(fake, fake, fake, 0, fake, C.c_void_p(0x2000), None, fake, None) == ARG
    assert lib.cddt_resample(fake, fake, fake, 1, fake, fake, None, fake, None) == ARG  # out == particles


def test_host_fault_injection(lib, monkeypatch):
    """CDDT_FAULT makes an entry point return a failure status after its
    argument checks and before any device call (the only calls made here
    return at the fault point)."""
    from paper_1705_01167_gb300 import cddt
    h = C.c_void_p(0x1234)
    fake = C.c_void_p(0x1000)
    for kind, status in (("oom", cddt.CDDT_ERR_OOM), ("launch", cddt.CDDT_ERR_CUDA),
                         ("timeout", cddt.CDDT_ERR_TIMEOUT)):
        monkeypatch.setenv("CDDT_FAULT", kind)
        assert lib.cddt_build(fake, 10, 10, 8, 10.0, 0, None, C.byref(h)) == status
        assert not h.value  # no handle made
        monkeypatch.setenv("CDDT_FAULT", f"{kind}:cddt_build")
        assert lib.cddt_build(fake, 10, 10, 8, 10.0, 0, None, C.byref(h)) == status
    # argument errors still come first
    monkeypatch.setenv("CDDT_FAULT", "oom")
    assert lib.cddt_build(fake, 0, 10, 8, 10.0, 0, None, C.byref(h)) == cddt.CDDT_ERR_ARG


def test_checked_variant_builds_and_exports():
    """The bounds-checked variant (-DCDDT_CHECKED=1) builds, reports itself
    and exports the same symbols as the normal library."""
    import ctypes

    from paper_1705_01167_gb300 import build
    from paper_1705_01167_gb300 import cddt as G
    lib = ctypes.CDLL(build.build_checked())
    lib.cddt_checked_build.restype = ctypes.c_int32
    assert lib.cddt_checked_build() == 1
    for name in G.EXPORTED:
        assert hasattr(lib, name), name
    normal = ctypes.CDLL(build.build())
    normal.cddt_checked_build.restype = ctypes.c_int32
    assert normal.cddt_checked_build() == 0


def test_trace_host_side(lib):
    """The call trace: enable / disable, an empty report with its header, a
    short buffer truncated with the needed length reported, and calls that
    fail their argument checks while tracing is on still return ARG."""
    from paper_1705_01167_gb300 import cddt
    assert lib.cddt_trace_enable(2) == cddt.CDDT_ERR_ARG
    assert lib.cddt_trace_enable(1) == cddt.CDDT_OK
    try:
        h = C.c_void_p(0)
        assert lib.cddt_build(None, 10, 10, 8, 10.0, 0, None, C.byref(h)) == cddt.CDDT_ERR_ARG
        need = C.c_int64()
        assert lib.cddt_trace_report(None, 0, C.byref(need)) == cddt.CDDT_OK
        header = b"entry,calls,total_ms,mean_ms,min_ms,max_ms\n"
        assert need.value >= len(header) + 1
        buf = C.create_string_buffer(8)
        assert lib.cddt_trace_report(buf, 8, C.byref(need)) == cddt.CDDT_OK
        assert buf.value == header[:7]
        assert lib.cddt_trace_report(None, 5, None) == cddt.CDDT_ERR_ARG
        assert cddt.trace_report() == []
    finally:
        assert lib.cddt_trace_enable(0) == cddt.CDDT_OK


def test_c_example_builds_and_runs_without_a_device(tmp_path):
    """The C ABI from plain C: tests/c_example/cddt_example.c compiles with gcc
    against include/cddt.h and libcddt.so; without a CUDA device it checks the
    argument and no-device statuses and exits 2."""
    import subprocess

    import torch

    from tests.c_example.build_example import build_example
    exe = build_example(str(tmp_path))
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    if torch.cuda.is_available():
        assert r.returncode == 0, r.stdout + r.stderr
    else:
        assert r.returncode == 2, r.stdout + r.stderr
        assert "no CUDA device" in r.stdout


def test_no_cpu_fallback():
    """Without the built library the binding raises instead of computing
    anything itself, and host tensors are refused: there is no CPU path."""
    import subprocess
    import sys

    code = ("import paper_1705_01167_gb300.build as b, paper_1705_01167_gb300.cddt as G\n"
            "b.LIB = '/nonexistent/libcddt.so'\n"
            "try:\n    G.load(build_if_missing=False)\nexcept RuntimeError as e:\n    print('raised:', e)\n")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300,
                       cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    assert r.returncode == 0 and "raised: libcddt.so is not built" in r.stdout, r.stdout + r.stderr
    import torch

    from paper_1705_01167_gb300 import cddt
    with pytest.raises(ValueError, match="CUDA tensor"):
        cddt.CDDT(torch.zeros((8, 8), dtype=torch.uint8), 8, 10.0)


def test_header_compiles_as_c_and_cpp(tmp_path):
    """include/cddt.h stands alone in C11 and C++17 translation units with
    every warning an error (it needs only <stdint.h>)."""
    import subprocess
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "use.c"
    src.write_text('#include "cddt.h"\nint main(void) { return cddt_version() > 0 ? 0 : 1; }\n')
    for cc, std, lang in (("gcc", "-std=c11", "c"), ("g++", "-std=c++17", "c++")):
        r = subprocess.run([cc, std, "-x", lang, "-Wall", "-Wextra", "-Werror", "-pedantic", f"-I{inc}",
                            "-fsyntax-only", str(src)], capture_output=True, text=True)
        assert r.returncode == 0, (cc, r.stderr)
