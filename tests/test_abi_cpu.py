"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports every entry point
that include/raysplats.h declares, and rejects bad arguments on the host (no GPU needed: these
calls return before touching the device).  Also checks that the product path never reaches the
oracle."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "raysplats.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rs_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2501_19196_gb300 import build, native
    build.build()
    return native.load()


def test_header_declares_the_path_calls():
    names = declared_functions()
    for must in ("rs_build_accel", "rs_render", "rs_render_backward", "rs_accel_destroy", "rs_state_destroy",
                 "rs_last_error", "rs_abi_version"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2501_19196_gb300 import native
    path = native.library_path()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(rs_\w+)", out))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)
    assert set(native.exported_symbols()) <= exported


def test_abi_version_and_default_tune(lib):
    from paper_2501_19196_gb300 import native
    assert lib.rs_abi_version() == 1
    t = native.default_tune()
    assert (t.tile_w, t.tile_h, t.kbuf, t.leaf_size, t.morton_bits, t.traversal, t.hit_list) == \
        (8, 4, 32, 32, 21, 2, 256)


def test_host_validation_rejects_bad_arguments(lib):
    from paper_2501_19196_gb300 import native
    acc = ctypes.c_void_p()
    t = native.default_tune()
    # NULL scene
    assert lib.rs_build_accel(None, 11.3, ctypes.byref(t), ctypes.byref(acc), None) == native.RS_ERR_INVALID_ARG
    assert b"NULL" in lib.rs_last_error()
    # n = 0
    g = native.RsGaussians(0, 1, 1, 1, 1, 1)
    assert lib.rs_build_accel(ctypes.byref(g), 11.3, ctypes.byref(t), ctypes.byref(acc), None) == \
        native.RS_ERR_INVALID_ARG
    # bad tile / kbuf / leaf / Q_box
    g = native.RsGaussians(10, 16, 16, 16, 16, 16)
    for field, val in (("tile_w", 3), ("kbuf", 12), ("leaf_size", 0), ("leaf_size", 33), ("morton_bits", 7), ("block_warps", 9),
                       ("traversal", 4), ("smem_nodes", 513), ("hit_list", -1), ("hit_list", 4097)):
        bad = native.default_tune(**{field: val})
        if field == "tile_w":
            bad.tile_h = 10
        assert lib.rs_build_accel(ctypes.byref(g), 11.3, ctypes.byref(bad), ctypes.byref(acc), None) == \
            native.RS_ERR_INVALID_ARG, field
    assert lib.rs_build_accel(ctypes.byref(g), -1.0, ctypes.byref(t), ctypes.byref(acc), None) == \
        native.RS_ERR_INVALID_ARG
    assert not acc  # nothing was created
    # backward without a forward state
    dl = native.RsFrameGrad(16, None)
    out = native.RsGaussianGrads(None, None, None, None, None)
    assert lib.rs_render_backward(ctypes.byref(g), None, None, ctypes.byref(dl), ctypes.byref(t),
                                  ctypes.byref(out), None) == native.RS_ERR_INVALID_ARG
    # destroy accepts NULL
    assert lib.rs_accel_destroy(None) == 0 and lib.rs_state_destroy(None) == 0


def test_injected_allocation_failure_frees_the_new_handle(lib):
    """rs_test_fail_alloc(1): the first device allocation of a new accel fails before any CUDA
    call, the half-built handle is freed and *inout stays NULL; the hook then disarms itself."""
    from paper_2501_19196_gb300 import native
    t = native.default_tune()
    g = native.RsGaussians(10, 16, 16, 16, 16, 16)
    acc = ctypes.c_void_p()
    assert lib.rs_test_fail_alloc(-1) == native.RS_ERR_INVALID_ARG
    assert lib.rs_test_fail_alloc(1) == native.RS_OK
    assert lib.rs_build_accel(ctypes.byref(g), 11.3, ctypes.byref(t), ctypes.byref(acc), None) == native.RS_ERR_OOM
    assert b"injected allocation failure" in lib.rs_last_error()
    assert not acc
    assert lib.rs_test_fail_alloc(0) == native.RS_OK


def test_product_path_never_reaches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2501_19196_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), f
                assert "liboracle" not in src and "raysplats_oracle" not in src, f
    # and the oracle never imports the product package
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            src = open(os.path.join(ROOT, "oracle", f)).read()
            assert not re.search(r"^\s*(import|from)\s+paper_2501_19196_gb300\b", src, flags=re.M), f
            assert "libraysplats" not in src, f
