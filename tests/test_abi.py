"""C-ABI library checks that need no GPU: it builds for sm_103a, loads, and
exports every entry point include/aln.h declares; host-side argument checks."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "aln.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(aln_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    from paper_1502_01645_gb300 import build_lib, aln
    build_lib.build()
    return aln.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_1502_01645_gb300 import aln
    declared = _declared()
    assert declared, "header parse found no entry points"
    assert sorted(aln.EXPORTS) == declared
    for name in declared:
        assert hasattr(lib, name), f"libaln does not export {name}"


def test_library_targets_sm103a_only():
    from paper_1502_01645_gb300 import build_lib
    assert build_lib.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_host_only_entry_points(lib):
    from paper_1502_01645_gb300 import aln
    assert aln.aln_version() == 201
    o = aln.aln_default_options()
    assert o.precision == aln.PREC_SPLIT_BF16 and o.max_refine == 8 and o.stagnation == 100
    assert aln.status_string(aln.ERR_NONFINITE) == "ALN_ERR_NONFINITE"
    assert aln.status_string(99) == "ALN_ERR_UNKNOWN"


def test_null_and_invalid_arguments_are_rejected_without_a_device(lib):
    from paper_1502_01645_gb300 import aln
    # NULL context / output pointer: rejected before any CUDA call.
    assert lib.aln_create(None, None, None) == aln.ERR_INVALID_ARG
    assert lib.aln_prepare(None, None, 1, 1, 1, 0, None, 1, 1) == aln.ERR_INVALID_ARG
    assert lib.aln_solve(None, 1e-6, 0, None, 1, None, None) == aln.ERR_INVALID_ARG
    assert lib.aln_kkt_residual(None, None, 1, None, None) == aln.ERR_INVALID_ARG
    assert lib.aln_export_scaled(None, None, 1, None, 1, None) == aln.ERR_INVALID_ARG
    assert lib.aln_get_stats(None, None) == aln.ERR_INVALID_ARG
    assert lib.aln_prepare_grouped(None, 1, None, 0) == aln.ERR_INVALID_ARG
    assert lib.aln_nmf(None, None, 4, 4, 4, 2, None, 4, None, 2, 1, 1e-6, 0, None) == \
        aln.ERR_INVALID_ARG
    assert lib.aln_prepare_csc(None, 4, 2, None, None, None, 0, None, 1, 4) == \
        aln.ERR_INVALID_ARG
    o = aln.aln_default_options()
    o.precision = 7
    ctx = ctypes.c_void_p()
    assert lib.aln_create(ctypes.byref(ctx), ctypes.byref(o), None) == aln.ERR_INVALID_ARG
    # option checks come before any CUDA call
    for field, bad in (("gram_split", 4), ("group_cluster", 3), ("group_cluster", 16),
                       ("refine_gain", 17), ("iter_kernel", 4), ("wait_limit_us", -1),
                       ("test_barrier_skew", -1), ("test_barrier_skew", 1025),
                       ("group_graph", 2), ("group_graph", -1), ("autotune", 3),
                       ("autotune", -1), ("autotune", 1), ("autotune", 2)):
        o = aln.aln_default_options()
        setattr(o, field, bad)  # autotune 1 and 2 without a cache path are invalid too
        assert lib.aln_create(ctypes.byref(ctx), ctypes.byref(o), None) == aln.ERR_INVALID_ARG
    o = aln.aln_default_options()
    o.autotune, o.autotune_cache = 1, b""
    assert lib.aln_create(ctypes.byref(ctx), ctypes.byref(o), None) == aln.ERR_INVALID_ARG
    assert lib.aln_set_wait_limit(None, 1000, 0) == aln.ERR_INVALID_ARG
    lib.aln_destroy(None)  # accepted


def test_binding_has_no_cpu_fallback(monkeypatch, tmp_path):
    """The product path fails loudly when the library is missing."""
    from paper_1502_01645_gb300 import aln
    monkeypatch.setattr(aln, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        aln.load(str(tmp_path / "missing.so"))
