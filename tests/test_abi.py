"""The C-ABI library builds, loads and exports every function include/ls.h declares
(no compute call: these run without a GPU)."""
import os
import re

import pytest

import paper_2007_12718_gb300 as ls
from paper_2007_12718_gb300 import build as lsbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def lib():
    if not os.path.exists(ls.LIB_PATH):
        lsbuild.build()
    return ls.load_library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "ls.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ls_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_boundary():
    names = declared_functions()
    for required in ("ls_build", "ls_apply", "ls_matvec", "ls_solve", "ls_free"):
        assert required in names


def test_every_declared_symbol_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(ls.EXPORTED) <= set(declared_functions())


def test_host_only_calls(lib):
    o = ls.default_opts()
    assert (o.order_matvec, o.order_precond, o.leaf_side, o.gmres_maxit) == (10, 4, 8, 100)
    assert abs(o.gmres_tol - 1e-10) < 1e-25
    assert lib.ls_strerror(ls.LS_ENOCONV) == b"GMRES did not reach the tolerance"
    assert lib.ls_strerror(ls.LS_EINVAL) == b"invalid argument"


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError):
        ls.load_library.__wrapped__(str(tmp_path / "nope.so")) if hasattr(ls.load_library, "__wrapped__") \
            else _load_fresh(str(tmp_path / "nope.so"))


def _load_fresh(path):
    saved = ls._lib
    ls._lib = None
    try:
        return ls.load_library(path)
    finally:
        ls._lib = saved


def test_fault_injection_specs(lib):
    """Host-side only: the injection hook parses its specs (nothing runs on a GPU)."""
    for spec in ("alloc:1", "alloc:25", "nan_b", ""):
        ls.ls_fault_inject(spec)
    for spec in ("alloc:0", "alloc:-3", "alloc:x", "oom", "nan_b "):
        with pytest.raises(ls.LSError) as e:
            ls.ls_fault_inject(spec)
        assert e.value.code == ls.LS_EINVAL
    ls.ls_fault_inject("")
    assert ls.ls_allocations() >= 0


def test_no_gpu_build_fails_cleanly(lib):
    """Without a CUDA device the entry points return an error code (no crash, no
    exception across the ABI); on a GPU machine this is covered by the GPU tests."""
    import numpy as np
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(ls.LSError) as e:
        ls.ls_build(32, 1 / 32, 20.0, np.zeros((32, 32)), 1e-4)
    assert e.value.code in (ls.LS_ECUDA, ls.LS_ENOMEM)


def test_load_refuses_missing_and_foreign_files(lib, tmp_path):
    """ls_load checks the file before any device work."""
    import ctypes
    out = ctypes.c_void_p()
    assert lib.ls_load(str(tmp_path / "absent").encode(), None, ctypes.byref(out)) == ls.LS_EINVAL
    junk = tmp_path / "junk"
    junk.write_bytes(b"not a handle file" * 10)
    assert lib.ls_load(str(junk).encode(), None, ctypes.byref(out)) == ls.LS_EINVAL
    assert not out.value
