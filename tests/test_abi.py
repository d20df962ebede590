"""The C-ABI library builds, loads and exports every symbol include/slg.h declares.

No GPU work is launched here: only symbol lookup and calls that touch no device.
"""
import ctypes
import os
import re

import pytest

import paper_2201_11326_gb300 as slg
from paper_2201_11326_gb300 import build as slg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\*]+\s+\**(slg_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    slg_build.build()
    return slg.lib()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("slg_load", "slg_count", "slg_build", "slg_build_window", "slg_bound",
                     "slg_plan_windows", "slg_free", "slg_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_symbol():
    for n in declared_symbols():
        assert n in slg._SIGS, f"{n} has no Python binding"


def test_version_and_error_string(lib):
    assert lib.slg_version() >= 100
    assert isinstance(lib.slg_last_error(), bytes)


def test_null_arguments_rejected_without_device(lib):
    # argument checks that happen before any CUDA call
    out = ctypes.c_void_p()
    assert lib.slg_load(None, None, 0, 0, None, ctypes.byref(out)) == slg.SLG_EINVAL
    assert lib.slg_load(None, None, -1, 0, None, None) == slg.SLG_EINVAL
    assert lib.slg_count(None, 1, None, None) == slg.SLG_EINVAL
    assert b"NULL" in lib.slg_last_error() or len(lib.slg_last_error()) > 0


def test_library_links_no_oracle():
    # the product library shares nothing with the oracle
    import subprocess
    out = subprocess.run(["nm", "-D", slg.library_path()], capture_output=True, text=True).stdout
    assert "oracle_" not in out


def test_no_gpu_means_an_error_not_a_cpu_fallback(lib):
    # without a CUDA device the library reports a CUDA error; nothing is computed on the CPU
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    off = (ctypes.c_int32 * 3)(0, 2, 3)
    idx = (ctypes.c_int32 * 3)(0, 1, 1)
    out = ctypes.c_void_p()
    rc = lib.slg_load(off, idx, 2, 2, None, ctypes.byref(out))
    assert rc in (slg.SLG_ECUDA, slg.SLG_ENOMEM) and not out.value
    assert lib.slg_last_error()  # with a message
    import numpy as np
    with pytest.raises(slg.SlgError):
        slg.slg_load(np.array([0, 2, 3], np.int32), np.array([0, 1, 1], np.int32), 2, 2)


def test_header_compiles_as_c_and_cpp(tmp_path):
    # the boundary is plain C: it compiles alone as C99 and as C++, without warnings
    import shutil
    import subprocess
    src = tmp_path / "use.c"
    src.write_text('#include "slg.h"\nint main(void) { return slg_version() > 0 ? 0 : 1; }\n')
    inc = os.path.join(ROOT, "include")
    for cc, extra in (("gcc", ["-std=c99"]), ("g++", ["-std=c++17", "-x", "c++"])):
        if not shutil.which(cc):
            pytest.skip(f"{cc} not found")
        r = subprocess.run([cc, *extra, "-Wall", "-Wextra", "-Werror", "-I", inc, "-c", str(src),
                            "-o", str(tmp_path / "use.o")], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_new_entry_points_reject_null_without_device(lib):
    i32 = ctypes.c_int32()
    i64 = ctypes.c_int64()
    s = (ctypes.c_int32 * 2)(2, 4)
    assert lib.slg_stream_window(None, 2, 0, None, None, None, 16, ctypes.byref(i32),
                                 ctypes.byref(i64)) == slg.SLG_EINVAL
    assert lib.slg_ensemble_stream_window(None, s, 2, 0, None, None, None, 16, ctypes.byref(i32),
                                          ctypes.byref(i64)) == slg.SLG_EINVAL
    assert lib.slg_ensemble_fill_stats(None, 0, None) == slg.SLG_EINVAL
    assert lib.slg_set_ensemble_filter(None, 0) == slg.SLG_EINVAL
    assert lib.slg_set_staging(None, -1) == slg.SLG_EINVAL
