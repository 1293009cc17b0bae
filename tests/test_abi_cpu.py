"""C ABI checks that need no GPU: the library loads, exports every entry point that
include/awgrid.h declares, and rejects bad arguments before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2508_17187_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2508_17187_gb300 import build
        build.build()
    return _lib.load()


def header_functions():
    src = open(os.path.join(ROOT, "include", "awgrid.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return re.findall(r"^\s*(?:awg_status|const char\s*\*|int64_t)\s+(\w+)\s*\(", src, flags=re.M)


def test_every_declared_symbol_is_exported(lib):
    from paper_2508_17187_gb300 import _lib
    names = header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(names) == sorted(_lib.EXPORTED)


def test_bad_arguments_fail_before_the_device(lib):
    from paper_2508_17187_gb300._lib import CfParams
    out = ctypes.c_void_p()
    p = CfParams()
    p.grid_n = 15
    p.cell_rad = 1e-6
    p.oversampling = 20
    p.max_support = 7
    p.ps_support = 7
    p.use_ps = 1
    p.n_pa_bins = 1
    p.n_subbands = 1
    assert lib.cf_set_create(ctypes.byref(p), None, ctypes.byref(out)) == 1
    assert b"grid_n" in lib.awg_last_error()
    p.grid_n = 512
    p.max_support = 65
    assert lib.cf_set_create(ctypes.byref(p), None, ctypes.byref(out)) == 2
    p.max_support = 7
    p.use_w = 1
    p.n_wplanes = 1
    assert lib.cf_set_create(ctypes.byref(p), None, ctypes.byref(out)) == 1
    assert lib.cf_set_create(None, None, ctypes.byref(out)) == 1
    assert lib.cf_set_create(ctypes.byref(p), None, None) == 1
    assert lib.plan_create(None, None, 0, None, 1, None, None, None, None, ctypes.byref(out)) == 1
    assert lib.grid_visibilities(None, None, None, None, 4, None, None, None, 0, None) == 1
    assert lib.degrid_visibilities(None, None, None, None, 4, 0, None) == 1
    assert lib.grid_normalize(None, None, 1, None, 0, None) == 1
    assert lib.cf_set_destroy(None) == 1
    assert lib.plan_destroy(None) == 1
    assert lib.awg_kernel_launches() >= 0


def test_python_binding_refuses_cpu_tensors():
    torch = pytest.importorskip("torch")
    from paper_2508_17187_gb300 import api
    with pytest.raises(ValueError, match="CUDA"):
        api._need(torch.zeros(3), "x", torch.float32)


def test_cf_cache_load_rejects_bad_files_before_the_device(lib, tmp_path):
    """cf_set_load checks the file (existence, magic, version, parameter layout, a complete header)
    before it touches the device; every failure is INVALID_ARG with a message naming the file."""
    from paper_2508_17187_gb300._lib import CfParams
    out = ctypes.c_void_p()
    lib.awg_last_error.restype = ctypes.c_char_p

    def load(path):
        return lib.cf_set_load(str(path).encode(), None, ctypes.byref(out))

    assert load(tmp_path / "missing.awgcf") == 1 and out.value is None
    assert b"cannot open" in lib.awg_last_error()
    junk = tmp_path / "junk.awgcf"
    junk.write_bytes(b"not a cache file at all")
    assert load(junk) == 1 and b"not a CF cache file" in lib.awg_last_error()
    magic = b"AWGCFSET"
    bad_version = tmp_path / "v.awgcf"
    bad_version.write_bytes(magic + (99).to_bytes(4, "little") + ctypes.sizeof(CfParams).to_bytes(4, "little"))
    assert load(bad_version) == 1 and b"version" in lib.awg_last_error()
    bad_layout = tmp_path / "l.awgcf"
    bad_layout.write_bytes(magic + (1).to_bytes(4, "little") + (ctypes.sizeof(CfParams) + 8).to_bytes(4, "little"))
    assert load(bad_layout) == 1 and b"layout" in lib.awg_last_error()
    truncated = tmp_path / "t.awgcf"
    truncated.write_bytes(magic + (1).to_bytes(4, "little") + ctypes.sizeof(CfParams).to_bytes(4, "little") + b"\0" * 16)
    assert load(truncated) == 1 and b"truncated" in lib.awg_last_error()
    assert lib.cf_set_save(None, str(junk).encode()) == 1
    assert lib.cf_set_load(None, None, ctypes.byref(out)) == 1
