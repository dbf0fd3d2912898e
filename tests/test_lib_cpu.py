"""Host-side checks of the C-ABI library that need no GPU: it loads, exports
every entry point that include/pwadv.h declares, and rejects bad arguments
before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pwadv.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2009_12850_b300 import build
    build.build()
    from paper_2009_12850_b300 import _lib
    return _lib


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(pw_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_symbols_exported(lib):
    names = declared_functions()
    assert len(names) >= 20, names
    for n in names:
        assert hasattr(lib._c, n), f"{n} declared in pwadv.h but not exported"
    # and the binding covers exactly the declared set
    assert set(lib.exported_symbols()) == set(names)


def test_version_and_strings(lib):
    assert lib.pw_version() == 1
    assert lib.status_string(lib.PW_OK) == "ok"
    assert "align" in lib.status_string(lib.PW_ERR_ALIGN)
    assert lib.status_string(-99) == "unknown status"


def test_null_arguments_rejected(lib):
    c = lib._c
    z = ctypes.c_void_p(0)
    assert c.pw_advect(z, z, z, z, z, z, z, 0, z) == lib.PW_ERR_ARG
    assert "mesh" in lib.last_error()
    assert c.pw_advect_adjoint(z, *([z] * 9), 1.0, 0, z) == lib.PW_ERR_ARG
    assert c.pw_euler_adjoint(z, *([z] * 9), 0.5, z) == lib.PW_ERR_ARG
    assert c.pw_halo_periodic(z, z, z, z, z) == lib.PW_ERR_ARG
    assert c.pw_euler(z, *([z] * 6), 0.5, z) == lib.PW_ERR_ARG
    assert c.pw_mesh_layout(z, None, None, None, None) == lib.PW_ERR_ARG
    assert c.pw_mesh_set_tile(z, 8, 32) == lib.PW_ERR_ARG
    assert c.pw_advect_batched(z, 0, z) == lib.PW_ERR_ARG
    assert c.pw_batch_set_schedule(z, 1, z) == lib.PW_ERR_ARG
    assert c.pw_advect_step(z, *([z] * 6), 0.5, z) == lib.PW_ERR_ARG
    arr = (ctypes.c_void_p * 1)()
    assert c.pw_advect_scalars(z, z, z, z, 1, arr, arr, 0, z) == lib.PW_ERR_ARG
    assert c.pw_pipeline_create(z, 0, ctypes.byref(ctypes.c_void_p())) == lib.PW_ERR_ARG
    assert c.pw_pipeline_sync(z) == lib.PW_ERR_ARG
    assert c.pw_pipeline_slab(z, None, None) == lib.PW_ERR_ARG
    assert c.pw_advect_host(z, *([z] * 6), 0, None, None, z) == lib.PW_ERR_ARG
    assert "pipeline" in lib.last_error()
    assert c.pw_advect_host_scalars(z, *([z] * 6), 1, arr, arr, 0, None, None, z) == lib.PW_ERR_ARG
    assert c.pw_pipeline_reserve_scalars(z, 2) == lib.PW_ERR_ARG
    assert c.pw_advect_scalars_step(z, z, z, z, 1, arr, arr, 0.5, z) == lib.PW_ERR_ARG
    lib.pw_mesh_destroy(z)   # NULL is allowed
    lib.pw_batch_destroy(z)
    lib.pw_pipeline_destroy(z)


def test_bad_descriptors_rejected(lib):
    c = lib._c
    out = ctypes.c_void_p()
    for kw in ({"nx": 0}, {"nz": 0}, {"nz": 5000}, {"dx": 0.0}, {"dy": -1.0}, {"dtype": 7}, {"algo": 9}):
        d = lib.pw_mesh_desc()
        d.nx, d.ny, d.nz, d.dx, d.dy = 8, 8, 8, 50.0, 50.0
        d.dtype, d.algo = lib.PW_F32, 0
        for k, v in kw.items():
            setattr(d, k, v)
        st = c.pw_mesh_create(ctypes.byref(d), None, ctypes.byref(out))
        assert st in (lib.PW_ERR_SHAPE, lib.PW_ERR_ARG, lib.PW_ERR_DTYPE), (kw, st)
        assert not out.value


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """The binding raises instead of falling back when the .so is absent."""
    import importlib.util
    src = os.path.join(ROOT, "paper_2009_12850_b300", "_lib.py")
    spec = importlib.util.spec_from_file_location("pw_lib_copy", str(tmp_path / "_lib.py"))
    (tmp_path / "_lib.py").write_text(open(src).read())
    mod = importlib.util.module_from_spec(spec)
    with pytest.raises(ImportError):
        spec.loader.exec_module(mod)


def test_residual_ratios_host_arithmetic(lib):
    """pw_residual_ratios is pure host arithmetic: R_E = sum W phi S / sum W |phi S|,
    R_M = sum W S / sum W |S| per component, 0 for a zero denominator."""
    sums = [1.0, 4.0, -3.0, 6.0, 0.0, 0.0, 2.0, 8.0, -5.0, 10.0, 0.5, 0.0]
    r = lib.pw_residual_ratios(sums)
    assert r == [0.25, 0.0, -0.5, -0.5, 0.25, 0.0]
    c = lib._c
    assert c.pw_residual_ratios(None, None) == lib.PW_ERR_ARG
    assert c.pw_mesh_algo(ctypes.c_void_p(0), None) == lib.PW_ERR_ARG
    assert "split" in lib.status_string(lib.PW_ERR_RANGE)
