"""The allocation-free conservation sums, checked against pw_residuals.

pw_residuals_noalloc is for callers that must not allocate device memory when
they ask for the diagnostics (a caching allocator owns the free memory, or an
allocation would stall a time-stepping loop) and that may not hold a mesh.  It
keeps its scratch in a static device array, so this test calls it through the
C-ABI twice in a row -- the second call reuses whatever the first left in that
array -- and compares both results with the mesh-based pw_residuals within the
tolerance of the other residual tests.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2009_12850_b300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    from paper_2009_12850_b300 import build
    build.build()
    from paper_2009_12850_b300 import api
    return api


def _noalloc(L, m, U, S, stream):
    c = m.coefficients()
    out = L.pw_residuals_noalloc(m.nx, m.ny, m.nz, m.nzp, {"f64": L.PW_F64, "f32": L.PW_F32, "bf16": L.PW_BF16,
                                                              "bf16_out": L.PW_BF16_OUT}[m.dtype],
                                 list(c["W_uv"]), list(c["W_w"]),
                                 *(ctypes.c_void_p(t.data_ptr()) for t in U),
                                 *(ctypes.c_void_p(t.data_ptr()) for t in S), stream)
    return np.array(out).reshape(3, 4)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "bf16_out"])
def test_noalloc_matches_residuals_twice(pw, dtype):
    from paper_2009_12850_b300 import _lib as L
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # two different problems back to back: the second call must not depend on
    # what the first left in the shared scratch array
    for nx, ny, nz, seed in ((40, 30, 24, 1), (23, 37, 61, 2)):
        m = pw.Mesh(nx, ny, nz, 50.0, dtype=dtype, algo="native")
        U = [m.from_interior(a) for a in synthetic.wind_fields(nx, ny, nz, seed)]
        S = m.advect(*U)
        ref = m.residual_sums(*U, *S)
        for _ in range(2):
            got = _noalloc(L, m, U, S, stream)
            for q in range(3):
                for t in range(4):
                    den = ref[q, 1] if t < 2 else ref[q, 3]
                    assert abs(got[q, t] - ref[q, t]) <= 1e-13 * den, (dtype, q, t, got[q, t], ref[q, t])


def test_noalloc_rejects_oversized_columns(pw):
    from paper_2009_12850_b300 import _lib as L
    m = pw.Mesh(8, 8, 8, 50.0, dtype="f32")
    U = [m.zeros() for _ in range(3)]
    S = [m.empty_out() for _ in range(3)]
    nz = L.PW_NOALLOC_MAX_NZ + 1 if hasattr(L, "PW_NOALLOC_MAX_NZ") else 4097
    with pytest.raises(L.PWError) as e:
        L.pw_residuals_noalloc(8, 8, nz, (nz + 7) // 8 * 8, L.PW_F32, [1.0] * nz, [1.0] * nz,
                               *(ctypes.c_void_p(t.data_ptr()) for t in U + S),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert e.value.status == L.PW_ERR_SHAPE
    assert "PW_NOALLOC_MAX_NZ" in str(e.value)


def test_noalloc_refuses_host_memory(pw):
    """A pinned host buffer in place of a device field is refused before any
    launch (PW_ERR_ARG), as is a weight list of the wrong length."""
    from paper_2009_12850_b300 import _lib as L
    m = pw.Mesh(8, 8, 8, 50.0, dtype="f32")
    U = [m.zeros() for _ in range(3)]
    S = [m.empty_out() for _ in range(3)]
    host = torch.zeros(m.shape, dtype=torch.float32, pin_memory=True)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptrs = [ctypes.c_void_p(t.data_ptr()) for t in U + S]
    ptrs[1] = ctypes.c_void_p(host.data_ptr())
    with pytest.raises(L.PWError) as e:
        L.pw_residuals_noalloc(8, 8, 8, m.nzp, L.PW_F32, [1.0] * 8, [1.0] * 8, *ptrs, stream)
    assert e.value.status == L.PW_ERR_ARG and "v is not device memory" in str(e.value)
    with pytest.raises(ValueError):
        L.pw_residuals_noalloc(8, 8, 8, m.nzp, L.PW_F32, [1.0] * 7, [1.0] * 8,
                               *(ctypes.c_void_p(t.data_ptr()) for t in U + S), stream)
