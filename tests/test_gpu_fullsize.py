"""Parity at the full sizes the benchmark runs, in its launch configuration
(default tiles, halo fill by the library, then the stencil): sampled outputs of
the 1024x1024x128 bandwidth workload (FP64 split and native, FP32, BF16) and of
the 512x512x160 precision workload, each compared with the FP64 oracle
evaluated point by point."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_12850_b300 import synthetic

from parity import TOL_F32_COND, TOL_F64, compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    from paper_2009_12850_b300 import build
    build.build()
    from paper_2009_12850_b300 import api
    return api


@pytest.fixture(scope="module")
def large_fields():
    return synthetic.fields_for(synthetic.LARGE)


def rounded(arrs, dtype):
    if dtype == "f64":
        return list(arrs)
    t = {"f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    return [torch.from_numpy(a).to(t).to(torch.float64).numpy() for a in arrs]


def sample_points(nx, ny, nz, n, seed):
    rng = np.random.default_rng(seed)
    pts = np.stack([rng.integers(0, nx, n), rng.integers(0, ny, n), rng.integers(0, nz, n)], 1)
    # corners, the ground, the level under the lid, tile and chunk edges
    edges = [[0, 0, 0], [nx - 1, ny - 1, nz - 1], [0, ny - 1, nz - 2], [nx - 1, 0, 0], [63, 64, nz - 1],
             [64, 3, 63], [nx - 1, ny // 2, 64], [nx // 2, ny - 1, 1], [127, 128, 127 % nz]]
    return np.concatenate([pts, np.array(edges) % np.array([nx, ny, nz])])


def check_sampled(m, fields, S, c, pts, tn, tc):
    vals, cond = oracle.advect_points(c, *fields, pts)
    idx = torch.from_numpy(pts).to(m.device)
    for q, name in enumerate(("su", "sv", "sw")):
        got = m.interior(S[q])[idx[:, 0], idx[:, 1], idx[:, 2]].double().cpu().numpy()
        compare(name, got, vals[:, q], cond[:, q], tn, tc)


@pytest.mark.parametrize("dtype,algo", [("f64", "auto"), ("f64", "native"), ("f32", "auto"), ("bf16", "auto")])
def test_bandwidth_workload_sampled(pw, large_fields, dtype, algo):
    wl = synthetic.LARGE
    m = pw.Mesh(wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, dtype=dtype, algo=algo)
    f = rounded(large_fields, dtype)
    U = [m.from_interior(a, fill_halo=False) for a in f]
    S = [m.empty_out() for _ in range(3)]
    m.halo(*U)
    m.advect(*U, *S)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    c = oracle.Coeffs(wl.nz, wl.dx, wl.dy)
    tol = (TOL_F64, TOL_F64) if dtype == "f64" else (TOL_F32_COND, TOL_F32_COND)
    check_sampled(m, f, S, c, sample_points(wl.nx, wl.ny, wl.nz, 6000, 31), *tol)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_precision_workload_sampled(pw, dtype):
    wl = synthetic.PRECISION
    m = pw.Mesh(wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, dtype=dtype)
    f = rounded(synthetic.fields_for(wl), dtype)
    U = [m.from_interior(a) for a in f]
    S = m.advect(*U)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    c = oracle.Coeffs(wl.nz, wl.dx, wl.dy)
    tol = (TOL_F64, TOL_F64) if dtype == "f64" else (TOL_F32_COND, TOL_F32_COND)
    check_sampled(m, f, S, c, sample_points(wl.nx, wl.ny, wl.nz, 6000, 32), *tol)
