"""Seeded randomized parity sweep: random domain shapes (including 1-wide and
non-multiple-of-tile sizes), random tile shapes and every arithmetic path, for
the wind stencil, the scalars, the fused step and ULTIMATE-QUICKEST (random
steps and wind directions), each against the FP64 oracle on the same inputs."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_12850_b300 import synthetic

from parity import TOL_F32_COND, TOL_F64, compare

pytestmark = pytest.mark.gpu

KINDS = [("f64", "split"), ("f64", "native"), ("f32", "auto"), ("bf16", "auto")]


@pytest.fixture(scope="module")
def pw():
    from paper_2009_12850_b300 import build
    build.build()
    from paper_2009_12850_b300 import api
    return api


def cases(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx = int(rng.choice([1, 2, 3, int(rng.integers(4, 90))]))
        ny = int(rng.choice([1, 2, 3, int(rng.integers(4, 90))]))
        nz = int(rng.choice([1, 2, 3, int(rng.integers(4, 200))]))
        tile = (int(rng.integers(1, 9)), int(rng.choice([1, 5, 16, 33, 64, 128])))
        dx, dy = float(rng.uniform(10, 200)), float(rng.uniform(10, 200))
        out.append((nx, ny, nz, tile, dx, dy, int(rng.integers(1 << 30))))
    return out


def rounded(arrs, dtype):
    t = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    return [torch.from_numpy(np.ascontiguousarray(a)).to(t).to(torch.float64).numpy() for a in arrs]


def tol(dtype):
    return TOL_F64 if dtype == "f64" else TOL_F32_COND


@pytest.mark.parametrize("case", cases(12, 2024), ids=lambda c: f"{c[0]}x{c[1]}x{c[2]}_t{c[3][0]}-{c[3][1]}")
@pytest.mark.parametrize("dtype,algo", KINDS)
def test_random_stencil(pw, case, dtype, algo):
    nx, ny, nz, tile, dx, dy, seed = case
    m = pw.Mesh(nx, ny, nz, dx, dy, dtype=dtype, algo=algo)
    m.set_tile(*tile)
    f = rounded(synthetic.wind_fields(nx, ny, nz, seed), dtype)
    U = [m.from_interior(a) for a in f]
    S = m.advect(*U)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    ref, cond = oracle.advect(oracle.Coeffs(nz, dx, dy), *f, want_cond=True)
    for q in range(3):
        compare("s" + "uvw"[q], m.interior(S[q]).double().cpu().numpy(), ref[q], cond[q], tol(dtype), tol(dtype))


@pytest.mark.parametrize("case", cases(8, 2025), ids=lambda c: f"{c[0]}x{c[1]}x{c[2]}_t{c[3][0]}-{c[3][1]}")
@pytest.mark.parametrize("dtype,algo", KINDS)
def test_random_scalars_and_step(pw, case, dtype, algo):
    nx, ny, nz, tile, dx, dy, seed = case
    m = pw.Mesh(nx, ny, nz, dx, dy, dtype=dtype, algo=algo)
    m.set_tile(min(tile[0], 8), tile[1])
    f = rounded(synthetic.wind_fields(nx, ny, nz, seed), dtype)
    n = 1 + seed % 7
    phis = rounded(synthetic.scalar_fields(nx, ny, nz, n, seed + 1), dtype)
    U = [m.from_interior(a) for a in f]
    P = [m.from_interior(a) for a in phis]
    SP = m.advect_scalars(*U, P)
    N = m.step(*U, dt=0.3)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    c = oracle.Coeffs(nz, dx, dy)
    for q, phi in enumerate(phis):
        ref, cond = oracle.advect_scalar(c, *f, phi, want_cond=True)
        compare(f"scalar{q}", m.interior(SP[q]).double().cpu().numpy(), ref, cond, tol(dtype), tol(dtype))
    xref = oracle.euler(c, *f, 0.3, 1)
    _, cond = oracle.advect(c, *f, want_cond=True)
    ulp = {"f64": 2.0 ** -52, "f32": 2.0 ** -23, "bf16": 2.0 ** -8}[dtype]
    for q in range(3):
        got = m.interior(N[q]).double().cpu().numpy()
        r = xref[q].copy()
        if q == 2:
            r[:, :, -1] = 0.0
        bound = tol(dtype) * 0.3 * cond[q] + ulp * (np.abs(f[q]) + np.abs(r))
        assert np.all(np.abs(got - r) <= bound), q


@pytest.mark.parametrize("dtype,algo", KINDS)
def test_tallest_columns(pw, dtype, algo):
    """nz = PW_MAX_NZ (4096 levels: many k chunks, the stretched grid down to its
    finest level): wind and scalar sources against the oracle."""
    from paper_2009_12850_b300 import _lib as L
    nx, ny, nz = 6, 5, L.PW_MAX_NZ
    m = pw.Mesh(nx, ny, nz, 50.0, dtype=dtype, algo=algo)
    f = rounded(synthetic.wind_fields(nx, ny, nz, 91), dtype)
    phis = rounded(synthetic.scalar_fields(nx, ny, nz, 2, 92), dtype)
    U = [m.from_interior(a) for a in f]
    P = [m.from_interior(a) for a in phis]
    S = m.advect(*U)
    SP = m.advect_scalars(*U, P)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    c = oracle.Coeffs(nz, 50.0, 50.0)
    ref, cond = oracle.advect(c, *f, want_cond=True)
    for q in range(3):
        compare("s" + "uvw"[q], m.interior(S[q]).double().cpu().numpy(), ref[q], cond[q], tol(dtype), tol(dtype))
    for q, phi in enumerate(phis):
        r, cd = oracle.advect_scalar(c, *f, phi, want_cond=True)
        compare(f"scalar{q}", m.interior(SP[q]).double().cpu().numpy(), r, cd, tol(dtype), tol(dtype))


def test_too_tall_column_rejected(pw):
    from paper_2009_12850_b300 import _lib as L
    with pytest.raises(L.PWError):
        pw.Mesh(4, 4, L.PW_MAX_NZ + 1, 50.0, dtype="f32")


# FP32 ULTIMATE-QUICKEST: the bound of test_gpu_tvd.py (a face's rounding, then
# the six flux terms, within 32 units of 2^-24 of the condition sum)
TOL_TVD_F32 = 32 * 2.0 ** -24


@pytest.mark.parametrize("case", cases(10, 2026), ids=lambda c: f"{c[0]}x{c[1]}x{c[2]}_t{c[3][0]}-{c[3][1]}")
@pytest.mark.parametrize("dtype,algo", KINDS)
def test_random_tvd(pw, case, dtype, algo):
    """ULTIMATE-QUICKEST on random shapes and tiles, with a random step (Courant
    numbers from near 0 to above 1) and winds of both signs, several scalars."""
    nx, ny, nz, tile, dx, dy, seed = case
    m = pw.Mesh(nx, ny, nz, dx, dy, dtype=dtype, algo=algo)
    m.set_tile(min(tile[0], 8), tile[1])
    rng = np.random.default_rng(seed)
    u, v, w = synthetic.wind_fields(nx, ny, nz, seed, u_mean=float(rng.uniform(-6, 6)),
                                    v_mean=float(rng.uniform(-6, 6)), u_std=3.0, v_std=3.0, w_std=1.0)
    f = rounded([u, v, w], dtype)
    n = 1 + seed % 4
    phis = rounded(synthetic.scalar_fields(nx, ny, nz, n, seed + 1), dtype)
    dt = float(rng.uniform(0.05, 1.3) * min(dx, dy) / 8.0)
    U = [m.from_interior(a) for a in f]
    P = [m.from_interior(a) for a in phis]
    S = m.advect_tvd(*U, P, dt)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    c = oracle.Coeffs(nz, dx, dy)
    t = TOL_F64 if dtype == "f64" else TOL_TVD_F32
    for q, phi in enumerate(phis):
        ref, cond = oracle.advect_tvd(c, *f, phi, dt, want_cond=True)
        compare(f"t{q}", m.interior(S[q]).double().cpu().numpy(), ref, cond, t if dtype == "f64" else 1e-5, t)
