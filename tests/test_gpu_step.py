"""GPU tests of the fused forward Euler steps (pw_advect_step for the wind,
pw_advect_scalars_step for theta and q): the new state against one Euler step
of the FP64 oracle, bit for bit against the unfused stencil + pw_euler
sequence, halo images, the lid, several steps in a row, and the argument
checks."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_12850_b300 import synthetic

from parity import TOL_F32_COND, TOL_F64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    from paper_2009_12850_b300 import build
    build.build()
    from paper_2009_12850_b300 import api
    return api


def rounded(arrs, dtype):
    t = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    return [torch.from_numpy(np.ascontiguousarray(a)).to(t).to(torch.float64).numpy() for a in arrs]


SHAPES = [(40, 24, 16), (37, 23, 13), (5, 7, 1), (1, 9, 6), (9, 1, 5), (3, 3, 2), (50, 17, 130)]
KINDS = [("f64", "split"), ("f64", "native"), ("f32", "auto"), ("bf16", "auto")]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("dtype,algo", KINDS)
def test_step_matches_oracle_euler(pw, shape, dtype, algo):
    nx, ny, nz = shape
    dt = 0.75
    m = pw.Mesh(nx, ny, nz, 50.0, 35.0, dtype=dtype, algo=algo)
    f = rounded(synthetic.wind_fields(nx, ny, nz, 61), dtype)
    U = [m.from_interior(a) for a in f]
    N = m.step(*U, dt=dt)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    c = oracle.Coeffs(nz, 50.0, 35.0)
    ref = oracle.euler(c, *f, dt, 1)
    _, cond = oracle.advect(c, *f, want_cond=True)
    tol, ulp = {"f64": (TOL_F64, 2.0 ** -52), "f32": (TOL_F32_COND, 2.0 ** -23), "bf16": (TOL_F32_COND, 2.0 ** -8)}[dtype]
    for q in range(3):
        got = m.interior(N[q]).double().cpu().numpy()
        r = ref[q].copy()
        if q == 2:
            r[:, :, -1] = 0.0  # the lid of the new state is 0
        bound = tol * dt * cond[q] + ulp * (np.abs(f[q]) + np.abs(r))
        err = np.abs(got - r)
        assert np.all(err <= bound), (q, float((err / np.maximum(bound, 1e-300)).max()))


@pytest.mark.parametrize("shape", [(40, 24, 16), (3, 3, 2), (1, 9, 6), (50, 17, 130)],
                         ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("dtype,algo", [("f64", "split"), ("f64", "native"), ("f32", "auto")])
def test_step_equals_advect_then_euler(pw, shape, dtype, algo):
    """The fused step writes exactly what pw_advect + pw_euler (which also
    refreshes the halos) leave in the fields, halos included."""
    nx, ny, nz = shape
    dt = 0.5
    m = pw.Mesh(nx, ny, nz, 40.0, dtype=dtype, algo=algo)
    f = synthetic.wind_fields(nx, ny, nz, 62)
    U = [m.from_interior(a) for a in f]
    N = m.step(*U, dt=dt)
    X = [t.clone() for t in U]
    S = m.advect(*X)
    m.euler(*X, *S, dt)
    torch.cuda.synchronize()
    X[2][:, :, nz - 1] = 0.0  # the unfused update leaves the lid as it was (0 here)
    for a, b in zip(N, X):
        assert torch.equal(a[:, :, :nz], b[:, :, :nz])


def test_step_lid_and_halos(pw):
    nx, ny, nz = 12, 10, 9
    m = pw.Mesh(nx, ny, nz, 50.0, dtype="f32")
    f = list(synthetic.wind_fields(nx, ny, nz, 63))
    f[2] = f[2].copy()
    f[2][:, :, -1] = 5.0  # a stored lid value is never read and not carried over
    U = [m.from_interior(a) for a in f]
    N = m.step(*U, dt=1.0)
    torch.cuda.synchronize()
    assert torch.all(N[2][:, :, nz - 1] == 0)
    for t in N:
        h = t.clone()
        m.halo(h)
        torch.cuda.synchronize()
        assert torch.equal(h[:, :, :nz], t[:, :, :nz])


@pytest.mark.parametrize("dtype,algo", [("f64", "split"), ("f32", "auto")])
def test_steps_in_a_row(pw, dtype, algo):
    nx, ny, nz = 33, 27, 21
    m = pw.Mesh(nx, ny, nz, 50.0, dtype=dtype, algo=algo)
    f = synthetic.wind_fields(nx, ny, nz, 64)
    A = [m.from_interior(a) for a in f]
    B = [m.empty() for _ in range(3)]
    X = [t.clone() for t in A]
    for _ in range(4):
        m.step(*A, *B, dt=0.25)
        A, B = B, A
        S = m.advect(*X)
        m.euler(*X, *S, 0.25)
    torch.cuda.synchronize()
    for a, x in zip(A, X):
        assert torch.equal(m.interior(a), m.interior(x))
    c = oracle.Coeffs(nz, 50.0, 50.0)
    ref = oracle.euler(c, *f, 0.25, 4)
    for q in range(3):
        got = m.interior(A[q]).double().cpu().numpy()
        scale = np.abs(ref[q]).max()
        tol = 1e-12 if dtype == "f64" else 1e-5
        assert np.abs(got - ref[q]).max() <= tol * scale


def test_step_argument_errors(pw):
    from paper_2009_12850_b300 import _lib as L
    m = pw.Mesh(8, 8, 8, 50.0, dtype="f32")
    U = [m.zeros() for _ in range(3)]
    N = [m.zeros() for _ in range(3)]
    with pytest.raises(L.PWError):
        m.step(*U, U[0], N[1], N[2])
    with pytest.raises(L.PWError):
        m.step(*U, N[0], N[0], N[2])
    with pytest.raises(L.PWError):
        m.step(*U, *N, dt=float("nan"))
    assert m.device_status() == 0


# --------------------------------------------------------------------------
# the fused step of the scalars (theta, q)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(40, 24, 16), (5, 7, 1), (1, 9, 6), (37, 23, 13), (50, 17, 130)],
                         ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("dtype,algo", KINDS)
def test_scalar_step_matches_oracle(pw, shape, dtype, algo):
    nx, ny, nz = shape
    dt = 0.6
    m = pw.Mesh(nx, ny, nz, 45.0, 30.0, dtype=dtype, algo=algo)
    f = rounded(synthetic.wind_fields(nx, ny, nz, 71), dtype)
    phis = rounded(synthetic.scalar_fields(nx, ny, nz, 3, 72), dtype)
    U = [m.from_interior(a) for a in f]
    P = [m.from_interior(a) for a in phis]
    N = m.step_scalars(*U, P, dt=dt)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    c = oracle.Coeffs(nz, 45.0, 30.0)
    tol, ulp = {"f64": (TOL_F64, 2.0 ** -52), "f32": (TOL_F32_COND, 2.0 ** -23), "bf16": (TOL_F32_COND, 2.0 ** -8)}[dtype]
    for q, phi in enumerate(phis):
        s, cond = oracle.advect_scalar(c, *f, phi, want_cond=True)
        r = phi + dt * s
        got = m.interior(N[q]).double().cpu().numpy()
        bound = tol * dt * cond + ulp * (np.abs(phi) + np.abs(r))
        err = np.abs(got - r)
        assert np.all(err <= bound), (q, float((err / np.maximum(bound, 1e-300)).max()))
        h = N[q].clone()
        m.halo(h)
        torch.cuda.synchronize()
        assert torch.equal(h[:, :, :nz], N[q][:, :, :nz])


@pytest.mark.parametrize("dtype,algo", [("f64", "split"), ("f64", "native"), ("f32", "auto")])
def test_scalar_step_equals_advect_then_euler(pw, dtype, algo):
    nx, ny, nz = 33, 21, 19
    m = pw.Mesh(nx, ny, nz, 40.0, dtype=dtype, algo=algo)
    f = synthetic.wind_fields(nx, ny, nz, 73)
    phis = synthetic.scalar_fields(nx, ny, nz, 3, 74)
    U = [m.from_interior(a) for a in f]
    P = [m.from_interior(a) for a in phis]
    N = m.step_scalars(*U, P, dt=0.4)
    X = [t.clone() for t in P]
    S = m.advect_scalars(*U, X)
    m.euler(*X, *S, 0.4)  # the Euler update of any three fields, halos refreshed
    torch.cuda.synchronize()
    for a, b in zip(N, X):
        assert torch.equal(a[:, :, :nz], b[:, :, :nz])


def test_scalar_step_argument_errors(pw):
    from paper_2009_12850_b300 import _lib as L
    m = pw.Mesh(8, 8, 8, 50.0, dtype="f32")
    U = [m.zeros() for _ in range(3)]
    P = [m.zeros() for _ in range(2)]
    with pytest.raises(L.PWError):
        m.step_scalars(*U, P, [P[0], m.zeros()])          # output aliases an input
    with pytest.raises(L.PWError):
        m.step_scalars(*U, P, dt=float("inf"))
    assert m.device_status() == 0
