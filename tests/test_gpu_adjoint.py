"""GPU parity of the hand-written adjoint (A7) through the C-ABI against the
oracle's transpose, plus the alpha/beta and Euler-adjoint conventions."""
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


def setup(pw, nx, ny, nz, dtype, seed=4, algo="native"):
    m = pw.Mesh(nx, ny, nz, 50.0, 30.0, dtype=dtype, algo=algo)
    u, v, w = synthetic.wind_fields(nx, ny, nz, seed)
    rng = np.random.default_rng(seed + 100)
    y = [rng.standard_normal((nx, ny, nz)) for _ in range(3)]
    y[2][:, :, -1] = rng.standard_normal((nx, ny))   # sw on the lid has no effect
    t = {"f64": torch.float64, "f32": torch.float32}[dtype]
    fr = [torch.from_numpy(a).to(t).double().numpy() for a in (u, v, w)]
    yr = [torch.from_numpy(a).to(t).double().numpy() for a in y]
    return m, fr, yr


def gpu_adjoint(m, f, y, alpha=1.0, beta=0, init=None):
    U = [m.from_interior(a) for a in f]
    Y = [m.from_interior(a, fill_halo=False) for a in y]
    G = [m.zeros() for _ in range(3)]
    if init is not None:
        for g, a in zip(G, init):
            m.interior(g).copy_(torch.from_numpy(a).to(g.dtype))
    m.adjoint(*U, *Y, *G, alpha=alpha, beta=beta)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    return [m.interior(g).double().cpu().numpy() for g in G], G


@pytest.mark.parametrize("shape", [(24, 20, 16), (37, 23, 13), (5, 7, 1), (1, 6, 5), (7, 1, 4), (3, 3, 2),
                                   (12, 10, 300)], ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("dtype,algo", [("f64", "native"), ("f64", "split"), ("f32", "auto")])
def test_adjoint_matches_oracle(pw, shape, dtype, algo):
    """The FP64 adjoint in native FP64 and in double-float (split) arithmetic,
    and the FP32 adjoint, against the oracle's transpose: 1e-12 normwise and of
    each point's gradient condition sum for FP64."""
    nx, ny, nz = shape
    m, f, y = setup(pw, nx, ny, nz, dtype, algo=algo)
    c = oracle.Coeffs(nz, 50.0, 30.0)
    y_eff = [y[0], y[1], y[2].copy()]
    y_eff[2][:, :, -1] = 0.0
    ref = oracle.adjoint(c, *f, *y_eff)
    cond = oracle.adjoint_cond(c, *f, *y_eff)
    got, G = gpu_adjoint(m, f, y)
    tol_n, tol_c = (TOL_F64, TOL_F64) if dtype == "f64" else (1e-5, 2 * TOL_F32_COND)
    for q in range(3):
        compare(f"g{'uvw'[q]}", got[q], ref[q], cond[q], tol_n, tol_c)
    assert not got[2][:, :, -1].any()
    # halos of the outputs are not written (they stay 0 here)
    h = G[0].double().cpu().numpy()
    assert not h[:2].any() and not h[:, :2].any()


@pytest.mark.parametrize("algo", ["native", "split"])
def test_alpha_beta(pw, algo):
    nx, ny, nz = 16, 12, 9
    m, f, y = setup(pw, nx, ny, nz, "f64", algo=algo)
    base, _ = gpu_adjoint(m, f, y)
    rng = np.random.default_rng(9)
    init = [rng.standard_normal((nx, ny, nz)) for _ in range(3)]
    got, _ = gpu_adjoint(m, f, y, alpha=-2.5, beta=1, init=init)
    for q in range(3):
        np.testing.assert_allclose(got[q], init[q] - 2.5 * base[q], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("algo", ["native", "split"])
def test_euler_adjoint(pw, algo):
    nx, ny, nz = 18, 14, 10
    dt = 0.5
    m, f, y = setup(pw, nx, ny, nz, "f64", algo=algo)
    base, _ = gpu_adjoint(m, f, y)
    U = [m.from_interior(a) for a in f]
    Y = [m.from_interior(a, fill_halo=False) for a in y]
    G = m.euler_adjoint(*U, *Y, dt=dt)
    torch.cuda.synchronize()
    for q in range(3):
        want = y[q] + dt * base[q]
        if q == 2:
            want = want.copy()
            want[:, :, -1] = 0.0
        np.testing.assert_allclose(m.interior(G[q]).double().cpu().numpy(), want, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("algo", ["native", "split"])
def test_dot_product_identity_on_device(pw, algo):
    """<J e, y> = <e, J^T y> with J e from the GPU forward by central differences
    (exact up to rounding: the sources are quadratic)."""
    nx, ny, nz = 20, 16, 12
    m, f, y = setup(pw, nx, ny, nz, "f64", algo=algo)
    rng = np.random.default_rng(5)
    e = [rng.standard_normal((nx, ny, nz)) for _ in range(3)]
    e[2][:, :, -1] = 0.0
    y[2][:, :, -1] = 0.0

    def fwd(fields):
        U = [m.from_interior(a) for a in fields]
        S = m.advect(*U)
        return [m.interior(s).double().cpu().numpy() for s in S]

    sp = fwd([f[q] + e[q] for q in range(3)])
    sm = fwd([f[q] - e[q] for q in range(3)])
    Je = [(sp[q] - sm[q]) / 2 for q in range(3)]
    JTy, _ = gpu_adjoint(m, f, y)
    lhs = sum(float(np.sum(Je[q] * y[q])) for q in range(3))
    rhs = sum(float(np.sum(e[q] * JTy[q])) for q in range(3))
    scale = sum(float(np.sum(np.abs(Je[q] * y[q]))) for q in range(3))
    assert abs(lhs - rhs) <= 1e-12 * scale


@pytest.mark.parametrize("kind", ["huge", "nan"])
def test_split_adjoint_out_of_range_is_reported(pw, kind):
    """The double-float adjoint reports inputs outside its range (here an
    incoming gradient) as PW_ERR_RANGE, like the forward."""
    from paper_2009_12850_b300 import _lib as L
    nx, ny, nz = 14, 12, 10
    m, f, y = setup(pw, nx, ny, nz, "f64", algo="split")
    y[1][5, 6, 3] = 2.0 ** 41 if kind == "huge" else np.nan
    U = [m.from_interior(a) for a in f]
    Y = [m.from_interior(a, fill_halo=False) for a in y]
    G = [m.zeros() for _ in range(3)]
    m.adjoint(*U, *Y, *G)
    torch.cuda.synchronize()
    assert m.device_status() == L.PW_ERR_RANGE
    assert m.device_status() == 0
