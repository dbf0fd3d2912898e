"""GPU parity of the forward path through the C-ABI: coefficients (A1), periodic
halo fill (A2), the PW stencil in FP64 (A3) and FP32 / BF16 storage (A4), the
conservation sums (A5), the Euler update and the argument checks that need a
device.  The reference is the FP64 CPU oracle on the same seeded inputs."""
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


def make(pw, nx, ny, nz, dx=50.0, dy=None, dtype="f64", algo="auto", seed=3, **kw):
    m = pw.Mesh(nx, ny, nz, dx, dy, dtype=dtype, algo=algo, **kw)
    u, v, w = synthetic.wind_fields(nx, ny, nz, seed)
    return m, (u, v, w)


def rounded(arrs, dtype):
    t = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    return [torch.from_numpy(a).to(t).to(torch.float64).numpy() for a in arrs]


def run_forward(pw, m, fields, beta=0, init=None):
    U = [m.from_interior(a) for a in fields]
    S = [m.empty_out() for _ in range(3)]
    if init is not None:
        for s, a in zip(S, init):
            s.zero_()
            m.interior(s).copy_(torch.from_numpy(a).to(s.dtype))
    m.advect(*U, *S, beta=beta)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    return [m.interior(s).double().cpu().numpy() for s in S], U, S


SHAPES = [(64, 64, 64), (37, 23, 13), (5, 7, 1), (1, 9, 6), (9, 1, 5), (3, 3, 2), (50, 17, 130),
          (16, 24, 300)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("algo", ["native", "split"])
def test_forward_f64(pw, shape, algo):
    nx, ny, nz = shape
    m, f = make(pw, nx, ny, nz, dx=50.0, dy=35.0, algo=algo)
    c = oracle.Coeffs(nz, 50.0, 35.0)
    (ref, cond) = oracle.advect(c, *f, want_cond=True)
    got, _, _ = run_forward(pw, m, f)
    for q in range(3):
        compare(f"s{'uvw'[q]}", got[q], ref[q], cond[q], TOL_F64, TOL_F64)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("shape", [(64, 64, 64), (37, 23, 13), (5, 7, 1), (16, 24, 300), (50, 17, 130)],
                         ids=lambda s: "x".join(map(str, s)) if isinstance(s, tuple) else s)
def test_forward_reduced(pw, dtype, shape):
    nx, ny, nz = shape
    m, f = make(pw, nx, ny, nz, dx=25.0, dtype=dtype)
    c = oracle.Coeffs(nz, 25.0, 25.0)
    fr = rounded(f, dtype)   # the values the kernel actually sees
    ref, cond = oracle.advect(c, *fr, want_cond=True)
    got, _, _ = run_forward(pw, m, f)
    for q in range(3):
        compare(f"{dtype} s{'uvw'[q]}", got[q], ref[q], cond[q], 1e-5, TOL_F32_COND)


@pytest.mark.parametrize("algo", ["native", "split"])
def test_forward_accumulate(pw, algo):
    nx, ny, nz = 20, 12, 11
    m, f = make(pw, nx, ny, nz, algo=algo)
    c = oracle.Coeffs(nz, 50.0, 50.0)
    ref, cond = oracle.advect(c, *f, want_cond=True)
    rng = np.random.default_rng(1)
    init = [rng.standard_normal((nx, ny, nz)) for _ in range(3)]
    got, _, _ = run_forward(pw, m, f, beta=1, init=init)
    for q in range(3):
        compare("beta=1", got[q] - init[q], ref[q], cond[q] + np.abs(init[q]), 1e-12, 1e-12)


def test_outputs_untouched_outside_interior(pw):
    nx, ny, nz = 12, 10, 13
    m, f = make(pw, nx, ny, nz, dtype="f32")
    U = [m.from_interior(a) for a in f]
    S = [m.empty_out().fill_(7.0) for _ in range(3)]
    m.advect(*U, *S)
    torch.cuda.synchronize()
    for s in S:
        h = s.cpu().numpy()
        mask = np.ones(h.shape, bool)
        mask[2:nx + 2, 2:ny + 2, :nz] = False
        assert np.all(h[mask] == 7.0)


@pytest.mark.parametrize("algo", ["native", "split"])
def test_lid_value_ignored(pw, algo):
    nx, ny, nz = 16, 16, 12
    m, f = make(pw, nx, ny, nz, algo=algo)
    u, v, w = f
    w2 = w.copy()
    w2[:, :, -1] = 123.0
    a, _, _ = run_forward(pw, m, (u, v, w))
    b, _, _ = run_forward(pw, m, (u, v, w2))
    for q in range(3):
        assert np.array_equal(a[q], b[q])
    W = m.from_interior(w2)
    assert not m.check_lid(W)
    assert m.check_lid(m.from_interior(w))


def test_uniform_flow_exact_zero(pw):
    nx, ny, nz = 24, 20, 17
    for dtype, algo in (("f64", "native"), ("f64", "split"), ("f32", "auto"), ("bf16", "auto")):
        m = pw.Mesh(nx, ny, nz, 40.0, 30.0, dtype=dtype, algo=algo)
        u = np.full((nx, ny, nz), 7.25)
        v = np.full((nx, ny, nz), -3.5)
        w = np.zeros((nx, ny, nz))
        got, _, _ = run_forward(pw, m, (u, v, w))
        for g in got:
            assert not g.any(), dtype


def test_coefficients_match_oracle(pw):
    for nz, kw in ((64, {}), (3, {}), (1, {}), (7, {"dz": np.linspace(5, 30, 7), "rho_n": np.linspace(1.2, 0.9, 7),
                                                      "rho_w": np.linspace(1.19, 0.89, 7)})):
        m = pw.Mesh(4, 4, nz, 50.0, **kw)
        c = oracle.Coeffs(nz, 50.0, 50.0, dz=kw.get("dz"), rho_n=kw.get("rho_n"), rho_w=kw.get("rho_w"))
        g = m.coefficients()
        for name in ("dz", "zf", "zn", "dzn", "rho_n", "rho_w", "tzc1", "tzc2", "tzd1", "tzd2"):
            np.testing.assert_allclose(g[name], getattr(c, name), rtol=4e-16 * 8, atol=0, err_msg=name)
        wuv, ww = oracle.weights(c)
        np.testing.assert_allclose(g["W_uv"], wuv, rtol=4e-15)
        np.testing.assert_allclose(g["W_w"], ww, rtol=4e-15)
        assert g["tcx"] == 0.25 / 50.0


@pytest.mark.parametrize("shape", [(8, 6, 5), (1, 1, 3), (2, 3, 9), (1, 5, 4), (33, 2, 17)])
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_halo_fill_bit_exact(pw, shape, dtype):
    nx, ny, nz = shape
    m = pw.Mesh(nx, ny, nz, 50.0, dtype=dtype)
    rng = np.random.default_rng(2)
    a = rng.standard_normal((nx, ny, nz))
    t = m.from_interior(a, fill_halo=False)
    m.halo(t)
    torch.cuda.synchronize()
    h = t.double().cpu().numpy()
    ar = torch.from_numpy(a).to(m.in_dtype).double().numpy()
    ii = (np.arange(nx + 4) - 2) % nx
    jj = (np.arange(ny + 4) - 2) % ny
    want = ar[ii][:, jj]
    assert np.array_equal(h[:, :, :nz], want)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_euler_update_and_halo(pw, dtype):
    nx, ny, nz = 19, 6, 11
    m, f = make(pw, nx, ny, nz, dtype=dtype, algo="native")
    U = [m.from_interior(a) for a in f]
    S = list(m.advect(*U))
    before = [m.interior(x).double().cpu().numpy().copy() for x in U]
    sv = [m.interior(s).double().cpu().numpy() for s in S]
    m.euler(*U, *S, 0.5)
    torch.cuda.synchronize()
    for q in range(3):
        h = U[q].double().cpu().numpy()
        want = before[q] + 0.5 * sv[q]
        got = h[2:nx + 2, 2:ny + 2, :nz]
        eps = 2.2e-16 if dtype == "f64" else 1.2e-7
        assert np.all(np.abs(got - want) <= 2 * eps * (np.abs(want) + 1e-30))
        ii = (np.arange(nx + 4) - 2) % nx
        jj = (np.arange(ny + 4) - 2) % ny
        assert np.array_equal(h[:, :, :nz], got[ii][:, jj])


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_residual_sums(pw, dtype):
    nx, ny, nz = 40, 30, 24
    m, f = make(pw, nx, ny, nz, dtype=dtype, algo="native")
    U = [m.from_interior(a) for a in f]
    S = m.advect(*U)
    gsum = m.residual_sums(*U, *S)
    c = oracle.Coeffs(nz, 50.0, 50.0)
    fr = [m.interior(x).double().cpu().numpy() for x in U]
    sr = [m.interior(s).double().cpu().numpy() for s in S]
    ref = oracle.residual_sums(c, *fr, *sr)
    # the same products summed in another order: relative to the |.| sums
    for q in range(3):
        for t in range(4):
            den = ref[q, 1] if t < 2 else ref[q, 3]
            assert abs(gsum[q, t] - ref[q, t]) <= 1e-13 * den, (q, t, gsum[q, t], ref[q, t])
    # and deterministic run to run
    again = m.residual_sums(*U, *S)
    assert np.array_equal(gsum, again)
    if dtype == "f64":
        re, rm = m.residuals(*U, *S)
        assert max(abs(r) for r in re) < 1e-13


@pytest.mark.parametrize("case", ["huge", "tiny", "subnormal", "mixed_wide"])
def test_residual_sums_outside_fast_range(pw, case):
    """Fields the double-float pass cannot carry (|x| from 2^56 up, nonzero
    values below 2^-100, or sums of magnitudes below 2^-40) still give the FP64
    sums: the library recomputes them in plain FP64.  Native FP64 stencil, so
    the sources are the oracle's to 1e-12."""
    nx, ny, nz = 21, 18, 13
    m, f = make(pw, nx, ny, nz, algo="native")
    f = [a.copy() for a in f]
    rng = np.random.default_rng(5)
    if case == "huge":
        f[0][3, 4, 5] = 2.0 ** 60
    elif case == "tiny":
        f = [a * 1e-35 for a in f]
    elif case == "subnormal":
        f[1][2, 2, 2] = 5e-324
    else:
        f = [a * np.exp2(rng.uniform(-30, 30, a.shape)) for a in f]
    f[2][:, :, -1] = 0.0
    U = [m.from_interior(a) for a in f]
    S = m.advect(*U)
    gsum = m.residual_sums(*U, *S)
    c = oracle.Coeffs(nz, 50.0, 50.0)
    sr = [m.interior(s).double().cpu().numpy() for s in S]
    ref = oracle.residual_sums(c, *f, *sr)
    for q in range(3):
        for t in range(4):
            den = ref[q, 1] if t < 2 else ref[q, 3]
            assert abs(gsum[q, t] - ref[q, t]) <= 1e-13 * den, (case, q, t, gsum[q, t], ref[q, t])
    assert np.array_equal(gsum, m.residual_sums(*U, *S))


def test_argument_errors_on_device(pw):
    from paper_2009_12850_b300 import _lib as L
    m = pw.Mesh(8, 8, 8, 50.0, dtype="f32")
    U = [m.zeros() for _ in range(3)]
    S = [m.empty_out() for _ in range(3)]
    with pytest.raises(L.PWError) as e:
        m.advect(*U, *S, beta=2)
    assert e.value.status == L.PW_ERR_ARG
    # misaligned pointer
    big = torch.zeros(m.total + 4, device="cuda")
    bad = big[1:m.total + 1]
    with pytest.raises(L.PWError) as e:
        m.advect(bad, U[1], U[2], *S)
    assert e.value.status == L.PW_ERR_ALIGN
    with pytest.raises(L.PWError):
        m.advect(U[0], U[1], U[2], U[0], S[1], S[2])   # output aliases input
    with pytest.raises(TypeError):
        m.advect(U[0].double(), U[1], U[2], *S)
    with pytest.raises(L.PWError):
        m.set_tile(0, 32)
    m64 = pw.Mesh(8, 8, 8, 50.0, dtype="bf16")
    V = [m64.zeros() for _ in range(3)]
    with pytest.raises(L.PWError) as e:
        m64.adjoint(*V, *V, *V)
    assert e.value.status in (L.PW_ERR_DTYPE, L.PW_ERR_ARG)


@pytest.mark.parametrize("tile", [(1, 1), (3, 5), (8, 7), (16, 64), (4, 1000)])
def test_tiles_do_not_change_results(pw, tile):
    nx, ny, nz = 45, 29, 20
    m, f = make(pw, nx, ny, nz, dtype="f32")
    a, _, _ = run_forward(pw, m, f)
    m.set_tile(*tile)
    b, _, _ = run_forward(pw, m, f)
    for q in range(3):
        assert np.array_equal(a[q], b[q])


# the split arithmetic: inputs below 2^40 in magnitude; the 1e-12 condition
# bound alone holds when every nonzero value is at least 2^-40, and in general
# |err| <= 1e-12 cond + 2^-100 B + 2^-140 with B = sum |c| (|phi| + |a1| + |a2|)
SPLIT_LO, SPLIT_HI = 2.0 ** -40, 2.0 ** 40
FLOOR_ABS = 2.0 ** -140


def _log_uniform(rng, lo, hi, shape, zeros=0.1):
    """Random signs and magnitudes spread evenly in log2 over [lo, hi), with a
    fraction of exact zeros."""
    x = np.exp2(rng.uniform(np.log2(lo), np.log2(hi), shape)) * rng.choice([-1.0, 1.0], shape)
    x = np.minimum(np.abs(x), np.nextafter(hi, 0)) * np.sign(x)
    x[rng.random(shape) < zeros] = 0.0
    return x


def local_max(fields):
    """Largest |value| of any field over the 3x3x3 neighbourhood of each point
    (periodic in x and y; every operand of a point's stencil lies in it)."""
    a = np.maximum.reduce([np.abs(f) for f in fields])
    for ax in (0, 1):
        a = np.maximum.reduce([a, np.roll(a, 1, ax), np.roll(a, -1, ax)])
    up = np.concatenate([a[:, :, 1:], a[:, :, -1:]], axis=2)
    dn = np.concatenate([a[:, :, :1], a[:, :, :-1]], axis=2)
    return np.maximum.reduce([a, up, dn])


def check_split_bound(name, got, ref, cond, floor):
    err = np.abs(got - ref)
    bad = err > 1e-12 * cond + floor
    assert not bad.any(), (f"{name}: {int(bad.sum())} points above 1e-12 cond + floor; worst excess "
                           f"{float((err - 1e-12 * cond - floor).max()):.3e}")


@pytest.mark.parametrize("lo,hi", [(2.0 ** -40, 2.0 ** -36), (1e-6, 1e-5), (1.0, 10.0), (1e9, 1e10),
                                   (2.0 ** 36, 2.0 ** 40), (2.0 ** -40, 2.0 ** 40), (2.0 ** -12, 2.0 ** 12)],
                         ids=lambda x: f"{x:.3g}")
def test_split_magnitude_range(pw, lo, hi):
    """The split path keeps 1e-12 of each point's condition sum (2^-140 of
    absolute slack) for values across [2^-40, 2^40) -- at both ends, and with
    magnitudes mixed over the whole range inside one stencil -- with mixed signs
    and exact zeros, and reports nothing."""
    nx, ny, nz = 24, 20, 18
    m = pw.Mesh(nx, ny, nz, 50.0, dtype="f64", algo="split")
    rng = np.random.default_rng(21)
    f = [_log_uniform(rng, lo, hi, (nx, ny, nz)) for _ in range(3)]
    f[2][:, :, -1] = 0.0
    c = oracle.Coeffs(nz, 50.0, 50.0)
    ref, cond = oracle.advect(c, *f, want_cond=True)
    got, _, _ = run_forward(pw, m, f)
    for q in range(3):
        check_split_bound(f"split [{lo:g}, {hi:g}) s{'uvw'[q]}", got[q], ref[q], cond[q], FLOOR_ABS)
    assert m.device_status() == 0


@pytest.mark.parametrize("lo,hi", [(2.0 ** -130, 2.0 ** -100), (2.0 ** -110, 2.0 ** -60), (2.0 ** -90, 2.0 ** -40),
                                   (2.0 ** -130, 2.0 ** 39)], ids=lambda x: f"{x:.3g}")
def test_split_small_values(pw, lo, hi):
    """Values below 2^-40 (down to and past the 2^-110 read-as-zero limit,
    alone and mixed with large ones): within 1e-12 cond + 2^-100 B + 2^-140,
    B bounded by 1.5 x (largest |value| around the point) x (the condition sum
    of all-ones fields); nothing is reported."""
    nx, ny, nz = 22, 19, 15
    m = pw.Mesh(nx, ny, nz, 50.0, dtype="f64", algo="split")
    rng = np.random.default_rng(23)
    f = [_log_uniform(rng, lo, hi, (nx, ny, nz)) for _ in range(3)]
    f[2][:, :, -1] = 0.0
    c = oracle.Coeffs(nz, 50.0, 50.0)
    ref, cond = oracle.advect(c, *f, want_cond=True)
    _, q1 = oracle.advect(c, *[np.ones((nx, ny, nz))] * 3, want_cond=True)
    vloc = local_max(f)
    got, _, _ = run_forward(pw, m, f)
    for q in range(3):
        floor = 2.0 ** -100 * 1.5 * vloc * q1[q] + FLOOR_ABS
        check_split_bound(f"split small [{lo:g}, {hi:g}) s{'uvw'[q]}", got[q], ref[q], cond[q], floor)
    assert m.device_status() == 0


@pytest.mark.parametrize("corner", ["small", "large"])
def test_split_coefficient_corners(pw, corner):
    """Mesh coefficients at the ends of the accepted ranges (tcx, tcy, tzc,
    tzd in [2^-16, 2^8], 0.25 rho in [2^-36, 2^24]) with values at the matching
    ends of theirs: the smallest values with the smallest coefficients and
    density (the products nearest underflow) and the largest with the largest
    (nearest overflow)."""
    nx, ny, nz = 20, 17, 12
    if corner == "small":
        # 0.25 rho = 2^-36; tzc = 0.25 rho_w / (rho_n dz) = 0.25 / dz = 2^-16; tcx = 2^-16
        rho, dz, dx = np.full(nz, 2.0 ** -34), np.full(nz, 2.0 ** 14), 0.25 * 2.0 ** 16
        vlo, vhi = SPLIT_LO, 2.0 ** -36
    else:
        # 0.25 rho = 2^24; tzc = 0.25 / dz = 2^8; tcx = 2^8
        rho, dz, dx = np.full(nz, 2.0 ** 26), np.full(nz, 2.0 ** -10), 0.25 * 2.0 ** -8
        vlo, vhi = 2.0 ** 36, SPLIT_HI
    m = pw.Mesh(nx, ny, nz, dx, dz=dz, rho_n=rho, rho_w=rho, rho0=rho[0], H=1.0, dtype="f64", algo="split")
    assert m.algo == "split"
    rng = np.random.default_rng(22)
    f = [_log_uniform(rng, vlo, vhi, (nx, ny, nz), zeros=0.05) for _ in range(3)]
    f[2][:, :, -1] = 0.0
    c = oracle.Coeffs(nz, dx, dx, dz=dz, rho_n=rho, rho_w=rho, rho0=rho[0], H=1.0)
    ref, cond = oracle.advect(c, *f, want_cond=True)
    got, _, _ = run_forward(pw, m, f)
    for q in range(3):
        check_split_bound(f"split {corner} corner s{'uvw'[q]}", got[q], ref[q], cond[q], FLOOR_ABS)
    assert m.device_status() == 0


@pytest.mark.parametrize("bad", ["huge", "nan", "inf"])
@pytest.mark.parametrize("field", [0, 1, 2])
def test_split_out_of_range_is_reported(pw, bad, field):
    """An input at or above 2^40 in magnitude, NaN or Inf sets PW_ERR_RANGE in
    the mesh status (sticky until cleared; the next clean call reports 0); every
    point whose stencil does not touch the value still meets the bound.  Tiny
    values and subnormal doubles read as 0 without a report."""
    from paper_2009_12850_b300 import _lib as L
    nx, ny, nz = 19, 16, 14
    m, f = make(pw, nx, ny, nz, algo="split")
    value = {"huge": -(2.0 ** 40), "nan": np.nan, "inf": np.inf}[bad]
    i, j, k = 9, 7, 5
    g = [a.copy() for a in f]
    g[field][i, j, k] = value
    U = [m.from_interior(a) for a in g]
    S = m.advect(*U)
    torch.cuda.synchronize()
    assert m.device_status(clear=False) == L.PW_ERR_RANGE
    assert m.device_status() == L.PW_ERR_RANGE      # read and clear
    assert m.device_status() == 0
    # points more than one cell from (i, j, k) in x or y do not see the value
    c = oracle.Coeffs(nz, 50.0, 50.0)
    ref, cond = oracle.advect(c, *f, want_cond=True)
    far = np.ones((nx, ny, nz), bool)
    far[i - 2:i + 3, j - 2:j + 3, :] = False
    for q in range(3):
        out = m.interior(S[q]).double().cpu().numpy()
        compare("far points", out[far], ref[q][far], cond[q][far], TOL_F64, TOL_F64)
    # the same fields in range give no report
    m.advect(*[m.from_interior(a) for a in f])
    torch.cuda.synchronize()
    assert m.device_status() == 0
    # values below 2^-110 and subnormal doubles read as 0, without a report
    for tiny in (2.0 ** -111, 5e-324):
        g = [a.copy() for a in f]
        g[field][i, j, k] = tiny
        m.advect(*[m.from_interior(a) for a in g])
        torch.cuda.synchronize()
        assert m.device_status() == 0


def test_coefficients_outside_split_range(pw):
    """A mesh whose coefficients leave [2^-16, 2^8] (here tcx = 0.25/dx with
    dx = 10 km... 2.5e-6 < 2^-16) is refused for the split arithmetic and runs
    native FP64 under auto, still within 1e-12 of the oracle."""
    from paper_2009_12850_b300 import _lib as L
    nx, ny, nz, dx = 12, 10, 9, 1.0e5
    with pytest.raises(L.PWError) as e:
        pw.Mesh(nx, ny, nz, dx, dtype="f64", algo="split")
    assert e.value.status == L.PW_ERR_RANGE
    m = pw.Mesh(nx, ny, nz, dx, dtype="f64", algo="auto")
    assert m.algo == "native"
    assert pw.Mesh(nx, ny, nz, 50.0, dtype="f64").algo == "split"
    assert pw.Mesh(nx, ny, nz, dx, dtype="f32").algo == "auto"
    f = synthetic.wind_fields(nx, ny, nz, 4)
    c = oracle.Coeffs(nz, dx, dx)
    ref, cond = oracle.advect(c, *f, want_cond=True)
    got, _, _ = run_forward(pw, m, f)
    for q in range(3):
        compare("auto -> native", got[q], ref[q], cond[q], TOL_F64, TOL_F64)


@pytest.mark.parametrize("tile", [(1, 1), (3, 5), (8, 7), (4, 1000), (2, 64)])
def test_split_tiles(pw, tile):
    nx, ny, nz = 45, 29, 70
    m, f = make(pw, nx, ny, nz, algo="split")
    c = oracle.Coeffs(nz, 50.0, 50.0)
    ref, cond = oracle.advect(c, *f, want_cond=True)
    m.set_tile(*tile)
    got, _, _ = run_forward(pw, m, f)
    for q in range(3):
        compare("split tile", got[q], ref[q], cond[q], TOL_F64, TOL_F64)


@pytest.mark.parametrize("dtype,algo", [("f32", "auto"), ("f64", "split"), ("f64", "native")])
def test_timeout_status_is_reported_and_sticky(pw, dtype, algo):
    """A bounded wait that runs out (a barrier nothing completes, ~10 ms) sets
    PW_ERR_TIMEOUT; while it is set the stencil does nothing; clearing it
    restores normal operation.  No fault, no hang."""
    from paper_2009_12850_b300 import _lib as L
    nx, ny, nz = 20, 16, 12
    m, f = make(pw, nx, ny, nz, dtype=dtype, algo=algo)
    U = [m.from_interior(a) for a in f]
    S = [m.empty_out().fill_(3.0) for _ in range(3)]
    m.selftest_timeout(20_000_000)
    torch.cuda.synchronize()
    assert m.device_status(clear=False) == L.PW_ERR_TIMEOUT
    m.advect(*U, *S)
    torch.cuda.synchronize()
    for s in S:
        assert torch.all(m.interior(s) == 3.0)       # skipped while the status is set
    assert m.device_status(clear=True) == L.PW_ERR_TIMEOUT
    assert m.device_status() == 0
    m.advect(*U, *S)
    torch.cuda.synchronize()
    c = oracle.Coeffs(nz, 50.0, 50.0)
    fr = rounded(f, dtype)
    ref, cond = oracle.advect(c, *fr, want_cond=True)
    tol = (TOL_F64, TOL_F64) if dtype == "f64" else (1e-5, TOL_F32_COND)
    for q in range(3):
        compare("after clear", m.interior(S[q]).double().cpu().numpy(), ref[q], cond[q], *tol)
