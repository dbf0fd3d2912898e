"""GPU parity of the ULTIMATE-QUICKEST scalar scheme (pw_advect_tvd, the
positivity-preserving scheme named in section 3.1) through the C-ABI against the
FP64 oracle: every storage kind, ragged shapes, Courant numbers below and above
1, many scalars, tiles, accumulation, the lid, untouched halos, argument checks,
the scheme's own properties on the device, and every point of theta + 5 q on a
full 1024x1024x128 launch."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_12850_b300 import synthetic

from parity import TOL_F64, compare, compare_slabs

pytestmark = pytest.mark.gpu

# FP32 arithmetic on exactly representable inputs.  Per face: the Courant number
# (two roundings), QUICKEST (at most 8 roundings, each of a quantity bounded by
# |phi_U| + |phi_C| + |phi_D| times a factor below 2), the bound
# phi_U + (phi_C - phi_U)/c (3 roundings of quantities bounded by |phi_U| +
# |phi_D|; the clamps select exactly), the flux a f and its coefficient (3); then
# six flux terms summed (5 roundings of partial sums bounded by the condition
# sum).  32 u of the condition sum covers this with room to spare.
TOL_TVD_F32 = 32 * 2.0 ** -24
# bfloat16 sources: the FP32 result rounded once more, |s| <= cond
TOL_TVD_BF16_OUT = TOL_TVD_F32 + 2.0 ** -8 * (1 + TOL_TVD_F32)


@pytest.fixture(scope="module")
def pw():
    from paper_2009_12850_b300 import build
    build.build()
    from paper_2009_12850_b300 import api
    return api


def rounded(arrs, dtype):
    t = {"f64": torch.float64, "f64n": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16,
         "bf16_out": torch.bfloat16}[dtype]
    return [torch.from_numpy(np.ascontiguousarray(a)).to(t).to(torch.float64).numpy() for a in arrs]


def run_tvd(m, wind, phis, dt, beta=0, init=None):
    U = [m.from_interior(a) for a in wind]
    P = [m.from_interior(a) for a in phis]
    S = [m.empty_out() for _ in phis]
    if init is not None:
        for s, a in zip(S, init):
            s.zero_()
            m.interior(s).copy_(torch.from_numpy(a).to(s.dtype))
    m.advect_tvd(*U, P, dt, S, beta=beta)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    return [m.interior(s).double().cpu().numpy() for s in S]


def mesh(pw, nx, ny, nz, dx, dy=None, dtype="f64"):
    """dtype "f64" is the double-float kernel (the FP64 default), "f64n" native FP64."""
    if dtype == "f64n":
        return pw.Mesh(nx, ny, nz, dx, dy if dy is not None else dx, dtype="f64", algo="native")
    return pw.Mesh(nx, ny, nz, dx, dy if dy is not None else dx, dtype=dtype)


def tolerances(dtype):
    if dtype in ("f64", "f64n"):
        return TOL_F64, TOL_F64
    if dtype == "bf16_out":   # the bfloat16 output alone rounds by up to 2^-8 of |s|
        return 2.0 ** -7, TOL_TVD_BF16_OUT
    return 1e-5, TOL_TVD_F32


SHAPES = [(64, 64, 64), (37, 23, 13), (5, 7, 1), (1, 9, 6), (9, 1, 5), (3, 3, 2), (50, 17, 130),
          (16, 24, 300), (2, 2, 33)]
DTYPES = ["f64", "f64n", "f32", "bf16", "bf16_out"]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("dt", [2.0, 9.0])
def test_tvd_matches_oracle(pw, shape, dtype, dt):
    # dt = 2 s: Courant numbers around 0.2 (dx 50 m, winds 5 +- 1 m/s);
    # dt = 9 s: around 0.9, some above 1 (the limiter's window closes there)
    nx, ny, nz = shape
    m = mesh(pw, nx, ny, nz, 50.0, 35.0, dtype=dtype)
    wind = rounded(synthetic.wind_fields(nx, ny, nz, 21), dtype)
    phis = rounded(synthetic.scalar_fields(nx, ny, nz, 2, 22), dtype)
    got = run_tvd(m, wind, phis, dt)
    c = oracle.Coeffs(nz, 50.0, 35.0)
    tn, tc = tolerances(dtype)
    for q, phi in enumerate(phis):
        ref, cond = oracle.advect_tvd(c, *wind, phi, dt, want_cond=True)
        compare(f"s{q}", got[q], ref, cond, tn, tc)


@pytest.mark.parametrize("dtype", ["f64", "f64n", "f32"])
def test_tvd_steep_and_signed_data(pw, dtype):
    """Fronts, plateaus, extrema and sign changes (every branch of the limiter:
    exact ties between neighbours, monotone runs where the Courant bound acts,
    extrema), with winds of both signs in every direction."""
    nx, ny, nz = 33, 26, 45
    rng = np.random.default_rng(23)
    u = 6.0 * rng.standard_normal((nx, ny, nz))
    v = 6.0 * rng.standard_normal((nx, ny, nz))
    w = 2.0 * rng.standard_normal((nx, ny, nz))
    w[:, :, -1] = 0.0
    phi = np.where(rng.random((nx, ny, nz)) < 0.5, 1.0, 0.0) + np.round(rng.standard_normal((nx, ny, nz)), 1)
    phi[:, :, 10:20] = 2.5  # a plateau: ties between neighbours
    wind, phis = rounded([u, v, w], dtype), rounded([phi], dtype)
    m = mesh(pw, nx, ny, nz, 40.0, dtype=dtype)
    c = oracle.Coeffs(nz, 40.0, 40.0)
    tn, tc = tolerances(dtype)
    for dt in (1.0, 4.0, 12.0):
        got = run_tvd(m, wind, phis, dt)[0]
        ref, cond = oracle.advect_tvd(c, *wind, phis[0], dt, want_cond=True)
        compare(f"dt{dt}", got, ref, cond, tn, tc)


@pytest.mark.parametrize("n", [1, 3, 16])
@pytest.mark.parametrize("dtype", ["f64", "f64n", "f32"])
def test_tvd_counts_are_independent(pw, n, dtype):
    """n scalars in one call equal n calls of one scalar, bit for bit, and match
    the oracle."""
    nx, ny, nz = 21, 34, 70
    m = mesh(pw, nx, ny, nz, 40.0, dtype=dtype)
    wind = rounded(synthetic.wind_fields(nx, ny, nz, 24), dtype)
    phis = rounded(synthetic.scalar_fields(nx, ny, nz, n, 25), dtype)
    together = run_tvd(m, wind, phis, 3.0)
    c = oracle.Coeffs(nz, 40.0, 40.0)
    tn, tc = tolerances(dtype)
    for q, phi in enumerate(phis):
        alone = run_tvd(m, wind, [phi], 3.0)[0]
        assert np.array_equal(together[q], alone), q
        ref, cond = oracle.advect_tvd(c, *wind, phi, 3.0, want_cond=True)
        compare(f"s{q}", together[q], ref, cond, tn, tc)


@pytest.mark.parametrize("tile_i", [1, 4, 7, 64, 300])
@pytest.mark.parametrize("dtype", ["f64", "f64n"])
def test_tvd_tiles_do_not_change_results(pw, tile_i, dtype):
    nx, ny, nz = 45, 29, 40
    m = mesh(pw, nx, ny, nz, 50.0, dtype=dtype)
    wind = synthetic.wind_fields(nx, ny, nz, 26)
    phis = synthetic.scalar_fields(nx, ny, nz, 2, 27)
    base = run_tvd(m, wind, phis, 5.0)
    m.set_tile(m.get_tile()[0], tile_i)
    other = run_tvd(m, wind, phis, 5.0)
    for a, b in zip(base, other):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("dtype", DTYPES)
def test_tvd_accumulate(pw, dtype):
    nx, ny, nz = 19, 22, 17
    m = mesh(pw, nx, ny, nz, 30.0, dtype=dtype)
    wind = rounded(synthetic.wind_fields(nx, ny, nz, 28), dtype)
    phis = rounded(synthetic.scalar_fields(nx, ny, nz, 2, 29), dtype)
    rng = np.random.default_rng(30)
    init = [rng.standard_normal((nx, ny, nz)) for _ in phis]
    if dtype == "bf16_out":
        init = rounded(init, "bf16")
    fresh = run_tvd(m, wind, phis, 2.0)
    acc = run_tvd(m, wind, phis, 2.0, beta=1, init=init)
    for a, f, i in zip(acc, fresh, init):
        if dtype == "bf16_out":
            # the FP32 sum of the stored value and the unrounded source, rounded
            # once (2^-8 of the sum); f itself is that source rounded (2^-8 of |f|)
            assert np.all(np.abs(a - (i + f)) <= 2.0 ** -8 * (np.abs(i + f) + 2 * np.abs(f)))
        else:
            tol = 1e-15 if dtype in ("f64", "f64n") else 2.0 ** -23
            assert np.allclose(a, i + f, rtol=tol, atol=tol * np.abs(i + f).max())


@pytest.mark.parametrize("dtype", ["f64", "f64n"])
def test_tvd_lid_and_halos_untouched(pw, dtype):
    nx, ny, nz = 13, 11, 9
    m = mesh(pw, nx, ny, nz, 30.0, dtype=dtype)
    u, v, w = synthetic.wind_fields(nx, ny, nz, 31)
    phi = synthetic.scalar_fields(nx, ny, nz, 1, 32)[0]
    base = run_tvd(m, [u, v, w], [phi], 2.0)[0]
    w2 = w.copy()
    w2[:, :, -1] = 7.0   # the lid value is never read
    assert np.array_equal(run_tvd(m, [u, v, w2], [phi], 2.0)[0], base)
    # only interior points of the source are written
    U = [m.from_interior(a) for a in (u, v, w)]
    P = m.from_interior(phi)
    S = m.empty_out()
    S.fill_(123.0)
    m.advect_tvd(*U, [P], 2.0, [S])
    torch.cuda.synchronize()
    mask = torch.ones(m.shape, dtype=torch.bool, device=m.device)
    mask[2:nx + 2, 2:ny + 2, :nz] = False
    assert torch.all(S[mask] == 123.0)


@pytest.mark.parametrize("dtype", ["f64", "f64n", "f32"])
def test_tvd_properties_on_device(pw, dtype):
    """What the scheme guarantees, checked on the device results at a size past
    a few tiles: one-dimensional uniform flow with c <= 1 keeps every value in
    the initial range and does not raise the total variation along the flow;
    Courant number 1 is an exact shift; a constant field stays constant under a
    divergence-free (uniform) wind."""
    nx, ny, nz = 200, 3, 2
    m = mesh(pw, nx, ny, nz, 10.0, dtype=dtype)
    rng = np.random.default_rng(33)
    line = np.where(np.arange(nx) % 23 < 9, 1.0, 0.0) + 0.1 * rng.random(nx)
    phi = rounded([np.broadcast_to(line[:, None, None], (nx, ny, nz)).copy()], dtype)[0]
    zero = np.zeros((nx, ny, nz))
    for U in (4.0, -4.0):
        for cr in (0.3, 0.8, 1.0):
            dt = cr * 10.0 / abs(U)
            s = run_tvd(m, [zero + U, zero, zero], [phi], dt)[0]
            new = phi + dt * s
            tol = 1e-13 if dtype in ("f64", "f64n") else 1e-5
            assert new.max() <= phi.max() + tol and new.min() >= phi.min() - tol
            tv = lambda a: np.abs(np.diff(np.r_[a, a[:1]])).sum()
            assert tv(new[:, 1, 0]) <= tv(phi[:, 1, 0]) * (1 + tol)
            if cr == 1.0:
                np.testing.assert_allclose(new, np.roll(phi, 1 if U > 0 else -1, axis=0), atol=tol)
    s = run_tvd(m, [zero + 3.0, zero - 2.0, zero], [zero + 4.5], 2.0)[0]
    assert np.abs(s).max() <= (1e-15 if dtype in ("f64", "f64n") else 1e-6)


def test_tvd_argument_errors(pw):
    from paper_2009_12850_b300 import _lib as L
    nx, ny, nz = 8, 8, 8
    m = pw.Mesh(nx, ny, nz, 30.0, dtype="f32")
    u, v, w = [m.from_interior(a) for a in synthetic.wind_fields(nx, ny, nz, 34)]
    p = m.from_interior(synthetic.scalar_fields(nx, ny, nz, 1, 35)[0])
    s = m.empty_out()
    for dt in (0.0, -1.0, float("inf"), float("nan")):
        with pytest.raises(L.PWError):
            m.advect_tvd(u, v, w, [p], dt, [s])
    with pytest.raises(L.PWError):
        m.advect_tvd(u, v, w, [p], 1.0, [s], beta=2)
    with pytest.raises(L.PWError):
        m.advect_tvd(u, v, w, [p], 1.0, [u])         # output aliases the wind
    with pytest.raises(L.PWError):
        m.advect_tvd(u, v, w, [p, p], 1.0, [s, s])
    with pytest.raises(L.PWError):
        m.advect_tvd(u, v, w, [], 1.0, [])
    assert m.device_status() == 0


@pytest.mark.parametrize("dtype", ["f64", "f64n", "f32", "bf16"])
def test_tvd_full_size_every_point(pw, dtype):
    """theta + 5 q on the 1024x1024x128 bandwidth workload (dx 25 m, dt 2 s) in the
    launch configuration the benchmark times (all six scalars in one call): every
    point of every scalar against the oracle (all host cores)."""
    oracle.set_threads(0)
    wl = synthetic.LARGE
    nx, ny, nz, dt = wl.nx, wl.ny, wl.nz, 2.0
    m = mesh(pw, nx, ny, nz, wl.dx, wl.dy, dtype=dtype)
    wind = rounded(synthetic.fields_for(wl), dtype)
    phis = synthetic.scalar_fields(nx, ny, nz, 6, wl.seed + 100)
    for q in range(len(phis)):   # one at a time: each field is 1 GB in FP64
        phis[q] = rounded([phis[q]], dtype)[0]
    U = [m.from_interior(a) for a in wind]
    P = [m.from_interior(a) for a in phis]
    S = [m.empty_out() for _ in phis]
    m.advect_tvd(*U, P, dt, S)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    del U, P
    c = oracle.Coeffs(nz, wl.dx, wl.dy)
    tn, tc = tolerances(dtype)
    for q in range(len(phis)):
        ref, cond = oracle.advect_tvd(c, *wind, phis[q], dt, want_cond=True)
        got = m.interior(S[q]).double().cpu().numpy()
        compare_slabs(f"s{q}", got, ref, cond, tn, tc)
        del ref, cond, got


def test_tvd_split_range_is_reported(pw):
    """The double-float kernel reads values outside its range as 0 and says so
    in the mesh status word; native FP64 has no such limit."""
    from paper_2009_12850_b300 import _lib as L
    nx, ny, nz = 12, 10, 9
    u, v, w = synthetic.wind_fields(nx, ny, nz, 36)
    phi = synthetic.scalar_fields(nx, ny, nz, 1, 37)[0]
    m = mesh(pw, nx, ny, nz, 30.0, dtype="f64")
    # in range: no report
    run_tvd(m, [u, v, w], [phi], 2.0)
    for bad in (float("nan"), float("inf"), 2.0 ** 61):
        p2 = phi.copy()
        p2[3, 4, 5] = bad
        U = [m.from_interior(a) for a in (u, v, w)]
        S = m.empty_out()
        m.advect_tvd(*U, [m.from_interior(p2)], 2.0, [S])
        torch.cuda.synchronize()
        assert m.device_status() == L.PW_ERR_RANGE
    u2 = u.copy()
    u2[1, 1, 1] = 2.0 ** 41
    U = [m.from_interior(a) for a in (u2, v, w)]
    S = m.empty_out()
    m.advect_tvd(*U, [m.from_interior(phi)], 2.0, [S])
    torch.cuda.synchronize()
    assert m.device_status() == L.PW_ERR_RANGE
    # native FP64 takes the large value as it is
    mn = mesh(pw, nx, ny, nz, 30.0, dtype="f64n")
    p2 = phi.copy()
    p2[3, 4, 5] = 2.0 ** 61
    got = run_tvd(mn, [u, v, w], [p2], 2.0)[0]
    ref, cond = oracle.advect_tvd(oracle.Coeffs(nz, 30.0, 30.0), u, v, w, p2, 2.0, want_cond=True)
    compare("native", got, ref, cond, TOL_F64, TOL_F64)
