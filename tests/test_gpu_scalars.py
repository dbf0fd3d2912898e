"""GPU parity of the scalar (theta, q) PW advection through the C-ABI against the
FP64 oracle: FP64 (double-float split and native FP64), FP32 and BF16 storage, ragged
shapes, grouping of many scalars, accumulation, argument checks, and every
point of theta + 5 q on a full 1024x1024x128 launch."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_12850_b300 import synthetic

from parity import TOL_F32_COND, TOL_F64, compare, compare_slabs

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


def run_scalars(pw, m, wind, phis, beta=0, init=None):
    U = [m.from_interior(a) for a in wind]
    P = [m.from_interior(a) for a in phis]
    S = [m.empty_out() for _ in phis]
    if init is not None:
        for s, a in zip(S, init):
            s.zero_()
            m.interior(s).copy_(torch.from_numpy(a).to(s.dtype))
    m.advect_scalars(*U, P, S, beta=beta)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    return [m.interior(s).double().cpu().numpy() for s in S]


def tolerances(dtype):
    return (TOL_F64, TOL_F64) if dtype == "f64" else (TOL_F32_COND, TOL_F32_COND)


SHAPES = [(64, 64, 64), (37, 23, 13), (5, 7, 1), (1, 9, 6), (9, 1, 5), (3, 3, 2), (50, 17, 130),
          (16, 24, 300)]


KINDS = [("f64", "split"), ("f64", "native"), ("f32", "auto"), ("bf16", "auto")]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("dtype,algo", KINDS)
def test_scalars_match_oracle(pw, shape, dtype, algo):
    nx, ny, nz = shape
    m = pw.Mesh(nx, ny, nz, 50.0, 35.0, dtype=dtype, algo=algo)
    wind = rounded(synthetic.wind_fields(nx, ny, nz, 11), dtype)
    phis = rounded(synthetic.scalar_fields(nx, ny, nz, 3, 12), dtype)
    got = run_scalars(pw, m, wind, phis)
    c = oracle.Coeffs(nz, 50.0, 35.0)
    tn, tc = tolerances(dtype)
    for q, phi in enumerate(phis):
        ref, cond = oracle.advect_scalar(c, *wind, phi, want_cond=True)
        compare(f"s{q}", got[q], ref, cond, tn, tc)


@pytest.mark.parametrize("n", [1, 2, 5, 9, 16])
@pytest.mark.parametrize("dtype,algo", [("f64", "split"), ("f64", "native"), ("f32", "auto")])
def test_scalar_counts_and_groups(pw, n, dtype, algo):
    nx, ny, nz = 21, 34, 70
    m = pw.Mesh(nx, ny, nz, 40.0, dtype=dtype, algo=algo)
    wind = rounded(synthetic.wind_fields(nx, ny, nz, 13), dtype)
    phis = rounded(synthetic.scalar_fields(nx, ny, nz, n, 14), dtype)
    got = run_scalars(pw, m, wind, phis)
    c = oracle.Coeffs(nz, 40.0, 40.0)
    tn, tc = tolerances(dtype)
    for q, phi in enumerate(phis):
        ref, cond = oracle.advect_scalar(c, *wind, phi, want_cond=True)
        compare(f"s{q}", got[q], ref, cond, tn, tc)


@pytest.mark.parametrize("n", [6, 16])
@pytest.mark.parametrize("dtype,algo", [("f64", "split"), ("f64", "native"), ("f32", "auto"), ("bf16", "auto")])
def test_scalar_grouping_does_not_change_results(pw, n, dtype, algo):
    """Each scalar's source is independent of the group the launch puts it in:
    n scalars in one call (automatic groups) equal n calls of one scalar, bit
    for bit, on a tall column (several k chunks) with ragged sizes."""
    nx, ny, nz = 37, 19, 101
    m = pw.Mesh(nx, ny, nz, 45.0, dtype=dtype, algo=algo)
    wind = synthetic.wind_fields(nx, ny, nz, 17)
    phis = synthetic.scalar_fields(nx, ny, nz, n, 18)
    together = run_scalars(pw, m, wind, phis)
    for q, phi in enumerate(phis):
        alone = run_scalars(pw, m, wind, [phi])[0]
        assert np.array_equal(together[q], alone), q


@pytest.mark.parametrize("tile", [(1, 16), (2, 7), (4, 64), (8, 32), (3, 200)])
@pytest.mark.parametrize("algo", ["split", "native"])
def test_scalar_tiles_do_not_change_results(pw, tile, algo):
    nx, ny, nz = 45, 29, 40
    m = pw.Mesh(nx, ny, nz, 50.0, dtype="f64", algo=algo)
    wind = synthetic.wind_fields(nx, ny, nz, 15)
    phis = synthetic.scalar_fields(nx, ny, nz, 4, 16)
    base = run_scalars(pw, m, wind, phis)
    m.set_tile(*tile)
    other = run_scalars(pw, m, wind, phis)
    for a, b in zip(base, other):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("dtype,algo", [("f64", "split"), ("f64", "native"), ("f32", "auto")])
def test_scalar_accumulate(pw, dtype, algo):
    nx, ny, nz = 19, 22, 17
    m = pw.Mesh(nx, ny, nz, 30.0, dtype=dtype, algo=algo)
    wind = rounded(synthetic.wind_fields(nx, ny, nz, 17), dtype)
    phis = rounded(synthetic.scalar_fields(nx, ny, nz, 2, 18), dtype)
    rng = np.random.default_rng(19)
    init = [rng.standard_normal((nx, ny, nz)) for _ in phis]
    init = rounded(init, dtype)
    got = run_scalars(pw, m, wind, phis, beta=1, init=init)
    c = oracle.Coeffs(nz, 30.0, 30.0)
    tn, tc = tolerances(dtype)
    for q, phi in enumerate(phis):
        ref, cond = oracle.advect_scalar(c, *wind, phi, want_cond=True)
        compare(f"s{q}", got[q], ref + init[q], cond + np.abs(init[q]), 2 * tn, 2 * tc)


@pytest.mark.parametrize("algo", ["split", "native"])
def test_scalar_uniform_and_lid(pw, algo):
    nx, ny, nz = 12, 10, 9
    m = pw.Mesh(nx, ny, nz, 50.0, dtype="f64", algo=algo)
    U, V, W = np.full((nx, ny, nz), 4.0), np.full((nx, ny, nz), -2.0), np.zeros((nx, ny, nz))
    got = run_scalars(pw, m, (U, V, W), [np.full((nx, ny, nz), 301.5)])
    assert not got[0].any()
    wind = list(synthetic.wind_fields(nx, ny, nz, 20))
    phis = synthetic.scalar_fields(nx, ny, nz, 1, 21)
    a = run_scalars(pw, m, wind, phis)
    wind[2] = wind[2].copy()
    wind[2][:, :, -1] = 1e3
    b = run_scalars(pw, m, wind, phis)
    assert np.array_equal(a[0], b[0])


def test_scalar_outputs_untouched_outside_interior(pw):
    nx, ny, nz = 9, 8, 7
    m = pw.Mesh(nx, ny, nz, 50.0, dtype="f32")
    wind = synthetic.wind_fields(nx, ny, nz, 22)
    phis = synthetic.scalar_fields(nx, ny, nz, 2, 23)
    U = [m.from_interior(a) for a in wind]
    P = [m.from_interior(a) for a in phis]
    S = [torch.full(m.shape, 7.0, dtype=torch.float32, device=m.device) for _ in phis]
    m.advect_scalars(*U, P, S)
    torch.cuda.synchronize()
    for s in S:
        mask = torch.ones(m.shape, dtype=torch.bool, device=m.device)
        mask[2:nx + 2, 2:ny + 2, :nz] = False
        assert torch.all(s[mask] == 7.0)


def test_scalar_argument_errors(pw):
    from paper_2009_12850_b300 import _lib as L
    nx, ny, nz = 8, 8, 8
    m = pw.Mesh(nx, ny, nz, 50.0, dtype="f32")
    U = [m.zeros() for _ in range(3)]
    P = [m.zeros() for _ in range(17)]
    S = [m.empty_out() for _ in range(17)]
    with pytest.raises(L.PWError):
        m.advect_scalars(*U, P, S)                       # 17 > PW_MAX_SCALARS
    with pytest.raises(L.PWError):
        m.advect_scalars(*U, [], [])                     # none
    with pytest.raises(L.PWError):
        m.advect_scalars(*U, P[:2], [S[0], S[0]])        # outputs alias
    with pytest.raises(L.PWError):
        m.advect_scalars(*U, P[:1], [U[0]])              # output aliases the wind
    with pytest.raises(L.PWError):
        m.advect_scalars(*U, P[:2], [P[1], S[0]])        # output aliases a scalar
    with pytest.raises(L.PWError):
        m.advect_scalars(*U, P[:1], S[:1], beta=2)
    assert m.device_status() == 0


@pytest.mark.parametrize("dtype,algo", KINDS)
def test_scalars_full_size_every_point(pw, dtype, algo):
    """1024x1024x128 (the bandwidth workload) with theta + 5 q in one call and the
    default tiles and groups, as the benchmark runs it: every output point of every
    scalar against the oracle on the values the kernel sees (all host cores)."""
    oracle.set_threads(0)
    wl = synthetic.LARGE
    nx, ny, nz = wl.nx, wl.ny, wl.nz
    m = pw.Mesh(nx, ny, nz, wl.dx, wl.dy, dtype=dtype, algo=algo)
    wind = rounded(synthetic.fields_for(wl), dtype)
    phis = synthetic.scalar_fields(nx, ny, nz, 6, wl.seed + 100)
    for q in range(len(phis)):   # one at a time: each field is 1 GB in FP64
        phis[q] = rounded([phis[q]], dtype)[0]
    U = [m.from_interior(a) for a in wind]
    P = [m.from_interior(a) for a in phis]
    S = m.advect_scalars(*U, P)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    del U, P
    c = oracle.Coeffs(nz, wl.dx, wl.dy)
    tn, tc = tolerances(dtype)
    for q in range(len(phis)):
        ref, cond = oracle.advect_scalar(c, *wind, phis[q], want_cond=True)
        got = m.interior(S[q]).double().cpu().numpy()
        compare_slabs(f"s{q}", got, ref, cond, tn, tc)
        del ref, cond, got


def _log_uniform(rng, lo, hi, shape, zeros=0.1):
    x = np.exp2(rng.uniform(np.log2(lo), np.log2(hi), shape)) * rng.choice([-1.0, 1.0], shape)
    x = np.minimum(np.abs(x), np.nextafter(hi, 0)) * np.sign(x)
    x[rng.random(shape) < zeros] = 0.0
    return x


@pytest.mark.parametrize("lo,hi,wide_wind", [(2.0 ** -60, 2.0 ** -56, False), (1e-17, 1e-15, False),
                                             (1e-6, 1e3, False), (2.0 ** 56, 2.0 ** 60, False),
                                             (2.0 ** -110, 2.0 ** 60, False), (2.0 ** -60, 2.0 ** 60, True)],
                         ids=lambda x: f"{x:.3g}" if isinstance(x, float) else str(x))
def test_split_scalars_magnitude_range(pw, lo, hi, wide_wind):
    """The double-float path keeps the split bound for scalars across their
    range (below 2^60; moisture fields far below 1e-12 kg/kg included), with
    mixed signs and exact zeros, also under winds spread over [2^-40, 2^40):
    |err| <= 1e-12 cond + 2^-100 B + 2^-140, B = sum |h| (|wind| + |phi|) <=
    2 (largest |value| around the point) x (the condition sum of all-ones
    fields); nothing is reported."""
    nx, ny, nz = 23, 19, 33
    m = pw.Mesh(nx, ny, nz, 50.0, dtype="f64", algo="split")
    rng = np.random.default_rng(26)
    if wide_wind:
        wind = [_log_uniform(rng, 2.0 ** -40, 2.0 ** 40, (nx, ny, nz)) for _ in range(3)]
        wind[2][:, :, -1] = 0.0
    else:
        wind = synthetic.wind_fields(nx, ny, nz, 25)
    phi = _log_uniform(rng, lo, hi, (nx, ny, nz))
    got = run_scalars(pw, m, wind, [phi])
    c = oracle.Coeffs(nz, 50.0, 50.0)
    ref, cond = oracle.advect_scalar(c, *wind, phi, want_cond=True)
    ones = np.ones((nx, ny, nz))
    _, q1 = oracle.advect_scalar(c, ones, ones, ones, ones, want_cond=True)
    a = np.maximum.reduce([np.abs(x) for x in list(wind) + [phi]])
    for ax in (0, 1):
        a = np.maximum.reduce([a, np.roll(a, 1, ax), np.roll(a, -1, ax)])
    a = np.maximum.reduce([a, np.concatenate([a[:, :, 1:], a[:, :, -1:]], 2),
                           np.concatenate([a[:, :, :1], a[:, :, :-1]], 2)])
    err = np.abs(got[0] - ref)
    lim = 1e-12 * cond + 2.0 ** -100 * 2 * a * q1 + 2.0 ** -140
    assert np.all(err <= lim), float((err - lim).max())
    assert m.device_status() == 0


@pytest.mark.parametrize("bad", ["huge_scalar", "nan_scalar", "inf_scalar", "huge_wind"])
def test_split_scalars_out_of_range_is_reported(pw, bad):
    """A scalar at or above 2^60 in magnitude (or NaN, Inf), or a wind at or
    above 2^40, sets PW_ERR_RANGE."""
    from paper_2009_12850_b300 import _lib as L
    nx, ny, nz = 17, 15, 12
    m = pw.Mesh(nx, ny, nz, 50.0, dtype="f64", algo="split")
    wind = list(synthetic.wind_fields(nx, ny, nz, 27))
    phi = synthetic.scalar_fields(nx, ny, nz, 1, 28)[0]
    value = {"huge_scalar": 2.0 ** 60, "nan_scalar": np.nan, "inf_scalar": -np.inf, "huge_wind": 2.0 ** 40}[bad]
    if bad == "huge_wind":
        wind[1][8, 7, 4] = value
    else:
        phi[8, 7, 4] = value
    U = [m.from_interior(a) for a in wind]
    m.advect_scalars(*U, [m.from_interior(phi)])
    torch.cuda.synchronize()
    assert m.device_status() == L.PW_ERR_RANGE
    assert m.device_status() == 0
