"""Fields past 2^31 elements: 2048 x 2048 x 520 points (2052 x 2052 x 520 with
the halos, 2.19e9 elements per field, so element and byte offsets of the last
columns need 64 bits in every kernel).  The fields are a 64 x 64 block of
seeded noise repeated over the domain; the stencil is local and periodic, so
the exact result at every one of the 2.2e9 points is the oracle's result on
the single periodic block, repeated.  Device memory: about 60 GB (FP32) and
125 GB (FP64) at the peak of each test."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_12850_b300 import synthetic

from parity import TOL_F32_COND, TOL_F64

pytestmark = pytest.mark.gpu

B, REP, NZ = 64, 32, 520          # block edge, repeats per horizontal direction, levels
N = B * REP                       # 2048


@pytest.fixture(scope="module")
def pw():
    from paper_2009_12850_b300 import build
    build.build()
    from paper_2009_12850_b300 import api
    return api


def big_fields(m, block, dtype):
    out = []
    for a in block:
        t = torch.from_numpy(a).to(device="cuda", dtype=dtype)
        out.append(m.from_interior(t.repeat(REP, REP, 1)))
        del t
    torch.cuda.empty_cache()
    return out


def check_tiled(m, got, ref, bound):
    """|got - tile(ref)| <= tile(bound) at every interior point, 64 rows of x at a time."""
    g = m.interior(got).view(REP, B, REP, B, NZ)
    r = torch.from_numpy(ref).cuda().view(1, B, 1, B, NZ)
    b = torch.from_numpy(bound).cuda().view(1, B, 1, B, NZ)
    worst = 0.0
    for a in range(REP):
        err = (g[a:a + 1].double() - r).abs()
        worst = max(worst, float((err / b.clamp_min(1e-300)).max()))
        del err
    return worst


def test_fp32_advect_and_step_past_2_31_elements(pw):
    torch.cuda.empty_cache()
    m = pw.Mesh(N, N, NZ, 50.0, dtype="f32")
    assert (N + 4) * (N + 4) * m.nzp > 2 ** 31
    block = [torch.from_numpy(a).float().double().numpy() for a in synthetic.wind_fields(B, B, NZ, 401)]
    U = big_fields(m, block, torch.float32)
    c = oracle.Coeffs(NZ, 50.0, 50.0)
    ref, cond = oracle.advect(c, *block, want_cond=True)
    S = m.advect(*U)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    for q in range(3):
        assert check_tiled(m, S[q], ref[q], TOL_F32_COND * cond[q]) <= 1.0, q
    del S
    torch.cuda.empty_cache()
    dt = 0.5
    N1 = m.step(*U, dt=dt)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    xr = oracle.euler(c, *block, dt, 1)
    for q in range(3):
        r = xr[q].copy()
        if q == 2:
            r[:, :, -1] = 0.0
        bound = TOL_F32_COND * dt * cond[q] + 2.0 ** -23 * (np.abs(block[q]) + np.abs(r))
        assert check_tiled(m, N1[q], r, bound) <= 1.0, q
    # the step wrote the periodic halo images of the new state: refilling them changes nothing
    h = N1[0].clone()
    m.halo(h)
    torch.cuda.synchronize()
    assert torch.equal(h[:, :, :NZ], N1[0][:, :, :NZ])
    del U, N1, h, m
    torch.cuda.empty_cache()


def test_fp64_split_advect_past_2_31_elements(pw):
    torch.cuda.empty_cache()
    m = pw.Mesh(N, N, NZ, 50.0, dtype="f64")
    block = list(synthetic.wind_fields(B, B, NZ, 402))
    U = big_fields(m, block, torch.float64)
    ref, cond = oracle.advect(oracle.Coeffs(NZ, 50.0, 50.0), *block, want_cond=True)
    S = m.advect(*U)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    for q in range(3):
        assert check_tiled(m, S[q], ref[q], TOL_F64 * cond[q]) <= 1.0, q
    del U, S, m
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_scalars_past_2_31_elements(pw, dtype):
    torch.cuda.empty_cache()
    m = pw.Mesh(N, N, NZ, 50.0, dtype=dtype)
    t = {"f32": torch.float32, "f64": torch.float64}[dtype]
    rnd = lambda a: torch.from_numpy(a).to(t).double().numpy()   # noqa: E731
    wind = [rnd(a) for a in synthetic.wind_fields(B, B, NZ, 403)]
    phis = [rnd(a) for a in synthetic.scalar_fields(B, B, NZ, 1, 404)]
    U = big_fields(m, wind, t)
    P = big_fields(m, phis, t)
    SP = m.advect_scalars(*U, P)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    ref, cond = oracle.advect_scalar(oracle.Coeffs(NZ, 50.0, 50.0), *wind, phis[0], want_cond=True)
    tol = TOL_F64 if dtype == "f64" else TOL_F32_COND
    assert check_tiled(m, SP[0], ref, tol * cond) <= 1.0
    del U, P, SP, m
    torch.cuda.empty_cache()


def test_fp32_adjoint_past_2_31_elements(pw):
    torch.cuda.empty_cache()
    m = pw.Mesh(N, N, NZ, 50.0, dtype="f32")
    rnd = lambda a: torch.from_numpy(a).float().double().numpy()   # noqa: E731
    wind = [rnd(a) for a in synthetic.wind_fields(B, B, NZ, 405)]
    rng = np.random.default_rng(406)
    y = [rnd(rng.standard_normal((B, B, NZ))) for _ in range(3)]
    y[2][:, :, -1] = 0.0   # sw on the lid has no effect
    U = big_fields(m, wind, torch.float32)
    Y = []
    for a in y:   # the adjoint fills the halo columns of the incoming gradients itself
        g = torch.from_numpy(a).to(device="cuda", dtype=torch.float32)
        Y.append(m.from_interior(g.repeat(REP, REP, 1), fill_halo=False))
        del g
    G = m.adjoint(*U, *Y)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    c = oracle.Coeffs(NZ, 50.0, 50.0)
    ref = oracle.adjoint(c, *wind, *y)
    cond = oracle.adjoint_cond(c, *wind, *y)
    for q in range(3):
        assert check_tiled(m, G[q], ref[q], 2 * TOL_F32_COND * cond[q]) <= 1.0, q
    del U, Y, G, m
    torch.cuda.empty_cache()
