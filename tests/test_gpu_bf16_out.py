"""GPU tests of the bfloat16-output storage (PW_BF16_OUT: u, v, w and the
sources in bfloat16, FP32 arithmetic).  Its arithmetic is that of the
bfloat16-input mesh (PW_BF16, FP32 sources), so every source must equal that
path's FP32 source rounded once to bfloat16 (round to nearest even, which is
also torch's conversion); against the FP64 oracle the error is the FP32 bound
of the condition sum plus 2^-8 |S| for the final rounding."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_12850_b300 import synthetic

from parity import TOL_F32_COND

pytestmark = pytest.mark.gpu

BF16_U = 2.0 ** -8  # unit roundoff of bfloat16 (8 significant bits)


@pytest.fixture(scope="module")
def pw():
    from paper_2009_12850_b300 import build
    build.build()
    from paper_2009_12850_b300 import api
    return api


def pair(pw, nx, ny, nz, dx=40.0, dy=30.0):
    return (pw.Mesh(nx, ny, nz, dx, dy, dtype="bf16_out"), pw.Mesh(nx, ny, nz, dx, dy, dtype="bf16"))


SHAPES = [(40, 24, 16), (37, 23, 13), (5, 7, 1), (1, 9, 6), (33, 17, 130), (64, 64, 64)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_sources_are_the_bf16_path_rounded(pw, shape):
    nx, ny, nz = shape
    mo, mb = pair(pw, nx, ny, nz)
    f = synthetic.wind_fields(nx, ny, nz, 301)
    Uo = [mo.from_interior(a) for a in f]
    Ub = [mb.from_interior(a) for a in f]
    So = mo.advect(*Uo)
    Sb = mb.advect(*Ub)
    torch.cuda.synchronize()
    assert mo.device_status() == 0
    for a, b in zip(So, Sb):
        assert a.dtype == torch.bfloat16
        assert torch.equal(mo.interior(a), mb.interior(b).to(torch.bfloat16))


@pytest.mark.parametrize("shape", [(40, 24, 16), (33, 17, 130)], ids=lambda s: "x".join(map(str, s)))
def test_error_against_the_oracle(pw, shape):
    nx, ny, nz = shape
    mo, _ = pair(pw, nx, ny, nz)
    f = synthetic.wind_fields(nx, ny, nz, 302)
    fr = [torch.from_numpy(a).to(torch.bfloat16).double().numpy() for a in f]
    S = mo.advect(*[mo.from_interior(a) for a in f])
    torch.cuda.synchronize()
    ref, cond = oracle.advect(oracle.Coeffs(nz, 40.0, 30.0), *fr, want_cond=True)
    for q in range(3):
        got = mo.interior(S[q]).double().cpu().numpy()
        bound = TOL_F32_COND * cond[q] * (1 + BF16_U) + BF16_U * np.abs(ref[q])
        err = np.abs(got - ref[q])
        assert np.all(err <= bound), (q, float((err / np.maximum(bound, 1e-300)).max()))


def test_accumulate_rounds_the_sum(pw):
    nx, ny, nz = 29, 18, 11
    mo, mb = pair(pw, nx, ny, nz)
    f = synthetic.wind_fields(nx, ny, nz, 303)
    rng = np.random.default_rng(304)
    init = [torch.from_numpy(rng.standard_normal((nx, ny, nz))).to(torch.bfloat16) for _ in range(3)]
    So = [mo.zeros(mo.out_dtype) for _ in range(3)]
    for s, a in zip(So, init):
        mo.interior(s).copy_(a)
    mo.advect(*[mo.from_interior(a) for a in f], *So, beta=1)
    Sb = mb.advect(*[mb.from_interior(a) for a in f])
    torch.cuda.synchronize()
    for s, b, a in zip(So, Sb, init):
        # the new source is rounded to bfloat16, added to the old value in FP32, rounded again
        new = mb.interior(b).to(torch.bfloat16).float()
        want = (a.cuda().float() + new).to(torch.bfloat16)
        assert torch.equal(mo.interior(s), want)


def test_outputs_untouched_outside_interior(pw):
    nx, ny, nz = 12, 10, 13
    mo, _ = pair(pw, nx, ny, nz)
    f = synthetic.wind_fields(nx, ny, nz, 305)
    S = [mo.empty_out().fill_(7.0) for _ in range(3)]
    mo.advect(*[mo.from_interior(a) for a in f], *S)
    torch.cuda.synchronize()
    mask = torch.ones(mo.shape, dtype=torch.bool, device=S[0].device)
    mask[2:nx + 2, 2:ny + 2, :nz] = False
    for s in S:
        assert torch.all(s[mask] == 7.0)


def test_step_scalars_and_residuals(pw):
    nx, ny, nz = 31, 19, 14
    mo, mb = pair(pw, nx, ny, nz)
    f = synthetic.wind_fields(nx, ny, nz, 306)
    phis = synthetic.scalar_fields(nx, ny, nz, 3, 307)
    Uo, Ub = [mo.from_interior(a) for a in f], [mb.from_interior(a) for a in f]
    Po, Pb = [mo.from_interior(a) for a in phis], [mb.from_interior(a) for a in phis]
    # the fused step writes the field type for both storages: identical
    for a, b in zip(mo.step(*Uo, dt=0.4), mb.step(*Ub, dt=0.4)):
        assert torch.equal(a[:, :, :nz], b[:, :, :nz])
    for a, b in zip(mo.step_scalars(*Uo, Po, dt=0.4), mb.step_scalars(*Ub, Pb, dt=0.4)):
        assert torch.equal(a[:, :, :nz], b[:, :, :nz])
    # scalar sources: the FP32 sources of the bfloat16-input mesh, rounded
    for a, b in zip(mo.advect_scalars(*Uo, Po), mb.advect_scalars(*Ub, Pb)):
        assert a.dtype == torch.bfloat16
        assert torch.equal(mo.interior(a), mb.interior(b).to(torch.bfloat16))
    # conservation sums read bfloat16 sources
    So = mo.advect(*Uo)
    re, rm = mo.residuals(*Uo, *So)
    sums = mo.residual_sums(*Uo, *So)
    fo = [mo.interior(t).double().cpu().numpy() for t in Uo]
    so = [mo.interior(t).double().cpu().numpy() for t in So]
    want = oracle.residual_sums(oracle.Coeffs(nz, 40.0, 30.0), *fo, *so)
    np.testing.assert_allclose(sums, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    assert all(abs(x) < 1e-2 for x in re)
    assert mo.device_status() == 0


def test_host_pipeline_matches_device(pw):
    nx, ny, nz = 30, 16, 12
    mo, _ = pair(pw, nx, ny, nz)
    pipe = pw.Pipeline(mo, 7)
    f = synthetic.wind_fields(nx, ny, nz, 308)
    H = []
    for a in f:
        t = pipe.empty_host()
        t[2:nx + 2, 2:ny + 2, :nz] = torch.from_numpy(a).to(t.dtype)
        H.append(t)
    O = [pipe.empty_host(out=True) for _ in range(3)]
    pipe.advect_host(*H, *O)
    pipe.sync()
    S = mo.advect(*[mo.from_interior(a) for a in f])
    torch.cuda.synchronize()
    for o, s in zip(O, S):
        assert o.dtype == torch.bfloat16
        assert torch.equal(o[2:nx + 2, 2:ny + 2, :nz], mo.interior(s).cpu())


def test_unsupported_entry_points_refuse(pw):
    from paper_2009_12850_b300 import _lib as L
    mo, _ = pair(pw, 8, 8, 8)
    U = [mo.zeros() for _ in range(3)]
    S = [mo.zeros(mo.out_dtype) for _ in range(3)]
    with pytest.raises(L.PWError):
        mo.adjoint(*U, *S)
    with pytest.raises(L.PWError):
        mo.euler(*U, *S, 0.1)
    with pytest.raises(L.PWError):
        mo.halo_fold(*U)
    with pytest.raises(L.PWError):
        pw.Batch([mo])
    assert mo.device_status() == 0
