"""GPU parity of the stencil on bfloat16 fields with long columns (32 to 300
levels, padded last k chunks) through the C-ABI: against the FP64 oracle on the
values the kernel sees, bfloat16 sources equal to the FP32 sources rounded,
accumulation, tiles, the lid and untouched halos, with ragged rows and ragged
tile marches."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_12850_b300 import synthetic

from parity import TOL_F32_COND, compare

pytestmark = pytest.mark.gpu

BF16_U = 2.0 ** -8
SHAPES = [(37, 23, 32), (19, 9, 64), (8, 17, 96), (5, 40, 160), (9, 11, 300), (1, 9, 64), (40, 1, 32),
          (3, 3, 128), (70, 33, 64)]


@pytest.fixture(scope="module")
def pw():
    from paper_2009_12850_b300 import build
    build.build()
    from paper_2009_12850_b300 import api
    return api


def bf16_values(arrs):
    return [torch.from_numpy(a).to(torch.bfloat16).double().numpy() for a in arrs]


def run(m, f, beta=0, init=None):
    U = [m.from_interior(a) for a in f]
    S = [m.empty_out() for _ in range(3)]
    if init is not None:
        for s, a in zip(S, init):
            s.zero_()
            m.interior(s).copy_(a.to(s.dtype))
    m.advect(*U, *S, beta=beta)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    return [m.interior(s).clone() for s in S]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("dtype", ["bf16", "bf16_out"])
def test_bf16_long_matches_oracle(pw, shape, dtype):
    nx, ny, nz = shape
    m = pw.Mesh(nx, ny, nz, 30.0, 45.0, dtype=dtype)
    f = synthetic.wind_fields(nx, ny, nz, 401)
    ref, cond = oracle.advect(oracle.Coeffs(nz, 30.0, 45.0), *bf16_values(f), want_cond=True)
    got = [s.double().cpu().numpy() for s in run(m, f)]
    for q in range(3):
        if dtype == "bf16":
            compare(f"s{'uvw'[q]}", got[q], ref[q], cond[q], 1e-5, TOL_F32_COND)
        else:
            bound = TOL_F32_COND * cond[q] * (1 + BF16_U) + BF16_U * np.abs(ref[q])
            err = np.abs(got[q] - ref[q])
            assert np.all(err <= bound), (q, float((err / np.maximum(bound, 1e-300)).max()))


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_bf16_long_bf16_sources_are_fp32_sources_rounded(pw, shape):
    nx, ny, nz = shape
    mo = pw.Mesh(nx, ny, nz, 30.0, 45.0, dtype="bf16_out")
    mb = pw.Mesh(nx, ny, nz, 30.0, 45.0, dtype="bf16")
    f = synthetic.wind_fields(nx, ny, nz, 402)
    for a, b in zip(run(mo, f), run(mb, f)):
        assert a.dtype == torch.bfloat16
        assert torch.equal(a, b.to(torch.bfloat16))


@pytest.mark.parametrize("dtype", ["bf16", "bf16_out"])
def test_bf16_long_accumulate(pw, dtype):
    nx, ny, nz = 21, 13, 96
    m = pw.Mesh(nx, ny, nz, 30.0, dtype=dtype)
    f = synthetic.wind_fields(nx, ny, nz, 403)
    rng = np.random.default_rng(404)
    init = [torch.from_numpy(rng.standard_normal((nx, ny, nz))).to(m.out_dtype).cuda() for _ in range(3)]
    fresh = run(m, f)
    acc = run(m, f, beta=1, init=init)
    for a, s, i in zip(acc, fresh, init):
        # the stored value plus the (rounded) new source in FP32, rounded to the output type
        assert torch.equal(a, (i.float() + s.float()).to(a.dtype))


@pytest.mark.parametrize("tile_i", [1, 3, 16, 1000])
def test_bf16_long_tiles_do_not_change_results(pw, tile_i):
    nx, ny, nz = 45, 29, 64
    m = pw.Mesh(nx, ny, nz, 50.0, dtype="bf16")
    f = synthetic.wind_fields(nx, ny, nz, 405)
    base = run(m, f)
    m.set_tile(m.get_tile()[0], tile_i)
    for a, b in zip(base, run(m, f)):
        assert torch.equal(a, b)


@pytest.mark.parametrize("dtype", ["bf16", "bf16_out"])
def test_bf16_long_lid_ignored_and_outside_untouched(pw, dtype):
    nx, ny, nz = 12, 10, 32
    m = pw.Mesh(nx, ny, nz, 30.0, dtype=dtype)
    u, v, w = synthetic.wind_fields(nx, ny, nz, 406)
    w2 = w.copy()
    w2[:, :, -1] = 123.0
    a = run(m, (u, v, w))
    b = run(m, (u, v, w2))
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    assert torch.all(a[2][:, :, nz - 1] == 0)
    U = [m.from_interior(x) for x in (u, v, w)]
    S = [m.empty_out().fill_(7.0) for _ in range(3)]
    m.advect(*U, *S)
    torch.cuda.synchronize()
    mask = torch.ones(m.shape, dtype=torch.bool, device=S[0].device)
    mask[2:nx + 2, 2:ny + 2, :nz] = False
    for s in S:
        assert torch.all(s[mask] == 7.0)
