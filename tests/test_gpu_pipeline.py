"""GPU tests of the host-memory step (pw_advect_host): results against the FP64
oracle and bit for bit against the device path (halo fill + stencil), slab
widths from 1 column to the whole domain, accumulation, host halos left alone,
scalars (theta, q) travelling with the wind,
the per-slab callbacks, and reuse of one pipeline over several steps."""
import threading

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


def host_fields(pipe, arrs):
    m = pipe.mesh
    out = []
    for a in arrs:
        t = pipe.empty_host()
        t[2:m.nx + 2, 2:m.ny + 2, :m.nz] = torch.from_numpy(a).to(t.dtype)
        out.append(t)
    return out


def device_reference(pw, m, arrs, beta=0, init=None):
    U = [m.from_interior(a) for a in arrs]
    S = [m.zeros(m.out_dtype) for _ in range(3)]
    if init is not None:
        for s, a in zip(S, init):
            m.interior(s).copy_(torch.from_numpy(a).to(s.dtype))
    m.advect(*U, *S, beta=beta)
    torch.cuda.synchronize()
    return [m.interior(s).cpu() for s in S]


CASES = [((40, 24, 16), 7), ((40, 24, 16), 1), ((40, 24, 16), 40), ((40, 24, 16), 100), ((33, 5, 9), 0),
         ((1, 12, 6), 0), ((2, 3, 2), 1), ((64, 64, 64), 16)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])) + f"_slab{c[1]}")
@pytest.mark.parametrize("dtype,algo", [("f64", "split"), ("f64", "native"), ("f32", "auto"), ("bf16", "auto")])
def test_host_step_matches_device_and_oracle(pw, case, dtype, algo):
    (nx, ny, nz), slab = case
    m = pw.Mesh(nx, ny, nz, 50.0, 30.0, dtype=dtype, algo=algo)
    pipe = pw.Pipeline(m, slab)
    f = synthetic.wind_fields(nx, ny, nz, 41)
    f = [torch.from_numpy(a).to(m.in_dtype).double().numpy() for a in f]
    H = host_fields(pipe, f)
    O = [pipe.empty_host(out=True) for _ in range(3)]
    pipe.advect_host(*H, *O)
    pipe.sync()
    assert m.device_status() == 0
    got = [o[2:nx + 2, 2:ny + 2, :nz] for o in O]
    ref_dev = device_reference(pw, m, f)
    for a, b in zip(got, ref_dev):
        assert torch.equal(a, b)
    ref, cond = oracle.advect(oracle.Coeffs(nz, 50.0, 30.0), *f, want_cond=True)
    tol = TOL_F64 if dtype == "f64" else TOL_F32_COND
    for q in range(3):
        compare("s", got[q].double().numpy(), ref[q], cond[q], tol, tol)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_host_step_accumulate_and_halos_untouched(pw, dtype):
    nx, ny, nz = 29, 18, 11
    m = pw.Mesh(nx, ny, nz, 40.0, dtype=dtype)
    pipe = pw.Pipeline(m, 6)
    f = synthetic.wind_fields(nx, ny, nz, 42)
    rng = np.random.default_rng(43)
    init = [rng.standard_normal((nx, ny, nz)) for _ in range(3)]
    H = host_fields(pipe, f)
    O = []
    for a in init:
        t = torch.full(m.shape, -7.0, dtype=m.out_dtype).pin_memory()
        t[2:nx + 2, 2:ny + 2, :nz] = torch.from_numpy(a).to(t.dtype)
        O.append(t)
    pipe.advect_host(*H, *O, beta=1)
    pipe.sync()
    ref_dev = device_reference(pw, m, f, beta=1, init=init)
    mask = torch.ones(m.shape, dtype=torch.bool)
    mask[2:nx + 2, 2:ny + 2, :nz] = False
    for o, r in zip(O, ref_dev):
        assert torch.equal(o[2:nx + 2, 2:ny + 2, :nz], r)
        assert torch.all(o[mask] == -7.0)


def test_callbacks_report_every_slab_in_order(pw):
    nx, ny, nz = 50, 20, 10
    m = pw.Mesh(nx, ny, nz, 50.0, dtype="f32")
    pipe = pw.Pipeline(m, 8)
    assert pipe.slab == 8 and pipe.nslab == 7
    f = synthetic.wind_fields(nx, ny, nz, 44)
    H = host_fields(pipe, f)
    O = [pipe.empty_host(out=True) for _ in range(3)]
    seen, lock = [], threading.Lock()
    ready = []

    def on_slab(i0, i1):
        with lock:
            seen.append((i0, i1))
            # the slab is already in the host arrays when the callback runs
            ready.append(bool(torch.any(O[0][i0 + 2:i1 + 2, 2:ny + 2, :nz] != 0)))

    pipe.advect_host(*H, *O, on_slab=on_slab)
    pipe.sync()
    assert seen == [(i, min(i + 8, nx)) for i in range(0, nx, 8)]
    assert all(ready)
    # a second call waits for the first one's callbacks before reusing them
    seen.clear()
    pipe.advect_host(*H, *O, on_slab=on_slab)
    pipe.advect_host(*H, *O, on_slab=on_slab)
    pipe.sync()
    assert len(seen) == 2 * pipe.nslab


def test_pipeline_reuse_over_steps(pw):
    """Several steps through one pipeline with different inputs, no sync in
    between except the final one; each step's output matches its own input."""
    nx, ny, nz = 37, 21, 13
    m = pw.Mesh(nx, ny, nz, 50.0, dtype="f64")
    pipe = pw.Pipeline(m, 5)
    outs = []
    for step in range(3):
        f = synthetic.wind_fields(nx, ny, nz, 50 + step)
        H = host_fields(pipe, f)
        O = [pipe.empty_host(out=True) for _ in range(3)]
        pipe.advect_host(*H, *O)
        outs.append((f, H, O))
    pipe.sync()
    for f, _, O in outs:
        ref_dev = device_reference(pw, m, f)
        for o, r in zip(O, ref_dev):
            assert torch.equal(o[2:nx + 2, 2:ny + 2, :nz], r)


def test_pipeline_argument_errors(pw):
    from paper_2009_12850_b300 import _lib as L
    m = pw.Mesh(8, 8, 8, 50.0, dtype="f32")
    with pytest.raises(L.PWError):
        pw.Pipeline(m, -1)
    pipe = pw.Pipeline(m, 3)
    H = [pipe.empty_host() for _ in range(3)]
    O = [pipe.empty_host(out=True) for _ in range(3)]
    with pytest.raises(L.PWError):
        pipe.advect_host(*H, O[0], O[0], O[2])
    with pytest.raises(L.PWError):
        pipe.advect_host(*H, *O, beta=3)
    with pytest.raises(TypeError):
        pipe.advect_host(*H, H[0].double(), O[1], O[2])


@pytest.mark.parametrize("dtype,algo", [("f64", "split"), ("f32", "auto"), ("bf16", "auto")])
@pytest.mark.parametrize("slab", [1, 6, 0, 100])
def test_host_step_with_scalars(pw, dtype, algo, slab):
    """theta + q travel with the wind: every source equals the device path's,
    bit for bit, and host halos of the outputs are left alone."""
    nx, ny, nz = 31, 19, 14
    m = pw.Mesh(nx, ny, nz, 45.0, dtype=dtype, algo=algo)
    pipe = pw.Pipeline(m, slab)
    pipe.reserve_scalars(3)
    f = synthetic.wind_fields(nx, ny, nz, 81)
    phis = synthetic.scalar_fields(nx, ny, nz, 3, 82)
    H = host_fields(pipe, f)
    HP = host_fields(pipe, phis)
    O = [torch.full(m.shape, -3.0, dtype=m.out_dtype).pin_memory() for _ in range(3)]
    OP = [torch.full(m.shape, -3.0, dtype=m.out_dtype).pin_memory() for _ in range(3)]
    pipe.advect_host(*H, *O, scalars=HP, sources=OP)
    pipe.sync()
    assert m.device_status() == 0
    U = [m.from_interior(torch.from_numpy(a).to(m.in_dtype)) for a in f]
    P = [m.from_interior(torch.from_numpy(a).to(m.in_dtype)) for a in phis]
    S = m.advect(*U)
    SP = m.advect_scalars(*U, P)
    torch.cuda.synchronize()
    mask = torch.ones(m.shape, dtype=torch.bool)
    mask[2:nx + 2, 2:ny + 2, :nz] = False
    for o, s in zip(O + OP, list(S) + list(SP)):
        assert torch.equal(o[2:nx + 2, 2:ny + 2, :nz], m.interior(s).cpu())
        assert torch.all(o[mask] == -3.0)


def test_host_step_scalars_need_reserved_buffers(pw):
    from paper_2009_12850_b300 import _lib as L
    m = pw.Mesh(12, 10, 8, 50.0, dtype="f32")
    pipe = pw.Pipeline(m, 4)
    H = [pipe.empty_host() for _ in range(3)]
    O = [pipe.empty_host(out=True) for _ in range(3)]
    HP = [pipe.empty_host() for _ in range(2)]
    OP = [pipe.empty_host(out=True) for _ in range(2)]
    with pytest.raises(L.PWError):
        pipe.advect_host(*H, *O, scalars=HP, sources=OP)
    pipe.reserve_scalars(1)
    with pytest.raises(L.PWError):
        pipe.advect_host(*H, *O, scalars=HP, sources=OP)
    pipe.reserve_scalars(2)
    pipe.advect_host(*H, *O, scalars=HP, sources=OP)
    with pytest.raises(L.PWError):
        pipe.advect_host(*H, *O, scalars=HP, sources=[OP[0], O[0]])   # an output listed twice
    pipe.sync()
    assert m.device_status() == 0
