"""Parity at the full sizes of the two workloads the other GPU files check on
small stand-ins: the 64-member uneven ensemble (batched, autotuned,
graph-replayed halo + advect, as the benchmark runs it; every output point of
every member against the oracle), and the 10-step
adjoint loop on 256 x 256 x 96 (FP32 and FP64 gradients against the oracle's
exact loop gradient, central differences at 16 random points, and the
dot-product test of the single-step adjoint)."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2009_12850_b300 import synthetic

from parity import TOL_F32_COND

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    from paper_2009_12850_b300 import build
    build.build()
    from paper_2009_12850_b300 import api
    return api


def test_ensemble_full_size_every_point(pw, tmp_path):
    oracle.set_threads(0)
    members = synthetic.ensemble(64)
    meshes, fields, sources = [], [], []
    for mb in members:
        m = pw.Mesh(mb.nx, mb.ny, mb.nz, mb.dx, mb.dx, dtype="f32")
        f = synthetic.wind_fields(mb.nx, mb.ny, mb.nz, mb.seed)
        meshes.append(m)
        fields.append([m.from_interior(a.astype(np.float32), fill_halo=False) for a in f])  # halos: the batch
        sources.append([m.empty_out() for _ in range(3)])
        del f
    b = pw.Batch(meshes)
    b.bind(fields, sources)
    b.autotune(os.path.join(tmp_path, "tune.txt"))
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        b.halo(stream=side)
        b.advect(stream=side)
    torch.cuda.current_stream().wait_stream(side)
    with torch.cuda.graph(graph):
        b.halo()
        b.advect()
    graph.replay()
    torch.cuda.synchronize()
    assert b.status() == 0
    for mb, m, s in zip(members, meshes, sources):
        # the member's fields again (seeded), as the kernel saw them: rounded to FP32
        fr = [a.astype(np.float32).astype(np.float64) for a in synthetic.wind_fields(mb.nx, mb.ny, mb.nz, mb.seed)]
        ref, cond = oracle.advect(oracle.Coeffs(mb.nz, mb.dx, mb.dx), *fr, want_cond=True)
        for q in range(3):
            got = m.interior(s[q]).double().cpu().numpy()
            err = np.abs(got - ref[q])
            assert np.all(err <= TOL_F32_COND * cond[q] + 1e-30), (m.nx, m.ny, m.nz, q, float(err.max()))


NX, NY, NZ, DT, STEPS = 256, 256, 96, 0.5, 10


@pytest.fixture(scope="module")
def loop_fields():
    f = synthetic.wind_fields(NX, NY, NZ, 602)
    return f


def test_adjoint_loop_full_size_gradients(pw, loop_fields):
    from paper_2009_12850_b300 import autograd as AG
    # one oracle loop on the FP64 fields serves both storages: rounding the
    # inputs to FP32 moves the gradient by ~1e-7 relative, far inside the FP32 bound
    c = oracle.Coeffs(NZ, 50.0, 50.0)
    Lref, gref = oracle.loss_and_grad(c, *loop_fields, DT, STEPS)
    for dtype, algo, tol in (("f32", "auto", 1e-5), ("f64", "native", 1e-10), ("f64", "split", 1e-10)):
        m = pw.Mesh(NX, NY, NZ, 50.0, dtype=dtype, algo=algo)
        U = [m.from_interior(a).requires_grad_(True) for a in loop_fields]
        L = AG.source_energy_loss(m, *U, dt=DT, steps=STEPS, checkpoint_every=2)
        L.backward()
        assert m.device_status() == 0
        assert abs(L.item() - Lref) <= tol * abs(Lref), (dtype, L.item(), Lref)
        for q in range(3):
            got = m.interior(U[q].grad).double().cpu().numpy()
            err = np.abs(got - gref[q]).max() / np.abs(gref[q]).max()
            assert err < tol, (dtype, q, err)
        del U, L, m
        torch.cuda.empty_cache()


def test_adjoint_loop_full_size_finite_differences(pw, loop_fields):
    """Central differences of the FP64 loop loss at 16 random points, h in {1e-3, 1e-4}."""
    from paper_2009_12850_b300 import autograd as AG
    m = pw.Mesh(NX, NY, NZ, 50.0, dtype="f64", algo="native")
    U = [m.from_interior(a).requires_grad_(True) for a in loop_fields]
    AG.source_energy_loss(m, *U, dt=DT, steps=STEPS).backward()
    base = [u.detach().clone() for u in U]
    rng = np.random.default_rng(603)

    def loss_at(q, i, j, k, h):
        X = [b.clone() for b in base]
        m.interior(X[q])[i, j, k] += h
        m.halo(X[q])
        with torch.no_grad():
            return AG.source_energy_loss(m, *X, dt=DT, steps=STEPS).item()

    for _ in range(16):
        q = int(rng.integers(0, 3))
        i, j = int(rng.integers(0, NX)), int(rng.integers(0, NY))
        k = int(rng.integers(0, NZ - 1 if q == 2 else NZ))
        gv = m.interior(U[q].grad)[i, j, k].item()
        errs = [abs((loss_at(q, i, j, k, h) - loss_at(q, i, j, k, -h)) / (2 * h) - gv) for h in (1e-3, 1e-4)]
        assert errs[1] <= 1e-6 * max(1.0, abs(gv)) or errs[1] < errs[0] / 20, (q, i, j, k, gv, errs)


def test_adjoint_dot_product_full_size(pw, loop_fields):
    """<J x, y> = <x, J^T y> for the single-step Jacobian at the 256 x 256 x 96
    state, FP64: S is quadratic, so J x = (S(u + x) - S(u - x)) / 2 exactly up
    to rounding."""
    m = pw.Mesh(NX, NY, NZ, 50.0, dtype="f64", algo="native")
    rng = np.random.default_rng(604)
    U = [m.from_interior(a) for a in loop_fields]
    xs = [rng.standard_normal((NX, NY, NZ)) for _ in range(3)]
    ys = [rng.standard_normal((NX, NY, NZ)) for _ in range(3)]
    xs[2][:, :, -1] = 0.0
    ys[2][:, :, -1] = 0.0
    Xp = [m.from_interior(a + b) for a, b in zip(loop_fields, xs)]
    Xm = [m.from_interior(a - b) for a, b in zip(loop_fields, xs)]
    Sp, Sm = m.advect(*Xp), m.advect(*Xm)
    Y = [m.from_interior(a, fill_halo=False) for a in ys]
    G = m.adjoint(*U, *Y)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    lhs = sum(float(((m.interior(a) - m.interior(b)) / 2 * torch.from_numpy(y).cuda()).sum())
              for a, b, y in zip(Sp, Sm, ys))
    rhs = sum(float((m.interior(g) * torch.from_numpy(x).cuda()).sum()) for g, x in zip(G, xs))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs)), (lhs, rhs)
