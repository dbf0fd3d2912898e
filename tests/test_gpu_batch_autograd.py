"""GPU tests of the batched persistent stencil and autotuner (A6) and of the
differentiable path (A7): autograd through the adjoint kernels, the
checkpointed Euler loop against the oracle, and finite differences."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2009_12850_b300 import synthetic

from parity import TOL_F32_COND, compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    from paper_2009_12850_b300 import build
    build.build()
    from paper_2009_12850_b300 import api
    return api


def small_ensemble(n=7, seed=5):
    rng = np.random.default_rng(seed)
    out = []
    for q in range(n):
        nx, ny = int(rng.integers(3, 40)), int(rng.integers(2, 45))
        nz = int(rng.choice([1, 2, 7, 13, 40, 64, 70, 130]))
        out.append((nx, ny, nz, float(rng.uniform(25, 100)), 100 + q))
    return out


def build_batch(pw, members):
    meshes, fields, sources, host = [], [], [], []
    for nx, ny, nz, dx, seed in members:
        m = pw.Mesh(nx, ny, nz, dx, dtype="f32")
        f = synthetic.wind_fields(nx, ny, nz, seed)
        meshes.append(m)
        fields.append([m.from_interior(a) for a in f])
        sources.append([m.empty_out() for _ in range(3)])
        host.append(f)
    b = pw.Batch(meshes)
    b.bind(fields, sources)
    return b, meshes, fields, sources, host


def test_batched_matches_single_and_oracle(pw):
    members = small_ensemble()
    b, meshes, fields, sources, host = build_batch(pw, members)
    b.advect()
    torch.cuda.synchronize()
    assert b.status() == 0
    for (nx, ny, nz, dx, _), m, f, s, h in zip(members, meshes, fields, sources, host):
        single = m.advect(*f)
        for q in range(3):
            a = m.interior(s[q]).cpu().numpy()
            assert np.array_equal(a, m.interior(single[q]).cpu().numpy())
        c = oracle.Coeffs(nz, dx, dx)
        fr = [torch.from_numpy(x).float().double().numpy() for x in h]
        ref, cond = oracle.advect(c, *fr, want_cond=True)
        for q in range(3):
            compare("batched", m.interior(s[q]).double().cpu().numpy(), ref[q], cond[q], 1e-5, TOL_F32_COND)


def test_batched_halo(pw):
    members = small_ensemble(5, seed=8)
    b, meshes, fields, sources, host = build_batch(pw, members)
    want = []
    for m, f in zip(meshes, fields):
        want.append([t.clone() for t in f])
        for t in f:   # scramble the halos
            t[:2].fill_(1e9)
            t[:, -2:].fill_(-1e9)
    b.halo()
    torch.cuda.synchronize()
    for m, f, w in zip(meshes, fields, want):
        for t, x in zip(f, w):
            assert torch.equal(t[:, :, :m.nz], x[:, :, :m.nz])


def test_batched_autotune_cache_and_graph(pw, tmp_path):
    members = small_ensemble(6, seed=11)
    b, meshes, fields, sources, host = build_batch(pw, members)
    b.advect()
    torch.cuda.synchronize()
    ref = [[m.interior(t).clone() for t in s] for m, s in zip(meshes, sources)]
    cache = str(tmp_path / "tune.txt")
    ms = b.autotune(cache)
    assert ms > 0
    assert "batch n=6" in open(cache).read()
    assert b.autotune(cache) == -1.0      # second call reads the cache
    for s in sources:
        for t in s:
            t.zero_()
    # capture halo + advect in a CUDA graph and replay it twice
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        b.halo(stream=stream)
        b.advect(stream=stream)
    torch.cuda.current_stream().wait_stream(stream)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.halo()
        b.advect()
    for s in sources:
        for t in s:
            t.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for m, s, r in zip(meshes, sources, ref):
        for t, x in zip(s, r):
            assert torch.equal(m.interior(t), x)


def test_mesh_autotune(pw, tmp_path):
    for dtype, algo in (("f32", "auto"), ("f64", "split"), ("f64", "native")):
        m = pw.Mesh(48, 40, 33, 50.0, dtype=dtype, algo=algo)
        f = [m.from_interior(a) for a in synthetic.wind_fields(48, 40, 33, 3)]
        s0 = [t.clone() for t in m.advect(*f)]
        S = [m.empty_out() for _ in range(3)]
        cache = str(tmp_path / "t.txt")
        assert m.autotune(*f, *S, cache_path=cache) > 0
        tile = m.get_tile()
        m.set_tile(4, 3)
        assert m.autotune(*f, *S, cache_path=cache) == -1.0 and m.get_tile() == tile
        s1 = m.advect(*f)
        for a, b in zip(s0, s1):
            assert torch.equal(m.interior(a), m.interior(b))


# ---------------------------------------------------------------- autograd
def test_autograd_advect_matches_oracle_adjoint(pw):
    from paper_2009_12850_b300 import autograd as AG
    nx, ny, nz = 12, 10, 9
    m = pw.Mesh(nx, ny, nz, 50.0, dtype="f64", algo="native")
    f = synthetic.wind_fields(nx, ny, nz, 6)
    U = [m.from_interior(a).requires_grad_(True) for a in f]
    rng = np.random.default_rng(3)
    y = [rng.standard_normal((nx, ny, nz)) for _ in range(3)]
    y[2][:, :, -1] = 0.0
    S = AG.advect(m, *U)
    L = sum((m.interior(s) * torch.from_numpy(yy).cuda()).sum() for s, yy in zip(S, y))
    L.backward()
    c = oracle.Coeffs(nz, 50.0, 50.0)
    ref = oracle.adjoint(c, *f, *y)
    for q in range(3):
        g = U[q].grad
        np.testing.assert_allclose(m.interior(g).cpu().numpy(), ref[q], rtol=1e-11, atol=1e-12)
        h = g.cpu().numpy()
        assert not h[:2].any() and not h[-2:].any() and not h[:, :2].any() and not h[:, -2:].any()


@pytest.mark.parametrize("dtype,algo", [("f64", "native"), ("f64", "split")])
def test_checkpointed_loop_gradient_matches_oracle(pw, dtype, algo):
    from paper_2009_12850_b300 import autograd as AG
    nx, ny, nz, dt, steps = 16, 12, 10, 0.5, 10
    m = pw.Mesh(nx, ny, nz, 50.0, dtype=dtype, algo=algo)
    f = synthetic.wind_fields(nx, ny, nz, 7)
    U = [m.from_interior(a).requires_grad_(True) for a in f]
    L = AG.source_energy_loss(m, *U, dt=dt, steps=steps, checkpoint_every=2)
    L.backward()
    c = oracle.Coeffs(nz, 50.0, 50.0)
    Lref, gref = oracle.loss_and_grad(c, *f, dt, steps)
    assert abs(L.item() - Lref) <= 1e-11 * abs(Lref)
    for q in range(3):
        got = m.interior(U[q].grad).cpu().numpy()
        err = np.abs(got - gref[q]).max() / np.abs(gref[q]).max()
        assert err < 1e-10, (q, err)


def test_checkpoint_segments_do_not_change_gradient(pw):
    from paper_2009_12850_b300 import autograd as AG
    nx, ny, nz = 10, 9, 8
    m = pw.Mesh(nx, ny, nz, 50.0, dtype="f64", algo="native")
    f = synthetic.wind_fields(nx, ny, nz, 9)
    grads = []
    for every in (1, 2, 3, 10):
        U = [m.from_interior(a).requires_grad_(True) for a in f]
        AG.source_energy_loss(m, *U, dt=0.5, steps=10, checkpoint_every=every).backward()
        grads.append([u.grad.clone() for u in U])
    for g in grads[1:]:
        for a, b in zip(grads[0], g):
            assert torch.allclose(a, b, rtol=1e-13, atol=1e-15)


def test_loop_gradient_finite_differences(pw):
    """Central differences at 16 random points with h in {1e-3, 1e-4} (FP64)."""
    from paper_2009_12850_b300 import autograd as AG
    nx, ny, nz, dt, steps = 14, 12, 10, 0.5, 10
    m = pw.Mesh(nx, ny, nz, 50.0, dtype="f64", algo="native")
    f = synthetic.wind_fields(nx, ny, nz, 10)
    U = [m.from_interior(a).requires_grad_(True) for a in f]
    AG.source_energy_loss(m, *U, dt=dt, steps=steps).backward()
    rng = np.random.default_rng(12)

    def loss(fields):
        with torch.no_grad():
            X = [m.from_interior(a) for a in fields]
            return AG.source_energy_loss(m, *X, dt=dt, steps=steps).item()

    for _ in range(16):
        q = int(rng.integers(0, 3))
        i, j = int(rng.integers(0, nx)), int(rng.integers(0, ny))
        k = int(rng.integers(0, nz - 1 if q == 2 else nz))
        gv = m.interior(U[q].grad)[i, j, k].item()
        errs = []
        for h in (1e-3, 1e-4):
            fp = [a.copy() for a in f]
            fm = [a.copy() for a in f]
            fp[q][i, j, k] += h
            fm[q][i, j, k] -= h
            errs.append(abs((loss(fp) - loss(fm)) / (2 * h) - gv))
        assert errs[1] <= 1e-6 * max(1.0, abs(gv)) or errs[1] < errs[0] / 20, (q, i, j, k, gv, errs)


def test_fp32_loop_gradient_vs_fp64(pw):
    from paper_2009_12850_b300 import autograd as AG
    nx, ny, nz = 24, 20, 16
    f = synthetic.wind_fields(nx, ny, nz, 13)
    out = {}
    for dtype in ("f32", "f64"):
        m = pw.Mesh(nx, ny, nz, 50.0, dtype=dtype, algo="native")
        U = [m.from_interior(a).requires_grad_(True) for a in f]
        AG.source_energy_loss(m, *U, dt=0.5, steps=10).backward()
        out[dtype] = [m.interior(u.grad).double().cpu().numpy() for u in U]
    for a, b in zip(out["f32"], out["f64"]):
        assert np.abs(a - b).max() / np.abs(b).max() < 1e-4


def test_batch_reorder_keeps_halo_and_stencil_consistent(pw):
    """Changing the CTA size changes the members' tile shapes and hence their
    work order; the halo fill and the stencil must follow the new order, under
    either tile schedule."""
    members = [(24, 40, 160, 30.0, 1), (56, 16, 64, 60.0, 2), (40, 40, 97, 45.0, 3),
               (16, 72, 130, 80.0, 4), (48, 24, 70, 25.0, 5), (8, 8, 150, 99.0, 6)]
    b, meshes, fields, sources, host = build_batch(pw, members)
    want = [[m.interior(s).clone() for s in m.advect(*f)] for m, f in zip(meshes, fields)]
    halos = [[t.clone() for t in f] for f in fields]
    for persistent, threads, tile_i in ((1, 128, 16), (1, 512, 64), (0, 256, 8), (0, 384, 32), (0, 96, 64),
                                        (1, 224, 128)):
        b.set_schedule(persistent)
        b.set_tile(threads, tile_i)
        for f in fields:
            for t in f:
                t[:2].fill_(1e9)
                t[:, -2:].fill_(-1e9)
        b.halo()
        for s in sources:
            for t in s:
                t.zero_()
        b.advect()
        torch.cuda.synchronize()
        assert b.status() == 0
        for m, f, h, s, w in zip(meshes, fields, halos, sources, want):
            for t, x in zip(f, h):
                assert torch.equal(t[:, :, :m.nz], x[:, :, :m.nz]), (persistent, threads, tile_i)
            for t, x in zip(s, w):
                assert torch.equal(m.interior(t), x), (persistent, threads, tile_i)
