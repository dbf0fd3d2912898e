"""Stray-write detection without a sanitizer: every field and source lives
inside a larger device (or pinned host) buffer whose guard zones before and
after it hold a canary value.  After each operation the guard zones must be
intact, the operands it only reads must be unchanged bit for bit, and the
operands it writes must be unchanged outside the region it documents (the
interior points k < nz for sources; the halo columns for the halo fills).
Shapes are ragged (sizes not multiples of any tile or vector width, nz = 1 and
odd column lengths), so the tails of every kernel are exercised."""
import pytest
import torch

from paper_2009_12850_b300 import synthetic

pytestmark = pytest.mark.gpu

GUARD = 4096        # elements on each side (16-byte multiple for every dtype)
CANARY = -1280.0    # exactly representable in every storage type (bfloat16 included)

SHAPES = [(13, 7, 9), (5, 3, 1), (33, 17, 67), (1, 9, 6), (40, 24, 130)]
KINDS = [("f64", "split"), ("f64", "native"), ("f32", "auto"), ("bf16", "auto"), ("bf16_out", "auto")]


@pytest.fixture(scope="module")
def pw():
    from paper_2009_12850_b300 import build
    build.build()
    from paper_2009_12850_b300 import api
    return api


class Guarded:
    """A mesh-layout tensor inside a canary-filled buffer."""

    def __init__(self, m, dtype, pin_host=False):
        n = m.total
        if pin_host:
            self.buf = torch.full((n + 2 * GUARD,), CANARY, dtype=dtype).pin_memory()
        else:
            self.buf = torch.full((n + 2 * GUARD,), CANARY, dtype=dtype, device="cuda")
        self.t = self.buf[GUARD:GUARD + n].view(m.shape)

    def guards_intact(self):
        return bool((self.buf[:GUARD] == CANARY).all()) and bool((self.buf[-GUARD:] == CANARY).all())


def interior_mask(m, device="cuda"):
    mask = torch.zeros(m.shape, dtype=torch.bool, device=device)
    mask[2:m.nx + 2, 2:m.ny + 2, :m.nz] = True
    return mask


def fields(pw, m, seed, n=3, scalars=False):
    arrs = (synthetic.scalar_fields(m.nx, m.ny, m.nz, n, seed) if scalars
            else synthetic.wind_fields(m.nx, m.ny, m.nz, seed))
    out = []
    for a in arrs:
        g = Guarded(m, m.in_dtype)
        g.t.zero_()
        m.interior(g.t).copy_(torch.from_numpy(a).to(device="cuda", dtype=m.in_dtype))
        m.halo(g.t)
        out.append(g)
    return out


def snapshot(gs):
    return [g.t.clone() for g in gs]


def unchanged(gs, snaps):
    return all(g.guards_intact() and torch.equal(g.t, s) for g, s in zip(gs, snaps))


def sources(m, n=3):
    return [Guarded(m, m.out_dtype) for _ in range(n)]


def written_only_inside(m, gs):
    """Outside the interior the sources still hold the canary; guards intact."""
    mask = interior_mask(m)
    return all(g.guards_intact() and bool((g.t[~mask] == CANARY).all()) for g in gs)


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("dtype,algo", KINDS)
def test_advect_and_scalars_write_only_their_outputs(pw, shape, dtype, algo):
    m = pw.Mesh(*shape, 45.0, 35.0, dtype=dtype, algo=algo)
    U = fields(pw, m, 501)
    P = fields(pw, m, 502, n=2, scalars=True)
    su, sp = snapshot(U), snapshot(P)
    S = sources(m)
    m.advect(*(g.t for g in U), *(g.t for g in S))
    SP = sources(m, 2)
    m.advect_scalars(*(g.t for g in U), [g.t for g in P], [g.t for g in SP])
    torch.cuda.synchronize()
    assert m.device_status() == 0
    assert unchanged(U, su) and unchanged(P, sp)
    assert written_only_inside(m, S) and written_only_inside(m, SP)
    # accumulate mode reads and writes the same interior only
    m.advect(*(g.t for g in U), *(g.t for g in S), beta=1)
    torch.cuda.synchronize()
    assert unchanged(U, su) and written_only_inside(m, S)


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "bf16_out"])
def test_tvd_writes_only_its_outputs(pw, shape, dtype):
    m = pw.Mesh(*shape, 45.0, 35.0, dtype=dtype)
    U = fields(pw, m, 511)
    P = fields(pw, m, 512, n=3, scalars=True)
    su, sp = snapshot(U), snapshot(P)
    SP = sources(m, 3)
    for beta in (0, 1):
        m.advect_tvd(*(g.t for g in U), [g.t for g in P], 4.0, [g.t for g in SP], beta=beta)
        torch.cuda.synchronize()
        assert m.device_status() == 0
        assert unchanged(U, su) and unchanged(P, sp)
        assert written_only_inside(m, SP)


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("dtype,algo", KINDS)
def test_fused_steps_stay_in_their_fields(pw, shape, dtype, algo):
    m = pw.Mesh(*shape, 45.0, 35.0, dtype=dtype, algo=algo)
    U = fields(pw, m, 503)
    P = fields(pw, m, 504, n=2, scalars=True)
    su, sp = snapshot(U), snapshot(P)
    N = [Guarded(m, m.in_dtype) for _ in range(3)]
    NP = [Guarded(m, m.in_dtype) for _ in range(2)]
    m.step(*(g.t for g in U), *(g.t for g in N), dt=0.3)
    m.step_scalars(*(g.t for g in U), [g.t for g in P], [g.t for g in NP], dt=0.3)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    assert unchanged(U, su) and unchanged(P, sp)
    # the new state covers interior and halo columns of k < nz; padding levels keep the canary
    pad = torch.zeros(m.shape, dtype=torch.bool, device="cuda")
    pad[:, :, m.nz:] = True
    for g in N + NP:
        assert g.guards_intact()
        assert bool((g.t[pad] == CANARY).all())
        assert bool(torch.isfinite(g.t[~pad].float()).all())


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("dtype,algo", [("f64", "native"), ("f64", "split"), ("f32", "auto")])
def test_adjoint_euler_and_sums_stay_in_their_fields(pw, shape, dtype, algo):
    m = pw.Mesh(*shape, 45.0, 35.0, dtype=dtype, algo=algo)
    U = fields(pw, m, 505)
    Y = fields(pw, m, 506)
    su, sy = snapshot(U), snapshot(Y)
    G = [Guarded(m, m.in_dtype) for _ in range(3)]
    m.adjoint(*(g.t for g in U), *(g.t for g in Y), *(g.t for g in G))
    torch.cuda.synchronize()
    assert m.device_status() == 0
    assert unchanged(U, su)
    # gsu, gsv, gsw: only their halo columns are rewritten with periodic copies,
    # which they already held, so they are unchanged
    assert unchanged(Y, sy)
    assert written_only_inside(m, G)
    # conservation sums read only
    S = sources(m)
    m.advect(*(g.t for g in U), *(g.t for g in S))
    ss = snapshot(S)
    m.residual_sums(*(g.t for g in U), *(g.t for g in S))
    torch.cuda.synchronize()
    assert unchanged(U, su) and unchanged(S, ss)
    # Euler update: interior plus halo images of the fields, sources read only
    m.euler(*(g.t for g in U), *(g.t for g in S), 0.2)
    torch.cuda.synchronize()
    assert unchanged(S, ss)
    pad = torch.zeros(m.shape, dtype=torch.bool, device="cuda")
    pad[:, :, m.nz:] = True
    for g, s in zip(U, su):
        assert g.guards_intact()
        assert torch.equal(g.t[pad], s[pad])


def test_batched_members_stay_in_their_fields(pw):
    members = [(13, 7, 67), (40, 24, 130), (5, 3, 64), (33, 17, 70)]
    meshes = [pw.Mesh(*s, 40.0, dtype="f32") for s in members]
    U = [fields(pw, m, 507 + q) for q, m in enumerate(meshes)]
    su = [snapshot(f) for f in U]
    S = [sources(m) for m in meshes]
    b = pw.Batch(meshes)
    b.bind([[g.t for g in f] for f in U], [[g.t for g in s] for s in S])
    b.halo()
    b.advect()
    torch.cuda.synchronize()
    assert b.status() == 0
    for m, f, s0, s in zip(meshes, U, su, S):
        assert unchanged(f, s0)     # the halo fill rewrites halos with the same periodic copies
        assert written_only_inside(m, s)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16_out"])
def test_host_pipeline_stays_in_its_arrays(pw, dtype):
    nx, ny, nz = 29, 11, 13
    m = pw.Mesh(nx, ny, nz, 45.0, dtype=dtype)
    pipe = pw.Pipeline(m, 6)
    pipe.reserve_scalars(1)
    arrs = list(synthetic.wind_fields(nx, ny, nz, 510)) + list(synthetic.scalar_fields(nx, ny, nz, 1, 511))
    H = []
    for a in arrs:
        g = Guarded(m, m.in_dtype, pin_host=True)
        g.t.zero_()
        g.t[2:nx + 2, 2:ny + 2, :nz] = torch.from_numpy(a).to(m.in_dtype)
        H.append(g)
    sh = [g.t.clone() for g in H]
    O = [Guarded(m, m.out_dtype, pin_host=True) for _ in range(4)]
    pipe.advect_host(*(g.t for g in H[:3]), *(g.t for g in O[:3]), scalars=[H[3].t], sources=[O[3].t])
    pipe.sync()
    assert m.device_status() == 0
    assert all(g.guards_intact() and torch.equal(g.t, s) for g, s in zip(H, sh))
    mask = interior_mask(m, device="cpu")
    for g in O:
        assert g.guards_intact()
        assert bool((g.t[~mask] == CANARY).all())
        assert bool(torch.isfinite(g.t[mask].float()).all())
