"""Pins of the FP64 CPU oracle against what the scheme and the mathematics fix
(no GPU): hand-evaluated worked examples, closed-form coefficients, exact
invariants of the Piacsek-Williams form (uniform flow, energy conservation,
skew-adjointness, the momentum / divergence identity), second-order convergence
to the continuous skew-symmetric tendency, and the adjoint by dot-product and
brute-force tests.  A final test plants plausible mistakes in copies of the
oracle source and checks that these pins catch every one.
"""
import json
import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_2009_12850_b300 import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def unit_coeffs(nz=4):
    return oracle.Coeffs(nz, 1.0, 1.0, dz=np.ones(nz), rho_n=np.ones(nz), rho_w=np.ones(nz), rho0=1.0)


def grid_idx(n=4):
    return np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")


def rand_fields(rng, nx, ny, nz, lid=True):
    u = 5 + rng.standard_normal((nx, ny, nz))
    v = 5 + rng.standard_normal((nx, ny, nz))
    w = 0.3 * rng.standard_normal((nx, ny, nz))
    if lid:
        w[:, :, -1] = 0.0
    return u, v, w


def stretched(nz, dx=37.0, dy=53.0):
    return oracle.Coeffs(nz, dx, dy)


def wdot(c, a, b, grid):
    wuv, ww = oracle.weights(c)
    W = wuv if grid < 2 else ww
    return float(np.sum(W[None, None, :] * a * b))


# --------------------------------------------------------------------------
# pins (each returns normally or raises AssertionError)
# --------------------------------------------------------------------------
def pin_worked_examples():
    spec = json.load(open(os.path.join(GOLDEN, "pw_worked_examples.json")))
    c = unit_coeffs()
    I, J, K = grid_idx()
    z = np.zeros((4, 4, 4))
    ex = {e["name"]: e["expect"] for e in spec["examples"]}
    # E1
    su, sv, sw = oracle.advect(c, 1.0 + I, z, z)
    np.testing.assert_array_equal(su, np.broadcast_to(np.array(ex["E1"]["su_i"])[:, None, None], su.shape))
    assert not sv.any() and not sw.any()
    # E2
    w = np.broadcast_to(np.array([1.0, 2.0, 1.0, 0.0]), (4, 4, 4)).copy()
    su, sv, sw = oracle.advect(c, 1.0 + K, z, w)
    np.testing.assert_array_equal(su, np.broadcast_to(np.array(ex["E2"]["su_k"]), su.shape))
    np.testing.assert_array_equal(sw, np.broadcast_to(np.array(ex["E2"]["sw_k"]), sw.shape))
    assert not sv.any()
    # E3
    su, sv, sw = oracle.advect(c, 2.0 + 0 * I, 1.0 + I, z)
    np.testing.assert_array_equal(sv, np.broadcast_to(np.array(ex["E3"]["sv_i"])[:, None, None], sv.shape))
    assert not su.any() and not sw.any()
    # E4
    w = np.zeros((4, 4, 4))
    w[:, :, 0] = (1.0 + I)[:, :, 0]
    su, sv, sw = oracle.advect(c, 1.0 + K, z, w)
    np.testing.assert_array_equal(sw, np.broadcast_to(np.array(ex["E4"]["sw_ik"])[:, None, :], sw.shape))
    np.testing.assert_array_equal(su, np.broadcast_to(np.array(ex["E4"]["su_ik"])[:, None, :], su.shape))
    assert not sv.any()
    # E5
    su, sv, sw = oracle.advect(c, 1.0 + J, 1.0 + I, z)
    np.testing.assert_array_equal(su, np.broadcast_to(np.array(ex["E5"]["su_ij"])[:, :, None], su.shape))
    np.testing.assert_array_equal(sv, np.broadcast_to(np.array(ex["E5"]["sv_ij"])[:, :, None], sv.shape))
    assert not sw.any()


def pin_coefficients():
    spec = json.load(open(os.path.join(GOLDEN, "pw_coefficients_nz3.json")))
    c = oracle.Coeffs(3, 50.0, 50.0)
    np.testing.assert_allclose(c.dz, spec["dz"], rtol=1e-15)
    np.testing.assert_allclose(c.zf, spec["zf"], rtol=1e-15)
    np.testing.assert_allclose(c.zn, spec["zn"], rtol=1e-15)
    np.testing.assert_allclose(c.dzn[:2], spec["dzn"], rtol=1e-15)
    for name in ("tzc1", "tzc2", "tzd1", "tzd2"):
        want = np.array([a * math.exp(e / 8000.0) for a, e in spec[name]])
        np.testing.assert_allclose(getattr(c, name), want, rtol=2e-15, atol=0, err_msg=name)
    assert c.tcx == 0.25 / 50.0 and c.tcy == 0.25 / 50.0


def pin_uniform_flow():
    rng = np.random.default_rng(5)
    nz = 9
    c = oracle.Coeffs(nz, 31.0, 17.0, dz=rng.uniform(5, 50, nz), rho_n=rng.uniform(0.5, 1.5, nz),
                      rho_w=rng.uniform(0.5, 1.5, nz))
    U = np.full((6, 5, nz), 7.25)
    V = np.full((6, 5, nz), -3.5)
    W = np.zeros((6, 5, nz))
    for s in oracle.advect(c, U, V, W):
        assert not s.any()


def pin_energy():
    rng = np.random.default_rng(6)
    for nx, ny, nz in ((7, 5, 6), (4, 9, 2), (3, 3, 1)):
        c = stretched(nz)
        u, v, w = rand_fields(rng, nx, ny, nz)
        (su, sv, sw), _ = oracle.advect(c, u, v, w, want_cond=True)
        for g, (phi, s) in enumerate(((u, su), (v, sv), (w, sw))):
            num = wdot(c, phi, s, g)
            den = wdot(c, np.abs(phi), np.abs(s), g)
            assert abs(num) <= 1e-14 * den + 1e-300, (g, num, den)


def pin_skew_adjoint():
    rng = np.random.default_rng(7)
    nx, ny, nz = 6, 5, 7
    c = stretched(nz)
    a = rand_fields(rng, nx, ny, nz)
    for g in range(3):
        phi = rng.standard_normal((nx, ny, nz))
        psi = rng.standard_normal((nx, ny, nz))
        if g == 2:
            phi[:, :, -1] = 0.0
            psi[:, :, -1] = 0.0
        lhs = wdot(c, psi, oracle.src(c, g, *a, phi), g)
        rhs = -wdot(c, oracle.src(c, g, *a, psi), phi, g)
        scale = wdot(c, np.abs(psi), np.abs(oracle.src(c, g, *a, phi)), g)
        assert abs(lhs - rhs) <= 1e-13 * scale, (g, lhs, rhs)


def streamfunction_flow(rng, nx, ny, nz, dx, dy):
    """w = 0 and (u, v) = (-d psi/dy, d psi/dx) from a corner streamfunction:
    psi[i, j] sits at (x_{i+1/2}, y_{j+1/2}); discretely divergence-free."""
    psi = rng.standard_normal((nx, ny, nz))
    u = -(psi - np.roll(psi, 1, axis=1)) / dy
    v = (psi - np.roll(psi, 1, axis=0)) / dx
    return 5 + u, 3 + v, np.zeros((nx, ny, nz))


def pin_momentum_divergence_free():
    rng = np.random.default_rng(8)
    nx, ny, nz, dx, dy = 8, 6, 5, 40.0, 60.0
    c = stretched(nz, dx, dy)
    u, v, w = streamfunction_flow(rng, nx, ny, nz, dx, dy)
    # the flow really is divergence-free at every cell centre
    div = (u - np.roll(u, 1, axis=0)) / dx + (v - np.roll(v, 1, axis=1)) / dy
    assert np.abs(div).max() < 1e-13
    su, sv, sw = oracle.advect(c, u, v, w)
    assert not sw.any()
    for g, s in ((0, su), (1, sv)):
        tot = wdot(c, np.ones_like(s), s, g)
        assert abs(tot) <= 1e-14 * wdot(c, np.ones_like(s), np.abs(s), g), (g, tot)


def pin_momentum_identity():
    rng = np.random.default_rng(9)
    nx, ny, nz = 7, 6, 8
    c = stretched(nz)
    u, v, w = rand_fields(rng, nx, ny, nz)
    s = oracle.advect(c, u, v, w)
    for g, phi in enumerate((u, v, w)):
        D = oracle.face_divergence(c, g, u, v, w)
        lhs = wdot(c, np.ones_like(phi), s[g], g)
        rhs = wdot(c, phi, D, g)
        scale = wdot(c, np.ones_like(phi), np.abs(s[g]), g)
        assert abs(lhs - rhs) <= 1e-13 * scale, (g, lhs, rhs)
        assert abs(lhs) > 1e-6 * scale  # arbitrary fields: the integral does not vanish


def continuum_fields(H):
    import sympy as sp
    x, y, z = sp.symbols("x y z", real=True)
    Lx, Ly, Z = 2000.0, 1600.0, 1000.0
    kx, ky = 2 * sp.pi / Lx, 2 * sp.pi / Ly
    u = 3 + sp.sin(kx * x + 0.4) * sp.cos(ky * y) * (1 + 0.3 * sp.cos(sp.pi * z / Z))
    v = 2 + sp.cos(kx * x) * sp.sin(ky * y + 0.7) * (1 + 0.2 * z / Z)
    w = 0.5 * sp.sin(sp.pi * z / Z) * sp.cos(kx * x + 0.1) * sp.sin(ky * y + 0.2)
    rho = 1.2 * sp.exp(-z / H)
    div = (sp.diff(rho * u, x) + sp.diff(rho * v, y) + sp.diff(rho * w, z)) / rho
    out = []
    for phi in (u, v, w):
        S = -(u * sp.diff(phi, x) + v * sp.diff(phi, y) + w * sp.diff(phi, z)) - phi * div / 2
        out.append(sp.lambdify((x, y, z), S, "numpy"))
    fl = [sp.lambdify((x, y, z), f, "numpy") for f in (u, v, w)]
    return fl, out, (Lx, Ly, Z)


def pin_continuum_second_order():
    H = 1500.0
    fl, Sl, (Lx, Ly, Z) = continuum_fields(H)
    errs = []
    for N in (12, 24, 48):
        nx = ny = nz = N
        dx, dy, dz = Lx / nx, Ly / ny, Z / nz
        c = oracle.Coeffs(nz, dx, dy, dz=np.full(nz, dz), rho0=1.2, H=H)
        i = np.arange(nx)[:, None, None]
        j = np.arange(ny)[None, :, None]
        zn = ((np.arange(nz) + 0.5) * dz)[None, None, :]
        zf = ((np.arange(nz) + 1.0) * dz)[None, None, :]
        pts = [((i + 0.5) * dx, j * dy, zn), (i * dx, (j + 0.5) * dy, zn), (i * dx, j * dy, zf)]
        F = [np.broadcast_to(fl[q](*pts[q]), (nx, ny, nz)).astype(np.float64).copy() for q in range(3)]
        F[2][:, :, -1] = 0.0
        S = oracle.advect(c, *F)
        e = 0.0
        for q in range(3):
            ref = np.broadcast_to(Sl[q](*pts[q]), (nx, ny, nz))
            mask = np.ones((nx, ny, nz), bool)
            if q == 2:
                mask[:, :, -1] = False
            e = max(e, float(np.abs(S[q] - ref)[mask].max() / np.abs(ref).max()))
        errs.append(e)
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.8 and 3.3 < r2 < 4.8, errs


def jvp(c, x, e):
    """J(x) e by central difference; exact (up to rounding) since S is quadratic."""
    p = oracle.advect(c, *(x[q] + e[q] for q in range(3)))
    m = oracle.advect(c, *(x[q] - e[q] for q in range(3)))
    return tuple((p[q] - m[q]) / 2 for q in range(3))


def pin_adjoint_dot():
    rng = np.random.default_rng(10)
    nx, ny, nz = 6, 7, 6
    c = stretched(nz)
    x = rand_fields(rng, nx, ny, nz)
    e = list(rand_fields(rng, nx, ny, nz))
    y = [rng.standard_normal((nx, ny, nz)) for _ in range(3)]
    Je = jvp(c, x, e)
    JTy = oracle.adjoint(c, *x, *y)
    lhs = sum(float(np.sum(Je[q] * y[q])) for q in range(3))
    rhs = sum(float(np.sum(e[q] * JTy[q])) for q in range(3))
    scale = sum(float(np.sum(np.abs(Je[q] * y[q]))) for q in range(3))
    assert abs(lhs - rhs) <= 1e-13 * scale, (lhs, rhs)
    # the lid face is not a degree of freedom
    assert not JTy[2][:, :, -1].any()


def pin_adjoint_bruteforce():
    rng = np.random.default_rng(11)
    nx, ny, nz = 3, 4, 4
    c = stretched(nz)
    x = rand_fields(rng, nx, ny, nz)
    y = [rng.standard_normal((nx, ny, nz)) for _ in range(3)]
    JTy = oracle.adjoint(c, *x, *y)
    n = nx * ny * nz
    for q in range(3):
        col = np.zeros(n)
        for m in range(n):
            e = [np.zeros((nx, ny, nz)) for _ in range(3)]
            e[q].reshape(-1)[m] = 1.0
            if q == 2 and m % nz == nz - 1:
                col[m] = 0.0          # lid value is never read
                continue
            Je = jvp(c, x, e)
            col[m] = sum(float(np.sum(Je[r] * y[r])) for r in range(3))
        np.testing.assert_allclose(JTy[q].reshape(-1), col, rtol=1e-12, atol=1e-12)


def pin_loop_gradient():
    rng = np.random.default_rng(12)
    nx, ny, nz, dt, steps = 5, 4, 5, 0.5, 4
    c = stretched(nz, 50.0, 50.0)
    x = rand_fields(rng, nx, ny, nz)
    L, g = oracle.loss_and_grad(c, *x, dt, steps)
    for trial in range(8):
        q = int(rng.integers(0, 3))
        i, j = int(rng.integers(0, nx)), int(rng.integers(0, ny))
        k = int(rng.integers(0, nz - 1 if q == 2 else nz))
        fd = []
        for h in (1e-3, 1e-4):
            xp = [a.copy() for a in x]
            xm = [a.copy() for a in x]
            xp[q][i, j, k] += h
            xm[q][i, j, k] -= h
            Lp, _ = oracle.loss_and_grad(c, *xp, dt, steps)
            Lm, _ = oracle.loss_and_grad(c, *xm, dt, steps)
            fd.append((Lp - Lm) / (2 * h))
        gv = g[q][i, j, k]
        e1, e2 = abs(fd[0] - gv), abs(fd[1] - gv)
        tol = 1e-7 * max(1.0, abs(gv))
        assert e2 <= tol or e2 < e1 / 20, (q, i, j, k, gv, fd)


def pin_cond_and_points():
    rng = np.random.default_rng(13)
    nx, ny, nz = 5, 6, 7
    c = stretched(nz)
    u, v, w = rand_fields(rng, nx, ny, nz)
    (su, sv, sw), (cu, cv, cw) = oracle.advect(c, u, v, w, want_cond=True)
    for s, cc in ((su, cu), (sv, cv), (sw, cw)):
        assert np.all(np.abs(s) <= cc * (1 + 1e-15))
    pts = np.array([[0, 0, 0], [4, 5, 6], [2, 3, 0], [1, 0, 6], [3, 2, 5]])
    vals, cond = oracle.advect_points(c, u, v, w, pts)
    for p, (i, j, k) in enumerate(pts):
        assert vals[p, 0] == su[i, j, k] and vals[p, 1] == sv[i, j, k] and vals[p, 2] == sw[i, j, k]
        assert cond[p, 0] == cu[i, j, k] and cond[p, 2] == cw[i, j, k]


def pin_lid_ignored():
    """The lid face w(nz-1) is 0 by definition: whatever is stored there must not
    change any source or gradient."""
    rng = np.random.default_rng(15)
    nx, ny, nz = 5, 4, 6
    c = stretched(nz)
    u, v, w = rand_fields(rng, nx, ny, nz)
    w2 = w.copy()
    w2[:, :, -1] = 100.0 * rng.standard_normal((nx, ny))
    for a, b in zip(oracle.advect(c, u, v, w), oracle.advect(c, u, v, w2)):
        assert np.array_equal(a, b)
    y = [rng.standard_normal((nx, ny, nz)) for _ in range(3)]
    for a, b in zip(oracle.adjoint(c, u, v, w, *y), oracle.adjoint(c, u, v, w2, *y)):
        assert np.array_equal(a, b)


# --------------------------------------------------------------------------
# scalars (theta, q): the cell-centred form
# --------------------------------------------------------------------------
def pin_scalar_worked_examples():
    spec = json.load(open(os.path.join(GOLDEN, "pw_scalar_worked_examples.json")))
    ex = {e["name"]: e["expect"] for e in spec["examples"]}
    c = unit_coeffs()
    I, J, K = grid_idx()
    z = np.zeros((4, 4, 4))
    s = oracle.advect_scalar(c, 1.0 + z, z, z, 1.0 * I)
    np.testing.assert_array_equal(s, np.broadcast_to(np.array(ex["S1"]["s_i"])[:, None, None], s.shape))
    w = np.broadcast_to(np.array([1.0, 2.0, 1.0, 0.0]), (4, 4, 4)).copy()
    s = oracle.advect_scalar(c, z, z, w, 1.0 * K)
    np.testing.assert_array_equal(s, np.broadcast_to(np.array(ex["S2"]["s_k"]), s.shape))
    s = oracle.advect_scalar(c, z, 1.0 + J, z, 1.0 + z)
    np.testing.assert_array_equal(s, np.broadcast_to(np.array(ex["S3"]["s_j"])[None, :, None], s.shape))
    s = oracle.advect_scalar(c, 1.0 + J, 2.0 + z, z, 1.0 * (I + J))
    np.testing.assert_array_equal(s, np.broadcast_to(np.array(ex["S4"]["s_ij"])[:, :, None], s.shape))
    # stretched, stratified column: a unit spike of phi at level k0 under w = 1
    # gives hz1(k0+1) one level up and -hz2(k0-1) one level down
    co = spec["coefficients_nz3"]
    c3 = oracle.Coeffs(3, co["dx"], co["dx"])
    hz1 = [a * math.exp(e / 8000.0) for a, e in co["hz1"]]
    hz2 = [a * math.exp(e / 8000.0) for a, e in co["hz2"]]
    assert c3.hx == co["hx"] and c3.hy == co["hx"]
    np.testing.assert_allclose(c3.hz1, hz1, rtol=2e-15, atol=0)
    np.testing.assert_allclose(c3.hz2, hz2, rtol=2e-15, atol=0)
    one = np.ones((3, 3, 3))
    w = one.copy()
    w[:, :, -1] = 0.0
    for k0 in range(3):
        phi = np.zeros((3, 3, 3))
        phi[:, :, k0] = 1.0
        s = oracle.advect_scalar(c3, 0 * one, 0 * one, w, phi)
        col = s[1, 2]
        if k0 + 1 < 3:
            assert abs(col[k0 + 1] - hz1[k0 + 1]) <= 2e-15 * hz1[k0 + 1], (k0, col)
        if k0 >= 1:
            assert abs(col[k0 - 1] + hz2[k0 - 1]) <= 2e-15 * hz2[k0 - 1], (k0, col)
        assert col[k0] == 0.0


def pin_scalar_uniform_and_centred():
    rng = np.random.default_rng(21)
    nx, ny, nz, dx, dy = 6, 5, 7, 31.0, 17.0
    c = oracle.Coeffs(nz, dx, dy, dz=rng.uniform(5, 50, nz), rho_n=rng.uniform(0.5, 1.5, nz),
                      rho_w=rng.uniform(0.5, 1.5, nz))
    U, V, W = np.full((nx, ny, nz), 7.25), np.full((nx, ny, nz), -3.5), np.zeros((nx, ny, nz))
    assert not oracle.advect_scalar(c, U, V, W, np.full((nx, ny, nz), 2.5)).any()
    # constant horizontal wind: minus the centred advective derivative
    phi = rng.standard_normal((nx, ny, nz))
    s = oracle.advect_scalar(c, U, V, W, phi)
    want = (-7.25 * (np.roll(phi, -1, 0) - np.roll(phi, 1, 0)) / (2 * dx)
            + 3.5 * (np.roll(phi, -1, 1) - np.roll(phi, 1, 1)) / (2 * dy))
    np.testing.assert_allclose(s, want, rtol=0, atol=1e-14 * np.abs(want).max())


def pin_scalar_energy_and_skew():
    rng = np.random.default_rng(22)
    for nx, ny, nz in ((7, 5, 6), (4, 9, 2), (3, 3, 1)):
        c = stretched(nz)
        u, v, w = rand_fields(rng, nx, ny, nz)
        phi, psi = rng.standard_normal((2, nx, ny, nz)) + 290.0
        s, cond = oracle.advect_scalar(c, u, v, w, phi, want_cond=True)
        assert np.all(np.abs(s) <= cond * (1 + 1e-15))
        num, den = wdot(c, phi, s, 0), wdot(c, np.abs(phi), np.abs(s), 0)
        assert abs(num) <= 1e-14 * den + 1e-300, (num, den)
        lhs = wdot(c, psi, s, 0)
        rhs = -wdot(c, oracle.advect_scalar(c, u, v, w, psi), phi, 0)
        assert abs(lhs - rhs) <= 1e-13 * wdot(c, np.abs(psi), np.abs(s), 0), (lhs, rhs)


def pin_scalar_divergence_identity():
    """Summation by parts: sum W s = 1/2 sum W phi D with D the anelastic
    divergence of the cell's face fluxes (written out here, not by the oracle)."""
    rng = np.random.default_rng(23)
    nx, ny, nz, dx, dy = 7, 6, 8, 37.0, 53.0
    c = stretched(nz, dx, dy)
    u, v, w = rand_fields(rng, nx, ny, nz)
    phi = 300.0 + rng.standard_normal((nx, ny, nz))
    s = oracle.advect_scalar(c, u, v, w, phi)
    fw = c.rho_w[None, None, :] * w
    fw[:, :, -1] = 0.0                                   # lid
    below = np.concatenate([np.zeros((nx, ny, 1)), fw[:, :, :-1]], axis=2)   # ground
    D = ((u - np.roll(u, 1, 0)) / dx + (v - np.roll(v, 1, 1)) / dy
         + (fw - below) / (c.rho_n * c.dz)[None, None, :])
    lhs = wdot(c, np.ones_like(s), s, 0)
    rhs = 0.5 * wdot(c, phi, D, 0)
    scale = wdot(c, np.ones_like(s), np.abs(s), 0)
    assert abs(lhs - rhs) <= 1e-13 * scale, (lhs, rhs)
    assert abs(lhs) > 1e-6 * scale
    # a discretely divergence-free wind conserves every scalar
    x = streamfunction_flow(rng, nx, ny, nz, dx, dy)
    s = oracle.advect_scalar(c, *x, phi)
    assert abs(wdot(c, np.ones_like(s), s, 0)) <= 1e-14 * wdot(c, np.ones_like(s), np.abs(s), 0)


def pin_scalar_continuum_second_order():
    import sympy as sp
    H = 1500.0
    x, y, zz = sp.symbols("x y z", real=True)
    Lx, Ly, Z = 2000.0, 1600.0, 1000.0
    kx, ky = 2 * sp.pi / Lx, 2 * sp.pi / Ly
    u = 3 + sp.sin(kx * x + 0.4) * sp.cos(ky * y) * (1 + 0.3 * sp.cos(sp.pi * zz / Z))
    v = 2 + sp.cos(kx * x) * sp.sin(ky * y + 0.7) * (1 + 0.2 * zz / Z)
    w = 0.5 * sp.sin(sp.pi * zz / Z) * sp.cos(kx * x + 0.1) * sp.sin(ky * y + 0.2)
    th = 300 + 2 * sp.cos(kx * x + 0.3) * sp.sin(ky * y + 1.1) + 5 * sp.sin(sp.pi * zz / (2 * Z))
    rho = 1.2 * sp.exp(-zz / H)
    div = (sp.diff(rho * u, x) + sp.diff(rho * v, y) + sp.diff(rho * w, zz)) / rho
    S = -(u * sp.diff(th, x) + v * sp.diff(th, y) + w * sp.diff(th, zz)) - th * div / 2
    fl = [sp.lambdify((x, y, zz), f, "numpy") for f in (u, v, w, th)]
    Sl = sp.lambdify((x, y, zz), S, "numpy")
    errs = []
    for N in (12, 24, 48):
        dx, dy, dz = Lx / N, Ly / N, Z / N
        c = oracle.Coeffs(N, dx, dy, dz=np.full(N, dz), rho0=1.2, H=H)
        i = np.arange(N)[:, None, None]
        j = np.arange(N)[None, :, None]
        zn = ((np.arange(N) + 0.5) * dz)[None, None, :]
        zf = ((np.arange(N) + 1.0) * dz)[None, None, :]
        pts = [((i + 0.5) * dx, j * dy, zn), (i * dx, (j + 0.5) * dy, zn), (i * dx, j * dy, zf),
               (i * dx, j * dy, zn)]
        F = [np.broadcast_to(fl[q](*pts[q]), (N, N, N)).astype(np.float64).copy() for q in range(4)]
        F[2][:, :, -1] = 0.0
        s = oracle.advect_scalar(c, *F)
        ref = np.broadcast_to(Sl(*pts[3]), (N, N, N))
        errs.append(float(np.abs(s - ref).max() / np.abs(ref).max()))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.8 and 3.3 < r2 < 4.8, errs


def pin_scalar_lid_and_points():
    rng = np.random.default_rng(24)
    nx, ny, nz = 5, 4, 6
    c = stretched(nz)
    u, v, w = rand_fields(rng, nx, ny, nz)
    phi = rng.standard_normal((nx, ny, nz))
    w2 = w.copy()
    w2[:, :, -1] = 100.0 * rng.standard_normal((nx, ny))
    s, cond = oracle.advect_scalar(c, u, v, w, phi, want_cond=True)
    assert np.array_equal(s, oracle.advect_scalar(c, u, v, w2, phi))
    pts = np.array([[0, 0, 0], [4, 3, 5], [2, 1, 0], [1, 0, 5], [3, 2, 3]])
    vals, cv = oracle.scalar_points(c, u, v, w, phi, pts)
    for p, (i, j, k) in enumerate(pts):
        assert vals[p] == s[i, j, k] and cv[p] == cond[i, j, k]


def pin_euler_energy_step():
    """One forward-Euler step changes each component's energy by exactly
    dt^2 sum W S^2: sum W (phi + dt S)^2 - sum W phi^2 = 2 dt sum W phi S + dt^2
    sum W S^2, and the first sum vanishes (energy identity of the PW form)."""
    rng = np.random.default_rng(25)
    nx, ny, nz, dt = 6, 5, 7, 7.0
    c = stretched(nz)
    x = rand_fields(rng, nx, ny, nz)
    s = oracle.advect(c, *x)
    xn = oracle.euler(c, *x, dt, 1)
    for g in range(3):
        e0, e1 = wdot(c, x[g], x[g], g), wdot(c, xn[g], xn[g], g)
        want = dt * dt * wdot(c, s[g], s[g], g)
        assert want > 1e-3 * e0
        assert abs((e1 - e0) - want) <= 1e-12 * (e0 + want), (g, e1 - e0, want)


def pin_euler_closed_forms():
    """A 1-D profile carried by a uniform crossing wind: with rho and dz
    constant the PW sources at the levels away from the ground and the lid
    reduce to the centred advective derivative, so one Euler step is
    phi - dt U (phi(+1) - phi(-1)) / (2 h) there, and the carrying components do
    not change.  Fixes the sign of every component's update and the dt factor."""
    nx, ny, nz, dx, dy, dz, dt = 7, 6, 6, 40.0, 30.0, 20.0, 3.0
    U, V = 6.5, -4.25
    c = oracle.Coeffs(nz, dx, dy, dz=np.full(nz, dz), rho_n=np.ones(nz), rho_w=np.ones(nz), rho0=1.0)
    i = np.arange(nx)[:, None, None] * np.ones((1, ny, nz))
    j = np.arange(ny)[None, :, None] * np.ones((nx, 1, nz))
    prof = lambda n, t: np.sin(2 * np.pi * t / n) + 0.3 * np.cos(4 * np.pi * t / n)
    inner = slice(1, nz - 2)
    # v carried along x by u = U (w = 0): every level
    a = 5.0 + prof(nx, i)
    u, v, w = np.full((nx, ny, nz), U), a.copy(), np.zeros((nx, ny, nz))
    xn = oracle.euler(c, u, v, w, dt, 1)
    want = a - dt * U * (np.roll(a, -1, 0) - np.roll(a, 1, 0)) / (2 * dx)
    np.testing.assert_allclose(xn[1], want, rtol=0, atol=1e-13 * np.abs(a).max())
    assert np.array_equal(xn[0], u) and not xn[2].any()
    # u carried along y by v = V (w = 0): every level
    b = 3.0 + prof(ny, j)
    u, v = b.copy(), np.full((nx, ny, nz), V)
    xn = oracle.euler(c, u, v, w, dt, 1)
    want = b - dt * V * (np.roll(b, -1, 1) - np.roll(b, 1, 1)) / (2 * dy)
    np.testing.assert_allclose(xn[0], want, rtol=0, atol=1e-13 * np.abs(b).max())
    assert np.array_equal(xn[1], v) and not xn[2].any()
    # w carried along x by u = U, v = V: levels 1 .. nz-3 (the column of w is
    # uniform there, so its vertical terms cancel)
    a = 0.4 * prof(nx, i)
    a[:, :, -1] = 0.0
    u, v = np.full((nx, ny, nz), U), np.full((nx, ny, nz), V)
    xn = oracle.euler(c, u, v, a, dt, 1)
    want = a - dt * U * (np.roll(a, -1, 0) - np.roll(a, 1, 0)) / (2 * dx)
    np.testing.assert_allclose(xn[2][:, :, inner], want[:, :, inner], rtol=0, atol=1e-14)
    np.testing.assert_allclose(xn[0][:, :, inner], U, rtol=0, atol=1e-14)
    np.testing.assert_allclose(xn[1][:, :, inner], V, rtol=0, atol=1e-14)


def pin_euler_fixed_point_and_steps():
    """Uniform horizontal flow is a fixed point of the step (bit for bit), and n
    steps in one call equal n calls of one step (bit for bit)."""
    rng = np.random.default_rng(26)
    nz = 5
    c = stretched(nz)
    U = np.full((5, 4, nz), 7.25)
    V = np.full((5, 4, nz), -3.5)
    W = np.zeros((5, 4, nz))
    for a, b in zip(oracle.euler(c, U, V, W, 0.5, 3), (U, V, W)):
        assert np.array_equal(a, b)
    x = rand_fields(rng, 5, 6, nz)
    one = x
    for _ in range(3):
        one = oracle.euler(c, *one, 0.5, 1)
    three = oracle.euler(c, *x, 0.5, 3)
    for a, b in zip(one, three):
        assert np.array_equal(a, b)
    assert not np.array_equal(three[0], x[0])


def pin_adjoint_cond():
    """The gradient's condition sums (every contribution taken in absolute
    value).  S is homogeneous of degree 2 in (u, v, w), and so is its
    absolute-value form, so by Euler's theorem
      sum_P cond_g(P) |x(P)| = 2 sum_m |y(m)| cond_S(m)
    with cond_S the forward condition sums; the triangle inequality gives
    |J^T y| <= cond_g pointwise, with equality wherever every contribution to a
    point has one sign (checked on a one-point y over positive fields)."""
    rng = np.random.default_rng(27)
    nx, ny, nz = 6, 7, 6
    c = stretched(nz)
    x = rand_fields(rng, nx, ny, nz)
    x = (x[0] - 5.0, x[1] - 5.0, x[2])           # mixed signs
    y = [rng.standard_normal((nx, ny, nz)) for _ in range(3)]
    y[2][:, :, -1] = 0.0
    g = oracle.adjoint(c, *x, *y)
    cg = oracle.adjoint_cond(c, *x, *y)
    _, cs = oracle.advect(c, *x, want_cond=True)
    lhs = sum(float(np.sum(cg[q] * np.abs(x[q]))) for q in range(3))
    rhs = 2.0 * sum(float(np.sum(np.abs(y[q]) * cs[q])) for q in range(3))
    assert abs(lhs - rhs) <= 1e-13 * rhs, (lhs, rhs)
    for q in range(3):
        assert np.all(np.abs(g[q]) <= cg[q] * (1 + 1e-14))
    # equality where all contributions share a sign: y = 1 at su(i, j, k) only
    xp = rand_fields(rng, nx, ny, nz)
    xp = (np.abs(xp[0]) + 1, np.abs(xp[1]) + 1, np.abs(xp[2]))
    i, j, k = 3, 3, 2
    y1 = [np.zeros((nx, ny, nz)) for _ in range(3)]
    y1[0][i, j, k] = 1.0
    g1 = oracle.adjoint(c, *xp, *y1)
    c1 = oracle.adjoint_cond(c, *xp, *y1)
    for q, p in ((0, (i - 1, j, k)), (0, (i + 1, j, k)), (1, (i, j - 1, k)), (1, (i + 1, j, k))):
        assert c1[q][p] > 0
        assert abs(abs(g1[q][p]) - c1[q][p]) <= 1e-15 * c1[q][p], (q, p, g1[q][p], c1[q][p])
    assert abs(g1[0][i, j, k]) < c1[0][i, j, k] * (1 - 1e-6)      # contributions of both signs



# --------------------------------------------------------------------------
# pins of the ULTIMATE-QUICKEST scalar scheme (section 3.1's second scheme)
# --------------------------------------------------------------------------
def tvd_column_coeffs(dz):
    n = len(dz)
    return oracle.Coeffs(n, 1.0, 1.0, dz=np.asarray(dz, float), rho_n=np.ones(n), rho_w=np.ones(n), rho0=1.0)


def pin_tvd_worked_examples():
    spec = json.load(open(os.path.join(GOLDEN, "tvd_worked_examples.json")))
    c = tvd_column_coeffs(spec["grid"]["dz"])
    z = np.zeros((1, 1, 4))
    for e in spec["examples"]:
        w = np.array(e["w"]).reshape(1, 1, 4)
        phi = np.array(e["phi"]).reshape(1, 1, 4)
        s = oracle.advect_tvd(c, z + 3.0, z - 2.0, w, phi, e["dt"])[0, 0]
        np.testing.assert_allclose(s, e["expect"], rtol=0, atol=1e-14, err_msg=e["name"])


def pin_tvd_coefficients_and_constants():
    # fz1, fz2 are the doubled scalar PW coefficients with the ground and lid faces dropped
    c = stretched(9)
    np.testing.assert_allclose(c.fz1[1:], 2 * c.hz1[1:], rtol=1e-15)
    np.testing.assert_allclose(c.fz2[:-1], 2 * c.hz2[:-1], rtol=1e-15)
    assert c.fz1[0] == 0.0 and c.fz2[-1] == 0.0
    # a constant field: every face carries the constant, so s = C * (inflow - outflow)
    rng = np.random.default_rng(31)
    nx, ny, nz = 6, 5, 9
    u, v, w = rand_fields(rng, nx, ny, nz)
    u, v = u - 5 + 2 * rng.standard_normal(u.shape), v - 5 + 2 * rng.standard_normal(v.shape)
    C = 2.75
    s = oracle.advect_tvd(c, u, v, w, np.full((nx, ny, nz), C), dt=3.0)
    wb = np.concatenate([np.zeros((nx, ny, 1)), w[:, :, :-1]], axis=2)   # w(k-1), ground 0
    wt = w.copy()
    wt[:, :, -1] = 0.0                                                     # lid
    div = ((np.roll(u, 1, 0) - u) / c.dx + (np.roll(v, 1, 1) - v) / c.dy
           + c.fz1[None, None, :] * wb - c.fz2[None, None, :] * wt)
    np.testing.assert_allclose(s, C * div, rtol=1e-13, atol=1e-13 * np.abs(C * div).max())


def pin_tvd_courant_one_shift():
    rng = np.random.default_rng(32)
    # x and y: uniform flow of Courant number 1 moves every cell one cell on
    for axis, (nx, ny) in ((0, (11, 3)), (1, (3, 13))):
        c = oracle.Coeffs(2, 40.0, 25.0)
        h = c.dx if axis == 0 else c.dy
        phi = rng.random((nx, ny, 2)) * 10 - 3
        for U in (7.0, -7.0):
            wind = [np.zeros((nx, ny, 2)) for _ in range(3)]
            wind[axis][:] = U
            dt = h / abs(U)
            new = phi + dt * oracle.advect_tvd(c, *wind, phi, dt)
            np.testing.assert_allclose(new, np.roll(phi, 1 if U > 0 else -1, axis), rtol=0, atol=1e-13)
            # above Courant number 1 the limiter's window [t_C, t_C / c] is empty
            # and closes on its lower end: every face takes the upwind value
            dt = 1.6 * h / abs(U)
            up = np.roll(phi, 1, axis) if U > 0 else np.roll(phi, -1, axis)
            new = phi + dt * oracle.advect_tvd(c, *wind, phi, dt)
            np.testing.assert_allclose(new, phi - 1.6 * (phi - up), rtol=0, atol=1e-13)
    # z on a stretched column of unit density: w(k) = dz(C)/dt makes every
    # interior face Courant 1, so each cell's content dz(k) phi(k) moves one cell
    dz = np.array([3.0, 5.0, 2.0, 7.0, 4.0, 6.0, 1.5])
    nz = len(dz)
    c = tvd_column_coeffs(dz)
    phi = rng.random((2, 1, nz)) + 0.5
    M = dz * phi
    dt = 0.25
    for up in (True, False):
        w = np.zeros((2, 1, nz))
        w[:, :, :-1] = dz[:-1] / dt if up else -dz[1:] / dt
        new = phi + dt * oracle.advect_tvd(c, np.zeros_like(w), np.zeros_like(w), w, phi, dt)
        if up:
            Mn = np.concatenate([np.zeros((2, 1, 1)), M[:, :, :-1]], axis=2)
            Mn[:, :, -1] += M[:, :, -1]
        else:
            Mn = np.concatenate([M[:, :, 1:], np.zeros((2, 1, 1))], axis=2)
            Mn[:, :, 0] += M[:, :, 0]
        np.testing.assert_allclose(new * dz, Mn, rtol=0, atol=1e-13)


def quad_cell_means(x0, h, a, b, q):
    """Cell means over [x0 - h/2, x0 + h/2] of a + b x + q x^2."""
    P = lambda x: a * x + b * x * x / 2 + q * x ** 3 / 3
    return (P(x0 + h / 2) - P(x0 - h / 2)) / h


def pin_tvd_quadratic_exact():
    # QUICKEST is exact on the cell means of a parabola; on a monotone one the
    # limiter leaves it alone, so one step equals the translated cell means
    a, b, q = 3.0, 0.7, 0.02
    for axis, n in ((0, 48), (1, 40), (2, 36)):
        shape = [2, 2, 2]
        shape[axis] = n
        if axis < 2:
            c = oracle.Coeffs(2, 1.0, 1.0)
        else:
            c = tvd_column_coeffs(np.ones(n))
        x = np.arange(n, dtype=float)
        line = quad_cell_means(x, 1.0, a, b, q)
        phi = np.broadcast_to(line.reshape([n if d == axis else 1 for d in range(3)]), shape).copy()
        for cr in (0.25, 0.6, 0.9):
            for U in (2.0, -2.0):
                wind = [np.zeros(shape) for _ in range(3)]
                wind[axis][:] = U
                if axis == 2:
                    wind[2][:, :, -1] = 0.0
                dt = cr / abs(U)
                new = phi + dt * oracle.advect_tvd(c, *wind, phi, dt)
                exact = quad_cell_means(x - U * dt, 1.0, a, b, q)
                got = np.moveaxis(new, axis, 0)[:, 0, 0]
                lo, hi = 3, n - 3   # away from the periodic seam and the ground / lid
                np.testing.assert_allclose(got[lo:hi], exact[lo:hi], rtol=1e-13, err_msg=f"axis {axis} c {cr} U {U}")


def total_variation(line):
    return float(np.abs(np.diff(np.r_[line, line[:1]])).sum())


def pin_tvd_total_variation():
    # one dimension, uniform flow, c <= 1: no new extrema and no growth of the
    # total variation, on random and on step data
    rng = np.random.default_rng(33)
    for axis in (0, 1):
        n = 40
        shape = [1, 1, 1]
        shape[axis] = n
        c = oracle.Coeffs(1, 1.0, 1.0)
        for trial in range(12):
            line = rng.random(n) if trial % 2 else (np.arange(n) % 9 < 4) + 0.05 * rng.random(n)
            for cr in (0.15, 0.5, 0.85, 1.0):
                for U in (1.0, -1.0):
                    wind = [np.zeros(shape) for _ in range(3)]
                    wind[axis][:] = U
                    p = line.reshape(shape).copy()
                    for _ in range(4):
                        new = p + cr * oracle.advect_tvd(c, *wind, p, cr)
                        assert total_variation(new.ravel()) <= total_variation(p.ravel()) * (1 + 1e-14) + 1e-14
                        assert new.max() <= line.max() + 1e-14 and new.min() >= line.min() - 1e-14
                        p = new


def pin_tvd_conservation_and_mirror():
    rng = np.random.default_rng(34)
    nx, ny, nz = 7, 6, 10
    c = stretched(nz)
    u, v, w = rand_fields(rng, nx, ny, nz)
    u = u - 5 + 3 * rng.standard_normal(u.shape)
    phi = rng.random((nx, ny, nz)) * 4
    s, cond = oracle.advect_tvd(c, u, v, w, phi, dt=2.0, want_cond=True)
    # flux form: the density-weighted sum of the sources is 0 (periodic sides,
    # no flux through the ground or the lid)
    W = (c.rho_n * c.dz)[None, None, :]
    assert abs(np.sum(W * s)) <= 1e-13 * np.sum(W * cond)
    # reflecting x (cell i -> nx-1-i; the face of u(i) -> that of u(nx-2-i),
    # whose velocity changes sign) reflects the source
    r = lambda f: f[::-1]
    ur = -np.roll(u[::-1], -1, axis=0)
    sr = oracle.advect_tvd(c, ur, r(v), r(w), r(phi), dt=2.0)
    np.testing.assert_allclose(sr, r(s), rtol=0, atol=1e-13 * np.abs(s).max())
    # the same reflection in y
    sy = oracle.advect_tvd(c, u[:, ::-1], -np.roll(v[:, ::-1], -1, axis=1), w[:, ::-1], phi[:, ::-1], dt=2.0)
    np.testing.assert_allclose(sy, s[:, ::-1], rtol=0, atol=1e-13 * np.abs(s).max())


def pin_tvd_lid_and_points():
    rng = np.random.default_rng(35)
    nx, ny, nz = 5, 4, 7
    c = stretched(nz)
    u, v, w = rand_fields(rng, nx, ny, nz)
    phi = rng.standard_normal((nx, ny, nz))
    s, cond = oracle.advect_tvd(c, u, v, w, phi, dt=1.5, want_cond=True)
    w2 = w.copy()
    w2[:, :, -1] = 1e3                      # the lid value is never read
    np.testing.assert_array_equal(oracle.advect_tvd(c, u, v, w2, phi, dt=1.5), s)
    assert np.all(cond >= np.abs(s) * (1 - 1e-15))
    pts = np.array([[i, j, k] for i in range(nx) for j in range(ny) for k in range(nz)][::3])
    o, oc = oracle.tvd_points(c, u, v, w, phi, 1.5, pts)
    np.testing.assert_array_equal(o, s[pts[:, 0], pts[:, 1], pts[:, 2]])
    np.testing.assert_array_equal(oc, cond[pts[:, 0], pts[:, 1], pts[:, 2]])


PINS = [pin_worked_examples, pin_lid_ignored, pin_coefficients, pin_uniform_flow, pin_energy, pin_skew_adjoint,
        pin_momentum_divergence_free, pin_momentum_identity, pin_continuum_second_order,
        pin_adjoint_dot, pin_adjoint_bruteforce, pin_cond_and_points,
        pin_euler_energy_step, pin_euler_closed_forms, pin_euler_fixed_point_and_steps, pin_adjoint_cond,
        pin_scalar_worked_examples, pin_scalar_uniform_and_centred, pin_scalar_energy_and_skew,
        pin_scalar_divergence_identity, pin_scalar_continuum_second_order, pin_scalar_lid_and_points,
        pin_tvd_worked_examples, pin_tvd_coefficients_and_constants, pin_tvd_courant_one_shift,
        pin_tvd_quadratic_exact, pin_tvd_total_variation, pin_tvd_conservation_and_mirror, pin_tvd_lid_and_points]


@pytest.mark.parametrize("pin", PINS + [pin_loop_gradient], ids=lambda f: f.__name__)
def test_pin(pin):
    pin()


def test_default_stretch_and_generators():
    dz = synthetic.default_dz(9)
    assert dz[0] == 10.0 and abs(dz[-1] - 40.0) < 1e-12
    assert np.allclose(dz[1:] / dz[:-1], 4 ** (1 / 8))
    c = oracle.Coeffs(9, 50.0, 50.0)
    np.testing.assert_allclose(c.dz, dz, rtol=1e-15)
    u, v, w = synthetic.wind_fields(8, 8, 6, 1)
    assert not w[:, :, -1].any()
    u2, _, _ = synthetic.wind_fields(8, 8, 6, 1)
    assert np.array_equal(u, u2)


def test_residuals_match_identities():
    rng = np.random.default_rng(14)
    nx, ny, nz = 6, 6, 6
    c = stretched(nz)
    u, v, w = rand_fields(rng, nx, ny, nz)
    s = oracle.advect(c, u, v, w)
    (re, rm) = oracle.residuals(c, u, v, w, *s)
    assert max(abs(r) for r in re) < 1e-14
    assert all(abs(r) > 1e-8 for r in rm)     # arbitrary fields: momentum not conserved
    x = streamfunction_flow(rng, nx, ny, nz, 37.0, 53.0)
    (re2, rm2) = oracle.residuals(c, *x, *oracle.advect(c, *x))
    assert abs(rm2[0]) < 1e-14 and abs(rm2[1]) < 1e-14 and max(abs(r) for r in re2) < 1e-14


# --------------------------------------------------------------------------
# planted mistakes: each must be caught by at least one pin
# --------------------------------------------------------------------------
MUTANTS = {
    "su_x_sign": ("                - at(g, p, i + 1, j, k) * (at(g, u, i, j, k) + at(g, u, i + 1, j, k)));\n    c = fabs(g->tcx) * (fabs(at(g, p, i - 1, j, k)) * (fabs(at(g, u, i - 1, j, k)) + fabs(at(g, u, i, j, k)))",
                  "                + at(g, p, i + 1, j, k) * (at(g, u, i, j, k) + at(g, u, i + 1, j, k)));\n    c = fabs(g->tcx) * (fabs(at(g, p, i - 1, j, k)) * (fabs(at(g, u, i - 1, j, k)) + fabs(at(g, u, i, j, k)))"),
    "su_y_index": ("(at(g, v, i, j - 1, k) + at(g, v, i + 1, j - 1, k))\n                    - at(g, p, i, j + 1, k)",
                   "(at(g, v, i, j - 1, k) + at(g, v, i - 1, j - 1, k))\n                    - at(g, p, i, j + 1, k)"),
    "sv_drop_tzc2": ("        s = s - g->tzc2[k] * at(g, p, i, j, k + 1) * (at(g, w, i, j, k) + at(g, w, i, j + 1, k));",
                     "        s = s;"),
    "su_swap_tzc": ("        s = s + g->tzc1[k] * at(g, p, i, j, k - 1) * (at(g, w, i, j, k - 1) + at(g, w, i + 1, j, k - 1));",
                    "        s = s + g->tzc2[k] * at(g, p, i, j, k - 1) * (at(g, w, i, j, k - 1) + at(g, w, i + 1, j, k - 1));"),
    "tzc1_wrong_rho": ("        double rw_below = (k == 0) ? rho0 : rhow[k - 1];",
                       "        double rw_below = (k == 0) ? rho0 : rhon[k - 1];"),
    "tzd2_wrong_level": ("            tzd2[k] = 0.25 * rhon[k + 1] / (rhow[k] * dzn[k]);",
                         "            tzd2[k] = 0.25 * rhon[k] / (rhow[k] * dzn[k]);"),
    "sw_x_transposed": ("(at(g, u, i - 1, j, k) + at(g, u, i - 1, j, k + 1))\n                - at(g, p, i + 1, j, k) * (at(g, u, i, j, k) + at(g, u, i, j, k + 1)));\n    c = fabs(g->tcx) * (fabs(at(g, p, i - 1, j, k)) * (fabs(at(g, u, i - 1, j, k)) + fabs(at(g, u, i - 1, j, k + 1)))",
                        "(at(g, u, i - 1, j, k) + at(g, u, i, j, k + 1))\n                - at(g, p, i + 1, j, k) * (at(g, u, i, j, k) + at(g, u, i, j, k + 1)));\n    c = fabs(g->tcx) * (fabs(at(g, p, i - 1, j, k)) * (fabs(at(g, u, i - 1, j, k)) + fabs(at(g, u, i - 1, j, k + 1)))"),
    "sw_reads_lid": ("    if (k + 1 < nz - 1) {   /* phi(k+1) is the lid when k+1 = nz-1: 0 */",
                     "    if (k < nz - 1) {   /* phi(k+1) is the lid when k+1 = nz-1: 0 */"),
    "adjoint_table_offset": ("    {1, CX, -1, +1, 0, 0, 0, 0, 0, 0, 0, +1, 0, 0},",
                             "    {1, CX, -1, +1, 0, 0, 0, 0, 0, 0, +1, 0, 0, 0},"),
    "adjoint_sign": ("    {2, D2, -1, 0, 0, +1, 2, 0, 0, 0, 0, 0, +1, 3},",
                     "    {2, D2, +1, 0, 0, +1, 2, 0, 0, 0, 0, 0, +1, 3},"),
    "stretch_exponent": ("        else dz[k] = 10.0 * pow(4.0, (double)k / (double)(nz - 1));",
                         "        else dz[k] = 10.0 * pow(4.0, (double)k / (double)nz);"),
    "dzn_offset": ("    for (int k = 0; k < nz; k++) dzn[k] = (k < nz - 1) ? zn[k + 1] - zn[k] : 0.0;",
                   "    for (int k = 0; k < nz; k++) dzn[k] = (k < nz - 1) ? zf[k + 1] - zf[k] : 0.0;"),
    "scalar_x_sign": ("* at(g, p, i - 1, j, k) - at(g, u, i, j, k) * at(g, p, i + 1, j, k));",
                      "* at(g, p, i - 1, j, k) + at(g, u, i, j, k) * at(g, p, i + 1, j, k));"),
    "scalar_y_face": ("    s = s + g->tcy * (at(g, v, i, j - 1, k) * at(g, p, i, j - 1, k)",
                      "    s = s + g->tcy * (at(g, v, i, j, k) * at(g, p, i, j - 1, k)"),
    "scalar_drop_top": ("        s = s - hz2[k] * at(g, w, i, j, k) * at(g, p, i, j, k + 1);",
                        "        s = s;"),
    "scalar_bottom_level": ("        s = s + hz1[k] * at(g, w, i, j, k - 1) * at(g, p, i, j, k - 1);",
                            "        s = s + hz1[k] * at(g, w, i, j, k) * at(g, p, i, j, k - 1);"),
    "scalar_hz1_rho": ("        hz1[k] = 0.5 * rho_face_below / (rhon[k] * dz[k]);",
                       "        hz1[k] = 0.5 * rhow[k] / (rhon[k] * dz[k]);"),
    "scalar_ground_density": ("        double rho_face_below = (k == 0) ? rho0 : rhow[k - 1];",
                              "        double rho_face_below = (k == 0) ? rhon[0] : rhow[k - 1];"),
    "scalar_quarter_width": ("        hz2[k] = 0.5 * rhow[k] / (rhon[k] * dz[k]);",
                             "        hz2[k] = 0.25 * rhow[k] / (rhon[k] * dz[k]);"),
    "euler_dt_squared": ("            u[m] = u[m] + dt * s[m];",
                         "            u[m] = u[m] + dt * dt * s[m];"),
    "euler_v_takes_su": ("            v[m] = v[m] + dt * s[n + m];",
                         "            v[m] = v[m] + dt * s[m];"),
    "euler_w_sign": ("            w[m] = w[m] + dt * s[2 * n + m];",
                     "            w[m] = w[m] - dt * s[2 * n + m];"),
    "euler_stale_sources": ("        pwo_advect(nx, ny, nz, tcx, tcy, tzc1, tzc2, tzd1, tzd2, u, v, w,\n                   s, s + n",
                            "        if (t == 0) pwo_advect(nx, ny, nz, tcx, tcy, tzc1, tzc2, tzd1, tzd2, u, v, w,\n                   s, s + n"),
    "adjoint_cond_signed_face_sum": ("gs[T->src][P] += fabs(sc) * (fabs(a[Q1]) + fabs(a[Q2]));",
                                     "gs[T->src][P] += fabs(sc * (a[Q1] + a[Q2]));"),
    "adjoint_cond_wrong_point": ("                        gs[T->a][Q2] += fabs(sc * phi);",
                                 "                        gs[T->a][Q1] += fabs(sc * phi);"),
    "adjoint_cond_drops_phi": ("                        gs[T->a][Q1] += fabs(sc * phi);",
                               "                        gs[T->a][Q1] += fabs(sc);"),
    "tvd_quick_coefficient": ("- (1.0 - c * c) / 6.0 * (pd - 2.0 * pc + pu);",
                              "- 1.0 / 8.0 * (pd - 2.0 * pc + pu);"),
    "tvd_courant_half": ("    return 0.5 * (pc + pd) - 0.5 * c * (pd - pc)",
                         "    return 0.5 * (pc + pd) - 0.25 * c * (pd - pc)"),
    "tvd_extrema_unlimited": ("    if (!monotone) return pc;",
                              "    if (!monotone) return quickest(pu, pc, pd, c);"),
    "tvd_no_courant_bound": ("    double top = (c > tc) ? tc / c : 1.0;   /* min(1, tc / c) */",
                             "    double top = 1.0;"),
    "tvd_no_lower_bound": ("    if (tf < tc) tf = tc;",
                           "    (void)0;"),
    "tvd_negative_far_cell": ("    return ultimate(pr2, pr, pl, c);",
                              "    return ultimate(pl2, pr, pl, c);"),
    "tvd_courant_downwind_width": ("        c = fabs(a) * g->dt / g->dz[a >= 0.0 ? k - 1 : k];",
                                   "        c = fabs(a) * g->dt / g->dz[k];"),
    "tvd_fz1_density": ("        fz1[k] = (k > 0) ? rhow[k - 1] / (rhon[k] * dz[k]) : 0.0;",
                        "        fz1[k] = (k > 0) ? rhon[k - 1] / (rhon[k] * dz[k]) : 0.0;"),
    "tvd_ground_far_cell": ("                     k + 1 < nz ? tat(g, p, i, j, k + 1) : 0.0, k >= 2, k + 1 < nz, &m);",
                            "                     k + 1 < nz ? tat(g, p, i, j, k + 1) : 0.0, 1, k + 1 < nz, &m);"),
    "tvd_y_inflow_sign": ("    s = s + a * f / g->dy;",
                          "    s = s - a * f / g->dy;"),
    "tvd_x_face_shift": ("    f = tvd_face(a, c, tat(g, p, i - 1, j, k), tat(g, p, i, j, k), tat(g, p, i + 1, j, k),\n                 tat(g, p, i + 2, j, k), 1, 1, &m);",
                         "    f = tvd_face(a, c, tat(g, p, i - 2, j, k), tat(g, p, i - 1, j, k), tat(g, p, i, j, k),\n                 tat(g, p, i + 1, j, k), 1, 1, &m);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "pw_oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, name
    mpath = tmp_path / "mut.c"
    mpath.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so), str(mpath), "-lm"],
                   check=True)
    caught = []
    with oracle.use_library(str(so)):
        for pin in PINS:
            try:
                pin()
            except AssertionError:
                caught.append(pin.__name__)
    assert caught, f"planted mistake {name} passed every pin"
