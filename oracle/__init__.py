"""FP64 CPU oracle of the Piacsek-Williams advection source terms (and of the
ULTIMATE-QUICKEST scalar scheme the paper names beside it).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and the CPU legs of
bench.py may import this package; the library and its Python binding never do.
It shares no code with the CUDA path.

Arrays here are interior-only numpy float64 arrays of shape (nx, ny, nz), k
fastest, periodic in i and j by modulo indexing.  The C source (pw_oracle.c)
holds every formula with its derivation; this module only marshals arguments.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_L = ctypes.POINTER(ctypes.c_long)


def lib():
    global _lib
    if _lib is None:
        path = _lib_path_override[-1] if _lib_path_override else _build.build()
        L = ctypes.CDLL(path)
        L.pwo_set_threads.argtypes = [ctypes.c_int]
        L.pwo_set_threads.restype = ctypes.c_int
        L.pwo_coeffs.argtypes = [ctypes.c_int, _D, _D, _D, ctypes.c_double, ctypes.c_double] + [_D] * 10
        L.pwo_coeffs.restype = ctypes.c_int
        L.pwo_src.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double] * 2 + [_D] * 4 + [_D] * 4 + [_D, _D]
        L.pwo_src.restype = None
        L.pwo_advect.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [_D] * 4 + [_D] * 3 + [_D] * 6
        L.pwo_advect.restype = None
        L.pwo_advect_points.argtypes = ([ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [_D] * 4 + [_D] * 3
                                        + [ctypes.c_long, _L, _D, _D])
        L.pwo_advect_points.restype = None
        L.pwo_adjoint.argtypes = ([ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [_D] * 4 + [_D] * 3
                                  + [_D] * 3 + [_D] * 3 + [ctypes.c_int])
        L.pwo_adjoint.restype = None
        L.pwo_adjoint_mode.argtypes = L.pwo_adjoint.argtypes + [ctypes.c_int]
        L.pwo_adjoint_mode.restype = None
        L.pwo_residual_sums.argtypes = [ctypes.c_int] * 3 + [_D] * 4 + [_D] * 6 + [_D]
        L.pwo_residual_sums.restype = None
        L.pwo_face_divergence.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double] * 2 + [_D] * 4 + [_D] * 3 + [_D]
        L.pwo_face_divergence.restype = None
        L.pwo_euler.argtypes = ([ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [_D] * 4 + [_D] * 3
                                + [ctypes.c_double, ctypes.c_int])
        L.pwo_euler.restype = ctypes.c_int
        L.pwo_scalar_coeffs.argtypes = [ctypes.c_int, _D, _D, _D, ctypes.c_double, _D, _D]
        L.pwo_scalar_coeffs.restype = None
        L.pwo_scalar_src.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [_D] * 2 + [_D] * 4 + [_D, _D]
        L.pwo_scalar_src.restype = None
        L.pwo_scalar_points.argtypes = ([ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [_D] * 2 + [_D] * 4
                                        + [ctypes.c_long, _L, _D, _D])
        L.pwo_scalar_points.restype = None
        L.pwo_tvd_coeffs.argtypes = [ctypes.c_int, _D, _D, _D, _D, _D]
        L.pwo_tvd_coeffs.restype = None
        L.pwo_tvd_src.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 3 + [_D] * 3 + [_D] * 4 + [_D, _D]
        L.pwo_tvd_src.restype = None
        L.pwo_tvd_points.argtypes = ([ctypes.c_int] * 3 + [ctypes.c_double] * 3 + [_D] * 3 + [_D] * 4
                                     + [ctypes.c_long, _L, _D, _D])
        L.pwo_tvd_points.restype = None
        _lib = L
    return _lib


class use_library:
    """Context manager: route every oracle call through another build of the C
    source (used by the tests that plant mistakes in a copy of the oracle)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        self._saved = lib()
        _lib = None
        _lib_path_override.append(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        _lib_path_override.pop()
        _lib = self._saved
        return False


_lib_path_override = []


def set_threads(n: int) -> int:
    """Set the OpenMP thread count of full-field sweeps; returns the count in use."""
    return lib().pwo_set_threads(int(n))


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Coeffs:
    """Vertical grid and PW coefficients (A1) for one mesh."""

    def __init__(self, nz, dx, dy, dz=None, rho_n=None, rho_w=None, rho0=1.2, H=8000.0):
        self.nz, self.dx, self.dy = int(nz), float(dx), float(dy)
        names = ["dz", "zf", "zn", "dzn", "rho_n", "rho_w", "tzc1", "tzc2", "tzd1", "tzd2"]
        arrs = {n: np.zeros(self.nz) for n in names}
        dz_in = None if dz is None else _f64(dz)
        rn_in = None if rho_n is None else _f64(rho_n)
        rw_in = None if rho_w is None else _f64(rho_w)
        rc = lib().pwo_coeffs(self.nz, _p(dz_in), _p(rn_in), _p(rw_in), float(rho0), float(H),
                              *[_p(arrs[n]) for n in names])
        if rc != 0:
            raise ValueError("oracle: bad coefficient arguments")
        for n in names:
            setattr(self, n, arrs[n])
        self.tcx = 0.25 / self.dx
        self.tcy = 0.25 / self.dy
        # scalar (theta, q) coefficients
        self.rho0 = float(rho0)
        self.hz1, self.hz2 = np.zeros(self.nz), np.zeros(self.nz)
        lib().pwo_scalar_coeffs(self.nz, _p(self.dz), _p(self.rho_n), _p(self.rho_w), self.rho0,
                                _p(self.hz1), _p(self.hz2))
        self.hx = 0.5 / self.dx
        self.hy = 0.5 / self.dy
        # flux-form vertical coefficients of the ULTIMATE-QUICKEST scheme
        self.fz1, self.fz2 = np.zeros(self.nz), np.zeros(self.nz)
        lib().pwo_tvd_coeffs(self.nz, _p(self.dz), _p(self.rho_n), _p(self.rho_w), _p(self.fz1), _p(self.fz2))

    def args(self):
        return (self.tcx, self.tcy, _p(self.tzc1), _p(self.tzc2), _p(self.tzd1), _p(self.tzd2))


def _shape(a):
    nx, ny, nz = a.shape
    return int(nx), int(ny), int(nz)


def advect(c: Coeffs, u, v, w, want_cond=False):
    """su, sv, sw (and the per-point condition sums if asked)."""
    u, v, w = _f64(u), _f64(v), _f64(w)
    nx, ny, nz = _shape(u)
    assert nz == c.nz
    out = [np.empty_like(u) for _ in range(3)]
    cond = [np.empty_like(u) for _ in range(3)] if want_cond else [None] * 3
    lib().pwo_advect(nx, ny, nz, *c.args(), _p(u), _p(v), _p(w),
                     *[_p(o) for o in out], *[_p(o) for o in cond])
    return (tuple(out), tuple(cond)) if want_cond else tuple(out)


def src(c: Coeffs, which, u, v, w, phi):
    """B(adv=(u,v,w); phi) on the u (0), v (1) or w (2) grid."""
    u, v, w, phi = _f64(u), _f64(v), _f64(w), _f64(phi)
    nx, ny, nz = _shape(u)
    out = np.empty_like(u)
    lib().pwo_src(int(which), nx, ny, nz, *c.args(), _p(u), _p(v), _p(w), _p(phi), _p(out), None)
    return out


def advect_points(c: Coeffs, u, v, w, pts):
    """S at the given (n, 3) integer points; returns (values, cond), each (n, 3)."""
    u, v, w = _f64(u), _f64(v), _f64(w)
    nx, ny, nz = _shape(u)
    pts = np.ascontiguousarray(pts, dtype=np.int64)
    n = pts.shape[0]
    out = np.empty((n, 3))
    cond = np.empty((n, 3))
    lib().pwo_advect_points(nx, ny, nz, *c.args(), _p(u), _p(v), _p(w), n,
                            pts.ctypes.data_as(_L), _p(out), _p(cond))
    return out, cond


def adjoint(c: Coeffs, u, v, w, gsu, gsv, gsw):
    """gu, gv, gw = J(u,v,w)^T (gsu, gsv, gsw)."""
    u, v, w = _f64(u), _f64(v), _f64(w)
    gsu, gsv, gsw = _f64(gsu), _f64(gsv), _f64(gsw)
    nx, ny, nz = _shape(u)
    g = [np.zeros_like(u) for _ in range(3)]
    lib().pwo_adjoint(nx, ny, nz, *c.args(), _p(u), _p(v), _p(w), _p(gsu), _p(gsv), _p(gsw),
                      *[_p(x) for x in g], 0)
    return tuple(g)


def adjoint_cond(c: Coeffs, u, v, w, gsu, gsv, gsw):
    """Per-point sums of |contribution| of the gradient (its condition sums)."""
    u, v, w = _f64(u), _f64(v), _f64(w)
    gsu, gsv, gsw = _f64(gsu), _f64(gsv), _f64(gsw)
    nx, ny, nz = _shape(u)
    g = [np.zeros_like(u) for _ in range(3)]
    lib().pwo_adjoint_mode(nx, ny, nz, *c.args(), _p(u), _p(v), _p(w), _p(gsu), _p(gsv), _p(gsw),
                           *[_p(x) for x in g], 0, 1)
    return tuple(g)


def advect_scalar(c: Coeffs, u, v, w, phi, want_cond=False):
    """PW source of the cell-centred scalar phi advected by (u, v, w)
    (and its per-point condition sums if asked)."""
    u, v, w, phi = _f64(u), _f64(v), _f64(w), _f64(phi)
    nx, ny, nz = _shape(u)
    assert nz == c.nz and phi.shape == u.shape
    out = np.empty_like(u)
    cond = np.empty_like(u) if want_cond else None
    lib().pwo_scalar_src(nx, ny, nz, c.hx, c.hy, _p(c.hz1), _p(c.hz2), _p(u), _p(v), _p(w), _p(phi),
                         _p(out), _p(cond))
    return (out, cond) if want_cond else out


def scalar_points(c: Coeffs, u, v, w, phi, pts):
    """Scalar source at the given (n, 3) integer points; returns (values, cond), each (n,)."""
    u, v, w, phi = _f64(u), _f64(v), _f64(w), _f64(phi)
    nx, ny, nz = _shape(u)
    pts = np.ascontiguousarray(pts, dtype=np.int64)
    n = pts.shape[0]
    out = np.empty(n)
    cond = np.empty(n)
    lib().pwo_scalar_points(nx, ny, nz, c.hx, c.hy, _p(c.hz1), _p(c.hz2), _p(u), _p(v), _p(w), _p(phi), n,
                            pts.ctypes.data_as(_L), _p(out), _p(cond))
    return out, cond


def advect_tvd(c: Coeffs, u, v, w, phi, dt, want_cond=False):
    """ULTIMATE-QUICKEST flux-form source of the scalar phi advected by
    (u, v, w) over one step dt (and its per-point condition sums if asked)."""
    u, v, w, phi = _f64(u), _f64(v), _f64(w), _f64(phi)
    nx, ny, nz = _shape(u)
    assert nz == c.nz and phi.shape == u.shape
    out = np.empty_like(u)
    cond = np.empty_like(u) if want_cond else None
    lib().pwo_tvd_src(nx, ny, nz, c.dx, c.dy, float(dt), _p(c.dz), _p(c.fz1), _p(c.fz2),
                      _p(u), _p(v), _p(w), _p(phi), _p(out), _p(cond))
    return (out, cond) if want_cond else out


def tvd_points(c: Coeffs, u, v, w, phi, dt, pts):
    """ULTIMATE-QUICKEST source at the given (n, 3) integer points; returns (values, cond)."""
    u, v, w, phi = _f64(u), _f64(v), _f64(w), _f64(phi)
    nx, ny, nz = _shape(u)
    pts = np.ascontiguousarray(pts, dtype=np.int64)
    n = pts.shape[0]
    out = np.empty(n)
    cond = np.empty(n)
    lib().pwo_tvd_points(nx, ny, nz, c.dx, c.dy, float(dt), _p(c.dz), _p(c.fz1), _p(c.fz2),
                         _p(u), _p(v), _p(w), _p(phi), n, pts.ctypes.data_as(_L), _p(out), _p(cond))
    return out, cond


def residual_sums(c: Coeffs, u, v, w, su, sv, sw):
    """(3, 4) array: per component [sum W phi S, sum W|phi S|, sum W S, sum W|S|]."""
    arrs = [_f64(a) for a in (u, v, w, su, sv, sw)]
    nx, ny, nz = _shape(arrs[0])
    out = np.zeros(12)
    lib().pwo_residual_sums(nx, ny, nz, _p(c.rho_n), _p(c.dz), _p(c.rho_w), _p(c.dzn),
                            *[_p(a) for a in arrs], _p(out))
    return out.reshape(3, 4)


def residuals(c: Coeffs, u, v, w, su, sv, sw):
    """R_E and R_M per component: ((RE_u, RE_v, RE_w), (RM_u, RM_v, RM_w))."""
    s = residual_sums(c, u, v, w, su, sv, sw)
    re = tuple(s[q, 0] / s[q, 1] if s[q, 1] != 0 else 0.0 for q in range(3))
    rm = tuple(s[q, 2] / s[q, 3] if s[q, 3] != 0 else 0.0 for q in range(3))
    return re, rm


def face_divergence(c: Coeffs, which, u, v, w):
    u, v, w = _f64(u), _f64(v), _f64(w)
    nx, ny, nz = _shape(u)
    out = np.empty_like(u)
    lib().pwo_face_divergence(int(which), nx, ny, nz, *c.args(), _p(u), _p(v), _p(w), _p(out))
    return out


def euler(c: Coeffs, u, v, w, dt, nsteps):
    """nsteps forward-Euler steps x <- x + dt S(x); returns new arrays."""
    u, v, w = _f64(u).copy(), _f64(v).copy(), _f64(w).copy()
    nx, ny, nz = _shape(u)
    rc = lib().pwo_euler(nx, ny, nz, *c.args(), _p(u), _p(v), _p(w), float(dt), int(nsteps))
    if rc != 0:
        raise MemoryError("oracle euler")
    return u, v, w


def weights(c: Coeffs):
    """Energy weights per level: (W_uv[nz], W_w[nz]) with the lid face weighted 0."""
    wuv = c.rho_n * c.dz
    ww = c.rho_w * c.dzn
    ww = ww.copy()
    ww[-1] = 0.0
    return wuv, ww


def loss_and_grad(c: Coeffs, u, v, w, dt, nsteps):
    """Adjoint-loop reference: L = sum(su^2 + sv^2 + sw^2) of S at the state after
    nsteps Euler steps, and dL/d(u0, v0, w0) by the oracle adjoint (FP64)."""
    states = []
    x = (_f64(u).copy(), _f64(v).copy(), _f64(w).copy())
    for _ in range(nsteps):
        states.append(x)
        s = advect(c, *x)
        x = tuple(x[q] + dt * s[q] for q in range(3))
    s = advect(c, *x)
    L = float(sum(np.sum(si * si) for si in s))
    g = adjoint(c, *x, *(2.0 * si for si in s))
    for t in reversed(range(nsteps)):
        jt = adjoint(c, *states[t], *g)
        g = tuple(g[q] + dt * jt[q] for q in range(3))
    return L, g
