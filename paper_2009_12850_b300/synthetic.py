"""Seeded synthetic inputs shaped like the paper's LES runs.

The paper's runs use MONC's "tank experiment" (warm and cold bubbles, sub-grid
on, five moisture fields; Results section), which is not available here.  These
generators stand in for it with the wind-field statistics and grid shapes of the
workloads this library is measured on.  They hold none of the advection
arithmetic: they only draw random numbers and lay out the vertical spacing used
to shape a height profile.  Every array is float64, interior only, shaped
(nx, ny, nz) with k fastest; the lid face w[..., nz-1] is set to 0.
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    seed: int
    kind: str = "wind"            # "wind" (mean + noise) or "shear"
    dtype: str = "f64"
    extra: dict = field(default_factory=dict)

    @property
    def points(self) -> int:
        return self.nx * self.ny * self.nz


# The five workloads: a 64^3 local domain (the weak-scaling local size of the
# paper's Results section), a 1024x1024x128 bandwidth run, a 512x512x160 precision
# study, a 64-member uneven ensemble and a 256x256x96 adjoint loop.
SMALL = Workload("pw_64x64x64_dx50", 64, 64, 64, 50.0, 50.0, 1234)
LARGE = Workload("pw_1024x1024x128_dx25", 1024, 1024, 128, 25.0, 25.0, 1235)
PRECISION = Workload("pw_512x512x160_shear_dx50", 512, 512, 160, 50.0, 50.0, 1236, kind="shear")
ENSEMBLE_SEED = 1237
ADJOINT = Workload("pw_adjoint_256x256x96_dx50", 256, 256, 96, 50.0, 50.0, 1238,
                   extra={"dt": 0.5, "steps": 10, "checkpoint_every": 2})
PAPER_STRONG = Workload("pw_2048x2048x64_dx25", 2048, 2048, 64, 25.0, 25.0, 1239, dtype="f32")


def default_dz(nz: int) -> np.ndarray:
    """Geometric stretch from 10 m at the ground to 40 m at the top."""
    if nz == 1:
        return np.full(1, 10.0)
    return 10.0 * 4.0 ** (np.arange(nz) / (nz - 1))


def wind_fields(nx, ny, nz, seed, u_mean=5.0, u_std=1.0, v_mean=5.0, v_std=1.0, w_std=0.3):
    """u, v = mean + N(0, std); w = N(0, w_std) with the lid face 0."""
    rng = np.random.default_rng(seed)
    u = u_mean + u_std * rng.standard_normal((nx, ny, nz))
    v = v_mean + v_std * rng.standard_normal((nx, ny, nz))
    w = w_std * rng.standard_normal((nx, ny, nz))
    w[:, :, nz - 1] = 0.0
    return u, v, w


def shear_fields(nx, ny, nz, seed, top_speed=15.0, noise=2.0, w_std=0.3, dz=None):
    """u rising linearly with height from 0 at the ground to top_speed at the lid,
    plus N(0, noise); v = N(0, noise); w = N(0, w_std) with the lid face 0.
    Heights are cell centres of the given spacing (default geometric stretch)."""
    dz = default_dz(nz) if dz is None else np.asarray(dz, dtype=np.float64)
    top = np.cumsum(dz)
    centre = top - 0.5 * dz
    profile = top_speed * centre / top[-1]
    rng = np.random.default_rng(seed)
    u = profile[None, None, :] + noise * rng.standard_normal((nx, ny, nz))
    v = noise * rng.standard_normal((nx, ny, nz))
    w = w_std * rng.standard_normal((nx, ny, nz))
    w[:, :, nz - 1] = 0.0
    return u, v, w


def scalar_fields(nx, ny, nz, n, seed, dz=None):
    """n cell-centred scalars: theta (K) first, then n - 1 moisture / tracer
    fields (kg/kg).  theta = 300 + 0.003 z + N(0, 0.5) (a stably stratified
    column with warm and cold perturbations); q_m = 1e-3 (m + 1) U(0, 1)."""
    dz = default_dz(nz) if dz is None else np.asarray(dz, dtype=np.float64)
    centre = np.cumsum(dz) - 0.5 * dz
    rng = np.random.default_rng(seed)
    out = [300.0 + 0.003 * centre[None, None, :] + 0.5 * rng.standard_normal((nx, ny, nz))]
    for m in range(1, n):
        out.append(1e-3 * (m + 1) * rng.random((nx, ny, nz)))
    return out


def fields_for(wl: Workload):
    if wl.kind == "shear":
        return shear_fields(wl.nx, wl.ny, wl.nz, wl.seed)
    return wind_fields(wl.nx, wl.ny, wl.nz, wl.seed)


@dataclass
class Member:
    nx: int
    ny: int
    nz: int
    dx: float
    seed: int


def ensemble(n=64, seed=ENSEMBLE_SEED, sizes=(32, 384), levels=(64, 160)):
    """n members with nx, ny drawn uniformly from the multiples of 8 in `sizes`,
    nz uniform in `levels`, dx = dy uniform in [25, 100] m."""
    rng = np.random.default_rng(seed)
    choices = np.arange(sizes[0], sizes[1] + 1, 8)
    out = []
    for m in range(n):
        nx = int(rng.choice(choices))
        ny = int(rng.choice(choices))
        nz = int(rng.integers(levels[0], levels[1] + 1))
        dx = float(rng.uniform(25.0, 100.0))
        out.append(Member(nx, ny, nz, dx, seed * 1000 + m))
    return out
