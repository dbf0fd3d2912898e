"""Helpers shared by the GPU parity tests: tolerances and comparisons of the
CUDA results (through the C-ABI) against the FP64 oracle."""
import numpy as np

import oracle

U32 = 2.0 ** -24
# FP64 target of the stencil: 1e-12 relative, normwise per field and pointwise
# against the condition sum (sum of |elementary products|) of each point.
TOL_F64 = 1e-12
# FP32 arithmetic on exactly-representable inputs: a handful of roundings per
# term (face sum, two products, coefficient, <= 6 accumulations).
TOL_F32_COND = 16 * U32


def coeffs_for(mesh_like, nz, dx, dy=None, dz=None, rho_n=None, rho_w=None, rho0=1.2, H=8000.0):
    return oracle.Coeffs(nz, dx, dx if dy is None else dy, dz=dz, rho_n=rho_n, rho_w=rho_w, rho0=rho0, H=H)


def compare(name, got, ref, cond, tol_norm, tol_cond):
    got = np.asarray(got, dtype=np.float64)
    err = np.abs(got - ref)
    scale = np.abs(ref).max()
    norm_rel = err.max() / scale if scale > 0 else err.max()
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(cond > 0, err / cond, np.where(err > 0, np.inf, 0.0))
    worst = float(ratio.max())
    assert norm_rel <= tol_norm, f"{name}: normwise {norm_rel:.3e} > {tol_norm:.1e}"
    assert worst <= tol_cond, f"{name}: pointwise err/cond {worst:.3e} > {tol_cond:.1e}"
    return {"max_abs": float(err.max()), "rms": float(np.sqrt(np.mean(err ** 2))),
            "norm_rel": float(norm_rel), "max_err_over_cond": worst}
