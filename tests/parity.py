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


def compare_slabs(name, got, ref, cond, tol_norm, tol_cond, slabs=16):
    """compare() over (nx, ny, nz) arrays of any size, one x slab at a time (the
    full-size fields are GBs; this keeps the temporaries to one slab).  Every
    point is checked."""
    nx = ref.shape[0]
    edges = np.linspace(0, nx, min(slabs, nx) + 1).astype(int)
    scale = max(float(np.abs(ref[a:b]).max()) for a, b in zip(edges[:-1], edges[1:]))
    emax, worst, sq = 0.0, 0.0, 0.0
    for a, b in zip(edges[:-1], edges[1:]):
        err = np.abs(np.asarray(got[a:b], dtype=np.float64) - ref[a:b])
        c = cond[a:b]
        with np.errstate(divide="ignore", invalid="ignore"):
            ratio = np.where(c > 0, err / c, np.where(err > 0, np.inf, 0.0))
        emax = max(emax, float(err.max()))
        worst = max(worst, float(ratio.max()))
        sq += float(np.sum(err * err))
    norm_rel = emax / scale if scale > 0 else emax
    assert norm_rel <= tol_norm, f"{name}: normwise {norm_rel:.3e} > {tol_norm:.1e}"
    assert worst <= tol_cond, f"{name}: pointwise err/cond {worst:.3e} > {tol_cond:.1e}"
    return {"max_abs": emax, "rms": (sq / ref.size) ** 0.5, "norm_rel": norm_rel, "max_err_over_cond": worst}


# Storage rounding.  An input stored with unit roundoff u perturbs each
# elementary product c phi (a1 + a2) by at most (2u + u^2) c |phi| (|a1| + |a2|),
# so against the FP64 oracle evaluated on the UNROUNDED fields the total error of
# a reduced-precision result is bounded by (2u + u^2) cond + the arithmetic error
# on the rounded values (TOL_F32_COND times their condition sum, at most
# (1 + u)^2 cond).  Rounding a source to bfloat16 adds at most 2^-8 |S|.
# (bfloat16: a conversion that rounds through FP32 first may add 2^-24 more)
U_STORE = {"f32": 2.0 ** -24, "bf16": 2.0 ** -8 + 2.0 ** -24, "bf16_out": 2.0 ** -8 + 2.0 ** -24}


def tol_unrounded(dtype):
    u = U_STORE[dtype]
    t = 2 * u + u * u + TOL_F32_COND * (1 + u) ** 2
    if dtype == "bf16_out":      # |S| <= cond, so the output rounding is <= 2^-8 (1 + t) cond
        t += 2.0 ** -8 * (1 + t)
    return t
