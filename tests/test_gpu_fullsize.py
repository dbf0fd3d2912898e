"""Parity at the full sizes the benchmark runs, in its launch configuration
(default tiles, halo fill by the library, then the stencil): EVERY output point
of the 1024x1024x128 bandwidth workload and of the 512x512x160 precision
workload against the FP64 oracle (all host cores).

FP64 (split and native): within 1e-12, normwise and of each point's condition
sum.  Reduced-precision storage is checked twice: against the oracle on the
values the kernel sees (the inputs rounded to the storage type: the arithmetic
error, 16 units of 2^-24 of the condition sum) and against the oracle on the
original FP64 fields (the total error including the storage rounding:
(2u + u^2) cond + the arithmetic error, u the storage unit roundoff, plus the
output rounding for bfloat16 sources)."""
import gc

import numpy as np
import pytest
import torch

import oracle
from paper_2009_12850_b300 import synthetic

from parity import TOL_F32_COND, TOL_F64, compare_slabs, tol_unrounded

pytestmark = pytest.mark.gpu

WORKLOADS = {"bandwidth": synthetic.LARGE, "precision": synthetic.PRECISION}


@pytest.fixture(scope="module")
def pw():
    from paper_2009_12850_b300 import build
    build.build()
    from paper_2009_12850_b300 import api
    oracle.set_threads(0)   # every host core
    return api


class _Refs:
    """FP64 oracle results per workload, computed once and kept for the module."""

    def __init__(self):
        self.cache = {}

    def get(self, key):
        if key not in self.cache:
            self.cache.clear()
            gc.collect()
            wl = WORKLOADS[key]
            f = synthetic.fields_for(wl)
            c = oracle.Coeffs(wl.nz, wl.dx, wl.dy)
            ref, cond = oracle.advect(c, *f, want_cond=True)
            self.cache[key] = (wl, f, c, ref, cond)
        return self.cache[key]


@pytest.fixture(scope="module")
def refs():
    return _Refs()


def rounded(arrs, dtype):
    t = {"f32": torch.float32, "bf16": torch.bfloat16, "bf16_out": torch.bfloat16}[dtype]
    return [torch.from_numpy(a).to(t).to(torch.float64).numpy() for a in arrs]


def run_bench_config(pw, wl, fields, dtype, algo):
    """Halo fill by the library then the stencil, default tiles (the bench's launch)."""
    m = pw.Mesh(wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, dtype=dtype, algo=algo)
    U = [m.from_interior(a, fill_halo=False) for a in fields]
    S = [m.empty_out() for _ in range(3)]
    m.halo(*U)
    m.advect(*U, *S)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    got = [m.interior(s).double().cpu().numpy() for s in S]
    del U, S, m
    torch.cuda.empty_cache()
    return got


CASES = [("bandwidth", "f64", "auto"), ("bandwidth", "f64", "native"), ("bandwidth", "f32", "auto"),
         ("bandwidth", "bf16", "auto"), ("bandwidth", "bf16_out", "auto"), ("precision", "f64", "auto"), ("precision", "f32", "auto"),
         ("precision", "bf16", "auto"), ("precision", "bf16_out", "auto")]


@pytest.mark.parametrize("key,dtype,algo", CASES, ids=lambda x: str(x))
def test_full_size_every_point(pw, refs, key, dtype, algo):
    wl, f, c, ref, cond = refs.get(key)
    if dtype == "f64":
        got = run_bench_config(pw, wl, f, dtype, algo)
        for q in range(3):
            compare_slabs(f"{key} {dtype}/{algo} s{'uvw'[q]}", got[q], ref[q], cond[q], TOL_F64, TOL_F64)
        return
    fr = rounded(f, dtype)
    got = run_bench_config(pw, wl, fr, dtype, algo)
    # total error against the oracle on the original fields (the bound is
    # pointwise in the condition sum; the normwise figure is only reported)
    tu = tol_unrounded(dtype)
    for q in range(3):
        compare_slabs(f"{key} {dtype} s{'uvw'[q]} vs unrounded", got[q], ref[q], cond[q], np.inf, tu)
    # arithmetic error against the oracle on the rounded fields
    ref_r, cond_r = oracle.advect(c, *fr, want_cond=True)
    del fr
    out_round = 2.0 ** -8 if dtype == "bf16_out" else 0.0     # bfloat16 sources (unit roundoff)
    tc = TOL_F32_COND + out_round * (1 + TOL_F32_COND)
    for q in range(3):
        compare_slabs(f"{key} {dtype} s{'uvw'[q]} vs rounded", got[q], ref_r[q], cond_r[q], 1e-5 + out_round, tc)
