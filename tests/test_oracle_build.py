"""The oracle build itself (CPU): the OpenMP sweep gives bit-identical results
on any number of threads, so the timed all-core oracle is the reference
oracle; and a build with floating-point contraction on (FMA), i.e. another
rounding order of the same formulas, stays within a few units of 2^-52 of the
condition sum -- far below the 1e-12 parity tolerance -- so the tolerance
measures the GPU kernels, not the oracle's own order of evaluation."""
import os
import subprocess

import numpy as np

import oracle
from paper_2009_12850_b300 import synthetic


def _fields(seed=5, shape=(23, 17, 19)):
    return synthetic.wind_fields(*shape, seed), synthetic.scalar_fields(*shape, 2, seed + 1)


def test_threads_give_identical_results():
    (u, v, w), phis = _fields()
    c = oracle.Coeffs(u.shape[2], 40.0, 30.0)
    n_all = oracle.set_threads(os.cpu_count() or 1)
    try:
        many = oracle.advect(c, u, v, w)
        many_phi = [oracle.advect_scalar(c, u, v, w, p) for p in phis]
        oracle.set_threads(1)
        one = oracle.advect(c, u, v, w)
        one_phi = [oracle.advect_scalar(c, u, v, w, p) for p in phis]
    finally:
        oracle.set_threads(n_all)
    for a, b in zip(list(many) + many_phi, list(one) + one_phi):
        assert np.array_equal(a, b)


def test_contracted_build_agrees_far_below_tolerance(tmp_path):
    (u, v, w), phis = _fields(seed=7)
    nz = u.shape[2]
    ref_c = oracle.Coeffs(nz, 40.0, 30.0)
    ref, cond = oracle.advect(ref_c, u, v, w, want_cond=True)
    ref_phi = [oracle.advect_scalar(ref_c, u, v, w, p, want_cond=True) for p in phis]
    src = os.path.join(os.path.dirname(oracle.__file__), "pw_oracle.c")
    so = tmp_path / "libfma.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=fast", "-march=native", "-fPIC", "-shared", "-o", str(so),
                    src, "-lm"], check=True)
    with oracle.use_library(str(so)):
        c = oracle.Coeffs(nz, 40.0, 30.0)
        got = oracle.advect(c, u, v, w)
        got_phi = [oracle.advect_scalar(c, u, v, w, p) for p in phis]
    worst = 0.0
    for g, r, k in list(zip(got, ref, cond)) + [(g, r, k) for g, (r, k) in zip(got_phi, ref_phi)]:
        worst = max(worst, float(np.max(np.abs(g - r) / np.maximum(k, 1e-300))))
    assert worst <= 64 * 2.0 ** -52, worst      # a few ulps of the condition sum
    assert worst < 1e-12 / 100                  # two orders below the parity tolerance
