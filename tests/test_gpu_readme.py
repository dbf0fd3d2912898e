"""The quick-start example of README.md runs as written, and its results agree
with the FP64 oracle."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2009_12850_b300 import synthetic

from parity import TOL_F64, compare

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_quick_start_runs():
    from paper_2009_12850_b300 import build
    build.build()
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, flags=re.S)
    assert blocks, "README.md has no python example"
    scope = {}
    exec(compile(blocks[0], "README.md", "exec"), scope)
    m, su, sv, sw = scope["m"], scope["su"], scope["sv"], scope["sw"]
    nx, ny, nz = scope["nx"], scope["ny"], scope["nz"]
    assert m.device_status() == 0
    f = synthetic.wind_fields(nx, ny, nz, seed=1)
    # the example's sources against the oracle on the same seeded fields
    ref, cond = oracle.advect(oracle.Coeffs(nz, 25.0, 25.0), *f, want_cond=True)
    for name, got, r, c in zip(("su", "sv", "sw"), (su, sv, sw), ref, cond):
        compare(name, m.interior(got).double().cpu().numpy(), r, c, TOL_F64, TOL_F64)
    assert len(scope["s_phi"]) == 6
    assert all(np.isfinite(m.interior(t).double().cpu().numpy()).all() for t in scope["s_phi"])
    # the ULTIMATE-QUICKEST sources of theta against the oracle
    theta = synthetic.scalar_fields(nx, ny, nz, 6, seed=2)[0]
    ref, cond = oracle.advect_tvd(oracle.Coeffs(nz, 25.0, 25.0), *f, theta, 2.0, want_cond=True)
    compare("s_tvd", m.interior(scope["s_tvd"][0]).double().cpu().numpy(), ref, cond, TOL_F64, TOL_F64)
