"""Arithmetic rates that shape the FP64 design, measured on the device by the
package's rate microbenchmark (paper_2009_12850_b300/rates/fp_rates.cu, also run
by `bench.py --fp-rates`): FP64 FMA and f64->f32 conversion are ~60x slower than
FP32 FMA on B300, while packed FP32x2 FMA keeps the FP32 lane rate (so
double-float arithmetic on the FP32 pipe beats native FP64).  Prints the
measured rates (run with -s)."""
import json
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2009_12850_b300", "rates", "fp_rates.cu")


def test_fp_rates(tmp_path):
    exe = str(tmp_path / "fp_rates")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                    SRC], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    r = json.loads(out)
    print(json.dumps(r, indent=1))
    assert r["ffma_per_clk_sm"] > 64
    assert r["ffma2_lanes_per_clk_sm"] > 0.8 * r["ffma_per_clk_sm"]
    assert r["dfma_per_clk_sm"] < r["ffma_per_clk_sm"] / 16
    assert r["cvt_f64_f32_per_clk_sm"] < r["ffma_per_clk_sm"] / 16
