"""The MUFU rates behind the compositing kernels' SFU roofline (bench.py: 32 ex2 and
16 rcp results per SM and clock, against 128 FP32 FMA lanes): measured by the
throughput loops of tests/alu_rates.cu and compared as clock-free ratios."""
import json
import os
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.gpu
def test_mufu_rates_relative_to_fp32_fma():
    import bench
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "alu_rates")
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                        os.path.join(HERE, "alu_rates.cu")], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120).stdout
    r = json.loads(out.strip().splitlines()[-1])
    print(r)
    assert r["status"] == "no error" and r["sms"] == bench.SMS
    fma_lanes = bench.FP32_LANES_PER_SM
    assert r["ex2_per_s"] / r["fma_per_s"] == pytest.approx(bench.MUFU_EX2_PER_SM_CLK / fma_lanes, rel=0.15)
    assert r["rcp_per_s"] / r["fma_per_s"] == pytest.approx(bench.MUFU_RCP_PER_SM_CLK / fma_lanes, rel=0.15)
