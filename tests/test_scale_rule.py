"""Host logic of the float16 storage scale (BP_OPT_PROJ_SCALE): the rule that
picks the power of four from a batch's max|p| (proj_scale_k), compiled for
the host from the library's own header and checked over every float
exponent -- no GPU needed."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_scale_rule_puts_the_maximum_in_its_band(tmp_path):
    nvcc = shutil.which("nvcc") or os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = tmp_path / "scale_rule_check"
    subprocess.check_call([nvcc, "-std=c++17", "-O1", "-x", "cu", os.path.join(HERE, "scale_rule_check.cu"),
                           "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout
    assert out.stdout.startswith("ok ")
    assert int(out.stdout.split()[1]) > 1000
