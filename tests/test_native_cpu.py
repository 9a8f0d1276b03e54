"""Host-compiled checks of device building blocks (no GPU needed): the
in-register DFT of the FFT passes against the DFT definition."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="needs nvcc")
def test_register_dft_matches_definition():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "reg_dft_check")
        subprocess.run([nvcc, "-std=c++17", "-O2", "-o", exe,
                        os.path.join(HERE, "native", "reg_dft_check.cu")], check=True,
                       capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    vals = dict(line.split() for line in out.strip().splitlines())
    assert float(vals["max_rel_err_f32"]) < 1e-6
    assert float(vals["max_rel_err_f64"]) < 1e-14
