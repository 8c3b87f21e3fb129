"""Host builds of the CUDA path's element header (plain C++ outside nvcc),
without a GPU: the element tangent against central differences of the element
residual, its transpose, diagonal, linearisation-store and design-sensitivity
variants against it (tests/host/element_consistency_check.cpp), and the
specialised element columns of the assembled Jacobian against the general
products (tests/host/element_columns_check.cpp), and the packed-pair FP32
products against the scalar ones (tests/host/element_pairs_check.cpp)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("prog", ["element_consistency_check", "element_columns_check",
                                  "element_pairs_check"])
def test_element_routines_on_the_host(tmp_path, prog):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / prog)
    subprocess.run([cxx, "-std=c++17", "-O1", os.path.join(HERE, "host", prog + ".cpp"), "-o", exe],
                   check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
