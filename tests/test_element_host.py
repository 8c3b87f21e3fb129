"""Host build of the CUDA path's element header: the specialised element
columns of the assembled Jacobian equal the general element products
(tests/host/element_columns_check.cpp), without a GPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_element_columns_match_general_products(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "element_columns_check")
    subprocess.run([cxx, "-std=c++17", "-O1", os.path.join(HERE, "host", "element_columns_check.cpp"),
                    "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert float(r.stdout.strip()) <= 1e-12
