"""Host builds of the CUDA path's element header (plain C++ outside nvcc),
without a GPU: the element tangent against central differences of the element
residual, its transpose, diagonal, linearisation-store and design-sensitivity
variants against it (tests/host/element_consistency_check.cpp), and the
specialised element columns of the assembled Jacobian against the general
products (tests/host/element_columns_check.cpp), the packed-pair FP32
products against the scalar ones (tests/host/element_pairs_check.cpp), the
element rows against the oracle, and the benchmark's per-element flop figures
against a count of the routines (tests/host/element_flop_count.cpp)."""
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


def test_element_rows_match_the_oracle(tmp_path):
    """The CUDA path's element routines (host build) against the oracle's element
    residual and its complex-step Jacobian, element by element: the residual rows,
    J v and J^T v in FP64 to 1e-13 of the largest row, and the FP32 packed-pair
    J v and J^T v to 2e-6 (FP32 rounding of the inputs and of about 10^2 terms per
    row).  Seeded random elements, parameters (with the benchmark's and the quarter
    cavity's materials), gravity directions and sources.  Unlike the consistency
    checks above, this catches an error shared by the residual and its
    derivatives (a weight, a sign, a transposed index)."""
    import numpy as np
    from oracle import element as El
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "rows")
    subprocess.run([cxx, "-std=c++17", "-O1", os.path.join(HERE, "host", "element_rows_print.cpp"),
                    "-o", exe], check=True)
    rng = np.random.default_rng(5150)
    cases, lines = [], []
    for t in range(24):
        h = 1.0 / (4 + 7 * t)
        Gr, Pr = 10.0 ** (2 + t % 5), (0.71, 1.0)[t % 2]
        am, qa, qf, Ck = ((1e4, 1.0, 1.0, 0.1), (1e5, 8.0, 0.881, 1e-2))[t % 2]
        eg = ((0.0, 0.0, -1.0), (0.0, -1.0, 0.0), (0.6, 0.0, -0.8))[t % 3]
        gam = 0.05 + 0.9 * rng.uniform()
        s = (0.0, 1e4 * rng.uniform())[t % 2]
        x = rng.standard_normal((8, 5)) * np.array([0.5, 0.5, 0.5, 50.0, 1.0])
        v = rng.standard_normal((8, 5))
        x32, v32 = x.astype(np.float32).astype(float), v.astype(np.float32).astype(float)
        cases.append((El.Params(h, Gr, Pr, am, qa, qf, Ck, eg), gam, s, x, v, x32, v32))
        lines.append(" ".join("%.17g" % z for z in (h, Gr, Pr, am, qa, qf, Ck) + eg + (gam, s)))
        lines.append(" ".join("%.17g" % z for z in x32.ravel()))
        lines.append(" ".join("%.17g" % z for z in v32.ravel()))
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                       check=True)
    out = np.array([[float(z) for z in l.split()] for l in r.stdout.strip().splitlines()])
    assert out.shape == (5 * len(cases), 40)
    eye = np.eye(40).reshape(40, 8, 5)
    for k, (prm, gam, s, x, v, x32, v32) in enumerate(cases):
        se = np.array([s])
        R = El.element_residual(x32[None], np.array([gam]), prm, se=se)[0].ravel()
        Jc = El.element_residual(x32[None] + 1e-30j * eye, np.full(40, gam), prm,
                                 se=np.full(40, s)).imag.reshape(40, 40) / 1e-30
        J = Jc.T  # J[row, col]
        vv = v32.ravel()
        refs = [R, J @ vv, J.T @ vv, J @ vv, J.T @ vv]
        tols = [1e-13, 1e-13, 1e-13, 2e-6, 2e-6]
        for q, (ref, tol) in enumerate(zip(refs, tols)):
            got = out[5 * k + q]
            err = np.abs(got - ref).max() / np.abs(ref).max()
            assert err <= tol, (k, q, err)


def test_flop_counts_match_the_benchmark(tmp_path):
    """The per-element operation counts that the benchmark's ALU roofline divides
    by the measured time are those of the element routines as they stand: the
    routines instantiated with a counting number type
    (tests/host/element_flop_count.cpp) give exactly bench.FLOPS_PER_ELEM."""
    import importlib.util
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "flops")
    subprocess.run([cxx, "-std=c++17", "-O1", os.path.join(HERE, "host", "element_flop_count.cpp"),
                    "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, check=True)
    counts = {l.split()[0]: int(l.split()[1]) for l in r.stdout.strip().splitlines()}
    spec = importlib.util.spec_from_file_location("bench_consts", os.path.join(HERE, "..", "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    assert counts == bench.FLOPS_PER_ELEM
