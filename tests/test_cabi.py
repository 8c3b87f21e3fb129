"""CPU checks of the C-ABI library: it builds, loads, and exports every function
that include/nc.h declares; size queries work without a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "nc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nc_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1508_04596_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared()
    for n in ("nc_setup", "nc_residual", "nc_jvp", "nc_jtvp", "nc_newton_solve",
              "nc_adjoint_solve", "nc_sensitivity", "nc_objective"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_sizes_without_device(lib):
    from paper_1508_04596_gb300 import nc
    p = nc.make_params(192, 192, 384, 1 / 192, 1e6, 0.71)
    nn, ne, nd = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
    assert nc.lib.nc_sizes(ctypes.byref(p), ctypes.byref(nn), ctypes.byref(ne), ctypes.byref(nd)) == 0
    assert (nn.value, ne.value, nd.value) == (14_340_865, 14_155_776, 71_704_325)
    bad = nc.make_params(0, 1, 1, 1.0, 1.0, 1.0)
    assert nc.lib.nc_sizes(ctypes.byref(bad), None, None, None) == 1
    assert nc.lib.nc_status_string(4) == b"non-finite value"


def test_default_opts(lib):
    from paper_1508_04596_gb300 import nc
    o = nc.default_opts()
    assert (o.rtol_newton, o.rtol_lin, o.restart, o.mixed) == (1e-8, 1e-5, 30, 1)
    assert (o.galerkin, o.assembled, o.rtol_adjoint) == (0, 0, 1e-10)


@pytest.mark.parametrize("struct,fill,last", [("SolveOpts", "nc_default_opts", "adjoint_start"),
                                             ("MmaOpts", "nc_default_mma_opts", "df0_scale")])
def test_option_structs_match_the_header(lib, struct, fill, last):
    """The ctypes mirrors of the option structs have the C layout: the library's
    default-filling call writes the mirror's last field and nothing beyond it."""
    from paper_1508_04596_gb300 import nc
    T = getattr(nc, struct)
    n = ctypes.sizeof(T)
    buf = (ctypes.c_ubyte * (n + 64))(*([0xA5] * (n + 64)))
    o = T.from_buffer(buf)
    getattr(nc.lib, fill)(ctypes.byref(o))
    assert bytes(buf[n:]) == b"\xa5" * 64
    ref = T()
    getattr(nc.lib, fill)(ctypes.byref(ref))
    assert getattr(o, last) == getattr(ref, last) and getattr(ref, last) != getattr(
        T.from_buffer_copy(b"\xa5" * n), last)


def test_quarter_workloads_have_the_papers_sizes(lib):
    """The quarter-cavity workloads are the paper's three meshes (Sec. 6.2-6.4,
    tests/golden/paper_dof_counts.txt, the paper's middle index vertical there
    and z here): nc_sizes gives the printed DOF and element counts."""
    from paper_1508_04596_gb300 import nc, synth
    path = os.path.join(ROOT, "tests", "golden", "paper_dof_counts.txt")
    printed = {(int(r[0]), int(r[2]), int(r[1])): (int(r[3]), int(r[4]))
               for r in (l.split() for l in open(path) if l.strip() and not l.startswith("#"))}
    seen = set()
    for name, cfg in synth.WORKLOADS.items():
        if cfg.get("bcs") != "quarter":
            continue
        key = (cfg["nx"], cfg["ny"], cfg["nz"])
        p = nc.make_params(*key, cfg["h"], cfg["Gr"], cfg["Pr"])
        nn, ne, nd = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        assert nc.lib.nc_sizes(ctypes.byref(p), ctypes.byref(nn), ctypes.byref(ne), ctypes.byref(nd)) == 0
        assert (nd.value, ne.value) == printed[key], name
        assert cfg["h"] * cfg["nz"] == pytest.approx(1.0)  # unit cavity height
        seen.add(key)
    assert len(seen) == 3


def test_fma_probe_rejects_invalid_arguments(lib):
    """nc_fma_probe checks its arguments before touching the device: an unknown
    precision, no blocks, an iteration count that is not a positive multiple of
    16 or a NULL output are NC_ERR_ARG (no GPU needed)."""
    f = lib.nc_fma_probe
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p]
    dummy = ctypes.c_void_p(16)  # never dereferenced: every call below is rejected first
    assert f(7, 1, 16, dummy, None) == 1
    assert f(0, 0, 16, dummy, None) == 1
    assert f(1, 1, 15, dummy, None) == 1
    assert f(1, 1, 0, dummy, None) == 1
    assert f(0, 1, 16, None, None) == 1
