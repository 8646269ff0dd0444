"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/bonsai_gb.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bonsai_gb.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "defined")))


@pytest.fixture(scope="module")
def lib():
    from paper_1412_0659_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_path():
    names = _declared()
    for n in ("tree_build", "tree_forces", "tree_step", "bonsai_create", "bonsai_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_1412_0659_gb300 import capi
    assert sorted(capi.EXPORTED) == _declared()


def test_strerror_without_gpu(lib):
    lib.bonsai_strerror.restype = ctypes.c_char_p
    assert lib.bonsai_strerror(0) == b"ok"
    assert lib.bonsai_strerror(-3) == b"walk buffer overflow"


def test_null_arguments_are_rejected_without_touching_the_device(lib):
    # argument checks run before any CUDA call
    assert lib.bonsai_create(None, None, None) == -1
    assert lib.tree_build(None, None, None, ctypes.c_int64(10)) == -1
    assert lib.tree_forces(None, ctypes.c_float(0.4), ctypes.c_float(0.01), None, None) == -1
    assert lib.tree_step(None, ctypes.c_double(0.1)) == -1


def test_product_path_has_no_cpu_fallback(tmp_path):
    """The binding refuses to run when the CUDA library is absent."""
    from paper_1412_0659_gb300 import capi
    with pytest.raises(RuntimeError, match="not built"):
        capi._lib, saved = None, capi._lib
        try:
            capi.load(str(tmp_path / "missing.so"))
        finally:
            capi._lib = saved


def test_product_sources_do_not_reference_the_oracle():
    pkg = os.path.join(ROOT, "paper_1412_0659_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "bonsai_oracle" not in txt, f


def test_galaxy_parameters_and_checks_without_gpu():
    """bonsai_galaxy_sec4 is host code: the Sec. IV counts for n particles
    (those of the oracle's generator), and the generator's argument checks
    reject bad models before any CUDA call."""
    from oracle import galaxy_ics as gi
    from paper_1412_0659_gb300 import capi
    for n in (1000, 1 << 20, (1 << 32) - 1):
        g = capi.bonsai_galaxy_sec4(n, 7)
        assert (g.n_halo, g.n_disk, g.n_bulge) == gi.counts(n)
        o = gi.milky_way_sec4(n, 7)
        for k in ("G", "M_halo", "a_halo", "M_bulge", "a_bulge", "r_t", "dr_t", "M_disk", "R_d",
                  "z0", "R_max", "Q", "R_Q"):
            assert getattr(g, k) == getattr(o, k), k
    for n in (0, -5, 1 << 32):
        with pytest.raises(capi.BonsaiError):
            capi.bonsai_galaxy_sec4(n, 1)
    lib = capi.load()
    for field, value in (("n_halo", -1), ("a_bulge", 0.0), ("Q", float("nan")), ("M_disk", 0.0),
                         ("R_Q", -1.0), ("G", float("inf"))):
        g = capi.bonsai_galaxy_sec4(4096, 1)
        setattr(g, field, value)
        rc = lib.bonsai_galaxy_generate(ctypes.byref(g), None, None, None, None)
        assert rc == capi.BONSAI_EINVAL, field
    g = capi.bonsai_galaxy_sec4(4096, 1)
    assert lib.bonsai_galaxy_generate(ctypes.byref(g), None, None, None, None) == capi.BONSAI_EINVAL
