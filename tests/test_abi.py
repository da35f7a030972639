"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every function include/etdrdpif.h declares, and rejects invalid
problems before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2001_11220_gb300 import _binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2001_11220_gb300 import build
    build.build()
    return B.load()


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(etd_[a-z_0-9]+)\s*\(", txt)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(B.EXPORTS) == names


def _create(lib, n=(8, 8), bc=(0, 0), D=(0.1,), kind=0, ns=None, k=0.1, prec=0, length=None):
    from paper_2001_11220_gb300.api import make_grid, make_reaction
    g = make_grid(n, bc, length)
    r = make_reaction(kind, len(D) if ns is None else ns, (1.0, 2.0))
    Darr = (ctypes.c_double * max(1, len(D)))(*D)
    ctx = ctypes.c_void_p()
    st = lib.etd_create(ctypes.byref(g), Darr, ctypes.byref(r), k, prec, None, ctypes.byref(ctx))
    return st, ctx


@pytest.mark.parametrize("kw,status", [
    (dict(n=(2, 8)), B.ETD_ERR_INVALID_ARG),
    (dict(n=(8, 20000)), B.ETD_ERR_INVALID_ARG),
    (dict(bc=(0, 3)), B.ETD_ERR_INVALID_ARG),
    (dict(D=(-1.0,)), B.ETD_ERR_INVALID_ARG),
    (dict(D=(float("nan"),)), B.ETD_ERR_INVALID_ARG),
    (dict(k=0.0), B.ETD_ERR_INVALID_ARG),
    (dict(k=float("inf")), B.ETD_ERR_INVALID_ARG),
    (dict(prec=7), B.ETD_ERR_INVALID_ARG),
    (dict(kind=2, D=(0.1,)), B.ETD_ERR_INVALID_ARG),       # Brusselator needs two species
    (dict(kind=5, D=(0.1, 0.2)), B.ETD_ERR_INVALID_ARG),   # enzyme needs one species
    (dict(kind=9), B.ETD_ERR_INVALID_ARG),
    (dict(D=(0.1, 0.1, 0.1), kind=1), B.ETD_ERR_UNSUPPORTED),
    (dict(length=(1.0, -1.0)), B.ETD_ERR_INVALID_ARG),
])
def test_create_rejects_invalid_problems(lib, kw, status):
    st, ctx = _create(lib, **kw)
    assert st == status, lib.etd_last_error(None)
    assert not ctx.value
    assert lib.etd_last_error(None)


def _create_coupled(lib, Dm, kind=6, ns=2, n=(8, 8), bc=(2, 2)):
    from paper_2001_11220_gb300.api import make_grid, make_reaction
    g = make_grid(n, bc)
    r = make_reaction(kind, ns, (1.3,))
    Darr = (ctypes.c_double * 4)(*Dm)
    ctx = ctypes.c_void_p()
    return lib.etd_create_coupled(ctypes.byref(g), Darr, ctypes.byref(r), 0.05, 0, None, ctypes.byref(ctx)), ctx


@pytest.mark.parametrize("kw,status", [
    (dict(Dm=(1.0, -0.5, 0.4, 1.0)), B.ETD_ERR_UNSUPPORTED),      # not of the form [[p, -q], [q, p]]
    (dict(Dm=(1.0, 0.0, 0.0, 2.0)), B.ETD_ERR_UNSUPPORTED),       # diagonal but unequal
    (dict(Dm=(-1.0, -0.5, 0.5, -1.0)), B.ETD_ERR_INVALID_ARG),    # real part p < 0
    (dict(Dm=(1.0, float("nan"), 0.5, 1.0)), B.ETD_ERR_INVALID_ARG),
    (dict(Dm=(1.0, -0.5, 0.5, 1.0), kind=2), B.ETD_ERR_UNSUPPORTED),  # Brusselator: not a coupled reaction
    (dict(Dm=(1.0, -0.5, 0.5, 1.0), ns=1), B.ETD_ERR_INVALID_ARG),
    (dict(Dm=(1.0, -0.5, 0.5, 1.0), n=(2, 8)), B.ETD_ERR_INVALID_ARG),
    (dict(Dm=(0.0, -1.0, 1.0, 0.0), n=(2,), bc=(1,)), B.ETD_ERR_INVALID_ARG),  # d = 1 line of 2 nodes
])
def test_create_coupled_rejects_before_any_device_call(lib, kw, status):
    st, ctx = _create_coupled(lib, **kw)
    assert st == status, lib.etd_last_error(None)
    assert not ctx.value


def test_schrodinger_reaction_needs_the_coupled_create(lib):
    st, ctx = _create(lib, D=(1.0, 1.0), kind=7)
    assert st == B.ETD_ERR_UNSUPPORTED and not ctx.value
    assert b"coupled" in lib.etd_last_error(None)


def test_dim_must_be_2_or_3(lib):
    g = B.etd_grid()
    g.dim = 4
    r = B.etd_reaction()
    r.nspecies = 1
    D = (ctypes.c_double * 1)(0.1)
    ctx = ctypes.c_void_p()
    assert lib.etd_create(ctypes.byref(g), D, ctypes.byref(r), 0.1, 0, None, ctypes.byref(ctx)) == B.ETD_ERR_INVALID_ARG
    assert b"dim" in lib.etd_last_error(None)


def test_null_arguments(lib):
    assert lib.etd_step(None, None, 0.0) == B.ETD_ERR_INVALID_ARG
    assert lib.etd_run(None, None, 0.0, 1) == B.ETD_ERR_INVALID_ARG
    assert lib.etd_get_info(None, None) == B.ETD_ERR_INVALID_ARG
    assert lib.etd_check_finite(None, None, None) == B.ETD_ERR_INVALID_ARG
    lib.etd_destroy(None)
    assert lib.etd_last_error(None)


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2001_11220_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "etd_oracle" not in txt, f
