"""The C-ABI library builds for sm_103a, loads without a GPU and exports every entry point
that include/esi.h declares; argument validation needs no device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"ESI_API\s+[\w\s\*]+?\b(esi_\w+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2211_06300_gb300 import build, esi
    build.build()
    return esi.load_library(require_gpu=False)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["esi_create", "esi_forward", "esi_adjoint", "esi_gradient", "esi_dft_extract",
              "esi_cg_solve", "esi_pc_load", "esi_destroy", "esi_status_string", "esi_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2211_06300_gb300 import esi
    for n in _declared():
        assert hasattr(lib, n), n
    assert set(esi.EXPORTS) == set(_declared())


def test_status_strings_and_argument_checks_need_no_gpu(lib):
    from paper_2211_06300_gb300 import esi
    assert lib.esi_status_string(0) == b"ok"
    assert lib.esi_status_string(esi.ESI_ERR_CFL).startswith(b"time step")
    h = ctypes.c_void_p()
    assert lib.esi_create(ctypes.byref(h), None, None, None, 1e-3, 10, None) == esi.ESI_ERR_ARG
    g = esi.EsiGrid(ndim=4, nz=1, ny=1, nx=1, dx=1.0, nb=0, sponge_R=0.1, sponge_vref=1.0,
                    dtype=0)
    gm = esi.EsiGeometry(ns=0)
    st = lib.esi_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(gm),
                        ctypes.c_void_p(16), 1e-3, 10, None)
    assert st == esi.ESI_ERR_ARG
    assert lib.esi_forward(None, None, None, None) == esi.ESI_ERR_ARG
    assert lib.esi_set_shot_groups(None, 2, None) == esi.ESI_ERR_ARG
    assert lib.esi_launch_count(None) == 0
