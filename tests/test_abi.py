"""The C-ABI library builds for sm_103a, loads, and exports every symbol esdcg.h declares
(no GPU needed: no compute call is made)."""
import ctypes
import re

import paper_2203_08498_gb300 as esd


def test_library_exports_every_declared_symbol():
    L = esd.lib()
    assert len(esd.HEADER_SYMBOLS) >= 20
    for name in esd.HEADER_SYMBOLS:
        assert hasattr(L, name), name


def test_binding_covers_the_header():
    for name in esd.HEADER_SYMBOLS:
        assert hasattr(esd, name), f"binding lacks {name}"


def test_params_default_without_gpu():
    p = esd.esd_params_default()
    assert p.precond == esd.PRECOND_IC0 and p.maxit_cap == 20000 and p.rank_tol == 1e-12
