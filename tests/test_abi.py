"""The C-ABI library builds, loads and exports every symbol include/ppr.h
declares; host-only entry points behave without a GPU."""
import ctypes as C
import math
import os
import re
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1903_11749_gb300 import build as B
    B.build()
    from paper_1903_11749_gb300 import ppr
    return ppr.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ppr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(ppr_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("ppr_load_graph", "ppr_run", "ppr_topk", "ppr_sparse_rows", "ppr_wait", "ppr_create"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    from paper_1903_11749_gb300 import ppr
    assert set(declared_functions()) == set(ppr._SIGS)


def test_version(lib):
    assert lib.ppr_version() == 1


def test_threshold_matches_definition(lib):
    rng = np.random.Generator(np.random.PCG64(3))
    for a in list(rng.random(300)) + [0.15, 0.2, 0.5]:
        assert lib.ppr_alpha_threshold(float(a)) == math.floor(Fraction(float(a)) * 2**32)
    for bad in (0.0, 1.0, -1.0, 2.0**-40, float("nan"), float("inf")):
        assert lib.ppr_alpha_threshold(bad) == 0


def test_create_without_gpu_reports_an_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    rc = lib.ppr_create(0, C.byref(h))
    assert rc == -3  # PPR_ECUDA
    assert b"device" in lib.ppr_last_error()


def test_binding_raises_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1903_11749_gb300 import ppr
    with pytest.raises(ppr.PPRError):
        ppr.Context(0)
