"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/nasch.h declares; its host-side helpers (slowdown threshold,
Floyd initialisation) agree with the oracle.  No kernel is launched here."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2309_14311_gb300 import build as B
from paper_2309_14311_gb300 import nasch as NS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(nasch_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    B.build()
    return NS.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("nasch_create", "nasch_run", "nasch_read_state", "nasch_stats", "nasch_set_state",
                     "nasch_read_grid", "nasch_destroy", "nasch_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_built_for_sm_103a_only():
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


@pytest.mark.parametrize("p", [0.0, 1.0, 0.13, 0.5, 2.0**-32, 0.999999, 1 / 3])
def test_threshold_matches_oracle(lib, p):
    assert NS.slow_threshold(p) == O.slow_threshold(p)


@pytest.mark.parametrize("L,N,seed,road", [(1000, 200, 1, 0), (1, 1, 3, 0), (10, 10, 4, 1), (10**6, 12345, 7, 99),
                                           (2**24, 2**20, 1, 0), (2**31, 1000, 5, 3)])
def test_library_floyd_matches_oracle(lib, L, N, seed, road):
    assert np.array_equal(NS.floyd_init(L, N, seed, road), O.floyd_init(L, N, seed, road))


def test_errors_are_reported_not_raised_across_the_abi(lib):
    with pytest.raises(NS.NaschError) as e:
        NS.floyd_init(10, 11, 1)
    assert e.value.status == NS.EINVAL
    h = ctypes.c_void_p()
    st = lib.nasch_create(0, 0, 5, 0.1, 1, ctypes.byref(h))
    assert st == NS.EINVAL and b"L=0" in lib.nasch_last_error()
    st = lib.nasch_create(10, 5, 200, 0.1, 1, ctypes.byref(h))
    assert st == NS.EINVAL and b"vmax" in lib.nasch_last_error()
    st = lib.nasch_create(10, 5, 5, 1.5, 1, ctypes.byref(h))
    assert st == NS.EINVAL and b"p=" in lib.nasch_last_error()
    # open roads: alpha and beta in [0, 1], grid layout only (checked before any device work)
    prm = NS.Params()
    lib.nasch_params_init(ctypes.byref(prm))
    prm.L, prm.N, prm.vmax, prm.p = 1000, 10, 5, 0.1
    for a, b in ((-0.5, 0.5), (0.5, 2.0), (float("nan"), 0.5)):
        assert lib.nasch_create_open(ctypes.byref(prm), a, b, ctypes.byref(h)) == NS.EINVAL
        assert b"alpha" in lib.nasch_last_error()
    prm.layout = NS.LAYOUTS["agent"]
    assert lib.nasch_create_open(ctypes.byref(prm), 0.5, 0.5, ctypes.byref(h)) == NS.EINVAL
    assert b"grid layout" in lib.nasch_last_error()
    assert lib.nasch_run_output(None, 10, 5, None, 0, None, 0, 0) == NS.EINVAL


def test_no_gpu_fails_loudly(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(NS.NaschError) as e:
        NS.Road(1000, 200, 5, 0.13, 1)
    assert e.value.status == NS.ECUDA
