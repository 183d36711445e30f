"""The C ABI library builds, loads and exports every entry point declared in include/msqoc.h,
and its host-side argument validation rejects malformed descriptions before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2407_13950_gb300 import build as B
from paper_2407_13950_gb300 import msqoc
from paper_2407_13950_gb300 import synthetic as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(msqoc_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    names = declared_entry_points()
    assert "msqoc_eval_gradient" in names and "msqoc_create_problem" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(msqoc.EXPORTED) <= set(names)
    assert msqoc.load().msqoc_version() >= 100


def _create(H, C, T=10.0, nsteps=100, M=2, opt=None):
    lib = msqoc.load()
    h = ctypes.c_void_p()
    st = lib.msqoc_create_problem(ctypes.byref(H) if H is not None else None,
                                  ctypes.byref(C) if C is not None else None, None, T, nsteps, M, 0.0,
                                  ctypes.byref(opt) if opt is not None else None, ctypes.byref(h))
    return st, h


def _desc(q=2, L=3, ness=2, jx=None, ncar=None, d1=6):
    xi = np.full(q, 1.0)
    xc = np.zeros((q, q))
    nf = np.asarray(ncar if ncar is not None else [2] * q, dtype=np.int32)
    om = np.zeros(max(int(nf.sum()), 1))
    keep = [xi, xc, nf, om]
    jxa = None
    if jx is not None:
        jxa = np.asarray(jx, dtype=np.float64)
        keep.append(jxa)
    H = msqoc.Hamiltonian(q, L, ness, xi.ctypes.data, xc.ctypes.data, None, None if jxa is None else jxa.ctypes.data)
    C = msqoc.Controls(nf.ctypes.data, om.ctypes.data, d1)
    return H, C, keep


def test_validation_rejects_malformed_descriptions_without_a_gpu():
    H, C, keep = _desc()
    assert _create(None, C)[0] == -1
    assert _create(H, None)[0] == -1
    Hb, Cb, k2 = _desc(q=0)
    assert _create(Hb, Cb)[0] == -1
    Hb, Cb, k3 = _desc(L=5, q=2)
    assert _create(Hb, Cb)[0] == -6            # no kernel for 5 levels
    Hb, Cb, k4 = _desc(jx=np.array([[0.0, 0.1], [0.0, 0.0]]))
    assert _create(Hb, Cb)[0] == -6            # dipole exchange needs 2-level subsystems
    Hb, Cb, k4b = _desc(jx=np.array([[0.0, np.nan], [0.0, 0.0]]))
    assert _create(Hb, Cb)[0] == -1            # non-finite exchange
    Hb, Cb, k5 = _desc(d1=2)
    assert _create(Hb, Cb)[0] == -1            # fewer than 3 splines
    Hb, Cb, k6 = _desc(ncar=[2, 0])
    assert _create(Hb, Cb)[0] == -1            # subsystem without carrier
    assert _create(H, C, T=-1.0)[0] == -1
    assert _create(H, C, nsteps=10, M=11)[0] == -1  # more windows than steps
    assert _create(H, C, M=0)[0] == -1
    opt = msqoc.Options(0, 0, -1)
    assert _create(H, C, opt=opt)[0] == -1     # negative checkpoint interval
    assert "checkpoint" in msqoc.last_error()
    lib = msqoc.load()
    assert lib.msqoc_create_problem(None, None, None, 1.0, 1, 1, 0.0, None, None) == -1
    assert lib.msqoc_destroy_problem(None) == 0


def test_binding_rejects_wrong_dtypes():
    with pytest.raises(TypeError):
        msqoc._ptr(np.zeros(3, dtype=np.float32))
    with pytest.raises(TypeError):
        msqoc._ptr(np.zeros((3, 3))[:, 0])


def test_bounded_wait_selftest_rejects_spin_counts_outside_its_range():
    lib = msqoc.load()
    for spins in (0, -3, (1 << 18) + 1):
        assert lib.msqoc_selftest_bounded_wait(spins, 0, None) == -1     # no device work
