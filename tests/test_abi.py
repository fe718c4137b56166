"""CPU-side checks of the C ABI: the library loads, exports every entry point
declared in include/pmlsh.h, and its host-only functions (chi-square
parameters, budget, argument validation) behave.  No GPU work is launched."""
import ctypes
import math
import os
import re

import pytest

import oracle
import paper_2107_05537_gb300 as pm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(pmlsh_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = pm.lib()
    names = _declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(L, name), name


def test_params_match_oracle_and_closed_forms():
    for m in range(1, 17):
        for c in (1.2, 1.5, 2.0, 4.0):
            t, a2, b = pm.params(m, c, 1 / math.e)
            to, a2o, bo = oracle.params(m, c, 1 / math.e)
            assert t == pytest.approx(to, rel=1e-14)
            # alpha2 = 1 - Pr[chi^2 > x] loses digits when alpha2 is tiny
            assert a2 == pytest.approx(a2o, rel=1e-8, abs=1e-15)
            assert b == pytest.approx(2 * a2, rel=1e-15)
    # m = 2: t^2 = -2 ln alpha1
    t, _, _ = pm.params(2, 1.5, 0.05)
    assert t * t == pytest.approx(-2 * math.log(0.05), rel=1e-13)


def test_budget_matches_oracle():
    for n, beta, k in ((10_000, 0.2809, 10), (1_000_000, 0.2809, 50), (10, 0.4, 1),
                       (7, 1.0, 7), (123_457, 0.0967, 100)):
        assert pm.budget(n, beta, k) == oracle.budget(n, beta, k)


def test_argument_validation_needs_no_gpu():
    L = pm.lib()
    h = ctypes.c_void_p()
    # n = 0 is rejected before any device work
    x = (ctypes.c_float * 4)()
    assert L.pmlsh_build(ctypes.cast(x, ctypes.c_void_p), 0, 4, None, None, ctypes.byref(h)) == 1
    assert b"n must be" in L.pmlsh_last_error()
    assert L.pmlsh_build(None, 10, 4, None, None, ctypes.byref(h)) == 1
    o = pm.KnnOpts()
    L.pmlsh_knn_opts_default(ctypes.byref(o))
    assert (o.k, o.c, o.beta) == (10, 1.5, 0.2809)
    assert L.pmlsh_knn(None, None, 5, ctypes.byref(o), None, None, None, None, None) == 1
    a = ctypes.c_double()
    assert L.pmlsh_params(0, 1.5, 0.3, ctypes.byref(a), None, None) == 1
    assert L.pmlsh_params(15, 1.0, 0.3, ctypes.byref(a), None, None) == 1
    assert L.pmlsh_params(15, 1.5, 1.0, ctypes.byref(a), None, None) == 1
    bo = pm.BuildOpts()
    L.pmlsh_build_opts_default(ctypes.byref(bo))
    assert (bo.m, bo.s, bo.leaf_size) == (15, 5, 256)
    bo.m = 17
    assert L.pmlsh_build(ctypes.cast(x, ctypes.c_void_p), 1, 4, ctypes.byref(bo), None,
                         ctypes.byref(h)) == 1


def test_cost_model_argument_validation_needs_no_gpu():
    L = pm.lib()
    h = ctypes.c_void_p()
    x = (ctypes.c_float * 4)()
    bo = pm.BuildOpts()
    L.pmlsh_build_opts_default(ctypes.byref(bo))
    bo.leaf_size = -2          # only 0 (measured), -1 (cost model) or 16..1024
    assert L.pmlsh_build(ctypes.cast(x, ctypes.c_void_p), 1, 4, ctypes.byref(bo), None,
                         ctypes.byref(h)) == 1
    assert b"leaf_size" in L.pmlsh_last_error()
    out = (ctypes.c_double * 4)()
    assert L.pmlsh_distance_sample(None, 4, 0, ctypes.cast(out, ctypes.c_void_p), None) == 1
    assert L.pmlsh_cost_model(None, ctypes.cast(out, ctypes.c_void_p), 4, None, 0, None, None, None) == 1
    assert L.pmlsh_export_leaf_entries(None, None, None, None, None, None, None) == 1
