"""CPU checks of the C-ABI library: it loads, exports every symbol the headers
declare, and rejects malformed problems on the host before touching a device."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2412_09285_b300 import build
    build.build()
    from paper_2412_09285_b300 import fem
    return fem


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(fem_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol(lib):
    names = _declared_symbols()
    assert "fem_create_problem" in names and "fem_anneal" in names and "fem_read_best" in names
    so = C.CDLL(lib.LIB_PATH)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def test_status_strings(lib):
    assert lib.status_string(0) == "FEM_OK"
    assert lib.status_string(lib.FEM_ERR_TIMEOUT) == "FEM_ERR_TIMEOUT"


def _desc(lib, n, ei, ej, w=None, kind=0, q=2):
    d = lib.fem_problem_desc()
    d.kind, d.n, d.q = kind, n, q
    keep = [np.asarray(ei, np.int32), np.asarray(ej, np.int32)]
    d.n_edges = len(ei)
    d.ei, d.ej = keep[0].ctypes.data, keep[1].ctypes.data
    if w is not None:
        keep.append(np.asarray(w, np.float64))
        d.w = keep[-1].ctypes.data
    return d, keep


@pytest.mark.parametrize("case,ei,ej,w", [
    ("self-loop", [0, 1], [1, 1], None),
    ("out of range", [0, 5], [1, 2], None),
    ("negative index", [0, -1], [1, 2], None),
    ("duplicate", [0, 1, 0], [1, 2, 1], None),
    ("duplicate reversed", [0, 1], [1, 0], None),
    ("zero weight", [0, 1], [1, 2], [1.0, 0.0]),
    ("nan weight", [0, 1], [1, 2], [1.0, float("nan")]),
])
def test_malformed_graphs_rejected_on_host(lib, case, ei, ej, w):
    d, keep = _desc(lib, 4, ei, ej, w)
    with pytest.raises(lib.FemError) as e:
        lib.fem_create_problem(d)
    assert e.value.status == lib.FEM_ERR_INVALID_ARG, case


def test_bad_kind_and_q_rejected(lib):
    d, keep = _desc(lib, 4, [0], [1], None, kind=7)
    with pytest.raises(lib.FemError) as e:
        lib.fem_create_problem(d)
    assert e.value.status == lib.FEM_ERR_INVALID_ARG
    d, keep = _desc(lib, 4, [0], [1], None, kind=0, q=3)
    with pytest.raises(lib.FemError) as e:
        lib.fem_create_problem(d)
    assert e.value.status == lib.FEM_ERR_INVALID_ARG
    d, keep = _desc(lib, 4, [0], [1], [-1.0], kind=1, q=4)
    with pytest.raises(lib.FemError) as e:
        lib.fem_create_problem(d)
    assert e.value.status == lib.FEM_ERR_INVALID_ARG


def test_null_arguments_rejected(lib):
    so = lib._lib
    assert so.fem_create_problem(None, None, None) == lib.FEM_ERR_INVALID_ARG
    assert so.fem_anneal(None, None, None) == lib.FEM_ERR_INVALID_ARG
    assert so.fem_read_best(None, None, None, None, None, None) == lib.FEM_ERR_INVALID_ARG
    so.fem_destroy(None)  # no-op


@pytest.mark.parametrize("schedule,bmin,bmax,n", [("exponential", 0.05, 5.0, 2000),
                                                  ("inverse_proportional", 1 / 1.16, 1 / 6e-5, 1000),
                                                  ("exponential", 0.3, 0.3, 1)])
def test_schedule_value_is_the_oracle_schedule(lib, schedule, bmin, bmax, n):
    """fem_schedule_value (host-only) gives the beta and lambda schedule the oracle uses."""
    import oracle as O
    ref_b = O.beta_schedule(schedule, bmin, bmax, n)
    ref_l = O.lambda_ramp(0.7, n)
    for t in sorted({0, min(1, n - 1), n // 3, n - 1}):
        b, lam = lib.fem_schedule_value(t, n, schedule=schedule, beta_min=bmin, beta_max=bmax, lambda_max=0.7)
        assert b == pytest.approx(ref_b[t], rel=1e-13) and lam == pytest.approx(ref_l[t], rel=1e-13, abs=1e-15)
    with pytest.raises(lib.FemError) as e:
        lib.fem_schedule_value(n, n)
    assert e.value.status == lib.FEM_ERR_INVALID_ARG
