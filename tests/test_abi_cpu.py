"""The C-ABI library loads and exports every declared symbol; host-side
argument validation returns the documented status codes (no GPU needed:
all checks happen before the first CUDA call)."""

import ctypes
import os
import re

import pytest

from tests._lib import ensure_built

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pb():
    ensure_built()
    from paper_1409_8116_gb300 import binding
    return binding


def _declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"\b(poisfft_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol(pb):
    lib = ctypes.CDLL(pb.LIB_PATH)
    declared = _declared_symbols()
    assert "poisfft_solve" in declared and "poisfft_plan_create" in declared
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert set(pb.EXPORTED) <= set(declared)


def test_status_strings(pb):
    for st in [0, -1, -2, -3, -4, -5, -6, -7, -8]:
        assert pb.status_string(st) and pb.status_string(st) != "unknown status"
    assert pb.status_string(12345) == "unknown status"


@pytest.mark.parametrize("args,expect", [
    (((8, 8, 8), (1, 1, 1), (0, 0, 0), 1, 0), None),                 # valid -> CUDA error without GPU, OK with
    (((8, 8, 8), (1, 1, 1), (0, 0, 0), 7, 0), -1),                   # bad approx
    (((8, 8, 8), (1, 1, 1), (0, 0, 0), 1, 5), -1),                   # bad dtype
    (((8, 0, 8), (1, 1, 1), (0, 0, 0), 1, 0), -1),                   # n < 1
    (((8, 8, 8), (1, -1, 1), (0, 0, 0), 1, 0), -1),                  # L <= 0
    (((8, 8, 8), (1, 1, 1), (0, 9, 0), 1, 0), -1),                   # bad bc code
    (((8, 1, 8), (1, 1, 1), (0, 3, 0), 1, 0), -1),                   # NR needs n >= 2
    (((8, 8, 8), (1, 1, 1), (0, 0, 2, 4, 0, 0), 1, 0), -2),          # faces of one axis differ
    (((8, 8, 8), (1, 1, 1), (0, 0, 0, 0, 0, 3), 1, 0), -2),
    (((8, 8, 8), (1, 1, 1), (2, 0, 4), 1, 0), None),                 # x non-periodic with periodic y
    (((8, 8, 8), (1, 1, 1), (4, 4, 0), 1, 0), None),                 # x non-periodic with periodic z
    (((8, 8, 8), (1, 1, 1), (0, 2, 4), 1, 2), None),                 # MIXED (FD2)
    (((8, 8, 8), (1, 1, 1), (0, 2, 4), 0, 2), -8),                   # MIXED needs FD2 eigenvalues
])
def test_plan_create_validation(pb, args, expect):
    rc, plan = pb.plan_create(*args)
    if expect is None:
        assert rc in (pb.OK, pb.ERR_CUDA)
        if rc == pb.OK:
            pb.destroy(plan)
    else:
        assert rc == expect
        assert not plan.value


def test_dims_out_of_range(pb):
    plan = ctypes.c_void_p()
    n = (ctypes.c_int64 * 4)(4, 4, 4, 4)
    L = (ctypes.c_double * 4)(1, 1, 1, 1)
    bc = (ctypes.c_int * 8)(*([0] * 8))
    assert pb.lib.poisfft_plan_create(ctypes.byref(plan), 4, n, L, bc, 1, 0) == pb.ERR_INVALID_ARG
    assert pb.lib.poisfft_plan_create(ctypes.byref(plan), 0, n, L, bc, 1, 0) == pb.ERR_INVALID_ARG
    assert pb.lib.poisfft_plan_create(None, 3, n, L, bc, 1, 0) == pb.ERR_INVALID_ARG


def test_null_plan_calls(pb):
    assert pb.lib.poisfft_solve(None, None, None, None) == pb.ERR_INVALID_ARG
    assert pb.lib.poisfft_solve_host(None, None, None, None) == pb.ERR_INVALID_ARG
    assert pb.lib.poisfft_solve_host_async(None, None, None, None) == pb.ERR_INVALID_ARG
    assert pb.lib.poisfft_check(None, None) == pb.ERR_INVALID_ARG
    assert pb.lib.poisfft_destroy(None) == pb.OK
    info = (ctypes.c_int64 * 4)()
    assert pb.lib.poisfft_plan_info(None, info) == pb.ERR_INVALID_ARG


def test_mixed_dtype_host_checks(pb):
    """MIXED is a plan dtype (Sec. 3: one solver object per precision); the
    calls that do not implement it say so before any CUDA call."""
    assert pb.MIXED == 2
    assert pb.lib.poisfft_plan_set_refinements(None, 1) == pb.ERR_INVALID_ARG
    g = ctypes.c_double()
    rc = pb.solve_noalloc((8, 8), (1, 1), (pb.P, pb.NS), pb.FD2, pb.MIXED, ctypes.addressof(g), ctypes.addressof(g))
    assert rc == pb.ERR_NOT_IMPLEMENTED
    n = (ctypes.c_int64 * 3)(8, 8, 8)
    L = (ctypes.c_double * 3)(1, 1, 1)
    bc = (ctypes.c_int * 6)(*([0] * 6))
    dims = (ctypes.c_int * 1)(3)
    b = ctypes.c_void_p()
    assert pb.lib.poisfft_batch_create(ctypes.byref(b), 1, dims, n, L, bc, 1, pb.MIXED) == pb.ERR_NOT_IMPLEMENTED


def test_bf16x3_needs_a_1024_point_strided_axis(pb):
    """The tensor-core form serves 1024-point strided axes; plans without
    one are refused at planning time, before any CUDA call."""
    assert pb.BF16X3 == 3
    for n, bc in [((64, 64, 64), (0, 0, 0)), ((1024, 64, 64), (0, 0, 4)), ((100, 1024, 1024), (0, 0, 4)),
                  ((1024, 1024), (4, 4))]:
        rc, plan = pb.plan_create(n, (1,) * len(n), bc, 1, pb.BF16X3)
        assert rc == pb.ERR_NOT_IMPLEMENTED, (n, bc, rc)
    rc, plan = pb.plan_create((64, 64, 1024), (1, 1, 1), (0, 0, 4), 1, pb.BF16X3)
    assert rc in (pb.OK, pb.ERR_CUDA)
    if rc == pb.OK:
        pb.destroy(plan)


def test_injected_size_fault_is_reported_before_any_cuda_call(pb, monkeypatch):
    """Host-side fault injection: POISFFT_FAULT=size makes planning report
    an unsupported size; without the variable the same plan is valid."""
    monkeypatch.setenv("POISFFT_FAULT", "size")
    rc, plan = pb.plan_create((32, 32, 32), (1, 1, 1), (0, 2, 4), 1, 0)
    assert rc == pb.ERR_UNSUPPORTED_SIZE and not plan.value
    monkeypatch.delenv("POISFFT_FAULT")
    rc, plan = pb.plan_create((32, 32, 32), (1, 1, 1), (0, 2, 4), 1, 0)
    assert rc in (pb.OK, pb.ERR_CUDA)
    if rc == pb.OK:
        pb.destroy(plan)
