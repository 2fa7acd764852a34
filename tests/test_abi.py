"""The C-ABI library loads without a GPU and exports every entry point that
include/ibfe.h declares; argument checks that run before any CUDA call
return their documented codes."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "include", "ibfe.h")


def declared():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ib_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2503_22695_gb300 import _build
    return C.CDLL(_build.build())


def test_header_declares_the_operators():
    names = declared()
    for want in ("ib_plan_create", "ib_plan_destroy", "ib_fe_force", "ib_spread", "ib_interp",
                 "ib_spread_adj", "ib_interp_adj", "ib_fe_force_adj", "ib_forward",
                 "ib_backward", "ib_plan_sync_status", "ib_status_str"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared():
        assert hasattr(lib, name), name


def test_host_side_argument_checks(lib):
    lib.ib_status_str.restype = C.c_char_p
    assert lib.ib_status_str(0) == b"ok"
    assert lib.ib_version() == 100
    # the active-tension waveform is host arithmetic: same values as the oracle's
    import oracle
    lib.ib_active_tension.restype = C.c_double
    lib.ib_active_tension.argtypes = [C.c_double]
    for t in [i * 0.0137 for i in range(200)] + [-0.3, 0.65, 0.8, 2.45]:
        assert lib.ib_active_tension(t) == pytest.approx(oracle.active_tension(t), rel=1e-14,
                                                         abs=1e-9)
    out = C.c_void_p()
    # null mesh / grid / out pointer: rejected before touching the device
    assert lib.ib_plan_create(None, None, 0, 0, None, C.byref(out)) == 1
    assert lib.ib_plan_create(None, None, 0, 0, None, None) == 1
    for fn in ("ib_fe_force", "ib_spread", "ib_interp", "ib_spread_adj", "ib_interp_adj",
               "ib_fe_force_adj", "ib_forward"):
        assert getattr(lib, fn)(*([None] * 9)) == 1, fn
    assert lib.ib_backward(*([None] * 13)) == 1
    assert lib.ib_plan_get_tuning(None, None) == 1
    assert lib.ib_plan_set_tuning(None, None) == 1
    assert lib.ib_plan_autotune(*([None] * 7)) == 1
    assert lib.ib_plan_destroy(None) == 1
    assert lib.ib_plan_sync_status(None, None) == 1


def test_host_fault_injection(lib, monkeypatch):
    """IBFE_FAULT makes the named entry point fail before any work (host only),
    so error propagation can be tested without a GPU fault."""
    out = C.c_void_p()
    monkeypatch.setenv("IBFE_FAULT", "ib_plan_create:5")
    assert lib.ib_plan_create(None, None, 0, 0, None, C.byref(out)) == 5  # IB_ERR_TIMEOUT
    monkeypatch.setenv("IBFE_FAULT", "ib_forward")
    assert lib.ib_forward(*([None] * 9)) == 2                              # IB_ERR_CUDA
    assert lib.ib_plan_create(None, None, 0, 0, None, C.byref(out)) == 1  # not injected
    monkeypatch.delenv("IBFE_FAULT")
    assert lib.ib_forward(*([None] * 9)) == 1
    # the Python binding turns the injected status into IBError
    from paper_2503_22695_gb300 import ibfe
    monkeypatch.setenv("IBFE_FAULT", "ib_forward:3")
    args = (None, None, 0, None, None, None, None, None, None)
    assert ibfe._lib.ib_forward(*args) == ibfe.IB_ERR_NONFINITE
    with pytest.raises(ibfe.IBError) as e:
        ibfe._chk(ibfe._lib.ib_forward(*args), "ib_forward")
    assert e.value.code == ibfe.IB_ERR_NONFINITE


def test_plan_creation_checks_the_element_type_before_the_device(lib):
    """Element type and grid checks of ib_plan_create run on the host, for
    every element (P2 tetrahedra included), before any CUDA call."""
    from paper_2503_22695_gb300 import ibfe
    conn = (C.c_int32 * 10)(*range(10))
    X = (C.c_float * 30)()
    out = C.c_void_p()
    grid_ok = ibfe._Grid((C.c_int32 * 3)(16, 16, 16), 1.0 / 16, (C.c_double * 3)(0, 0, 0))
    grid_bad_h = ibfe._Grid((C.c_int32 * 3)(16, 16, 16), 0.0, (C.c_double * 3)(0, 0, 0))
    grid_ragged = ibfe._Grid((C.c_int32 * 3)(16, 12, 16), 1.0 / 16, (C.c_double * 3)(0, 0, 0))
    for elem in (ibfe.IB_ELEM_HEX8, ibfe.IB_ELEM_TET4, ibfe.IB_ELEM_TET10):
        mesh = ibfe._Mesh(10, 1, C.cast(conn, C.c_void_p), C.cast(X, C.c_void_p), None, None,
                          elem)
        assert lib.ib_plan_create(C.byref(mesh), C.byref(grid_bad_h), 0, 0, None,
                                  C.byref(out)) == ibfe.IB_ERR_INVALID_ARG
        assert lib.ib_plan_create(C.byref(mesh), C.byref(grid_ragged), 0, 0, None,
                                  C.byref(out)) == ibfe.IB_ERR_UNSUPPORTED
    for bad in (3, -1):
        mesh = ibfe._Mesh(10, 1, C.cast(conn, C.c_void_p), C.cast(X, C.c_void_p), None, None,
                          bad)
        assert lib.ib_plan_create(C.byref(mesh), C.byref(grid_ok), 0, 0, None,
                                  C.byref(out)) == ibfe.IB_ERR_INVALID_ARG
    assert out.value is None
