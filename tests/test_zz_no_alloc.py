"""The plan-free energy entry point, for callers that cannot allocate device
memory (runtimes that own all device memory through their own pool, loops
that must not enter the allocator).  It is called through the C ABI and must
agree with the energy of the plan-based ib_fe_force, and with the FP64
oracle's energy for every material law with and without active tension,
within the energy tolerance of the parity tests, on two calls in a row (its
scratch array is shared between calls).

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2503_22695_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ENERGY_RTOL = 1e-5   # FP32 split-position energy tolerance of the parity tests


@pytest.mark.parametrize("make", [lambda: I.block_problem(fp64=False), I.shell_problem])
def test_noalloc_energy_matches_plan_energy(make):
    import torch
    from paper_2503_22695_gb300 import ibfe
    p = make()
    dev = "cuda"
    conn = torch.from_numpy(p.conn).to(dev)
    X = torch.from_numpy(p.X).to(dev)
    fib = torch.from_numpy(p.fibres).to(dev)
    mid = torch.from_numpy(p.mat_id).to(dev)
    pos = ibfe.Pos(cell=torch.from_numpy(p.cell).to(dev), off=torch.from_numpy(p.off).to(dev))
    mats = [ibfe.Material(m.model, m.params) for m in p.materials]
    plan = ibfe.Plan(conn, X, p.grid.n, p.grid.h, fibres=fib, mat_id=mid)
    _, want = ibfe.ib_fe_force(plan, mats, pos, energy=True)
    # straight through the C ABI
    lib = ibfe._lib
    mesh = ibfe._Mesh(p.n_nodes, p.n_elems, conn.data_ptr(), X.data_ptr(), fib.data_ptr(),
                      mid.data_ptr())
    arr, nm = ibfe._mats(mats)
    for _ in range(2):
        out = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        rc = lib.ib_fe_energy_noalloc(C.byref(mesh), arr, nm, C.byref(pos._s), float(p.grid.h),
                                      C.c_void_p(out.data_ptr()),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == ibfe.IB_OK
        got = float(out.item())
        assert got == pytest.approx(want, rel=ENERGY_RTOL)


LAWS = [
    (I.NEO_HOOKEAN, (0.5, 100.0)),
    (I.FIBRE1, I.FIBRE1_LEAFLET),
    (I.HO, I.HO_DEFAULT),
    (I.STD_REINF, I.STD_REINF_COOK),
    (I.FIBRE2, I.FIBRE2_AV),
]


@pytest.mark.parametrize("Ta", [0.0, 5.0])
@pytest.mark.parametrize("model,params", LAWS)
def test_noalloc_energy_matches_oracle_for_every_law(model, params, Ta):
    import torch
    from paper_2503_22695_gb300 import ibfe
    p = I.block_problem(seed=1050, fp64=False)
    p.materials = [I.Material(model, params, Ta)]
    dev = "cuda"
    conn = torch.from_numpy(p.conn).to(dev)
    X = torch.from_numpy(p.X).to(dev)
    fib = torch.from_numpy(p.fibres).to(dev)
    pos = ibfe.Pos(cell=torch.from_numpy(p.cell).to(dev), off=torch.from_numpy(p.off).to(dev))
    mats = [ibfe.Material(model, params, Ta)]
    _, want = oracle.Model(p).fe_force(I.from_split(p.cell, p.off, p.grid))
    for _ in range(2):
        out = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        ibfe.ib_fe_energy_noalloc(conn, X, mats, pos, p.grid.h, out, fibres=fib)
        assert float(out.item()) == pytest.approx(want, rel=ENERGY_RTOL)


def test_noalloc_rejects_oversized_mesh():
    import torch
    from paper_2503_22695_gb300 import ibfe
    E = 262144 + 1
    conn = torch.zeros((8, E), dtype=torch.int32, device="cuda")
    X = torch.zeros((3, 8), dtype=torch.float32, device="cuda")
    pos = ibfe.Pos(cell=torch.zeros((3, 8), dtype=torch.int32, device="cuda"),
                   off=torch.zeros((3, 8), dtype=torch.float32, device="cuda"))
    out = torch.zeros((1,), dtype=torch.float64, device="cuda")
    with pytest.raises(ibfe.IBError) as e:
        ibfe.ib_fe_energy_noalloc(conn, X, [ibfe.Material(0, (0.5, 100.0))], pos, 1 / 32, out)
    assert e.value.code == ibfe.IB_ERR_CAPACITY
