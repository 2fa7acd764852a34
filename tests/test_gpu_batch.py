"""Batched form: independent hexahedral shells of uneven sizes, each on its
own periodic grid, packed into one plan (one launch per stage over all of
them, one CUDA graph per pass).

* Every instance equals the single-instance entry points bit for bit
  (ib_forward, ib_backward and the parameter gradients), although the packed
  plan is tuned once for the whole batch and the single plans keep their
  default tuning.
* The 48-instance parameter sweep (grids 32^3..128^3, 2k..20k hexahedra, HO
  parameters a, b, a_f, b_f each scaled by U(0.7, 1.3)) against the FP64
  oracle at the FP32 tolerances, forward and backward (the position
  gradient away from the few elements with a Gauss point within 5e-7 of the
  fibres' tension-only kink, where the Hessian jumps).
* The same 48 instances through FP64 plans (the plain FP64 GPU form): within
  1e-10 of the oracle, and the batched FP32 results within the FP32
  tolerances of them.
* Graph replays are identical.
"""
import numpy as np
import pytest

import oracle
from paper_2503_22695_gb300 import inputs as I

from helpers import kink_nodes, np_, rel_l2

pytestmark = pytest.mark.gpu

TOL = dict(G=1e-5, f=1e-5, U=1e-6, adj=2e-5)


def _instances(probs, seed):
    import torch
    from paper_2503_22695_gb300 import ibfe
    rng = np.random.default_rng(seed)
    out = []
    for p in probs:
        d = dict(conn=torch.from_numpy(p.conn).cuda(), X=torch.from_numpy(p.X).cuda(),
                 fibres=torch.from_numpy(p.fibres).cuda(), mat_id=torch.from_numpy(p.mat_id).cuda(),
                 n=p.grid.n, h=p.grid.h, mats=[ibfe.Material(m.model, m.params) for m in p.materials],
                 cell=torch.from_numpy(p.cell).cuda(), off=torch.from_numpy(p.off).cuda(),
                 u=torch.from_numpy(p.u).cuda())
        N, sh = p.n_nodes, (3,) + tuple(p.u.shape[1:])
        d.update(G=torch.empty((3, N), device="cuda"), f=torch.empty(sh, device="cuda"),
                 U=torch.empty((3, N), device="cuda"),
                 gU=torch.from_numpy(rng.normal(size=(3, N)).astype(np.float32)).cuda(),
                 gf=torch.from_numpy(rng.normal(size=sh).astype(np.float32)).cuda(),
                 gG=torch.from_numpy(rng.normal(size=(3, N)).astype(np.float32)).cuda(),
                 gu=torch.empty(sh, device="cuda"), gx=torch.empty((3, N), device="cuda"))
        out.append(d)
    return out


def test_batch_matches_single_instance_bitwise():
    import torch
    from paper_2503_22695_gb300 import ibfe
    probs = I.batch_problems(seed=7000, count=6, sizes=(32, 64), elems=(300, 2500))
    inst = _instances(probs, 7000)
    batch = ibfe.Batch(inst)
    batch.forward()
    batch.adjoint()
    gp = batch.gparams()
    torch.cuda.synchronize()
    for i, d in enumerate(inst):
        plan = ibfe.Plan(d["conn"], d["X"], d["n"], d["h"], fibres=d["fibres"], mat_id=d["mat_id"])
        pos = ibfe.Pos(cell=d["cell"], off=d["off"])
        G, f, U = ibfe.ib_forward(plan, d["mats"], pos, d["u"])
        assert torch.equal(G, d["G"]) and torch.equal(f, d["f"]) and torch.equal(U, d["U"]), i
        gx, gu, gpi = ibfe.ib_backward(plan, d["mats"], pos, d["u"], G, d["gG"], d["gf"],
                                       d["gU"])
        assert torch.equal(gu, d["gu"]) and torch.equal(gx, d["gx"]), i
        nm = len(d["mats"])
        assert torch.equal(gpi.cpu(), gp[i, :nm]), i
        assert torch.count_nonzero(gp[i, nm:]) == 0


def test_batch_graph_replays_identically():
    import torch
    from paper_2503_22695_gb300 import ibfe
    probs = I.batch_problems(seed=7100, count=4, sizes=(32, 64), elems=(300, 2500))
    inst = _instances(probs, 7100)
    batch = ibfe.Batch(inst)
    batch.forward()
    first = [d["f"].clone() for d in inst]
    for d in inst:
        d["f"].fill_(float("nan"))
    batch.forward()
    torch.cuda.synchronize()
    for a, d in zip(first, inst):
        assert torch.equal(a, d["f"])


def _oracle_of(p):
    return oracle.Model(grid=p.grid, conn=p.conn, X=p.X.astype(np.float64),
                        fibres=p.fibres.astype(np.float64), mat_id=p.mat_id,
                        materials=p.materials)


@pytest.fixture(scope="module")
def sweep():
    """The 48-instance sweep: batched FP32 forward and backward on the device."""
    import torch
    from paper_2503_22695_gb300 import ibfe
    probs = I.batch_problems()
    assert len(probs) == 48
    assert {p.grid.n[0] for p in probs} <= {32, 64, 96, 128}
    # 2k..20k hexahedra, up to the rounding of the mesh dimensions
    assert min(p.n_elems for p in probs) >= 1900 and max(p.n_elems for p in probs) <= 21000
    inst = _instances(probs, 5)
    batch = ibfe.Batch(inst)
    batch.forward()
    batch.adjoint()
    gp = batch.gparams()
    torch.cuda.synchronize()
    out = [{k: np_(d[k]) for k in ("G", "f", "U", "gx", "gu", "gU", "gf", "gG")} for d in inst]
    return probs, out, gp.numpy(), batch.tuning()


def test_batch_sweep_forward_matches_oracle(sweep):
    probs, out, _, _ = sweep
    for i, (p, o) in enumerate(zip(probs, out)):
        orc = _oracle_of(p)
        x = I.from_split(p.cell, p.off, p.grid)
        Go, _ = orc.fe_force(x)
        assert rel_l2(o["G"], Go) <= TOL["G"], i
        G32 = o["G"].astype(np.float64)          # the spread input both sides see
        assert rel_l2(o["f"], orc.spread(x, G32)) <= TOL["f"], i
        assert rel_l2(o["U"], orc.interp(x, p.u.astype(np.float64))) <= TOL["U"], i


def test_batch_sweep_backward_matches_oracle(sweep):
    probs, out, gp, _ = sweep
    for i, (p, o) in enumerate(zip(probs, out)):
        orc = _oracle_of(p)
        x = I.from_split(p.cell, p.off, p.grid)
        G = o["G"].astype(np.float64)
        gU, gf, gG = (o[k].astype(np.float64) for k in ("gU", "gf", "gG"))
        # gx = Hv(gG + S^T gf) + (dS/dx)^T gf + (dJ/dx)^T gU
        guo, gxi = orc.interp_adj(x, p.u.astype(np.float64), gU)
        gGs, gxs = orc.spread_adj(x, G, gf)
        Hv, gpo = orc.fe_force_adj(x, gG + gGs)
        # the Hessian jumps at the tension-only fibre kink (I4 = 1): on the
        # nodes of the elements with a Gauss point within 5e-7 of it either
        # branch is valid for FP32 inputs; every other node must match
        keep = np.ones(p.n_nodes, bool)
        keep[kink_nodes(p, x)] = False
        assert keep.sum() >= 0.99 * p.n_nodes, i
        assert rel_l2(o["gx"][:, keep], (gxi + gxs + Hv)[:, keep]) <= TOL["adj"], i
        assert rel_l2(o["gu"], guo) <= TOL["adj"], i
        k = I.N_PARAMS[p.materials[0].model]
        assert rel_l2(gp[i, 0, :k], gpo[0, :k]) <= TOL["adj"], i


def test_batch_sweep_against_fp64_gpu_form(sweep):
    """The plain FP64 GPU form of the same 48 instances (one FP64 plan each,
    positions and data widened exactly) meets 1e-10 against the oracle; the
    batched FP32 results are within the FP32 tolerances of it."""
    import torch
    from paper_2503_22695_gb300 import ibfe
    probs, out, _, _ = sweep
    for i, (p, o) in enumerate(zip(probs, out)):
        g = p.grid
        x = I.from_split(p.cell, p.off, g)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
        plan = ibfe.Plan(torch.from_numpy(p.conn).cuda(), dev(p.X), g.n, g.h, g.origin,
                         fibres=dev(p.fibres), mat_id=torch.from_numpy(p.mat_id).cuda(),
                         precision=ibfe.IB_FP64)
        mats = [ibfe.Material(m.model, m.params) for m in p.materials]
        G64, f64, U64 = (np_(t) for t in ibfe.ib_forward(plan, mats, ibfe.Pos(x64=dev(x)),
                                                           dev(p.u)))
        orc = _oracle_of(p)
        Go, _ = orc.fe_force(x)
        assert rel_l2(G64, Go) <= 1e-10, i
        assert rel_l2(f64, orc.spread(x, G64)) <= 1e-10, i
        assert rel_l2(U64, orc.interp(x, p.u.astype(np.float64))) <= 1e-10, i
        # matched accuracy: the batched FP32 form against the FP64 GPU form
        assert rel_l2(o["G"], G64) <= TOL["G"], i
        assert rel_l2(o["f"], f64) <= TOL["f"], i
        assert rel_l2(o["U"], U64) <= TOL["U"], i
        del plan
