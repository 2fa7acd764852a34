"""Batched form: independent shells of uneven sizes on their own grids, run
as one captured CUDA graph; every instance must equal the single-instance
entry points bitwise (ib_forward and ib_backward), and the graph must replay
identically."""
import numpy as np
import pytest

from paper_2503_22695_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _instances(count=6, seed=7000):
    import torch
    from paper_2503_22695_gb300 import ibfe
    probs = I.batch_problems(seed=seed, count=count, sizes=(32, 64), elems=(300, 2500))
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
    inst = _instances()
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
        assert torch.equal(gu, d["gu"]) and torch.equal(gx, d["gx"])
        nm = len(d["mats"])
        assert torch.equal(gpi.cpu(), gp[i, :nm])
        assert torch.count_nonzero(gp[i, nm:]) == 0


def test_batch_graph_replays_identically():
    import torch
    from paper_2503_22695_gb300 import ibfe
    inst = _instances(count=4, seed=7100)
    batch = ibfe.Batch(inst)
    batch.forward()
    first = [d["f"].clone() for d in inst]
    for d in inst:
        d["f"].fill_(float("nan"))
    batch.forward()
    torch.cuda.synchronize()
    for a, d in zip(first, inst):
        assert torch.equal(a, d["f"])
