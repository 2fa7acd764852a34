"""GPU parity of the penalty tethers of the solid boundary (Section 5)
against the oracle: nodal force and energy, the force adjoint, the fused
forward/backward and the explicit IB step with the x-minimum face of the
block tethered (hexahedra; the force and adjoint also on quadratic
tetrahedra), in FP32 (1e-5 force, 2e-5 adjoint) and FP64 (1e-12)."""
import numpy as np
import pytest

from oracle import fluid as OF
from paper_2503_22695_gb300 import inputs as I

from helpers import Case, np_, rel_l2

pytestmark = pytest.mark.gpu

KAPPA = 1e6


def _case(fp64, weighted, p2=False):
    import torch
    base = I.block_problem(fp64=fp64)
    c = Case(I.tet10_problem(base) if p2 else base)
    X = c.prob.X
    nodes = np.flatnonzero(X[0] <= X[0].min() + 1e-12).astype(np.int32)
    w = None
    if weighted:
        w = np.random.default_rng(3).uniform(0.5, 2.0, size=len(nodes)) * c.prob.grid.h ** 2
        w = c.rounded(w)
    c.nodes = nodes
    c.w = w
    c.ibfe.ib_plan_set_penalty(c.plan, torch.from_numpy(nodes).cuda(), KAPPA,
                               None if w is None else c.to_dev(w))
    return c


@pytest.mark.parametrize("fp64,weighted,p2", [(False, False, False), (False, True, False),
                                               (True, False, False), (False, False, True),
                                               (True, False, True)])
def test_penalty_force_energy_and_adjoint(fp64, weighted, p2):
    """Hexahedra, and quadratic tetrahedra (whose tether weights are the
    scaled-diagonal lumped masses)."""
    c = _case(fp64, weighted, p2)
    t = 1e-12 if fp64 else 1e-5
    G, en = c.ibfe.ib_fe_force(c.plan, c.mats, c.pos, energy=True)
    Ge, ee = c.orc.fe_force(c.x_np)
    Gp, ep = c.orc.penalty(c.x_np, c.nodes, KAPPA, c.w)
    assert np.abs(Gp).max() > 0.1 * np.abs(Ge).max()   # the tethers matter
    assert rel_l2(np_(G), Ge + Gp) <= t
    assert en == pytest.approx(ee + ep, rel=t)
    # adjoint: the tethers' force is linear with G(X) = 0, so its Jacobian
    # times v is the oracle's tether force at X + v
    v = c.rounded(np.random.default_rng(4).normal(size=(3, c.prob.n_nodes)))
    Hv, gp = c.ibfe.ib_fe_force_adj(c.plan, c.mats, c.pos, c.to_dev(v))
    Hve, gpe = c.orc.fe_force_adj(c.x_np, v)
    Hvp, _ = c.orc.penalty(c.prob.X.astype(np.float64) + v, c.nodes, KAPPA, c.w)
    assert rel_l2(np_(Hv), Hve + Hvp) <= (1e-12 if fp64 else 2e-5)
    k = I.N_PARAMS[c.prob.materials[0].model]
    assert rel_l2(gp[0, :k].numpy(), gpe[0, :k]) <= (1e-12 if fp64 else 2e-5)


def test_penalty_in_forward_backward_and_step():
    import torch
    from paper_2503_22695_gb300 import ibfe
    c = _case(False, False)
    G, f, U = ibfe.ib_forward(c.plan, c.mats, c.pos, c.u)
    Ge, _ = c.orc.fe_force(c.x_np)
    Gp, _ = c.orc.penalty(c.x_np, c.nodes, KAPPA)
    assert rel_l2(np_(G), Ge + Gp) <= 1e-5
    assert rel_l2(np_(f), c.orc.spread(c.x_np, Ge + Gp)) <= 1e-5
    # fused backward = composition of the separate adjoints (tethers included)
    rng = np.random.default_rng(5)
    gG = c.to_dev(c.rounded(rng.normal(size=(3, c.prob.n_nodes))))
    gx, _, _ = ibfe.ib_backward(c.plan, c.mats, c.pos, None, None, gG, want_params=False)
    Hv, _ = ibfe.ib_fe_force_adj(c.plan, c.mats, c.pos, gG, want_params=False)
    assert torch.equal(gx, Hv)
    # explicit IB step: the oracle step with the tethers' force added
    fl = ibfe.Fluid(c.prob.grid.n, c.prob.grid.h, 1.0, 0.02, 1e-3)
    u = c.u.clone()
    G1, f1, U1, _ = ibfe.ib_step(c.plan, fl, c.mats, c.pos, u)
    fo = c.orc.spread(c.x_np, Ge + Gp)
    _, _, uo = OF.fluid_step(c.u_np, fo, 1.0, 0.02, 1e-3, c.prob.grid.h)
    assert rel_l2(np_(G1), Ge + Gp) <= 1e-5
    assert rel_l2(np_(u), uo) <= 1e-5
    assert rel_l2(np_(U1), c.orc.interp(c.x_np, uo)) <= 1e-5


def test_penalty_removal_and_argument_checks():
    import torch
    from paper_2503_22695_gb300 import ibfe
    c = _case(False, False)
    G1 = np_(ibfe.ib_fe_force(c.plan, c.mats, c.pos))
    ibfe.ib_plan_set_penalty(c.plan, None)
    G0 = np_(ibfe.ib_fe_force(c.plan, c.mats, c.pos))
    assert rel_l2(G0, c.orc.fe_force(c.x_np)[0]) <= 1e-5
    assert not np.array_equal(G0, G1)
    nodes = torch.from_numpy(c.nodes).cuda()
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(ibfe.IBError) as e:
            ibfe.ib_plan_set_penalty(c.plan, nodes, bad)
        assert e.value.code == ibfe.IB_ERR_INVALID_ARG
