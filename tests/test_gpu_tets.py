"""GPU parity on tetrahedral meshes: linear (P1, the element of the paper's
valve meshes, Section 5) and quadratic (P2, the element of its Cook
membrane): the block and the 128^3 shell with every hexahedron split into six
tetrahedra (and, for P2, a node added at the middle of every edge, displaced
in the current configuration), against the FP64 oracle with the same 4-point
rule.  Tolerances as in the main parity suite: FP32 split plans 1e-5 (force,
spread), 1e-6 (interpolation), 2e-5 (adjoint outputs); FP64 plans 1e-12."""
import numpy as np
import pytest

from oracle import fluid as OF
from paper_2503_22695_gb300 import inputs as I

from helpers import Case, np_, rel_l2

pytestmark = pytest.mark.gpu

TOL32 = dict(G=1e-5, f=1e-5, U=1e-6, adj=2e-5)

_cache = {}


def case(name, quad=0, order=1):
    key = (name, quad, order)
    if key not in _cache:
        base = {"block32": lambda: I.block_problem(fp64=False),
                "block64": lambda: I.block_problem(),
                "shell128": lambda: I.shell_problem()}[name]()
        prob = I.tet_problem(base) if order == 1 else I.tet10_problem(base)
        _cache[key] = Case(prob, quad=quad)
    return _cache[key]


def tol(c, k):
    return 1e-12 if c.fp64 else TOL32[k]


NAMES = ["block32", "block64", "shell128"]
ORDERS = [1, 2]


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("name", NAMES)
def test_tet_force_energy_and_adjoint(name, order):
    c = case(name, order=order)
    assert c.plan.elem == (c.ibfe.IB_ELEM_TET4 if order == 1 else c.ibfe.IB_ELEM_TET10)
    G, en = c.ibfe.ib_fe_force(c.plan, c.mats, c.pos, energy=True)
    Go, eno = c.orc.fe_force(c.x_np)
    assert rel_l2(np_(G), Go) <= tol(c, "G")
    assert en == pytest.approx(eno, rel=tol(c, "G"))
    v = c.rounded(np.random.default_rng(41).normal(size=(3, c.prob.n_nodes)))
    Hv, gp = c.ibfe.ib_fe_force_adj(c.plan, c.mats, c.pos, c.to_dev(v))
    Hvo, gpo = c.orc.fe_force_adj(c.x_np, v)
    assert rel_l2(np_(Hv), Hvo) <= tol(c, "adj")
    k = I.N_PARAMS[c.prob.materials[0].model]
    assert rel_l2(gp[0, :k].numpy(), gpo[0, :k]) <= tol(c, "adj")


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("name", NAMES)
def test_tet_spread_interp_and_mass(name, order):
    c = case(name, order=order)
    ib = c.ibfe
    m = np_(ib.ib_lumped_mass(c.plan))
    assert rel_l2(m, c.orc.mass()) <= (1e-14 if c.fp64 else 1e-6)
    Go, _ = c.orc.fe_force(c.x_np)
    G = c.rounded(Go)
    f = ib.ib_spread(c.plan, c.pos, c.to_dev(G))
    assert rel_l2(np_(f), c.orc.spread(c.x_np, G)) <= tol(c, "f")
    U = ib.ib_interp(c.plan, c.pos, c.u)
    assert rel_l2(np_(U), c.orc.interp(c.x_np, c.u_np)) <= tol(c, "U")
    # the fused forward equals the three operators
    G2, f2, U2 = ib.ib_forward(c.plan, c.mats, c.pos, c.u)
    assert rel_l2(np_(G2), Go) <= tol(c, "G")
    assert rel_l2(np_(U2), np_(U)) <= (1e-15 if c.fp64 else 1e-7)


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("name", ["block32", "block64"])
def test_tet_fused_backward(name, order):
    c = case(name, order=order)
    ib = c.ibfe
    rng = np.random.default_rng(42)
    n = c.prob.n_nodes
    G = c.to_dev(c.rounded(c.orc.fe_force(c.x_np)[0]))
    gG = c.rounded(rng.normal(size=(3, n)))
    gU = c.rounded(rng.normal(size=(3, n)))
    gf = c.rounded(rng.normal(size=c.plan.grid_shape()))
    gx, gu, gp = ib.ib_backward(c.plan, c.mats, c.pos, c.u, G, c.to_dev(gG), c.to_dev(gf),
                                c.to_dev(gU))
    guo, gxi = c.orc.interp_adj(c.x_np, c.u_np, gU)
    gGs, gxs = c.orc.spread_adj(c.x_np, np_(G), gf)
    Hv, gpo = c.orc.fe_force_adj(c.x_np, gG + gGs)
    t = tol(c, "adj")
    assert rel_l2(np_(gx), gxi + gxs + Hv) <= t
    assert rel_l2(np_(gu), guo) <= t
    k = I.N_PARAMS[c.prob.materials[0].model]
    assert rel_l2(gp[0, :k].cpu().numpy(), gpo[0, :k]) <= t


@pytest.mark.parametrize("order", ORDERS)
def test_tet_nodal_rule_and_ib_step(order):
    """The nodal quadrature rule on tetrahedra, and one explicit IB step."""
    from paper_2503_22695_gb300 import ibfe
    c = case("block32", quad=ibfe.IB_QUAD_NODAL, order=order)
    Go, _ = c.orc.fe_force(c.x_np)
    G = c.rounded(Go)
    f = ibfe.ib_spread(c.plan, c.pos, c.to_dev(G))
    assert rel_l2(np_(f), c.orc.spread_nodal(c.x_np, G)) <= 1e-5
    c2 = case("block32", order=order)
    fl = ibfe.Fluid(c2.prob.grid.n, c2.prob.grid.h, 1.0, 0.02, 1e-3)
    u = c2.u.clone()
    x0 = c2.x_np.copy()
    G1, f1, U1, _ = ibfe.ib_step(c2.plan, fl, c2.mats, c2.pos, u)
    Gs, fs, us, _, Us, x1o = OF.ib_step(c2.orc, x0, c2.u_np, 1.0, 0.02, 1e-3)
    x1 = I.from_split(np_(c2.pos.cell), np_(c2.pos.off), c2.prob.grid)
    assert rel_l2(np_(G1), Gs) <= 1e-5
    assert rel_l2(np_(u), us) <= 1e-5
    assert rel_l2(x1 - x0, x1o - x0) <= 1e-5
