"""GPU parity of the nodal quadrature rule (Section 4.4: the coupling points
are the nodes) against the oracle's nodal functions, on the same seeded
inputs as the Gauss-rule tests.  Tolerances as there: FP32 split plans 1e-5
(spread force), 1e-6 (interpolated velocity), 2e-5 (adjoint outputs); FP64
plans 1e-12."""
import numpy as np
import pytest

from paper_2503_22695_gb300 import inputs as I

from helpers import Case, np_, rel_l2

pytestmark = pytest.mark.gpu

TOL32 = dict(G=1e-5, f=1e-5, U=1e-6, adj=2e-5)
TOL64 = 1e-12
NODAL = 1


def tol(case, key):
    return TOL64 if case.fp64 else TOL32[key]


_cache = {}


def case(name):
    if name not in _cache:
        p = {"block64": lambda: I.block_problem(),
             "block32": lambda: I.block_problem(fp64=False),
             "seam32": lambda: I.block_problem(seed=1001, fp64=False, centre=(0.01, 0.985, 0.5)),
             "seam64": lambda: I.block_problem(seed=1002, fp64=True, centre=(0.99, 0.5, 0.012)),
             "shell128": lambda: I.shell_problem(),
             "shell256": lambda: I.shell_sheets_problem()}[name]()
        _cache[name] = Case(p, quad=NODAL)
    return _cache[name]


SMALL = ["block64", "block32", "seam32", "seam64", "shell128"]


@pytest.mark.parametrize("name", SMALL + ["shell256"])
def test_nodal_forward(name):
    c = case(name)
    G, f, U = c.ibfe.ib_forward(c.plan, c.mats, c.pos, c.u)
    Go, _ = c.orc.fe_force(c.x_np)
    assert rel_l2(np_(G), Go) <= tol(c, "G")
    Gr = c.rounded(Go)
    # spreading of the same nodal forces on both sides
    f1 = c.ibfe.ib_spread(c.plan, c.pos, c.to_dev(Gr))
    fo = c.orc.spread_nodal(c.x_np, Gr)
    assert rel_l2(np_(f1), fo) <= tol(c, "f")
    assert np.all(np_(f1)[fo == 0] == 0)
    assert rel_l2(np_(f), c.orc.spread_nodal(c.x_np, np_(G))) <= tol(c, "f")
    Uo = c.orc.interp_nodal(c.x_np, c.u_np)
    assert rel_l2(np_(U), Uo) <= tol(c, "U")
    assert np.array_equal(np_(U), np_(c.ibfe.ib_interp(c.plan, c.pos, c.u)))


@pytest.mark.parametrize("name", SMALL)
def test_nodal_adjoint_identity_on_device(name):
    c = case(name)
    G = c.rounded(np.random.default_rng(5).normal(size=(3, c.prob.n_nodes)))
    f = np_(c.ibfe.ib_spread(c.plan, c.pos, c.to_dev(G)))
    U = np_(c.ibfe.ib_interp(c.plan, c.pos, c.u))
    lhs = c.prob.grid.h ** 3 * np.sum(f * c.u_np)
    assert lhs == pytest.approx(np.sum(G * U), rel=1e-11 if c.fp64 else 1e-5)


@pytest.mark.parametrize("name", SMALL + ["shell256"])
def test_nodal_adjoints(name):
    c = case(name)
    rng = np.random.default_rng(6)
    n = c.prob.n_nodes
    G = c.rounded(c.orc.fe_force(c.x_np)[0])
    gf = c.rounded(rng.normal(size=c.plan.grid_shape()))
    gU = c.rounded(rng.normal(size=(3, n)))
    t = tol(c, "adj")
    gG, gx = c.ibfe.ib_spread_adj(c.plan, c.pos, c.to_dev(G), c.to_dev(gf))
    gGo, gxo = c.orc.spread_nodal_adj(c.x_np, G, gf)
    assert rel_l2(np_(gG), gGo) <= t and rel_l2(np_(gx), gxo) <= t
    gu, gx2 = c.ibfe.ib_interp_adj(c.plan, c.pos, c.u, c.to_dev(gU))
    guo, gx2o = c.orc.interp_nodal_adj(c.x_np, c.u_np, gU)
    assert rel_l2(np_(gu), guo) <= t and rel_l2(np_(gx2), gx2o) <= t
    # fused backward: gx = Hv(gG_s) + (df/dx)^T gf + (dU/dx)^T gU
    gxb, gub, gpb = c.ibfe.ib_backward(c.plan, c.mats, c.pos, c.u, c.to_dev(G), None,
                                       c.to_dev(gf), c.to_dev(gU))
    Hv, gpo = c.orc.fe_force_adj(c.x_np, gGo)
    assert rel_l2(np_(gxb), gxo + gx2o + Hv) <= t
    assert rel_l2(np_(gub), guo) <= t
    for m, mat in enumerate(c.prob.materials):
        k = I.N_PARAMS[mat.model]
        assert rel_l2(gpb[m, :k].cpu().numpy(), gpo[m, :k]) <= t


def test_nodal_spread_bitwise_reproducible():
    c = case("shell128")
    Gd = c.to_dev(c.rounded(c.orc.fe_force(c.x_np)[0]))
    f1 = np_(c.ibfe.ib_spread(c.plan, c.pos, Gd))
    for _ in range(3):
        assert np.array_equal(f1, np_(c.ibfe.ib_spread(c.plan, c.pos, Gd)))
