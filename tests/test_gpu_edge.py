"""GPU parity on the hard inputs of the method, against the FP64 oracle.

* Positions on the grid lines: split offsets exactly 0 and exactly
  1 - 2^-24, nodes on tile faces and across the periodic seam, with the
  Gauss rule and with the nodal rule (whose coupling points are the nodes
  themselves, so the kernel is evaluated exactly at the support edges).
* One 8^3-cell tile holding 2,744 Gauss points (three work items of one
  tile, merged).
* Penalty tethers at kappa = 5e6 (the aortic-valve tube of Section 5) beside
  elastic forces thousands of times smaller: the spread force is compared on
  the faces farther than 4 h from every tethered node as well as globally.
* Near incompressibility: kappa / a = 2e4 with |J - 1| <= 6e-5 while
  |F - I| is near 5e-2, where tr(F - I) cancels in J - 1.

Tolerances are the stated FP32 ones: relative L2 1e-5 for forces (nodal and
spread), 1e-6 for interpolated velocities, 2e-5 for adjoints; each field is
also held per face / per node against its own largest magnitude.
"""
import numpy as np
import pytest

from paper_2503_22695_gb300 import inputs as I

from helpers import Case, np_, rel_l2

pytestmark = pytest.mark.gpu


def max_rel(a, b):
    """Largest per-entry error over the largest reference magnitude."""
    return float(np.abs(np.asarray(a) - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("quad", [0, 1])
@pytest.mark.parametrize("which", ["aligned", "dense"])
def test_spread_interp_on_hard_positions(which, quad):
    p = I.grid_aligned_problem() if which == "aligned" else I.dense_tile_problem()
    c = Case(p, quad=quad)
    rng = np.random.default_rng(31)
    G = c.rounded(rng.normal(size=(3, p.n_nodes)))
    f = np_(c.ibfe.ib_spread(c.plan, c.pos, c.to_dev(G)))
    if quad:
        fo = c.orc.spread_nodal(c.x_np, G)
        Uo = c.orc.interp_nodal(c.x_np, c.u_np)
    else:
        fo = c.orc.spread(c.x_np, G)
        Uo = c.orc.interp(c.x_np, c.u_np)
    assert rel_l2(f, fo) <= 1e-5
    assert max_rel(f, fo) <= 1e-6
    assert np.all(f[fo == 0] == 0)
    U = np_(c.ibfe.ib_interp(c.plan, c.pos, c.u))
    assert rel_l2(U, Uo) <= 1e-6
    assert max_rel(U, Uo) <= 1e-6
    # the same inputs twice: the same bits
    assert np.array_equal(f, np_(c.ibfe.ib_spread(c.plan, c.pos, c.to_dev(G))))


def test_offsets_are_the_adversarial_values():
    p = I.grid_aligned_problem()
    vals = set(np.unique(p.off).tolist())
    assert vals == {0.0, float(np.float32(1) - np.float32(2.0 ** -24))}
    assert p.cell.min() < 0 < p.cell.max()          # straddles the seam in x
    q = I.dense_tile_problem()
    assert q.n_gauss > 2 * 1024


def _face_positions(grid, comp):
    n0, n1, n2 = grid.n
    h = grid.h
    s = [0.5, 0.5, 0.5]
    s[comp] = 0.0
    z, y, x = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
    return [(x + s[0]) * h, (y + s[1]) * h, (z + s[2]) * h]


def test_spread_with_stiff_tethers_far_field():
    # The block has moved rigidly by about a quarter cell (small elastic
    # strain, node noise 0.002 h) and the tethers of its x-minimum face pull
    # it back: their forces are more than a thousand times the elastic ones.
    import dataclasses
    import torch
    p = I.block_problem(seed=1040, fp64=False, noise=0.002)
    x = p.x + np.array([0.23, -0.17, 0.11])[:, None] * p.grid.h
    cell, off = I.to_split(x, p.grid)
    p = dataclasses.replace(p, x=x, cell=cell, off=off)
    c = Case(p)
    X = p.X
    nodes = np.flatnonzero(X[0] <= X[0].min() + 1e-12).astype(np.int32)
    kappa = 5e6
    c.ibfe.ib_plan_set_penalty(c.plan, torch.from_numpy(nodes).cuda(), kappa, None)
    Ge, _ = c.orc.fe_force(c.x_np)
    Gp, _ = c.orc.penalty(c.x_np, nodes, kappa)
    ratio = np.abs(Gp).max() / np.abs(Ge).max()
    assert ratio > 1e3                                  # the tethers dominate
    # the device's nodal force with the tethers
    Gd, _ = c.ibfe.ib_fe_force(c.plan, c.mats, c.pos, energy=True)
    assert rel_l2(np_(Gd), Ge + Gp) <= 1e-5
    G = c.rounded(Ge + Gp)
    f = np_(c.ibfe.ib_spread(c.plan, c.pos, c.to_dev(G)))
    fo = c.orc.spread(c.x_np, G)
    assert rel_l2(f, fo) <= 1e-5
    # faces farther than 4 h from every tethered node (periodic distance)
    g = p.grid
    L = g.n[0] * g.h
    tx = c.x_np[:, nodes]
    far_err, far_ref = 0.0, 0.0
    nfar = 0
    for comp in range(3):
        P = _face_positions(g, comp)
        d2 = np.full(P[0].shape, np.inf)
        for k in range(len(nodes)):
            dd = 0.0
            for d in range(3):
                t = np.abs(P[d] - tx[d, k]) % L
                t = np.minimum(t, L - t)
                dd = dd + t * t
            d2 = np.minimum(d2, dd)
        far = (d2 > (4 * g.h) ** 2) & (fo[comp] != 0)
        nfar += int(far.sum())
        far_err += float(np.sum((f[comp][far] - fo[comp][far]) ** 2))
        far_ref += float(np.sum(fo[comp][far] ** 2))
    assert nfar > 1000
    assert np.sqrt(far_err / far_ref) <= 1e-5


@pytest.mark.parametrize("model", [I.NEO_HOOKEAN, I.HO])
@pytest.mark.parametrize("precision", ["dfvol", "fp64", "split"])
def test_nearly_incompressible_force_and_hvp(model, precision):
    """kappa / a >= 2e4, |J - 1| <= 6e-5, |F - I| near 5e-2.  With
    IB_FP32_SPLIT_DFVOL (J - 1 from double-float kinematics) the force and
    Hessian-vector product meet the FP32 tolerances.  FP64 plans meet 1e-9:
    the same amplification of rounding by |F - I| / |J - 1| (about 1e3 here)
    acts on double, in the oracle as on the device (8.6e-11 measured).
    IB_FP32_SPLIT forms J - 1 from the FP32 displacement gradient, whose
    rounding (near 1e-7 |F - I|) is amplified by |F - I| / |J - 1|: its stated
    accuracy in this regime is 5e-3 (1.3e-3 measured)."""
    p = I.incompressible_problem(model=model, fp64=precision == "fp64")
    c = Case(p)
    _, J = c.orc.gauss_info(c.x_np)
    assert np.abs(J - 1).max() <= 1e-4
    plan = c.plan
    if precision == "dfvol":
        g = p.grid
        plan = c.ibfe.Plan(c.conn, c.X, g.n, g.h, g.origin, fibres=c.fib, mat_id=c.mat_id,
                           precision=c.ibfe.IB_FP32_SPLIT_DFVOL)
    tol_g, tol_adj = {"dfvol": (1e-5, 2e-5), "fp64": (1e-9, 1e-9), "split": (5e-3, 5e-3)}[
        precision]
    G, en = c.ibfe.ib_fe_force(plan, c.mats, c.pos, energy=True)
    Go, eno = c.orc.fe_force(c.x_np)
    assert rel_l2(np_(G), Go) <= tol_g
    assert en == pytest.approx(eno, rel=max(tol_g, 1e-12))
    v = c.rounded(np.random.default_rng(32).normal(size=(3, p.n_nodes)))
    Hv, gp = c.ibfe.ib_fe_force_adj(plan, c.mats, c.pos, c.to_dev(v))
    Hvo, gpo = c.orc.fe_force_adj(c.x_np, v)
    assert rel_l2(np_(Hv), Hvo) <= tol_adj
    k = I.N_PARAMS[model]
    assert rel_l2(gp[0, :k].numpy(), gpo[0, :k]) <= tol_adj
    if precision == "dfvol":   # the rest of the path is the split one
        f1 = np_(c.ibfe.ib_spread(plan, c.pos, G))
        f2 = np_(c.ibfe.ib_spread(c.plan, c.pos, G))
        assert np.array_equal(f1, f2)
