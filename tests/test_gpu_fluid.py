"""GPU parity of the fluid step and the explicit IB step (Section 4.2)
against the FP64 oracle, whose discrete Helmholtz and Poisson solves are
exact (FFT-diagonalised).

The GPU solves them with a fixed number of multigrid V-cycles, so parity is
the multigrid's convergence plus rounding: FP32 plans 1e-5 relative L2 on
u^{n+1}, U, G, f and the displacement, 2e-5 on the pressure; FP64 plans,
with enough cycles, 1e-10.
"""
import numpy as np
import pytest

from oracle import fluid as OF
from paper_2503_22695_gb300 import inputs as I

from helpers import Case, np_, rel_l2

pytestmark = pytest.mark.gpu

RHO, MU, DT = 1.0, 0.02, 2e-4


def _fields(n, fp64, seed):
    g = I.Grid(tuple(n), 1.0 / n[0])
    rng = np.random.Generator(np.random.PCG64(seed))
    u = I.fourier_velocity(g, 6, rng, dtype=np.float64)
    u = u + 0.1 * rng.normal(size=u.shape)           # not solenoidal: the projection acts
    f = 50.0 * rng.normal(size=u.shape)
    dt = np.float64 if fp64 else np.float32
    return g, u.astype(dt).astype(np.float64), f.astype(dt).astype(np.float64)


def _dev(a, fp64):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda",
                                                         torch.float64 if fp64 else torch.float32)


@pytest.mark.parametrize("n,fp64", [((32, 32, 32), False), ((64, 64, 64), False),
                                    ((32, 16, 48), False), ((96, 96, 96), False),
                                    ((32, 32, 32), True), ((48, 24, 40), True)])
def test_fluid_step_matches_oracle(n, fp64):
    from paper_2503_22695_gb300 import ibfe
    g, u, f = _fields(n, fp64, seed=100 + n[0] + n[2])
    fl = ibfe.Fluid(g.n, g.h, RHO, MU, DT, precision=ibfe.IB_FP64 if fp64 else ibfe.IB_FP32_SPLIT)
    if fp64:
        fl.set_cycles(6, 24)
    un, p, res = ibfe.ib_fluid_step(fl, _dev(u, fp64), _dev(f, fp64), residuals=True)
    _, po, uo = OF.fluid_step(u, f, RHO, MU, DT, g.h)
    tu, tp = (1e-10, 1e-10) if fp64 else (1e-5, 2e-5)
    assert rel_l2(np_(un), uo) <= tu
    assert rel_l2(np_(p), po) <= tp
    assert res[0] <= (1e-11 if fp64 else 1e-5) and res[1] <= (1e-11 if fp64 else 1e-5), res
    # the result is discretely solenoidal
    div = OF.divergence(np_(un).astype(np.float64), g.h)
    assert np.abs(div).max() <= (1e-9 if fp64 else 2e-5) * np.abs(uo).max() / g.h


def test_fluid_step_in_place_and_reproducible():
    import torch
    from paper_2503_22695_gb300 import ibfe
    g, u, f = _fields((64, 32, 32), False, seed=5)
    fl = ibfe.Fluid(g.n, g.h, RHO, MU, DT)
    ud, fd = _dev(u, False), _dev(f, False)
    a, pa, _ = ibfe.ib_fluid_step(fl, ud, fd)
    b, pb, _ = ibfe.ib_fluid_step(fl, ud, fd)
    assert torch.equal(a, b) and torch.equal(pa, pb)
    uin = ud.clone()
    c, pc, _ = ibfe.ib_fluid_step(fl, uin, fd, u_next=uin)
    assert c.data_ptr() == uin.data_ptr()
    assert torch.equal(c, a) and torch.equal(pc, pa)
    # the graph replay (no residuals) and the direct launches (residuals)
    # run the same kernels in the same order
    d, pd, res = ibfe.ib_fluid_step(fl, ud, fd, residuals=True)
    assert torch.equal(d, a) and torch.equal(pd, pa) and res[1] < 1e-5
    assert fl.cycles() == [2, 6]
    # no force: the same as a zero force
    z, pz, _ = ibfe.ib_fluid_step(fl, ud, None)
    z2, pz2, _ = ibfe.ib_fluid_step(fl, ud, torch.zeros_like(fd))
    assert torch.equal(z, z2) and torch.equal(pz, pz2)


def test_fluid_levels_and_argument_checks():
    from paper_2503_22695_gb300 import ibfe
    assert ibfe.Fluid((256, 256, 256), 1 / 256, 1.0, 0.01, 1e-4).levels() == 6   # 256 .. 8
    assert ibfe.Fluid((32, 16, 48), 1 / 32, 1.0, 0.01, 1e-4).levels() == 4      # .. (4, 2, 6)
    assert ibfe.Fluid((40, 40, 6), 1 / 40, 1.0, 0.01, 1e-4).levels() == 2       # (20, 20, 3)
    with pytest.raises(ibfe.IBError) as e:
        ibfe.Fluid((33, 32, 32), 1 / 32, 1.0, 0.01, 1e-4)
    assert e.value.code == ibfe.IB_ERR_UNSUPPORTED
    for bad in [(0.0, 0.01, 1e-4), (1.0, -1.0, 1e-4), (1.0, 0.01, 0.0)]:
        with pytest.raises(ibfe.IBError) as e:
            ibfe.Fluid((32, 32, 32), 1 / 32, *bad)
        assert e.value.code == ibfe.IB_ERR_INVALID_ARG
    fl = ibfe.Fluid((32, 32, 32), 1 / 32, 1.0, 0.01, 1e-4)
    with pytest.raises(ibfe.IBError):
        fl.set_cycles(0, 8)


def test_fluid_odd_coarsest_level_converges():
    """(40, 40, 6) coarsens once to (20, 20, 3): the coarsest solve uses
    weighted Jacobi (odd dimension); more cycles reach the same solution."""
    from paper_2503_22695_gb300 import ibfe
    g, u, f = _fields((40, 40, 6), False, seed=9)
    fl = ibfe.Fluid(g.n, g.h, RHO, MU, DT)
    fl.set_cycles(2, 40)
    un, p, res = ibfe.ib_fluid_step(fl, _dev(u, False), _dev(f, False), residuals=True)
    _, po, uo = OF.fluid_step(u, f, RHO, MU, DT, g.h)
    assert rel_l2(np_(un), uo) <= 1e-5
    assert rel_l2(np_(p), po) <= 1e-4


@pytest.mark.parametrize("name", ["block32", "block64", "shell128"])
def test_ib_step_matches_oracle(name):
    """One explicit IB step: G and f of x^n, u^{n+1}, U (interpolated at x^n)
    and the displacement dt U, against the oracle's step on the same inputs."""
    import torch
    from paper_2503_22695_gb300 import ibfe
    prob = {"block32": lambda: I.block_problem(fp64=False),
            "block64": lambda: I.block_problem(),
            "shell128": lambda: I.shell_problem()}[name]()
    c = Case(prob)
    g = prob.grid
    dt = 1e-3
    fl = ibfe.Fluid(g.n, g.h, RHO, MU, dt, precision=ibfe.IB_FP64 if c.fp64 else ibfe.IB_FP32_SPLIT)
    if c.fp64:
        fl.set_cycles(6, 24)
    u = c.u.clone()
    x0 = c.x_np.copy()
    G, f, U, p = ibfe.ib_step(c.plan, fl, c.mats, c.pos, u)
    torch.cuda.synchronize()
    Go, fo, uo, po, Uo, x1o = OF.ib_step(c.orc, x0, c.u_np, RHO, MU, dt)
    if c.fp64:
        x1 = np_(c.pos.x64)
    else:
        x1 = I.from_split(np_(c.pos.cell), np_(c.pos.off), g)
        assert np_(c.pos.off).min() >= 0.0 and np_(c.pos.off).max() < 1.0
    t = 1e-10 if c.fp64 else 1e-5
    assert rel_l2(np_(G), Go) <= t
    assert rel_l2(np_(f), fo) <= t
    assert rel_l2(np_(u), uo) <= t
    assert rel_l2(np_(U), Uo) <= t
    assert rel_l2(x1 - x0, x1o - x0) <= t
    # the positions were advanced in place: a second step starts from x^{n+1}
    G2, _, _, _ = ibfe.ib_step(c.plan, fl, c.mats, c.pos, u)
    G2o, _ = c.orc.fe_force(x1)
    assert rel_l2(np_(G2), G2o) <= (1e-10 if c.fp64 else 1e-5)
