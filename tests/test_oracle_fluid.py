"""Pins for the FP64 fluid step (Section 4.2, Chorin projection on the
periodic MAC grid): the discrete operators against closed forms and against
each other, the exact solves against the stencil, and the step against the
behaviour the scheme fixes (divergence-free result, gradients absorbed by the
pressure, implicit viscous decay of a single mode, momentum balance)."""
import math

import numpy as np
import pytest

import oracle
from oracle import fluid as F
from paper_2503_22695_gb300 import inputs as I


def _mode(shape, k, h, shift=(0.0, 0.0, 0.0)):
    """cos(2 pi k.x) sampled at lattice points (i + shift) h, shape (n2, n1, n0)."""
    n2, n1, n0 = shape
    L = np.array([n0, n1, n2]) * h
    x0 = (np.arange(n0) + shift[0]) * h
    x1 = (np.arange(n1) + shift[1]) * h
    x2 = (np.arange(n2) + shift[2]) * h
    th = (2 * math.pi * k[0] * x0 / L[0])[None, None, :] + \
         (2 * math.pi * k[1] * x1 / L[1])[None, :, None] + \
         (2 * math.pi * k[2] * x2 / L[2])[:, None, None]
    return np.cos(th)


@pytest.mark.parametrize("shape,k", [((8, 8, 8), (1, 0, 0)), ((16, 12, 10), (2, -3, 1)),
                                     ((6, 10, 14), (0, 4, 5))])
def test_laplacian_of_a_mode_is_its_symbol(shape, k):
    """Lap_h cos(2 pi k.x) = sum_d (2 cos(2 pi k_d / n_d) - 2)/h^2 cos(2 pi k.x)."""
    h = 1.0 / 16
    m = _mode(shape, k, h, shift=(0.3, 0.1, 0.7))
    n2, n1, n0 = shape
    lam = sum((2 * math.cos(2 * math.pi * kd / nd) - 2) / h ** 2
              for kd, nd in zip(k, (n0, n1, n2)))
    np.testing.assert_allclose(F.laplacian(m, h), lam * m, atol=1e-10 * abs(lam) + 1e-12)
    # second order towards the continuum -|2 pi k / L|^2 as h -> 0
    if k == (1, 0, 0):
        errs = []
        for n in (16, 32, 64):
            hh = 1.0 / n
            lam_h = (2 * math.cos(2 * math.pi / n) - 2) / hh ** 2
            errs.append(abs(lam_h + (2 * math.pi) ** 2))
        assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.01)
        assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.01)


def test_divergence_of_gradient_is_laplacian_and_fourier_fields_are_solenoidal():
    """div_h grad_h = Lap_h on the MAC grid (face / centre shifts consistent),
    and the seeded divergence-free Fourier fields (built from the MAC-modified
    wavevector) have zero discrete divergence under this divergence."""
    rng = np.random.default_rng(1)
    h = 1.0 / 12
    p = rng.normal(size=(10, 12, 14))
    np.testing.assert_allclose(F.divergence(F.gradient(p, h), h), F.laplacian(p, h),
                               atol=1e-10 * np.abs(F.laplacian(p, h)).max())
    g = I.Grid((16, 12, 20), 1.0 / 16)
    u = I.fourier_velocity(g, 6, np.random.Generator(np.random.PCG64(3)), dtype=np.float64)
    assert np.abs(F.divergence(u, g.h)).max() < 1e-10 * np.abs(u).max() / g.h
    # a plain shifted mode is not solenoidal: the check has teeth
    assert np.abs(F.divergence(u[[1, 2, 0]], g.h)).max() > 1e-2 * np.abs(u).max() / g.h


@pytest.mark.parametrize("alpha,beta", [(50.0, 0.01), (1.0, 1.0), (1e4, 3e-3)])
def test_helmholtz_solve_satisfies_the_stencil(alpha, beta):
    rng = np.random.default_rng(2)
    h = 1.0 / 16
    r = rng.normal(size=(16, 12, 8))
    phi = F.solve_helmholtz(r, alpha, beta, h)
    res = alpha * phi - beta * F.laplacian(phi, h) - r
    assert np.abs(res).max() < 1e-11 * np.abs(r).max()


def test_poisson_solve_satisfies_the_stencil_with_zero_mean():
    rng = np.random.default_rng(3)
    h = 1.0 / 20
    r = rng.normal(size=(10, 20, 14))
    phi = F.solve_poisson(r, h)
    assert abs(phi.mean()) < 1e-13 * np.abs(phi).max()
    res = F.laplacian(phi, h) - (r - r.mean())
    assert np.abs(res).max() < 1e-10 * np.abs(r).max()


def test_projection_result_is_solenoidal_and_idempotent():
    rng = np.random.default_rng(4)
    h = 1.0 / 16
    u = rng.normal(size=(3, 16, 16, 16))
    f = rng.normal(size=(3, 16, 16, 16))
    _, p, un = F.fluid_step(u, f, rho=1.0, mu=0.02, dt=1e-3, h=h)
    assert np.abs(F.divergence(un, h)).max() < 1e-9 * np.abs(un).max() / h
    assert abs(p.mean()) < 1e-12 * np.abs(p).max()
    # a solenoidal field with no force and no viscosity is left as it is
    _, p2, un2 = F.fluid_step(un, np.zeros_like(f), rho=1.0, mu=0.0, dt=1e-3, h=h)
    np.testing.assert_allclose(un2, un, atol=1e-11 * np.abs(un).max())
    assert np.abs(p2).max() < 1e-9 * np.abs(un).max() * h


def test_gradient_forcing_is_absorbed_by_the_pressure():
    """f = grad_h phi on a fluid at rest (mu = 0): the velocity stays zero and
    the pressure is phi / rho up to its mean (Section 4.2 with u^n = 0)."""
    rng = np.random.default_rng(5)
    h = 1.0 / 12
    phi = rng.normal(size=(12, 12, 12))
    f = F.gradient(phi, h)
    rho, dt = 1.3, 2e-3
    _, p, un = F.fluid_step(np.zeros_like(f), f, rho=rho, mu=0.0, dt=dt, h=h)
    assert np.abs(un).max() < 1e-10 * np.abs(f).max() * dt / rho
    np.testing.assert_allclose(p, (phi - phi.mean()) / rho, atol=1e-10 * np.abs(phi).max())


def test_viscous_decay_of_a_solenoidal_mode():
    """A divergence-free single mode with no force decays by the implicit-Euler
    factor 1 / (1 - dt mu lambda(k) / rho) in one step (lambda < 0)."""
    g = I.Grid((16, 16, 16), 1.0 / 16)
    h = g.h
    shape = (16, 16, 16)
    k = (2, 1, 0)
    u = np.zeros((3,) + shape)
    # u = (0, 0, w(x, y)): solenoidal for any w independent of z
    u[2] = _mode(shape, k, h, shift=(0.5, 0.5, 0.0))
    assert np.abs(F.divergence(u, h)).max() < 1e-12
    rho, mu, dt = 1.0, 0.05, 4e-3
    lam = sum((2 * math.cos(2 * math.pi * kd / 16) - 2) / h ** 2 for kd in k)
    _, p, un = F.fluid_step(u, np.zeros_like(u), rho, mu, dt, h)
    np.testing.assert_allclose(un, u / (1 - dt * mu * lam / rho), atol=1e-12)
    assert np.abs(p).max() < 1e-9


def test_kinetic_energy_does_not_grow_without_forcing():
    g = I.Grid((16, 16, 16), 1.0 / 16)
    u = I.fourier_velocity(g, 8, np.random.Generator(np.random.PCG64(9)), dtype=np.float64)
    e0 = np.sum(u * u)
    for _ in range(3):
        _, _, u = F.fluid_step(u, np.zeros_like(u), 1.0, 0.01, 1e-3, g.h)
        e1 = np.sum(u * u)
        assert e1 <= e0 * (1 + 1e-14)
        e0 = e1


def test_ib_step_momentum_balance_and_position_update():
    """One explicit IB step on the elastic block: the spread force carries no
    net force (internal forces), so the mean velocity is unchanged; the nodes
    move by dt times the interpolated new velocity."""
    p = I.block_problem(seed=1000, n=16, blocks=(4, 4, 2), fp64=True)
    m = oracle.Model(p)
    rho, mu, dt = 1.0, 0.01, 5e-4
    u = p.u.astype(np.float64)
    G, f, un, pr, U, x1 = F.ib_step(m, p.x, u, rho, mu, dt)
    assert np.abs(G).max() > 0
    assert np.abs(f.sum(axis=(1, 2, 3))).max() < 1e-10 * np.abs(f).max()
    np.testing.assert_allclose(un.mean(axis=(1, 2, 3)), u.mean(axis=(1, 2, 3)),
                               atol=1e-12 * np.abs(u).max())
    assert np.abs(F.divergence(un, p.grid.h)).max() < 1e-9 * np.abs(un).max() / p.grid.h
    np.testing.assert_allclose(U, m.interp(p.x, un), rtol=0, atol=0)
    np.testing.assert_allclose(x1, p.x + dt * U, rtol=0, atol=0)
