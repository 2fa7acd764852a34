"""FP64 fluid step of the explicit IB scheme -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this module; the product path never loads it.

Section 4.2 splits each time step by Chorin's projection on the MAC grid:

    rho/dt (u* - u^n) - mu Lap_h u* = f^{n+1}          (Helmholtz)
    Lap_h p^{n+1} = (1/dt) div_h u*                    (Poisson)
    u^{n+1} = u* - dt grad_h p^{n+1}                   (correction)

and moves the structure with the interpolated new velocity,
(X^{n+1} - X^n)/dt = int u^{n+1} delta(x - X^n) dx, the force density f^{n+1}
being spread from the nodal forces of the configuration X^n.

Here the box is periodic (the domain of the coupling operators), so every
discrete operator is a circulant convolution and the discrete Helmholtz and
Poisson equations are solved exactly by diagonalising them with the FFT
(numpy's, a library primitive): the discrete Laplacian multiplies the Fourier
mode k by lambda(k) = sum_d (2 cos(2 pi k_d / n_d) - 2) / h^2.  This is the
definition of the discrete solution the multigrid of the GPU path iterates
towards, not an approximation of it.

MAC layout (shared convention with the coupling operators): fields are
[3][n2][n1][n0] (component, z, y, x); component c lives at the lower c-face,
the pressure at cell centres.  Hence
    (div u)(i)    = sum_c (u^c(i + e_c) - u^c(i)) / h
    (grad p)^c(i) = (p(i) - p(i - e_c)) / h
so that div grad = Lap_h (the 7-point Laplacian) exactly.
"""
from __future__ import annotations

import numpy as np

# spatial axis of field arrays [..., n2, n1, n0] for component / direction c
_AXIS = {0: -1, 1: -2, 2: -3}


def _roll(a, c, s):
    """a(i + s e_c) on the periodic lattice."""
    return np.roll(a, -s, axis=_AXIS[c])


def laplacian(phi, h):
    """7-point Laplacian of a scalar lattice field [n2][n1][n0] (periodic)."""
    out = -6.0 * phi
    for c in range(3):
        out = out + _roll(phi, c, 1) + _roll(phi, c, -1)
    return out / (h * h)


def divergence(u, h):
    """Cell-centred divergence of a MAC field u [3][n2][n1][n0]."""
    return sum(_roll(u[c], c, 1) - u[c] for c in range(3)) / h


def gradient(p, h):
    """Face-centred gradient [3][n2][n1][n0] of a cell-centred p."""
    return np.stack([(p - _roll(p, c, -1)) / h for c in range(3)])


def symbol(shape, h):
    """lambda(k) of the 7-point Laplacian for a lattice of shape (n2, n1, n0)."""
    lam = np.zeros(shape)
    for ax, n in zip((0, 1, 2), shape):
        k = np.arange(n)
        s = (2.0 * np.cos(2.0 * np.pi * k / n) - 2.0) / (h * h)
        sh = [1, 1, 1]
        sh[ax] = n
        lam = lam + s.reshape(sh)
    return lam


def solve_helmholtz(rhs, alpha, beta, h):
    """phi with (alpha - beta Lap_h) phi = rhs, alpha > 0 (exact, by FFT)."""
    lam = symbol(rhs.shape, h)
    return np.real(np.fft.ifftn(np.fft.fftn(rhs) / (alpha - beta * lam)))


def solve_poisson(rhs, h):
    """The mean-zero phi with Lap_h phi = rhs - mean(rhs) (exact, by FFT)."""
    lam = symbol(rhs.shape, h)
    r = np.fft.fftn(rhs)
    lam[0, 0, 0] = 1.0
    r = r / lam
    r[0, 0, 0] = 0.0
    return np.real(np.fft.ifftn(r))


def fluid_step(u, f, rho, mu, dt, h):
    """One projection step of Section 4.2: (u*, p^{n+1}, u^{n+1})."""
    u = np.asarray(u, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    a = rho / dt
    ustar = np.stack([solve_helmholtz(a * u[c] + f[c], a, mu, h) for c in range(3)])
    p = solve_poisson(divergence(ustar, h) / dt, h)
    unew = ustar - dt * gradient(p, h)
    return ustar, p, unew


def ib_step(model, x, u, rho, mu, dt):
    """One explicit IB step (Section 4.2) from nodes x^n [3][N] and u^n.

    The nodal forces G^{n+1} of the configuration x^n are spread at x^n, the
    fluid is advanced by `fluid_step`, the new velocity is interpolated at x^n
    (U, with the lumped projection onto the nodes) and the nodes move by
    dt U.  `model` is an oracle.Model holding mesh, grid and materials.
    Returns (G, f, u^{n+1}, p, U, x^{n+1}).
    """
    h = model.grid_py.h
    G, _ = model.fe_force(x)
    f = model.spread(x, G)
    _, p, unew = fluid_step(u, f, rho, mu, dt, h)
    U = model.interp(x, unew)
    return G, f, unew, p, U, x + dt * U
