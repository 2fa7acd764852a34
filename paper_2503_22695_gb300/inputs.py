"""Seeded synthetic inputs for the immersed-boundary coupling step.

This module is shared by the CUDA path's tests/benchmark and by the FP64
oracle's tests.  It holds only input construction -- meshes, fibre fields,
node deformations, periodic velocity fields, material tables and the
conversion of positions to the split (integer cell + FP32 offset) storage
format.  It contains none of the method's arithmetic (no shape functions,
quadrature, stresses, delta kernels, spreading or interpolation).

Geometry stands in for the paper's cardiac models (Section 6: image-based
left ventricle, porcine aortic valve, mitral valve), whose data are not
available: a truncated thick prolate-ellipsoidal shell meshed with trilinear
hexahedra (ventricle-like) and thin curved cylindrical sheets (leaflet-like).

Every array is generated with numpy ``Generator(PCG64(seed))``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# Material model identifiers (same numbering as the C ABI's ib_model).
NEO_HOOKEAN = 0   # Psi = a (I1bar - 3) + kappa/2 (ln J)^2        (Section 6.3)
FIBRE1 = 1        # fibre-reinforced model 1, Psi_2               (Section 3)
HO = 2            # Holzapfel-Ogden, Psi_4                        (Section 3)
STD_REINF = 3     # modified standard reinforcing, Psi_1 (I4f, I5f) (Section 3)
FIBRE2 = 4        # fibre-reinforced model 2, Psi_3               (Section 3)

N_PARAMS = {NEO_HOOKEAN: 2, FIBRE1: 4, HO: 9, STD_REINF: 4, FIBRE2: 5}
PARAM_NAMES = {
    NEO_HOOKEAN: ("a", "kappa"),
    FIBRE1: ("C1", "af", "bf", "kappa"),
    HO: ("a", "b", "af", "bf", "as", "bs", "afs", "bfs", "kappa"),
    STD_REINF: ("GT", "GL", "EL", "kappa"),
    FIBRE2: ("C10", "C01", "af", "bf", "kappa"),
}

# Holzapfel-Ogden defaults in kPa-scaled units: a, b, af, bf are the centres of
# the batched parameter sweep; as, bs, afs, bfs are the left-ventricle table of
# Section 6.1 converted from dyn/cm^2 to kPa (1 kPa = 1e4 dyn/cm^2);
# kappa = 1e6 dyn/cm^2 = 100 kPa.
HO_DEFAULT = (0.059, 8.02, 18.47, 16.03, 0.5562, 0.7746, 0.3905, 1.695, 100.0)
# Mitral anterior leaflet (Section 6.3 table) in kPa: C1 = 17.4, af = 31.3, bf = 55.93.
FIBRE1_LEAFLET = (17.4, 31.3, 55.93, 100.0)
# Cook's membrane (Section 4 table) in its printed unit dyn/cm^2:
# G_T = 8, G_L = 160, E_L = 1200, kappa_stab = 112.
STD_REINF_COOK = (8.0, 160.0, 1200.0, 112.0)
# Aortic valve leaflets (Section 6.2 table) in kPa: C10 = 1.21, C01 = 7.99,
# af = 24.23, bf = 57.62, kappa = 100.
FIBRE2_AV = (1.21, 7.99, 24.23, 57.62, 100.0)

# VTK hexahedron corner order in the reference cube [-1,1]^3.
HEX_CORNERS = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                        [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], dtype=np.int64)


@dataclasses.dataclass
class Grid:
    """Periodic MAC grid: n[d] cells of width h, box [origin, origin + n h)."""
    n: tuple
    h: float
    origin: tuple = (0.0, 0.0, 0.0)


@dataclasses.dataclass
class Material:
    model: int
    params: tuple
    active: float = 0.0   # active fibre tension T_a at the current time (Section 6.1)


@dataclasses.dataclass
class Problem:
    """One coupling-step input set (all arrays in structure-of-arrays layout)."""
    name: str
    grid: Grid
    conn: np.ndarray        # int32 [8][E], VTK hex order
    X: np.ndarray           # float32 (or float64) [3][N] reference coordinates
    fibres: np.ndarray      # float32 (or float64) [6][E]: e_f (3) then e_s (3)
    mat_id: np.ndarray      # int32 [E]
    materials: List[Material]
    x: np.ndarray           # float64 [3][N] current positions (before storage)
    cell: np.ndarray        # int32 [3][N] split position: integer cell
    off: np.ndarray         # float32 [3][N] split position: offset in [0,1)
    u: np.ndarray           # float32 (or float64) [3][n2][n1][n0] MAC velocity
    fp64: bool = False

    @property
    def n_nodes(self) -> int:
        return int(self.X.shape[1])

    @property
    def n_elems(self) -> int:
        return int(self.conn.shape[1])

    @property
    def n_gauss(self) -> int:
        """Points of the element rule: 8 per hexahedron, 4 per tetrahedron
        (linear or quadratic)."""
        return (8 if self.conn.shape[0] == 8 else 4) * self.n_elems


# ----------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------

def _structured_hex(nodes_ijk: np.ndarray, periodic_i: bool = False):
    """Connectivity of a structured (ni x nj x nk) node lattice.

    nodes_ijk has shape (ni, nj, nk, 3).  Element (i,j,k) uses lattice corners
    (i+di, j+dj, k+dk) in VTK order with (di,dj,dk) = (corner+1)/2.  With
    periodic_i the i index wraps (closed circumferential direction).
    Returns conn int32 [8][E] and coordinates float64 [3][N].
    """
    ni, nj, nk, _ = nodes_ijk.shape
    ei = ni if periodic_i else ni - 1
    ej, ek = nj - 1, nk - 1
    idx = np.arange(ni * nj * nk).reshape(ni, nj, nk)
    I, J, K = np.meshgrid(np.arange(ei), np.arange(ej), np.arange(ek), indexing="ij")
    conn = np.empty((8, ei * ej * ek), dtype=np.int64)
    for a, (ci, cj, ck) in enumerate(HEX_CORNERS):
        ii = (I + (ci + 1) // 2) % ni
        jj = J + (cj + 1) // 2
        kk = K + (ck + 1) // 2
        conn[a] = idx[ii, jj, kk].ravel()
    X = nodes_ijk.reshape(-1, 3).T.copy()
    return conn, X


def _orient(conn: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Flip element corner order where the corner-0 edge triple is left-handed.

    Plain geometry: the triple product of the three edges leaving corner 0.
    """
    p0 = X[:, conn[0]]
    e1 = X[:, conn[1]] - p0
    e3 = X[:, conn[3]] - p0
    e4 = X[:, conn[4]] - p0
    vol = np.einsum("ie,ie->e", np.cross(e1.T, e3.T).T, e4)
    bad = vol < 0
    if bad.any():
        # mirror the local xi axis: swap corners 0<->1, 3<->2, 4<->5, 7<->6
        perm = [1, 0, 3, 2, 5, 4, 7, 6]
        conn = conn.copy()
        conn[:, bad] = conn[perm][:, bad]
    return conn


# The six tetrahedra of a hexahedron around its 0-6 diagonal (VTK corners):
# the paths 0->1->2->6, 0->1->5->6, 0->3->2->6, 0->3->7->6, 0->4->5->6,
# 0->4->7->6.  Hexahedra of one structured grid all split this way agree on
# every shared face diagonal, so the tetrahedral mesh is conforming.
_HEX_TETS = ((0, 1, 2, 6), (0, 1, 5, 6), (0, 3, 2, 6), (0, 3, 7, 6), (0, 4, 5, 6), (0, 4, 7, 6))


def hex_to_tets(conn: np.ndarray, X: np.ndarray, *per_elem):
    """Split hexahedra [8][E] into tetrahedra [4][6E] with positive volume
    (two corners swapped where the triple product is negative); per-element
    arrays ([k][E] or [E]) are repeated for the six children."""
    E = conn.shape[1]
    tets = np.stack([conn[list(t)] for t in _HEX_TETS], axis=2).reshape(4, 6 * E)
    p0 = X[:, tets[0]]
    vol = np.einsum("ie,ie->e", np.cross((X[:, tets[1]] - p0).T, (X[:, tets[2]] - p0).T).T,
                    X[:, tets[3]] - p0)
    flip = vol < 0
    tets[1, flip], tets[2, flip] = tets[2, flip].copy(), tets[1, flip].copy()
    out = [np.ascontiguousarray(tets)]
    for a in per_elem:
        out.append(np.repeat(a, 6, axis=-1))
    return tuple(out)


def box_block(nx: int, ny: int, nz: int, edge: float, centre) -> tuple:
    """A rectangular block of nx*ny*nz cubes of side `edge` centred at `centre`."""
    c = np.asarray(centre, dtype=np.float64)
    gx = (np.arange(nx + 1) - nx / 2) * edge + c[0]
    gy = (np.arange(ny + 1) - ny / 2) * edge + c[1]
    gz = (np.arange(nz + 1) - nz / 2) * edge + c[2]
    P = np.stack(np.meshgrid(gx, gy, gz, indexing="ij"), axis=-1)
    conn, X = _structured_hex(P)
    return _orient(conn, X), X


def ellipsoid_shell(n_c: int, n_l: int, n_t: int, outer=(0.2, 0.2, 0.35), wall=0.05,
                    centre=(0.5, 0.5, 0.5), theta=(math.pi / 40, 7 * math.pi / 12)):
    """Truncated thick prolate-ellipsoidal shell (left-ventricle stand-in).

    Surfaces s in [0,1] (0 = inner/endocardium, 1 = outer/epicardium) are
    ellipsoids with semi-axes outer - (1-s)*wall.  The polar angle theta is
    measured from the apex (-z); the range leaves an open apex cap and a base
    above the equator.  The circumferential angle is closed (periodic).
    Returns conn [8][E], X [3][N], fibres [6][E].

    Fibre field (Section 6.1 describes a rule-based helix angle rotating
    transmurally): alpha = -60 deg + 120 deg * s at the element centroid;
    e_f = cos(alpha) e_circ + sin(alpha) e_long, e_s = outward wall normal.
    """
    ax, ay, az = outer
    c = np.asarray(centre, dtype=np.float64)
    phi = 2 * math.pi * np.arange(n_c) / n_c
    th = np.linspace(theta[0], theta[1], n_l + 1)
    s = np.linspace(0.0, 1.0, n_t + 1)

    def surf(ph, t, ss):
        rx, ry, rz = ax - (1 - ss) * wall, ay - (1 - ss) * wall, az - (1 - ss) * wall
        return np.stack([c[0] + rx * np.sin(t) * np.cos(ph),
                         c[1] + ry * np.sin(t) * np.sin(ph),
                         c[2] - rz * np.cos(t)], axis=-1)

    PH, TH, S = np.meshgrid(phi, th, s, indexing="ij")
    P = surf(PH, TH, S)
    conn, X = _structured_hex(P, periodic_i=True)

    # centroid parameters of each element (same element enumeration order)
    dphi = 2 * math.pi / n_c
    pc = (np.arange(n_c) + 0.5) * dphi
    tc = 0.5 * (th[:-1] + th[1:])
    sc = 0.5 * (s[:-1] + s[1:])
    PC, TC, SC = np.meshgrid(pc, tc, sc, indexing="ij")
    PC, TC, SC = PC.ravel(), TC.ravel(), SC.ravel()
    rx, ry, rz = ax - (1 - SC) * wall, ay - (1 - SC) * wall, az - (1 - SC) * wall
    e_circ = np.stack([-rx * np.sin(TC) * np.sin(PC), ry * np.sin(TC) * np.cos(PC),
                       np.zeros_like(PC)], axis=0)
    e_long = np.stack([rx * np.cos(TC) * np.cos(PC), ry * np.cos(TC) * np.sin(PC),
                       rz * np.sin(TC)], axis=0)
    # outward normal of the ellipsoid x^2/rx^2 + y^2/ry^2 + z^2/rz^2 = 1
    pos = np.stack([rx * np.sin(TC) * np.cos(PC), ry * np.sin(TC) * np.sin(PC),
                    -rz * np.cos(TC)], axis=0)
    nrm = pos / np.stack([rx * rx, ry * ry, rz * rz], axis=0)
    fib = _fibre_frame(e_circ, e_long, nrm, np.deg2rad(-60.0 + 120.0 * SC))
    return _orient(conn, X), X, fib


def _fibre_frame(t1, t2, nrm, alpha):
    """Orthonormal (e_f, e_s): e_f in the tangent plane at angle alpha from t1."""
    t1 = t1 / np.linalg.norm(t1, axis=0)
    n = nrm / np.linalg.norm(nrm, axis=0)
    t2 = t2 - np.sum(t2 * t1, axis=0) * t1
    t2 = t2 / np.linalg.norm(t2, axis=0)
    ef = np.cos(alpha) * t1 + np.sin(alpha) * t2
    ef = ef / np.linalg.norm(ef, axis=0)
    es = n - np.sum(n * ef, axis=0) * ef
    es = es / np.linalg.norm(es, axis=0)
    return np.concatenate([ef, es], axis=0)


def cylinder_sheet(n_a: int, n_x: int, n_t: int, radius=0.15, arc=1.6, length=0.12,
                   thick=0.01, axis_point=(0.5, 0.66, 0.62), facing=-1.0):
    """A thin curved sheet: a cylindrical arc (leaflet stand-in).

    The cylinder axis is parallel to x through axis_point; the arc spans
    angle `arc` around the direction `facing` * e_y; the sheet has n_a
    elements along the arc, n_x along the axis and n_t through the thickness.
    Fibres run along the arc (the long direction); e_s is the sheet normal.
    """
    cx, cy, cz = axis_point
    psi = np.linspace(-arc / 2, arc / 2, n_a + 1)
    xs = np.linspace(cx - length / 2, cx + length / 2, n_x + 1)
    rs = np.linspace(radius - thick / 2, radius + thick / 2, n_t + 1)
    PS, XS, RS = np.meshgrid(psi, xs, rs, indexing="ij")
    P = np.stack([XS, cy + facing * RS * np.cos(PS), cz + RS * np.sin(PS)], axis=-1)
    conn, X = _structured_hex(P)
    pc = 0.5 * (psi[:-1] + psi[1:])
    PC = np.repeat(pc, n_x * n_t)
    e_arc = np.stack([np.zeros_like(PC), -facing * np.sin(PC), np.cos(PC)], axis=0)
    e_ax = np.stack([np.ones_like(PC), np.zeros_like(PC), np.zeros_like(PC)], axis=0)
    nrm = np.stack([np.zeros_like(PC), facing * np.cos(PC), np.sin(PC)], axis=0)
    fib = _fibre_frame(e_arc, e_ax, nrm, np.zeros_like(PC))
    return _orient(conn, X), X, fib


# ----------------------------------------------------------------------------
# deformations, velocity fields, storage format
# ----------------------------------------------------------------------------

def smooth_deformation(X: np.ndarray, rng: np.random.Generator, centre=(0.5, 0.5, 0.5),
                       half_length=0.35, twist=0.3, amp=0.015, axial=0.02,
                       modes=3) -> np.ndarray:
    """Radial + twist deformation of a structure about the z axis.

    x = c + R_z(tau zeta) [(1 + eps(X)) (X_perp - c_perp)] + (1 + eps_z)(X_z - c_z) e_z
    with zeta = (X_z - c_z)/half_length, tau ~ U(+-twist),
    eps = sum_m A_m sin(2 pi k_m . X + phase_m), A_m ~ U(+-amp), k_m integer
    with |k|_inf <= 1, eps_z ~ U(+-axial).
    """
    c = np.asarray(centre, dtype=np.float64)
    tau = rng.uniform(-twist, twist)
    epsz = rng.uniform(-axial, axial)
    eps = np.zeros(X.shape[1])
    for _ in range(modes):
        k = rng.integers(-1, 2, size=3)
        A = rng.uniform(-amp, amp)
        ph = rng.uniform(0, 2 * math.pi)
        eps += A * np.sin(2 * math.pi * (k @ X) + ph)
    zeta = (X[2] - c[2]) / half_length
    ang = tau * zeta
    dx, dy = (1 + eps) * (X[0] - c[0]), (1 + eps) * (X[1] - c[1])
    x = np.empty_like(X)
    x[0] = c[0] + np.cos(ang) * dx - np.sin(ang) * dy
    x[1] = c[1] + np.sin(ang) * dx + np.cos(ang) * dy
    x[2] = c[2] + (1 + epsz) * (X[2] - c[2])
    return x


def fourier_velocity(grid: Grid, n_modes: int, rng: np.random.Generator,
                     kmax: int = 4, dtype=np.float32) -> np.ndarray:
    """A periodic MAC velocity field, a sum of discretely divergence-free modes.

    Component c lives on the lower c-faces: face (i0,i1,i2) of component c is
    at origin + (i + s_c) h with s_c[d] = 0 for d == c and 1/2 otherwise.
    Each mode is Re(A exp(2 pi i k.x)) with integer wavevector |k|_inf <= kmax
    and complex amplitude A orthogonal to the MAC-modified wavevector
    2 sin(pi k_d h)/h, so the discrete MAC divergence of every mode vanishes.
    Returns an array [3][n2][n1][n0].
    """
    n0, n1, n2 = grid.n
    h = grid.h
    L = np.array(grid.n, dtype=np.float64) * h
    o = np.asarray(grid.origin, dtype=np.float64)
    ks, amps = [], []
    for _ in range(n_modes):
        while True:
            k = rng.integers(-kmax, kmax + 1, size=3)
            if np.any(k != 0):
                break
        kt = 2.0 * np.sin(math.pi * k * h / L) / h   # MAC-modified wavevector
        a = rng.normal(size=3)
        b = rng.normal(size=3)
        kn = kt / np.linalg.norm(kt)
        a -= (a @ kn) * kn
        b -= (b @ kn) * kn
        ks.append(k)
        amps.append(a + 1j * b)
    u = np.zeros((3, n2, n1, n0), dtype=np.float64)
    if n_modes == 0:
        return u.astype(dtype)
    # exp(i theta) factorises over the three axes: build, per component, the
    # (i2,i1) x mode matrix and the mode x i0 matrix and contract over modes.
    for c in range(3):
        s = [0.5, 0.5, 0.5]
        s[c] = 0.0
        B = np.empty((n2 * n1, n_modes), dtype=np.complex128)
        E0 = np.empty((n_modes, n0), dtype=np.complex128)
        for m, (k, A) in enumerate(zip(ks, amps)):
            e = [np.exp(2j * math.pi * k[d] * (o[d] + (np.arange(grid.n[d]) + s[d]) * h) / L[d])
                 for d in range(3)]
            B[:, m] = (A[c] * np.outer(e[2], e[1])).ravel()
            E0[m] = e[0]
        u[c] = (B.real @ E0.real - B.imag @ E0.imag).reshape(n2, n1, n0)
    return u.astype(dtype)


def to_split(x: np.ndarray, grid: Grid):
    """Store positions as (integer cell, FP32 offset in [0,1)) in units of h.

    The position represented is origin + (cell + off) h exactly (the offset is
    the float32 rounding of the fractional part; a rounding up to 1.0 is
    carried into the cell).  Cells are NOT wrapped: a structure may straddle
    the periodic seam and keeps continuous coordinates.
    """
    o = np.asarray(grid.origin, dtype=np.float64)[:, None]
    t = (x - o) / grid.h
    cell = np.floor(t)
    off = (t - cell).astype(np.float32)
    carry = off >= np.float32(1.0)
    cell = cell + carry
    off = np.where(carry, np.float32(0.0), off).astype(np.float32)
    return cell.astype(np.int32), off


def from_split(cell: np.ndarray, off: np.ndarray, grid: Grid) -> np.ndarray:
    """Positions represented by a split storage (FP64, exact sum)."""
    o = np.asarray(grid.origin, dtype=np.float64)[:, None]
    return o + (cell.astype(np.float64) + off.astype(np.float64)) * grid.h


# ----------------------------------------------------------------------------
# the named workloads
# ----------------------------------------------------------------------------

def _finish(name, grid, conn, X, fib, mat_id, mats, x, u_modes, rng, fp64=False):
    ftype = np.float64 if fp64 else np.float32
    Xs = X.astype(ftype)
    cell, off = to_split(x, grid)
    u = fourier_velocity(grid, u_modes, rng, dtype=ftype)
    return Problem(name=name, grid=grid, conn=np.ascontiguousarray(conn.astype(np.int32)),
                   X=np.ascontiguousarray(Xs), fibres=np.ascontiguousarray(fib.astype(ftype)),
                   mat_id=np.ascontiguousarray(mat_id.astype(np.int32)), materials=mats,
                   x=x, cell=np.ascontiguousarray(cell), off=np.ascontiguousarray(off),
                   u=np.ascontiguousarray(u), fp64=fp64)


def block_problem(seed: int = 1000, n: int = 32, blocks=(8, 8, 2), noise=0.2,
                  fp64: bool = True, mu: float = 1.0, kappa: float = 100.0,
                  u_modes: int = 4, centre=None) -> Problem:
    """Elastic block in a periodic unit box (the plain FP64 workload at 32^3).

    8x8x2 trilinear hexes of edge h centred in the box, node positions
    perturbed by uniform +-noise*h, neo-Hookean mu = 1 (a = mu/2), kappa = 100,
    velocity a sum of `u_modes` divergence-free Fourier modes.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    h = 1.0 / n
    grid = Grid((n, n, n), h)
    centre = (0.5, 0.5, 0.5) if centre is None else centre
    conn, X = box_block(*blocks, edge=h, centre=centre)
    if not fp64:
        X = X.astype(np.float32).astype(np.float64)
    x = X + rng.uniform(-noise * h, noise * h, size=X.shape)
    fib = np.zeros((6, conn.shape[1]))
    fib[0] = 1.0
    fib[4] = 1.0
    mats = [Material(NEO_HOOKEAN, (mu / 2.0, kappa))]
    return _finish("block", grid, conn, X, fib, np.zeros(conn.shape[1]), mats, x,
                   u_modes, rng, fp64)


def shell_problem(seed: int = 2000, n: int = 128, dims=(60, 40, 6), u_modes: int = 4,
                  ho=HO_DEFAULT, twist=0.3, amp=0.015, axial=0.02, fp64=False) -> Problem:
    """Ventricle-like HO shell on an n^3 grid (128^3, 60x40x6 hexes by default)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    grid = Grid((n, n, n), 1.0 / n)
    conn, X, fib = ellipsoid_shell(*dims)
    X = X.astype(np.float32).astype(np.float64)
    x = smooth_deformation(X, rng, twist=twist, amp=amp, axial=axial)
    mats = [Material(HO, tuple(ho))]
    return _finish("shell", grid, conn, X, fib, np.zeros(conn.shape[1]), mats, x,
                   u_modes, rng, fp64)


def shell_sheets_problem(seed: int = 3000, n: int = 256, dims=(160, 100, 10),
                         sheet=(80, 40, 2), u_modes: int = 16) -> Problem:
    """Large workload: the shell at 160x100x10 plus two 80x40x2 leaflet sheets.

    HO for the shell (material 0), fibre-reinforced model 1 for the sheets
    (material 1); 172,800 elements and 1,382,400 Gauss points at the defaults.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    grid = Grid((n, n, n), 1.0 / n)
    c1, X1, f1 = ellipsoid_shell(*dims)
    c2, X2, f2 = cylinder_sheet(*sheet, axis_point=(0.5, 0.66, 0.62), facing=-1.0)
    c3, X3, f3 = cylinder_sheet(*sheet, axis_point=(0.5, 0.34, 0.62), facing=1.0)
    n1, n2 = X1.shape[1], X2.shape[1]
    conn = np.concatenate([c1, c2 + n1, c3 + n1 + n2], axis=1)
    X = np.concatenate([X1, X2, X3], axis=1).astype(np.float32).astype(np.float64)
    fib = np.concatenate([f1, f2, f3], axis=1)
    mat_id = np.concatenate([np.zeros(c1.shape[1]), np.ones(c2.shape[1] + c3.shape[1])])
    x = smooth_deformation(X, rng)
    mats = [Material(HO, HO_DEFAULT), Material(FIBRE1, FIBRE1_LEAFLET)]
    return _finish("shell+sheets", grid, conn, X, fib, mat_id, mats, x, u_modes, rng)


def material_mix_problem(seed: int = 6000, n: int = 64, dims=(30, 20, 4), models=None,
                         fp64: bool = False, twist=0.3, amp=0.015, axial=0.02,
                         active=0.0) -> Problem:
    """The shell with elements cycling through several laws (mat_id = e mod k).

    `models` lists the ib_model codes (default: all five laws of Section 3 and
    Section 6.3), each with its standard parameter set: neo-Hookean a = 0.5,
    kappa = 100; Psi_2 leaflet; Psi_4 HO; Psi_1 Cook's membrane constants;
    Psi_3 aortic-valve constants.  The smooth twist stretches some fibres and
    shortens others, so the tension-only clamp of Psi_2/Psi_4 and the
    two-sided fibre term of Psi_3 are both exercised.  `active` is the active
    tension T_a of every material (Section 6.1), or a list with one per model.
    """
    params = {NEO_HOOKEAN: (0.5, 100.0), FIBRE1: FIBRE1_LEAFLET, HO: HO_DEFAULT,
              STD_REINF: STD_REINF_COOK, FIBRE2: FIBRE2_AV}
    models = list(params) if models is None else list(models)
    rng = np.random.Generator(np.random.PCG64(seed))
    grid = Grid((n, n, n), 1.0 / n)
    conn, X, fib = ellipsoid_shell(*dims)
    if not fp64:
        X = X.astype(np.float32).astype(np.float64)
    x = smooth_deformation(X, rng, twist=twist, amp=amp, axial=axial)
    Ta = list(active) if isinstance(active, (list, tuple)) else [float(active)] * len(models)
    mats = [Material(m, tuple(params[m]), Ta[i]) for i, m in enumerate(models)]
    mat_id = np.arange(conn.shape[1]) % len(models)
    return _finish("mix", grid, conn, X, fib, mat_id, mats, x, 4, rng, fp64)


def tet_problem(base: Problem) -> Problem:
    """The same structure and inputs with every hexahedron split into six
    linear tetrahedra (the element of the paper's valve meshes)."""
    conn, fib, mid = hex_to_tets(base.conn, base.X.astype(np.float64), base.fibres, base.mat_id)
    return dataclasses.replace(base, name=base.name + "-tet", conn=conn.astype(np.int32),
                               fibres=np.ascontiguousarray(fib.astype(base.fibres.dtype)),
                               mat_id=np.ascontiguousarray(mid.astype(np.int32)))


# P2 edge nodes in VTK order: the vertex pair of each of the six edges
TET10_EDGES = ((0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3))


def tets_to_quadratic(conn4: np.ndarray, n_nodes: int):
    """Quadratic tetrahedra [10][E] from linear ones [4][E]: one new node per
    distinct edge, numbered n_nodes, n_nodes + 1, ... in ascending order of
    the edge's (smaller, larger) vertex pair.  Returns (conn10, edges) with
    edges [2][n_edges] the vertex pair of each new node."""
    E = conn4.shape[1]
    a = np.stack([conn4[i] for i, _ in TET10_EDGES]).astype(np.int64)
    b = np.stack([conn4[j] for _, j in TET10_EDGES]).astype(np.int64)
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    keys = (lo * n_nodes + hi).ravel()
    uniq, inv = np.unique(keys, return_inverse=True)
    conn10 = np.concatenate([conn4, (n_nodes + inv).reshape(6, E)], axis=0)
    return np.ascontiguousarray(conn10.astype(np.int32)), np.stack([uniq // n_nodes,
                                                                   uniq % n_nodes])


def tet10_problem(base: Problem, seed: int = 77, bend: float = 0.1) -> Problem:
    """The same structure as quadratic (P2) tetrahedra, the element of the
    paper's Cook membrane (Section 5): every hexahedron split into six
    tetrahedra, a node added at the middle of every edge.  The new nodes sit
    at the edge midpoints in the reference configuration (straight-sided
    elements) and, in the current one, at the midpoints of the current edge
    ends displaced by a seeded uniform +-bend r per coordinate, r the
    smallest inradius (3 volume / surface) of the current tetrahedra sharing
    the edge, so that the current elements are curved but far from
    inverted."""
    t = tet_problem(base)
    conn10, edges = tets_to_quadratic(t.conn, t.n_nodes)
    rng = np.random.Generator(np.random.PCG64(seed))
    X64 = t.X.astype(np.float64)
    Xm = 0.5 * (X64[:, edges[0]] + X64[:, edges[1]])
    xm = 0.5 * (t.x[:, edges[0]] + t.x[:, edges[1]])
    v = [t.x[:, t.conn[i]] for i in range(4)]
    vol = np.abs(np.einsum("ie,ie->e", np.cross((v[1] - v[0]).T, (v[2] - v[0]).T).T,
                           v[3] - v[0])) / 6.0
    area = sum(0.5 * np.linalg.norm(np.cross((v[j] - v[i]).T, (v[k] - v[i]).T), axis=1)
               for i, j, k in ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)))
    r = np.full(edges.shape[1], np.inf)
    np.minimum.at(r, (conn10[4:] - t.n_nodes).ravel(), np.tile(3.0 * vol / area, 6))
    xm = xm + rng.uniform(-bend, bend, size=xm.shape) * r
    X = np.concatenate([X64, Xm], axis=1).astype(t.X.dtype)
    x = np.concatenate([t.x, xm], axis=1)
    cell, off = to_split(x, t.grid)
    return dataclasses.replace(t, name=base.name + "-tet10", conn=conn10,
                               X=np.ascontiguousarray(X), x=x,
                               cell=np.ascontiguousarray(cell), off=np.ascontiguousarray(off))


def grid_aligned_problem(seed: int = 6000, n: int = 32, dims=(8, 8, 8), start=(-3, 5, 12),
                         u_modes: int = 4) -> Problem:
    """Hexahedra of edge h whose nodes sit exactly on grid lines (split
    offsets exactly 0), a seeded half of them moved by -2^-24 h along seeded
    axes (cell - 1, offset 1 - 2^-24, the largest float32 below 1).  The block
    spans cells start .. start + dims: by default it straddles the periodic
    seam in x and tile faces (multiples of 8 cells) in y and z.  FP32 split.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    h = 1.0 / n
    grid = Grid((n, n, n), h)
    ijk = np.stack(np.meshgrid(*[np.arange(dims[d] + 1) + start[d] for d in range(3)],
                               indexing="ij"), axis=-1)
    conn, K = _structured_hex(ijk.astype(np.float64))
    conn = _orient(conn, K)
    X = K * h
    move = (rng.uniform(size=K.shape) < 0.5)
    x = X - move * (2.0 ** -24) * h
    fib = np.zeros((6, conn.shape[1]))
    fib[0] = 1.0
    fib[4] = 1.0
    mats = [Material(NEO_HOOKEAN, (0.5, 100.0))]
    return _finish("aligned", grid, conn, X, fib, np.zeros(conn.shape[1]), mats, x, u_modes,
                   rng)


def dense_tile_problem(seed: int = 6100, n: int = 32, dims=(7, 7, 7), tile=(1, 1, 1),
                       noise: float = 0.2, u_modes: int = 4) -> Problem:
    """A block of dims hexahedra of edge h packed inside one 8^3-cell tile
    (7^3 elements: 2,744 Gauss points in that tile), nodes perturbed by
    +-noise h.  FP32 split."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = 1.0 / n
    grid = Grid((n, n, n), h)
    centre = [(8 * tile[d] + 4) * h for d in range(3)]
    conn, X = box_block(*dims, edge=h, centre=centre)
    X = X.astype(np.float32).astype(np.float64)
    x = X + rng.uniform(-noise * h, noise * h, size=X.shape)
    fib = np.zeros((6, conn.shape[1]))
    fib[0] = 1.0
    fib[4] = 1.0
    mats = [Material(NEO_HOOKEAN, (0.5, 100.0))]
    return _finish("densetile", grid, conn, X, fib, np.zeros(conn.shape[1]), mats, x, u_modes,
                   rng)


def incompressible_problem(seed: int = 6200, n: int = 32, blocks=(8, 8, 2), kappa: float = 1e4,
                           model: int = NEO_HOOKEAN, stretch: float = 0.01, angle: float = 0.05,
                           noise: float = 2e-5, fp64: bool = False) -> Problem:
    """Nearly incompressible block: x = c + R D (X - c) + noise, D = diag(1 + s,
    1 + s, (1 + s)^-2) (volume preserving), R a rotation by `angle` about a
    seeded axis, node noise +-noise h; with kappa = 1e4 the bulk modulus
    dwarfs the shear modulus (kappa / a = 2e4 for the neo-Hookean block) and
    |J - 1| stays near 1e-4 while |F - I| is near 5e-2, so tr(F - I) cancels
    in J - 1.  FP32 split unless fp64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = 1.0 / n
    grid = Grid((n, n, n), h)
    c = np.array([0.5, 0.5, 0.5])
    conn, X = box_block(*blocks, edge=h, centre=c)
    if not fp64:
        X = X.astype(np.float32).astype(np.float64)
    a = rng.normal(size=3)
    a /= np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    R = np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * (K @ K)
    D = np.diag([1 + stretch, 1 + stretch, (1 + stretch) ** -2])
    x = c[:, None] + (R @ D) @ (X - c[:, None]) + rng.uniform(-noise * h, noise * h, X.shape)
    fib = np.zeros((6, conn.shape[1]))
    fib[0] = 1.0
    fib[4] = 1.0
    params = (0.5, kappa) if model == NEO_HOOKEAN else HO_DEFAULT[:8] + (kappa,)
    mats = [Material(model, params)]
    return _finish("incompressible", grid, conn, X, fib, np.zeros(conn.shape[1]), mats, x, 4,
                   rng, fp64)


def batch_problems(seed: int = 5000, count: int = 48, sizes=(32, 64, 96, 128),
                   elems=(2000, 20000)) -> List[Problem]:
    """Independent HO shells on their own grids (parameter-sweep batch).

    Grid n_i drawn from `sizes`; transmural n_t in [2,6]; (n_c, n_l) scaled so
    E_i ~ U[elems]; HO a, b, af, bf each scaled by U(0.7, 1.3).
    """
    out = []
    for i in range(count):
        rng = np.random.Generator(np.random.PCG64(seed + i))
        n = int(rng.choice(sizes))
        nt = int(rng.integers(2, 7))
        target = rng.uniform(*elems)
        nl = max(4, int(round(math.sqrt(target / nt / 1.5))))
        nc = max(6, int(round(target / nt / nl)))
        ho = list(HO_DEFAULT)
        for j in range(4):
            ho[j] *= rng.uniform(0.7, 1.3)
        p = shell_problem(seed=seed + 100 + i, n=n, dims=(nc, nl, nt), ho=tuple(ho))
        p.name = f"batch{i}"
        out.append(p)
    return out


def named(name: str) -> Problem:
    """The standard workloads by name."""
    if name == "block32":
        return block_problem()
    if name == "shell128":
        return shell_problem()
    if name == "shell256":
        return shell_sheets_problem()
    raise KeyError(name)
