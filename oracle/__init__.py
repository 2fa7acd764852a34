"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package.  The product path (the CUDA
library and its Python binding) never loads it.

The numerics live in ``ibref.cpp`` (plain C++17, double precision); this
module compiles it with g++ on first use and exposes numpy wrappers whose
inputs are the same arrays the GPU path receives (FP32 values are widened
exactly to FP64; split positions are rebuilt exactly as origin + (cell+off) h).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ibref.cpp")
_HDR = os.path.join(_HERE, "ibref.h")
_OUT = os.path.join(_HERE, "_build", "libibref.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (g++ -O2, no fast-math) into oracle/_build/."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    stale = (not os.path.exists(_OUT) or
             max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)) > os.path.getmtime(_OUT))
    if force or stale:
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-fPIC", "-shared",
                               "-ffp-contract=off", _SRC, "-o", tmp])
        os.replace(tmp, _OUT)
    return _OUT


class _Grid(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("h", C.c_double), ("origin", C.c_double * 3)]


class _Mesh(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_elems", C.c_int32),
                ("conn", C.c_void_p), ("X", C.c_void_p), ("fibres", C.c_void_p),
                ("mat_id", C.c_void_p), ("elem", C.c_int32)]


class _Mats(C.Structure):
    _fields_ = [("n_mats", C.c_int32), ("model", C.c_void_p), ("params", C.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.or_active_tension.restype = C.c_double
            L.or_active_tension.argtypes = [C.c_double]
            L.or_phi.restype = C.c_double
            L.or_phi.argtypes = [C.c_double]
            L.or_dphi.restype = C.c_double
            L.or_dphi.argtypes = [C.c_double]
            L.or_support_count.restype = C.c_int64
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Model:
    """Oracle view of one problem: mesh, grid, materials and positions (all FP64)."""

    def __init__(self, prob=None, *, grid=None, conn=None, X=None, fibres=None, mat_id=None,
                 materials=None):
        if prob is not None:
            grid, conn, X = prob.grid, prob.conn, prob.X
            fibres, mat_id, materials = prob.fibres, prob.mat_id, prob.materials
        self.grid_py = grid
        self.conn = np.ascontiguousarray(conn, dtype=np.int32)
        self.X = _f64(X)
        self.fibres = None if fibres is None else _f64(fibres)
        self.mat_id = None if mat_id is None else np.ascontiguousarray(mat_id, dtype=np.int32)
        self.N = self.X.shape[1]
        self.E = self.conn.shape[1]
        self.elem = {8: 0, 4: 1, 10: 2}[self.conn.shape[0]]  # hexahedra, P1 or P2 tetrahedra
        self.nq = 8 if self.elem == 0 else 4                  # points of the element rule
        self._mesh = _Mesh(self.N, self.E, _p(self.conn), _p(self.X), _p(self.fibres),
                           _p(self.mat_id), self.elem)
        if grid is not None:
            self._grid = _Grid((C.c_int32 * 3)(*grid.n), float(grid.h),
                               (C.c_double * 3)(*[float(v) for v in grid.origin]))
        self.set_materials(materials or [])

    def set_materials(self, materials):
        self.materials = list(materials)
        nm = max(1, len(self.materials))
        self._models = np.zeros(nm, dtype=np.int32)
        self._params = np.zeros((nm, 10), dtype=np.float64)
        for i, m in enumerate(self.materials):
            self._models[i] = m.model
            self._params[i, :len(m.params)] = m.params
            self._params[i, 9] = getattr(m, "active", 0.0)
        self._mats = _Mats(len(self.materials), _p(self._models), _p(self._params))

    # -- positions -----------------------------------------------------------
    def positions(self, cell, off):
        """Exact FP64 positions origin + (cell + off) h from split storage."""
        g = self.grid_py
        o = np.asarray(g.origin, dtype=np.float64)[:, None]
        return o + (cell.astype(np.float64) + off.astype(np.float64)) * g.h

    # -- operators -----------------------------------------------------------
    def _chk(self, rc, what):
        if rc != 0:
            raise RuntimeError(f"oracle {what} failed with code {rc}")

    def mass(self):
        m = np.empty(self.N)
        self._chk(lib().or_lumped_mass(C.byref(self._mesh), _p(m)), "mass")
        return m

    def gauss_info(self, x):
        x = _f64(x)
        w = np.empty((self.nq, self.E))
        J = np.empty((self.nq, self.E))
        self._chk(lib().or_gauss_info(C.byref(self._mesh), _p(x), _p(w), _p(J)), "gauss_info")
        return w, J

    def fe_force(self, x):
        x = _f64(x)
        G = np.empty((3, self.N))
        en = C.c_double(0.0)
        self._chk(lib().or_fe_force(C.byref(self._mesh), C.byref(self._mats), _p(x), _p(G),
                                    C.byref(en)), "fe_force")
        return G, en.value

    def penalty(self, x, nodes, kappa, weights=None):
        """Penalty tethers of the solid boundary (Section 5: the fixed face of
        Cook's membrane, the fixed tube of the aortic valve): each listed node
        is pulled to its reference position by G_a = -kappa w_a (x_a - X_a),
        w_a the lumped mass (volume weight of the node, the nodal-rule weight
        of Section 4.4) unless weights are given; the energy is
        kappa/2 sum_a w_a |x_a - X_a|^2.  Returns (G [3][N], energy)."""
        x = _f64(x)
        nodes = np.asarray(nodes, dtype=np.int64)
        w = self.mass()[nodes] if weights is None else _f64(weights)
        d = x[:, nodes] - self.X[:, nodes]
        G = np.zeros((3, self.N))
        G[:, nodes] = -kappa * w * d
        return G, 0.5 * kappa * float(np.sum(w * np.sum(d * d, axis=0)))

    def fe_force_adj(self, x, v):
        x, v = _f64(x), _f64(v)
        Hv = np.empty((3, self.N))
        gp = np.zeros((len(self.materials), 10))
        self._chk(lib().or_fe_force_adj(C.byref(self._mesh), C.byref(self._mats), _p(x), _p(v),
                                        _p(Hv), _p(gp)), "fe_force_adj")
        return Hv, gp

    def _field(self):
        n0, n1, n2 = self.grid_py.n
        return np.empty((3, n2, n1, n0))

    def spread(self, x, G):
        x, G = _f64(x), _f64(G)
        f = self._field()
        self._chk(lib().or_spread(C.byref(self._grid), C.byref(self._mesh), _p(x), _p(G), _p(f)),
                  "spread")
        return f

    def spread_at(self, x, G, comp, idx):
        x, G = _f64(x), _f64(G)
        comp = np.ascontiguousarray(comp, dtype=np.int32)
        idx = np.ascontiguousarray(idx, dtype=np.int32).reshape(-1, 3)
        out = np.empty(len(comp))
        self._chk(lib().or_spread_at(C.byref(self._grid), C.byref(self._mesh), _p(x), _p(G),
                                     C.c_int64(len(comp)), _p(comp), _p(idx), _p(out)),
                  "spread_at")
        return out

    def interp(self, x, u, want_gauss=False):
        x, u = _f64(x), _f64(u)
        U = np.empty((3, self.N))
        Uq = np.empty((3, self.nq, self.E)) if want_gauss else None
        self._chk(lib().or_interp(C.byref(self._grid), C.byref(self._mesh), _p(x), _p(u), _p(U),
                                  _p(Uq)), "interp")
        return (U, Uq) if want_gauss else U

    def spread_adj(self, x, G, gf, want_gx=True):
        x, G, gf = _f64(x), _f64(G), _f64(gf)
        gG = np.empty((3, self.N))
        gx = np.empty((3, self.N)) if want_gx else None
        self._chk(lib().or_spread_adj(C.byref(self._grid), C.byref(self._mesh), _p(x), _p(G),
                                      _p(gf), _p(gG), _p(gx)), "spread_adj")
        return gG, gx

    def interp_adj(self, x, u, gU, want_gx=True):
        x, u, gU = _f64(x), _f64(u), _f64(gU)
        gu = self._field()
        gx = np.empty((3, self.N)) if want_gx else None
        self._chk(lib().or_interp_adj(C.byref(self._grid), C.byref(self._mesh), _p(x), _p(u),
                                      _p(gU), _p(gu), _p(gx)), "interp_adj")
        return gu, gx

    # nodal quadrature rule (Section 4.4): the coupling points are the nodes
    def spread_nodal(self, x, G):
        x, G = _f64(x), _f64(G)
        f = self._field()
        self._chk(lib().or_spread_nodal(C.byref(self._grid), C.c_int64(self.N), _p(x), _p(G),
                                        _p(f)), "spread_nodal")
        return f

    def spread_nodal_at(self, x, G, comp, idx):
        x, G = _f64(x), _f64(G)
        comp = np.ascontiguousarray(comp, dtype=np.int32)
        idx = np.ascontiguousarray(idx, dtype=np.int32).reshape(-1, 3)
        out = np.empty(len(comp))
        self._chk(lib().or_spread_nodal_at(C.byref(self._grid), C.c_int64(self.N), _p(x), _p(G),
                                           C.c_int64(len(comp)), _p(comp), _p(idx), _p(out)),
                  "spread_nodal_at")
        return out

    def interp_nodal(self, x, u):
        x, u = _f64(x), _f64(u)
        U = np.empty((3, self.N))
        self._chk(lib().or_interp_nodal(C.byref(self._grid), C.c_int64(self.N), _p(x), _p(u),
                                        _p(U)), "interp_nodal")
        return U

    def spread_nodal_adj(self, x, G, gf, want_gx=True):
        x, G, gf = _f64(x), _f64(G), _f64(gf)
        gG = np.empty((3, self.N))
        gx = np.empty((3, self.N)) if want_gx else None
        self._chk(lib().or_spread_nodal_adj(C.byref(self._grid), C.c_int64(self.N), _p(x), _p(G),
                                            _p(gf), _p(gG), _p(gx)), "spread_nodal_adj")
        return gG, gx

    def interp_nodal_adj(self, x, u, gU, want_gx=True):
        x, u, gU = _f64(x), _f64(u), _f64(gU)
        gu = self._field()
        gx = np.empty((3, self.N)) if want_gx else None
        self._chk(lib().or_interp_nodal_adj(C.byref(self._grid), C.c_int64(self.N), _p(x), _p(u),
                                            _p(gU), _p(gu), _p(gx)), "interp_nodal_adj")
        return gu, gx

    def support_count(self, x):
        x = _f64(x)
        r = lib().or_support_count(C.byref(self._grid), C.byref(self._mesh), _p(x))
        if r < 0:
            raise RuntimeError("oracle support_count failed")
        return int(r)


def active_tension(t: float) -> float:
    """T_a(t) of Section 6.1 in Pa (period 0.8 s)."""
    return lib().or_active_tension(float(t))


def phi(r: float) -> float:
    return lib().or_phi(float(r))


def dphi(r: float) -> float:
    return lib().or_dphi(float(r))


def _row(params, Ta):
    p = np.zeros(10)
    p[:len(params)] = params
    p[9] = Ta
    return p


def stress(model: int, params, F, ef=(1, 0, 0), es=(0, 1, 0), Ta=0.0):
    """(P, Psi) for one deformation gradient F (3x3); Ta is the active tension."""
    p = _row(params, Ta)
    F = _f64(np.asarray(F).reshape(9))
    ef, es = _f64(ef), _f64(es)
    P = np.empty(9)
    psi = C.c_double(0.0)
    rc = lib().or_stress(C.c_int32(model), _p(p), _p(F), _p(ef), _p(es), _p(P), C.byref(psi))
    if rc:
        raise RuntimeError("oracle stress failed")
    return P.reshape(3, 3), psi.value


def stress_dir(model: int, params, F, dF, ef=(1, 0, 0), es=(0, 1, 0), Ta=0.0):
    p = _row(params, Ta)
    F = _f64(np.asarray(F).reshape(9))
    dF = _f64(np.asarray(dF).reshape(9))
    ef, es = _f64(ef), _f64(es)
    dP = np.empty(9)
    rc = lib().or_stress_dir(C.c_int32(model), _p(p), _p(F), _p(dF), _p(ef), _p(es), _p(dP))
    if rc:
        raise RuntimeError("oracle stress_dir failed")
    return dP.reshape(3, 3)
