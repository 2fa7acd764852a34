"""Thin Python binding of libibfe (include/ibfe.h) over ctypes.

Argument marshalling only: every operator runs in the CUDA library.  Arrays
are torch tensors on the current CUDA device (PyTorch provides device memory
and streams); every call is issued on torch's current stream.  The binding
never falls back to another implementation: if the library cannot be loaded
the import fails.

Names follow the C ABI: ib_plan_create, ib_fe_force, ib_spread, ib_interp,
ib_forward, ib_spread_adj, ib_interp_adj, ib_fe_force_adj, ib_lumped_mass,
ib_plan_sync_status, ib_plan_destroy, ib_status_str, ib_version.  The
torch.autograd.Function classes FEForce, Spread and Interp route their
backward passes to the adjoint entry points.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libibfe.so")

IB_OK, IB_ERR_INVALID_ARG, IB_ERR_CUDA, IB_ERR_NONFINITE = 0, 1, 2, 3
IB_ERR_CAPACITY, IB_ERR_TIMEOUT, IB_ERR_UNSUPPORTED, IB_ERR_INVERTED = 4, 5, 6, 7
IB_NEO_HOOKEAN, IB_FIBRE1, IB_HO, IB_STD_REINF, IB_FIBRE2 = 0, 1, 2, 3, 4
IB_FP32_SPLIT, IB_FP64, IB_FP32_SPLIT_F32STAB, IB_FP32_SPLIT_DFVOL = 0, 1, 2, 3
IB_QUAD_GAUSS2, IB_QUAD_NODAL = 0, 1
IB_ELEM_HEX8, IB_ELEM_TET4, IB_ELEM_TET10 = 0, 1, 2
_ELEM_OF_NODES = {8: IB_ELEM_HEX8, 4: IB_ELEM_TET4, 10: IB_ELEM_TET10}
_NODES_OF_ELEM = {v: k for k, v in _ELEM_OF_NODES.items()}
IB_MAX_MATERIALS = 8
IB_PARAM_ROW = 10   # gradient row: the law's parameters, zeros, d/dT_a in column 9
STAGES = ("force", "gather", "points", "sort", "spread", "interp", "project", "reduce",
          "spread_push")
N_PARAMS = {IB_NEO_HOOKEAN: 2, IB_FIBRE1: 4, IB_HO: 9, IB_STD_REINF: 4, IB_FIBRE2: 5}


class IBError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {ib_status_str(code)} (status {code})")


class _Mesh(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_elems", C.c_int32), ("conn", C.c_void_p),
                ("X", C.c_void_p), ("fibres", C.c_void_p), ("mat_id", C.c_void_p),
                ("elem_type", C.c_int32)]


class _Grid(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("h", C.c_double), ("origin", C.c_double * 3)]


class _Pos(C.Structure):
    _fields_ = [("cell", C.c_void_p), ("off", C.c_void_p), ("x64", C.c_void_p),
                ("grad_unit", C.c_double)]


class _Mat(C.Structure):
    _fields_ = [("model", C.c_int32), ("n_params", C.c_int32), ("params", C.c_double * 9),
                ("Ta", C.c_double)]


class _Instance(C.Structure):
    _fields_ = [("mesh", _Mesh), ("grid", _Grid), ("n_mats", C.c_int32),
                ("mats", _Mat * 8), ("x", _Pos), ("u", C.c_void_p), ("G", C.c_void_p),
                ("f", C.c_void_p), ("U", C.c_void_p), ("gU", C.c_void_p), ("gf", C.c_void_p),
                ("gG", C.c_void_p), ("gu", C.c_void_p), ("gx", C.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libibfe.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    vp, i32, dp = C.c_void_p, C.c_int32, C.POINTER(C.c_double)
    sigs = {
        "ib_plan_create": [C.POINTER(_Mesh), C.POINTER(_Grid), i32, i32, vp, C.POINTER(vp)],
        "ib_plan_destroy": [vp],
        "ib_lumped_mass": [vp, vp, vp],
        "ib_fe_force": [vp, C.POINTER(_Mat), i32, C.POINTER(_Pos), vp, dp, vp],
        "ib_spread": [vp, C.POINTER(_Pos), vp, vp, vp],
        "ib_interp": [vp, C.POINTER(_Pos), vp, vp, vp],
        "ib_forward": [vp, C.POINTER(_Mat), i32, C.POINTER(_Pos), vp, vp, vp, vp, vp],
        "ib_spread_adj": [vp, C.POINTER(_Pos), vp, vp, vp, vp, vp],
        "ib_interp_adj": [vp, C.POINTER(_Pos), vp, vp, vp, vp, vp],
        "ib_fe_force_adj": [vp, C.POINTER(_Mat), i32, C.POINTER(_Pos), vp, vp, dp, vp],
        "ib_backward": [vp, C.POINTER(_Mat), i32, C.POINTER(_Pos), vp, vp, vp, vp, vp, vp, vp,
                        vp, vp],
        "ib_plan_sync_status": [vp, vp],
        "ib_plan_get_tuning": [vp, C.POINTER(i32)],
        "ib_plan_set_tuning": [vp, C.POINTER(i32)],
        "ib_plan_autotune": [vp, C.POINTER(_Mat), i32, C.POINTER(_Pos), vp, vp, C.POINTER(i32)],
        "ib_plan_set_profiling": [vp, i32],
        "ib_batch_create": [i32, C.POINTER(_Instance), i32, vp, C.POINTER(vp)],
        "ib_batch_forward": [vp, vp],
        "ib_batch_adjoint": [vp, vp],
        "ib_batch_gparams": [vp, dp, vp],
        "ib_batch_get_tuning": [vp, C.POINTER(i32)],
        "ib_batch_destroy": [vp],
        "ib_fe_energy_noalloc": [C.POINTER(_Mesh), C.POINTER(_Mat), i32, C.POINTER(_Pos),
                                 C.c_double, vp, vp],
        "ib_plan_profile": [vp, vp, dp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), i32],
        "ib_plan_set_penalty": [vp, vp, i32, vp, C.c_double],
        "ib_diag_wait_timeout": [C.c_double, vp],
        "ib_fluid_create": [C.POINTER(_Grid), i32, C.c_double, C.c_double, C.c_double, vp,
                            C.POINTER(vp)],
        "ib_fluid_destroy": [vp],
        "ib_fluid_set_cycles": [vp, i32, i32],
        "ib_fluid_levels": [vp, C.POINTER(i32)],
        "ib_fluid_get_cycles": [vp, C.POINTER(i32)],
        "ib_fluid_step": [vp, vp, vp, vp, vp, dp, vp],
        "ib_step": [vp, vp, C.POINTER(_Mat), i32, C.POINTER(_Pos), vp, vp, vp, vp, vp, vp],
    }
    for name, args in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.ib_status_str.argtypes = [C.c_int]
    L.ib_status_str.restype = C.c_char_p
    L.ib_version.argtypes = []
    L.ib_version.restype = C.c_int32
    L.ib_active_tension.argtypes = [C.c_double]
    L.ib_active_tension.restype = C.c_double
    return L


_lib = _load()


def ib_status_str(code: int) -> str:
    return _lib.ib_status_str(int(code)).decode()


def ib_version() -> int:
    return int(_lib.ib_version())


def ib_active_tension(t: float) -> float:
    """T_a(t) of Section 6.1 in Pa (period 0.8 s); Material.Ta takes it (in the
    parameter set's units)."""
    return float(_lib.ib_active_tension(float(t)))


def _chk(code: int, what: str):
    if code != IB_OK:
        raise IBError(code, what)


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


@dataclass
class Material:
    model: int
    params: Sequence[float]
    Ta: float = 0.0   # active fibre tension at the current time (Section 6.1)


def _mats(mats: Sequence[Material]):
    arr = (_Mat * len(mats))()
    for i, m in enumerate(mats):
        arr[i].model = int(m.model)
        arr[i].n_params = len(m.params)
        for k, v in enumerate(m.params):
            arr[i].params[k] = float(v)
        arr[i].Ta = float(getattr(m, "Ta", 0.0))
    return arr, len(mats)


class Pos:
    """Node positions: split (cell int32 [3][N] + off float32 [3][N]) or x64 [3][N].
    grad_unit: the length per which the adjoints return position derivatives
    (0: per unit length, d/dx; the grid's h: per unit of the offset, d/d off)."""

    def __init__(self, cell: torch.Tensor = None, off: torch.Tensor = None,
                 x64: torch.Tensor = None, grad_unit: float = 0.0):
        self.cell, self.off, self.x64 = cell, off, x64
        self._s = _Pos(None if cell is None else cell.data_ptr(),
                       None if off is None else off.data_ptr(),
                       None if x64 is None else x64.data_ptr(), float(grad_unit))


class Plan:
    """An ib_plan: one hexahedral or tetrahedral mesh on one periodic MAC grid."""

    def __init__(self, conn: torch.Tensor, X: torch.Tensor, n, h: float, origin=(0.0, 0.0, 0.0),
                 fibres: torch.Tensor = None, mat_id: torch.Tensor = None,
                 precision: int = IB_FP32_SPLIT, quad: int = IB_QUAD_GAUSS2):
        self.dtype = torch.float64 if precision == IB_FP64 else torch.float32
        self.quad = quad
        # hexahedra [8][E], linear [4][E] or quadratic [10][E] tetrahedra
        self.elem = _ELEM_OF_NODES.get(int(conn.shape[0]) if conn.dim() == 2 else 8, IB_ELEM_HEX8)
        _check(conn, torch.int32, (_NODES_OF_ELEM[self.elem], -1), "conn")
        _check(X, self.dtype, (3, -1), "X")
        if fibres is not None:
            _check(fibres, self.dtype, (6, conn.shape[1]), "fibres")
        if mat_id is not None:
            _check(mat_id, torch.int32, (conn.shape[1],), "mat_id")
        # the plan keeps these pointers: hold the tensors
        self._keep = (conn, X, fibres, mat_id)
        self.N, self.E = int(X.shape[1]), int(conn.shape[1])
        self.n, self.h, self.origin = tuple(int(v) for v in n), float(h), tuple(origin)
        self.precision = precision
        self.device = X.device
        mesh = _Mesh(self.N, self.E, conn.data_ptr(), X.data_ptr(),
                     None if fibres is None else fibres.data_ptr(),
                     None if mat_id is None else mat_id.data_ptr(), self.elem)
        grid = _Grid((C.c_int32 * 3)(*self.n), self.h, (C.c_double * 3)(*origin))
        out = C.c_void_p()
        _chk(_lib.ib_plan_create(C.byref(mesh), C.byref(grid), quad, precision, _stream(),
                                 C.byref(out)), "ib_plan_create")
        self._h = out

    @property
    def handle(self):
        return self._h

    def grid_shape(self):
        n0, n1, n2 = self.n
        return (3, n2, n1, n0)

    def __del__(self):
        if getattr(self, "_h", None):
            try:
                _lib.ib_plan_destroy(self._h)
            except Exception:
                pass
            self._h = None


class Fluid:
    """The fluid solver of Section 4.2 on a periodic MAC grid (ib_fluid_create)."""

    def __init__(self, n, h: float, rho: float, mu: float, dt: float,
                 precision: int = IB_FP32_SPLIT, origin=(0.0, 0.0, 0.0)):
        self.dtype = torch.float64 if precision == IB_FP64 else torch.float32
        self.n, self.h = tuple(int(v) for v in n), float(h)
        self.rho, self.mu, self.dt = float(rho), float(mu), float(dt)
        self.precision = precision
        grid = _Grid((C.c_int32 * 3)(*self.n), self.h, (C.c_double * 3)(*origin))
        out = C.c_void_p()
        _chk(_lib.ib_fluid_create(C.byref(grid), precision, self.rho, self.mu, self.dt,
                                  _stream(), C.byref(out)), "ib_fluid_create")
        self._h = out

    @property
    def handle(self):
        return self._h

    def grid_shape(self):
        n0, n1, n2 = self.n
        return (3, n2, n1, n0)

    def levels(self) -> int:
        v = C.c_int32()
        _chk(_lib.ib_fluid_levels(self._h, C.byref(v)), "ib_fluid_levels")
        return int(v.value)

    def cycles(self):
        """[Helmholtz, Poisson] V-cycles per step."""
        t = (C.c_int32 * 2)()
        _chk(_lib.ib_fluid_get_cycles(self._h, t), "ib_fluid_get_cycles")
        return list(t)

    def set_cycles(self, helmholtz: int, poisson: int):
        _chk(_lib.ib_fluid_set_cycles(self._h, int(helmholtz), int(poisson)),
             "ib_fluid_set_cycles")

    def __del__(self):
        if getattr(self, "_h", None):
            try:
                _lib.ib_fluid_destroy(self._h)
            except Exception:
                pass
            self._h = None


def ib_fluid_step(fluid: Fluid, u, f=None, u_next=None, p=None, residuals: bool = False):
    """One projection step: (u_next, p, residuals or None); u_next may be u."""
    sh = fluid.grid_shape()
    _check(u, fluid.dtype, sh, "u")
    if f is not None:
        _check(f, fluid.dtype, sh, "f")
    if u_next is None:
        u_next = torch.empty_like(u)
    _check(u_next, fluid.dtype, sh, "u_next")
    if p is None:
        p = torch.empty(sh[1:], dtype=fluid.dtype, device=u.device)
    _check(p, fluid.dtype, sh[1:], "p")
    res = (C.c_double * 2)() if residuals else None
    _chk(_lib.ib_fluid_step(fluid.handle, _ptr(u), _ptr(f), _ptr(u_next), _ptr(p), res,
                            _stream()), "ib_fluid_step")
    return u_next, p, (list(res) if residuals else None)


def ib_step(plan: Plan, fluid: Fluid, mats, x: Pos, u, G=None, f=None, U=None, p=None):
    """One explicit IB step (Section 4.2): x and u advance in place; returns
    (G, f, U, p) -- the nodal force and force density of x^n, the new velocity
    at x^n and the pressure."""
    sh = plan.grid_shape()
    _check(u, plan.dtype, sh, "u")
    G = _out(G, plan, (3, plan.N), "G")
    f = _out(f, plan, sh, "f")
    U = _out(U, plan, (3, plan.N), "U")
    if p is None:
        p = torch.empty(sh[1:], dtype=plan.dtype, device=u.device)
    _check(p, plan.dtype, sh[1:], "p")
    arr, nm = _mats(mats)
    _chk(_lib.ib_step(plan.handle, fluid.handle, arr, nm, C.byref(_pos(plan, x)), _ptr(u),
                      _ptr(G), _ptr(f), _ptr(U), _ptr(p), _stream()), "ib_step")
    return G, f, U, p


def _check(t, dtype, shape, name):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if len(shape) != t.dim() or any(s != -1 and s != d for s, d in zip(shape, t.shape)):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {shape}")


def _pos(plan: Plan, x: Pos):
    if plan.precision == IB_FP64:
        _check(x.x64, torch.float64, (3, plan.N), "x64")
    else:
        _check(x.cell, torch.int32, (3, plan.N), "cell")
        _check(x.off, torch.float32, (3, plan.N), "off")
    return x._s


def _out(t, plan, shape, name):
    if t is None:
        return torch.empty(shape, dtype=plan.dtype, device="cuda")
    _check(t, plan.dtype, shape, name)
    return t


def ib_plan_create(conn, X, n, h, origin=(0.0, 0.0, 0.0), fibres=None, mat_id=None,
                   precision=IB_FP32_SPLIT, quad=IB_QUAD_GAUSS2) -> Plan:
    return Plan(conn, X, n, h, origin, fibres, mat_id, precision, quad)


def ib_plan_destroy(plan: Plan):
    if plan._h:
        _chk(_lib.ib_plan_destroy(plan._h), "ib_plan_destroy")
        plan._h = None


def ib_lumped_mass(plan: Plan, mass=None):
    mass = _out(mass, plan, (plan.N,), "mass")
    _chk(_lib.ib_lumped_mass(plan.handle, _ptr(mass), _stream()), "ib_lumped_mass")
    return mass


def ib_fe_force(plan: Plan, mats, x: Pos, G=None, energy: bool = False):
    G = _out(G, plan, (3, plan.N), "G")
    arr, nm = _mats(mats)
    en = C.c_double(0.0)
    _chk(_lib.ib_fe_force(plan.handle, arr, nm, C.byref(_pos(plan, x)), _ptr(G),
                          C.byref(en) if energy else None, _stream()), "ib_fe_force")
    return (G, en.value) if energy else G


def ib_spread(plan: Plan, x: Pos, G, f=None):
    _check(G, plan.dtype, (3, plan.N), "G")
    f = _out(f, plan, plan.grid_shape(), "f")
    _chk(_lib.ib_spread(plan.handle, C.byref(_pos(plan, x)), _ptr(G), _ptr(f), _stream()),
         "ib_spread")
    return f


def ib_interp(plan: Plan, x: Pos, u, U=None):
    _check(u, plan.dtype, plan.grid_shape(), "u")
    U = _out(U, plan, (3, plan.N), "U")
    _chk(_lib.ib_interp(plan.handle, C.byref(_pos(plan, x)), _ptr(u), _ptr(U), _stream()),
         "ib_interp")
    return U


def ib_forward(plan: Plan, mats, x: Pos, u, G=None, f=None, U=None):
    _check(u, plan.dtype, plan.grid_shape(), "u")
    G = _out(G, plan, (3, plan.N), "G")
    f = _out(f, plan, plan.grid_shape(), "f")
    U = _out(U, plan, (3, plan.N), "U")
    arr, nm = _mats(mats)
    _chk(_lib.ib_forward(plan.handle, arr, nm, C.byref(_pos(plan, x)), _ptr(u), _ptr(G),
                         _ptr(f), _ptr(U), _stream()), "ib_forward")
    return G, f, U


def ib_spread_adj(plan: Plan, x: Pos, G, gf, want_gx: bool = True, gG=None, gx=None):
    _check(G, plan.dtype, (3, plan.N), "G")
    _check(gf, plan.dtype, plan.grid_shape(), "gf")
    gG = _out(gG, plan, (3, plan.N), "gG")
    gx = _out(gx, plan, (3, plan.N), "gx") if want_gx else None
    _chk(_lib.ib_spread_adj(plan.handle, C.byref(_pos(plan, x)), _ptr(G), _ptr(gf), _ptr(gG),
                            _ptr(gx), _stream()), "ib_spread_adj")
    return gG, gx


def ib_interp_adj(plan: Plan, x: Pos, u, gU, want_gx: bool = True, gu=None, gx=None):
    _check(gU, plan.dtype, (3, plan.N), "gU")
    if want_gx:
        _check(u, plan.dtype, plan.grid_shape(), "u")
    gu = _out(gu, plan, plan.grid_shape(), "gu")
    gx = _out(gx, plan, (3, plan.N), "gx") if want_gx else None
    _chk(_lib.ib_interp_adj(plan.handle, C.byref(_pos(plan, x)), _ptr(u if want_gx else None),
                            _ptr(gU), _ptr(gu), _ptr(gx), _stream()), "ib_interp_adj")
    return gu, gx


def ib_fe_force_adj(plan: Plan, mats, x: Pos, v, want_params: bool = True, Hv=None):
    _check(v, plan.dtype, (3, plan.N), "v")
    Hv = _out(Hv, plan, (3, plan.N), "Hv")
    arr, nm = _mats(mats)
    gp = (C.c_double * (IB_PARAM_ROW * nm))()
    _chk(_lib.ib_fe_force_adj(plan.handle, arr, nm, C.byref(_pos(plan, x)), _ptr(v), _ptr(Hv),
                              gp if want_params else None, _stream()), "ib_fe_force_adj")
    if not want_params:
        return Hv, None
    g = torch.tensor(list(gp), dtype=torch.float64).reshape(nm, IB_PARAM_ROW)
    return Hv, g


def ib_backward(plan: Plan, mats, x: Pos, u=None, G=None, gG=None, gf=None, gU=None,
                gx=None, gu=None, want_params: bool = True):
    """Fused backward of ib_forward: (gx, gu, gparams) for the cotangents
    (gG, gf, gU) of (G, f, U); any cotangent may be None (zero).  gparams is a
    device float64 tensor [n_mats][IB_PARAM_ROW] (None unless want_params); gu is None
    unless gU is given."""
    if gf is not None:
        _check(gf, plan.dtype, plan.grid_shape(), "gf")
        _check(G, plan.dtype, (3, plan.N), "G")
    if gG is not None:
        _check(gG, plan.dtype, (3, plan.N), "gG")
    if gU is not None:
        _check(gU, plan.dtype, (3, plan.N), "gU")
        _check(u, plan.dtype, plan.grid_shape(), "u")
        gu = _out(gu, plan, plan.grid_shape(), "gu")
    else:
        gu = None
    gx = _out(gx, plan, (3, plan.N), "gx")
    arr, nm = _mats(mats)
    gp = (torch.empty(nm, IB_PARAM_ROW, dtype=torch.float64, device=plan.device)
          if want_params else None)
    _chk(_lib.ib_backward(plan.handle, arr, nm, C.byref(_pos(plan, x)), _ptr(u), _ptr(G),
                          _ptr(gG), _ptr(gf), _ptr(gU), _ptr(gx), _ptr(gu), _ptr(gp),
                          _stream()), "ib_backward")
    return gx, gu, gp


def ib_plan_set_penalty(plan: Plan, nodes=None, kappa: float = 0.0, weights=None):
    """Tether the listed nodes (device int32 [n]) to their reference positions
    with stiffness kappa (weights: device Real [n], default the lumped mass);
    nodes=None removes the tethers.  The plan keeps the tensors alive."""
    if nodes is None or nodes.numel() == 0:
        plan._pen = None
        _chk(_lib.ib_plan_set_penalty(plan.handle, None, 0, None, 0.0), "ib_plan_set_penalty")
        return
    _check(nodes, torch.int32, (-1,), "nodes")
    if weights is not None:
        _check(weights, plan.dtype, (nodes.numel(),), "weights")
    plan._pen = (nodes, weights)
    _chk(_lib.ib_plan_set_penalty(plan.handle, _ptr(nodes), int(nodes.numel()), _ptr(weights),
                                  float(kappa)), "ib_plan_set_penalty")


def ib_diag_wait_timeout(ms: float = 20.0) -> int:
    """Run the bounded-wait diagnostic; returns the status (IB_ERR_TIMEOUT)."""
    return int(_lib.ib_diag_wait_timeout(float(ms), _stream()))


def ib_plan_get_tuning(plan: Plan):
    """[points per work item, force CTAs/SM, spreading CTAs/SM cap, interpolation cap]"""
    t = (C.c_int32 * 4)()
    _chk(_lib.ib_plan_get_tuning(plan.handle, t), "ib_plan_get_tuning")
    return list(t)


def ib_plan_set_tuning(plan: Plan, tuning):
    t = (C.c_int32 * 4)(*[int(v) for v in tuning])
    _chk(_lib.ib_plan_set_tuning(plan.handle, t), "ib_plan_set_tuning")


def ib_plan_autotune(plan: Plan, mats, x: Pos, u):
    """Time ib_forward over candidate tunings, keep the fastest, return it."""
    _check(u, plan.dtype, plan.grid_shape(), "u")
    arr, nm = _mats(mats)
    t = (C.c_int32 * 4)()
    _chk(_lib.ib_plan_autotune(plan.handle, arr, nm, C.byref(_pos(plan, x)), _ptr(u), _stream(),
                               t), "ib_plan_autotune")
    return list(t)


def ib_plan_sync_status(plan: Plan) -> int:
    return int(_lib.ib_plan_sync_status(plan.handle, _stream()))


def ib_fe_energy_noalloc(conn, X, mats, x: Pos, h: float, energy, fibres=None, mat_id=None):
    """Plan-free total elastic energy written into the device float64 tensor
    `energy` (one element); the library allocates nothing for it (see the C
    declaration for the limits and the shared-scratch caveats)."""
    _check(conn, torch.int32, (8, -1), "conn")
    _check(X, torch.float32, (3, -1), "X")
    _check(energy, torch.float64, (1,), "energy")
    N, E = int(X.shape[1]), int(conn.shape[1])
    _check(x.cell, torch.int32, (3, N), "cell")
    _check(x.off, torch.float32, (3, N), "off")
    if fibres is not None:
        _check(fibres, torch.float32, (6, E), "fibres")
    if mat_id is not None:
        _check(mat_id, torch.int32, (E,), "mat_id")
    mesh = _Mesh(N, E, conn.data_ptr(), X.data_ptr(),
                 None if fibres is None else fibres.data_ptr(),
                 None if mat_id is None else mat_id.data_ptr())
    arr, nm = _mats(mats)
    _chk(_lib.ib_fe_energy_noalloc(C.byref(mesh), arr, nm, C.byref(x._s), float(h),
                                   _ptr(energy), _stream()), "ib_fe_energy_noalloc")
    return energy


class Batch:
    """Independent hexahedral structures, each on its own grid, packed into one
    plan: every stage is one launch over all of them, and the forward and the
    backward are each one captured CUDA graph.

    `instances` is a list of dicts with the device tensors of each structure:
    conn, X, fibres (or None), mat_id (or None), n, h, origin, mats (list of
    Material), cell/off (FP32 split) or x64 (FP64), u, and the output tensors
    G, f, U; for the backward (ib_backward) also the cotangents gU, gf and
    optionally gG, and the outputs gu, gx.  The tensors must stay alive and in
    place: the graphs bake their addresses in."""

    def __init__(self, instances, precision: int = IB_FP32_SPLIT):
        n = len(instances)
        arr = (_Instance * n)()
        self._keep = instances
        self.n = n
        for i, d in enumerate(instances):
            a = arr[i]
            conn, X = d["conn"], d["X"]
            fib, mid = d.get("fibres"), d.get("mat_id")
            a.mesh = _Mesh(int(X.shape[1]), int(conn.shape[1]), conn.data_ptr(), X.data_ptr(),
                           None if fib is None else fib.data_ptr(),
                           None if mid is None else mid.data_ptr(),
                           _ELEM_OF_NODES.get(int(conn.shape[0]), IB_ELEM_HEX8))
            a.grid = _Grid((C.c_int32 * 3)(*d["n"]), float(d["h"]),
                           (C.c_double * 3)(*d.get("origin", (0.0, 0.0, 0.0))))
            mats = d["mats"]
            a.n_mats = len(mats)
            for k, m in enumerate(mats):
                a.mats[k].model = int(m.model)
                a.mats[k].n_params = len(m.params)
                for j, v in enumerate(m.params):
                    a.mats[k].params[j] = float(v)
                a.mats[k].Ta = float(getattr(m, "Ta", 0.0))
            a.x = _Pos(_p(d.get("cell")), _p(d.get("off")), _p(d.get("x64")), 0.0)
            for name in ("u", "G", "f", "U", "gU", "gf", "gG", "gu", "gx"):
                setattr(a, name, _p(d.get(name)))
        out = C.c_void_p()
        _chk(_lib.ib_batch_create(n, arr, precision, _stream(), C.byref(out)), "ib_batch_create")
        self._h = out

    def forward(self):
        _chk(_lib.ib_batch_forward(self._h, _stream()), "ib_batch_forward")

    def adjoint(self):
        _chk(_lib.ib_batch_adjoint(self._h, _stream()), "ib_batch_adjoint")

    def tuning(self):
        """The packed plan's tuning (points per work item, force CTAs per SM,
        spreading and interpolation CTA caps per SM)."""
        t = (C.c_int32 * 4)()
        _chk(_lib.ib_batch_get_tuning(self._h, t), "ib_batch_get_tuning")
        return list(t)

    def gparams(self):
        out = (C.c_double * (self.n * IB_MAX_MATERIALS * IB_PARAM_ROW))()
        _chk(_lib.ib_batch_gparams(self._h, out, _stream()), "ib_batch_gparams")
        return torch.tensor(list(out), dtype=torch.float64).reshape(self.n, IB_MAX_MATERIALS,
                                                                    IB_PARAM_ROW)

    def __del__(self):
        if getattr(self, "_h", None):
            try:
                _lib.ib_batch_destroy(self._h)
            except Exception:
                pass
            self._h = None


def _p(t):
    return None if t is None else t.data_ptr()


def ib_plan_set_profiling(plan: Plan, enable: bool):
    _chk(_lib.ib_plan_set_profiling(plan.handle, 1 if enable else 0), "ib_plan_set_profiling")


def ib_plan_profile(plan: Plan, reset: bool = True):
    """{stage: (milliseconds, calls, kernel launches)} since the last reset."""
    n = len(STAGES)
    ms = (C.c_double * n)()
    calls = (C.c_int64 * n)()
    launches = (C.c_int64 * n)()
    _chk(_lib.ib_plan_profile(plan.handle, _stream(), ms, calls, launches, 1 if reset else 0),
         "ib_plan_profile")
    return {s: (ms[i], int(calls[i]), int(launches[i])) for i, s in enumerate(STAGES)}


# ---------------------------------------------------------------------------
# autograd: positions enter as the split offset `off` (x = origin + (cell+off) h,
# so dL/doff = h dL/dx); material parameters as a float64 CPU tensor [n_mats][9]
# (the law's parameters) or [n_mats][10] (then column 9 is the active tension T_a).
# ---------------------------------------------------------------------------

def _mats_from(models, params: torch.Tensor):
    Ta = params[:, 9].tolist() if params.shape[1] > 9 else [0.0] * len(models)
    return [Material(m, params[i, :N_PARAMS[m]].tolist(), Ta[i]) for i, m in enumerate(models)]


def _param_grad(gp: torch.Tensor, models, params: torch.Tensor) -> torch.Tensor:
    # zero the unused columns of each row; keep d/dT_a only when params carries T_a
    gp = gp[:, :params.shape[1]].clone()
    for i, m in enumerate(models):
        gp[i, N_PARAMS[m]:9] = 0
    return gp


class FEForce(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan, models, cell, off, params):
        x = Pos(cell=cell, off=off.detach())
        G = ib_fe_force(plan, _mats_from(models, params.detach()), x)
        ctx.plan, ctx.models = plan, models
        ctx.save_for_backward(cell, off, params)
        return G

    @staticmethod
    def backward(ctx, gG):
        cell, off, params = ctx.saved_tensors
        plan = ctx.plan
        x = Pos(cell=cell, off=off.detach(), grad_unit=plan.h)   # d/d off
        Hv, gp = ib_fe_force_adj(plan, _mats_from(ctx.models, params.detach()), x,
                                 gG.contiguous())
        return None, None, None, Hv, _param_grad(gp, ctx.models, params)


class Spread(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan, cell, off, G):
        x = Pos(cell=cell, off=off.detach())
        f = ib_spread(plan, x, G.detach().contiguous())
        ctx.plan = plan
        ctx.save_for_backward(cell, off, G)
        return f

    @staticmethod
    def backward(ctx, gf):
        cell, off, G = ctx.saved_tensors
        x = Pos(cell=cell, off=off.detach(), grad_unit=ctx.plan.h)   # d/d off
        gG, gx = ib_spread_adj(ctx.plan, x, G.detach().contiguous(), gf.contiguous())
        return None, None, gx, gG


class Interp(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan, cell, off, u):
        x = Pos(cell=cell, off=off.detach())
        U = ib_interp(plan, x, u.detach().contiguous())
        ctx.plan = plan
        ctx.save_for_backward(cell, off, u)
        return U

    @staticmethod
    def backward(ctx, gU):
        cell, off, u = ctx.saved_tensors
        x = Pos(cell=cell, off=off.detach(), grad_unit=ctx.plan.h)   # d/d off
        gu, gx = ib_interp_adj(ctx.plan, x, u.detach().contiguous(), gU.contiguous())
        return None, None, gx, gu


class Coupling(torch.autograd.Function):
    """The whole coupling step: ib_forward forward, ib_backward backward."""

    @staticmethod
    def forward(ctx, plan, models, cell, off, params, u):
        ctx.set_materialize_grads(False)
        x = Pos(cell=cell, off=off.detach())
        G, f, U = ib_forward(plan, _mats_from(models, params.detach()), x,
                             u.detach().contiguous())
        ctx.plan, ctx.models = plan, models
        ctx.save_for_backward(cell, off, params, u, G)
        return G, f, U

    @staticmethod
    def backward(ctx, gG, gf, gU):
        cell, off, params, u, G = ctx.saved_tensors
        plan = ctx.plan
        x = Pos(cell=cell, off=off.detach(), grad_unit=plan.h)   # d/d off
        c = lambda t: None if t is None else t.contiguous()
        gx, gu, gp = ib_backward(plan, _mats_from(ctx.models, params.detach()), x,
                                 u.detach().contiguous(), G, c(gG), c(gf), c(gU))
        return None, None, None, gx, _param_grad(gp.cpu(), ctx.models, params), gu


class IBCoupling(torch.nn.Module):
    """G = FE force(x; theta), f = spread(x, G), U = interp(x, u), differentiable in
    the offsets, the material parameters and u (one fused forward and backward)."""

    def __init__(self, plan: Plan, models):
        super().__init__()
        self.plan, self.models = plan, list(models)

    def forward(self, cell, off, params, u):
        return Coupling.apply(self.plan, self.models, cell, off, params, u)
