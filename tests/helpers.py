"""Shared helpers for the GPU parity tests: move a seeded Problem to the
device and build the oracle's view of exactly the same values."""
import numpy as np

import oracle
from paper_2503_22695_gb300 import inputs as I


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (den if den > 0 else 1.0)


class Case:
    """A problem on the GPU (through the C ABI) and in the oracle."""

    def __init__(self, prob: I.Problem, quad: int = 0):
        import torch
        from paper_2503_22695_gb300 import ibfe
        self.prob = prob
        self.ibfe = ibfe
        self.fp64 = prob.fp64
        dt = torch.float64 if prob.fp64 else torch.float32
        self.dt = dt
        dev = "cuda"
        self.conn = torch.from_numpy(prob.conn).to(dev)
        self.X = torch.from_numpy(prob.X).to(dev, dt)
        self.fib = torch.from_numpy(prob.fibres).to(dev, dt)
        self.mat_id = torch.from_numpy(prob.mat_id).to(dev)
        g = prob.grid
        self.plan = ibfe.Plan(self.conn, self.X, g.n, g.h, g.origin, fibres=self.fib,
                              mat_id=self.mat_id,
                              precision=ibfe.IB_FP64 if prob.fp64 else ibfe.IB_FP32_SPLIT,
                              quad=quad)
        if prob.fp64:
            self.x_np = prob.x.copy()
            self.pos = ibfe.Pos(x64=torch.from_numpy(self.x_np).to(dev))
        else:
            self.cell = torch.from_numpy(prob.cell).to(dev)
            self.off = torch.from_numpy(prob.off).to(dev)
            self.pos = ibfe.Pos(cell=self.cell, off=self.off)
            self.x_np = I.from_split(prob.cell, prob.off, g)
        self.mats = [ibfe.Material(m.model, m.params, m.active) for m in prob.materials]
        self.u = torch.from_numpy(prob.u).to(dev, dt)
        # oracle sees the device values widened exactly to float64
        self.orc = oracle.Model(grid=g, conn=prob.conn, X=prob.X.astype(np.float64),
                                fibres=prob.fibres.astype(np.float64), mat_id=prob.mat_id,
                                materials=prob.materials)
        self.u_np = prob.u.astype(np.float64)

    def to_dev(self, a):
        import torch
        return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", self.dt)

    def rounded(self, a):
        """Round an oracle array to the device precision (the value both sides see)."""
        return np.asarray(a).astype(np.float64 if self.fp64 else np.float32).astype(np.float64)


def np_(t):
    return t.detach().double().cpu().numpy()


def hex_fibre_stretch(prob, x):
    """I4 - 1 = |F e|^2 - 1 of the fibre (e_f) and sheet (e_s) directions at the
    2x2x2 Gauss points of a trilinear hexahedral mesh (VTK corner order), in
    FP64: arrays [8][E] each.  F = (dx/dxi)(dX/dxi)^-1 from the shape-function
    gradients at xi = +-1/sqrt(3)."""
    sg = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                   [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], float)
    g = 1.0 / np.sqrt(3.0)
    X = prob.X.astype(np.float64)
    ef = prob.fibres[0:3].astype(np.float64)
    es = prob.fibres[3:6].astype(np.float64)
    d4f, d4s = [], []
    for q in range(8):
        xi = np.array([(1 if (q >> k) & 1 else -1) * g for k in range(3)])
        f = (1 + sg * xi) / 2                                   # [8 corners][3]
        dN = np.stack([sg[:, k] / 2 * np.prod(np.delete(f, k, axis=1), axis=1)
                       for k in range(3)], axis=1)              # dN_a/dxi_k
        J0 = np.einsum('iae,ak->eik', X[:, prob.conn], dN)
        Jx = np.einsum('iae,ak->eik', x[:, prob.conn], dN)
        F = Jx @ np.linalg.inv(J0)
        for e_dir, out in ((ef, d4f), (es, d4s)):
            Fe = np.einsum('eij,je->ei', F, e_dir)
            out.append((Fe ** 2).sum(axis=1) - 1.0)
    return np.array(d4f), np.array(d4s)


def kink_nodes(prob, x, band=5e-7):
    """Nodes of the elements with a Gauss point whose fibre or sheet stretch
    lies within `band` of 1.  The tension-only fibre terms make the Hessian
    jump at I4 = 1; an FP32 evaluation within rounding of the kink may take
    either branch, and both are valid for inputs within that rounding (the
    FP32 displacement gradient moves I4 - 1 by about 1.4e-7 on these
    meshes; the default band is 3.5 times that)."""
    d4f, d4s = hex_fibre_stretch(prob, x)
    near = ((np.abs(d4f) < band) | (np.abs(d4s) < band)).any(axis=0)
    return np.unique(prob.conn[:, near])
