"""Pins for the FP64 oracle: facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed-form
values, Peskin's kernel conditions, exact derivatives by central finite
differences, invariances of hyperelastic energies, conservation of total force
and torque under spreading, exactness of interpolation on constant and linear
fields, the discrete adjointness of spreading and interpolation (Section 4.4),
and brute-force sums over every grid face.
"""
import dataclasses
import math
import os

import numpy as np
import pytest

import oracle
from paper_2503_22695_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rot(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a*a+b*b-c*c-d*d, 2*(b*c-a*d), 2*(b*d+a*c)],
                     [2*(b*c+a*d), a*a-b*b+c*c-d*d, 2*(c*d-a*b)],
                     [2*(b*d-a*c), 2*(c*d+a*b), a*a-b*b-c*c+d*d]])


# ---------------------------------------------------------------------------
# 4-point kernel
# ---------------------------------------------------------------------------

def test_phi_closed_form_golden():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "peskin4_closed_form.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) >= 10
    for r, expr in rows:
        want = eval(expr, {"sqrt": math.sqrt})
        assert oracle.phi(float(r)) == pytest.approx(want, abs=1e-15), (r, expr)


def test_phi_peskin_conditions():
    # Peskin's conditions for the 4-point kernel: partition of unity, equal
    # even/odd sums, vanishing first moment, sum of squares 3/8.
    rng = np.random.default_rng(0)
    for r in rng.uniform(-3, 3, size=200):
        js = np.arange(-6, 7)
        w = np.array([oracle.phi(r - j) for j in js])
        assert w.sum() == pytest.approx(1.0, abs=1e-14)
        assert w[js % 2 == 0].sum() == pytest.approx(0.5, abs=1e-14)
        assert ((r - js) * w).sum() == pytest.approx(0.0, abs=1e-14)
        assert (w * w).sum() == pytest.approx(3.0 / 8.0, abs=1e-14)
        assert (w >= 0).all() and np.count_nonzero(w) <= 4


def test_dphi_is_derivative_and_c1():
    rng = np.random.default_rng(1)
    eps = 1e-6
    for r in np.concatenate([rng.uniform(-2.2, 2.2, size=100), [0.3, -1.7]]):
        if min(abs(abs(r) - 1), abs(abs(r) - 2), abs(r)) < 1e-4:
            continue
        fd = (oracle.phi(r + eps) - oracle.phi(r - eps)) / (2 * eps)
        assert oracle.dphi(r) == pytest.approx(fd, abs=1e-8)
    # C1 at |r| = 1 and |r| = 2; derivative sums to zero over the stencil
    for k in (1.0, 2.0):
        assert oracle.dphi(k - 1e-12) == pytest.approx(oracle.dphi(k + 1e-12), abs=1e-9)
    for r in rng.uniform(-3, 3, size=50):
        assert sum(oracle.dphi(r - j) for j in range(-6, 7)) == pytest.approx(0, abs=1e-13)


# ---------------------------------------------------------------------------
# constitutive laws
# ---------------------------------------------------------------------------

MODELS = [
    (I.NEO_HOOKEAN, (0.5, 100.0)),
    (I.FIBRE1, I.FIBRE1_LEAFLET),
    (I.HO, I.HO_DEFAULT),
    (I.STD_REINF, I.STD_REINF_COOK),
    (I.FIBRE2, I.FIBRE2_AV),
]


def _rand_F(rng, amp=0.15):
    F = np.eye(3) + rng.uniform(-amp, amp, size=(3, 3))
    assert np.linalg.det(F) > 0
    return F


def _fibres(rng):
    ef = rng.normal(size=3)
    ef /= np.linalg.norm(ef)
    es = rng.normal(size=3)
    es -= es @ ef * ef
    es /= np.linalg.norm(es)
    return ef, es


@pytest.mark.parametrize("model,params", MODELS)
def test_stress_is_energy_derivative(model, params):
    # P = dPsi/dF (Section 2: P = dW/dF) by central differences, away from the
    # tension-only kink I4 = 1.
    rng = np.random.default_rng(10 + model)
    checked = 0
    for _ in range(40):
        F = _rand_F(rng)
        ef, es = _fibres(rng)
        I4 = [np.sum((F @ e) ** 2) for e in (ef, es)]
        if min(abs(v - 1) for v in I4) < 1e-3:
            continue
        P, _ = oracle.stress(model, params, F, ef, es)
        eps = 1e-6
        fd = np.zeros((3, 3))
        for i in range(3):
            for j in range(3):
                dF = np.zeros((3, 3))
                dF[i, j] = eps
                fd[i, j] = (oracle.stress(model, params, F + dF, ef, es)[1] -
                            oracle.stress(model, params, F - dF, ef, es)[1]) / (2 * eps)
        np.testing.assert_allclose(P, fd, rtol=1e-7, atol=1e-7 * np.abs(P).max())
        checked += 1
    assert checked > 20


@pytest.mark.parametrize("model,params", MODELS)
def test_stress_reference_state_and_frame_invariance(model, params):
    rng = np.random.default_rng(20 + model)
    ef, es = _fibres(rng)
    P0, psi0 = oracle.stress(model, params, np.eye(3), ef, es)
    assert np.abs(P0).max() < 1e-13 and abs(psi0) < 1e-13
    for _ in range(10):
        F = _rand_F(rng)
        Q = rot(rng)
        P, psi = oracle.stress(model, params, F, ef, es)
        PQ, psiQ = oracle.stress(model, params, Q @ F, ef, es)
        assert psiQ == pytest.approx(psi, rel=1e-12, abs=1e-14)
        np.testing.assert_allclose(PQ, Q @ P, rtol=1e-10, atol=1e-12 * np.abs(P).max())


def test_neo_hookean_small_strain_lame():
    # a = mu/2: linearisation gives P = 2 mu eps + (kappa - 2 mu/3) tr(eps) I.
    mu, kappa = 1.0, 100.0
    rng = np.random.default_rng(3)
    A = rng.normal(size=(3, 3))
    d = 1e-6
    P, _ = oracle.stress(I.NEO_HOOKEAN, (mu / 2, kappa), np.eye(3) + d * A)
    eps = 0.5 * (A + A.T)
    lin = 2 * mu * eps + (kappa - 2 * mu / 3) * np.trace(eps) * np.eye(3)
    np.testing.assert_allclose(P / d, lin, rtol=1e-4, atol=1e-4)


def test_ho_isotropic_limit_is_neo_hookean():
    # a/(2b)(exp[b(I1bar-3)]-1) -> a/2 (I1bar-3) as b -> 0, so HO with no fibre
    # stiffness reduces to neo-Hookean with a_NH = a/2.
    rng = np.random.default_rng(4)
    F = _rand_F(rng)
    ef, es = _fibres(rng)
    a, kappa = 0.7, 50.0
    P_ho, psi_ho = oracle.stress(I.HO, (a, 1e-9, 0, 1, 0, 1, 0, 1, kappa), F, ef, es)
    P_nh, psi_nh = oracle.stress(I.NEO_HOOKEAN, (a / 2, kappa), F)
    np.testing.assert_allclose(P_ho, P_nh, rtol=1e-7, atol=1e-9)
    assert psi_ho == pytest.approx(psi_nh, rel=1e-7)


HO_SETS = [
    I.HO_DEFAULT,
    (0.5, 2.0, 3.0, 4.0, 1.5, 2.5, 0.8, 3.5, 40.0),
    (1.3, 0.4, 0.7, 9.0, 2.2, 0.3, 4.1, 0.6, 7.0),
]


@pytest.mark.parametrize("params", HO_SETS)
def test_ho_simple_shear_closed_form(params):
    # Psi_4 (Section 3) under simple shear of the fibre-sheet plane.  With e_f
    # and e_s orthonormal and F = I + g e_f (x) e_s: J = 1, I1bar - 3 = g^2,
    # I4f = 1, I4s = 1 + g^2, I8fs = e_f.C e_s = g, so
    #   Psi = a/(2b)(e^{b g^2} - 1) + a_s/(2b_s)(e^{b_s g^4} - 1)
    #       + a_fs/(2b_fs)(e^{b_fs g^2} - 1)
    # and its g-derivative is the shear stress e_f.P e_s = P : (e_f (x) e_s):
    #   a g e^{b g^2} + 2 a_s g^3 e^{b_s g^4} + a_fs g e^{b_fs g^2}.
    # Shearing the other way (F = I + g e_s (x) e_f) swaps the roles of the
    # fibre and sheet families (I4f = 1 + g^2, I4s = 1).  Each term has its own
    # exponent and prefactor, so a dropped square (I8 for I8^2), a missing 1/2
    # or a wrong rate constant in any of them fails here.
    a, b, af, bf, as_, bs, afs, bfs, kap = params
    rng = np.random.default_rng(41)
    for _ in range(3):
        ef, es = _fibres(rng)
        for g in (-0.45, -0.1, 0.03, 0.2, 0.6):
            for fam, (u, v, a4, b4) in enumerate(((ef, es, as_, bs), (es, ef, af, bf))):
                F = np.eye(3) + g * np.outer(u, v)
                P, psi = oracle.stress(I.HO, params, F, ef, es)
                want = (a / (2 * b) * np.expm1(b * g * g) + a4 / (2 * b4) * np.expm1(b4 * g ** 4)
                        + afs / (2 * bfs) * np.expm1(bfs * g * g))
                assert psi == pytest.approx(want, rel=1e-13, abs=1e-15)
                shear = (a * g * np.exp(b * g * g) + 2 * a4 * g ** 3 * np.exp(b4 * g ** 4)
                         + afs * g * np.exp(bfs * g * g))
                assert u @ P @ v == pytest.approx(shear, rel=1e-13, abs=1e-15)


@pytest.mark.parametrize("params", HO_SETS)
def test_ho_dilation_closed_form(params):
    # F = lam I: J = lam^3, I1bar = 3, I8fs = lam^2 e_f.e_s = 0 and
    # I4f = I4s = lam^2, so only the volumetric and the two fibre terms remain:
    #   Psi = kappa/2 (3 ln lam)^2 + sum_{i=f,s} a_i/(2b_i)(e^{b_i(lam^2-1)^2} - 1)
    # (the fibres carry tension only: zero for lam < 1); the pressure-like
    # derivative dPsi/dlam = P : I.
    a, b, af, bf, as_, bs, afs, bfs, kap = params
    ef, es = _fibres(np.random.default_rng(42))
    for lam in (0.93, 0.99, 1.02, 1.08):
        P, psi = oracle.stress(I.HO, params, lam * np.eye(3), ef, es)
        d = lam * lam - 1 if lam > 1 else 0.0
        want = kap / 2 * (3 * np.log(lam)) ** 2 + sum(
            ai / (2 * bi) * np.expm1(bi * d * d) for ai, bi in ((af, bf), (as_, bs)))
        assert psi == pytest.approx(want, rel=1e-13, abs=1e-15)
        dpsi = kap * 9 * np.log(lam) / lam + sum(
            2 * ai * d * lam * np.exp(bi * d * d) for ai, bi in ((af, bf), (as_, bs)))
        assert np.trace(P) == pytest.approx(dpsi, rel=1e-12, abs=1e-14)


def test_standard_reinforcing_isotropic_limit_is_neo_hookean():
    # Psi_1 with G_L = G_T and E_L = 3 G_T has no fibre terms
    # (G_T - G_L = 0, E_L + G_T - 4 G_L = 0): neo-Hookean with a = G_T/2.
    rng = np.random.default_rng(31)
    ef, es = _fibres(rng)
    for _ in range(4):
        F = _rand_F(rng)
        P1, psi1 = oracle.stress(I.STD_REINF, (2.0, 2.0, 6.0, 50.0), F, ef, es)
        P0, psi0 = oracle.stress(I.NEO_HOOKEAN, (1.0, 50.0), F, ef, es)
        np.testing.assert_allclose(P1, P0, rtol=1e-13, atol=1e-13)
        assert psi1 == pytest.approx(psi0, rel=1e-13, abs=1e-15)


def test_standard_reinforcing_fibre_terms_by_invariants():
    # Psi_1's anisotropic energy against I4 and I5 computed directly from C
    rng = np.random.default_rng(32)
    ef, es = _fibres(rng)
    GT, GL, EL, kap = I.STD_REINF_COOK
    for _ in range(4):
        F = _rand_F(rng)
        C = F.T @ F
        I4, I5 = ef @ C @ ef, ef @ C @ C @ ef
        J = np.linalg.det(F)
        I1b = J ** (-2 / 3) * np.trace(C)
        want = (GT / 2 * (I1b - 3) + (GT - GL) / 2 * (2 * I4 - I5 - 1) +
                (EL + GT - 4 * GL) / 8 * (I4 - 1) ** 2 + kap / 2 * np.log(J) ** 2)
        _, psi = oracle.stress(I.STD_REINF, I.STD_REINF_COOK, F, ef, es)
        assert psi == pytest.approx(want, rel=1e-12)


def test_fibre_model_2_limits():
    # Psi_3: C10 (exp[C01 (I1bar - 3)] - 1) tends to C10 C01 (I1bar - 3) as
    # C01 -> 0 (neo-Hookean with a = C10 C01), and its fibre term acts in
    # compression too (no tension-only clamp, unlike Psi_2).
    rng = np.random.default_rng(33)
    ef, es = _fibres(rng)
    F = _rand_F(rng)
    P3, _ = oracle.stress(I.FIBRE2, (2e6, 1e-6, 0.0, 1.0, 50.0), F, ef, es)
    P0, _ = oracle.stress(I.NEO_HOOKEAN, (2.0, 50.0), F, ef, es)
    np.testing.assert_allclose(P3, P0, rtol=1e-4, atol=1e-6)
    Fc = np.diag([0.95, 1.02, 1.03])            # fibre along x compressed
    x = np.array([1.0, 0.0, 0.0])
    Pc, _ = oracle.stress(I.FIBRE2, (1.0, 1.0, 3.0, 2.0, 0.0), Fc, x, np.array([0, 1.0, 0]))
    Pn, _ = oracle.stress(I.FIBRE2, (1.0, 1.0, 0.0, 2.0, 0.0), Fc, x, np.array([0, 1.0, 0]))
    d = 0.95 ** 2 - 1
    assert Pc[0, 0] - Pn[0, 0] == pytest.approx(2 * 3.0 * d * np.exp(2.0 * d * d) * 0.95,
                                                rel=1e-12)


def test_fibres_carry_tension_only():
    # I4* = max(I4, 1): a compressed fibre adds nothing (Psi_2 and Psi_4).
    F = np.diag([0.9, 1.05, 1.0 / (0.9 * 1.05)])
    ef, es = np.array([1.0, 0, 0]), np.array([0, 1.0, 0])
    P1, _ = oracle.stress(I.FIBRE1, (1.0, 5.0, 2.0, 10.0), F, ef, es)
    P0, _ = oracle.stress(I.FIBRE1, (1.0, 0.0, 2.0, 10.0), F, ef, es)
    np.testing.assert_allclose(P1, P0, atol=1e-14)
    P1, _ = oracle.stress(I.FIBRE1, (1.0, 5.0, 2.0, 10.0), F, es, ef)   # fibre along y, stretched
    assert np.abs(P1 - P0).max() > 1e-3


@pytest.mark.parametrize("model,params", MODELS)
def test_stress_direction_derivative(model, params):
    rng = np.random.default_rng(30 + model)
    for _ in range(10):
        F = _rand_F(rng)
        ef, es = _fibres(rng)
        dF = rng.normal(size=(3, 3))
        eps = 1e-6
        I4 = [np.sum((F @ e) ** 2) for e in (ef, es)]
        if min(abs(v - 1) for v in I4) < 1e-3:
            continue
        fd = (oracle.stress(model, params, F + eps * dF, ef, es)[0] -
              oracle.stress(model, params, F - eps * dF, ef, es)[0]) / (2 * eps)
        dP = oracle.stress_dir(model, params, F, dF, ef, es)
        np.testing.assert_allclose(dP, fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())


# ---------------------------------------------------------------------------
# FE force, mass
# ---------------------------------------------------------------------------

def tiny_mesh(model=I.HO, params=I.HO_DEFAULT, n=16, blocks=(2, 2, 1), seed=7, noise=0.15):
    p = I.block_problem(seed=seed, n=n, blocks=blocks, noise=noise, fp64=True)
    rng = np.random.default_rng(seed)
    fib = np.zeros((6, p.n_elems))
    for e in range(p.n_elems):
        ef, es = _fibres(rng)
        fib[:3, e], fib[3:, e] = ef, es
    p.fibres = fib
    p.materials = [I.Material(model, params)]
    return p


# ---------------------------------------------------------------------------
# active fibre stress (Section 6.1)
# ---------------------------------------------------------------------------

ACTIVE = [(I.HO, I.HO_DEFAULT, 60.0), (I.NEO_HOOKEAN, (0.5, 100.0), 30.0),
          (I.FIBRE2, I.FIBRE2_AV, 45.0)]


@pytest.mark.parametrize("model,params,Ta", ACTIVE)
def test_active_stress_is_energy_derivative(model, params, Ta):
    """P^a = F S_a has the potential W_a(I4f) at fixed t, so P = dPsi/dF holds
    with the active term included (checked by central differences)."""
    rng = np.random.default_rng(70 + model)
    checked = 0
    for _ in range(30):
        F = _rand_F(rng)
        ef, es = _fibres(rng)
        I4 = [np.sum((F @ e) ** 2) for e in (ef, es)]
        if min(abs(v - 1) for v in I4) < 1e-3:
            continue
        P, _ = oracle.stress(model, params, F, ef, es, Ta=Ta)
        eps = 1e-6
        fd = np.zeros((3, 3))
        for i in range(3):
            for j in range(3):
                dF = np.zeros((3, 3))
                dF[i, j] = eps
                fd[i, j] = (oracle.stress(model, params, F + dF, ef, es, Ta=Ta)[1] -
                            oracle.stress(model, params, F - dF, ef, es, Ta=Ta)[1]) / (2 * eps)
        np.testing.assert_allclose(P, fd, rtol=1e-7, atol=1e-7 * np.abs(P).max())
        checked += 1
    assert checked > 15


def test_active_stress_closed_forms():
    """With no passive stiffness (neo-Hookean a = kappa = 0) the stress is the
    active term alone.  At F = I it is T_a e_f (x) e_f (T = T_a at I4f = 1) for
    any fibre direction; under a stretch lambda along e_f = x it is
    P_11 = T_a (1 + 4.9 (lambda - 1)) lambda (P = F S with S_11 = T), every
    other entry zero; its energy vanishes at F = I."""
    Ta = 37.0
    rng = np.random.default_rng(71)
    for _ in range(5):
        ef, es = _fibres(rng)
        P, psi = oracle.stress(I.NEO_HOOKEAN, (0.0, 0.0), np.eye(3), ef, es, Ta=Ta)
        np.testing.assert_allclose(P, Ta * np.outer(ef, ef), rtol=1e-14, atol=1e-14 * Ta)
        assert abs(psi) < 1e-14 * Ta
    for lam in (0.8, 0.95, 1.0, 1.1, 1.3):
        F = np.diag([lam, 1.0, 1.0])
        P, _ = oracle.stress(I.NEO_HOOKEAN, (0.0, 0.0), F, (1, 0, 0), (0, 1, 0), Ta=Ta)
        want = np.zeros((3, 3))
        want[0, 0] = Ta * (1 + 4.9 * (lam - 1)) * lam
        np.testing.assert_allclose(P, want, rtol=1e-14, atol=1e-14 * Ta)


@pytest.mark.parametrize("model,params,Ta", ACTIVE)
def test_active_stress_linear_in_tension_and_objective(model, params, Ta):
    rng = np.random.default_rng(72 + model)
    for _ in range(8):
        F = _rand_F(rng)
        ef, es = _fibres(rng)
        P0, psi0 = oracle.stress(model, params, F, ef, es)
        P1, psi1 = oracle.stress(model, params, F, ef, es, Ta=Ta)
        P2, psi2 = oracle.stress(model, params, F, ef, es, Ta=2 * Ta)
        np.testing.assert_allclose(P2 - P0, 2 * (P1 - P0), rtol=1e-10, atol=1e-12 * Ta)
        assert psi2 - psi0 == pytest.approx(2 * (psi1 - psi0), rel=1e-10, abs=1e-12 * Ta)
        Q = rot(rng)
        PQ, psiQ = oracle.stress(model, params, Q @ F, ef, es, Ta=Ta)
        np.testing.assert_allclose(PQ, Q @ P1, rtol=1e-10, atol=1e-12 * np.abs(P1).max())
        assert psiQ == pytest.approx(psi1, rel=1e-12, abs=1e-14)


def test_active_tension_waveform():
    """T_a(t) of Section 6.1: zero in diastole (t < 0.5 s), rising to its peak
    84260 (1 - e^-4.5) Pa at 0.65 s, mirror-symmetric about 0.65 s, back to
    zero at 0.8 s, repeated every 0.8 s (the cardiac cycle)."""
    Ta = oracle.active_tension
    for t in (0.0, 0.1, 0.3, 0.4999, 0.5, 0.8, 1.2, 1.6, 2.4):
        assert Ta(t) == pytest.approx(0.0, abs=1e-9)
    assert Ta(0.65) == pytest.approx(84260 * (1 - math.exp(-4.5)), rel=1e-14)
    for s in (0.01, 0.05, 0.1, 0.149):
        assert Ta(0.65 - s) == pytest.approx(Ta(0.65 + s), rel=1e-12)
    ts = np.linspace(0.5, 0.65, 40)
    v = [Ta(t) for t in ts]
    assert all(b > a for a, b in zip(v, v[1:]))
    assert max(Ta(t) for t in np.linspace(0, 0.8, 801)) <= Ta(0.65) + 1e-9
    for t in (0.55, 0.6, 0.7, 0.75):
        for k in (1, 2):
            assert Ta(t + 0.8 * k) == pytest.approx(Ta(t), rel=1e-9)


def test_active_force_gradients():
    """With T_a on: G = -dE/dx, the Hessian-vector product and the T_a
    gradient (column 9 of the parameter gradients) by central differences."""
    p = tiny_mesh(I.HO, I.HO_DEFAULT)
    Ta = 60.0
    p.materials = [I.Material(I.HO, I.HO_DEFAULT, Ta)]
    m = oracle.Model(p)
    x = p.x
    G, _ = m.fe_force(x)
    eps = 1e-6 * p.grid.h
    rng = np.random.default_rng(73)
    for _ in range(8):
        a, i = rng.integers(p.n_nodes), rng.integers(3)
        xp, xm = x.copy(), x.copy()
        xp[i, a] += eps
        xm[i, a] -= eps
        fd = -(m.fe_force(xp)[1] - m.fe_force(xm)[1]) / (2 * eps)
        assert G[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-8 * np.abs(G).max())
    v = rng.normal(size=x.shape)
    Hv, gp = m.fe_force_adj(x, v)
    e2 = 1e-7 * p.grid.h
    fd = (m.fe_force(x + e2 * v)[0] - m.fe_force(x - e2 * v)[0]) / (2 * e2)
    np.testing.assert_allclose(Hv, fd, rtol=1e-5, atol=1e-6 * np.abs(Hv).max())
    d = 1e-4
    m.set_materials([I.Material(I.HO, I.HO_DEFAULT, Ta + d)])
    Gp = m.fe_force(x)[0]
    m.set_materials([I.Material(I.HO, I.HO_DEFAULT, Ta - d)])
    Gm = m.fe_force(x)[0]
    assert gp[0, 9] == pytest.approx(np.sum(v * (Gp - Gm)) / (2 * d), rel=1e-7)
    # the passive gradients do not depend on how T_a enters
    m.set_materials([I.Material(I.HO, I.HO_DEFAULT)])
    _, gp0 = m.fe_force_adj(x, v)
    np.testing.assert_allclose(gp[0, :9], gp0[0, :9], rtol=1e-12)
    assert gp0[0, 9] == pytest.approx(gp[0, 9], rel=1e-12)  # dP/dT_a does not involve T_a


def test_mass_is_volume():
    p = I.block_problem(fp64=True)
    m = oracle.Model(p)
    assert m.mass().sum() == pytest.approx(128 * p.grid.h ** 3, rel=1e-13)
    assert (m.mass() > 0).all()


@pytest.mark.parametrize("model,params", MODELS)
def test_force_zero_in_reference_and_rigid_motion(model, params):
    p = tiny_mesh(model, params)
    m = oracle.Model(p)
    G, E = m.fe_force(p.X)
    scale = params[-1] * p.grid.h ** 2
    assert np.abs(G).max() < 1e-12 * scale and abs(E) < 1e-15
    Q = rot(np.random.default_rng(5))
    x = Q @ (p.X - 0.5) + 0.5 + np.array([[0.01], [-0.02], [0.03]])
    G, E = m.fe_force(x)
    assert np.abs(G).max() < 1e-11 * scale and abs(E) < 1e-15


@pytest.mark.parametrize("model,params", MODELS)
def test_force_is_minus_energy_gradient(model, params):
    p = tiny_mesh(model, params)
    m = oracle.Model(p)
    x = p.x
    G, _ = m.fe_force(x)
    # internal force: no net force and no net torque
    assert np.abs(G.sum(axis=1)).max() < 1e-12 * np.abs(G).max()
    torque = np.cross(x.T, G.T).sum(axis=0)
    assert np.abs(torque).max() < 1e-12 * np.abs(G).max()
    eps = 1e-6 * p.grid.h
    rng = np.random.default_rng(8)
    for _ in range(12):
        a, i = rng.integers(p.n_nodes), rng.integers(3)
        xp, xm = x.copy(), x.copy()
        xp[i, a] += eps
        xm[i, a] -= eps
        fd = -(m.fe_force(xp)[1] - m.fe_force(xm)[1]) / (2 * eps)
        assert G[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-8 * np.abs(G).max())


@pytest.mark.parametrize("model,params", MODELS)
def test_force_adjoint_hvp_and_params(model, params):
    p = tiny_mesh(model, params)
    m = oracle.Model(p)
    x = p.x
    rng = np.random.default_rng(9)
    v = rng.normal(size=x.shape)
    w = rng.normal(size=x.shape)
    Hv, gp = m.fe_force_adj(x, v)
    Hw, _ = m.fe_force_adj(x, w)
    # symmetric Hessian: <w, Hv> = <v, Hw>
    assert np.sum(w * Hv) == pytest.approx(np.sum(v * Hw), rel=1e-11)
    eps = 1e-7 * p.grid.h
    fd = (m.fe_force(x + eps * v)[0] - m.fe_force(x - eps * v)[0]) / (2 * eps)
    np.testing.assert_allclose(Hv, fd, rtol=1e-5, atol=1e-6 * np.abs(Hv).max())
    # dG/dtheta_k . v by differences in each parameter
    for k in range(len(params)):
        th = np.array(params, dtype=float)
        d = 1e-6 * max(abs(th[k]), 1e-3)
        tp, tm = th.copy(), th.copy()
        tp[k] += d
        tm[k] -= d
        m.set_materials([I.Material(model, tuple(tp))])
        Gp = m.fe_force(x)[0]
        m.set_materials([I.Material(model, tuple(tm))])
        Gm = m.fe_force(x)[0]
        m.set_materials([I.Material(model, tuple(th))])
        want = np.sum(v * (Gp - Gm)) / (2 * d)
        assert gp[0, k] == pytest.approx(want, rel=1e-5, abs=1e-9 * np.abs(gp).max()), k


# ---------------------------------------------------------------------------
# spreading and interpolation
# ---------------------------------------------------------------------------

def small_problem(n=8, blocks=(2, 2, 1), seed=11, centre=None):
    p = I.block_problem(seed=seed, n=n, blocks=blocks, noise=0.3, fp64=True, centre=centre)
    rng = np.random.default_rng(seed)
    G = rng.normal(size=(3, p.n_nodes))
    return p, G


@pytest.mark.parametrize("centre", [None, (0.02, 0.97, 0.5)])
def test_spread_matches_brute_force_over_all_faces(centre):
    # every face of the grid, every Gauss point, nearest periodic image;
    # the second case straddles the periodic seam in x and y.
    p, G = small_problem(centre=centre)
    m = oracle.Model(p)
    f = m.spread(p.x, G)
    n = p.grid.n[0]
    comp, idx = [], []
    for c in range(3):
        for i2 in range(n):
            for i1 in range(n):
                for i0 in range(n):
                    comp.append(c)
                    idx.append((i0, i1, i2))
    bf = m.spread_at(p.x, G, comp, idx).reshape(3, n, n, n)
    np.testing.assert_allclose(f, bf, rtol=1e-12, atol=1e-12 * np.abs(f).max())


def test_spread_conserves_force_and_torque():
    p, G = small_problem(n=16, blocks=(2, 3, 2))
    m = oracle.Model(p)
    f = m.spread(p.x, G)
    h = p.grid.h
    np.testing.assert_allclose(h ** 3 * f.reshape(3, -1).sum(axis=1), G.sum(axis=1),
                               rtol=1e-12, atol=1e-12)
    # torque: h^3 sum x_face x f = sum_q chi_q x P_q (first-moment condition),
    # with x_face the staggered face position of each component.
    n = p.grid.n[0]
    ii = np.arange(n)
    torque = np.zeros(3)
    pos = []
    for c in range(3):
        s = [0.5, 0.5, 0.5]
        s[c] = 0.0
        z, y, x = np.meshgrid((ii + s[2]) * h, (ii + s[1]) * h, (ii + s[0]) * h, indexing="ij")
        pos.append((x, y, z))
    # tau = sum r x f: tau_x = y f_z - z f_y, etc.
    torque[0] = np.sum(pos[2][1] * f[2]) - np.sum(pos[1][2] * f[1])
    torque[1] = np.sum(pos[0][2] * f[0]) - np.sum(pos[2][0] * f[2])
    torque[2] = np.sum(pos[1][0] * f[1]) - np.sum(pos[0][1] * f[0])
    torque *= h ** 3
    # same torque from the Lagrangian side: Gauss-point forces at chi_q equal
    # the nodal forces redistributed with the lumped projection; compute it via
    # interpolation of the linear fields x, y, z (exact by the first moment).
    want = np.zeros(3)
    lin = []
    for d in range(3):
        ud = np.zeros((3, n, n, n))
        for c in range(3):
            ud[c] = pos[c][d]
        lin.append(ud)
    # sum_q chi_q,d P_q,c = <G, interp(field that is x_d in component c)>
    Gd = {}
    for d in range(3):
        for c in range(3):
            u = np.zeros((3, n, n, n))
            u[c] = pos[c][d]
            U = m.interp(p.x, u)
            Gd[(d, c)] = np.sum(G[c] * U[c])
    want[0] = Gd[(1, 2)] - Gd[(2, 1)]
    want[1] = Gd[(2, 0)] - Gd[(0, 2)]
    want[2] = Gd[(0, 1)] - Gd[(1, 0)]
    np.testing.assert_allclose(torque, want, rtol=1e-11, atol=1e-13)


def test_interp_exact_on_constant_and_linear_fields():
    p, _ = small_problem(n=16, blocks=(3, 2, 2))
    m = oracle.Model(p)
    n = p.grid.n[0]
    h = p.grid.h
    const = np.array([0.3, -1.2, 2.5])
    u = np.broadcast_to(const[:, None, None, None], (3, n, n, n)).copy()
    U = m.interp(p.x, u)
    np.testing.assert_allclose(U, np.broadcast_to(const[:, None], U.shape), rtol=1e-13)
    # linear field (the structure sits away from the seam): U^IB_q = A chi_q + b
    A = np.random.default_rng(2).normal(size=(3, 3))
    b = np.array([0.1, 0.2, -0.3])
    ii = np.arange(n)
    for c in range(3):
        s = [0.5, 0.5, 0.5]
        s[c] = 0.0
        z, y, x = np.meshgrid((ii + s[2]) * h, (ii + s[1]) * h, (ii + s[0]) * h, indexing="ij")
        u[c] = A[c, 0] * x + A[c, 1] * y + A[c, 2] * z + b[c]
    _, Uq = m.interp(p.x, u, want_gauss=True)
    # chi_q of a trilinear element at a Gauss point, written with the corner
    # weights prod_d (1 + c_d xi_d)/8 (VTK corner signs)
    g = 1 / math.sqrt(3)
    for q in range(8):
        xi = np.array([(2 * ((q >> d) & 1) - 1) * g for d in range(3)])
        Nq = np.prod(1 + I.HEX_CORNERS * xi, axis=1) / 8
        chi = np.einsum("a,iae->ie", Nq, p.x[:, p.conn])
        np.testing.assert_allclose(Uq[:, q], A @ chi + b[:, None], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("centre", [None, (0.99, 0.5, 0.01)])
def test_spread_interp_adjoint_identity(centre):
    # Section 4.4: with the same quadrature, spreading and interpolation are
    # discretely adjoint: h^3 sum f.u = sum_a G_a . U_a.
    p, G = small_problem(n=16, blocks=(3, 3, 2), centre=centre)
    m = oracle.Model(p)
    rng = np.random.default_rng(12)
    u = rng.normal(size=(3, 16, 16, 16))
    f = m.spread(p.x, G)
    U = m.interp(p.x, u)
    lhs = p.grid.h ** 3 * np.sum(f * u)
    rhs = np.sum(G * U)
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_linear_adjoints():
    p, G = small_problem(n=16, blocks=(3, 2, 2))
    m = oracle.Model(p)
    rng = np.random.default_rng(13)
    gf = rng.normal(size=(3, 16, 16, 16))
    gU = rng.normal(size=G.shape)
    u = rng.normal(size=gf.shape)
    gG, _ = m.spread_adj(p.x, G, gf, want_gx=False)
    assert np.sum(gG * G) == pytest.approx(np.sum(gf * m.spread(p.x, G)), rel=1e-12)
    gu, _ = m.interp_adj(p.x, u, gU, want_gx=False)
    assert np.sum(gu * u) == pytest.approx(np.sum(gU * m.interp(p.x, u)), rel=1e-12)


def test_position_adjoints_by_differences():
    p, G = small_problem(n=16, blocks=(3, 2, 2))
    m = oracle.Model(p)
    rng = np.random.default_rng(14)
    gf = rng.normal(size=(3, 16, 16, 16))
    gU = rng.normal(size=G.shape)
    u = m.spread(p.x, rng.normal(size=G.shape))   # a smooth-ish field
    _, gx_s = m.spread_adj(p.x, G, gf)
    _, gx_i = m.interp_adj(p.x, u, gU)
    eps = 1e-6 * p.grid.h
    for _ in range(4):
        d = rng.normal(size=p.x.shape)
        fd_s = (np.sum(gf * m.spread(p.x + eps * d, G)) -
                np.sum(gf * m.spread(p.x - eps * d, G))) / (2 * eps)
        assert np.sum(gx_s * d) == pytest.approx(fd_s, rel=1e-6)
        fd_i = (np.sum(gU * m.interp(p.x + eps * d, u)) -
                np.sum(gU * m.interp(p.x - eps * d, u))) / (2 * eps)
        assert np.sum(gx_i * d) == pytest.approx(fd_i, rel=1e-6)


# ---------------------------------------------------------------------------
# nodal quadrature rule (Section 4.4): the coupling points are the nodes
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("centre", [None, (0.02, 0.97, 0.5)])
def test_nodal_spread_matches_brute_force_over_all_faces(centre):
    p, G = small_problem(centre=centre)
    m = oracle.Model(p)
    f = m.spread_nodal(p.x, G)
    n = p.grid.n[0]
    comp, idx = [], []
    for c in range(3):
        for i2 in range(n):
            for i1 in range(n):
                for i0 in range(n):
                    comp.append(c)
                    idx.append((i0, i1, i2))
    bf = m.spread_nodal_at(p.x, G, comp, idx).reshape(3, n, n, n)
    np.testing.assert_allclose(f, bf, rtol=1e-12, atol=1e-12 * np.abs(f).max())


def test_nodal_spread_conserves_force_and_torque():
    # zeroth and first moments of the 4-point kernel: h^3 sum f = sum_a G_a and
    # h^3 sum x_face x f = sum_a x_a x G_a
    p, G = small_problem(n=16, blocks=(2, 3, 2))
    m = oracle.Model(p)
    f = m.spread_nodal(p.x, G)
    h, n = p.grid.h, p.grid.n[0]
    np.testing.assert_allclose(h ** 3 * f.reshape(3, -1).sum(axis=1), G.sum(axis=1),
                               rtol=1e-12, atol=1e-12)
    ii = np.arange(n)
    pos = []
    for c in range(3):
        s = [0.5, 0.5, 0.5]
        s[c] = 0.0
        z, y, x = np.meshgrid((ii + s[2]) * h, (ii + s[1]) * h, (ii + s[0]) * h, indexing="ij")
        pos.append((x, y, z))
    torque = h ** 3 * np.array([
        np.sum(pos[2][1] * f[2]) - np.sum(pos[1][2] * f[1]),
        np.sum(pos[0][2] * f[0]) - np.sum(pos[2][0] * f[2]),
        np.sum(pos[1][0] * f[1]) - np.sum(pos[0][1] * f[0])])
    want = np.cross(p.x.T, G.T).sum(axis=0)
    np.testing.assert_allclose(torque, want, rtol=1e-11, atol=1e-13)


def test_nodal_interp_exact_on_constant_and_linear_fields():
    p, _ = small_problem(n=16, blocks=(3, 2, 2))
    m = oracle.Model(p)
    n, h = p.grid.n[0], p.grid.h
    const = np.array([0.3, -1.2, 2.5])
    u = np.broadcast_to(const[:, None, None, None], (3, n, n, n)).copy()
    np.testing.assert_allclose(m.interp_nodal(p.x, u),
                               np.broadcast_to(const[:, None], (3, p.n_nodes)), rtol=1e-13)
    A = np.random.default_rng(2).normal(size=(3, 3))
    b = np.array([0.1, 0.2, -0.3])
    ii = np.arange(n)
    for c in range(3):
        s = [0.5, 0.5, 0.5]
        s[c] = 0.0
        z, y, x = np.meshgrid((ii + s[2]) * h, (ii + s[1]) * h, (ii + s[0]) * h, indexing="ij")
        u[c] = A[c, 0] * x + A[c, 1] * y + A[c, 2] * z + b[c]
    np.testing.assert_allclose(m.interp_nodal(p.x, u), A @ p.x + b[:, None], rtol=1e-12,
                               atol=1e-12)


@pytest.mark.parametrize("centre", [None, (0.99, 0.5, 0.01)])
def test_nodal_spread_interp_adjoint_identity(centre):
    p, G = small_problem(n=16, blocks=(3, 3, 2), centre=centre)
    m = oracle.Model(p)
    u = np.random.default_rng(12).normal(size=(3, 16, 16, 16))
    lhs = p.grid.h ** 3 * np.sum(m.spread_nodal(p.x, G) * u)
    assert lhs == pytest.approx(np.sum(G * m.interp_nodal(p.x, u)), rel=1e-12)


def test_nodal_linear_and_position_adjoints():
    p, G = small_problem(n=16, blocks=(3, 2, 2))
    m = oracle.Model(p)
    rng = np.random.default_rng(15)
    gf = rng.normal(size=(3, 16, 16, 16))
    gU = rng.normal(size=G.shape)
    u = m.spread_nodal(p.x, rng.normal(size=G.shape))
    gG, gx_s = m.spread_nodal_adj(p.x, G, gf)
    gu, gx_i = m.interp_nodal_adj(p.x, u, gU)
    assert np.sum(gG * G) == pytest.approx(np.sum(gf * m.spread_nodal(p.x, G)), rel=1e-12)
    assert np.sum(gu * u) == pytest.approx(np.sum(gU * m.interp_nodal(p.x, u)), rel=1e-12)
    eps = 1e-6 * p.grid.h
    for _ in range(4):
        d = rng.normal(size=p.x.shape)
        fd_s = (np.sum(gf * m.spread_nodal(p.x + eps * d, G)) -
                np.sum(gf * m.spread_nodal(p.x - eps * d, G))) / (2 * eps)
        assert np.sum(gx_s * d) == pytest.approx(fd_s, rel=1e-6)
        fd_i = (np.sum(gU * m.interp_nodal(p.x + eps * d, u)) -
                np.sum(gU * m.interp_nodal(p.x - eps * d, u))) / (2 * eps)
        assert np.sum(gx_i * d) == pytest.approx(fd_i, rel=1e-6)


def test_loss_gradient_chain_by_differences():
    # the differentiation workload's loss on a small shell:
    # L = sum_a |U_a|^2 + sqrt(h^3 sum |f|^2), gradients in x and the 8 HO
    # parameters, against central differences on 20 seeded directions.
    p = I.shell_problem(seed=4000, n=32, dims=(12, 8, 2), u_modes=3, fp64=True)
    m = oracle.Model(p)
    h3 = p.grid.h ** 3

    def loss(x, th):
        m.set_materials([I.Material(I.HO, tuple(th))])
        G, _ = m.fe_force(x)
        f = m.spread(x, G)
        U = m.interp(x, p.u)
        return np.sum(U * U) + math.sqrt(h3 * np.sum(f * f))

    th0 = np.array(I.HO_DEFAULT)
    x0 = p.x
    m.set_materials([I.Material(I.HO, tuple(th0))])
    G, _ = m.fe_force(x0)
    f = m.spread(x0, G)
    U = m.interp(x0, p.u)
    nf = math.sqrt(h3 * np.sum(f * f))
    _, gx_i = m.interp_adj(x0, p.u, 2 * U)
    gG, gx_s = m.spread_adj(x0, G, h3 * f / nf)
    Hv, gth = m.fe_force_adj(x0, gG)
    gx = gx_i + gx_s + Hv
    rng = np.random.Generator(np.random.PCG64(4001))
    for _ in range(20):
        dx = rng.normal(size=x0.shape) * p.grid.h
        dth = rng.normal(size=9) * th0
        dth[8] = 0.0
        n = math.sqrt(np.sum((dx / p.grid.h) ** 2) + np.sum((dth / th0) ** 2))
        dx /= n
        dth /= n
        eps = 1e-6
        fd = (loss(x0 + eps * dx, th0 + eps * dth) - loss(x0 - eps * dx, th0 - eps * dth)) / (2 * eps)
        an = np.sum(gx * dx) + np.sum(gth[0, :9] * dth)
        assert an == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_material_table_conversions_golden():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "material_tables.txt"))
            if l.strip() and not l.startswith("#")]
    lv = {r[1]: float(r[4]) for r in rows if r[0] == "LV"}
    mv = {r[1]: float(r[4]) for r in rows if r[0] == "MV"}
    for r in rows:
        scale = {"dyn/cm2": 1e-4, "Pa": 1e-3, "-": 1.0}[r[3]]
        assert float(r[2]) * scale == pytest.approx(float(r[4]), rel=1e-12)
    # HO sheet/shear constants of the workloads are the LV table in kPa
    assert I.HO_DEFAULT[4] == pytest.approx(lv["as"], rel=1e-3)
    assert I.HO_DEFAULT[5] == pytest.approx(lv["bs"])
    assert I.HO_DEFAULT[6] == pytest.approx(lv["afs"], rel=1e-3)
    assert I.HO_DEFAULT[7] == pytest.approx(lv["bfs"])
    assert I.HO_DEFAULT[8] == pytest.approx(lv["kappa"])
    assert I.FIBRE1_LEAFLET[:3] == pytest.approx((mv["C1"], mv["af"], mv["bf"]))
    cm = {r[1]: float(r[2]) for r in rows if r[0] == "CM"}   # kept in dyn/cm^2
    assert I.STD_REINF_COOK == pytest.approx((cm["GT"], cm["GL"], cm["EL"], cm["kappa"]))
    av = {r[1]: float(r[4]) for r in rows if r[0] == "AV"}
    assert I.FIBRE2_AV[:4] == pytest.approx((av["C10"], av["C01"], av["af"], av["bf"]))


def test_workload_shapes_and_jacobians():
    p = I.shell_problem()
    assert (p.n_elems, p.n_nodes, p.n_gauss) == (14400, 17220, 115200)
    m = oracle.Model(p)
    w, J = m.gauss_info(p.x)
    assert (w > 0).all()
    assert J.min() > 0.9 and J.max() < 1.1
    b = I.block_problem()
    assert (b.n_elems, b.n_nodes, b.n_gauss) == (128, 243, 1024)


def test_differentiation_workload_oracle_gradient_by_differences():
    # The 128^3 ventricle shell: the oracle's adjoint gradient of
    # L = sum |U|^2 + sqrt(h^3 sum |f|^2) with respect to x and the 8 HO
    # parameters, against FP64 central differences (step 1e-6) along 20 seeded
    # directions normalised in (x/h, theta/theta0).
    p = I.shell_problem(fp64=True)
    m = oracle.Model(p)
    h3 = p.grid.h ** 3
    u = p.u.astype(np.float64)

    def loss(x, th):
        m.set_materials([I.Material(I.HO, tuple(th))])
        G, _ = m.fe_force(x)
        f = m.spread(x, G)
        U = m.interp(x, u)
        return np.sum(U * U) + math.sqrt(h3 * np.sum(f * f))

    th0 = np.array(I.HO_DEFAULT)
    x0 = p.x
    m.set_materials([I.Material(I.HO, tuple(th0))])
    G, _ = m.fe_force(x0)
    f = m.spread(x0, G)
    U = m.interp(x0, u)
    nf = math.sqrt(h3 * np.sum(f * f))
    _, gx_i = m.interp_adj(x0, u, 2 * U)
    gG, gx_s = m.spread_adj(x0, G, h3 * f / nf)
    Hv, gth = m.fe_force_adj(x0, gG)
    gx = gx_i + gx_s + Hv
    L0 = loss(x0, th0)
    rng = np.random.Generator(np.random.PCG64(4002))
    for _ in range(20):
        dx = rng.normal(size=x0.shape) * p.grid.h
        dth = rng.normal(size=9) * th0
        dth[8] = 0.0
        nrm = math.sqrt(np.sum((dx / p.grid.h) ** 2) + np.sum((dth[:8] / th0[:8]) ** 2))
        dx /= nrm
        dth /= nrm
        an = np.sum(gx * dx) + np.sum(gth[0, :9] * dth)
        # step 1e-6: the difference of two evaluations of L (~2.5e5) carries a
        # rounding error of order eps_mach |L|, i.e. eps_mach |L| / step in
        # the quotient; step 1e-5 leaves truncation below 1e-6 relative.
        for step, rel, absol in ((1e-6, 1e-6, np.finfo(float).eps * abs(L0) / 1e-6),
                                 (1e-5, 1e-5, 0.0)):
            fd = (loss(x0 + step * dx, th0 + step * dth) -
                  loss(x0 - step * dx, th0 - step * dth)) / (2 * step)
            assert an == pytest.approx(fd, rel=rel, abs=absol), step


# ---------------------------------------------------------------------------
# penalty tethers of the solid boundary (Section 5)
# ---------------------------------------------------------------------------

def _tethered(p):
    """The nodes of the block's x-minimum face (the 'fixed left face')."""
    return np.flatnonzero(p.X[0] <= p.X[0].min() + 1e-12)


def test_penalty_zero_at_reference_and_closed_form_translation():
    p = tiny_mesh(I.NEO_HOOKEAN, (0.5, 100.0))
    m = oracle.Model(p)
    nodes = _tethered(p)
    kappa = 1e6
    G, E = m.penalty(p.X, nodes, kappa)
    assert np.abs(G).max() == 0.0 and E == 0.0
    d = np.array([1e-3, -2e-3, 5e-4])[:, None]
    G, E = m.penalty(p.X + d, nodes, kappa)
    w = m.mass()[nodes]
    np.testing.assert_allclose(G[:, nodes], -kappa * w * d, rtol=1e-10)  # (X + d) - X rounds
    assert np.abs(np.delete(G, nodes, axis=1)).max() == 0.0
    assert E == pytest.approx(0.5 * kappa * w.sum() * float(np.sum(d * d)), rel=1e-10)
    # with the elastic force: a rigid translation strains nothing, so the
    # total force is the tethers' alone
    Ge, _ = m.fe_force(p.X + d)
    assert np.abs((Ge + G).sum(axis=1) + kappa * w.sum() * d[:, 0]).max() < 1e-9 * kappa * w.sum()


def test_penalty_force_is_minus_energy_gradient():
    p = tiny_mesh(I.NEO_HOOKEAN, (0.5, 100.0))
    m = oracle.Model(p)
    nodes = _tethered(p)
    rng = np.random.default_rng(31)
    w = rng.uniform(0.5, 2.0, size=len(nodes)) * p.grid.h ** 2
    G, _ = m.penalty(p.x, nodes, 5e6, weights=w)
    eps = 1e-6 * p.grid.h
    for _ in range(10):
        a, i = rng.choice(nodes), rng.integers(3)
        xp, xm = p.x.copy(), p.x.copy()
        xp[i, a] += eps
        xm[i, a] -= eps
        fd = -(m.penalty(xp, nodes, 5e6, w)[1] - m.penalty(xm, nodes, 5e6, w)[1]) / (2 * eps)
        assert G[i, a] == pytest.approx(fd, rel=1e-6)


# ---------------------------------------------------------------------------
# linear tetrahedra (P1) with the 4-point rule
# ---------------------------------------------------------------------------

def tiny_tets(model=I.HO, params=I.HO_DEFAULT, seed=7, blocks=(2, 2, 1)):
    return I.tet_problem(tiny_mesh(model, params, seed=seed, blocks=blocks))


def test_tet_rule_mass_and_volume():
    """The 4-point rule's weights sum to the element volume and each node's
    lumped mass is a quarter of its elements' volumes (P1 row sums)."""
    p = tiny_tets()
    m = oracle.Model(p)
    X = p.X
    w, _ = m.gauss_info(X)
    vol = np.zeros(p.n_elems)
    for e in range(p.n_elems):
        a, b, c, d = (X[:, p.conn[k, e]] for k in range(4))
        vol[e] = np.dot(np.cross(b - a, c - a), d - a) / 6.0
    assert (vol > 0).all()
    np.testing.assert_allclose(w.sum(axis=0), vol, rtol=1e-13)
    np.testing.assert_allclose(w, np.broadcast_to(vol / 4, w.shape), rtol=1e-13)
    mass = np.zeros(p.n_nodes)
    for k in range(4):
        np.add.at(mass, p.conn[k], vol / 4)
    np.testing.assert_allclose(m.mass(), mass, rtol=1e-13)
    # six tetrahedra fill each cube of the block exactly
    assert vol.sum() == pytest.approx(2 * 2 * 1 * p.grid.h ** 3, rel=1e-13)


@pytest.mark.parametrize("model,params", MODELS)
def test_tet_patch_test_and_energy_gradient(model, params):
    """P1 patch test: under an affine deformation every element has the same
    F, so interior nodes carry no force; G = -dE/dx by differences on a
    perturbed mesh; zero force at the reference and under rigid motion."""
    p = tiny_tets(model, params, blocks=(2, 2, 2))
    p.fibres = np.ascontiguousarray(np.repeat(p.fibres[:, :1], p.n_elems, axis=1))  # homogeneous
    m = oracle.Model(p)
    A = np.eye(3) + np.array([[0.05, 0.02, -0.01], [0.0, -0.03, 0.04], [0.01, 0.0, 0.02]])
    x = A @ (p.X - 0.5) + 0.5
    G, _ = m.fe_force(x)
    _, detF = m.gauss_info(x)
    np.testing.assert_allclose(detF, np.linalg.det(A), rtol=1e-12)
    X = p.X
    interior = np.flatnonzero(np.all([(X[d] > X[d].min() + 1e-12) & (X[d] < X[d].max() - 1e-12)
                                      for d in range(3)], axis=0))
    assert len(interior) > 0
    assert np.abs(G[:, interior]).max() < 1e-10 * np.abs(G).max()
    scale = params[-1] * p.grid.h ** 2
    G0, E0 = m.fe_force(X)
    assert np.abs(G0).max() < 1e-12 * scale and abs(E0) < 1e-15
    Q = rot(np.random.default_rng(6))
    G1, E1 = m.fe_force(Q @ (X - 0.5) + 0.5)
    assert np.abs(G1).max() < 1e-11 * scale and abs(E1) < 1e-15
    x = p.x
    G, _ = m.fe_force(x)
    eps = 1e-6 * p.grid.h
    rng = np.random.default_rng(12)
    for _ in range(8):
        a, i = rng.integers(p.n_nodes), rng.integers(3)
        xp, xm = x.copy(), x.copy()
        xp[i, a] += eps
        xm[i, a] -= eps
        fd = -(m.fe_force(xp)[1] - m.fe_force(xm)[1]) / (2 * eps)
        assert G[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-8 * np.abs(G).max())


def test_tet_adjoints_and_transfer_identities():
    """On the tetrahedral mesh: the force adjoint by differences, the spread
    against the brute-force sum over every face, force conservation, and the
    discrete adjointness of spreading and interpolation."""
    p = tiny_tets()
    m = oracle.Model(p)
    x = p.x
    rng = np.random.default_rng(13)
    v = rng.normal(size=x.shape)
    Hv, _ = m.fe_force_adj(x, v)
    eps = 1e-7 * p.grid.h
    fd = (m.fe_force(x + eps * v)[0] - m.fe_force(x - eps * v)[0]) / (2 * eps)
    np.testing.assert_allclose(Hv, fd, rtol=1e-5, atol=1e-6 * np.abs(Hv).max())
    G = rng.normal(size=x.shape)
    f = m.spread(x, G)
    n0, n1, n2 = p.grid.n
    comp = np.repeat(np.arange(3), n0 * n1 * n2).astype(np.int32)
    kk, jj, ii = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
    idx = np.tile(np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1), (3, 1))
    np.testing.assert_allclose(f.ravel(), m.spread_at(x, G, comp, idx), rtol=1e-12,
                               atol=1e-12 * np.abs(f).max())
    h3 = p.grid.h ** 3
    np.testing.assert_allclose(f.sum(axis=(1, 2, 3)) * h3, G.sum(axis=1), rtol=1e-12)
    u = rng.normal(size=(3, n2, n1, n0))
    U = m.interp(x, u)
    assert h3 * np.sum(f * u) == pytest.approx(np.sum(G * U), rel=1e-12)


# ---------------------------------------------------------------------------
# quadratic tetrahedra (P2) with the 4-point rule
# ---------------------------------------------------------------------------

def tiny_tet10(model=I.HO, params=I.HO_DEFAULT, seed=7, blocks=(2, 2, 1)):
    return I.tet10_problem(tiny_mesh(model, params, seed=seed, blocks=blocks))


_TA = (5 + 3 * np.sqrt(5)) / 20   # barycentric coordinates of the 4-point rule
_TB = (5 - np.sqrt(5)) / 20


def _rule_points_ref(p):
    """Reference positions of the rule points, from the vertices alone (the
    reference elements are straight-sided): X_q = a X_q + b sum_{i != q} X_i."""
    V = [p.X[:, p.conn[i]].astype(np.float64) for i in range(4)]
    return np.stack([_TB * sum(V) + (_TA - _TB) * V[q] for q in range(4)])  # [4][3][E]


def _quad_map(X):
    """A smooth quadratic deformation and its gradient, in closed form."""
    c = X - 0.5
    x = np.stack([c[0] + 0.3 * c[0] * c[1] + 0.2 * c[2] ** 2,
                  c[1] - 0.25 * c[0] ** 2 + 0.1 * c[1] * c[2],
                  c[2] + 0.15 * c[0] * c[2] - 0.2 * c[1] ** 2]) + 0.5
    F = np.zeros((3, 3) + X.shape[1:])
    F[0, 0], F[0, 1], F[0, 2] = 1 + 0.3 * c[1], 0.3 * c[0], 0.4 * c[2]
    F[1, 0], F[1, 1], F[1, 2] = -0.5 * c[0], 1 + 0.1 * c[2], 0.1 * c[1]
    F[2, 0], F[2, 1], F[2, 2] = 0.15 * c[2], -0.4 * c[1], 1 + 0.15 * c[0]
    return x, F


def test_tet10_quadratic_fields_are_reproduced():
    """P2 reproduces quadratic maps exactly: under x = phi(X) quadratic, det F
    at every rule point equals det grad phi there, and interpolating the
    coordinate field (the 4-point kernel reproduces linear functions) gives
    back the rule points phi(X_q): this pins the ten shape functions, their
    gradients and the rule's points (each from its closed form)."""
    p = tiny_tet10(blocks=(2, 2, 2))
    m = oracle.Model(p)
    x, _ = _quad_map(p.X)
    _, detF = m.gauss_info(x)
    Xq = _rule_points_ref(p)                         # [4][3][E]
    for q in range(4):
        _, Fq = _quad_map(Xq[q])
        np.testing.assert_allclose(detF[q], np.linalg.det(np.moveaxis(Fq, -1, 0)), rtol=1e-12)
    # coordinate field on the faces: u^c(face) = its c coordinate (no wrap
    # near the structure, which sits in the middle of the box)
    n0, n1, n2 = p.grid.n
    h = p.grid.h
    u = np.zeros((3, n2, n1, n0))
    u[0] += (np.arange(n0) * h)[None, None, :]
    u[1] += (np.arange(n1) * h)[None, :, None]
    u[2] += (np.arange(n2) * h)[:, None, None]
    _, Uq = m.interp(x, u, want_gauss=True)
    for q in range(4):
        chi, _ = _quad_map(Xq[q])
        # faces of component c sit at i h in direction c (no staggering there)
        np.testing.assert_allclose(Uq[:, q], chi, rtol=0, atol=1e-12)


def test_tet10_mass_is_the_scaled_diagonal():
    """Lumped P2 mass (diagonal scaling of Hinton, Rock and Zienkiewicz):
    positive, the element masses sum to the volume, and on a straight-sided
    element vertex : edge masses are the rule's sums of N^2, in closed form
    from the rule's barycentric coordinates: N_vertex = +-1/10 at the four
    points, N_edge = (1 + sqrt 5)/10 at two and (3 - sqrt 5)/10 at two."""
    p = tiny_tet10()
    m = oracle.Model(p)
    M = m.mass()
    assert (M > 0).all()
    assert M.sum() == pytest.approx(2 * 2 * 1 * p.grid.h ** 3, rel=1e-13)
    sv = 4 * 0.01
    se = 2 * ((1 + np.sqrt(5)) / 10) ** 2 + 2 * ((3 - np.sqrt(5)) / 10) ** 2
    one = dataclasses.replace(p, conn=np.ascontiguousarray(p.conn[:, :1]))
    M1 = oracle.Model(one).mass()
    V = np.dot(np.cross(*(p.X[:, p.conn[k, 0]] - p.X[:, p.conn[0, 0]] for k in (1, 2))),
               p.X[:, p.conn[3, 0]] - p.X[:, p.conn[0, 0]]) / 6
    np.testing.assert_allclose(M1[p.conn[:4, 0]], V * 0.01 / (sv + 6 * se / 4), rtol=1e-12)
    np.testing.assert_allclose(M1[p.conn[4:, 0]], V * (se / 4) / (sv + 6 * se / 4), rtol=1e-12)


@pytest.mark.parametrize("model,params", MODELS)
def test_tet10_patch_test_and_energy_gradient(model, params):
    """P2 patch test (interior nodes free of force under an affine
    deformation), G = -dE/dx by differences, zero force at the reference and
    under rigid motion."""
    p = tiny_tet10(model, params, blocks=(2, 2, 2))
    p.fibres = np.ascontiguousarray(np.repeat(p.fibres[:, :1], p.n_elems, axis=1))
    m = oracle.Model(p)
    A = np.eye(3) + np.array([[0.05, 0.02, -0.01], [0.0, -0.03, 0.04], [0.01, 0.0, 0.02]])
    G, _ = m.fe_force(A @ (p.X - 0.5) + 0.5)
    X = p.X
    interior = np.flatnonzero(np.all([(X[d] > X[d].min() + 1e-12) & (X[d] < X[d].max() - 1e-12)
                                      for d in range(3)], axis=0))
    assert len(interior) > 8
    assert np.abs(G[:, interior]).max() < 1e-10 * np.abs(G).max()
    scale = params[-1] * p.grid.h ** 2
    G0, E0 = m.fe_force(X)
    assert np.abs(G0).max() < 1e-12 * scale and abs(E0) < 1e-15
    Q = rot(np.random.default_rng(6))
    G1, E1 = m.fe_force(Q @ (X - 0.5) + 0.5)
    assert np.abs(G1).max() < 1e-11 * scale and abs(E1) < 1e-15
    x = p.x
    G, _ = m.fe_force(x)
    eps = 1e-6 * p.grid.h
    rng = np.random.default_rng(12)
    for _ in range(8):
        a, i = rng.integers(p.n_nodes), rng.integers(3)
        xp, xm = x.copy(), x.copy()
        xp[i, a] += eps
        xm[i, a] -= eps
        fd = -(m.fe_force(xp)[1] - m.fe_force(xm)[1]) / (2 * eps)
        assert G[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-8 * np.abs(G).max())


def test_tet10_adjoints_and_transfer_identities():
    """On the P2 mesh: the force adjoint by differences, the spread against
    the brute-force sum over every face, the discrete adjointness of spreading
    and interpolation, and a uniform force density (nodal forces g m_a) spread
    to a field whose total is g times the structure's volume (the shape
    functions sum to one at every rule point)."""
    p = tiny_tet10()
    m = oracle.Model(p)
    x = p.x
    rng = np.random.default_rng(13)
    v = rng.normal(size=x.shape)
    Hv, _ = m.fe_force_adj(x, v)
    eps = 1e-7 * p.grid.h
    fd = (m.fe_force(x + eps * v)[0] - m.fe_force(x - eps * v)[0]) / (2 * eps)
    np.testing.assert_allclose(Hv, fd, rtol=1e-5, atol=1e-6 * np.abs(Hv).max())
    G = rng.normal(size=x.shape)
    f = m.spread(x, G)
    n0, n1, n2 = p.grid.n
    comp = np.repeat(np.arange(3), n0 * n1 * n2).astype(np.int32)
    kk, jj, ii = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
    idx = np.tile(np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1), (3, 1))
    np.testing.assert_allclose(f.ravel(), m.spread_at(x, G, comp, idx), rtol=1e-12,
                               atol=1e-12 * np.abs(f).max())
    h3 = p.grid.h ** 3
    u = rng.normal(size=(3, n2, n1, n0))
    U = m.interp(x, u)
    assert h3 * np.sum(f * u) == pytest.approx(np.sum(G * U), rel=1e-12)
    g = np.array([0.3, -1.2, 0.7])
    fu = m.spread(x, g[:, None] * m.mass()[None, :])
    w, _ = m.gauss_info(x)
    np.testing.assert_allclose(fu.sum(axis=(1, 2, 3)) * h3, g * w.sum(), rtol=1e-12)


def test_tet10_mesh_construction():
    """The P2 generator shares one node per edge: on an nx x ny x nz block
    split into six tetrahedra per cube (all around the 0-6 diagonal) the
    distinct edges are the lattice edges, one face diagonal per face and one
    body diagonal per cube; every edge node sits at its edge's middle in the
    reference configuration and the quadratic mesh covers the same volume."""
    nx, ny, nz = 3, 2, 2
    p = tiny_mesh(blocks=(nx, ny, nz))
    q = I.tet10_problem(p)
    nv = (nx + 1) * (ny + 1) * (nz + 1)
    lattice = nx * (ny + 1) * (nz + 1) + (nx + 1) * ny * (nz + 1) + (nx + 1) * (ny + 1) * nz
    faces = nx * ny * (nz + 1) + nx * (ny + 1) * nz + (nx + 1) * ny * nz
    cubes = nx * ny * nz
    assert q.n_nodes == nv + lattice + faces + cubes
    assert q.conn.shape == (10, 6 * cubes)
    for k, (i, j) in enumerate(I.TET10_EDGES):
        np.testing.assert_allclose(q.X[:, q.conn[4 + k]],
                                   0.5 * (q.X[:, q.conn[i]] + q.X[:, q.conn[j]]), rtol=0, atol=1e-15)
    w, _ = oracle.Model(q).gauss_info(q.X)
    assert w.sum() == pytest.approx(cubes * p.grid.h ** 3, rel=1e-13)
