"""CPU pins of the test helpers that select what the GPU parity tests compare."""
import numpy as np

from paper_2503_22695_gb300 import inputs as I

from helpers import hex_fibre_stretch, kink_nodes


def test_fibre_stretch_under_uniform_stretch():
    # x = lam X: F = lam I at every Gauss point, so I4 - 1 = lam^2 |e|^2 - 1
    p = I.shell_problem()
    lam = 1.1
    d4f, d4s = hex_fibre_stretch(p, lam * p.X.astype(np.float64))
    nf = (p.fibres[0:3].astype(np.float64) ** 2).sum(axis=0)
    ns = (p.fibres[3:6].astype(np.float64) ** 2).sum(axis=0)
    assert np.allclose(d4f, lam ** 2 * nf - 1, rtol=0, atol=1e-12)
    assert np.allclose(d4s, lam ** 2 * ns - 1, rtol=0, atol=1e-12)


def test_kink_nodes_selects_the_elements_at_the_kink():
    # undeformed: every stretch is |e|^2 - 1 (FP32 fibres: within 1e-7 of 0),
    # so every node is near the kink; stretched by 1 %: none is
    p = I.shell_problem()
    X = p.X.astype(np.float64)
    assert len(kink_nodes(p, X)) == p.n_nodes
    assert len(kink_nodes(p, 1.01 * X)) == 0
