"""ib_forward and ib_backward captured in a CUDA graph.

The caller's stream is captured; the library's own side streams join the
capture through its fork and join events.  A replay of the graph gives the
outputs of direct calls bit for bit: FP32 split positions on the 128^3
ventricle shell (Gauss and nodal rules) and an FP64 block plan."""
import numpy as np
import pytest

from paper_2503_22695_gb300 import inputs as I

from helpers import Case

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("make,quad", [(I.shell_problem, 0), (I.shell_problem, 1),
                                       (I.block_problem, 0)])
def test_forward_backward_graph_replay_is_bitwise(make, quad):
    import torch
    c = Case(make(), quad=quad)
    ibfe = c.ibfe
    dev, dt, N = "cuda", c.dt, c.prob.n_nodes
    shape = tuple(c.plan.grid_shape())
    G = torch.empty((3, N), device=dev, dtype=dt)
    f = torch.empty(shape, device=dev, dtype=dt)
    U = torch.empty((3, N), device=dev, dtype=dt)
    gx = torch.empty((3, N), device=dev, dtype=dt)
    gu = torch.empty(shape, device=dev, dtype=dt)
    rng = np.random.default_rng(11)
    gU = torch.from_numpy(rng.normal(size=(3, N))).to(dev, dt)
    gf = torch.from_numpy(rng.normal(size=shape) * 1e-3).to(dev, dt)
    gG = torch.from_numpy(rng.normal(size=(3, N))).to(dev, dt)

    def run():
        ibfe.ib_forward(c.plan, c.mats, c.pos, c.u, G, f, U)
        return ibfe.ib_backward(c.plan, c.mats, c.pos, c.u, G, gG, gf, gU, gx=gx, gu=gu)[2]

    gp_ref = run()
    torch.cuda.synchronize()
    ref = [t.clone() for t in (G, f, U, gx, gu, gp_ref)]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        run()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        gp = run()
    for t in (G, f, U, gx, gu, gp):
        t.fill_(float("nan"))
    graph.replay()
    torch.cuda.synchronize()
    for name, a, b in zip(("G", "f", "U", "gx", "gu", "gparams"), (G, f, U, gx, gu, gp), ref):
        assert torch.equal(a, b), name
