"""Failure detection without a GPU fault, and order independence.

* The bounded wait that guards every TMA box gives up and reports
  IB_ERR_TIMEOUT when a transaction never arrives (a diagnostic kernel arms
  an mbarrier for bytes no copy delivers); the context stays usable.
* Spreading in FP32 plans sums exact integers, so the force field does not
  depend on the order of the elements: a mesh whose elements are permuted
  gives a bitwise-equal f for the same nodal forces.
"""
import dataclasses
import time

import numpy as np
import pytest

from paper_2503_22695_gb300 import inputs as I

from helpers import Case, np_, rel_l2

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    import torch
    from paper_2503_22695_gb300 import ibfe
    t0 = time.time()
    assert ibfe.ib_diag_wait_timeout(20.0) == ibfe.IB_ERR_TIMEOUT
    assert time.time() - t0 < 5.0
    with pytest.raises(ibfe.IBError):
        ibfe._chk(ibfe._lib.ib_diag_wait_timeout(-1.0, None), "ib_diag_wait_timeout")
    # the context is intact: a forward still matches the oracle
    c = Case(I.block_problem(fp64=False))
    G, f, U = ibfe.ib_forward(c.plan, c.mats, c.pos, c.u)
    torch.cuda.synchronize()
    assert rel_l2(np_(G), c.orc.fe_force(c.x_np)[0]) <= 1e-5
    assert ibfe.ib_plan_sync_status(c.plan) == ibfe.IB_OK


@pytest.mark.parametrize("name", ["block32", "shell128"])
def test_element_order_does_not_change_the_field(name):
    import torch
    from paper_2503_22695_gb300 import ibfe
    p = I.block_problem(fp64=False) if name == "block32" else I.shell_problem()
    c = Case(p)
    G = c.to_dev(c.rounded(np.random.default_rng(17).normal(size=(3, p.n_nodes))))
    f0 = np_(ibfe.ib_spread(c.plan, c.pos, G))
    perm = np.random.default_rng(18).permutation(p.n_elems)
    q = dataclasses.replace(p, conn=np.ascontiguousarray(p.conn[:, perm]),
                            fibres=np.ascontiguousarray(p.fibres[:, perm]),
                            mat_id=np.ascontiguousarray(p.mat_id[perm]))
    c2 = Case(q)
    f1 = np_(ibfe.ib_spread(c2.plan, c2.pos, G))
    assert np.array_equal(f0, f1)
    # nodal sums follow each mesh's incidence order: equal up to rounding
    G0, _ = ibfe.ib_fe_force(c.plan, c.mats, c.pos, energy=True)
    G1, _ = ibfe.ib_fe_force(c2.plan, c2.mats, c2.pos, energy=True)
    assert rel_l2(np_(G1), np_(G0)) <= 1e-6
    torch.cuda.synchronize()
