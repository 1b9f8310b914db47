"""Failure detection on the GPU without a fault: a bounded device-side wait that
runs out returns an error status, and the handle stays usable.

Every grid-wide barrier of the persistent kernels gives up after a cycle budget
(about 1 s by default), records the timeout in the barrier word and returns.
tp_set_wait_budget shrinks that budget for one problem: with a budget of one
cycle the first CTA to reach a barrier gives up before the others arrive, so
the solve ends with TP_ERR_TIMEOUT.  No kernel hangs, traps or faults.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fem, sens

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def topo():
    from paper_2012_08208_gb300 import topo as t
    return t


def test_barrier_timeout_returns_status_and_handle_recovers(topo):
    prob = W.small2d(70, 20, n_cases=2)
    p = topo.Problem.from_workload(prob)
    opts = topo.solve_opts(tol=1e-10, max_it=50000, precision=topo.TP_PREC_F64)
    p.set_wait_budget(1)
    info = p.solve(opts, check=False)
    assert info.status == topo.TP_ERR_TIMEOUT
    assert "timed out" in p.last_error()
    with pytest.raises(topo.TopoError) as e:
        p.solve(opts)
    assert e.value.status == topo.TP_ERR_TIMEOUT
    # the same handle, default budget: a normal solve that matches the oracle
    p.set_wait_budget(0)
    info = p.solve(opts)
    assert info.converged == 1
    U_ref = fem.solve(prob, prob.initial_density())
    c_ref = sens.compliance(prob, U_ref)
    assert p.sensitivities() == pytest.approx(c_ref, rel=1e-8)
    # the OC kernel's barriers take the same budget
    p.filter()
    p.set_wait_budget(1)
    with pytest.raises(topo.TopoError) as e:
        p.oc_update()
    assert e.value.status == topo.TP_ERR_TIMEOUT
    p.set_wait_budget(0)
    lam, vol, ch = p.oc_update()
    assert vol == pytest.approx(prob.volfrac * prob.n_el, rel=1e-8)
    p.close()


def test_wait_budget_rejects_out_of_range(topo):
    p = topo.Problem.from_workload(W.small2d(4, 2))
    for bad in (-1, 5_000_000_000):
        with pytest.raises(topo.TopoError) as e:
            p.set_wait_budget(bad)
        assert e.value.status == topo.TP_ERR_ARG
    p.close()
