"""The allocation-free OC update (tp_oc_update_noalloc) gives the same result as
the regular tp_oc_update, and both match the oracle's exact multiplier and
update (Eq. "update": lambda is the root of sum rho_new(lambda) = volfrac n_el).

tp_oc_update_noalloc is for callers that cannot allocate device memory when they
update the design (their framework's allocator owns the memory budget, or their
host forbids allocations after start-up, or the loop must not pay for
cudaMalloc / cudaFree).  Its scratch is one static device array shared by every
call, so this test calls it twice in a row, on different inputs, and compares
each call through the C-ABI with the regular entry point on the same inputs,
using the tolerances of the OC parity tests (lambda rel 1e-9, densities
max-abs 1e-6); each call is also compared with the oracle's exact piecewise
root for lambda and its update at that root.  This file is named so that
pytest collects it last.
"""
import numpy as np
import pytest

import workloads as W
from oracle import oc

pytestmark = pytest.mark.gpu


def _regular(topo, n, rho, dcf, vf, passive):
    prob = W.small2d(n, 1, volfrac=vf)
    if passive is not None:
        prob.passive = passive
    p = topo.Problem.from_workload(prob)
    p.set_density(rho)
    p.set(topo.TP_DCF, dcf)
    lam, vol, ch = p.oc_update()
    out = p.get(topo.TP_RHO)
    p.close()
    return out, lam, vol, ch


def test_noalloc_matches_regular_on_two_calls():
    import torch
    from paper_2012_08208_gb300 import topo

    assert torch.cuda.is_available()
    dev = torch.device("cuda", 0)
    cases = [(50000, 0.4, 11, False), (120000, 0.3, 12, True)]
    for n, vf, seed, with_passive in cases:
        rng = np.random.default_rng(seed)
        rho = rng.uniform(0.001, 1.0, n)
        dcf = W.random_sensitivity(n, seed=seed + 100)
        passive = None
        if with_passive:
            passive = (rng.uniform(size=n) < 0.1).astype(np.int8)
            rho[passive == 1] = 0.001
        ref, lam_r, vol_r, ch_r = _regular(topo, n, rho, dcf, vf, passive)
        rho_d = torch.from_numpy(rho).to(dev)
        dcf_d = torch.from_numpy(dcf).to(dev)
        out_d = torch.empty_like(rho_d)
        pas_d = torch.from_numpy(passive).to(dev) if passive is not None else None
        lam, vol, ch = topo.oc_update_noalloc(rho_d, dcf_d, out_d, vf, passive=pas_d)
        torch.cuda.synchronize()
        out = out_d.cpu().numpy()
        assert lam == pytest.approx(lam_r, rel=1e-9)
        assert np.max(np.abs(out - ref)) <= 1e-6
        assert vol == pytest.approx(vol_r, rel=1e-12)
        assert ch == pytest.approx(ch_r, rel=1e-12, abs=1e-15)
        if passive is not None:
            assert np.all(out[passive == 1] == 0.001)
        # against the oracle: exact root of the volume constraint, update there
        lam_exact = oc.exact_lambda(rho, dcf, vf, passive=passive)
        assert lam == pytest.approx(lam_exact, rel=1e-9)
        assert np.max(np.abs(out - oc.update(rho, dcf, lam_exact, passive=passive))) <= 1e-6
        assert vol == pytest.approx(vf * n, rel=1e-8)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2012_08208_gb300 import topo

    dev = torch.device("cuda", 0)
    n = topo.NOALLOC_MAX_ELEMENTS + 1
    rho = torch.full((n,), 0.5, dtype=torch.float64, device=dev)
    dcf = torch.full((n,), -1.0, dtype=torch.float64, device=dev)
    out = torch.empty_like(rho)
    with pytest.raises(topo.TopoError) as e:
        topo.oc_update_noalloc(rho, dcf, out, 0.5)
    assert e.value.status == topo.TP_ERR_ARG
