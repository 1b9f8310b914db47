"""Batched SIMP iterations of independent uneven 2D problems (one persistent CG
launch for all instances, graph-captured step) against the oracle, instance by
instance, on identical densities: compliance rel <= 1e-8, densities max-abs
<= 1e-6, lambda within 1e-9 of the exact root."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import filt, oc, simp

pytestmark = pytest.mark.gpu


def _small_batch():
    b = W.batch2d(6, seed=7, w_range=(8, 60))
    for w in b:
        w.tol = 1e-10
    return b


def test_batch_steps_match_oracle_per_instance(tmp_path):
    from paper_2012_08208_gb300 import topo
    ws = _small_batch()
    B = topo.Batch(ws)
    ty, cps = B.autotune(str(tmp_path / "tiles.json"))
    assert ty in (4, 8, 16) and 1 <= cps <= 8
    cache = json.load(open(tmp_path / "tiles.json"))
    assert len(cache) == 1 and list(cache.values())[0]["tile_rows"] == ty
    opts = topo.solve_opts(tol=1e-10, max_it=100000, precision=topo.TP_PREC_MIXED, update_drop=0.1)
    Wm = [filt.weights_for(w) for w in ws]
    rho = [w.initial_density() for w in ws]
    for step in range(3):
        info, comp = B.step(opts)
        assert info.converged == 1
        if step > 0:
            assert info.graph == 1
        for i, w in enumerate(ws):
            ref = simp.iteration(w, rho[i], W=Wm[i])
            assert abs(comp[i] - ref["c"]) <= 1e-8 * abs(ref["c"])
            rho_gpu, sc = B.get(i, topo.TP_RHO)
            lam_exact = oc.exact_lambda(rho[i], ref["dcf"], w.volfrac)
            assert sc[1] == pytest.approx(lam_exact, rel=1e-9)
            assert np.max(np.abs(rho_gpu - ref["rho_new"])) <= 1e-6
            assert sc[5] <= 1.2e-10
            rho[i] = rho_gpu
    B.close()


def test_batch_tile_shapes_give_the_same_answer():
    from paper_2012_08208_gb300 import topo
    ws = _small_batch()[:3]
    opts = topo.solve_opts(tol=1e-10, max_it=100000, precision=topo.TP_PREC_MIXED, update_drop=0.1)
    out = []
    for ty, cps in ((4, 1), (16, 4)):
        B = topo.Batch(ws)
        B.set_tiles(ty, cps)
        info, comp = B.step(opts)
        out.append(comp)
        B.close()
    assert np.allclose(out[0], out[1], rtol=1e-8)
