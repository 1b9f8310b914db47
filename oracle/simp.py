"""The SIMP loop of the paper's main program (Section 4; loop of Section 4.4):
FE solve -> objective and sensitivities -> filter -> OC bisection -> change.

The paper loops while change > 0.01 and loop < 2000; the workloads fix the
number of iterations instead (change is still reported).  One iteration here is
the reference for one GPU SIMP iteration on identical densities.
"""
from __future__ import annotations

import numpy as np

from . import fem, filt, helm, oc, sens


def iteration(prob, rho, W=None, solve_method="lu", rtol=1e-13, filter_mode=0, K0cache=None):
    """One SIMP iteration from density rho.  Returns a dict with u, c, dc, dcf,
    rho_new, lam, vol, change."""
    W = filt.weights_for(prob) if W is None else W
    passive = prob.passive
    AT = helm.operator(prob) if filter_mode == 2 else None
    if filter_mode == 0:
        rho_phys = rho
    elif filter_mode == 1:
        rho_phys = filt.density_filter(W, rho)
    else:  # the Helmholtz (PDE) filter of the paper's parallel runs
        rho_phys = helm.apply(prob, rho, AT=AT)
    K = fem.assemble(prob, rho_phys)
    U = fem.solve(prob, rho_phys, method=solve_method, rtol=rtol, K=K)
    c, ce, dc = sens.sensitivities(prob, rho_phys, U)
    if filter_mode == 0:
        dcf = filt.sensitivity_filter(W, rho, dc)
    elif filter_mode == 1:
        dcf = filt.density_filter_chain(W, dc)
    else:  # H is symmetric: d c / d rho = H (d c / d rho~)
        dcf = helm.apply(prob, dc, AT=AT)
    rho_new, lam, vol, change, nb = oc.bisect(rho, dcf, prob.volfrac, prob.move, prob.dmin, passive)
    return dict(u=U, c=c, ce=ce, dc=dc, dcf=dcf, rho_new=rho_new, lam=lam, vol=vol,
                change=change, n_bisect=nb)


def run(prob, n_iter=None, rho0=None, solve_method="lu", rtol=1e-13, callback=None, filter_mode=0):
    """Fixed-count SIMP loop; returns (rho, history list of per-iteration dicts
    without the large arrays)."""
    n_iter = prob.n_iter if n_iter is None else n_iter
    rho = prob.initial_density() if rho0 is None else rho0.copy()
    W = filt.weights_for(prob)
    hist = []
    for it in range(n_iter):
        out = iteration(prob, rho, W=W, solve_method=solve_method, rtol=rtol, filter_mode=filter_mode)
        hist.append(dict(it=it, c=out["c"], lam=out["lam"], vol=out["vol"], change=out["change"]))
        if callback is not None:
            callback(it, rho, out)
        rho = out["rho_new"]
    return rho, hist
