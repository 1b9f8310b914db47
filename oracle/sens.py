"""Compliance and element sensitivities (Section 3.2, sensitivity d f/d d = -p d^(p-1) U;
Section 4.4 objective/sensitivity projection; Section 5.3 sums over load cases).

With modified SIMP E_e = Emin + rho_e^p (E0 - Emin) and element energy
ce_e = u_e^T K0 u_e (K0 for unit modulus), the compliance of case k is
c_k = f_k^T u_k = sum_e E_e ce_{e,k}, and
dc_e = d c / d rho_e = -p rho_e^(p-1) (E0 - Emin) sum_k ce_{e,k}.
The paper's DG0 projection of d^p psi is the same element energy up to a
constant factor (the element volume and the factor 2 between u^T K u and
the integral of psi), which does not change the OC result.
"""
from __future__ import annotations

import numpy as np

from . import fem


def element_energy(prob, U):
    """ce_e = sum over cases of u_e^T K0 u_e, shape [n_el]."""
    K0 = fem.k0_for(prob)
    edofs = fem.edofs_for(prob)
    ce = np.zeros(edofs.shape[0])
    for c in range(U.shape[0]):
        ue = U[c][edofs]
        ce += np.einsum("ei,ij,ej->e", ue, K0, ue)
    return ce


def compliance(prob, U):
    """c = sum_k f_k^T u_k."""
    return float(sum(prob.loads[c] @ U[c] for c in range(U.shape[0])))


def sensitivities(prob, rho, U):
    """Returns (c, ce, dc): total compliance, summed element energies and
    dc_e = -p rho^(p-1) (E0 - Emin) ce_e."""
    ce = element_energy(prob, U)
    dc = -prob.penal * np.power(rho, prob.penal - 1.0) * (prob.E0 - prob.Emin) * ce
    return compliance(prob, U), ce, dc
