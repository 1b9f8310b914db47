"""Finite-element analysis for the oracle: modified-SIMP stiffness, assembly, solve.

Stiffness interpolation: the paper penalises the density as d^p (Eq. "simp_fn",
Eq. "simp"; form K = inner(density**penal*sigma(u), grad(v)) in Section 4.3).
We use the modified SIMP reading E_e = Emin + rho_e^p (E0 - Emin) (Emin = 1e-9)
so that K stays non-singular in void regions.

Discrete system (Section 3.1, Eq. "fe_form"): K(rho) = sum_e E_e P_e^T K0 P_e.
Dirichlet DOFs are eliminated: K_ff u_f = f_f, u = 0 on fixed DOFs.
The paper solves with PETSc's default sparse LU (Section 4.3); the oracle uses
SciPy's SuperLU, and SciPy's own CG (Jacobi-preconditioned) only where a direct
factorisation does not fit.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import element, mesh


def young(rho, E0=1.0, Emin=1e-9, penal=3.0):
    """E_e = Emin + rho^p (E0 - Emin)."""
    return Emin + np.power(rho, penal) * (E0 - Emin)


def k0_for(prob):
    return element.k0_q4(1.0, prob.nu) if prob.dim == 2 else element.k0_h8(1.0, prob.nu)


def edofs_for(prob):
    return mesh.element_dofs(prob.dim, prob.nelx, prob.nely, prob.nelz)


def assemble(prob, rho, K0=None, edofs=None):
    """Global K(rho) as CSR (no boundary conditions applied)."""
    K0 = k0_for(prob) if K0 is None else K0
    edofs = edofs_for(prob) if edofs is None else edofs
    E = young(rho, prob.E0, prob.Emin, prob.penal)
    nd = edofs.shape[1]
    rows = np.repeat(edofs, nd, axis=1).ravel()
    cols = np.tile(edofs, (1, nd)).ravel()
    vals = (E[:, None, None] * K0[None, :, :]).reshape(len(E), -1).ravel()
    K = sp.coo_matrix((vals, (rows, cols)), shape=(prob.n_dof, prob.n_dof)).tocsr()
    K.sum_duplicates()
    return K


def matvec_bc(prob, rho, u, K=None):
    """Operator with Dirichlet rows replaced by identity: y_free = (K u_masked)_free,
    y_fixed = u_fixed, where u_masked has its fixed entries set to zero."""
    K = assemble(prob, rho) if K is None else K
    fixed = prob.fixed.astype(bool)
    um = np.where(fixed, 0.0, u)
    y = K @ um
    return np.where(fixed, u, y)


def matvec_elementwise(prob, rho, u):
    """Matrix-free reference product y = sum_e E_e P_e^T K0 P_e u (no BCs);
    a second, assembly-free statement of the same sum."""
    K0 = k0_for(prob)
    edofs = edofs_for(prob)
    E = young(rho, prob.E0, prob.Emin, prob.penal)
    ue = u[edofs]  # [n_el, nd]
    fe = (ue @ K0.T) * E[:, None]
    return np.bincount(edofs.ravel(), weights=fe.ravel(), minlength=prob.n_dof)


def matvec_rows(prob, rho, u, dofs, absolute=False):
    """Rows `dofs` of the boundary-conditioned operator, evaluated one by one from
    the element sum (for sampled checks at sizes the assembled matrix cannot
    reach).  Returns y[dofs] exactly as matvec_bc would.  With absolute=True
    the same rows of |K| |u| (the scale of the rounding error of the sum)."""
    K0 = k0_for(prob)
    if absolute:
        K0 = np.abs(K0)
        u = np.abs(u)
    dim = prob.dim
    nx, ny, nz = prob.nelx, prob.nely, prob.nelz
    fixed = prob.fixed.astype(bool)
    corners = element.Q4_NODES if dim == 2 else element.H8_NODES
    out = np.zeros(len(dofs))
    for t, g in enumerate(dofs):
        g = int(g)
        if fixed[g]:
            out[t] = u[g]
            continue
        node, comp = divmod(g, dim)
        i = node % (nx + 1)
        j = (node // (nx + 1)) % (ny + 1)
        k = node // ((nx + 1) * (ny + 1)) if dim == 3 else 0
        acc = 0.0
        for c, off in enumerate(corners):
            ei, ej = i - off[0], j - off[1]
            ek = k - off[2] if dim == 3 else 0
            if ei < 0 or ej < 0 or ei >= nx or ej >= ny:
                continue
            if dim == 3 and (ek < 0 or ek >= nz):
                continue
            e = ei + nx * (ej + ny * ek)
            Ee = prob.Emin + rho[e] ** prob.penal * (prob.E0 - prob.Emin)
            row = dim * c + comp
            for m, offm in enumerate(corners):
                ni, nj = ei + offm[0], ej + offm[1]
                nk = ek + offm[2] if dim == 3 else 0
                nm = ni + (nx + 1) * (nj + (ny + 1) * nk)
                for s in range(dim):
                    dm = dim * nm + s
                    if fixed[dm]:
                        continue
                    acc += Ee * K0[row, dim * m + s] * u[dm]
        out[t] = acc
    return out


def solve(prob, rho, method="lu", rtol=1e-13, maxiter=200000, K=None, x0=None, callback=None):
    """Displacements u[n_cases, n_dof] of K(rho) u_k = f_k with u = 0 on fixed DOFs.
    method 'lu': SuperLU factorisation of K_ff, shared by all load cases.
    method 'cg': SciPy's Jacobi-preconditioned CG on K_ff to relative residual rtol;
    `callback` (optional) is handed to SciPy's CG, which calls it once per
    iteration (e.g. to count iterations)."""
    K = assemble(prob, rho) if K is None else K
    free = np.flatnonzero(prob.fixed == 0)
    Kff = K[free][:, free].tocsc()
    U = np.zeros((prob.n_cases, prob.n_dof))
    if method == "lu":
        lu = spla.splu(Kff, permc_spec="COLAMD")
        for c in range(prob.n_cases):
            U[c, free] = lu.solve(prob.loads[c, free])
        return U
    dinv = 1.0 / Kff.diagonal()
    M = spla.LinearOperator(Kff.shape, matvec=lambda v: dinv * v)
    for c in range(prob.n_cases):
        b = prob.loads[c, free]
        xs = None if x0 is None else x0[c, free]
        x, info = spla.cg(Kff, b, x0=xs, rtol=rtol, atol=0.0, maxiter=maxiter, M=M, callback=callback)
        if info != 0:
            raise RuntimeError(f"oracle CG did not converge (info={info})")
        U[c, free] = x
    return U


def rel_residual(prob, rho, U, K=None):
    """True relative residual ||f - K u||_2 / ||f||_2 over the free DOFs, per case."""
    K = assemble(prob, rho) if K is None else K
    free = prob.fixed == 0
    out = []
    for c in range(prob.n_cases):
        r = (prob.loads[c] - K @ U[c])[free]
        out.append(np.linalg.norm(r) / np.linalg.norm(prob.loads[c][free]))
    return np.array(out)


def jacobi_diag(prob, rho, K=None):
    """Diagonal of the boundary-conditioned operator (1 on fixed rows)."""
    K = assemble(prob, rho) if K is None else K
    d = K.diagonal().copy()
    d[prob.fixed.astype(bool)] = 1.0
    return d
