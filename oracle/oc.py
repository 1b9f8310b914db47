"""Optimality-criteria update with bisection on the Lagrange multiplier
(Section 3.2, Eq. "kkt", Eq. "update"; Section 3.2.1 "The bisection method";
code of Section 4.4).

Update with move limit m = 0.2, damping eta = 0.5 and lower bound dmin = 0.001:
  B_e = -dc~_e / lambda   (d g / d rho_e = 1 for unit elements)
  rho_new = max(dmin, max(rho - m, min(1, min(rho + m, rho * B_e^eta))))
Bisection: g(rho_new(lambda)) = sum(rho_new) - volfrac * N; if it is positive the
lower bound moves up to the midpoint, otherwise the upper bound moves down.

Readings where the paper is silent or differs from the workloads:
  * bracket [0, 1e9], upper end multiplied by 10 while the volume at it is still
    above target; stop when l2 - l1 <= 1e-9 (l1 + l2) (relative, instead of the
    paper's absolute 1e-4 with l2 = 1e5);
  * the final density uses the midpoint of the final bracket;
  * passive elements are held at dmin inside the bisection (volume exact);
  * a non-negative dc~ (cannot occur for compliance) gives B = 0.
"""
from __future__ import annotations

import numpy as np


def update(rho, dcf, lam, move=0.2, dmin=1e-3, passive=None, eta=0.5):
    B = np.maximum(-dcf, 0.0) / lam
    cand = rho * np.power(B, eta)
    new = np.maximum(dmin, np.maximum(rho - move, np.minimum(1.0, np.minimum(rho + move, cand))))
    if passive is not None:
        new = np.where(passive == 1, dmin, new)
    return new


def bisect(rho, dcf, volfrac, move=0.2, dmin=1e-3, passive=None, rel_tol=1e-9,
           l2_init=1e9, max_iter=1000):
    """Returns (rho_new, lambda, volume, change, n_halvings)."""
    target = volfrac * rho.size
    l1, l2 = 0.0, l2_init
    while np.sum(update(rho, dcf, l2, move, dmin, passive)) > target and l2 < 1e300:
        l2 *= 10.0
    it = 0
    while (l2 - l1) > rel_tol * (l1 + l2) and it < max_iter:
        mid = 0.5 * (l1 + l2)
        if np.sum(update(rho, dcf, mid, move, dmin, passive)) - target > 0:
            l1 = mid
        else:
            l2 = mid
        it += 1
    lam = 0.5 * (l1 + l2)
    new = update(rho, dcf, lam, move, dmin, passive)
    return new, lam, float(np.sum(new)), float(np.max(np.abs(new - rho))), it


def volume_at(rho, dcf, lam, move=0.2, dmin=1e-3, passive=None):
    return float(np.sum(update(rho, dcf, lam, move, dmin, passive)))


def exact_lambda(rho, dcf, volfrac, move=0.2, dmin=1e-3, passive=None):
    """Exact root of V(lambda) = volfrac * N.

    With s = lambda^(-1/2) and B_e = rho_e sqrt(max(-dc~_e, 0)), each element's
    new density is clamp(B_e s, lo_e, hi_e) with lo_e = max(dmin, rho_e - m),
    hi_e = min(1, rho_e + m); V is piecewise linear and non-decreasing in s.
    Sorting the breakpoints lo_e / B_e and hi_e / B_e gives the piece that holds
    the target, solved in closed form.  Returns lambda (None if no root)."""
    target = volfrac * rho.size
    act = np.ones(rho.size, dtype=bool) if passive is None else (passive != 1)
    const = float(np.sum(~act)) * dmin
    r = rho[act]
    Bc = r * np.sqrt(np.maximum(-dcf[act], 0.0))
    lo = np.maximum(dmin, r - move)
    hi = np.minimum(1.0, r + move)
    zero = Bc <= 0
    const += float(np.sum(lo[zero]))
    Bc, lo, hi = Bc[~zero], lo[~zero], hi[~zero]
    s_lo, s_hi = lo / Bc, hi / Bc
    # events: at s_lo an element starts growing (slope +B), at s_hi it stops (slope -B)
    ev_s = np.concatenate([s_lo, s_hi])
    ev_db = np.concatenate([Bc, -Bc])
    order = np.argsort(ev_s, kind="stable")
    ev_s, ev_db = ev_s[order], ev_db[order]
    # V(s) = const + sum(lo) + sum_{active} (B s - lo) + sum_{done} (hi - lo)
    base = const + float(np.sum(lo))
    slope, offset = 0.0, 0.0  # V = base + slope * s + offset
    prev = 0.0
    cur = base
    for s, db in zip(ev_s, ev_db):
        v_here = base + slope * s + offset
        if v_here >= target and slope > 0:
            s_star = (target - base - offset) / slope
            return 1.0 / (s_star * s_star)
        # crossing an event at s: adjust slope and offset so V stays continuous
        if db > 0:
            slope += db
            offset -= db * s  # growing element contributes B (s' - s_lo)
        else:
            slope += db
            offset -= db * s  # element capped: removes B s', adds B s_hi
        prev = s
        cur = v_here
    if slope > 0:
        s_star = (target - base - offset) / slope
        return 1.0 / (s_star * s_star)
    return None
