"""FP64 CPU oracle of the optimisation loop of Sec. 7 (test infrastructure only).

The paper updates the design with MMA, a third-party optimiser that is not part of the
method.  Both here and on the GPU its place is taken by a projected-gradient step:

    y       = chi - move * g / max|g|                       (steepest descent, move limit)
    chi_new = clamp(y - mu, max(0, chi - move), min(1, chi + move))

with mu >= 0 the smallest shift for which mean(chi_new) <= vol_frac (the volume
constraint of Sec. 7.1 for elements of equal size).  This chi_new is the Euclidean
projection of y onto {box} intersected with {mean <= vol_frac}, found here by bisection on
mu because mean(chi_new) falls monotonically as mu grows.

``optimize`` runs the loop of Sec. 7.2 with exact solves (sequential time stepping) for
the state and the adjoint and the discrete-adjoint sensitivity, all from the oracle.
"""
from __future__ import annotations

import numpy as np

from . import assemble_load, exact, objective, sensitivity, simp

BISECTION_STEPS = 64


def design_update(chi, g, vol_frac, move):
    """One projected-gradient design update (see the module docstring)."""
    chi = np.asarray(chi, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    gmax = np.abs(g).max() if g.size else 0.0
    step = g / gmax if gmax > 0.0 else np.zeros_like(g)
    y = chi - move * step
    lo = np.maximum(0.0, chi - move)
    hi = np.minimum(1.0, chi + move)

    def shifted(mu):
        return np.minimum(np.maximum(y - mu, lo), hi)

    if shifted(0.0).mean() <= vol_frac:
        return shifted(0.0), 0.0
    # mean(shifted(a)) > vol_frac >= mean(shifted(b)) (b = 2 puts every element on its
    # lower bound; if even that is above vol_frac, the move limit wins and mu = 2)
    a, b = 0.0, 2.0
    for _ in range(BISECTION_STEPS):
        mid = 0.5 * (a + b)
        if shifted(mid).mean() > vol_frac:
            a = mid
        else:
            b = mid
    return shifted(b), b


def optimize(N, NT, L, tT, simp6, q, iters, vol_frac=0.5, move=0.2, chi0=0.5, theta_ref=1e6):
    """The loop of Sec. 7.2 for ``iters`` design updates from chi = chi0, exact solves.

    Returns the list of designs (iters + 1 of them, the start included) and the list of
    objective values Theta = b^T u dt / theta_ref of the first iters designs.
    """
    dx, dt = L / N, tT / NT
    b = assemble_load(N, NT, dx, q)
    chi = np.full(N, float(chi0))
    designs, thetas = [chi.copy()], []
    for _ in range(iters):
        k, c = simp(chi, simp6)
        u = exact(N, NT, L, tT, k, c, b)
        lam = exact(N, NT, L, tT, k, c, b * (dt / theta_ref), adj=True)
        thetas.append(objective(N, NT, dt, b, u, theta_ref))
        g = sensitivity(N, NT, L, tT, chi, simp6, u, lam)
        chi, _ = design_update(chi, g, vol_frac, move)
        designs.append(chi.copy())
    return designs, thetas
