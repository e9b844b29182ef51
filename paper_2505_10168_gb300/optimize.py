"""The optimisation loop of Sec. 7 on the GPU.

min Theta = b^T u dt / Theta_ref over the design chi, subject to J(chi) u = b,
0 <= chi <= 1 and mean(chi) <= vol_frac (Sec. 7.1).  Every cycle re-assembles the levels
for the current design (SIMP material, then the chosen coarse reassembly K, R, P, or D from
the design field itself) on a hierarchy fixed at the start (the design-independent D_eff of
Sec. 7.2 gives the same coarsening path for every design), solves the state and the
adjoint J^T lam = b dt / Theta_ref (up to that positive factor) by STMG (warm restarts
start from the previous cycle's u and lam; cold restarts from 0), evaluates Theta and the
discrete-adjoint sensitivity,
and updates the design with ``design_update`` -- the projected-gradient step that stands
in for the paper's MMA optimiser.  The loop stops when Theta has changed by less than rtol
(relative) for `patience` consecutive cycles (Sec. 7.2: 0.1 % for 5 cycles).
"""
from __future__ import annotations

import numpy as np
import torch

from . import Solver, deff_simp, design_update, simp


def optimize(N, NT, L, tT, simp6, q, vol_frac=0.5, move=0.2, chi0=0.5, theta_ref=1e6, warm=True, max_iter=200,
             rtol=1e-3, patience=5, device="cuda", **solver_opts):
    """Runs the loop; q: (NT+1) x N element loads (host or device).  Solver options (nu,
    num_levels, interp, reassembly, tol, ...) pass through to ``Solver``.

    Returns a dict with the final design ``chi`` (numpy) and ``history``: one entry per cycle
    with theta and the primal / adjoint cycle counts, statuses and relative residuals."""
    dev = torch.device(device)
    chi = torch.full((N,), float(chi0), dtype=torch.float64, device=dev)
    opts = dict(deff_fixed=deff_simp(simp6), reassembly="R")
    opts.update(solver_opts)
    design_path = opts["reassembly"] == "D"
    history = []
    if design_path:  # D-reassembly re-applies SIMP on every level itself
        opts.pop("reassembly")
        solver = Solver(N, NT, L, tT, chi=chi, simp6=simp6, **opts)
    else:  # K, R, P: the material of the current design, by the SIMP kernel
        k = torch.empty_like(chi)
        c = torch.empty_like(chi)
        simp(chi, simp6, k, c)
        solver = Solver(N, NT, L, tT, k, c, **opts)
    with solver:
        qd = torch.as_tensor(np.ascontiguousarray(q), dtype=torch.float64, device=dev)
        b = torch.empty((NT + 1, N + 1), dtype=torch.float64, device=dev)
        solver.assemble_load(qd, b)
        # The adjoint of the objective solves J^T lam = b dt / Theta_ref; the loop solves
        # J^T lam = b instead: the positive factor dt / Theta_ref scales the sensitivity and
        # drops out of the normalised design step.
        u = torch.zeros_like(b)
        lam = torch.zeros_like(b)
        g = torch.empty_like(chi)
        calm = 0
        for it in range(max_iter):
            if it > 0:
                if design_path:
                    solver.update_design(chi)
                else:
                    simp(chi, simp6, k, c)
                    solver.update_material(k, c)
            restart = warm and it > 0
            st_u, cyc_u, rr_u = solver.solve(u, b=b, warm=restart)
            st_l, cyc_l, rr_l = solver.solve_adjoint(lam, b, warm=restart)
            theta = solver.objective(b, u, theta_ref)
            history.append(dict(theta=theta, cycles=cyc_u, adj_cycles=cyc_l, status=st_u, adj_status=st_l,
                                relres=rr_u, adj_relres=rr_l))
            if len(history) > 1:
                prev = history[-2]["theta"]
                calm = calm + 1 if abs(theta - prev) < rtol * abs(prev) else 0
                if calm >= patience:
                    break
            solver.sensitivity(chi, simp6, u, lam, g)
            design_update(chi, g, vol_frac, move, chi)
        torch.cuda.synchronize(dev)
    return dict(chi=chi.cpu().numpy(), history=history)


def main():
    """Problem 7's optimisation (Sec. 7.1) with the paper's settings; prints one line per cycle."""
    import argparse

    from . import workloads as wl

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--interp", default="C", choices=["C", "B"])
    ap.add_argument("--reassembly", default="R", choices=["K", "R", "D", "P"])
    ap.add_argument("--cold", action="store_true")
    ap.add_argument("--max-iter", type=int, default=200)
    a = ap.parse_args()
    p = wl.paper_problem(7, N=a.n, NT=a.n)
    q = wl.load_paper(a.n, a.n, p["L"], p["tT"])
    r = optimize(a.n, a.n, p["L"], p["tT"], p["simp"], q, warm=not a.cold, max_iter=a.max_iter, num_levels=6, nu=20,
                 interp=a.interp, reassembly=a.reassembly, tol=1e-9)
    for i, h in enumerate(r["history"]):
        print(i, "%.6f" % h["theta"], h["cycles"], h["adj_cycles"], h["status"], h["adj_status"])


if __name__ == "__main__":
    main()
