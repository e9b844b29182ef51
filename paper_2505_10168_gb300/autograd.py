"""Differentiable STMG solve: u(chi) with a hand-written adjoint backward.

Forward: SIMP material (Sec. 2.1) from the design field chi, then the STMG solve of
J(chi) u = b (Alg. 1).  Backward, for an upstream gradient g_u = dL/du: the adjoint
STMG solve J^T lam = g_u with the same hierarchy and the unchanged causal prolongation
(Sec. 7.2), then the fused sensitivity kernel dL/dchi_e = -lam^T (dJ/dchi_e) u.  For the
compliance Theta = b^T u dt / Theta_ref (Sec. 7.1) the upstream gradient is
b dt / Theta_ref, which is the paper's adjoint right-hand side.

With ``slab_rows = K`` the forward keeps only every K-th time level of u; the backward
rebuilds each slab of K levels exactly from its checkpoint inside the sensitivity kernel
(``stmg_sensitivity_slabs``), so the backward holds no full copy of u.

All arithmetic runs in libstmg.so; this module only wires it into torch.autograd.
"""
from __future__ import annotations

import torch

from . import Solver, simp


class _SolveFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, chi, q, solver, simp6, slab_rows):
        N, NT = solver.nel, solver.nt
        dev = chi.device
        k = torch.empty(N, dtype=torch.float64, device=dev)
        c = torch.empty_like(k)
        simp(chi, simp6, k, c)
        solver.update_material(k, c)
        b = torch.empty((NT + 1, N + 1), dtype=torch.float64, device=dev)
        solver.assemble_load(q, b)
        u = torch.empty_like(b)
        status, cycles, relres = solver.solve(u, b=b)
        if status != "ok":
            raise RuntimeError("STMG forward solve stopped: %s after %d cycles (relres %.3e)" % (status, cycles, relres))
        ctx.solver, ctx.simp6, ctx.slab_rows = solver, list(simp6), slab_rows
        if slab_rows:
            ckpt = u[::slab_rows][: (NT + slab_rows - 1) // slab_rows].contiguous()
            ctx.save_for_backward(chi, q, ckpt)
        else:
            ctx.save_for_backward(chi, q, u)
        ctx.stats = (cycles, relres)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        chi, q, saved = ctx.saved_tensors
        solver = ctx.solver
        lam = torch.empty_like(grad_u, dtype=torch.float64)
        status, cycles, relres = solver.solve_adjoint(lam, grad_u.contiguous().to(torch.float64))
        if status != "ok":
            raise RuntimeError("STMG adjoint solve stopped: %s after %d cycles (relres %.3e)" % (status, cycles, relres))
        g = torch.empty_like(chi)
        if ctx.slab_rows:
            b = torch.empty_like(lam)
            solver.assemble_load(q, b)
            solver.sensitivity_slabs(chi, ctx.simp6, b, saved, ctx.slab_rows, lam, g)
        else:
            solver.sensitivity(chi, ctx.simp6, saved, lam, g)
        return g, None, None, None, None


def solve(chi, q, solver: Solver, simp6, slab_rows: int = 0):
    """u = STMG solution for the design field chi and element loads q.

    chi: (nel,) float64 CUDA tensor (requires_grad for a gradient); q: (nt+1, nel) loads;
    solver: a ``Solver`` of the same grid (its material is replaced); simp6: SIMP
    parameters (k_ins, k_con, c_ins, c_con, p_k, p_c); slab_rows: 0 keeps u for the
    backward, K > 0 keeps only every K-th time level.
    """
    return _SolveFn.apply(chi, q, solver, simp6, int(slab_rows))


class _ComplianceFn(torch.autograd.Function):
    """Theta = b^T u dt / Theta_ref by stmg_objective; the backward hands b dt / Theta_ref
    (times the upstream gradient) to u by stmg_objective_gradient."""

    @staticmethod
    def forward(ctx, u, b, solver, theta_ref):
        ctx.save_for_backward(b)
        ctx.solver, ctx.theta_ref = solver, float(theta_ref)
        theta = solver.objective(b.contiguous(), u.contiguous(), ctx.theta_ref)
        return torch.tensor(theta, dtype=torch.float64, device=u.device)

    @staticmethod
    def backward(ctx, grad_theta):
        (b,) = ctx.saved_tensors
        grad_u = torch.empty_like(b)
        ctx.solver.objective_gradient(b.contiguous(), grad_u, ctx.theta_ref, float(grad_theta))
        return grad_u, None, None, None


def compliance(u, b, solver: Solver, theta_ref=1.0):
    """Theta = b^T u dt / Theta_ref (Sec. 7.1) of the state u for the nodal load b on the
    solver's grid, differentiable in u (forward and backward in the library)."""
    return _ComplianceFn.apply(u, b, solver, float(theta_ref))
