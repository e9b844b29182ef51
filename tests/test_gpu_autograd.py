"""GPU: time-slab recomputation of the forward state and the autograd adjoint backward.

Tolerances: slab recomputation is exact time stepping in FP64; it evaluates each step's
two Thomas recurrences as a parallel scan, whose rounding order differs from the oracle's
sequential Thomas, and over up to 4096 unknowns per step that difference reaches ~2e-11
of max|u| (bound used: 1e-10).  Gradients from
STMG solves to relative residual 1e-11 agree with the oracle's exact-solve gradient to
1e-7 relative, and with central differences of Theta (h = 1e-6, exact oracle solves) to
1e-5 relative (the finite-difference truncation and rounding error at h = 1e-6).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2505_10168_gb300 as pkg
from paper_2505_10168_gb300 import autograd as ag
from paper_2505_10168_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def T(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("N,NT,K", [(96, 200, 7), (96, 200, 64), (96, 200, 200), (700, 64, 1), (4096, 40, 16)])
def test_recompute_slabs_matches_exact_solution(N, NT, K):
    chi = 0.05 + 0.95 * wl.uniform(31, N)
    s6 = wl.simp_params(1e-3, 1.0, 0.4, 1.0)
    k, c = oracle.simp(chi, s6)
    q = wl.load_paper(N, NT, 1.0, 0.5) * 1e-6
    b = oracle.assemble_load(N, NT, 1.0 / N, q)
    ue = oracle.exact(N, NT, 1.0, 0.5, k, c, b)
    g = pkg.Solver(N, NT, 1.0, 0.5, k, c)
    ckpt = np.ascontiguousarray(ue[::K][: (NT + K - 1) // K])
    u = torch.empty((NT + 1, N + 1), dtype=torch.float64, device=DEV)
    g.recompute_slabs(T(b), T(ckpt), K, u)
    assert rel(u.cpu().numpy(), ue) < 1e-10
    g.close()


def _cfg4(N, NT):
    w = wl.random_design(N=N, NT=NT)
    return w, T(w["chi"]), T(w["q"])


@pytest.mark.parametrize("slab_rows", [0, 64])
def test_autograd_compliance_gradient_matches_oracle(slab_rows):
    N, NT = 256, 1024
    w, chi0, q = _cfg4(N, NT)
    s6 = w["simp"]
    solver = pkg.Solver(N, NT, 1.0, 1.0, np.ones(N), np.ones(N), nu=w["nu"], tol=1e-11)
    chi = chi0.clone().requires_grad_(True)
    u = ag.solve(chi, q, solver, s6, slab_rows=slab_rows)
    b = torch.empty_like(u)
    solver.assemble_load(q, b)
    theta = ag.compliance(u, b, solver)
    theta.backward()
    ko, co = oracle.simp(w["chi"], s6)
    bo = oracle.assemble_load(N, NT, 1.0 / N, w["q"])
    uo = oracle.exact(N, NT, 1.0, 1.0, ko, co, bo)
    lo = oracle.exact(N, NT, 1.0, 1.0, ko, co, bo * solver.dt, adj=True)
    go = oracle.sensitivity(N, NT, 1.0, 1.0, w["chi"], s6, uo, lo)
    assert float(theta) == pytest.approx(oracle.objective(N, NT, solver.dt, bo, uo), rel=1e-9)
    assert rel(chi.grad.cpu().numpy(), go) < 1e-7
    solver.close()


def test_random_design_gradient_against_central_differences():
    """The differentiation workload at full size (1024 x 4096): autograd gradient of the
    compliance against central differences with h = 1e-6 on 32 random elements.  The
    solves stop at 1e-10: at this grid the FP64 evaluation of J u cancels ~1e6-fold
    (|J_ij u_j| / |b_i|), which puts the attainable relative residual near 5e-11."""
    w, chi0, q = _cfg4(1024, 4096)
    N, NT, s6 = w["N"], w["NT"], w["simp"]
    solver = pkg.Solver(N, NT, 1.0, 1.0, np.ones(N), np.ones(N), nu=w["nu"], tol=1e-10)
    chi = chi0.clone().requires_grad_(True)
    u = ag.solve(chi, q, solver, s6, slab_rows=256)
    b = torch.empty_like(u)
    solver.assemble_load(q, b)
    ag.compliance(u, b, solver).backward()
    grad = chi.grad.cpu().numpy()
    bo = oracle.assemble_load(N, NT, 1.0 / N, w["q"])
    dt = 1.0 / NT

    def theta(x):
        k, c = oracle.simp(x, s6)
        return oracle.objective(N, NT, dt, bo, oracle.exact(N, NT, 1.0, 1.0, k, c, bo))

    h = 1e-6
    scale = np.abs(grad).max()
    for e in w["fd_elements"]:
        xp, xm = w["chi"].copy(), w["chi"].copy()
        xp[e] += h
        xm[e] -= h
        fd = (theta(xp) - theta(xm)) / (2 * h)
        assert abs(grad[e] - fd) <= 1e-5 * scale, (e, grad[e], fd)
    solver.close()


def test_objective_and_its_gradient_in_the_library():
    """stmg_objective gives Theta = b^T u dt / Theta_ref (Sec. 7.1) and
    stmg_objective_gradient seed * b dt / Theta_ref, the adjoint right-hand side of Sec.
    7.2; autograd.compliance uses both.  Host arrays are refused by the gradient call."""
    N, NT = 64, 128
    w, chi0, q = _cfg4(N, NT)
    solver = pkg.Solver(N, NT, 1.0, 1.0, np.ones(N), np.ones(N))
    b = torch.empty((NT + 1, N + 1), dtype=torch.float64, device=DEV)
    solver.assemble_load(q, b)
    u = T(wl.uniform(9, (NT + 1) * (N + 1)).reshape(NT + 1, N + 1))
    theta = solver.objective(b, u, theta_ref=2.0)
    bo = oracle.assemble_load(N, NT, 1.0 / N, w["q"])
    assert theta == pytest.approx(oracle.objective(N, NT, solver.dt, bo, u.cpu().numpy()) / 2.0, rel=1e-13)
    g = torch.empty_like(b)
    solver.objective_gradient(b, g, theta_ref=2.0, seed=3.0)
    assert torch.equal(g, b * (3.0 * solver.dt / 2.0))
    uu = u.clone().requires_grad_(True)
    ag.compliance(uu, b, solver, theta_ref=2.0).backward()
    assert torch.equal(uu.grad, b * (solver.dt / 2.0))
    with pytest.raises(pkg.STMGError, match="einval"):
        solver.objective_gradient(b.cpu(), g)
    solver.close()
