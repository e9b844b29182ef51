"""Exact scaling with the right-hand side (GPU).

J is linear, and every step of the solve (FP64 arithmetic, the FP32 cycles of the mixed
scheme, the termination norms) commutes with a power-of-two scale of b as long as no value
leaves the range of its format.  The FP32 parts run on copies scaled by 2^k with k taken
from ||b||, so J u = 2^m b must take the same cycles, report the same relative residual and
return exactly 2^m u, bit for bit, also for m far outside the FP32 range: a square r^2 of
an unscaled residual of 2^-200 b would flush to zero in FP32 (a false convergence) and an
unscaled FP32 defect would flush to zero (no progress).  The unscaled solution itself is
checked against the oracle's exact time stepping.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2505_10168_gb300 as pkg
from paper_2505_10168_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")

N, NT = 96, 320


def _problem():
    u = wl.uniform(71, 2 * N)
    k = np.exp(np.log(1e-3) * u[:N])
    c = 0.5 + u[N:]
    b = wl.uniform(72, (NT + 1) * (N + 1)).reshape(NT + 1, N + 1) - 0.3
    return k, c, b


def _solve(precision, adj, b, k, c, tT):
    s = pkg.Solver(N, NT, 1.0, tT, torch.tensor(k, device=DEV), torch.tensor(c, device=DEV),
                   precision=precision, tol=1e-10, max_coarse_dofs=64)
    out = torch.empty((NT + 1, N + 1), dtype=torch.float64, device=DEV)
    bd = torch.tensor(b, device=DEV)
    st, cyc, rr = s.solve_adjoint(out, bd) if adj else s.solve(out, b=bd)
    s.close()
    return st, cyc, rr, out.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("adj", [False, True])
def test_solution_scales_exactly_with_b(precision, adj):
    k, c, b = _problem()
    tT = 0.05
    st0, cyc0, rr0, u0 = _solve(precision, adj, b, k, c, tT)
    assert st0 == "ok" and rr0 < 1e-10
    ue = oracle.exact(N, NT, 1.0, tT, k, c, b, adj=adj)
    assert np.abs(u0 - ue).max() / np.abs(ue).max() < (1e-9 if precision == "fp64" else 1e-8)
    for m in (-200, -60, 60, 200):
        st, cyc, rr, um = _solve(precision, adj, np.ldexp(b, m), k, c, tT)
        assert (st, cyc) == (st0, cyc0), m
        assert rr == rr0, m
        assert np.array_equal(um, np.ldexp(u0, m)), m
