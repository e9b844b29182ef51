"""Sparse FP64 oracle of the Galerkin reassembly (P-method, Sec. 5.1) -- TEST INFRASTRUCTURE ONLY.

Level 0 is the all-at-once matrix of Sec. 2.2 with the Dirichlet treatment of Appendix A,
J = B J_Neu B + W (I - B), assembled as a scipy.sparse matrix from the global mass and
stiffness matrices.  P_l is the Kronecker product of the 1D stencils of Sec. 3.1 / 5.1
(linear in x; causal or bilinear in t), R_l = s P_l^T (s = 1 for x, 1/2 for t), and every
coarser matrix is the sparse triple product J_{l+1} = R_l J_l P_l.  Alg. 1 runs on these
matrices as written: damped Jacobi with D = diag(J_l), the coarse-grid correction, and an
exact solve on the coarsest level by sparse LU; the adjoint uses J_l^T with the same P, R
(Sec. 7.2).  The coarsening path is Alg. 3's with the K-averaged material standing in for
the coarse k and c (Sec. 5.1); it is taken from the structured oracle's planner run with
reassembly K.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import Hierarchy


def _mk_sparse(N, dx, k, c):
    """Global consistent mass M and stiffness K of linear elements, tridiagonal."""
    k, c = np.asarray(k, float), np.asarray(c, float)
    md = np.zeros(N + 1)
    md[:N] += c * dx / 3.0
    md[1:] += c * dx / 3.0
    kd = np.zeros(N + 1)
    kd[:N] += k / dx
    kd[1:] += k / dx
    M = sp.diags([c * dx / 6.0, md, c * dx / 6.0], [-1, 0, 1], format="csr")
    K = sp.diags([-k / dx, kd, -k / dx], [-1, 0, 1], format="csr")
    return M, K


def all_at_once(N, NT, L, tT, k, c):
    """J = B J_Neu B + W (I - B) (Sec. 2.2, Appendix A) as a sparse matrix."""
    dx, dt = L / N, tT / NT
    M, K = _mk_sparse(N, dx, k, c)
    W = np.max(c) * dx / dt + np.max(k) / dx
    first = sp.diags([np.r_[1.0, np.zeros(NT)]], [0])
    later = sp.diags([np.r_[0.0, np.ones(NT)]], [0])
    below = sp.diags([np.ones(NT)], [-1])
    Jn = sp.kron(first, W * sp.identity(N + 1)) + sp.kron(later, M / dt + K) - sp.kron(below, M / dt)
    mask = np.ones((NT + 1, N + 1))
    mask[0, :] = 0.0
    mask[:, 0] = 0.0
    B = sp.diags([mask.ravel()], [0])
    I = sp.identity((NT + 1) * (N + 1))
    return (B @ Jn @ B + W * (I - B)).tocsr()


def _p_x(Nf):
    Nc = Nf // 2
    rows, cols, vals = [], [], []
    for j in range(Nc + 1):
        for i, w in ((2 * j - 1, 0.5), (2 * j, 1.0), (2 * j + 1, 0.5)):
            if 0 <= i <= Nf:
                rows.append(i), cols.append(j), vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(Nf + 1, Nc + 1))


def _p_t(NTf, interp):
    NTc = NTf // 2
    rows, cols, vals = [], [], []
    for m in range(NTc + 1):
        taps = ((2 * m, 1.0), (2 * m + 1, 1.0)) if interp == "C" else ((2 * m - 1, 0.5), (2 * m, 1.0), (2 * m + 1, 0.5))
        for n, w in taps:
            if 0 <= n <= NTf:
                rows.append(n), cols.append(m), vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(NTf + 1, NTc + 1))


class GalerkinHierarchy:
    """Levels J_0 (rediscretised) and J_{l+1} = R_l J_l P_l, with Alg. 1 on them."""

    def __init__(self, N, NT, L, tT, k, c, *, nu=5, omega=0.5, interp="C", **planner):
        plan = Hierarchy(N, NT, L, tT, k, c, nu=nu, omega=omega, interp=interp, reassembly="K", **planner)
        self.nu, self.omega, self.interp = nu, omega, interp
        self.path = plan.path()
        self.plan = plan
        J = all_at_once(N, NT, L, tT, k, c)
        self.levels = []
        for l, ch in enumerate(self.path + "."):
            lv = dict(N=N, NT=NT, J=J, D=J.diagonal().copy())
            if ch != ".":
                if ch == "x":
                    P, s = sp.kron(sp.identity(NT + 1), _p_x(N)), 1.0
                    N //= 2
                else:
                    P, s = sp.kron(_p_t(NT, interp), sp.identity(N + 1)), 0.5
                    NT //= 2
                lv["P"] = P.tocsr()
                lv["R"] = (s * P.T).tocsr()
                J = (lv["R"] @ J @ lv["P"]).tocsr()
                J.eliminate_zeros()
            self.levels.append(lv)
        self._lu = {}

    @property
    def nlevels(self):
        return len(self.levels)

    def shape(self, l):
        lv = self.levels[l]
        return (lv["NT"] + 1, lv["N"] + 1)

    def _J(self, l, adj):
        J = self.levels[l]["J"]
        return J.T.tocsr() if adj else J

    def apply(self, l, u, adj=False):
        return (self._J(l, adj) @ np.ravel(u)).reshape(self.shape(l))

    def residual(self, l, u, b, adj=False):
        return (np.ravel(b) - self._J(l, adj) @ np.ravel(u)).reshape(self.shape(l))

    def smooth(self, l, u, b, nsweeps, adj=False):
        J, D = self._J(l, adj), self.levels[l]["D"]
        u, b = np.ravel(u).astype(float).copy(), np.ravel(b)
        for _ in range(nsweeps):
            u = u + self.omega * (b - J @ u) / D
        return u.reshape(self.shape(l))

    def restrict(self, l, r):
        return (self.levels[l]["R"] @ np.ravel(r)).reshape(self.shape(l + 1))

    def prolong_add(self, l, z, u):
        return (np.ravel(u) + self.levels[l]["P"] @ np.ravel(z)).reshape(self.shape(l))

    def exact_level(self, l, b, adj=False):
        key = (l, adj)
        if key not in self._lu:
            self._lu[key] = spla.splu(self._J(l, adj).tocsc())
        return self._lu[key].solve(np.ravel(b).astype(float)).reshape(self.shape(l))

    def _cycle(self, l, u, b, adj):
        if l == self.nlevels - 1:
            return self.exact_level(l, b, adj)
        u = self.smooth(l, u, b, self.nu, adj)
        bc = self.restrict(l, self.residual(l, u, b, adj))
        z = self._cycle(l + 1, np.zeros(self.shape(l + 1)), bc, adj)
        u = self.prolong_add(l, z, u)
        return self.smooth(l, u, b, self.nu, adj)

    def vcycle(self, u, b, adj=False):
        """One cycle of Alg. 1 on level 0."""
        return self._cycle(0, np.reshape(u, self.shape(0)), np.reshape(b, self.shape(0)), adj)

    def solve(self, b, adj=False, tol=1e-10, div_tol=1e9, max_cycles=100, u0=None):
        """Sec. 3.1 solver loop; returns (u, status, cycles, residual history)."""
        b = np.reshape(b, self.shape(0)).astype(float)
        u = np.zeros(self.shape(0)) if u0 is None else np.reshape(u0, self.shape(0)).astype(float).copy()
        nb = np.linalg.norm(b)
        hist = [np.linalg.norm(self.residual(0, u, b, adj)) / nb]
        status, cyc = "max_cycles", 0
        if hist[0] < tol:
            return u, "converged", 0, np.array(hist)
        for cyc in range(1, max_cycles + 1):
            u = self.vcycle(u, b, adj)
            hist.append(np.linalg.norm(self.residual(0, u, b, adj)) / nb)
            if not hist[-1] <= div_tol:
                status = "diverged"
                break
            if hist[-1] < tol:
                status = "converged"
                break
        return u, status, cyc, np.array(hist)
