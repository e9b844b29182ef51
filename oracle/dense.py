"""Dense-matrix brute force for tiny space-time grids (TEST INFRASTRUCTURE ONLY).

This module pins the structured oracle in ``stmg_oracle.c``.  It shares nothing with it:
it assembles the global FE matrices with ``np.add.at``, builds the all-at-once matrix as
explicit blocks (Sec. 2.2), applies the Dirichlet treatment of Appendix A as the matrix
product ``B J_Neu B + W (I - B)``, builds P from Kronecker products of 1D stencil matrices
(Sec. 3.1, 5.1) and runs Alg. 1 with dense linear algebra (``np.linalg.solve`` on the
coarsest level).  Vectors are flattened (time level major, node minor).
"""
from __future__ import annotations

import numpy as np


def global_mk(N, dx, k, c):
    """Global consistent mass M and stiffness K of linear elements (Sec. 2.2)."""
    M = np.zeros((N + 1, N + 1))
    K = np.zeros((N + 1, N + 1))
    me = np.array([[2.0, 1.0], [1.0, 2.0]]) / 6.0
    ke = np.array([[1.0, -1.0], [-1.0, 1.0]])
    for e in range(N):
        idx = np.ix_([e, e + 1], [e, e + 1])
        np.add.at(M, idx, c[e] * dx * me)
        np.add.at(K, idx, k[e] / dx * ke)
    return M, K


def w_diri(dx, dt, k, c):
    """Appendix A: W_Diri = max c dx/dt + max k/dx."""
    return np.max(c) * dx / dt + np.max(k) / dx


def dirichlet_mask(N, NT):
    """Diagonal of B: 0 on the initial row and on node 0, 1 elsewhere (Appendix A)."""
    B = np.ones((NT + 1, N + 1))
    B[0, :] = 0.0
    B[:, 0] = 0.0
    return B.ravel()


def all_at_once(N, NT, L, tT, k, c):
    """J = B J_Neu B + W (I - B) with the block lower-bidiagonal J_Neu of Sec. 2.2."""
    dx, dt = L / N, tT / NT
    M, K = global_mk(N, dx, k, c)
    W = w_diri(dx, dt, k, c)
    n = (NT + 1) * (N + 1)
    Jn = np.zeros((n, n))
    Jn[: N + 1, : N + 1] = W * np.eye(N + 1)
    for t in range(1, NT + 1):
        r = slice(t * (N + 1), (t + 1) * (N + 1))
        rp = slice((t - 1) * (N + 1), t * (N + 1))
        Jn[r, r] = M / dt + K
        Jn[r, rp] = -M / dt
    Bd = dirichlet_mask(N, NT)
    B = np.diag(Bd)
    return B @ Jn @ B + W * (np.eye(n) - B)


def load_vector(N, NT, dx, q):
    """b = B b_Neu with b_Neu,n = integral of q_n N_i (element-wise constant q)."""
    q = np.asarray(q, dtype=np.float64).reshape(NT + 1, N)
    bn = np.zeros((NT + 1, N + 1))
    bn[:, :N] += q * dx / 2.0
    bn[:, 1:] += q * dx / 2.0
    return (dirichlet_mask(N, NT) * bn.ravel())


def p1d_x(Nf):
    """1D x-prolongation 1/2 [1 2 1]: (Nf+1) x (Nf/2+1)."""
    Nc = Nf // 2
    P = np.zeros((Nf + 1, Nc + 1))
    for j in range(Nc + 1):
        P[2 * j, j] = 1.0
        if 2 * j - 1 >= 0:
            P[2 * j - 1, j] = 0.5
        if 2 * j + 1 <= Nf:
            P[2 * j + 1, j] = 0.5
    return P


def p1d_t(NTf, interp="C"):
    """1D t-prolongation: causal [1;1] (forward only) or bilinear 1/2 [1;2;1]."""
    NTc = NTf // 2
    P = np.zeros((NTf + 1, NTc + 1))
    for m in range(NTc + 1):
        P[2 * m, m] = 1.0
        if interp == "C":
            if 2 * m + 1 <= NTf:
                P[2 * m + 1, m] = 1.0
        else:
            if 2 * m - 1 >= 0:
                P[2 * m - 1, m] = 0.5
            if 2 * m + 1 <= NTf:
                P[2 * m + 1, m] = 0.5
    return P


def prolongation(N, NT, kind, interp="C"):
    """Space-time P as a Kronecker product (time index major)."""
    if kind == "x":
        return np.kron(np.eye(NT + 1), p1d_x(N)), 1.0
    return np.kron(p1d_t(NT, interp), np.eye(N + 1)), 0.5


def simp_material(chi, simp6):
    """SIMP interpolation of Sec. 2.1 for design values chi (vectorised)."""
    k_ins, k_con, c_ins, c_con, p_k, p_c = [float(v) for v in simp6]
    chi = np.asarray(chi, dtype=np.float64)
    return k_ins + (k_con - k_ins) * chi ** p_k, c_ins + (c_con - c_ins) * chi ** p_c


def coarse_material(k, c, kind, reassembly, chi=None, simp6=None):
    """Coarse k, c (and the coarse design field, with D) of one coarsening step: t keeps
    the material (and chi); x merges element pairs by conductivity (K), resistivity (R)
    or design-field (D: mean chi of the pair, SIMP re-applied) averaging (Sec. 3.1, 5.1).
    Returns (k, c, chi)."""
    if kind == "t":
        return k.copy(), c.copy(), (None if chi is None else chi.copy())
    if reassembly == "D":
        chi_c = 0.5 * (chi[0::2] + chi[1::2])
        kc, cc = simp_material(chi_c, simp6)
        return kc, cc, chi_c
    k0, k1 = k[0::2], k[1::2]
    c2 = (c[0::2] + c[1::2]) / 2.0
    if reassembly == "R":
        return 2.0 * k0 * k1 / (k0 + k1), c2, None
    return (k0 + k1) / 2.0, c2, None


class DenseHierarchy:
    """Dense levels for a given coarsening path (string of 'x'/'t').

    reassembly "K" / "R" / "D": every level is the all-at-once J of its own grid and
    averaged material (Sec. 3.1, 5.1; "D" needs the design field chi and simp6, and the
    level-0 material is SIMP of chi); "P": every coarse J is the Galerkin product R J P
    of the level above (Sec. 5.1)."""

    def __init__(self, N, NT, L, tT, k, c, path, interp="C", reassembly="R", chi=None, simp6=None):
        self.levels = []
        if reassembly == "D":
            chi = np.asarray(chi, float)
            k, c = simp_material(chi, simp6)
        k, c = np.asarray(k, float), np.asarray(c, float)
        J = all_at_once(N, NT, L, tT, k, c)
        for l in range(len(path) + 1):
            lv = dict(N=N, NT=NT, J=J, D=np.diag(J).copy(), k=k, c=c, chi=chi)
            if l < len(path):
                kind = path[l]
                P, s = prolongation(N, NT, kind, interp)
                lv["P"], lv["R"] = P, s * P.T
                k, c, chi = coarse_material(k, c, kind, "K" if reassembly == "P" else reassembly, chi, simp6)
                if kind == "x":
                    N //= 2
                else:
                    NT //= 2
                if reassembly == "P":
                    J = lv["R"] @ lv["J"] @ P
                else:
                    J = all_at_once(N, NT, L, tT, k, c)
            self.levels.append(lv)

    def vcycle(self, l, u, b, nu=5, omega=0.5, adj=False):
        lv = self.levels[l]
        J = lv["J"].T if adj else lv["J"]
        if l == len(self.levels) - 1:
            return np.linalg.solve(J, b)
        for _ in range(nu):
            u = u + omega * (b - J @ u) / lv["D"]
        bc = lv["R"] @ (b - J @ u)
        z = self.vcycle(l + 1, np.zeros_like(bc), bc, nu, omega, adj)
        u = u + lv["P"] @ z
        for _ in range(nu):
            u = u + omega * (b - J @ u) / lv["D"]
        return u
