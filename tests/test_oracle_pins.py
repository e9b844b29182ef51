"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test ties one oracle function to something other than itself: the printed stencil
and W_Diri formula, a dense direct solve of the all-at-once system, the separable modal
closed form, the printed lambda_eff values, a dense Kronecker-product brute-force V-cycle,
the adjoint identity, central finite differences, and the paper's qualitative claims.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import dense
from paper_2505_10168_gb300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _rand_material(seed, N, contrast=1e3):
    u = wl.uniform(seed, 2 * N)
    k = np.exp(np.log(1.0 / contrast) * u[:N])
    c = 0.5 + u[N:]
    return k, c


def _rand_vec(seed, shape):
    return wl.uniform(seed, int(np.prod(shape))).reshape(shape) - 0.5


# ---------------------------------------------------------------- assembly (Sec. 2.2, App. A)

def test_interior_stencil_matches_printed_stencil():
    g = _gold("stencil_sec2.json")
    N, NT, L, tT, kc, cc = 8, 8, 1.3, 0.9, 0.7, 1.9
    H = oracle.Hierarchy(N, NT, L, tT, np.full(N, kc), np.full(N, cc), num_levels=1)
    dx, dt = L / N, tT / NT
    expect = cc * dx / dt * np.array(g["mass"]) + kc / dx * np.array(g["stiffness"])
    n, i = 4, 4
    row = np.zeros((NT + 1, N + 1))
    for m in range(NT + 1):
        for j in range(N + 1):
            e = np.zeros((NT + 1, N + 1))
            e[m, j] = 1.0
            row[m, j] = H.apply(0, e)[n, i]
    got = np.array([[row[n + 1, i - 1], row[n + 1, i], row[n + 1, i + 1]],
                    [row[n, i - 1], row[n, i], row[n, i + 1]],
                    [row[n - 1, i - 1], row[n - 1, i], row[n - 1, i + 1]]])
    np.testing.assert_allclose(got, expect, rtol=1e-14, atol=1e-12)
    row[n - 1:n + 2, i - 1:i + 2] = 0.0
    assert np.all(row == 0.0), "J has entries outside the 6-point stencil"


def test_dirichlet_weight_formula():
    N, NT, L, tT = 6, 5, 2.0, 3.0
    k, c = _rand_material(11, N)
    H = oracle.Hierarchy(N, NT, L, tT, k, c, num_levels=1)
    W = c.max() * (L / N) / (tT / NT) + k.max() / (L / N)
    for (m, j) in [(0, 0), (0, 3), (2, 0), (NT, 0)]:
        e = np.zeros((NT + 1, N + 1))
        e[m, j] = 1.0
        y = H.apply(0, e)
        assert y[m, j] == pytest.approx(W, rel=1e-15)
        y[m, j] = 0.0
        assert np.all(y == 0.0)  # Dirichlet columns are eliminated


@pytest.mark.parametrize("N,NT", [(2, 2), (4, 8), (8, 4), (5, 3), (1, 6)])
def test_operator_matches_dense_all_at_once(N, NT):
    L, tT = 1.7, 0.6
    k, c = _rand_material(N * 31 + NT, N)
    H = oracle.Hierarchy(N, NT, L, tT, k, c, num_levels=1)
    J = dense.all_at_once(N, NT, L, tT, k, c)
    u = _rand_vec(5, (NT + 1, N + 1))
    scale = np.abs(J).max() * np.abs(u).max()
    np.testing.assert_allclose(H.apply(0, u).ravel(), J @ u.ravel(), rtol=0, atol=1e-14 * scale)
    np.testing.assert_allclose(H.apply(0, u, adj=True).ravel(), J.T @ u.ravel(), rtol=0, atol=1e-14 * scale)
    np.testing.assert_allclose(H.diag(0).ravel(), np.diag(J), rtol=1e-15)


def test_load_vector_matches_dense():
    N, NT, L = 7, 5, 1.4
    q = _rand_vec(3, (NT + 1, N)) + 2.0
    b = oracle.assemble_load(N, NT, L / N, q)
    np.testing.assert_allclose(b.ravel(), dense.load_vector(N, NT, L / N, q), rtol=1e-15, atol=0)
    assert np.all(b[0] == 0) and np.all(b[:, 0] == 0)


# ---------------------------------------------------------------- exact solution

@pytest.mark.parametrize("N,NT", [(2, 2), (4, 8), (8, 4), (3, 7)])
@pytest.mark.parametrize("adj", [False, True])
def test_exact_time_stepping_matches_dense_lu(N, NT, adj):
    L, tT = 1.0, 2.0
    k, c = _rand_material(N + 7 * NT, N, contrast=1e4)
    J = dense.all_at_once(N, NT, L, tT, k, c)
    b = _rand_vec(17, (NT + 1, N + 1))  # includes Dirichlet entries, as on coarse levels
    u = oracle.exact(N, NT, L, tT, k, c, b, adj=adj)
    ref = np.linalg.solve(J.T if adj else J, b.ravel())
    np.testing.assert_allclose(u.ravel(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_exact_matches_modal_closed_form():
    """Constant k, c: v_j(i) = sin(theta_j i), theta_j = (2j-1) pi / (2N) are the generalized
    eigenvectors of (K, M) on nodes 1..N with mu_j = 6k(1-cos th)/(c dx^2 (2+cos th)); the
    backward-Euler recurrence is a_j(n) = (a_j(n-1) + dt g_j(n)) / (1 + dt mu_j)."""
    N, NT, L, tT, kc, cc = 32, 64, 1.0, 0.5, 0.8, 1.3
    dx, dt = L / N, tT / NT
    q = wl.load_paper(N, NT, L, tT) * 1e-6
    b = oracle.assemble_load(N, NT, dx, q)
    u = oracle.exact(N, NT, L, tT, np.full(N, kc), np.full(N, cc), b)
    i = np.arange(1, N + 1)
    th = (2 * np.arange(1, N + 1) - 1) * np.pi / (2 * N)
    V = np.sin(np.outer(i, th))  # columns v_j
    mu = 6 * kc * (1 - np.cos(th)) / (cc * dx * dx * (2 + np.cos(th)))
    M, _ = dense.global_mk(N, dx, np.full(N, kc), np.full(N, cc))
    Mi = M[1:, 1:]
    nrm = np.einsum("ij,ik,kj->j", V, Mi, V)
    a = np.zeros(N)
    ref = np.zeros((NT + 1, N + 1))
    for n in range(1, NT + 1):
        g = V.T @ b[n, 1:] / nrm
        a = (a + dt * g) / (1 + dt * mu)
        ref[n, 1:] = V @ a
    np.testing.assert_allclose(u, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


# ---------------------------------------------------------------- planner (Alg. 3/4, Sec. 5.1)

@pytest.mark.parametrize("prob", ["problem7", "problem8"])
def test_lambda_eff_printed_values(prob):
    g = _gold("lambda_eff_sec5.json")[prob]
    p = wl.paper_problem(int(prob[-1]), tT=g["tT"])
    k, c = oracle.simp(p["chi"], p["simp"])
    H = oracle.Hierarchy(p["N"], p["NT"], p["L"], p["tT"], k, c, num_levels=1)
    assert round(H.levels[0]["lambda_eff"], g["digits"]) == g["lambda_eff"]


def test_alg3_path_uniform_material():
    # k = c = 1, L = 1, N = 64, NT = 64, tT chosen so that lambda = 2 on level 1:
    # x: 2 -> 0.5 -> 0.125 (< 0.25: t) -> 0.25 (not < 0.25: x) -> 0.0625 (t) -> 0.125 (t)
    N = NT = 64
    tT = 2.0 * NT / N ** 2
    H = oracle.Hierarchy(N, NT, 1.0, tT, np.ones(N), np.ones(N), num_levels=7)
    assert H.path() == "xxtxtt"
    lam = [lv["lambda_eff"] for lv in H.levels]
    np.testing.assert_allclose(lam, [2, 0.5, 0.125, 0.25, 0.0625, 0.125, 0.25], rtol=1e-14)


def test_alg4_min_elements_forces_t():
    N = NT = 64
    tT = 2.0 * NT / N ** 2 * 64  # lambda = 128: pure x-coarsening under Alg. 3
    H3 = oracle.Hierarchy(N, NT, 1.0, tT, np.ones(N), np.ones(N), num_levels=6)
    H4 = oracle.Hierarchy(N, NT, 1.0, tT, np.ones(N), np.ones(N), num_levels=6, min_nel=16)
    assert H3.path() == "xxxxx"
    assert H4.path() == "xxttt"  # N/2 < 16 once N = 16


def test_coarse_material_rules():
    N, NT = 8, 4
    k, c = _rand_material(21, N, contrast=1e5)
    for reasm, expect in [("R", 2 * k[0::2] * k[1::2] / (k[0::2] + k[1::2])), ("K", (k[0::2] + k[1::2]) / 2)]:
        H = oracle.Hierarchy(N, NT, 1.0, 1e-6, k, c, num_levels=2, reassembly=reasm, lambda_crit=0.0)
        assert H.path() == "x"
        np.testing.assert_allclose(H.levels[1]["k"], expect, rtol=1e-14)
        np.testing.assert_allclose(H.levels[1]["c"], (c[0::2] + c[1::2]) / 2, rtol=1e-15)
    H = oracle.Hierarchy(N, NT, 1.0, 1e-9, k, c, num_levels=2, lambda_crit=1e300)
    assert H.path() == "t"
    np.testing.assert_array_equal(H.levels[1]["k"], k)
    assert H.levels[1]["dt"] == pytest.approx(2e-9 / NT * 1.0, rel=1e-15)


def test_design_dependent_vs_fixed_deff():
    p = wl.paper_problem(7, tT=10.0)
    k, c = oracle.simp(p["chi"], p["simp"])
    s = p["simp"]
    deff = np.sqrt(s[0] / s[2] * s[1] / s[3])  # Sec. 7.2: sqrt(D_SIMP(0) D_SIMP(1))
    Hf = oracle.Hierarchy(256, 256, p["L"], p["tT"], k, c, num_levels=6, deff_fixed=deff)
    Hd = oracle.Hierarchy(256, 256, p["L"], p["tT"], k, c, num_levels=6)
    assert Hf.levels[0]["lambda_eff"] == pytest.approx(Hd.levels[0]["lambda_eff"], rel=1e-12)
    lam = [lv["lambda_eff"] for lv in Hf.levels]
    for l, lv in enumerate(Hf.levels[:-1]):  # fixed D_eff: lambda scales only with dt/dx^2
        f = 4.0 if lv["next"] == oracle.XCOARSEN else 0.5
        assert lam[l + 1] == pytest.approx(lam[l] / f, rel=1e-14)


# ---------------------------------------------------------------- transfer operators (Sec. 3.1)

@pytest.mark.parametrize("kind,interp", [("x", "C"), ("t", "C"), ("x", "B"), ("t", "B")])
def test_prolong_restrict_match_kronecker(kind, interp):
    N, NT = 8, 8
    k, c = _rand_material(4, N)
    lc = 1e300 if kind == "t" else 0.0
    H = oracle.Hierarchy(N, NT, 1.0, 1.0, k, c, num_levels=2, lambda_crit=lc, interp=interp)
    assert H.path() == kind
    P, s = dense.prolongation(N, NT, kind, interp)
    z = _rand_vec(8, H.shape(1))
    u = _rand_vec(9, H.shape(0))
    np.testing.assert_allclose(H.prolong_add(0, z, u).ravel(), u.ravel() + P @ z.ravel(), rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(H.restrict(0, u).ravel(), s * P.T @ u.ravel(), rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("interp", ["C", "B"])
def test_time_prolongation_reproduces_polynomials(interp):
    """Sec. 3.1 / 5.1: the causal t-prolongation copies a coarse value to the fine levels
    2m and 2m+1 (it reproduces functions constant in time), the bilinear one interpolates
    linearly between t_2m and t_2m+2 (it reproduces every function linear in t).  The
    restriction is R = 1/2 P^T, so <R r, z> = 1/2 <r, P z> for all r, z."""
    N, NT, tT = 6, 16, 2.0
    k, c = _rand_material(5, N)
    H = oracle.Hierarchy(N, NT, 1.0, tT, k, c, num_levels=2, lambda_crit=1e300, interp=interp)
    assert H.path() == "t"
    tc = np.arange(NT // 2 + 1) * (2.0 * tT / NT)
    tf = np.arange(NT + 1) * (tT / NT)
    a, b = wl.uniform(61, N + 1), wl.uniform(62, N + 1) - 0.5
    zc = a[None, :] + 0.0 * tc[:, None]
    np.testing.assert_allclose(H.prolong_add(0, zc, np.zeros((NT + 1, N + 1))), a[None, :] + 0.0 * tf[:, None],
                               rtol=1e-15, atol=0)
    zl = a[None, :] + b[None, :] * tc[:, None]
    fine = H.prolong_add(0, zl, np.zeros((NT + 1, N + 1)))
    lin = a[None, :] + b[None, :] * tf[:, None]
    if interp == "B":
        np.testing.assert_allclose(fine, lin, rtol=1e-14, atol=1e-15)
    else:  # causal: fine row 2m+1 holds the value of t_2m, one fine step behind
        np.testing.assert_allclose(fine[0::2], lin[0::2], rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(fine[1::2], lin[0:-1:2], rtol=1e-14, atol=1e-15)
    r = _rand_vec(63, H.shape(0))
    z = _rand_vec(64, H.shape(1))
    lhs = np.sum(H.restrict(0, r) * z)
    rhs = 0.5 * np.sum(r * H.prolong_add(0, z, np.zeros(H.shape(0))))
    assert lhs == pytest.approx(rhs, rel=1e-13)


def test_bilinear_t_restriction_by_hand():
    """Sec. 5.1 bilinear t-restriction on one column: b_c[m] = 1/2 (r[2m] + 1/2 r[2m-1] +
    1/2 r[2m+1]), the missing rows -1 and NT+1 dropped."""
    N, NT = 2, 8
    H = oracle.Hierarchy(N, NT, 1.0, 1.0, np.ones(N), np.ones(N), num_levels=2, lambda_crit=1e300, interp="B")
    r = np.zeros((NT + 1, N + 1))
    r[:, 1] = np.arange(1.0, NT + 2.0)  # r[n] = n + 1
    got = H.restrict(0, r)[:, 1]
    expect = [0.5 * (1.0 + 0.5 * 2.0), 0.5 * (3.0 + 0.5 * 2.0 + 0.5 * 4.0), 0.5 * (5.0 + 0.5 * 4.0 + 0.5 * 6.0),
              0.5 * (7.0 + 0.5 * 6.0 + 0.5 * 8.0), 0.5 * (9.0 + 0.5 * 8.0)]
    np.testing.assert_allclose(got, expect, rtol=1e-15)


# ---------------------------------------------------------------- SIMP material model (Sec. 2.1)

def test_simp_hand_values():
    """k = k_ins + (k_con - k_ins) chi^p_k, c = c_ins + (c_con - c_ins) chi^p_c at points
    worked out by hand, with p_k != p_c so that a swapped exponent fails."""
    s6 = [1e-3, 1.0, 0.2, 1.5, 3.0, 2.0]
    chi = np.array([0.0, 0.25, 0.5, 1.0])
    k, c = oracle.simp(chi, s6)
    # chi^3 = 0, 1/64, 1/8, 1; chi^2 = 0, 1/16, 1/4, 1; k_con - k_ins = 0.999, c_con - c_ins = 1.3
    np.testing.assert_allclose(k, [1e-3, 0.016609375, 0.125875, 1.0], rtol=1e-15)
    np.testing.assert_allclose(c, [0.2, 0.28125, 0.525, 1.5], rtol=1e-15)
    k2, c2 = oracle.simp(np.array([0.5]), [2.0, 10.0, 3.0, 7.0, 1.0, 4.0])  # p_k = 1: linear in chi
    assert k2[0] == pytest.approx(6.0, rel=1e-15) and c2[0] == pytest.approx(3.25, rel=1e-15)


# ---------------------------------------------------------------- D-reassembly (Sec. 5.1)

def test_design_reassembly_levels_match_dense():
    """D-reassembly: on x-coarsening the coarse design value is the mean of the pair and
    the SIMP model is re-applied; t-coarsening keeps chi.  Level by level against the dense
    brute force, and by hand on one pair: chi = (0.2, 0.6) gives simp(0.4), which differs
    from both the arithmetic (K) and the harmonic (R) mean of the pair's k."""
    N, NT = 16, 16
    chi = 0.05 + 0.9 * wl.uniform(71, N)
    chi[0], chi[1] = 0.2, 0.6
    s6 = [1e-4, 1.0, 0.3, 1.0, 3.0, 2.0]
    k, c = oracle.simp(chi, s6)
    H = oracle.Hierarchy(N, NT, 1.0, 0.05, k, c, chi=chi, simp6=s6, reassembly="D", max_coarse_dofs=10)
    path = H.path()
    assert "x" in path and "t" in path
    D = dense.DenseHierarchy(N, NT, 1.0, 0.05, k, c, path, reassembly="D", chi=chi, simp6=s6)
    for l, lv in enumerate(D.levels):
        np.testing.assert_allclose(H.levels[l]["k"], lv["k"], rtol=1e-14)
        np.testing.assert_allclose(H.levels[l]["c"], lv["c"], rtol=1e-14)
    first_x = path.index("x") + 1
    k04 = 1e-4 + (1.0 - 1e-4) * 0.4 ** 3
    assert H.levels[first_x]["k"][0] == pytest.approx(k04, rel=1e-14)
    assert H.levels[first_x]["c"][0] == pytest.approx(0.3 + 0.7 * 0.16, rel=1e-14)
    ka, kh = (k[0] + k[1]) / 2, 2 * k[0] * k[1] / (k[0] + k[1])
    assert abs(k04 - ka) > 0.01 * k04 and abs(k04 - kh) > 0.01 * k04


@pytest.mark.parametrize("adj", [False, True])
def test_design_reassembly_vcycle_matches_dense(adj):
    N, NT = 16, 16
    chi = 0.05 + 0.9 * wl.uniform(72, N)
    s6 = [1e-3, 1.0, 0.5, 1.0, 3.0, 1.0]
    k, c = oracle.simp(chi, s6)
    deff = np.sqrt((k / c).min() * (k / c).max())
    tT = 0.5 * (1.0 / N) ** 2 / deff * NT
    H = oracle.Hierarchy(N, NT, 1.0, tT, k, c, chi=chi, simp6=s6, reassembly="D", max_coarse_dofs=20, nu=3)
    path = H.path()
    assert len(path) >= 2 and "x" in path
    D = dense.DenseHierarchy(N, NT, 1.0, tT, k, c, path, reassembly="D", chi=chi, simp6=s6)
    b = _rand_vec(33, H.shape(0))
    u = np.zeros(H.shape(0))
    ud = u.ravel().copy()
    for cyc in range(3):
        u = H.vcycle(u, b, adj=adj)
        ud = D.vcycle(0, ud, b.ravel(), nu=3, adj=adj)
        np.testing.assert_allclose(u.ravel(), ud, rtol=0, atol=1e-12 * np.abs(ud).max())


# ---------------------------------------------------------------- V-cycle (Alg. 1) vs dense brute force

@pytest.mark.parametrize("N,NT,lam", [(8, 8, 2.0), (16, 8, 0.05), (8, 16, 0.3), (16, 16, 1.0)])
@pytest.mark.parametrize("reasm", ["R", "K"])
@pytest.mark.parametrize("adj", [False, True])
@pytest.mark.parametrize("interp", ["C", "B"])
def test_vcycle_matches_dense_bruteforce(N, NT, lam, reasm, adj, interp):
    k, c = _rand_material(N + NT, N, contrast=1e3)
    deff = np.sqrt((k / c).min() * (k / c).max())
    tT = lam * (1.0 / N) ** 2 / deff * NT
    H = oracle.Hierarchy(N, NT, 1.0, tT, k, c, reassembly=reasm, max_coarse_dofs=20, nu=3, interp=interp)
    path = H.path()
    assert len(path) >= 2
    D = dense.DenseHierarchy(N, NT, 1.0, tT, k, c, path, reassembly=reasm, interp=interp)
    b = _rand_vec(31, H.shape(0))
    u = np.zeros(H.shape(0))
    ud = u.ravel().copy()
    for cyc in range(3):
        u = H.vcycle(u, b, adj=adj)
        ud = D.vcycle(0, ud, b.ravel(), nu=3, adj=adj)
        np.testing.assert_allclose(u.ravel(), ud, rtol=0, atol=1e-12 * np.abs(ud).max())


def test_level_operators_match_dense_on_every_level():
    N, NT = 16, 16
    k, c = _rand_material(77, N, contrast=1e4)
    H = oracle.Hierarchy(N, NT, 1.0, 0.02, k, c, max_coarse_dofs=10)
    D = dense.DenseHierarchy(N, NT, 1.0, 0.02, k, c, H.path())
    for l, lv in enumerate(D.levels):
        u = _rand_vec(40 + l, H.shape(l))
        np.testing.assert_allclose(H.apply(l, u).ravel(), lv["J"] @ u.ravel(), rtol=0,
                                   atol=1e-13 * np.abs(lv["J"]).max())
        assert H.levels[l]["W"] == pytest.approx(dense.w_diri(1.0 / lv["N"], 0.02 / lv["NT"], lv["k"], lv["c"]),
                                                 rel=1e-13)


# ---------------------------------------------------------------- solver loop and invariants

def test_rod_blocks_converges_to_exact_solution():
    cfg = wl.rod_blocks()
    N, NT = cfg["N"], cfg["NT"]
    H = oracle.Hierarchy(N, NT, cfg["L"], cfg["tT"], cfg["k"], cfg["c"])
    b = oracle.assemble_load(N, NT, cfg["L"] / N, cfg["q"])
    u, st, cyc, hist = H.solve(b, tol=1e-10)
    assert st == "converged" and hist[-1] < 1e-10 and cyc < 40
    ue = oracle.exact(N, NT, cfg["L"], cfg["tT"], cfg["k"], cfg["c"], b)
    assert np.abs(u - ue).max() <= 1e-8 * np.abs(ue).max()
    rho = (hist[-1] / hist[0]) ** (1.0 / cyc)  # Sec. 3.1 convergence factor estimate
    assert rho < 0.6


def test_linearity_of_the_cycle():
    cfg = wl.rod_blocks()
    N, NT = cfg["N"], cfg["NT"]
    H = oracle.Hierarchy(N, NT, cfg["L"], cfg["tT"], cfg["k"], cfg["c"])
    b = _rand_vec(3, H.shape(0))
    u1 = H.vcycle(np.zeros(H.shape(0)), b)
    u2 = H.vcycle(np.zeros(H.shape(0)), 1024.0 * b)  # power of two: scaling is exact
    np.testing.assert_array_equal(u2, 1024.0 * u1)


def test_adjoint_identity_and_cycle_counts():
    cfg = wl.random_design(N=64, NT=128)
    N, NT = cfg["N"], cfg["NT"]
    k, c = oracle.simp(cfg["chi"], cfg["simp"])
    dt = cfg["tT"] / NT
    b = oracle.assemble_load(N, NT, cfg["L"] / N, cfg["q"])
    u = oracle.exact(N, NT, cfg["L"], cfg["tT"], k, c, b)
    lam = oracle.exact(N, NT, cfg["L"], cfg["tT"], k, c, b * dt, adj=True)
    theta = oracle.objective(N, NT, dt, b, u)
    assert float(np.sum(lam * b)) == pytest.approx(theta, rel=1e-12)
    H = oracle.Hierarchy(N, NT, cfg["L"], cfg["tT"], k, c)
    _, s1, c1, _ = H.solve(b, tol=1e-10)
    lam2, s2, c2, _ = H.solve(b * dt, adj=True, tol=1e-10)
    assert s1 == s2 == "converged"
    assert abs(c1 - c2) <= max(3, 0.3 * c1)  # Sec. 7.3: adjoint counts close to primal
    assert np.abs(lam2 - lam).max() <= 1e-8 * np.abs(lam).max()


@pytest.mark.parametrize("penalise_c", [False, True])
def test_sensitivity_matches_central_differences(penalise_c):
    N, NT, L, tT = 24, 40, 1.0, 1.0
    chi = 0.1 + 0.8 * wl.uniform(12, N)
    s = wl.simp_params(1e-3, 1.0, 0.3 if penalise_c else 1.0, 1.0)
    q = wl.load_paper(N, NT, L, tT) * 1e-6
    dt = tT / NT
    b = oracle.assemble_load(N, NT, L / N, q)

    def theta(x):
        k, c = oracle.simp(x, s)
        return oracle.objective(N, NT, dt, b, oracle.exact(N, NT, L, tT, k, c, b))

    k, c = oracle.simp(chi, s)
    u = oracle.exact(N, NT, L, tT, k, c, b)
    lam = oracle.exact(N, NT, L, tT, k, c, b * dt, adj=True)
    g = oracle.sensitivity(N, NT, L, tT, chi, s, u, lam)
    # h = 1e-5: truncation error O(h^2) ~ 1e-10 relative, rounding noise ~ 100 eps Theta / h.
    h = 1e-5
    th0 = theta(chi)
    for e in [0, 1, 5, 11, N - 2, N - 1]:
        xp, xm = chi.copy(), chi.copy()
        xp[e] += h
        xm[e] -= h
        fd = (theta(xp) - theta(xm)) / (2 * h)
        assert g[e] == pytest.approx(fd, rel=1e-6, abs=100 * np.finfo(float).eps * th0 / h)


def test_solver_reports_divergence_and_max_cycles():
    cfg = wl.rod_blocks()
    N, NT = cfg["N"], cfg["NT"]
    b = oracle.assemble_load(N, NT, 1.0 / N, cfg["q"])
    H = oracle.Hierarchy(N, NT, 1.0, 1.0, cfg["k"], cfg["c"], nu=1)
    _, st, cyc, _ = H.solve(b, tol=1e-30, max_cycles=3)
    assert st == "max_cycles" and cyc == 3
    Hbad = oracle.Hierarchy(N, NT, 1.0, 1.0, cfg["k"], cfg["c"], omega=2.5)  # over-damped smoother
    _, st, _, hist = Hbad.solve(b, tol=1e-10, div_tol=1e3)
    assert st == "diverged" and hist[-1] > 1e3


def test_zero_rhs_gives_zero():
    H = oracle.Hierarchy(8, 8, 1.0, 1.0, np.ones(8), np.ones(8))
    u, st, cyc, _ = H.solve(np.zeros(H.shape(0)))
    assert st == "converged" and cyc == 0 and np.all(u == 0)


def _two_grid_factor(N, NT, L, tT, k, c, kind):
    lc = 1e300 if kind == "t" else 0.0
    H = oracle.Hierarchy(N, NT, L, tT, k, c, num_levels=2, lambda_crit=lc, reassembly="K")
    assert H.path() == kind
    b = oracle.assemble_load(N, NT, L / N, wl.load_paper(N, NT, L, tT))
    _, _, cyc, hist = H.solve(b, tol=1e-9, max_cycles=100)
    return (hist[-1] / hist[0]) ** (1.0 / cyc)


def test_two_grid_crossover_uniform_material():
    """Sec. 3.2: t-coarsening wins for small lambda, x-coarsening for large, crossing near 0.1."""
    g = _gold("coarsening_crossover.json")
    N = NT = 64
    rows = []
    for p in [-6, -4, -2, 0, 2]:
        lam = 2.0 ** p
        tT = lam * NT / N ** 2
        rows.append((lam, _two_grid_factor(N, NT, 1.0, tT, np.ones(N), np.ones(N), "x"),
                     _two_grid_factor(N, NT, 1.0, tT, np.ones(N), np.ones(N), "t")))
    for lam, fx, ft in rows:
        if lam <= g["lambda_crit_uniform"] / 4:
            assert ft < fx, (lam, fx, ft)
        if lam >= g["lambda_crit_uniform"] * 4:
            assert fx < ft, (lam, fx, ft)


@pytest.mark.slow
def test_two_grid_crossover_band_problem2():
    """Sec. 4: for problem 2 the x/t curves cross inside 2^-3 <= lambda_eff <= 2^-1."""
    g = _gold("coarsening_crossover.json")
    lo, hi = g["band_log2"]
    N = NT = 128
    p = wl.paper_problem(2, N=N, NT=NT)
    k, c = oracle.simp(p["chi"], p["simp"])
    d = k / c
    deff = np.sqrt(d.min() * d.max())
    res = {}
    for e in [lo - 2, hi + 2]:
        tT = 2.0 ** e * (1.0 / N) ** 2 / deff * NT
        res[e] = (_two_grid_factor(N, NT, 1.0, tT, k, c, "x"), _two_grid_factor(N, NT, 1.0, tT, k, c, "t"))
    assert res[lo - 2][1] < res[lo - 2][0]  # below the band: t-coarsening better
    assert res[hi + 2][0] < res[hi + 2][1]  # above the band: x-coarsening better


def _factor_problem7(N_l, interp):
    p = wl.paper_problem(7, tT=10.0)
    k, c = oracle.simp(p["chi"], p["simp"])
    H = oracle.Hierarchy(p["N"], p["NT"], p["L"], p["tT"], k, c, num_levels=N_l, interp=interp, reassembly="R")
    b = oracle.assemble_load(p["N"], p["NT"], p["L"] / p["N"], wl.load_paper(p["N"], p["NT"], p["L"], p["tT"]))
    _, st, cyc, hist = H.solve(b, tol=1e-9, max_cycles=100)
    return (hist[-1] / hist[0]) ** (1.0 / cyc)


@pytest.mark.slow
def test_causal_beats_bilinear_on_problem7_deep_hierarchies():
    """Sec. 5.2: on problem 7 the methods are close for N_l <= 5, and for N_l >= 6 causal
    interpolation converges noticeably faster than bilinear (CR vs BR here)."""
    for N_l in (6, 8):
        assert _factor_problem7(N_l, "C") < _factor_problem7(N_l, "B")


# ---------------------------------------------------------------------------------------
# Optimisation loop of Sec. 7 (projected-gradient stand-in for MMA)
# ---------------------------------------------------------------------------------------
def _projection_by_qp(y, lo, hi, vol):
    """Euclidean projection of y onto {lo <= x <= hi, mean(x) <= vol} by a generic QP solver."""
    from scipy.optimize import minimize

    n = y.size
    res = minimize(lambda x: 0.5 * np.sum((x - y) ** 2), np.clip(y, lo, hi), jac=lambda x: x - y,
                   bounds=list(zip(lo, hi)), constraints=[{"type": "ineq", "fun": lambda x: vol - x.mean(),
                                                            "jac": lambda x: -np.ones(n) / n}],
                   method="SLSQP", options={"ftol": 1e-15, "maxiter": 500})
    assert res.success, res.message
    return res.x


@pytest.mark.parametrize("case", range(6))
def test_design_update_is_the_projection(case):
    from oracle.optim import design_update

    rng = np.random.default_rng(40 + case)
    n = 24
    chi = rng.random(n) if case < 4 else np.full(n, 0.5)
    g = rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 3)
    if case == 5:
        g = -np.abs(g)  # every element wants more material: the volume bound is active
    vol, move = (0.5, 0.2) if case != 3 else (0.1, 0.05)  # case 3: move limit keeps mean above vol
    x, mu = design_update(chi, g, vol, move)
    y = chi - move * g / np.abs(g).max()
    lo, hi = np.maximum(0, chi - move), np.minimum(1, chi + move)
    assert np.all(x >= lo) and np.all(x <= hi)
    free = (x > lo + 1e-12) & (x < hi - 1e-12)
    np.testing.assert_allclose(x[free], y[free] - mu, rtol=0, atol=1e-14)
    if case == 3:
        assert mu == 2.0 and np.array_equal(x, lo)
        return
    if mu > 0:
        assert abs(x.mean() - vol) < 1e-14
        np.testing.assert_allclose(x, _projection_by_qp(y, lo, hi, vol), rtol=0, atol=1e-7)
    else:
        assert x.mean() <= vol
        np.testing.assert_allclose(x, np.clip(y, lo, hi), rtol=0, atol=1e-15)


def test_design_update_special_cases():
    from oracle.optim import design_update

    chi = np.linspace(0.1, 0.6, 11)
    x, mu = design_update(chi, np.zeros(11), 0.5, 0.2)  # no gradient, constraint inactive
    assert mu == 0.0 and np.array_equal(x, chi)
    x, mu = design_update(np.full(8, 0.5), np.ones(8), 0.5, 0.2)  # uniform gradient: uniform step
    np.testing.assert_allclose(x, 0.3, rtol=0, atol=0)
    x, mu = design_update(np.full(8, 0.5), -np.ones(8), 0.5, 0.2)  # uniform step back onto the bound
    assert abs(mu - 0.2) < 1e-15 and np.allclose(x, 0.5, rtol=0, atol=1e-15)


def test_optimisation_loop_descends_on_problem7():
    """Problem 7's materials and load (Sec. 7.1) on a 32 x 32 grid: the design stays
    feasible and the compliance falls at every update from the uniform start."""
    from oracle.optim import optimize

    N = NT = 32
    p = wl.paper_problem(7, N=N, NT=NT)
    q = wl.load_paper(N, NT, p["L"], p["tT"])
    designs, thetas = optimize(N, NT, p["L"], p["tT"], p["simp"], q, iters=12)
    for x in designs:
        assert np.all((x >= 0) & (x <= 1)) and x.mean() <= 0.5 + 1e-14
    assert all(b < a for a, b in zip(thetas, thetas[1:]))
    assert thetas[-1] < 0.93 * thetas[0]


# ---------------------------------------------------------------------------------------
# Galerkin reassembly (P-method, Sec. 5.1): J_{l+1} = R_l J_l P_l
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("interp", ["C", "B"])
@pytest.mark.parametrize("lam", [0.02, 3.0])
def test_galerkin_sparse_levels_match_dense_products(interp, lam):
    from oracle.galerkin import GalerkinHierarchy

    N, NT = 8, 8
    rng = np.random.default_rng(90)
    k, c = 10.0 ** rng.uniform(-2, 0, N), 0.5 + rng.random(N)
    tT = lam * NT / N ** 2 / np.sqrt((k / c).min() * (k / c).max())
    G = GalerkinHierarchy(N, NT, 1.0, tT, k, c, interp=interp, num_levels=4)
    D = dense.DenseHierarchy(N, NT, 1.0, tT, k, c, G.path, interp=interp, reassembly="P")
    for l in range(G.nlevels):
        np.testing.assert_allclose(G.levels[l]["J"].toarray(), D.levels[l]["J"], rtol=0, atol=1e-12 * np.abs(D.levels[l]["J"]).max())
    b = rng.standard_normal(G.shape(0))
    for adj in (False, True):
        want = D.vcycle(0, np.zeros(b.size), b.ravel(), adj=adj)
        got = G.vcycle(np.zeros(G.shape(0)), b, adj=adj)
        np.testing.assert_allclose(got.ravel(), want, rtol=0, atol=1e-11 * np.abs(want).max())


@pytest.mark.parametrize("interp", ["C", "B"])
def test_galerkin_t_coarsening_blocks_by_hand(interp):
    """k = c = 1, N = 3, NT = 4, one t-coarsening.  With A' and B' the same-step and
    previous-step blocks of a time row (node 0 masked to the Dirichlet row W e_0), the fine
    rows are W I (n = 0), A' (n = 1), B' | A' (n >= 2).  Causal P = [1; 1] per pair and
    R = P^T / 2 give coarse rows (W I + A')/2; B'/2 | A' + B'/2; B'/2 | A'/2.  Bilinear P
    (1/2, 1, 1/2) and R = P^T / 2 give for coarse row 1: A'/8 + B'/4 | 3A'/4 + B'/2 | A'/8."""
    from oracle.galerkin import GalerkinHierarchy

    N, NT, tT = 3, 4, 0.01
    k, c = np.ones(N), np.ones(N)
    dx, dt = 1.0 / N, tT / NT
    M, K = dense.global_mk(N, dx, k, c)
    W = dense.w_diri(dx, dt, k, c)
    E = np.diag([0.0, 1.0, 1.0, 1.0])
    I = np.eye(N + 1)
    A = E @ (M / dt + K) @ E + W * (I - E)
    B = E @ (-M / dt) @ E
    G = GalerkinHierarchy(N, NT, 1.0, tT, k, c, interp=interp, num_levels=2)
    assert G.path == "t"
    Jc = G.levels[1]["J"].toarray()
    blk = lambda m, mp: Jc[m * 4:(m + 1) * 4, mp * 4:(mp + 1) * 4]  # noqa: E731
    Z = np.zeros((4, 4))
    if interp == "C":
        want = {(0, 0): (W * I + A) / 2, (0, 1): Z, (1, 0): B / 2, (1, 1): A + B / 2, (1, 2): Z,
                (2, 1): B / 2, (2, 2): A / 2}
    else:
        want = {(1, 0): A / 8 + B / 4, (1, 1): 3 * A / 4 + B / 2, (1, 2): A / 8}
    for (m, mp), w in want.items():
        np.testing.assert_allclose(blk(m, mp), w, rtol=0, atol=1e-12 * W)


def test_galerkin_on_problem7_matches_the_paper():
    """Sec. 5.2, problem 7 (N = NT = 256): with bilinear interpolation the Galerkin
    hierarchy (BP) is stable up to 4 levels and blows up beyond; with causal interpolation
    (CP) the convergence factor stays within a few percent of the K-method's (CK)."""
    from oracle.galerkin import GalerkinHierarchy

    N = NT = 256
    p = wl.paper_problem(7, N=N, NT=NT)
    k, c = oracle.simp(p["chi"], p["simp"])
    b = oracle.assemble_load(N, NT, p["L"] / N, wl.load_paper(N, NT, p["L"], p["tT"]))

    def rho(H, nl):
        u, st, cyc, hist = H.solve(b, tol=1e-9, max_cycles=100)
        return st, (hist[-1] / hist[0]) ** (1.0 / max(cyc, 1))

    for nl in (4, 5, 6):
        st, r = rho(GalerkinHierarchy(N, NT, p["L"], p["tT"], k, c, interp="B", num_levels=nl), nl)
        if nl == 4:
            assert st == "converged" and r < 0.6
        else:
            assert st == "diverged" and r > 100.0
    for nl in (3, 5):
        st, r = rho(GalerkinHierarchy(N, NT, p["L"], p["tT"], k, c, interp="C", num_levels=nl), nl)
        stk, rk = rho(oracle.Hierarchy(N, NT, p["L"], p["tT"], k, c, reassembly="K", num_levels=nl), nl)
        assert st == stk == "converged" and abs(r - rk) < 0.05 * rk
