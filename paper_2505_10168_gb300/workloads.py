"""Seeded synthetic inputs for the STMG library and for its tests.

This module only draws numbers and lays out input fields: design fields, two-phase
conductivity blocks, element heat loads, serving request mixes.  It holds none of the
method's arithmetic (no material interpolation, no assembly, no operators), so that the
CUDA path and the CPU oracle can both be fed from it without sharing any of the method.

Random numbers come from splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15, then the output mix
z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27; z *= 0x94D049BB133111EB; z ^= z>>31.
A uniform double in [0, 1) is (z >> 11) * 2^-53.

Workloads (all with T = 0 at t = 0 and x = 0, adiabatic at x = L):

* ``rod_blocks``: L = 1, t_end = 1, 128 x 128, c = 1, conductivity in 16 blocks of 8
  elements, each block k = 1e-3 or 1 with probability 1/2 (seed 1), load q = 1.
* ``filtered_simp``: 4096 x 16384, design field chi ~ U(0,1) (seed 2) smoothed by a
  centred 16-element box filter (window [e-8, e+7], mean over the elements inside the
  domain), SIMP k_ins = 1e-4, k_con = 1, p_k = 3, c = 1; q = 1 on elements with
  x_e < 0.1, else 0.
* ``filtered_simp_high_contrast``: as filtered_simp with k_ins = 1e-6.
* ``random_design``: 1024 x 4096, chi ~ U(0.05, 1) (seed 4), k_ins = 1e-3, p_k = 3, c = 1,
  q = 1; 32 elements for finite differences drawn with seed 5 (the differentiation
  workload, solved with nu = 20).

Each returns a dict whose ``name`` states the field and the grid, e.g.
"filtered-simp-4096x16384".
* ``serving_requests``: 512 requests (seed 6), N log-uniform in [256, 4096] and NT
  log-uniform in [512, 16384], both rounded to multiples of 64; two-phase 8-element
  blocks with k in {k_min, 1}, k_min = 10^-U(3,6); forward or adjoint with p = 1/2;
  Poisson arrival gaps.
* ``paper_problem``: design fields and materials of the paper's problems 1-9
  (Sec. 4 Table of problems 1-6, Sec. 5.2 problems 7-9) and its test heat load (Sec. 3.1).
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n outputs of splitmix64 started from ``seed``, skipping ``offset`` outputs."""
    idx = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1) from splitmix64."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def box_filter(v: np.ndarray, width: int = 16) -> np.ndarray:
    """Centred moving average over [e - width/2, e + width/2 - 1], clipped to the domain."""
    n = v.size
    cs = np.concatenate([[0.0], np.cumsum(v)])
    e = np.arange(n)
    lo = np.maximum(e - width // 2, 0)
    hi = np.minimum(e + width // 2 - 1, n - 1)
    return (cs[hi + 1] - cs[lo]) / (hi - lo + 1)


def two_phase_blocks(seed: int, n: int, block: int, k_low: float, k_high: float = 1.0) -> np.ndarray:
    """Conductivity in blocks of ``block`` elements, each k_low or k_high with p = 1/2."""
    nb = (n + block - 1) // block
    pick = uniform(seed, nb) < 0.5
    kb = np.where(pick, k_low, k_high)
    return np.repeat(kb, block)[:n].copy()


def element_centres(N: int, L: float) -> np.ndarray:
    """x_e = (e + 1/2) dx (Sec. 2.2)."""
    return (np.arange(N) + 0.5) * (L / N)


def load_uniform(N: int, NT: int, value: float = 1.0) -> np.ndarray:
    """Element loads q[n, e] for time levels n = 0..NT (row 0 is never used)."""
    return np.full((NT + 1, N), value)


def load_left_strip(N: int, NT: int, L: float, x_end: float = 0.1) -> np.ndarray:
    """q = 1 on elements with x_e < x_end, else 0, at every time level."""
    row = (element_centres(N, L) < x_end).astype(np.float64)
    return np.broadcast_to(row, (NT + 1, N)).copy()


def load_paper(N: int, NT: int, L: float, tT: float) -> np.ndarray:
    """Test heat load of Sec. 3.1: (1 + cos(200[(x_e/L-1/2)^2 + (t_j/t_T-1/2)^2])) 1e6."""
    xe = element_centres(N, L) / L - 0.5
    tj = np.arange(NT + 1) * (tT / NT) / tT - 0.5
    return (1.0 + np.cos(200.0 * (xe[None, :] ** 2 + tj[:, None] ** 2))) * 1e6


def simp_params(k_ins, k_con, c_ins, c_con, p_k=3.0, p_c=2.0) -> np.ndarray:
    """Parameter vector (k_ins, k_con, c_ins, c_con, p_k, p_c) of the SIMP model."""
    return np.array([k_ins, k_con, c_ins, c_con, p_k, p_c], dtype=np.float64)


def rod_blocks():
    N = NT = 128
    k = two_phase_blocks(1, N, 8, 1e-3, 1.0)
    return dict(name="rod-blocks-%dx%d" % (N, NT), N=N, NT=NT, L=1.0, tT=1.0, k=k, c=np.ones(N), chi=None, simp=None,
                q=load_uniform(N, NT), tol=1e-10)


def _chi_filtered(seed, N):
    return box_filter(uniform(seed, N), 16)


def filtered_simp(N=4096, NT=16384, k_ins=1e-4, seed=2, name="filtered-simp"):
    chi = _chi_filtered(seed, N)
    return dict(name="%s-%dx%d" % (name, N, NT), N=N, NT=NT, L=1.0, tT=1.0, chi=chi, simp=simp_params(k_ins, 1.0, 1.0, 1.0),
                k=None, c=None, q=load_left_strip(N, NT, 1.0), tol=1e-8)


def filtered_simp_high_contrast(N=4096, NT=16384):
    return filtered_simp(N, NT, k_ins=1e-6, name="filtered-simp-kins1e-6")


def random_design(N=1024, NT=4096):
    chi = 0.05 + 0.95 * uniform(4, N)
    fd = np.sort(np.floor(uniform(5, 32) * N).astype(np.int64))
    return dict(name="random-design-%dx%d" % (N, NT), N=N, NT=NT, L=1.0, tT=1.0, chi=chi, simp=simp_params(1e-3, 1.0, 1.0, 1.0),
                k=None, c=None, q=load_uniform(N, NT), fd_elements=fd, theta_ref=1.0, tol=1e-10, nu=20)


def _round64(v):
    return int(max(64, 64 * round(v / 64.0)))


def serving_requests(n=512, seed=6, nx=(256, 4096), nt=(512, 16384), rate=1.0):
    """Request mix for the serving workload; ``rate`` is the mean arrivals per second."""
    u = uniform(seed, 6 * n).reshape(n, 6)
    reqs = []
    t = 0.0
    for r in range(n):
        N = _round64(math.exp(math.log(nx[0]) + u[r, 0] * (math.log(nx[1]) - math.log(nx[0]))))
        NT = _round64(math.exp(math.log(nt[0]) + u[r, 1] * (math.log(nt[1]) - math.log(nt[0]))))
        kmin = 10.0 ** -(3.0 + 3.0 * u[r, 2])
        adjoint = bool(u[r, 3] < 0.5)
        t += -math.log(1.0 - u[r, 4]) / rate
        reqs.append(dict(id=r, N=N, NT=NT, L=1.0, tT=1.0, kmin=kmin, adjoint=adjoint, arrival=t,
                         k_seed=1000003 * (seed + 1) + r))
    return reqs


def request_fields(req):
    """Conductivity, heat capacity and element load of one serving request."""
    N, NT = req["N"], req["NT"]
    k = two_phase_blocks(req["k_seed"], N, 8, req["kmin"], 1.0)
    return k, np.ones(N), load_uniform(N, NT)


# --- the paper's own test problems (inputs only) ---------------------------------------

def f01(v):
    """Clamp to [0, 1] (Sec. 4, the function f_01)."""
    return np.clip(v, 0.0, 1.0)


PROBLEMS_1_6 = {  # k_ins, c_ins, x_offset, (log2 t_T range)  -- Sec. 4 table
    1: (1e-2, 1.0, 0.5, (-10, -2)),
    2: (1e-4, 1.0, 0.5, (-7, 1)),
    3: (1e-4, 1.0, 0.15, (-7, 1)),
    4: (1e-4, 1.0, 0.85, (-7, 1)),
    5: (1.0, 1e-4, 0.5, (-20, -12)),
    6: (1e-4, 1e-4, 0.5, (-12, -4)),
}

# Sec. 5.2 material table: aluminium conductor and epoxy insulator (k in W/m/K, c in J/m^3/K)
AL_EPOXY = dict(k_con=2.14e2, c_con=2.41e6, k_ins=1.97e-1, c_ins=1.67e6)


def paper_problem(num, N=256, NT=256, tT=None, F=0.03):
    """Design field, SIMP parameters and domain of problems 1-9."""
    if num in PROBLEMS_1_6:
        k_ins, c_ins, xoff, _ = PROBLEMS_1_6[num]
        L = 1.0
        chi = f01(0.5 - 10.0 * (element_centres(N, L) - xoff))
        s = simp_params(k_ins, 1.0, c_ins, 1.0)
        return dict(N=N, NT=NT, L=L, tT=tT if tT is not None else 1.0, chi=chi, simp=s)
    L = 0.1
    m = AL_EPOXY
    s = simp_params(m["k_ins"], m["k_con"], m["c_ins"], m["c_con"])
    xe = element_centres(N, L)
    if num == 7:
        chi = f01(0.5 - (5.0 / L) * (xe - L / 2.0))
        tdef = 10.0
    elif num == 8:
        chi = f01(np.abs((xe - L / 2.0) / L) * 2.0 / F - 1.0)
        tdef = 100.0
    elif num == 9:
        chi = 1.0 - f01(np.abs((xe - L / 2.0) / L) * 2.0 / F - 1.0)
        tdef = 100.0
    else:
        raise ValueError(num)
    return dict(N=N, NT=NT, L=L, tT=tT if tT is not None else tdef, chi=chi, simp=s)
