"""FP64 CPU oracle for the space-time multigrid method (arXiv 2505.10168).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product library never imports
this package, and this package never imports the product library.

Two independent parts:

* ``stmg_oracle.c`` (loaded here through ctypes): the structured oracle -- element-by-
  element operator application (Sec. 2.2, Appendix A), damped Jacobi (Sec. 3.1),
  prolongation/restriction from the stencil columns (Sec. 3.1, 5.1), the coarsening
  strategy (Alg. 3/4), the V-cycle (Alg. 1), exact implicit time stepping, the
  adjoint (Sec. 7.2) and the sensitivity.
* ``dense.py``: dense-matrix brute force for tiny grids, used only to pin the above.

Arrays are float64 numpy arrays; a space-time vector has shape (NT+1, N+1)
(time level, node).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stmg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

INTERP = {"C": 0, "B": 1}
REASM = {"K": 0, "R": 1, "D": 2}
XCOARSEN, TCOARSEN = 1, 2
STATUS = {0: "converged", 1: "diverged", 2: "max_cycles", 3: "einval"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction: products rounded as written)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Opts(C.Structure):
    _fields_ = [
        ("nu", C.c_int),
        ("omega", C.c_double),
        ("lambda_crit", C.c_double),
        ("interp", C.c_int),
        ("reassembly", C.c_int),
        ("min_nel", C.c_int),
        ("num_levels", C.c_int),
        ("max_levels", C.c_int),
        ("max_coarse_dofs", C.c_longlong),
        ("deff_fixed", C.c_double),
    ]


_lib = None
_dp = C.POINTER(C.c_double)


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        vp = C.c_void_p
        lib.or_create.restype = vp
        lib.or_create.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp, _dp, _dp, C.POINTER(_Opts)]
        lib.or_destroy.argtypes = [vp]
        lib.or_nlevels.argtypes = [vp]
        lib.or_level_info.argtypes = [vp, C.c_int, C.POINTER(C.c_int), _dp]
        lib.or_level_material.argtypes = [vp, C.c_int, _dp, _dp]
        lib.or_apply.argtypes = [vp, C.c_int, C.c_int, _dp, _dp]
        lib.or_diag.argtypes = [vp, C.c_int, _dp]
        lib.or_residual.argtypes = [vp, C.c_int, C.c_int, _dp, _dp, _dp]
        lib.or_smooth.argtypes = [vp, C.c_int, C.c_int, C.c_int, _dp, _dp]
        lib.or_restrict.argtypes = [vp, C.c_int, _dp, _dp]
        lib.or_prolong_add.argtypes = [vp, C.c_int, _dp, _dp]
        lib.or_exact_level.argtypes = [vp, C.c_int, C.c_int, _dp, _dp]
        lib.or_vcycle.argtypes = [vp, C.c_int, _dp, _dp]
        lib.or_solve.restype = C.c_int
        lib.or_solve.argtypes = [vp, C.c_int, _dp, _dp, C.c_int, C.c_double, C.c_double, C.c_int,
                                 C.POINTER(C.c_int), _dp]
        lib.or_exact.restype = C.c_int
        lib.or_exact.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp, C.c_int, _dp, _dp]
        lib.or_objective.restype = C.c_double
        lib.or_objective.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp]
        lib.or_sensitivity.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp, _dp, _dp, _dp]
        lib.or_simp.argtypes = [C.c_int, _dp, _dp, _dp, _dp]
        lib.or_assemble_load.argtypes = [C.c_int, C.c_int, C.c_double, _dp, _dp]
        _lib = lib
    return _lib


def _p(a):
    """Pointer to a C-contiguous float64 array (None -> NULL)."""
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle arrays must be contiguous float64"
    return a.ctypes.data_as(_dp)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def simp(chi, simp6):
    """Sec. 2.1 SIMP interpolation: returns (k, c) per element."""
    chi = _f64(chi)
    s = _f64(simp6)
    k = np.empty_like(chi)
    c = np.empty_like(chi)
    _load().or_simp(chi.size, _p(chi), _p(s), _p(k), _p(c))
    return k, c


def assemble_load(N, NT, dx, q):
    """Nodal load b = B b_Neu from element loads q[(NT+1), N] (Sec. 2.2, Appendix A)."""
    q = _f64(q).reshape(NT + 1, N)
    b = np.empty((NT + 1, N + 1))
    _load().or_assemble_load(N, NT, dx, _p(q), _p(b))
    return b


def exact(N, NT, L, tT, k, c, b, adj=False):
    """Exact discrete solution of J u = b (adj: J^T u = b) by implicit time stepping."""
    k, c, b = _f64(k), _f64(c), _f64(b).reshape(NT + 1, N + 1)
    u = np.empty((NT + 1, N + 1))
    _load().or_exact(N, NT, L, tT, _p(k), _p(c), int(adj), _p(b), _p(u))
    return u


def objective(N, NT, dt, b, u, theta_ref=1.0):
    """Theta = b^T u dt / Theta_ref (Sec. 7.1)."""
    return _load().or_objective(N, NT, dt, theta_ref, _p(_f64(b)), _p(_f64(u)))


def sensitivity(N, NT, L, tT, chi, simp6, u, lam):
    """dTheta/dchi_e = -Lambda^T (dJ/dchi_e) u (discrete adjoint, Sec. 7.2)."""
    g = np.empty(N)
    _load().or_sensitivity(N, NT, L, tT, _p(_f64(chi)), _p(_f64(simp6)), _p(_f64(u)), _p(_f64(lam)), _p(g))
    return g


class Hierarchy:
    """Oracle STMG hierarchy: Alg. 3/4 planner plus per-level operators and Alg. 1."""

    def __init__(self, N, NT, L, tT, k, c, *, chi=None, simp6=None, nu=5, omega=0.5, lambda_crit=0.25,
                 interp="C", reassembly="R", min_nel=0, num_levels=0, max_levels=30, max_coarse_dofs=512,
                 deff_fixed=0.0):
        lib = _load()
        self.N, self.NT, self.L, self.tT = N, NT, L, tT
        o = _Opts(nu, omega, lambda_crit, INTERP[interp], REASM[reassembly], min_nel, num_levels, max_levels,
                  max_coarse_dofs, deff_fixed)
        self._k, self._c, self._chi, self._s = _f64(k), _f64(c), _f64(chi), _f64(simp6)
        h = lib.or_create(N, NT, L, tT, _p(self._k), _p(self._c), _p(self._chi), _p(self._s), C.byref(o))
        if not h:
            raise ValueError("oracle rejected the problem definition")
        self._h = h
        self.nlevels = lib.or_nlevels(h)
        self.levels = []
        for l in range(self.nlevels):
            ints = (C.c_int * 3)()
            dbl = (C.c_double * 4)()
            lib.or_level_info(h, l, ints, dbl)
            kk = np.empty(ints[0])
            cc = np.empty(ints[0])
            lib.or_level_material(h, l, _p(kk), _p(cc))
            self.levels.append(dict(N=ints[0], NT=ints[1], next=ints[2], dx=dbl[0], dt=dbl[1], W=dbl[2],
                                    lambda_eff=dbl[3], k=kk, c=cc))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_destroy(h)
            self._h = None

    def shape(self, l):
        lv = self.levels[l]
        return (lv["NT"] + 1, lv["N"] + 1)

    def apply(self, l, u, adj=False):
        u = _f64(u).reshape(self.shape(l))
        y = np.empty_like(u)
        _load().or_apply(self._h, l, int(adj), _p(u), _p(y))
        return y

    def diag(self, l):
        d = np.empty(self.shape(l))
        _load().or_diag(self._h, l, _p(d))
        return d

    def residual(self, l, u, b, adj=False):
        u, b = _f64(u).reshape(self.shape(l)), _f64(b).reshape(self.shape(l))
        r = np.empty_like(u)
        _load().or_residual(self._h, l, int(adj), _p(u), _p(b), _p(r))
        return r

    def smooth(self, l, u, b, nsweeps, adj=False):
        u = _f64(u).reshape(self.shape(l)).copy()
        b = _f64(b).reshape(self.shape(l))
        _load().or_smooth(self._h, l, int(adj), nsweeps, _p(u), _p(b))
        return u

    def restrict(self, l, r):
        r = _f64(r).reshape(self.shape(l))
        bc = np.empty(self.shape(l + 1))
        _load().or_restrict(self._h, l, _p(r), _p(bc))
        return bc

    def prolong_add(self, l, z, u):
        z = _f64(z).reshape(self.shape(l + 1))
        u = _f64(u).reshape(self.shape(l)).copy()
        _load().or_prolong_add(self._h, l, _p(z), _p(u))
        return u

    def exact_level(self, l, b, adj=False):
        b = _f64(b).reshape(self.shape(l))
        u = np.empty_like(b)
        _load().or_exact_level(self._h, l, int(adj), _p(b), _p(u))
        return u

    def vcycle(self, u, b, adj=False):
        u = _f64(u).reshape(self.shape(0)).copy()
        b = _f64(b).reshape(self.shape(0))
        _load().or_vcycle(self._h, int(adj), _p(u), _p(b))
        return u

    def solve(self, b, adj=False, tol=1e-10, div_tol=1e9, max_cycles=100, u0=None):
        """Sec. 3.1 solver loop; returns (u, status, cycles, residual history)."""
        b = _f64(b).reshape(self.shape(0))
        u = np.zeros(self.shape(0)) if u0 is None else _f64(u0).reshape(self.shape(0)).copy()
        hist = np.zeros(max_cycles + 1)
        cyc = C.c_int(0)
        st = _load().or_solve(self._h, int(adj), _p(b), _p(u), int(u0 is not None), tol, div_tol, max_cycles,
                              C.byref(cyc), _p(hist))
        return u, STATUS[st], cyc.value, hist[: cyc.value + 1].copy()

    def path(self):
        """Coarsening path as a string of 'x'/'t' (one letter per coarsening)."""
        return "".join({XCOARSEN: "x", TCOARSEN: "t"}[lv["next"]] for lv in self.levels[:-1])
