"""GB300-native space-time multigrid (STMG) for 1D transient heat conduction.

Python face of the C ABI in include/stmg.h (libstmg.so): the method runs entirely in the
library's CUDA kernels; this module only marshals arguments.  See ``Solver`` for the
handle API and ``workloads`` for the seeded synthetic inputs.
"""
from __future__ import annotations

import ctypes as C

from . import _binding as B
from ._binding import STMGError

__all__ = ["Solver", "STMGError", "simp", "deff_simp", "lib", "kernel_launches"]

lib = B.lib


def kernel_launches():
    """Kernels the library has launched in this process (``stmg_kernel_launches``)."""
    return int(B.lib().stmg_kernel_launches())


def simp(chi, simp6, k, c, stream=None):
    """SIMP material model (Sec. 2.1) on the device: chi -> k, c (torch CUDA tensors)."""
    s = (C.c_double * 6)(*[float(v) for v in simp6])
    st = B.lib().stmg_simp(B.numel(chi), B.ptr(chi), s, B.ptr(k), B.ptr(c),
                           stream if stream is not None else B.default_stream())
    B.check(st)
    return k, c


def deff_simp(simp6):
    """Design-independent D_eff of Sec. 7.2 for the SIMP parameters (``stmg_deff_simp``)."""
    s = (C.c_double * 6)(*[float(v) for v in simp6])
    out = C.c_double(0.0)
    B.check(B.lib().stmg_deff_simp(s, C.byref(out)))
    return out.value


def design_update(chi, g, vol_frac, move, out, stream=None):
    """Projected-gradient design update of the optimisation loop (Sec. 7.2; stand-in for
    MMA): out = clamp(chi - move g / max|g| - mu, max(0, chi - move), min(1, chi + move))
    with the volume shift mu >= 0 (``stmg_design_update``).  out may be chi."""
    st = B.lib().stmg_design_update(B.numel(chi), B.ptr(chi), B.ptr(g), float(vol_frac), float(move), B.ptr(out),
                                    stream if stream is not None else B.default_stream())
    B.check(st)
    return out


class Solver:
    """One STMG hierarchy (``stmg_create``) on one CUDA stream.

    Space-time arrays have (nt+1) x (nel+1) float64 values (time level major); element
    arrays have nel values; element loads (nt+1) x nel.  Arrays can live on the GPU or
    on the host.  Options are the fields of ``stmg_opts`` (nu, omega, lambda_crit,
    reassembly 'R'/'K', min_nel, num_levels, max_levels, max_coarse_dofs, deff_fixed,
    precision 'fp64'/'mixed', tol, div_tol, max_cycles).
    """

    def __init__(self, nel, nt, L, t_end, k=None, c=None, stream=None, chi=None, simp6=None, **opts):
        """k, c: element material; or chi + simp6 for a design-field hierarchy (D-reassembly)."""
        self.nel, self.nt, self.L, self.t_end = int(nel), int(nt), float(L), float(t_end)
        self.opts = B.make_opts(**opts)
        self.stream = stream if stream is not None else B.default_stream()
        h = C.c_void_p()
        if chi is not None:
            s6 = (C.c_double * 6)(*[float(v) for v in simp6])
            st = B.lib().stmg_create_design(C.byref(h), self.nel, self.nt, self.L, self.t_end, B.ptr(chi), s6,
                                            C.byref(self.opts), self.stream)
        else:
            st = B.lib().stmg_create(C.byref(h), self.nel, self.nt, self.L, self.t_end, B.ptr(k), B.ptr(c),
                                     C.byref(self.opts), self.stream)
        B.check(st)
        self._h = h

    # -- lifetime --------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            B.lib().stmg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    @property
    def shape(self):
        return (self.nt + 1, self.nel + 1)

    @property
    def dt(self):
        return self.t_end / self.nt

    # -- solves ----------------------------------------------------------------------
    def update_material(self, k, c):
        B.check(B.lib().stmg_update_material(self._h, B.ptr(k), B.ptr(c)), self._h)

    def update_design(self, chi):
        B.check(B.lib().stmg_update_design(self._h, B.ptr(chi)), self._h)

    def assemble_load(self, q, b):
        B.check(B.lib().stmg_assemble_load(self._h, B.ptr(q), B.ptr(b)), self._h)
        return b

    def solve(self, u, q=None, b=None, warm=False):
        """J u = b (or the load q).  Returns (status, cycles, relres); u is written."""
        cyc, rel = C.c_int(0), C.c_double(0.0)
        st = B.lib().stmg_solve(self._h, B.ptr(q), B.ptr(b), B.ptr(u), int(warm), C.byref(cyc), C.byref(rel))
        return B.check(st, self._h, ok=(0, 4, 5)), cyc.value, rel.value

    def solve_adjoint(self, lam, rhs, warm=False):
        """J^T lam = rhs.  Returns (status, cycles, relres); lam is written."""
        cyc, rel = C.c_int(0), C.c_double(0.0)
        st = B.lib().stmg_solve_adjoint(self._h, B.ptr(rhs), B.ptr(lam), int(warm), C.byref(cyc), C.byref(rel))
        return B.check(st, self._h, ok=(0, 4, 5)), cyc.value, rel.value

    def sensitivity(self, chi, simp6, u, lam, g):
        s = (C.c_double * 6)(*[float(v) for v in simp6])
        B.check(B.lib().stmg_sensitivity(self._h, B.ptr(chi), s, B.ptr(u), B.ptr(lam), B.ptr(g)), self._h)
        return g

    def recompute_slabs(self, b, ckpt, slab_rows, u):
        """Fill u from checkpoint rows 0, K, 2K, ... by exact time stepping per slab."""
        B.check(B.lib().stmg_recompute_slabs(self._h, B.ptr(b), B.ptr(ckpt), int(slab_rows), B.ptr(u)), self._h)
        return u

    def sensitivity_slabs(self, chi, simp6, b, ckpt, slab_rows, lam, g):
        """Sensitivity with the forward state recomputed from checkpoints."""
        s = (C.c_double * 6)(*[float(v) for v in simp6])
        B.check(B.lib().stmg_sensitivity_slabs(self._h, B.ptr(chi), s, B.ptr(b), B.ptr(ckpt), int(slab_rows),
                                                B.ptr(lam), B.ptr(g)), self._h)
        return g

    def objective(self, b, u, theta_ref=1.0):
        """Theta = b^T u dt / theta_ref (Sec. 7.1), ``stmg_objective``."""
        out = C.c_double(0.0)
        B.check(B.lib().stmg_objective(self._h, B.ptr(b), B.ptr(u), float(theta_ref), C.byref(out)), self._h)
        return out.value

    def objective_gradient(self, b, grad_u, theta_ref=1.0, seed=1.0):
        """grad_u = seed * b dt / theta_ref, the gradient of Theta in u
        (``stmg_objective_gradient``; device arrays)."""
        B.check(B.lib().stmg_objective_gradient(self._h, B.ptr(b), float(theta_ref), float(seed), B.ptr(grad_u)),
                self._h)
        return grad_u

    # -- hierarchy -------------------------------------------------------------------
    @property
    def num_levels(self):
        return B.lib().stmg_num_levels(self._h)

    def level_info(self, l):
        n, nt, nx = C.c_int(), C.c_int(), C.c_int()
        dx, dt, w, lam = C.c_double(), C.c_double(), C.c_double(), C.c_double()
        B.check(B.lib().stmg_level_info(self._h, l, C.byref(n), C.byref(nt), C.byref(nx), C.byref(dx), C.byref(dt),
                                        C.byref(w), C.byref(lam)), self._h)
        return dict(N=n.value, NT=nt.value, next=nx.value, dx=dx.value, dt=dt.value, W=w.value, lambda_eff=lam.value)

    def level_material(self, l):
        import numpy as np

        N = self.level_info(l)["N"]
        k, c = np.empty(N), np.empty(N)
        B.check(B.lib().stmg_level_material(self._h, l, k.ctypes.data_as(B._dp), c.ctypes.data_as(B._dp)), self._h)
        return k, c

    def path(self):
        return "".join({1: "x", 2: "t"}[self.level_info(l)["next"]] for l in range(self.num_levels - 1))

    # -- building blocks ---------------------------------------------------------------
    def apply(self, level, u, y, adjoint=False):
        B.check(B.lib().stmg_apply(self._h, level, int(adjoint), B.ptr(u), B.ptr(y)), self._h)
        return y

    def smooth(self, level, u, b, nsweeps, adjoint=False):
        B.check(B.lib().stmg_smooth(self._h, level, int(adjoint), int(nsweeps), B.ptr(u), B.ptr(b)), self._h)
        return u

    def restrict(self, level, r, bc):
        B.check(B.lib().stmg_restrict(self._h, level, B.ptr(r), B.ptr(bc)), self._h)
        return bc

    def prolong_add(self, level, z, u):
        B.check(B.lib().stmg_prolong_add(self._h, level, B.ptr(z), B.ptr(u)), self._h)
        return u

    def exact_solve(self, level, b, u, adjoint=False):
        B.check(B.lib().stmg_exact_solve(self._h, level, int(adjoint), B.ptr(b), B.ptr(u)), self._h)
        return u

    def vcycle(self, u, b, adjoint=False):
        B.check(B.lib().stmg_vcycle(self._h, int(adjoint), B.ptr(u), B.ptr(b)), self._h)
        return u

    MIXED_PASS_KINDS = {"down": 0, "up": 1, "defect": 2, "up32": 3}

    def mixed_pass(self, level, kind, adjoint=False):
        """Enqueue one step of the mixed scheme on the solver's own vectors (``kind``: "down",
        "up" (on level 0 into the FP64 iterate), "up32" (into the FP32 iterate) or "defect"),
        without synchronising: for timing single passes."""
        B.check(B.lib().stmg_mixed_pass(self._h, int(level), int(adjoint), self.MIXED_PASS_KINDS[kind]), self._h)
