"""The allocation-free sensitivity entry point against the handle-based one.

stmg_sensitivity_noalloc exists for callers that cannot allocate device memory when
they need a gradient (allocation can synchronise the whole device, or their memory is
fixed up front).  It keeps its scratch in a fixed array inside the library, so this
test calls it twice in a row with different inputs and checks each result against
stmg_sensitivity (and the first also against the CPU oracle), and checks that oversize
problems and host arrays are refused.
This file is collected last so that a run stopping at the first failure has already
run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
import paper_2505_10168_gb300 as pkg
from paper_2505_10168_gb300 import _binding as B
from paper_2505_10168_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _noalloc(nel, nt, L, tT, chi, simp6, u, lam, g, stream=None):
    s6 = (C.c_double * 6)(*[float(v) for v in simp6])
    return B.lib().stmg_sensitivity_noalloc(nel, nt, L, tT, B.ptr(chi), s6, B.ptr(u), B.ptr(lam), B.ptr(g),
                                           stream if stream is not None else B.default_stream())


def _inputs(seed, N, NT):
    chi = torch.tensor(0.1 + 0.8 * wl.uniform(seed, N), device=DEV)
    u = torch.tensor(wl.uniform(seed + 1, (NT + 1) * (N + 1)).reshape(NT + 1, N + 1) - 0.5, device=DEV)
    lam = torch.tensor(wl.uniform(seed + 2, (NT + 1) * (N + 1)).reshape(NT + 1, N + 1) - 0.5, device=DEV)
    return chi, u, lam


def test_noalloc_sensitivity_matches_stmg_sensitivity_twice():
    N, NT, L, tT = 300, 700, 1.3, 0.7  # several time chunks with a ragged last one
    s6 = wl.simp_params(1e-3, 1.0, 0.2, 1.0)  # penalised heat capacity: both terms active
    ref_solver = pkg.Solver(N, NT, L, tT, np.ones(N), np.ones(N))
    for call, seed in enumerate([11, 29]):
        chi, u, lam = _inputs(seed, N, NT)
        ref = torch.empty(N, dtype=torch.float64, device=DEV)
        ref_solver.sensitivity(chi, s6, u, lam, ref)
        out = torch.full((N,), float("nan"), dtype=torch.float64, device=DEV)
        st = _noalloc(N, NT, L, tT, chi, s6, u, lam, out)
        assert B.STATUS[st] == "ok", B.lib().stmg_last_error(None)
        torch.cuda.synchronize()
        err = (out - ref).abs().max().item() / ref.abs().max().item()
        assert err < 1e-12, (call, err)
        if call == 0:  # and once against the CPU oracle's sensitivity, independently of the GPU
            go = oracle.sensitivity(N, NT, L, tT, chi.cpu().numpy(), s6, u.cpu().numpy(), lam.cpu().numpy())
            assert np.abs(out.cpu().numpy() - go).max() / np.abs(go).max() < 1e-12
    ref_solver.close()


def test_noalloc_rejects_oversize_and_host_arrays():
    N = 4096
    NT = 32768  # needs 2 * 129 * 4096 scratch values, above the fixed maximum
    chi = torch.zeros(N, dtype=torch.float64, device=DEV)
    g = torch.zeros(N, dtype=torch.float64, device=DEV)
    small = torch.zeros(4, dtype=torch.float64, device=DEV)
    s6 = wl.simp_params(1e-3, 1.0, 1.0, 1.0)
    st = _noalloc(N, NT, 1.0, 1.0, chi, s6, small, small, g)
    assert B.STATUS[st] == "einval"
    assert b"maximum" in B.lib().stmg_last_error(None)
    # a single element over more time steps than one launch's grid holds in time chunks
    # (65536 chunks of 256 rows): refused on the host, before any array is touched
    one = torch.zeros(1, dtype=torch.float64, device=DEV)
    st = _noalloc(1, 65535 * 256, 1.0, 1.0, one, s6, small, small, one)
    assert B.STATUS[st] == "einval"
    assert b"time chunks" in B.lib().stmg_last_error(None)
    n, nt = 8, 8
    chi_h = np.full(n, 0.5)
    u_h = np.zeros((nt + 1, n + 1))
    st = _noalloc(n, nt, 1.0, 1.0, chi_h, s6, u_h, u_h, np.zeros(n))
    assert B.STATUS[st] == "einval"
    assert b"device memory" in B.lib().stmg_last_error(None)
