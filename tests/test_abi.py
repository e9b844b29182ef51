"""The C-ABI library loads and exports every function that include/stmg.h declares (CPU only)."""
import ctypes
import os
import re

import pytest

from paper_2505_10168_gb300 import _binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(stmg_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(_binding.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 20
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    assert _declared() <= set(_binding._SIGS)


def test_default_opts_and_errors_without_gpu():
    lib = _binding.lib()
    o = _binding.make_opts()
    assert (o.nu, o.omega, o.lambda_crit, o.max_cycles, o.tol) == (5, 0.5, 0.25, 100, 1e-10)
    h = ctypes.c_void_p()
    # invalid sizes are rejected on the host before any device work
    st = lib.stmg_create(ctypes.byref(h), 0, 4, 1.0, 1.0, None, None, None, None)
    assert _binding.STATUS[st] == "einval" and not h.value
    assert b"nel" in lib.stmg_last_error(None)
    with pytest.raises(_binding.STMGError):
        _binding.make_opts(no_such_option=1)
    assert _binding.STATUS[lib.stmg_mixed_pass(None, 0, 0, 0)] == "einval"


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs (options, server options, request,
    result) have the C compiler's size and field offsets, field by field and by name."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = [("stmg_opts", _binding.Opts), ("stmg_server_opts", _binding.ServerOpts),
             ("stmg_request", _binding.Request), ("stmg_result", _binding.Result)]
    lines = ['#include "stmg.h"', "#include <stddef.h>", "#include <stdio.h>", "int main(void) {"]
    expect = []
    for cname, cls in pairs:
        lines.append('  printf("%%zu\\n", sizeof(%s));' % cname)
        expect.append(ctypes.sizeof(cls))
        for fname, _ in cls._fields_:
            lines.append('  printf("%%zu\\n", offsetof(%s, %s));' % (cname, fname))
            expect.append(getattr(cls, fname).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(ROOT, "include")
    subprocess.run([cc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True, capture_output=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == expect


def test_noalloc_placement_rule(tmp_path):
    """stmg_sensitivity_noalloc takes device memory of the current device or managed
    memory, and refuses host memory and device memory of another GPU (which the current
    device cannot read without peer access).  The rule is checked here on the host,
    against the CUDA runtime's own cudaMemoryType values, without any device."""
    import shutil
    import subprocess

    cxx = shutil.which("g++") or shutil.which("c++")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if cxx is None or not os.path.exists(os.path.join(cuda_inc, "driver_types.h")):
        pytest.skip("no C++ compiler or CUDA headers")
    src = tmp_path / "placement.cc"
    src.write_text("\n".join([
        "#include <cstdio>",
        "#include <driver_types.h>",
        '#include "stmg_placement.h"',
        "using namespace stmg;",
        "int main() {",
        "  int bad = 0;",
        "  bad += noalloc_placement(cudaMemoryTypeDevice, 0, 0) != kPlaceUsable;",
        "  bad += noalloc_placement(cudaMemoryTypeDevice, 3, 3) != kPlaceUsable;",
        "  bad += noalloc_placement(cudaMemoryTypeDevice, 1, 0) != kPlaceOtherDevice;",
        "  bad += noalloc_placement(cudaMemoryTypeDevice, 0, 2) != kPlaceOtherDevice;",
        "  bad += noalloc_placement(cudaMemoryTypeManaged, 1, 0) != kPlaceUsable;",
        "  bad += noalloc_placement(cudaMemoryTypeHost, 0, 0) != kPlaceNotDevice;",
        "  bad += noalloc_placement(cudaMemoryTypeUnregistered, 0, 0) != kPlaceNotDevice;",
        '  std::printf("%d\\n", bad);',
        "  return 0;",
        "}",
    ]) + "\n")
    exe = tmp_path / "placement"
    csrc = os.path.join(ROOT, "paper_2505_10168_gb300", "csrc")
    subprocess.run([cxx, "-std=c++17", "-I", csrc, "-I", cuda_inc, str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert out == ["0"]


def test_deff_simp_on_the_host():
    """stmg_deff_simp (Sec. 7.2): sqrt(min D * max D) of D_SIMP = k_SIMP / c_SIMP over chi in
    [0, 1], host arithmetic only.  With c constant the extrema are k_ins and k_con; with a
    penalised c the minimum lies inside (0, 1), where a bounded scalar minimiser finds it."""
    import math

    import paper_2505_10168_gb300 as pkg

    assert pkg.deff_simp([1e-3, 1.0, 1.0, 1.0, 3.0, 1.0]) == pytest.approx(math.sqrt(1e-3), rel=1e-15)
    assert pkg.deff_simp([1e-6, 2.0, 0.5, 0.5, 3.0, 2.0]) == pytest.approx(math.sqrt(2e-6 / 0.25), rel=1e-15)
    s6 = [0.01, 1.0, 0.1, 1.0, 3.0, 1.0]
    d = lambda x: (0.01 + 0.99 * x ** 3) / (0.1 + 0.9 * x)  # noqa: E731
    from scipy.optimize import minimize_scalar

    m = minimize_scalar(d, bounds=(0.0, 1.0), method="bounded", options={"xatol": 1e-12})
    assert 0.0 < m.x < 1.0 and m.fun < d(0.0)
    assert pkg.deff_simp(s6) == pytest.approx(math.sqrt(m.fun * d(1.0)), rel=1e-7)
    with pytest.raises(_binding.STMGError):
        pkg.deff_simp([0.0, 1.0, 1.0, 1.0, 3.0, 1.0])


def test_grid_size_limit_on_the_host():
    """A space-time vector is indexed with 32-bit DOF numbers: (nel+1)(nt+1) must stay
    below 2^31.  The largest grid below the limit is planned (its footprint is positive);
    the first one at the limit is refused by stmg_footprint and by stmg_create before any
    device work, with a message."""
    lib = _binding.lib()
    o = _binding.make_opts()
    import numpy as np

    k = np.ones(32767)
    assert (32767 + 1) * (65534 + 1) < 2 ** 31 and (32767 + 1) * (65535 + 1) == 2 ** 31
    assert lib.stmg_footprint(32767, 65534, 1.0, 1.0, k.ctypes.data, k.ctypes.data, ctypes.byref(o)) > 0
    assert lib.stmg_footprint(32767, 65535, 1.0, 1.0, k.ctypes.data, k.ctypes.data, ctypes.byref(o)) == -1
    h = ctypes.c_void_p()
    st = lib.stmg_create(ctypes.byref(h), 32767, 65535, 1.0, 1.0, k.ctypes.data, k.ctypes.data, None, None)
    assert _binding.STATUS[st] == "einval" and not h.value
    assert b"2^31" in lib.stmg_last_error(None)
