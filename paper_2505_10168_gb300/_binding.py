"""ctypes binding of libstmg.so (include/stmg.h).  Argument marshalling only.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays; they must be contiguous
float64.  Their raw pointers are handed to the C ABI, which accepts device or host
memory.  There is no fallback: if the library is missing every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libstmg.so")

STATUS = {0: "ok", 1: "einval", 2: "enomem", 3: "ecuda", 4: "diverged", 5: "max_cycles"}
FP64, MIXED = 0, 1
REASM = {"K": 0, "R": 1, "D": 2, "P": 3}


class STMGError(RuntimeError):
    pass


class Opts(C.Structure):
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
        ("precision", C.c_int),
        ("tol", C.c_double),
        ("div_tol", C.c_double),
        ("max_cycles", C.c_int),
        ("mixed_first_cycles", C.c_int),
        ("mixed_inner_cycles", C.c_int),
    ]


class ServerOpts(C.Structure):
    _fields_ = [("workers", C.c_int), ("budget_bytes", C.c_longlong), ("cache", C.c_int), ("max_nu", C.c_int)]


class Request(C.Structure):
    _fields_ = [("nel", C.c_int), ("nt", C.c_int), ("L", C.c_double), ("t_end", C.c_double),
                ("k_el", C.c_void_p), ("c_el", C.c_void_p), ("q_el", C.c_void_p), ("q_value", C.c_double),
                ("adjoint", C.c_int), ("out", C.c_void_p), ("opts", Opts)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("cycles", C.c_int), ("relres", C.c_double), ("theta", C.c_double),
                ("t_submit", C.c_double), ("t_start", C.c_double), ("t_end", C.c_double), ("bytes", C.c_longlong),
                ("worker", C.c_int), ("nu", C.c_int)]


_lib = None
_vp = C.c_void_p
_i = C.c_int
_d = C.c_double
_ip = C.POINTER(C.c_int)
_dp = C.POINTER(C.c_double)

_SIGS = {
    "stmg_default_opts": (None, [C.POINTER(Opts)]),
    "stmg_last_error": (C.c_char_p, [_vp]),
    "stmg_create": (_i, [C.POINTER(_vp), _i, _i, _d, _d, _vp, _vp, C.POINTER(Opts), _vp]),
    "stmg_update_material": (_i, [_vp, _vp, _vp]),
    "stmg_create_design": (_i, [C.POINTER(_vp), _i, _i, _d, _d, _vp, _dp, C.POINTER(Opts), _vp]),
    "stmg_update_design": (_i, [_vp, _vp]),
    "stmg_create_with_allocator": (_i, [C.POINTER(_vp), _i, _i, _d, _d, _vp, _vp, C.POINTER(Opts), _vp, _vp, _vp,
                                        _vp]),
    "stmg_device_bytes": (C.c_longlong, [_vp]),
    "stmg_footprint": (C.c_longlong, [_i, _i, _d, _d, _vp, _vp, C.POINTER(Opts)]),
    "stmg_destroy": (None, [_vp]),
    "stmg_simp": (_i, [_i, _vp, _dp, _vp, _vp, _vp]),
    "stmg_design_update": (_i, [_i, _vp, _vp, _d, _d, _vp, _vp]),
    "stmg_assemble_load": (_i, [_vp, _vp, _vp]),
    "stmg_solve": (_i, [_vp, _vp, _vp, _vp, _i, _ip, _dp]),
    "stmg_solve_adjoint": (_i, [_vp, _vp, _vp, _i, _ip, _dp]),
    "stmg_sensitivity": (_i, [_vp, _vp, _dp, _vp, _vp, _vp]),
    "stmg_objective": (_i, [_vp, _vp, _vp, _d, _dp]),
    "stmg_objective_gradient": (_i, [_vp, _vp, _d, _d, _vp]),
    "stmg_deff_simp": (_i, [_dp, _dp]),
    "stmg_recompute_slabs": (_i, [_vp, _vp, _vp, _i, _vp]),
    "stmg_sensitivity_slabs": (_i, [_vp, _vp, _dp, _vp, _vp, _i, _vp, _vp]),
    "stmg_num_levels": (_i, [_vp]),
    "stmg_level_info": (_i, [_vp, _i, _ip, _ip, _ip, _dp, _dp, _dp, _dp]),
    "stmg_level_material": (_i, [_vp, _i, _dp, _dp]),
    "stmg_apply": (_i, [_vp, _i, _i, _vp, _vp]),
    "stmg_smooth": (_i, [_vp, _i, _i, _i, _vp, _vp]),
    "stmg_restrict": (_i, [_vp, _i, _vp, _vp]),
    "stmg_prolong_add": (_i, [_vp, _i, _vp, _vp]),
    "stmg_exact_solve": (_i, [_vp, _i, _i, _vp, _vp]),
    "stmg_vcycle": (_i, [_vp, _i, _vp, _vp]),
    "stmg_mixed_pass": (_i, [_vp, _i, _i, _i]),
    "stmg_sensitivity_noalloc": (_i, [_i, _i, _d, _d, _vp, _dp, _vp, _vp, _vp, _vp]),
    "stmg_kernel_launches": (C.c_ulonglong, []),
    "stmg_set_stream": (_i, [_vp, _vp]),
    "stmg_server_default_opts": (None, [C.POINTER(ServerOpts)]),
    "stmg_server_create": (_i, [C.POINTER(_vp), C.POINTER(ServerOpts)]),
    "stmg_server_submit": (_i, [_vp, C.POINTER(Request), C.POINTER(C.c_longlong)]),
    "stmg_server_result": (_i, [_vp, C.c_longlong, _i, C.POINTER(Result)]),
    "stmg_server_drain": (_i, [_vp]),
    "stmg_server_now": (_d, [_vp]),
    "stmg_server_peak_bytes": (C.c_longlong, [_vp]),
    "stmg_server_destroy": (None, [_vp]),
}


def lib():
    """Load libstmg.so (built by __graft_entry__.build()); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise STMGError("libstmg.so is not built (run __graft_entry__.build()); there is no fallback path")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def ptr(a):
    """Raw data pointer of a contiguous float64 torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise STMGError("numpy arrays must be C-contiguous float64")
        return a.ctypes.data
    import torch

    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise STMGError("tensors must be contiguous float64")
        return a.data_ptr()
    raise STMGError("unsupported array type %r" % type(a))


def numel(a):
    return a.size if isinstance(a, np.ndarray) else a.numel()


def default_stream():
    """The current torch CUDA stream handle if torch has a GPU, else NULL (0)."""
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def check(status, handle=None, ok=(0,)):
    if status in ok:
        return STATUS[status]
    msg = lib().stmg_last_error(handle).decode(errors="replace")
    raise STMGError("%s: %s" % (STATUS.get(status, status), msg))


def make_opts(**kw):
    o = Opts()
    lib().stmg_default_opts(C.byref(o))
    for key, val in kw.items():
        if key == "reassembly" and isinstance(val, str):
            val = REASM[val]
        if key == "interp" and isinstance(val, str):
            val = {"C": 0, "B": 1}[val]
        if key == "precision" and isinstance(val, str):
            val = {"fp64": FP64, "mixed": MIXED}[val]
        if not hasattr(o, key):
            raise STMGError("unknown option %s" % key)
        setattr(o, key, val)
    return o
