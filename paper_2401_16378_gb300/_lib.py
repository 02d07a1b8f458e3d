"""ctypes view of libpauli.so (the C ABI declared in include/pauli.h).

Loading never falls back to anything: if the shared library is missing the import of a
compute function raises, naming the build step.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpauli.so")

PAULI_C64, PAULI_C128 = 0, 1
PAULI_AUTO, PAULI_PLAIN, PAULI_XORDIAG = 0, 1, 2
STATUS = {0: "PAULI_OK", 1: "PAULI_ERR_ARG", 2: "PAULI_ERR_NULL", 3: "PAULI_ERR_ALIGN", 4: "PAULI_ERR_ALIAS",
          5: "PAULI_ERR_DTYPE", 6: "PAULI_ERR_NOMEM", 7: "PAULI_ERR_CUDA", 8: "PAULI_ERR_TIMEOUT",
          9: "PAULI_ERR_UNSUPPORTED"}

# name -> (restype, argtypes); every function the header declares.
_vp, _i, _i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
_vpp = ctypes.POINTER(ctypes.c_void_p)
_ip = ctypes.POINTER(ctypes.c_int)
SIGNATURES = {
    "pauli_decompose": (_i, [_vp, _i, _i, _i, _vp, _i, _vp]),
    "pauli_decompose_workspace_size": (_i, [_i, _i, _i, _i, ctypes.POINTER(ctypes.c_size_t)]),
    "pauli_decompose_ws": (_i, [_vp, _i, _i, _i, _vp, _i, _vp, ctypes.c_size_t, _vp]),
    "pauli_workspace_status": (_i, [_vp, _vp]),
    "pauli_release_workspaces": (_i, [_vp]),
    "pauli_compose": (_i, [_vp, _i, _i, _i, _vp, _i, _vp]),
    "pauli_decompose_hermitian": (_i, [_vp, _i, _i, _i, _vp, _i, _vp]),
    "pauli_decompose_real": (_i, [_vp, _i, _i, _i, _vp, _i, _vp]),
    "pauli_decompose_hermitian_upper": (_i, [_vp, _i, _i, _i, _vp, _i, _vp]),
    "pauli_weighted_norm": (_i, [_vp, _i, _i, _i, _vp, _vp, _vp]),
    "pauli_decompose_weighted_norm": (_i, [_vp, _i, _i, _i, _vp, _vp, _vp, _i, _vp]),
    "pauli_compose_weighted": (_i, [_vp, _i, _i, _i, _vp, _vp, _vp, _i, _vp]),
    "pauli_weighted_norm_grad": (_i, [_vp, _i, _i, _i, _vp, _vp, _vp, _vp]),
    "pauli_coeffs_at": (_i, [_vp, _i, _i, _vp, _i64, _vp, _vp]),
    "pauli_decompose_list": (_i, [_vpp, _ip, _i, _i, _vpp, _i, _vp]),
    "pauli_decompose_host": (_i, [_vp, _i, _i, _i, _vp, _vp, _vp, _i, _vp]),
    "pauli_decompose_host_stream": (_i, [_vpp, _vpp, _i, _i, _i, _vpp, _vpp, _i, _vp]),
    "pauli_compose_batched": (_i, [_vpp, _ip, _i, _i, _vpp, _i, _vp]),
    "pauli_xhi_layout": (_i, [_vp, _i, _i, _i, _i, _vp, _vp]),
    "pauli_decompose_xhi": (_i, [_vp, _i, _i, _i, _i, _vp, _i, _vp]),
    "pauli_decompose_batch_static": (_i, [_vpp, _ip, _i, _i, _vpp, _vp]),
    "pauli_plan_create": (_i, [_ip, _i, _i, _i, _i, ctypes.POINTER(ctypes.c_void_p)]),
    "pauli_plan_create_hermitian": (_i, [_ip, _i, _i, _i, _i, ctypes.POINTER(ctypes.c_void_p)]),
    "pauli_plan_bind": (_i, [_vp, _vpp, _vpp]),
    "pauli_plan_execute": (_i, [_vp, _vp]),
    "pauli_plan_graph_launch": (_i, [_vp, _vp]),
    "pauli_plan_status": (_i, [_vp]),
    "pauli_plan_set_stall": (_i, [_vp, _i]),
    "pauli_plan_destroy": (None, [_vp]),
    "pauli_set_variant": (_i, [_i, _i, _i, _i]),
    "pauli_get_variant": (_i, [_i, _i, _i]),
    "pauli_stream_status": (_i, [_vp]),
    "pauli_last_error": (ctypes.c_char_p, []),
    "pauli_version": (_i, []),
    "pauli_debug_fail_next_launches": (None, [_i]),
    "pauli_debug_stall_next_tiled": (None, []),
}

_lock = threading.Lock()
_lib = None


class PauliError(RuntimeError):
    """A libpauli call returned a status other than PAULI_OK."""

    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


def load() -> ctypes.CDLL:
    """Load libpauli.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
            fresh = True
        else:
            fresh = False
    if fresh and os.environ.get("PAULI_AUTOTUNE", "1") != "0":
        from . import autotune  # applies the tuned launch shapes measured on this GPU model

        autotune.apply_cached()
    return _lib


def check(status: int) -> None:
    if status != 0:
        raise PauliError(status, load().pauli_last_error().decode(errors="replace"))
