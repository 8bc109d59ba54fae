"""ctypes binding of libhubsv.so (the C ABI declared in include/hubsv.h).

Argument marshalling only.  The library is loaded on first use; if it has not
been built the call raises instead of falling back to anything else.
"""

from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_uint32, c_void_p

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhubsv.so")

HUB_OK, HUB_EINVAL, HUB_EUNSUPPORTED, HUB_ENOMEM, HUB_ECUDA, HUB_ETIMEOUT = range(6)
STATUS_NAMES = {0: "HUB_OK", 1: "HUB_EINVAL", 2: "HUB_EUNSUPPORTED", 3: "HUB_ENOMEM",
                4: "HUB_ECUDA", 5: "HUB_ETIMEOUT"}

EXPORTS = [
    "hub_square_lattice", "hub_create", "hub_destroy", "ans_create", "ans_create_multi",
    "ans_destroy", "ans_num_params", "ans_num_qubits", "state_prepare", "energy",
    "energy_grad", "hub_apply_h", "ans_plan_stats", "ans_set_tile", "ans_set_runs", "hub_sync",
    "hub_last_error", "ans_plan_describe", "ans_profile", "ans_profile_read", "energy_noalloc",
    "overlap_grad", "spin_correlation", "ans_workspace_bytes", "ans_set_threads",
]


class HubError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class HubLattice(ctypes.Structure):
    _fields_ = [("n_sites", c_int32), ("n_bonds", c_int32), ("bonds", POINTER(c_int32)),
                ("mode_up", POINTER(c_int32)), ("mode_dn", POINTER(c_int32))]


class HubGroup(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("n_terms", c_int32), ("terms", POINTER(c_int32)),
                ("param", c_int32)]


_lib = None


def lib():
    """The loaded library; raises if libhubsv.so has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            "libhubsv.so is not built: run `python -m paper_2408_00836_gb300.build` "
            "(or __graft_entry__.build()); there is no fallback path")
    L = ctypes.CDLL(LIB_PATH)
    st = c_int32
    sig = {
        "hub_square_lattice": (st, [c_int32, c_int32, c_int32, POINTER(c_int32), POINTER(c_int32), POINTER(c_int32)]),
        "hub_create": (st, [POINTER(HubLattice), POINTER(c_double), POINTER(c_double), POINTER(c_double),
                            c_int32, c_int32, POINTER(c_void_p)]),
        "hub_destroy": (None, [c_void_p]),
        "ans_create": (st, [c_void_p, c_int32, c_int32, POINTER(HubGroup), POINTER(c_void_p)]),
        "ans_create_multi": (st, [POINTER(c_void_p), c_int32, c_int32, c_int32, POINTER(HubGroup),
                                  POINTER(c_void_p)]),
        "ans_destroy": (None, [c_void_p]),
        "ans_num_params": (c_int32, [c_void_p]),
        "ans_num_qubits": (c_int32, [c_void_p]),
        "state_prepare": (st, [c_void_p, c_int32, POINTER(c_double), POINTER(c_int32), c_void_p, c_int32,
                               c_int64, c_void_p]),
        "energy": (st, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int64, c_uint32, c_void_p]),
        "energy_noalloc": (st, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int64, c_uint32, c_void_p]),
        "energy_grad": (st, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int32,
                             c_int64, c_uint32, c_void_p]),
        "hub_apply_h": (st, [c_void_p, c_void_p, c_void_p, c_int32, c_int64, c_void_p]),
        "overlap_grad": (st, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p,
                              c_void_p, c_int32, c_int64, c_uint32, c_void_p]),
        "spin_correlation": (st, [c_void_p, c_void_p, c_void_p, c_int32, c_int64, c_void_p]),
        "ans_workspace_bytes": (st, [c_void_p, c_int32, c_int32, c_uint32, c_int64, POINTER(ctypes.c_uint64),
                                     POINTER(c_int32)]),
        "ans_plan_stats": (st, [c_void_p, c_int32, c_int32, c_uint32, POINTER(c_int32), POINTER(c_double)]),
        "ans_set_tile": (st, [c_void_p, c_int32, c_int32]),
        "ans_set_threads": (st, [c_void_p, c_int32, c_int32, c_int32]),
        "ans_set_runs": (st, [c_void_p, c_int32, c_int32]),
        "ans_plan_describe": (st, [c_void_p, c_int32, c_int32, c_uint32, POINTER(c_int64), c_int32,
                                   POINTER(c_int32)]),
        "ans_profile": (st, [c_void_p, c_int32]),
        "ans_profile_read": (st, [c_void_p, POINTER(c_double), c_int32, POINTER(c_int32)]),
        "hub_sync": (st, [c_void_p]),
        "hub_last_error": (c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(status: int) -> None:
    if status != HUB_OK:
        msg = lib().hub_last_error()
        raise HubError(status, msg.decode() if msg else "")
