"""Loads libp2m.so (built in-tree by ``build.py``) and declares the C ABI of
include/p2m.h for ctypes.  A missing library is an ImportError: there is no
fallback implementation."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libp2m.so")

STATUS = {0: "ok", 1: "invalid argument", 2: "invalid mesh", 3: "duplicate vertex position",
          4: "out of memory", 5: "CUDA error", 6: "work queue error", 7: "I/O error",
          8: "no CUDA device", 9: "size exceeds a limit"}


class P2MError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)} (status {code})")


def check(code, where="p2m"):
    if code != 0:
        raise P2MError(code, where)


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -c 'import __graft_entry__ as g; g.build()'`")

lib = ctypes.CDLL(LIB_PATH)

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_INT = ctypes.c_int

_SIGS = {
    "p2m_default_opts": (None, [_P]),
    "p2m_build": (_INT, [_P, _P, _P]),
    "p2m_build_mixed": (_INT, [_P, _P, _I64, _P, _P]),
    "p2m_destroy": (None, [_P]),
    "p2m_query": (_INT, [_P, _P, _I64, _P, _P, _P, _P, _P, _P, _P]),
    "p2m_query_host": (_INT, [_P, _P, _I64, _P, _P, _P, _P, _P]),
    "p2m_nearest_vertex": (_INT, [_P, _P, _I64, _P, _P]),
    "p2m_pipe_create": (_INT, [_P, _I64, _INT, _P]),
    "p2m_pipe_submit": (_INT, [_P, _P, _I64, _P, _P, _P, _P]),
    "p2m_pipe_submit_device": (_INT, [_P, _P, _I64, _P, _P, _P, _P, _P]),
    "p2m_pipe_join": (_INT, [_P, _P]),
    "p2m_pipe_wait": (_INT, [_P]),
    "p2m_pipe_destroy": (None, [_P]),
    "p2m_query_noalloc": (_INT, [_P, _P, _I64, _P, _P, _P, _P, _P]),
    "p2m_get_tuning": (_INT, [_P, _P]),
    "p2m_set_tuning": (_INT, [_P, _P]),
    "p2m_reserve": (_INT, [_P, _I64]),
    "p2m_set_timing": (_INT, [_P, _INT]),
    "p2m_timing_summary": (_INT, [_P, _P]),
    "p2m_query_counters": (_INT, [_P, _P, _I64, _P, _P]),
    "p2m_backward": (_INT, [_P, _P, _P, _P, _P, _P, _I64, _P, _P, _P]),
    "p2m_update_vertices": (_INT, [_P, _P, _I64, _INT, _P]),
    "p2m_batch_create": (_INT, [_P, _P, _INT, _P]),
    "p2m_batch_run": (_INT, [_P, _P]),
    "p2m_batch_get_tuning": (_INT, [_P, _P]),
    "p2m_batch_set_tuning": (_INT, [_P, _P]),
    "p2m_batch_autotune": (_INT, [_P, _INT, _P, _P]),
    "p2m_batch_check": (_INT, [_P, _P]),
    "p2m_batch_destroy": (None, [_P]),
    "p2m_query_batched": (_INT, [_P, _P, _INT, _P]),
    "p2m_autotune": (_INT, [_P, _P, _I64, _INT, _P, _P]),
    "p2m_get_edges": (_INT, [_P, _P, _P]),
    "p2m_stats": (_INT, [_P, _P]),
    "p2m_flood_stats": (_INT, [_P, _P]),
    "p2m_cell_stats": (_INT, [_P, _P]),
    "p2m_domain": (_INT, [_P, _P]),
    "p2m_get_list": (_INT, [_P, ctypes.c_int32, _P, _P, _P, _I64, _P]),
    "p2m_save": (_INT, [_P, ctypes.c_char_p]),
    "p2m_load": (_INT, [ctypes.c_char_p, _P]),
    "p2m_status_string": (ctypes.c_char_p, [_INT]),
}

for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)
