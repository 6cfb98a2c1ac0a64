"""ctypes declarations of the C ABI in include/ising_ds.h.

Loading fails with an exception when libising_gb300.so has not been built:
there is no fallback implementation.
"""

from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int32, c_int64, c_uint64, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libising_gb300.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EBUSY, ENOTSUP = range(7)
LAYOUT_DENSE, LAYOUT_CSR = 0, 1
F64, F32, I8, I32 = 0, 1, 2, 3
CONV_PHYSICS, CONV_PAPER = 0, 1
MEM_HOST, MEM_DEVICE = 0, 1
PREC_AUTO, PREC_FP32_PLAIN, PREC_TC, PREC_BF16, PREC_FP8 = range(5)
PATH_PLAIN, PATH_TC, PATH_SPARSE = range(3)
PRUNE_ZERO_RULE = 1
SERVER_PACK = 1
DS_PROFILE = 1
DS_STREAMING = 2
DS_NO_AUTOTUNE = 4
DS_CONVERGE = 8
DS_RELAXED = 16


class Instance(ctypes.Structure):
    _fields_ = [("n", c_int64), ("layout", c_int32), ("j_dtype", c_int32), ("J", c_void_p),
                ("indptr", c_void_p), ("indices", c_void_p), ("nnz", c_int64),
                ("h_dtype", c_int32), ("reserved0", c_int32), ("h", c_void_p),
                ("j_scale", c_double), ("convention", c_int32), ("mem", c_int32)]


class DSParams(ctypes.Structure):
    _fields_ = [("restarts", c_int64), ("steps", c_int64), ("lr", c_double), ("mu", c_double),
                ("beta1", c_double), ("beta2", c_double), ("eps", c_double),
                ("seed", c_uint64), ("precision", c_int32), ("flags", c_int32)]


class DSStats(ctypes.Structure):
    _fields_ = [("best_restart", c_int64), ("best_step", c_int64),
                ("last_best_energy", c_double), ("last_best_restart", c_int64),
                ("steps_done", c_int64), ("path", c_int32), ("precision", c_int32),
                ("device_ms", c_double), ("kernel_ms", c_double),
                ("kernel_launches", c_int64), ("resident", c_int32), ("operand_planes", c_int32),
                ("tile_restarts", c_int32), ("tile_pair", c_int32)]


class ServerCfg(ctypes.Structure):
    _fields_ = [("budget_bytes", c_uint64), ("max_active", c_int32), ("chunk_steps", c_int32),
                ("flags", c_int32), ("helper_threads", c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("status", c_int32), ("done", c_int32), ("n", c_int64),
                ("best_energy", c_double), ("best_restart", c_int64), ("best_step", c_int64),
                ("footprint", c_int64), ("t_submit_ms", c_double), ("t_admit_ms", c_double),
                ("t_done_ms", c_double), ("steps_done", c_int64), ("reached", c_int32),
                ("cancelled", c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", c_int64), ("rounds", c_int64), ("chunks", c_int64),
                ("pack_chunks", c_int64), ("packs_created", c_int64), ("target_checks", c_int64),
                ("setup_ms", c_double), ("setup_upload_ms", c_double),
                ("setup_prune_ms", c_double), ("setup_session_ms", c_double),
                ("advance_ms", c_double), ("pack_create_ms", c_double),
                ("check_ms", c_double), ("finish_ms", c_double), ("release_ms", c_double),
                ("idle_ms", c_double), ("elapsed_ms", c_double)]


_PROTOS = {
    "ising_version": (c_int, []),
    "ising_create": (c_int, [POINTER(c_void_p), c_int, c_void_p]),
    "ising_destroy": (c_int, [c_void_p]),
    "ising_last_error": (c_char_p, [c_void_p]),
    "ising_set_stream": (c_int, [c_void_p, c_void_p]),
    "ising_synchronize": (c_int, [c_void_p]),
    "ising_energy": (c_int, [c_void_p, POINTER(Instance), c_void_p, c_int64, c_void_p,
                             c_void_p, c_void_p, c_int]),
    "ising_energy_noalloc": (c_int, [POINTER(Instance), c_void_p, c_int64, c_void_p, c_void_p]),
    "ising_energy_noalloc_error": (c_char_p, []),
    "ising_prune": (c_int, [c_void_p, POINTER(Instance), c_int, POINTER(c_void_p)]),
    "ising_prune_info": (c_int, [c_void_p, POINTER(c_int64), POINTER(c_int64),
                                 POINTER(c_double), POINTER(c_double), POINTER(c_int32)]),
    "ising_prune_reduced": (c_int, [c_void_p, POINTER(Instance)]),
    "ising_prune_reduced_copy": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int]),
    "ising_prune_record": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                   c_void_p, c_void_p, c_int]),
    "ising_prune_free": (c_int, [c_void_p]),
    "ising_reconstruct": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int]),
    "ising_select_domain": (c_int, [c_void_p, POINTER(Instance), POINTER(DSParams), c_void_p,
                                    POINTER(c_double), POINTER(DSStats), c_int]),
    "ising_solve": (c_int, [c_void_p, POINTER(Instance), POINTER(DSParams), c_int, c_void_p,
                            POINTER(c_double), POINTER(DSStats), c_int]),
    "ising_ds_create": (c_int, [c_void_p, POINTER(Instance), POINTER(DSParams),
                                POINTER(c_void_p)]),
    "ising_ds_run": (c_int, [c_void_p, c_int64]),
    "ising_ds_finish": (c_int, [c_void_p]),
    "ising_ds_export_state": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                      POINTER(c_int64), c_int]),
    "ising_ds_import_state": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int]),
    "ising_ds_coupling": (c_int, [c_void_p, c_void_p, c_int]),
    "ising_ds_trace": (c_int, [c_void_p, c_void_p, c_int64, POINTER(c_int64)]),
    "ising_ds_last_energies": (c_int, [c_void_p, c_void_p, c_int]),
    "ising_ds_restart_best": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int]),
    "ising_ds_convergence": (c_int, [c_void_p, c_void_p, c_int]),
    "ising_ds_work": (c_int, [c_void_p, POINTER(c_int64)]),
    "ising_ds_set_tiles": (c_int, [c_void_p, c_int32, c_int32]),
    "ising_selftest_waits": (c_int, [c_void_p, c_int64, c_void_p]),
    "ising_ds_result": (c_int, [c_void_p, c_void_p, POINTER(c_double), POINTER(DSStats), c_int]),
    "ising_ds_destroy": (c_int, [c_void_p]),
    "ising_pack_create": (c_int, [c_void_p, POINTER(c_void_p), c_int32, POINTER(c_void_p)]),
    "ising_pack_run": (c_int, [c_void_p, c_int64]),
    "ising_pack_destroy": (c_int, [c_void_p]),
    "ising_server_create": (c_int, [c_void_p, POINTER(ServerCfg), POINTER(c_void_p)]),
    "ising_server_submit": (c_int, [c_void_p, POINTER(Instance), POINTER(DSParams), c_int,
                                    POINTER(c_uint64)]),
    "ising_server_submit_target": (c_int, [c_void_p, POINTER(Instance), POINTER(DSParams), c_int,
                                           c_double, POINTER(c_uint64)]),
    "ising_server_stats_get": (c_int, [c_void_p, POINTER(ServerStats)]),
    "ising_server_error": (c_int, [c_void_p, c_uint64, c_char_p, c_int64]),
    "ising_server_cancel": (c_int, [c_void_p, c_uint64]),
    "ising_server_poll": (c_int, [c_void_p, c_uint64, POINTER(Result), c_void_p]),
    "ising_server_wait": (c_int, [c_void_p, c_uint64, c_double, POINTER(Result), c_void_p]),
    "ising_server_release": (c_int, [c_void_p, c_uint64]),
    "ising_server_destroy": (c_int, [c_void_p]),
}

_lib = None


def load() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; "
            "g.build()\"` (there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _PROTOS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def optional(name: str, res, args):
    """Declare an entry point that newer builds add; returns None if absent."""
    lib = load()
    fn = getattr(lib, name, None)
    if fn is not None:
        fn.restype = res
        fn.argtypes = args
    return fn
