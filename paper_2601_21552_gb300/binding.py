"""Thin ctypes binding over libscuba (include/scuba.h). Argument marshalling
only: every step of the satisfiability check runs in the library (host C++
encoder/verifier, CUDA kernels for the solve). There is no fallback: if the
library is missing this module raises at import.

The names match the C ABI (scuba_encode_batch, scuba_solve_batch, ...);
the small classes below only hold the marshalled arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SCUBA_LIBRARY=checked selects the checked build (device bounds checks that
# report through the call's status); anything else the regular library
LIB_PATH = os.path.join(_HERE, "_build", "libscuba_checked.so"
                        if os.environ.get("SCUBA_LIBRARY") == "checked" else "libscuba.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libscuba.so not built ({LIB_PATH}); run __graft_entry__.build() "
                      "or python paper_2601_21552_gb300/build.py")

_lib = ctypes.CDLL(LIB_PATH)

SCUBA_UNSAT, SCUBA_SAT, SCUBA_UNKNOWN = 0, 1, 2
SCUBA_OK = 0
SCUBA_ERR_ARG, SCUBA_ERR_CUDA, SCUBA_ERR_NOMEM = -1, -2, -3
SCUBA_ERR_TIMEOUT, SCUBA_ERR_MALFORMED, SCUBA_ERR_ABORTED, SCUBA_ERR_TOO_LARGE = -4, -5, -6, -7
SCUBA_ERR_INTERNAL = -8
SCUBA_HEUR_ACTIVITY, SCUBA_HEUR_LEARNED = 0, 1
SCUBA_SEARCH_DPLL, SCUBA_SEARCH_CDCL = 0, 1

_vp = ctypes.c_void_p
_i32, _i64 = ctypes.c_int32, ctypes.c_int64


class scuba_cnf_batch(ctypes.Structure):
    _fields_ = [("num_instances", _i32), ("max_vars", _i32), ("total_clauses", _i64),
                ("total_lits", _i64), ("total_vars", _i64), ("inst_clause_begin", _vp),
                ("clause_begin", _vp), ("lits", _vp), ("inst_num_vars", _vp),
                ("inst_var_begin", _vp)]


class scuba_options(ctypes.Structure):
    _fields_ = [("heuristic", _i32), ("learned_depth", _i32), ("mlp_weights", _vp),
                ("decision_budget", _i64), ("time_budget_ms", _i64), ("split", _i32),
                ("warps_per_block", _i32), ("blocks_per_sm", _i32), ("split_interval", _i32),
                ("split_min", _i32), ("trail_placement", _i32), ("finish_ns", _vp),
                ("profile", _vp),
                ("stats", _vp), ("order", _vp), ("abort_flag", _vp),
                ("search_event_begin", _vp), ("search_event_end", _vp),
                ("inst_num_inputs", _vp), ("trace", _vp), ("search", _i32),
                ("restart_unit", _i32), ("learnt_words", _i64), ("split_depth", _i32),
                ("share_lbd", _i32)]


class scuba_trace(ctypes.Structure):
    _fields_ = [("depth", _i32), ("max_nodes", _i64), ("max_rows", _i64), ("counts", _vp),
                ("node_inst", _vp), ("node_depth", _vp), ("node_row", _vp),
                ("node_nrows", _vp), ("node_closed", _vp), ("x", _vp), ("target", _vp),
                ("var", _vp)]


SCUBA_NSTATS = 6
STAT_NAMES = ("decisions", "conflicts", "propagations", "visits", "act_reads", "undone")


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("scuba_options_init", _i32, [ctypes.POINTER(scuba_options)])
_sig("scuba_solve_batch", _i32, [ctypes.POINTER(scuba_cnf_batch), _vp, _vp, _vp])
_sig("scuba_solve_batch_ex", _i32, [ctypes.POINTER(scuba_cnf_batch), _vp, _vp, _vp,
                                    ctypes.POINTER(scuba_options)])
_sig("scuba_solve_batch_host", _i32, [ctypes.POINTER(scuba_cnf_batch), _vp, _vp, _vp,
                                      ctypes.POINTER(scuba_options)])
_sig("scuba_solve_units", _i32, [ctypes.POINTER(scuba_cnf_batch), _i32, _vp, _vp, _vp, _vp, _vp,
                                 _vp, _vp, ctypes.POINTER(scuba_options)])
_sig("scuba_solve_batch_noalloc", _i32, [ctypes.POINTER(scuba_cnf_batch), _vp, _vp, _vp,
                                         ctypes.POINTER(scuba_options)])
_sig("scuba_propagate_batch", _i32, [ctypes.POINTER(scuba_cnf_batch), _vp, _vp, _vp, _vp, _vp])
_sig("scuba_sync_status", _i32, [_vp])
_sig("scuba_release", None, [])
_sig("scuba_last_error", ctypes.c_char_p, [])
_sig("scuba_version", _i32, [])
_sig("scuba_abi_sizes", _i32, [_vp])
_sig("scuba_encode_batch", _i32, [_i32, _vp, _vp, _i32, ctypes.POINTER(_vp)])
_sig("scuba_encoded_sizes", _i32, [_vp, _vp])
_sig("scuba_encoded_copy", _i32, [_vp, _vp, _vp, _vp, _vp, _vp])
_sig("scuba_encoded_inputs", _i32, [_vp, _vp, _vp, _vp])
_sig("scuba_encoded_free", None, [_vp])
_sig("scuba_encoded_release_clauses", _i32, [_vp])
_sig("scuba_verify_batch", _i32, [_vp, _vp, _vp, _vp, _vp, _i32, _vp])
_sig("scuba_mlp_layout", _i32, [_vp])
_sig("scuba_mlp_init", _i32, [_vp, _vp, ctypes.c_uint64, _vp])
_sig("scuba_mlp_pack", _i32, [_vp, _vp, _vp])
_sig("scuba_mlp_forward", _i32, [_vp, _i64, _vp, _vp, _vp])
_sig("scuba_mlp_grad", _i32, [ctypes.POINTER(scuba_trace), _i64, _i64, _vp, _vp, _vp, _vp])
_sig("scuba_mlp_train", _i32, [ctypes.POINTER(scuba_trace), _i64, _vp, _vp, _vp, _vp, _i32,
                               _i32, ctypes.c_float, _vp, _vp])

EXPORTED = [
    "scuba_options_init", "scuba_solve_batch", "scuba_solve_batch_ex", "scuba_solve_units",
    "scuba_solve_batch_host", "scuba_solve_batch_noalloc", "scuba_propagate_batch",
    "scuba_sync_status", "scuba_release", "scuba_last_error",
    "scuba_version", "scuba_abi_sizes", "scuba_encode_batch", "scuba_encoded_sizes", "scuba_encoded_copy",
    "scuba_encoded_inputs", "scuba_encoded_free", "scuba_encoded_release_clauses",
    "scuba_verify_batch",
    "scuba_mlp_layout", "scuba_mlp_init", "scuba_mlp_pack", "scuba_mlp_forward",
    "scuba_mlp_grad", "scuba_mlp_train",
]
SCUBA_MLP_WEIGHT_BYTES = 2448
SCUBA_MLP_NPARAM = 1153


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(_vp)


def _check_layout():
    sz = np.zeros(2, dtype=np.int64)
    _lib.scuba_abi_sizes(_np_ptr(sz))
    mine = (ctypes.sizeof(scuba_cnf_batch), ctypes.sizeof(scuba_options))
    if tuple(int(x) for x in sz) != mine:
        raise ImportError(f"libscuba struct layout {tuple(sz)} != binding {mine}; rebuild")


_check_layout()


def last_error() -> str:
    return (_lib.scuba_last_error() or b"").decode()


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise RuntimeError(f"{what} failed with status {rc}: {last_error()}")
    return rc


def scuba_options_init() -> scuba_options:
    o = scuba_options()
    _check(_lib.scuba_options_init(ctypes.byref(o)), "scuba_options_init")
    return o


# ---------------------------------------------------------------------------
# Host side: encode, CSR, verify
# ---------------------------------------------------------------------------

class Encoded:
    """Owner of a scuba_encoded handle plus its CSR copied out as numpy."""

    def __init__(self, handle, irs_buf, ir_offsets):
        self.handle = handle
        self.irs_buf = irs_buf
        self.ir_offsets = ir_offsets
        s = np.zeros(6, dtype=np.int64)
        _check(_lib.scuba_encoded_sizes(handle, _np_ptr(s)), "scuba_encoded_sizes")
        self.n, self.total_clauses, self.total_lits, self.total_vars, self.max_vars, \
            self.total_input_bits = (int(x) for x in s)
        n = self.n
        self.inst_clause_begin = np.zeros(n + 1, np.int64)
        self.clause_begin = np.zeros(self.total_clauses + 1, np.int64)
        self.lits = np.zeros(max(self.total_lits, 1), np.int32)
        self.inst_num_vars = np.zeros(max(n, 1), np.int32)
        self.inst_var_begin = np.zeros(n + 1, np.int64)
        _check(_lib.scuba_encoded_copy(handle, _np_ptr(self.inst_clause_begin),
                                       _np_ptr(self.clause_begin), _np_ptr(self.lits),
                                       _np_ptr(self.inst_num_vars),
                                       _np_ptr(self.inst_var_begin)), "scuba_encoded_copy")
        self.lits = self.lits[:self.total_lits]
        self.inst_num_vars = self.inst_num_vars[:n]

    def inputs(self):
        iib = np.zeros(self.n + 1, np.int64)
        nwords = 0
        # widths array length = total FREE words; bound by input bits
        widths = np.zeros(max(self.total_input_bits, 1), np.int32)
        var = np.zeros(max(self.total_input_bits, 1), np.int32)
        _check(_lib.scuba_encoded_inputs(self.handle, _np_ptr(iib), _np_ptr(widths),
                                         _np_ptr(var)), "scuba_encoded_inputs")
        nwords = int(iib[-1])
        return iib, widths[:nwords], var[:self.total_input_bits]

    def release_clauses(self) -> None:
        """Free the library-side clause storage (the numpy CSR copies stay)."""
        _check(_lib.scuba_encoded_release_clauses(self.handle), "scuba_encoded_release_clauses")

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.scuba_encoded_free(self.handle)
            self.handle = None


def scuba_encode_batch(irs: list, nthreads: int = 0) -> Encoded:
    offs = np.zeros(len(irs) + 1, dtype=np.int64)
    for i, a in enumerate(irs):
        offs[i + 1] = offs[i] + len(a)
    buf = np.ascontiguousarray(np.concatenate(irs) if irs else np.zeros(1, np.int64),
                               dtype=np.int64)
    h = _vp()
    _check(_lib.scuba_encode_batch(len(irs), _np_ptr(buf), _np_ptr(offs), int(nthreads),
                                   ctypes.byref(h)), "scuba_encode_batch")
    return Encoded(h, buf, offs)


def scuba_verify_batch(enc: Encoded, verdict: np.ndarray, model: np.ndarray,
                       nthreads: int = 0) -> tuple[int, np.ndarray]:
    verdict = np.ascontiguousarray(verdict, dtype=np.uint8)
    model = np.ascontiguousarray(model, dtype=np.uint8)
    ok = np.zeros(max(enc.n, 1), np.uint8)
    fails = _check(_lib.scuba_verify_batch(enc.handle, _np_ptr(enc.irs_buf),
                                           _np_ptr(enc.ir_offsets), _np_ptr(verdict),
                                           _np_ptr(model), int(nthreads), _np_ptr(ok)),
                   "scuba_verify_batch")
    return fails, ok[:enc.n]


# ---------------------------------------------------------------------------
# Device side: solve
# ---------------------------------------------------------------------------

def make_batch(n, max_vars, total_clauses, total_lits, total_vars, icb, cb, lits, nv, vb):
    """Fill a scuba_cnf_batch from integer device (or host) addresses."""
    b = scuba_cnf_batch()
    b.num_instances = int(n)
    b.max_vars = int(max_vars)
    b.total_clauses = int(total_clauses)
    b.total_lits = int(total_lits)
    b.total_vars = int(total_vars)
    b.inst_clause_begin = icb
    b.clause_begin = cb
    b.lits = lits
    b.inst_num_vars = nv
    b.inst_var_begin = vb
    return b


def scuba_solve_batch_ex(batch: scuba_cnf_batch, verdict_ptr: int, model_ptr, stream_ptr,
                         opt: scuba_options | None = None) -> int:
    if opt is None:
        opt = scuba_options_init()
    return _check(_lib.scuba_solve_batch_ex(ctypes.byref(batch), verdict_ptr, model_ptr,
                                            stream_ptr, ctypes.byref(opt)),
                  "scuba_solve_batch_ex")


def scuba_solve_batch(batch: scuba_cnf_batch, verdict_ptr: int, model_ptr, stream_ptr) -> int:
    return _check(_lib.scuba_solve_batch(ctypes.byref(batch), verdict_ptr, model_ptr,
                                         stream_ptr), "scuba_solve_batch")


def scuba_solve_batch_host(batch: scuba_cnf_batch, verdict: np.ndarray, model,
                           stream_ptr=None, opt: scuba_options | None = None) -> int:
    if opt is None:
        opt = scuba_options_init()
    return _lib.scuba_solve_batch_host(ctypes.byref(batch), _np_ptr(verdict),
                                       _np_ptr(model) if model is not None else None,
                                       stream_ptr, ctypes.byref(opt))


def scuba_solve_batch_noalloc(batch: scuba_cnf_batch, verdict_ptr: int, model_ptr, stream_ptr,
                              opt: scuba_options | None = None) -> int:
    """Allocation-free solve (fixed static scratch); waits and returns the
    device status. Raises on argument/size errors like the other calls."""
    if opt is None:
        opt = scuba_options_init()
    return _check(_lib.scuba_solve_batch_noalloc(ctypes.byref(batch), verdict_ptr, model_ptr,
                                                 stream_ptr, ctypes.byref(opt)),
                  "scuba_solve_batch_noalloc")


def scuba_solve_units(batch: scuba_cnf_batch, n_units: int, unit_inst_ptr, asm_begin_ptr,
                      asm_lits_ptr, unit_model_begin_ptr, verdict_ptr, model_ptr, stream_ptr,
                      opt: scuba_options | None = None) -> int:
    if opt is None:
        opt = scuba_options_init()
    return _check(_lib.scuba_solve_units(ctypes.byref(batch), int(n_units), unit_inst_ptr,
                                         asm_begin_ptr, asm_lits_ptr, unit_model_begin_ptr,
                                         verdict_ptr, model_ptr, stream_ptr, ctypes.byref(opt)),
                  "scuba_solve_units")


def scuba_sync_status(stream_ptr=None) -> int:
    return _lib.scuba_sync_status(stream_ptr)


def scuba_release() -> None:
    _lib.scuba_release()


def scuba_version() -> int:
    return _lib.scuba_version()
