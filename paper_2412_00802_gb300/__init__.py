"""GB300 (sm_103a) hypothesis evaluation for ALCQI(D) description logic.

Python binding of the C ABI declared in ``include/hedl.h``: each ``hedl_*``
function here marshals its arguments (torch CUDA tensors to device pointers,
numpy arrays to host pointers, the current torch stream to a cudaStream_t)
and calls the function of the same name in ``libhedl.so``.  Every evaluation
step runs in the library's CUDA kernels; there is no Python or CPU fallback,
and importing a function that needs the library fails loudly if it has not
been built (``paper_2412_00802_gb300.build.build()``).

``DeviceKB`` is a convenience owner: it copies host (numpy) arrays of a
knowledge base into torch device tensors (concept bitsets, role CSRs, property
columns, numeric and string concrete roles, the string table; the patterns
go to the library as host bytes), registers them and keeps them alive, and
offers ``score`` / ``eval`` that allocate outputs and workspaces with torch.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhedl.so")

HEDL_OK = 0
ERRORS = {-1: "HEDL_ERR_INVALID_ARG", -2: "HEDL_ERR_BAD_PROGRAM", -3: "HEDL_ERR_WORKSPACE_TOO_SMALL",
          -4: "HEDL_ERR_CUDA", -5: "HEDL_ERR_TIMEOUT", -6: "HEDL_ERR_BAD_KB", -7: "HEDL_ERR_NO_EXAMPLES",
          -8: "HEDL_ERR_OOM"}
HEDL_KB_NO_VALIDATE = 1
HEDL_NO_CSE = 1
HEDL_NO_GRAPH = 2
HEDL_PLAIN = 4
HEDL_LEVELS = 8
HEDL_NO_SLICE = 16
HEDL_SLICE_ALL = 32
HEDL_TEST_UNSAT_DEP = 0x100
HEDL_MAX_STACK = 64
HEDL_NOALLOC_SCRATCH_BYTES = 16 << 20

# exported symbols (one per declaration in include/hedl.h)
SYMBOLS = ("hedl_row_words", "hedl_kb_load", "hedl_kb_plan_only", "hedl_kb_free", "hedl_examples_set", "hedl_examples_counts",
           "hedl_validate", "hedl_plan_batch", "hedl_plan_batch_parallel", "hedl_plan_batch_device", "hedl_plan_info_get", "hedl_plan_image",
           "hedl_plan_free",
           "hedl_plan_execute",
           "hedl_plan_replay", "hedl_workspace_size", "hedl_score_batch", "hedl_eval_concept",
           "hedl_eval_concept_noalloc", "hedl_sync_status", "hedl_tuning_get", "hedl_tuning_set",
           "hedl_autotune_workspace_size", "hedl_autotune", "hedl_mlp_param_count", "hedl_mlp_create",
           "hedl_mlp_free", "hedl_mlp_get", "hedl_mlp_get_moments", "hedl_mlp_workspace_size", "hedl_encode", "hedl_mlp_forward",
           "hedl_mlp_gradients", "hedl_mlp_train_step", "hedl_scores_from_counts", "hedl_select_workspace_size",
           "hedl_select_top", "hedl_canonical_batch", "hedl_mlp_fit_target_map", "hedl_mlp_set_target_map",
           "hedl_mlp_get_target_map", "hedl_mlp_set_gemm", "hedl_mlp_status", "hedl_stat_scores",
           "hedl_last_error")


class HedlError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.msg = msg


class hedl_csr(ctypes.Structure):
    _fields_ = [("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("n_edges", ctypes.c_uint32)]


class hedl_numeric_role(ctypes.Structure):
    _fields_ = [("row_ptr", ctypes.c_void_p), ("vals", ctypes.c_void_p), ("n_vals", ctypes.c_uint32)]


class hedl_string_role(ctypes.Structure):
    _fields_ = [("row_ptr", ctypes.c_void_p), ("ids", ctypes.c_void_p), ("n_vals", ctypes.c_uint32)]


class hedl_kb_desc(ctypes.Structure):
    _fields_ = [("n_indiv", ctypes.c_uint32), ("n_concepts", ctypes.c_uint32), ("concept_bits", ctypes.c_void_p),
                ("n_roles", ctypes.c_uint32), ("roles", ctypes.c_void_p), ("inv_roles", ctypes.c_void_p),
                ("n_props", ctypes.c_uint32), ("prop_vals", ctypes.c_void_p), ("prop_stride", ctypes.c_uint64),
                ("n_num_roles", ctypes.c_uint32), ("num_roles", ctypes.c_void_p),
                ("n_str_roles", ctypes.c_uint32), ("str_roles", ctypes.c_void_p),
                ("n_strings", ctypes.c_uint32), ("str_off", ctypes.c_void_p), ("str_chars", ctypes.c_void_p),
                ("n_str_chars", ctypes.c_uint32),
                ("n_patterns", ctypes.c_uint32), ("pat_off", ctypes.c_void_p), ("pat_chars", ctypes.c_void_p)]


def _byte_table(items) -> Tuple[np.ndarray, np.ndarray]:
    """Byte strings as (uint32 offsets [len+1], uint8 bytes)."""
    items = [bytes(x) for x in items]
    off = np.zeros(len(items) + 1, np.uint32)
    if items:
        np.cumsum([len(x) for x in items], out=off[1:])
    return off, np.frombuffer(b"".join(items) or b"\0", np.uint8).copy()


class hedl_plan_info(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint32) for k in ("n_hyps", "n_nodes", "n_segments", "n_slots", "n_levels", "n_items",
                                                "tile_words", "n_role_ops", "n_role_groups", "n_data_ops",
                                                "n_atom_loads", "warp_words")] + \
               [(k, ctypes.c_uint64) for k in ("total_insns", "workspace_bytes", "image_bytes", "model_bytes")]


class hedl_tuning(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint32) for k in ("warps_per_cta", "words_per_lane", "rounds", "ctas_per_sm",
                                                "wait_timeout_ms", "stage_fillers", "role_block", "full_occupancy")]


_lib = None
_lock = threading.Lock()


def library(path: Optional[str] = None):
    """Load libhedl.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with paper_2412_00802_gb300.build.build()")
        L = ctypes.CDLL(p)
        P, U32, U64, I = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        sig = {
            "hedl_row_words": (U32, [U32]),
            "hedl_kb_load": (I, [P, ctypes.c_uint, P, ctypes.POINTER(P)]),
            "hedl_kb_plan_only": (I, [P, ctypes.POINTER(P)]),
            "hedl_kb_free": (None, [P]),
            "hedl_examples_set": (I, [P, P, P, P]),
            "hedl_examples_counts": (I, [P, ctypes.POINTER(U32), ctypes.POINTER(U32)]),
            "hedl_validate": (I, [P, P, U32]),
            "hedl_canonical_batch": (I, [P, P, U32, P]),
            "hedl_plan_batch": (I, [P, P, P, U32, ctypes.c_uint, ctypes.POINTER(P)]),
            "hedl_plan_batch_parallel": (I, [P, P, P, U32, ctypes.c_uint, U32, ctypes.POINTER(P)]),
            "hedl_plan_batch_device": (I, [P, P, P, U32, U64, ctypes.c_uint, P, ctypes.POINTER(P)]),
            "hedl_plan_info_get": (I, [P, ctypes.POINTER(hedl_plan_info)]),
            "hedl_plan_image": (I, [P, P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
            "hedl_plan_free": (None, [P]),
            "hedl_plan_execute": (I, [P, P, P, P, P, ctypes.c_size_t, P]),
            "hedl_plan_replay": (I, [P, P, P, P, P, ctypes.c_size_t, P]),
            "hedl_workspace_size": (I, [P, P, P, U32, ctypes.c_uint, ctypes.POINTER(ctypes.c_size_t)]),
            "hedl_score_batch": (I, [P, P, P, U32, P, P, ctypes.c_size_t, ctypes.c_uint, P]),
            "hedl_eval_concept": (I, [P, P, U32, P, P, ctypes.c_size_t, ctypes.c_uint, P]),
            "hedl_eval_concept_noalloc": (I, [P, P, U32, P, P]),
            "hedl_sync_status": (I, [P, P]),
            "hedl_tuning_get": (I, [P, ctypes.POINTER(hedl_tuning)]),
            "hedl_tuning_set": (I, [P, ctypes.POINTER(hedl_tuning)]),
            "hedl_autotune_workspace_size": (I, [P, P, P, U32, ctypes.POINTER(ctypes.c_size_t)]),
            "hedl_autotune": (I, [P, P, P, U32, P, ctypes.c_size_t, ctypes.c_char_p, P, ctypes.POINTER(hedl_tuning)]),
            "hedl_mlp_param_count": (U64, []),
            "hedl_mlp_create": (I, [P, ctypes.POINTER(P)]),
            "hedl_mlp_free": (None, [P]),
            "hedl_mlp_get": (I, [P, P, P, ctypes.POINTER(U32)]),
            "hedl_mlp_get_moments": (I, [P, P, P]),
            "hedl_mlp_workspace_size": (I, [U32, ctypes.POINTER(ctypes.c_size_t)]),
            "hedl_encode": (I, [P, P, U32, P, U32, P, U32, P, P, P]),
            "hedl_stat_scores": (I, [P, U32, P, P]),
            "hedl_mlp_forward": (I, [P, P, U32, P, P, ctypes.c_size_t, P]),
            "hedl_mlp_gradients": (I, [P, P, P, U32, P, P, ctypes.c_size_t, P]),
            "hedl_mlp_train_step": (I, [P, P, P, U32, ctypes.c_float, P, P, ctypes.c_size_t, P]),
            "hedl_scores_from_counts": (I, [P, U32, P, P]),
            "hedl_mlp_fit_target_map": (I, [P, P, U32, ctypes.c_float, P]),
            "hedl_mlp_set_target_map": (I, [P, P]),
            "hedl_mlp_get_target_map": (I, [P, P]),
            "hedl_mlp_set_gemm": (I, [P, ctypes.c_uint]),
            "hedl_mlp_status": (I, [P, P]),
            "hedl_select_workspace_size": (I, [U32, ctypes.POINTER(ctypes.c_size_t)]),
            "hedl_select_top": (I, [P, U32, U32, P, P, ctypes.c_size_t, P]),
            "hedl_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        if path is None:
            _lib = L
        return L


def hedl_last_error() -> str:
    return library().hedl_last_error().decode()


def _check(rc: int):
    if rc != HEDL_OK:
        raise HedlError(rc, hedl_last_error())


def _stream(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _dptr(t) -> Optional[int]:
    """Device pointer of a CUDA tensor (None for None)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _host_u64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint64)


def _host_u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


# ---------------------------------------------------------------------------- C-ABI calls
def hedl_row_words(n_indiv: int) -> int:
    return int(library().hedl_row_words(n_indiv))


class KBHandle:
    """An opaque hedl_kb* plus the tensors it borrows (kept alive here)."""

    def __init__(self, ptr: int, keep: list, n: int, wp: int):
        self.ptr = ptr
        self.keep = keep
        self.n = n
        self.wp = wp

    def __del__(self):
        try:
            if self.ptr:
                library().hedl_kb_free(self.ptr)
                self.ptr = None
        except Exception:
            pass


def hedl_kb_load(n_indiv: int, concept_bits, roles: Sequence[Tuple[object, object]],
                 inv_roles: Sequence[Tuple[object, object]], prop_vals, flags: int = 0, stream=None,
                 num_roles: Sequence[Tuple[object, object]] = (), str_roles: Sequence[Tuple[object, object]] = (),
                 str_table: Optional[Tuple[object, object, int, int]] = None,
                 patterns: Sequence[bytes] = ()) -> KBHandle:
    """concept_bits: CUDA [C, row_words] 32-bit tensor; roles / inv_roles: (row_ptr, col) CUDA int32 tensors;
    prop_vals: CUDA float32 [P, stride] (or None); num_roles: (row_ptr int32, vals float32) CUDA tensors
    of the numeric concrete roles (property ids P + q); str_roles: (row_ptr, ids) CUDA int32 tensors of
    the string concrete roles; str_table: (offsets int32 [S+1], chars uint8) CUDA tensors, S and the
    number of chars; patterns: the substring patterns (host bytes)."""
    n_roles = len(roles)
    csr = (hedl_csr * max(n_roles, 1))()
    icsr = (hedl_csr * max(n_roles, 1))()
    for r in range(n_roles):
        rp, col = roles[r]
        csr[r] = hedl_csr(_dptr(rp), _dptr(col) if col.numel() else None, int(col.numel()))
        rp, col = inv_roles[r]
        icsr[r] = hedl_csr(_dptr(rp), _dptr(col) if col.numel() else None, int(col.numel()))
    n_c = int(concept_bits.shape[0]) if concept_bits is not None else 0
    n_p = int(prop_vals.shape[0]) if prop_vals is not None else 0
    Q = len(num_roles)
    nums = (hedl_numeric_role * max(Q, 1))()
    for q, (rp, vals) in enumerate(num_roles):
        nums[q] = hedl_numeric_role(_dptr(rp), _dptr(vals) if vals.numel() else None, int(vals.numel()))
    SR = len(str_roles)
    strs = (hedl_string_role * max(SR, 1))()
    for q, (rp, ids) in enumerate(str_roles):
        strs[q] = hedl_string_role(_dptr(rp), _dptr(ids) if ids.numel() else None, int(ids.numel()))
    t_off, t_chars, n_str, n_chars = str_table if str_table is not None else (None, None, 0, 0)
    p_off, p_chars = _byte_table(patterns)
    d = hedl_kb_desc(n_indiv, n_c, _dptr(concept_bits) if n_c else None, n_roles,
                     ctypes.addressof(csr) if n_roles else None, ctypes.addressof(icsr) if n_roles else None,
                     n_p, _dptr(prop_vals) if n_p else None, int(prop_vals.stride(0)) if n_p else 0,
                     Q, ctypes.addressof(nums) if Q else None,
                     SR, ctypes.addressof(strs) if SR else None,
                     n_str, _dptr(t_off) if n_str else None, _dptr(t_chars) if n_chars else None, n_chars,
                     len(patterns), p_off.ctypes.data if patterns else None, p_chars.ctypes.data if patterns else None)
    out = ctypes.c_void_p()
    _check(library().hedl_kb_load(ctypes.byref(d), flags, _stream(stream), ctypes.byref(out)))
    return KBHandle(out.value, [concept_bits, roles, inv_roles, prop_vals, num_roles, str_roles, str_table],
                    n_indiv, hedl_row_words(n_indiv))


def hedl_kb_plan_only(n_indiv: int, n_concepts: int, role_edges: Sequence[int], n_props: int,
                      num_role_vals: Sequence[int] = (), str_role_vals: Sequence[int] = (), n_strings: int = 0,
                      n_patterns: int = 0) -> KBHandle:
    """Planning-only handle from sizes (no CUDA call; works without a GPU)."""
    R = len(role_edges)
    csr = (hedl_csr * max(R, 1))()
    for r, e in enumerate(role_edges):
        csr[r] = hedl_csr(None, None, int(e))
    Q = len(num_role_vals)
    nums = (hedl_numeric_role * max(Q, 1))()
    for q, m in enumerate(num_role_vals):
        nums[q] = hedl_numeric_role(None, None, int(m))
    SR = len(str_role_vals)
    strs = (hedl_string_role * max(SR, 1))()
    for q, m in enumerate(str_role_vals):
        strs[q] = hedl_string_role(None, None, int(m))
    d = hedl_kb_desc(n_indiv, n_concepts, None, R, ctypes.addressof(csr) if R else None,
                     ctypes.addressof(csr) if R else None, n_props, None, n_indiv,
                     Q, ctypes.addressof(nums) if Q else None, SR, ctypes.addressof(strs) if SR else None,
                     n_strings, None, None, 0, n_patterns, None, None)
    out = ctypes.c_void_p()
    _check(library().hedl_kb_plan_only(ctypes.byref(d), ctypes.byref(out)))
    return KBHandle(out.value, [csr, nums, strs], n_indiv, hedl_row_words(n_indiv))


def hedl_kb_free(kb: KBHandle):
    if kb.ptr:
        library().hedl_kb_free(kb.ptr)
        kb.ptr = None


def hedl_examples_set(kb: KBHandle, pos_bits, neg_bits, stream=None):
    _check(library().hedl_examples_set(kb.ptr, _dptr(pos_bits), _dptr(neg_bits), _stream(stream)))
    kb.keep.append((pos_bits, neg_bits))


def hedl_examples_counts(kb: KBHandle) -> Tuple[int, int]:
    a, b = ctypes.c_uint32(), ctypes.c_uint32()
    _check(library().hedl_examples_counts(kb.ptr, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def hedl_validate(kb: KBHandle, prog) -> None:
    p = _host_u64(prog)
    _check(library().hedl_validate(kb.ptr, p.ctypes.data if p.size else None, p.size))


def hedl_canonical_batch(progs, offs) -> np.ndarray:
    """Canonical forms (AND / OR operands in ascending byte order) of host programs, same offsets."""
    p, o = _host_u64(progs), _host_u32(offs)
    out = np.empty_like(p)
    _check(library().hedl_canonical_batch(p.ctypes.data if p.size else None, o.ctypes.data, o.size - 1,
                                          out.ctypes.data if out.size else None))
    return out


class Plan:
    def __init__(self, ptr: int):
        self.ptr = ptr

    def __del__(self):
        try:
            if self.ptr:
                library().hedl_plan_free(self.ptr)
                self.ptr = None
        except Exception:
            pass


def hedl_plan_batch(kb: KBHandle, progs, offs, flags: int = 0) -> Plan:
    p, o = _host_u64(progs), _host_u32(offs)
    out = ctypes.c_void_p()
    _check(library().hedl_plan_batch(kb.ptr, p.ctypes.data if p.size else None, o.ctypes.data, o.size - 1, flags,
                                     ctypes.byref(out)))
    return Plan(out.value)


def hedl_plan_batch_parallel(kb: KBHandle, progs, offs, flags: int = 0, n_threads: int = 0) -> Plan:
    """The no-sharing, no-slicing plan of the batch, built per hypothesis on n_threads host threads."""
    p, o = _host_u64(progs), _host_u32(offs)
    out = ctypes.c_void_p()
    _check(library().hedl_plan_batch_parallel(kb.ptr, p.ctypes.data if p.size else None, o.ctypes.data, o.size - 1,
                                              flags, n_threads, ctypes.byref(out)))
    return Plan(out.value)


def hedl_plan_batch_device(kb: KBHandle, progs_dev, offs_dev, n_insns: int, flags: int = 0, stream=None) -> Plan:
    """The no-sharing, no-slicing plan of the batch built on the device from DEVICE programs
    (progs_dev: int64/uint64 tensor of n_insns instructions, offs_dev: int32 tensor [H+1])."""
    out = ctypes.c_void_p()
    _check(library().hedl_plan_batch_device(kb.ptr, _dptr(progs_dev), _dptr(offs_dev), offs_dev.numel() - 1,
                                            n_insns, flags, _stream(stream), ctypes.byref(out)))
    return Plan(out.value)


def hedl_plan_info_get(plan: Plan) -> Dict[str, int]:
    info = hedl_plan_info()
    _check(library().hedl_plan_info_get(plan.ptr, ctypes.byref(info)))
    return {k: int(getattr(info, k)) for k, _ in hedl_plan_info._fields_}


def hedl_plan_image(plan: Plan) -> np.ndarray:
    """The plan's image (uint8, host copy): the work queue the interpreter reads."""
    lib = library()
    n = ctypes.c_size_t(0)
    rc = lib.hedl_plan_image(plan.ptr, None, 0, ctypes.byref(n))   # sizes it (fails only on a NULL plan)
    if rc != 0 and n.value == 0:
        _check(rc)
    out = np.zeros(n.value, np.uint8)
    if n.value:
        _check(lib.hedl_plan_image(plan.ptr, out.ctypes.data, out.size, ctypes.byref(n)))
    return out


def hedl_plan_free(plan: Plan):
    if plan.ptr:
        library().hedl_plan_free(plan.ptr)
        plan.ptr = None


def hedl_plan_execute(kb: KBHandle, plan: Plan, counts, out_bits, ws, stream=None):
    _check(library().hedl_plan_execute(kb.ptr, plan.ptr, _dptr(counts), _dptr(out_bits), _dptr(ws),
                                       ws.numel() * ws.element_size(), _stream(stream)))


def hedl_plan_replay(kb: KBHandle, plan: Plan, counts, out_bits, ws, stream=None):
    _check(library().hedl_plan_replay(kb.ptr, plan.ptr, _dptr(counts), _dptr(out_bits), _dptr(ws),
                                      ws.numel() * ws.element_size(), _stream(stream)))


def hedl_workspace_size(kb: KBHandle, progs, offs, flags: int = 0) -> int:
    p, o = _host_u64(progs), _host_u32(offs)
    out = ctypes.c_size_t()
    _check(library().hedl_workspace_size(kb.ptr, p.ctypes.data if p.size else None, o.ctypes.data, o.size - 1,
                                         flags, ctypes.byref(out)))
    return out.value


def hedl_score_batch(kb: KBHandle, progs, offs, counts, ws, flags: int = 0, stream=None):
    p, o = _host_u64(progs), _host_u32(offs)
    _check(library().hedl_score_batch(kb.ptr, p.ctypes.data if p.size else None, o.ctypes.data, o.size - 1,
                                      _dptr(counts), _dptr(ws), ws.numel() * ws.element_size(), flags,
                                      _stream(stream)))


def hedl_eval_concept(kb: KBHandle, prog, out_bits, ws, flags: int = 0, stream=None):
    p = _host_u64(prog)
    _check(library().hedl_eval_concept(kb.ptr, p.ctypes.data if p.size else None, p.size, _dptr(out_bits),
                                       _dptr(ws), ws.numel() * ws.element_size(), flags, _stream(stream)))


def hedl_eval_concept_noalloc(kb: KBHandle, prog, out_bits, stream=None):
    """Evaluate one program into out_bits using the library's built-in scratch (no allocation)."""
    p = _host_u64(prog)
    _check(library().hedl_eval_concept_noalloc(kb.ptr, p.ctypes.data if p.size else None, p.size,
                                               _dptr(out_bits), _stream(stream)))


def hedl_sync_status(kb: KBHandle, stream=None):
    _check(library().hedl_sync_status(kb.ptr, _stream(stream)))


def hedl_tuning_get(kb: KBHandle) -> Dict[str, int]:
    t = hedl_tuning()
    _check(library().hedl_tuning_get(kb.ptr, ctypes.byref(t)))
    return {k: int(getattr(t, k)) for k, _ in hedl_tuning._fields_}


def hedl_tuning_set(kb: KBHandle, **kw):
    t = hedl_tuning(**{**hedl_tuning_get(kb), **kw})
    _check(library().hedl_tuning_set(kb.ptr, ctypes.byref(t)))


def hedl_autotune_workspace_size(kb: KBHandle, progs, offs) -> int:
    p, o = _host_u64(progs), _host_u32(offs)
    out = ctypes.c_size_t()
    _check(library().hedl_autotune_workspace_size(kb.ptr, p.ctypes.data if p.size else None, o.ctypes.data,
                                                  o.size - 1, ctypes.byref(out)))
    return out.value


def hedl_autotune(kb: KBHandle, progs, offs, ws, cache_path: Optional[str] = None, stream=None) -> Dict[str, int]:
    """Time candidate launch shapes on the probe batch and keep the fastest; returns it."""
    p, o = _host_u64(progs), _host_u32(offs)
    t = hedl_tuning()
    _check(library().hedl_autotune(kb.ptr, p.ctypes.data if p.size else None, o.ctypes.data, o.size - 1, _dptr(ws),
                                   ws.numel() * ws.element_size(), cache_path.encode() if cache_path else None,
                                   _stream(stream), ctypes.byref(t)))
    return {k: int(getattr(t, k)) for k, _ in hedl_tuning._fields_}


# ---------------------------------------------------------------------------- surrogate
ENC_DIM = 512


def hedl_mlp_param_count() -> int:
    return int(library().hedl_mlp_param_count())


class MLPHandle:
    def __init__(self, ptr):
        self.ptr = ptr

    def __del__(self):
        try:
            if self.ptr:
                library().hedl_mlp_free(self.ptr)
                self.ptr = None
        except Exception:
            pass


def hedl_mlp_create(params: np.ndarray) -> MLPHandle:
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.size != hedl_mlp_param_count():
        raise ValueError("wrong parameter count")
    out = ctypes.c_void_p()
    _check(library().hedl_mlp_create(p.ctypes.data, ctypes.byref(out)))
    return MLPHandle(out.value)


def hedl_mlp_free(m: MLPHandle):
    if m.ptr:
        library().hedl_mlp_free(m.ptr)
        m.ptr = None


def hedl_mlp_get(m: MLPHandle):
    n = hedl_mlp_param_count()
    p = np.zeros(n, np.float32)
    g = np.zeros(n, np.float32)
    step = ctypes.c_uint32()
    _check(library().hedl_mlp_get(m.ptr, p.ctypes.data, g.ctypes.data, ctypes.byref(step)))
    return p, g, step.value


def hedl_mlp_get_moments(m: MLPHandle):
    """Adam's first and second moments (float32 arrays of hedl_mlp_param_count() values)."""
    n = hedl_mlp_param_count()
    first = np.zeros(n, np.float32)
    second = np.zeros(n, np.float32)
    _check(library().hedl_mlp_get_moments(m.ptr, first.ctypes.data, second.ctypes.data))
    return first, second


def hedl_mlp_workspace_size(B: int) -> int:
    out = ctypes.c_size_t()
    _check(library().hedl_mlp_workspace_size(B, ctypes.byref(out)))
    return out.value


def hedl_encode(progs_dev, offs_dev, X, grid=None, prior=None, stats=None, n_stat_concepts=0, stream=None):
    """progs_dev: CUDA int64 tensor of instructions; offs_dev: CUDA int32 [H+1]; X: CUDA bf16 [H][512];
    grid: CUDA float32 [n_props][15] threshold boundaries or None; prior: CUDA float32 [H][2] or None;
    stats: CUDA int32 statistics table (n_stat_concepts atom scores, then n_props x 2 x 16) or None."""
    H = offs_dev.numel() - 1
    _check(library().hedl_encode(_dptr(progs_dev), _dptr(offs_dev), H, _dptr(grid),
                                 0 if grid is None else grid.shape[0], _dptr(stats), n_stat_concepts, _dptr(prior),
                                 _dptr(X), _stream(stream)))


def hedl_stat_scores(scores, out, stream=None):
    """out (CUDA int32 [n]) = round((scores[:, 0] - 1/2) * 32) for exact scores (CUDA float32 [n][2])."""
    _check(library().hedl_stat_scores(_dptr(scores), scores.shape[0], _dptr(out), _stream(stream)))


def hedl_mlp_forward(m: MLPHandle, X, Y, ws, stream=None):
    _check(library().hedl_mlp_forward(m.ptr, _dptr(X), X.shape[0], _dptr(Y), _dptr(ws),
                                      ws.numel() * ws.element_size(), _stream(stream)))


def hedl_mlp_gradients(m: MLPHandle, X, T, ws, loss=None, stream=None):
    _check(library().hedl_mlp_gradients(m.ptr, _dptr(X), _dptr(T), X.shape[0], _dptr(loss), _dptr(ws),
                                        ws.numel() * ws.element_size(), _stream(stream)))


def hedl_mlp_train_step(m: MLPHandle, X, T, lr: float, ws, loss=None, stream=None):
    _check(library().hedl_mlp_train_step(m.ptr, _dptr(X), _dptr(T), X.shape[0], lr, _dptr(loss), _dptr(ws),
                                         ws.numel() * ws.element_size(), _stream(stream)))


def hedl_mlp_fit_target_map(m: MLPHandle, T, tail_weight: float, stream=None):
    _check(library().hedl_mlp_fit_target_map(m.ptr, _dptr(T), T.shape[0], tail_weight, _stream(stream)))


def hedl_mlp_set_target_map(m: MLPHandle, tmap):
    a = np.ascontiguousarray(tmap, np.float32)
    _check(library().hedl_mlp_set_target_map(m.ptr, a.ctypes.data))


def hedl_mlp_get_target_map(m: MLPHandle) -> np.ndarray:
    a = np.zeros(5, np.float32)
    _check(library().hedl_mlp_get_target_map(m.ptr, a.ctypes.data))
    return a


HEDL_GEMM_TCGEN05 = 0
HEDL_GEMM_MMA_SYNC = 1


def hedl_mlp_set_gemm(m: MLPHandle, engine: int):
    _check(library().hedl_mlp_set_gemm(m.ptr, engine))


def hedl_mlp_status(m: MLPHandle, stream=None):
    _check(library().hedl_mlp_status(m.ptr, _stream(stream)))


def hedl_scores_from_counts(counts, scores, stream=None):
    _check(library().hedl_scores_from_counts(_dptr(counts), counts.shape[0], _dptr(scores), _stream(stream)))


def hedl_select_workspace_size(H: int) -> int:
    out = ctypes.c_size_t()
    _check(library().hedl_select_workspace_size(H, ctypes.byref(out)))
    return out.value


def hedl_select_top(Y, k: int, idx, ws, stream=None):
    _check(library().hedl_select_top(_dptr(Y), Y.shape[0], k, _dptr(idx), _dptr(ws),
                                     ws.numel() * ws.element_size(), _stream(stream)))


# ---------------------------------------------------------------------------- convenience owner
class DeviceKB:
    """Device copy (torch tensors) of a KB given as host numpy arrays, registered with the library."""

    def __init__(self, n: int, concept_bits: np.ndarray, row_ptr: List[np.ndarray], col: List[np.ndarray],
                 inv_row_ptr: List[np.ndarray], inv_col: List[np.ndarray], prop_vals: np.ndarray,
                 pos_bits: Optional[np.ndarray] = None, neg_bits: Optional[np.ndarray] = None,
                 device: str = "cuda", flags: int = 0, num_row_ptr: Sequence[np.ndarray] = (),
                 num_vals: Sequence[np.ndarray] = (), str_row_ptr: Sequence[np.ndarray] = (),
                 str_ids: Sequence[np.ndarray] = (), strings: Sequence[bytes] = (),
                 patterns: Sequence[bytes] = ()):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.n = n
        self.wp = hedl_row_words(n)
        t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).view(dt)).to(self.device)
        self.concepts = t(concept_bits.reshape(-1, self.wp), np.int32) if concept_bits.size else \
            torch.zeros((0, self.wp), dtype=torch.int32, device=self.device)
        self.roles = [(t(rp, np.int32), t(c, np.int32)) for rp, c in zip(row_ptr, col)]
        self.inv_roles = [(t(rp, np.int32), t(c, np.int32)) for rp, c in zip(inv_row_ptr, inv_col)]
        # property rows padded to a multiple of 4 floats (16-byte rows)
        P = prop_vals.shape[0] if prop_vals is not None else 0
        stride = (n + 3) // 4 * 4
        pv = np.full((P, stride), np.nan, dtype=np.float32)
        if P:
            pv[:, :n] = prop_vals
        self.props = torch.from_numpy(pv).to(self.device) if P else None
        self.num_roles = [(t(rp, np.int32), t(np.asarray(v, np.float32), np.float32))
                          for rp, v in zip(num_row_ptr, num_vals)]
        self.str_roles = [(t(rp, np.int32), t(np.asarray(ids, np.uint32), np.int32))
                          for rp, ids in zip(str_row_ptr, str_ids)]
        table = None
        if len(strings):
            off, chars = _byte_table(strings)
            table = (t(off, np.int32), torch.from_numpy(chars).to(self.device), len(strings), int(off[-1]))
        with torch.cuda.device(self.device):
            self.handle = hedl_kb_load(n, self.concepts if self.concepts.shape[0] else None, self.roles,
                                       self.inv_roles, self.props, flags, num_roles=self.num_roles,
                                       str_roles=self.str_roles, str_table=table, patterns=list(patterns))
            if pos_bits is not None:
                self.set_examples(pos_bits, neg_bits)
        self._ws = None

    @classmethod
    def from_synth(cls, kb, device: str = "cuda", flags: int = 0) -> "DeviceKB":
        return cls(kb.n, kb.concept_bits, kb.row_ptr, kb.col, kb.inv_row_ptr, kb.inv_col, kb.prop_vals,
                   kb.pos_bits, kb.neg_bits, device, flags, getattr(kb, "num_row_ptr", ()),
                   getattr(kb, "num_vals", ()), getattr(kb, "str_row_ptr", ()), getattr(kb, "str_ids", ()),
                   getattr(kb, "strings", ()), getattr(kb, "patterns", ()))

    def set_examples(self, pos_bits: np.ndarray, neg_bits: np.ndarray):
        self.pos = self.torch.from_numpy(np.ascontiguousarray(pos_bits).view(np.int32)).to(self.device)
        self.neg = self.torch.from_numpy(np.ascontiguousarray(neg_bits).view(np.int32)).to(self.device)
        hedl_examples_set(self.handle, self.pos, self.neg)

    def workspace(self, nbytes: int):
        torch = self.torch
        if self._ws is None or self._ws.numel() < nbytes:
            self._ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        return self._ws

    def score(self, progs, offs, flags: int = 0, out_bits: bool = False):
        """Counts uint32[H][4] (TP, FP, FN, TN) as numpy, plus instance sets uint32[H][wp] if out_bits."""
        torch = self.torch
        H = len(offs) - 1
        plan = hedl_plan_batch(self.handle, progs, offs, flags)
        info = hedl_plan_info_get(plan)
        ws = self.workspace(info["workspace_bytes"])
        counts = torch.zeros((H, 4), dtype=torch.int32, device=self.device)
        bits = torch.zeros((H, self.wp), dtype=torch.int32, device=self.device) if out_bits else None
        hedl_plan_execute(self.handle, plan, counts, bits, ws)
        hedl_sync_status(self.handle)
        c = counts.cpu().numpy().view(np.uint32)
        if out_bits:
            return c, bits.cpu().numpy().view(np.uint32)
        return c

    def autotune(self, progs, offs, cache_path: Optional[str] = None) -> Dict[str, int]:
        """Pick the fastest launch shape on a probe batch (allocates its scratch with torch)."""
        torch = self.torch
        need = hedl_autotune_workspace_size(self.handle, progs, offs)
        ws = torch.empty(need + 256 + 16 * (len(offs) - 1) + 256, dtype=torch.uint8, device=self.device)
        return hedl_autotune(self.handle, progs, offs, ws, cache_path)

    def eval(self, prog, flags: int = 0) -> np.ndarray:
        torch = self.torch
        offs = np.array([0, len(prog)], dtype=np.uint32)
        nbytes = hedl_workspace_size(self.handle, prog, offs, flags)
        ws = self.workspace(nbytes)
        out = torch.zeros(self.wp, dtype=torch.int32, device=self.device)
        hedl_eval_concept(self.handle, prog, out, ws, flags)
        hedl_sync_status(self.handle)
        return out.cpu().numpy().view(np.uint32)
