"""GB300-native Monte Carlo decoding of the 3D toric code (arXiv:2212.06985).

Thin ctypes binding over the C ABI of ``include/toric3d.h`` (libtoric3d.so,
built for sm_103a by ``build.py``).  Every function here only marshals
arguments -- torch tensors become device pointers, the current torch stream
becomes the CUDA stream -- and every step of the decoding path runs in the
library's CUDA kernels.  There is no CPU path: if the library cannot be
loaded, every call raises.

Bit-sliced arrays are torch.int64 tensors used as raw 64-bit words
(``[3L^3, words]``; sample 64*w + j is bit j of word w).
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

__all__ = [
    "TannerGraph", "tanner_prepare",
    "T3DError", "RunCfg", "lib", "n_bits", "words_for", "table1_schedule",
    "toric3d_noise", "toric3d_syndrome", "toric3d_flip", "toric3d_pflip",
    "toric3d_bp_step", "toric3d_bp_decide", "toric3d_bp_decide_workspace_bytes", "toric3d_bp", "toric3d_logical",
    "toric3d_pack", "toric3d_unpack", "toric3d_run_cycles",
    "toric3d_flip_workspace_bytes", "toric3d_bp_message_bytes",
    "toric3d_bp_workspace_bytes", "toric3d_run_workspace_bytes", "make_run_cfg",
    "toric3d_profile_enable", "toric3d_profile_reset", "toric3d_profile_read", "KERNEL_KINDS",
    "EXPORTED_SYMBOLS", "replica_sample0", "BatchItem", "make_batch", "toric3d_run_batch",
    "toric3d_run_batch_workspace_bytes", "toric3d_set_blocks_per_sm", "toric3d_get_blocks_per_sm",
    "toric3d_autotune_batch", "toric3d_flip_noalloc", "toric3d_gate_workspace_bytes", "toric3d_gate",
    "toric3d_flip_until_clear_workspace_bytes", "toric3d_flip_until_clear",
    "toric3d_bp_meta_workspace_bytes", "toric3d_bp_meta", "toric3d_bp_meta_message_bytes", "toric3d_bp_meta_step",
    "toric3d_tanner_bytes", "toric3d_tanner_prepare", "toric3d_tanner_noise", "toric3d_tanner_syndrome",
    "toric3d_tanner_flip_workspace_bytes", "toric3d_tanner_pflip", "toric3d_tanner_bp_workspace_bytes",
    "toric3d_tanner_bp", "toric3d_tanner_bp_message_bytes", "toric3d_tanner_bp_step",
]

EXPORTED_SYMBOLS = [
    "toric3d_last_error", "toric3d_abi_version", "toric3d_noise", "toric3d_syndrome",
    "toric3d_flip_workspace_bytes", "toric3d_flip", "toric3d_pflip", "toric3d_bp_message_bytes",
    "toric3d_bp_step", "toric3d_bp_decide_workspace_bytes", "toric3d_bp_decide",
    "toric3d_bp_workspace_bytes", "toric3d_bp",
    "toric3d_logical", "toric3d_pack", "toric3d_unpack", "toric3d_run_workspace_bytes",
    "toric3d_run_cycles", "toric3d_run_batch_workspace_bytes", "toric3d_run_batch",
    "toric3d_set_blocks_per_sm", "toric3d_get_blocks_per_sm", "toric3d_autotune_batch",
    "toric3d_profile_enable", "toric3d_profile_reset", "toric3d_profile_read", "toric3d_flip_noalloc",
    "toric3d_flip_until_clear_workspace_bytes", "toric3d_flip_until_clear",
    "toric3d_cnn_param_count", "toric3d_cnn_blob_bytes", "toric3d_cnn_prepare", "toric3d_cnn_workspace_bytes",
    "toric3d_cnn_decode", "toric3d_cnn_train_workspace_bytes", "toric3d_cnn_train_step",
    "toric3d_gate_workspace_bytes", "toric3d_gate", "toric3d_cnn_status", "toric3d_cnn_debug_wait_limit",
    "toric3d_bp_meta_workspace_bytes", "toric3d_bp_meta", "toric3d_bp_meta_message_bytes", "toric3d_bp_meta_step",
    "toric3d_tanner_bytes", "toric3d_tanner_prepare", "toric3d_tanner_noise", "toric3d_tanner_syndrome",
    "toric3d_tanner_flip_workspace_bytes", "toric3d_tanner_pflip", "toric3d_tanner_bp_workspace_bytes",
    "toric3d_tanner_bp", "toric3d_tanner_bp_message_bytes", "toric3d_tanner_bp_step",
]

KERNEL_KINDS = {"noise": 0, "syndrome": 1, "flip": 2, "pflip": 3, "bp_step": 4, "bp_decide": 5,
                "logical": 6, "layout": 7, "cnn": 8}


class T3DError(RuntimeError):
    """A toric3d call returned an error status."""

    def __init__(self, status: int, message: str):
        super().__init__(f"toric3d error {status}: {message}")
        self.status = status


class Tanner(ctypes.Structure):
    """Mirror of ``t3d_tanner`` in include/toric3d.h."""

    _fields_ = [
        ("n_vars", ctypes.c_int64),
        ("n_checks", ctypes.c_int64),
        ("n_edges", ctypes.c_int64),
        ("max_var_degree", ctypes.c_int32),
        ("max_check_degree", ctypes.c_int32),
        ("cptr", ctypes.c_void_p),
        ("cvar", ctypes.c_void_p),
        ("vptr", ctypes.c_void_p),
        ("vedge", ctypes.c_void_p),
        ("vcheck", ctypes.c_void_p),
    ]


class RunCfg(ctypes.Structure):
    """Mirror of ``t3d_run_cfg`` in include/toric3d.h."""

    _fields_ = [
        ("L", ctypes.c_int32),
        ("T", ctypes.c_int32),
        ("p", ctypes.c_double),
        ("q", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("sample0", ctypes.c_uint64),
        ("n_samples", ctypes.c_int64),
        ("use_bp", ctypes.c_int32),
        ("bp_iters", ctypes.c_int32),
        ("bp_meas_nodes", ctypes.c_int32),
        ("n_apply", ctypes.c_int32),
        ("schedule", ctypes.c_char * 64),
        ("perfect_round", ctypes.c_int32),
        ("perfect_max_sweeps", ctypes.c_int32),
        ("cycle0", ctypes.c_uint32),
        ("use_graph", ctypes.c_int32),
        ("bp_chunk_samples", ctypes.c_int64),
        ("cnn_blob", ctypes.c_void_p),
        ("fallback_max_weight", ctypes.c_int32),
        ("fallback_sigmas", ctypes.c_double),
    ]


class BatchItem(ctypes.Structure):
    """Mirror of ``t3d_batch_item`` in include/toric3d.h."""

    _fields_ = [
        ("L", ctypes.c_int32),
        ("n_samples", ctypes.c_int64),
        ("sample0", ctypes.c_uint64),
        ("e", ctypes.c_void_p),
        ("mask", ctypes.c_void_p),
        ("counts8", ctypes.c_void_p),
        ("s_prev", ctypes.c_void_p),
        ("fallback_words", ctypes.c_void_p),
    ]


_lock = threading.Lock()
_lib = None
_P = ctypes.c_void_p


def lib():
    """Load libtoric3d.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            handle = ctypes.CDLL(path)
            _declare(handle)
            _lib = handle
    return _lib


def _declare(h):
    i32, i64, u32, u64, dbl, sz = (ctypes.c_int, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64,
                                   ctypes.c_double, ctypes.c_size_t)
    sig = {
        "toric3d_last_error": (ctypes.c_char_p, []),
        "toric3d_abi_version": (i32, []),
        "toric3d_noise": (i32, [i32, i64, _P, dbl, u64, u64, u32, _P]),
        "toric3d_syndrome": (i32, [i32, i64, _P, _P, dbl, u64, u64, u32, _P]),
        "toric3d_flip_workspace_bytes": (sz, [i32, i64]),
        "toric3d_flip": (i32, [i32, i64, _P, _P, i32, _P, sz, _P]),
        "toric3d_flip_noalloc": (i32, [i32, i64, _P, _P, i32, _P]),
        "toric3d_flip_until_clear_workspace_bytes": (sz, [i32, i64]),
        "toric3d_flip_until_clear": (i32, [i32, i64, _P, _P, i32, _P, _P, sz, _P]),
        "toric3d_pflip": (i32, [i32, i64, _P, _P, ctypes.c_char_p, i32, u32, u64, u64, u32, _P, sz, _P]),
        "toric3d_bp_message_bytes": (sz, [i32, i64]),
        "toric3d_bp_step": (i32, [i32, i64, _P, dbl, dbl, _P, _P, _P]),
        "toric3d_bp_decide_workspace_bytes": (sz, [i32, i64]),
        "toric3d_bp_decide": (i32, [i32, i64, _P, dbl, _P, _P, _P, _P, sz, _P]),
        "toric3d_bp_workspace_bytes": (sz, [i32, i64]),
        "toric3d_bp": (i32, [i32, i64, _P, _P, dbl, dbl, i32, _P, sz, _P, _P]),
        "toric3d_bp_meta_workspace_bytes": (sz, [i32, i64]),
        "toric3d_bp_meta": (i32, [i32, i64, _P, _P, dbl, dbl, i32, _P, sz, _P, _P]),
        "toric3d_bp_meta_message_bytes": (sz, [i32, i64]),
        "toric3d_tanner_bytes": (sz, [i64, i64, i64]),
        "toric3d_tanner_prepare": (i32, [i64, i64, _P, _P, _P, sz, ctypes.POINTER(Tanner)]),
        "toric3d_tanner_noise": (i32, [ctypes.POINTER(Tanner), i64, _P, dbl, u64, u64, u32, _P]),
        "toric3d_tanner_syndrome": (i32, [ctypes.POINTER(Tanner), i64, _P, _P, dbl, u64, u64, u32, _P]),
        "toric3d_tanner_flip_workspace_bytes": (sz, [ctypes.POINTER(Tanner), i64]),
        "toric3d_tanner_pflip": (i32, [ctypes.POINTER(Tanner), i64, _P, _P, ctypes.c_char_p, i32, u32, u64, u64, u32,
                                       _P, sz, _P]),
        "toric3d_tanner_bp_workspace_bytes": (sz, [ctypes.POINTER(Tanner), i64]),
        "toric3d_tanner_bp": (i32, [ctypes.POINTER(Tanner), i64, _P, _P, _P, i32, _P, sz, _P, _P]),
        "toric3d_tanner_bp_message_bytes": (sz, [ctypes.POINTER(Tanner), i64]),
        "toric3d_tanner_bp_step": (i32, [ctypes.POINTER(Tanner), i64, _P, _P, _P, _P, _P, sz, _P]),
        "toric3d_bp_meta_step": (i32, [i32, i64, _P, dbl, dbl, _P, _P, _P, sz, _P]),
        "toric3d_logical": (i32, [i32, i64, _P, _P, _P, _P]),
        "toric3d_gate_workspace_bytes": (ctypes.c_size_t, [i32, i64]),
        "toric3d_cnn_status": (i32, []),
        "toric3d_cnn_debug_wait_limit": (i32, [u64]),
        "toric3d_gate": (i32, [i32, i64, _P, ctypes.c_uint32, _P, _P, _P, ctypes.c_size_t, _P]),
        "toric3d_pack": (i32, [i64, i64, _P, _P, _P]),
        "toric3d_unpack": (i32, [i64, i64, _P, _P, _P]),
        "toric3d_run_workspace_bytes": (sz, [ctypes.POINTER(RunCfg)]),
        "toric3d_run_cycles": (i32, [ctypes.POINTER(RunCfg), _P, _P, sz, _P, _P, _P]),
        "toric3d_run_batch_workspace_bytes": (sz, [ctypes.POINTER(RunCfg), ctypes.POINTER(BatchItem), i32]),
        "toric3d_run_batch": (i32, [ctypes.POINTER(RunCfg), ctypes.POINTER(BatchItem), i32, _P, sz, _P]),
        "toric3d_set_blocks_per_sm": (None, [i32, i32]),
        "toric3d_get_blocks_per_sm": (i32, [i32]),
        "toric3d_autotune_batch": (i32, [ctypes.POINTER(RunCfg), ctypes.POINTER(BatchItem), i32, _P, sz,
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float), _P]),
        "toric3d_cnn_param_count": (i32, []),
        "toric3d_cnn_blob_bytes": (sz, []),
        "toric3d_cnn_prepare": (i32, [_P, _P, _P]),
        "toric3d_cnn_workspace_bytes": (sz, [i32, i64]),
        "toric3d_cnn_decode": (i32, [i32, i64, _P, _P, _P, _P, _P, _P, sz, _P]),
        "toric3d_cnn_train_workspace_bytes": (sz, [i32, i64]),
        "toric3d_cnn_train_step": (i32, [i32, i64, _P, _P, _P, _P, _P, _P, i32, ctypes.c_float, _P, _P, _P,
                                         _P, sz, _P]),
        "toric3d_profile_enable": (None, [i32]),
        "toric3d_profile_reset": (None, []),
        "toric3d_profile_read": (i32, [i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(h, name)
        fn.restype = res
        fn.argtypes = args


def _check(status: int):
    if status != 0:
        msg = lib().toric3d_last_error()
        raise T3DError(status, msg.decode() if msg else "")


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_cuda:
        raise ValueError("toric3d needs CUDA tensors (the library has no CPU path)")
    if not t.is_contiguous():
        raise ValueError("toric3d needs contiguous tensors")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def n_bits(L: int) -> int:
    return 3 * L ** 3


def words_for(n_samples: int) -> int:
    return (n_samples + 63) // 64


def table1_schedule(n_A: int, lambda_p: int) -> str:
    """F/P schedule of n_A rule applications in one code cycle where every
    lambda_p-th application (counted within the cycle) is p-flip (Table 1 and
    its footnote; Sec. 3.2 prints n_A = 5, lambda_p = 3 as F F P F F)."""
    if n_A < 1 or lambda_p < 1:
        raise ValueError("n_A and lambda_p must be positive")
    return "".join("P" if k % lambda_p == 0 else "F" for k in range(1, n_A + 1))


# ------------------------------------------------------------------ sizes
def toric3d_flip_workspace_bytes(L: int, words: int) -> int:
    return int(lib().toric3d_flip_workspace_bytes(L, words))


def toric3d_bp_message_bytes(L: int, n_samples: int) -> int:
    return int(lib().toric3d_bp_message_bytes(L, n_samples))


def toric3d_bp_workspace_bytes(L: int, chunk_samples: int) -> int:
    return int(lib().toric3d_bp_workspace_bytes(L, chunk_samples))


def toric3d_run_workspace_bytes(cfg: RunCfg) -> int:
    return int(lib().toric3d_run_workspace_bytes(ctypes.byref(cfg)))


# ------------------------------------------------------------------ calls
def toric3d_noise(L, e, p, seed, sample0, cycle, stream=None):
    _check(lib().toric3d_noise(L, e.shape[-1], _ptr(e), float(p), seed, sample0, cycle, _stream(stream)))


def toric3d_syndrome(L, e, s, q, seed, sample0, cycle, stream=None):
    _check(lib().toric3d_syndrome(L, e.shape[-1], _ptr(e), _ptr(s), float(q), seed, sample0, cycle,
                                  _stream(stream)))


def toric3d_flip(L, e, s, sweeps, work, stream=None):
    _check(lib().toric3d_flip(L, e.shape[-1], _ptr(e), _ptr(s), sweeps, _ptr(work),
                              work.numel() * work.element_size(), _stream(stream)))


def toric3d_flip_until_clear_workspace_bytes(L, words):
    return lib().toric3d_flip_until_clear_workspace_bytes(L, words)


def toric3d_flip_until_clear(L, e, s, max_sweeps, work, sweeps_done=None, stream=None):
    """Up to max_sweeps flip applications, the ones after the batch's syndrome cleared
    skipped on the device; sweeps_done: optional one-element int32 device tensor."""
    _check(lib().toric3d_flip_until_clear(L, e.shape[-1], _ptr(e), _ptr(s), max_sweeps,
                                          _ptr(sweeps_done) if sweeps_done is not None else None,
                                          _ptr(work), work.numel() * work.element_size(), _stream(stream)))


def toric3d_flip_noalloc(L, e, s, sweeps, stream=None):
    """toric3d_flip with the library's built-in 32 MiB scratch instead of a
    caller workspace (no device allocation anywhere in the call)."""
    _check(lib().toric3d_flip_noalloc(L, e.shape[-1], _ptr(e), _ptr(s), sweeps, _stream(stream)))


def toric3d_pflip(L, e, s, schedule, n_apply, sweep0, seed, sample0, cycle, work, stream=None):
    _check(lib().toric3d_pflip(L, e.shape[-1], _ptr(e), _ptr(s), schedule.encode(), n_apply, sweep0,
                               seed, sample0, cycle, _ptr(work), work.numel() * work.element_size(),
                               _stream(stream)))


def toric3d_bp_step(L, n_samples, s, p, q_meas, msg_in, msg_out, stream=None):
    _check(lib().toric3d_bp_step(L, n_samples, _ptr(s), float(p), float(q_meas), _ptr(msg_in),
                                 _ptr(msg_out), _stream(stream)))


def toric3d_bp_decide_workspace_bytes(L: int, n_samples: int) -> int:
    return int(lib().toric3d_bp_decide_workspace_bytes(L, n_samples))


def toric3d_bp_decide(L, n_samples, msg, p, e, s, work, llr_out=None, stream=None):
    _check(lib().toric3d_bp_decide(L, n_samples, _ptr(msg), float(p), _ptr(e), _ptr(s),
                                   _ptr(llr_out), _ptr(work), work.numel() * work.element_size(),
                                   _stream(stream)))


def toric3d_bp(L, n_samples, e, s, p, q_meas, iters, work, llr_out=None, stream=None):
    _check(lib().toric3d_bp(L, n_samples, _ptr(e), _ptr(s), float(p), float(q_meas), iters,
                            _ptr(work), work.numel() * work.element_size(), _ptr(llr_out),
                            _stream(stream)))


def toric3d_bp_meta_workspace_bytes(L: int, chunk_samples: int) -> int:
    return int(lib().toric3d_bp_meta_workspace_bytes(L, chunk_samples))


def toric3d_bp_meta_message_bytes(L: int, n_samples: int) -> int:
    return int(lib().toric3d_bp_meta_message_bytes(L, n_samples))


def toric3d_bp_meta_step(L, n_samples, s, p, q, msg_in, msg_out, work, stream=None):
    _check(lib().toric3d_bp_meta_step(L, n_samples, _ptr(s), float(p), float(q), _ptr(msg_in), _ptr(msg_out),
                                      _ptr(work), work.numel() * work.element_size(), _stream(stream)))


def toric3d_bp_meta(L, n_samples, e, s, p, q, iters, work, llr_out=None, stream=None):
    """BP with meta-checks (one per unit cube over its faces' measurement variables)."""
    _check(lib().toric3d_bp_meta(L, n_samples, _ptr(e), _ptr(s), float(p), float(q), iters,
                                 _ptr(work), work.numel() * work.element_size(), _ptr(llr_out),
                                 _stream(stream)))


def toric3d_logical(L, n_samples, e, mask=None, counts8=None, stream=None):
    _check(lib().toric3d_logical(L, n_samples, _ptr(e), _ptr(mask), _ptr(counts8), _stream(stream)))


def toric3d_pack(n_bits_, n_samples, bits, words, stream=None):
    _check(lib().toric3d_pack(n_bits_, n_samples, _ptr(bits), _ptr(words), _stream(stream)))


def toric3d_unpack(n_bits_, n_samples, words, bits, stream=None):
    _check(lib().toric3d_unpack(n_bits_, n_samples, _ptr(words), _ptr(bits), _stream(stream)))


def toric3d_gate_workspace_bytes(L, words) -> int:
    return int(lib().toric3d_gate_workspace_bytes(L, words))


def toric3d_gate(L, s, max_weight, gate, work, n_flagged=None, stream=None):
    _check(lib().toric3d_gate(L, s.shape[1], _ptr(s), max_weight, _ptr(gate), _ptr(n_flagged), _ptr(work),
                              work.numel() * work.element_size(), _stream(stream)))


def make_run_cfg(L, T, p, q, seed, n_samples, *, sample0=0, use_bp=False, bp_iters=0,
                 bp_meas_nodes=True, schedule="", n_apply=None, perfect_round=False,
                 perfect_max_sweeps=0, cycle0=0, use_graph=False, bp_chunk_samples=0, cnn_blob=None,
                 fallback_max_weight=-1, bp_meta_checks=False, fallback_sigmas=0.0) -> RunCfg:
    """bp_meta_checks: BP over the measurement variables joined by the cube meta-checks
    (bp_meas_nodes = 2 in the C struct; implies measurement variables).  fallback_sigmas:
    the learned decoder's fallback threshold also allows q 3L^3 + fallback_sigmas standard
    deviations of unsatisfied checks (the measurement errors any decoder leaves)."""
    c = RunCfg()
    c.L, c.T, c.p, c.q, c.seed = L, T, float(p), float(q), seed
    c.sample0, c.n_samples = sample0, n_samples
    c.use_bp, c.bp_iters = int(use_bp), bp_iters
    c.bp_meas_nodes = 2 if bp_meta_checks else int(bp_meas_nodes)
    c.n_apply = len(schedule) if n_apply is None else n_apply
    c.schedule = schedule.encode()
    c.perfect_round, c.perfect_max_sweeps = int(perfect_round), perfect_max_sweeps
    c.cycle0, c.use_graph, c.bp_chunk_samples = cycle0, int(use_graph), bp_chunk_samples
    c.cnn_blob, c.fallback_max_weight = _ptr(cnn_blob), fallback_max_weight
    c.fallback_sigmas = float(fallback_sigmas)
    return c


def toric3d_run_cycles(cfg: RunCfg, e, work, mask=None, counts8=None, stream=None):
    _check(lib().toric3d_run_cycles(ctypes.byref(cfg), _ptr(e), _ptr(work),
                                    work.numel() * work.element_size(), _ptr(mask), _ptr(counts8),
                                    _stream(stream)))


# ------------------------------------------------------------------ batches of lattices
def make_batch(items):
    """items: iterable of dicts with L, n_samples, e (device int64 tensor) and
    optional sample0, mask, counts8, s_prev, fallback_words -> ctypes array of BatchItem."""
    items = list(items)
    arr = (BatchItem * len(items))()
    for a, it in zip(arr, items):
        a.L, a.n_samples = it["L"], it["n_samples"]
        a.sample0 = it.get("sample0", 0)
        a.e = _ptr(it["e"])
        a.mask = _ptr(it.get("mask"))
        a.counts8 = _ptr(it.get("counts8"))
        a.s_prev = _ptr(it.get("s_prev"))
        a.fallback_words = _ptr(it.get("fallback_words"))
    return arr


def _as_batch(batch):
    if isinstance(batch, ctypes.Array):
        return batch
    items = list(batch)
    return (BatchItem * len(items))(*items)


def toric3d_run_batch_workspace_bytes(cfg: RunCfg, batch) -> int:
    batch = _as_batch(batch)
    return int(lib().toric3d_run_batch_workspace_bytes(ctypes.byref(cfg), batch, len(batch)))


def toric3d_run_batch(cfg: RunCfg, batch, work, stream=None):
    batch = _as_batch(batch)
    _check(lib().toric3d_run_batch(ctypes.byref(cfg), batch, len(batch), _ptr(work),
                                   work.numel() * work.element_size(), _stream(stream)))


def toric3d_set_blocks_per_sm(kind, blocks_per_sm: int):
    k = KERNEL_KINDS[kind] if isinstance(kind, str) else int(kind)
    lib().toric3d_set_blocks_per_sm(k, int(blocks_per_sm))


def toric3d_get_blocks_per_sm(kind) -> int:
    k = KERNEL_KINDS[kind] if isinstance(kind, str) else int(kind)
    return int(lib().toric3d_get_blocks_per_sm(k))


def toric3d_autotune_batch(cfg: RunCfg, batch, work, stream=None):
    """Tune the BP iteration's blocks-per-SM cap; returns (cap, ms per iteration)."""
    batch = _as_batch(batch)
    cap = ctypes.c_int()
    ms = ctypes.c_float()
    _check(lib().toric3d_autotune_batch(ctypes.byref(cfg), batch, len(batch), _ptr(work),
                                        work.numel() * work.element_size(), ctypes.byref(cap),
                                        ctypes.byref(ms), _stream(stream)))
    return cap.value, ms.value


# ------------------------------------------------------------------ kernel timing
def toric3d_profile_enable(on: bool = True):
    lib().toric3d_profile_enable(int(on))


def toric3d_profile_reset():
    lib().toric3d_profile_reset()


def toric3d_profile_read(kind) -> tuple[float, int]:
    """(summed device milliseconds, launches) recorded for one kernel kind."""
    k = KERNEL_KINDS[kind] if isinstance(kind, str) else int(kind)
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(lib().toric3d_profile_read(k, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


# ------------------------------------------------------------------ replicas
def replica_sample0(rank: int, samples_per_rank: int) -> int:
    """First global sample of a rank's disjoint range.  Ranges start on
    64-sample word boundaries, so every replica draws exactly the random
    numbers one large batch would (the generator is keyed by global sample)."""
    return rank * ((samples_per_rank + 63) // 64 * 64)


# ------------------------------------------------------------------ learned pre-decoder
def toric3d_cnn_param_count() -> int:
    return int(lib().toric3d_cnn_param_count())


def toric3d_cnn_blob_bytes() -> int:
    return int(lib().toric3d_cnn_blob_bytes())


def toric3d_cnn_prepare(params, blob, stream=None):
    _check(lib().toric3d_cnn_prepare(_ptr(params), _ptr(blob), _stream(stream)))


def toric3d_cnn_workspace_bytes(L: int, n_samples: int) -> int:
    return int(lib().toric3d_cnn_workspace_bytes(L, n_samples))


def toric3d_cnn_decode(L, n_samples, s_prev, s, e, blob, work, logits_out=None, stream=None):
    _check(lib().toric3d_cnn_decode(L, n_samples, _ptr(s_prev), _ptr(s), _ptr(e), _ptr(blob),
                                    _ptr(logits_out), _ptr(work), work.numel() * work.element_size(),
                                    _stream(stream)))


def toric3d_cnn_status():
    """Raise T3DError if a tensor-core pre-decoder kernel gave up a bounded wait."""
    _check(lib().toric3d_cnn_status())


def toric3d_cnn_debug_wait_limit(ns: int):
    """Test hook: shorten (ns > 0) or restore (0) the bound of the pre-decoder's
    waits that may give up."""
    _check(lib().toric3d_cnn_debug_wait_limit(int(ns)))


def toric3d_cnn_train_workspace_bytes(L: int, n_samples: int) -> int:
    return int(lib().toric3d_cnn_train_workspace_bytes(L, n_samples))


def toric3d_cnn_train_step(L, n_samples, s_prev, s, e_label, params, adam_m, adam_v, step, lr, blob,
                           work, loss_out, grads_out=None, stream=None):
    _check(lib().toric3d_cnn_train_step(L, n_samples, _ptr(s_prev), _ptr(s), _ptr(e_label), _ptr(params),
                                        _ptr(adam_m), _ptr(adam_v), int(step), float(lr), _ptr(blob),
                                        _ptr(grads_out), _ptr(loss_out), _ptr(work),
                                        work.numel() * work.element_size(), _stream(stream)))


# ------------------------------------------------------------------ generic Tanner graphs
class TannerGraph:
    """A code prepared for the toric3d_tanner_* calls: the C descriptor plus the
    device blob it points into (kept alive with this object)."""

    def __init__(self, desc: Tanner, blob):
        self.desc = desc
        self.blob = blob

    @property
    def n_vars(self):
        return int(self.desc.n_vars)

    @property
    def n_checks(self):
        return int(self.desc.n_checks)

    @property
    def n_edges(self):
        return int(self.desc.n_edges)

    def ref(self):
        return ctypes.byref(self.desc)


def tanner_prepare(cptr, cvar, n_vars: int, device="cuda:0") -> TannerGraph:
    """Checks in CSR form (host int32 arrays) -> a prepared graph on `device`."""
    import numpy as np
    cptr = np.ascontiguousarray(cptr, dtype=np.int32)
    cvar = np.ascontiguousarray(cvar, dtype=np.int32)
    m = len(cptr) - 1
    nbytes = int(lib().toric3d_tanner_bytes(n_vars, m, int(cptr[-1])))
    if nbytes == 0:
        raise T3DError(1, "invalid graph sizes")
    blob = torch.empty(nbytes, dtype=torch.uint8, device=device)
    desc = Tanner()
    _check(lib().toric3d_tanner_prepare(n_vars, m, cptr.ctypes.data_as(ctypes.c_void_p),
                                        cvar.ctypes.data_as(ctypes.c_void_p), _ptr(blob), nbytes,
                                        ctypes.byref(desc)))
    return TannerGraph(desc, blob)


def toric3d_tanner_noise(g: TannerGraph, n_samples, e, p, seed, sample0, cycle, stream=None):
    _check(lib().toric3d_tanner_noise(g.ref(), n_samples, _ptr(e), float(p), seed, sample0, cycle, _stream(stream)))


def toric3d_tanner_syndrome(g: TannerGraph, n_samples, e, s, q, seed, sample0, cycle, stream=None):
    _check(lib().toric3d_tanner_syndrome(g.ref(), n_samples, _ptr(e), _ptr(s), float(q), seed, sample0, cycle,
                                         _stream(stream)))


def toric3d_tanner_flip_workspace_bytes(g: TannerGraph, n_samples) -> int:
    return int(lib().toric3d_tanner_flip_workspace_bytes(g.ref(), n_samples))


def toric3d_tanner_pflip(g: TannerGraph, n_samples, e, s, schedule, n_apply, sweep0, seed, sample0, cycle, work,
                         stream=None):
    _check(lib().toric3d_tanner_pflip(g.ref(), n_samples, _ptr(e), _ptr(s), schedule.encode(), n_apply, sweep0, seed,
                                      sample0, cycle, _ptr(work), work.numel() * work.element_size(),
                                      _stream(stream)))


def toric3d_tanner_bp_workspace_bytes(g: TannerGraph, chunk_samples) -> int:
    return int(lib().toric3d_tanner_bp_workspace_bytes(g.ref(), chunk_samples))


def toric3d_tanner_bp(g: TannerGraph, n_samples, e, s, prior, iters, work, llr_out=None, stream=None):
    _check(lib().toric3d_tanner_bp(g.ref(), n_samples, _ptr(e), _ptr(s), _ptr(prior), iters, _ptr(work),
                                   work.numel() * work.element_size(), _ptr(llr_out), _stream(stream)))


def toric3d_tanner_bp_message_bytes(g: TannerGraph, n_samples) -> int:
    return int(lib().toric3d_tanner_bp_message_bytes(g.ref(), n_samples))


def toric3d_tanner_bp_step(g: TannerGraph, n_samples, s, prior, msg_in, msg_out, work, stream=None):
    _check(lib().toric3d_tanner_bp_step(g.ref(), n_samples, _ptr(s), _ptr(prior), _ptr(msg_in), _ptr(msg_out),
                                        _ptr(work), work.numel() * work.element_size(), _stream(stream)))
