"""CPU oracle for the 3D toric code decoders of arXiv:2212.06985.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may load this package; the CUDA library never
does, and this package imports nothing from it.  The arithmetic lives in plain
C (``t3d_oracle.c``, one sample at a time, uint8 bits, binary64 belief
propagation); this module only compiles it with gcc and marshals numpy arrays
through ctypes.

Parity pins (tests/test_oracle_*.py): Philox4x32-10 against its published
known-answer vectors and Triton's independent implementation; the syndrome map against the code parameters
[[3L^3, 3, L]] of Sec. 2; flip and p-flip against the worked examples of
Sec. 3 (Fig. 3(a) half cube, Fig. 3(b) planar error, Fig. 5 oscillating pair,
the opposite-face pair); BP against exact marginals on acyclic graphs and the
closed form of its first iteration; the logical readout against membranes and
stabilisers.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "t3d_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libt3d_oracle.so")
_lock = threading.Lock()
_lib = None

STREAM_QUBIT, STREAM_MEAS, STREAM_COIN = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Cfg(ctypes.Structure):
    """Run configuration; mirrors ``t3o_cfg`` in t3d_oracle.c."""

    _fields_ = [
        ("L", ctypes.c_int32),
        ("T", ctypes.c_int32),
        ("p", ctypes.c_double),
        ("q", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("use_bp", ctypes.c_int32),
        ("bp_iters", ctypes.c_int32),
        ("bp_meas_nodes", ctypes.c_int32),
        ("n_apply", ctypes.c_int32),
        ("schedule", ctypes.c_char * 64),
        ("perfect_round", ctypes.c_int32),
        ("perfect_max_sweeps", ctypes.c_int32),
        ("cycle0", ctypes.c_uint32),
        ("bp_meta", ctypes.c_int32),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


_P = ctypes.c_void_p


def _declare(L):
    u64, i64, i32, u32, dbl = (ctypes.c_uint64, ctypes.c_int64, ctypes.c_int,
                               ctypes.c_uint32, ctypes.c_double)
    sig = {
        "t3o_philox4x32": (None, [_P, _P, _P]),
        "t3o_prob_to_threshold": (u64, [dbl]),
        "t3o_bernoulli_count": (i64, [dbl, u64, i32, u64, u64, u64, u64, i64]),
        "t3o_bernoulli": (i32, [dbl, u64, i32, u64, u64, u64, u64]),
        "t3o_coin": (i32, [u64, u64, i32, u64, u64, u64]),
        "t3o_face_edges": (None, [i32, i64, _P]),
        "t3o_incidence": (None, [i32, _P, _P]),
        "t3o_syndrome": (None, [i32, _P, _P]),
        "t3o_noise": (None, [i32, _P, dbl, u64, u64, u32]),
        "t3o_measure": (None, [i32, _P, _P, dbl, u64, u64, u32]),
        "t3o_flip_once": (None, [i32, _P, _P]),
        "t3o_pflip_once": (None, [i32, _P, _P, u64, u64, u32, u32]),
        "t3o_flip_sequential": (i32, [i32, _P, _P, i32]),
        "t3o_bp": (None, [i32, i32, _P, _P, _P, dbl, dbl, i32, _P, _P, _P]),
        "t3o_toric_tanner": (None, [i32, _P, _P]),
        "t3o_bp_priors": (None, [i32, i32, _P, _P, _P, _P, i32, _P]),
        "t3o_bp_priors_from": (None, [i32, i32, _P, _P, _P, _P, i32, _P, _P, _P]),
        "t3o_cube_faces": (None, [i32, i64, _P]),
        "t3o_meta_syndrome": (None, [i32, _P, _P]),
        "t3o_meta_tanner": (None, [i32, _P, _P]),
        "t3o_bp_meta_decode_batch": (None, [i32, i64, _P, _P, dbl, dbl, i32, _P]),
        "t3o_bp_decode": (None, [i32, _P, _P, dbl, dbl, i32, i32, _P]),
        "t3o_logical": (i32, [i32, _P, _P]),
        "t3o_run_sample": (i32, [_P, u64, _P]),
        "t3o_run_batch": (None, [_P, u64, i64, _P, _P]),
        "t3o_noise_batch": (None, [i32, i64, _P, dbl, u64, u64, u32]),
        "t3o_measure_batch": (None, [i32, i64, _P, _P, dbl, u64, u64, u32]),
        "t3o_syndrome_batch": (None, [i32, i64, _P, _P]),
        "t3o_flip_batch": (None, [i32, i64, _P, _P, i32, u64, u64, u32, u32]),
        "t3o_logical_batch": (None, [i32, i64, _P, _P]),
        "t3o_bp_batch": (None, [i32, i64, _P, dbl, dbl, i32, i32, _P, _P, _P]),
        "t3o_bp_decode_batch": (None, [i32, i64, _P, _P, dbl, dbl, i32, i32, _P]),
        "t3o_abi_version": (i32, []),
        "t3o_tanner_syndrome_batch": (None, [i64, i64, _P, _P, i64, _P, _P]),
        "t3o_tanner_noise_batch": (None, [i64, i64, _P, dbl, u64, u64, u32]),
        "t3o_tanner_measure_batch": (None, [i64, i64, _P, _P, i64, _P, _P, dbl, u64, u64, u32]),
        "t3o_tanner_coin": (i32, [u64, i64, u32, u32, u64]),
        "t3o_tanner_rule_batch": (None, [i64, i64, _P, _P, i64, _P, _P, i32, u64, u64, u32, u32]),
        "t3o_tanner_bp_batch": (None, [i64, i64, _P, _P, i64, _P, _P, _P, i32, _P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a


def n_bits(L: int) -> int:
    return 3 * L * L * L


# ---------------------------------------------------------------- Philox / RNG
def philox4x32(counter, key):
    """One Philox4x32-10 block: counter (4 x uint32), key (2 x uint32) -> 4 x uint32."""
    c = np.ascontiguousarray(np.asarray(counter, dtype=np.uint64).astype(np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64).astype(np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().t3o_philox4x32(_ptr(c), _ptr(k), _ptr(out))
    return out


def prob_to_threshold(p: float) -> int:
    return int(lib().t3o_prob_to_threshold(float(p)))


def bernoulli(p, seed, stream, site, cycle, sweep, sample) -> int:
    return int(lib().t3o_bernoulli(float(p), seed, stream, site, cycle, sweep, sample))


def bernoulli_count(p, seed, stream, site, cycle, sweep, sample0, n) -> int:
    """Events among samples [sample0, sample0 + n) of one stream position."""
    return int(lib().t3o_bernoulli_count(float(p), seed, stream, site, cycle, sweep, sample0, n))


def coin(seed, L, edge, cycle, sweep, sample) -> int:
    """p-flip coin of edge index `edge` = d L^3 + site."""
    L3 = L ** 3
    return int(lib().t3o_coin(seed, edge % L3, edge // L3, cycle, sweep, sample))


# ---------------------------------------------------------------- lattice
def face_edges(L: int, f: int) -> np.ndarray:
    out = np.zeros(4, dtype=np.int64)
    lib().t3o_face_edges(L, f, _ptr(out))
    return out


def incidence(L: int):
    n = n_bits(L)
    fe = np.zeros((n, 4), dtype=np.int32)
    ef = np.zeros((n, 4), dtype=np.int32)
    lib().t3o_incidence(L, _ptr(fe), _ptr(ef))
    return fe, ef


def toric_tanner(L: int):
    n = n_bits(L)
    cptr = np.zeros(n + 1, dtype=np.int32)
    cvar = np.zeros(4 * n, dtype=np.int32)
    lib().t3o_toric_tanner(L, _ptr(cptr), _ptr(cvar))
    return cptr, cvar


def bp_priors(cptr, cvar, syn, prior, iters):
    """BP with one prior per variable on a CSR factor graph; returns the posteriors."""
    cptr = np.ascontiguousarray(cptr, dtype=np.int32)
    cvar = np.ascontiguousarray(cvar, dtype=np.int32)
    prior = np.ascontiguousarray(prior, dtype=np.float64)
    syn = _u8(syn)
    llr = np.zeros(len(prior), dtype=np.float64)
    lib().t3o_bp_priors(len(prior), len(cptr) - 1, _ptr(cptr), _ptr(cvar), _ptr(syn), _ptr(prior), iters,
                        _ptr(llr))
    return llr


def bp_priors_from(cptr, cvar, syn, prior, iters, cv_in=None):
    """bp_priors started from the check->variable messages cv_in (one per Tanner edge,
    CSR order; None = zero); returns (posteriors, the last check->variable messages)."""
    cptr = np.ascontiguousarray(cptr, dtype=np.int32)
    cvar = np.ascontiguousarray(cvar, dtype=np.int32)
    prior = np.ascontiguousarray(prior, dtype=np.float64)
    syn = _u8(syn)
    cv = None if cv_in is None else np.ascontiguousarray(cv_in, dtype=np.float64)
    assert cv is None or cv.shape == (cptr[-1],)
    cv_out = np.zeros(int(cptr[-1]), dtype=np.float64)
    llr = np.zeros(len(prior), dtype=np.float64)
    lib().t3o_bp_priors_from(len(prior), len(cptr) - 1, _ptr(cptr), _ptr(cvar), _ptr(syn), _ptr(prior), iters,
                             _ptr(cv), _ptr(cv_out), _ptr(llr))
    return llr, cv_out


def cube_faces(L: int, site: int) -> np.ndarray:
    out = np.zeros(6, dtype=np.int64)
    lib().t3o_cube_faces(L, site, _ptr(out))
    return out


def meta_syndrome(L: int, s) -> np.ndarray:
    s = _u8(s)
    m = np.zeros(L ** 3, dtype=np.uint8)
    lib().t3o_meta_syndrome(L, _ptr(s), _ptr(m))
    return m


def meta_tanner(L: int):
    n = n_bits(L)
    cptr = np.zeros(n + L ** 3 + 1, dtype=np.int32)
    cvar = np.zeros(5 * n + 6 * L ** 3, dtype=np.int32)
    lib().t3o_meta_tanner(L, _ptr(cptr), _ptr(cvar))
    return cptr, cvar


def bp_meta_decode_batch(L, e, s, p, q, iters):
    """BP with meta-checks on each sample; returns (e, s, llr [S][2 * 3L^3])."""
    e = _u8(e).copy()
    s = _u8(s).copy()
    llr = np.zeros((e.shape[0], 2 * e.shape[1]), dtype=np.float64)
    lib().t3o_bp_meta_decode_batch(L, e.shape[0], _ptr(e), _ptr(s), float(p), float(q), iters, _ptr(llr))
    return e, s, llr


# ---------------------------------------------------------------- single sample
def syndrome(L: int, e) -> np.ndarray:
    e = _u8(e)
    s = np.zeros(n_bits(L), dtype=np.uint8)
    lib().t3o_syndrome(L, _ptr(e), _ptr(s))
    return s


def noise(L, e, p, seed, sample, cycle):
    e = _u8(e).copy()
    lib().t3o_noise(L, _ptr(e), float(p), seed, sample, cycle)
    return e


def measure(L, e, q, seed, sample, cycle):
    e = _u8(e)
    s = np.zeros(n_bits(L), dtype=np.uint8)
    lib().t3o_measure(L, _ptr(e), _ptr(s), float(q), seed, sample, cycle)
    return s


def flip_once(L, e, s):
    e = _u8(e).copy()
    s = _u8(s).copy()
    lib().t3o_flip_once(L, _ptr(e), _ptr(s))
    return e, s


def pflip_once(L, e, s, seed, sample, cycle, sweep):
    e = _u8(e).copy()
    s = _u8(s).copy()
    lib().t3o_pflip_once(L, _ptr(e), _ptr(s), seed, sample, cycle, sweep)
    return e, s


def flip_sequential(L, e, s, max_flips=1 << 20):
    e = _u8(e).copy()
    s = _u8(s).copy()
    k = lib().t3o_flip_sequential(L, _ptr(e), _ptr(s), max_flips)
    return e, s, int(k)


def bp_general(cptr, cvar, syn, l0, lq, iters, m_in=None):
    """Generic product-sum BP (Eqs. 1-4) on a CSR Tanner graph."""
    cptr = np.ascontiguousarray(cptr, dtype=np.int32)
    cvar = np.ascontiguousarray(cvar, dtype=np.int32)
    syn = _u8(syn)
    nc = len(cptr) - 1
    nv = int(cvar.max()) + 1 if len(cvar) else 0
    ne = int(cptr[-1])
    if m_in is not None:
        m_in = np.ascontiguousarray(m_in, dtype=np.float64)
    m_out = np.zeros(ne, dtype=np.float64)
    llr = np.zeros(nv, dtype=np.float64)
    lib().t3o_bp(nv, nc, _ptr(cptr), _ptr(cvar), _ptr(syn), float(l0), float(lq), iters,
                 _ptr(m_in), _ptr(m_out), _ptr(llr))
    return m_out, llr


def bp_decode(L, e, s, p, q, meas_nodes, iters):
    e = _u8(e).copy()
    s = _u8(s).copy()
    llr = np.zeros(n_bits(L), dtype=np.float64)
    lib().t3o_bp_decode(L, _ptr(e), _ptr(s), float(p), float(q), int(meas_nodes), iters,
                        _ptr(llr))
    return e, s, llr


def logical(L, e):
    e = _u8(e)
    counts = np.zeros(3, dtype=np.int32)
    m = lib().t3o_logical(L, _ptr(e), _ptr(counts))
    return int(m), counts


def make_cfg(L, T, p, q, seed, *, use_bp=False, bp_iters=0, bp_meas_nodes=True,
             schedule="", n_apply=None, perfect_round=False, perfect_max_sweeps=0,
             cycle0=0, bp_meta=False) -> Cfg:
    c = Cfg()
    c.L, c.T, c.p, c.q, c.seed = L, T, float(p), float(q), seed
    c.use_bp, c.bp_iters, c.bp_meas_nodes = int(use_bp), bp_iters, int(bp_meas_nodes)
    c.n_apply = len(schedule) if n_apply is None else n_apply
    c.schedule = schedule.encode()
    c.perfect_round, c.perfect_max_sweeps = int(perfect_round), perfect_max_sweeps
    c.cycle0 = cycle0
    c.bp_meta = int(bp_meta)
    return c


def run_sample(cfg: Cfg, sample: int, e=None):
    n = n_bits(cfg.L)
    e = np.zeros(n, dtype=np.uint8) if e is None else _u8(e).copy()
    m = lib().t3o_run_sample(ctypes.byref(cfg), sample, _ptr(e))
    return int(m), e


# ---------------------------------------------------------------- batches [S][n]
def run_batch(cfg: Cfg, sample0: int, n_samples: int, e=None):
    n = n_bits(cfg.L)
    e = np.zeros((n_samples, n), dtype=np.uint8) if e is None else _u8(e).copy()
    mask = np.zeros(n_samples, dtype=np.uint8)
    lib().t3o_run_batch(ctypes.byref(cfg), sample0, n_samples, _ptr(e), _ptr(mask))
    return mask, e


def noise_batch(L, e, p, seed, sample0, cycle):
    e = _u8(e).copy()
    lib().t3o_noise_batch(L, e.shape[0], _ptr(e), float(p), seed, sample0, cycle)
    return e


def measure_batch(L, e, q, seed, sample0, cycle):
    e = _u8(e)
    s = np.zeros_like(e)
    lib().t3o_measure_batch(L, e.shape[0], _ptr(e), _ptr(s), float(q), seed, sample0, cycle)
    return s


def syndrome_batch(L, e):
    e = _u8(e)
    s = np.zeros_like(e)
    lib().t3o_syndrome_batch(L, e.shape[0], _ptr(e), _ptr(s))
    return s


def flip_batch(L, e, s, probabilistic=False, seed=0, sample0=0, cycle=0, sweep=0):
    e = _u8(e).copy()
    s = _u8(s).copy()
    lib().t3o_flip_batch(L, e.shape[0], _ptr(e), _ptr(s), int(probabilistic), seed, sample0,
                         cycle, sweep)
    return e, s


def logical_batch(L, e):
    e = _u8(e)
    mask = np.zeros(e.shape[0], dtype=np.uint8)
    lib().t3o_logical_batch(L, e.shape[0], _ptr(e), _ptr(mask))
    return mask


def bp_batch(L, s, p, q, meas_nodes, iters, m_in=None):
    """BP messages [S][4*3L^3] (Tanner-edge order of toric_tanner) and posteriors."""
    s = _u8(s)
    S, n = s.shape
    if m_in is not None:
        m_in = np.ascontiguousarray(m_in, dtype=np.float64)
    m_out = np.zeros((S, 4 * n), dtype=np.float64)
    llr = np.zeros((S, n), dtype=np.float64)
    lib().t3o_bp_batch(L, S, _ptr(s), float(p), float(q), int(meas_nodes), iters, _ptr(m_in),
                       _ptr(m_out), _ptr(llr))
    return m_out, llr


def bp_decode_batch(L, e, s, p, q, meas_nodes, iters):
    e = _u8(e).copy()
    s = _u8(s).copy()
    llr = np.zeros(e.shape, dtype=np.float64)
    lib().t3o_bp_decode_batch(L, e.shape[0], _ptr(e), _ptr(s), float(p), float(q),
                              int(meas_nodes), iters, _ptr(llr))
    return e, s, llr


# ---------------------------------------------------------------- generic Tanner graphs
def _csr(cptr, cvar):
    return np.ascontiguousarray(cptr, dtype=np.int32), np.ascontiguousarray(cvar, dtype=np.int32)


def tanner_syndrome_batch(cptr, cvar, e):
    """s = H e per sample; e [S][n] -> s [S][m] (checks in CSR form)."""
    cptr, cvar = _csr(cptr, cvar)
    e = _u8(e)
    s = np.zeros((e.shape[0], len(cptr) - 1), dtype=np.uint8)
    lib().t3o_tanner_syndrome_batch(e.shape[1], len(cptr) - 1, _ptr(cptr), _ptr(cvar), e.shape[0], _ptr(e), _ptr(s))
    return s


def tanner_noise_batch(e, p, seed, sample0, cycle):
    e = _u8(e).copy()
    lib().t3o_tanner_noise_batch(e.shape[1], e.shape[0], _ptr(e), float(p), seed, sample0, cycle)
    return e


def tanner_measure_batch(cptr, cvar, e, q, seed, sample0, cycle):
    cptr, cvar = _csr(cptr, cvar)
    e = _u8(e)
    s = np.zeros((e.shape[0], len(cptr) - 1), dtype=np.uint8)
    lib().t3o_tanner_measure_batch(e.shape[1], len(cptr) - 1, _ptr(cptr), _ptr(cvar), e.shape[0], _ptr(e), _ptr(s),
                                   float(q), seed, sample0, cycle)
    return s


def tanner_coin(seed, v, cycle, sweep, sample):
    return int(lib().t3o_tanner_coin(seed, v, cycle, sweep, sample))


def tanner_rule_batch(cptr, cvar, e, s, probabilistic=False, seed=0, sample0=0, cycle=0, sweep=0):
    """One parallel flip (or p-flip) application per sample; returns (e, s)."""
    cptr, cvar = _csr(cptr, cvar)
    e = _u8(e).copy()
    s = _u8(s).copy()
    lib().t3o_tanner_rule_batch(e.shape[1], len(cptr) - 1, _ptr(cptr), _ptr(cvar), e.shape[0], _ptr(e), _ptr(s),
                                int(probabilistic), seed, sample0, cycle, sweep)
    return e, s


def tanner_bp_batch(cptr, cvar, e, s, prior, iters):
    """BP with per-variable priors and the hard decision; returns (e, s, llr [S][n])."""
    cptr, cvar = _csr(cptr, cvar)
    e = _u8(e).copy()
    s = _u8(s).copy()
    prior = np.ascontiguousarray(prior, dtype=np.float64)
    llr = np.zeros(e.shape, dtype=np.float64)
    lib().t3o_tanner_bp_batch(e.shape[1], len(cptr) - 1, _ptr(cptr), _ptr(cvar), e.shape[0], _ptr(e), _ptr(s),
                              _ptr(prior), iters, _ptr(llr))
    return e, s, llr
