"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every entry point include/toric3d.h declares, sizes its
workspaces, and rejects invalid arguments with T3D_EINVAL before touching the
device."""
import ctypes
import os
import re

import pytest

import paper_2212_06985_gb300 as t3d

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EINVAL = 1


def _declared():
    text = open(os.path.join(ROOT, "include", "toric3d.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(toric3d_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    lib = t3d.lib()
    declared = _declared()
    assert len(declared) >= 17
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(t3d.EXPORTED_SYMBOLS) == declared


def test_abi_version():
    assert t3d.lib().toric3d_abi_version() == 1


def test_workspace_sizes():
    L, W = 4, 157
    assert t3d.toric3d_flip_workspace_bytes(L, W) == 3 * 64 * W * 8
    assert t3d.toric3d_flip_workspace_bytes(1, W) == 0
    assert t3d.toric3d_bp_message_bytes(4, 100) == 2 * 3 * 64 * 4 * 64 * 4
    assert t3d.toric3d_bp_workspace_bytes(4, 100) == 2 * (2 * 3 * 64 * 4 * 64 * 4 + 64 * 32)
    cfg = t3d.make_run_cfg(4, 4, 0.01, 0.01, 0, 10_000, schedule="F", n_apply=32)
    assert t3d.toric3d_run_workspace_bytes(cfg) == 2 * ((3 * 64 * 157 * 8 + 255) // 256 * 256)
    bad = t3d.make_run_cfg(4, 4, 0.01, 0.01, 0, 10_000, schedule="FX", n_apply=2)
    assert t3d.toric3d_run_workspace_bytes(bad) == 0


def _err():
    return t3d.lib().toric3d_last_error().decode()


FAKE = ctypes.c_void_p(0x10000)    # aligned, never dereferenced: calls fail validation first
MIS = ctypes.c_void_p(0x10004)


@pytest.mark.parametrize("call,needle", [
    (lambda l: l.toric3d_noise(1, 4, FAKE, 0.1, 0, 0, 1, None), "L=1"),
    (lambda l: l.toric3d_noise(4, 0, FAKE, 0.1, 0, 0, 1, None), "words"),
    (lambda l: l.toric3d_noise(4, 4, None, 0.1, 0, 0, 1, None), "NULL"),
    (lambda l: l.toric3d_noise(4, 4, MIS, 0.1, 0, 0, 1, None), "aligned"),
    (lambda l: l.toric3d_noise(4, 4, FAKE, 1.5, 0, 0, 1, None), "p="),
    (lambda l: l.toric3d_noise(4, 4, FAKE, 0.1, 0, 3, 1, None), "sample0"),
    (lambda l: l.toric3d_syndrome(4, 4, FAKE, FAKE, 0.1, 0, 0, 1, None), "overlap"),
    (lambda l: l.toric3d_flip(4, 4, FAKE, FAKE, 2, FAKE, 16, None), "workspace"),
    (lambda l: l.toric3d_pflip(4, 4, FAKE, FAKE, b"FQ", 2, 0, 0, 0, 1, FAKE, 1 << 20, None), "schedule"),
    (lambda l: l.toric3d_bp_step(4, 10, FAKE, 0.0, 0.1, None, FAKE, None), "0 < p < 1"),
    (lambda l: l.toric3d_bp_step(4, 10, FAKE, 0.1, 0.6, None, FAKE, None), "q_meas"),
    (lambda l: l.toric3d_bp(4, 10, FAKE, FAKE, 0.1, 0.1, 3, FAKE, 64, None, None), "workspace"),
    (lambda l: l.toric3d_logical(4, 0, FAKE, None, None, None), "n_samples"),
    (lambda l: l.toric3d_pack(0, 4, FAKE, FAKE, None), "empty"),
])
def test_invalid_arguments_are_rejected(call, needle):
    assert call(t3d.lib()) == EINVAL
    assert needle in _err()


def test_run_cycles_rejects_bad_configs():
    lib = t3d.lib()
    for kw in (dict(L=1), dict(p=-0.1), dict(sample0=10), dict(schedule="FFX", n_apply=3),
               dict(schedule="", n_apply=2), dict(use_bp=True, bp_iters=4, p=0.0)):
        base = dict(L=4, T=2, p=0.01, q=0.01, seed=0, n_samples=100, schedule="F", n_apply=1)
        base.update(kw)
        cfg = t3d.make_run_cfg(**base)
        assert lib.toric3d_run_cycles(ctypes.byref(cfg), FAKE, FAKE, 1 << 30, None, None, None) == EINVAL
    cfg = t3d.make_run_cfg(4, 2, 0.01, 0.01, 0, 100, schedule="F", n_apply=1)
    assert lib.toric3d_run_cycles(ctypes.byref(cfg), FAKE, FAKE, 64, None, None, None) == EINVAL
    assert "workspace" in _err()


def test_table1_schedule_matches_paper():
    import json
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "schedules.json")))
    for row in g["table1"]:
        assert t3d.table1_schedule(row["n_A"], row["lambda_p"]) == row["schedule"]


def test_batch_validation():
    lib = t3d.lib()
    cfg = t3d.make_run_cfg(4, 2, 0.01, 0.01, 0, 1, schedule="F", n_apply=1)
    items = (t3d.BatchItem * 9)()
    for it in items:
        it.L, it.n_samples, it.e = 4, 64, 0x10000
    assert lib.toric3d_run_batch(ctypes.byref(cfg), items, 9, FAKE, 1 << 30, None) == EINVAL
    assert lib.toric3d_run_batch(ctypes.byref(cfg), items, 0, FAKE, 1 << 30, None) == EINVAL
    items[1].L = 1
    assert lib.toric3d_run_batch(ctypes.byref(cfg), items, 2, FAKE, 1 << 30, None) == EINVAL
    assert "L=1" in _err()
    items[1].L = 5
    items[1].sample0 = 3
    assert lib.toric3d_run_batch(ctypes.byref(cfg), items, 2, FAKE, 1 << 30, None) == EINVAL
    items[1].sample0 = 0
    assert t3d.toric3d_run_batch_workspace_bytes(cfg, items[:2]) == sum(
        2 * ((3 * L ** 3 * 8 + 255) // 256 * 256) for L in (4, 5))
    bp = t3d.make_run_cfg(4, 2, 0.04, 0.04, 0, 1, use_bp=True, bp_iters=4, schedule="F", n_apply=1)
    items[0].L = 130
    assert lib.toric3d_run_batch(ctypes.byref(bp), items, 1, FAKE, 1 << 40, None) == EINVAL
    assert "L <= 128" in _err()


def test_tuning_table_roundtrip():
    t3d.toric3d_set_blocks_per_sm("bp_step", 3)
    assert t3d.toric3d_get_blocks_per_sm("bp_step") == 3
    t3d.toric3d_set_blocks_per_sm("bp_step", 0)
    assert t3d.toric3d_get_blocks_per_sm("bp_step") == 0


def test_learned_run_validation():
    lib = t3d.lib()
    items = (t3d.BatchItem * 1)()
    items[0].L, items[0].n_samples, items[0].e, items[0].s_prev = 4, 64, 0x10000, 0x20000
    blob = ctypes.c_void_p(0x30000)
    cfg = t3d.make_run_cfg(4, 2, 0.04, 0.04, 0, 64, use_bp=True, bp_iters=4, schedule="F", n_apply=1)
    cfg.cnn_blob = blob
    assert lib.toric3d_run_batch(ctypes.byref(cfg), items, 1, FAKE, 1 << 30, None) == EINVAL
    assert "use_bp must be 0" in _err()
    cfg = t3d.make_run_cfg(4, 2, 0.04, 0.04, 0, 64, schedule="F", n_apply=1, fallback_max_weight=5)
    cfg.cnn_blob = blob
    assert lib.toric3d_run_batch(ctypes.byref(cfg), items, 1, FAKE, 1 << 30, None) == EINVAL
    assert "bp_iters > 0" in _err()
    cfg.fallback_max_weight = -1
    items[0].s_prev = None
    assert lib.toric3d_run_batch(ctypes.byref(cfg), items, 1, FAKE, 1 << 30, None) == EINVAL
    assert "s_prev" in _err()
    assert lib.toric3d_run_cycles(ctypes.byref(cfg), FAKE, FAKE, 1 << 30, None, None, None) == EINVAL
    assert "toric3d_run_batch" in _err()
    items[0].s_prev = 0x20000
    # the learned decoder's workspace adds s_raw and the pre-decoder's scratch to the two state copies
    plain = t3d.make_run_cfg(4, 2, 0.04, 0.04, 0, 64, schedule="F", n_apply=1)
    assert t3d.toric3d_run_batch_workspace_bytes(cfg, items) > t3d.toric3d_run_batch_workspace_bytes(plain, items)
    fb = t3d.make_run_cfg(4, 2, 0.04, 0.04, 0, 64, schedule="F", n_apply=1, bp_iters=4, fallback_max_weight=9)
    fb.cnn_blob = blob
    assert t3d.toric3d_run_batch_workspace_bytes(fb, items) > t3d.toric3d_run_batch_workspace_bytes(cfg, items)


def test_gate_validation():
    lib = t3d.lib()
    assert lib.toric3d_gate(1, 1, FAKE, 0, FAKE, None, FAKE, 1 << 20, None) == EINVAL
    assert lib.toric3d_gate(4, 0, FAKE, 0, FAKE, None, FAKE, 1 << 20, None) == EINVAL
    assert lib.toric3d_gate(4, 1, FAKE, 0, None, None, FAKE, 1 << 20, None) == EINVAL
    need = t3d.toric3d_gate_workspace_bytes(4, 1)
    assert need > 0
    assert lib.toric3d_gate(4, 1, FAKE, 0, FAKE, None, FAKE, need - 8, None) == EINVAL
    assert "workspace" in _err()


def test_meta_check_bp_sizes_and_validation():
    lib = t3d.lib()
    L, S = 4, 100
    n, W = 3 * L ** 3, 2
    assert t3d.toric3d_bp_meta_message_bytes(L, S) == 7 * n * 64 * W * 4
    per_word = t3d.toric3d_bp_meta_workspace_bytes(L, 64)
    assert per_word >= 64 * 15 * n * 4 + L ** 3 * 32
    assert t3d.toric3d_bp_meta_workspace_bytes(L, S) == 2 * per_word
    assert t3d.toric3d_bp_meta_workspace_bytes(1, S) == 0
    other = ctypes.c_void_p(0x10000 + n * W * 8)
    assert lib.toric3d_bp_meta(L, S, FAKE, other, 0.04, 0.0, 5, FAKE, 1 << 30, None, None) == EINVAL
    assert "0 < q < 1" in _err()
    assert lib.toric3d_bp_meta(L, S, FAKE, other, 1.0, 0.04, 5, FAKE, 1 << 30, None, None) == EINVAL
    assert "0 < p < 1" in _err()
    assert lib.toric3d_bp_meta(L, S, FAKE, other, 0.04, 0.04, 5, FAKE, per_word - 1, None, None) == EINVAL
    assert "workspace too small" in _err()
    assert lib.toric3d_bp_meta(L, S, FAKE, other, 0.04, 0.04, 5, FAKE, per_word, FAKE, None) == EINVAL
    assert "llr_out" in _err()
    assert lib.toric3d_bp_meta(L, S, FAKE, ctypes.c_void_p(0x10008), 0.04, 0.04, 5, FAKE, 1 << 30, None,
                               None) == EINVAL
    assert "overlap" in _err()
    mb = t3d.toric3d_bp_meta_message_bytes(L, S)
    assert lib.toric3d_bp_meta_step(L, S, FAKE, 0.04, 0.04, FAKE, ctypes.c_void_p(0x10000 + mb - 16), FAKE,
                                    1 << 30, None) == EINVAL
    assert "overlap" in _err()
    # whole runs: meta-checks need BP and measurement errors
    cfg = t3d.make_run_cfg(L, 2, 0.04, 0.0, 0, S, use_bp=True, bp_iters=4, bp_meta_checks=True, schedule="F")
    assert cfg.bp_meas_nodes == 2
    assert lib.toric3d_run_cycles(ctypes.byref(cfg), FAKE, FAKE, 1 << 30, None, None, None) == EINVAL
    assert "meta-checks" in _err()
    cfg = t3d.make_run_cfg(L, 2, 0.04, 0.04, 0, S, use_bp=True, bp_iters=4, bp_meta_checks=True, schedule="F")
    plain = t3d.make_run_cfg(L, 2, 0.04, 0.04, 0, S, use_bp=True, bp_iters=4, schedule="F")
    assert t3d.toric3d_run_workspace_bytes(cfg) > t3d.toric3d_run_workspace_bytes(plain)


def _prep(cptr, cvar, n, blob=FAKE, nbytes=1 << 20):
    import numpy as np
    cptr = np.asarray(cptr, np.int32)
    cvar = np.asarray(cvar, np.int32)
    desc = t3d.Tanner()
    st = t3d.lib().toric3d_tanner_prepare(n, len(cptr) - 1, cptr.ctypes.data_as(ctypes.c_void_p),
                                          cvar.ctypes.data_as(ctypes.c_void_p), blob, nbytes, ctypes.byref(desc))
    return st, desc


@pytest.mark.parametrize("cptr,cvar,n,needle", [
    ([0, 2, 4], [0, 0, 1, 2], 3, "twice"),
    ([0, 2, 4], [0, 3, 1, 2], 3, "out of range"),
    ([0, 33], list(range(33)), 40, "degree 33"),
    ([1, 2], [0, 1], 3, "cptr[0]"),
    ([0, 2, 1], [0, 1], 3, "non-decreasing"),
    ([0, 0], [], 3, "edges"),
])
def test_tanner_prepare_rejects_bad_lists(cptr, cvar, n, needle):
    st, _ = _prep(cptr, cvar, n)
    assert st == EINVAL and needle in _err()


def test_tanner_prepare_rejects_variable_degree_above_32_and_small_blobs():
    cptr = list(range(0, 34))
    cvar = [0] * 33                  # variable 0 in 33 checks of degree 1
    st, _ = _prep(cptr, cvar, 1)
    assert st == EINVAL and "variable 0 has degree 33" in _err()
    need = t3d.lib().toric3d_tanner_bytes(3, 2, 4)
    assert need > 0
    st, _ = _prep([0, 2, 4], [0, 1, 1, 2], 3, nbytes=need - 1)
    assert st == EINVAL and "blob too small" in _err()
    st, _ = _prep([0, 2, 4], [0, 1, 1, 2], 3, blob=MIS)
    assert st == EINVAL and "aligned" in _err()


def test_tanner_calls_reject_unprepared_graphs():
    lib = t3d.lib()
    g = t3d.Tanner()   # all zero: not prepared
    assert lib.toric3d_tanner_noise(ctypes.byref(g), 64, FAKE, 0.1, 0, 0, 1, None) == EINVAL
    assert "not prepared" in _err()
    assert lib.toric3d_tanner_flip_workspace_bytes(None, 64) == 0
    assert lib.toric3d_tanner_bp_workspace_bytes(None, 64) == 0
