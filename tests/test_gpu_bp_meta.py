"""Parity of the FP32 CUDA BP with meta-checks (Sec. 4.1, last paragraph) with
the FP64 oracle (its BP on the explicit meta-check factor graph).

Per-iteration protocol (toric3d_bp_meta_step): the oracle takes the GPU's
messages of the previous iteration and runs one iteration, so each comparison
isolates one iteration of FP32 arithmetic.  Tolerance per message, as for the
plain BP:  1e-5 |ref| + 1e-6 (FP32 target) + 2.3e-16 exp(|ref|) (the oracle's
binary64 error in 2 atanh near the clamp) + the FP32 rounding of the inputs:
every variable->check input is a sum formed in at most six FP32 operations,
so it is off by at most 6u (|prior| + sum of |incoming|), u = 2^-24, and the
output moves by at most |dx| per input.
End to end (toric3d_bp_meta from the priors on both sides) the first two
iterations agree to that FP32 accuracy; after more, loopy BP amplifies the
per-iteration rounding along some trajectories (on this graph 2e-2 of |l| +
1e-3 after 10 to 20 iterations, 1e-1 after 15 on a consistent syndrome), so
there the posteriors are bounded only loosely (relative 0.5 of |l| + 1e-3:
the same trajectory), the hard decisions agree exactly wherever |l| > 1e-3,
and the e / s update always equals the GPU's own decision d = [l < 0]
applied as e ^= d, s ^= H d.  Long runs on strongly inconsistent syndromes
are chaotic (30 iterations at twice the assumed measurement-error rate ended
0.8 relative apart), so there only the per-iteration protocol is meaningful,
as for the plain BP."""
import numpy as np
import pytest
import torch

import oracle
import paper_2212_06985_gb300 as t3d
import toric3d_inputs as inp
from gpu_util import dev, download_bits, upload_bits, workspace

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _noisy(L, S, p, q, seed):
    n = 3 * L ** 3
    e = inp.random_bits(S, n, p, seed)
    return e, oracle.syndrome_batch(L, e) ^ inp.random_bits(S, n, q, seed + 1)


def _gpu(L, S, ebits, sbits, p, q, iters, chunk=None, want_llr=True):
    n = 3 * L ** 3
    e, s = upload_bits(ebits), upload_bits(sbits)
    llr = torch.full((2, n, S), float("nan"), dtype=torch.float32, device=dev()) if want_llr else None
    work = workspace(t3d.toric3d_bp_meta_workspace_bytes(L, chunk or S))
    t3d.toric3d_bp_meta(L, S, e, s, p, q, iters, work, llr)
    torch.cuda.synchronize()
    g = None
    if want_llr:
        g = llr.cpu().numpy().astype(np.float64)
        g = np.concatenate([g[0].T, g[1].T], axis=1)       # [S][2n], oracle order
    return download_bits(e, S), download_bits(s, S), g


def _gpu_rows(L, cptr, cvar):
    """Row of the GPU message buffer (float[7][3L^3][S']) of every oracle Tanner edge."""
    n = 3 * L ** 3
    rows = np.empty(cptr[-1], dtype=np.int64)
    f = np.arange(n)
    for j in range(4):
        rows[5 * f + j] = 4 * f + j
    rows[5 * f + 4] = 4 * n + f
    t = np.arange(5 * n, cptr[-1])
    k = (t - 5 * n) % 6                       # cube's faces: lower a0, upper a0, lower a1, ...
    face = cvar[t] - n
    rows[t] = np.where(k % 2 == 0, 5 * n, 6 * n) + face
    return rows


def test_gpu_rows_is_a_bijection():
    L = 3
    cptr, cvar = oracle.meta_tanner(L)
    rows = _gpu_rows(L, cptr, cvar)
    assert np.array_equal(np.sort(rows), np.arange(7 * 3 * L ** 3))


@pytest.mark.parametrize("L,S,p,q,iters", [(3, 70, 0.04, 0.04, 6), (4, 64, 0.05, 0.03, 5), (5, 33, 0.02, 0.02, 4),
                                           (5, 64, 0.04, 0.08, 12)])
def test_each_iteration_matches_oracle(L, S, p, q, iters):
    n = 3 * L ** 3
    ebits, sbits = _noisy(L, S, p, q, seed=3 * L)
    s = upload_bits(sbits)
    mb = t3d.toric3d_bp_meta_message_bytes(L, S)
    Sp = 64 * inp.words_for(S)
    cur = torch.zeros(mb // 4, dtype=torch.float32, device=dev())
    nxt = torch.zeros_like(cur)
    work = workspace(mb // 7)
    cptr, cvar = oracle.meta_tanner(L)
    rows = _gpu_rows(L, cptr, cvar)
    prior = np.r_[np.full(n, np.log((1 - p) / p)), np.full(n, np.log((1 - q) / q))]
    syn = [np.r_[sbits[i], oracle.meta_syndrome(L, sbits[i])] for i in range(S)]
    worst = 0.0
    for it in range(iters):
        t3d.toric3d_bp_meta_step(L, S, s, p, q, cur, nxt, work)
        torch.cuda.synchronize()
        m_in = cur.cpu().numpy().astype(np.float64).reshape(7 * n, Sp)
        m_out = nxt.cpu().numpy().astype(np.float64).reshape(7 * n, Sp)
        for i in range(S):
            cv_in = m_in[rows, i]
            _, ref = oracle.bp_priors_from(cptr, cvar, syn[i], prior, 1, cv_in)
            got = m_out[rows, i]
            A = np.zeros(2 * n)
            np.add.at(A, cvar, np.abs(cv_in))
            xb = 6 * U32 * (np.abs(prior) + A)          # bound on each variable's FP32 input sum
            per_check = np.add.reduceat(xb[cvar], cptr[:-1])
            others = np.repeat(per_check, np.diff(cptr)) - xb[cvar]
            tol = 1e-5 * np.abs(ref) + 1e-6 + 2.3e-16 * np.exp(np.minimum(np.abs(ref), 40.0)) + others
            err = np.abs(got - ref)
            assert (err <= tol).all(), (it, i, float(err.max()))
            worst = max(worst, float((err / tol).max()))
        cur, nxt = nxt, cur
    print(f"L={L}: worst error / tolerance over {iters} iterations: {worst:.3f}")


def test_step_arguments():
    L, S = 3, 10
    s = upload_bits(np.zeros((S, 3 * L ** 3), np.uint8))
    mb = t3d.toric3d_bp_meta_message_bytes(L, S)
    buf = torch.zeros(mb // 4 * 2, dtype=torch.float32, device=dev())
    with pytest.raises(RuntimeError, match="overlap"):
        t3d.toric3d_bp_meta_step(L, S, s, 0.04, 0.04, buf[:mb // 4], buf[8:8 + mb // 4], workspace(mb // 7))
    with pytest.raises(RuntimeError, match="work"):
        t3d.toric3d_bp_meta_step(L, S, s, 0.04, 0.04, buf[:mb // 4], buf[mb // 4:], workspace(mb // 7 - 256))


def _check_update(L, ebits, sbits, e, s, g):
    n = 3 * L ** 3
    d = (g[:, :n] < 0).astype(np.uint8)
    assert np.array_equal(e, ebits ^ d)
    assert np.array_equal(s, sbits ^ oracle.syndrome_batch(L, d))


@pytest.mark.parametrize("L,S,iters", [(3, 70, 1), (4, 64 * 2 + 5, 1), (4, 64 * 2 + 5, 2), (5, 33, 2)])
def test_first_iterations_match_oracle(L, S, iters):
    p, q = 0.04, 0.04
    ebits, sbits = _noisy(L, S, p, q, seed=L + 10 * iters)
    e, s, g = _gpu(L, S, ebits, sbits, p, q, iters)
    _, _, ref = oracle.bp_meta_decode_batch(L, ebits, sbits, p, q, iters)
    err = np.abs(g - ref)
    tol = 1e-5 * np.abs(ref) + 1e-5 + 2.3e-16 * np.exp(np.minimum(np.abs(ref), 40.0))
    print(f"L={L} iters={iters}: max |gpu - oracle| {err.max():.2e}")
    assert (err <= tol).all()
    _check_update(L, ebits, sbits, e, s, g)


@pytest.mark.parametrize("L,S,iters,q_noise", [(4, 200, 10, 0.04), (6, 70, 20, 0.04), (4, 100, 15, 0.0)])
def test_end_to_end_posteriors_and_decisions(L, S, iters, q_noise):
    p = q = 0.04
    ebits, sbits = _noisy(L, S, p, q_noise, seed=20 + L)
    e, s, g = _gpu(L, S, ebits, sbits, p, q, iters)
    e_ref, s_ref, ref = oracle.bp_meta_decode_batch(L, ebits, sbits, p, q, iters)
    rel = np.abs(g - ref) / (np.abs(ref) + 1e-3)
    print(f"max relative posterior error after {iters} iterations: {rel.max():.2e}")
    assert rel.max() < 0.5
    clear = np.abs(ref) > 1e-3
    assert np.array_equal((g < 0)[clear], (ref < 0)[clear])
    _check_update(L, ebits, sbits, e, s, g)
    # samples whose every posterior is clear of zero: the corrected state is the oracle's
    rows = clear.all(axis=1)
    assert rows.mean() > 0.9
    assert np.array_equal(e[rows], e_ref[rows]) and np.array_equal(s[rows], s_ref[rows])


def test_isolated_measurement_error_is_flagged():
    """One wrong outcome and no qubit error: the face's measurement variable is the
    only negative posterior and nothing is corrected."""
    L, S, p, q = 4, 64, 0.04, 0.04
    n = 3 * L ** 3
    ebits = np.zeros((S, n), dtype=np.uint8)
    sbits = np.zeros((S, n), dtype=np.uint8)
    faces = np.arange(S) * 7 % n
    sbits[np.arange(S), faces] = 1
    e, s, g = _gpu(L, S, ebits, sbits, p, q, 10)
    assert not e.any() and np.array_equal(s, sbits)
    meas = g[:, n:]
    assert (meas[np.arange(S), faces] < 0).all()
    meas[np.arange(S), faces] = 1.0
    assert (meas > 0).all() and (g[:, :n] > 0).all()


def test_chunking_is_invisible():
    """Chunks of one, two and all words run the same per-sample arithmetic: identical bits."""
    L, S, p = 4, 64 * 3 + 9, 0.05
    ebits, sbits = _noisy(L, S, p, p, seed=4)
    outs = [_gpu(L, S, ebits, sbits, p, p, 12, chunk=c, want_llr=False)[:2] for c in (64, 128, S)]
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1])


def test_zero_iterations_and_arguments():
    L, S = 3, 100
    n = 3 * L ** 3
    ebits, sbits = _noisy(L, S, 0.1, 0.1, seed=2)
    e, s, g = _gpu(L, S, ebits, sbits, 0.04, 0.03, 0)
    assert np.array_equal(e, ebits) and np.array_equal(s, sbits)
    assert np.allclose(g[:, :n], np.log(0.96 / 0.04), rtol=1e-6)
    assert np.allclose(g[:, n:], np.log(0.97 / 0.03), rtol=1e-6)
    eg, sg = upload_bits(ebits), upload_bits(sbits)
    small = workspace(t3d.toric3d_bp_meta_workspace_bytes(L, 64) - 1024)
    full = workspace(t3d.toric3d_bp_meta_workspace_bytes(L, S))
    with pytest.raises(RuntimeError, match="workspace too small"):
        t3d.toric3d_bp_meta(L, S, eg, sg, 0.04, 0.04, 5, small)
    with pytest.raises(RuntimeError, match="0 < q < 1"):
        t3d.toric3d_bp_meta(L, S, eg, sg, 0.04, 0.0, 5, full)
    with pytest.raises(RuntimeError, match="llr_out"):
        llr = torch.zeros((2, n, S), dtype=torch.float32, device=dev())
        t3d.toric3d_bp_meta(L, S, eg, sg, 0.04, 0.04, 5, workspace(t3d.toric3d_bp_meta_workspace_bytes(L, 1)), llr)
    torch.cuda.synchronize()
    assert np.array_equal(download_bits(eg, S), ebits)


def test_full_size_sampled():
    """L = 24, 1000 samples: the samples the oracle checks one by one (a handful)
    decode to the oracle's state, and every sample's residual syndrome is
    consistent with its correction."""
    L, S, p, iters = 24, 1000, 0.04, 10
    ebits, sbits = _noisy(L, S, p, p, seed=77)
    e, s, _ = _gpu(L, S, ebits, sbits, p, p, iters, want_llr=False)
    pick = [0, 1, 63, 64, 511, S - 1]
    e_ref, s_ref, ref = oracle.bp_meta_decode_batch(L, ebits[pick], sbits[pick], p, p, iters)
    for k, i in enumerate(pick):
        if (np.abs(ref[k]) > 1e-3).all():
            assert np.array_equal(e[i], e_ref[k]) and np.array_equal(s[i], s_ref[k]), i
    assert np.array_equal(s ^ sbits, oracle.syndrome_batch(L, e ^ ebits))


@pytest.mark.parametrize("use_graph,chunk", [(False, 0), (True, 0), (False, 128)])
def test_run_with_meta_checks_equals_stepwise(use_graph, chunk):
    """A whole run with bp_meta_checks is the cycle assembled from single calls
    (noise, measurement, toric3d_bp_meta, p-flip schedule), bit for bit."""
    L, S, T, p, seed, iters, sched = 5, 300, 3, 0.04, 6, 8, "PFFPFF"
    n, W = 3 * L ** 3, inp.words_for(S)
    e = torch.zeros((n, W), dtype=torch.int64, device=dev())
    s = torch.zeros_like(e)
    work = workspace(t3d.toric3d_bp_meta_workspace_bytes(L, S))
    fwork = workspace(t3d.toric3d_flip_workspace_bytes(L, W))
    for t in range(1, T + 1):
        t3d.toric3d_noise(L, e, p, seed, 0, t)
        t3d.toric3d_syndrome(L, e, s, p, seed, 0, t)
        t3d.toric3d_bp_meta(L, S, e, s, p, p, iters, work)
        t3d.toric3d_pflip(L, e, s, sched, 6, 0, seed, 0, t, fwork)
    mask_ref = torch.zeros(S, dtype=torch.uint8, device=dev())
    t3d.toric3d_logical(L, S, e, mask_ref)
    cfg = t3d.make_run_cfg(L, T, p, p, seed, S, use_bp=True, bp_iters=iters, bp_meta_checks=True,
                           schedule=sched, n_apply=6, use_graph=use_graph, bp_chunk_samples=chunk)
    e2 = torch.zeros_like(e)
    mask = torch.zeros(S, dtype=torch.uint8, device=dev())
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())   # inputs were written on the current stream
    with torch.cuda.stream(stream):
        t3d.toric3d_run_cycles(cfg, e2, workspace(t3d.toric3d_run_workspace_bytes(cfg)), mask, None)
    stream.synchronize()
    torch.cuda.synchronize()
    assert torch.equal(e2, e)
    assert torch.equal(mask, mask_ref)


def test_run_with_meta_checks_replays_oracle_cycle():
    """One cycle of a meta-check run against the oracle's run: bit-exact on every
    sample whose posteriors are clear of zero on the oracle side."""
    L, S, p, seed, iters = 4, 128, 0.05, 3, 6
    cfg = t3d.make_run_cfg(L, 1, p, p, seed, S, use_bp=True, bp_iters=iters, bp_meta_checks=True,
                           schedule="PFF", n_apply=3)
    e = torch.zeros((3 * L ** 3, inp.words_for(S)), dtype=torch.int64, device=dev())
    t3d.toric3d_run_cycles(cfg, e, workspace(t3d.toric3d_run_workspace_bytes(cfg)), None, None)
    torch.cuda.synchronize()
    got = download_bits(e, S)
    _, ora_e = oracle.run_batch(oracle.make_cfg(L, 1, p, p, seed, use_bp=True, bp_iters=iters, bp_meta=True,
                                                schedule="PFF", n_apply=3), 0, S)
    e0 = oracle.noise_batch(L, np.zeros((S, 3 * L ** 3), np.uint8), p, seed, 0, 1)
    s0 = oracle.measure_batch(L, e0, p, seed, 0, 1)
    _, _, ref = oracle.bp_meta_decode_batch(L, e0, s0, p, p, iters)
    rows = (np.abs(ref) > 1e-3).all(axis=1)
    assert rows.mean() > 0.9
    assert np.array_equal(got[rows], ora_e[rows])
