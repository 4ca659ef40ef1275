"""Parity of the FP32 CUDA belief propagation with the FP64 oracle (Sec. 4.1).

Per-iteration protocol: iteration 1 starts both sides from the priors; for
every later iteration the oracle is seeded with the GPU's FP32 messages of the
previous iteration, so each comparison isolates one iteration of FP32
arithmetic.  Tolerance per message:
    |gpu - ref| <= 1e-5 |ref| + 1e-6 + 2.3e-16 exp(|ref|)
The first two terms are the FP32 target; the last bounds the oracle's own
binary64 error in 2 atanh(P) when P is within a few ulps of 1 (messages near
the clamp of 30), where 1 - P carries one ulp of 2^-53 relative to e^-|ref|.
End to end (all iterations on each side), posteriors agree to a tolerance
derived from the per-iteration bound grown over the iterations, and hard
decisions agree exactly wherever |l| > 1e-4."""
import numpy as np
import pytest
import torch

import oracle
import paper_2212_06985_gb300 as t3d
import toric3d_inputs as inp
from gpu_util import dev, download_bits, gpu_messages_to_oracle, message_index, upload_bits, workspace

pytestmark = pytest.mark.gpu


def _tol(ref):
    return 1e-5 * np.abs(ref) + 1e-6 + 2.3e-16 * np.exp(np.minimum(np.abs(ref), 40.0))


def _noisy_syndromes(L, S, p, q, seed):
    n = 3 * L ** 3
    e = inp.random_bits(S, n, p, seed)
    return e, oracle.syndrome_batch(L, e) ^ inp.random_bits(S, n, q, seed + 1)


@pytest.mark.parametrize("L,S,p,q,meas", [(4, 96, 0.04, 0.04, True), (3, 40, 0.05, 0.05, True),
                                          (4, 64, 0.04, 0.04, False), (5, 33, 0.02, 0.02, True)])
def test_bp_each_iteration_matches_oracle(L, S, p, q, meas):
    _, sbits = _noisy_syndromes(L, S, p, q, seed=L * 7 + S)
    s = upload_bits(sbits)
    fe, _ = oracle.incidence(L)
    idx = message_index(L, fe)
    nfl = t3d.toric3d_bp_message_bytes(L, S) // 4
    A = torch.zeros(nfl, dtype=torch.float32, device=dev())
    B = torch.zeros_like(A)
    qm = q if meas else 0.0
    t3d.toric3d_bp_step(L, S, s, p, qm, None, A)
    gpu = gpu_messages_to_oracle(A, L, S, idx)
    ref, _ = oracle.bp_batch(L, sbits, p, q, meas, 1)
    worst = 0.0
    for it in range(2, 17):
        assert (np.abs(gpu - ref) <= _tol(ref)).all(), f"iteration {it - 1}"
        worst = max(worst, float((np.abs(gpu - ref) / _tol(ref)).max()))
        t3d.toric3d_bp_step(L, S, s, p, qm, A, B)
        ref, _ = oracle.bp_batch(L, sbits, p, q, meas, 1, m_in=gpu)
        gpu = gpu_messages_to_oracle(B, L, S, idx)
        A, B = B, A
    assert (np.abs(gpu - ref) <= _tol(ref)).all()
    print(f"worst error / tolerance over 16 iterations: {worst:.3f}")


@pytest.mark.parametrize("L,S,iters,meas", [(4, 200, 16, True), (6, 70, 20, True), (4, 100, 30, False)])
def test_bp_end_to_end_posteriors_and_decisions(L, S, iters, meas):
    p = q = 0.04
    ebits, sbits = _noisy_syndromes(L, S, p, q, seed=3 + L)
    e, s = upload_bits(ebits), upload_bits(sbits)
    n = 3 * L ** 3
    llr = torch.zeros((n, S), dtype=torch.float32, device=dev())
    work = workspace(t3d.toric3d_bp_workspace_bytes(L, S))
    t3d.toric3d_bp(L, S, e, s, p, q if meas else 0.0, iters, work, llr)
    g = llr.cpu().numpy().T.astype(np.float64)
    _, ref = oracle.bp_batch(L, sbits, p, q, meas, iters)
    rel = np.abs(g - ref) / (np.abs(ref) + 1e-3)
    print(f"max relative posterior error after {iters} iterations: {rel.max():.2e}")
    assert rel.max() < 1e-3
    clear = np.abs(ref) > 1e-4
    assert np.array_equal((g < 0)[clear], (ref < 0)[clear])
    # the e / s update is exactly the GPU's own hard decision d = [l < 0]
    d = (g < 0).astype(np.uint8)
    assert np.array_equal(download_bits(e, S), ebits ^ d)
    assert np.array_equal(download_bits(s, S), sbits ^ oracle.syndrome_batch(L, d))


def test_bp_chunking_is_invisible():
    L, S, p = 4, 300, 0.04
    ebits, sbits = _noisy_syndromes(L, S, p, p, seed=9)
    outs = []
    for chunk in (64, 128, S):
        e, s = upload_bits(ebits), upload_bits(sbits)
        t3d.toric3d_bp(L, S, e, s, p, p, 12, workspace(t3d.toric3d_bp_workspace_bytes(L, chunk)))
        outs.append((download_bits(e, S), download_bits(s, S)))
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1])


def test_bp_decide_without_messages_uses_prior():
    L, S = 3, 50
    n = 3 * L ** 3
    ebits = inp.random_bits(S, n, 0.2, 1)
    e, s = upload_bits(ebits), upload_bits(np.zeros_like(ebits))
    t3d.toric3d_bp_decide(L, S, None, 0.3, e, s)     # l0 > 0: no correction
    assert np.array_equal(download_bits(e, S), ebits)
    t3d.toric3d_bp_decide(L, S, None, 0.7, e, s)     # l0 < 0: flip every qubit
    assert np.array_equal(download_bits(e, S), ebits ^ 1)
    assert download_bits(s, S).sum() == 0            # H applied to all-ones is zero (4 edges per face)
