"""Parity of the FP32 CUDA belief propagation with the FP64 oracle (Sec. 4.1).

Per-iteration protocol: iteration 1 starts both sides from the priors; for
every later iteration the oracle is seeded with the GPU's FP32 messages of the
previous iteration, so each comparison isolates one iteration of FP32
arithmetic.  Tolerance per message (derived from the arithmetic):
    |gpu - ref| <= 1e-5 |ref| + 1e-6                       FP32 target
                 + 2.3e-16 exp(|ref|)                      oracle's own error
                 + 3 u sum_{i != j} (|l0| + sum |m_in|)    FP32 input sums
The second term bounds the oracle's binary64 error in 2 atanh(P) when 1 - P
~ e^-|ref| is resolved to one ulp of 2^-53 (messages near the clamp of 30).
The third bounds the FP32 rounding of each variable->check input
x = l0 + m_a + m_b + m_c (three roundings of at most u = 2^-24 times the sum
of magnitudes), propagated through Eq. 2, whose output moves by at most
|dx| per input; it only matters when opposite-sign saturated messages cancel
(measurement variables off).
End to end (all iterations on each side, with measurement variables on or
consistent syndromes) hard decisions agree exactly wherever |l| > 1e-4.
Posteriors are only bounded loosely there (relative 1e-2 of |l| + 1e-3):
loopy BP amplifies the per-iteration FP32 rounding along some trajectories
(about 1e-3 after 20 iterations), which is why message parity is established
iteration by iteration.  Loopy BP on an inconsistent syndrome without
measurement variables is chaotic (messages pinned at the clamp flip sign), so
there only the per-iteration protocol is meaningful."""
import numpy as np
import pytest
import torch

import oracle
import paper_2212_06985_gb300 as t3d
import toric3d_inputs as inp
from gpu_util import dev, download_bits, gpu_messages_to_oracle, message_index, upload_bits, workspace

pytestmark = pytest.mark.gpu


U32 = 2.0 ** -24


def _tol(ref, input_bound=0.0):
    return (1e-5 * np.abs(ref) + 1e-6 + 2.3e-16 * np.exp(np.minimum(np.abs(ref), 40.0))
            + input_bound)


def _input_rounding_bound(m_in, face_edges, l0):
    """Per Tanner edge (f -> E_j): 3u times the sum, over the face's other three
    edges i, of |l0| + the magnitudes of the three messages summed into x_{i->f}."""
    S, ne = m_in.shape
    n = ne // 4
    fe = np.asarray(face_edges, dtype=np.int64).reshape(-1)      # Tanner edge -> variable
    absm = np.abs(m_in)
    A = np.zeros((S, n))
    np.add.at(A, (slice(None), fe), absm)                        # sum of |incoming| per edge
    xin = abs(l0) + A[:, fe] - absm                              # magnitudes summed into x_{v->f}
    per_face = xin.reshape(S, n, 4)
    others = per_face.sum(axis=2, keepdims=True) - per_face
    return (3 * U32 * others).reshape(S, ne)


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
    l0 = float(np.log((1 - p) / p))
    bound = 0.0
    worst = 0.0
    for it in range(1, 17):
        tol = _tol(ref, bound)
        bad = np.abs(gpu - ref) > tol
        if bad.any():
            i = np.argwhere(bad)[0]
            raise AssertionError(f"iteration {it}: sample {i[0]} tanner edge {i[1]}: gpu {gpu[tuple(i)]!r} "
                                 f"ref {ref[tuple(i)]!r} tol {tol[tuple(i)]!r} ({int(bad.sum())} bad)")
        worst = max(worst, float((np.abs(gpu - ref) / _tol(ref)).max()))
        if it == 16:
            break
        t3d.toric3d_bp_step(L, S, s, p, qm, A, B)
        ref, _ = oracle.bp_batch(L, sbits, p, q, meas, 1, m_in=gpu)
        bound = _input_rounding_bound(gpu, fe, l0)
        gpu = gpu_messages_to_oracle(B, L, S, idx)
        A, B = B, A
    print(f"worst error / (1e-5 rel + 1e-6 abs + oracle term) over 16 iterations: {worst:.3f}")


@pytest.mark.parametrize("L,S,iters,meas,q_noise", [(4, 200, 16, True, 0.04), (6, 70, 20, True, 0.04),
                                                   (4, 100, 30, False, 0.0)])
def test_bp_end_to_end_posteriors_and_decisions(L, S, iters, meas, q_noise):
    p = q = 0.04
    ebits, sbits = _noisy_syndromes(L, S, p, q_noise, seed=3 + L)
    e, s = upload_bits(ebits), upload_bits(sbits)
    n = 3 * L ** 3
    llr = torch.zeros((n, S), dtype=torch.float32, device=dev())
    work = workspace(t3d.toric3d_bp_workspace_bytes(L, S))
    t3d.toric3d_bp(L, S, e, s, p, q if meas else 0.0, iters, work, llr)
    g = llr.cpu().numpy().T.astype(np.float64)
    _, ref = oracle.bp_batch(L, sbits, p, q, meas, iters)
    rel = np.abs(g - ref) / (np.abs(ref) + 1e-3)
    print(f"max relative posterior error after {iters} iterations: {rel.max():.2e}")
    assert rel.max() < 1e-2
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
    for chunk in (64, 128, 192, S):
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
    work = workspace(t3d.toric3d_bp_decide_workspace_bytes(L, S))
    t3d.toric3d_bp_decide(L, S, None, 0.3, e, s, work)     # l0 > 0: no correction
    assert np.array_equal(download_bits(e, S), ebits)
    t3d.toric3d_bp_decide(L, S, None, 0.7, e, s, work)     # l0 < 0: flip every qubit
    assert np.array_equal(download_bits(e, S), ebits ^ 1)
    assert download_bits(s, S).sum() == 0            # H applied to all-ones is zero (4 edges per face)


def test_bp_decide_api_from_stepped_messages():
    L, S, p, iters = 4, 150, 0.04, 5
    ebits, sbits = _noisy_syndromes(L, S, p, p, seed=21)
    e, s = upload_bits(ebits), upload_bits(sbits)
    nfl = t3d.toric3d_bp_message_bytes(L, S) // 4
    A = torch.zeros(nfl, dtype=torch.float32, device=dev())
    B = torch.zeros_like(A)
    t3d.toric3d_bp_step(L, S, s, p, p, None, A)
    for _ in range(iters - 1):
        t3d.toric3d_bp_step(L, S, s, p, p, A, B)
        A, B = B, A
    n = 3 * L ** 3
    llr = torch.zeros((n, S), dtype=torch.float32, device=dev())
    t3d.toric3d_bp_decide(L, S, A, p, e, s, workspace(t3d.toric3d_bp_decide_workspace_bytes(L, S)), llr)
    g = llr.cpu().numpy().T.astype(np.float64)
    _, ref = oracle.bp_batch(L, sbits, p, p, True, iters)
    assert np.abs(g - ref).max() < 1e-3
    d = (g < 0).astype(np.uint8)
    assert np.array_equal(download_bits(e, S), ebits ^ d)
    assert np.array_equal(download_bits(s, S), sbits ^ oracle.syndrome_batch(L, d))
